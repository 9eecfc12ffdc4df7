"""Input generators: sizes, coefficients and determinism of the synthetic workloads."""
import numpy as np
import pytest

from oracle import phipm_oracle as O
from paper_0907_4631_gb300 import workloads as wl


def test_rng_determinism_and_moments():
    a = wl.normal(123, 4, 100_000)
    assert np.array_equal(a, wl.normal(123, 4, 100_000))
    assert not np.array_equal(a, wl.normal(123, 5, 100_000))
    assert abs(a.mean()) < 5 / np.sqrt(a.size) and abs(a.var() - 1) < 0.02
    u = wl.uniform(9, 1, 100_000, -1.0, 1.0)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01
    r = wl.randint(9, 2, 10_000, 1, 4)
    assert set(np.unique(r)) == {1, 2, 3, 4}
    # the vectorised generator equals a plain-integer SplitMix64 (Steele, Lea & Flood 2014)
    M = (1 << 64) - 1

    def mix(z):
        z = (z + 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)
    seed, stream = 77, 3
    key = mix(mix((seed * 0x100000001B3 + 0x632BE59BD9B4E019) & M) ^ stream)
    ref = [mix((i * 0xD1B54A32D192ED03 + key) & M) for i in range(5)]
    assert [int(x) for x in wl.random_u64(seed, stream, 5)] == ref


def test_laplacian_2d_32():
    st = wl.laplacian(2, 32)
    assert st.n == 1024 and st.nnz() == 4992
    assert st.c_center == pytest.approx(-4356.0) and st.c_plus[0] == pytest.approx(1089.0)
    A = wl.stencil_to_csr(st)
    assert A.nnz == 4992 and O.Operator(A).norm_inf() == pytest.approx(8712.0)


def test_convection_diffusion_512():
    st = wl.convection_diffusion_2d(512, 1.0, 50.0, 50.0)
    assert st.c_center == pytest.approx(-1_052_676.0)
    assert st.c_plus[0] == pytest.approx(250_344.0) and st.c_plus[1] == pytest.approx(250_344.0)
    assert st.c_minus[0] == pytest.approx(275_994.0) and st.c_minus[1] == pytest.approx(275_994.0)
    A = wl.stencil_to_csr(st)
    assert A.n == 262_144 and A.nnz == 1_308_672
    assert A.rowptr.dtype == np.int32 and A.colind.dtype == np.int32
    assert O.Operator(A).norm_inf() == pytest.approx(2_105_352.0)
    for i in [0, 1, 511, 512, 100_000, 262_143]:
        cols = A.colind[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)


def test_laplacian_3d_128():
    st = wl.laplacian(3, 128)
    assert st.n == 2_097_152
    assert st.c_center == pytest.approx(-99_846.0) and st.c_plus[2] == pytest.approx(16_641.0)
    assert O.Operator(st).norm_inf() == pytest.approx(199_692.0)


@pytest.mark.parametrize("st", [wl.laplacian(2, 9), wl.laplacian(3, 5), wl.convection_diffusion_2d(7, 0.3, 40.0, -25.0),
                                wl.laplacian(1, 11)])
def test_stencil_matvec_equals_csr(st):
    A = wl.stencil_to_csr(st)
    x = wl.normal(3, 3, st.n)
    assert np.allclose(O.Operator(st).matvec(x), O.Operator(A).matvec(x), rtol=1e-14, atol=1e-12)
    assert A.nnz == st.nnz()
    D = wl.csr_to_dense(A)
    assert np.allclose(D @ x, O.Operator(A).matvec(x))


def test_batched_generators():
    probs = wl.batched_convdiff_problems(count=32)
    for pr in probs:
        assert 64 <= pr.meta["side"] <= 256 and 1 <= pr.p <= 4
        assert 0.1 <= pr.meta["d"] <= 10.0 and all(abs(v) <= 100 for v in pr.meta["v"])
        assert pr.n == pr.meta["side"] ** 2 and len(pr.b) == pr.p + 1
    again = wl.batched_convdiff_problems(count=2)
    assert np.array_equal(again[1].b[0], probs[1].b[0])
    pe = wl.peclet_convdiff_problems(count=8)
    for pr in pe:
        assert pr.n == 16384 and 1.0 <= pr.meta["pe"] <= 1e3
