"""Seeded synthetic inputs for the phipm hot path (operators and vectors).

This module only *builds inputs*: operators in CSR or constant-coefficient
stencil form, and the vectors b_0..b_p of the problem statement
u(t) = sum_k t^k phi_k(tA) b_k (Sec. 3.3, Eq. lincomb2).  It holds none of the
method's arithmetic, so both the CPU oracle and the CUDA path may use it.

Random numbers come from a counter-based generator (SplitMix64 applied to
(seed, stream, index)), written here from its published definition, so the
same seed gives bit-identical integers on every platform and numpy version.
Uniform doubles take the top 53 bits; normals use the Box-Muller cosine branch.

Operator conventions (shared by every workload):
  * grids hold only interior unknowns, h = 1/(N+1), homogeneous Dirichlet data;
  * unknowns are numbered lexicographically with x fastest: i = x + nx*(y + ny*z);
  * a stencil row is  (Ax)_i = c_center x_i + sum_d c_minus[d] x_{i-e_d} + c_plus[d] x_{i+e_d},
    with neighbours outside the grid dropped;
  * Laplacian: A = Delta_h (diagonal -2*ndim/h^2, neighbours +1/h^2), so e^{tA} decays;
  * convection-diffusion u_t = d Lap u - v . grad u with central differences:
    west/east = d/h^2 +/- vx/(2h)  (x-1 gets +, x+1 gets -), same for y.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_M64 = (1 << 64) - 1


# --------------------------------------------------------------------------------------
# counter-based random numbers
# --------------------------------------------------------------------------------------
def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (Steele, Lea & Flood 2014)."""
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    k = _splitmix64(np.array([(seed * 0x100000001B3 + 0x632BE59BD9B4E019) & _M64], dtype=np.uint64))
    k = _splitmix64(k ^ np.array([stream & _M64], dtype=np.uint64))
    return k[0]


def random_u64(seed: int, stream: int, count: int) -> np.ndarray:
    idx = np.arange(count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _splitmix64(idx * np.uint64(0xD1B54A32D192ED03) + _key(seed, stream))


def uniform(seed: int, stream: int, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """count doubles uniform in [lo, hi)."""
    u = (random_u64(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """count standard normal doubles (Box-Muller, cosine branch)."""
    r = random_u64(seed, stream, 2 * count)
    u1 = ((r[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)  # (0, 1]
    u2 = (r[1::2] >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def randint(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    """count integers uniform in {lo..hi} inclusive."""
    span = hi - lo + 1
    return lo + (random_u64(seed, stream, count) % np.uint64(span)).astype(np.int64)


# --------------------------------------------------------------------------------------
# operators
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class Stencil:
    """Constant-coefficient 5-point (2D) or 7-point (3D) stencil, Dirichlet 0."""
    ndim: int
    nx: int
    ny: int
    nz: int
    c_center: float
    c_minus: tuple
    c_plus: tuple

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def dims(self) -> tuple:
        return (self.nx, self.ny, self.nz)[: self.ndim]

    def nnz(self) -> int:
        """Number of structural nonzeros of the matrix the stencil represents."""
        total = self.n
        for d, nd in enumerate(self.dims):
            total += 2 * (self.n // nd) * (nd - 1)
        return total


@dataclasses.dataclass
class CSR:
    """Square CSR matrix: int32 row pointers / sorted int32 column indices, float64 values."""
    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    values: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.values.size)


def laplacian(ndim: int, N: int) -> Stencil:
    h = 1.0 / (N + 1)
    c = 1.0 / (h * h)
    off = tuple([c] * ndim + [0.0] * (3 - ndim))
    return Stencil(ndim, N, N if ndim > 1 else 1, N if ndim > 2 else 1, -2.0 * ndim * c, off, off)


def convection_diffusion_2d(N: int, d: float, vx: float, vy: float) -> Stencil:
    h = 1.0 / (N + 1)
    dd = d / (h * h)
    cm = (dd + vx / (2 * h), dd + vy / (2 * h), 0.0)
    cp = (dd - vx / (2 * h), dd - vy / (2 * h), 0.0)
    return Stencil(2, N, N, 1, -4.0 * dd, cm, cp)


def stencil_to_csr(st: Stencil) -> CSR:
    """Assemble the CSR matrix of a stencil (columns sorted within each row)."""
    n = st.n
    nx, ny, nz = st.nx, st.ny, st.nz
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    strides = (1, nx, nx * ny)
    coords = (x, y, z)
    sizes = (nx, ny, nz)
    cols, vals, rows = [], [], []
    # order of entries by column offset: -e_z, -e_y, -e_x, 0, +e_x, +e_y, +e_z  (sorted)
    entries = []
    for d in reversed(range(st.ndim)):
        entries.append((-strides[d], d, -1, st.c_minus[d]))
    entries.append((0, None, 0, st.c_center))
    for d in range(st.ndim):
        entries.append((strides[d], d, +1, st.c_plus[d]))
    for off, d, sgn, c in entries:
        if d is None:
            mask = np.ones(n, dtype=bool)
        elif sgn < 0:
            mask = coords[d] > 0
        else:
            mask = coords[d] < sizes[d] - 1
        rows.append(idx[mask])
        cols.append(idx[mask] + off)
        vals.append(np.full(int(mask.sum()), c, dtype=np.float64))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), vals)


def dense_to_csr(A: np.ndarray) -> CSR:
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    rows, cols = np.nonzero(A)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return CSR(n, np.cumsum(rowptr).astype(np.int32), cols.astype(np.int32), A[rows, cols].copy())


def csr_to_dense(A: CSR) -> np.ndarray:
    D = np.zeros((A.n, A.n))
    for i in range(A.n):
        for k in range(A.rowptr[i], A.rowptr[i + 1]):
            D[i, A.colind[k]] += A.values[k]
    return D


def random_sparse(seed: int, n: int, per_row: int, scale: float = 1.0, symmetric: bool = False) -> CSR:
    """Random sparse test matrix with a negative-shifted diagonal (for small parity cases)."""
    cols = randint(seed, 1, n * per_row, 0, n - 1).reshape(n, per_row)
    vals = normal(seed, 2, n * per_row).reshape(n, per_row) * scale
    D = np.zeros((n, n))
    for i in range(n):
        for k in range(per_row):
            D[i, cols[i, k]] += vals[i, k]
    if symmetric:
        D = 0.5 * (D + D.T)
    D -= np.diag(np.abs(D).sum(axis=1) * 0.5 + scale)
    return dense_to_csr(D)


# --------------------------------------------------------------------------------------
# problems
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    """One phipm problem: u(t_end) = sum_k t_end^k phi_k(t_end A) b_k."""
    name: str
    op: object           # Stencil or CSR
    b: list              # p+1 float64 arrays
    t_end: float
    tol: float
    symm: int            # -1 auto, 0 no, 1 yes
    precision: str = "f64"   # "f64" or "f32" (FP32 basis + SpMV)
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.op.n

    @property
    def p(self) -> int:
        return len(self.b) - 1


def _normal_vectors(seed: int, n: int, count: int) -> list:
    return [normal(seed, 100 + k, n) for k in range(count)]


def _uniform_vectors(seed: int, n: int, count: int, lo: float, hi: float) -> list:
    return [uniform(seed, 100 + k, n, lo, hi) for k in range(count)]


def laplacian_2d_problem(N: int = 32, p: int = 3, t_end: float = 0.01, tol: float = 1e-8,
                         seed: int = 1000, as_csr: bool = False) -> Problem:
    """Plain phipm FP64: 2D 5-point Dirichlet Laplacian on an N x N grid, b_k ~ N(0,1)."""
    st = laplacian(2, N)
    op = stencil_to_csr(st) if as_csr else st
    return Problem(f"laplacian2d_{N}", op, _normal_vectors(seed, st.n, p + 1), t_end, tol, 1,
                   meta=dict(N=N, seed=seed, stencil=st))


def convdiff_2d_problem(N: int = 512, d: float = 1.0, v: tuple = (50.0, 50.0), p: int = 4,
                        t_end: float = 1e-3, tol: float = 1e-8, seed: int = 2000,
                        as_csr: bool = True) -> Problem:
    """FP64 nonsymmetric: 2D convection-diffusion, central differences, CSR float64/int32."""
    st = convection_diffusion_2d(N, d, v[0], v[1])
    op = stencil_to_csr(st) if as_csr else st
    return Problem(f"convdiff2d_{N}", op, _normal_vectors(seed, st.n, p + 1), t_end, tol, 0,
                   meta=dict(N=N, d=d, v=v, seed=seed, stencil=st))


def laplacian_3d_problem(N: int = 128, p: int = 2, t_end: float = 1e-4, tol: float = 1e-5,
                         seed: int = 3000, precision: str = "f32") -> Problem:
    """Precision form: 3D 7-point Laplacian stencil on N^3, b_k ~ U[-1,1]."""
    st = laplacian(3, N)
    return Problem(f"laplacian3d_{N}", st, _uniform_vectors(seed, st.n, p + 1, -1.0, 1.0), t_end, tol, 1,
                   precision=precision, meta=dict(N=N, seed=seed, stencil=st))


def batched_convdiff_problems(count: int = 256, side_lo: int = 64, side_hi: int = 256,
                              t_end: float = 1e-3, tol: float = 1e-8, seed0: int = 4000) -> list:
    """Batched form: independent 2D convection-diffusion problems of uneven size and p.

    Per problem i (seed seed0+i): side ~ U{side_lo..side_hi}, d log-uniform [0.1, 10],
    v ~ U[-100,100]^2, p ~ U{1..4}, b_k ~ N(0,1)."""
    probs = []
    for i in range(count):
        s = seed0 + i
        side = int(randint(s, 1, 1, side_lo, side_hi)[0])
        d = float(10.0 ** uniform(s, 2, 1, -1.0, 1.0)[0])
        v = uniform(s, 3, 2, -100.0, 100.0)
        p = int(randint(s, 4, 1, 1, 4)[0])
        st = convection_diffusion_2d(side, d, float(v[0]), float(v[1]))
        probs.append(Problem(f"batch_{i}", stencil_to_csr(st), _normal_vectors(s, st.n, p + 1), t_end, tol, 0,
                             meta=dict(side=side, d=d, v=(float(v[0]), float(v[1])), seed=s, stencil=st)))
    return probs


def peclet_convdiff_problems(count: int = 1024, N: int = 128, pe_lo: float = 1.0, pe_hi: float = 1e3,
                             t_end: float = 1e-3, tol: float = 1e-8, seed0: int = 5000) -> list:
    """Held-out batch: convection-diffusion N x N, d = 1, |v| = Pe log-uniform, random direction."""
    probs = []
    for i in range(count):
        s = seed0 + i
        pe = float(10.0 ** uniform(s, 2, 1, math.log10(pe_lo), math.log10(pe_hi))[0])
        ang = float(uniform(s, 3, 1, 0.0, 2.0 * math.pi)[0])
        p = int(randint(s, 4, 1, 1, 4)[0])
        vx, vy = pe * math.cos(ang), pe * math.sin(ang)
        st = convection_diffusion_2d(N, 1.0, vx, vy)
        probs.append(Problem(f"pe_{i}", stencil_to_csr(st), _normal_vectors(s, st.n, p + 1), t_end, tol, 0,
                             meta=dict(pe=pe, angle=ang, seed=s, stencil=st)))
    return probs
