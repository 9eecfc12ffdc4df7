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


@dataclasses.dataclass
class VarCoefConvDiff:
    """Data of the built-in matrix-free operator PHIPM_FN_VARCOEF_CONVDIFF (include/phipm.h):
    a grid, the diffusivity field kappa (n values > 0), velocity fields (n values each, or
    None) and the scalars 1/h^2 and 1/(2h) per dimension.  Only inputs: the product itself
    runs in the library's kernels (and, separately, in the oracle)."""
    ndim: int
    nx: int
    ny: int
    nz: int
    kappa: np.ndarray
    vel: list                      # ndim entries, arrays or None
    h: float
    norm_bound: float = 0.0        # <= 0: the library computes ||A||_inf on the device
    cost: int = 0                  # <= 0: the grid operator's structural nonzeros
    fn: int = 0

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def fields(self) -> list:
        return [self.kappa] + [self.vel[d] if d < len(self.vel) else None for d in range(3)]

    @property
    def scal(self) -> list:
        s2 = [1.0 / (self.h * self.h) if d < self.ndim else 0.0 for d in range(3)]
        s1 = [1.0 / (2.0 * self.h) if d < self.ndim else 0.0 for d in range(3)]
        return s2 + s1


def varcoef_convdiff(ndim: int, N: int, speed: float, seed: int, kappa_amp: float = 0.5) -> VarCoefConvDiff:
    """A smooth positive diffusivity 1 + kappa_amp sin(2 pi x) cos(pi y) (cos(pi z) in 3D)
    plus a small seeded perturbation, and, for speed > 0, a rotating velocity field of that
    magnitude, v = speed (cos(pi y), sin(pi x)[, cos(pi x)]), on the N^ndim interior grid,
    h = 1 / (N + 1)."""
    h = 1.0 / (N + 1)
    g = np.arange(1, N + 1) * h
    dims = [N] * ndim + [1] * (3 - ndim)
    z, y, x = np.meshgrid(g if ndim > 2 else [0.5], g if ndim > 1 else [0.5], g, indexing="ij")
    n = N ** ndim
    kap = 1.0 + kappa_amp * np.sin(2 * np.pi * x) * np.cos(np.pi * y) * (np.cos(np.pi * z) if ndim > 2 else 1.0)
    kap = kap.reshape(-1) * (1.0 + 0.05 * uniform(seed, 7, n, -1.0, 1.0))
    vel = [None] * ndim
    if speed > 0:
        comps = [np.cos(np.pi * y), np.sin(np.pi * x), np.cos(np.pi * x)]
        vel = [speed * comps[d].reshape(-1) for d in range(ndim)]
    return VarCoefConvDiff(ndim, dims[0], dims[1], dims[2], kap, vel, h)


def varcoef_convdiff_problem(ndim: int = 2, N: int = 64, speed: float = 20.0, p: int = 2, t_end: float = 1e-3,
                             tol: float = 1e-8, seed: int = 6000) -> Problem:
    """A matrix-free phipm problem (Sec. 3.5): the variable-coefficient operator above,
    b_k ~ N(0, 1)."""
    op = varcoef_convdiff(ndim, N, speed, seed)
    return Problem(f"varcoef_{ndim}d_{N}", op, _normal_vectors(seed, op.n, p + 1), t_end, tol,
                   1 if speed == 0 else 0, meta=dict(seed=seed))


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


def nine_point(N: int, center: float = 8.0, neighbour: float = -1.0) -> CSR:
    """Nine-point matrix on an N x N grid of unknowns (x fastest): every unknown couples
    to the up to eight grid neighbours with |dx|, |dy| <= 1.  Its sparsity is that of
    the nine-point Laplacian of Sec. 4.2 (N = 30: n = 900, nnz = (3N-2)^2 = 7,744).
    The default values (8 on the diagonal, -1 off it) make a symmetric positive
    definite matrix with eigenvalues in (0, 12)."""
    n = N * N
    idx = np.arange(n, dtype=np.int64)
    x, y = idx % N, idx // N
    rows, cols, vals = [], [], []
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            mask = (x + dx >= 0) & (x + dx < N) & (y + dy >= 0) & (y + dy < N)
            rows.append(idx[mask])
            cols.append(idx[mask] + dx + N * dy)
            vals.append(np.full(int(mask.sum()), center if dx == 0 and dy == 0 else neighbour))
    rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return CSR(n, np.cumsum(rowptr).astype(np.int32), cols[order].astype(np.int32), vals[order].astype(np.float64))


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


def nine_point_phi_sum_problem(N: int = 30, p: int = 4, t_end: float = 2.0,
                               tol: float = 2.0 ** -26) -> Problem:
    """Sec. 4.2, Experiment 2 on the nine-point matrix: sum_{k<=4} t^k phi_k(tA) b_k with
    every b_k = [1, ..., 1], t = 2, Tol = sqrt(machine epsilon).  The paper's matrix values
    are not printed; the stand-in is A = -S with S = nine_point(N) (diagonal 8, off-diagonal
    -1), so that e^{tA} decays as the Laplacian's does."""
    S = nine_point(N)
    A = CSR(S.n, S.rowptr, S.colind, -S.values)
    return Problem(f"ninepoint{N}_phi{p}", A, [np.ones(S.n) for _ in range(p + 1)], t_end, tol, 1,
                   meta=dict(N=N))


def nine_point_round_trip(N: int = 30, t_end: float = 2.0, tol: float = 1e-14) -> tuple:
    """Sec. 4.2, Experiment 1's third case: w = e^{tA} b_0, then e^{-tA} w, which returns b_0
    in exact arithmetic; b_0 = [1, ..., 1], t = 2, Tol = 1e-14, A = -nine_point(N).
    Returns (A, -A) as CSR, b_0, t_end and tol."""
    S = nine_point(N)
    A = CSR(S.n, S.rowptr, S.colind, -S.values)
    B = CSR(S.n, S.rowptr, S.colind, S.values.copy())
    return A, B, np.ones(S.n), t_end, tol


@dataclasses.dataclass
class HestonGrid:
    """Grid and coefficients of the Heston PDE of Sec. 4.1 (u' = A u + b_1)."""
    ns: int = 100           # points in s: s_i = i ds, i = 1..ns (s = 0 and s = S are not grid points)
    nv: int = 51            # points in v: v_j = j dv, j = 0..nv-1 (v = 0 is, v = V is not)
    K: float = 100.0        # strike
    S: float = 800.0        # 8 K
    V: float = 5.0
    kappa: float = 2.0
    eta: float = 0.2        # the mean level of v (the parameter list prints it as nu)
    lam: float = 0.3
    rho: float = 0.8
    rd: float = 0.03
    rf: float = 0.0
    T: float = 1.0

    @property
    def ds(self) -> float:
        return self.S / (self.ns + 1)

    @property
    def dv(self) -> float:
        return self.V / self.nv

    def s(self) -> np.ndarray:
        return self.ds * np.arange(1, self.ns + 1)

    def v(self) -> np.ndarray:
        return self.dv * np.arange(self.nv)


def heston_operator(g: HestonGrid | None = None) -> tuple:
    """Assemble the semi-discrete Heston system u' = A u + b_1, u(0) = b_0 of Sec. 4.1.

    Unknowns U_{i,j} = U(s_i, v_j) numbered i + ns j (s fastest).  Rows with v_j > 0 use
    the printed second-order differences for U_s, U_ss, U_v, U_vv and U_sv of
        U_t = v s^2/2 U_ss + rho lam v s U_sv + lam^2 v/2 U_vv + (rd - rf) s U_s
              + kappa (eta - v) U_v - rd U;
    rows with v = 0 use the boundary equation U_t = (rd - rf) s U_s + kappa eta U_v - rd U
    with the printed one-sided U_v.  Boundary data: U = 0 at s = 0 and U = s at v = V
    (both into b_1), U_s = 1 at s = S through the ghost value U(S, v) = U(s_ns, v) + ds.
    b_0 is the payoff max(s - K, 0).  Returns (CSR A, b_0, b_1, grid)."""
    g = g or HestonGrid()
    ns, nv, ds, dv = g.ns, g.nv, g.ds, g.dv
    s, v = g.s(), g.v()
    n = ns * nv
    rows, cols, vals = [], [], []
    b1 = np.zeros(n)

    def add(r, i, j, c):
        """Coefficient c on U at grid index (i, j); i = -1 is s = 0, i = ns is s = S, j = nv is v = V."""
        if j == nv:
            s_i = ds * (i + 1)
            b1[r] += c * s_i                  # U(s, V) = s
        elif i < 0:
            pass                              # U(0, v) = 0
        elif i == ns:
            rows.append(r); cols.append(ns - 1 + ns * j); vals.append(c)
            b1[r] += c * ds                   # ghost: U(S, v) = U(s_ns, v) + ds
        else:
            rows.append(r); cols.append(i + ns * j); vals.append(c)

    for j in range(nv):
        for i in range(ns):
            r = i + ns * j
            a_s = (g.rd - g.rf) * s[i] / (2 * ds)
            if j == 0:
                c = g.kappa * g.eta / (2 * dv)
                add(r, i + 1, 0, a_s); add(r, i - 1, 0, -a_s)
                add(r, i, 0, -3 * c); add(r, i, 1, 4 * c); add(r, i, 2, -c)
            else:
                a_ss = 0.5 * v[j] * s[i] ** 2 / ds ** 2
                a_vv = 0.5 * g.lam ** 2 * v[j] / dv ** 2
                a_v = g.kappa * (g.eta - v[j]) / (2 * dv)
                a_sv = g.rho * g.lam * v[j] * s[i] / (4 * ds * dv)
                add(r, i + 1, j, a_ss + a_s); add(r, i - 1, j, a_ss - a_s); add(r, i, j, -2 * a_ss)
                add(r, i, j + 1, a_vv + a_v); add(r, i, j - 1, a_vv - a_v); add(r, i, j, -2 * a_vv)
                add(r, i + 1, j + 1, a_sv); add(r, i - 1, j - 1, a_sv)
                add(r, i - 1, j + 1, -a_sv); add(r, i + 1, j - 1, -a_sv)
            add(r, i, j, -g.rd)
    rows, cols, vals = np.asarray(rows), np.asarray(cols), np.asarray(vals, dtype=np.float64)
    # merge duplicates (ghost folding), drop exact zeros, sort columns within rows
    key = rows.astype(np.int64) * n + cols
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    uniq, start = np.unique(key, return_index=True)
    merged = np.add.reduceat(vals, start)
    keep = merged != 0.0
    uniq, merged = uniq[keep], merged[keep]
    r_u = (uniq // n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r_u + 1, 1)
    A = CSR(n, np.cumsum(rowptr).astype(np.int32), (uniq % n).astype(np.int32), merged)
    b0 = np.maximum(np.tile(s, nv) - g.K, 0.0)
    return A, b0, b1, g


def heston_problem(tol: float = 1e-4) -> Problem:
    """Sec. 4.1: u(T) = e^{TA} b_0 + T phi_1(TA) b_1 for the 100 x 51 Heston grid, T = 1."""
    A, b0, b1, g = heston_operator()
    return Problem(f"heston_{g.ns}x{g.nv}", A, [b0, b1], g.T, tol, 0, meta=dict(grid=g))
