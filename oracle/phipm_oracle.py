"""Plain FP64 CPU oracle of the phipm algorithm (Niesen & Wright, Sec. 3).

TEST INFRASTRUCTURE ONLY: used by tests, smoke() and bench.py's CPU-baseline
leg; never by the product path.  Shares no code with the CUDA implementation.

It follows the paper step by step, slow and plain:
  * Arnoldi with modified Gram-Schmidt exactly as Algorithm 1, Lanczos as
    Algorithm 2 (with the index reading below), recomputed from scratch at
    every attempt as Algorithm 3 prints it;
  * the augmented matrix of Eq. (hathm), extended by one row/column so that
    phi_{p+1} is available for the corrector of Eq. (phipapprox2);
  * exp by the degree-13 diagonal Pade approximant with scaling and squaring
    (Sec. 3.1), powers formed one by one, the linear system solved by LU with
    partial pivoting (numpy.linalg.solve);
  * the error estimate of Eq. (errest), the step of Eq. (step), the
    w-recurrence of Eq. (wrecurrence), the initial step of Eq. (tau_0);
  * the controller of Sec. 3.4: Eqs. (taunew), (6), (2), (7), (3), cost model
    Eqs. (4), (5), (8), and Algorithms 3 and 4.

Readings where the paper is silent, garbled or contradicts itself
(the same readings hold for the CUDA path):
  R2  augmented matrix has size m+p+1; phi_j(tau H) e_1 is column m+j-1
      (0-based); tau multiplies only the H block.
  R3  Lanczos: t_{j+1,j} = t_{j,j+1} = ||w||, v_{j+1} = w / t_{j+1,j}.
  R4  the estimate of Eq. (errest) applied to tau*A and scaled by tau^p:
      eps = tau^{p+1} beta |h_{m+1,m}| |[phi_{p+1}(tau H) e_1]_m|.
  R5  m_init = 10 (Algorithm 3), m_max = 64 (parameter), m >= 1.
  R6  Tol is the tolerance of Eq. (taunew), absolute, on the 2-norm.
  R7  Eq. (6) is printed inverted; with eps ~ tau^{q+1} the order estimate is
      q = log(eps/eps_old) / log(tau/tau_old) - 1; clamped to [0, m], and
      replaced by m/4 when not finite.
  R8  tau changes by at most the factors of Algorithm 3: [tau/5, 2 tau].
  R9  u and t advance with the tau of the accepted attempt; the tau and m
      the controller produced in that attempt seed the next step.
  R10 the m branch is taken when C(tau, m_new) <= C(tau_new, m); accept iff
      omega <= delta.
  R11 "m was reduced" in Algorithm 4 reads "m was changed".
  R12 happy breakdown when h_{j+1,j} <= breakdown_tol * ||A||_inf: the
      Krylov space is invariant, m := j and the corrector and eps vanish.
      beta = 0 gives F = 0, eps = 0.  kappa <= 1 or not finite -> 2.
      A non-finite eps rejects the attempt and divides tau by 5; ten in a
      row is an error.  If b_0 = 0 the tau_0 formula uses max_k ||b_k||_inf;
      if every b_k is 0 the result is 0.
  R13 m_new is rounded up (the smallest integer meeting the tolerance) and
      clamped to [1, m_max] before its cost is evaluated; a tau_new of +inf
      (eps = 0) costs ceil(0) = 0 steps.
  R14 the expm cost factor M of Eq. (8) uses ||H_hat||_1 of the current
      attempt for both candidates; theta_13 = 5.37 as printed; the same s
      drives the scaling of the exponential.
  R15 the cost model follows the symmetry of A (Lanczos or Arnoldi formula of
      Eq. 4), whatever orthogonalisation an implementation uses.
  R19 the m branch is only taken when it changes m: if m_new, restricted to a
      factor 4/3 and to [1, m_max], equals the current m (m at m_max with the
      tolerance still missed, say), tau changes instead.  Sec. 3.4 does not
      say what happens at the bound; taken literally the rejected attempt
      would repeat unchanged for ever.
  R20 phip, the fixed-dimension variant of Sec. 4.2 (the same code with m
      held constant), is this algorithm with the m branch never taken: m
      stays m_init (a happy breakdown shortens it as in R12) and every
      attempt updates tau.
  R23 phi_method "eigen" (symmetric A): phi_p(tau T) e_1 and phi_{p+1}(tau T) e_1 are
      taken from the eigen-decomposition of the Lanczos matrix, the direct route
      Sec. 5 suggests; the cost model still charges the exponential of Eq. (8), so
      the controller's decisions are those of the augmented route.
  R24 a matrix-free A (Sec. 3.5 accepts a function computing A b) supplies, besides
      the product, an upper bound of ||A||_inf and the cost N_A of one product, which
      Eq. (tau_0), the breakdown threshold and Eq. (4) need; symmetry is not detected
      (nonsymmetric unless symm = 1), as Sec. 3.5 prescribes for implicit A.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

DEFAULTS = dict(
    gamma=0.8,          # safety factor, Sec. 3.4
    delta=1.2,          # acceptance threshold, Sec. 3.4
    m_init=10,          # Algorithm 3
    m_max=64,           # reading R5
    theta13=5.37,       # Eq. (8)
    breakdown_tol=1e-12,
    max_steps=1_000_000,
    max_rejects=1_000_000,
    adapt_m=True,       # False: the fixed-dimension variant phip of Sec. 4.2
    phi_method="augmented",   # "eigen": phi of the Lanczos matrix directly (symmetric A only)
)


# --------------------------------------------------------------------------------------
# the operator A (the oracle's own matrix-vector product)
# --------------------------------------------------------------------------------------
class Operator:
    """A as CSR (scipy.sparse product), as a constant-coefficient stencil, or matrix-free
    (R24): an object with apply(x) -> A x, n, and the two scalars the method needs from A,
    norm_inf (an upper bound of ||A||_inf, for Eq. tau_0 and the breakdown threshold) and
    nnz (the cost of one product in the units of Eq. 4's N_A)."""

    def __init__(self, op):
        self.src = op
        if callable(getattr(op, "apply", None)):
            self.kind = "function"
            self.n = int(op.n)
            self.nnz = int(op.nnz)
        elif hasattr(op, "rowptr"):
            self.kind = "csr"
            self.n = int(op.n)
            self.M = sp.csr_matrix((np.asarray(op.values, dtype=np.float64),
                                    np.asarray(op.colind), np.asarray(op.rowptr)), shape=(self.n, self.n))
            self.nnz = int(self.M.nnz)
        else:
            self.kind = "stencil"
            self.n = int(op.n)
            self.nnz = int(op.nnz())

    def matvec(self, x: np.ndarray) -> np.ndarray:
        if self.kind == "function":
            return np.asarray(self.src.apply(x), dtype=np.float64)
        if self.kind == "csr":
            return self.M @ x
        st = self.src
        X = x.reshape(st.nz, st.ny, st.nx)   # x fastest
        Y = st.c_center * X
        # axis of dimension d in the (z, y, x) array
        for d in range(st.ndim):
            ax = 2 - d
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ax] = slice(0, -1)
            hi[ax] = slice(1, None)
            Y[tuple(hi)] += st.c_minus[d] * X[tuple(lo)]   # neighbour i - e_d
            Y[tuple(lo)] += st.c_plus[d] * X[tuple(hi)]    # neighbour i + e_d
        return Y.reshape(-1)

    def norm_inf(self) -> float:
        """||A||_inf, the maximum absolute row sum (matrix-free: the bound supplied)."""
        if self.kind == "function":
            return float(self.src.norm_inf)
        if self.kind == "csr":
            return float(np.max(np.asarray(abs(self.M).sum(axis=1)).ravel())) if self.n else 0.0
        st = self.src
        s = abs(st.c_center)
        for d in range(st.ndim):
            s += abs(st.c_minus[d]) + abs(st.c_plus[d])
        return float(s)

    def is_symmetric(self) -> bool:
        if self.kind == "function":     # not detectable: nonsymmetric unless symm says so (Sec. 3.5)
            return False
        if self.kind == "csr":
            D = self.M - self.M.T
            return D.count_nonzero() == 0 or float(abs(D).max()) == 0.0
        st = self.src
        return all(st.c_minus[d] == st.c_plus[d] for d in range(st.ndim))


# --------------------------------------------------------------------------------------
# Krylov projections (Sec. 3.1)
# --------------------------------------------------------------------------------------
def arnoldi(matvec, v: np.ndarray, m: int, bd_abs: float):
    """Algorithm 1 (modified Gram-Schmidt).

    Returns (V, H, m_eff): V is (m_eff+1, n) with rows v_1..v_{m_eff+1},
    H is (m_eff+1, m_eff).  Stops at happy breakdown h_{j+1,j} <= bd_abs
    (then v_{m_eff+1} = 0 and h_{m_eff+1,m_eff} = 0)."""
    n = v.size
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    V[0] = v / np.linalg.norm(v)
    for j in range(m):
        w = matvec(V[j])
        for i in range(j + 1):
            H[i, j] = V[i] @ w
            w = w - H[i, j] * V[i]
        hn = np.linalg.norm(w)
        if hn <= bd_abs:
            return V[: j + 2] * np.r_[np.ones(j + 1), 0.0][:, None], _trim(H, j + 1, zero_last=True), j + 1
        H[j + 1, j] = hn
        V[j + 1] = w / hn
    return V, H, m


def lanczos(matvec, v: np.ndarray, m: int, bd_abs: float):
    """Algorithm 2 (three-term recurrence) with t_{j+1,j} = t_{j,j+1} = ||w||."""
    n = v.size
    V = np.zeros((m + 1, n))
    T = np.zeros((m + 1, m))
    V[0] = v / np.linalg.norm(v)
    for j in range(m):
        w = matvec(V[j])
        T[j, j] = V[j] @ w
        if j > 0:
            w = w - T[j - 1, j] * V[j - 1]      # t_{j,j-1} v_{j-1}
        w = w - T[j, j] * V[j]
        hn = np.linalg.norm(w)
        if hn <= bd_abs:
            return V[: j + 2] * np.r_[np.ones(j + 1), 0.0][:, None], _trim(T, j + 1, zero_last=True), j + 1
        T[j + 1, j] = hn
        if j + 1 < m:
            T[j, j + 1] = hn
        V[j + 1] = w / hn
    return V, T, m


def _trim(H: np.ndarray, m: int, zero_last: bool) -> np.ndarray:
    out = np.array(H[: m + 1, :m])
    if zero_last:
        out[m, m - 1] = 0.0
    return out


# --------------------------------------------------------------------------------------
# augmented matrix and its exponential (Sec. 3.1)
# --------------------------------------------------------------------------------------
def augmented_matrix(H_m: np.ndarray, tau: float, p: int) -> np.ndarray:
    """Eq. (hathm) extended by one (reading R2): size m+p+1.

    [[tau H_m, e_1, 0], [0, 0, I_p], [0, 0, 0]] ; the top m entries of column
    m+j-1 of its exponential are phi_j(tau H_m) e_1, j = 1..p+1."""
    m = H_m.shape[0]
    N = m + p + 1
    Hh = np.zeros((N, N))
    Hh[:m, :m] = tau * H_m
    Hh[0, m] = 1.0
    for i in range(p):
        Hh[m + i, m + i + 1] = 1.0
    return Hh


def pade13_coefficients() -> list:
    """c_j of the [13/13] Pade approximant of e^x: (26-j)! 13! / (26! j! (13-j)!)."""
    f = math.factorial
    return [f(26 - j) * f(13) / (f(26) * f(j) * f(13 - j)) for j in range(14)]


def squarings(norm1: float, theta13: float) -> int:
    """s = ceil(log2(||A||_1 / theta_13))_+ (Sec. 3.1)."""
    if norm1 <= theta13 or norm1 == 0.0:
        return 0
    return max(0, int(math.ceil(math.log2(norm1 / theta13))))


def expm_pade13(A: np.ndarray, theta13: float = DEFAULTS["theta13"]) -> np.ndarray:
    """exp(A) by the degree-13 diagonal Pade approximant with scaling and squaring."""
    N = A.shape[0]
    norm1 = float(np.max(np.abs(A).sum(axis=0))) if N else 0.0
    s = squarings(norm1, theta13)
    X = A / (2.0 ** s)
    c = pade13_coefficients()
    P = c[0] * np.eye(N)
    Q = c[0] * np.eye(N)
    Xk = np.eye(N)
    for j in range(1, 14):
        Xk = Xk @ X
        P = P + c[j] * Xk
        Q = Q + ((-1.0) ** j) * c[j] * Xk
    R = np.linalg.solve(Q, P)
    for _ in range(s):
        R = R @ R
    return R


# --------------------------------------------------------------------------------------
# phi of the symmetric Lanczos matrix directly (the alternative Sec. 5 proposes to the
# augmented exponential when A is symmetric): phi_j(tau T) e_1 = Q phi_j(tau L) Q^T e_1
# with T = Q L Q^T (numpy's symmetric eigensolver as the library step)
# --------------------------------------------------------------------------------------
def phi_scalars(z: np.ndarray, kmax: int) -> np.ndarray:
    """phi_0(z) .. phi_kmax(z) for real z (rows k).  |z| < 1: the series
    phi_k(z) = sum_i z^i / (i+k)! of Eq. (phifunctions), summed to 30 terms; otherwise
    phi_0 = e^z and the recurrence of Eq. (phirelation), phi_k = (phi_{k-1} - 1/(k-1)!)/z."""
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros((kmax + 1, z.size))
    small = np.abs(z) < 1.0
    for k in range(kmax + 1):
        zs = z[small]
        acc = np.zeros_like(zs)
        term = np.full_like(zs, 1.0 / math.factorial(k))
        for i in range(30):
            acc = acc + term
            term = term * zs / (i + 1 + k)
        out[k, small] = acc
    zb = z[~small]
    prev = np.exp(zb)
    out[0, ~small] = prev
    for k in range(1, kmax + 1):
        prev = (prev - 1.0 / math.factorial(k - 1)) / zb
        out[k, ~small] = prev
    return out


def phi_columns_tridiagonal(T_m: np.ndarray, tau: float, p: int):
    """phi_p(tau T_m) e_1 and phi_{p+1}(tau T_m) e_1 (phi_0 = exp for p = 0) of a symmetric
    tridiagonal T_m, through its eigen-decomposition; the same vectors as the top m
    entries of columns m+p-1 and m+p of exp(H_hat) (reading R2)."""
    lam, Q = np.linalg.eigh(T_m)
    ph = phi_scalars(tau * lam, p + 1)
    q1 = Q[0, :]
    return Q @ (ph[p] * q1), Q @ (ph[p + 1] * q1)


def expm_cost_factor(norm1: float, theta13: float = DEFAULTS["theta13"]) -> float:
    """M of Eq. (8): 44/3 + 2 ceil(log2(||A||_1/5.37))_+."""
    return 44.0 / 3.0 + 2.0 * squarings(norm1, theta13)


def step_cost(m: float, p: int, nnz: int, n: int, M: float, symmetric: bool) -> float:
    """C_1(m) of Eq. (4)."""
    if symmetric:
        return (m + p) * nnz + 3.0 * (m + p) * n + M * (m + p + 1) ** 3
    return (m + p) * nnz + (m * m + 3 * p + 2) * n + M * (m + p + 1) ** 3


def total_cost(tau: float, m: float, t_left: float, p: int, nnz: int, n: int, M: float, symmetric: bool) -> float:
    """C(tau, m) of Eq. (5)."""
    return math.ceil(t_left / tau) * step_cost(m, p, nnz, n, M, symmetric)


def initial_tau(norm_A: float, norm_b0: float, tol: float, m_bar: float) -> float:
    """Eq. (tau_0), evaluated in logarithms."""
    lg = (math.log(tol) + (m_bar + 1.0) * (math.log(m_bar + 1.0) - 1.0)
          + 0.5 * math.log(2.0 * math.pi * (m_bar + 1.0)) - math.log(4.0 * norm_A * norm_b0))
    return 10.0 / norm_A * math.exp(lg / m_bar)


# --------------------------------------------------------------------------------------
# the controller (Sec. 3.4, Algorithm 4 and the branch of Algorithm 3)
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class AttemptMemory:
    """What Algorithm 4 remembers from the previous attempt within one step."""
    rejected: bool = False        # previous attempt of this step was rejected
    tau_changed: bool = False     # ... and it changed tau
    m_changed: bool = False       # ... and it changed m
    q_from_formula: bool = False  # q_hat came from Eq. (6) (computed or kept)
    k_from_formula: bool = False  # kappa_hat came from Eq. (7)
    q_hat: float = 0.0
    kappa_hat: float = 2.0
    eps_old: float = 0.0
    tau_old: float = 0.0
    m_old: int = 0


def controller(eps: float, omega: float, tau: float, m: int, mem: AttemptMemory, prm: dict):
    """Algorithm 4: returns (q_hat, tau_new, kappa_hat, m_new_real); updates mem's q/kappa."""
    gamma = prm["gamma"]
    if mem.rejected and mem.tau_changed:
        q = math.log(eps / mem.eps_old) / math.log(tau / mem.tau_old) - 1.0 if (
            eps > 0 and mem.eps_old > 0 and tau != mem.tau_old) else float("nan")
        if not math.isfinite(q):
            q, from_f = m / 4.0, False
        else:
            q, from_f = min(max(q, 0.0), float(m)), True
    elif mem.rejected and mem.q_from_formula:
        q, from_f = mem.q_hat, True
    else:
        q, from_f = m / 4.0, False
    mem.q_hat, mem.q_from_formula = q, from_f
    tau_new = tau * (gamma / omega) ** (1.0 / (q + 1.0)) if omega > 0 else math.inf

    if mem.rejected and mem.m_changed:
        k = (eps / mem.eps_old) ** (1.0 / (mem.m_old - m)) if (
            eps > 0 and mem.eps_old > 0 and m != mem.m_old) else float("nan")
        if not math.isfinite(k) or k <= 1.0:
            k, kf = 2.0, False
        else:
            kf = True
    elif mem.rejected and mem.k_from_formula:
        k, kf = mem.kappa_hat, True
    else:
        k, kf = 2.0, False
    mem.kappa_hat, mem.k_from_formula = k, kf
    m_new = m + math.log(omega / gamma) / math.log(k) if omega > 0 else -math.inf
    return q, tau_new, k, m_new


def w_recurrence(matvec, u: np.ndarray, b: list, t: float) -> list:
    """Eq. (wrecurrence): w_0 = u(t_k), w_j = A w_{j-1} + sum_{l=0}^{p-j} t_k^l/l! b_{j+l}."""
    p = len(b) - 1
    W = [u]
    for j in range(1, p + 1):
        wj = matvec(W[j - 1])
        for ell in range(0, p - j + 1):
            wj = wj + (t ** ell / math.factorial(ell)) * b[j + ell]
        W.append(wj)
    return W


def step_update(F: np.ndarray, W: list, tau: float) -> np.ndarray:
    """Eq. (step): u_{k+1} = tau^p phi_p(tau A) w_p + sum_{j<p} tau^j/j! w_j, with F the first term."""
    u = F.copy()
    for j in range(len(W) - 1):
        u = u + (tau ** j / math.factorial(j)) * W[j]
    return u


def omega_ratio(eps: float, tau: float, t_end: float, tol: float) -> float:
    """omega of Eq. (taunew): t_end ||eps|| / (tau Tol)."""
    return t_end * eps / (tau * tol)


def krylov_attempt(matvec, krylov, v: np.ndarray, tau: float, m: int, p: int, bd_abs: float,
                   theta13: float = DEFAULTS["theta13"], phi_method: str = "augmented"):
    """One attempt of Algorithm 3: F ~ tau^p phi_p(tau A) v and its estimate eps.

    Krylov projection (Algorithm 1 or 2), augmented matrix (Eq. hathm, R2),
    exponential, then Eq. (phipapprox2) and Eq. (errest) for tau*A, scaled by
    tau^p (reading R4).  Returns (F, eps, m_eff, ||H_hat||_1, beta)."""
    n = v.size
    beta = float(np.linalg.norm(v))
    if beta == 0.0:
        return np.zeros(n), 0.0, m, float(p > 0), 0.0
    V, H, m_eff = krylov(matvec, v, m, bd_abs)
    Hh = augmented_matrix(H[:m_eff, :m_eff], tau, p)
    norm1_Hh = float(np.max(np.abs(Hh).sum(axis=0)))
    if phi_method == "eigen":       # symmetric T_m (Lanczos): phi directly, Sec. 5
        phi_p, phi_p1 = phi_columns_tridiagonal(H[:m_eff, :m_eff], tau, p)
    else:
        E = expm_pade13(Hh, theta13)
        phi_p = E[:m_eff, m_eff + p - 1] if p >= 1 else E[:m_eff, 0]
        phi_p1 = E[:m_eff, m_eff + p]
    h_last = H[m_eff, m_eff - 1]
    F = (tau ** p) * beta * (V[:m_eff].T @ phi_p + tau * h_last * phi_p1[m_eff - 1] * V[m_eff])
    eps = (tau ** (p + 1)) * beta * abs(h_last) * abs(phi_p1[m_eff - 1])
    return F, eps, m_eff, norm1_Hh, beta


# --------------------------------------------------------------------------------------
# phipm (Algorithm 3)
# --------------------------------------------------------------------------------------
class PhipmError(RuntimeError):
    pass


@dataclasses.dataclass
class Stats:
    steps: int = 0
    rejects: int = 0
    matvecs: int = 0
    expms: int = 0
    err_est_sum: float = 0.0


def phipm(t_end: float, A, b, tol: float = 1e-7, symm: int = -1, params: dict | None = None,
          trace: list | None = None):
    """u(t_end) = sum_k t_end^k phi_k(t_end A) b_k by Algorithm 3 (Sec. 3.3-3.5).

    A: workloads.Stencil / workloads.CSR (or an oracle Operator); b: list of
    p+1 float64 vectors.  Returns (u, Stats).  If trace is a list, one dict per
    attempt is appended to it."""
    prm = dict(DEFAULTS)
    if params:
        prm.update(params)
    op = A if isinstance(A, Operator) else Operator(A)
    b = [np.asarray(x, dtype=np.float64) for x in b]
    p = len(b) - 1
    n = op.n
    stats = Stats()
    if tol <= 0:
        tol = 1e-7                          # default tolerance, Sec. 3.5
    symmetric = op.is_symmetric() if symm < 0 else bool(symm)
    krylov = lanczos if symmetric else arnoldi
    norm_A = op.norm_inf()
    nnz = op.nnz
    norm_b0 = float(np.max(np.abs(b[0]))) if n else 0.0
    if norm_b0 == 0.0:
        norm_b0 = max((float(np.max(np.abs(x))) for x in b), default=0.0) if n else 0.0
    if n == 0 or norm_b0 == 0.0:
        return np.zeros(n), stats
    m_max = int(prm["m_max"])
    m = min(int(prm["m_init"]), m_max)
    bd_abs = prm["breakdown_tol"] * max(norm_A, np.finfo(float).tiny)
    if norm_A == 0.0:                       # A = 0: u = sum_k t^k/k! b_k, one step is exact
        tau = t_end
    else:
        tau = min(initial_tau(norm_A, norm_b0, tol, 0.5 * (prm["m_init"] + m_max)), t_end)

    u = b[0].copy()
    t = 0.0
    nonfinite_run = 0
    while t < t_end:
        # Eq. (wrecurrence): w_0 = u, w_j = A w_{j-1} + sum_l t^l/l! b_{j+l}
        W = w_recurrence(op.matvec, u, b, t)
        stats.matvecs += p
        mem = AttemptMemory()
        while True:
            tau_used, m_used = tau, m
            F, eps, m_eff, norm1_Hh, beta = krylov_attempt(op.matvec, krylov, W[p], tau_used, m_used, p, bd_abs,
                                                           prm["theta13"],
                                                           prm["phi_method"] if symmetric else "augmented")
            if beta > 0.0:
                stats.matvecs += m_eff
                stats.expms += 1
            if not math.isfinite(eps):
                nonfinite_run += 1
                stats.rejects += 1
                if nonfinite_run >= 10:
                    raise PhipmError("non-finite error estimate")
                tau = tau / 5.0
                mem = AttemptMemory()
                continue
            nonfinite_run = 0
            m = m_eff
            omega = omega_ratio(eps, tau_used, t_end, tol)
            q, tau_new, kap, m_new_real = controller(eps, omega, tau_used, m, mem, prm)
            m_new = min(max(math.ceil(m_new_real), 1), m_max) if math.isfinite(m_new_real) else (
                1 if m_new_real < 0 else m_max)
            M = expm_cost_factor(norm1_Hh, prm["theta13"])           # Eq. (8), reading R14
            t_left = t_end - t
            c_tau = total_cost(tau_new, m, t_left, p, nnz, n, M, symmetric)
            c_m = total_cost(tau_used, m_new, t_left, p, nnz, n, M, symmetric)
            m_cand = min(max(m_new, (3 * m) // 4, 1), math.ceil(4 * m / 3), m_max)
            if c_tau < c_m or m_cand == m or not prm["adapt_m"]:   # Algorithm 3 branch; R19; phip
                tau = min(max(tau_new, tau_used / 5.0), 2.0 * tau_used, t_left)
                branch = "tau"
            else:
                m = m_cand
                branch = "m"
            accepted = omega <= prm["delta"]
            if trace is not None:
                trace.append(dict(step=stats.steps, t=t, tau=tau_used, m=m_eff, eps=eps, omega=omega,
                                  accepted=accepted, q_hat=q, kappa_hat=kap, tau_new=tau_new,
                                  m_new=m_new, branch=branch, beta=beta, next_tau=tau, next_m=m,
                                  cost_tau=c_tau, cost_m=c_m))
            if accepted:
                break
            stats.rejects += 1
            if stats.rejects > prm["max_rejects"]:
                raise PhipmError("too many rejected attempts")
            mem.rejected = True
            mem.tau_changed = branch == "tau"
            mem.m_changed = branch == "m"
            mem.eps_old, mem.tau_old, mem.m_old = eps, tau_used, m_eff
        # Eq. (step): u_{k+1} = tau^p phi_p(tau A) w_p + sum_{j<p} tau^j/j! w_j
        u = step_update(F, W, tau_used)
        stats.steps += 1
        stats.err_est_sum += eps
        if stats.steps > prm["max_steps"]:
            raise PhipmError("too many steps")
        last = tau_used >= t_end - t
        t = t_end if last else t + tau_used
        tau = min(tau, t_end - t) if t < t_end else tau
    return u, stats


def phip(t_end: float, A, b, tol: float = 1e-7, symm: int = -1, m: int = 30,
         params: dict | None = None, trace: list | None = None):
    """The fixed-dimension variant of Sec. 4.2 (m = 30 there): phipm with adapt_m off (R20).
    m_max keeps its default (it enters only Eq. tau_0 through m_bar)."""
    prm = dict(params or {})
    prm.update(adapt_m=False, m_init=m)
    return phipm(t_end, A, b, tol, symm, prm, trace)


def shifted_inputs(b: list, t1: float) -> list:
    """Inputs that restart Eq. (phide) at t1 (Lemma 2.1 / Eq. steppre):
    b'_0 = u(t1) is supplied by the caller; b'_i = sum_{l=0}^{p-i} t1^l/l! b_{i+l}."""
    p = len(b) - 1
    out = [None]
    for i in range(1, p + 1):
        acc = np.zeros_like(b[i])
        for ell in range(0, p - i + 1):
            acc = acc + (t1 ** ell / math.factorial(ell)) * b[i + ell]
        out.append(acc)
    return out
