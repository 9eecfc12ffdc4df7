// The phipm method on the device (Niesen & Wright, Sec. 3), written once over
// a "team" of CTAs that share one problem:
//   GridTeam  every CTA of a cooperative launch; bounded grid barriers,
//             per-CTA partial sums reduced in a fixed order (deterministic);
//   CtaTeam   one CTA; __syncthreads.
// S is the element type of the Krylov basis: double (FP64 mode) or float
// (FP32 mode: basis and SpMV in FP32 with FP32 accumulation, dot products
// accumulated as exact float products in float pairs, H / expm / eps in FP64).
//
// Every CTA of a team runs the same scalar code (controller, cost model) on
// bit-identical inputs, so all CTAs take the same decisions without a broadcast.
#pragma once
#include "phipm_common.cuh"

// FP32 basis mode: bound on ||F|| / ||u|| per step (F = tau^p phi_p(tau A) w_p)
#define PM_F32_AMP 32.0

template <class S> struct Elem;
template <> struct Elem<double> {
  typedef double Acc;
  __device__ static __forceinline__ Acc zero() { return 0.0; }
  __device__ static __forceinline__ void dot(Acc& a, double x, double y) { a = fma(x, y, a); }
  __device__ static __forceinline__ double val(const Acc& a) { return a; }
  __device__ static __forceinline__ double cvt(double x) { return x; }
  __device__ static __forceinline__ double coef(double c) { return c; }
};
template <> struct Elem<float> {
  typedef F2Acc Acc;
  __device__ static __forceinline__ Acc zero() { F2Acc a; a.hi = 0.f; a.lo = 0.f; return a; }
  __device__ static __forceinline__ void dot(Acc& a, float x, float y) { f2_add_prod(a, x, y); }
  __device__ static __forceinline__ double val(const Acc& a) { return f2_value(a); }
  __device__ static __forceinline__ float cvt(double x) { return (float)x; }
  __device__ static __forceinline__ float coef(double c) { return (float)c; }
};

// per-CTA shared state
struct PmShared {
  double H[(PM_MAXM + 1) * PM_MAXM];   // H[i * PM_MAXM + j], Hessenberg / tridiagonal
  double red[PM_WARPS][8];
  double coef[PM_NSLOT];               // reduced sums of the current phase
  double h1[PM_NSLOT];                 // first Gram-Schmidt pass coefficients
  float hf[PM_NSLOT];                  // coefficients as float (FP32 update)
  double phi0[PM_NA], phi1[PM_NA];     // phi_p(tau H) e1 and phi_{p+1}(tau H) e1
  double ucoef[PM_NSLOT + PM_MAXP + 1];
  double mat_norm;
  double dred[PM_NSLOT + PM_WARPS];    // per-unit partial dots (vector, row chunk)
  int ipiv[PM_NA];
  int flag;
};

struct PmWork {
  double* partials;     // [2][G][PM_NSLOT] (grid team)
  double* phi_g;        // [2][2][PM_NA]   (grid team)
  double* expm;         // per-CTA: 8 * PM_NA2 doubles
};

// ------------------------------------------------------------------------------------
// team reductions of K values held in s.coef[0..K) by each CTA
// ------------------------------------------------------------------------------------
template <class Team>
__device__ bool team_sum(const Team& team, PmShared& s, int K, const PmWork& w, int& parity) {
  if (!Team::multi) { __syncthreads(); return true; }
  const int G = team.size(), r = team.rank();
  double* P = w.partials + (size_t)parity * G * PM_NSLOT;
  parity ^= 1;
  for (int k = threadIdx.x; k < K; k += blockDim.x) P[(size_t)r * PM_NSLOT + k] = s.coef[k];
  if (!team.sync()) return false;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < K; k += PM_WARPS) {
    double a = 0.0;
    for (int g = lane; g < G; g += 32) a += __ldcg(&P[(size_t)g * PM_NSLOT + k]);
    a = pm_warp_sum(a);
    if (lane == 0) s.coef[k] = a;
  }
  __syncthreads();
  return true;
}

template <class Team>
__device__ bool team_max(const Team& team, PmShared& s, int K, const PmWork& w, int& parity) {
  if (!Team::multi) { __syncthreads(); return true; }
  const int G = team.size(), r = team.rank();
  double* P = w.partials + (size_t)parity * G * PM_NSLOT;
  parity ^= 1;
  for (int k = threadIdx.x; k < K; k += blockDim.x) P[(size_t)r * PM_NSLOT + k] = s.coef[k];
  if (!team.sync()) return false;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < K; k += PM_WARPS) {
    double a = -1.0;
    for (int g = lane; g < G; g += 32) a = fmax(a, __ldcg(&P[(size_t)g * PM_NSLOT + k]));
    a = pm_warp_max(a);
    if (lane == 0) s.coef[k] = a;
  }
  __syncthreads();
  return true;
}

// block-wide sums of 8 per-thread values into out[0..cnt)
__device__ __forceinline__ void block_sum8(PmShared& s, double v[8], int cnt, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k < cnt) {
      double a = pm_warp_sum(v[k]);
      if (lane == 0) s.red[warp][k] = a;
    }
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double a = 0.0;
    for (int q = 0; q < PM_WARPS; ++q) a += s.red[q][threadIdx.x];
    out[threadIdx.x] = a;
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------
// SpMV rows
// ------------------------------------------------------------------------------------
// y_r = (A x)_r with x given by a loader functor (element index -> value of type T)
template <class T, class XL>
__device__ __forceinline__ T spmv_row(const DevOp& A, int r, const XL& x) {
  if (A.kind == 0) {
    const int k0 = __ldg(&A.rowptr[r]), k1 = __ldg(&A.rowptr[r + 1]);
    T acc = T(0);
    if (sizeof(T) == 8) {
      for (int k = k0; k < k1; ++k) acc = fma((double)__ldg(&A.val[k]), (double)x(__ldg(&A.colind[k])), (double)acc);
    } else {
      for (int k = k0; k < k1; ++k) acc = fmaf(__ldg(&A.valf[k]), (float)x(__ldg(&A.colind[k])), (float)acc);
    }
    return acc;
  }
  const int nx = A.nx, ny = A.ny;
  const int ix = r % nx;
  const int iy = (r / nx) % ny;
  const int iz = r / (nx * ny);
  T acc = T(A.cc) * x(r);
  if (ix > 0) acc += T(A.cm[0]) * x(r - 1);
  if (ix < nx - 1) acc += T(A.cp[0]) * x(r + 1);
  if (A.ndim > 1) {
    if (iy > 0) acc += T(A.cm[1]) * x(r - nx);
    if (iy < ny - 1) acc += T(A.cp[1]) * x(r + nx);
  }
  if (A.ndim > 2) {
    const int pl = nx * ny;
    if (iz > 0) acc += T(A.cm[2]) * x(r - pl);
    if (iz < A.nz - 1) acc += T(A.cp[2]) * x(r + pl);
  }
  return acc;
}

template <class T> struct LoadScaled {
  const T* p; double s;
  __device__ __forceinline__ T operator()(int i) const { return (T)((double)p[i] * s); }
};
template <class T> struct LoadScaledF {    // FP32 vector times a float scale
  const T* p; float s;
  __device__ __forceinline__ T operator()(int i) const { return p[i] * s; }
};
struct LoadD {
  const double* p;
  __device__ __forceinline__ double operator()(int i) const { return p[i]; }
};
struct LoadDtoF {                         // FP64 vector scaled, rounded to float
  const double* p; double s;
  __device__ __forceinline__ float operator()(int i) const { return (float)(p[i] * s); }
};

// ------------------------------------------------------------------------------------
// Gram-Schmidt passes over this CTA's rows [lo, hi)
// ------------------------------------------------------------------------------------
// d_i = sum_r V[i0+i][r] y[r], i < nv, into s.coef[0..nv).  Work is split into
// units (vector i, row chunk c) handled by one warp each, so the cross-lane sum
// runs once per unit rather than once per vector per warp.
template <class S> struct Quad;
template <> struct Quad<float> {
  float x[4];
  __device__ __forceinline__ void load(const float* p) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
  }
  __device__ __forceinline__ void store(float* p) const { *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]); }
};
template <> struct Quad<double> {
  double x[4];
  __device__ __forceinline__ void load(const double* p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
  }
  __device__ __forceinline__ void store(double* p) const {
    reinterpret_cast<double2*>(p)[0] = make_double2(x[0], x[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(x[2], x[3]);
  }
};

// d_i = sum_r V[i0+i][r] y[r], i < nv, into s.coef[0..nv).  Work is split into
// units (vector i, row chunk c) handled by one warp each, so the cross-lane sum
// runs once per unit rather than once per vector per warp.  lo is a multiple of
// 64 and vectors are 256-byte aligned, so chunks start on 16-byte boundaries.
template <class S>
__device__ void dots_cta(const S* __restrict__ V, long long ld, int i0, int nv, const S* __restrict__ y, int lo, int hi,
                         PmShared& s) {
  typedef Elem<S> E;
  typedef typename E::Acc Acc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = hi - lo;
  int cpv = (PM_WARPS + nv - 1) / nv;                     // chunks per vector
  cpv = max(1, min(cpv, (rows + 255) / 256));
  const int units = nv * cpv;
  const int chunk = (((rows + cpv - 1) / cpv) + 127) & ~127;
  for (int un = warp; un < units; un += PM_WARPS) {
    const int i = un / cpv, c = un - i * cpv;
    const int a = lo + c * chunk;
    const int b = min(hi, a + chunk);
    const S* v = V + (size_t)(i0 + i) * ld;
    Acc acc0 = E::zero(), acc1 = E::zero();
    int e = a + 4 * lane;
    for (; e + 128 + 3 < b; e += 256) {
      Quad<S> v0, y0, v1, y1;
      v0.load(v + e); y0.load(y + e); v1.load(v + e + 128); y1.load(y + e + 128);
#pragma unroll
      for (int k = 0; k < 4; ++k) { E::dot(acc0, v0.x[k], y0.x[k]); E::dot(acc1, v1.x[k], y1.x[k]); }
    }
    for (; e + 3 < b; e += 128) {
      Quad<S> v0, y0;
      v0.load(v + e); y0.load(y + e);
#pragma unroll
      for (int k = 0; k < 4; ++k) E::dot(acc0, v0.x[k], y0.x[k]);
    }
    for (int r = e; r < b && r < e + 4; ++r) E::dot(acc1, v[r], y[r]);
    const double d = pm_warp_sum(E::val(acc0) + E::val(acc1));
    if (lane == 0) s.dred[un] = d;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < cpv; ++c) t += s.dred[i * cpv + c];
    s.coef[i] = t;
  }
  __syncthreads();
}

// y[r] -= sum_{i<nv} h_i V[i][r] over this CTA's rows, four consecutive rows per
// thread; returns this thread's sum of y[r]^2.  Element types: FP64 with FP64
// coefficients, or FP32 with the coefficients rounded to FP32 (FP32 accumulation).
template <class S, class C>
__device__ __forceinline__ double update_rows(S* __restrict__ y, const S* __restrict__ V, long long ld, int nv,
                                              const C* h, int lo, int hi) {
  double nrm = 0.0;
  for (int r = lo + 4 * threadIdx.x; r < hi; r += 4 * blockDim.x) {
    if (r + 3 < hi) {
      Quad<S> a, b;
      a.load(y + r);
#pragma unroll
      for (int k = 0; k < 4; ++k) b.x[k] = S(0);
      int i = 0;
      for (; i + 1 < nv; i += 2) {
        Quad<S> v0, v1;
        v0.load(V + (size_t)i * ld + r);
        v1.load(V + (size_t)(i + 1) * ld + r);
        const S h0 = (S)h[i], h1 = (S)h[i + 1];
#pragma unroll
        for (int k = 0; k < 4; ++k) { a.x[k] = fma(-h0, v0.x[k], a.x[k]); b.x[k] = fma(-h1, v1.x[k], b.x[k]); }
      }
      if (i < nv) {
        Quad<S> v0;
        v0.load(V + (size_t)i * ld + r);
        const S h0 = (S)h[i];
#pragma unroll
        for (int k = 0; k < 4; ++k) a.x[k] = fma(-h0, v0.x[k], a.x[k]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        a.x[k] += b.x[k];
        nrm = fma((double)a.x[k], (double)a.x[k], nrm);
      }
      a.store(y + r);
    } else {
      for (int q = r; q < hi; ++q) {
        S a = y[q];
        for (int i = 0; i < nv; ++i) a = fma(-(S)h[i], V[(size_t)i * ld + q], a);
        y[q] = a;
        nrm = fma((double)a, (double)a, nrm);
      }
    }
  }
  return nrm;
}

// ------------------------------------------------------------------------------------
// dense kernels of one CTA on small matrices (FP64): the exponential of H_hat
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void mm_cta(double* C, const double* A, const double* B, int N) {
  const int NN = N * N;
  for (int e = threadIdx.x; e < NN; e += blockDim.x) {
    const int i = e / N, j = e - i * N;
    const double* a = A + i * PM_NA;
    double acc = 0.0;
    for (int k = 0; k < N; ++k) acc = fma(a[k], B[k * PM_NA + j], acc);
    C[i * PM_NA + j] = acc;
  }
  __syncthreads();
}

// exp(Hh) by the degree-13 Pade approximant (even/odd split) with s squarings;
// writes the top m entries of columns ca and cb to out0/out1.
__device__ void expm_cta(PmShared& s, double tau, int m, int p, int N, int sq, const double* bc, double* ws,
                         int ca, int cb, double* out0, double* out1) {
  double* X = ws;
  double* X2 = ws + 1 * PM_NA2;
  double* X4 = ws + 2 * PM_NA2;
  double* X6 = ws + 3 * PM_NA2;
  double* T1 = ws + 4 * PM_NA2;
  double* T2 = ws + 5 * PM_NA2;
  double* U = ws + 6 * PM_NA2;
  double* Vm = ws + 7 * PM_NA2;
  const double sc = ldexp(1.0, -sq);
  const int NN = N * N;
  // X = H_hat / 2^s with H_hat = [[tau H_m, e_1, 0], [0, 0, I_p], [0, 0, 0]]  (Eq. hathm, size m+p+1)
  for (int e = threadIdx.x; e < NN; e += blockDim.x) {
    const int i = e / N, j = e - i * N;
    double v = 0.0;
    if (i < m && j < m) v = tau * s.H[i * PM_MAXM + j];
    else if (i == 0 && j == m) v = 1.0;
    else if (i >= m && j == i + 1) v = 1.0;
    X[i * PM_NA + j] = v * sc;
  }
  __syncthreads();
  (void)p;
  mm_cta(X2, X, X, N);
  mm_cta(X4, X2, X2, N);
  mm_cta(X6, X4, X2, N);
  for (int e = threadIdx.x; e < NN; e += blockDim.x) {
    const int i = e / N, j = e - i * N, o = i * PM_NA + j;
    T1[o] = bc[13] * X6[o] + bc[11] * X4[o] + bc[9] * X2[o];
    T2[o] = bc[12] * X6[o] + bc[10] * X4[o] + bc[8] * X2[o];
  }
  __syncthreads();
  mm_cta(U, X6, T1, N);                  // U <- X6 * T1  (odd inner)
  mm_cta(Vm, X6, T2, N);                 // V <- X6 * T2  (even)
  for (int e = threadIdx.x; e < NN; e += blockDim.x) {
    const int i = e / N, j = e - i * N, o = i * PM_NA + j;
    const double id = (i == j) ? 1.0 : 0.0;
    T1[o] = U[o] + bc[7] * X6[o] + bc[5] * X4[o] + bc[3] * X2[o] + bc[1] * id;
    Vm[o] = Vm[o] + bc[6] * X6[o] + bc[4] * X4[o] + bc[2] * X2[o] + bc[0] * id;
  }
  __syncthreads();
  mm_cta(U, X, T1, N);                   // U = X * (...)
  // P = V + U -> T2 ;  Q = V - U -> X2 (reuse)
  for (int e = threadIdx.x; e < NN; e += blockDim.x) {
    const int i = e / N, j = e - i * N, o = i * PM_NA + j;
    T2[o] = Vm[o] + U[o];
    X2[o] = Vm[o] - U[o];
  }
  __syncthreads();
  double* Q = X2;
  double* R = T2;
  // LU with partial pivoting of Q; the same row swaps applied to R (= P)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k < N; ++k) {
    if (warp == 0) {
      double best = -1.0;
      int bi = k;
      for (int i = k + lane; i < N; i += 32) {
        double a = fabs(Q[i * PM_NA + k]);
        if (a > best) { best = a; bi = i; }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) s.ipiv[k] = bi;
    }
    __syncthreads();
    const int pv = s.ipiv[k];
    if (pv != k) {
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double t = Q[k * PM_NA + j]; Q[k * PM_NA + j] = Q[pv * PM_NA + j]; Q[pv * PM_NA + j] = t;
        t = R[k * PM_NA + j]; R[k * PM_NA + j] = R[pv * PM_NA + j]; R[pv * PM_NA + j] = t;
      }
      __syncthreads();
    }
    const double piv = Q[k * PM_NA + k];
    for (int i = k + 1 + threadIdx.x; i < N; i += blockDim.x) Q[i * PM_NA + k] /= piv;
    __syncthreads();
    const int rows = N - k - 1;
    const int tot = rows * (2 * N - k - 1);   // trailing Q block (rows x (N-k-1)) and R rows (rows x N)
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int i = k + 1 + e / (2 * N - k - 1);
      const int c = e % (2 * N - k - 1);
      const double l = Q[i * PM_NA + k];
      if (c < N - k - 1) {
        const int j = k + 1 + c;
        Q[i * PM_NA + j] = fma(-l, Q[k * PM_NA + j], Q[i * PM_NA + j]);
      } else {
        const int j = c - (N - k - 1);
        R[i * PM_NA + j] = fma(-l, R[k * PM_NA + j], R[i * PM_NA + j]);
      }
    }
    __syncthreads();
  }
  // back substitution U R = (L^{-1} P R) column-parallel over all N columns
  for (int k = N - 1; k >= 0; --k) {
    const double d = Q[k * PM_NA + k];
    for (int j = threadIdx.x; j < N; j += blockDim.x) R[k * PM_NA + j] /= d;
    __syncthreads();
    const int tot = k * N;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int i = e / N, j = e - i * N;
      R[i * PM_NA + j] = fma(-Q[i * PM_NA + k], R[k * PM_NA + j], R[i * PM_NA + j]);
    }
    __syncthreads();
  }
  // squarings
  double* cur = R;
  double* oth = U;
  for (int q = 0; q < sq; ++q) {
    mm_cta(oth, cur, cur, N);
    double* t = cur; cur = oth; oth = t;
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    out0[i] = cur[i * PM_NA + ca];
    out1[i] = cur[i * PM_NA + cb];
  }
  __syncthreads();
}

__device__ __forceinline__ int pm_squarings(double norm1, double theta) {
  if (!(norm1 > theta)) return 0;
  const double v = ceil(log2(norm1 / theta));
  return v > 0 ? (int)v : 0;
}

// ------------------------------------------------------------------------------------
// the solver
// ------------------------------------------------------------------------------------
struct Ctl {   // controller memory of Algorithm 4 within one step
  bool rejected, tau_changed, m_changed, qf, kf;
  double q, kap, eps_old, tau_old;
  int m_old;
};

template <class Team, class S>
__device__ void phipm_device(const Team& team, const DevProblem& P, const DevParams& prm, DevResult& res,
                             PmShared& s, const PmWork& w, double* expm_ws) {
  typedef Elem<S> E;
  typedef typename E::Acc Acc;
  const int n = P.A.n, p = P.p;
  const int tid = threadIdx.x, nth = blockDim.x;
  int lo, hi;
  pm_rows(n, team.rank(), team.size(), lo, hi);
  const long long ld = P.ld;
  S* V = (S*)P.V;
  S* Y = (S*)P.Y;
  double* W = P.W;
  double* u = P.u;                        // current solution u(t_k)
  double* ualt = P.W + (size_t)p * P.ld;  // spare vector (FP32 guard)
  int parity = 0;
  int status = PM_OK;
  long long steps = 0, rejects = 0, matvecs = 0, expms = 0, kry_steps = 0, gs_vectors = 0;
  double err_sum = 0.0;
  double r_normA = 0.0, r_normb = 0.0, r_last_tau = 0.0;
  int r_last_m = 0;
  bool symmetric = false;
  for (int e = threadIdx.x; e < (PM_MAXM + 1) * PM_MAXM; e += blockDim.x) s.H[e] = 0.0;
  __syncthreads();

#define PM_SYNC_OR_FAIL() do { if (!team.sync()) { status = PM_ETIMEOUT; goto done; } } while (0)
#define PM_SUM_OR_FAIL(K) do { if (!team_sum(team, s, (K), w, parity)) { status = PM_ETIMEOUT; goto done; } } while (0)
#define PM_MAX_OR_FAIL(K) do { if (!team_max(team, s, (K), w, parity)) { status = PM_ETIMEOUT; goto done; } } while (0)

  // ---------------- setup (a1): ||A||_inf, ||b_0||_inf, max_k ||b_k||_inf, symmetry; u = b_0
  {
    double na = 0.0, nb0 = 0.0, nball = 0.0, asym = 0.0;
    for (int r = lo + tid; r < hi; r += nth) {
      if (P.A.kind == 0) {
        const int k0 = P.A.rowptr[r], k1 = P.A.rowptr[r + 1];
        double rs = 0.0;
        for (int k = k0; k < k1; ++k) {
          const double a = P.A.val[k];
          rs += fabs(a);
          if (P.symm < 0) {       // look for the transposed entry in row colind[k]
            const int c = P.A.colind[k];
            const int q0 = P.A.rowptr[c], q1 = P.A.rowptr[c + 1];
            bool found = false;
            for (int q = q0; q < q1; ++q)
              if (P.A.colind[q] == r) { found = true; if (P.A.val[q] != a) asym = 1.0; }
            if (!found && a != 0.0) asym = 1.0;
          }
        }
        na = fmax(na, rs);
      }
      const double b0 = fabs(P.b[0][r]);
      nb0 = fmax(nb0, b0);
      nball = fmax(nball, b0);
      for (int k = 1; k <= p; ++k) nball = fmax(nball, fabs(P.b[k][r]));
      u[r] = P.b[0][r];
    }
    const double t0 = pm_warp_max(na), t1 = pm_warp_max(nb0), t2 = pm_warp_max(nball), t3 = pm_warp_max(asym);
    __shared__ double red4[PM_WARPS][4];
    if ((tid & 31) == 0) { red4[tid >> 5][0] = t0; red4[tid >> 5][1] = t1; red4[tid >> 5][2] = t2; red4[tid >> 5][3] = t3; }
    __syncthreads();
    if (tid < 4) {
      double a = 0.0;
      for (int q = 0; q < PM_WARPS; ++q) a = fmax(a, red4[q][tid]);
      s.coef[tid] = a;
    }
    __syncthreads();
    PM_MAX_OR_FAIL(4);
  }
  {
    double normA;
    if (P.A.kind == 0) {
      normA = s.coef[0];
    } else {
      normA = fabs(P.A.cc);
      for (int d = 0; d < P.A.ndim; ++d) normA += fabs(P.A.cm[d]) + fabs(P.A.cp[d]);
    }
    double normb = s.coef[1];
    const double normb_all = s.coef[2];
    if (P.symm >= 0) symmetric = P.symm != 0;
    else if (P.A.kind == 0) symmetric = s.coef[3] == 0.0;
    else {
      symmetric = true;
      for (int d = 0; d < P.A.ndim; ++d) symmetric = symmetric && (P.A.cm[d] == P.A.cp[d]);
    }
    if (normb == 0.0) normb = normb_all;
    r_normA = normA;
    r_normb = normb;
    if (n == 0 || normb == 0.0) {        // every b_k = 0: u = 0
      for (int r = lo + tid; r < hi; r += nth) u[r] = 0.0;
      goto done;
    }
    const double tol = P.tol > 0.0 ? P.tol : 1e-7;
    const double t_end = P.t_end;
    const int m_max = prm.m_max;
    int m = min(prm.m_init, m_max);
    const double bd_abs = prm.breakdown_tol * fmax(normA, 2.2250738585072014e-308);
    double tau;
    if (normA == 0.0) {
      tau = t_end;
    } else {       // Eq. (tau_0) in logarithms, m_bar = (m_init + m_max)/2
      const double mb = 0.5 * (prm.m_init + m_max);
      const double lg = log(tol) + (mb + 1.0) * (log(mb + 1.0) - 1.0) + 0.5 * log(2.0 * 3.141592653589793 * (mb + 1.0)) -
                        log(4.0 * normA * normb);
      tau = fmin(10.0 / normA * exp(lg / mb), t_end);
    }
    const long long nnzA = P.A.nnz;
    PM_SYNC_OR_FAIL();          // u = b_0 complete before the first SpMV

    double t = 0.0;
    int nonfinite = 0;
    while (t < t_end) {
      // ---------------- w-recurrence (a2), Eq. (wrecurrence): p SpMVs in FP64
      double beta, unorm;
      {
        double tl[PM_MAXP + 1];
        tl[0] = 1.0;
        for (int l = 1; l <= p; ++l) tl[l] = tl[l - 1] * t / (double)l;
        for (int j = 1; j <= p; ++j) {
          const double* xin = (j == 1) ? u : W + (size_t)(j - 2) * ld;
          double* wout = W + (size_t)(j - 1) * ld;
          double nrm = 0.0;
          LoadD xl{xin};
          for (int r = lo + tid; r < hi; r += nth) {
            double y = spmv_row<double>(P.A, r, xl);
            for (int l = 0; l <= p - j; ++l) y = fma(tl[l], P.b[j + l][r], y);
            wout[r] = y;
            if (j == p) nrm = fma(y, y, nrm);
          }
          matvecs += 1;
          if (j == p) {
            double un = 0.0;
            for (int r = lo + tid; r < hi; r += nth) un = fma(u[r], u[r], un);
            double v[8] = {nrm, un, 0, 0, 0, 0, 0, 0};
            block_sum8(s, v, 2, s.coef);
            PM_SUM_OR_FAIL(2);
          } else {
            PM_SYNC_OR_FAIL();
          }
        }
        if (p == 0) {
          double nrm = 0.0;
          for (int r = lo + tid; r < hi; r += nth) nrm = fma(u[r], u[r], nrm);
          double v[8] = {nrm, nrm, 0, 0, 0, 0, 0, 0};
          block_sum8(s, v, 2, s.coef);
          PM_SUM_OR_FAIL(2);
        }
        beta = sqrt(s.coef[0]);
        unorm = sqrt(s.coef[1]);
      }
      const double* wp = (p == 0) ? u : W + (size_t)(p - 1) * ld;
      int kcur = 0;            // Arnoldi / Lanczos steps done for this w_p
      bool invariant = false;  // happy breakdown reached
      double ynorm_last = 0.0; // ||y|| of the last step (h_{kcur+1,kcur})
      Ctl ctl;
      ctl.rejected = ctl.tau_changed = ctl.m_changed = ctl.qf = ctl.kf = false;
      ctl.q = 0.0; ctl.kap = 2.0; ctl.eps_old = 0.0; ctl.tau_old = 0.0; ctl.m_old = 0;
      bool accepted = false;
      while (!accepted) {
        const double tau_used = tau;
        int m_used = m;
        double eps = 0.0, hlast = 0.0;
        int sq = 0;
        double norm1 = (p > 0) ? 1.0 : 0.0;
        if (beta > 0.0) {
          // ---------------- Krylov extension (a3/a4) to m steps
          const int target = invariant ? kcur : m;
          if (kcur < target) {
            const int j0 = kcur;       // first step of this extension
            for (int j = j0; j < target; ++j) {
              // phase A: x = v_j ; y = A x ; first-pass dots
              if (j == 0) {
                const double inv = 1.0 / beta;
                for (int r = lo + tid; r < hi; r += nth) V[r] = E::cvt(wp[r] * inv);
              } else if (j == j0) {
                // v_j already normalised in V[j] by the end of the previous extension
              } else {
                const S* yprev = Y + (size_t)((j - 1) & 1) * ld;
                const double inv = 1.0 / ynorm_last;
                for (int r = lo + tid; r < hi; r += nth) V[(size_t)j * ld + r] = E::cvt((double)yprev[r] * inv);
              }
              __syncthreads();
              S* ycur = Y + (size_t)(j & 1) * ld;
              if (j == 0) {
                if (sizeof(S) == 8) {
                  LoadScaled<double> xl{wp, 1.0 / beta};
                  for (int r = lo + tid; r < hi; r += nth) ycur[r] = (S)spmv_row<double>(P.A, r, xl);
                } else {
                  LoadDtoF xl{wp, 1.0 / beta};
                  for (int r = lo + tid; r < hi; r += nth) ycur[r] = (S)spmv_row<float>(P.A, r, xl);
                }
              } else if (j == j0) {
                const S* xv = V + (size_t)j * ld;
                if (sizeof(S) == 8) {
                  LoadD xl{(const double*)xv};
                  for (int r = lo + tid; r < hi; r += nth) ycur[r] = (S)spmv_row<double>(P.A, r, xl);
                } else {
                  LoadScaledF<float> xl{(const float*)xv, 1.0f};
                  for (int r = lo + tid; r < hi; r += nth) ycur[r] = (S)spmv_row<float>(P.A, r, xl);
                }
              } else {
                const S* yprev = Y + (size_t)((j - 1) & 1) * ld;
                if (sizeof(S) == 8) {
                  LoadScaled<double> xl{(const double*)yprev, 1.0 / ynorm_last};
                  for (int r = lo + tid; r < hi; r += nth) ycur[r] = (S)spmv_row<double>(P.A, r, xl);
                } else {
                  LoadScaledF<float> xl{(const float*)yprev, (float)(1.0 / ynorm_last)};
                  for (int r = lo + tid; r < hi; r += nth) ycur[r] = (S)spmv_row<float>(P.A, r, xl);
                }
              }
              matvecs += 1;
              kry_steps += 1;
              __syncthreads();
              const bool lanczos = symmetric && sizeof(S) == 8;
              if (!lanczos) gs_vectors += j + 1;
              const int i0 = lanczos ? j : 0;          // Lanczos: only t_jj = v_j^T y here
              const int nv = j + 1 - i0;
              // dots d_i = v_i . y over my rows
              dots_cta<S>(V, ld, i0, nv, ycur, lo, hi, s);
              PM_SUM_OR_FAIL(nv);
              if (lanczos) {
                // Algorithm 2: y <- y - t_{j,j-1} v_{j-1} - t_jj v_j ; t_{j+1,j} = ||y||
                const double tjj = s.coef[0];
                const double tjm = (j > 0) ? s.H[(j - 1) * PM_MAXM + j] : 0.0;
                __syncthreads();
                double nrm = 0.0;
                for (int r = lo + tid; r < hi; r += nth) {
                  double y = (double)ycur[r];
                  if (j > 0) y = fma(-tjm, (double)V[(size_t)(j - 1) * ld + r], y);
                  y = fma(-tjj, (double)V[(size_t)j * ld + r], y);
                  ycur[r] = (S)y;
                  nrm = fma(y, y, nrm);
                }
                double v[8] = {nrm, 0, 0, 0, 0, 0, 0, 0};
                block_sum8(s, v, 1, s.coef);
                PM_SUM_OR_FAIL(1);
                const double hn = sqrt(s.coef[0]);
                if (tid == 0) {
                  s.H[j * PM_MAXM + j] = tjj;
                  if (j + 1 < PM_MAXM + 1) s.H[(j + 1) * PM_MAXM + j] = hn;
                  if (j + 1 < PM_MAXM) s.H[j * PM_MAXM + j + 1] = hn;
                  if (j > 0) s.H[(j - 1) * PM_MAXM + j] = tjm;
                }
                __syncthreads();
                ynorm_last = hn;
              } else {
                // CGS2: y -= V h1 ; h2 = V^T y ; y -= V h2 ; h = h1 + h2
                for (int k = tid; k < nv; k += nth) { s.h1[k] = s.coef[k]; s.hf[k] = E::coef(s.coef[k]); }
                __syncthreads();
                for (int pass = 0; pass < 2; ++pass) {
                  double nrm;
                  if (sizeof(S) == 8) nrm = update_rows<S, double>(ycur, V, ld, nv, s.h1, lo, hi);
                  else nrm = update_rows<S, float>(ycur, V, ld, nv, s.hf, lo, hi);
                  __syncthreads();
                  if (pass == 0) {
                    dots_cta<S>(V, ld, 0, nv, ycur, lo, hi, s);
                    PM_SUM_OR_FAIL(nv);
                    for (int k = tid; k < nv; k += nth) {
                      const double h2 = s.coef[k];
                      s.H[k * PM_MAXM + j] = s.h1[k] + h2;
                      s.h1[k] = h2;
                      s.hf[k] = E::coef(h2);
                    }
                    __syncthreads();
                  } else {
                    double v[8] = {nrm, 0, 0, 0, 0, 0, 0, 0};
                    block_sum8(s, v, 1, s.coef);
                    PM_SUM_OR_FAIL(1);
                  }
                }
                const double hn = sqrt(s.coef[0]);
                if (tid == 0) s.H[(j + 1) * PM_MAXM + j] = hn;
                __syncthreads();
                ynorm_last = hn;
              }
              if (ynorm_last <= bd_abs) {      // happy breakdown (R12): invariant subspace
                if (tid == 0) s.H[(j + 1) * PM_MAXM + j] = 0.0;
                __syncthreads();
                ynorm_last = 0.0;
                invariant = true;
                kcur = j + 1;
                break;
              }
              kcur = j + 1;
            }
            // normalise the last vector: v_{kcur} = y / ||y||  (my rows)
            if (ynorm_last > 0.0) {
              const S* yl = Y + (size_t)((kcur - 1) & 1) * ld;
              const double inv = 1.0 / ynorm_last;
              for (int r = lo + tid; r < hi; r += nth) V[(size_t)kcur * ld + r] = E::cvt((double)yl[r] * inv);
            }
          }
          m_used = min(m, kcur);
          hlast = s.H[m_used * PM_MAXM + m_used - 1];
          if (invariant && m_used == kcur) hlast = 0.0;
          // ---------------- augmented matrix (Eq. hathm + R2) and its exponential (a5)
          const int N = m_used + p + 1;
          // ||H_hat||_1 = max(tau ||H_m||_1, 1): the augmented columns each hold a single 1
          if (tid < 32) {
            double mx = 0.0;
            for (int jj = tid; jj < m_used; jj += 32) {
              double cs = 0.0;
              for (int i = 0; i < m_used; ++i) cs += fabs(s.H[i * PM_MAXM + jj]);
              mx = fmax(mx, tau_used * cs);
            }
            mx = pm_warp_max(mx);
            if (tid == 0) s.mat_norm = fmax(mx, 1.0);
          }
          __syncthreads();
          norm1 = s.mat_norm;
          sq = pm_squarings(norm1, prm.theta13);
          const int ca = (p >= 1) ? m_used + p - 1 : 0;
          const int cb = m_used + p;
          if (Team::multi) {
            double* pg = w.phi_g + (size_t)(expms & 1) * 2 * PM_NA;
            if (team.rank() == 0) expm_cta(s, tau_used, m_used, p, N, sq, prm.pade_b, expm_ws, ca, cb, pg, pg + PM_NA);
            PM_SYNC_OR_FAIL();
            for (int i = tid; i < m_used; i += nth) { s.phi0[i] = __ldcg(&pg[i]); s.phi1[i] = __ldcg(&pg[PM_NA + i]); }
            __syncthreads();
          } else {
            expm_cta(s, tau_used, m_used, p, N, sq, prm.pade_b, expm_ws, ca, cb, s.phi0, s.phi1);
          }
          expms += 1;
          // ---------------- error estimate (a6), Eq. (errest) with R4
          eps = pow(tau_used, p + 1) * beta * fabs(hlast) * fabs(s.phi1[m_used - 1]);
        } else {
          m_used = m;
        }
        if (!isfinite(eps)) {
          nonfinite += 1;
          rejects += 1;
          if (nonfinite >= 10) { status = PM_ENONFINITE; goto done; }
          tau = tau / 5.0;
          ctl.rejected = ctl.tau_changed = ctl.m_changed = ctl.qf = ctl.kf = false;
          continue;
        }
        nonfinite = 0;
        m = m_used;
        // ---------------- controller (a7): Eq. (taunew), Algorithm 4, Eqs. (2)-(8)
        const double omega = t_end * eps / (tau_used * tol);
        double q;
        bool qf;
        if (ctl.rejected && ctl.tau_changed) {
          q = (eps > 0.0 && ctl.eps_old > 0.0 && tau_used != ctl.tau_old)
                  ? log(eps / ctl.eps_old) / log(tau_used / ctl.tau_old) - 1.0 : nan("");
          if (!isfinite(q)) { q = m / 4.0; qf = false; }
          else { q = fmin(fmax(q, 0.0), (double)m); qf = true; }
        } else if (ctl.rejected && ctl.qf) {
          q = ctl.q; qf = true;
        } else {
          q = m / 4.0; qf = false;
        }
        ctl.q = q; ctl.qf = qf;
        const double tau_new = (omega > 0.0) ? tau_used * pow(prm.gamma / omega, 1.0 / (q + 1.0)) : INFINITY;
        double kap;
        bool kf;
        if (ctl.rejected && ctl.m_changed) {
          kap = (eps > 0.0 && ctl.eps_old > 0.0 && m != ctl.m_old)
                    ? pow(eps / ctl.eps_old, 1.0 / (double)(ctl.m_old - m)) : nan("");
          if (!isfinite(kap) || kap <= 1.0) { kap = 2.0; kf = false; }
          else kf = true;
        } else if (ctl.rejected && ctl.kf) {
          kap = ctl.kap; kf = true;
        } else {
          kap = 2.0; kf = false;
        }
        ctl.kap = kap; ctl.kf = kf;
        const double m_new_real = (omega > 0.0) ? m + log(omega / prm.gamma) / log(kap) : -INFINITY;
        int m_new;
        if (isfinite(m_new_real)) {
          const double c = fmin(fmax(ceil(m_new_real), 1.0), (double)m_max);
          m_new = (int)c;
        } else {
          m_new = (m_new_real < 0.0) ? 1 : m_max;
        }
        const double Mf = 44.0 / 3.0 + 2.0 * pm_squarings(norm1, prm.theta13);
        const double t_left = t_end - t;
        auto C1 = [&](double mm) {
          if (symmetric) return (mm + p) * (double)nnzA + 3.0 * (mm + p) * n + Mf * (mm + p + 1) * (mm + p + 1) * (mm + p + 1);
          return (mm + p) * (double)nnzA + (mm * mm + 3 * p + 2) * (double)n + Mf * (mm + p + 1) * (mm + p + 1) * (mm + p + 1);
        };
        const double c_tau = ceil(t_left / tau_new) * C1((double)m);
        const double c_m = ceil(t_left / tau_used) * C1((double)m_new);
        bool branch_tau;
        if (c_tau < c_m) {
          tau = fmin(fmin(fmax(tau_new, tau_used / 5.0), 2.0 * tau_used), t_left);
          branch_tau = true;
        } else {
          int mm = max(max(m_new, (3 * m) / 4), 1);
          mm = min(min(mm, (4 * m + 2) / 3), m_max);
          m = mm;
          branch_tau = false;
        }
        if (omega <= prm.delta) {
          // ---------------- accept: Eq. (step) (a8), F by Eq. (phipapprox2)
          if (tid == 0) {
            const double tp = pow(tau_used, p);
            if (beta > 0.0) {
              for (int i = 0; i < m_used; ++i) s.ucoef[i] = tp * beta * s.phi0[i];
              s.ucoef[m_used] = (hlast != 0.0) ? tp * tau_used * beta * hlast * s.phi1[m_used - 1] : 0.0;
            }
            double d = 1.0;
            for (int jj = 0; jj < p; ++jj) {
              s.ucoef[PM_NSLOT + jj] = d;
              d = d * tau_used / (double)(jj + 1);
            }
          }
          __syncthreads();
          // FP32 basis: F carries a relative rounding error of about u32 and cancels against
          // sum_j tau^j/j! w_j in Eq. (step); the candidate goes to a spare vector so that
          // ||F|| / ||u_new|| can be bounded before it replaces u.
          const bool guard = (sizeof(S) == 4) && p >= 2 && beta > 0.0;
          double* udst = guard ? ualt : u;
          const int nvv = (beta > 0.0) ? ((s.ucoef[m_used] != 0.0) ? m_used + 1 : m_used) : 0;
          double un = 0.0;
          for (int r = lo + tid; r < hi; r += nth) {
            double acc = 0.0;
            for (int i = 0; i < nvv; ++i) acc = fma(s.ucoef[i], (double)V[(size_t)i * ld + r], acc);
            if (p >= 1) acc = fma(s.ucoef[PM_NSLOT], u[r], acc);
            for (int jj = 1; jj < p; ++jj) acc = fma(s.ucoef[PM_NSLOT + jj], W[(size_t)(jj - 1) * ld + r], acc);
            udst[r] = acc;
            un = fma(acc, acc, un);
          }
          if (guard) {
            double v[8] = {un, 0, 0, 0, 0, 0, 0, 0};
            block_sum8(s, v, 1, s.coef);
            PM_SUM_OR_FAIL(1);
            const double unew = sqrt(s.coef[0]);
            double fn = 0.0;
            for (int i = 0; i < m_used; ++i) fn = fma(s.phi0[i], s.phi0[i], fn);
            fn = pow(tau_used, p) * beta * sqrt(fn);
            if (fn > PM_F32_AMP * unew && unew > 0.0) {
              rejects += 1;
              if (rejects > prm.max_rejects) { status = PM_EMAXSTEPS; goto done; }
              tau = tau_used * pow(0.5 * PM_F32_AMP * unew / fn, 1.0 / (double)(p - 1));
              ctl.rejected = ctl.tau_changed = ctl.m_changed = ctl.qf = ctl.kf = false;
              continue;
            }
            double* t2 = u; u = ualt; ualt = t2;
          }
          accepted = true;
          steps += 1;
          err_sum += eps;
          if (steps > prm.max_steps) { status = PM_EMAXSTEPS; goto done; }
          const bool last = tau_used >= t_end - t;
          t = last ? t_end : t + tau_used;
          if (t < t_end) tau = fmin(tau, t_end - t);
          r_last_tau = tau_used;
          r_last_m = m_used;
          PM_SYNC_OR_FAIL();    // u complete before the next SpMV reads neighbours
        } else {
          rejects += 1;
          if (rejects > prm.max_rejects) { status = PM_EMAXSTEPS; goto done; }
          ctl.rejected = true;
          ctl.tau_changed = branch_tau;
          ctl.m_changed = !branch_tau;
          ctl.eps_old = eps;
          ctl.tau_old = tau_used;
          ctl.m_old = m_used;
        }
      }
    }
  }
  if (u != P.u) {
    for (int r = lo + tid; r < hi; r += nth) P.u[r] = u[r];
  }
done:
  if (team.rank() == 0 && threadIdx.x == 0) {
    res.status = status;
    res.steps = steps;
    res.rejects = rejects;
    res.matvecs = matvecs;
    res.expms = expms;
    res.kry_steps = kry_steps;
    res.gs_vectors = gs_vectors;
    res.err_est_sum = err_sum;
    res.normA = r_normA;
    res.normb = r_normb;
    res.symmetric = symmetric ? 1 : 0;
    res.last_tau = r_last_tau;
    res.last_m = r_last_m;
  }
#undef PM_SYNC_OR_FAIL
#undef PM_SUM_OR_FAIL
#undef PM_MAX_OR_FAIL
}
