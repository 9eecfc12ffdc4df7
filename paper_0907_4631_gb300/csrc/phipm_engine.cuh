// The phipm method on the device (Niesen & Wright, Sec. 3), written once over
// a "team" of CTAs that share one problem (GridTeam: every CTA of a cooperative
// launch; CtaTeam: one CTA) and over the element type S of the Krylov basis
// (phipm_elem.cuh).  Every CTA of a team runs the same scalar code (controller,
// cost model) on bit-identical inputs, so all CTAs take the same decisions
// without a broadcast.
#pragma once
#include <type_traits>
#include "phipm_common.cuh"
#include "phipm_mlp.cuh"

// FP32 basis mode: bound on ||F|| / ||u_new|| per step (F = tau^p phi_p(tau A) w_p)
#define PM_F32_AMP 32.0
// Selective second Gram-Schmidt pass (FP64 and float-pair bases): a candidate that
// keeps at least sqrt(PM_ETA2) = 1/4 of its norm through the first projection is
// orthogonal to the basis to a few units of rounding after that one projection (the
// Daniel-Gragg-Kaufman-Stewart bound: loss at most about eps / 0.25), so its second
// pass is skipped.  The FP32 basis always takes both passes.
#define PM_ETA2 0.0625
#define PM_DRED (PM_WARPS * (PM_NSLOT + 2))   // partials of a dot pass (vector x warp) or of a team fold
#define PM_ZW_BYTES 65536                      // shared staging of the two vectors every product of a dot pass reads

// Scalar state of one problem.  Thread 0 writes it, every thread reads it after
// the next barrier: on GB300 a scalar FP64 expression evaluated by all threads
// would cost a warp-wide FP64 instruction per warp on a pipe of about 2 FMA/clk/SM.
struct PmScal {
  double t, tau, tau_used, beta, eps, hlast, norm1, hn, inv, tol, t_end, normA, normb, bd_abs, err_sum;
  double fnorm, last_tau, omega, last_omega, m_new;
  double tp;                            // tau^p of the accepted attempt
  double fz, fw, fab, dcoef;            // lagged Gram-Schmidt: z.z, z.w, a.b, d
  double fww, fbb;                      // w.w and ||b||^2 (first-pass retention of the next candidate)
  int skipz;                            // the current candidate keeps its single projection
  double tl[PM_MAXP + 1];
  df32 inv2;
  float invf;
  int m, m_used, kcur, invariant, sq, nonfinite, nvv, measure, outcome, status, go, symmetric, lanczos, last_m;
  int m_req, attempt, source, step_rejects, prev_rejects;
  int xv_k, xv_s;                       // action form of this attempt's exponential (xv_s = 0: squaring form)
  long long steps, rejects, expms, trace_idx;
  float feat[MLP_IN];
};

// per-CTA shared state
struct PmShared {
  double H[(PM_MAXM + 1) * PM_MAXM];   // H[i * PM_MAXM + j], Hessenberg / tridiagonal
  double red[PM_WARPS][8];
  double coef[2 * PM_NSLOT + 4];       // reduced sums of the current phase
  double h1[PM_NSLOT];                 // Gram-Schmidt coefficients a (candidate's second pass)
  double hb[PM_NSLOT];                 // Gram-Schmidt coefficients b (new vector's first pass)
  double hdd[PM_NSLOT];                // coefficients of the current update (FP64 basis)
  float hf[PM_NSLOT];                  // ... as float (FP32 basis)
  df32 hd[PM_NSLOT];                   // ... as float pairs (float-pair basis)
  double hdd2[PM_NSLOT];               // second coefficient set of a fused two-output update
  float hf2[PM_NSLOT];
  df32 hd2[PM_NSLOT];
  double phi0[PM_NA], phi1[PM_NA];     // phi_p(tau H) e1 and phi_{p+1}(tau H) e1
  double ucoef[PM_NSLOT + PM_MAXP + 1];
  float ucf[PM_NSLOT];
  df32 ucd[PM_NSLOT];
  double dred[PM_DRED];                // per-segment partial dots of one pass
  double lu[PM_NA2];                   // LU factors of the Pade denominator (every CTA its own)
  double rdiag[PM_NA];                 // reciprocals of U's diagonal
  int piv[PM_NA];
  int perm[PM_NA];                     // the row interchanges of the LU as one permutation
  float mh[2][MLP_H];                  // learned controller: hidden activations (warp 0)
  PmScal sc;
  unsigned long long mbar;             // completion barrier of the stencil product's bulk copy
  alignas(16) unsigned char zw[PM_ZW_BYTES];   // this CTA's rows of z and A z during a dot pass;
                                               // the stencil product's staged rows during a product
};

struct PmWork {
  double* partials;     // [2][G][PM_PSTRIDE] (grid team)
  double* expm;         // team-shared exponential scratch: PM_EXPM_DOUBLES doubles
};

#define PM_PSTRIDE (2 * PM_NSLOT + 4)

// Sums of E::Red partials across a warp (float pairs for the FP32 and float-pair
// bases, FP64 otherwise), and their 8-byte slots in shared memory.
template <class E>
__device__ __forceinline__ typename E::Red red_warp_sum(typename E::Red v) {
  if constexpr (E::kind == 0) {
    return pm_warp_sum(v);
  } else {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      F2Acc t;
      t.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
      t.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
      v = f2_add(v, t);
    }
    return v;
  }
}
// The sum of PM_WARPS (16) partials p[q * stride], q < 16, by one warp: lanes 0..15 load
// one each and four shuffle levels add them (fixed order, so deterministic), against a
// chain of 16 dependent adds by one thread (each FP64 add about 65 cycles).  Every lane
// of the warp must call it; lane 0 holds the total.
template <class E>
__device__ __forceinline__ typename E::Red red_sum16(const double* p, int stride) {
  static_assert(PM_WARPS == 16, "one partial per lane of a half warp");
  const int lane = threadIdx.x & 31;
  typename E::Red v;
  if (lane < PM_WARPS) memcpy(&v, p + lane * stride, sizeof(v));
  else v = E::red_zero();
#pragma unroll
  for (int o = 8; o; o >>= 1) {
    typename E::Red t;
    if constexpr (E::kind == 0) {
      t = __shfl_xor_sync(0xffffffffu, v, o);
    } else {
      t.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
      t.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    }
    v = E::red_add(v, t);
  }
  return v;
}

template <class R>
__device__ __forceinline__ void red_put(double* p, const R& r) {
  static_assert(sizeof(R) == sizeof(double), "a partial fills one 8-byte slot");
  memcpy(p, &r, sizeof(R));
}
template <class R>
__device__ __forceinline__ R red_get(const double* p) {
  R r;
  memcpy(&r, p, sizeof(R));
  return r;
}


// ------------------------------------------------------------------------------------
// team reductions of K values held in s.coef[0..K) by each CTA
// ------------------------------------------------------------------------------------
// After the team barrier every CTA folds the G partial rows P[g][0..K) into
// s.coef[0..K).  The G x K loads are cut into units (k, block of CTAs) so that each
// thread has up to PM_RB independent L2 loads in flight (a lane-strided loop leaves
// one load per lane outstanding and pays the L2 latency G / 32 times per k); units
// are folded in a fixed order, so every CTA gets bit-identical results.  With PAIR
// the partials are float pairs (F2Acc in the 8-byte slots) folded by f2_add on the
// FP32 pipe (the FP32 and float-pair bases; every CTA folds all G x K partials).
#define PM_RB 16
template <bool PAIR>
__device__ __forceinline__ void team_fold_sum(PmShared& s, const double* P, int G, int K) {
  if (K <= 0) { __syncthreads(); return; }
  int nb = (G + PM_RB - 1) / PM_RB;
  nb = max(1, min(nb, PM_DRED / K));
  const int gpb = (G + nb - 1) / nb;          // CTAs per unit
  for (int u = threadIdx.x; u < K * nb; u += blockDim.x) {
    const int k = u / nb, b = u - k * nb;
    const int g0 = b * gpb, g1 = min(G, g0 + gpb);
    if constexpr (PAIR) {
      F2Acc a = f2_zero();
      for (int g = g0; g < g1; g += PM_RB) {
        float2 v[PM_RB];
#pragma unroll
        for (int q = 0; q < PM_RB; ++q)
          v[q] = (g + q < g1) ? __ldcg(reinterpret_cast<const float2*>(&P[(size_t)(g + q) * PM_PSTRIDE + k]))
                              : make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < PM_RB; ++q) {
          F2Acc t;
          t.hi = v[q].x;
          t.lo = v[q].y;
          a = f2_add(a, t);
        }
      }
      red_put(&s.dred[u], a);
    } else {
      double a = 0.0;
      for (int g = g0; g < g1; g += PM_RB) {
        double v[PM_RB];
#pragma unroll
        for (int q = 0; q < PM_RB; ++q) v[q] = (g + q < g1) ? __ldcg(&P[(size_t)(g + q) * PM_PSTRIDE + k]) : 0.0;
#pragma unroll
        for (int q = 0; q < PM_RB; ++q) a = a + v[q];
      }
      s.dred[u] = a;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    if constexpr (PAIR) {
      F2Acc a = red_get<F2Acc>(&s.dred[k * nb]);
      for (int b = 1; b < nb; ++b) a = f2_add(a, red_get<F2Acc>(&s.dred[k * nb + b]));
      s.coef[k] = f2_value(a);
    } else {
      double a = s.dred[k * nb];
      for (int b = 1; b < nb; ++b) a = a + s.dred[k * nb + b];
      s.coef[k] = a;
    }
  }
  __syncthreads();
}

// the same fold for maxima (FP64; rare: norms of A)
__device__ __forceinline__ void team_fold_max(PmShared& s, const double* P, int G, int K) {
  if (K <= 0) { __syncthreads(); return; }
  int nb = (G + PM_RB - 1) / PM_RB;
  nb = max(1, min(nb, PM_DRED / K));
  const int gpb = (G + nb - 1) / nb;
  for (int u = threadIdx.x; u < K * nb; u += blockDim.x) {
    const int k = u / nb, b = u - k * nb;
    const int g0 = b * gpb, g1 = min(G, g0 + gpb);
    double a = -INFINITY;
    for (int g = g0; g < g1; g += PM_RB) {
      double v[PM_RB];
#pragma unroll
      for (int q = 0; q < PM_RB; ++q) v[q] = (g + q < g1) ? __ldcg(&P[(size_t)(g + q) * PM_PSTRIDE + k]) : -INFINITY;
#pragma unroll
      for (int q = 0; q < PM_RB; ++q) a = fmax(a, v[q]);
    }
    s.dred[u] = a;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double a = s.dred[k * nb];
    for (int b = 1; b < nb; ++b) a = fmax(a, s.dred[k * nb + b]);
    s.coef[k] = a;
  }
  __syncthreads();
}

template <bool PAIR, class Team>
__device__ bool team_sum(const Team& team, PmShared& s, int K, const PmWork& w, int& parity) {
  if (!Team::multi) { __syncthreads(); return true; }
  const int G = team.size(), r = team.rank();
  double* P = w.partials + (size_t)parity * G * PM_PSTRIDE;
  parity ^= 1;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    if constexpr (PAIR) red_put(&P[(size_t)r * PM_PSTRIDE + k], f2_split(s.coef[k]));
    else P[(size_t)r * PM_PSTRIDE + k] = s.coef[k];
  }
  if (!team.sync()) return false;
  team_fold_sum<PAIR>(s, P, G, K);
  return true;
}

template <class Team>
__device__ bool team_max(const Team& team, PmShared& s, int K, const PmWork& w, int& parity) {
  if (!Team::multi) { __syncthreads(); return true; }
  const int G = team.size(), r = team.rank();
  double* P = w.partials + (size_t)parity * G * PM_PSTRIDE;
  parity ^= 1;
  for (int k = threadIdx.x; k < K; k += blockDim.x) P[(size_t)r * PM_PSTRIDE + k] = s.coef[k];
  if (!team.sync()) return false;
  team_fold_max(s, P, G, K);
  return true;
}

// block-wide sums of up to 8 per-thread values into out[0..cnt)
__device__ __forceinline__ void block_sum(PmShared& s, const double* v, int cnt, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k < cnt) {
      const double a = pm_warp_sum(v[k]);
      if (lane == 0) s.red[warp][k] = a;
    }
  }
  __syncthreads();
  for (int k = warp; k < cnt; k += PM_WARPS) {
    const double a = red_sum16<Elem<double>>(&s.red[0][k], 8);
    if (lane == 0) out[k] = a;
  }
  __syncthreads();
}

__device__ __forceinline__ void split_range(int total, int rank, int G, int& lo, int& hi) {
  const int chunk = (total + G - 1) / G;
  lo = min(total, rank * chunk);
  hi = min(total, lo + chunk);
}

// ------------------------------------------------------------------------------------
// SpMV: y_r = (A x)_r, x given by a loader (element index -> S)
// ------------------------------------------------------------------------------------
// Loads of data that other CTAs of the team wrote during this launch go through
// L2 (ld.global.cg): the L1 of an SM is not coherent with other SMs' stores, and
// a line cached before a team barrier could otherwise be read stale after it.
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ df32 ld_cg(const df32* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  df32 r;
  r.hi = v.x;
  r.lo = v.y;
  return r;
}
// x(i) for the SpMV.  With CG (grid team) rows outside this CTA's [lo, hi), written
// by other CTAs during the launch, are read through L2; the CTA's own rows, written
// only by itself (row blocks are 64-aligned, so no cache line is shared between
// CTAs), use the L1-cached path, where stencil neighbours reuse each other's lines.
template <class S, bool CG> struct VecLoad {
  const S* p;
  int lo, hi;
  __device__ __forceinline__ S operator()(int i) const {
    if constexpr (CG) {
      if ((unsigned)(i - lo) >= (unsigned)(hi - lo)) return ld_cg(p + i);
    }
    return p[i];
  }
};
template <class S, bool CG> struct DLoadAs {      // FP64 vector read as S
  const double* p;
  int lo, hi;
  __device__ __forceinline__ S operator()(int i) const {
    if constexpr (CG) {
      if ((unsigned)(i - lo) >= (unsigned)(hi - lo)) return Elem<S>::from_d(__ldcg(p + i));
    }
    return Elem<S>::from_d(p[i]);
  }
};

// Row r of a built-in matrix-free operator (kind 2) applied to x (an index -> double
// loader), in FP64; with asum, also the row's sum of absolute entries (for ||A||_inf).
// PHIPM_FN_VARCOEF_CONVDIFF (include/phipm.h): for each dimension d, the diffusion
// fluxes through the two faces with face diffusivities (kappa_i + kappa_nb) / 2
// (kappa_i at the boundary, where x is 0) and the central-difference convection term.
template <class XF>
__device__ __forceinline__ double fn_row(const DevOp& A, int r, const XF& x, double* asum) {
  const int nx = A.nx, ny = A.ny;
  const unsigned line = pm_udiv((unsigned)r, A.mnx);
  const int c[3] = {r - (int)line * nx, (A.ndim > 1) ? (int)line - (int)pm_udiv(line, A.mny) * ny : 0,
                    (A.ndim > 2) ? (int)pm_udiv(line, A.mny) : 0};
  const int ext[3] = {nx, ny, A.nz};
  const int stride[3] = {1, nx, nx * ny};
  const double* kap = A.fld[0];
  const double k0 = kap[r], xr = x(r);
  double acc = 0.0, as = 0.0;
  for (int d = 0; d < A.ndim; ++d) {
    const bool hm = c[d] > 0, hp = c[d] < ext[d] - 1;
    const double xm = hm ? x(r - stride[d]) : 0.0, xp = hp ? x(r + stride[d]) : 0.0;
    const double km = hm ? 0.5 * (k0 + kap[r - stride[d]]) : k0;
    const double kp = hp ? 0.5 * (k0 + kap[r + stride[d]]) : k0;
    const double sd = A.fsc[d], cd = A.fsc[3 + d];
    const double v = A.fld[1 + d] ? A.fld[1 + d][r] : 0.0;
    acc += sd * (kp * (xp - xr) - km * (xr - xm)) - cd * v * (xp - xm);
    if (asum) {
      as += sd * (kp + km);
      if (hp) as += fabs(sd * kp - cd * v);
      if (hm) as += fabs(sd * km + cd * v);
    }
  }
  if (asum) *asum = as;
  return acc;
}

template <class S, class XL>
__device__ __forceinline__ S spmv_row(const DevOp& A, int r, const XL& x) {
  if (A.kind == 2) return Elem<S>::from_d(fn_row(A, r, [&](int i) { return Elem<S>::to_d(x(i)); }, nullptr));
  if constexpr (Elem<S>::kind == 0) {
    double acc = 0.0;
    if (A.kind == 0) {
      const int k0 = __ldg(&A.rowptr[r]), k1 = __ldg(&A.rowptr[r + 1]);
      for (int k = k0; k < k1; ++k) acc = fma(__ldg(&A.val[k]), x(__ldg(&A.colind[k])), acc);
      return acc;
    }
    const int nx = A.nx, ny = A.ny, ix = r % nx, iy = (r / nx) % ny, iz = r / (nx * ny);
    acc = A.cc * x(r);
    if (ix > 0) acc = fma(A.cm[0], x(r - 1), acc);
    if (ix < nx - 1) acc = fma(A.cp[0], x(r + 1), acc);
    if (A.ndim > 1) {
      if (iy > 0) acc = fma(A.cm[1], x(r - nx), acc);
      if (iy < ny - 1) acc = fma(A.cp[1], x(r + nx), acc);
    }
    if (A.ndim > 2) {
      const int pl = nx * ny;
      if (iz > 0) acc = fma(A.cm[2], x(r - pl), acc);
      if (iz < A.nz - 1) acc = fma(A.cp[2], x(r + pl), acc);
    }
    return acc;
  } else if constexpr (Elem<S>::kind == 1) {
    float acc = 0.f;
    if (A.kind == 0) {
      const int k0 = __ldg(&A.rowptr[r]), k1 = __ldg(&A.rowptr[r + 1]);
      for (int k = k0; k < k1; ++k) acc = fmaf(__ldg(&A.valf[k]), x(__ldg(&A.colind[k])), acc);
      return acc;
    }
    const int nx = A.nx, ny = A.ny, ix = r % nx, iy = (r / nx) % ny, iz = r / (nx * ny);
    acc = A.cc2.hi * x(r);
    if (ix > 0) acc = fmaf(A.cm2[0].hi, x(r - 1), acc);
    if (ix < nx - 1) acc = fmaf(A.cp2[0].hi, x(r + 1), acc);
    if (A.ndim > 1) {
      if (iy > 0) acc = fmaf(A.cm2[1].hi, x(r - nx), acc);
      if (iy < ny - 1) acc = fmaf(A.cp2[1].hi, x(r + nx), acc);
    }
    if (A.ndim > 2) {
      const int pl = nx * ny;
      if (iz > 0) acc = fmaf(A.cm2[2].hi, x(r - pl), acc);
      if (iz < A.nz - 1) acc = fmaf(A.cp2[2].hi, x(r + pl), acc);
    }
    return acc;
  } else {
    F2Acc acc = f2_zero();
    if (A.kind == 0) {
      const int k0 = __ldg(&A.rowptr[r]), k1 = __ldg(&A.rowptr[r + 1]);
      for (int k = k0; k < k1; ++k) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(&A.val2[k]));
        df32 av;
        av.hi = a.x;
        av.lo = a.y;
        f2_add_prod(acc, av, x(__ldg(&A.colind[k])));
      }
      return f2_round(acc);
    }
    const int nx = A.nx, ny = A.ny, ix = r % nx, iy = (r / nx) % ny, iz = r / (nx * ny);
    f2_add_prod(acc, A.cc2, x(r));
    if (ix > 0) f2_add_prod(acc, A.cm2[0], x(r - 1));
    if (ix < nx - 1) f2_add_prod(acc, A.cp2[0], x(r + 1));
    if (A.ndim > 1) {
      if (iy > 0) f2_add_prod(acc, A.cm2[1], x(r - nx));
      if (iy < ny - 1) f2_add_prod(acc, A.cp2[1], x(r + nx));
    }
    if (A.ndim > 2) {
      const int pl = nx * ny;
      if (iz > 0) f2_add_prod(acc, A.cm2[2], x(r - pl));
      if (iz < A.nz - 1) f2_add_prod(acc, A.cp2[2], x(r + pl));
    }
    return f2_round(acc);
  }
}

// Two CSR rows r and r2 (r2 < 0: none) at once: both rows' extents, then up to
// PM_CSR_U column indices and values of each, then the matching x entries, so that the
// three dependent loads of a row (extent, index, x) overlap with the other row's and
// every load of one level is in flight together.  Short rows (the 5-point operators)
// take one round.  Arithmetic as in spmv_row.
#define PM_CSR_U 6
template <class S, class XL>
__device__ __forceinline__ void spmv_csr_pair(const DevOp& A, int r, int r2, const XL& x, S& y0, S& y1) {
  typedef Elem<S> E;
  constexpr int kind = E::kind;
  typedef typename std::conditional<kind == 0, double, typename std::conditional<kind == 1, float, F2Acc>::type>::type
      Acc;
  typedef typename std::conditional<kind == 0, double, typename std::conditional<kind == 1, float, df32>::type>::type
      Val;
  Acc c0, c1;
  if constexpr (kind == 2) { c0 = f2_zero(); c1 = f2_zero(); }
  else { c0 = 0; c1 = 0; }
  const int a0 = __ldg(&A.rowptr[r]), b0 = __ldg(&A.rowptr[r + 1]);
  int a1 = 0, b1 = 0;
  if (r2 >= 0) {
    a1 = __ldg(&A.rowptr[r2]);
    b1 = __ldg(&A.rowptr[r2 + 1]);
  }
  const int len = max(b0 - a0, b1 - a1);
  for (int t = 0; t < len; t += PM_CSR_U) {
    int col0[PM_CSR_U], col1[PM_CSR_U];
    Val v0[PM_CSR_U], v1[PM_CSR_U];
#pragma unroll
    for (int u = 0; u < PM_CSR_U; ++u) {
      const int k0 = a0 + t + u, k1 = a1 + t + u;
      col0[u] = (k0 < b0) ? __ldg(&A.colind[k0]) : -1;
      col1[u] = (k1 < b1) ? __ldg(&A.colind[k1]) : -1;
      if constexpr (kind == 0) {
        v0[u] = (k0 < b0) ? __ldg(&A.val[k0]) : 0.0;
        v1[u] = (k1 < b1) ? __ldg(&A.val[k1]) : 0.0;
      } else if constexpr (kind == 1) {
        v0[u] = (k0 < b0) ? __ldg(&A.valf[k0]) : 0.f;
        v1[u] = (k1 < b1) ? __ldg(&A.valf[k1]) : 0.f;
      } else {
        const float2 q0 = (k0 < b0) ? __ldg(reinterpret_cast<const float2*>(&A.val2[k0])) : make_float2(0.f, 0.f);
        const float2 q1 = (k1 < b1) ? __ldg(reinterpret_cast<const float2*>(&A.val2[k1])) : make_float2(0.f, 0.f);
        v0[u].hi = q0.x; v0[u].lo = q0.y;
        v1[u].hi = q1.x; v1[u].lo = q1.y;
      }
    }
    S x0[PM_CSR_U], x1[PM_CSR_U];
#pragma unroll
    for (int u = 0; u < PM_CSR_U; ++u) {
      x0[u] = (col0[u] >= 0) ? x(col0[u]) : E::from_d(0.0);
      x1[u] = (col1[u] >= 0) ? x(col1[u]) : E::from_d(0.0);
    }
#pragma unroll
    for (int u = 0; u < PM_CSR_U; ++u) {
      if (col0[u] >= 0) {
        if constexpr (kind == 0) c0 = fma(v0[u], x0[u], c0);
        else if constexpr (kind == 1) c0 = fmaf(v0[u], x0[u], c0);
        else f2_add_prod(c0, v0[u], x0[u]);
      }
      if (col1[u] >= 0) {
        if constexpr (kind == 0) c1 = fma(v1[u], x1[u], c1);
        else if constexpr (kind == 1) c1 = fmaf(v1[u], x1[u], c1);
        else f2_add_prod(c1, v1[u], x1[u]);
      }
    }
  }
  if constexpr (kind == 2) {
    y0 = f2_round(c0);
    y1 = f2_round(c1);
  } else {
    y0 = c0;
    y1 = c1;
  }
}

// ------------------------------------------------------------------------------------
// staging of a stencil product's rows through the TMA bulk-copy engine
// ------------------------------------------------------------------------------------
struct Stage {
  unsigned char* buf;            // shared memory, 16-byte aligned, PM_ZW_BYTES
  unsigned long long* mbar;      // the CTA's mbarrier (initialised by phipm_device)
  unsigned* phase;               // how many phases of it this thread has waited for
  long long timeout;             // bound of the wait, clock64 cycles
};

__device__ __forceinline__ unsigned pm_smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void pm_mbar_init(unsigned long long* mbar) {   // thread 0; a __syncthreads follows
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n\tfence.mbarrier_init.release.cluster;"
               :: "r"(pm_smem_addr(mbar)) : "memory");
}

// x[a, b) into stg.buf by one bulk asynchronous copy (cp.async.bulk) that completes on
// the mbarrier; every thread waits for that phase, bounded by stg.timeout.  Returns the
// same answer in every thread of the CTA: false if some thread's wait gave up.  The
// addresses and the size must be multiples of 16 bytes (the caller checks).  x was written
// by generic stores of this launch (this CTA's and, before a team barrier, other CTAs'):
// every thread orders its generic accesses of global and shared memory before the
// copy's async-proxy accesses with proxy fences, ahead of the barrier that precedes the
// copy's issue.
template <class S>
__device__ bool stage_rows(const Stage& stg, const S* x, int a, int b) {
  const unsigned bytes = (unsigned)(b - a) * (unsigned)sizeof(S);
  const unsigned mb = pm_smem_addr(stg.mbar);
  asm volatile("fence.proxy.async.global;\n\tfence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();                                    // earlier readers of the buffer are done
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mb), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(pm_smem_addr(stg.buf)), "l"(x + a), "r"(bytes), "r"(mb) : "memory");
  }
  const unsigned par = *stg.phase & 1u;
  *stg.phase += 1;
  bool ok = false;
  const long long t0 = clock64();
  for (;;) {
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(mb), "r"(par) : "memory");
    if (done) { ok = true; break; }
    if (clock64() - t0 > stg.timeout) break;
  }
  return __syncthreads_and(ok ? 1 : 0) != 0;
}

// One stencil row from its centre value and six neighbours (zero where the
// neighbour is outside the grid, which adds nothing), in spmv_row's order.
template <class S>
__device__ __forceinline__ S stencil_point(const DevOp& A, S xc, S xl, S xr, S ym, S yp, S zm, S zp) {
  if constexpr (Elem<S>::kind == 0) {
    double acc = A.cc * xc;
    acc = fma(A.cm[0], xl, acc);
    acc = fma(A.cp[0], xr, acc);
    if (A.ndim > 1) { acc = fma(A.cm[1], ym, acc); acc = fma(A.cp[1], yp, acc); }
    if (A.ndim > 2) { acc = fma(A.cm[2], zm, acc); acc = fma(A.cp[2], zp, acc); }
    return acc;
  } else if constexpr (Elem<S>::kind == 1) {
    float acc = A.cc2.hi * xc;
    acc = fmaf(A.cm2[0].hi, xl, acc);
    acc = fmaf(A.cp2[0].hi, xr, acc);
    if (A.ndim > 1) { acc = fmaf(A.cm2[1].hi, ym, acc); acc = fmaf(A.cp2[1].hi, yp, acc); }
    if (A.ndim > 2) { acc = fmaf(A.cm2[2].hi, zm, acc); acc = fmaf(A.cp2[2].hi, zp, acc); }
    return acc;
  } else {
    F2Acc acc = f2_zero();
    f2_add_prod(acc, A.cc2, xc);
    f2_add_prod(acc, A.cm2[0], xl);
    f2_add_prod(acc, A.cp2[0], xr);
    if (A.ndim > 1) { f2_add_prod(acc, A.cm2[1], ym); f2_add_prod(acc, A.cp2[1], yp); }
    if (A.ndim > 2) { f2_add_prod(acc, A.cm2[2], zm); f2_add_prod(acc, A.cp2[2], zp); }
    return f2_round(acc);
  }
}

// Stencil product over this CTA's rows [lo, hi) taken as 16-byte quads of four
// consecutive rows (nx a multiple of 4, so a quad never crosses a grid line; lo and
// hi are multiples of 4 except hi = n, whose ragged rows take the per-row path).  Per
// quad: the quad itself, its two x-neighbours and the quads of the y- and z-neighbour
// lines, seven loads for four rows instead of twenty-eight, all issued before the
// arithmetic, two quads per thread per pass for FP32 (one for the 8-byte types, whose
// quads need twice the registers).  Row coordinates come from multiply-high
// divisions (pm_udiv).  With CG, quads outside [lo, hi) (written by other CTAs of the
// team) are read through L2; every quad lies wholly inside or outside, since lo, hi,
// nx and nx ny are multiples of 4.
template <class S, bool CG, bool STAGED, class Epi>
__device__ __forceinline__ bool stencil_rows4_body(const DevOp& A, const S* __restrict__ x, int lo, int hi,
                                                   const Epi& epi, const Stage* stg) {
  typedef Elem<S> E;
  const int nx = A.nx, ny = A.ny, nz = A.nz, pl = nx * ny;
  const int nq = (hi - lo) >> 2;
  const S zero = E::zero_elem();
  // With a stage, the rows [sa, sb) = this CTA's rows and the grid lines next to them in
  // y are copied into shared memory by the TMA engine when they fit; the x- and
  // y-neighbours then come from shared memory and only the z-neighbour quads from L2.
  // sa and sb are multiples of 4 rows (lo of 64, nx and n of 4), so the copy starts and
  // ends on 16-byte boundaries.
  int sa = 0, sb = 0;
  const S* sx = nullptr;
  if (STAGED && hi > lo) {
    sa = max(0, lo - nx);
    sb = min(A.n, hi + nx);
    if ((long long)(sb - sa) * (long long)sizeof(S) <= (long long)PM_ZW_BYTES) {
      if (!stage_rows<S>(*stg, x, sa, sb)) return false;
      sx = reinterpret_cast<const S*>(stg->buf) - sa;   // indexed by absolute row
    } else {
      sa = sb = 0;
    }
  }
  auto staged = [&](int r) { return STAGED && (unsigned)(r - sa) < (unsigned)(sb - sa); };
  auto outside = [&](int r) { return CG && (unsigned)(r - lo) >= (unsigned)(hi - lo); };
  auto ldq = [&](Quad<S>& q, int r, bool ok) {
    if (!ok) {
#pragma unroll
      for (int k = 0; k < 4; ++k) q.x[k] = zero;
    } else if (staged(r)) {
      q.load(sx + r);
    } else if (outside(r)) {
      q.load_cg(x + r);
    } else {
      q.load(x + r);
    }
  };
  auto lds = [&](int r, bool ok) -> S { return !ok ? zero : staged(r) ? sx[r] : outside(r) ? ld_cg(x + r) : x[r]; };
  constexpr int U = sizeof(S) == 4 ? 2 : 1;
  for (int q0 = threadIdx.x; q0 < nq; q0 += U * blockDim.x) {
    Quad<S> c[U], ym[U], yp[U], zm[U], zp[U];
    S xl[U], xr[U];
    int rr[U];
    bool act[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int qi = q0 + u * blockDim.x;
      act[u] = qi < nq;
      const int r = lo + 4 * (act[u] ? qi : q0);
      rr[u] = r;
      const unsigned line = pm_udiv((unsigned)r, A.mnx);
      const int ix = r - (int)line * nx;
      int iy = 0, iz = 0;
      if (A.ndim > 1) {
        iz = (int)pm_udiv(line, A.mny);
        iy = (int)line - iz * ny;
      }
      ldq(c[u], r, true);
      xl[u] = lds(r - 1, ix > 0);
      xr[u] = lds(r + 4, ix + 4 < nx);
      ldq(ym[u], r - nx, A.ndim > 1 && iy > 0);
      ldq(yp[u], r + nx, A.ndim > 1 && iy < ny - 1);
      ldq(zm[u], r - pl, A.ndim > 2 && iz > 0);
      ldq(zp[u], r + pl, A.ndim > 2 && iz < nz - 1);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!act[u]) continue;
      Quad<S> y;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const S l = (k == 0) ? xl[u] : c[u].x[k - 1];
        const S rgt = (k == 3) ? xr[u] : c[u].x[k + 1];
        y.x[k] = stencil_point<S>(A, c[u].x[k], l, rgt, ym[u].x[k], yp[u].x[k], zm[u].x[k], zp[u].x[k]);
      }
      epi.quad(rr[u], y);
    }
  }
  VecLoad<S, CG> xl{x, lo, hi};
  for (int r = lo + 4 * nq + threadIdx.x; r < hi; r += blockDim.x) epi.row(r, spmv_row<S>(A, r, xl));
  return true;
}

// the staged and the plain form are separate instances, so that the plain loop carries
// no staging tests
template <class S, bool CG, class Epi>
__device__ __forceinline__ bool stencil_rows4_epi(const DevOp& A, const S* __restrict__ x, int lo, int hi,
                                                  const Epi& epi, const Stage* stg = nullptr) {
  if (stg != nullptr) return stencil_rows4_body<S, CG, true>(A, x, lo, hi, epi, stg);
  return stencil_rows4_body<S, CG, false>(A, x, lo, hi, epi, nullptr);
}

// epilogue of a plain product: out = (A x) * sc (scale) or A x
template <class S>
struct StoreScaled {
  S* out;
  typename Elem<S>::Coef sc;
  bool scale;
  __device__ __forceinline__ void quad(int r, Quad<S>& y) const {
    if (scale) {
#pragma unroll
      for (int k = 0; k < 4; ++k) y.x[k] = Elem<S>::scale(y.x[k], sc);
    }
    y.store(out + r);
  }
  __device__ __forceinline__ void row(int r, S v) const { out[r] = scale ? Elem<S>::scale(v, sc) : v; }
};

template <class S, bool CG>
__device__ __forceinline__ bool stencil_rows4(const DevOp& A, const S* __restrict__ x, S* __restrict__ out,
                                              typename Elem<S>::Coef sc, bool scale, int lo, int hi,
                                              const Stage* stg) {
  return stencil_rows4_epi<S, CG>(A, x, lo, hi, StoreScaled<S>{out, sc, scale}, stg);
}

template <class XL> struct IsVecLoad { static constexpr bool value = false; };
template <class S, bool CG> struct IsVecLoad<VecLoad<S, CG>> {
  static constexpr bool value = true;
  static constexpr bool cg = CG;
};

// out[r] = (A x)[r] * sc over this CTA's rows (CSR rows two at a time per thread,
// stencil rows two at a time too: their neighbour loads are independent, so a pass has
// both rows' loads in flight instead of paying the load latency once per row)
template <class S, class XL>
__device__ __forceinline__ bool spmv_rows(const DevOp& A, const XL& x, S* __restrict__ out,
                                          typename Elem<S>::Coef sc, bool scale, int lo, int hi,
                                          const Stage* stg = nullptr) {
  typedef Elem<S> E;
  const int nth = blockDim.x;
  if (A.kind == 0) {
    for (int r = lo + threadIdx.x; r < hi; r += 2 * nth) {
      const int r2 = (r + nth < hi) ? r + nth : -1;
      S y0, y1;
      spmv_csr_pair<S>(A, r, r2, x, y0, y1);
      out[r] = scale ? E::scale(y0, sc) : y0;
      if (r2 >= 0) out[r2] = scale ? E::scale(y1, sc) : y1;
    }
  } else {
    if constexpr (IsVecLoad<XL>::value) {
      if (A.kind == 1 && A.quad) return stencil_rows4<S, IsVecLoad<XL>::cg>(A, x.p, out, sc, scale, lo, hi, stg);
    }
    for (int r = lo + threadIdx.x; r < hi; r += 2 * nth) {
      const int r2 = r + nth;
      const S y0 = spmv_row<S>(A, r, x);
      const S y1 = (r2 < hi) ? spmv_row<S>(A, r2, x) : y0;
      out[r] = scale ? E::scale(y0, sc) : y0;
      if (r2 < hi) out[r2] = scale ? E::scale(y1, sc) : y1;
    }
  }
  return true;
}

// epilogue of a w-recurrence product, Eq. (wrecurrence): w_j = A w_{j-1} +
// sum_{l <= p-j} t^l / l! b_{j+l}, and the FP64 sum of squares of w_p
struct WEpi {
  double* out;
  const double* const* b;    // b_j, b_{j+1}, ...
  const double* tl;          // t^l / l!
  int nl;                    // l = 0 .. nl
  bool norm;
  mutable double nrm;        // this thread's sum of squares
  __device__ __forceinline__ double fin(int r, double y) const {
    for (int l = 0; l <= nl; ++l) y = fma(tl[l], b[l][r], y);
    if (norm) nrm = fma(y, y, nrm);
    return y;
  }
  __device__ __forceinline__ void quad(int r, Quad<double>& y) const {
#pragma unroll
    for (int k = 0; k < 4; ++k) y.x[k] = fin(r + k, y.x[k]);
    y.store(out + r);
  }
  __device__ __forceinline__ void row(int r, double v) const { out[r] = fin(r, v); }
};

// ------------------------------------------------------------------------------------
// Gram-Schmidt passes over this CTA's rows [lo, hi)
// ------------------------------------------------------------------------------------
// Row-owner form of dots_cta for one or two products (Lanczos): each thread owns
// four consecutive rows per tile of 4 x blockDim rows (16-byte accesses; lo is a
// multiple of 64 and vectors are 256-byte aligned), loads its quad of y once per
// tile together with the (at most two) vectors' quads; each warp reduces its
// partial per vector and accumulates it over the tiles in s.dred[i][warp]; d_i
// then sums the warps in order (deterministic).  With more vectors the per-vector
// warp reductions serialise the loads, and the run-per-warp form below is faster.
template <class S>
__device__ void dots_rows(const S* __restrict__ V, long long ld, int nv, const S* __restrict__ y, int lo, int hi,
                         bool with_norm, PmShared& s) {
  typedef Elem<S> E;
  typedef typename E::Acc Acc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nvec = nv + (with_norm ? 1 : 0);
  if (hi <= lo) {
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) s.coef[i] = 0.0;
    __syncthreads();
    return;
  }
  double* red = s.dred;                      // [nvec][PM_WARPS]
  const int span = 4 * blockDim.x;
  for (int base = lo; base < hi; base += span) {
    const int r = base + 4 * threadIdx.x;
    const int nr = max(0, min(4, hi - r));   // rows of this thread in the tile
    if (base + 128 * warp >= hi) {           // no rows for this warp: its partials are zero
      if (base == lo && lane == 0)           // (skips the FP64 warp sums of small problems)
        for (int i = 0; i < nvec; ++i) red_put(&red[i * PM_WARPS + warp], E::red_zero());
      continue;
    }
    Quad<S> yq;
    if (nr == 4) {
      yq.load(y + r);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) yq.x[k] = (k < nr) ? y[r + k] : E::from_d(0.0);
    }
    constexpr int NG = 2;                      // vectors per group
    for (int i0 = 0; i0 < nvec; i0 += NG) {
      typename E::Red d[NG];
      Quad<S> vq[NG];
#pragma unroll
      for (int u = 0; u < NG; ++u) {
        const int i = i0 + u;
        if (i < nvec) {
          const S* v = (i < nv) ? V + (size_t)i * ld : y;
          if (nr == 4) {
            vq[u].load(v + r);
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) vq[u].x[k] = (k < nr) ? v[r + k] : E::from_d(0.0);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < NG; ++u) {
        if (i0 + u < nvec) {
          Acc acc = E::zero();
          E::dot4(acc, vq[u].x, yq.x);
          d[u] = red_warp_sum<E>(E::red_of(acc, E::zero()));
        }
      }
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < NG; ++u) {
          const int i = i0 + u;
          if (i < nvec) {
            double* slot = &red[i * PM_WARPS + warp];
            red_put(slot, E::red_add(base == lo ? E::red_zero() : red_get<typename E::Red>(slot), d[u]));
          }
        }
      }
    }
  }
  __syncthreads();
  for (int i = warp; i < nvec; i += PM_WARPS) {
    const typename E::Red t = red_sum16<E>(&red[i * PM_WARPS], 1);
    if (lane == 0) s.coef[i] = E::red_val(t);
  }
  __syncthreads();
}

// d_i = sum_r V[i][r] y[r], i < nv, into s.coef[0..nv); with_norm adds sum y^2
// as s.coef[nv].  The nvec x rows products, taken vector after vector, are cut
// into PM_WARPS equal contiguous runs, one per warp, so every warp streams a long
// run (four 16-byte loads of V and of y per lane in flight) whatever nvec is.  A
// run crosses at most a few vector boundaries; each piece (segment) leaves one
// warp-reduced partial in s.dred, and d_i sums the partials of its segments in
// warp order (deterministic).  Rows of vectors are 256-byte aligned from lo, a
// multiple of 64, so quads start on row offsets that are multiples of 4.
#define PM_DSEG (PM_DRED / PM_WARPS)   // segments per warp
template <class S>
__device__ __forceinline__ typename Elem<S>::Red dot_segment(const S* __restrict__ v, const S* __restrict__ y, int a,
                                                            int b) {
  typedef Elem<S> E;
  typedef typename E::Acc Acc;
  const int lane = threadIdx.x & 31;
  Acc acc0 = E::zero(), acc1 = E::zero();
  const int qa = min(b, (a + 3) & ~3);      // quads cover [qa, qb)
  const int qb = max(qa, b & ~3);
  if (a + lane < qa) E::dot(acc1, v[a + lane], y[a + lane]);        // head: at most 3 rows
  int e = qa + 4 * lane;
  for (; e + 384 + 3 < qb; e += 512) {
    Quad<S> v0, y0, v1, y1, v2, y2, v3, y3;
    v0.load(v + e); y0.load(y + e);
    v1.load(v + e + 128); y1.load(y + e + 128);
    v2.load(v + e + 256); y2.load(y + e + 256);
    v3.load(v + e + 384); y3.load(y + e + 384);
    if constexpr (E::kind == 1) {
      E::dot4(acc0, v0.x, y0.x);
      E::dot4(acc1, v1.x, y1.x);
      E::dot4(acc0, v2.x, y2.x);
      E::dot4(acc1, v3.x, y3.x);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        E::dot(acc0, v0.x[k], y0.x[k]);
        E::dot(acc1, v1.x[k], y1.x[k]);
        E::dot(acc0, v2.x[k], y2.x[k]);
        E::dot(acc1, v3.x[k], y3.x[k]);
      }
    }
  }
  for (; e + 3 < qb; e += 128) {
    Quad<S> v0, y0;
    v0.load(v + e); y0.load(y + e);
    E::dot4(acc0, v0.x, y0.x);
  }
  if (qb + lane < b) E::dot(acc0, v[qb + lane], y[qb + lane]);      // tail: at most 3 rows
  return E::red_of(acc0, acc1);
}

// The run-per-warp pass of dots_cta (more than two products); the CTA's rows of y are
// staged in shared memory when they fit (every product reads them).
template <class S>
__device__ __forceinline__ void dots_part(const S* __restrict__ V, long long ld, int nv, const S* __restrict__ y,
                                          int lo, int hi, bool with_norm, PmShared& s) {
  typedef Elem<S> E;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long rows = hi - lo;
  const int nvec = nv + (with_norm ? 1 : 0);
  const long long total = (long long)nvec * rows;
  if (total == 0) {
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) s.coef[i] = 0.0;
    __syncthreads();
    return;
  }
  if (rows * (long long)sizeof(S) <= (long long)PM_ZW_BYTES) {
    constexpr int VEC = 16 / sizeof(S);
    S* sy = reinterpret_cast<S*>(s.zw);
    const int nq = (int)(rows / VEC);
    for (int q = threadIdx.x; q < nq; q += blockDim.x)
      reinterpret_cast<float4*>(sy)[q] = *reinterpret_cast<const float4*>(y + lo + q * VEC);
    for (int r = nq * VEC + threadIdx.x; r < rows; r += blockDim.x) sy[r] = y[lo + r];
    __syncthreads();
    y = sy - lo;                                  // indexed by absolute row, like V
  }
  // run length, a multiple of 4 rows.  A run meets at most run / rows + 2 vectors,
  // and run <= nvec rows / 16 + 4 rows with nvec <= 65 keeps that below 12 <= PM_DSEG.
  const long long run = (((total + PM_WARPS - 1) / PM_WARPS) + 3) & ~3ll;
  long long f = (long long)warp * run;
  const long long fend = min(total, f + run);
  if (f < fend) {
    int i = (int)(f / rows);                 // first vector of this run
    long long r0 = f - (long long)i * rows;
    for (int seg = 0; f < fend; ++seg, ++i, r0 = 0) {
      const long long r1 = min(rows, r0 + (fend - f));
      const S* v = (i < nv) ? V + (size_t)i * ld : y;
      const typename E::Red d = red_warp_sum<E>(dot_segment<S>(v, y, lo + (int)r0, lo + (int)r1));
      if (lane == 0) red_put(&s.dred[warp * PM_DSEG + seg], d);
      f += r1 - r0;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    const long long fa = (long long)i * rows, fb = fa + rows - 1;
    typename E::Red t = E::red_zero();
    for (long long w = fa / run; w <= fb / run && w < PM_WARPS; ++w)
      t = E::red_add(t, red_get<typename E::Red>(&s.dred[w * PM_DSEG + (int)(i - (w * run) / rows)]));
    s.coef[i] = E::red_val(t);
  }
  __syncthreads();
}

// Out of line, so that it does not add to the register pressure of the Arnoldi loop
// (it serves the rarer passes: the completion of an extension's last candidate and the
// candidate's third projection; the Lanczos steps call dots_rows directly).
template <class S>
__device__ __noinline__ void dots_cta(const S* __restrict__ V, long long ld, int nv, const S* __restrict__ y, int lo,
                                      int hi, bool with_norm, PmShared& s) {
  const int nvec = nv + (with_norm ? 1 : 0);
  if (nvec <= 2) {           // one or two products: one pass over rows, y loaded once
    dots_rows<S>(V, ld, nv, y, lo, hi, with_norm, s);
    return;
  }
  dots_part<S>(V, ld, nv, y, lo, hi, with_norm, s);
}

// y[r] -= sum_{i<nv} h_i V[i][r] over this CTA's rows, four consecutive rows
// per thread (16-byte accesses).  FP64: FMA in FP64; FP32: FMA in FP32 with the
// coefficients rounded to FP32; float pairs: the sum is accumulated as a float
// pair and subtracted once.
template <class S>
__device__ __forceinline__ void update_rows(S* __restrict__ y, const S* __restrict__ V, long long ld, int nv,
                                           const typename Elem<S>::Coef* h, int lo, int hi) {
  typedef Elem<S> E;
  for (int r = lo + 4 * threadIdx.x; r < hi; r += 4 * blockDim.x) {
    if (r + 3 < hi) {
      Quad<S> a;
      a.load(y + r);
      if constexpr (E::kind == 2) {
        F2Acc acc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] = f2_zero();
        int i = 0;
        for (; i + 3 < nv; i += 4) {          // four basis quads in flight
          Quad<S> v0, v1, v2, v3;
          v0.load(V + (size_t)i * ld + r);
          v1.load(V + (size_t)(i + 1) * ld + r);
          v2.load(V + (size_t)(i + 2) * ld + r);
          v3.load(V + (size_t)(i + 3) * ld + r);
          const df32 h0 = h[i], h1 = h[i + 1], h2 = h[i + 2], h3 = h[i + 3];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            f2_add_prod(acc[k], h0, v0.x[k]);
            f2_add_prod(acc[k], h1, v1.x[k]);
            f2_add_prod(acc[k], h2, v2.x[k]);
            f2_add_prod(acc[k], h3, v3.x[k]);
          }
        }
        for (; i < nv; ++i) {
          Quad<S> v0;
          v0.load(V + (size_t)i * ld + r);
          const df32 h0 = h[i];
#pragma unroll
          for (int k = 0; k < 4; ++k) f2_add_prod(acc[k], h0, v0.x[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) a.x[k] = df_sub(a.x[k], f2_round(acc[k]));
      } else {
        Quad<S> b;
#pragma unroll
        for (int k = 0; k < 4; ++k) b.x[k] = S(0);
        int i = 0;
        for (; i + 3 < nv; i += 4) {
          Quad<S> v0, v1, v2, v3;
          v0.load(V + (size_t)i * ld + r);
          v1.load(V + (size_t)(i + 1) * ld + r);
          v2.load(V + (size_t)(i + 2) * ld + r);
          v3.load(V + (size_t)(i + 3) * ld + r);
          const S h0 = h[i], h1 = h[i + 1], h2 = h[i + 2], h3 = h[i + 3];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            a.x[k] = fma(-h0, v0.x[k], a.x[k]);
            b.x[k] = fma(-h1, v1.x[k], b.x[k]);
            a.x[k] = fma(-h2, v2.x[k], a.x[k]);
            b.x[k] = fma(-h3, v3.x[k], b.x[k]);
          }
        }
        for (; i < nv; ++i) {
          Quad<S> v0;
          v0.load(V + (size_t)i * ld + r);
          const S h0 = h[i];
#pragma unroll
          for (int k = 0; k < 4; ++k) a.x[k] = fma(-h0, v0.x[k], a.x[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) a.x[k] += b.x[k];
      }
      a.store(y + r);
    } else {
      for (int q = r; q < hi; ++q) {
        if constexpr (E::kind == 2) {
          F2Acc acc = f2_zero();
          for (int i = 0; i < nv; ++i) f2_add_prod(acc, h[i], V[(size_t)i * ld + q]);
          y[q] = df_sub(y[q], f2_round(acc));
        } else {
          S a = y[q];
          for (int i = 0; i < nv; ++i) a = fma(-(S)h[i], V[(size_t)i * ld + q], a);
          y[q] = a;
        }
      }
    }
  }
}

// Two dot products per left vector in one pass, for the lagged Gram-Schmidt step
// (WIDE: more loads in flight per lane, measured faster when one CTA streams a whole
// problem and slower for the short runs of a grid team):
// with L_i = V_i (i < nv), L_nv = z and, with_ww, L_{nv+1} = w (nvec left vectors),
// s.coef[i] = L_i . z and s.coef[nvec + i] = L_i . w.  Runs per warp as in dots_cta;
// each segment leaves two warp-reduced partials in s.dred (even / odd slots).
template <class S, bool WIDE>
__device__ __forceinline__ void dot_segment2(const S* __restrict__ v, const S* __restrict__ z,
                                             const S* __restrict__ w, int a, int b, typename Elem<S>::Red& dz,
                                             typename Elem<S>::Red& dw) {
  typedef Elem<S> E;
  typedef typename E::Acc Acc;
  const int lane = threadIdx.x & 31;
  Acc z0 = E::zero(), z1 = E::zero(), w0 = E::zero(), w1 = E::zero();
  const int qa = min(b, (a + 3) & ~3);
  const int qb = max(qa, b & ~3);
  if (a + lane < qa) { E::dot(z1, v[a + lane], z[a + lane]); E::dot(w1, v[a + lane], w[a + lane]); }
  int e = qa;
  if constexpr (sizeof(S) == 8) {
    // lane owns elements 2l, 2l+1 and 64+2l, 65+2l of each 128-element block: every
    // 16-byte load instruction of a warp covers 512 contiguous bytes
    auto ld2 = [](const S* p, S& x0, S& x1) {
      const float4 q = *reinterpret_cast<const float4*>(p);
      S t0, t1;
      memcpy(&t0, &q.x, 8);
      memcpy(&t1, &q.z, 8);
      x0 = t0;
      x1 = t1;
    };
    for (; WIDE && e + 255 < qb; e += 256) {    // one CTA per problem: two blocks in flight
      S va, vb, vc, vd, za, zb, zc, zd, wa, wb, wc, wd;
      S xa, xb, xc, xd, ya, yb, yc, yd, ua, ub, uc, ud;
      const int p0 = e + 2 * lane, p1 = p0 + 64, p2 = p0 + 128, p3 = p0 + 192;
      ld2(v + p0, va, vb); ld2(v + p1, vc, vd); ld2(v + p2, xa, xb); ld2(v + p3, xc, xd);
      ld2(z + p0, za, zb); ld2(z + p1, zc, zd); ld2(z + p2, ya, yb); ld2(z + p3, yc, yd);
      ld2(w + p0, wa, wb); ld2(w + p1, wc, wd); ld2(w + p2, ua, ub); ld2(w + p3, uc, ud);
      E::dot(z0, va, za); E::dot(z1, vb, zb); E::dot(z0, vc, zc); E::dot(z1, vd, zd);
      E::dot(w0, va, wa); E::dot(w1, vb, wb); E::dot(w0, vc, wc); E::dot(w1, vd, wd);
      E::dot(z0, xa, ya); E::dot(z1, xb, yb); E::dot(z0, xc, yc); E::dot(z1, xd, yd);
      E::dot(w0, xa, ua); E::dot(w1, xb, ub); E::dot(w0, xc, uc); E::dot(w1, xd, ud);
    }
    for (; e + 127 < qb; e += 128) {
      S va, vb, vc, vd, za, zb, zc, zd, wa, wb, wc, wd;
      const int p0 = e + 2 * lane, p1 = p0 + 64;
      ld2(v + p0, va, vb); ld2(v + p1, vc, vd);
      ld2(z + p0, za, zb); ld2(z + p1, zc, zd);
      ld2(w + p0, wa, wb); ld2(w + p1, wc, wd);
      E::dot(z0, va, za); E::dot(z1, vb, zb); E::dot(z0, vc, zc); E::dot(z1, vd, zd);
      E::dot(w0, va, wa); E::dot(w1, vb, wb); E::dot(w0, vc, wc); E::dot(w1, vd, wd);
    }
  }
  e += 4 * lane;
  if constexpr (sizeof(S) == 4) {
    // FP32 basis: four quads of V per lane in flight (64 bytes; 32 KB per SM), enough
    // bytes in flight to stream the basis from HBM at full bandwidth
    for (; e + 384 + 3 < qb; e += 512) {
      Quad<S> vq[4], zq[4], wq[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) vq[u].load(v + e + 128 * u);
#pragma unroll
      for (int u = 0; u < 4; ++u) { zq[u].load(z + e + 128 * u); wq[u].load(w + e + 128 * u); }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        E::dot4((u & 1) ? z1 : z0, vq[u].x, zq[u].x);
        E::dot4((u & 1) ? w1 : w0, vq[u].x, wq[u].x);
      }
    }
  }
  for (; e + 128 + 3 < qb; e += 256) {        // two quads of each operand per lane in flight
    Quad<S> v0, v1, z0q, z1q, w0q, w1q;
    v0.load(v + e); z0q.load(z + e); w0q.load(w + e);
    v1.load(v + e + 128); z1q.load(z + e + 128); w1q.load(w + e + 128);
    E::dot4(z0, v0.x, z0q.x);
    E::dot4(w0, v0.x, w0q.x);
    E::dot4(z1, v1.x, z1q.x);
    E::dot4(w1, v1.x, w1q.x);
  }
  for (; e + 3 < qb; e += 128) {
    Quad<S> v0, z0q, w0q;
    v0.load(v + e); z0q.load(z + e); w0q.load(w + e);
    E::dot4(z0, v0.x, z0q.x);
    E::dot4(w0, v0.x, w0q.x);
  }
  if (qb + lane < b) { E::dot(z0, v[qb + lane], z[qb + lane]); E::dot(w0, v[qb + lane], w[qb + lane]); }
  dz = E::red_of(z0, z1);
  dw = E::red_of(w0, w1);
}

template <class S, bool WIDE>
__device__ __noinline__ void dots2_cta(const S* __restrict__ V, long long ld, int nv, const S* __restrict__ z,
                                       const S* __restrict__ w, int lo, int hi, bool with_ww, PmShared& s) {
  typedef Elem<S> E;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long rows = hi - lo;
  const int nvec = nv + 1 + (with_ww ? 1 : 0);
  const long long total = (long long)nvec * rows;
  if (total == 0) {
    for (int i = threadIdx.x; i < 2 * nvec; i += blockDim.x) s.coef[i] = 0.0;
    __syncthreads();
    return;
  }
  // Every product of the pass reads this CTA's rows of z and w: when they fit, they are
  // staged in shared memory once, so that L2 serves only the basis vectors (otherwise
  // z and w would cross L2 once per vector).  Same arithmetic and order either way.
  // Both staged copies start on 16-byte boundaries (the passes read them with 16-byte
  // loads at offsets that are multiples of 16 bytes from lo, as they read z and w).
  constexpr int VEC = 16 / sizeof(S);            // elements per 16-byte copy
  const long long rows16 = (rows + VEC - 1) / VEC * VEC;
  const S* zb = z;
  const S* wb = w;
  if (2 * rows16 * (long long)sizeof(S) <= (long long)PM_ZW_BYTES) {
    S* sz = reinterpret_cast<S*>(s.zw);
    S* sw = sz + rows16;
    const int nq = (int)(rows / VEC);
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      reinterpret_cast<float4*>(sz)[q] = *reinterpret_cast<const float4*>(z + lo + q * VEC);
      reinterpret_cast<float4*>(sw)[q] = *reinterpret_cast<const float4*>(w + lo + q * VEC);
    }
    for (int r = nq * VEC + threadIdx.x; r < rows; r += blockDim.x) {
      sz[r] = z[lo + r];
      sw[r] = w[lo + r];
    }
    __syncthreads();
    zb = sz - lo;                                 // indexed by absolute row, like z and w
    wb = sw - lo;
  }
  // as in dots_cta: a run meets fewer than 12 vectors, so 2 x 12 slots fit PM_DSEG
  const long long run = (((total + PM_WARPS - 1) / PM_WARPS) + 3) & ~3ll;
  long long f = (long long)warp * run;
  const long long fend = min(total, f + run);
  if (f < fend) {
    int i = (int)(f / rows);
    long long r0 = f - (long long)i * rows;
    for (int seg = 0; f < fend; ++seg, ++i, r0 = 0) {
      const long long r1 = min(rows, r0 + (fend - f));
      const S* v = (i < nv) ? V + (size_t)i * ld : (i == nv) ? zb : wb;
      typename E::Red dz, dw;
      dot_segment2<S, WIDE>(v, zb, wb, lo + (int)r0, lo + (int)r1, dz, dw);
      if constexpr (E::kind == 0) {
        // both sums in one tree: at the first level the lower half-warp keeps z and the
        // upper half keeps w, so five FP64 adds finish both (an FP64 warp instruction
        // costs the same however many of its lanes are active)
        const bool up = lane >= 16;
        double keep = up ? dw : dz;
        keep += __shfl_xor_sync(0xffffffffu, up ? dz : dw, 16);
#pragma unroll
        for (int o = 8; o; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
        if ((lane & 15) == 0) s.dred[warp * PM_DSEG + 2 * seg + (up ? 1 : 0)] = keep;
      } else {
        dz = red_warp_sum<E>(dz);
        dw = red_warp_sum<E>(dw);
        if (lane == 0) {
          red_put(&s.dred[warp * PM_DSEG + 2 * seg], dz);
          red_put(&s.dred[warp * PM_DSEG + 2 * seg + 1], dw);
        }
      }
      f += r1 - r0;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    const long long fa = (long long)i * rows, fb = fa + rows - 1;
    typename E::Red tz = E::red_zero(), tw = E::red_zero();
    for (long long w2 = fa / run; w2 <= fb / run && w2 < PM_WARPS; ++w2) {
      const int sl = (int)w2 * PM_DSEG + 2 * (int)(i - (w2 * run) / rows);
      tz = E::red_add(tz, red_get<typename E::Red>(&s.dred[sl]));
      tw = E::red_add(tw, red_get<typename E::Red>(&s.dred[sl + 1]));
    }
    s.coef[i] = E::red_val(tz);
    s.coef[nvec + i] = E::red_val(tw);
  }
  __syncthreads();
}

// The pass of an Arnoldi step whose candidate z keeps its single projection (no second
// Gram-Schmidt pass, see the Krylov loop): one product per basis element,
//   s.coef[i] = V_i . w (i < nv), s.coef[nv] = z.z, s.coef[nv+1] = z.w, s.coef[nv+2] = w.w,
// as the runs of dots_cta over the nv + 3 (left, right) pairs, z and w staged in shared
// memory when they fit.
template <class S>
__device__ __noinline__ void dots_skip_cta(const S* __restrict__ V, long long ld, int nv, const S* __restrict__ z,
                                           const S* __restrict__ w, int lo, int hi, PmShared& s) {
  typedef Elem<S> E;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long rows = hi - lo;
  const int nvec = nv + 3;
  const long long total = (long long)nvec * rows;
  if (total == 0) {
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) s.coef[i] = 0.0;
    __syncthreads();
    return;
  }
  constexpr int VEC = 16 / sizeof(S);
  const long long rows16 = (rows + VEC - 1) / VEC * VEC;
  const S* zb = z;
  const S* wb = w;
  if (2 * rows16 * (long long)sizeof(S) <= (long long)PM_ZW_BYTES) {
    S* sz = reinterpret_cast<S*>(s.zw);
    S* sw = sz + rows16;
    const int nq = (int)(rows / VEC);
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      reinterpret_cast<float4*>(sz)[q] = *reinterpret_cast<const float4*>(z + lo + q * VEC);
      reinterpret_cast<float4*>(sw)[q] = *reinterpret_cast<const float4*>(w + lo + q * VEC);
    }
    for (int r = nq * VEC + threadIdx.x; r < rows; r += blockDim.x) {
      sz[r] = z[lo + r];
      sw[r] = w[lo + r];
    }
    __syncthreads();
    zb = sz - lo;
    wb = sw - lo;
  }
  const long long run = (((total + PM_WARPS - 1) / PM_WARPS) + 3) & ~3ll;
  long long f = (long long)warp * run;
  const long long fend = min(total, f + run);
  if (f < fend) {
    int i = (int)(f / rows);
    long long r0 = f - (long long)i * rows;
    for (int seg = 0; f < fend; ++seg, ++i, r0 = 0) {
      const long long r1 = min(rows, r0 + (fend - f));
      const S* a = (i < nv) ? V + (size_t)i * ld : (i == nv + 2) ? wb : zb;
      const S* b = (i == nv) ? zb : wb;
      const typename E::Red d = red_warp_sum<E>(dot_segment<S>(a, b, lo + (int)r0, lo + (int)r1));
      if (lane == 0) red_put(&s.dred[warp * PM_DSEG + seg], d);
      f += r1 - r0;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    const long long fa = (long long)i * rows, fb = fa + rows - 1;
    typename E::Red t = E::red_zero();
    for (long long w2 = fa / run; w2 <= fb / run && w2 < PM_WARPS; ++w2)
      t = E::red_add(t, red_get<typename E::Red>(&s.dred[w2 * PM_DSEG + (int)(i - (w2 * run) / rows)]));
    s.coef[i] = E::red_val(t);
  }
  __syncthreads();
}

// Fused update of the lagged Gram-Schmidt step over this CTA's rows:
//   q = (z - sum_{i<nv} a_i V_i) * inv                  (written to qout when qout != 0)
//   z' = (w - sum_{i<nv} b_i V_i - d q) * inv            (written to zout when zout != 0)
// mode PM_UPD_Q_IS_Z: q = z (z is the normalised basis vector itself); PM_UPD_SCALE:
// q = z * inv (the candidate keeps its single projection, a = 0); PM_UPD_REORTH: as
// above.  Four consecutive rows per thread, four basis quads in flight, each loaded
// once for both sums.  zout may alias z (each thread reads its rows of z before
// writing them).
#define PM_UPD_Q_IS_Z 0
#define PM_UPD_SCALE 1
#define PM_UPD_REORTH 2
template <class S>
__device__ __forceinline__ void upd2_finish(Quad<S>& q, Quad<S>& zn, const Quad<S>& zq, const Quad<S>& wq,
                                            typename Elem<S>::Coef d, typename Elem<S>::Coef inv, int mode) {
  typedef Elem<S> E;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if constexpr (E::kind == 2) {
      q.x[k] = (mode != PM_UPD_Q_IS_Z) ? df_mul(q.x[k], inv) : zq.x[k];
      zn.x[k] = df_mul(df_sub(zn.x[k], df_mul(d, q.x[k])), inv);
    } else {
      q.x[k] = (mode != PM_UPD_Q_IS_Z) ? q.x[k] * (S)inv : zq.x[k];
      zn.x[k] = fma(-(S)d, q.x[k], zn.x[k]) * (S)inv;
    }
  }
}

template <class S>
__device__ void update_rows2(const S* __restrict__ V, long long ld, int nv, const typename Elem<S>::Coef* ca,
                             const typename Elem<S>::Coef* cb, typename Elem<S>::Coef d, typename Elem<S>::Coef inv,
                             const S* z, const S* __restrict__ w, S* qout, S* zout, int mode, int lo, int hi) {
  typedef Elem<S> E;
  for (int r = lo + 4 * threadIdx.x; r < hi; r += 4 * blockDim.x) {
    if (r + 3 < hi) {
      Quad<S> q, zn, zq, wq;
      if constexpr (E::kind == 2) {
        F2Acc sa[4], sb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) { sa[k] = f2_zero(); sb[k] = f2_zero(); }
        int i = 0;
        for (; i + 3 < nv; i += 4) {
          Quad<S> v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u].load(V + (size_t)(i + u) * ld + r);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const df32 au = ca[i + u], bu = cb[i + u];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              if (mode == PM_UPD_REORTH) f2_add_prod(sa[k], au, v[u].x[k]);
              f2_add_prod(sb[k], bu, v[u].x[k]);
            }
          }
        }
        for (; i < nv; ++i) {
          Quad<S> v0;
          v0.load(V + (size_t)i * ld + r);
          const df32 au = ca[i], bu = cb[i];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (mode == PM_UPD_REORTH) f2_add_prod(sa[k], au, v0.x[k]);
            f2_add_prod(sb[k], bu, v0.x[k]);
          }
        }
        zq.load(z + r);
        wq.load(w + r);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          q.x[k] = df_sub(zq.x[k], f2_round(sa[k]));
          zn.x[k] = df_sub(wq.x[k], f2_round(sb[k]));
        }
      } else {
        zq.load(z + r);
        wq.load(w + r);
#pragma unroll
        for (int k = 0; k < 4; ++k) { q.x[k] = zq.x[k]; zn.x[k] = wq.x[k]; }
        int i = 0;
        for (; i + 3 < nv; i += 4) {
          Quad<S> v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u].load(V + (size_t)(i + u) * ld + r);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const S au = (S)ca[i + u], bu = (S)cb[i + u];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              if (mode == PM_UPD_REORTH) q.x[k] = fma(-au, v[u].x[k], q.x[k]);
              zn.x[k] = fma(-bu, v[u].x[k], zn.x[k]);
            }
          }
        }
        for (; i < nv; ++i) {
          Quad<S> v0;
          v0.load(V + (size_t)i * ld + r);
          const S au = (S)ca[i], bu = (S)cb[i];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (mode == PM_UPD_REORTH) q.x[k] = fma(-au, v0.x[k], q.x[k]);
            zn.x[k] = fma(-bu, v0.x[k], zn.x[k]);
          }
        }
      }
      upd2_finish<S>(q, zn, zq, wq, d, inv, mode);
      if (qout) q.store(qout + r);
      if (zout) zn.store(zout + r);
    } else {
      for (int t = r; t < hi; ++t) {       // ragged end: one row at a time
        Quad<S> q, zn, zq, wq;
        if constexpr (E::kind == 2) {
          F2Acc sa = f2_zero(), sb = f2_zero();
          for (int i = 0; i < nv; ++i) {
            const df32 vi = V[(size_t)i * ld + t];
            if (mode == PM_UPD_REORTH) f2_add_prod(sa, ca[i], vi);
            f2_add_prod(sb, cb[i], vi);
          }
          zq.x[0] = z[t];
          wq.x[0] = w[t];
          q.x[0] = df_sub(zq.x[0], f2_round(sa));
          zn.x[0] = df_sub(wq.x[0], f2_round(sb));
        } else {
          zq.x[0] = z[t];
          wq.x[0] = w[t];
          S qa = zq.x[0], zb = wq.x[0];
          for (int i = 0; i < nv; ++i) {
            const S vi = V[(size_t)i * ld + t];
            if (mode == PM_UPD_REORTH) qa = fma(-(S)ca[i], vi, qa);
            zb = fma(-(S)cb[i], vi, zb);
          }
          q.x[0] = qa;
          zn.x[0] = zb;
        }
#pragma unroll
        for (int k = 1; k < 4; ++k) { q.x[k] = q.x[0]; zn.x[k] = zn.x[0]; zq.x[k] = zq.x[0]; wq.x[k] = wq.x[0]; }
        upd2_finish<S>(q, zn, zq, wq, d, inv, mode);
        if (qout) qout[t] = q.x[0];
        if (zout) zout[t] = zn.x[0];
      }
    }
  }
}

// Out-of-line copy for the rarely taken paths (second projection, completing the
// last candidate), so that they do not add to the register pressure of the main loop.
template <class S>
__device__ __noinline__ void update_rows2_cold(const S* V, long long ld, int nv, const typename Elem<S>::Coef* ca,
                                               typename Elem<S>::Coef inv, const S* z, const S* w, S* qout,
                                               int lo, int hi) {
  update_rows2<S>(V, ld, nv, ca, ca, Elem<S>::coef(0.0), inv, z, w, qout, nullptr, PM_UPD_REORTH, lo, hi);
}

// ------------------------------------------------------------------------------------
// accept step (Eq. step) over this CTA's rows: udst = F + sum_{j<p} tau^j/j! w_j with
// F = sum_{i<nvv} ucoef_i v_i (coefficients s.ucoef / s.ucf / s.ucd, the powers of tau
// at s.ucoef[PM_NSLOT + j]).  Four rows per thread with 16-byte accesses when u and
// udst allow them (the basis and W are 256-byte aligned, lo a multiple of 64 rows), so
// that a thread has a quarter of the dependent load round trips; every row takes the
// same operations in the same order as in the one-row form below.  Returns this
// thread's sum of squares of the new rows when guard is set.
// ------------------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ double accept_krylov_row(const S* __restrict__ V, long long ld, const PmShared& s, int nvv,
                                                    int r) {
  typedef Elem<S> E;
  if constexpr (E::kind == 0) {
    double acc = 0.0;
    for (int i = 0; i < nvv; ++i) acc = fma(s.ucoef[i], V[(size_t)i * ld + r], acc);
    return acc;
  } else {
    F2Acc fa = f2_zero();
    if constexpr (E::kind == 1) {
      // chunks of four terms in FP32, the chunks summed as a float pair (the
      // coefficients are FP32-rounded already, a relative error of u32 per term)
      int i = 0;
      for (; i + 3 < nvv; i += 4) {
        float q = s.ucf[i] * V[(size_t)i * ld + r];
        q = fmaf(s.ucf[i + 1], V[(size_t)(i + 1) * ld + r], q);
        q = fmaf(s.ucf[i + 2], V[(size_t)(i + 2) * ld + r], q);
        q = fmaf(s.ucf[i + 3], V[(size_t)(i + 3) * ld + r], q);
        f2_add_float(fa, q);
      }
      for (; i < nvv; ++i) f2_add_prod(fa, s.ucf[i], V[(size_t)i * ld + r]);
    } else {
      for (int i = 0; i < nvv; ++i) f2_add_prod(fa, s.ucd[i], V[(size_t)i * ld + r]);
    }
    return f2_value(fa);
  }
}

template <class S>
__device__ __forceinline__ double accept_rows(const S* __restrict__ V, long long ld, const PmShared& s, int nvv,
                                              int p, const double* u, const double* __restrict__ W, double* udst,
                                              bool guard, int lo, int hi) {
  typedef Elem<S> E;
  double un = 0.0;
  int r0 = lo;
  if (((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(udst)) & 15) == 0) {
    const int nq = (hi - lo) >> 2;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      const int r = lo + 4 * q;
      Quad<double> acc;
      if constexpr (E::kind == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) acc.x[k] = 0.0;
        int i = 0;
        for (; i + 1 < nvv; i += 2) {
          Quad<double> v0, v1;
          v0.load(V + (size_t)i * ld + r);
          v1.load(V + (size_t)(i + 1) * ld + r);
#pragma unroll
          for (int k = 0; k < 4; ++k) acc.x[k] = fma(s.ucoef[i], v0.x[k], acc.x[k]);
#pragma unroll
          for (int k = 0; k < 4; ++k) acc.x[k] = fma(s.ucoef[i + 1], v1.x[k], acc.x[k]);
        }
        if (i < nvv) {
          Quad<double> v0;
          v0.load(V + (size_t)i * ld + r);
#pragma unroll
          for (int k = 0; k < 4; ++k) acc.x[k] = fma(s.ucoef[i], v0.x[k], acc.x[k]);
        }
      } else {
        F2Acc fa[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) fa[k] = f2_zero();
        if constexpr (E::kind == 1) {
          int i = 0;
          for (; i + 3 < nvv; i += 4) {
            Quad<float> v[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) v[t].load(V + (size_t)(i + t) * ld + r);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              float c = s.ucf[i] * v[0].x[k];
              c = fmaf(s.ucf[i + 1], v[1].x[k], c);
              c = fmaf(s.ucf[i + 2], v[2].x[k], c);
              c = fmaf(s.ucf[i + 3], v[3].x[k], c);
              f2_add_float(fa[k], c);
            }
          }
          for (; i < nvv; ++i) {
            Quad<float> v0;
            v0.load(V + (size_t)i * ld + r);
#pragma unroll
            for (int k = 0; k < 4; ++k) f2_add_prod(fa[k], s.ucf[i], v0.x[k]);
          }
        } else {
          for (int i = 0; i < nvv; ++i) {
            Quad<df32> v0;
            v0.load(V + (size_t)i * ld + r);
#pragma unroll
            for (int k = 0; k < 4; ++k) f2_add_prod(fa[k], s.ucd[i], v0.x[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) acc.x[k] = f2_value(fa[k]);
      }
      if (p >= 1) {
        Quad<double> uq;
        uq.load(u + r);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc.x[k] = fma(s.ucoef[PM_NSLOT], uq.x[k], acc.x[k]);
      }
      for (int jj = 1; jj < p; ++jj) {
        Quad<double> wq;
        wq.load(W + (size_t)(jj - 1) * ld + r);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc.x[k] = fma(s.ucoef[PM_NSLOT + jj], wq.x[k], acc.x[k]);
      }
      acc.store(udst + r);
      if (guard) {
#pragma unroll
        for (int k = 0; k < 4; ++k) un = fma(acc.x[k], acc.x[k], un);
      }
    }
    r0 = lo + 4 * nq;
  }
  for (int r = r0 + threadIdx.x; r < hi; r += blockDim.x) {
    double acc = accept_krylov_row<S>(V, ld, s, nvv, r);
    if (p >= 1) acc = fma(s.ucoef[PM_NSLOT], u[r], acc);
    for (int jj = 1; jj < p; ++jj) acc = fma(s.ucoef[PM_NSLOT + jj], W[(size_t)(jj - 1) * ld + r], acc);
    udst[r] = acc;
    if (guard) un = fma(acc, acc, un);
  }
  return un;
}

// ------------------------------------------------------------------------------------
// the exponential of the augmented matrix, spread over the team's CTAs
// ------------------------------------------------------------------------------------
#define PM_EXPM_MATS 13
#define PM_EXPM_DOUBLES (PM_EXPM_MATS * PM_NA2 + 2 * PM_NA + PM_NA)

template <bool CG>
__device__ __forceinline__ double ldx(const double* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// C = A * B on the elements [e0, e1) of the N x N result (row-major, stride PM_NA).
// Grid team (MULTI): a CTA owns a few elements; one warp per element with the lanes
// splitting k, so all loads of an element are in flight at once (operands written
// by other CTAs: through L2).  One CTA: one thread per element, operands written by
// this CTA (L1-cached).
static_assert(3 * 32 >= PM_NA, "three k-slices per lane cover the augmented matrix");
template <bool MULTI>
__device__ __forceinline__ void mm_elems(double* C, const double* A, const double* B, int N, int e0, int e1) {
  if constexpr (MULTI) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = e0 + warp; e < e1; e += PM_WARPS) {
      const int i = e / N, j = e - i * N;
      double c = 0.0;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int k = lane + 32 * q;
        if (k < N) c = fma(__ldcg(&A[i * PM_NA + k]), __ldcg(&B[k * PM_NA + j]), c);
      }
      c = pm_warp_sum(c);
      if (lane == 0) C[i * PM_NA + j] = c;
    }
  } else {
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int i = e / N, j = e - i * N;
      const double* a = A + i * PM_NA;
      double c0 = 0.0, c1 = 0.0;
      int k = 0;
      for (; k + 1 < N; k += 2) {
        c0 = fma(a[k], B[k * PM_NA + j], c0);
        c1 = fma(a[k + 1], B[(k + 1) * PM_NA + j], c1);
      }
      if (k < N) c0 = fma(a[k], B[k * PM_NA + j], c0);
      C[i * PM_NA + j] = c0 + c1;
    }
  }
}

// squarings s = max(0, ceil(log2(||X||_1 / theta))) that bring ||X||_1 down to theta (Eq. 8)
__device__ __forceinline__ int pm_squarings(double norm1, double theta) {
  if (!(norm1 > theta)) return 0;
  const double v = ceil(log2(norm1 / theta));
  return v > 0 ? (int)v : 0;
}

// The squarings of the scaled exponential R (exp of the scaled augmented matrix) on the
// team: sq - 1 full squarings (oth as scratch), the last one forming only columns ca
// and cb; on return every CTA holds the top m entries of those columns in
// s.phi0 / s.phi1.  out holds 2 PM_NA doubles of team-shared scratch.
template <class Team>
__device__ bool expm_square_out(const Team& team, PmShared& s, double* R, double* R2, double* out, int N, int m,
                                int sq, int e0, int e1, int ca, int cb) {
  const int G = team.size(), rk = team.rank();
  double* cur = R;
  double* oth = R2;
  for (int q = 0; q + 1 < sq; ++q) {
    mm_elems<Team::multi>(oth, cur, cur, N, e0, e1);
    if (!team.sync()) return false;
    double* t = cur; cur = oth; oth = t;
  }
  {
    int r0, r1;
    split_range(2 * N, rk, G, r0, r1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = r0 + warp; e < r1; e += PM_WARPS) {     // one warp per entry, lanes split k
      const int which = e / N, i = e - which * N;
      const int col = which ? cb : ca;
      double v;
      if (sq == 0) {
        v = ldx<Team::multi>(&cur[i * PM_NA + col]);
      } else {
        double c0 = 0.0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int k = lane + 32 * q;
          if (k < N) c0 = fma(ldx<Team::multi>(&cur[i * PM_NA + k]), ldx<Team::multi>(&cur[k * PM_NA + col]), c0);
        }
        v = pm_warp_sum(c0);
      }
      if (lane == 0) out[which * PM_NA + i] = v;
    }
  }
  if (!team.sync()) return false;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    s.phi0[i] = ldx<Team::multi>(&out[i]);
    s.phi1[i] = ldx<Team::multi>(&out[PM_NA + i]);
  }
  __syncthreads();
  return true;
}

// exp(H_hat) by the degree-18 Taylor polynomial of X = H_hat / 2^sq, sum_k X^k / k!,
// evaluated by Paterson-Stockmeyer with the powers X, X^2, X^3, X^4 and four Horner
// steps in X^4, then sq squarings (sq from ||H_hat||_1 and theta, the largest norm whose
// truncation term stays below 2^-53 e^-theta).  Every stage is a team-parallel matrix
// product followed by one team barrier.  The Pade form needs a pivoted LU and two
// triangular solves, sequences of N CTA-wide steps, which cost more than the Taylor
// form's extra product and squarings on grid and cluster teams (115 -> 50 us per
// exponential on the 512^2 solve) and on one CTA too (709 -> 571 us per solve on the
// 32^2 one).  tc[k] = 1 / k!.  Same output as expm_team's Pade form.
template <class Team>
__device__ bool expm_taylor_team(const Team& team, PmShared& s, const double* tc, double theta, double norm1,
                                 double tau, int m, int p, double* ws, int ca, int cb) {
  const int N = m + p + 1, NN = N * N;
  const int G = team.size(), rk = team.rank();
  const int sq = pm_squarings(norm1, theta);
  double* X = ws;
  double* X2 = ws + 1 * PM_NA2;
  double* X3 = ws + 2 * PM_NA2;
  double* X4 = ws + 3 * PM_NA2;
  double* Y = ws + 4 * PM_NA2;
  double* Y2 = ws + 5 * PM_NA2;
  double* out = ws + PM_EXPM_MATS * PM_NA2;
  int e0, e1;
  split_range(NN, rk, G, e0, e1);
  const double sc = ldexp(1.0, -sq);
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int i = e / N, j = e - i * N;
    double v = 0.0;
    if (i < m && j < m) v = tau * s.H[i * PM_MAXM + j];
    else if (i == 0 && j == m) v = 1.0;
    else if (i >= m && j == i + 1) v = 1.0;
    X[i * PM_NA + j] = v * sc;
  }
  if (!team.sync()) return false;
  mm_elems<Team::multi>(X2, X, X, N, e0, e1);
  if (!team.sync()) return false;
  mm_elems<Team::multi>(X3, X2, X, N, e0, e1);
  mm_elems<Team::multi>(X4, X2, X2, N, e0, e1);
  __syncthreads();
  // the top block B_4 = c16 I + c17 X + c18 X^2, then Y <- B_j + X^4 Y for j = 3 .. 0 with
  // B_j = c_{4j} I + c_{4j+1} X + c_{4j+2} X^2 + c_{4j+3} X^3
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int i = e / N, j = e - i * N, o = i * PM_NA + j;
    Y[o] = (i == j ? tc[16] : 0.0) + tc[17] * ldx<Team::multi>(&X[o]) + tc[18] * X2[o];
  }
  if (!team.sync()) return false;
  double* cur = Y;
  double* nxt = Y2;
  for (int jb = 3; jb >= 0; --jb) {
    mm_elems<Team::multi>(nxt, X4, cur, N, e0, e1);
    __syncthreads();
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int i = e / N, j = e - i * N, o = i * PM_NA + j;
      nxt[o] += (i == j ? tc[4 * jb] : 0.0) + tc[4 * jb + 1] * ldx<Team::multi>(&X[o]) + tc[4 * jb + 2] * X2[o] +
                tc[4 * jb + 3] * X3[o];
    }
    if (!team.sync()) return false;
    double* t = cur; cur = nxt; nxt = t;
  }
  // squarings into the two matrices the products no longer need
  return expm_square_out(team, s, cur, (cur == Y) ? Y2 : Y, out, N, m, sq, e0, e1, ca, cb);
}

// warps per SM sub-partition that threads 0 .. nthreads-1 fill (warp w runs on sub-partition w % 4)
__device__ __forceinline__ int pm_warps_per_sp(int nthreads) { return ((nthreads + 31) / 32 + 3) / 4; }

// The two columns ca, cb of exp(H_hat) without forming exp(H_hat): the action
// F = exp(H_hat) [e_ca e_cb] as (T_k(H_hat / sd))^sd applied to the two unit vectors, T_k
// the degree-k Taylor polynomial, with ||H_hat||_1 / sd <= theta_k, where theta_k bounds
// the truncated tail by 2^-53 e^-theta_k as for the squaring form (the action route of
// Al-Mohy and Higham, SIAM J. Sci. Comput. 33, 2011, with the forward tail bound).  The
// products are H_hat times two N-vectors; H_hat is upper Hessenberg (tridiagonal when
// tri, the Lanczos case) plus the unit entries of Eq. (hathm), so a step costs about
// N m multiply-adds (3 N tridiagonal) against N^3 per matrix product.  On GB300 an FP64
// warp instruction holds its SM sub-partition's FP64 pipe for about 64 cycles however
// few lanes are active, so the outputs are spread one per thread over the first warps
// (tridiagonal: one (row, vector) pair per thread, H_hat / sd as three diagonals and the
// unit entries precomputed) or four lanes per row (Hessenberg: the lanes split the
// columns of H, shuffle sum, each lane forming both vectors).  On return every thread
// sees the top m entries of the columns in s.phi0 / s.phi1.
static __device__ __noinline__ void expmv_cta(PmShared& s, const DevParams& prm, double tau, int m, int p, int ca,
                                              int cb, int kdeg, int sd, bool tri) {
  // The terms are kept unscaled, Bt_j = (H_hat / sd)^j Bt_0, and enter the sum as
  // F += Bt_j / j! (1/j! from the host): one FP64 multiply-add per output instead of a
  // scaling and an add.  |Bt_j| <= theta_k^j |Bt_0| <= 6^40 |Bt_0| stays far inside the
  // FP64 range.  Each output (row, vector) has one owning thread for the whole call
  // (2N <= 146 tridiagonal, 4N <= 292 Hessenberg threads of the 512), which keeps its
  // coefficients and its entry of F in registers.
  const int N = m + p + 1;
  const int tid = threadIdx.x;
  double* Bc = s.lu;                       // [2][PM_NA] current term
  double* Bn = s.lu + 2 * PM_NA;           // [2][PM_NA] next term
  const double isd = prm.inv_int[sd];
  for (int t = tid; t < 2 * PM_NA; t += blockDim.x) {
    const int i = t % PM_NA;
    Bc[t] = (i == ((t < PM_NA) ? ca : cb)) ? 1.0 : 0.0;
  }
  constexpr int KS = 4;                    // lanes per dense row
  const int L = (m + KS - 1) / KS;         // columns of H per lane
  // this thread's output: tridiagonal (col, i) = (tid / N, tid % N); dense row i = tid / KS
  // with lane q = tid % KS (lane 0 owns the outputs of both vectors)
  const bool own_t = tri && tid < 2 * N;
  const int tc = (tid < N) ? 0 : 1, ti = tid - tc * N;
  const bool own_d = !tri && tid < N * KS;
  const int di = tid / KS, dq = tid - di * KS;
  double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;   // H_hat / sd: sub, diagonal, super, unit entry
  int im = 0, ip = 0, ia = 0;                       // their columns (clamped into [0, N))
  double f0 = 0.0, f1 = 0.0;                        // F entries owned (f1: second vector, dense lane 0)
  if (own_t) {
    const double ts = tau * isd;
    const double* h = &s.H[ti * PM_MAXM];
    d0 = (ti < m && ti > 0) ? ts * h[ti - 1] : 0.0;
    d1 = (ti < m) ? ts * h[ti] : 0.0;
    d2 = (ti + 1 < m) ? ts * h[ti + 1] : 0.0;
    d3 = (ti == 0 || (ti >= m && ti < m + p)) ? isd : 0.0;   // H_hat[0][m], H_hat[i][i+1]
    im = ti > 0 ? ti - 1 : 0;
    ip = ti + 1 < N ? ti + 1 : ti;
    const int a = (ti == 0) ? m : ti + 1;
    ia = a < N ? a : ti;
    f0 = (ti == (tc ? cb : ca)) ? 1.0 : 0.0;
  }
  if (own_d && dq == 0) {
    f0 = (di == ca) ? 1.0 : 0.0;
    f1 = (di == cb) ? 1.0 : 0.0;
  }
  __syncthreads();
  // dense: whole warps take part in the shuffles, lanes past N * KS with zero sums
  const int nt = (N * KS + 31) & ~31;
  for (int st = 0; st < sd; ++st) {
    for (int j = 1; j <= kdeg; ++j) {
      const double cj = prm.xv_invfact[j];
      if (own_t) {
        const double* b = Bc + tc * PM_NA;
        double v = d1 * b[ti];
        v = fma(d0, b[im], v);
        v = fma(d2, b[ip], v);
        v = fma(d3, b[ia], v);
        Bn[tc * PM_NA + ti] = v;
        f0 = fma(cj, v, f0);
      } else if (!tri && tid < nt) {
        double a0 = 0.0, a1 = 0.0;
        if (own_d && di < m) {
          const int k0 = max(dq * L, di - 1 > 0 ? di - 1 : 0), k1 = min(m, (dq + 1) * L);
          const double* h = &s.H[di * PM_MAXM];
          for (int k = k0; k < k1; ++k) {
            a0 = fma(h[k], Bc[k], a0);
            a1 = fma(h[k], Bc[PM_NA + k], a1);
          }
        }
        a0 += __shfl_xor_sync(0xffffffffu, a0, 1);
        a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
        a0 += __shfl_xor_sync(0xffffffffu, a0, 2);
        a1 += __shfl_xor_sync(0xffffffffu, a1, 2);
        if (own_d && dq == 0) {
          double v0, v1;
          if (di < m) {
            v0 = tau * a0;
            v1 = tau * a1;
            if (di == 0) { v0 += Bc[m]; v1 += Bc[PM_NA + m]; }
          } else {
            v0 = (di < m + p) ? Bc[di + 1] : 0.0;
            v1 = (di < m + p) ? Bc[PM_NA + di + 1] : 0.0;
          }
          v0 *= isd;
          v1 *= isd;
          Bn[di] = v0;
          Bn[PM_NA + di] = v1;
          f0 = fma(cj, v0, f0);
          f1 = fma(cj, v1, f1);
        }
      }
      __syncthreads();
      double* t2 = Bc; Bc = Bn; Bn = t2;
    }
    // the next step starts from the partial sum: Bt_0 = F
    if (own_t) Bc[tc * PM_NA + ti] = f0;
    if (own_d && dq == 0) {
      Bc[di] = f0;
      Bc[PM_NA + di] = f1;
    }
    __syncthreads();
  }
  if (own_t && ti < m) (tc ? s.phi1 : s.phi0)[ti] = f0;
  if (own_d && dq == 0 && di < m) {
    s.phi0[di] = f0;
    s.phi1[di] = f1;
  }
  __syncthreads();
}

// exp(H_hat) with H_hat = [[tau H_m, e_1, 0], [0, 0, I_p], [0, 0, 0]] (Eq. hathm,
// size N = m+p+1), degree-13 Pade approximant (even/odd split) with sq
// squarings (Sec. 3.1).  Products are split over the team by elements; every CTA
// factorises the denominator in its own shared memory; the right-hand sides are
// split by columns; only columns ca and cb of the last square are formed.
// On return every CTA holds the top m entries of those columns in s.phi0/phi1.
template <class Team>
__device__ bool expm_team(const Team& team, PmShared& s, const DevParams& prm, double norm1, double tau, int m, int p,
                          int sq, double* ws, int ca, int cb) {
  if (prm.expm_taylor)
    return expm_taylor_team(team, s, prm.taylor_c, prm.taylor_theta, norm1, tau, m, p, ws, ca, cb);
  const double* bc = prm.pade_b;
  const int N = m + p + 1, NN = N * N;
  const int G = team.size(), rk = team.rank();
  double* X = ws;
  double* X2 = ws + 1 * PM_NA2;
  double* X4 = ws + 2 * PM_NA2;
  double* X6 = ws + 3 * PM_NA2;
  double* T1 = ws + 4 * PM_NA2;
  double* T2 = ws + 5 * PM_NA2;
  double* U = ws + 6 * PM_NA2;
  double* Vm = ws + 7 * PM_NA2;
  double* U2 = ws + 8 * PM_NA2;
  double* Pm = ws + 9 * PM_NA2;
  double* Q = ws + 10 * PM_NA2;
  double* R = ws + 11 * PM_NA2;
  double* R2 = ws + 12 * PM_NA2;
  double* out = ws + PM_EXPM_MATS * PM_NA2;
  int e0, e1;
  split_range(NN, rk, G, e0, e1);
  const double sc = ldexp(1.0, -sq);
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int i = e / N, j = e - i * N;
    double v = 0.0;
    if (i < m && j < m) v = tau * s.H[i * PM_MAXM + j];
    else if (i == 0 && j == m) v = 1.0;
    else if (i >= m && j == i + 1) v = 1.0;
    X[i * PM_NA + j] = v * sc;
  }
  if (!team.sync()) return false;
  mm_elems<Team::multi>(X2, X, X, N, e0, e1);
  if (!team.sync()) return false;
  mm_elems<Team::multi>(X4, X2, X2, N, e0, e1);
  if (!team.sync()) return false;
  mm_elems<Team::multi>(X6, X4, X2, N, e0, e1);
  __syncthreads();
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int i = e / N, j = e - i * N, o = i * PM_NA + j;
    T1[o] = bc[13] * X6[o] + bc[11] * X4[o] + bc[9] * X2[o];
    T2[o] = bc[12] * X6[o] + bc[10] * X4[o] + bc[8] * X2[o];
  }
  if (!team.sync()) return false;
  mm_elems<Team::multi>(U, X6, T1, N, e0, e1);
  mm_elems<Team::multi>(Vm, X6, T2, N, e0, e1);
  __syncthreads();
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int i = e / N, j = e - i * N, o = i * PM_NA + j;
    const double id = (i == j) ? 1.0 : 0.0;
    U[o] = U[o] + bc[7] * X6[o] + bc[5] * X4[o] + bc[3] * X2[o] + bc[1] * id;
    Vm[o] = Vm[o] + bc[6] * X6[o] + bc[4] * X4[o] + bc[2] * X2[o] + bc[0] * id;
  }
  if (!team.sync()) return false;
  mm_elems<Team::multi>(U2, X, U, N, e0, e1);     // odd part X * (...)
  __syncthreads();
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int i = e / N, j = e - i * N, o = i * PM_NA + j;
    Pm[o] = Vm[o] + U2[o];           // numerator
    Q[o] = Vm[o] - U2[o];            // denominator
  }
  if (!team.sync()) return false;
  // LU factorisation with partial pivoting of Q, by every CTA in its own shared
  // memory (at most 73 x 73): no CTA waits for another, the factors are bit-identical
  // in every CTA (same inputs, same order), and the solves below read them at shared-
  // memory latency.  Q was formed by other CTAs: read through L2.
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* L = s.lu;
    for (int i = warp; i < N; i += PM_WARPS)
      for (int j = lane; j < N; j += 32) L[i * PM_NA + j] = ldx<Team::multi>(&Q[i * PM_NA + j]);
    __syncthreads();
    for (int k = 0; k < N; ++k) {
      if (warp == 0) {
        // pivot search on integer keys: the bit patterns of |x| order as the values do,
        // and integer compares stay off the FP64 pipe (on GB300 every FP64 warp
        // instruction, compares included, occupies it for about 64 cycles)
        long long best = -1;
        int bi = k;
        for (int i = k + lane; i < N; i += 32) {
          const long long a = __double_as_longlong(L[i * PM_NA + k]) & 0x7fffffffffffffffll;
          if (a > best) { best = a; bi = i; }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (bi != k)
          for (int j = lane; j < N; j += 32) {
            const double t = L[k * PM_NA + j];
            L[k * PM_NA + j] = L[bi * PM_NA + j];
            L[bi * PM_NA + j] = t;
          }
        __syncwarp();
        const double rp = 1.0 / L[k * PM_NA + k];
        for (int i = k + 1 + lane; i < N; i += 32) L[i * PM_NA + k] *= rp;
        if (lane == 0) {
          s.piv[k] = bi;
          s.rdiag[k] = rp;
        }
      }
      __syncthreads();
      // trailing update, its r x r elements spread flat over the CTA (fewest FP64 warp
      // instructions: their cost does not depend on how many lanes are active)
      const int r = N - k - 1;
      for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int i = k + 1 + e / r, j = k + 1 + e % r;
        L[i * PM_NA + j] = fma(-L[i * PM_NA + k], L[k * PM_NA + j], L[i * PM_NA + j]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {            // the row interchanges as one permutation: row i of P R = row perm[i] of P
      for (int i = 0; i < N; ++i) s.perm[i] = i;
      for (int k = 0; k < N; ++k) {
        const int pk = s.piv[k];
        if (pk != k) { const int t = s.perm[k]; s.perm[k] = s.perm[pk]; s.perm[pk] = t; }
      }
    }
    __syncthreads();
  }
  // R = Q^{-1} P on the CTA's columns [c0, c1) (columns split over the team), in place in
  // R: every substitution step updates all of the CTA's columns at once, the elements
  // spread flat over its threads (one CTA-wide barrier per step)
  {
    int c0, c1;
    split_range(N, rk, G, c0, c1);
    const int nc = c1 - c0;
    const double* L = s.lu;
    for (int e = threadIdx.x; e < N * nc; e += blockDim.x) {
      const int i = e / nc, j = c0 + e % nc;
      R[i * PM_NA + j] = ldx<Team::multi>(&Pm[s.perm[i] * PM_NA + j]);
    }
    __syncthreads();
    for (int k = 0; k + 1 < N && nc > 0; ++k) {     // unit lower triangular
      const int r = N - k - 1;
      for (int e = threadIdx.x; e < r * nc; e += blockDim.x) {
        const int i = k + 1 + e / nc, j = c0 + e % nc;
        R[i * PM_NA + j] = fma(-L[i * PM_NA + k], R[k * PM_NA + j], R[i * PM_NA + j]);
      }
      __syncthreads();
    }
    for (int k = N - 1; k >= 0 && nc > 0; --k) {    // upper triangular
      for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x) R[k * PM_NA + j] *= s.rdiag[k];
      __syncthreads();
      for (int e = threadIdx.x; e < k * nc; e += blockDim.x) {
        const int i = e / nc, j = c0 + e % nc;
        R[i * PM_NA + j] = fma(-L[i * PM_NA + k], R[k * PM_NA + j], R[i * PM_NA + j]);
      }
      __syncthreads();
    }
  }
  if (!team.sync()) return false;
  return expm_square_out(team, s, R, R2, out, N, m, sq, e0, e1, ca, cb);
}


// ------------------------------------------------------------------------------------
// the solver
// ------------------------------------------------------------------------------------
struct Ctl {   // controller memory of Algorithm 4 within one step (thread 0 only)
  bool rejected, tau_changed, m_changed, qf, kf;
  double q, kap, eps_old, tau_old;
  int m_old;
};

__device__ __forceinline__ void ctl_reset(Ctl& c) {
  c.rejected = c.tau_changed = c.m_changed = c.qf = c.kf = false;
  c.q = 0.0; c.kap = 2.0; c.eps_old = 0.0; c.tau_old = 0.0; c.m_old = 0;
}

template <class S> __device__ __forceinline__ typename Elem<S>::Coef* coef_array(PmShared& s);
template <> __device__ __forceinline__ double* coef_array<double>(PmShared& s) { return s.hdd; }
template <> __device__ __forceinline__ float* coef_array<float>(PmShared& s) { return s.hf; }
template <> __device__ __forceinline__ df32* coef_array<df32>(PmShared& s) { return s.hd; }
template <class S> __device__ __forceinline__ typename Elem<S>::Coef* coef_array2(PmShared& s);
template <> __device__ __forceinline__ double* coef_array2<double>(PmShared& s) { return s.hdd2; }
template <> __device__ __forceinline__ float* coef_array2<float>(PmShared& s) { return s.hf2; }
template <> __device__ __forceinline__ df32* coef_array2<df32>(PmShared& s) { return s.hd2; }
template <class S> __device__ __forceinline__ typename Elem<S>::Coef scal_inv(const PmScal& c);
template <> __device__ __forceinline__ double scal_inv<double>(const PmScal& c) { return c.inv; }
template <> __device__ __forceinline__ float scal_inv<float>(const PmScal& c) { return c.invf; }
template <> __device__ __forceinline__ df32 scal_inv<df32>(const PmScal& c) { return c.inv2; }

__device__ __forceinline__ void set_inv(PmScal& c, double x) {   // thread 0: 1/x in every form
  c.inv = 1.0 / x;
  c.invf = (float)c.inv;
  c.inv2 = df_from_d(c.inv);
}

// Algorithm 3's attempt outcome after the controller (thread 0 decides)
#define PM_ATT_RETRY 0     // non-finite estimate or FP32 guard: try again with a smaller tau
#define PM_ATT_REJECT 1    // omega > delta
#define PM_ATT_ACCEPT 2    // omega <= delta
#define PM_ATT_FAIL 3      // status set

template <class Team, class S>
__device__ __forceinline__ void phipm_device(const Team& team, const DevProblem& P, const DevParams& prm, DevResult& res,
                             PmShared& s, const PmWork& w) {
  typedef Elem<S> E;
  typedef typename E::Coef C;
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
  C* hc = coef_array<S>(s);               // coefficients of the current update, as S needs them
  PmScal& c = s.sc;                       // scalar state: written by thread 0, read after a barrier
  int parity = 0;
  long long matvecs = 0, kry_steps = 0, gs_vectors = 0, reorth_vectors = 0;
  Ctl ctl;                                // thread 0's controller memory
  ctl_reset(ctl);
#ifdef PM_PHASE_PROBE
  long long pm_t_last = clock64();
#endif
  // the stencil products stage their rows through the TMA engine (stage_rows)
  unsigned tma_phase = 0;
  const Stage stage{s.zw, &s.mbar, &tma_phase, prm.timeout_cycles};
  const Stage* stg = prm.stencil_stage ? &stage : nullptr;
  if (tid == 0) pm_mbar_init(&s.mbar);
  for (int e = tid; e < (PM_MAXM + 1) * PM_MAXM; e += nth) s.H[e] = 0.0;
  if (tid == 0) {
    c.status = PM_OK;
    c.steps = c.rejects = c.expms = 0;
    c.err_sum = 0.0;
    c.normA = c.normb = c.last_tau = 0.0;
    c.last_m = 0;
    c.symmetric = 0;
  }
  __syncthreads();

#define PM_SYNC_OR_FAIL() do { if (!team.sync()) { if (tid == 0) c.status = PM_ETIMEOUT; goto done; } } while (0)
// team sums: PM_SUM_OR_FAIL in FP64 (norms of the FP64 vectors u and w_p, whose squares
// can leave the float range); PM_BSUM_OR_FAIL for dot products of basis-type vectors,
// folded as float pairs when the basis is FP32 or float pairs (their partials were
// already accumulated in that format)
#define PM_SUM_OR_FAIL(K) do { if (!team_sum<false>(team, s, (K), w, parity)) { if (tid == 0) c.status = PM_ETIMEOUT; goto done; } } while (0)
#define PM_BSUM_OR_FAIL(K) do { if (!team_sum<(Elem<S>::kind != 0)>(team, s, (K), w, parity)) { if (tid == 0) c.status = PM_ETIMEOUT; goto done; } } while (0)
#define PM_SPMV_OR_FAIL(call) do { if (!(call)) { if (tid == 0) c.status = PM_ETIMEOUT; goto done; } } while (0)
#define PM_MAX_OR_FAIL(K) do { if (!team_max(team, s, (K), w, parity)) { if (tid == 0) c.status = PM_ETIMEOUT; goto done; } } while (0)

  // ---------------- setup (a1): ||A||_inf, ||b_0||_inf, max_k ||b_k||_inf, symmetry; u = b_0
  {
    double na = 0.0, nb0 = 0.0, nball = 0.0, asym = 0.0;
    for (int r = lo + tid; r < hi; r += nth) {
      if (P.A.kind == 2 && !(P.A.fnorm > 0.0)) {    // matrix-free, no bound given: row sums
        double rs = 0.0;
        fn_row(P.A, r, [&](int i) { return 0.0; }, &rs);
        na = fmax(na, rs);
      }
      if (P.A.kind == 0) {
        const int k0 = P.A.rowptr[r], k1 = P.A.rowptr[r + 1];
        double rs = 0.0;
        for (int k = k0; k < k1; ++k) {
          const double a = P.A.val[k];
          rs += fabs(a);
          if (P.symm < 0) {       // look for the transposed entry in row colind[k]
            const int cc = P.A.colind[k];
            const int q0 = P.A.rowptr[cc], q1 = P.A.rowptr[cc + 1];
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
    if ((tid & 31) == 0) { s.red[tid >> 5][0] = t0; s.red[tid >> 5][1] = t1; s.red[tid >> 5][2] = t2; s.red[tid >> 5][3] = t3; }
    __syncthreads();
    if (tid < 4) {
      double a = 0.0;
      for (int q = 0; q < PM_WARPS; ++q) a = fmax(a, s.red[q][tid]);
      s.coef[tid] = a;
    }
    __syncthreads();
    PM_MAX_OR_FAIL(4);
  }
  if (tid == 0) {
    double normA;
    if (P.A.kind == 0) {
      normA = s.coef[0];
    } else if (P.A.kind == 2) {
      normA = (P.A.fnorm > 0.0) ? P.A.fnorm : s.coef[0];
    } else {
      normA = fabs(P.A.cc);
      for (int d = 0; d < P.A.ndim; ++d) normA += fabs(P.A.cm[d]) + fabs(P.A.cp[d]);
    }
    double normb = s.coef[1];
    bool symmetric;
    if (P.symm >= 0) symmetric = P.symm != 0;
    else if (P.A.kind == 0) symmetric = s.coef[3] == 0.0;
    else if (P.A.kind == 2) symmetric = false;    // a function's symmetry is not detected (symm = 1 declares it)
    else {
      symmetric = true;
      for (int d = 0; d < P.A.ndim; ++d) symmetric = symmetric && (P.A.cm[d] == P.A.cp[d]);
    }
    if (normb == 0.0) normb = s.coef[2];
    c.normA = normA;
    c.normb = normb;
    c.symmetric = symmetric ? 1 : 0;
    // Lanczos (Algorithm 2) for symmetric A with an FP64-class basis; the FP32
    // basis always uses full Arnoldi orthogonalisation (the three-term recurrence
    // loses orthogonality in FP32)
    c.lanczos = (symmetric && E::kind != 1) ? 1 : 0;
    c.go = (n > 0 && normb > 0.0) ? 1 : 0;
    c.tol = P.tol > 0.0 ? P.tol : 1e-7;
    c.t_end = P.t_end;
    c.m = min(prm.m_init, prm.m_max);
    c.bd_abs = prm.breakdown_tol * fmax(normA, 2.2250738585072014e-308);
    if (normA == 0.0) {
      c.tau = c.t_end;
    } else {       // Eq. (tau_0) in logarithms, m_bar = (m_init + m_max)/2
      const double mb = 0.5 * (prm.m_init + prm.m_max);
      const double lg = log(c.tol) + (mb + 1.0) * (log(mb + 1.0) - 1.0) +
                        0.5 * log(2.0 * 3.141592653589793 * (mb + 1.0)) - log(4.0 * normA * normb);
      c.tau = fmin(10.0 / normA * exp(lg / mb), c.t_end);
    }
    c.t = 0.0;
    c.nonfinite = 0;
    c.last_omega = 1.0;
    c.prev_rejects = 0;
    c.step_rejects = 0;
  }
  __syncthreads();
  if (!c.go) {        // every b_k = 0: u = 0
    for (int r = lo + tid; r < hi; r += nth) u[r] = 0.0;
    goto done;
  }
  PM_SYNC_OR_FAIL();  // u = b_0 complete before the first SpMV
  PM_MARK(0);

  while (c.t < c.t_end) {
    // ---------------- w-recurrence (a2), Eq. (wrecurrence): p SpMVs in FP64
    if (tid == 0) {
      c.tl[0] = 1.0;
      for (int l = 1; l <= p; ++l) c.tl[l] = c.tl[l - 1] * c.t / (double)l;
    }
    __syncthreads();
    for (int j = 1; j <= p; ++j) {
      const double* xin = (j == 1) ? u : W + (size_t)(j - 2) * ld;
      double* wout = W + (size_t)(j - 1) * ld;
      VecLoad<double, Team::multi> xl{xin, lo, hi};
      WEpi we{wout, P.b + j, c.tl, p - j, j == p, 0.0};
      if (P.A.kind == 1 && P.A.quad) {
        PM_SPMV_OR_FAIL((stencil_rows4_epi<double, Team::multi>(P.A, xin, lo, hi, we, stg)));
      } else {
        for (int r = lo + tid; r < hi; r += nth) we.row(r, spmv_row<double>(P.A, r, xl));
      }
      const double nrm = we.nrm;
      matvecs += 1;
      if (j == p) {
        const double v[1] = {nrm};
        block_sum(s, v, 1, s.coef);
        PM_SUM_OR_FAIL(1);
      } else {
        PM_SYNC_OR_FAIL();
      }
    }
    if (p == 0) {
      double nrm = 0.0;
      for (int r = lo + tid; r < hi; r += nth) nrm = fma(u[r], u[r], nrm);
      const double v[1] = {nrm};
      block_sum(s, v, 1, s.coef);
      PM_SUM_OR_FAIL(1);
    }
    PM_MARK(1);
    if (tid == 0) {
      c.beta = sqrt(s.coef[0]);
      if (c.beta > 0.0) set_inv(c, c.beta);
      c.kcur = 0;          // Arnoldi / Lanczos steps done for this w_p
      c.invariant = 0;     // happy breakdown reached
      c.skipz = 0;
      c.hn = 0.0;          // ||y|| of the last step (h_{kcur+1,kcur})
      c.attempt = 0;
      c.source = 0;
      ctl_reset(ctl);
    }
    __syncthreads();
    if (prm.mlp != nullptr && (c.steps == 0 || prm.mlp_every_step) && tid < 32) {
      // learned controller (a11): propose (tau, m) for the first attempt of the first
      // step, in place of Eq. (tau_0) and m_init, or (mlp_every_step) for the first
      // attempt of every step, from the live state: the tau and m Algorithm 4 carried
      // into the step, omega of the last accepted attempt and the last step's rejects.
      // After a rejected attempt Algorithm 4 takes over for the rest of the step.
      const float* blob = prm.mlp;
      if (tid == 0) {
        const double raw[MLP_IN] = {log10(c.normA * c.t_end), log10(c.tol), (double)p, log10(c.tau * c.normA),
                                    c.m / 64.0, log10(fmax(c.last_omega, 1e-6)), (double)c.prev_rejects,
                                    log10((double)n)};
        for (int i = 0; i < MLP_IN; ++i)
          c.feat[i] = (float)((raw[i] - blob[MLP_NP + i]) / blob[MLP_NP + MLP_IN + i]);
      }
      __syncwarp();
      float x[MLP_IN];
      bool ok = true;
      for (int i = 0; i < MLP_IN; ++i) { x[i] = c.feat[i]; ok = ok && isfinite(x[i]); }
      if (ok) {
        float y[MLP_OUT];
        mlp_warp_forward(blob, x, s.mh[0], s.mh[1], y);
        if (tid == 0) {
          const double lr = (double)y[0] * blob[MLP_NP + 2 * MLP_IN + 2] + blob[MLP_NP + 2 * MLP_IN];
          const double mm = (double)y[1] * blob[MLP_NP + 2 * MLP_IN + 3] + blob[MLP_NP + 2 * MLP_IN + 1];
          if (isfinite(lr) && isfinite(mm)) {
            if (c.steps == 0) {
              // the first step: Eq. (tau_0) and m_init are guesses, so the proposal may move
              // tau by 1/32 .. 8 and m anywhere in [1, m_max]
              const double ratio = exp2(fmin(fmax(lr, -5.0), 3.0));
              c.tau = fmin(c.tau * ratio, c.t_end - c.t);
              c.m = (int)fmin(fmax(rint(64.0 * mm), 1.0), (double)prm.m_max);
            } else {
              // later steps start from Algorithm 4's measured proposal, and the network may
              // only raise its tau, up to 2 tau; m stays Algorithm 4's.  Algorithm 3 lets tau
              // grow by at most 2x per step, so a network that lowered tau (or m, which
              // Algorithm 4 mostly keeps) on every step would ratchet the step size down for
              // good; a raised tau that fails is rejected and the paper's controller retries.
              const double ratio = exp2(fmin(fmax(lr, 0.0), 1.0));
              c.tau = fmin(c.tau * ratio, c.t_end - c.t);
            }
            c.source = 1;
          }
        }
      }
    }
    __syncthreads();
    const double* wp = (p == 0) ? u : W + (size_t)(p - 1) * ld;
    for (;;) {   // attempts of one step (Algorithm 3, inner loop)
      PM_MARK(2);
      if (tid == 0) {
        c.tau_used = c.tau;
        c.m_req = c.m;
        c.m_used = c.m;
        c.m_new = NAN;
        c.eps = 0.0;
        c.hlast = 0.0;
        c.sq = 0;
        c.norm1 = (p > 0) ? 1.0 : 0.0;
      }
      __syncthreads();
      if (c.beta > 0.0) {
        // ---------------- Krylov extension (a3/a4) to m steps
        const int target = c.invariant ? c.kcur : c.m;
        const int j0 = c.kcur;   // first step of this extension
        if (j0 < target && !c.lanczos) {
          // Arnoldi with lagged (delayed) classical Gram-Schmidt and reorthogonalisation:
          // iteration j applies A to the candidate z for v_j (projected once, not yet
          // reorthogonalised or normalised), and one pass over V_0..V_{j-1} gives both
          // the candidate's second-pass coefficients a = V^T z (with z.z) and the new
          // vector's coefficients b = V^T w (with z.w), w = A z.  With nu = ||z - V a||
          // (Pythagoras), v_j = (z - V a) / nu, column j-1 of H gains a and nu, and by
          // the Arnoldi relation A v_j = (w - V_{j+1} H a) / nu, whose projections are
          // known without touching the vectors again:
          //   H[i][j] (first pass) = (b_i - (H a)_i) / nu,   i < j,
          //   H[j][j] (first pass) = (d - (H a)_j) / nu,     d = (z.w - a.b) / nu,
          //   next candidate       = (w - V b - d v_j) / nu.
          // One pass of dot products, one team reduction, one fused update and one team
          // barrier per step, against two of each for classical Gram-Schmidt applied
          // twice.  The last candidate is completed after the loop.  At the first
          // iteration of an extension the candidate is v_j itself (a = 0, nu = 1).
          // With the FP64-class bases the second pass is selective: the pass also forms
          // w.w and ||b||^2, which give by Pythagoras how much of w the next candidate
          // keeps; when it keeps at least a quarter of its norm, the next step skips that
          // candidate's second pass (a = 0) and streams the basis with one product per
          // element (dots_skip_cta, PM_UPD_SCALE) instead of two.
          S* Z = Y;                          // candidate (own rows + halo)
          S* Wv = Y + ld;                    // A applied to the candidate
          C* ca = coef_array<S>(s);
          C* cb = coef_array2<S>(s);
          for (int j = j0; j < target; ++j) {
            const bool zfinal = (j == j0);
            const S* zp = zfinal ? V + (size_t)j * ld : Z;
            if (j == 0) {
              const C sc = scal_inv<S>(c);   // 1/beta
              DLoadAs<S, Team::multi> xl{wp, lo, hi};
              for (int r = lo + tid; r < hi; r += nth) V[r] = E::from_d(wp[r] * c.inv);
              spmv_rows<S>(P.A, xl, Wv, sc, true, lo, hi);
            } else {
              VecLoad<S, Team::multi> xl{zp, lo, hi};
              PM_SPMV_OR_FAIL(spmv_rows<S>(P.A, xl, Wv, scal_inv<S>(c), false, lo, hi, stg));
            }
            matvecs += 1;
            kry_steps += 1;
            gs_vectors += j;
            __syncthreads();
            PM_MARK(3);
            // single: z keeps its one projection (or is v_j itself): only V^T w is needed
            const bool single = zfinal || c.skipz;
            if (!single) reorth_vectors += j;
            const bool with_ww = E::kind != 1;
            int ib, izw, iww, K;                 // where b, z.w and w.w land in s.coef
            if (single) {
              dots_skip_cta<S>(V, ld, j, zp, Wv, lo, hi, s);
              ib = 0; izw = j + 1; iww = j + 2; K = j + 3;
            } else {
              dots2_cta<S, !Team::multi>(V, ld, j, zp, Wv, lo, hi, with_ww, s);
              const int nvec = j + 1 + (with_ww ? 1 : 0);
              ib = nvec; izw = nvec + j; iww = nvec + j + 1; K = 2 * nvec;
            }
            PM_MARK(4);
            PM_BSUM_OR_FAIL(K);
            PM_MARK(5);
            // scalars by one warp (||a||^2, a.b, ||b||^2); a and b copied by every thread
            if (tid < 32) {
              double aa = 0.0, ab = 0.0, bb = 0.0;
              for (int k = tid; k < j; k += 32) {
                const double ak = single ? 0.0 : s.coef[k], bk = s.coef[ib + k];
                aa = fma(ak, ak, aa);
                ab = fma(ak, bk, ab);
                bb = fma(bk, bk, bb);
              }
              aa = pm_warp_sum(aa);
              ab = pm_warp_sum(ab);
              bb = pm_warp_sum(bb);
              if (tid == 0) {
                c.fz = s.coef[j];                // z.z
                c.fw = s.coef[izw];              // z.w
                c.fww = with_ww ? s.coef[iww] : 0.0;   // w.w
                c.fab = ab;                      // a.b
                c.fbb = bb;                      // ||b||^2
                c.hn = zfinal ? 1.0 : c.fz - aa; // nu^2 by Pythagoras
                c.measure = (single || aa <= 0.25 * c.fz) ? 0 : 1;   // else: project the candidate again
              }
            }
            for (int k = tid; k < j; k += nth) {
              const double ak = single ? 0.0 : s.coef[k], bk = s.coef[ib + k];
              s.h1[k] = ak;
              s.hb[k] = bk;
              ca[k] = E::coef(ak);
              cb[k] = E::coef(bk);
            }
            __syncthreads();
            if (c.measure) {
              // q0 = z - V a into v_j's slot, then its own projections a2 and norm
              update_rows2_cold<S>(V, ld, j, ca, E::coef(1.0), zp, Wv, V + (size_t)j * ld, lo, hi);
              __syncthreads();
              dots_cta<S>(V, ld, j, V + (size_t)j * ld, lo, hi, true, s);
              PM_BSUM_OR_FAIL(j + 1);
              if (tid < 32) {
                double aa = 0.0;
                for (int k = tid; k < j; k += 32) aa = fma(s.coef[k], s.coef[k], aa);
                aa = pm_warp_sum(aa);
                if (tid == 0) {
                  const double q0 = s.coef[j];
                  c.hn = (aa <= 0.25 * q0) ? q0 - aa : 0.0;   // still not orthogonal: numerically in the span
                }
              }
              for (int k = tid; k < j; k += nth) {
                s.h1[k] += s.coef[k];
                ca[k] = E::coef(s.h1[k]);
              }
              __syncthreads();
              if (tid < 32) {
                double ab = 0.0;
                for (int k = tid; k < j; k += 32) ab = fma(s.h1[k], s.hb[k], ab);
                ab = pm_warp_sum(ab);
                if (tid == 0) c.fab = ab;
              }
              __syncthreads();
            }
            if (tid == 0) {
              c.hn = sqrt(fmax(c.hn, 0.0));
              if (!zfinal && c.hn <= c.bd_abs) {   // happy breakdown (R12): span(v_0..v_{j-1}) is invariant
                c.invariant = 1;
                c.kcur = j;
                c.hn = 0.0;
              } else {
                set_inv(c, c.hn);
                c.dcoef = (c.fw - c.fab) * c.inv;  // d = (z.w - a.b) / nu
                // the next candidate w - V b - d v_j keeps ||.||^2 = w.w - ||b||^2 - d^2 of
                // w.w (Pythagoras); if that is at least PM_ETA2 w.w, one projection leaves it
                // orthogonal to working accuracy and its second pass is skipped
                const double keep = c.fww - c.fbb - c.dcoef * c.dcoef;
                c.skipz = (with_ww && c.fww > 0.0 && keep >= PM_ETA2 * c.fww) ? 1 : 0;
              }
            }
            __syncthreads();
            if (c.invariant) {
              for (int k = tid; k < j; k += nth) s.H[k * PM_MAXM + j - 1] += s.h1[k];
              if (tid == 0) s.H[j * PM_MAXM + j - 1] = 0.0;
              __syncthreads();
              break;
            }
            PM_MARK(6);
            // columns j-1 (second pass, subdiagonal nu) and j (first pass) of H, row l by
            // thread l; H is next read after later barriers, so the update starts at once
            for (int l = tid; l <= j; l += nth) {
              if (l < j) {
                double g = 0.0;
                for (int i = max(l - 1, 0); i < j - 1; ++i) g = fma(s.H[l * PM_MAXM + i], s.h1[i], g);
                double hl = s.H[l * PM_MAXM + j - 1];
                if (!zfinal) {
                  hl += s.h1[l];
                  s.H[l * PM_MAXM + j - 1] = hl;
                }
                g = fma(hl, s.h1[j - 1], g);
                s.H[l * PM_MAXM + j] = (s.hb[l] - g) * c.inv;
              } else {
                if (j > 0 && !zfinal) s.H[j * PM_MAXM + j - 1] = c.hn;
                const double g = (j > 0) ? c.hn * s.h1[j - 1] : 0.0;
                s.H[j * PM_MAXM + j] = (c.dcoef - g) * c.inv;
              }
            }
            update_rows2<S>(V, ld, j, ca, cb, E::coef(c.dcoef), scal_inv<S>(c), zp, Wv,
                            zfinal ? nullptr : V + (size_t)j * ld, Z,
                            zfinal ? PM_UPD_Q_IS_Z : single ? PM_UPD_SCALE : PM_UPD_REORTH, lo, hi);
            PM_MARK(7);
            PM_SYNC_OR_FAIL();                 // the next SpMV reads other CTAs' rows of the candidate
            PM_MARK(8);
            if (tid == 0) c.kcur = j;          // complete columns 0 .. j-1
          }
          if (!c.invariant) {
            // complete the last candidate: v_target and column target-1 (its second
            // projection only when the candidate needs one; otherwise just its norm)
            const int nq = target;
            const int na = c.skipz ? 0 : nq;   // basis vectors the completion pass reads
            gs_vectors += na;
            dots_cta<S>(V, ld, na, Z, lo, hi, true, s);
            PM_BSUM_OR_FAIL(na + 1);
            for (int k = tid; k < nq; k += nth) s.h1[k] = (k < na) ? s.coef[k] : 0.0;
            if (tid < 32) {
              double aa = 0.0;
              for (int k = tid; k < na; k += 32) aa = fma(s.coef[k], s.coef[k], aa);
              aa = pm_warp_sum(aa);
              if (tid == 0) {
                c.fz = s.coef[na];
                c.hn = c.fz - aa;
                c.measure = (aa <= 0.25 * c.fz) ? 0 : 1;
              }
            }
            __syncthreads();
            if (c.measure) {
              for (int k = tid; k < nq; k += nth) ca[k] = E::coef(s.h1[k]);
              __syncthreads();
              update_rows2_cold<S>(V, ld, nq, ca, E::coef(1.0), Z, Wv, V + (size_t)nq * ld, lo, hi);
              __syncthreads();
              dots_cta<S>(V, ld, nq, V + (size_t)nq * ld, lo, hi, true, s);
              PM_BSUM_OR_FAIL(nq + 1);
              if (tid < 32) {
                double aa = 0.0;
                for (int k = tid; k < nq; k += 32) aa = fma(s.coef[k], s.coef[k], aa);
                aa = pm_warp_sum(aa);
                if (tid == 0) {
                  const double q0 = s.coef[nq];
                  c.hn = (aa <= 0.25 * q0) ? q0 - aa : 0.0;
                }
              }
              for (int k = tid; k < nq; k += nth) s.h1[k] += s.coef[k];
              __syncthreads();
            }
            for (int k = tid; k < nq; k += nth) s.H[k * PM_MAXM + nq - 1] += s.h1[k];
            if (tid == 0) {
              c.hn = sqrt(fmax(c.hn, 0.0));
              c.kcur = nq;
              if (c.hn <= c.bd_abs) {          // happy breakdown (R12)
                s.H[nq * PM_MAXM + nq - 1] = 0.0;
                c.hn = 0.0;
                c.invariant = 1;
              } else {
                s.H[nq * PM_MAXM + nq - 1] = c.hn;
                set_inv(c, c.hn);
              }
            }
            __syncthreads();
            if (!c.invariant) {
              for (int k = tid; k < nq; k += nth) ca[k] = E::coef(s.h1[k]);
              __syncthreads();
              update_rows2_cold<S>(V, ld, nq, ca, scal_inv<S>(c), Z, Wv, V + (size_t)nq * ld, lo, hi);
              __syncthreads();
            }
          }
        } else if (j0 < target) {
          for (int j = j0; j < target; ++j) {
            // phase A: write v_j (my rows), y = A v_j
            S* ycur = Y + (size_t)(j & 1) * ld;
            const S* yprev = Y + (size_t)((j + 1) & 1) * ld;
            const C sc = scal_inv<S>(c);   // 1/beta at j = 0, else 1/||y_{j-1}||
            if (j == 0) {
              DLoadAs<S, Team::multi> xl{wp, lo, hi};
              for (int r = lo + tid; r < hi; r += nth) V[r] = E::from_d(wp[r] * c.inv);
              spmv_rows<S>(P.A, xl, ycur, sc, true, lo, hi);
            } else if (j == j0) {
              VecLoad<S, Team::multi> xl{V + (size_t)j * ld, lo, hi};   // v_j normalised at the end of the previous extension
              PM_SPMV_OR_FAIL(spmv_rows<S>(P.A, xl, ycur, sc, false, lo, hi, stg));
            } else {
              VecLoad<S, Team::multi> xl{yprev, lo, hi};
              for (int r = lo + tid; r < hi; r += nth) V[(size_t)j * ld + r] = E::scale(yprev[r], sc);
              PM_SPMV_OR_FAIL(spmv_rows<S>(P.A, xl, ycur, sc, true, lo, hi, stg));
            }
            matvecs += 1;
            kry_steps += 1;
            __syncthreads();
            {
              // Algorithm 2: t_jj = v_j^T y ; y <- y - t_{j,j-1} v_{j-1} - t_jj v_j ; t_{j+1,j} = ||y||
              dots_rows<S>(V + (size_t)j * ld, ld, 1, ycur, lo, hi, false, s);
              PM_BSUM_OR_FAIL(1);
              if (tid == 0) {
                const double tjj = s.coef[0];
                s.H[j * PM_MAXM + j] = tjj;
                if (j > 0) { hc[0] = E::coef(s.H[(j - 1) * PM_MAXM + j]); hc[1] = E::coef(tjj); }
                else hc[0] = E::coef(tjj);
              }
              __syncthreads();
              if (j > 0) update_rows<S>(ycur, V + (size_t)(j - 1) * ld, ld, 2, hc, lo, hi);
              else update_rows<S>(ycur, V, ld, 1, hc, lo, hi);
              __syncthreads();
              dots_rows<S>(ycur, ld, 0, ycur, lo, hi, true, s);
              PM_BSUM_OR_FAIL(1);
              if (tid == 0) {
                const double hn = sqrt(s.coef[0]);
                s.H[(j + 1) * PM_MAXM + j] = hn;
                if (j + 1 < PM_MAXM) s.H[j * PM_MAXM + j + 1] = hn;
                c.hn = hn;
              }
            }
            if (tid == 0) {
              c.kcur = j + 1;
              if (c.hn <= c.bd_abs) {      // happy breakdown (R12): invariant subspace
                s.H[(j + 1) * PM_MAXM + j] = 0.0;
                c.hn = 0.0;
                c.invariant = 1;
              } else {
                set_inv(c, c.hn);
              }
            }
            __syncthreads();
            if (c.invariant) break;
          }
          // normalise the last vector: v_{kcur} = y / ||y||  (my rows)
          if (!c.invariant) {
            const S* yl = Y + (size_t)((c.kcur - 1) & 1) * ld;
            const C sc = scal_inv<S>(c);
            for (int r = lo + tid; r < hi; r += nth) V[(size_t)c.kcur * ld + r] = E::scale(yl[r], sc);
          }
        }
        PM_MARK(9);
        // ---------------- augmented matrix (Eq. hathm + R2) and its exponential (a5)
        // ||H_hat||_1 = max(tau ||H_m||_1, 1): the augmented columns each hold a single 1
        if (tid < 32) {
          const int mu = min(c.m, c.kcur);
          double mx = 0.0;
          for (int jj = tid; jj < mu; jj += 32) {
            double cs = 0.0;
            for (int i = 0; i < mu; ++i) cs += fabs(s.H[i * PM_MAXM + jj]);
            mx = fmax(mx, c.tau_used * cs);
          }
          mx = pm_warp_max(mx);
          if (tid == 0) {
            c.m_used = mu;
            c.hlast = (c.invariant && mu == c.kcur) ? 0.0 : s.H[mu * PM_MAXM + mu - 1];
            c.norm1 = fmax(mx, 1.0);
            c.sq = pm_squarings(c.norm1, prm.theta13);
            // the action form's degree k and steps sd: the fewest products k sd with
            // ||H_hat||_1 / sd <= theta_k, in FP32 with a margin (s rounds up); taken in mode
            // 0 by one-CTA teams where its estimated cycles (k sd products of H_hat with two
            // vectors) are below those of the squaring form's 7 + s matrix products (a
            // multi-CTA team splits those products over its CTAs, the action form cannot)
            c.xv_k = 0;
            c.xv_s = 0;
            if (prm.expm_action == 2 || (prm.expm_action == 0 && prm.expm_taylor && team.size() == 1)) {
              const float nf = (float)c.norm1 * 1.0000005f;
              int bk = 0, bs = 0, best = 1 << 30;
              for (int k = 2; k <= PM_XV_KMAX; ++k) {
                const float q = ceilf(nf * prm.xv_itheta[k]);
                if (!(q <= (float)PM_XV_SMAX)) continue;
                const int ss = max(1, (int)q);
                if (k * ss < best) { best = k * ss; bk = k; bs = ss; }
              }
              bool take = bs > 0 && prm.expm_action == 2;
              if (bs > 0 && prm.expm_action == 0) {
                // cycles, counting FP64 warp instructions per sub-partition at 64 cycles
                // each: a vector step (tridiagonal: 6 per output thread; Hessenberg: two
                // multiply-adds per column of a lane's slice, 8 more) plus 250 for its
                // barrier, against 7 + s products of N^3 multiply-adds at 2 per cycle
                const int N = mu + p + 1;
                const int wsp = pm_warps_per_sp(c.lanczos ? 2 * N : 4 * N);
                const float per = 250.f + 64.f * (float)wsp * (c.lanczos ? 6.f : (float)(2 * ((mu + 3) / 4) + 8));
                const float sqt = fmaxf(0.f, ceilf(log2f(nf / (float)prm.taylor_theta)));
                const float Nf = (float)N;
                take = (float)best * per < (7.f + sqt) * 0.5f * Nf * Nf * Nf;
              }
              if (take) { c.xv_k = bk; c.xv_s = bs; }
            }
          }
        }
        __syncthreads();
        const int mu = c.m_used;
        const int ca = (p >= 1) ? mu + p - 1 : 0;
        const int cb = mu + p;
        if (c.xv_s > 0) {
          expmv_cta(s, prm, c.tau_used, mu, p, ca, cb, c.xv_k, c.xv_s, c.lanczos != 0);
        } else if (!expm_team(team, s, prm, c.norm1, c.tau_used, mu, p, c.sq, w.expm, ca, cb)) {
          if (tid == 0) c.status = PM_ETIMEOUT;
          goto done;
        }
      }
      PM_MARK(11);
      // ---------------- error estimate (a6) and controller (a7): thread 0
      if (tid == 0) {
        const int mu = c.m_used;
        if (c.beta > 0.0) {
          c.expms += 1;
          c.eps = pow(c.tau_used, p + 1) * c.beta * fabs(c.hlast) * fabs(s.phi1[mu - 1]);   // Eq. (errest), R4
        }
        if (!isfinite(c.eps)) {
          c.omega = c.eps;
          c.m_new = NAN;
          c.nonfinite += 1;
          c.rejects += 1;
          c.outcome = PM_ATT_RETRY;
          if (c.nonfinite >= 10) { c.status = PM_ENONFINITE; c.outcome = PM_ATT_FAIL; }
          c.tau = c.tau / 5.0;
          ctl_reset(ctl);
        } else {
          c.nonfinite = 0;
          const double eps = c.eps, tau_used = c.tau_used;
          int m = mu;
          const int m_max = prm.m_max;
          const double omega = c.t_end * eps / (tau_used * c.tol);          // Eq. (taunew)
          c.omega = omega;
          // Algorithm 4
          double q;
          bool qf;
          if (ctl.rejected && ctl.tau_changed) {
            q = (eps > 0.0 && ctl.eps_old > 0.0 && tau_used != ctl.tau_old)
                    ? log(eps / ctl.eps_old) / log(tau_used / ctl.tau_old) - 1.0 : nan("");   // Eq. (6), R7
            if (!isfinite(q)) { q = m / 4.0; qf = false; }
            else { q = fmin(fmax(q, 0.0), (double)m); qf = true; }
          } else if (ctl.rejected && ctl.qf) {
            q = ctl.q; qf = true;
          } else {
            q = m / 4.0; qf = false;
          }
          ctl.q = q; ctl.qf = qf;
          const double tau_new = (omega > 0.0) ? tau_used * pow(prm.gamma / omega, 1.0 / (q + 1.0)) : INFINITY;  // Eq. (2)
          double kap;
          bool kf;
          if (ctl.rejected && ctl.m_changed) {
            kap = (eps > 0.0 && ctl.eps_old > 0.0 && m != ctl.m_old)
                      ? pow(eps / ctl.eps_old, 1.0 / (double)(ctl.m_old - m)) : nan("");       // Eq. (7)
            if (!isfinite(kap) || kap <= 1.0) { kap = 2.0; kf = false; }
            else kf = true;
          } else if (ctl.rejected && ctl.kf) {
            kap = ctl.kap; kf = true;
          } else {
            kap = 2.0; kf = false;
          }
          ctl.kap = kap; ctl.kf = kf;
          const double m_new_real = (omega > 0.0) ? m + log(omega / prm.gamma) / log(kap) : -INFINITY;   // Eq. (3)
          c.m_new = m_new_real;
          int m_new;
          if (isfinite(m_new_real)) m_new = (int)fmin(fmax(ceil(m_new_real), 1.0), (double)m_max);
          else m_new = (m_new_real < 0.0) ? 1 : m_max;
          // cost model, Eqs. (4), (5), (8) with R13-R15
          const double Mf = 44.0 / 3.0 + 2.0 * c.sq;     // c.sq = the squarings of this attempt's exponential
          const double t_left = c.t_end - c.t;
          const double nnzA = (double)P.A.nnz;
          auto C1 = [&](double mm) {
            const double e3 = Mf * (mm + p + 1) * (mm + p + 1) * (mm + p + 1);
            if (c.symmetric) return (mm + p) * nnzA + 3.0 * (mm + p) * n + e3;
            return (mm + p) * nnzA + (mm * mm + 3 * p + 2) * (double)n + e3;
          };
          const double c_tau = ceil(t_left / tau_new) * C1((double)m);
          const double c_m = ceil(t_left / tau_used) * C1((double)m_new);
          // m within a factor 4/3 of the current one and within [1, m_max]; when that
          // leaves m as it is (m at a bound), only a change of tau can alter the attempt.
          // The fixed-dimension variant (phip) always changes tau.
          const int m_cand = min(min(max(max(m_new, (3 * m) / 4), 1), (4 * m + 2) / 3), m_max);
          bool branch_tau;
          if (c_tau < c_m || m_cand == m || prm.fixed_m) {
            c.tau = fmin(fmin(fmax(tau_new, tau_used / 5.0), 2.0 * tau_used), t_left);
            branch_tau = true;
          } else {
            m = m_cand;
            branch_tau = false;
          }
          c.m = m;
          if (omega <= prm.delta) {
            c.outcome = PM_ATT_ACCEPT;
            // coefficients of Eq. (step) (a8) with F of Eq. (phipapprox2): the corrector's
            // here, the mu others (tp beta phi0[i]) by the whole CTA in the accept block
            const double tp = pow(tau_used, p);
            c.tp = tp;
            int nvv = 0;
            if (c.beta > 0.0) {
              s.ucoef[mu] = (c.hlast != 0.0) ? tp * tau_used * c.beta * c.hlast * s.phi1[mu - 1] : 0.0;
              nvv = (s.ucoef[mu] != 0.0) ? mu + 1 : mu;
            }
            c.nvv = nvv;
            double d = 1.0;
            for (int jj = 0; jj < p; ++jj) {
              s.ucoef[PM_NSLOT + jj] = d;
              d = d * tau_used / (double)(jj + 1);
            }
          } else {
            c.outcome = PM_ATT_REJECT;
            c.rejects += 1;
            if (c.rejects > prm.max_rejects) { c.status = PM_EMAXSTEPS; c.outcome = PM_ATT_FAIL; }
            ctl.rejected = true;
            ctl.tau_changed = branch_tau;
            ctl.m_changed = !branch_tau;
            ctl.eps_old = eps;
            ctl.tau_old = tau_used;
            ctl.m_old = mu;
          }
        }
        // attempt record (G15): written by one CTA of the team
        c.trace_idx = -1;
        if (prm.trace != nullptr && team.rank() == 0) {
          const unsigned long long idx = atomicAdd(prm.trace_count, 1ull);
          if ((long long)idx < prm.trace_cap) {
            TraceRec& tr = prm.trace[idx];
            tr.problem = P.id;
            tr.step = (int)c.steps;
            tr.attempt = c.attempt;
            tr.accepted = (c.outcome == PM_ATT_ACCEPT) ? 1 : 0;
            tr.m_req = c.m_req;
            tr.m_used = mu;
            tr.p = p;
            tr.n = n;
            tr.t = c.t;
            tr.t_end = c.t_end;
            tr.tau = c.tau_used;
            tr.eps = c.eps;
            tr.omega = c.omega;
            tr.norm_a = c.normA;
            tr.tol = c.tol;
            tr.m_new = c.m_new;
            tr.source = c.source;
            tr.rejects_prev = c.prev_rejects;
            c.trace_idx = (long long)idx;
          }
        }
        c.attempt += 1;
        c.source = 0;
        if (c.outcome != PM_ATT_ACCEPT) c.step_rejects += 1;
      }
      __syncthreads();
      PM_MARK(12);
      if (c.outcome == PM_ATT_FAIL) goto done;
      if (c.outcome != PM_ATT_ACCEPT) continue;
      {
        // ---------------- accept: u_{k+1} = F + sum_{j<p} tau^j/j! w_j  (Eq. step)
        // FP32 basis: F carries a relative rounding error of about u32 and cancels
        // against the polynomial part; the candidate goes to a spare vector so that
        // ||F|| / ||u_new|| can be bounded before it replaces u.
        const bool guard = (E::kind == 1) && p >= 2 && c.beta > 0.0;
        if (c.beta > 0.0) {
          // the coefficients tp beta phi0[i] of F, i < mu, in FP64, FP32 and float pairs
          const int mu = c.m_used, nvv = c.nvv;
          const double tb = c.tp * c.beta;
          for (int i = tid; i < nvv; i += nth) {
            const double v = (i < mu) ? tb * s.phi0[i] : s.ucoef[i];
            s.ucoef[i] = v;
            s.ucf[i] = (float)v;
            s.ucd[i] = df_from_d(v);
          }
          if (guard && tid < 32) {               // ||F|| without the corrector (FP32 guard)
            double fn = 0.0;
            for (int i = tid; i < mu; i += 32) fn = fma(s.phi0[i], s.phi0[i], fn);
            fn = pm_warp_sum(fn);
            if (tid == 0) c.fnorm = tb * sqrt(fn);
          }
          __syncthreads();
        }
        double* udst = guard ? ualt : u;
        const double un = accept_rows<S>(V, ld, s, c.nvv, p, u, W, udst, guard, lo, hi);
        if (guard) {
          const double v[1] = {un};
          block_sum(s, v, 1, s.coef);
          PM_SUM_OR_FAIL(1);
          if (tid == 0) {
            const double unew = sqrt(s.coef[0]);
            c.outcome = PM_ATT_ACCEPT;
            if (c.fnorm > PM_F32_AMP * unew && unew > 0.0) {
              c.rejects += 1;
              c.outcome = PM_ATT_RETRY;
              if (c.rejects > prm.max_rejects) { c.status = PM_EMAXSTEPS; c.outcome = PM_ATT_FAIL; }
              c.tau = c.tau_used * pow(0.5 * PM_F32_AMP * unew / c.fnorm, 1.0 / (double)(p - 1));
              c.m = c.m_used;
              c.step_rejects += 1;
              if (c.trace_idx >= 0) prm.trace[c.trace_idx].accepted = 0;
              ctl_reset(ctl);
            }
          }
          __syncthreads();
          if (c.outcome == PM_ATT_FAIL) goto done;
          if (c.outcome == PM_ATT_RETRY) continue;
          double* t2 = u; u = ualt; ualt = t2;
        }
        if (tid == 0) {
          c.steps += 1;
          c.err_sum += c.eps;
          if (c.steps > prm.max_steps) c.status = PM_EMAXSTEPS;
          const bool last = c.tau_used >= c.t_end - c.t;
          c.t = last ? c.t_end : c.t + c.tau_used;
          if (c.t < c.t_end) c.tau = fmin(c.tau, c.t_end - c.t);
          c.last_tau = c.tau_used;
          c.last_m = c.m_used;
          c.last_omega = c.omega;
          c.prev_rejects = c.step_rejects;
          c.step_rejects = 0;
        }
        PM_SYNC_OR_FAIL();    // u complete before the next SpMV reads neighbours; c visible
        PM_MARK(13);
        if (c.status != PM_OK) goto done;
        break;
      }
    }
  }
  if (u != P.u) {
    for (int r = lo + tid; r < hi; r += nth) P.u[r] = u[r];
  }
done:
  __syncthreads();
  if (team.rank() == 0 && threadIdx.x == 0) {
    res.status = c.status;
    res.steps = c.steps;
    res.rejects = c.rejects;
    res.matvecs = matvecs;
    res.expms = c.expms;
    res.kry_steps = kry_steps;
    res.gs_vectors = gs_vectors;
    res.reorth_vectors = reorth_vectors;
    res.err_est_sum = c.err_sum;
    res.normA = c.normA;
    res.normb = c.normb;
    res.symmetric = c.symmetric;
    res.last_tau = c.last_tau;
    res.last_m = c.last_m;
  }
#undef PM_SYNC_OR_FAIL
#undef PM_SUM_OR_FAIL
#undef PM_BSUM_OR_FAIL
#undef PM_MAX_OR_FAIL
#undef PM_SPMV_OR_FAIL
}
