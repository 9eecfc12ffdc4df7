// Shared device-side definitions of the phipm engine: problem descriptors,
// teams (who cooperates on one problem), bounded barriers and reductions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "phipm_elem.cuh"

#define PM_MAXM 64
#define PM_MAXP 8
#define PM_NA (PM_MAXM + PM_MAXP + 1)   // largest augmented matrix, Eq. (hathm) + 1
#define PM_NA2 (PM_NA * PM_NA)
#define PM_XV_KMAX 40                   // largest Taylor degree of the action form of exp(H_hat)
#define PM_XV_SMAX 64                   // largest number of its steps
#define PM_THREADS 512
#define PM_WARPS (PM_THREADS / 32)
#define PM_NSLOT 66                     // partial sums per reduction (j+1 <= 65, +1)

// status codes (mirror phipm_status in include/phipm.h)
#define PM_OK 0
#define PM_EINVAL 1
#define PM_ENONFINITE 4
#define PM_EMAXSTEPS 5
#define PM_ETIMEOUT 6
#define PM_EBOUNDS 7
#define PM_ENOTRUN 9      // batched: the launch stopped before a team took this problem

struct DevOp {
  int kind;          // 0 CSR, 1 stencil, 2 built-in function (matrix-free)
  int n;
  long long nnz;     // structural nonzeros (cost model, Eq. 4)
  const int* rowptr;
  const int* colind;
  const double* val;     // CSR values, FP64 (caller's)
  const float* valf;     // CSR values, FP32 copy (workspace; FP32 basis)
  const df32* val2;      // CSR values as float pairs (workspace; float-pair basis)
  int ndim, nx, ny, nz;
  double cc, cm[3], cp[3];
  df32 cc2, cm2[3], cp2[3];   // stencil coefficients as float pairs (hi alone for FP32)
  int quad;                   // stencil with nx a multiple of 4: rows taken four at a time
  int fn;                     // kind 2 (matrix-free): built-in function id
  unsigned long long mnx, mny;   // multiply-high divisors by nx and ny (pm_udiv; 0 for 1)
  const double* fld[4];       // kind 2: the function's fields (device arrays, may be null)
  double fsc[6];              // kind 2: the function's scalars
  double fnorm;               // kind 2: caller's bound of ||A||_inf (<= 0: computed)
};

// x / d for 0 <= x < 2^32 as the high word of x * m, m = floor((2^64 - 1) / d) + 1 for
// d >= 2: with m = 2^64 / d + e, 0 <= e < 1, x m / 2^64 = x / d + x e / 2^64 and
// x e / 2^64 < 2^-32 < 1 / d, which never reaches the next integer.  m = 0 encodes d = 1.
__device__ __forceinline__ unsigned pm_udiv(unsigned x, unsigned long long m) {
  return m ? (unsigned)__umul64hi((unsigned long long)x, m) : x;
}

// One attempt record; the same layout as phipm_trace_record in include/phipm.h.
struct TraceRec {
  int problem, step, attempt, accepted, m_req, m_used, p, n;
  double t, t_end, tau, eps, omega, norm_a, tol, m_new;
  int source, rejects_prev;
};

struct DevParams {
  double gamma, delta, theta13, breakdown_tol;
  int m_init, m_max;
  int fixed_m;           // 1: the m branch of Algorithm 3 is never taken (phip)
  int mlp_every_step;    // 1: the learned controller proposes the first attempt of every step
  long long max_steps, max_rejects;
  long long timeout_cycles;
  int stencil_stage;     // 1: stencil products stage their rows through the TMA engine
  int pad1;
  double pade_b[14];     // degree-13 Pade coefficients, computed on the host from their closed form
  double taylor_c[19];   // 1 / k!, k <= 18 (the Taylor exponential of multi-CTA teams)
  double taylor_theta;   // largest ||X||_1 for which the degree-18 Taylor truncation term is below 2^-53 e^-||X||
  int expm_taylor;       // 1: the exponential by the degree-18 Taylor form; 0: the degree-13 Pade form
  int expm_action;       // 0: phi columns by the action form where it is estimated cheaper; 1: never; 2: always
  float xv_itheta[PM_XV_KMAX + 1];   // 1 / theta_k of the action form's degree-k Taylor polynomial
  double inv_int[PM_XV_SMAX + 1];    // 1 / j
  double xv_invfact[PM_XV_KMAX + 1]; // 1 / j!
  const float* mlp;      // learned-controller blob (device), or null
  TraceRec* trace;       // attempt records (device), or null
  unsigned long long* trace_count;
  long long trace_cap;
#ifdef PM_PHASE_PROBE
  unsigned long long* phase_ticks;   // probe build: clock cycles per solver phase (PM_NPHASE)
#endif
};

// Phase timers, compiled in only by a probe build (-DPM_PHASE_PROBE): thread 0 of the
// team's first CTA adds the clock cycles since its previous mark to ticks[k].
#define PM_NPHASE 16
#ifdef PM_PHASE_PROBE
#define PM_MARK(k)                                                              \
  do {                                                                          \
    if (prm.phase_ticks && team.rank() == 0 && threadIdx.x == 0) {              \
      const long long pm_t_now = clock64();                                     \
      prm.phase_ticks[k] += (unsigned long long)(pm_t_now - pm_t_last);         \
      pm_t_last = pm_t_now;                                                     \
    }                                                                           \
  } while (0)
#else
#define PM_MARK(k) do { } while (0)
#endif

struct DevProblem {
  DevOp A;
  int id;                // index of the problem in the call (traces)
  int p;
  int symm;              // -1 detect, 0, 1
  double t_end, tol;
  const double* b[PM_MAXP + 1];
  double* u;             // current solution u(t_k) = w_0, FP64, caller's buffer
  // workspace (device)
  void* V;               // (m_max+1) basis vectors of length ld, element type S
  double* W;             // w_1..w_p and one spare vector, FP64, length ld each
  void* Y;               // 2 buffers of length ld (unnormalised Krylov vector), type S
  long long ld;
};

struct DevResult {
  int status;
  int symmetric;
  long long steps, rejects, matvecs, expms;
  long long kry_steps, gs_vectors, reorth_vectors;
  double err_est_sum;
  double normA, normb;
  double last_tau;
  int last_m;
  int pad;
};

// ------------------------------------------------------------------------------------
// bounded waits
// ------------------------------------------------------------------------------------
// Barrier over the G CTAs of a cooperative launch on one 64-bit arrival counter
// that the host zeroes before the launch and that only grows: the k-th barrier is
// passed once it reaches k G.  Each CTA counts its own barriers (gen, thread 0),
// so arriving takes one acquire-release atomic and waiting one acquire load per
// poll, with no generation word and no separate fences.  The spin is bounded by
// timeout cycles (the clock is read at every poll); on expiry the error word is set
// and every later barrier returns within 16 polls (err is checked every 16 polls).
__device__ __forceinline__ unsigned long long pm_atom_add_acq_rel(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long pm_ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ bool pm_grid_barrier(unsigned long long* cnt, int G, int* err, long long timeout,
                                                unsigned long long& gen) {
  __syncthreads();
  __shared__ int s_fail;
  if (threadIdx.x == 0) {
    s_fail = 0;
    gen += 1;
    const unsigned long long target = gen * (unsigned long long)G;
    const unsigned long long prev = pm_atom_add_acq_rel(cnt, 1ull);
    if (prev + 1 < target) {
      const long long t0 = clock64();
      for (unsigned it = 1; pm_ld_acquire64(cnt) < target; ++it) {
        if (clock64() - t0 > timeout) { atomicCAS(err, 0, PM_ETIMEOUT); s_fail = 1; break; }
        if ((it & 15u) == 0 && *((volatile int*)err) != 0) { s_fail = 1; break; }
      }
    }
  }
  __syncthreads();
  return s_fail == 0;
}

// A team is the set of CTAs that work on one problem.
struct GridTeam {
  unsigned long long* bar;               // arrival counter, zero at launch
  int* err;
  long long timeout;
  mutable unsigned long long gen = 0;    // barriers passed (used by thread 0)
  __device__ int rank() const { return blockIdx.x; }
  __device__ int size() const { return gridDim.x; }
  __device__ bool sync() const { return pm_grid_barrier(bar, gridDim.x, err, timeout, gen); }
  static constexpr bool multi = true;
};

struct CtaTeam {
  __device__ int rank() const { return 0; }
  __device__ int size() const { return 1; }
  __device__ bool sync() const { __syncthreads(); return true; }
  static constexpr bool multi = false;
};

// Barrier over the K CTAs of a thread-block cluster: the same counting protocol as
// pm_grid_barrier on a 64-bit counter in rank 0's shared memory, reached through
// distributed shared memory with cluster-scope acquire / release (no L2 round trip),
// bounded by timeout cycles and the launch's error word.
__device__ __forceinline__ unsigned long long pm_atom_add_cluster(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.cluster.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long pm_ld_acquire_cluster(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.cluster.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ bool pm_cluster_barrier(unsigned long long* cnt, int K, int* err, long long timeout,
                                                   unsigned long long& gen) {
  __syncthreads();
  __shared__ int s_cfail;
  if (threadIdx.x == 0) {
    s_cfail = 0;
    gen += 1;
    const unsigned long long target = gen * (unsigned long long)K;
    const unsigned long long prev = pm_atom_add_cluster(cnt, 1ull);
    if (prev + 1 < target) {
      const long long t0 = clock64();
      for (unsigned it = 1; pm_ld_acquire_cluster(cnt) < target; ++it) {
        if (clock64() - t0 > timeout) { atomicCAS(err, 0, PM_ETIMEOUT); s_cfail = 1; break; }
        if ((it & 15u) == 0 && *((volatile int*)err) != 0) { s_cfail = 1; break; }
      }
    }
  }
  __syncthreads();
  return s_cfail == 0;
}

// A team of the K CTAs of one cluster (batched form: one problem per cluster).
struct ClusterTeam {
  unsigned long long* bar;               // rank 0's arrival counter (distributed shared memory)
  int* err;
  long long timeout;
  int r, k;
  mutable unsigned long long gen = 0;
  __device__ int rank() const { return r; }
  __device__ int size() const { return k; }
  __device__ bool sync() const { return pm_cluster_barrier(bar, k, err, timeout, gen); }
  static constexpr bool multi = true;
};

// ------------------------------------------------------------------------------------
// reductions
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double pm_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double pm_warp_max(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Rows owned by CTA r of a team of G CTAs for a vector of length n.
__device__ __forceinline__ void pm_rows(int n, int r, int G, int& lo, int& hi) {
  long long chunk = ((long long)n + G - 1) / G;
  chunk = (chunk + 63) & ~63ll;
  long long a = chunk * r, b = a + chunk;
  lo = (int)(a < n ? a : n);
  hi = (int)(b < n ? b : n);
}
