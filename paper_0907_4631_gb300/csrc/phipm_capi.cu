// Host side of the C ABI declared in include/phipm.h.  The solver kernels that
// run the device engine (phipm_engine.cuh) live in phipm_kernels.cu and are
// reached through phipm_launch.h:
//   k_solve_grid     one problem, every CTA of a cooperative launch;
//   k_solve_queue    a persistent CTA per slot that pulls problems from an
//                    atomic queue, largest first (batched form and small
//                    single problems);
//   k_solve_cluster  the same queue served by thread-block clusters of K CTAs.
// This file holds the small kernels (value conversion, the controller network's
// training) and the allocation-free solve.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <map>
#include <vector>

#include "phipm.h"
#include "phipm_launch.h"
#include "phipm_mlp_train.cuh"

// ------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------
// CSR values converted for the FP32 basis (valf) or the float-pair basis (val2);
// blockIdx.y selects the problem, blockIdx.x strides over its values.
__global__ void k_convert_values(const DevProblem* probs, int count, int mode) {
  const int id = blockIdx.y;
  if (id >= count) return;
  const DevOp& A = probs[id].A;
  if (A.kind != 0) return;
  const long long nnz = A.nnz;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x) {
    const double v = A.val[k];
    if (mode == 1) {
      ((float*)A.valf)[k] = (float)v;
    } else {
      df32 d;
      d.hi = __double2float_rn(v);
      d.lo = __double2float_rn(v - (double)d.hi);
      ((df32*)A.val2)[k] = d;
    }
  }
}

// ------------------------------------------------------------------------------------
// handle
// ------------------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  bool ensure(size_t bytes) {
    if (bytes <= cap) return true;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = std::max(bytes, (size_t)256);
    if (cudaMalloc(&p, want) != cudaSuccess) { p = nullptr; return false; }
    cap = want;
    return true;
  }
  void release() { if (p) cudaFree(p); p = nullptr; cap = 0; }
};

struct HostBuf {
  void* p = nullptr;
  size_t cap = 0;
  bool ensure(size_t bytes) {
    if (bytes <= cap) return true;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    if (cudaMallocHost(&p, std::max(bytes, (size_t)256)) != cudaSuccess) { p = nullptr; return false; }
    cap = std::max(bytes, (size_t)256);
    return true;
  }
  void release() { if (p) cudaFreeHost(p); p = nullptr; cap = 0; }
};

struct phipm_handle {
  int device = 0;
  int num_sms = 0;
  phipm_params params;
  std::string err;
  DevBuf ws;          // V, W, Y of the grid solve / queue slots
  DevBuf sync;        // barrier words + error flag + queue counter
  DevBuf partials, expm, conv, res, probs, order;
  DevBuf h_rowptr, h_colind, h_vals, h_b, h_u;   // device staging for phipm_solve_host
  HostBuf res_host, probs_host;
  int grid_blocks[3] = {0, 0, 0};    // cooperative grid size per precision
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // around the solver kernel
  DevBuf trace;                      // attempt records
  long long trace_cap = 0;
  long long trace_last = 0;          // records produced by the last solve call
  HostBuf trace_count_host;
  DevBuf mlp_blob, mlp_part;         // learned controller weights; training partials
  bool has_mlp = false;
  // batched form: the launch sequence captured once as a CUDA graph, replayed on gstream
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<unsigned char> gkey;
  // team size per size class (precision, operator kind, floor(log2 n)), from the
  // autotuner or a loaded cache; team_force overrides (0 = use the table / default)
  std::map<int, std::pair<int, double>> tuned;
  int team_force = 0;
  int last_batch_team = 0;           // cluster size K of the last batched launch
  // cluster size per batch class (precision, floor(log2 count), floor(log2 largest n)),
  // from phipm_autotune_batched or a loaded cache; batch_req forces K while the tuner runs
  std::map<int, std::pair<int, double>> tuned_batch;
  int batch_req = 0;
#ifdef PM_PHASE_PROBE
  DevBuf phase;                      // probe build: clock cycles per solver phase
#endif
};

static phipm_status fail(phipm_handle* h, phipm_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}
static phipm_status cuda_fail(phipm_handle* h, cudaError_t e, const char* what) {
  return fail(h, PHIPM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

extern "C" void phipm_default_params(phipm_params* o) {
  if (!o) return;
  o->gamma = 0.8;
  o->delta = 1.2;
  o->m_init = 10;
  o->m_max = 64;
  o->theta13 = 5.37;
  o->breakdown_tol = 1e-12;
  o->max_steps = 1000000;
  o->max_rejects = 1000000;
  o->precision = PHIPM_F64;
  o->controller = 0;
  o->timeout_cycles = 20000000000ll;   // about 10 s at 2 GHz
  o->stencil_stage = 0;
  o->expm_pade = 0;
  o->expm_action = 0;
}

static bool params_ok(const phipm_params& p, std::string& why) {
  if (!(p.gamma > 0 && p.gamma < p.delta)) { why = "need 0 < gamma < delta"; return false; }
  if (p.m_max < 1 || p.m_max > PHIPM_M_MAX) { why = "m_max out of [1, 64]"; return false; }
  if (p.m_init < 1 || p.m_init > p.m_max) { why = "m_init out of [1, m_max]"; return false; }
  if (!(p.theta13 > 0)) { why = "theta13 must be positive"; return false; }
  if (!(p.breakdown_tol >= 0)) { why = "breakdown_tol must be >= 0"; return false; }
  if (p.precision != PHIPM_F64 && p.precision != PHIPM_F32_MIXED && p.precision != PHIPM_F64_PAIR) {
    why = "unknown precision";
    return false;
  }
  if (p.controller < 0 || p.controller > 3) { why = "unknown controller"; return false; }
  if (p.timeout_cycles <= 0) { why = "timeout_cycles must be positive"; return false; }
  if (p.stencil_stage != 0 && p.stencil_stage != 1) { why = "stencil_stage must be 0 or 1"; return false; }
  if (p.expm_pade != 0 && p.expm_pade != 1) { why = "expm_pade must be 0 or 1"; return false; }
  if (p.expm_action < 0 || p.expm_action > 2) { why = "expm_action must be 0, 1 or 2"; return false; }
  return true;
}

template <class S>
static cudaError_t setup_kernels(int smem) {
  cudaError_t e = pm_grid_setup<S>(smem);
  if (e != cudaSuccess) return e;
  e = pm_cluster_setup<S>(smem);
  if (e != cudaSuccess) return e;
  return pm_queue_setup<S>(smem);
}

// Co-resident clusters of K CTAs for the precision (0 when the GPU cannot hold one).
static int cluster_capacity(int precision, int K) {
  const int smem = (int)sizeof(PmShared);
  if (precision == PHIPM_F32_MIXED) return pm_cluster_capacity<float>(K, smem);
  if (precision == PHIPM_F64_PAIR) return pm_cluster_capacity<df32>(K, smem);
  return pm_cluster_capacity<double>(K, smem);
}

static cudaError_t launch_cluster_any(int precision, int K, int clusters, cudaStream_t stream, const DevProblem* probs,
                                      const int* order, int count, const DevParams& prm, DevResult* res,
                                      unsigned char* slots, const SlotLayout& lay, int* queue, double* partials,
                                      int* err) {
  if (precision == PHIPM_F32_MIXED)
    return pm_cluster_launch<float>(K, clusters, stream, probs, order, count, prm, res, slots, lay, queue, partials, err);
  if (precision == PHIPM_F64_PAIR)
    return pm_cluster_launch<df32>(K, clusters, stream, probs, order, count, prm, res, slots, lay, queue, partials, err);
  return pm_cluster_launch<double>(K, clusters, stream, probs, order, count, prm, res, slots, lay, queue, partials, err);
}

extern "C" phipm_status phipm_create(phipm_handle** out, const phipm_params* params) {
  if (!out) return PHIPM_EINVAL;
  *out = nullptr;
  phipm_handle* h = new phipm_handle();
  phipm_default_params(&h->params);
  if (params) {
    std::string why;
    if (!params_ok(*params, why)) { delete h; return PHIPM_EINVAL; }
    h->params = *params;
  }
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) { delete h; return PHIPM_ECUDA; }
  e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) { delete h; return PHIPM_ECUDA; }
  const int smem = (int)sizeof(PmShared);
  if (setup_kernels<double>(smem) != cudaSuccess || setup_kernels<float>(smem) != cudaSuccess ||
      setup_kernels<df32>(smem) != cudaSuccess) {
    delete h;
    return PHIPM_ECUDA;
  }
  const int occ[3] = {pm_grid_occupancy<double>(smem), pm_grid_occupancy<float>(smem), pm_grid_occupancy<df32>(smem)};
  for (int i = 0; i < 3; ++i) h->grid_blocks[i] = std::max(1, occ[i]) * h->num_sms;
  if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem)) !=
      cudaSuccess) {
    delete h;
    return PHIPM_ECUDA;
  }
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->gev, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return PHIPM_ECUDA;
  }
  if (!h->sync.ensure(4096) || !h->res.ensure(sizeof(DevResult)) || !h->res_host.ensure(sizeof(DevResult)) ||
      !h->expm.ensure(PM_EXPM_DOUBLES * sizeof(double)) || !h->trace_count_host.ensure(sizeof(unsigned long long))) {
    delete h;
    return PHIPM_ENOMEM;
  }
  *out = h;
  return PHIPM_OK;
}

extern "C" void phipm_destroy(phipm_handle* h) {
  if (!h) return;
  DevBuf* bufs[] = {&h->ws, &h->sync, &h->partials, &h->expm, &h->conv, &h->res, &h->probs,
                    &h->order, &h->h_rowptr, &h->h_colind, &h->h_vals, &h->h_b, &h->h_u,
                    &h->trace, &h->mlp_blob, &h->mlp_part};
  for (DevBuf* b : bufs) b->release();
  h->res_host.release();
  h->probs_host.release();
  h->trace_count_host.release();
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->gev) cudaEventDestroy(h->gev);
  if (h->gstream) cudaStreamDestroy(h->gstream);
  delete h;
}

extern "C" const char* phipm_last_error(const phipm_handle* h) { return h ? h->err.c_str() : "null handle"; }

extern "C" phipm_status phipm_set_params(phipm_handle* h, const phipm_params* params) {
  if (!h || !params) return PHIPM_EINVAL;
  std::string why;
  if (!params_ok(*params, why)) return fail(h, PHIPM_EINVAL, why);
  h->params = *params;
  return PHIPM_OK;
}

// ------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------
// theta(deg): the largest theta with sum_{k>deg} theta^k / k! <= 2^-53 e^-theta (the
// truncated Taylor tail relative to the smallest possible |exp|), by bisection; for the
// degree-18 squaring form and, as 1 / theta_k rounded up in FP32 (so that the steps
// s = ceil(||H_hat|| / theta_k), formed in FP32 with a margin, never fall short), for the
// action form's degrees k <= PM_XV_KMAX.  Computed once per process (every solve call
// builds its parameter block).
struct ThetaTables {
  double theta18;
  float itheta[PM_XV_KMAX + 1];
  double inv_int[PM_XV_SMAX + 1];
  double invfact[PM_XV_KMAX + 1];
};
static double theta_of(int deg) {
  auto tail = [deg](double th) {
    double term = 1.0, sum = 0.0;
    for (int k = 1; k <= deg + 160; ++k) {
      term *= th / (double)k;
      if (k > deg) sum += term;
    }
    return sum;
  };
  double lo = 0.0, hi = (double)deg + 1.0;
  for (int it = 0; it < 100; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (tail(mid) <= std::ldexp(1.0, -53) * std::exp(-mid)) lo = mid; else hi = mid;
  }
  return lo;
}
static const ThetaTables& theta_tables() {
  static const ThetaTables t = [] {
    ThetaTables r;
    r.theta18 = theta_of(18);
    r.itheta[0] = 0.f;
    for (int k = 1; k <= PM_XV_KMAX; ++k) r.itheta[k] = std::nextafter((float)(1.0 / theta_of(k)), INFINITY);
    r.inv_int[0] = 0.0;
    for (int j = 1; j <= PM_XV_SMAX; ++j) r.inv_int[j] = 1.0 / (double)j;
    double f = 1.0;
    for (int j = 0; j <= PM_XV_KMAX; ++j) {
      r.invfact[j] = f;
      f /= (double)(j + 1);
    }
    return r;
  }();
  return t;
}

static DevParams make_params(const phipm_params& p) {
  DevParams d;
  memset(&d, 0, sizeof(d));      // padding too: the batched form keys its captured graph on these bytes
  d.gamma = p.gamma;
  d.delta = p.delta;
  d.theta13 = p.theta13;
  d.breakdown_tol = p.breakdown_tol;
  d.m_init = p.m_init;
  d.m_max = p.m_max;
  d.fixed_m = (p.controller == PHIPM_CTRL_FIXED_M) ? 1 : 0;
  d.mlp_every_step = (p.controller == PHIPM_CTRL_LEARNED_STEPS) ? 1 : 0;
  d.stencil_stage = p.stencil_stage;
  d.max_steps = p.max_steps;
  d.max_rejects = p.max_rejects;
  d.timeout_cycles = p.timeout_cycles;
  d.mlp = nullptr;
  d.trace = nullptr;
  d.trace_count = nullptr;
  d.trace_cap = 0;
#ifdef PM_PHASE_PROBE
  d.phase_ticks = nullptr;
#endif
  // [13/13] Pade coefficients of e^x, c_j = (26-j)! 13! / (26! j! (13-j)!), from their closed form
  double c = 1.0;
  for (int j = 0; j <= 13; ++j) {
    d.pade_b[j] = c;
    c = c * (double)(13 - j) / ((double)(26 - j) * (double)(j + 1));
  }
  // degree-18 Taylor form: 1/k!; its theta and the action form's from theta_tables()
  double f = 1.0;
  for (int k = 0; k <= 18; ++k) {
    d.taylor_c[k] = f;
    f /= (double)(k + 1);
  }
  const ThetaTables& tt = theta_tables();
  d.taylor_theta = tt.theta18;
  d.expm_taylor = p.expm_pade ? 0 : 1;
  d.expm_action = p.expm_action;
  for (int k = 0; k <= PM_XV_KMAX; ++k) d.xv_itheta[k] = tt.itheta[k];
  for (int j = 0; j <= PM_XV_SMAX; ++j) d.inv_int[j] = tt.inv_int[j];
  for (int j = 0; j <= PM_XV_KMAX; ++j) d.xv_invfact[j] = tt.invfact[j];
  return d;
}

static phipm_status check_operator(phipm_handle* h, const phipm_operator* A, long long& nnz_model) {
  if (!A) return fail(h, PHIPM_EINVAL, "operator is NULL");
  if (A->kind == PHIPM_OP_CSR) {
    if (A->csr.n < 0 || A->csr.nnz < 0) return fail(h, PHIPM_EINVAL, "negative CSR sizes");
    if (A->csr.n > 0 && (!A->csr.rowptr || (A->csr.nnz > 0 && (!A->csr.colind || !A->csr.values))))
      return fail(h, PHIPM_EINVAL, "CSR arrays missing");
    nnz_model = A->csr.nnz;
    return PHIPM_OK;
  }
  if (A->kind == PHIPM_OP_STENCIL) {
    const phipm_stencil& st = A->st;
    if (st.ndim < 1 || st.ndim > 3) return fail(h, PHIPM_EINVAL, "stencil ndim must be 1, 2 or 3");
    if (st.nx < 1 || st.ny < 1 || st.nz < 1) return fail(h, PHIPM_EINVAL, "stencil extents must be >= 1");
    if ((st.ndim < 2 && st.ny != 1) || (st.ndim < 3 && st.nz != 1)) return fail(h, PHIPM_EINVAL, "unused stencil extents must be 1");
    const long long n = (long long)st.nx * st.ny * st.nz;
    if (n > 0x7fffffffll) return fail(h, PHIPM_EINVAL, "stencil too large for int32 indexing");
    const long long dims[3] = {st.nx, st.ny, st.nz};
    nnz_model = n;
    for (int d = 0; d < st.ndim; ++d) nnz_model += 2 * (n / dims[d]) * (dims[d] - 1);
    return PHIPM_OK;
  }
  if (A->kind == PHIPM_OP_FUNCTION) {
    const phipm_function& f = A->fn;
    if (f.fn != PHIPM_FN_VARCOEF_CONVDIFF) return fail(h, PHIPM_EINVAL, "unknown built-in function");
    if (f.ndim < 1 || f.ndim > 3) return fail(h, PHIPM_EINVAL, "function ndim must be 1, 2 or 3");
    if (f.nx < 1 || f.ny < 1 || f.nz < 1) return fail(h, PHIPM_EINVAL, "function grid extents must be >= 1");
    if ((f.ndim < 2 && f.ny != 1) || (f.ndim < 3 && f.nz != 1)) return fail(h, PHIPM_EINVAL, "unused extents must be 1");
    const long long n = (long long)f.nx * f.ny * f.nz;
    if (n > 0x7fffffffll) return fail(h, PHIPM_EINVAL, "function grid too large for int32 indexing");
    if (!f.field[0]) return fail(h, PHIPM_EINVAL, "the diffusivity field is NULL");
    for (int d = 0; d < 6; ++d)
      if (!std::isfinite(f.scal[d])) return fail(h, PHIPM_EINVAL, "function scalars must be finite");
    if (!std::isfinite(f.norm_inf)) return fail(h, PHIPM_EINVAL, "norm_inf must be finite");
    if (f.cost > 0) {
      nnz_model = f.cost;
    } else {
      const long long dims[3] = {f.nx, f.ny, f.nz};
      nnz_model = n;
      for (int d = 0; d < f.ndim; ++d) nnz_model += 2 * (n / dims[d]) * (dims[d] - 1);
    }
    return PHIPM_OK;
  }
  return fail(h, PHIPM_EINVAL, "unknown operator kind");
}

static int op_n(const phipm_operator* A) {
  if (A->kind == PHIPM_OP_CSR) return A->csr.n;
  if (A->kind == PHIPM_OP_FUNCTION) return A->fn.nx * A->fn.ny * A->fn.nz;
  return A->st.nx * A->st.ny * A->st.nz;
}

static df32 host_split(double c) {   // c = hi + lo with hi = fl32(c)
  df32 r;
  r.hi = (float)c;
  r.lo = (float)(c - (double)r.hi);
  return r;
}

static DevOp make_devop(const phipm_operator* A, long long nnz_model) {
  DevOp o;
  memset(&o, 0, sizeof(o));
  o.kind = A->kind == PHIPM_OP_CSR ? 0 : A->kind == PHIPM_OP_FUNCTION ? 2 : 1;
  o.n = op_n(A);
  o.nnz = nnz_model;
  if (o.kind == 2) {
    const phipm_function& f = A->fn;
    o.fn = f.fn;
    o.ndim = f.ndim;
    o.nx = f.nx;
    o.ny = f.ny;
    o.nz = f.nz;
    for (int d = 0; d < 4; ++d) o.fld[d] = f.field[d];
    for (int d = 0; d < 6; ++d) o.fsc[d] = f.scal[d];
    o.fnorm = f.norm_inf;
    o.mnx = o.nx >= 2 ? (~0ull / (unsigned long long)o.nx) + 1 : 0;
    o.mny = o.ny >= 2 ? (~0ull / (unsigned long long)o.ny) + 1 : 0;
  } else if (o.kind == 0) {
    o.rowptr = A->csr.rowptr;
    o.colind = A->csr.colind;
    o.val = A->csr.values;
  } else {
    o.ndim = A->st.ndim;
    o.nx = A->st.nx;
    o.ny = A->st.ny;
    o.nz = A->st.nz;
    o.cc = A->st.c_center;
    o.cc2 = host_split(o.cc);
    o.quad = (o.nx % 4 == 0) ? 1 : 0;
    o.mnx = o.nx >= 2 ? (~0ull / (unsigned long long)o.nx) + 1 : 0;
    o.mny = o.ny >= 2 ? (~0ull / (unsigned long long)o.ny) + 1 : 0;
    for (int d = 0; d < 3; ++d) {
      o.cm[d] = A->st.c_minus[d];
      o.cp[d] = A->st.c_plus[d];
      o.cm2[d] = host_split(o.cm[d]);
      o.cp2[d] = host_split(o.cp[d]);
    }
  }
  return o;
}

// The four-row stencil product reads u (the caller's buffer, w_0 of the recurrence)
// with 16-byte loads; a u that is only 8-byte aligned takes the one-row product.
static void fit_quad_to_u(DevProblem& P) {
  if (P.A.kind == 1 && (reinterpret_cast<uintptr_t>(P.u) & 15) != 0) P.A.quad = 0;
}

static long long round_ld(long long n) { return std::max(64ll, (n + 63) & ~63ll); }
static size_t elem_bytes(int precision) { return precision == PHIPM_F32_MIXED ? 4 : 8; }

static phipm_status map_status(int s) {
  switch (s) {
    case PM_OK: return PHIPM_OK;
    case PM_EINVAL: return PHIPM_EINVAL;
    case PM_ENONFINITE: return PHIPM_ENONFINITE;
    case PM_EMAXSTEPS: return PHIPM_EMAXSTEPS;
    case PM_ETIMEOUT: return PHIPM_ETIMEOUT;
    case PM_EBOUNDS: return PHIPM_EBOUNDS;
    case PM_ENOTRUN: return PHIPM_ENOTRUN;
    default: return PHIPM_ECUDA;
  }
}

static const char* status_text(phipm_status s) {
  switch (s) {
    case PHIPM_OK: return "ok";
    case PHIPM_EINVAL: return "invalid argument";
    case PHIPM_ENOMEM: return "out of device memory";
    case PHIPM_ECUDA: return "CUDA error";
    case PHIPM_ENONFINITE: return "ten non-finite error estimates in a row";
    case PHIPM_EMAXSTEPS: return "step or reject limit exceeded";
    case PHIPM_ETIMEOUT: return "a device-side wait timed out";
    case PHIPM_EBOUNDS: return "device bounds check failed";
    case PHIPM_ETOOLARGE: return "problem larger than the static scratch";
    case PHIPM_ENOTRUN: return "not solved: the batched launch stopped before this problem";
  }
  return "unknown";
}

static void fill_stats(phipm_stats* o, const DevResult& r, float kernel_ms) {
  o->steps = r.steps;
  o->rejects = r.rejects;
  o->matvecs = r.matvecs;
  o->expms = r.expms;
  o->err_est_sum = r.err_est_sum;
  o->krylov_steps = r.kry_steps;
  o->gs_vectors = r.gs_vectors;
  o->reorth_vectors = r.reorth_vectors;
  o->kernel_ms = kernel_ms;
}

static SlotLayout slot_layout(long long nmax, int pmax, int m_max, size_t es) {
  SlotLayout lay;
  lay.ld = round_ld(nmax);
  lay.v_off = 0;
  lay.w_off = (long long)(m_max + 1) * lay.ld * (long long)es;
  lay.y_off = lay.w_off + (long long)(pmax + 1) * lay.ld * 8;
  lay.e_off = lay.y_off + 2 * lay.ld * (long long)es;
  lay.e_off = (lay.e_off + 255) & ~255ll;
  lay.bytes = (lay.e_off + (long long)PM_EXPM_DOUBLES * 8 + 255) & ~255ll;   // slots stay 256-byte aligned
  return lay;
}

static cudaError_t launch_queue_any(int precision, int blocks, cudaStream_t stream, const DevProblem* probs,
                                    const int* order, int count, const DevParams& prm, DevResult* res,
                                    unsigned char* slots, const SlotLayout& lay, int* queue) {
  if (precision == PHIPM_F32_MIXED)
    return pm_queue_launch<float>(blocks, stream, probs, order, count, prm, res, slots, lay, queue);
  if (precision == PHIPM_F64_PAIR)
    return pm_queue_launch<df32>(blocks, stream, probs, order, count, prm, res, slots, lay, queue);
  return pm_queue_launch<double>(blocks, stream, probs, order, count, prm, res, slots, lay, queue);
}

static int queue_occupancy(int precision) {
  const int smem = (int)sizeof(PmShared);
  const int occ = precision == PHIPM_F32_MIXED ? pm_queue_occupancy<float>(smem)
                  : precision == PHIPM_F64_PAIR ? pm_queue_occupancy<df32>(smem)
                                                : pm_queue_occupancy<double>(smem);
  return std::max(1, occ);
}

// Attach the learned controller and the trace buffer of the handle to a launch.
static phipm_status attach_runtime(phipm_handle* h, DevParams& prm, cudaStream_t stream) {
#ifdef PM_PHASE_PROBE
  if (!h->phase.p) {
    if (!h->phase.ensure(PM_NPHASE * sizeof(unsigned long long))) return fail(h, PHIPM_ENOMEM, "phase timers");
    cudaMemset(h->phase.p, 0, PM_NPHASE * sizeof(unsigned long long));
  }
  prm.phase_ticks = (unsigned long long*)h->phase.p;
#endif
  if (h->params.controller == PHIPM_CTRL_LEARNED || h->params.controller == PHIPM_CTRL_LEARNED_STEPS) {
    if (!h->has_mlp) return fail(h, PHIPM_EINVAL, "a learned controller needs phipm_set_controller_weights");
    prm.mlp = (const float*)h->mlp_blob.p;
  }
  if (h->trace_cap > 0) {
    prm.trace = (TraceRec*)h->trace.p;
    prm.trace_count = (unsigned long long*)((char*)h->sync.p + 3072);
    prm.trace_cap = h->trace_cap;
    cudaError_t e = cudaMemsetAsync(prm.trace_count, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "trace reset");
  }
  return PHIPM_OK;
}

// After the solver kernel: fetch the number of trace records (host copy is read after the sync).
static cudaError_t fetch_trace_count(phipm_handle* h, const DevParams& prm, cudaStream_t stream) {
  if (!prm.trace) return cudaSuccess;
  return cudaMemcpyAsync(h->trace_count_host.p, prm.trace_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                         stream);
}

// Problems below this size run on one CTA; larger ones on every SM.
static const int kGridMinN = 16384;

// Reserve converted-value storage for CSR problems (FP32 / float-pair bases)
// and point each descriptor at its slice.
static bool assign_conversions(phipm_handle* h, DevProblem* probs, int count, int precision) {
  if (precision == PHIPM_F64) return true;
  const size_t es = precision == PHIPM_F32_MIXED ? 4 : 8;
  size_t total = 0;
  for (int i = 0; i < count; ++i)
    if (probs[i].A.kind == 0) total += ((size_t)probs[i].A.nnz * es + 255) & ~(size_t)255;
  if (total == 0) return true;
  if (!h->conv.ensure(total)) return false;
  size_t off = 0;
  for (int i = 0; i < count; ++i) {
    if (probs[i].A.kind != 0) continue;
    void* p = (char*)h->conv.p + off;
    if (precision == PHIPM_F32_MIXED) probs[i].A.valf = (const float*)p;
    else probs[i].A.val2 = (const df32*)p;
    off += ((size_t)probs[i].A.nnz * es + 255) & ~(size_t)255;
  }
  return true;
}

static int conv_blocks(long long nnz) { return (int)std::max(1ll, std::min(4096ll, (nnz + 255) / 256)); }

static bool any_csr(const DevProblem* probs, int count) {
  for (int i = 0; i < count; ++i)
    if (probs[i].A.kind == 0 && probs[i].A.nnz > 0) return true;
  return false;
}

// ------------------------------------------------------------------------------------
// single solve
// ------------------------------------------------------------------------------------
static int ilog2(long long n) {
  int lg = 0;
  while (lg < 62 && (2ll << lg) <= n) ++lg;    // floor(log2 n), 0 for n <= 1
  return lg;
}
static int size_class(int prec, int kind, int n) { return prec * 10000 + kind * 1000 + ilog2(n); }
static int batch_class(int prec, int count, int nmax) { return prec * 10000 + ilog2(count) * 100 + ilog2(nmax); }

// CTAs that cooperate on one problem: forced, tuned for the size class, or the default
// (every SM from n = 16384 on, else one CTA).
static int choose_team(const phipm_handle* h, int prec, int kind, int n) {
  const int gmax = h->grid_blocks[prec];
  if (h->team_force > 0) return std::min(h->team_force, gmax);
  const auto it = h->tuned.find(size_class(prec, kind, n));
  if (it != h->tuned.end()) return std::min(it->second.first, gmax);
  return n >= kGridMinN ? gmax : 1;
}

// team_req: 0 = choose_team, 1 = one CTA, G >= 2 = cooperative grid of G CTAs
static phipm_status solve_impl(phipm_handle* h, int team_req, double t_end, const phipm_operator* A, int32_t p,
                               const double* const* b, double tol, int32_t symm, double* u, phipm_stats* stats,
                               void* stream_) {
  if (!h) return PHIPM_EINVAL;
  cudaStream_t stream = (cudaStream_t)stream_;
  long long nnz_model = 0;
  phipm_status st = check_operator(h, A, nnz_model);
  if (st != PHIPM_OK) return st;
  if (!(t_end > 0) || !std::isfinite(t_end)) return fail(h, PHIPM_EINVAL, "t_end must be positive and finite");
  if (p < 0 || p > PHIPM_P_MAX) return fail(h, PHIPM_EINVAL, "p out of [0, 8]");
  if (!std::isfinite(tol)) return fail(h, PHIPM_EINVAL, "tol must be finite");
  if (symm < -1 || symm > 1) return fail(h, PHIPM_EINVAL, "symm must be -1, 0 or 1");
  const int n = op_n(A);
  if (n > 0 && (!b || !u)) return fail(h, PHIPM_EINVAL, "b or u is NULL");
  for (int k = 0; k <= p && n > 0; ++k)
    if (!b[k]) return fail(h, PHIPM_EINVAL, "b[k] is NULL");
  if (stats) memset(stats, 0, sizeof(*stats));
  if (n == 0) return PHIPM_OK;

  const int prec = h->params.precision;
  const size_t es = elem_bytes(prec);
  cudaError_t e;
  DevProblem P;
  memset(&P, 0, sizeof(P));
  P.A = make_devop(A, nnz_model);
  P.p = p;
  P.symm = symm;
  P.t_end = t_end;
  P.tol = tol;
  for (int k = 0; k <= p; ++k) P.b[k] = b[k];
  P.u = u;
  fit_quad_to_u(P);
  if (!assign_conversions(h, &P, 1, prec)) return fail(h, PHIPM_ENOMEM, "value conversion buffer");
  DevParams prm = make_params(h->params);
  st = attach_runtime(h, prm, stream);
  if (st != PHIPM_OK) return st;
  const int M1 = h->params.m_max + 1;
  DevResult* res_h = (DevResult*)h->res_host.p;
  DevResult* res_d = (DevResult*)h->res.p;
  const bool convert = prec != PHIPM_F64 && any_csr(&P, 1);
  const int team = team_req > 0 ? std::min(team_req, h->grid_blocks[prec]) : choose_team(h, prec, A->kind, n);

  // teams of 2..8 CTAs run as one thread-block cluster (barriers in distributed shared
  // memory); larger teams as a cooperative grid
  int cK = 0;
  if (team >= 2 && team <= 8) {
    cK = cluster_capacity(prec, team);
    cK = cK >= 1 ? team : 0;
  }
  if (team >= 2 && cK == 0) {
    const long long ld = round_ld(n);
    const size_t vbytes = (size_t)M1 * ld * es, wbytes = (size_t)(p + 1) * ld * 8, ybytes = 2 * (size_t)ld * es;
    if (!h->ws.ensure(vbytes + wbytes + ybytes)) return fail(h, PHIPM_ENOMEM, "workspace");
    P.V = h->ws.p;
    P.W = (double*)((char*)h->ws.p + vbytes);
    P.Y = (char*)h->ws.p + vbytes + wbytes;
    P.ld = ld;
    const int G = team;
    if (!h->partials.ensure((size_t)2 * G * PM_PSTRIDE * sizeof(double))) return fail(h, PHIPM_ENOMEM, "partials");
    if (convert) {
      if (!h->probs.ensure(sizeof(DevProblem)) || !h->probs_host.ensure(sizeof(DevProblem)))
        return fail(h, PHIPM_ENOMEM, "descriptors");
      memcpy(h->probs_host.p, &P, sizeof(P));
      if ((e = cudaMemcpyAsync(h->probs.p, h->probs_host.p, sizeof(P), cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_fail(h, e, "descriptor upload");
      k_convert_values<<<dim3(conv_blocks(P.A.nnz), 1), 256, 0, stream>>>((const DevProblem*)h->probs.p, 1, prec);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "value conversion");
    }
    PmWork w{(double*)h->partials.p, (double*)h->expm.p};
    unsigned long long* bar = (unsigned long long*)h->sync.p;
    int* err = (int*)((char*)h->sync.p + 1024);
    if ((e = cudaMemsetAsync(h->sync.p, 0, 2048, stream)) != cudaSuccess) return cuda_fail(h, e, "memset");
    if ((e = cudaMemsetAsync(res_d, 0, sizeof(DevResult), stream)) != cudaSuccess) return cuda_fail(h, e, "memset");
    cudaEventRecord(h->ev0, stream);
    e = prec == PHIPM_F32_MIXED ? pm_grid_launch<float>(G, stream, P, prm, res_d, w, bar, err)
        : prec == PHIPM_F64_PAIR ? pm_grid_launch<df32>(G, stream, P, prm, res_d, w, bar, err)
                                 : pm_grid_launch<double>(G, stream, P, prm, res_d, w, bar, err);
    if (e != cudaSuccess) return cuda_fail(h, e, "cooperative launch");
    cudaEventRecord(h->ev1, stream);
  } else {
    const SlotLayout lay = slot_layout(n, p, h->params.m_max, es);
    if (!h->ws.ensure((size_t)lay.bytes)) return fail(h, PHIPM_ENOMEM, "workspace");
    if (!h->probs.ensure(sizeof(DevProblem)) || !h->order.ensure(sizeof(int)) ||
        !h->probs_host.ensure(sizeof(DevProblem) + sizeof(int)))
      return fail(h, PHIPM_ENOMEM, "descriptors");
    memcpy(h->probs_host.p, &P, sizeof(P));
    const int zero = 0;
    memcpy((char*)h->probs_host.p + sizeof(DevProblem), &zero, sizeof(int));
    int* queue = (int*)((char*)h->sync.p + 2048);
    if ((e = cudaMemcpyAsync(h->probs.p, h->probs_host.p, sizeof(DevProblem), cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h->order.p, (char*)h->probs_host.p + sizeof(DevProblem), sizeof(int), cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(queue, 0, sizeof(int), stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(res_d, 0, sizeof(DevResult), stream)) != cudaSuccess)
      return cuda_fail(h, e, "descriptor upload");
    if (convert) {
      k_convert_values<<<dim3(conv_blocks(P.A.nnz), 1), 256, 0, stream>>>((const DevProblem*)h->probs.p, 1, prec);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "value conversion");
    }
    if (cK >= 2) {
      if (!h->partials.ensure((size_t)2 * cK * PM_PSTRIDE * sizeof(double))) return fail(h, PHIPM_ENOMEM, "partials");
      int* err = (int*)((char*)h->sync.p + 1024);
      if ((e = cudaMemsetAsync(err, 0, sizeof(int), stream)) != cudaSuccess) return cuda_fail(h, e, "memset");
    }
    cudaEventRecord(h->ev0, stream);
    if (cK >= 2) {
      const DevProblem* pd = (const DevProblem*)h->probs.p;
      const int* od = (const int*)h->order.p;
      unsigned char* ws = (unsigned char*)h->ws.p;
      double* pt = (double*)h->partials.p;
      int* err = (int*)((char*)h->sync.p + 1024);
      e = launch_cluster_any(prec, cK, 1, stream, pd, od, 1, prm, res_d, ws, lay, queue, pt, err);
    } else {
      e = launch_queue_any(prec, 1, stream, (const DevProblem*)h->probs.p, (const int*)h->order.p, 1, prm, res_d,
                           (unsigned char*)h->ws.p, lay, queue);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "launch");
    cudaEventRecord(h->ev1, stream);
  }
  if ((e = cudaMemcpyAsync(res_h, res_d, sizeof(DevResult), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
    return cuda_fail(h, e, "result copy");
  if ((e = fetch_trace_count(h, prm, stream)) != cudaSuccess) return cuda_fail(h, e, "trace count");
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(h, e, "solve");
  if (prm.trace) h->trace_last = (long long)*(unsigned long long*)h->trace_count_host.p;
  if (stats) {
    float kms = 0.f;
    cudaEventElapsedTime(&kms, h->ev0, h->ev1);
    fill_stats(stats, *res_h, kms);
  }
  st = map_status(res_h->status);
  if (st != PHIPM_OK) return fail(h, st, status_text(st));
  return PHIPM_OK;
}

extern "C" phipm_status phipm_solve(phipm_handle* h, double t_end, const phipm_operator* A, int32_t p,
                                   const double* const* b, double tol, int32_t symm, double* u,
                                   phipm_stats* stats, void* stream) {
  return solve_impl(h, 0, t_end, A, p, b, tol, symm, u, stats, stream);
}

// ------------------------------------------------------------------------------------
// host-buffer solve: H2D of the operator and b, device solve, D2H of u
// ------------------------------------------------------------------------------------
extern "C" phipm_status phipm_solve_host(phipm_handle* h, double t_end, const phipm_operator* A_host, int32_t p,
                                        const double* const* b_host, double tol, int32_t symm, double* u_host,
                                        phipm_stats* stats, void* stream_) {
  if (!h) return PHIPM_EINVAL;
  cudaStream_t stream = (cudaStream_t)stream_;
  long long nnz_model = 0;
  phipm_status st = check_operator(h, A_host, nnz_model);
  if (st != PHIPM_OK) return st;
  if (A_host->kind == PHIPM_OP_FUNCTION) return fail(h, PHIPM_EINVAL, "host-buffer solve: CSR or stencil operators");
  if (p < 0 || p > PHIPM_P_MAX) return fail(h, PHIPM_EINVAL, "p out of [0, 8]");
  const int n = op_n(A_host);
  if (n > 0 && (!b_host || !u_host)) return fail(h, PHIPM_EINVAL, "b or u is NULL");
  phipm_operator Ad = *A_host;
  cudaError_t e;
  if (A_host->kind == PHIPM_OP_CSR && n > 0) {
    const long long nnz = A_host->csr.nnz;
    if (!h->h_rowptr.ensure((size_t)(n + 1) * 4) || !h->h_colind.ensure((size_t)std::max(nnz, 1ll) * 4) ||
        !h->h_vals.ensure((size_t)std::max(nnz, 1ll) * 8))
      return fail(h, PHIPM_ENOMEM, "operator staging");
    if ((e = cudaMemcpyAsync(h->h_rowptr.p, A_host->csr.rowptr, (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (nnz > 0 && (e = cudaMemcpyAsync(h->h_colind.p, A_host->csr.colind, (size_t)nnz * 4, cudaMemcpyHostToDevice, stream)) != cudaSuccess) ||
        (nnz > 0 && (e = cudaMemcpyAsync(h->h_vals.p, A_host->csr.values, (size_t)nnz * 8, cudaMemcpyHostToDevice, stream)) != cudaSuccess))
      return cuda_fail(h, e, "operator upload");
    Ad.csr.rowptr = (const int32_t*)h->h_rowptr.p;
    Ad.csr.colind = (const int32_t*)h->h_colind.p;
    Ad.csr.values = (const double*)h->h_vals.p;
  }
  const size_t vb = ((size_t)std::max(n, 1) * 8 + 255) & ~(size_t)255;
  if (!h->h_b.ensure(vb * (p + 1)) || !h->h_u.ensure(vb)) return fail(h, PHIPM_ENOMEM, "vector staging");
  const double* bd[PHIPM_P_MAX + 1];
  for (int k = 0; k <= p; ++k) {
    bd[k] = (const double*)((char*)h->h_b.p + vb * k);
    if (n > 0) {
      if (!b_host[k]) return fail(h, PHIPM_EINVAL, "b[k] is NULL");
      if ((e = cudaMemcpyAsync((void*)bd[k], b_host[k], (size_t)n * 8, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_fail(h, e, "b upload");
    }
  }
  st = phipm_solve(h, t_end, &Ad, p, bd, tol, symm, (double*)h->h_u.p, stats, stream_);
  if (st != PHIPM_OK) return st;
  if (n > 0) {
    if ((e = cudaMemcpyAsync(u_host, h->h_u.p, (size_t)n * 8, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
      return cuda_fail(h, e, "u download");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(h, e, "u download");
  }
  return PHIPM_OK;
}

// ------------------------------------------------------------------------------------
// batched: one persistent launch, one CTA per problem at a time, largest first
// ------------------------------------------------------------------------------------
extern "C" phipm_status phipm_solve_batched(phipm_handle* h, int32_t count, const double* t_end,
                                           const phipm_operator* A, const int32_t* p,
                                           const double* const* const* b, const double* tol,
                                           const int32_t* symm, double* const* u, phipm_stats* stats,
                                           phipm_status* per_problem, void* stream_) {
  if (!h) return PHIPM_EINVAL;
  cudaStream_t stream = (cudaStream_t)stream_;
  if (count < 0) return fail(h, PHIPM_EINVAL, "count < 0");
  if (count == 0) return PHIPM_OK;
  if (!t_end || !A || !p || !b || !tol || !symm || !u) return fail(h, PHIPM_EINVAL, "NULL array argument");
  const int prec = h->params.precision;
  const size_t es = elem_bytes(prec);
  std::vector<DevProblem> probs(count);
  std::vector<double> cost(count);
  int nmax = 1, pmax = 1;
  for (int i = 0; i < count; ++i) {
    long long nnz_model = 0;
    phipm_status st = check_operator(h, &A[i], nnz_model);
    if (st != PHIPM_OK) return st;
    if (!(t_end[i] > 0) || !std::isfinite(t_end[i])) return fail(h, PHIPM_EINVAL, "t_end must be positive and finite");
    if (p[i] < 0 || p[i] > PHIPM_P_MAX) return fail(h, PHIPM_EINVAL, "p out of [0, 8]");
    if (symm[i] < -1 || symm[i] > 1) return fail(h, PHIPM_EINVAL, "symm must be -1, 0 or 1");
    if (!std::isfinite(tol[i])) return fail(h, PHIPM_EINVAL, "tol must be finite");
    const int n = op_n(&A[i]);
    if (n > 0 && (!b[i] || !u[i])) return fail(h, PHIPM_EINVAL, "b[i] or u[i] is NULL");
    DevProblem& P = probs[i];
    memset(&P, 0, sizeof(P));
    P.A = make_devop(&A[i], nnz_model);
    P.p = p[i];
    P.symm = symm[i];
    P.t_end = t_end[i];
    P.tol = tol[i];
    for (int k = 0; k <= p[i]; ++k) {
      if (n > 0 && !b[i][k]) return fail(h, PHIPM_EINVAL, "b[i][k] is NULL");
      P.b[k] = b[i][k];
    }
    P.u = u[i];
    fit_quad_to_u(P);
    nmax = std::max(nmax, n);
    pmax = std::max(pmax, (int)p[i]);
    cost[i] = (double)nnz_model + (double)n * 16.0;
  }
  if (!assign_conversions(h, probs.data(), count, prec)) return fail(h, PHIPM_ENOMEM, "value conversion buffer");
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  const SlotLayout lay = slot_layout(nmax, pmax, h->params.m_max, es);
  // Team per problem: one CTA (queue) or a cluster of K CTAs.  phipm_set_team forces K
  // (up to 8); else the K that phipm_autotune_batched measured fastest for this batch
  // class; else K grows with the share of the largest problem in the batch's work: with
  // ratio = SMs x largest cost / total cost, K = 1 below 0.5 (many similar problems keep
  // every SM busy), 2 below 1, else 4.
  int K;
  const auto tb = h->tuned_batch.find(batch_class(prec, count, nmax));
  if (h->batch_req > 0) {
    K = h->batch_req;
  } else if (h->team_force > 0) {
    K = std::min(h->team_force, 8);
  } else if (tb != h->tuned_batch.end()) {
    K = tb->second.first;
  } else {
    double cmax = 0.0, csum = 0.0;
    for (int i = 0; i < count; ++i) {
      cmax = std::max(cmax, cost[i]);
      csum += cost[i];
    }
    const double ratio = csum > 0.0 ? h->num_sms * cmax / csum : 0.0;
    K = ratio < 0.5 ? 1 : ratio < 1.0 ? 2 : 4;
  }
  int clusters = 0;
  if (K >= 2) {
    clusters = cluster_capacity(prec, K);
    if (clusters < 1) K = 1;
  }
  if (K < 2) K = 1;
  h->last_batch_team = K;
  const int slots = K >= 2 ? std::max(1, std::min(count, clusters))
                           : std::max(1, std::min(count, queue_occupancy(prec) * h->num_sms));
  if (K >= 2 && !h->partials.ensure((size_t)slots * 2 * K * PM_PSTRIDE * sizeof(double)))
    return fail(h, PHIPM_ENOMEM, "partials");
  if (!h->ws.ensure((size_t)lay.bytes * slots)) return fail(h, PHIPM_ENOMEM, "workspace");
  const size_t pb = sizeof(DevProblem) * count, ob = sizeof(int) * count, rb = sizeof(DevResult) * count;
  // pinned host staging: descriptors, queue order, and the records every result starts
  // from (status "not run", overwritten by the solver; a problem that no team took
  // because the launch stopped early keeps it)
  const size_t r0 = (pb + ob + 15) & ~(size_t)15;
  if (!h->probs.ensure(pb) || !h->order.ensure(ob) || !h->res.ensure(rb) || !h->probs_host.ensure(r0 + rb) ||
      !h->res_host.ensure(rb))
    return fail(h, PHIPM_ENOMEM, "descriptors");
  for (int i = 0; i < count; ++i) probs[i].id = i;
  memcpy(h->probs_host.p, probs.data(), pb);
  memcpy((char*)h->probs_host.p + pb, order.data(), ob);
  {
    DevResult init;
    memset(&init, 0, sizeof(init));
    init.status = PM_ENOTRUN;
    for (int i = 0; i < count; ++i) memcpy((char*)h->probs_host.p + r0 + (size_t)i * sizeof(DevResult), &init, sizeof(init));
  }
  DevParams prm = make_params(h->params);
  {
    const phipm_status st = attach_runtime(h, prm, stream);
    if (st != PHIPM_OK) return st;
  }
  int* queue = (int*)((char*)h->sync.p + 2048);
  cudaError_t e;
  long long max_nnz = 0;
  for (int i = 0; i < count; ++i) max_nnz = std::max(max_nnz, probs[i].A.kind == 0 ? probs[i].A.nnz : 0ll);
  const bool convert = prec != PHIPM_F64 && any_csr(probs.data(), count);
  // Everything baked into the graph: sizes, buffers, launch shape and parameters.
  // Descriptors are read from pinned host memory at every replay.
  std::vector<unsigned char> key;
  auto put = [&key](const void* p, size_t n) { key.insert(key.end(), (const unsigned char*)p, (const unsigned char*)p + n); };
  const void* ptrs[] = {h->probs.p, h->probs_host.p, h->order.p, h->res.p, h->res_host.p, h->ws.p, h->sync.p,
                        h->trace_count_host.p};
  put(ptrs, sizeof(ptrs));
  put(&count, sizeof(count));
  put(&slots, sizeof(slots));
  put(&K, sizeof(K));
  const void* pp = h->partials.p;
  put(&pp, sizeof(pp));
  put(&lay, sizeof(lay));
  put(&prec, sizeof(prec));
  put(&convert, sizeof(convert));
  put(&max_nnz, sizeof(max_nnz));
  put(&prm, sizeof(prm));
  if (!h->gexec || key != h->gkey) {
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail(h, e, "graph capture");
    cudaStream_t gs = h->gstream;
    cudaMemcpyAsync(h->probs.p, h->probs_host.p, pb, cudaMemcpyHostToDevice, gs);
    cudaMemcpyAsync(h->order.p, (char*)h->probs_host.p + pb, ob, cudaMemcpyHostToDevice, gs);
    cudaMemsetAsync(queue, 0, sizeof(int), gs);
    cudaMemcpyAsync(h->res.p, (char*)h->probs_host.p + r0, rb, cudaMemcpyHostToDevice, gs);
    if (prm.trace) cudaMemsetAsync(prm.trace_count, 0, sizeof(unsigned long long), gs);
    if (convert)
      k_convert_values<<<dim3(conv_blocks(max_nnz) / 8 + 1, count), 256, 0, gs>>>((const DevProblem*)h->probs.p,
                                                                                 count, prec);
    if (K >= 2) {
      int* err = (int*)((char*)h->sync.p + 1024);
      cudaMemsetAsync(err, 0, sizeof(int), gs);
      const DevProblem* pd = (const DevProblem*)h->probs.p;
      const int* od = (const int*)h->order.p;
      DevResult* rd = (DevResult*)h->res.p;
      unsigned char* ws = (unsigned char*)h->ws.p;
      double* pt = (double*)h->partials.p;
      launch_cluster_any(prec, K, slots, gs, pd, od, count, prm, rd, ws, lay, queue, pt, err);
    } else {
      launch_queue_any(prec, slots, gs, (const DevProblem*)h->probs.p, (const int*)h->order.p, count, prm,
                       (DevResult*)h->res.p, (unsigned char*)h->ws.p, lay, queue);
    }
    cudaMemcpyAsync(h->res_host.p, h->res.p, rb, cudaMemcpyDeviceToHost, gs);
    fetch_trace_count(h, prm, gs);
    e = cudaStreamEndCapture(h->gstream, &graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { h->gexec = nullptr; return cuda_fail(h, e, "graph instantiate"); }
    h->gkey = key;
  }
  // order after the caller's stream, replay, wait
  if ((e = cudaEventRecord(h->gev, stream)) != cudaSuccess || (e = cudaStreamWaitEvent(h->gstream, h->gev, 0)) != cudaSuccess)
    return cuda_fail(h, e, "stream order");
  cudaEventRecord(h->ev0, h->gstream);
  if ((e = cudaGraphLaunch(h->gexec, h->gstream)) != cudaSuccess) return cuda_fail(h, e, "graph launch");
  cudaEventRecord(h->ev1, h->gstream);
  if ((e = cudaStreamSynchronize(h->gstream)) != cudaSuccess) return cuda_fail(h, e, "batched solve");
  if (prm.trace) h->trace_last = (long long)*(unsigned long long*)h->trace_count_host.p;
  float kms = 0.f;
  cudaEventElapsedTime(&kms, h->ev0, h->ev1);
  const DevResult* rh = (const DevResult*)h->res_host.p;
  phipm_status overall = PHIPM_OK;
  for (int i = 0; i < count; ++i) {
    const phipm_status si = map_status(rh[i].status);
    if (per_problem) per_problem[i] = si;
    if (stats) fill_stats(&stats[i], rh[i], kms);
    if (si != PHIPM_OK && overall == PHIPM_OK) overall = si;
  }
  if (overall != PHIPM_OK) return fail(h, overall, status_text(overall));
  return PHIPM_OK;
}

// ------------------------------------------------------------------------------------
// traces and the learned controller
// ------------------------------------------------------------------------------------
static_assert(sizeof(TraceRec) == sizeof(phipm_trace_record), "trace record layout");

extern "C" phipm_status phipm_trace_enable(phipm_handle* h, int64_t capacity) {
  if (!h) return PHIPM_EINVAL;
  if (capacity < 0) return fail(h, PHIPM_EINVAL, "capacity < 0");
  if (capacity > 0 && !h->trace.ensure((size_t)capacity * sizeof(TraceRec))) return fail(h, PHIPM_ENOMEM, "trace buffer");
  h->trace_cap = capacity;
  h->trace_last = 0;
  return PHIPM_OK;
}

extern "C" phipm_status phipm_trace_read(phipm_handle* h, phipm_trace_record* out, int64_t max, int64_t* count) {
  if (!h || (max > 0 && !out)) return PHIPM_EINVAL;
  if (count) *count = h->trace_last;
  const long long k = std::min<long long>(std::min<long long>(max, h->trace_last), h->trace_cap);
  if (k <= 0) return PHIPM_OK;
  cudaError_t e = cudaMemcpy(out, h->trace.p, (size_t)k * sizeof(TraceRec), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "trace copy");
  return PHIPM_OK;
}

extern "C" phipm_status phipm_set_controller_weights(phipm_handle* h, const float* blob, size_t count) {
  if (!h) return PHIPM_EINVAL;
  if (count == 0) { h->has_mlp = false; return PHIPM_OK; }
  if (!blob || count != (size_t)PHIPM_CONTROLLER_FLOATS)
    return fail(h, PHIPM_EINVAL, "controller blob must hold PHIPM_CONTROLLER_FLOATS floats");
  for (size_t i = 0; i < count; ++i)
    if (!std::isfinite(blob[i])) return fail(h, PHIPM_EINVAL, "controller blob is not finite");
  for (int i = 0; i < MLP_IN; ++i)
    if (!(blob[MLP_NP + MLP_IN + i] > 0.f)) return fail(h, PHIPM_EINVAL, "feature scales must be positive");
  if (!h->mlp_blob.ensure(count * sizeof(float))) return fail(h, PHIPM_ENOMEM, "controller weights");
  cudaError_t e = cudaMemcpy(h->mlp_blob.p, blob, count * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "controller weights");
  h->has_mlp = true;
  return PHIPM_OK;
}

static int mlp_blocks(phipm_handle* h, long long n) {
  const long long want = (n + MLP_WARPS * 4 - 1) / (MLP_WARPS * 4);
  return (int)std::max(1ll, std::min<long long>(want, h->num_sms));
}

extern "C" phipm_status phipm_mlp_forward(phipm_handle* h, const float* w, const float* X, int64_t n, float* Y,
                                         void* stream_) {
  if (!h || n < 0 || (n > 0 && (!w || !X || !Y))) return PHIPM_EINVAL;
  if (n == 0) return PHIPM_OK;
  cudaStream_t stream = (cudaStream_t)stream_;
  const int G = (int)std::max(1ll, std::min<long long>((n + 7) / 8, 4ll * h->num_sms));
  k_mlp_forward<<<G, 256, 0, stream>>>(w, X, n, Y);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  return e == cudaSuccess ? PHIPM_OK : cuda_fail(h, e, "mlp forward");
}

extern "C" phipm_status phipm_mlp_grad(phipm_handle* h, const float* w, const float* X, const float* T, int64_t n,
                                      float* grad, float* loss, void* stream_) {
  if (!h || n <= 0 || !w || !X || !T || !grad) return PHIPM_EINVAL;
  cudaStream_t stream = (cudaStream_t)stream_;
  const int G = mlp_blocks(h, n);
  if (!h->mlp_part.ensure((size_t)G * MLP_PART * sizeof(float))) return fail(h, PHIPM_ENOMEM, "mlp partials");
  k_mlp_grad<<<G, MLP_WARPS * 32, sizeof(MlpSmem), stream>>>(w, X, T, n, (float*)h->mlp_part.p);
  k_mlp_adam<<<(MLP_NP + 256) / 256, 256, 0, stream>>>(nullptr, nullptr, nullptr, (const float*)h->mlp_part.p, G,
                                                       grad, loss, 0, 0.f, 0.f, 0.f, 0.f);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  return e == cudaSuccess ? PHIPM_OK : cuda_fail(h, e, "mlp gradient");
}

extern "C" phipm_status phipm_mlp_train(phipm_handle* h, float* w, float* m, float* v, const float* X, const float* T,
                                       int64_t n, int32_t iters, int64_t t0, float lr, float* losses, void* stream_) {
  if (!h || n <= 0 || iters < 0 || !w || !m || !v || !X || !T || !(lr > 0.f)) return PHIPM_EINVAL;
  cudaStream_t stream = (cudaStream_t)stream_;
  const int G = mlp_blocks(h, n);
  if (!h->mlp_part.ensure((size_t)G * MLP_PART * sizeof(float) + (size_t)std::max(iters, 1) * sizeof(float)))
    return fail(h, PHIPM_ENOMEM, "mlp partials");
  float* lossdev = (float*)((char*)h->mlp_part.p + (size_t)G * MLP_PART * sizeof(float));
  for (int it = 0; it < iters; ++it) {
    k_mlp_grad<<<G, MLP_WARPS * 32, sizeof(MlpSmem), stream>>>(w, X, T, n, (float*)h->mlp_part.p);
    k_mlp_adam<<<(MLP_NP + 256) / 256, 256, 0, stream>>>(w, m, v, (const float*)h->mlp_part.p, G, nullptr,
                                                         lossdev + it, t0 + it + 1, lr, 0.9f, 0.999f, 1e-8f);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && losses && iters > 0)
    e = cudaMemcpyAsync(losses, lossdev, (size_t)iters * sizeof(float), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  return e == cudaSuccess ? PHIPM_OK : cuda_fail(h, e, "mlp training");
}

// ------------------------------------------------------------------------------------
// team-size autotuner: per size class, the number of CTAs that cooperate on a solve
// ------------------------------------------------------------------------------------
extern "C" phipm_status phipm_autotune(phipm_handle* h, double t_end, const phipm_operator* A, int32_t p,
                                      const double* const* b, double tol, int32_t symm, double* u,
                                      phipm_tune_entry* report, int32_t max_report, int32_t* n_report,
                                      void* stream) {
  if (!h || !A) return PHIPM_EINVAL;
  if (n_report) *n_report = 0;
  const int prec = h->params.precision;
  const int n = op_n(A);
  if (n <= 0) return fail(h, PHIPM_EINVAL, "autotune needs n > 0");
  const int gmax = h->grid_blocks[prec];
  std::vector<int> cand = {1};
  for (int g : {2, 4, 8, 16, 32})
    if (g <= gmax && (long long)n >= 64ll * g) cand.push_back(g);
  for (int div : {4, 2, 1}) {                 // fractions of the co-resident grid
    const int g = gmax / div;
    if (g >= 2 && (long long)n >= 64ll * g && std::find(cand.begin(), cand.end(), g) == cand.end()) cand.push_back(g);
  }
  int best = 0, k = 0;
  double best_ms = 0.0;
  for (int g : cand) {
    phipm_stats st;
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {       // the second run is timed (the first pays first-touch costs)
      const phipm_status r = solve_impl(h, g, t_end, A, p, b, tol, symm, u, &st, stream);
      if (r != PHIPM_OK) return r;
      ms = (float)st.kernel_ms;
    }
    if (report && k < max_report) {
      report[k].team = g;
      report[k].kernel_ms = ms;
    }
    ++k;
    if (best == 0 || ms < best_ms) { best = g; best_ms = ms; }
  }
  if (n_report) *n_report = std::min(k, max_report);
  h->tuned[size_class(prec, A->kind, n)] = {best, best_ms};
  return PHIPM_OK;
}

extern "C" phipm_status phipm_autotune_batched(phipm_handle* h, int32_t count, const double* t_end,
                                              const phipm_operator* A, const int32_t* p,
                                              const double* const* const* b, const double* tol, const int32_t* symm,
                                              double* const* u, phipm_tune_entry* report, int32_t max_report,
                                              int32_t* n_report, void* stream) {
  if (!h) return PHIPM_EINVAL;
  if (n_report) *n_report = 0;
  if (count <= 0 || !A) return fail(h, PHIPM_EINVAL, "autotune_batched needs count > 0");
  const int prec = h->params.precision;
  int nmax = 1;
  for (int i = 0; i < count; ++i) nmax = std::max(nmax, op_n(&A[i]));
  std::vector<phipm_stats> st((size_t)count);
  int best = 0, k = 0;
  double best_ms = 0.0;
  for (int K : {1, 2, 4, 8}) {
    if (K >= 2 && cluster_capacity(prec, K) < 1) continue;
    h->batch_req = K;
    double ms = 0.0;
    phipm_status r = PHIPM_OK;
    for (int rep = 0; rep < 2 && r == PHIPM_OK; ++rep) {   // the second run is timed (the first captures the graph)
      r = phipm_solve_batched(h, count, t_end, A, p, b, tol, symm, u, st.data(), nullptr, stream);
      ms = st[0].kernel_ms;
    }
    h->batch_req = 0;
    if (r != PHIPM_OK) return r;
    if (report && k < max_report) {
      report[k].team = K;
      report[k].kernel_ms = ms;
    }
    ++k;
    if (best == 0 || ms < best_ms) { best = K; best_ms = ms; }
  }
  if (n_report) *n_report = std::min(k, max_report);
  h->tuned_batch[batch_class(prec, count, nmax)] = {best, best_ms};
  return PHIPM_OK;
}

extern "C" phipm_status phipm_set_team(phipm_handle* h, int32_t team) {
  if (!h) return PHIPM_EINVAL;
  if (team < 0) return fail(h, PHIPM_EINVAL, "team < 0");
  h->team_force = team;
  return PHIPM_OK;
}

extern "C" int32_t phipm_batched_team(const phipm_handle* h) { return h ? h->last_batch_team : 0; }

#ifdef PM_PHASE_PROBE
// Probe build only: the accumulated clock cycles per solver phase (PM_NPHASE values), then zero them.
extern "C" phipm_status phipm_probe_phase_ticks(phipm_handle* h, unsigned long long* out) {
  if (!h || !out || !h->phase.p) return PHIPM_EINVAL;
  if (cudaMemcpy(out, h->phase.p, PM_NPHASE * sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PHIPM_ECUDA;
  cudaMemset(h->phase.p, 0, PM_NPHASE * sizeof(unsigned long long));
  return PHIPM_OK;
}
#endif

extern "C" int32_t phipm_team_for(const phipm_handle* h, int32_t precision, int32_t kind, int32_t n) {
  if (!h || precision < 0 || precision > 2 || kind < 0 || kind > 2 || n <= 0) return 0;
  return choose_team(h, precision, kind, n);
}

// Cache file: one JSON object, {"sms": S, "entries": [{"precision": P, "kind": K,
// "log2n": L, "team": G, "ms": T}, ...]}.  Entries for another SM count are ignored
// on load.
extern "C" phipm_status phipm_tune_save(phipm_handle* h, const char* path) {
  if (!h || !path) return PHIPM_EINVAL;
  FILE* f = fopen(path, "w");
  if (!f) return fail(h, PHIPM_EINVAL, std::string("cannot write ") + path);
  fprintf(f, "{\"sms\": %d, \"entries\": [", h->num_sms);
  bool first = true;
  for (const auto& kv : h->tuned) {
    const int key = kv.first;
    fprintf(f, "%s\n  {\"precision\": %d, \"kind\": %d, \"log2n\": %d, \"team\": %d, \"ms\": %.6g}", first ? "" : ",",
            key / 10000, (key / 1000) % 10, key % 1000, kv.second.first, kv.second.second);
    first = false;
  }
  fprintf(f, "\n], \"batch_entries\": [");
  first = true;
  for (const auto& kv : h->tuned_batch) {
    const int key = kv.first;
    fprintf(f, "%s\n  {\"precision\": %d, \"log2count\": %d, \"log2nmax\": %d, \"team\": %d, \"ms\": %.6g}",
            first ? "" : ",", key / 10000, (key / 100) % 100, key % 100, kv.second.first, kv.second.second);
    first = false;
  }
  fprintf(f, "\n]}\n");
  const bool ok = fclose(f) == 0;
  return ok ? PHIPM_OK : fail(h, PHIPM_EINVAL, std::string("cannot write ") + path);
}

static bool json_int(const std::string& obj, const char* key, long long& out) {
  const std::string k = std::string("\"") + key + "\"";
  size_t i = obj.find(k);
  if (i == std::string::npos) return false;
  i = obj.find(':', i + k.size());
  if (i == std::string::npos) return false;
  ++i;
  while (i < obj.size() && (obj[i] == ' ' || obj[i] == '\t' || obj[i] == '\n' || obj[i] == '\r')) ++i;
  char* end = nullptr;
  const long long v = strtoll(obj.c_str() + i, &end, 10);
  if (end == obj.c_str() + i) return false;
  out = v;
  return true;
}

extern "C" phipm_status phipm_tune_load(phipm_handle* h, const char* path) {
  if (!h || !path) return PHIPM_EINVAL;
  FILE* f = fopen(path, "r");
  if (!f) return fail(h, PHIPM_EINVAL, std::string("cannot read ") + path);
  std::string text;
  char buf[4096];
  size_t r;
  while ((r = fread(buf, 1, sizeof(buf), f)) > 0 && text.size() < (1u << 20)) text.append(buf, r);
  fclose(f);
  long long sms = 0;
  const size_t lb = text.find('[');
  if (lb == std::string::npos || !json_int(text.substr(0, lb), "sms", sms))
    return fail(h, PHIPM_EINVAL, "tuning cache: no sms / entries");
  if (sms != h->num_sms) return PHIPM_OK;     // tuned on another GPU: nothing applies
  std::map<int, std::pair<int, double>> add, add_batch;
  size_t pos = lb;
  while (true) {
    const size_t a = text.find('{', pos), z = (a == std::string::npos) ? a : text.find('}', a);
    if (a == std::string::npos || z == std::string::npos) break;
    const std::string obj = text.substr(a, z - a + 1);
    long long pr, kd, lg, tm, lc;
    if (json_int(obj, "log2count", lc)) {     // a batched entry: cluster size K per batch class
      if (!json_int(obj, "precision", pr) || !json_int(obj, "log2nmax", lg) || !json_int(obj, "team", tm) || pr < 0 ||
          pr > 2 || lc < 0 || lc > 31 || lg < 0 || lg > 31 || (tm != 1 && tm != 2 && tm != 4 && tm != 8))
        return fail(h, PHIPM_EINVAL, "tuning cache: malformed batch entry");
      add_batch[(int)(pr * 10000 + lc * 100 + lg)] = {(int)tm, 0.0};
    } else {
      if (!json_int(obj, "precision", pr) || !json_int(obj, "kind", kd) || !json_int(obj, "log2n", lg) ||
          !json_int(obj, "team", tm) || pr < 0 || pr > 2 || kd < 0 || kd > 2 || lg < 0 || lg > 30 || tm < 1 ||
          tm > 1 << 20)
        return fail(h, PHIPM_EINVAL, "tuning cache: malformed entry");
      add[(int)(pr * 10000 + kd * 1000 + lg)] = {(int)tm, 0.0};
    }
    pos = z + 1;
  }
  for (const auto& kv : add) h->tuned[kv.first] = kv.second;
  for (const auto& kv : add_batch) h->tuned_batch[kv.first] = kv.second;
  return PHIPM_OK;
}

// ------------------------------------------------------------------------------------
// allocation-free solve: the workspace of one single-CTA FP64 solve lives in a
// file-scope device array (n <= PHIPM_NOALLOC_MAX_N)
// ------------------------------------------------------------------------------------
namespace {
constexpr long long kNaLd = PHIPM_NOALLOC_MAX_N;                        // multiple of 64
constexpr long long kNaV = 0;                                           // (m_max+1) basis vectors
constexpr long long kNaW = kNaV + (PM_MAXM + 1) * kNaLd * 8;            // w_1..w_p + spare
constexpr long long kNaY = kNaW + (PM_MAXP + 1) * kNaLd * 8;            // two Krylov vectors
constexpr long long kNaE = (kNaY + 2 * kNaLd * 8 + 255) & ~255ll;       // exponential scratch
constexpr long long kNaR = (kNaE + (long long)PM_EXPM_DOUBLES * 8 + 255) & ~255ll;   // result record
constexpr long long kNaBytes = (kNaR + (long long)sizeof(DevResult) + 255) & ~255ll;
}  // namespace

// Only the host-side address lookup below may name this array from host code:
// on the host its name is a stand-in, not a device address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

__global__ void __launch_bounds__(PM_THREADS, 1)
k_solve_noalloc(DevProblem P, DevParams prm, unsigned char* scratch) {
  extern __shared__ __align__(16) unsigned char pm_smem[];
  PmShared& s = *reinterpret_cast<PmShared*>(pm_smem);
  DevResult* res = reinterpret_cast<DevResult*>(scratch + kNaR);
  if (threadIdx.x == 0) memset(res, 0, sizeof(DevResult));   // the array keeps the last call's contents
  __syncthreads();
  P.V = scratch + kNaV;
  P.W = reinterpret_cast<double*>(scratch + kNaW);
  P.Y = scratch + kNaY;
  P.ld = kNaLd;
  PmWork w{nullptr, reinterpret_cast<double*>(scratch + kNaE)};
  CtaTeam team;
  phipm_device<CtaTeam, double>(team, P, prm, *res, s, w);
}

namespace {
std::mutex g_noalloc_mu;
constexpr int kNaMaxDevices = 64;
unsigned char* g_noalloc_ptr[kNaMaxDevices] = {nullptr};
}  // namespace

extern "C" phipm_status phipm_solve_noalloc(double t_end, const phipm_operator* A, int32_t p,
                                           const double* const* b, double tol, int32_t symm, double* u,
                                           phipm_stats* stats, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  long long nnz_model = 0;
  if (check_operator(nullptr, A, nnz_model) != PHIPM_OK) return PHIPM_EINVAL;
  if (!(t_end > 0) || !std::isfinite(t_end) || !std::isfinite(tol) || symm < -1 || symm > 1 || p < 0)
    return PHIPM_EINVAL;
  const int n = op_n(A);
  if (n > PHIPM_NOALLOC_MAX_N || p > PHIPM_P_MAX) return PHIPM_ETOOLARGE;
  if (n > 0 && (!b || !u)) return PHIPM_EINVAL;
  for (int k = 0; k <= p && n > 0; ++k)
    if (!b[k]) return PHIPM_EINVAL;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (n == 0) return PHIPM_OK;
  // once per device, with that device current: the array's device address
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return PHIPM_ECUDA;
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return PHIPM_ECUDA;
      if (cudaFuncSetAttribute(k_solve_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PmShared)) !=
          cudaSuccess)
        return PHIPM_ECUDA;
      g_noalloc_ptr[dev] = (unsigned char*)ptr;
    }
    scratch = g_noalloc_ptr[dev];
  }
  phipm_params defaults;
  phipm_default_params(&defaults);
  DevProblem P;
  memset(&P, 0, sizeof(P));
  P.A = make_devop(A, nnz_model);
  P.p = p;
  P.symm = symm;
  P.t_end = t_end;
  P.tol = tol;
  for (int k = 0; k <= p; ++k) P.b[k] = b[k];
  P.u = u;
  fit_quad_to_u(P);
  const DevParams prm = make_params(defaults);
  k_solve_noalloc<<<1, PM_THREADS, sizeof(PmShared), stream>>>(P, prm, scratch);
  if (cudaGetLastError() != cudaSuccess) return PHIPM_ECUDA;
  DevResult r;
  if (cudaMemcpyAsync(&r, scratch + kNaR, sizeof(DevResult), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
    return PHIPM_ECUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return PHIPM_ECUDA;
  if (stats) fill_stats(stats, r, 0.f);
  return map_status(r.status);
}
