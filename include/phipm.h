/*
 * phipm.h -- C ABI of the GB300 (sm_103a) phipm library.
 *
 * Computes u(t_end) = sum_{k=0}^{p} t_end^k phi_k(t_end A) b_k, the solution at
 * t_end of u'(t) = A u + sum_{j=1}^{p} t^{j-1}/(j-1)! b_j, u(0) = b_0
 * (Niesen & Wright, Sec. 3.3, Eqs. lincomb2 and phide), by the adaptive
 * time-stepped Krylov method of Sec. 3 (Algorithms 3 and 4): each step builds
 * the Krylov basis of A for w_p (Arnoldi, Algorithm 1, or Lanczos, Algorithm 2),
 * exponentiates the augmented matrix of Eq. (hathm), applies the corrector of
 * Eq. (phipapprox2), and lets the error estimate of Eq. (errest) adapt the step
 * size tau and the Krylov dimension m (Sec. 3.4).  The call follows the paper's
 * interface [u, stats] = phipm(t, A, b, tol, symm, m) of Sec. 3.5.
 *
 * Every step of the method runs in CUDA kernels on the device of the calling
 * thread; there is no CPU fallback.  If the library cannot run on the GPU it
 * returns PHIPM_ECUDA.
 *
 * Conventions for every entry point:
 *   - Errors are returned as phipm_status codes; the library never traps or
 *     aborts.  phipm_last_error(h) holds a message for the last failure.
 *   - "device" pointers are CUDA global-memory pointers owned by the caller;
 *     "host" pointers are ordinary host memory owned by the caller.
 *   - Calls are ordered on the stream passed in (a cudaStream_t given as
 *     void*; NULL is the legacy default stream).  A solve returns after one
 *     stream synchronisation, so stats and status are final on return.
 *   - A handle is not thread-safe: use one handle per host thread.
 */
#ifndef PHIPM_H
#define PHIPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PHIPM_OK = 0,
  PHIPM_EINVAL = 1,       /* invalid argument (sizes, pointers, p, tol, operator) */
  PHIPM_ENOMEM = 2,       /* device workspace allocation failed                    */
  PHIPM_ECUDA = 3,        /* a CUDA call failed (no device, launch error, ...)     */
  PHIPM_ENONFINITE = 4,   /* ten non-finite error estimates in a row               */
  PHIPM_EMAXSTEPS = 5,    /* params.max_steps or params.max_rejects exceeded       */
  PHIPM_ETIMEOUT = 6,     /* a bounded device-side wait gave up                    */
  PHIPM_EBOUNDS = 7,      /* a device-side bounds check failed                     */
  PHIPM_ETOOLARGE = 8,    /* problem larger than phipm_solve_noalloc's static scratch */
  PHIPM_ENOTRUN = 9       /* batched: the launch stopped (another problem's error) before
                             this problem was solved; its u is not valid               */
} phipm_status;

typedef enum {
  PHIPM_F64 = 0,          /* basis, SpMV and all vector work in IEEE FP64 (FP64 pipe)        */
  PHIPM_F32_MIXED = 1,    /* basis and SpMV in FP32 with FP32 accumulation; Gram-Schmidt
                             dot products summed in FP32 over chunks of four products and
                             accumulated across chunks as float pairs; coefficients, norms, H,
                             the exponential, eps and u in FP64                              */
  PHIPM_F64_PAIR = 2      /* FP64-class accuracy on the FP32 pipe: the basis is stored as
                             float pairs hi+lo (8 bytes, about 48 significant bits) and every
                             SpMV, dot and update of the Krylov phase uses error-free float
                             transforms; the w-recurrence, H, the exponential, eps and u are
                             FP64.  Results differ from PHIPM_F64 by about 2^-48 times the
                             cancellation factor ||F|| / ||u|| of Eq. (step).                 */
} phipm_precision;
/* Range of the two float-based modes: their Krylov vectors and the partial sums of their
 * dot products are float pairs or floats, so the candidate vectors, A times them and
 * their products must stay inside the float range (about 3e38); in practice ||A|| up
 * to about 1e12.  The norms of u and w_p are always summed in FP64. */

typedef enum { PHIPM_OP_CSR = 0, PHIPM_OP_STENCIL = 1, PHIPM_OP_FUNCTION = 2 } phipm_op_kind;

/* CSR matrix, n x n.  rowptr[n+1], colind[nnz] (0-based, int32), values[nnz] (FP64).
 * For phipm_solve*: device pointers.  For phipm_solve_host: host pointers. */
typedef struct {
  int32_t n;
  int32_t nnz;
  const int32_t* rowptr;
  const int32_t* colind;
  const double* values;
} phipm_csr;

/* Constant-coefficient stencil on an nx x ny x nz grid of interior unknowns with
 * homogeneous Dirichlet data, numbered i = x + nx*(y + ny*z) (x fastest):
 *   (Ax)_i = c_center x_i + sum_{d<ndim} ( c_minus[d] x_{i-e_d} + c_plus[d] x_{i+e_d} ),
 * with neighbours outside the grid dropped.  ndim = 1, 2 or 3; unused extents = 1. */
typedef struct {
  int32_t ndim, nx, ny, nz;
  double c_center;
  double c_minus[3];
  double c_plus[3];
} phipm_stencil;

/* Matrix-free operator (Sec. 3.5: A may be given as a function that computes A x).
 * A persistent GPU kernel can only apply device code of its own module, so the
 * functions are built into the library and selected by id; the caller passes their
 * data (device arrays and scalars) and, as with a function handle, may pass an upper
 * bound of ||A||_inf (Eq. tau_0 and the breakdown threshold) and the cost N_A of one
 * product (Eq. 4).  Symmetry is not detected: symm = -1 treats A as nonsymmetric
 * (Arnoldi); pass symm = 1 for a symmetric function.
 *
 * PHIPM_FN_VARCOEF_CONVDIFF, variable-coefficient convection-diffusion on the
 * nx x ny x nz grid of interior unknowns (i = x + nx (y + ny z), Dirichlet 0), with
 * the diffusivity kappa = field[0] (n values > 0) and velocities v_d = field[1 + d]
 * (n values, NULL = 0):
 *   (A x)_i = sum_{d<ndim} ( s_d [ kp (x_{i+e_d} - x_i) - km (x_i - x_{i-e_d}) ]
 *                            - c_d v_{d,i} (x_{i+e_d} - x_{i-e_d}) ),
 * kp = (kappa_i + kappa_{i+e_d}) / 2 and km = (kappa_i + kappa_{i-e_d}) / 2 (kappa_i
 * alone where the neighbour lies outside the grid, where x is 0), s_d = scal[d]
 * (1 / h_d^2) and c_d = scal[3 + d] (1 / (2 h_d)).  Symmetric when every v_d is NULL. */
typedef enum { PHIPM_FN_VARCOEF_CONVDIFF = 0 } phipm_fn_id;
typedef struct {
  int32_t fn;                 /* phipm_fn_id                                            */
  int32_t ndim, nx, ny, nz;   /* grid (unused extents 1)                                */
  int32_t reserved;
  const double* field[4];     /* device arrays of n values; meaning per function        */
  double scal[6];             /* scalars of the function                                */
  double norm_inf;            /* an upper bound of ||A||_inf; <= 0: computed on the device */
  int64_t cost;               /* N_A of Eq. (4); <= 0: the grid operator's structural nonzeros */
} phipm_function;

typedef struct {
  int32_t kind;           /* phipm_op_kind */
  phipm_csr csr;          /* used when kind == PHIPM_OP_CSR      */
  phipm_stencil st;       /* used when kind == PHIPM_OP_STENCIL  */
  phipm_function fn;      /* used when kind == PHIPM_OP_FUNCTION */
} phipm_operator;

/* stats(1..4) of Sec. 3.5 plus the sum of accepted error estimates.
 * matvecs counts the products with A actually performed (the basis is reused
 * when only tau changes and extended when m grows).  krylov_steps counts
 * Arnoldi/Lanczos steps; gs_vectors sums, over the Arnoldi steps (and the
 * completion of each extension's last vector), the number of earlier basis
 * vectors each orthogonalisation pass reads (j at step j; 0 for Lanczos steps).
 * kernel_ms is the device time of the solver kernel, from CUDA events on the
 * call's stream.  reorth_vectors sums j over the Arnoldi steps whose pass also
 * formed the candidate's second projection (always with the FP32 basis; only when
 * the first projection kept less than a quarter of the vector's norm with the
 * FP64-class bases); those passes take two products per basis element, the others one. */
typedef struct {
  int64_t steps;
  int64_t rejects;
  int64_t matvecs;
  int64_t expms;
  double err_est_sum;
  int64_t krylov_steps;
  int64_t gs_vectors;
  double kernel_ms;
  int64_t reorth_vectors;
} phipm_stats;

/* Method parameters.  phipm_default_params() gives the paper's values:
 * gamma = 0.8, delta = 1.2 (Sec. 3.4), m_init = 10 (Algorithm 3), m_max = 64,
 * theta13 = 5.37 (Eq. 8), breakdown_tol = 1e-12 (relative to ||A||_inf). */
typedef struct {
  double gamma;
  double delta;
  int32_t m_init;
  int32_t m_max;          /* 1 <= m_max <= PHIPM_M_MAX */
  double theta13;
  double breakdown_tol;
  int64_t max_steps;
  int64_t max_rejects;
  int32_t precision;      /* phipm_precision */
  int32_t controller;     /* phipm_controller: 0 = the paper's controller; 1, 3 = learned
                             proposals (see below); 2 = fixed Krylov dimension (phip) */
  int64_t timeout_cycles; /* bound on every device-side spin-wait, in clock64 cycles */
  int32_t stencil_stage;  /* 1: a stencil product first copies the CTA's rows and the grid
                             lines next to them into shared memory with one TMA bulk copy
                             (when they fit 64 KB); 0 (default): it reads them as 16-byte
                             quads through L1, measured faster on GB300 */
  int32_t expm_pade;      /* 1: exp of the augmented matrix by the degree-13 Pade approximant
                             with scaling and squaring (the paper's choice, Sec. 3.1); 0
                             (default): by the degree-18 Taylor polynomial (Paterson-
                             Stockmeyer) with scaling and squaring, no LU, faster on GB300.
                             Both are accurate to about the unit roundoff; the cost model of
                             Eq. (4) charges the Pade form either way. */
  int32_t expm_action;    /* how the two columns phi_p(tau H) e1, phi_{p+1}(tau H) e1 of
                             exp(H_hat) are formed.  0 (default): per attempt, as the action of
                             exp(H_hat) on the two unit vectors (the degree-k Taylor polynomial
                             of H_hat / s applied s times, k and s from ||H_hat||_1 with the same
                             2^-53 tail bound; products of H_hat with vectors, upper Hessenberg
                             or tridiagonal, each CTA on its own) where a cost estimate puts it
                             below the full exponential with squarings, else the full
                             exponential (expm_pade selects its form); 1: always the full
                             exponential; 2: the action form whenever s <= 64.  With
                             expm_pade = 1, mode 0 keeps the Pade exponential. */
} phipm_params;

/* Controllers.  PHIPM_CTRL_FIXED_M is the fixed-dimension variant the paper
 * compares phipm with (phip, Sec. 4.2): the same algorithm with the m branch of
 * Algorithm 3 never taken, so every attempt uses m = m_init (shortened only by a
 * happy breakdown, as in phipm) and only tau adapts (Eq. taunew with the q
 * estimate of Eq. 6). */
typedef enum {
  PHIPM_CTRL_PAPER = 0,
  PHIPM_CTRL_LEARNED = 1,        /* the network proposes the first attempt of the first step */
  PHIPM_CTRL_FIXED_M = 2,
  PHIPM_CTRL_LEARNED_STEPS = 3   /* the network proposes the first attempt of every step     */
} phipm_controller;

#define PHIPM_M_MAX 64
#define PHIPM_P_MAX 8

void phipm_default_params(phipm_params* out);

typedef struct phipm_handle phipm_handle;

/* Create a handle on the current CUDA device.  params may be NULL (defaults).
 * The handle owns its device workspace (grown on demand, freed by destroy). */
phipm_status phipm_create(phipm_handle** h, const phipm_params* params);
void phipm_destroy(phipm_handle* h);
const char* phipm_last_error(const phipm_handle* h);
phipm_status phipm_set_params(phipm_handle* h, const phipm_params* params);

/* Single problem, device buffers (Sec. 3.5 interface).
 *   t_end  > 0, finite
 *   A      operator; CSR arrays are device pointers
 *   p      0 <= p <= PHIPM_P_MAX; b[0..p] are p+1 device pointers to n FP64 values
 *   tol    absolute tolerance Tol of Eq. (taunew) on the 2-norm; <= 0 selects 1e-7
 *   symm   1 symmetric (Lanczos), 0 not (Arnoldi), -1 detect on the device
 *   u      device pointer to n FP64 values, written (may not alias any b[k])
 *   stats  host pointer, may be NULL
 *   stream cudaStream_t (as void*)
 * The precision of the basis and SpMV is params.precision. */
phipm_status phipm_solve(phipm_handle* h, double t_end, const phipm_operator* A, int32_t p,
                         const double* const* b, double tol, int32_t symm, double* u,
                         phipm_stats* stats, void* stream);

/* Same computation with every array in host memory (CSR arrays, b[k], u):
 * copies the operator and b to the device, solves, and copies u back.  CSR and
 * stencil operators only (PHIPM_EINVAL for a function operator). */
phipm_status phipm_solve_host(phipm_handle* h, double t_end, const phipm_operator* A_host,
                              int32_t p, const double* const* b_host, double tol, int32_t symm,
                              double* u_host, phipm_stats* stats, void* stream);

/* Batched: count independent problems in one persistent launch.  Arrays of
 * length count in host memory: t_end, A (CSR arrays device pointers), p, b
 * (b[i] is a host array of p[i]+1 device pointers), tol, symm, u (device
 * pointers).  stats and per_problem (host, may be NULL) receive one entry per
 * problem.  Returns PHIPM_OK only if every problem succeeded.  Problems are
 * taken largest first by teams of one CTA or of a K-CTA thread-block cluster
 * (see phipm_set_team); the launch sequence is captured once as a CUDA graph
 * and replayed while sizes, buffers, parameters and team size are unchanged. */
phipm_status phipm_solve_batched(phipm_handle* h, int32_t count, const double* t_end,
                                 const phipm_operator* A, const int32_t* p,
                                 const double* const* const* b, const double* tol,
                                 const int32_t* symm, double* const* u, phipm_stats* stats,
                                 phipm_status* per_problem, void* stream);

/* ---------------------------------------------------------------------------
 * Attempt traces (the records behind the paper's Figs. 2-3, Sec. 4.1: t, tau,
 * m, the estimate and accept/reject of every attempt), and the learned (tau, m)
 * controller trained on them.
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t problem;    /* index of the problem in the call (0 for single solves)          */
  int32_t step;       /* accepted steps before this attempt                              */
  int32_t attempt;    /* attempt number within the step, from 0                          */
  int32_t accepted;   /* 1 if omega <= delta                                             */
  int32_t m_req;      /* Krylov dimension requested for the attempt                      */
  int32_t m_used;     /* dimension used (smaller after a happy breakdown)                */
  int32_t p;          /* number of phi terms minus one                                   */
  int32_t n;          /* problem size                                                    */
  double t;           /* start of the step                                               */
  double t_end;
  double tau;         /* step size of the attempt                                        */
  double eps;         /* error estimate, Eq. (errest) with the tau^{p+1} scaling         */
  double omega;       /* t_end eps / (tau Tol), Eq. (taunew)                             */
  double norm_a;      /* ||A||_inf                                                       */
  double tol;
  double m_new;       /* unrounded, unrestricted m_new of Eq. (3) from this attempt      */
  int32_t source;     /* 0: tau, m from Algorithms 3-4; 1: proposed by the learned controller */
  int32_t rejects_prev; /* rejected attempts in the previous step                        */
} phipm_trace_record;

/* Record up to capacity attempts of every later solve call (0 disables).  The
 * buffer restarts at each call.  phipm_trace_read copies up to max records of the
 * last call to host memory and sets *count to the number the call produced
 * (records beyond capacity are dropped). */
phipm_status phipm_trace_enable(phipm_handle* h, int64_t capacity);
phipm_status phipm_trace_read(phipm_handle* h, phipm_trace_record* out, int64_t max, int64_t* count);

/* The controller network: 8 inputs, two hidden layers of 64 GELU units, 2
 * outputs, FP32; PHIPM_MLP_PARAMS weights laid out as W1[64x8], b1[64],
 * W2[64x64], b2[64], W3[2x64], b3[2] (row-major).  A controller blob appends
 * x_mean[8], x_std[8], y_mean[2], y_std[2].
 *
 * Inputs (before normalisation), at the start of a step:
 *   log10(||A||_inf t_end), log10(Tol), p, log10(tau_start ||A||_inf),
 *   m_start / 64, log10(omega of the previous accepted attempt), rejected
 *   attempts in the previous step, log10(n),
 * where tau_start, m_start are the values Algorithm 3 carries into the step.
 * Outputs: log2(tau / tau_start) and m / 64 of the proposal.  With
 * params.controller = PHIPM_CTRL_LEARNED and a blob installed, the first attempt
 * of the first step uses the proposal in place of Eq. (tau_0) and m_init (tau
 * ratio clamped to [1/32, 8] and to the interval, m to [1, m_max]); the error
 * estimate still accepts or rejects it, and the paper's controller handles every
 * later attempt and step.  With PHIPM_CTRL_LEARNED_STEPS the first step is
 * proposed as above, and the first attempt of every later step takes Algorithm 4's
 * proposal with its tau raised by the network's ratio clamped to [1, 2] (m stays
 * Algorithm 4's; a lowering correction would compound, since Algorithm 3 grows tau
 * at most 2x per step); after a rejected attempt the paper's controller takes over
 * for the rest of the step.  The two
 * modes want networks trained on different labels (learned.py). */
#define PHIPM_MLP_PARAMS 4866
#define PHIPM_CONTROLLER_FLOATS (PHIPM_MLP_PARAMS + 20)
phipm_status phipm_set_controller_weights(phipm_handle* h, const float* blob, size_t count);

/* Device pointers; X is [n x 8], T and Y are [n x 2], row-major FP32.
 * phipm_mlp_forward: Y = f(X) with weights w (PHIPM_MLP_PARAMS, no normalisation).
 * phipm_mlp_grad: grad = d/dw mean((f(X) - T)^2) over all n*2 entries, and *loss.
 * phipm_mlp_train: `iters` full-batch Adam steps on w with moments m, v (device,
 * PHIPM_MLP_PARAMS each), step counter starting at t0+1; losses (host, may be NULL)
 * receives the loss before each step. */
phipm_status phipm_mlp_forward(phipm_handle* h, const float* w, const float* X, int64_t n, float* Y, void* stream);
phipm_status phipm_mlp_grad(phipm_handle* h, const float* w, const float* X, const float* T, int64_t n,
                            float* grad, float* loss, void* stream);
phipm_status phipm_mlp_train(phipm_handle* h, float* w, float* m, float* v, const float* X, const float* T,
                             int64_t n, int32_t iters, int64_t t0, float lr, float* losses, void* stream);

/* Allocation-free solve (the paper has no counterpart; this is a library service).
 *
 * For callers that must not allocate device memory: for example a plugin whose
 * host application reserves all device memory up front and refuses further
 * cudaMalloc calls, or a latency-bound loop that cannot afford cudaMalloc's
 * implicit device synchronisation.  phipm_create allocates (its workspace, its
 * events), so this entry point needs no handle and calls no cudaMalloc,
 * cudaFree or other allocating routine.  Its workspace is one file-scope
 * __device__ array of about 5.5 MB that every GPU which loads the library holds
 * until the process exits.
 *
 * Same arguments and result as phipm_solve with the default parameters
 * (PHIPM_F64, one CTA per solve), device buffers, except that n must be at most
 * PHIPM_NOALLOC_MAX_N and p at most PHIPM_P_MAX; larger problems return
 * PHIPM_ETOOLARGE before any GPU work.  stats->kernel_ms is 0.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  With CUDA's lazy module loading (the default), that lookup
 * is also when the device first sets the array aside, so a caller that reserves
 * all device memory up front should make one call per device before reserving
 * it (or run with CUDA_MODULE_LOADING=EAGER).  The address is then kept per
 * device for the life of the process: do not reset the device
 * (cudaDeviceReset) or replace its primary context between calls.  All calls
 * share the one array, which keeps the last call's contents (the kernel clears
 * what must start at zero): calls whose work overlaps on the GPU, e.g. on two
 * streams at once, race on it and must be serialised by the caller.  The call
 * synchronises the stream before returning. */
#define PHIPM_NOALLOC_MAX_N 8192
phipm_status phipm_solve_noalloc(double t_end, const phipm_operator* A, int32_t p, const double* const* b,
                                 double tol, int32_t symm, double* u, phipm_stats* stats, void* stream);

/* ---------------------------------------------------------------------------
 * Team-size autotuner (the paper has no counterpart; a library service).
 *
 * A solve runs on a team of CTAs: one CTA (the whole problem in one SM's shared
 * state) or a cooperative grid of G CTAs, each owning a 64-row-aligned block
 * of every vector, with grid-wide reductions and barriers between phases.  The
 * best G depends on n, the operator and the precision: more CTAs add memory
 * parallelism and split the exponential, but every Krylov step pays two or
 * three grid barriers.  Without tuning a solve uses one CTA below n = 16384 and
 * every co-resident CTA from there on.
 *
 * phipm_autotune solves the given problem (arguments as phipm_solve; device
 * buffers) with each candidate team size -- 1, 2, 4, 8, 16, 32 and 1/4, 1/2 and
 * all of the co-resident grid, keeping only sizes that leave every CTA at least
 * 64 rows -- timing the second of two solves per candidate, and records the
 * fastest for the problem's size class (precision, operator kind, floor(log2 n)).
 * Later phipm_solve / phipm_solve_host calls of that class use it.  u holds the
 * last solve's result.  report (host, may be NULL) receives up to max_report
 * (team, kernel_ms) pairs in the order tried; *n_report (may be NULL) their count.
 * Errors are those of phipm_solve.
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t team;        /* CTAs cooperating on the solve (1 = one CTA)  */
  int32_t reserved;
  double kernel_ms;    /* solver kernel time of the timed solve         */
} phipm_tune_entry;
phipm_status phipm_autotune(phipm_handle* h, double t_end, const phipm_operator* A, int32_t p,
                            const double* const* b, double tol, int32_t symm, double* u,
                            phipm_tune_entry* report, int32_t max_report, int32_t* n_report, void* stream);
/* Batched counterpart: solves the batch (arguments as phipm_solve_batched) with
 * each cluster size K = 1, 2, 4, 8 that the GPU can hold (K CTAs per problem; 1 =
 * one CTA per problem), timing the second of two launches per K, and records the
 * fastest for the batch class (precision, floor(log2 count), floor(log2 of the
 * largest n)); later phipm_solve_batched calls of that class use it.  u holds the
 * last launch's results.  report / n_report as for phipm_autotune (team = K). */
phipm_status phipm_autotune_batched(phipm_handle* h, int32_t count, const double* t_end, const phipm_operator* A,
                                    const int32_t* p, const double* const* const* b, const double* tol,
                                    const int32_t* symm, double* const* u, phipm_tune_entry* report,
                                    int32_t max_report, int32_t* n_report, void* stream);
/* Force a team size for every later solve of this handle (0 = the tuned table or
 * the default; larger than the co-resident grid is clamped to it).  For
 * phipm_solve_batched the team is a thread-block cluster of up to 8 CTAs per
 * problem (1 = one CTA per problem); without a forced or tuned K the batch picks
 * 1, 2 or 4 from the share of its largest problem in the total work. */
phipm_status phipm_set_team(phipm_handle* h, int32_t team);
/* The team size a solve of this shape would use now (0 for invalid arguments). */
int32_t phipm_team_for(const phipm_handle* h, int32_t precision, int32_t kind, int32_t n);
/* CTAs per problem (the cluster size K; 1 = one CTA per problem) of the last
 * phipm_solve_batched call on this handle; 0 before the first. */
int32_t phipm_batched_team(const phipm_handle* h);
/* Save / load the tuned tables as JSON: {"sms": S, "entries": [{"precision": P,
 * "kind": K, "log2n": L, "team": G, "ms": T}, ...], "batch_entries": [{"precision": P,
 * "log2count": C, "log2nmax": L, "team": K, "ms": T}, ...]}.  Loading merges the entries
 * into the handle's table when S equals this GPU's SM count and ignores the file
 * otherwise; a file that cannot be read or parsed returns PHIPM_EINVAL and
 * changes nothing. */
phipm_status phipm_tune_save(phipm_handle* h, const char* path);
phipm_status phipm_tune_load(phipm_handle* h, const char* path);

#ifdef __cplusplus
}
#endif
#endif /* PHIPM_H */
