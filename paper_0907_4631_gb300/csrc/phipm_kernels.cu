// The solver kernels and their launchers (phipm_launch.h).  The build compiles this
// file once per (basis element type, team form) pair, with
//   PM_ELEM  0: double (IEEE FP64 basis), 1: float (FP32 basis), 2: df32 (float pairs)
//   PM_FORM  0: k_solve_grid, 1: k_solve_queue, 2: k_solve_cluster,
// so that the nine solver instances compile in parallel.  Every instance runs the
// same device engine (phipm_engine.cuh) over its team.
#include "phipm_launch.h"

#if !defined(PM_ELEM) || !defined(PM_FORM)
#error "compile with -DPM_ELEM=0|1|2 -DPM_FORM=0|1|2"
#endif
#if PM_ELEM == 0
typedef double PmElemT;
#elif PM_ELEM == 1
typedef float PmElemT;
#else
typedef df32 PmElemT;
#endif

#if PM_FORM == 0
// ------------------------------------------------------------------------------------
// one problem on every CTA of a cooperative launch
// ------------------------------------------------------------------------------------
template <class S>
__global__ void __launch_bounds__(PM_THREADS, 1)
k_solve_grid(DevProblem P, DevParams prm, DevResult* res, PmWork w, unsigned long long* bar, int* err) {
  extern __shared__ __align__(16) unsigned char pm_smem[];
  PmShared& s = *reinterpret_cast<PmShared*>(pm_smem);
  GridTeam team{bar, err, prm.timeout_cycles, 0ull};
  phipm_device<GridTeam, S>(team, P, prm, *res, s, w);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int e = *((volatile int*)err);
    if (e != 0 && res->status == PM_OK) res->status = e;
  }
}

template <class S>
cudaError_t pm_grid_setup(int smem) {
  return cudaFuncSetAttribute(k_solve_grid<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
template <class S>
int pm_grid_occupancy(int smem) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve_grid<S>, PM_THREADS, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}
template <class S>
cudaError_t pm_grid_launch(int G, cudaStream_t stream, const DevProblem& P, const DevParams& prm, DevResult* res,
                           const PmWork& w, unsigned long long* bar, int* err) {
  DevProblem p = P;
  DevParams q = prm;
  PmWork ww = w;
  void* args[] = {(void*)&p, (void*)&q, (void*)&res, (void*)&ww, (void*)&bar, (void*)&err};
  return cudaLaunchCooperativeKernel((const void*)k_solve_grid<S>, dim3(G), dim3(PM_THREADS), args, sizeof(PmShared),
                                     stream);
}
template cudaError_t pm_grid_setup<PmElemT>(int);
template int pm_grid_occupancy<PmElemT>(int);
template cudaError_t pm_grid_launch<PmElemT>(int, cudaStream_t, const DevProblem&, const DevParams&, DevResult*,
                                             const PmWork&, unsigned long long*, int*);

#elif PM_FORM == 1
// ------------------------------------------------------------------------------------
// persistent CTAs pulling problems from an atomic queue
// ------------------------------------------------------------------------------------
template <class S>
__global__ void __launch_bounds__(PM_THREADS, 1)
k_solve_queue(const DevProblem* probs, const int* order, int count, DevParams prm, DevResult* res,
              unsigned char* slots, SlotLayout lay, int* queue) {
  extern __shared__ __align__(16) unsigned char pm_smem[];
  PmShared& s = *reinterpret_cast<PmShared*>(pm_smem);
  __shared__ int s_next;
  unsigned char* base = slots + (size_t)blockIdx.x * lay.bytes;
  CtaTeam team;
  PmWork w{nullptr, (double*)(base + lay.e_off)};
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
    __syncthreads();
    const int q = s_next;
    __syncthreads();
    if (q >= count) break;
    const int id = order[q];
    DevProblem P = probs[id];
    P.V = base + lay.v_off;
    P.W = (double*)(base + lay.w_off);
    P.Y = base + lay.y_off;
    P.ld = lay.ld;
    phipm_device<CtaTeam, S>(team, P, prm, res[id], s, w);
    __syncthreads();
  }
}


template <class S>
cudaError_t pm_queue_setup(int smem) {
  return cudaFuncSetAttribute(k_solve_queue<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
template <class S>
int pm_queue_occupancy(int smem) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve_queue<S>, PM_THREADS, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}
template <class S>
cudaError_t pm_queue_launch(int blocks, cudaStream_t stream, const DevProblem* probs, const int* order, int count,
                            const DevParams& prm, DevResult* res, unsigned char* slots, const SlotLayout& lay,
                            int* queue) {
  k_solve_queue<S><<<blocks, PM_THREADS, sizeof(PmShared), stream>>>(probs, order, count, prm, res, slots, lay, queue);
  return cudaGetLastError();
}
template cudaError_t pm_queue_setup<PmElemT>(int);
template int pm_queue_occupancy<PmElemT>(int);
template cudaError_t pm_queue_launch<PmElemT>(int, cudaStream_t, const DevProblem*, const int*, int, const DevParams&,
                                              DevResult*, unsigned char*, const SlotLayout&, int*);

#else
// ------------------------------------------------------------------------------------
// persistent thread-block clusters, one problem per cluster at a time
// ------------------------------------------------------------------------------------
// Batched form with a team of K CTAs per problem: each thread-block cluster is one
// team (rows split over its CTAs, reductions through per-cluster partials, barriers
// on a counter in rank 0's shared memory) and pulls problems from the atomic queue.
// Large problems of an uneven batch then get K SMs' bandwidth instead of one.
__device__ __forceinline__ unsigned pm_cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned pm_cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned pm_cluster_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void pm_cluster_arrive_wait() {   // full cluster barrier (hardware)
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
template <class T>
__device__ __forceinline__ T* pm_map_rank(T* p, unsigned rank) {   // generic address of p in CTA rank's smem
  T* q;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(q) : "l"(p), "r"(rank));
  return q;
}

template <class S>
__global__ void __launch_bounds__(PM_THREADS, 1)
k_solve_cluster(const DevProblem* probs, const int* order, int count, DevParams prm, DevResult* res,
                unsigned char* slots, SlotLayout lay, int* queue, double* partials, int* err) {
  extern __shared__ __align__(16) unsigned char pm_smem[];
  PmShared& s = *reinterpret_cast<PmShared*>(pm_smem);
  __shared__ unsigned long long s_bar;
  __shared__ int s_next;
  const unsigned rank = pm_cluster_rank(), K = pm_cluster_size(), cid = pm_cluster_id();
  if (threadIdx.x == 0) {
    s_bar = 0;
    s_next = 0;
  }
  pm_cluster_arrive_wait();            // every CTA's counter initialised before remote use
  ClusterTeam team{pm_map_rank(&s_bar, 0), err, prm.timeout_cycles, (int)rank, (int)K, 0ull};
  const int* next0 = pm_map_rank(&s_next, 0);
  unsigned char* base = slots + (size_t)cid * lay.bytes;
  PmWork w{partials + (size_t)cid * 2 * K * PM_PSTRIDE, (double*)(base + lay.e_off)};
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) s_next = atomicAdd(queue, 1);
    if (!team.sync()) break;
    const int q = *((volatile const int*)next0);
    if (!team.sync()) break;           // read before rank 0 takes the next problem
    if (q >= count) break;
    const int id = order[q];
    DevProblem P = probs[id];
    P.V = base + lay.v_off;
    P.W = (double*)(base + lay.w_off);
    P.Y = base + lay.y_off;
    P.ld = lay.ld;
    phipm_device<ClusterTeam, S>(team, P, prm, res[id], s, w);
    if (rank == 0 && threadIdx.x == 0) {
      const int e = *((volatile int*)err);
      if (e != 0 && res[id].status == PM_OK) res[id].status = e;
    }
  }
  pm_cluster_arrive_wait();            // no CTA leaves while others may still read rank 0's memory
}

static cudaLaunchConfig_t cluster_config(int K, int clusters, int smem, cudaStream_t stream, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * K));
  cfg.blockDim = dim3(PM_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)K;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}
template <class S>
cudaError_t pm_cluster_setup(int smem) {
  return cudaFuncSetAttribute(k_solve_cluster<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
template <class S>
int pm_cluster_capacity(int K, int smem) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config(K, 1, smem, nullptr, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_solve_cluster<S>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}
template <class S>
cudaError_t pm_cluster_launch(int K, int clusters, cudaStream_t stream, const DevProblem* probs, const int* order,
                              int count, const DevParams& prm, DevResult* res, unsigned char* slots,
                              const SlotLayout& lay, int* queue, double* partials, int* err) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config(K, clusters, (int)sizeof(PmShared), stream, attr);
  return cudaLaunchKernelEx(&cfg, k_solve_cluster<S>, probs, order, count, prm, res, slots, lay, queue, partials, err);
}
template cudaError_t pm_cluster_setup<PmElemT>(int);
template int pm_cluster_capacity<PmElemT>(int, int);
template cudaError_t pm_cluster_launch<PmElemT>(int, int, cudaStream_t, const DevProblem*, const int*, int,
                                                const DevParams&, DevResult*, unsigned char*, const SlotLayout&, int*,
                                                double*, int*);
#endif
