// Launchers of the solver kernels.  The kernels (phipm_kernels.cu) are compiled
// once per (basis element type, team form) in separate translation units, so the
// library builds in parallel; the C ABI (phipm_capi.cu) reaches them only through
// the functions declared here, each explicitly instantiated for S = double, float
// and df32 in the translation unit that holds its kernel.
//
// Team forms: a cooperative grid of G CTAs on one problem (k_solve_grid); a
// persistent CTA per queue slot pulling problems largest first (k_solve_queue);
// a K-CTA thread-block cluster per queue slot (k_solve_cluster).
#pragma once
#include <cuda_runtime.h>

#include "phipm_engine.cuh"

// Workspace of one queue slot (one CTA or one cluster): V, W, Y and the exponential scratch.
struct SlotLayout {
  long long ld;                          // vector stride (elements)
  long long v_off, w_off, y_off, e_off;  // byte offsets inside the slot
  long long bytes;                       // bytes per slot (multiple of 256)
};

// Allow sizeof(PmShared) bytes of dynamic shared memory for the kernel.
template <class S> cudaError_t pm_grid_setup(int smem);
template <class S> cudaError_t pm_queue_setup(int smem);
template <class S> cudaError_t pm_cluster_setup(int smem);

// CTAs of the kernel resident per SM (0 on error).
template <class S> int pm_grid_occupancy(int smem);
template <class S> int pm_queue_occupancy(int smem);
// Co-resident clusters of K CTAs (0 when the GPU cannot hold one).
template <class S> int pm_cluster_capacity(int K, int smem);

// Cooperative launch of G CTAs on problem P (bar: arrival counter, zero; err: error word, zero).
template <class S>
cudaError_t pm_grid_launch(int G, cudaStream_t stream, const DevProblem& P, const DevParams& prm, DevResult* res,
                           const PmWork& w, unsigned long long* bar, int* err);
// Persistent queue: `blocks` CTAs take problems order[0..count) from the counter *queue (zero).
template <class S>
cudaError_t pm_queue_launch(int blocks, cudaStream_t stream, const DevProblem* probs, const int* order, int count,
                            const DevParams& prm, DevResult* res, unsigned char* slots, const SlotLayout& lay,
                            int* queue);
// Persistent queue of `clusters` teams of K CTAs (partials: 2 K PM_PSTRIDE doubles per team).
template <class S>
cudaError_t pm_cluster_launch(int K, int clusters, cudaStream_t stream, const DevProblem* probs, const int* order,
                              int count, const DevParams& prm, DevResult* res, unsigned char* slots,
                              const SlotLayout& lay, int* queue, double* partials, int* err);
