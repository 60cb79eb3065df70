// Empty-barrier floors: the cost of one synchronisation of each scope a rod kernel can
// use, measured with nothing else in the loop.  The paper's multi-block kernel pays an
// inter-block barrier per exchange (Section 2.2, Fig. 5); these floors are what a
// persistent step kernel's latency per step is compared against.
#include <cooperative_groups.h>

#include <string>

#include "../../include/corde.h"
#include "corde_variants.cuh"

namespace cg = cooperative_groups;

namespace {

__global__ void floor_block(int n_iters, int* sink) {
  int acc = 0;
  for (int i = 0; i < n_iters; ++i) {
    __syncthreads();
    acc += i;
  }
  if (threadIdx.x == 0 && acc == -1) *sink = acc;
}

__global__ void floor_warp(int n_iters, int* sink) {
  int acc = 0;
  for (int i = 0; i < n_iters; ++i) {
    __syncwarp();
    acc += i;
  }
  if (threadIdx.x == 0 && acc == -1) *sink = acc;
}

__global__ void floor_cluster(int n_iters, int* sink) {
  cg::cluster_group cl = cg::this_cluster();
  int acc = 0;
  for (int i = 0; i < n_iters; ++i) {
    cl.sync();
    acc += i;
  }
  if (threadIdx.x == 0 && acc == -1) *sink = acc;
}

__global__ void floor_grid(int n_iters, int* sink) {
  cg::grid_group g = cg::this_grid();
  int acc = 0;
  for (int i = 0; i < n_iters; ++i) {
    g.sync();
    acc += i;
  }
  if (threadIdx.x == 0 && acc == -1) *sink = acc;
}

}  // namespace

extern "C" {

// Empty-barrier floor (synchronous): ns per barrier over n_iters back-to-back barriers
// in one launch, minus nothing (the launch overhead is amortised by n_iters).
//  scope 0: __syncthreads in one block of `threads` threads;
//  scope 1: __syncwarp in one warp;
//  scope 2: cluster barrier over a cluster of `cluster` blocks of `threads` threads;
//  scope 3: cooperative grid sync over `cluster` blocks per SM on every SM (cooperative
//           launch: co-residency is checked by the runtime, the launch fails otherwise).
int rod_barrier_floor(int scope, int threads, int cluster, int n_iters, double* ns_per_barrier, void* stream) {
  if (!ns_per_barrier || n_iters < 1 || threads < 1 || threads > 1024 || cluster < 1 || cluster > 16 ||
      scope < 0 || scope > 3)
    return corde::set_error(CORDE_ERR_ARG, "rod_barrier_floor: bad scope or sizes");
  cudaStream_t s = (cudaStream_t)stream;
  int* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(int)) != cudaSuccess) return corde::set_error(CORDE_ERR_OOM, "rod_barrier_floor");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t err = cudaSuccess;
  auto run = [&](bool timed) -> cudaError_t {
    if (timed) cudaEventRecord(e0, s);
    cudaError_t e = cudaSuccess;
    if (scope == 0) {
      floor_block<<<1, threads, 0, s>>>(n_iters, sink);
      e = cudaGetLastError();
    } else if (scope == 1) {
      floor_warp<<<1, 32, 0, s>>>(n_iters, sink);
      e = cudaGetLastError();
    } else if (scope == 2) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cluster);
      cfg.blockDim = dim3(threads);
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cluster;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      if (cluster > 8) {
        e = cudaFuncSetAttribute(floor_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
      }
      e = cudaLaunchKernelEx(&cfg, floor_cluster, n_iters, sink);
    } else {
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      void* args[] = {&n_iters, &sink};
      e = cudaLaunchCooperativeKernel((void*)floor_grid, dim3(sms * cluster), dim3(threads), args, 0, s);
    }
    if (timed) cudaEventRecord(e1, s);
    return e;
  };
  err = run(false);
  if (err == cudaSuccess) err = run(true);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return corde::set_error(CORDE_ERR_CUDA, std::string("rod_barrier_floor: ") + cudaGetErrorString(err));
  }
  *ns_per_barrier = (double)ms * 1e6 / n_iters;
  return CORDE_OK;
}

}  // extern "C"
