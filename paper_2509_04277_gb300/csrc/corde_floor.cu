// Empty-barrier floors: the cost of one synchronisation of each scope a rod kernel can
// use, measured with nothing else in the loop; and the device's FP32 FMA throughput, the
// peak the step kernels' arithmetic is measured against.  The paper's multi-block kernel pays an
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

// FP32 issue peak: every thread runs 8 independent fused multiply-add chains (enough
// independent work per warp to hide the FMA latency at a few resident warps per SMSP).
// PACKED: the chains are float2 pairs through the paired-lane FMA (__ffma2_rn), which
// does two FMAs per lane and instruction.  The values stay bounded (a < 1).
template <bool PACKED>
__global__ void fp32_peak_kernel(int n_iters, float a, float b, float* sink) {
  if constexpr (PACKED) {
    float2 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = make_float2(1e-3f * threadIdx.x + k, 2e-3f * threadIdx.x - k);
    const float2 A = make_float2(a, a), B = make_float2(b, b);
#pragma unroll 4
    for (int i = 0; i < n_iters; ++i) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = __ffma2_rn(x[k], A, B);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k].x + x[k].y;
    if (s == -1.f) *sink = s;
  } else {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1e-3f * threadIdx.x + k;
#pragma unroll 4
    for (int i = 0; i < n_iters; ++i) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == -1.f) *sink = s;
  }
}

}  // namespace

extern "C" {

int rod_device_info(int* n_sms, int* max_threads_per_sm) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && n_sms) e = cudaDeviceGetAttribute(n_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && max_threads_per_sm)
    e = cudaDeviceGetAttribute(max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return corde::set_error(CORDE_ERR_UNSUPPORTED, std::string("rod_device_info: ") + cudaGetErrorString(e));
  }
  return CORDE_OK;
}

// FP32 FMA throughput (synchronous): blocks_per_sm x (number of SMs) blocks of `threads`
// threads, each thread 8 independent FMA chains of n_iters steps (packed = 1: float2
// chains through the paired-lane FMA); one untimed launch, then one timed.
int rod_fp32_peak(int packed, int blocks_per_sm, int threads, int n_iters, double* tflops, void* stream) {
  if (!tflops || n_iters < 1 || threads < 32 || threads > 1024 || (threads & 31) || blocks_per_sm < 1 ||
      blocks_per_sm > 32 || (packed != 0 && packed != 1))
    return corde::set_error(CORDE_ERR_ARG, "rod_fp32_peak: bad sizes");
  int sms = 0;
  if (int rc = rod_device_info(&sms, nullptr)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  float* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return corde::set_error(CORDE_ERR_OOM, "rod_fp32_peak");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const dim3 grid(sms * blocks_per_sm), block(threads);
  auto launch = [&]() {
    if (packed)
      fp32_peak_kernel<true><<<grid, block, 0, s>>>(n_iters, 0.9999f, 1e-4f, sink);
    else
      fp32_peak_kernel<false><<<grid, block, 0, s>>>(n_iters, 0.9999f, 1e-4f, sink);
    return cudaGetLastError();
  };
  cudaError_t err = launch();
  if (err == cudaSuccess) err = cudaEventRecord(e0, s);
  if (err == cudaSuccess) err = launch();
  if (err == cudaSuccess) err = cudaEventRecord(e1, s);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return corde::set_error(CORDE_ERR_CUDA, std::string("rod_fp32_peak: ") + cudaGetErrorString(err));
  }
  const double flops = (double)grid.x * threads * (double)n_iters * 8.0 * (packed ? 4.0 : 2.0);
  *tflops = flops / ((double)ms * 1e-3) / 1e12;
  return CORDE_OK;
}

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
