// Long rods over a thread-block cluster (and, beyond what a cluster holds, over a
// cooperative grid): the rod's elements are split over C blocks of one
// cluster (block c holds threads c NT ... c NT + NT - 1 of the rod), the per-step
// exchanges of the first and last element of each block read the neighbouring block's
// exchange buffer through distributed shared memory, and every exchange barrier is a
// cluster barrier.  This is the GB300 form of the paper's multi-block kernel (Section 2.2:
// the rod spread over several SMs, inter-block synchronisation at each data exchange,
// border elements exchanged between blocks; Fig. 5): the cluster barrier is a hardware
// barrier over co-scheduled blocks, so no global-memory spin counter is needed, and the
// halo stays on chip.
#include <cooperative_groups.h>

#include "corde_step.cuh"
#include "corde_variants.cuh"

namespace corde {
namespace {

template <int EPT, int NT>
__global__ void __launch_bounds__(NT)
cluster_step_kernel(const RodDev* __restrict__ rods, const int* __restrict__ work, float4* __restrict__ x4,
                    float4* __restrict__ v4, float4* __restrict__ q4, float4* __restrict__ o4,
                    const float4* __restrict__ u4, const float4* __restrict__ k4, const float4* __restrict__ drive,
                    int n_steps, float4* __restrict__ traj, int64_t n_elem, int C, MailboxDev mb,
                    float4* __restrict__ pos_out) {
  static_assert(EPT % 2 == 0, "elements per thread must be even (red-black sweeps)");
  extern __shared__ float4 smem[];
  pdl_begin();
  cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
  const int c = (int)cluster.block_rank();
  const int rid = work[blockIdx.x / C];
  const RodDev R = rods[rid];
  const ClusterHalo<NT> H{(int)threadIdx.x, c, C};
  run_rod<EPT, NT>(R, H, rid, x4, x4, v4, q4, o4, u4, k4, drive, n_steps, traj, n_elem, mb, smem, pos_out);
  // no block leaves while a neighbour may still read its exchange buffer
  cluster.sync();
}

template <int EPT, int NT>
cudaError_t launch_cluster_t(const StepArgs& a, int n_rods, int C, cudaStream_t s) {
  constexpr int smem = step_smem_bytes<EPT, NT>();
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(cluster_step_kernel<EPT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  if (C > 8) {
    cudaError_t e = cudaFuncSetAttribute(cluster_step_kernel<EPT, NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  return launch_kernel(cluster_step_kernel<EPT, NT>, dim3(n_rods * C), dim3(NT), smem, s, a.pdl, C, a.rods, a.work,
                       a.x4, a.v4, a.q4, a.o4, a.u4, a.k4, a.drive, a.n_steps, a.traj, a.n_elem, C, a.mb, a.pos_out);
}

// The same rod spread over C blocks of a cooperative grid (rods longer than a cluster
// holds): GridHalo publishes each block's edge slots in global memory (gh: per rod
// 2 x C x kHaloSlots x 2 float4) and synchronises with grid syncs.  Several rods can share
// a launch (block b holds block b % C of rod work[b / C]); every grid sync then spans
// them all, which only keeps them in step.
template <int EPT, int NT>
__global__ void __launch_bounds__(NT)
grid_step_kernel(const RodDev* __restrict__ rods, const int* __restrict__ work, float4* __restrict__ x4,
                 float4* __restrict__ v4, float4* __restrict__ q4, float4* __restrict__ o4,
                 const float4* __restrict__ u4, const float4* __restrict__ k4, const float4* __restrict__ drive,
                 int n_steps, float4* __restrict__ traj, int64_t n_elem, int C, float4* __restrict__ gh,
                 MailboxDev mb, float4* __restrict__ pos_out) {
  static_assert(EPT % 2 == 0, "elements per thread must be even (red-black sweeps)");
  extern __shared__ float4 smem[];
  const int k = blockIdx.x / C, c = blockIdx.x - k * C;
  const int rid = work[k];
  const RodDev R = rods[rid];
  const GridHalo<NT> H{(int)threadIdx.x, c, C, gh + (size_t)k * 2 * C * kHaloSlots * 2, smem + 2 * EPT * NT};
  run_rod<EPT, NT>(R, H, rid, x4, x4, v4, q4, o4, u4, k4, drive, n_steps, traj, n_elem, mb, smem, pos_out);
}

template <int EPT, int NT>
cudaError_t launch_grid_t(const StepArgs& a, int n_rods, int C, cudaStream_t s) {
  constexpr int smem = step_smem_bytes<EPT, NT>();
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(grid_step_kernel<EPT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_rods * C);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, grid_step_kernel<EPT, NT>, a.rods, a.work, a.x4, a.v4, a.q4, a.o4, a.u4, a.k4,
                            a.drive, a.n_steps, a.traj, a.n_elem, C, a.grid_halo, a.mb, a.pos_out);
}

// Blocks of grid_step_kernel<EPT, NT> resident on the whole device at once (occupancy API
// x SMs): the largest cooperative grid it can launch.
template <int EPT, int NT>
int grid_blocks_t() {
  constexpr int smem = step_smem_bytes<EPT, NT>();
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(grid_step_kernel<EPT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grid_step_kernel<EPT, NT>, NT, smem) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * sms;
}

}  // namespace

const ClusterVariant kClusterVariants[] = {
    {2, 256, &launch_cluster_t<2, 256>, &launch_grid_t<2, 256>, &grid_blocks_t<2, 256>},
    {4, 256, &launch_cluster_t<4, 256>, &launch_grid_t<4, 256>, &grid_blocks_t<4, 256>},
    {4, 512, &launch_cluster_t<4, 512>, &launch_grid_t<4, 512>, &grid_blocks_t<4, 512>},
};
const int kNumClusterVariants = 3;

}  // namespace corde
