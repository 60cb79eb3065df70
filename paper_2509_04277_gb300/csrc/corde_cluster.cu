// Long rods over a thread-block cluster: the rod's elements are split over C blocks of one
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
                    int n_steps, float4* __restrict__ traj, int64_t n_elem, int C) {
  static_assert(EPT % 2 == 0, "elements per thread must be even (red-black sweeps)");
  extern __shared__ float4 smem[];
  float4* par_u = smem;
  float4* par_k = smem + EPT * NT;
  float4* halo = smem + 2 * EPT * NT;
  cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
  const int c = (int)cluster.block_rank();
  const int rid = work[blockIdx.x / C];
  const RodDev R = rods[rid];
  const int t = threadIdx.x;
  const ClusterHalo<NT> H{t, c, C};
  const int e0 = H.tg() * EPT;

  float3 r[EPT], v[EPT], om[EPT];
  float4 q[EPT];
  float w[EPT];
  load_rod<EPT, NT>(R, t, H.tg(), x4, v4, q4, o4, u4, k4, r, v, q, om, w, par_u, par_k);
  float3 v_drive = zero3(), w_drive = zero3();
  if (drive != nullptr) {
    v_drive = f3(drive[2 * rid]);
    w_drive = f3(drive[2 * rid + 1]);
  }
  int xc = 0;
  for (int step = 0; step < n_steps; ++step) {
    step_body<EPT, NT, false>(R, H, r, v, q, om, w, par_u, par_k, halo, xc, v_drive, w_drive, nullptr, nullptr);
    if (traj != nullptr) {
#pragma unroll
      for (int e = 0; e < EPT; ++e)
        if (e0 + e < R.n) traj[(int64_t)step * n_elem + R.off + e0 + e] = make_float4(r[e].x, r[e].y, r[e].z, w[e]);
    }
  }
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = e0 + e;
    if (i < R.n) {
      x4[R.off + i] = make_float4(r[e].x, r[e].y, r[e].z, w[e]);
      v4[R.off + i] = make_float4(v[e].x, v[e].y, v[e].z, 0.f);
      q4[R.off + i] = q[e];
      o4[R.off + i] = make_float4(om[e].x, om[e].y, om[e].z, 0.f);
    }
  }
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
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_rods * C);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cluster_step_kernel<EPT, NT>, a.rods, a.work, a.x4, a.v4, a.q4, a.o4, a.u4, a.k4,
                            a.drive, a.n_steps, a.traj, a.n_elem, C);
}

}  // namespace

const ClusterVariant kClusterVariants[] = {
    {2, 256, &launch_cluster_t<2, 256>},
    {4, 256, &launch_cluster_t<4, 256>},
    {4, 512, &launch_cluster_t<4, 512>},
};
const int kNumClusterVariants = 3;

}  // namespace corde
