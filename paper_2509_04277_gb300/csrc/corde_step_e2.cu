// Step-kernel instantiations with 2 elements per thread.
#include "corde_step.cuh"
#include "corde_variants.cuh"

namespace corde {

template <int EPT, int NT>
static cudaError_t launch_step(const StepArgs& a, int n_blocks, cudaStream_t s) {
  constexpr int smem = step_smem_bytes<EPT, NT>();
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(step_kernel<EPT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  return launch_kernel(step_kernel<EPT, NT>, dim3(n_blocks), dim3(NT), smem, s, a.pdl, 0, a.rods, a.work, a.x4,
                       a.v4, a.q4, a.o4, a.u4, a.k4, a.drive, a.n_steps, a.traj, a.n_elem, a.mb, a.pos_out);
}

template <int EPT, int NT>
static cudaError_t preload_step() {
  cudaFuncAttributes at;
  return cudaFuncGetAttributes(&at, step_kernel<EPT, NT>);
}

#define V(NT) {2, NT, step_smem_bytes<2, NT>(), &launch_step<2, NT>, &preload_step<2, NT>}
const StepVariant kStepVariantsE2[] = {V(32), V(64), V(128), V(256), V(512)};
#undef V
const int kNumStepVariantsE2 = 5;

}  // namespace corde
