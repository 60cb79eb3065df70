// Registry of the compiled step-kernel variants (elements per thread x threads per block).
#pragma once

#include <string>
#include <utility>

#include "corde_common.cuh"

namespace corde {

// Records the message returned by rod_last_error() and passes the code through.
int set_error(int code, const std::string& msg);

struct StepArgs {
  const RodDev* rods;
  const int* work;
  float4 *x4, *v4, *q4, *o4;
  const float4 *u4, *k4;
  const float4* drive;
  int n_steps;
  float4* traj;    // optional: positions after every step, [n_steps][n_elem]
  int64_t n_elem;
  MailboxDev mb;   // mailbox of the launch (period 0: none)
  int4* self_stats;  // self-collision statistics per rod (corde_self.cu), or NULL
  unsigned char* self_skin;  // self-collision skin lists kept between launches (corde_self.cu), or NULL
  float4* pos_out;   // optional: positions (r, w) after the launch, [n_elem] (device or mapped host)
  float4* grid_halo; // rods on a cooperative grid: their global exchange slots
  int pdl;           // 1: launch with programmatic stream serialisation (the kernel may start
                     // before the stream's previous kernel ends; it waits in pdl_begin)
};

// Launches kernel<<<grid, block, smem, s>>>(args...), with the programmatic-serialisation
// attribute when pdl != 0 and as clusters of `cluster` blocks along x when cluster > 0.
template <class... KArgs, class... Args>
cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, int smem, cudaStream_t s, int pdl,
                          int cluster, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  int na = 0;
  if (pdl) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (cluster > 0) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = (unsigned)cluster;
    at[na].val.clusterDim.y = 1;
    at[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = (unsigned)na;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

typedef cudaError_t (*StepLaunchFn)(const StepArgs& a, int n_blocks, cudaStream_t s);
// Loads the variant's kernel into the current context now (cudaFuncGetAttributes), so
// that its first launch does not load the module (lazy loading takes device memory).
typedef cudaError_t (*StepPreloadFn)();

struct StepVariant {
  int ept;
  int nt;
  int smem_bytes;
  StepLaunchFn launch;
  StepPreloadFn preload;
  int capacity() const { return ept * nt; }
};

// Arguments of the reverse (adjoint) kernel; see corde_adjoint.cu.
struct AdjointArgs {
  const RodDev* rods;
  const int* work;
  const float4* ckpt;    // [n_ckpt][4][n_elem]: x4, v4, q4, o4 at steps 0, K, 2K, ...
  float4* seg_states;    // scratch [K][4][n_elem]
  const float4 *u4, *k4;
  const float4* drive;
  const float4* dLdpos;  // [n_steps][n_elem] or NULL
  int n_steps, ckpt_every;
  int64_t n_elem;
  float4 *dpos0, *dvel0, *dquat0, *domega0, *dK, *duhat;
  // Record mode (sweep_rec != NULL): the first pass over a checkpoint segment keeps, per
  // step and block, the velocities before every constraint half-sweep (compact layout:
  // before the first even and every odd one) (sweep_rec[(s gridDim + b) slots 3 EPT NT / 4
  // ...] float4, 2 rec_iters or rec_iters + 1 slots), and seg_states holds K + 1 states
  // (positions, frames and angular velocities: the neighbour data of each step comes
  // from them); the reverse pass then reads them instead of recomputing each step.  NULL:
  // recompute mode.
  float4* sweep_rec = nullptr;
  int rec_iters = 0;
};
// Reverse-kernel modes: 0 recompute; 1 record, one sweep buffer (the copy of a step's
// records waits for the reverse of the step after it); 2 record, two sweep buffers (the
// copy overlaps that reverse).  compact: 1 + n_iters record slots per step instead of
// 2 n_iters (the adjoint rebuilds the inputs of the later even half-sweeps: less memory
// traffic and shared memory, a longer reverse).  All give the same gradients.
// Shared memory of the reverse kernel: parameters, exchange buffers and one (modes 0, 1)
// or two (mode 2) sweep-velocity buffers.
int adjoint_smem_bytes(int nt, int n_iters, int mode = 0, bool compact = false);
// mode > 0 exactly when a.sweep_rec is set (cudaErrorInvalidValue otherwise).
cudaError_t launch_adjoint(int nt, int mode, bool compact, const AdjointArgs& a, int n_blocks, int smem,
                           cudaStream_t s);
// Loads the recompute-mode reverse kernels of `nt` threads (both layouts) into the
// current context.
cudaError_t preload_adjoint(int nt);
// Resident blocks per SM of the reverse kernel of `nt` threads with `smem` bytes of
// dynamic shared memory (occupancy API).
cudaError_t adjoint_occupancy(int nt, int mode, bool compact, int smem, int* blocks);
// The pipelined reverse kernel (record mode, two sweep buffers, full layout): a cluster of
// two blocks per rod (grid 2 n_rods), the first recording the checkpoint segments and the
// second reversing them one segment behind.  Its scratch is twice record mode's: segment
// states and records in two sets, by segment parity.  smem should keep one block per SM.
cudaError_t launch_adjoint_pipe(int nt, const AdjointArgs& a, int n_rods, int smem, cudaStream_t s);
constexpr int kAdjointMaxNodes = 512;

// Rods with self-collision (corde_self.cu): one rod per block, at most 1024 nodes.
extern const StepVariant kSelfVariants[];
extern const int kNumSelfVariants;
constexpr int kSelfMaxNodes = 1024;
// Bytes per rod of StepArgs::self_skin: a rod's skin list kept between launches (rods in
// blocks of up to 512 nodes); its first int is the valid flag, cleared to discard it.
extern const int kSelfSkinBytes;

// Catheter/guidewire pairs (corde_pair.cu): pairs[i] = (outer rod, inner rod, mode, 0);
// ept in {2, 4}, nt (threads per rod) in {32, ..., 256}.
cudaError_t launch_pair(int ept, int nt, const StepArgs& a, const int4* pairs, int n_pairs, cudaStream_t s);

// Long rods over a thread-block cluster (corde_cluster.cu): C blocks of NT threads, EPT
// elements per thread, one rod per cluster; launch(args, n_rods, C, stream).
typedef cudaError_t (*ClusterLaunchFn)(const StepArgs& a, int n_rods, int C, cudaStream_t s);
struct ClusterVariant {
  int ept;
  int nt;
  ClusterLaunchFn launch;       // a cluster of C blocks per rod
  ClusterLaunchFn launch_grid;  // C blocks per rod in a cooperative grid (a.grid_halo: the rods'
                                // global exchange slots, 2 x C x kHaloSlots x 2 float4 per rod)
  int (*grid_blocks)();         // the most blocks a cooperative grid of this variant can hold
  int capacity(int C) const { return ept * nt * C; }
};
extern const ClusterVariant kClusterVariants[];
extern const int kNumClusterVariants;
constexpr int kMaxCluster = 16;

// Defined in the per-EPT instantiation units.
extern const StepVariant kStepVariantsE2[];
extern const int kNumStepVariantsE2;
extern const StepVariant kStepVariantsE4[];
extern const int kNumStepVariantsE4;

}  // namespace corde
