// Registry of the compiled step-kernel variants (elements per thread x threads per block).
#pragma once

#include <string>

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
};

typedef cudaError_t (*StepLaunchFn)(const StepArgs& a, int n_blocks, cudaStream_t s);

struct StepVariant {
  int ept;
  int nt;
  int smem_bytes;
  StepLaunchFn launch;
  int capacity() const { return ept * nt; }
};

// Defined in the per-EPT instantiation units.
extern const StepVariant kStepVariantsE2[];
extern const int kNumStepVariantsE2;
extern const StepVariant kStepVariantsE4[];
extern const int kNumStepVariantsE4;

}  // namespace corde
