// Device-side data structures and small vector/quaternion helpers of the CoRdE stepper.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace corde {

enum : int { F_INEXT = 1, F_CLAMP = 2, F_TUBE = 4, F_SELF = 8 };
constexpr int kHaloSlots = 3;  // neighbour-exchange slots per thread and exchange
constexpr int kPosSlots = 4;  // ring of position snapshots per rod (mailbox)

// Per-rod constants used by the step kernel (derived once at creation, FP64 -> FP32).
struct RodDev {
  int off;      // first global element of the rod
  int n;        // nodes N
  int flags;    // F_INEXT | F_CLAMP | F_TUBE | F_SELF
  int n_iters;  // constraint iterations per step
  float dt, l0, two_over_l, lKp;  // time step, rest length, 2 / l_j, l0 * Kp
  float Ks, inv_l0, damp, self_dist;  // stretch stiffness, 1 / l0, 1 / (1 + alpha dt), 2 r
  float gx, gy, gz, self_reach;       // gravity acceleration of a dynamic node (g / mass_scale), 3 r
  float J1, J3, Jinv1, Jinv3;     // inertial frame inertia diag (J1, J1, J3) and inverses
  float tube_cx, tube_cy, tube_cz, tube_rc;  // vessel centreline: circle in the plane z = cz
  float tube_allow, tube_mu, self_mu, self_sep;  // inner radius minus rod radius, Coulomb friction;
                                                 // self-contact friction, smallest index gap
};
static_assert(sizeof(RodDev) == 112, "RodDev layout");

// Mailbox of a running launch, in mapped pinned host memory (Section 2.2: the haptic thread
// writes the device state into the running kernel and reads the feedback back at a rate
// higher than the kernel launches).  Disabled when period == 0.
//  in_seq / in_drive: seqlock word and [n_rods][8] drive rows written by the host;
//  out: [n_rods][2] records of 8 words (seq, step, x, y, z, vx, vy, vz): record 0 the
//       base node, record 1 the tip node, each under its own seqlock;
//  log: (global step, input seq) of every input a rod picked up, *log_count entries;
//  pos_seq / pos (optional): position snapshots published every period steps into a ring of
//       kPosSlots slots per rod: pos_seq[rid][32] words = (publications, _, _, _) then per
//       slot (_, step low, step high, _); pos[slot][n_elem] = (x, y, z, inverse mass).  A
//       slot is rewritten only after the count that retires it is visible.
struct MailboxDev {
  const unsigned* in_seq;
  const float* in_drive;
  unsigned* out;
  int2* log;
  int* log_count;
  int log_cap;
  int period;
  long long step0;  // global index of the launch's first step
  unsigned* pos_seq;
  float4* pos;
  long long n_elem;  // elements of the handle (slot stride of pos)
  // lock-step (single-block rods): at every poll point wait for a new input, at most
  // wait_ns of GPU time; a wait that runs out sets bit 0 of *status and ends the launch
  int lockstep;
  unsigned* status;
  unsigned long long wait_ns;
};

// System-scope loads/stores/fences for memory shared with the host while a kernel runs.
__device__ __forceinline__ unsigned ld_acquire_sys(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.sys.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_sys(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.sys.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ float ld_relaxed_sys_f(const float* p) {
  float v;
  asm volatile("ld.relaxed.sys.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_sys(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.sys.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys(unsigned* p, unsigned v) {
  asm volatile("st.release.sys.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_sys() { asm volatile("fence.acq_rel.sys;" ::: "memory"); }
// One 16-byte volatile store (system-visible, like the component-wise volatile stores it
// replaces: one transaction across the CPU-GPU link instead of four).
__device__ __forceinline__ void st_volatile_f4(float4* p, float4 v) {
  asm volatile("st.volatile.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Programmatic dependent launch.  A stepping kernel starts with this: it lets the stream's
// next kernel be scheduled at once (that kernel only starts its own prologue early), then
// waits until the stream's previous kernel has completed and its writes are visible.  Every
// global access of the kernel comes after the wait, so the result does not depend on
// whether the launch carried the programmatic-serialisation attribute (without it the wait
// returns at once).
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------- float3 helpers

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3& operator+=(float3& a, float3 b) { a = a + b; return a; }
__device__ __forceinline__ float3& operator-=(float3& a, float3 b) { a = a - b; return a; }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 zero3() { return f3(0.f, 0.f, 0.f); }

// ---------------------------------------------------------------- quaternions (x, y, z, w)

// Vector part of conj(a) (x) b: the relative rotation of frame b seen from frame a.
__device__ __forceinline__ float3 im_conj_mul(float4 a, float4 b) {
  return f3(a.w * b.x - a.x * b.w - a.y * b.z + a.z * b.y,
            a.w * b.y - a.y * b.w - a.z * b.x + a.x * b.z,
            a.w * b.z - a.z * b.w - a.x * b.y + a.y * b.x);
}

// Third director d3 = R(q) e_z of a unit quaternion.
__device__ __forceinline__ float3 director3(float4 q) {
  return f3(2.f * (q.x * q.z + q.w * q.y), 2.f * (q.y * q.z - q.w * q.x), 1.f - 2.f * (q.x * q.x + q.y * q.y));
}

// R(q)^T v for a unit quaternion (world -> body).
__device__ __forceinline__ float3 rotate_inv(float4 q, float3 v) {
  const float3 u = f3(q.x, q.y, q.z);
  const float3 uxv = cross3(u, v);
  const float3 t = uxv - q.w * v;
  return v + 2.f * cross3(u, t);
}

// Discrete Darboux vector u = (2 / l) Im(conj(qa) (x) qb) (Eq. 5-6 with the B_k reading).
__device__ __forceinline__ float3 darboux(float4 qa, float4 qb, float two_over_l) {
  return two_over_l * im_conj_mul(qa, qb);
}

}  // namespace corde
