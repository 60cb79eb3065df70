// Device-side data structures and small vector/quaternion helpers of the CoRdE stepper.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace corde {

enum : int { F_INEXT = 1, F_CLAMP = 2 };

// Per-rod constants used by the step kernel (derived once at creation, FP64 -> FP32).
struct RodDev {
  int off;      // first global element of the rod
  int n;        // nodes N
  int flags;    // F_INEXT | F_CLAMP
  int n_iters;  // constraint iterations per step
  float dt, l0, two_over_l, lKp;  // time step, rest length, 2 / l_j, l0 * Kp
  float Ks, inv_l0, damp, pad0;   // stretch stiffness, 1 / l0, 1 / (1 + alpha dt)
  float gx, gy, gz, pad1;         // gravity acceleration of a dynamic node (g / mass_scale)
  float J1, J3, Jinv1, Jinv3;     // inertial frame inertia diag (J1, J1, J3) and inverses
};
static_assert(sizeof(RodDev) == 80, "RodDev layout");

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
