// Persistent multi-step CoRdE kernel: one thread block per rod, EPT consecutive
// elements per thread kept in registers for the whole launch (Section 2.2: the state is
// loaded once per launch and many time steps run before it is written back).
//
// Per time step, in the order of Fig. 5:
//   1. exchange: each thread publishes its first element's (r, w, q) to its left and its
//      last element's (r, w) to its right neighbour;
//   2. elastic forces and torques of the joints and segments the thread owns (bend and
//      twist, Eq. 3 with Eq. 5-6; penalty, Eq. 8; stretch, Eq. 2 for extensible rods);
//      the contribution of a thread's last joint / segment to the right neighbour's
//      first element is carried over in a second exchange;
//   3. force integration: v += dt (F / m~ + g / mass_scale), omega += dt J~^-1 (tau -
//      omega x J~ omega), implicit Rayleigh damping; the kinematic base takes the drive;
//   4. n_iters iterations of red-black distance-constraint impulses (inextensible
//      variant, Section 2.1 "Constraints"): the even segments of a thread are local
//      (EPT is even and every thread starts on an even element); the odd sweep needs one
//      exchange (boundary velocities) for the segment crossing each thread boundary;
//   5. integration of the velocities: r += dt v, q <- normalize(q + dt/2 q (x) (0, omega))
//      (the frames' update needs only omega, final after step 3, so it runs before the
//      sweeps of step 4 and fills their latency).
// A step costs 2 + n_iters block barriers (the paper's single-block kernel uses two
// __syncthreads per constraint iteration, one thread per element).  Neighbour data moves
// through a ping-pong pair of shared-memory buffers, so one barrier per exchange suffices.
//
// The step body is a device function shared by the forward kernel and the adjoint's
// recomputation, so both run the same arithmetic.
#pragma once

#include <cooperative_groups.h>
#include <type_traits>

#include "corde_common.cuh"

namespace corde {

template <int NT>
__device__ __forceinline__ void block_sync() {
  if constexpr (NT == 32) {
    __syncwarp();
  } else {
    __syncthreads();
  }
}

// Neighbour access and barrier of a rod held by one thread block (t = thread of the rod;
// SYNC_NT threads take part in each barrier: NT, or more when several rods share the block
// in lockstep).  Exchange buffers hold `slots` x NT float4, slot-major.  PAIR2 selects the
// layout of the three-float slots (see put3).
template <int NT, int SYNC_NT, bool PAIR2 = false>
struct BlockHalo {
  static constexpr bool kCluster = false;
  int t;
  __device__ __forceinline__ int tg() const { return t; }
  __device__ __forceinline__ int rod_threads() const { return NT; }
  __device__ __forceinline__ bool has_next() const { return t + 1 < NT; }
  __device__ __forceinline__ bool has_prev() const { return t > 0; }
  __device__ __forceinline__ float4 next(const float4* hb, int slot) const { return hb[slot * NT + t + 1]; }
  __device__ __forceinline__ float4 prev(const float4* hb, int slot) const { return hb[slot * NT + t - 1]; }
  // three-float slots, one float per component (component c of slot s at float
  // (3 s + c) NT + t): a neighbour's vector is three 32-bit loads, issued together.  With
  // PAIR2 the x and y components sit together as a float2 (float2 3 s NT / 2 + t) and z
  // at float (3 s + 2) NT + t: two loads instead of three (measured: 2.96 against 3.01
  // us/step for the 512-node rod at two elements per thread; the four-element batch
  // variants keep three, 1.6 % faster for them)
  __device__ __forceinline__ void put3(float4* hb, int slot, float3 a) const {
    float* f = reinterpret_cast<float*>(hb) + 3 * slot * NT;
    if constexpr (PAIR2) {
      f[2 * t] = a.x;  // two 32-bit stores: no register pair to form on the way to the barrier
      f[2 * t + 1] = a.y;
      f[2 * NT + t] = a.z;
    } else {
      f[t] = a.x;
      f[NT + t] = a.y;
      f[2 * NT + t] = a.z;
    }
  }
  __device__ __forceinline__ float3 get3(const float4* hb, int slot, int u) const {
    const float* f = reinterpret_cast<const float*>(hb) + 3 * slot * NT;
    if constexpr (PAIR2) {
      const float2 xy = reinterpret_cast<const float2*>(f)[u];
      return f3(xy.x, xy.y, f[2 * NT + u]);
    } else {
      return f3(f[u], f[NT + u], f[2 * NT + u]);
    }
  }
  __device__ __forceinline__ float3 next3(const float4* hb, int slot) const { return get3(hb, slot, t + 1); }
  __device__ __forceinline__ float3 prev3(const float4* hb, int slot) const { return get3(hb, slot, t - 1); }
  __device__ __forceinline__ void sync() const { block_sync<SYNC_NT>(); }
  // a barrier in two halves (arrive after the exchange stores, wait before the neighbour
  // loads); one block has no split barrier, so the wait is the whole barrier
  __device__ __forceinline__ void arrive(const float4*) const {}
  __device__ __forceinline__ void wait() const { block_sync<SYNC_NT>(); }
  // block-wide OR of x (a barrier)
  __device__ __forceinline__ int any(int x) const {
    if constexpr (SYNC_NT == 32) {
      return __any_sync(0xffffffffu, x);
    } else {
      return __syncthreads_or(x);
    }
  }
};

// A rod spread over the C thread blocks of a cluster (block c holds threads c NT ...
// c NT + NT - 1 of the rod): the neighbours of a block's first and last thread live in
// the adjacent blocks, whose exchange buffers are read through distributed shared
// memory; the barrier is the cluster barrier (release / acquire).
template <int NT>
struct ClusterHalo {
  static constexpr bool kCluster = true;
  int t, c, C;
  __device__ __forceinline__ int tg() const { return c * NT + t; }
  __device__ __forceinline__ int rod_threads() const { return C * NT; }
  __device__ __forceinline__ bool has_next() const { return t + 1 < NT || c + 1 < C; }
  __device__ __forceinline__ bool has_prev() const { return t > 0 || c > 0; }
  __device__ __forceinline__ float4 next(const float4* hb, int slot) const {
    if (t + 1 < NT) return hb[slot * NT + t + 1];
    const float4* remote = cooperative_groups::this_cluster().map_shared_rank(hb, c + 1);
    return remote[slot * NT];
  }
  __device__ __forceinline__ float4 prev(const float4* hb, int slot) const {
    if (t > 0) return hb[slot * NT + t - 1];
    const float4* remote = cooperative_groups::this_cluster().map_shared_rank(hb, c - 1);
    return remote[slot * NT + NT - 1];
  }
  // three-float slots: whole float4 slots here (one remote access per vector)
  __device__ __forceinline__ void put3(float4* hb, int slot, float3 a) const {
    hb[slot * NT + t] = make_float4(a.x, a.y, a.z, 0.f);
  }
  __device__ __forceinline__ float3 next3(const float4* hb, int slot) const { return f3(next(hb, slot)); }
  __device__ __forceinline__ float3 prev3(const float4* hb, int slot) const { return f3(prev(hb, slot)); }
  __device__ __forceinline__ void sync() const { cooperative_groups::this_cluster().sync(); }
  // OR of x over the rod's threads on all C blocks (a block-wide OR, each block's result
  // in its shared memory, read by every thread through distributed shared memory between
  // two cluster barriers)
  __device__ __forceinline__ int any(int x) const {
    __shared__ int block_or;
    const int b = __syncthreads_or(x);
    if (t == 0) block_or = b;
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    cl.sync();
    int r = 0;
    for (int k = 0; k < C; ++k) r |= *cl.map_shared_rank(&block_or, k);
    cl.sync();
    return r;
  }
  // the cluster barrier in two halves: thread-local work between them overlaps its latency
  __device__ __forceinline__ void arrive(const float4*) const {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  }
  __device__ __forceinline__ void wait() const { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
};

// A rod spread over C blocks of a cooperative grid (block c holds threads c NT ...
// c NT + NT - 1 of the rod): the paper's multi-block "universal" kernel for rods longer
// than one cluster holds.  Each block's first and last thread also publish their exchange
// slots in global memory (a ping-pong pair per exchange parity), the barrier is a grid
// sync, and a block's edge thread reads its neighbour block's slots from L2 (ld.cg, past
// any stale L1 line).  The runtime launches the grid only if all its blocks are resident
// at once, so the grid sync cannot wait on a block that never runs.
template <int NT>
struct GridHalo {
  static constexpr bool kCluster = true;
  int t, c, C;
  float4* gh;           // this rod's slots: [2 parities][C blocks][kHaloSlots][first, last]
  const float4* halo0;  // the block's shared exchange buffer of parity 0
  __device__ __forceinline__ int tg() const { return c * NT + t; }
  __device__ __forceinline__ int rod_threads() const { return C * NT; }
  __device__ __forceinline__ bool has_next() const { return t + 1 < NT || c + 1 < C; }
  __device__ __forceinline__ bool has_prev() const { return t > 0 || c > 0; }
  __device__ __forceinline__ float4* gslot(const float4* hb, int blk, int slot, int edge) const {
    const int par = hb != halo0 ? 1 : 0;
    return gh + (((par * C + blk) * kHaloSlots + slot) * 2 + edge);
  }
  __device__ __forceinline__ float4 next(const float4* hb, int slot) const {
    if (t + 1 < NT) return hb[slot * NT + t + 1];
    return __ldcg(gslot(hb, c + 1, slot, 0));
  }
  __device__ __forceinline__ float4 prev(const float4* hb, int slot) const {
    if (t > 0) return hb[slot * NT + t - 1];
    return __ldcg(gslot(hb, c - 1, slot, 1));
  }
  // three-float slots: whole float4 slots here (one global access per vector)
  __device__ __forceinline__ void put3(float4* hb, int slot, float3 a) const {
    hb[slot * NT + t] = make_float4(a.x, a.y, a.z, 0.f);
  }
  __device__ __forceinline__ float3 next3(const float4* hb, int slot) const { return f3(next(hb, slot)); }
  __device__ __forceinline__ float3 prev3(const float4* hb, int slot) const { return f3(prev(hb, slot)); }
  __device__ __forceinline__ void sync() const { cooperative_groups::this_grid().sync(); }
  // after the exchange stores: the block's first and last thread copy their slots (written
  // by themselves just before) to global memory; the grid sync then publishes them
  __device__ __forceinline__ void arrive(const float4* hb) const {
    if (t == 0 || t == NT - 1) {
#pragma unroll
      for (int s = 0; s < kHaloSlots; ++s) __stcg(gslot(hb, c, s, t == 0 ? 0 : 1), hb[s * NT + t]);
    }
  }
  __device__ __forceinline__ void wait() const { cooperative_groups::this_grid().sync(); }
  // block-wide OR (rods on a grid run without the mailbox, the only user of a rod-wide OR)
  __device__ __forceinline__ int any(int x) const { return __syncthreads_or(x); }
};

// Bend/twist torques of the joint between frames a and b (Eq. 3): with
// D = conj(qa) (x) qb, u = (2/l) Im(D) and m = 2 K (u - u-hat), the body torques are
// tau_a = 1/2 Im(D (x) (0, m)) and tau_b = -1/2 Im(conj(D) (x) (0, m)).
__device__ __forceinline__ void joint_torques(float4 qa, float4 qb, float4 uh, float4 K, float two_over_l,
                                              float3& ta, float3& tb) {
  const float dw = qa.x * qb.x + qa.y * qb.y + qa.z * qb.z + qa.w * qb.w;
  const float3 dv = im_conj_mul(qa, qb);
  const float3 u = two_over_l * dv;
  const float3 m = f3(2.f * K.x * (u.x - uh.x), 2.f * K.y * (u.y - uh.y), 2.f * K.z * (u.z - uh.z));
  const float3 c = cross3(dv, m);
  ta = 0.5f * (dw * m + c);
  tb = 0.5f * (c - dw * m);
}

// Segment forces between nodes a and b and the penalty torque on frame q (Eq. 8, and
// Eq. 2 when the rod is extensible).  Penalty: E = 1/2 l0 Kp |t - d3|^2 gives the force
// l0 Kp (d3 - (t . d3) t) / |e| on node b (opposite on a) and the torque l0 Kp d3 x t,
// which in the body frame (d3 = e_z) is l0 Kp (-t_b.y, t_b.x, 0) with t_b = R(q)^T t.
__device__ __forceinline__ void segment_forces(float3 ra, float3 rb, float4 q, const RodDev& R, bool extensible,
                                               float3& fa, float3& fb, float3& tq) {
  const float3 e = rb - ra;
  const float ee = dot3(e, e);
  const float il = rsqrtf(ee);
  const float3 t = il * e;
  const float3 d3 = director3(q);
  const float c = dot3(t, d3);
  const float3 f = (R.lKp * il) * (d3 - c * t);
  fb = f;
  fa = -f;
  if (extensible) {
    const float len = ee * il;
    const float3 fs = (R.Ks * (len * R.inv_l0 - 1.f)) * t;
    fa += fs;
    fb -= fs;
  }
  const float3 tb = rotate_inv(q, t);
  tq = f3(-R.lKp * tb.y, R.lKp * tb.x, 0.f);
}

// Impulse of one distance constraint (predictive: makes the segment length l0 after the
// update).  With e = r_b - r_a (fixed during the sweeps of a step) and
// d = (r_b + dt v_b) - (r_a + dt v_a) = e + dt (v_b - v_a) (the node difference is exact
// for neighbouring nodes, whereas r + dt v would round dt v against |r|), returns
// g = lambda n = -(|d| - l0) / (dt (w_a + w_b)) d / |d| = (l0 / |d| - 1) inv_dtW d;
// the caller applies v_a -= w_a g, v_b += w_b g.  inv_dtW = 1 / (dt (w_a + w_b)) is
// computed once per step (0 for a constraint that does not exist: then e is a safe
// non-zero vector and g = 0).
__device__ __forceinline__ float3 constraint_impulse(float3 e, float3 va, float3 vb, float inv_dtW, float l0,
                                                     float dt) {
  const float3 d = f3(__fmaf_rn(dt, __fsub_rn(vb.x, va.x), e.x), __fmaf_rn(dt, __fsub_rn(vb.y, va.y), e.y),
                      __fmaf_rn(dt, __fsub_rn(vb.z, va.z), e.z));
  const float dd = __fmaf_rn(d.x, d.x, __fmaf_rn(d.y, d.y, __fmul_rn(d.z, d.z)));
  const float s = __fmul_rn(__fmaf_rn(l0, rsqrtf(dd), -1.f), inv_dtW);
  return f3(__fmul_rn(s, d.x), __fmul_rn(s, d.y), __fmul_rn(s, d.z));
}

// Predictive impulse with the masses folded into per-launch scales: with
// c_a = w_a / (dt (w_a + w_b)) and c_b = w_b / (dt (w_a + w_b)) (0 for a constraint that does
// not exist), v_a -= (l0 c_a / |d| - c_a) d and v_b += (l0 c_b / |d| - c_b) d: the update of
// constraint_impulse with two dependent operations after the reciprocal square root
// instead of four (it holds four scales per constraint in registers instead of one).
__device__ __forceinline__ void constraint_apply(float3 e, float3& va, float3& vb, float ca, float l0ca, float cb,
                                                 float l0cb, float dt) {
  const float3 d = f3(__fmaf_rn(dt, __fsub_rn(vb.x, va.x), e.x), __fmaf_rn(dt, __fsub_rn(vb.y, va.y), e.y),
                      __fmaf_rn(dt, __fsub_rn(vb.z, va.z), e.z));
  const float dd = __fmaf_rn(d.x, d.x, __fmaf_rn(d.y, d.y, __fmul_rn(d.z, d.z)));
  const float il = rsqrtf(dd);
  const float sa = __fmaf_rn(l0ca, il, -ca), sb = __fmaf_rn(l0cb, il, -cb);
  va = f3(__fmaf_rn(-sa, d.x, va.x), __fmaf_rn(-sa, d.y, va.y), __fmaf_rn(-sa, d.z, va.z));
  vb = f3(__fmaf_rn(sb, d.x, vb.x), __fmaf_rn(sb, d.y, vb.y), __fmaf_rn(sb, d.z, vb.z));
}

// Two independent constraints in the two lanes of packed FP32x2 operations (Blackwell
// fma/mul/add.f32x2): lane x and lane y each compute exactly what constraint_impulse
// computes for them (round-to-nearest per lane), with half the instructions.
struct Vec3x2 {
  float2 x, y, z;
};
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// b - a as one packed fused operation, a (-1) + b: exactly the difference, rounded once
// (a separate negation would put one more operation on the impulse chain)
__device__ __forceinline__ float2 sub2(float2 b, float2 a) { return __ffma2_rn(a, make_float2(-1.f, -1.f), b); }
__device__ __forceinline__ Vec3x2 constraint_impulse2(const Vec3x2& e, const Vec3x2& va, const Vec3x2& vb,
                                                      float2 inv_dtW, float l0, float dt) {
  const float2 dt2 = make_float2(dt, dt);
  const float2 dx = __ffma2_rn(dt2, sub2(vb.x, va.x), e.x);
  const float2 dy = __ffma2_rn(dt2, sub2(vb.y, va.y), e.y);
  const float2 dz = __ffma2_rn(dt2, sub2(vb.z, va.z), e.z);
  const float2 dd = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
  const float2 il = make_float2(rsqrtf(dd.x), rsqrtf(dd.y));
  const float2 sv = __fmul2_rn(__ffma2_rn(make_float2(l0, l0), il, make_float2(-1.f, -1.f)), inv_dtW);
  return Vec3x2{__fmul2_rn(sv, dx), __fmul2_rn(sv, dy), __fmul2_rn(sv, dz)};
}

// The two odd constraints across a thread's boundaries with folded scales: right (the
// thread's last node, the next thread's first) and left (the previous thread's last node,
// the thread's first).  e_bnd holds their segment vectors (lane x right, lane y left),
// l_bnd and c_bnd the folded scales of the thread's own node in each (right: -c_a, left:
// +c_b), vn and vp the neighbours' velocities; updates the thread's last and first
// velocities.  Scalar operations: the two constraints are independent chains, and paired
// lanes would put register-pair moves on this latency-bound path (measured 2.82 against
// 2.89 us/step for the 512-node rod).  The adjoint repeats this update on recorded
// velocities, so both use this one function.
__device__ __forceinline__ void boundary_apply(const Vec3x2& e_bnd, float2 l_bnd, float2 c_bnd, float dt, float3 vn,
                                               float3 vp, float3& v_last, float3& v_first) {
  auto one = [dt](float ex, float ey, float ez, float3 va, float3 vb, float l, float c, float3& vo) {
    const float dx = __fmaf_rn(dt, __fsub_rn(vb.x, va.x), ex);
    const float dy = __fmaf_rn(dt, __fsub_rn(vb.y, va.y), ey);
    const float dz = __fmaf_rn(dt, __fsub_rn(vb.z, va.z), ez);
    const float dd = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
    const float il = rsqrtf(dd);
    // right: v_last -= c_a (l0 / |d| - 1) d ; left: v_first += c_b (l0 / |d| - 1) d
    const float scl = __fmaf_rn(l, il, -c);
    vo = f3(__fmaf_rn(scl, dx, vo.x), __fmaf_rn(scl, dy, vo.y), __fmaf_rn(scl, dz, vo.z));
  };
  const float3 vl = v_last, vf = v_first;
  one(e_bnd.x.x, e_bnd.y.x, e_bnd.z.x, vl, vn, l_bnd.x, c_bnd.x, v_last);
  one(e_bnd.x.y, e_bnd.y.y, e_bnd.z.y, vp, vf, l_bnd.y, c_bnd.y, v_first);
}

// Per-step data of one constraint: e = r_b - r_a and 1 / (dt (w_a + w_b)); a constraint
// that does not exist (or joins two kinematic nodes) gets 0 and a safe e.
__device__ __forceinline__ float3 segment_vector(float3 ra, float3 rb) {
  return f3(__fsub_rn(rb.x, ra.x), __fsub_rn(rb.y, ra.y), __fsub_rn(rb.z, ra.z));
}
__device__ __forceinline__ float inv_dt_wsum(bool exists, float wa, float wb, float dt) {
  const float ws = __fadd_rn(wa, wb);
  return (exists && ws > 0.f) ? __frcp_rn(__fmul_rn(dt, ws)) : 0.f;
}
__device__ __forceinline__ float3 safe_segment(float inv, float3 e, float l0) {
  return inv != 0.f ? e : f3(0.f, 0.f, l0);
}

// Contact of node (r, v) with the wall of an analytic vessel (collision constraint C_c with
// Coulomb friction, Section 2.1 "Constraints"; a tube stands in for the vessel meshes):
// the centreline is the circle of radius rc about (cx, cy) in the plane z = cz; the node
// must stay within `allow` (inner radius minus rod radius) of it.  With p = r + dt v the
// predicted position and c the centreline point nearest to p, delta = p - c is normal to
// the centreline; if |delta| > allow the
// normal velocity changes by dvn = -(|delta| - allow) / dt along n = delta / |delta| (the
// predicted node lands on the wall) and the tangential velocity shrinks by at most
// mu |dvn| (Coulomb).  Kinematic nodes (w = 0) are skipped.
__device__ __forceinline__ void tube_contact(float3 r, float3& v, float w, const RodDev& R, float dt,
                                             float inv_dt) {
  // offset of the predicted position from the vessel centre, radially (rho) and along z
  const float px = fmaf(dt, v.x, r.x - R.tube_cx), py = fmaf(dt, v.y, r.y - R.tube_cy);
  const float pz = fmaf(dt, v.z, r.z - R.tube_cz);
  const float rho2 = fmaxf(fmaf(px, px, py * py), 1e-30f);
  const float irho = rsqrtf(rho2);
  const float s = fmaf(rho2, irho, -R.tube_rc);  // rho - rc: radial offset from the centreline
  const float d2 = fmaxf(fmaf(s, s, pz * pz), 1e-30f);  // |delta|^2, delta = p - c
  const float il = rsqrtf(d2);
  const float a = s * irho * il;
  const float3 n = f3(px * a, py * a, pz * il);  // delta / |delta|
  // branch-free: a node out of contact (or kinematic) gets dvn = 0 and keep = 1, which
  // leaves v unchanged exactly
  const bool hit = (w > 0.f) && (d2 > R.tube_allow * R.tube_allow);
  const float dvn = hit ? (R.tube_allow - d2 * il) * inv_dt : 0.f;
  const float vn = dot3(v, n);
  const float3 vt = v - vn * n;
  const float vt2 = fmaxf(dot3(vt, vt), 1e-30f);
  const float keep = hit ? fmaxf(0.f, 1.f - R.tube_mu * fabsf(dvn) * rsqrtf(vt2)) : 1.f;
  // v + dvn n - (1 - keep) vt  =  keep v + (dvn + (1 - keep) vn) n
  const float c = fmaf(1.f - keep, vn, dvn);
  v = f3(fmaf(keep, v.x, c * n.x), fmaf(keep, v.y, c * n.y), fmaf(keep, v.z, c * n.z));
}

// Hook into the constraint loop of step_body: before_iterations() once per step before
// the sweeps, after_odd() after every iteration's odd sweep.  The plain rod needs none;
// the catheter/guidewire pair applies its binding constraints there.
struct NoHook {
  template <int EPT>
  __device__ __forceinline__ void before_iterations(const float3 (&)[EPT], const float (&)[EPT]) const {}
  template <int EPT>
  __device__ __forceinline__ void after_odd(const float3 (&)[EPT], float3 (&)[EPT], const float (&)[EPT]) const {}
};

// Neighbour data of one step, kept by the adjoint's recomputation.
struct StepNeighbours {
  float3 r_next, r_prev;
  float w_next, w_prev;
  float4 q_next;
};

// Per-thread constants of a launch that step_body derives on its first step: the
// constraint scales 1 / (dt (w_a + w_b)) of the thread's even, odd and boundary segments
// (inverse masses do not change during a launch) and, with two elements per thread, the
// folded per-node scales of constraint_apply.
template <int EPT>
struct StepCache {
  static constexpr int NE = EPT / 2, NO = EPT / 2 > 1 ? EPT / 2 - 1 : 1;
  // fold the masses into the impulse scales (fewer dependent operations per impulse, more
  // registers: with four elements per thread the 128-register budget of the batch layout
  // would spill)
  static constexpr bool kFold = EPT == 2;
  bool ready = false;
  float i_even[NE], i_odd[NO], i_right, i_left;
  float ca_even[NE], cb_even[NE], la_even[NE], lb_even[NE];
  float2 c_bnd, l_bnd;  // per lane the scale of the thread's own node (right: -c_a, left: +c_b)
};

// Dynamic shared memory of a <EPT, NT> block: per-element joint parameters (u-hat and
// K), element-major so that thread t's accesses are conflict-free, then the two
// ping-pong exchange buffers of kHaloSlots float4 slots per thread.
template <int EPT, int NT>
constexpr int step_smem_bytes() {
  return (2 * EPT * NT + 2 * kHaloSlots * NT) * (int)sizeof(float4);
}

// Velocity records of one step for the adjoint, slot-major and then by component,
// element and thread ([slots][3][EPT][NT] floats): a thread's vector is three coalesced
// 32-bit accesses, and a step's record is one contiguous block (12 B per node and slot).
template <int EPT, int NT>
__device__ __forceinline__ void rec_put(float4* rec, int slot, int e, int u, float3 v) {
  float* f = reinterpret_cast<float*>(rec) + (slot * 3 * EPT + e) * NT + u;
  f[0] = v.x;
  f[EPT * NT] = v.y;
  f[2 * EPT * NT] = v.z;
}
template <int EPT, int NT>
__device__ __forceinline__ float3 rec_get(const float4* rec, int slot, int e, int u) {
  const float* f = reinterpret_cast<const float*>(rec) + (slot * 3 * EPT + e) * NT + u;
  return f3(f[0], f[EPT * NT], f[2 * EPT * NT]);
}

// One time step of the rod; H (BlockHalo or ClusterHalo) gives the thread's place in the
// rod, its neighbours' exchange slots and the barrier; sc holds the launch constants
// (default-constructed before the first step).  STORE (for the adjoint) writes the
// neighbour data to *nb and velocities to sweep_v (rec_put): with STORE == 1 those
// before every constraint half-sweep (2 n_iters slots: 2 it before the even and 2 it + 1
// before the odd half-sweep of iteration it); with STORE == 2 (compact) those before the
// first even half-sweep (slot 0) and before every odd one (slot 1 + it), from which the
// adjoint rebuilds the others.
template <int EPT, int NT, int STORE, class Halo, class Hook = NoHook>
__device__ __forceinline__ void step_body(const RodDev& R, const Halo& H, float3 (&r)[EPT], float3 (&v)[EPT],
                                          float4 (&q)[EPT], float3 (&om)[EPT], const float (&w)[EPT],
                                          const float4* par_u, const float4* par_k, float4* halo, int& xc,
                                          StepCache<EPT>& sc, const float3 v_drive, const float3 w_drive,
                                          float4* sweep_v, StepNeighbours* nb, const Hook& hook = Hook()) {
  const int t = H.t;
  const int e0 = H.tg() * EPT;
  const int n = R.n;
  const bool inext = (R.flags & F_INEXT) != 0;
  const bool clamp = (R.flags & F_CLAMP) != 0;
  const float dt = R.dt;
  const float half_dt = 0.5f * dt;

  // ---- exchange 1: first element's position, inverse mass and frame to the left
  // neighbour, last element's position and inverse mass to the right neighbour (the
  // positions hold for the whole step: the constraint sweeps change velocities only)
  float4* hb = halo + (xc & 1) * kHaloSlots * NT;
  ++xc;
  hb[t] = make_float4(r[0].x, r[0].y, r[0].z, w[0]);
  hb[NT + t] = q[0];
  hb[2 * NT + t] = make_float4(r[EPT - 1].x, r[EPT - 1].y, r[EPT - 1].z, w[EPT - 1]);
  H.arrive(hb);

  // ---- elastic forces and torques.  Joint j couples frames j and j + 1, segment j nodes
  // j and j + 1 (with frame j); all but the thread's last joint and segment are local, and
  // they run while the exchange barrier waits.
  float3 F[EPT], tau[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    F[e] = zero3();
    tau[e] = zero3();
  }
  float3 F_carry = zero3(), tau_carry = zero3();
  auto joint_and_segment = [&](int e, float4 qb, float3 rb) {
    const int j = e0 + e;
    if (j <= n - 3) {
      float3 ta, tb;
      joint_torques(q[e], qb, par_u[e * NT + t], par_k[e * NT + t], R.two_over_l, ta, tb);
      tau[e] += ta;
      if (e + 1 < EPT) {
        tau[(e + 1) % EPT] += tb;
      } else {
        tau_carry = tb;
      }
    }
    if (j <= n - 2) {
      float3 fa, fb, tq;
      segment_forces(r[e], rb, q[e], R, !inext, fa, fb, tq);
      F[e] += fa;
      tau[e] += tq;
      if (e + 1 < EPT) {
        F[(e + 1) % EPT] += fb;
      } else {
        F_carry = fb;
      }
    }
  };
#pragma unroll
  for (int e = 0; e + 1 < EPT; ++e) joint_and_segment(e, q[e + 1], r[e + 1]);

  H.wait();
  float3 r_next = zero3(), r_prev = zero3();
  float w_next = 0.f, w_prev = 0.f;
  float4 q_next = make_float4(0.f, 0.f, 0.f, 1.f);
  const bool has_next = H.has_next(), has_prev = H.has_prev();
  if (has_next) {
    const float4 a = H.next(hb, 0);
    r_next = f3(a);
    w_next = a.w;
    q_next = H.next(hb, 1);
  }
  if (has_prev) {
    const float4 a = H.prev(hb, 2);
    r_prev = f3(a);
    w_prev = a.w;
  }
  if constexpr (STORE) {
    nb->r_next = r_next;
    nb->r_prev = r_prev;
    nb->w_next = w_next;
    nb->w_prev = w_prev;
    nb->q_next = q_next;
  }
  // the thread's last joint and segment reach into the next thread's first element
  joint_and_segment(EPT - 1, q_next, r_next);
  // ---- exchange 2: carries to the right neighbour's first element
  hb = halo + (xc & 1) * kHaloSlots * NT;
  ++xc;
  H.put3(hb, 0, F_carry);
  H.put3(hb, 1, tau_carry);
  H.arrive(hb);

  // ---- while the exchange barrier completes: the constraint geometry of this step (the
  // positions and masses do not change in the sweeps) and the force integration of
  // elements 1 .. EPT - 1, which take no carry
  constexpr int NE = StepCache<EPT>::NE, NO = StepCache<EPT>::NO;
  float3 e_even[NE], e_odd[NO], e_r = zero3(), e_l = zero3();
  if (inext) {
    if (!sc.ready) {
#pragma unroll
      for (int k = 0; k < NE; ++k) sc.i_even[k] = inv_dt_wsum(e0 + 2 * k + 1 <= n - 1, w[2 * k], w[2 * k + 1], dt);
#pragma unroll
      for (int k = 0; k < NO; ++k) {
        const bool ex = EPT / 2 > 1 && e0 + 2 * k + 2 <= n - 1;
        sc.i_odd[k] = inv_dt_wsum(ex, w[(2 * k + 1) % EPT], w[(2 * k + 2) % EPT], dt);
      }
      // the two boundary constraints: right (my last, next first), left (previous last,
      // my first)
      sc.i_right = inv_dt_wsum(has_next && e0 + EPT <= n - 1, w[EPT - 1], w_next, dt);
      sc.i_left = inv_dt_wsum(has_prev && e0 <= n - 1, w_prev, w[0], dt);
      if constexpr (StepCache<EPT>::kFold) {
#pragma unroll
        for (int k = 0; k < NE; ++k) {
          sc.ca_even[k] = w[2 * k] * sc.i_even[k];
          sc.cb_even[k] = w[2 * k + 1] * sc.i_even[k];
          sc.la_even[k] = R.l0 * sc.ca_even[k];
          sc.lb_even[k] = R.l0 * sc.cb_even[k];
        }
        sc.c_bnd = make_float2(-w[EPT - 1] * sc.i_right, w[0] * sc.i_left);
        sc.l_bnd = make_float2(R.l0 * sc.c_bnd.x, R.l0 * sc.c_bnd.y);
      }
      sc.ready = true;
    }
#pragma unroll
    for (int k = 0; k < NE; ++k) e_even[k] = safe_segment(sc.i_even[k], segment_vector(r[2 * k], r[2 * k + 1]), R.l0);
#pragma unroll
    for (int k = 0; k < NO; ++k)
      e_odd[k] = safe_segment(sc.i_odd[k], segment_vector(r[(2 * k + 1) % EPT], r[(2 * k + 2) % EPT]), R.l0);
    e_r = safe_segment(sc.i_right, segment_vector(r[EPT - 1], r_next), R.l0);
    e_l = safe_segment(sc.i_left, segment_vector(r_prev, r[0]), R.l0);
  }
  auto integrate = [&](int e) {
    const int i = e0 + e;
    if (w[e] > 0.f) {
      const float3 a = f3(w[e] * F[e].x + R.gx, w[e] * F[e].y + R.gy, w[e] * F[e].z + R.gz);
      v[e] = R.damp * (v[e] + dt * a);
    }
    const bool frame_dynamic = (i <= n - 2) && !(clamp && i == 0);
    if (frame_dynamic) {
      const float3 o = om[e];
      const float3 Jw = f3(R.J1 * o.x, R.J1 * o.y, R.J3 * o.z);
      const float3 rhs = tau[e] - cross3(o, Jw);
      const float3 on = f3(o.x + dt * R.Jinv1 * rhs.x, o.y + dt * R.Jinv1 * rhs.y, o.z + dt * R.Jinv3 * rhs.z);
      om[e] = R.damp * on;
    }
  };
#pragma unroll
  for (int e = 1; e < EPT; ++e) integrate(e);
  H.wait();
  if (has_prev) {
    F[0] += H.prev3(hb, 0);
    tau[0] += H.prev3(hb, 1);
  }
  integrate(0);
  if (clamp && e0 == 0) {
    v[0] = v_drive;
    om[0] = w_drive;
  }
  // ---- integrate the angular velocities into the frames (semi-implicit Euler): the
  // constraint sweeps change only the node velocities, so the frames' update is final
  // here and overlaps the sweeps' latency
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    if (e0 + e <= n - 2) {
      const float4 a = q[e];
      const float3 o = om[e];
      // q (x) (0, omega)
      const float dx = a.w * o.x + a.y * o.z - a.z * o.y;
      const float dy = a.w * o.y + a.z * o.x - a.x * o.z;
      const float dz = a.w * o.z + a.x * o.y - a.y * o.x;
      const float dwq = -(a.x * o.x + a.y * o.y + a.z * o.z);
      const float4 b = make_float4(a.x + half_dt * dx, a.y + half_dt * dy, a.z + half_dt * dz, a.w + half_dt * dwq);
      const float inv = rsqrtf(b.x * b.x + b.y * b.y + b.z * b.z + b.w * b.w);
      q[e] = make_float4(b.x * inv, b.y * inv, b.z * inv, b.w * inv);
    }
  }

  // ---- distance-constraint iterations (inextensible rod), red-black
  if (inext) {
    hook.template before_iterations<EPT>(r, w);
    const float inv_dt = 1.f / dt;
    // the two boundary constraints, right in lane x and left in lane y
    const Vec3x2 e_bnd{make_float2(e_r.x, e_l.x), make_float2(e_r.y, e_l.y), make_float2(e_r.z, e_l.z)};
    const float2 w_bnd = make_float2(-w[EPT - 1], w[0]);

    // one iteration; tube_on (a compile-time bool) adds the vessel contact
    auto iteration = [&](int it, auto tube_on) {
      if constexpr (STORE) {
#pragma unroll
        for (int e = 0; e < EPT; ++e)
          if (STORE == 1 || it == 0)
            rec_put<EPT, NT>(sweep_v, STORE == 1 ? 2 * it : 0, e, t, v[e]);
      }
      // even segments (e0 + 2k, e0 + 2k + 1): local to the thread, two per packed op
      if constexpr (StepCache<EPT>::kFold) {
#pragma unroll
        for (int k = 0; k < NE; ++k)
          constraint_apply(e_even[k], v[2 * k], v[2 * k + 1], sc.ca_even[k], sc.la_even[k], sc.cb_even[k],
                           sc.lb_even[k], dt);
      } else if constexpr (NE == 1) {
        const float3 g = constraint_impulse(e_even[0], v[0], v[1], sc.i_even[0], R.l0, dt);
        v[0] -= w[0] * g;
        v[1] += w[1] * g;
      } else {
#pragma unroll
        for (int k = 0; k + 1 < NE; k += 2) {
          const int a0 = 2 * k, b0 = 2 * k + 1, a1 = 2 * k + 2, b1 = 2 * k + 3;
          const Vec3x2 ep{make_float2(e_even[k].x, e_even[k + 1].x), make_float2(e_even[k].y, e_even[k + 1].y),
                          make_float2(e_even[k].z, e_even[k + 1].z)};
          const Vec3x2 va{make_float2(v[a0].x, v[a1].x), make_float2(v[a0].y, v[a1].y), make_float2(v[a0].z, v[a1].z)};
          const Vec3x2 vb{make_float2(v[b0].x, v[b1].x), make_float2(v[b0].y, v[b1].y), make_float2(v[b0].z, v[b1].z)};
          const Vec3x2 g = constraint_impulse2(ep, va, vb, make_float2(sc.i_even[k], sc.i_even[k + 1]), R.l0, dt);
          v[a0] -= w[a0] * f3(g.x.x, g.y.x, g.z.x);
          v[a1] -= w[a1] * f3(g.x.y, g.y.y, g.z.y);
          v[b0] += w[b0] * f3(g.x.x, g.y.x, g.z.x);
          v[b1] += w[b1] * f3(g.x.y, g.y.y, g.z.y);
        }
        if constexpr (NE % 2 == 1) {
          const int a = EPT - 2, b = EPT - 1;
          const float3 g = constraint_impulse(e_even[NE - 1], v[a], v[b], sc.i_even[NE - 1], R.l0, dt);
          v[a] -= w[a] * g;
          v[b] += w[b] * g;
        }
      }
      if constexpr (STORE) {
#pragma unroll
        for (int e = 0; e < EPT; ++e)
          rec_put<EPT, NT>(sweep_v, STORE == 1 ? 2 * it + 1 : it + 1, e, t, v[e]);
      }
      // exchange 3: velocities of the first and last element
      hb = halo + (xc & 1) * kHaloSlots * NT;
      ++xc;
      H.put3(hb, 0, v[0]);
      H.put3(hb, 1, v[EPT - 1]);
      H.arrive(hb);
      // odd segments inside the thread: they move elements 1 .. EPT - 2 only, which the
      // exchange and the boundary segments do not read, so they run while the barrier waits
#pragma unroll
      for (int k = 0; k + 1 < EPT / 2; ++k) {
        const int a = 2 * k + 1, b = 2 * k + 2;
        const float3 g = constraint_impulse(e_odd[k], v[a], v[b], sc.i_odd[k], R.l0, dt);
        v[a] -= w[a] * g;
        v[b] += w[b] * g;
      }
      H.wait();
      // odd segments across the two thread boundaries (two independent scalar chains)
      {
        const float3 vn = has_next ? H.next3(hb, 0) : zero3();
        const float3 vp = has_prev ? H.prev3(hb, 1) : zero3();
        if constexpr (StepCache<EPT>::kFold) {
          boundary_apply(e_bnd, sc.l_bnd, sc.c_bnd, dt, vn, vp, v[EPT - 1], v[0]);
        } else {
          const float3 gr = constraint_impulse(e_r, v[EPT - 1], vn, sc.i_right, R.l0, dt);
          const float3 gl = constraint_impulse(e_l, vp, v[0], sc.i_left, R.l0, dt);
          v[EPT - 1] = f3(__fmaf_rn(w_bnd.x, gr.x, v[EPT - 1].x), __fmaf_rn(w_bnd.x, gr.y, v[EPT - 1].y),
                          __fmaf_rn(w_bnd.x, gr.z, v[EPT - 1].z));
          v[0] = f3(__fmaf_rn(w_bnd.y, gl.x, v[0].x), __fmaf_rn(w_bnd.y, gl.y, v[0].y), __fmaf_rn(w_bnd.y, gl.z, v[0].z));
        }
      }
      // collision response (analytic vessel), per node
      if constexpr (decltype(tube_on)::value) {
#pragma unroll
        for (int e = 0; e < EPT; ++e)
          if (e0 + e < n) tube_contact(r[e], v[e], w[e], R, dt, inv_dt);
      }
      hook.template after_odd<EPT>(r, v, w);
    };
    if (R.flags & F_TUBE) {
      for (int it = 0; it < R.n_iters; ++it) iteration(it, std::true_type());
    } else if constexpr (std::is_same<Hook, NoHook>::value && EPT == 2) {
      // the plain rod: unrolled (ten iterations, the paper's count, run as one block of code)
#pragma unroll 10
      for (int it = 0; it < R.n_iters; ++it) iteration(it, std::false_type());
    } else if constexpr (std::is_same<Hook, NoHook>::value) {
#pragma unroll 2
      for (int it = 0; it < R.n_iters; ++it) iteration(it, std::false_type());
    } else {
      for (int it = 0; it < R.n_iters; ++it) iteration(it, std::false_type());
    }
  }

  // ---- integrate the node velocities into the positions (semi-implicit Euler)
#pragma unroll
  for (int e = 0; e < EPT; ++e) r[e] += dt * v[e];
}

// Loads the rod's elements owned by thread tg of the rod (registers) and their joint
// parameters (shared memory slot t, read back only by the same thread).
template <int EPT, int NT>
__device__ __forceinline__ void load_rod(const RodDev& R, const int t, const int tg, const float4* __restrict__ x4,
                                         const float4* __restrict__ v4, const float4* __restrict__ q4,
                                         const float4* __restrict__ o4, const float4* __restrict__ u4,
                                         const float4* __restrict__ k4, float3 (&r)[EPT], float3 (&v)[EPT],
                                         float4 (&q)[EPT], float3 (&om)[EPT], float (&w)[EPT], float4* par_u,
                                         float4* par_k) {
  const int e0 = tg * EPT;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = e0 + e;
    if (i < R.n) {
      const float4 a = x4[R.off + i];
      r[e] = f3(a);
      w[e] = a.w;
      v[e] = f3(v4[R.off + i]);
      q[e] = q4[R.off + i];
      om[e] = f3(o4[R.off + i]);
      if (par_u != nullptr) {
        par_u[e * NT + t] = u4[R.off + i];
        par_k[e * NT + t] = k4[R.off + i];
      }
    } else {
      r[e] = zero3();
      v[e] = zero3();
      om[e] = zero3();
      q[e] = make_float4(0.f, 0.f, 0.f, 1.f);
      w[e] = 0.f;
    }
  }
}

// One non-blocking read attempt of the drive mailbox (seqlock: the host makes the word odd
// while it writes).  Returns true, with the drive row of rod `rid`, for a new consistent
// input; a torn or unchanged input is skipped (read again at the next poll).
__device__ __forceinline__ bool mailbox_poll(const MailboxDev& mb, int rid, unsigned& last, float3& vd, float3& wd,
                                             float* slot3 = nullptr) {
  const unsigned s1 = ld_acquire_sys(mb.in_seq);
  if ((s1 & 1u) || s1 == last || s1 == 0u) return false;
  float d[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) d[k] = ld_relaxed_sys_f(mb.in_drive + 8 * (int64_t)rid + k);
  fence_acq_rel_sys();
  if (ld_relaxed_sys(mb.in_seq) != s1) return false;
  vd = f3(d[0], d[1], d[2]);
  wd = f3(d[4], d[5], d[6]);
  if (slot3 != nullptr) *slot3 = d[3];
  last = s1;
  return true;
}

__device__ __forceinline__ void mailbox_log(const MailboxDev& mb, long long step, unsigned seq) {
  const int k = atomicAdd(mb.log_count, 1);
  if (k < mb.log_cap) mb.log[k] = make_int2((int)step, (int)seq);
}

// Lock-step: wait for a new input, bounded by mb.wait_ns of GPU time (and an iteration
// cap), backing off between reads.  Returns false, with bit 0 of the status set, when the
// wait runs out.
__device__ __forceinline__ bool mailbox_wait(const MailboxDev& mb, int rid, unsigned& last, float3& vd, float3& wd,
                                             long long step, float* slot3 = nullptr) {
  const unsigned long long t0 = global_ns();
  for (int k = 0; k < (1 << 26); ++k) {
    if (mailbox_poll(mb, rid, last, vd, wd, slot3)) {
      mailbox_log(mb, step, last);
      return true;
    }
    if (global_ns() - t0 > mb.wait_ns) break;
    __nanosleep(256);
  }
  st_release_sys(mb.status, 1u);
  return false;
}

// Seqlock write of one feedback record (seq, step, position, velocity).
__device__ __forceinline__ void mailbox_write(unsigned* rec, unsigned& seq, long long step, float3 r, float3 v) {
  st_relaxed_sys(rec, seq + 1u);
  fence_acq_rel_sys();
  st_relaxed_sys(rec + 1, (unsigned)step);
  st_relaxed_sys(rec + 2, __float_as_uint(r.x));
  st_relaxed_sys(rec + 3, __float_as_uint(r.y));
  st_relaxed_sys(rec + 4, __float_as_uint(r.z));
  st_relaxed_sys(rec + 5, __float_as_uint(v.x));
  st_relaxed_sys(rec + 6, __float_as_uint(v.y));
  st_relaxed_sys(rec + 7, __float_as_uint(v.z));
  seq += 2u;
  st_release_sys(rec, seq);
}

// Mailbox work of one rod inside a launch (Section 2.2: the haptic thread exchanges input
// and feedback with the running kernel): before every `period`-th step the drive is polled
// (or, in lock-step, waited for); after it the base/tip records and the position snapshot
// are written.  H provides the barrier (and, for single blocks, the block-wide OR).
template <int EPT>
struct RodMailbox {
  const MailboxDev& mb;  // the launch's parameter
  const RodDev& R;
  int rid, e0, group;
  bool owns_base, owns_tip;
  // With position snapshots the base record is written by the rod's thread 32 (another
  // warp, the same block), from values the base's thread stages in shared memory, so the
  // base's thread goes straight on to the next input wait.
  bool writes_base;
  unsigned last = 0u, seq_base = 0u, seq_tip = 0u, seq_pos = 0u;
  unsigned* rec_base = nullptr;
  unsigned* rec_tip = nullptr;

  // rod_threads: threads holding the rod; group: the rod's index in its block (0, or the
  // pair kernel's group)
  __device__ __forceinline__ RodMailbox(const MailboxDev& m, const RodDev& R_, int rid_, int e0_, int rod_threads,
                                        int group_ = 0)
      : mb(m), R(R_), rid(rid_), e0(e0_), group(group_) {
    owns_base = e0 == 0;
    owns_tip = e0 <= R.n - 1 && R.n - 1 < e0 + EPT;
    writes_base = (mb.pos != nullptr && rod_threads > 32) ? e0 == 32 * EPT : owns_base;
    if (mb.period > 0) {
      rec_base = mb.out + 16 * (int64_t)rid;
      rec_tip = rec_base + 8;
      if (writes_base) seq_base = ld_relaxed_sys(rec_base) & ~1u;
      if (owns_tip) seq_tip = ld_relaxed_sys(rec_tip) & ~1u;
      // every thread keeps the publication count (it selects the ring slot); read before
      // the first barrier, so before any publication of this launch
      if (mb.pos != nullptr) seq_pos = ld_relaxed_sys(mb.pos_seq + 32 * (int64_t)rid);
    }
  }

  // Before step `step`; true when the launch must stop (a lock-step wait ran out).  A new
  // input replaces the drive (and *slot3, the drive row's slot 3, when given).
  template <class Halo>
  __device__ __forceinline__ bool before_step(const Halo& H, int step, float3& vd, float3& wd,
                                              float* slot3 = nullptr) {
    if (mb.period <= 0 || step % mb.period != 0) return false;
    if (mb.lockstep) {
      // lock-step: the base's thread waits (bounded) for the next input; the rod's other
      // threads wait at the OR (block or cluster) and all leave together if it ran out
      int lost = 0;
      if (owns_base) lost = !mailbox_wait(mb, rid, last, vd, wd, mb.step0 + step, slot3);
      return H.any(lost) != 0;
    }
    if (owns_base && mailbox_poll(mb, rid, last, vd, wd, slot3)) mailbox_log(mb, mb.step0 + step, last);
    return false;
  }

  // After step `step`: the position snapshot, then the feedback records.
  template <class Halo>
  __device__ __forceinline__ void after_step(const Halo& H, int step, const float3 (&r)[EPT], const float3 (&v)[EPT],
                                             const float (&w)[EPT]) {
    if (mb.period <= 0 || (step + 1) % mb.period != 0) return;
    __shared__ float4 base_stage[2][2];  // [group]: base position, velocity
    if (mb.pos != nullptr) {
      // Snapshot p of every position into ring slot p % kPosSlots, its step into the
      // slot's header, then the publication count p + 1 (release).  The first thread's
      // fence after that release orders the count before the next snapshot's stores, so
      // a slot is rewritten (at publication p + 4) only after count p + 4 is visible: a
      // host that copied slot p % kPosSlots and then still reads a count <= p + 3 copied
      // publication p whole.  The fence comes after the release, so the host sees the
      // count without waiting for it.
      unsigned* hdr = mb.pos_seq + 32 * (int64_t)rid;
      const int slot = (int)(seq_pos % kPosSlots);
      unsigned* sh = hdr + 4 + 4 * slot;
      if (owns_base) {
        base_stage[group][0] = make_float4(r[0].x, r[0].y, r[0].z, 0.f);
        base_stage[group][1] = make_float4(v[0].x, v[0].y, v[0].z, 0.f);
      }
      // system-scope stores (volatile), ordered before the first thread's release by the
      // barrier (release/acquire among the rod's threads) and its system-scope fence
      float4* dst = mb.pos + slot * mb.n_elem + R.off;
#pragma unroll
      for (int e = 0; e < EPT; ++e)
        if (e0 + e < R.n) st_volatile_f4(dst + e0 + e, make_float4(r[e].x, r[e].y, r[e].z, w[e]));
      H.sync();
      if (owns_base) {
        fence_acq_rel_sys();
        const long long st = mb.step0 + step + 1;
        st_relaxed_sys(sh + 1, (unsigned)(st & 0xffffffffll));
        st_relaxed_sys(sh + 2, (unsigned)(st >> 32));
        st_release_sys(hdr, seq_pos + 1u);
        fence_acq_rel_sys();
      }
      ++seq_pos;
    }
    // base and tip records after the snapshot: their fences do not delay it
    if (writes_base) {
      float3 rb = r[0], vb = v[0];
      if (!owns_base) {  // staged before the snapshot's barrier
        rb = f3(base_stage[group][0]);
        vb = f3(base_stage[group][1]);
      }
      mailbox_write(rec_base, seq_base, mb.step0 + step + 1, rb, vb);
    }
    if (owns_tip) {
#pragma unroll
      for (int e = 0; e < EPT; ++e)
        if (e0 + e == R.n - 1) mailbox_write(rec_tip, seq_tip, mb.step0 + step + 1, r[e], v[e]);
    }
  }
};

// The launch of one rod by the threads described by H: load, n_steps steps (with the
// optional trajectory output and mailbox), store.
template <int EPT, int NT, class Halo>
__device__ __forceinline__ void run_rod(const RodDev& R, const Halo& H, const int rid, const float4* __restrict__ x4in,
                                        float4* __restrict__ x4, float4* __restrict__ v4, float4* __restrict__ q4,
                                        float4* __restrict__ o4, const float4* __restrict__ u4,
                                        const float4* __restrict__ k4, const float4* __restrict__ drive, int n_steps,
                                        float4* __restrict__ traj, int64_t n_elem, const MailboxDev& mb, float4* smem,
                                        float4* __restrict__ pos_out) {
  float4* par_u = smem;
  float4* par_k = smem + EPT * NT;
  float4* halo = smem + 2 * EPT * NT;
  const int t = H.t;
  const int e0 = H.tg() * EPT;
  float3 r[EPT], v[EPT], om[EPT];
  float4 q[EPT];
  float w[EPT];
  load_rod<EPT, NT>(R, t, H.tg(), x4in, v4, q4, o4, u4, k4, r, v, q, om, w, par_u, par_k);
  float3 v_drive = zero3(), w_drive = zero3();
  if (drive != nullptr) {
    v_drive = f3(drive[2 * rid]);
    w_drive = f3(drive[2 * rid + 1]);
  }
  RodMailbox<EPT> box(mb, R, rid, e0, H.rod_threads());

  int xc = 0;  // exchange counter selects the ping-pong buffer
  StepCache<EPT> sc;  // launch constants of the step (filled on the first step)
  for (int step = 0; step < n_steps; ++step) {
    if (box.before_step(H, step, v_drive, w_drive)) break;
    step_body<EPT, NT, false>(R, H, r, v, q, om, w, par_u, par_k, halo, xc, sc, v_drive, w_drive, nullptr, nullptr);
    if (traj != nullptr) {
#pragma unroll
      for (int e = 0; e < EPT; ++e)
        if (e0 + e < R.n) traj[(int64_t)step * n_elem + R.off + e0 + e] = make_float4(r[e].x, r[e].y, r[e].z, w[e]);
    }
    box.after_step(H, step, r, v, w);
  }

#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = e0 + e;
    if (i < R.n) {
      x4[R.off + i] = make_float4(r[e].x, r[e].y, r[e].z, w[e]);
      v4[R.off + i] = make_float4(v[e].x, v[e].y, v[e].z, 0.f);
      q4[R.off + i] = q[e];
      o4[R.off + i] = make_float4(om[e].x, om[e].y, om[e].z, 0.f);
      if (pos_out != nullptr) pos_out[R.off + i] = make_float4(r[e].x, r[e].y, r[e].z, w[e]);
    }
  }
}

// n_steps time steps of one rod per block.  traj (optional): positions after every step,
// [n_steps][n_elements] float4 with .w the inverse mass; pos_out (optional): positions after
// the last step, [n_elements] float4 (device or mapped host memory).
template <int EPT, int NT>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : 512 / NT)
step_kernel(const RodDev* __restrict__ rods, const int* __restrict__ work, float4* __restrict__ x4,
            float4* __restrict__ v4, float4* __restrict__ q4, float4* __restrict__ o4,
            const float4* __restrict__ u4, const float4* __restrict__ k4, const float4* __restrict__ drive,
            int n_steps, float4* __restrict__ traj, int64_t n_elem, MailboxDev mb, float4* __restrict__ pos_out) {
  static_assert(EPT % 2 == 0, "elements per thread must be even (red-black sweeps)");
  extern __shared__ float4 smem[];
  pdl_begin();
  const int rid = work[blockIdx.x];
  const RodDev R = rods[rid];
  const BlockHalo<NT, NT, EPT == 2> H{(int)threadIdx.x};
  run_rod<EPT, NT>(R, H, rid, x4, x4, v4, q4, o4, u4, k4, drive, n_steps, traj, n_elem, mb, smem, pos_out);
}

}  // namespace corde
