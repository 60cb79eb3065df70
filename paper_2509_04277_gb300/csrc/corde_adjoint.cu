// Hand-written adjoint of the multi-step rollout (reverse-mode differentiation through
// the step of Fig. 5), with checkpoint-and-recompute.
//
// One thread block per rod, two elements per thread (the step kernel's <2, NT> layout).
// The forward rollout (rod_rollout) stores a checkpoint every K steps.  The reverse
// kernel walks the segments backwards.  For each segment it runs the K steps forward
// from the checkpoint, keeping the states and (record mode) the velocities the
// constraint half-sweeps start from in scratch memory; in recompute mode each step is
// run once more just before its reverse, its velocity records in shared memory.  Then,
// for each step (last to first), it applies the transposed Jacobian of the step:
//   r' = r + dt v2, q' = normalize(q + dt/2 q (x) (0, omega1))       (position update)
//   v2 = P(r, v1): 2 n_iters half-sweeps of distance impulses          (constraints)
//   v1 = damp (v + dt (w F + g)), omega1 = damp (omega + dt J^-1 (tau - omega x J omega))
//   F, tau = elastic forces / torques of Eq. 2, 3, 8 (second derivatives of the energies)
// Gradients flow to the initial positions and velocities and, accumulated over all
// steps, to the per-joint stiffness (K1, K2, K3) and intrinsic Darboux vectors u-hat.
#include "corde_step.cuh"
#include "corde_variants.cuh"

namespace corde {
namespace {

__device__ __forceinline__ float4 qmul4(float4 a, float4 b) {
  return make_float4(a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y, a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
                     a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w, a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z);
}
__device__ __forceinline__ float4 pure(float3 v) { return make_float4(v.x, v.y, v.z, 0.f); }
__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 scale4(float s, float4 a) { return make_float4(s * a.x, s * a.y, s * a.z, s * a.w); }
__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// VJP of joint_torques: given the adjoints of (ta, tb), the adjoints of qa, qb, K, u-hat.
__device__ __forceinline__ void joint_torques_vjp(float4 qa, float4 qb, float4 uh, float4 K, float two_over_l,
                                                  float3 ta_bar, float3 tb_bar, float4& qa_bar, float4& qb_bar,
                                                  float3& K_bar, float3& uh_bar) {
  const float dw = dot4(qa, qb);
  const float3 dv = im_conj_mul(qa, qb);
  const float3 u = two_over_l * dv;
  const float3 du = f3(u.x - uh.x, u.y - uh.y, u.z - uh.z);
  const float3 m = f3(2.f * K.x * du.x, 2.f * K.y * du.y, 2.f * K.z * du.z);
  const float3 cv_bar = 0.5f * (ta_bar + tb_bar);
  const float3 diff = ta_bar - tb_bar;
  const float dw_bar = 0.5f * dot3(m, diff);
  const float3 m_bar = 0.5f * dw * diff + cross3(cv_bar, dv);
  float3 dv_bar = cross3(m, cv_bar);
  K_bar = f3(2.f * du.x * m_bar.x, 2.f * du.y * m_bar.y, 2.f * du.z * m_bar.z);
  const float3 u_bar = f3(2.f * K.x * m_bar.x, 2.f * K.y * m_bar.y, 2.f * K.z * m_bar.z);
  uh_bar = -u_bar;
  dv_bar += two_over_l * u_bar;
  // dv = Im(conj(qa) (x) qb): d/dqb = qa (x) (0, .), d/dqa = -qb (x) (0, .); dw = qa . qb
  qa_bar = add4(scale4(dw_bar, qb), scale4(-1.f, qmul4(qb, pure(dv_bar))));
  qb_bar = add4(scale4(dw_bar, qa), qmul4(qa, pure(dv_bar)));
}

// VJP of rotate_inv(q, v) = v + 2 u x (u x v - w v) (u, w: vector and real part of q).
__device__ __forceinline__ void rotate_inv_vjp(float4 q, float3 v, float3 o_bar, float3& v_bar, float4& q_bar) {
  const float3 u = f3(q.x, q.y, q.z);
  const float3 s = cross3(u, v) - q.w * v;
  const float3 z_bar = 2.f * o_bar;
  float3 u_bar = cross3(s, z_bar);
  const float3 s_bar = cross3(z_bar, u);
  u_bar += cross3(v, s_bar);
  v_bar = o_bar + cross3(s_bar, u) - q.w * s_bar;
  q_bar = make_float4(u_bar.x, u_bar.y, u_bar.z, -dot3(v, s_bar));
}

// VJP of director3.
__device__ __forceinline__ float4 director3_vjp(float4 q, float3 a) {
  return make_float4(2.f * (q.z * a.x - q.w * a.y) - 4.f * q.x * a.z, 2.f * (q.w * a.x + q.z * a.y) - 4.f * q.y * a.z,
                     2.f * (q.x * a.x + q.y * a.y), 2.f * (q.y * a.x - q.x * a.y));
}

// VJP of segment_forces.
__device__ __forceinline__ void segment_forces_vjp(float3 ra, float3 rb, float4 q, const RodDev& R, bool extensible,
                                                   float3 fa_bar, float3 fb_bar, float3 tq_bar, float3& ra_bar,
                                                   float3& rb_bar, float4& q_bar) {
  const float3 e = rb - ra;
  const float ee = dot3(e, e);
  const float il = rsqrtf(ee);
  const float3 t = il * e;
  const float3 d3 = director3(q);
  const float c = dot3(t, d3);
  const float k = R.lKp;
  const float3 f_bar = fb_bar - fa_bar;
  const float3 g = d3 - c * t;
  float il_bar = k * dot3(g, f_bar);
  float3 d3_bar = (k * il) * f_bar;
  const float c_bar = -k * il * dot3(t, f_bar);
  float3 t_bar = (-k * il * c) * f_bar;
  t_bar += c_bar * d3;
  d3_bar += c_bar * t;
  float ee_bar = 0.f;
  if (extensible) {
    const float len = ee * il;
    const float3 fs_bar = fa_bar - fb_bar;
    t_bar += (R.Ks * (len * R.inv_l0 - 1.f)) * fs_bar;
    const float len_bar = R.Ks * R.inv_l0 * dot3(t, fs_bar);
    ee_bar += il * len_bar;
    il_bar += ee * len_bar;
  }
  // torque l0 Kp (-t_b.y, t_b.x, 0), t_b = R(q)^T t
  const float3 tb_bar = f3(k * tq_bar.y, -k * tq_bar.x, 0.f);
  float3 t_bar2;
  float4 q_bar_rot;
  rotate_inv_vjp(q, t, tb_bar, t_bar2, q_bar_rot);
  t_bar += t_bar2;
  q_bar = add4(q_bar_rot, director3_vjp(q, d3_bar));
  // t = il e, il = ee^(-1/2), ee = e . e
  float3 e_bar = il * t_bar;
  il_bar += dot3(e, t_bar);
  ee_bar += -0.5f * il * il * il * il_bar;
  e_bar += (2.f * ee_bar) * e;
  ra_bar = -e_bar;
  rb_bar = e_bar;
}

// Adjoint of one distance constraint (pre-update velocities va, vb): with
// g = s d and dg/dd = M = -(1/(dt W)) [(1 - l0/L) I + (l0/L) n n^T], returns
// d_bar = M (-wa va_bar + wb vb_bar); the caller applies va_bar -= dt d_bar,
// vb_bar += dt d_bar, ra_bar -= d_bar, rb_bar += d_bar.
__device__ __forceinline__ float3 constraint_vjp(float3 ra, float3 va, float3 rb, float3 vb, float wa, float wb,
                                                 float3 va_bar, float3 vb_bar, float l0, float dt) {
  const float3 d = f3(__fmaf_rn(dt, __fsub_rn(vb.x, va.x), __fsub_rn(rb.x, ra.x)),
                      __fmaf_rn(dt, __fsub_rn(vb.y, va.y), __fsub_rn(rb.y, ra.y)),
                      __fmaf_rn(dt, __fsub_rn(vb.z, va.z), __fsub_rn(rb.z, ra.z)));
  const float dd = __fmaf_rn(d.x, d.x, __fmaf_rn(d.y, d.y, __fmul_rn(d.z, d.z)));
  const float il = rsqrtf(dd);
  const float3 n = il * d;
  const float3 g_bar = f3(__fmaf_rn(wb, vb_bar.x, -__fmul_rn(wa, va_bar.x)),
                          __fmaf_rn(wb, vb_bar.y, -__fmul_rn(wa, va_bar.y)),
                          __fmaf_rn(wb, vb_bar.z, -__fmul_rn(wa, va_bar.z)));
  const float rho = l0 * il;
  const float inv = -__frcp_rn(__fmul_rn(dt, wa + wb));
  return inv * ((1.f - rho) * g_bar + (rho * dot3(n, g_bar)) * n);
}

// Asynchronous 16-byte global -> shared copies (completed by cp_async_wait_all).
__device__ __forceinline__ void cp_async16(float4* dst_smem, const float4* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// constraint_vjp in two parts.  The geometry (direction n and l0/L of the predicted
// segment) depends only on the recorded velocities, so it is computed before the
// exchange of the adjoint velocities; inv = -1/(dt W) is constant over a step, and 0
// for a constraint that does not exist (its geometry is then a safe unit vector and the
// returned d_bar is 0).  Same arithmetic as constraint_vjp.
struct VjpGeo {
  float3 n;
  float rho;
};
__device__ __forceinline__ float vjp_inv(bool exists, float wa, float wb, float dt) {
  return (exists && wa + wb > 0.f) ? -__frcp_rn(__fmul_rn(dt, wa + wb)) : 0.f;
}
__device__ __forceinline__ VjpGeo vjp_geo(float3 ra, float3 va, float3 rb, float3 vb, float inv, float l0,
                                          float dt) {
  float3 d = f3(__fmaf_rn(dt, __fsub_rn(vb.x, va.x), __fsub_rn(rb.x, ra.x)),
                __fmaf_rn(dt, __fsub_rn(vb.y, va.y), __fsub_rn(rb.y, ra.y)),
                __fmaf_rn(dt, __fsub_rn(vb.z, va.z), __fsub_rn(rb.z, ra.z)));
  if (inv == 0.f) d = f3(0.f, 0.f, 1.f);
  const float dd = __fmaf_rn(d.x, d.x, __fmaf_rn(d.y, d.y, __fmul_rn(d.z, d.z)));
  const float il = rsqrtf(dd);
  return VjpGeo{il * d, l0 * il};
}
__device__ __forceinline__ float3 vjp_apply(const VjpGeo& G, float inv, float wa, float wb, float3 va_bar,
                                            float3 vb_bar) {
  const float3 g_bar = f3(__fmaf_rn(wb, vb_bar.x, -__fmul_rn(wa, va_bar.x)),
                          __fmaf_rn(wb, vb_bar.y, -__fmul_rn(wa, va_bar.y)),
                          __fmaf_rn(wb, vb_bar.z, -__fmul_rn(wa, va_bar.z)));
  return inv * ((1.f - G.rho) * g_bar + (G.rho * dot3(G.n, g_bar)) * G.n);
}

// One step of the reverse pass.  sweep_v holds the step's velocity records in the layout
// step_body writes with STORE == 2 (COMPACT) or STORE == 1.
template <int EPT, int NT, bool COMPACT>
__device__ __forceinline__ void reverse_step(const RodDev& R, const int t, const float3 (&r)[EPT],
                                             const float4 (&q)[EPT], const float3 (&om)[EPT], const float (&w)[EPT],
                                             const float3 (&om1)[EPT], const float4 (&qo)[EPT],
                                             const StepNeighbours& nb, const float4* par_u, const float4* par_k,
                                             float4* halo, int& xc, const float4* sweep_v,
                                             const StepCache<EPT>& sc, float3 (&rb)[EPT],
                                             float3 (&vb)[EPT], float4 (&qb)[EPT], float3 (&ob)[EPT],
                                             float3 (&Kb)[EPT], float3 (&ub)[EPT]) {
  const int e0 = t * EPT;
  const int n = R.n;
  const bool inext = (R.flags & F_INEXT) != 0;
  const bool clamp = (R.flags & F_CLAMP) != 0;
  const float dt = R.dt;
  const float half_dt = 0.5f * dt;

  // ---- position update: r' = r + dt v2, q' = normalize(q + dt/2 q (x) (0, omega1))
  float3 vb2[EPT], ob1[EPT];
  float4 qbi[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = e0 + e;
    vb2[e] = vb[e] + dt * rb[e];
    ob1[e] = ob[e];
    qbi[e] = zero4();
    if (i <= n - 2) {
      const float4 a = q[e];
      const float3 o = om1[e];
      const float dx = a.w * o.x + a.y * o.z - a.z * o.y;
      const float dy = a.w * o.y + a.z * o.x - a.x * o.z;
      const float dz = a.w * o.z + a.x * o.y - a.y * o.x;
      const float dwq = -(a.x * o.x + a.y * o.y + a.z * o.z);
      const float4 p = make_float4(a.x + half_dt * dx, a.y + half_dt * dy, a.z + half_dt * dz, a.w + half_dt * dwq);
      const float inv = rsqrtf(dot4(p, p));
      const float4 pb = scale4(inv, add4(qb[e], scale4(-dot4(qo[e], qb[e]), qo[e])));
      qbi[e] = add4(pb, scale4(half_dt, qmul4(pb, make_float4(-o.x, -o.y, -o.z, 0.f))));
      ob1[e] += half_dt * im_conj_mul(a, pb);
    }
  }

  // ---- constraint half-sweeps in reverse order (odd, then even, last iteration first)
  if (inext) {
    const BlockHalo<NT, NT> H{t};
    // -1 / (dt W) of every constraint the thread touches (constant over the step)
    constexpr int NE = EPT / 2, NO = EPT / 2 - 1 > 0 ? EPT / 2 - 1 : 1;
    float inv_e[NE], inv_o[NO];
#pragma unroll
    for (int k = 0; k < NE; ++k) inv_e[k] = vjp_inv(e0 + 2 * k + 1 <= n - 1, w[2 * k], w[2 * k + 1], dt);
#pragma unroll
    for (int k = 0; k < NO; ++k)
      inv_o[k] = vjp_inv(EPT / 2 > 1 && e0 + 2 * k + 2 <= n - 1, w[(2 * k + 1) % EPT], w[(2 * k + 2) % EPT], dt);
    const float inv_r = vjp_inv(t + 1 < NT && e0 + EPT <= n - 1, w[EPT - 1], nb.w_next, dt);
    const float inv_l = vjp_inv(t > 0 && e0 <= n - 1, nb.w_prev, w[0], dt);
    const int tn = min(t + 1, NT - 1), tp = max(t - 1, 0);  // in-range neighbour slots
    // the forward's boundary segment vectors (positions are fixed during the sweeps)
    static_assert(!COMPACT || EPT == 2, "the rebuilt even-sweep input assumes no odd segment inside a thread");
    const float3 e_r = safe_segment(sc.i_right, segment_vector(r[EPT - 1], nb.r_next), R.l0);
    const float3 e_l = safe_segment(sc.i_left, segment_vector(nb.r_prev, r[0]), R.l0);
    const Vec3x2 e_bnd{make_float2(e_r.x, e_l.x), make_float2(e_r.y, e_l.y), make_float2(e_r.z, e_l.z)};
#pragma unroll 2
    for (int it = R.n_iters - 1; it >= 0; --it) {
      // geometry of this iteration's constraints, from the recorded velocities
      const int so = COMPACT ? 1 + it : 2 * it + 1;  // record slot before the odd half-sweep
      // the velocities before the even half-sweep: recorded; in the compact layout only for
      // the first iteration, and for a later one the odd half-sweep of the iteration before
      // repeated on its recorded input (the forward's own arithmetic, so the same values)
      float3 ve[EPT];
      {
        // slot 2 it; compact: slot 0, or the record before the previous odd half-sweep
        const int sp = COMPACT ? it : 2 * it;
#pragma unroll
        for (int e = 0; e < EPT; ++e) ve[e] = rec_get<EPT, NT>(sweep_v, sp, e, t);
        if (COMPACT && it > 0) {
          const float3 vn = t + 1 < NT ? rec_get<EPT, NT>(sweep_v, sp, 0, tn) : zero3();
          const float3 vp = t > 0 ? rec_get<EPT, NT>(sweep_v, sp, EPT - 1, tp) : zero3();
          boundary_apply(e_bnd, sc.l_bnd, sc.c_bnd, dt, vn, vp, ve[EPT - 1], ve[0]);
        }
      }
      VjpGeo g_o[NO], g_e[NE];
#pragma unroll
      for (int k = 0; k + 1 < EPT / 2; ++k) {
        const int a = 2 * k + 1, b = 2 * k + 2;
        g_o[k] = vjp_geo(r[a], rec_get<EPT, NT>(sweep_v, so, a, t), r[b], rec_get<EPT, NT>(sweep_v, so, b, t),
                         inv_o[k], R.l0, dt);
      }
      const VjpGeo g_r = vjp_geo(r[EPT - 1], rec_get<EPT, NT>(sweep_v, so, EPT - 1, t), nb.r_next,
                                 rec_get<EPT, NT>(sweep_v, so, 0, tn), inv_r, R.l0, dt);
      const VjpGeo g_l = vjp_geo(nb.r_prev, rec_get<EPT, NT>(sweep_v, so, EPT - 1, tp), r[0],
                                 rec_get<EPT, NT>(sweep_v, so, 0, t), inv_l, R.l0, dt);
#pragma unroll
      for (int k = 0; k < NE; ++k) {
        const int a = 2 * k, b = 2 * k + 1;
        g_e[k] = vjp_geo(r[a], ve[a], r[b], ve[b], inv_e[k], R.l0, dt);
      }
      // exchange of the adjoint velocities of the first and last element
      float4* hb = halo + (xc & 1) * kHaloSlots * NT;
      ++xc;
      H.put3(hb, 0, vb2[0]);
      H.put3(hb, 1, vb2[EPT - 1]);
      // odd segments inside the thread (elements 1 .. EPT - 2: not exchanged)
#pragma unroll
      for (int k = 0; k + 1 < EPT / 2; ++k) {
        const int a = 2 * k + 1, b = 2 * k + 2;
        const float3 db = vjp_apply(g_o[k], inv_o[k], w[a], w[b], vb2[a], vb2[b]);
        vb2[a] -= dt * db;
        vb2[b] += dt * db;
        rb[a] -= db;
        rb[b] += db;
      }
      block_sync<NT>();
      const float3 vn_bar = H.next3(hb, 0), vp_bar = H.prev3(hb, 1);  // read only where the constraint exists
      {
        const float3 db = vjp_apply(g_r, inv_r, w[EPT - 1], nb.w_next, vb2[EPT - 1], t + 1 < NT ? vn_bar : zero3());
        vb2[EPT - 1] -= dt * db;
        rb[EPT - 1] -= db;
      }
      {
        const float3 db = vjp_apply(g_l, inv_l, nb.w_prev, w[0], t > 0 ? vp_bar : zero3(), vb2[0]);
        vb2[0] += dt * db;
        rb[0] += db;
      }
#pragma unroll
      for (int k = 0; k < NE; ++k) {
        const int a = 2 * k, b = 2 * k + 1;
        const float3 db = vjp_apply(g_e[k], inv_e[k], w[a], w[b], vb2[a], vb2[b]);
        vb2[a] -= dt * db;
        vb2[b] += dt * db;
        rb[a] -= db;
        rb[b] += db;
      }
    }
  }

  // ---- force integration: v1 = damp (v + dt (w F + g)), omega1 = damp (...)
  float3 Fb[EPT], Tb[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = e0 + e;
    if (w[e] > 0.f) {
      Fb[e] = (R.damp * dt * w[e]) * vb2[e];
      vb[e] = R.damp * vb2[e];
    } else {
      Fb[e] = zero3();
      vb[e] = zero3();
    }
    const bool frame_dynamic = (i <= n - 2) && !(clamp && i == 0);
    if (frame_dynamic) {
      const float3 b = f3(R.Jinv1 * ob1[e].x, R.Jinv1 * ob1[e].y, R.Jinv3 * ob1[e].z);
      Tb[e] = (R.damp * dt) * b;
      const float3 o = om[e];
      const float3 Jw = f3(R.J1 * o.x, R.J1 * o.y, R.J3 * o.z);
      const float3 oxb = cross3(o, b);
      const float3 Joxb = f3(R.J1 * oxb.x, R.J1 * oxb.y, R.J3 * oxb.z);
      ob[e] = R.damp * (ob1[e] + dt * (Joxb - cross3(Jw, b)));
    } else {
      Tb[e] = zero3();
      ob[e] = zero3();
    }
  }

  // ---- elastic forces and torques (transposed)
  float4* hb = halo + (xc & 1) * kHaloSlots * NT;
  ++xc;
  hb[t] = make_float4(Fb[0].x, Fb[0].y, Fb[0].z, 0.f);
  hb[NT + t] = make_float4(Tb[0].x, Tb[0].y, Tb[0].z, 0.f);
  block_sync<NT>();
  float3 Fb_next = zero3(), Tb_next = zero3();
  if (t + 1 < NT) {
    Fb_next = f3(hb[t + 1]);
    Tb_next = f3(hb[NT + t + 1]);
  }
  float3 r_carry = zero3();
  float4 q_carry = zero4();
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int j = e0 + e;
    const float4 qn = (e + 1 < EPT) ? q[(e + 1) % EPT] : nb.q_next;
    const float3 rn = (e + 1 < EPT) ? r[(e + 1) % EPT] : nb.r_next;
    if (j <= n - 3) {
      const float3 tbar_b = (e + 1 < EPT) ? Tb[(e + 1) % EPT] : Tb_next;
      float4 qa_bar, qn_bar;
      float3 K_bar, uh_bar;
      joint_torques_vjp(q[e], qn, par_u[e * NT + t], par_k[e * NT + t], R.two_over_l, Tb[e], tbar_b, qa_bar, qn_bar,
                        K_bar, uh_bar);
      qbi[e] = add4(qbi[e], qa_bar);
      if (e + 1 < EPT) {
        qbi[(e + 1) % EPT] = add4(qbi[(e + 1) % EPT], qn_bar);
      } else {
        q_carry = qn_bar;
      }
      Kb[e] += K_bar;
      ub[e] += uh_bar;
    }
    if (j <= n - 2) {
      const float3 fbar_b = (e + 1 < EPT) ? Fb[(e + 1) % EPT] : Fb_next;
      float3 ra_bar, rn_bar;
      float4 q_bar;
      segment_forces_vjp(r[e], rn, q[e], R, !inext, Fb[e], fbar_b, Tb[e], ra_bar, rn_bar, q_bar);
      rb[e] += ra_bar;
      if (e + 1 < EPT) {
        rb[(e + 1) % EPT] += rn_bar;
      } else {
        r_carry = rn_bar;
      }
      qbi[e] = add4(qbi[e], q_bar);
    }
  }
  hb = halo + (xc & 1) * kHaloSlots * NT;
  ++xc;
  hb[t] = make_float4(r_carry.x, r_carry.y, r_carry.z, 0.f);
  hb[NT + t] = q_carry;
  block_sync<NT>();
  if (t > 0) {
    rb[0] += f3(hb[t - 1]);
    qbi[0] = add4(qbi[0], hb[NT + t - 1]);
  }
#pragma unroll
  for (int e = 0; e < EPT; ++e) qb[e] = qbi[e];
}

// Reverse pass over the whole rollout of one rod per block.  MODE 0: recompute every
// step before its reverse; 1: record mode with one sweep buffer (a step's records are
// copied in after the step before it is reversed); 2: record mode with two buffers (the
// copy overlaps the reverse of the step before).  PIPE (record mode, two buffers, full
// layout): each rod has a cluster of two blocks; the first records the segments, the
// second reverses them one segment behind, so that the recording of segment k - 1 runs
// while segment k is reversed (segment scratch in two sets, by segment parity; one
// cluster barrier per segment).
template <int NT, int MODE, bool COMPACT, bool PIPE = false>
__global__ void __launch_bounds__(NT)
adjoint_kernel(AdjointArgs a) {
  static_assert(!PIPE || (MODE == 2 && !COMPACT), "the pipelined form records the full layout");
  constexpr bool RECORD = MODE > 0;
  constexpr int STORE = COMPACT ? 2 : 1;  // step_body's record layout
  constexpr int NBUF = MODE == 2 ? 2 : 1;
  constexpr int EPT = 2;
  static_assert((3 * EPT * NT) % 4 == 0, "a record slot is a whole number of 16-byte pieces");
  extern __shared__ float4 smem[];
  float4* par_u = smem;
  float4* par_k = smem + EPT * NT;
  float4* halo = smem + 2 * EPT * NT;
  float4* sweep_v = halo + 2 * kHaloSlots * NT;
  // float4 per (step, block) record: 1 + n_iters (compact) or 2 n_iters slots of 3 EPT NT
  // floats (rec_put)
  const int64_t rec_stride = (int64_t)(COMPACT ? a.rec_iters + 1 : 2 * a.rec_iters) * 3 * EPT * NT / 4;

  const int rod_slot = PIPE ? (int)blockIdx.x / 2 : (int)blockIdx.x;  // the rod's place in the launch
  const int n_slots = PIPE ? (int)gridDim.x / 2 : (int)gridDim.x;
  const int role = PIPE ? (int)(blockIdx.x & 1) : 0;  // PIPE: 0 records, 1 reverses (the cluster rank)
  const int rid = a.work[rod_slot];
  const RodDev R = a.rods[rid];
  const int t = threadIdx.x;
  const int e0 = t * EPT;
  const int64_t E = a.n_elem;
  float3 v_drive = zero3(), w_drive = zero3();
  if (a.drive != nullptr) {
    v_drive = f3(a.drive[2 * rid]);
    w_drive = f3(a.drive[2 * rid + 1]);
  }

  float3 r[EPT], v[EPT], om[EPT];
  float4 q[EPT];
  float w[EPT];
  float3 rb[EPT], vb[EPT], ob[EPT], Kb[EPT], ub[EPT];
  float4 qb[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    rb[e] = vb[e] = ob[e] = Kb[e] = ub[e] = zero3();
    qb[e] = zero4();
  }
  const BlockHalo<NT, NT> H{t};
  int xc = 0;
  StepCache<EPT> sc;  // launch constants of the step (filled on the first step)
  const int n_seg = (a.n_steps + a.ckpt_every - 1) / a.ckpt_every;
  bool params_loaded = false;
  // segment scratch: states 0 .. K and the velocity records of segment seg (two sets by
  // segment parity with PIPE)
  auto seg_base = [&](int seg) {
    return a.seg_states + (PIPE ? (int64_t)(seg & 1) * (a.ckpt_every + 1) * 4 * E : (int64_t)0);
  };
  auto rec_at = [&](int seg, int s) {
    return a.sweep_rec + ((int64_t)(PIPE ? (seg & 1) * a.ckpt_every : 0) + s) * n_slots * rec_stride +
           (int64_t)rod_slot * rec_stride;
  };
  // copies step s's record into a shared buffer: 16-byte pieces spread over the block
  // (a barrier orders them before any thread's reads; a block or cluster barrier orders
  // the recording pass's stores before them)
  auto fetch = [&](int seg, int s, float4* dst) {
    const float4* src = rec_at(seg, s);
    const int slots = R.n_iters > 0 ? (COMPACT ? R.n_iters + 1 : 2 * R.n_iters) : 0;
    const int n16 = slots * 3 * EPT * NT / 4;
    for (int k = t; k < n16; k += NT) cp_async16(dst + k, src + k);
    cp_async_commit();
  };
  // rounds: without PIPE round j records (or recomputes) segment n_seg - 1 - j and then
  // reverses it; with PIPE round j records segment n_seg - 1 - j (first block) while the
  // second block reverses segment n_seg - j
  const int n_round = PIPE ? n_seg + 1 : n_seg;
  for (int j = 0; j < n_round; ++j) {
    const int rec_seg = n_seg - 1 - j;
    const int rev_seg = PIPE ? n_seg - j : rec_seg;
    const bool do_rec = rec_seg >= 0 && role == 0;
    const bool do_rev = rev_seg >= 0 && rev_seg < n_seg && (!PIPE || role == 1);
    if (do_rec || !params_loaded) {
      // the recording (or recomputing) block loads the segment's checkpoint; a reversing
      // block only the inverse masses and joint parameters, once
      const int ls = do_rec ? rec_seg : n_seg - 1;
      const float4* ck = a.ckpt + (int64_t)ls * 4 * E;
      load_rod<EPT, NT>(R, t, t, ck, ck + E, ck + 2 * E, ck + 3 * E, a.u4, a.k4, r, v, q, om, w,
                        params_loaded ? nullptr : par_u, par_k);
      params_loaded = true;
    }
    if (do_rec) {
      const int cnt = min(a.ckpt_every, a.n_steps - rec_seg * a.ckpt_every);
      auto put_state = [&](int s) {
        float4* st = seg_base(rec_seg) + (int64_t)s * 4 * E + R.off;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          if (e0 + e < R.n) {
            st[e0 + e] = make_float4(r[e].x, r[e].y, r[e].z, w[e]);
            if constexpr (!RECORD) st[E + e0 + e] = make_float4(v[e].x, v[e].y, v[e].z, 0.f);  // record mode reads none
            st[2 * E + e0 + e] = q[e];
            st[3 * E + e0 + e] = make_float4(om[e].x, om[e].y, om[e].z, 0.f);
          }
        }
      };
      if constexpr (RECORD) {
        // forward over the segment, keeping states 0 .. cnt and the velocity records
        for (int s = 0; s < cnt; ++s) {
          put_state(s);
          StepNeighbours nb;
          step_body<EPT, NT, STORE>(R, H, r, v, q, om, w, par_u, par_k, halo, xc, sc, v_drive, w_drive,
                                    rec_at(rec_seg, s), &nb);
        }
        put_state(cnt);
      } else {
        // recompute the segment's states into scratch
        for (int s = 0; s < cnt; ++s) {
          put_state(s);
          if (s + 1 < cnt)
            step_body<EPT, NT, 0>(R, H, r, v, q, om, w, par_u, par_k, halo, xc, sc, v_drive, w_drive, nullptr,
                                  nullptr);
        }
      }
    }
    if (!do_rev) {
      if constexpr (PIPE) cooperative_groups::this_cluster().sync();
      continue;
    }
    const int seg = rev_seg;
    const int t0 = seg * a.ckpt_every;
    const int cnt = min(a.ckpt_every, a.n_steps - t0);
    if constexpr (RECORD) {
      // the recording pass's stores are visible here: a block barrier follows each step's
      // records within step_body, or (PIPE) the cluster barrier ended the round that wrote
      // them
      fetch(seg, cnt - 1, sweep_v + ((cnt - 1) % NBUF) * rec_stride);
    }
    // reverse the segment's steps
    if constexpr (RECORD) {
      // Each step's inputs are loaded one step ahead, while the step before is reversed:
      // the state before it, its neighbour data and the loss gradient after it.  The frame
      // and angular velocity after step s are the state before step s + 1.  The segment
      // states are read from L2 (ld.cg): with PIPE another SM wrote them.
      float3 pr[EPT], pom[EPT], pg[EPT];
      float4 pq[EPT], pn0, pn1, pn2;
      float4 nq[EPT];
      float3 nom[EPT];
      auto prefetch = [&](int s) {
        const float4* st = seg_base(seg) + (int64_t)s * 4 * E + R.off;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          pg[e] = zero3();
          if (e0 + e < R.n) {
            pr[e] = f3(__ldcg(st + e0 + e));
            pq[e] = __ldcg(st + 2 * E + e0 + e);
            pom[e] = f3(__ldcg(st + 3 * E + e0 + e));
            if (a.dLdpos != nullptr) pg[e] = f3(a.dLdpos[(int64_t)(t0 + s) * E + R.off + e0 + e]);
          }
        }
        // the neighbour data of the step: the neighbouring threads' nodes in the same state
        // (read where the constraint or joint exists; an in-range node elsewhere)
        const int in = min(e0 + EPT, R.n - 1), ip = min(max(e0 - 1, 0), R.n - 1);
        pn0 = __ldcg(st + in);
        pn1 = __ldcg(st + ip);
        pn2 = __ldcg(st + 2 * E + in);
      };
      {
        const float4* sn = seg_base(seg) + (int64_t)cnt * 4 * E + R.off;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          nq[e] = q[e];
          nom[e] = om[e];
          if (e0 + e < R.n) {
            nq[e] = __ldcg(sn + 2 * E + e0 + e);
            nom[e] = f3(__ldcg(sn + 3 * E + e0 + e));
          }
        }
      }
      prefetch(cnt - 1);
      for (int s = cnt - 1; s >= 0; --s) {
        float3 r_in[EPT], om_in[EPT];
        float4 q_in[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          if (e0 + e < R.n) {
            r[e] = pr[e];
            q[e] = pq[e];
            om[e] = pom[e];
          }
          r_in[e] = r[e];
          q_in[e] = q[e];
          om_in[e] = om[e];
          if (a.dLdpos != nullptr && e0 + e < R.n) rb[e] += pg[e];  // loss gradient after this step
          if (e0 + e < R.n) {
            q[e] = nq[e];
            om[e] = nom[e];
          }
          nq[e] = q_in[e];
          nom[e] = om_in[e];
        }
        StepNeighbours nb;
        nb.r_next = f3(pn0);
        nb.w_next = pn0.w;
        nb.r_prev = f3(pn1);
        nb.w_prev = pn1.w;
        nb.q_next = pn2;
        // step s's sweeps (threads read their neighbours' entries too); with two buffers the
        // copy of step s - 1's starts once every thread is done with the buffer it reuses
        // (step s + 1's), with one buffer once every thread is done with step s's
        cp_async_wait_all();
        block_sync<NT>();
        if (s > 0) {
          if constexpr (NBUF == 2) fetch(seg, s - 1, sweep_v + ((s - 1) & 1) * rec_stride);
          prefetch(s - 1);
        }
        reverse_step<EPT, NT, COMPACT>(R, t, r_in, q_in, om_in, w, om, q, nb, par_u, par_k, halo, xc,
                                       sweep_v + (s % NBUF) * rec_stride, sc, rb, vb, qb, ob, Kb, ub);
        if constexpr (NBUF == 1) {
          if (s > 0) {
            block_sync<NT>();
            fetch(seg, s - 1, sweep_v);
          }
        }
      }
    } else {
      // each step's state and loss gradient loaded one step ahead, as in record mode
      float3 pr[EPT], pv[EPT], pom[EPT], pg[EPT];
      float4 pq[EPT];
      auto prefetch = [&](int s) {
        const float4* st = seg_base(seg) + (int64_t)s * 4 * E + R.off;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          pg[e] = zero3();
          if (e0 + e < R.n) {
            pr[e] = f3(st[e0 + e]);
            pv[e] = f3(st[E + e0 + e]);
            pq[e] = st[2 * E + e0 + e];
            pom[e] = f3(st[3 * E + e0 + e]);
            if (a.dLdpos != nullptr) pg[e] = f3(a.dLdpos[(int64_t)(t0 + s) * E + R.off + e0 + e]);
          }
        }
      };
      prefetch(cnt - 1);
      for (int s = cnt - 1; s >= 0; --s) {
        float3 r_in[EPT], om_in[EPT], g_s[EPT];
        float4 q_in[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          if (e0 + e < R.n) {
            r[e] = pr[e];
            v[e] = pv[e];
            q[e] = pq[e];
            om[e] = pom[e];
          }
          r_in[e] = r[e];
          q_in[e] = q[e];
          om_in[e] = om[e];
          g_s[e] = pg[e];
        }
        if (s > 0) prefetch(s - 1);
        StepNeighbours nb;
        step_body<EPT, NT, STORE>(R, H, r, v, q, om, w, par_u, par_k, halo, xc, sc, v_drive, w_drive, sweep_v, &nb);
        // loss gradient with respect to the positions after this step
        if (a.dLdpos != nullptr) {
#pragma unroll
          for (int e = 0; e < EPT; ++e)
            if (e0 + e < R.n) rb[e] += g_s[e];
        }
        reverse_step<EPT, NT, COMPACT>(R, t, r_in, q_in, om_in, w, om, q, nb, par_u, par_k, halo, xc, sweep_v, sc,
                                       rb, vb, qb, ob, Kb, ub);
      }
    }
    if constexpr (PIPE) cooperative_groups::this_cluster().sync();  // end of the round
  }
  if (PIPE && role == 0) return;  // the recording block holds no gradients
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = e0 + e;
    if (i < R.n) {
      const int64_t o = R.off + i;
      if (a.dpos0) a.dpos0[o] = make_float4(rb[e].x, rb[e].y, rb[e].z, 0.f);
      if (a.dvel0) a.dvel0[o] = make_float4(vb[e].x, vb[e].y, vb[e].z, 0.f);
      if (a.dquat0) a.dquat0[o] = qb[e];
      if (a.domega0) a.domega0[o] = make_float4(ob[e].x, ob[e].y, ob[e].z, 0.f);
      if (a.dK) a.dK[o] = make_float4(Kb[e].x, Kb[e].y, Kb[e].z, 0.f);
      if (a.duhat) a.duhat[o] = make_float4(ub[e].x, ub[e].y, ub[e].z, 0.f);
    }
  }
}

using AdjointFn = void (*)(AdjointArgs);
template <int NT>
AdjointFn adjoint_fn_nt(int mode, bool compact) {
  switch (mode) {
    case 0: return compact ? adjoint_kernel<NT, 0, true> : adjoint_kernel<NT, 0, false>;
    case 1: return compact ? adjoint_kernel<NT, 1, true> : adjoint_kernel<NT, 1, false>;
    case 2: return compact ? adjoint_kernel<NT, 2, true> : adjoint_kernel<NT, 2, false>;
    default: return nullptr;
  }
}
// The reverse kernel of `nt` threads in `mode`, with the compact record layout or not
// (nullptr for a thread count that does not exist).
AdjointFn adjoint_fn(int nt, int mode, bool compact) {
  switch (nt) {
    case 32: return adjoint_fn_nt<32>(mode, compact);
    case 64: return adjoint_fn_nt<64>(mode, compact);
    case 128: return adjoint_fn_nt<128>(mode, compact);
    case 256: return adjoint_fn_nt<256>(mode, compact);
    default: return nullptr;
  }
}

// The pipelined reverse kernel (record mode, two buffers, full layout) of `nt` threads.
AdjointFn adjoint_pipe_fn(int nt) {
  switch (nt) {
    case 32: return adjoint_kernel<32, 2, false, true>;
    case 64: return adjoint_kernel<64, 2, false, true>;
    case 128: return adjoint_kernel<128, 2, false, true>;
    case 256: return adjoint_kernel<256, 2, false, true>;
    default: return nullptr;
  }
}

}  // namespace

int adjoint_smem_bytes(int nt, int n_iters, int mode, bool compact) {
  const int ept = 2;
  const int it = n_iters > 0 ? n_iters : 1;
  const int sweep = (compact ? it + 1 : 2 * it) * 3 * ept * nt / 4;  // record slots of one step, in float4
  return (2 * ept * nt + 2 * kHaloSlots * nt + (mode == 2 ? 2 : 1) * sweep) * (int)sizeof(float4);
}

cudaError_t adjoint_occupancy(int nt, int mode, bool compact, int smem, int* blocks) {
  const AdjointFn fn = adjoint_fn(nt, mode, compact);
  if (fn == nullptr) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, nt, (size_t)smem);
}

cudaError_t preload_adjoint(int nt) {
  for (int c = 0; c < 2; ++c) {
    const AdjointFn fn = adjoint_fn(nt, 0, c != 0);
    if (fn == nullptr) return cudaErrorInvalidValue;
    cudaFuncAttributes at;
    cudaError_t e = cudaFuncGetAttributes(&at, fn);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_adjoint(int nt, int mode, bool compact, const AdjointArgs& a, int n_blocks, int smem,
                           cudaStream_t s) {
  if ((mode > 0) != (a.sweep_rec != nullptr)) return cudaErrorInvalidValue;
  const AdjointFn fn = adjoint_fn(nt, mode, compact);
  if (fn == nullptr) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  fn<<<n_blocks, nt, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_pipe(int nt, const AdjointArgs& a, int n_rods, int smem, cudaStream_t s) {
  if (a.sweep_rec == nullptr) return cudaErrorInvalidValue;
  const AdjointFn fn = adjoint_pipe_fn(nt);
  if (fn == nullptr) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * n_rods);
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, a);
}

}  // namespace corde
