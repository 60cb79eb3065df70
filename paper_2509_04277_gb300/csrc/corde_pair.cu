// Catheter/guidewire pair in one thread block (Section 3.4): the outer rod (catheter)
// on threads [0, NT), the inner rod (guidewire) on threads [NT, 2 NT), stepped in
// lockstep by the shared step body, with the binding constraints C_b (Section 2.1
// "Constraints": distance constraints of rest length zero) applied after every
// iteration's odd distance sweep.
//
// Binding reading: both rods share the rest segment length l0; inner node i is bound to
// the outer centreline point at arclength (i + beta) l0 - segment k = floor(i + beta),
// fraction a = (i + beta) - k - when 0 <= k <= N_outer - 2.  beta, the inner rod's
// insertion relative to the outer rod in segments, is a per-launch input (slot 3 of the
// inner rod's drive row).  Mode 1 (v1, one-way): the outer rod is not moved by binding.
// Mode 2 (v2, two-way): the impulse is shared by inverse mass.  Mode 0 (v0): no binding.
// The impulses are applied in two colors (even inner nodes, then odd), so that within a
// color no two constraints touch the same outer node; the outer rod's velocities are
// staged in shared memory for the inner threads to read (and, in v2, to update).
#include "corde_step.cuh"
#include "corde_variants.cuh"

namespace corde {
namespace {

template <int SYNC_NT, int EPT, bool DYN_BETA>
struct PairHook {
  int group;       // 0 outer, 1 inner
  int t;           // thread index within the group
  int mode;        // 0, 1, 2
  const float* beta_sh;  // binding offset beta (shared: the mailbox may change it between steps)
  mutable int k0;        // floor(beta) of this step
  mutable float alpha;   // beta - k0
  int n_out;       // outer nodes
  int n_in;        // inner nodes
  float dt;
  float4* out_r;   // [capacity] outer positions and inverse masses (once per step)
  float4* out_v;   // [capacity] outer velocities (every iteration)
  // per step, inner nodes only (positions and masses are fixed during the sweeps):
  mutable float3 rp[EPT];   // node position minus its binding point on the outer centreline
  mutable float inv[EPT];   // -1 / (dt w_eff), 0 when the node has no binding this step
  mutable float sk[EPT], sk1[EPT];  // v2: (1 - a) w_k and a w_k+1, the outer nodes' shares

  template <int E>
  __device__ __forceinline__ void before_iterations(const float3 (&r)[E], const float (&w)[E]) const {
    if (mode == 0) return;
    if constexpr (DYN_BETA) {
      const float beta = *beta_sh;  // written before this step's force-phase barriers
      k0 = (int)floorf(beta);
      alpha = beta - floorf(beta);
    }
    if (group == 0) {
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int i = t * EPT + e;
        if (i < n_out) out_r[i] = make_float4(r[e].x, r[e].y, r[e].z, w[e]);
      }
    }
    block_sync<SYNC_NT>();
    if (group == 1) {
      const float a = alpha, b = 1.f - alpha;
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int i = t * EPT + e;
        const int k = i + k0;
        inv[e] = 0.f;
        rp[e] = zero3();
        sk[e] = sk1[e] = 0.f;
        if (i >= n_in || k < 0 || k > n_out - 2) continue;
        const float4 rk = out_r[k], rk1 = out_r[k + 1];
        const float wk = mode == 2 ? rk.w : 0.f, wk1 = mode == 2 ? rk1.w : 0.f;
        const float weff = w[e] + b * b * wk + a * a * wk1;
        if (!(weff > 0.f)) continue;
        const float3 pc = f3(b * rk.x + a * rk1.x, b * rk.y + a * rk1.y, b * rk.z + a * rk1.z);
        rp[e] = r[e] - pc;
        inv[e] = -1.f / (dt * weff);
        sk[e] = b * wk;
        sk1[e] = a * wk1;
      }
    }
  }

  // One inner node's binding: lambda = -(d) / (dt w_eff) with d the predicted offset from
  // its binding point; the node moves by w lambda, in v2 the two outer nodes by their shares.
  __device__ __forceinline__ float3 binding(int e, float3 ve, float3& vk, float3& vk1) const {
    const float a = alpha, b = 1.f - alpha;
    const float3 vc = f3(b * vk.x + a * vk1.x, b * vk.y + a * vk1.y, b * vk.z + a * vk1.z);
    const float3 d = rp[e] + dt * (ve - vc);
    return inv[e] * d;
  }

  template <int E>
  __device__ __forceinline__ void after_odd(const float3 (&r)[E], float3 (&v)[E], const float (&w)[E]) const {
    if (mode == 0) return;
    if (group == 0) {
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int i = t * EPT + e;
        if (i < n_out) out_v[i] = make_float4(v[e].x, v[e].y, v[e].z, 0.f);
      }
    }
    block_sync<SYNC_NT>();
    if (mode == 1) {
      // one-way: the outer rod does not move, so the two colors are independent and run
      // together (the same result as in order)
      if (group == 1) {
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          // branch-free: an unbound node (inv = 0) reads an in-range point and adds an
          // exact zero
          const int k = min(max(t * EPT + e + k0, 0), n_out - 2);
          float3 vk = f3(out_v[k]), vk1 = f3(out_v[k + 1]);
          v[e] += w[e] * binding(e, v[e], vk, vk1);
        }
      }
      return;
    }
#pragma unroll
    for (int color = 0; color < 2; ++color) {
      if (group == 1) {
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          if ((e & 1) != color || inv[e] == 0.f) continue;  // EPT is even: node parity = e parity
          const int k = t * EPT + e + k0;
          float3 vk = f3(out_v[k]), vk1 = f3(out_v[k + 1]);
          const float3 lam = binding(e, v[e], vk, vk1);
          v[e] += w[e] * lam;
          const float3 dk = sk[e] * lam, dk1 = sk1[e] * lam;
          out_v[k] = make_float4(vk.x - dk.x, vk.y - dk.y, vk.z - dk.z, 0.f);
          out_v[k + 1] = make_float4(vk1.x - dk1.x, vk1.y - dk1.y, vk1.z - dk1.z, 0.f);
        }
      }
      block_sync<SYNC_NT>();
    }
    if (group == 0) {
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int i = t * EPT + e;
        if (i < n_out) v[e] = f3(out_v[i]);
      }
    }
  }
};

template <int EPT, int NT>
constexpr int pair_smem_bytes() {
  // two rods' parameters and exchange slots, the outer rod's staged positions and
  // velocities, and one slot for the binding offset
  return (2 * (2 * EPT * NT + 2 * kHaloSlots * NT) + 2 * EPT * NT + 1) * (int)sizeof(float4);
}

// MB: launched with the mailbox (inputs, and so beta, may change between steps).
template <int EPT, int NT, bool MB>
__global__ void __launch_bounds__(2 * NT)
pair_kernel(const RodDev* __restrict__ rods, const int4* __restrict__ pairs, float4* __restrict__ x4,
            float4* __restrict__ v4, float4* __restrict__ q4, float4* __restrict__ o4,
            const float4* __restrict__ u4, const float4* __restrict__ k4, const float4* __restrict__ drive,
            int n_steps, float4* __restrict__ pos_out, MailboxDev mb) {
  extern __shared__ float4 smem[];
  pdl_begin();
  const int group = threadIdx.x / NT;
  const int t = threadIdx.x - group * NT;
  const int4 pr = pairs[blockIdx.x];  // (outer rod, inner rod, mode, 0)
  const int rid = group == 0 ? pr.x : pr.y;
  const RodDev R = rods[rid];
  float4* gs = smem + group * (2 * EPT * NT + 2 * kHaloSlots * NT);
  float4* par_u = gs;
  float4* par_k = gs + EPT * NT;
  float4* halo = gs + 2 * EPT * NT;
  float4* out_r = smem + 2 * (2 * EPT * NT + 2 * kHaloSlots * NT);
  float4* out_v = out_r + EPT * NT;
  float& beta_sh = reinterpret_cast<float*>(out_v + EPT * NT)[0];

  float3 r[EPT], v[EPT], om[EPT];
  float4 q[EPT];
  float w[EPT];
  load_rod<EPT, NT>(R, t, t, x4, v4, q4, o4, u4, k4, r, v, q, om, w, par_u, par_k);
  float3 v_drive = zero3(), w_drive = zero3();
  float beta = 0.f;
  if (drive != nullptr) {
    const float4 d0 = drive[2 * rid];
    v_drive = f3(d0);
    w_drive = f3(drive[2 * rid + 1]);
    beta = drive[2 * pr.y].w;
  }
  PairHook<2 * NT, EPT, MB> hook;
  hook.group = group;
  hook.t = t;
  hook.mode = pr.z;
  hook.beta_sh = &beta_sh;
  hook.k0 = (int)floorf(beta);
  hook.alpha = beta - floorf(beta);
  hook.n_out = rods[pr.x].n;
  hook.n_in = rods[pr.y].n;
  hook.dt = R.dt;
  hook.out_r = out_r;
  hook.out_v = out_v;

  const BlockHalo<NT, 2 * NT> H{t};
  int xc = 0;
  StepCache<EPT> sc;  // launch constants of the step (filled on the first step)
  if constexpr (MB) {
    // beta is written by the inner rod's first thread only (here, and by its mailbox polls)
    if (group == 1 && t == 0) beta_sh = beta;
    RodMailbox<EPT> box(mb, R, rid, t * EPT, NT, group);
    for (int step = 0; step < n_steps; ++step) {
      if (box.before_step(H, step, v_drive, w_drive, group == 1 ? &beta_sh : nullptr)) break;
      step_body<EPT, NT, false>(R, H, r, v, q, om, w, par_u, par_k, halo, xc, sc, v_drive, w_drive, nullptr, nullptr,
                                hook);
      box.after_step(H, step, r, v, w);
    }
  } else {
    for (int step = 0; step < n_steps; ++step)
      step_body<EPT, NT, false>(R, H, r, v, q, om, w, par_u, par_k, halo, xc, sc, v_drive, w_drive, nullptr, nullptr,
                                hook);
  }
  const int e0 = t * EPT;
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

template <int EPT, int NT, bool MB>
cudaError_t launch_pair_mb(const StepArgs& a, const int4* pairs, int n_pairs, cudaStream_t s) {
  constexpr int smem = pair_smem_bytes<EPT, NT>();
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(pair_kernel<EPT, NT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  return launch_kernel(pair_kernel<EPT, NT, MB>, dim3(n_pairs), dim3(2 * NT), smem, s, a.pdl, 0, a.rods, pairs, a.x4,
                       a.v4, a.q4, a.o4, a.u4, a.k4, a.drive, a.n_steps, a.pos_out, a.mb);
}

template <int EPT, int NT>
cudaError_t launch_pair_t(const StepArgs& a, const int4* pairs, int n_pairs, cudaStream_t s) {
  return a.mb.period > 0 ? launch_pair_mb<EPT, NT, true>(a, pairs, n_pairs, s)
                         : launch_pair_mb<EPT, NT, false>(a, pairs, n_pairs, s);
}

}  // namespace

cudaError_t launch_pair(int ept, int nt, const StepArgs& a, const int4* pairs, int n_pairs, cudaStream_t s) {
  if (ept == 2) {
    switch (nt) {
      case 32: return launch_pair_t<2, 32>(a, pairs, n_pairs, s);
      case 64: return launch_pair_t<2, 64>(a, pairs, n_pairs, s);
      case 128: return launch_pair_t<2, 128>(a, pairs, n_pairs, s);
      case 256: return launch_pair_t<2, 256>(a, pairs, n_pairs, s);
    }
  } else if (ept == 4) {
    switch (nt) {
      case 32: return launch_pair_t<4, 32>(a, pairs, n_pairs, s);
      case 64: return launch_pair_t<4, 64>(a, pairs, n_pairs, s);
      case 128: return launch_pair_t<4, 128>(a, pairs, n_pairs, s);
      case 256: return launch_pair_t<4, 256>(a, pairs, n_pairs, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace corde
