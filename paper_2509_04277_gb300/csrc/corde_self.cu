// Self-collision of a rod held by one thread block ("Collisions and self-collisions", and
// Section 2.1 "Constraints": contact constraints C_c handle self-collisions with Coulomb
// friction).
//
// Every mass point carries a sphere of the rod radius r.  Once per step, on the positions
// the constraint stage starts from, the block finds every pair (i, j) with
// |i - j| >= min_sep and |r_i - r_j| < 3 r (contact distance 2 r plus a skin of r):
//   broad phase  - bounding spheres wrap groups of 8 neighbouring mass points (centre: the
//                  group's middle point, radius: its farthest point); every sphere is
//                  checked against all others, with the 3 r reach added, into a bit
//                  matrix of overlapping group pairs;
//   narrow phase - each mass point checks the points of every group overlapping its own
//                  group (sphere-sphere distance test) and keeps its partners, ascending,
//                  in a list of at most 16 in shared memory;
//   compaction   - the pairs (i < j) get consecutive slots (a block prefix sum over the
//                  points' counts of larger partners), and every list entry is replaced by
//                  its pair's slot.
// In every constraint iteration, after the distance sweeps (and the vessel contact), the
// velocities are staged in shared memory, every pair is evaluated once, spread evenly
// over the threads (Jacobi: all from the staged velocities), and each mass point sums its
// pairs in ascending partner order.  For a pair with predicted offset
// delta = (r_j - r_i) + dt (v_j - v_i) shorter than 2 r, phi = 2 r - |delta|,
// n = delta / |delta|, du_n = phi / dt, relative tangential velocity u_t,
//   J = (du_n n - min(1, mu du_n / |u_t|) u_t) / (w_i + w_j)        (+J on j, -J on i),
// and a point takes the penetration-weighted mean of its pairs:
//   dv_i = -w_i sum_j phi_ij J_ij / sum_j phi_ij.
// No pair is lost to the broad phase: a pair within reach lies in groups whose spheres,
// grown by the reach, overlap.  Rods of at most 1024 nodes (everything lives in shared
// memory); a mass point with more than 16 partners keeps the first 16, and pairs beyond
// 3 per mass point are dropped; either raises the overflow flag of the rod's statistics.
#include "corde_step.cuh"
#include "corde_variants.cuh"

namespace corde {
namespace {

constexpr int kSelfGroup = 8;     // mass points per bounding sphere
constexpr int kSelfMaxCand = 16;  // partners kept per mass point
constexpr int kSelfPairsPerNode = 3;  // compacted pair capacity: 3 pairs per mass point
constexpr unsigned short kSelfNone = 0xffffu;  // list entry dropped (pair capacity exceeded)
constexpr unsigned short kSelfDown = 0x8000u;  // list entry flag: this point is the pair's larger index

// Shared-memory layout of the self-collision area (bytes from its start).
template <int EPT, int NT>
struct SelfLayout {
  static constexpr int NN = EPT * NT;                                // node capacity
  static constexpr int NG = (NN + kSelfGroup - 1) / kSelfGroup;      // bounding spheres
  static constexpr int NGW = (NG + 31) / 32;                         // words per bit row
  static constexpr int NP = kSelfPairsPerNode * NN;                  // pair capacity
  static_assert(NP < 0x8000, "pair slots must fit 15 bits");
  static constexpr int off_r = 0;                                    // float4 [NN]: r, w
  static constexpr int off_v = off_r + NN * 16;                      // float4 [NN]: v
  static constexpr int off_pj = off_v + NN * 16;                     // float4 [NP]: phi J, phi
  static constexpr int off_g = off_pj + NP * 16;                     // float4 [NG]: centre, radius
  static constexpr int off_bits = off_g + NG * 16;                   // unsigned [NG][NGW]
  static constexpr int off_cnt = off_bits + ((NG * NGW * 4 + 15) / 16) * 16;  // int [NN]: partners
  static constexpr int off_up = off_cnt + NN * 4;                    // int [NN]: first pair slot << 8 | up
  static constexpr int off_pa = off_up + NN * 4;                     // ushort2 [NP]: (i, j), i < j
  static constexpr int off_scan = off_pa + NP * 4;                   // int [NT / 32 + 1]: warp sums
  static constexpr int off_stat = off_scan + ((NT / 32 + 1) * 4 + 15) / 16 * 16;  // int [4]
  static constexpr int off_list = off_stat + 16;                     // uint16 [kSelfMaxCand][NN]
  static constexpr int bytes = off_list + kSelfMaxCand * NN * 2;
};

template <int NT>
__device__ __forceinline__ int block_or(int x) {
  if constexpr (NT == 32) {
    return __any_sync(0xffffffffu, x);
  } else {
    return __syncthreads_or(x);
  }
}

// Exclusive prefix sum of one int per thread over the block; *total receives the sum.
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int x, int* warp_sums, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if constexpr (NT == 32) {
    *total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - x;
  } else {
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int s = lane < NT / 32 ? warp_sums[lane] : 0;
      int si = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, si, o);
        if (lane >= o) si += y;
      }
      if (lane < NT / 32) warp_sums[lane] = si - s;
      if (lane == NT / 32 - 1) warp_sums[NT / 32] = si;
    }
    __syncthreads();
    *total = warp_sums[NT / 32];
    return warp_sums[wid] + incl - x;
  }
}

template <int EPT, int NT>
struct SelfHook {
  using L = SelfLayout<EPT, NT>;
  unsigned char* base;
  int t, n, min_sep;
  float dt, inv_dt, dist, reach, mu;
  mutable int active;   // block-uniform: some pair exists this step
  mutable int n_pairs;  // compacted pairs this step (block-uniform)

  __device__ __forceinline__ float4* sr() const { return reinterpret_cast<float4*>(base + L::off_r); }
  __device__ __forceinline__ float4* sv() const { return reinterpret_cast<float4*>(base + L::off_v); }
  __device__ __forceinline__ float4* pj() const { return reinterpret_cast<float4*>(base + L::off_pj); }
  __device__ __forceinline__ float4* gs() const { return reinterpret_cast<float4*>(base + L::off_g); }
  __device__ __forceinline__ unsigned* bits() const { return reinterpret_cast<unsigned*>(base + L::off_bits); }
  __device__ __forceinline__ int* cnt() const { return reinterpret_cast<int*>(base + L::off_cnt); }
  __device__ __forceinline__ int* up() const { return reinterpret_cast<int*>(base + L::off_up); }
  __device__ __forceinline__ ushort2* pa() const { return reinterpret_cast<ushort2*>(base + L::off_pa); }
  __device__ __forceinline__ int* scan() const { return reinterpret_cast<int*>(base + L::off_scan); }
  __device__ __forceinline__ int* stat() const { return reinterpret_cast<int*>(base + L::off_stat); }
  __device__ __forceinline__ unsigned short* list() const {
    return reinterpret_cast<unsigned short*>(base + L::off_list);
  }

  // Detection: broad phase over bounding spheres, narrow phase over mass points, then the
  // pairs (i < j) compacted into slots and every list entry turned into its pair's slot.
  template <int E>
  __device__ __forceinline__ void before_iterations(const float3 (&r)[E], const float (&w)[E]) const {
    float4* R4 = sr();
    const int e0 = t * EPT;
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      if (e0 + e < n) R4[e0 + e] = make_float4(r[e].x, r[e].y, r[e].z, w[e]);
    if (t < 3) stat()[t] = 0;
    block_sync<NT>();
    const int ng = (n + kSelfGroup - 1) / kSelfGroup;
    for (int g = t; g < ng; g += NT) {
      const int k0 = g * kSelfGroup;
      const float4 c = R4[min(k0 + kSelfGroup / 2, n - 1)];
      float rad2 = 0.f;
#pragma unroll
      for (int kk = 0; kk < kSelfGroup; ++kk) {
        const float4 p = R4[min(k0 + kk, n - 1)];
        const float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
        rad2 = fmaxf(rad2, dx * dx + dy * dy + dz * dz);
      }
      gs()[g] = make_float4(c.x, c.y, c.z, sqrtf(rad2));
    }
    block_sync<NT>();
    const int nw = (ng + 31) / 32;
    for (int task = t; task < ng * nw; task += NT) {
      const int a = task / nw, wd = task - a * nw;
      const float4 ca = gs()[a];
      unsigned word = 0u;
#pragma unroll 8
      for (int bb = 0; bb < 32; ++bb) {
        const int b = min(wd * 32 + bb, ng - 1);
        const float4 cb = gs()[b];
        const float dx = cb.x - ca.x, dy = cb.y - ca.y, dz = cb.z - ca.z;
        const float lim = (ca.w + cb.w + reach) * 1.001f + 1e-6f;  // conservative against rounding
        if (wd * 32 + bb < ng && dx * dx + dy * dy + dz * dz <= lim * lim) word |= 1u << bb;
      }
      bits()[a * L::NGW + wd] = word;
    }
    block_sync<NT>();
    const float reach2 = reach * reach, dist2 = dist * dist;
    int n_up[EPT];
    int my_up = 0;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int i = e0 + e;
      n_up[e] = 0;
      if (i >= n) continue;
      const float4 ri = R4[i];
      const int a = i / kSelfGroup;
      int c = 0, ups = 0, touching = 0;
      for (int wd = 0; wd < nw; ++wd) {
        unsigned word = bits()[a * L::NGW + wd];
        while (word) {
          const int jb = (wd * 32 + __ffs(word) - 1) * kSelfGroup;
          word &= word - 1u;
#pragma unroll
          for (int jj = 0; jj < kSelfGroup; ++jj) {
            const int j = jb + jj;
            const float4 rj = R4[min(j, n - 1)];
            const float dx = rj.x - ri.x, dy = rj.y - ri.y, dz = rj.z - ri.z;
            const float d2 = dx * dx + dy * dy + dz * dz;
            if (j < n && abs(i - j) >= min_sep && d2 < reach2) {
              if (c < kSelfMaxCand) {
                list()[c * L::NN + i] = (unsigned short)j;
                ups += j > i;
              }
              ++c;
              touching += d2 < dist2;
            }
          }
        }
      }
      if (c > kSelfMaxCand) atomicOr(&stat()[3], 1);
      const int kept = min(c, kSelfMaxCand);
      cnt()[i] = kept;
      n_up[e] = ups;
      my_up += ups;
      if (kept > 0) {
        atomicAdd(&stat()[0], kept);
        atomicMax(&stat()[1], c);
        atomicAdd(&stat()[2], touching);
      }
    }
    // compacted pair slots: node i owns slots [first_i, first_i + up_i) for its partners j > i
    int total = 0;
    int first = block_exclusive_scan<NT>(my_up, scan(), &total);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int i = e0 + e;
      if (i >= n) continue;
      up()[i] = (first << 8) | n_up[e];
      const int c = cnt()[i];
      int k2 = 0;
      for (int k = 0; k < c; ++k) {
        const int j = list()[k * L::NN + i];
        if (j > i) {
          const int slot = first + k2++;
          if (slot < L::NP) pa()[slot] = make_ushort2((unsigned short)i, (unsigned short)j);
        }
      }
      first += n_up[e];
    }
    if (total > L::NP) {
      if (t == 0) atomicOr(&stat()[3], 2);
      total = L::NP;
    }
    n_pairs = total;
    block_sync<NT>();
    // list entries -> pair slots (partners below: find this point in the partner's slots)
    int any = 0;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int i = e0 + e;
      if (i >= n) continue;
      const int c = cnt()[i];
      const int fi = up()[i] >> 8;
      int k2 = 0;
      for (int k = 0; k < c; ++k) {
        const int j = list()[k * L::NN + i];
        int slot;
        unsigned short flag = 0;
        if (j > i) {
          slot = fi + k2++;
        } else {
          const int uj = up()[j];
          const int fj = uj >> 8, nj = uj & 0xff;
          slot = L::NP;
          for (int q = 0; q < nj; ++q)
            if (fj + q < L::NP && pa()[fj + q].y == i) slot = fj + q;
          flag = kSelfDown;
        }
        list()[k * L::NN + i] = slot < L::NP ? (unsigned short)(slot | flag) : kSelfNone;
      }
      any |= c > 0;
    }
    active = block_or<NT>(any);
  }

  // Response: every pair evaluated once from the staged velocities (Jacobi), then each
  // mass point takes the penetration-weighted mean of its pairs, in ascending partner order.
  template <int E>
  __device__ __forceinline__ void after_odd(const float3 (&r)[E], float3 (&v)[E], const float (&w)[E]) const {
    if (!active) return;
    const int e0 = t * EPT;
    float4* V4 = sv();
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      if (e0 + e < n) V4[e0 + e] = make_float4(v[e].x, v[e].y, v[e].z, 0.f);
    block_sync<NT>();
    const float4* R4 = sr();
    float4* P4 = pj();
    const float dist2 = dist * dist;
    for (int p0 = 0; p0 < n_pairs; p0 += 2 * NT) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = p0 + h * NT + t;
        if (p >= n_pairs) continue;
        const ushort2 ij = pa()[p];
        const float4 ri = R4[ij.x], rj = R4[ij.y];
        const float3 u = f3(V4[ij.y]) - f3(V4[ij.x]);
        const float3 delta = (f3(rj) - f3(ri)) + dt * u;
        const float d2 = dot3(delta, delta);
        const float wsum = ri.w + rj.w;
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (d2 < dist2 && d2 > 0.f && wsum > 0.f) {
          const float il = rsqrtf(d2);
          const float phi = dist - d2 * il;
          const float3 nrm = il * delta;
          const float dun = phi * inv_dt;
          const float3 ut = u - dot3(u, nrm) * nrm;
          const float ut2 = dot3(ut, ut);
          const float cut = ut2 > 0.f ? fminf(1.f, mu * dun * rsqrtf(ut2)) : 0.f;
          const float3 J = (phi * __frcp_rn(wsum)) * (dun * nrm - cut * ut);
          out = make_float4(J.x, J.y, J.z, phi);
        }
        P4[p] = out;
      }
    }
    block_sync<NT>();
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int i = e0 + e;
      if (i >= n || !(w[e] > 0.f)) continue;
      const int c = cnt()[i];
      float3 acc = zero3();
      float wphi = 0.f;
      for (int k = 0; k < c; ++k) {
        const unsigned short ent = list()[k * L::NN + i];
        if (ent == kSelfNone) continue;
        const float4 s = P4[ent & 0x7fff];
        if (ent & kSelfDown) acc += f3(s);
        else acc -= f3(s);
        wphi += s.w;
      }
      if (wphi > 0.f) v[e] += (w[e] / wphi) * acc;
    }
  }
};

template <int EPT, int NT>
constexpr int self_smem_bytes() {
  return step_smem_bytes<EPT, NT>() + SelfLayout<EPT, NT>::bytes;
}

template <int EPT, int NT>
__global__ void __launch_bounds__(NT)
self_step_kernel(const RodDev* __restrict__ rods, const int* __restrict__ work, float4* __restrict__ x4,
                 float4* __restrict__ v4, float4* __restrict__ q4, float4* __restrict__ o4,
                 const float4* __restrict__ u4, const float4* __restrict__ k4, const float4* __restrict__ drive,
                 int n_steps, int4* __restrict__ stats) {
  extern __shared__ float4 smem[];
  const int rid = work[blockIdx.x];
  const RodDev R = rods[rid];
  const int t = threadIdx.x;
  float4* par_u = smem;
  float4* par_k = smem + EPT * NT;
  float4* halo = smem + 2 * EPT * NT;
  unsigned char* self_base = reinterpret_cast<unsigned char*>(smem + 2 * EPT * NT + 2 * kHaloSlots * NT);

  float3 r[EPT], v[EPT], om[EPT];
  float4 q[EPT];
  float w[EPT];
  load_rod<EPT, NT>(R, t, t, x4, v4, q4, o4, u4, k4, r, v, q, om, w, par_u, par_k);
  float3 v_drive = zero3(), w_drive = zero3();
  if (drive != nullptr) {
    v_drive = f3(drive[2 * rid]);
    w_drive = f3(drive[2 * rid + 1]);
  }
  SelfHook<EPT, NT> hook;
  hook.base = self_base;
  hook.t = t;
  hook.n = R.n;
  hook.min_sep = (int)R.self_sep;
  hook.dt = R.dt;
  hook.inv_dt = 1.f / R.dt;
  hook.dist = R.self_dist;
  hook.reach = R.self_reach;
  hook.mu = R.self_mu;
  hook.active = 0;
  hook.n_pairs = 0;
  if (t == 0) hook.stat()[3] = 0;  // overflow flag of this launch (read after the last barrier)

  const BlockHalo<NT, NT> H{t};
  int xc = 0;
  for (int step = 0; step < n_steps; ++step)
    step_body<EPT, NT, false>(R, H, r, v, q, om, w, par_u, par_k, halo, xc, v_drive, w_drive, nullptr, nullptr,
                              hook);
  const int e0 = t * EPT;
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
  block_sync<NT>();
  if (t == 0 && stats != nullptr) {
    const int* st = hook.stat();
    int4 out = stats[rid];
    out.x = st[0] / 2;  // candidate pairs at the last detection
    out.y = st[1];      // most partners of one mass point
    out.z = st[2] / 2;  // pairs whose spheres overlap at the last detection
    out.w |= st[3];     // 1: a partner list overflowed, 2: the pair slots overflowed (sticky)
    stats[rid] = out;
  }
}

template <int EPT, int NT>
cudaError_t launch_self_t(const StepArgs& a, int n_blocks, cudaStream_t s) {
  constexpr int smem = self_smem_bytes<EPT, NT>();
  static_assert(smem <= 227 * 1024, "self-collision shared memory");
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(self_step_kernel<EPT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  self_step_kernel<EPT, NT><<<n_blocks, NT, smem, s>>>(a.rods, a.work, a.x4, a.v4, a.q4, a.o4, a.u4, a.k4, a.drive,
                                                        a.n_steps, a.self_stats);
  return cudaGetLastError();
}

}  // namespace

const StepVariant kSelfVariants[] = {
    {2, 32, self_smem_bytes<2, 32>(), &launch_self_t<2, 32>},
    {2, 64, self_smem_bytes<2, 64>(), &launch_self_t<2, 64>},
    {2, 128, self_smem_bytes<2, 128>(), &launch_self_t<2, 128>},
    {2, 256, self_smem_bytes<2, 256>(), &launch_self_t<2, 256>},
    {2, 512, self_smem_bytes<2, 512>(), &launch_self_t<2, 512>},
    {4, 128, self_smem_bytes<4, 128>(), &launch_self_t<4, 128>},
    {4, 256, self_smem_bytes<4, 256>(), &launch_self_t<4, 256>},
};
const int kNumSelfVariants = 7;

}  // namespace corde
