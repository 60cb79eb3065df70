// Self-collision of a rod held by one thread block ("Collisions and self-collisions", and
// Section 2.1 "Constraints": contact constraints C_c handle self-collisions with Coulomb
// friction).
//
// Every mass point carries a sphere of the rod radius r.  Once per step, on the positions
// the constraint stage starts from, the block finds every pair (i < j) with
// j - i >= min_sep and |r_i - r_j| < 3 r (contact distance 2 r plus a skin of r):
//   broad phase  - bounding spheres wrap groups of 8 neighbouring mass points (centre: the
//                  group's middle point, radius: its farthest point); every sphere is
//                  checked against all others, with the 3 r reach added, into a bit
//                  matrix of overlapping group pairs;
//   narrow phase - each mass point i checks the points j > i of every group overlapping
//                  its own (sphere-sphere distance test) and keeps them, ascending, in a
//                  list of at most 16 in shared memory;
//   compaction   - the pairs get consecutive slots, ordered by (i, j) (a block prefix sum
//                  over the points' counts).
// Skin list (rods in blocks of up to 512 nodes): the broad and narrow phases run with the
// reach grown by two skin widths s = 1.5 r and keep every point's partners in a list, with
// the positions they were found at; the build's narrow phase lists its own step's
// partners at the plain reach too, and on later steps each point only tests its listed
// partners at the plain reach.  A pair within the reach now was within reach + 2 s at the
// build as long as no mass point has moved more than s since, so the block rebuilds the
// list as soon as one has moved more than 0.999 s (and when it has none: the list and the
// positions it was built at are kept in device memory from one launch to the next,
// discarded when the rod's self-collision settings change; a build that overflowed the
// list is repeated on the next step): the candidate pairs of every step are exactly those
// of the full detection.
// In every constraint iteration, after the distance sweeps (and the vessel contact), the
// velocities are staged in shared memory and (Jacobi: everything from the staged
// velocities)
//   1. every pair's predicted offset delta = (r_j - r_i) + dt (v_j - v_i) is tested and the
//      pairs with |delta| < 2 r are listed, each warp its own in a scratch of its own;
//   2. right away, spread over the warp's lanes, each listed pair gets phi = 2 r - |delta|,
//      n = delta / |delta|, du_n = phi / dt, the relative tangential velocity u_t and
//        J = (du_n n - min(1, mu du_n / |u_t|) u_t) / (w_i + w_j)   (+J on j, -J on i),
//      and its slot is appended to both mass points' short lists;
//   3. each mass point sums its pairs in ascending slot order (= ascending partner order,
//      so the result does not depend on the order of step 2) and takes the
//      penetration-weighted mean  dv_i = -w_i sum_j phi_ij J_ij / sum_j phi_ij.
// No pair is lost to the broad phase: a pair within reach lies in groups whose spheres,
// grown by the reach, overlap.  Rods of at most 1024 nodes (everything lives in shared
// memory).  Beyond 16 larger partners of a point, 3 pairs per point, or 16 touching pairs
// of a point, the excess is dropped and the overflow flag of the rod's statistics raised.
#include "corde_step.cuh"
#include "corde_variants.cuh"

namespace corde {
namespace {

constexpr int kSelfGroup = 8;         // mass points per bounding sphere
constexpr int kSelfMaxCand = 16;      // larger partners kept per mass point; touching pairs per point
constexpr int kSelfPairsPerNode = 3;  // compacted pair capacity: 3 pairs per mass point
constexpr int kSkinMax = 24;          // partners kept per mass point in the skin list
constexpr int kSkinNodes = 512;       // rods held by blocks of up to this many nodes keep a skin list

// A rod's skin list kept in device memory between launches (the record of rod r at
// r x kBytes): its valid flag, then every mass point's list count, listed partners
// ([kSkinMax][kSkinNodes] uint16) and position at the last build.
struct SelfSkinStore {
  static constexpr int off_cnt = 16;
  static constexpr int off_list = off_cnt + kSkinNodes;
  static constexpr int off_rb = off_list + kSkinMax * kSkinNodes * 2;
  static constexpr int kBytes = off_rb + kSkinNodes * 16;
};
static_assert(SelfSkinStore::off_rb % 16 == 0, "skin store layout");

// Shared-memory layout of the self-collision area (bytes from its start).
template <int EPT, int NT>
struct SelfLayout {
  static constexpr int NN = EPT * NT;                                // node capacity
  static constexpr int NG = (NN + kSelfGroup - 1) / kSelfGroup;      // bounding spheres
  static constexpr int NGH = (NG + 15) / 16;                         // 16-bit words per bit row
  static constexpr int NP = kSelfPairsPerNode * NN;                  // pair capacity
  static_assert(NP < 0x10000, "pair slots must fit 16 bits");
  static constexpr int off_r = 0;                                    // float4 [NN]: r, w
  static constexpr int off_v = off_r + NN * 16;                      // float4 [NN]: v
  static constexpr int off_pj = off_v + NN * 16;                     // float4 [NP]: phi J, phi
  static constexpr int off_q = off_pj + NP * 16;                     // float4 [NN]: r + dt v, w
  static constexpr int off_g = off_q + NN * 16;                      // float4 [NG]: centre, radius
  static constexpr int off_bits = off_g + NG * 16;                   // uint16 [NG][NGH]
  static constexpr int off_nact = off_bits + ((NG * NGH * 2 + 15) / 16) * 16;  // int [NN]
  static constexpr int off_pa = off_nact + NN * 4;                   // ushort2 [NP]: (i, j), i < j
  static constexpr int off_act = off_pa + NP * 4;                    // uint16 [NP]: touching pairs, 4 x 32 per warp
  static constexpr int off_scan = off_act + ((NP * 2 + 15) / 16) * 16;  // int [NT / 32 + 1]
  static constexpr int off_stat = off_scan + ((NT / 32 + 1) * 4 + 15) / 16 * 16;  // int [8]
  static constexpr int off_list = off_stat + 32;  // uint16 [kSelfMaxCand][NN]: partners, then slots
  // skin list (blocks of up to kSkinNodes nodes): partners j > i within the reach grown by
  // two skin widths at the last build, ascending, and their counts
  static constexpr bool kSkin = NN <= kSkinNodes;
  static constexpr int off_skin = off_list + kSelfMaxCand * NN * 2;  // uint16 [kSkinMax][NN]
  static constexpr int off_skincnt = off_skin + (kSkin ? kSkinMax * NN * 2 : 0);  // uint8 [NN]
  static constexpr int bytes = off_skincnt + (kSkin ? (NN + 15) / 16 * 16 : 0);
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
  mutable int n_pairs;  // compacted pairs this step (block-uniform)
  // skin list: positions of the thread's mass points at the last build, and whether the
  // block's list is complete (block-uniform)
  mutable float3 rb[EPT];
  mutable int skin_valid = 0;

  __device__ __forceinline__ float4* sr() const { return reinterpret_cast<float4*>(base + L::off_r); }
  __device__ __forceinline__ float4* sv() const { return reinterpret_cast<float4*>(base + L::off_v); }
  __device__ __forceinline__ float4* pj() const { return reinterpret_cast<float4*>(base + L::off_pj); }
  __device__ __forceinline__ float4* qp() const { return reinterpret_cast<float4*>(base + L::off_q); }
  __device__ __forceinline__ float4* gs() const { return reinterpret_cast<float4*>(base + L::off_g); }
  __device__ __forceinline__ unsigned short* bits() const {
    return reinterpret_cast<unsigned short*>(base + L::off_bits);
  }
  __device__ __forceinline__ int* nact() const { return reinterpret_cast<int*>(base + L::off_nact); }
  __device__ __forceinline__ ushort2* pa() const { return reinterpret_cast<ushort2*>(base + L::off_pa); }
  __device__ __forceinline__ unsigned short* act() const {
    return reinterpret_cast<unsigned short*>(base + L::off_act);
  }
  __device__ __forceinline__ int* scan() const { return reinterpret_cast<int*>(base + L::off_scan); }
  // stat: [0] pairs, [1] most larger partners, [2] overlapping pairs, [3] overflow, [5] builds
  __device__ __forceinline__ int* stat() const { return reinterpret_cast<int*>(base + L::off_stat); }
  __device__ __forceinline__ unsigned short* list() const {
    return reinterpret_cast<unsigned short*>(base + L::off_list);
  }
  __device__ __forceinline__ unsigned short* skin() const {
    return reinterpret_cast<unsigned short*>(base + L::off_skin);
  }
  __device__ __forceinline__ unsigned char* skin_cnt() const {
    return reinterpret_cast<unsigned char*>(base + L::off_skincnt);
  }

  // Bounding spheres of kSelfGroup mass points and the bit matrix of sphere pairs (a <= b)
  // closer than their radii plus `rch` (two barriers; R4 staged before).
  __device__ __forceinline__ void build_groups(float rch) const {
    const float4* R4 = sr();
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
    const int nh = (ng + 15) / 16;
    for (int task = t; task < ng * nh; task += NT) {
      const int a = task / nh, wd = task - a * nh;
      const float4 ca = gs()[a];
      unsigned word = 0u;
#pragma unroll
      for (int bb = 0; bb < 16; ++bb) {
        const int b = min(wd * 16 + bb, ng - 1);
        const float4 cb = gs()[b];
        const float dx = cb.x - ca.x, dy = cb.y - ca.y, dz = cb.z - ca.z;
        const float lim = (ca.w + cb.w + rch) * 1.001f + 1e-6f;  // conservative against rounding
        // pairs (i < j) only: groups b >= a
        if (wd * 16 + bb >= a && wd * 16 + bb < ng && dx * dx + dy * dy + dz * dz <= lim * lim) word |= 1u << bb;
      }
      bits()[a * L::NGH + wd] = (unsigned short)word;
    }
    block_sync<NT>();
  }

  // Detection: broad phase over bounding spheres, narrow phase over mass points, then the
  // pairs compacted into slots ordered by (i, j).
  template <int E>
  __device__ __forceinline__ void before_iterations(const float3 (&r)[E], const float (&w)[E]) const {
    float4* R4 = sr();
    const int e0 = t * EPT;
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      if (e0 + e < n) {
        R4[e0 + e] = make_float4(r[e].x, r[e].y, r[e].z, w[e]);
        nact()[e0 + e] = 0;
      }
    if (t < 3) stat()[t] = 0;
    const int ng = (n + kSelfGroup - 1) / kSelfGroup;
    const int nh = (ng + 15) / 16;
    const float reach2 = reach * reach, dist2 = dist * dist;
    // narrow phase of point i over the groups its bit row marks: the partners j > i
    // (j - i >= min_sep) with |r_i - r_j|^2 < rch2, ascending, into out[c NN + i] for c < cap;
    // returns their number; *touching counts those closer than the contact distance.  With
    // out_plain, those also within plain2 (<= rch2) go, ascending, into out_plain the same
    // way, *c_plain their number.
    auto narrow = [&](int i, float4 ri, float rch2, unsigned short* out, int cap, int* touching, float plain2,
                      unsigned short* out_plain, int* c_plain) {
      const int a = i / kSelfGroup;
      int c = 0, cp = 0;
      for (int wd = a / 16; wd < nh; ++wd) {
        unsigned word = bits()[a * L::NGH + wd];
        while (word) {
          const int jb = (wd * 16 + __ffs(word) - 1) * kSelfGroup;
          word &= word - 1u;
          unsigned hit = 0u, hitp = 0u;
#pragma unroll
          for (int jj = 0; jj < kSelfGroup; ++jj) {
            const int j = jb + jj;
            const float4 rj = R4[min(j, n - 1)];
            const float dx = rj.x - ri.x, dy = rj.y - ri.y, dz = rj.z - ri.z;
            const float d2 = dx * dx + dy * dy + dz * dz;
            const bool ok = j < n && j - i >= min_sep;
            if (ok && d2 < rch2) hit |= 1u << jj;
            if (ok && d2 < plain2) hitp |= 1u << jj;
            if (ok && d2 < dist2) ++*touching;
          }
          while (hit) {
            const int j = jb + __ffs(hit) - 1;
            hit &= hit - 1u;
            if (c < cap) out[c * L::NN + i] = (unsigned short)j;
            ++c;
          }
          if (out_plain != nullptr) {
            while (hitp) {
              const int j = jb + __ffs(hitp) - 1;
              hitp &= hitp - 1u;
              if (cp < kSelfMaxCand) out_plain[cp * L::NN + i] = (unsigned short)j;
              ++cp;
            }
          }
        }
      }
      if (c_plain != nullptr) *c_plain = cp;
      return c;
    };
    int n_up[EPT];
    int my_up = 0, st_max = 0, st_touch = 0, st_over = 0;
    // the candidate counts of this step come from a narrow phase (parked in nact), or
    // from the skin list's filter
    bool from_narrow = false;
    if constexpr (L::kSkin) {
      // rebuild the skin list when a mass point has moved more than 0.999 s since the last
      // build (s = reach / 2 = 1.5 r), or when there is none
      const float s = reach * 0.5f;
      const float move2 = (0.999f * s) * (0.999f * s);
      int moved = !skin_valid;
#pragma unroll
      for (int e = 0; e < EPT; ++e)
        if (e0 + e < n) {
          const float3 d = r[e] - rb[e];
          moved |= dot3(d, d) > move2;
        }
      if (block_or<NT>(moved)) {  // (a barrier: the staged positions are visible)
        // the build also lists this step's candidates at the plain reach (its groups cover
        // them), so the step needs no filter, and a list that overflowed needs no second pass
        const float rch = reach + 2.f * s;
        build_groups(rch);
        int over = 0;
#pragma unroll 1
        for (int e = 0; e < EPT; ++e) {
          const int i = e0 + e;
          if (i >= n) continue;
          int cp = 0;
          const int c = narrow(i, R4[i], rch * rch, skin(), kSkinMax, &st_touch, reach2, list(), &cp);
          skin_cnt()[i] = (unsigned char)min(c, kSkinMax);
          nact()[i] = cp;
          over |= c > kSkinMax;
        }
#pragma unroll
        for (int e = 0; e < EPT; ++e) rb[e] = r[e];
        skin_valid = !block_or<NT>(over);  // (a barrier: the lists are visible)
        if (t == 0) ++stat()[5];           // builds in this launch
        if (!skin_valid && t == 0) atomicOr(&stat()[3], 8);  // the next step builds again
        from_narrow = true;
      }
    } else {
      block_sync<NT>();
      build_groups(reach);
      // the full narrow phase (one copy of its code: its counts parked in nact)
#pragma unroll 1
      for (int e = 0; e < EPT; ++e) {
        const int i = e0 + e;
        if (i < n) nact()[i] = narrow(i, R4[i], reach2, list(), kSelfMaxCand, &st_touch, -1.f, nullptr, nullptr);
      }
      from_narrow = true;
    }
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int i = e0 + e;
      n_up[e] = 0;
      if (i >= n) continue;
      const float4 ri = R4[i];
      int c = 0, touching = 0;
      if (!from_narrow) {
        // the listed partners at the plain reach (ascending, as the full detection finds them)
        const int k = skin_cnt()[i];
        // four partners at a time: their loads issued together
        for (int m0 = 0; m0 < k; m0 += 4) {
          int jj[4];
          float4 rj[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) jj[u] = skin()[min(m0 + u, k - 1) * L::NN + i];
#pragma unroll
          for (int u = 0; u < 4; ++u) rj[u] = R4[jj[u]];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (m0 + u >= k) break;
            const float dx = rj[u].x - ri.x, dy = rj[u].y - ri.y, dz = rj[u].z - ri.z;
            const float d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < dist2) ++touching;
            if (d2 < reach2) {
              if (c < kSelfMaxCand) list()[c * L::NN + i] = (unsigned short)jj[u];
              ++c;
            }
          }
        }
      } else {
        c = nact()[i];
        nact()[i] = 0;
      }
      st_over |= c > kSelfMaxCand;
      n_up[e] = min(c, kSelfMaxCand);
      my_up += n_up[e];
      st_max = max(st_max, c);
      st_touch += touching;
    }
    // statistics: one shared atomic per warp
    const int w_up = __reduce_add_sync(0xffffffffu, my_up);
    st_touch = __reduce_add_sync(0xffffffffu, st_touch);
    st_max = __reduce_max_sync(0xffffffffu, st_max);
    st_over = __reduce_or_sync(0xffffffffu, st_over);
    if ((t & 31) == 0) {
      if (w_up > 0) {
        atomicAdd(&stat()[0], w_up);
        atomicMax(&stat()[1], st_max);
        atomicAdd(&stat()[2], st_touch);
      }
      if (st_over) atomicOr(&stat()[3], 1);
    }
    // compacted pair slots: point i owns [first_i, first_i + up_i), partners ascending
    int total = 0;
    int first = block_exclusive_scan<NT>(my_up, scan(), &total);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int i = e0 + e;
      if (i >= n) continue;
      for (int k = 0; k < n_up[e]; ++k) {
        const int slot = first + k;
        if (slot < L::NP) pa()[slot] = make_ushort2((unsigned short)i, list()[k * L::NN + i]);
      }
      first += n_up[e];
    }
    if (total > L::NP) {
      if (t == 0) atomicOr(&stat()[3], 2);
      total = L::NP;
    }
    n_pairs = total;
  }

  // Response (see the file header): touching pairs found, their impulses computed, and
  // every mass point's pairs summed in ascending slot order.
  template <int E>
  __device__ __forceinline__ void after_odd(const float3 (&r)[E], float3 (&v)[E], const float (&w)[E]) const {
    if (n_pairs == 0) return;  // block-uniform
    const int e0 = t * EPT;
    float4* V4 = sv();
    float4* Q4 = qp();  // predicted positions, read by the touch test only
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      if (e0 + e < n) {
        V4[e0 + e] = make_float4(v[e].x, v[e].y, v[e].z, 0.f);
        Q4[e0 + e] = make_float4(fmaf(dt, v[e].x, r[e].x), fmaf(dt, v[e].y, r[e].y), fmaf(dt, v[e].z, r[e].z), w[e]);
      }
    block_sync<NT>();
    const float4* R4 = sr();
    float4* P4 = pj();
    const float dist2 = dist * dist;
    const int lane = t & 31;
    // 1. which pairs touch: predicted positions closer than 2 r (the exact offset of step 2
    //    decides the impulse; a pair misjudged here within rounding of 2 r has phi = 0)
    constexpr int PH = 4;
    static_assert(L::NP >= PH * NT, "each warp lists its touching pairs of one pass in the pair area");
    unsigned short* wl = act() + (t >> 5) * (PH * 32);  // this warp's touching pairs
    for (int p0 = 0; p0 < n_pairs; p0 += PH * NT) {
      bool hit[PH];
      float4 qi[PH], qj[PH];
#pragma unroll
      for (int h = 0; h < PH; ++h) {
        const ushort2 ij = pa()[min(p0 + h * NT + t, n_pairs - 1)];
        qi[h] = Q4[ij.x];
        qj[h] = Q4[ij.y];
      }
#pragma unroll
      for (int h = 0; h < PH; ++h) {
        const float3 delta = f3(qj[h]) - f3(qi[h]);
        hit[h] = p0 + h * NT + t < n_pairs && dot3(delta, delta) < dist2 * 1.0001f && qi[h].w + qj[h].w > 0.f;
      }
      // the warp's hits listed in its own scratch and spread over its lanes
      unsigned m[PH];
      int tot = 0;
#pragma unroll
      for (int h = 0; h < PH; ++h) {
        m[h] = __ballot_sync(0xffffffffu, hit[h]);
        tot += __popc(m[h]);
      }
      if (tot > 0) {  // warp-uniform
        int at = 0;
        const unsigned below = (1u << lane) - 1u;
#pragma unroll
        for (int h = 0; h < PH; ++h) {
          if (hit[h]) wl[at + __popc(m[h] & below)] = (unsigned short)(p0 + h * NT + t);
          at += __popc(m[h]);
        }
        __syncwarp();
        // 2. impulses of the touching pairs
        for (int q = lane; q < tot; q += 32) {
          const int p = wl[q];
          const ushort2 ij = pa()[p];
          const float4 ri = R4[ij.x], rj = R4[ij.y];
          const float3 u = f3(V4[ij.y]) - f3(V4[ij.x]);
          const float3 delta = (f3(rj) - f3(ri)) + dt * u;
          const float d2 = dot3(delta, delta);
          const float il = rsqrtf(d2);
          const float phi = fmaxf(dist - d2 * il, 0.f);  // rounding at the contact distance
          const float3 nrm = il * delta;
          const float dun = phi * inv_dt;
          const float3 ut = u - dot3(u, nrm) * nrm;
          const float ut2 = dot3(ut, ut);
          const float cut = ut2 > 0.f ? fminf(1.f, mu * dun * rsqrtf(ut2)) : 0.f;
          const float3 J = (phi * __fdividef(1.f, ri.w + rj.w)) * (dun * nrm - cut * ut);  // approximate reciprocal: ~2 ulp
          P4[p] = make_float4(J.x, J.y, J.z, phi);
          const int ka = atomicAdd(&nact()[ij.x], 1);
          const int kb = atomicAdd(&nact()[ij.y], 1);
          if (ka < kSelfMaxCand) list()[ka * L::NN + ij.x] = (unsigned short)p;
          if (kb < kSelfMaxCand) list()[kb * L::NN + ij.y] = (unsigned short)p;
          if (ka >= kSelfMaxCand || kb >= kSelfMaxCand) atomicOr(&stat()[3], 4);
        }
        __syncwarp();  // (the scratch is reused by the next pass)
      }
    }
    block_sync<NT>();
    // 3. each mass point: its pairs in ascending slot order
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int i = e0 + e;
      if (i >= n) continue;
      const int k = min(nact()[i], kSelfMaxCand);
      if (k == 0) continue;
      nact()[i] = 0;
      if (!(w[e] > 0.f)) continue;
      float3 acc = zero3();
      float wphi = 0.f;
      if (k <= 2) {
        // one or two pairs: their slots in ascending order without a search
        const int s0 = list()[i];
        const int s1 = k == 2 ? list()[L::NN + i] : s0;
        const int lo = min(s0, s1), hi = max(s0, s1);
        const float4 a4 = P4[lo];
        const bool a_first = pa()[lo].x == i;
        float4 b4 = make_float4(0.f, 0.f, 0.f, 0.f);
        bool b_first = false;
        if (k == 2) {
          b4 = P4[hi];
          b_first = pa()[hi].x == i;
        }
        if (a_first) acc -= f3(a4);
        else acc += f3(a4);
        wphi += a4.w;
        if (k == 2) {
          if (b_first) acc -= f3(b4);
          else acc += f3(b4);
          wphi += b4.w;
        }
      } else {
        int prev = -1;
        for (int q = 0; q < k; ++q) {
          int next = 0x7fffffff;
          for (int m = 0; m < k; ++m) {
            const int sl = list()[m * L::NN + i];
            if (sl > prev && sl < next) next = sl;
          }
          prev = next;
          const float4 s4 = P4[next];
          if (pa()[next].x == i) acc -= f3(s4);
          else acc += f3(s4);
          wphi += s4.w;
        }
      }
      if (wphi > 0.f) v[e] += __fdividef(w[e], wphi) * acc;
    }
  }
};

template <int EPT, int NT>
constexpr int self_smem_bytes() {
  return step_smem_bytes<EPT, NT>() + SelfLayout<EPT, NT>::bytes;
}

template <int EPT, int NT>
__global__ void __launch_bounds__(NT, 1)
self_step_kernel(const RodDev* __restrict__ rods, const int* __restrict__ work, float4* __restrict__ x4,
                 float4* __restrict__ v4, float4* __restrict__ q4, float4* __restrict__ o4,
                 const float4* __restrict__ u4, const float4* __restrict__ k4, const float4* __restrict__ drive,
                 int n_steps, int4* __restrict__ stats, float4* __restrict__ pos_out, unsigned char* __restrict__ skin_g) {
  extern __shared__ float4 smem[];
  pdl_begin();
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
  hook.n_pairs = 0;
  if (t == 0) {
    hook.stat()[3] = 0;  // overflow flags of this launch (read after the last barrier)
    hook.stat()[5] = 0;  // skin-list builds of this launch
  }
  using L = SelfLayout<EPT, NT>;
  unsigned char* store = nullptr;  // this rod's skin list of the previous launch
  if constexpr (L::kSkin) {
    if (skin_g != nullptr) store = skin_g + (int64_t)rid * SelfSkinStore::kBytes;
  }
  if (store != nullptr) {
    // a list from an earlier launch stays valid as long as no mass point has moved more
    // than the skin width from the position it was built at, which the first step checks
    // (a change of the rod's self-collision settings clears the flag)
    hook.skin_valid = *reinterpret_cast<const int*>(store);
    if (hook.skin_valid) {
      const float4* rbg = reinterpret_cast<const float4*>(store + SelfSkinStore::off_rb);
      const unsigned short* lg = reinterpret_cast<const unsigned short*>(store + SelfSkinStore::off_list);
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int i = t * EPT + e;
        if (i >= R.n) continue;
        const int c = store[SelfSkinStore::off_cnt + i];
        hook.skin_cnt()[i] = (unsigned char)c;
        for (int m = 0; m < c; ++m) hook.skin()[m * L::NN + i] = lg[m * kSkinNodes + i];
        hook.rb[e] = f3(rbg[i]);
      }
    }
  }

  const BlockHalo<NT, NT> H{t};
  int xc = 0;
  StepCache<EPT> sc;  // launch constants of the step (filled on the first step)
  for (int step = 0; step < n_steps; ++step)
    step_body<EPT, NT, false>(R, H, r, v, q, om, w, par_u, par_k, halo, xc, sc, v_drive, w_drive, nullptr, nullptr,
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
      if (pos_out != nullptr) pos_out[R.off + i] = make_float4(r[e].x, r[e].y, r[e].z, w[e]);
    }
  }
  if (store != nullptr) {
    // the list and the positions it was built at, for the next launch (each thread its
    // own mass points, as it reads them back)
    if (hook.skin_valid) {
      float4* rbg = reinterpret_cast<float4*>(store + SelfSkinStore::off_rb);
      unsigned short* lg = reinterpret_cast<unsigned short*>(store + SelfSkinStore::off_list);
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int i = t * EPT + e;
        if (i >= R.n) continue;
        const int c = hook.skin_cnt()[i];
        store[SelfSkinStore::off_cnt + i] = (unsigned char)c;
        for (int m = 0; m < c; ++m) lg[m * kSkinNodes + i] = hook.skin()[m * L::NN + i];
        rbg[i] = make_float4(hook.rb[e].x, hook.rb[e].y, hook.rb[e].z, 0.f);
      }
    }
    if (t == 0) *reinterpret_cast<int*>(store) = hook.skin_valid;
  }
  block_sync<NT>();
  if (t == 0 && stats != nullptr) {
    const int* st = hook.stat();
    int4 out = stats[2 * rid];
    out.x = st[0];   // candidate pairs at the last detection
    out.y = st[1];   // most larger partners of one mass point
    out.z = st[2];   // pairs whose spheres overlap at the last detection
    out.w |= st[3];  // 1: partner list, 2: pair slots, 4: touching pairs of a point, 8: skin list overflowed
    stats[2 * rid] = out;
    stats[2 * rid + 1] = make_int4(st[5], 0, 0, 0);  // skin-list builds in the launch
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
  return launch_kernel(self_step_kernel<EPT, NT>, dim3(n_blocks), dim3(NT), smem, s, a.pdl, 0, a.rods, a.work, a.x4,
                       a.v4, a.q4, a.o4, a.u4, a.k4, a.drive, a.n_steps, a.self_stats, a.pos_out, a.self_skin);
}

}  // namespace

const StepVariant kSelfVariants[] = {
    {2, 32, self_smem_bytes<2, 32>(), &launch_self_t<2, 32>},
    {2, 64, self_smem_bytes<2, 64>(), &launch_self_t<2, 64>},
    {2, 128, self_smem_bytes<2, 128>(), &launch_self_t<2, 128>},
    {2, 256, self_smem_bytes<2, 256>(), &launch_self_t<2, 256>},
    {4, 128, self_smem_bytes<4, 128>(), &launch_self_t<4, 128>},
    {4, 256, self_smem_bytes<4, 256>(), &launch_self_t<4, 256>},
};
const int kNumSelfVariants = 6;
const int kSelfSkinBytes = SelfSkinStore::kBytes;

}  // namespace corde
