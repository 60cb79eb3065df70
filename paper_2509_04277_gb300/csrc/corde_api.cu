// C ABI of the CoRdE stepper: creation (derived constants and packing on the device),
// kernel-variant plans, the persistent step launches, state I/O and diagnostics.
#include <algorithm>
#include <atomic>
#include <climits>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/corde.h"
#include "corde_common.cuh"
#include "corde_variants.cuh"

using namespace corde;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

}  // namespace

namespace corde {
int set_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace corde

namespace {

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? CORDE_ERR_OOM : CORDE_ERR_CUDA,       \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
    }                                                                                     \
  } while (0)

// All compiled variants, in preference order of the default plan.
std::vector<StepVariant> all_variants() {
  std::vector<StepVariant> v;
  for (int i = 0; i < kNumStepVariantsE2; ++i) v.push_back(kStepVariantsE2[i]);
  for (int i = 0; i < kNumStepVariantsE4; ++i) v.push_back(kStepVariantsE4[i]);
  return v;
}

const std::vector<StepVariant>& variants() {
  static const std::vector<StepVariant> v = all_variants();
  return v;
}

int max_block_capacity() {
  int c = 0;
  for (const auto& v : variants()) c = std::max(c, v.capacity());
  return c;
}

int max_capacity() {
  int c = max_block_capacity();
  for (int i = 0; i < kNumClusterVariants; ++i) c = std::max(c, kClusterVariants[i].capacity(kMaxCluster));
  return c;
}

// Largest rod a cooperative grid of the current device holds (all its blocks resident).
int max_grid_capacity() {
  int c = 0;
  for (int i = 0; i < kNumClusterVariants; ++i)
    c = std::max(c, kClusterVariants[i].capacity(kClusterVariants[i].grid_blocks()));
  return c;
}

int find_cluster_variant(int ept, int nt) {
  for (int i = 0; i < kNumClusterVariants; ++i)
    if (kClusterVariants[i].ept == ept && kClusterVariants[i].nt == nt) return i;
  return -1;
}

// Default plan of a rod longer than one block holds: 1024 nodes per block (4 elements x
// 256 threads) over the fewest blocks, 2048 per block beyond 16 blocks.
void default_cluster_plan(int n, int* variant, int* C) {
  int v = find_cluster_variant(4, 256);
  int c = (n + 1023) / 1024;
  if (c > kMaxCluster) {
    v = find_cluster_variant(4, 512);
    c = (n + 2047) / 2048;
  }
  *variant = v;
  *C = std::max(2, c);
}

// Default plan of a rod longer than a cluster holds: 2048 nodes per block (4 elements x 512
// threads) over a cooperative grid.
void default_grid_plan(int n, int* variant, int* C) {
  *variant = find_cluster_variant(4, 512);
  *C = std::max(2, (n + 2047) / 2048);
}

int find_variant(int ept, int nt) {
  const auto& vs = variants();
  for (size_t i = 0; i < vs.size(); ++i)
    if (vs[i].ept == ept && vs[i].nt == nt) return (int)i;
  return -1;
}

// Default plan: two elements per thread up to one warp, four elements per thread above,
// with the smallest power-of-two block that holds the rod.
int default_variant(int n) {
  const int ept = n <= 64 ? 2 : 4;
  int nt = 32;
  while (nt * ept < n && nt < 512) nt *= 2;
  int v = find_variant(ept, nt);
  if (v >= 0 && variants()[v].capacity() >= n) return v;
  int best = -1;
  for (size_t i = 0; i < variants().size(); ++i)
    if (variants()[i].capacity() >= n && (best < 0 || variants()[i].capacity() < variants()[best].capacity()))
      best = (int)i;
  return best;
}

struct Bin {
  int variant;  // block variant index, or cluster variant index when cluster > 0
  int count;
  int* d_work;
  int cluster = 0;  // blocks per rod (0: one block per rod; -1: self-collision kernel, variant
                    // indexes kSelfVariants)
  int grid = 0;     // 1: the cluster variant's blocks form a cooperative grid
  float4* d_gh = nullptr;  // grid bins: the rods' global exchange slots
};

}  // namespace

struct corde_rods {
  int device = 0;
  int n_rods = 0;
  int64_t n_elem = 0;
  std::vector<int> n_nodes, off;
  std::vector<int> flags;
  std::vector<int> n_iters;
  std::vector<double> dt;
  std::vector<double> derived;  // [n_rods][16]
  RodDev* d_rods = nullptr;
  double* d_derived = nullptr;
  float4 *d_x = nullptr, *d_v = nullptr, *d_q = nullptr, *d_o = nullptr, *d_u = nullptr, *d_k = nullptr;
  float4* d_drive = nullptr;
  float4* d_drive_graph = nullptr;  // the drive the graph reads (copied in before each replay)
  int* d_elem_rod = nullptr;
  std::vector<int> plan;          // variant index per rod (block or cluster table)
  std::vector<int> plan_cluster;  // blocks per rod; 0: one block
  std::vector<char> plan_grid;    // 1: the rod's plan_cluster blocks form a cooperative grid
  std::vector<Bin> bins;
  int last_launches = 0;
  int pdl = 1;  // stepping kernels launched with programmatic stream serialisation
  // rollout / adjoint
  float4* d_ckpt = nullptr;  // [n_ckpt][4][E]
  size_t ckpt_cap = 0;       // float4 entries
  float4* d_seg = nullptr;   // [K (+1)][4][E] scratch of the reverse pass
  size_t seg_cap = 0;
  float4* d_sweep_rec = nullptr;  // record mode of the reverse pass: sweeps and neighbour data
  size_t sweep_rec_cap = 0;
  long long adj_record_budget = 1ll << 30;
  int ro_steps = 0, ro_every = 0;
  // last rod_adjoint's largest launch: mode, nt, blocks/SM, blocks, SMs, compact records,
  // pipelined
  int adj_info[7] = {0, 0, 0, 0, 0, 0, 0};
  int adj_pipe = 1;  // pipelined reverse where it applies (rod_set_adjoint_pipeline)
  std::vector<Bin> adj_bins;  // variant = threads per block
  // catheter/guidewire pairs
  std::vector<int4> pairs;     // (outer, inner, mode, 0)
  std::vector<char> paired;    // per rod
  std::vector<char> tube;      // per rod: vessel contact enabled
  std::vector<char> self;      // per rod: self-collision enabled
  int4* d_self_stats = nullptr;  // [n_rods][2] self-collision statistics
  unsigned char* d_self_skin = nullptr;  // [n_rods][kSelfSkinBytes] skin lists kept between launches
  struct PairBin {
    int ept, nt, count;
    int4* d_pairs;
  };
  std::vector<PairBin> pair_bins;
  // mailbox of running launches
  int mb_period = 0;
  void* mb_in_host = nullptr;   // 16-byte seqlock header + [n_rods][8] floats, mapped pinned
  void* mb_out_host = nullptr;  // [n_rods][2][8] words, mapped pinned
  void* mb_pos_host = nullptr;  // [n_rods][4] seqlock words, then [n_elem] float4 positions, mapped pinned
  MailboxDev mb_dev = {};
  unsigned mb_host_seq = 0;
  long long steps_done = 0;
  // CUDA graph of one rod_step (all bins forked onto parallel branches)
  int graph_mode = 1;  // 0 never, 1 when a step needs more than one launch, 2 always
  cudaGraphExec_t graph_exec = nullptr;
  int graph_steps = -1;
  const float4* graph_drive = nullptr;
  float4* graph_pos_out = nullptr;
  float4* io_pos = nullptr;  // positions output of the launch being issued (rod_step_io)
  int graph_launches = 0;
  cudaStream_t cap_stream = nullptr;
  std::vector<cudaStream_t> side;
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> join_ev;
};

namespace {

const double kPi = 3.14159265358979323846;

// Section 2.1 constants (Eq. 2-3 with the second-moment reading), lumped masses, frame
// inertias and the default rules for Kp and the inertial scaling; FP64, one thread per rod.
__global__ void derive_kernel(int n_rods, const RodParams* __restrict__ P, const int* __restrict__ off,
                              RodDev* __restrict__ rods, double* __restrict__ derived) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rods) return;
  const RodParams p = P[r];
  const int N = p.n_nodes;
  const double l0 = p.length / (N - 1);
  const double r2 = p.radius * p.radius;
  const double A = kPi * r2;
  const double I = kPi * r2 * r2 / 4.0;
  const double K1 = p.E_bend * I, K3 = p.G * 2.0 * I, Ks = p.E_stretch * A;
  const double Kp = p.Kp > 0 ? p.Kp : 100.0 * 4.0 * K1 / (p.length * p.length);
  const double m_el = p.density * A * l0;
  const double J_el = p.density * l0 * I;
  double ms = p.mass_scale;
  if (!(ms > 0)) {
    double k_node = Kp / l0;
    if (!p.inextensible && Ks / l0 > k_node) k_node = Ks / l0;
    const double w2 = p.dt * p.dt * 4.0 * k_node / m_el;
    ms = w2 / 0.25 > 1.0 ? w2 / 0.25 : 1.0;
  }
  double is = p.inertia_scale;
  if (!(is > 0)) {
    const double kb = K1 > K3 ? K1 : K3;
    const double w2 = p.dt * p.dt * (4.0 * kb / l0 + Kp * l0) / J_el;
    is = w2 / 0.25 > 1.0 ? w2 / 0.25 : 1.0;
  }
  const double J1 = is * J_el, J3 = is * 2.0 * J_el;
  RodDev R;
  R.off = off[r];
  R.n = N;
  R.flags = (p.inextensible ? F_INEXT : 0) | (p.clamp ? F_CLAMP : 0);
  R.n_iters = p.n_iters;
  R.dt = (float)p.dt;
  R.l0 = (float)l0;
  R.two_over_l = (float)(2.0 / l0);
  R.lKp = (float)(l0 * Kp);
  R.Ks = (float)Ks;
  R.inv_l0 = (float)(1.0 / l0);
  R.damp = (float)(1.0 / (1.0 + p.damping_alpha * p.dt));
  R.self_dist = 0.f;
  R.gx = (float)(p.gravity[0] / ms);
  R.gy = (float)(p.gravity[1] / ms);
  R.gz = (float)(p.gravity[2] / ms);
  R.self_reach = 0.f;
  R.J1 = (float)J1;
  R.J3 = (float)J3;
  R.Jinv1 = (float)(1.0 / J1);
  R.Jinv3 = (float)(1.0 / J3);
  R.tube_cx = R.tube_cy = R.tube_cz = R.tube_rc = 0.f;
  R.tube_allow = R.tube_mu = R.self_mu = R.self_sep = 0.f;
  rods[r] = R;
  double* d = derived + 16 * (size_t)r;
  d[0] = l0; d[1] = A; d[2] = I; d[3] = K1; d[4] = K1; d[5] = K3; d[6] = Ks; d[7] = Kp;
  d[8] = ms; d[9] = is; d[10] = m_el; d[11] = J1; d[12] = J1; d[13] = J3; d[14] = 1.0 / (ms * m_el); d[15] = 0.0;
}

// Packs caller arrays into the element-indexed float4 layout; per-joint stiffness and
// intrinsic Darboux vectors (computed from the rest frames with the step's formula, so
// that the rest state carries no bending torque).
__global__ void pack_kernel(int64_t E, const int* __restrict__ elem_rod, const RodDev* __restrict__ rods,
                            const RodParams* __restrict__ P, const double* __restrict__ derived,
                            const float* __restrict__ pos, const float* __restrict__ quat,
                            const float* __restrict__ rest, const float* __restrict__ vel,
                            const float* __restrict__ omega, const float* __restrict__ mul, float4* x4, float4* v4,
                            float4* q4, float4* o4, float4* u4, float4* k4) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  const int r = elem_rod[i];
  const RodDev R = rods[r];
  const RodParams p = P[r];
  const double* d = derived + 16 * (size_t)r;
  const int li = (int)(i - R.off);
  const int n = R.n;
  const int64_t fi = i - r;      // global frame index
  const int64_t ji = i - 2 * r;  // global joint index
  const double l0 = d[0];
  const double left = li > 0 ? l0 : 0.0, right = li < n - 1 ? l0 : 0.0;
  const double m = p.density * d[1] * (left + right) / 2.0;
  float w = (float)(1.0 / (d[8] * m));
  if ((R.flags & F_CLAMP) && li == 0) w = 0.f;
  x4[i] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], w);
  v4[i] = vel ? make_float4(vel[3 * i], vel[3 * i + 1], vel[3 * i + 2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
  if (li <= n - 2) {
    q4[i] = make_float4(quat[4 * fi], quat[4 * fi + 1], quat[4 * fi + 2], quat[4 * fi + 3]);
    o4[i] = omega ? make_float4(omega[3 * fi], omega[3 * fi + 1], omega[3 * fi + 2], 0.f)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    q4[i] = make_float4(0.f, 0.f, 0.f, 1.f);
    o4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (li <= n - 3) {
    const double m1 = mul ? mul[3 * ji] : 1.0, m2 = mul ? mul[3 * ji + 1] : 1.0, m3 = mul ? mul[3 * ji + 2] : 1.0;
    k4[i] = make_float4((float)(d[3] * m1), (float)(d[4] * m2), (float)(d[5] * m3), 0.f);
    float3 uh = zero3();
    if (rest) {
      const float4 a = make_float4(rest[4 * fi], rest[4 * fi + 1], rest[4 * fi + 2], rest[4 * fi + 3]);
      const float4 b = make_float4(rest[4 * fi + 4], rest[4 * fi + 5], rest[4 * fi + 6], rest[4 * fi + 7]);
      uh = darboux(a, b, R.two_over_l);
    }
    u4[i] = make_float4(uh.x, uh.y, uh.z, 0.f);
  } else {
    k4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    u4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Per-rod diagnostics: max segment-length error, max quaternion-norm error, count of
// non-finite values, elastic energy (FP64 accumulation).
__global__ void diag_kernel(const RodDev* __restrict__ rods, const double* __restrict__ derived,
                            const float4* __restrict__ x4, const float4* __restrict__ q4,
                            const float4* __restrict__ v4, const float4* __restrict__ o4,
                            const float4* __restrict__ u4, const float4* __restrict__ k4, double* out) {
  const int r = blockIdx.x;
  const RodDev R = rods[r];
  const double* d = derived + 16 * (size_t)r;
  const double l0 = d[0], Kp = d[7], Ks = d[6];
  double len_err = 0, qn_err = 0, nonfin = 0, energy = 0;
  for (int li = threadIdx.x; li < R.n; li += blockDim.x) {
    const int64_t i = R.off + li;
    const float4 a = x4[i], q = q4[i], v = v4[i], o = o4[i];
    const float vals[12] = {a.x, a.y, a.z, v.x, v.y, v.z, q.x, q.y, q.z, q.w, o.x, o.y};
    for (int k = 0; k < 12; ++k)
      if (!isfinite(vals[k])) nonfin += 1;
    if (li <= R.n - 2) {
      const float4 b = x4[i + 1];
      const double ex = (double)b.x - a.x, ey = (double)b.y - a.y, ez = (double)b.z - a.z;
      const double len = sqrt(ex * ex + ey * ey + ez * ez);
      len_err = fmax(len_err, fabs(len / l0 - 1.0));
      const double qn = sqrt((double)q.x * q.x + (double)q.y * q.y + (double)q.z * q.z + (double)q.w * q.w);
      qn_err = fmax(qn_err, fabs(qn - 1.0));
      const double tx = ex / len, ty = ey / len, tz = ez / len;
      const double dx = 2.0 * ((double)q.x * q.z + (double)q.w * q.y);
      const double dy = 2.0 * ((double)q.y * q.z - (double)q.w * q.x);
      const double dz = 1.0 - 2.0 * ((double)q.x * q.x + (double)q.y * q.y);
      energy += 0.5 * l0 * Kp * ((tx - dx) * (tx - dx) + (ty - dy) * (ty - dy) + (tz - dz) * (tz - dz));
      if (!(R.flags & F_INEXT)) energy += 0.5 * l0 * Ks * (len / l0 - 1.0) * (len / l0 - 1.0);
    }
    if (li <= R.n - 3) {
      const float4 b = q4[i + 1];
      const double ux = (2.0 / l0) * ((double)q.w * b.x - (double)q.x * b.w - (double)q.y * b.z + (double)q.z * b.y);
      const double uy = (2.0 / l0) * ((double)q.w * b.y - (double)q.y * b.w - (double)q.z * b.x + (double)q.x * b.z);
      const double uz = (2.0 / l0) * ((double)q.w * b.z - (double)q.z * b.w - (double)q.x * b.y + (double)q.y * b.x);
      const float4 uh = u4[i], K = k4[i];
      energy += 0.5 * l0 *
                (K.x * (ux - uh.x) * (ux - uh.x) + K.y * (uy - uh.y) * (uy - uh.y) + K.z * (uz - uh.z) * (uz - uh.z));
    }
  }
  __shared__ double red[4][256];
  red[0][threadIdx.x] = len_err;
  red[1][threadIdx.x] = qn_err;
  red[2][threadIdx.x] = nonfin;
  red[3][threadIdx.x] = energy;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      red[0][threadIdx.x] = fmax(red[0][threadIdx.x], red[0][threadIdx.x + s]);
      red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + s]);
      red[2][threadIdx.x] += red[2][threadIdx.x + s];
      red[3][threadIdx.x] += red[3][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) out[4 * r + k] = red[k][0];
}

int check_handle(rod_handle h) {
  if (!h) return fail(CORDE_ERR_ARG, "NULL rod handle");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return fail(CORDE_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  return CORDE_OK;
}

void free_bins(rod_handle h) {
  for (auto& b : h->bins) {
    cudaFree(b.d_work);
    cudaFree(b.d_gh);
  }
  h->bins.clear();
}

// Group rods by variant; each group's work list is sorted by decreasing length so that
// the longest rods start first.
void invalidate_graph(rod_handle h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  h->graph_exec = nullptr;
  h->graph_steps = -1;
}

int build_bins(rod_handle h) {
  invalidate_graph(h);
  free_bins(h);
  std::vector<std::tuple<int, int, int>> keys;  // (blocks per rod, variant, grid)
  auto key_of = [&](int r) { return std::make_tuple(h->plan_cluster[r], h->plan[r], (int)h->plan_grid[r]); };
  for (int r = 0; r < h->n_rods; ++r) {
    if (r < (int)h->paired.size() && h->paired[r]) continue;
    const auto k = key_of(r);
    if (std::find(keys.begin(), keys.end(), k) == keys.end()) keys.push_back(k);
  }
  std::sort(keys.begin(), keys.end());
  for (const auto& k : keys) {
    std::vector<int> rods;
    for (int r = 0; r < h->n_rods; ++r)
      if (key_of(r) == k && !(r < (int)h->paired.size() && h->paired[r])) rods.push_back(r);
    // heaviest rods first: a rod's work per step grows with its nodes times (the force
    // phase, about seven constraint iterations' worth, plus its constraint iterations)
    std::stable_sort(rods.begin(), rods.end(), [&](int a, int b) {
      return (int64_t)h->n_nodes[a] * (7 + h->n_iters[a]) > (int64_t)h->n_nodes[b] * (7 + h->n_iters[b]);
    });
    Bin b{std::get<1>(k), (int)rods.size(), nullptr, std::get<0>(k), std::get<2>(k)};
    CK(cudaMalloc(&b.d_work, rods.size() * sizeof(int)));
    CK(cudaMemcpy(b.d_work, rods.data(), rods.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (b.grid) {
      const size_t n4 = rods.size() * 2 * (size_t)b.cluster * kHaloSlots * 2;
      CK(cudaMalloc(&b.d_gh, n4 * sizeof(float4)));
      CK(cudaMemset(b.d_gh, 0, n4 * sizeof(float4)));
    }
    h->bins.push_back(b);
  }
  return CORDE_OK;
}

int launch_bins(rod_handle h, const std::vector<Bin>& bins, int n_steps, const float4* drive, cudaStream_t s,
                float4* traj = nullptr, const MailboxDev* mb = nullptr) {
  StepArgs a = {};
  a.rods = h->d_rods;
  a.x4 = h->d_x;
  a.v4 = h->d_v;
  a.q4 = h->d_q;
  a.o4 = h->d_o;
  a.u4 = h->d_u;
  a.k4 = h->d_k;
  a.drive = drive;
  a.n_steps = n_steps;
  a.traj = traj;
  a.n_elem = h->n_elem;
  a.self_stats = h->d_self_stats;
  a.self_skin = h->d_self_skin;
  a.pos_out = h->io_pos;
  a.pdl = h->pdl;
  if (mb) a.mb = *mb;
  int launches = 0;
  for (const auto& b : bins) {
    a.work = b.d_work;
    if (b.cluster < 0) {
      const StepVariant& v = kSelfVariants[b.variant];
      cudaError_t e = v.launch(a, b.count, s);
      if (e != cudaSuccess)
        return fail(CORDE_ERR_CUDA, std::string("self-collision step launch (ept=") + std::to_string(v.ept) +
                                        ", nt=" + std::to_string(v.nt) + "): " + cudaGetErrorString(e));
    } else if (b.cluster > 0 && b.grid) {
      const ClusterVariant& v = kClusterVariants[b.variant];
      a.grid_halo = b.d_gh;
      cudaError_t e = v.launch_grid(a, b.count, b.cluster, s);
      if (e != cudaSuccess)
        return fail(CORDE_ERR_CUDA, std::string("cooperative grid step launch (ept=") + std::to_string(v.ept) +
                                        ", nt=" + std::to_string(v.nt) + ", blocks=" + std::to_string(b.cluster) +
                                        "): " + cudaGetErrorString(e));
    } else if (b.cluster > 0) {
      const ClusterVariant& v = kClusterVariants[b.variant];
      cudaError_t e = v.launch(a, b.count, b.cluster, s);
      if (e != cudaSuccess)
        return fail(CORDE_ERR_CUDA, std::string("cluster step launch (ept=") + std::to_string(v.ept) + ", nt=" +
                                        std::to_string(v.nt) + ", cluster=" + std::to_string(b.cluster) +
                                        "): " + cudaGetErrorString(e));
    } else {
      const StepVariant& v = variants()[b.variant];
      cudaError_t e = v.launch(a, b.count, s);
      if (e != cudaSuccess)
        return fail(CORDE_ERR_CUDA, std::string("step launch (ept=") + std::to_string(v.ept) +
                                        ", nt=" + std::to_string(v.nt) + "): " + cudaGetErrorString(e));
    }
    ++launches;
  }
  h->last_launches = launches;
  return CORDE_OK;
}

// True if the kernel may dereference p (device, managed or mapped pinned host memory);
// *dev receives the device address.
bool device_accessible(const void* p, const void** dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    *dev = p;
    return reinterpret_cast<uintptr_t>(p) % 16 == 0;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr) {
    *dev = at.devicePointer;
    return reinterpret_cast<uintptr_t>(at.devicePointer) % 16 == 0;
  }
  return false;
}

int ensure_capacity(float4** buf, size_t* cap, size_t need) {
  if (*cap >= need) return CORDE_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  CK(cudaMalloc(buf, need * sizeof(float4)));
  *cap = need;
  return CORDE_OK;
}

template <class T>
int upload(const T* src, size_t count, T** dst, cudaStream_t s) {
  *dst = nullptr;
  if (!src) return CORDE_OK;
  CK(cudaMalloc(dst, count * sizeof(T) + 16));
  CK(cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyDefault, s));
  return CORDE_OK;
}

bool params_valid(const RodParams& p, std::string& why) {
  if (p.n_nodes < 2) { why = "n_nodes must be >= 2"; return false; }
  if (!(p.length > 0) || !(p.radius > 0) || !(p.density > 0) || !(p.dt > 0)) {
    why = "length, radius, density and dt must be positive";
    return false;
  }
  if (!(p.E_bend >= 0) || !(p.E_stretch >= 0) || !(p.G >= 0) || !(p.damping_alpha >= 0)) {
    why = "moduli and damping must be non-negative";
    return false;
  }
  if (p.n_iters < 0) { why = "n_iters must be >= 0"; return false; }
  return true;
}

// Launches every bin and pair bin of one rod_step.  With branches, bin k goes to
// branches[k] (for the forked graph capture); otherwise all go to s in order.
int launch_all(rod_handle h, int n_steps, const float4* d, cudaStream_t s, const std::vector<cudaStream_t>* branches,
               const MailboxDev* mb = nullptr) {
  int launches = 0;
  size_t k = 0;
  for (size_t b = 0; b < h->bins.size(); ++b, ++k) {
    cudaStream_t sk = branches ? (*branches)[k] : s;
    std::vector<Bin> one{h->bins[b]};
    if (int rc = launch_bins(h, one, n_steps, d, sk, nullptr, mb)) return rc;
    ++launches;
  }
  if (!h->pair_bins.empty()) {
    StepArgs a = {};
    a.rods = h->d_rods;
    a.work = nullptr;
    a.x4 = h->d_x;
    a.v4 = h->d_v;
    a.q4 = h->d_q;
    a.o4 = h->d_o;
    a.u4 = h->d_u;
    a.k4 = h->d_k;
    a.drive = d;
    a.n_steps = n_steps;
    a.traj = nullptr;
    a.pos_out = h->io_pos;
    a.n_elem = h->n_elem;
    a.pdl = h->pdl;
    if (mb) a.mb = *mb;
    for (const auto& pb : h->pair_bins) {
      cudaStream_t sk = branches ? (*branches)[k] : s;
      ++k;
      cudaError_t e = launch_pair(pb.ept, pb.nt, a, pb.d_pairs, pb.count, sk);
      if (e != cudaSuccess) return fail(CORDE_ERR_CUDA, std::string("pair launch: ") + cudaGetErrorString(e));
      ++launches;
    }
  }
  h->last_launches = launches;
  return CORDE_OK;
}

// Captures one rod_step into a CUDA graph whose kernel nodes run concurrently (fork on
// an event, one branch stream per bin, join), so that the bins fill the SMs together.
int capture_graph(rod_handle h, int n_steps, const float4* d) {
  invalidate_graph(h);
  const size_t nb = h->bins.size() + h->pair_bins.size();
  if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  if (!h->fork_ev) CK(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
  while (h->side.size() < nb) {
    cudaStream_t st;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    h->side.push_back(st);
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    h->join_ev.push_back(ev);
  }
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = CORDE_OK;
  cudaError_t e = cudaEventRecord(h->fork_ev, h->cap_stream);
  for (size_t k = 0; k < nb && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(h->side[k], h->fork_ev, 0);
  if (e == cudaSuccess) rc = launch_all(h, n_steps, d, h->cap_stream, &h->side);
  for (size_t k = 0; k < nb && e == cudaSuccess && rc == CORDE_OK; ++k) {
    e = cudaEventRecord(h->join_ev[k], h->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->cap_stream, h->join_ev[k], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
  if (rc != CORDE_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(CORDE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  cudaError_t e3 = cudaGraphInstantiate(&h->graph_exec, g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) {
    h->graph_exec = nullptr;
    return fail(CORDE_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
  }
  h->graph_steps = n_steps;
  h->graph_drive = d;
  h->graph_pos_out = h->io_pos;
  h->graph_launches = (int)nb;
  return CORDE_OK;
}

}  // namespace

extern "C" {

int rod_set_graph_mode(rod_handle h, int mode) {
  if (int rc = check_handle(h)) return rc;
  if (mode < 0 || mode > 2) return fail(CORDE_ERR_ARG, "graph mode must be 0, 1 or 2");
  h->graph_mode = mode;
  invalidate_graph(h);
  return CORDE_OK;
}

const char* rod_strerror(int code) {
  switch (code) {
    case CORDE_OK: return "ok";
    case CORDE_ERR_ARG: return "invalid argument";
    case CORDE_ERR_CUDA: return "CUDA runtime error";
    case CORDE_ERR_OOM: return "device out of memory";
    case CORDE_ERR_UNSUPPORTED: return "unsupported (rod too long for the compiled kernels, or no device)";
    case CORDE_ERR_NONFINITE: return "non-finite state";
    default: return "unknown error";
  }
}

const char* rod_last_error(void) { return g_last_error.c_str(); }

int rod_create(int n_rods, const RodParams* params, const float* pos, const float* quat, const float* rest_quat,
               const float* vel, const float* omega, const float* stiff_mul, void* stream, rod_handle* out) {
  if (!out) return fail(CORDE_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_rods < 1 || !params || !pos || !quat) return fail(CORDE_ERR_ARG, "need n_rods >= 1, params, pos and quat");
  const int cap = std::max(max_capacity(), max_grid_capacity());
  std::vector<int> nn(n_rods), off(n_rods);
  int64_t E = 0;
  for (int r = 0; r < n_rods; ++r) {
    std::string why;
    if (!params_valid(params[r], why)) return fail(CORDE_ERR_ARG, "rod " + std::to_string(r) + ": " + why);
    if (params[r].n_nodes > cap)
      return fail(CORDE_ERR_UNSUPPORTED, "rod " + std::to_string(r) + " has " + std::to_string(params[r].n_nodes) +
                                             " nodes; the compiled kernels hold at most " + std::to_string(cap));
    nn[r] = params[r].n_nodes;
    off[r] = (int)E;
    E += nn[r];
  }
  if (E > (int64_t)0x7fffffff) return fail(CORDE_ERR_ARG, "too many elements");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaStream_t s = (cudaStream_t)stream;

  rod_handle h = new corde_rods();
  h->device = dev;
  h->n_rods = n_rods;
  h->n_elem = E;
  h->n_nodes = nn;
  h->off = off;
  h->n_iters.resize(n_rods);
  h->dt.resize(n_rods);
  h->tube.assign(n_rods, 0);
  h->self.assign(n_rods, 0);
  for (int r = 0; r < n_rods; ++r) {
    h->n_iters[r] = params[r].inextensible ? params[r].n_iters : 0;
    h->dt[r] = params[r].dt;
  }
  const int64_t F = E - n_rods, J = E - 2 * (int64_t)n_rods;
  std::vector<int> elem_rod(E);
  for (int r = 0; r < n_rods; ++r)
    for (int k = 0; k < nn[r]; ++k) elem_rod[off[r] + k] = r;

  RodParams* d_params = nullptr;
  int *d_off = nullptr;
  float *d_pos = nullptr, *d_quat = nullptr, *d_rest = nullptr, *d_vel = nullptr, *d_om = nullptr, *d_mul = nullptr;
  auto cleanup_staging = [&]() {
    cudaFree(d_params); cudaFree(d_off); cudaFree(d_pos); cudaFree(d_quat); cudaFree(d_rest);
    cudaFree(d_vel); cudaFree(d_om); cudaFree(d_mul);
  };
  int rc = CORDE_OK;
  auto step_rc = [&](int c) { if (rc == CORDE_OK) rc = c; };
  do {
    const size_t b4 = (size_t)E * sizeof(float4);
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&h->d_rods, n_rods * sizeof(RodDev))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_derived, n_rods * 16 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_x, b4)) != cudaSuccess || (e = cudaMalloc(&h->d_v, b4)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_q, b4)) != cudaSuccess || (e = cudaMalloc(&h->d_o, b4)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_u, b4)) != cudaSuccess || (e = cudaMalloc(&h->d_k, b4)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_drive, n_rods * 2 * sizeof(float4))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_elem_rod, E * sizeof(int))) != cudaSuccess) {
      rc = fail(CORDE_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
      break;
    }
    step_rc(upload(params, n_rods, &d_params, s));
    step_rc(upload(off.data(), n_rods, &d_off, s));
    step_rc(upload(pos, 3 * E, &d_pos, s));
    step_rc(upload(quat, 4 * F, &d_quat, s));
    step_rc(upload(rest_quat, 4 * F, &d_rest, s));
    step_rc(upload(vel, 3 * E, &d_vel, s));
    step_rc(upload(omega, 3 * F, &d_om, s));
    step_rc(upload(stiff_mul, 3 * J, &d_mul, s));
    if (rc != CORDE_OK) break;
    if ((e = cudaMemcpyAsync(h->d_elem_rod, elem_rod.data(), E * sizeof(int), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(h->d_drive, 0, n_rods * 2 * sizeof(float4), s)) != cudaSuccess) {
      rc = fail(CORDE_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
      break;
    }
    derive_kernel<<<(n_rods + 127) / 128, 128, 0, s>>>(n_rods, d_params, d_off, h->d_rods, h->d_derived);
    pack_kernel<<<(unsigned)((E + 255) / 256), 256, 0, s>>>(E, h->d_elem_rod, h->d_rods, d_params, h->d_derived,
                                                           d_pos, d_quat, d_rest, d_vel, d_om, d_mul, h->d_x,
                                                           h->d_v, h->d_q, h->d_o, h->d_u, h->d_k);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      rc = fail(CORDE_ERR_CUDA, std::string("init kernels: ") + cudaGetErrorString(e));
      break;
    }
    h->derived.resize(16 * (size_t)n_rods);
    if ((e = cudaMemcpy(h->derived.data(), h->d_derived, 16 * n_rods * sizeof(double), cudaMemcpyDeviceToHost)) !=
        cudaSuccess) {
      rc = fail(CORDE_ERR_CUDA, std::string("copy derived: ") + cudaGetErrorString(e));
      break;
    }
    h->plan.resize(n_rods);
    h->plan_cluster.assign(n_rods, 0);
    h->plan_grid.assign(n_rods, 0);
    for (int r = 0; r < n_rods; ++r) {
      if (nn[r] <= max_block_capacity()) {
        h->plan[r] = default_variant(nn[r]);
      } else if (nn[r] <= max_capacity()) {
        default_cluster_plan(nn[r], &h->plan[r], &h->plan_cluster[r]);
      } else {
        default_grid_plan(nn[r], &h->plan[r], &h->plan_cluster[r]);
        h->plan_grid[r] = 1;
      }
    }
    rc = build_bins(h);
  } while (0);
  cleanup_staging();
  if (rc != CORDE_OK) {
    std::string msg = g_last_error;
    rod_destroy(h);
    g_last_error = msg;
    return rc;
  }
  *out = h;
  return CORDE_OK;
}

static int step_impl(rod_handle h, int n_steps, const float* drive, float4* pos_out, void* stream) {
  if (int rc = check_handle(h)) return rc;
  if (n_steps < 0) return fail(CORDE_ERR_ARG, "n_steps must be >= 0");
  if (n_steps == 0) {
    h->last_launches = 0;
    return CORDE_OK;
  }
  const float4* d = h->d_drive;
  if (drive) {
    // The kernel dereferences `drive`: accept device, managed or mapped pinned host memory.
    const void* dp = nullptr;
    if (!device_accessible(drive, &dp))
      return fail(CORDE_ERR_ARG, "drive must be 16-byte aligned device, managed or mapped pinned host memory");
    d = reinterpret_cast<const float4*>(dp);
  }
  if (h->mb_period > 0) {
    MailboxDev mb = h->mb_dev;
    mb.step0 = h->steps_done;
    if (int rc = launch_all(h, n_steps, d, (cudaStream_t)stream, nullptr, &mb)) return rc;
    h->steps_done += n_steps;
    return CORDE_OK;
  }
  const int n_launch = (int)h->bins.size() + (int)h->pair_bins.size();
  const bool use_graph = h->graph_mode == 2 || (h->graph_mode == 1 && n_launch > 1);
  h->steps_done += n_steps;
  if (!use_graph) return launch_all(h, n_steps, d, (cudaStream_t)stream, nullptr);
  if (!h->d_drive_graph) CK(cudaMalloc(&h->d_drive_graph, h->n_rods * 2 * sizeof(float4)));
  CK(cudaMemcpyAsync(h->d_drive_graph, d, h->n_rods * 2 * sizeof(float4), cudaMemcpyDefault, (cudaStream_t)stream));
  if (!h->graph_exec || h->graph_steps != n_steps || h->graph_drive != h->d_drive_graph ||
      h->graph_pos_out != pos_out) {
    if (int rc = capture_graph(h, n_steps, h->d_drive_graph)) return rc;
  }
  CK(cudaGraphLaunch(h->graph_exec, (cudaStream_t)stream));
  h->last_launches = h->graph_launches;
  return CORDE_OK;
}

int rod_step(rod_handle h, int n_steps, const float* drive, void* stream) {
  return step_impl(h, n_steps, drive, nullptr, stream);
}

int rod_step_io(rod_handle h, int n_steps, const float* drive, float* pos_out, void* stream) {
  if (int rc = check_handle(h)) return rc;
  float4* po = nullptr;
  if (pos_out) {
    const void* dp = nullptr;
    if (!device_accessible(pos_out, &dp))
      return fail(CORDE_ERR_ARG, "pos_out must be 16-byte aligned device, managed or mapped pinned host memory");
    po = reinterpret_cast<float4*>(const_cast<void*>(dp));
  }
  h->io_pos = po;
  const int rc = step_impl(h, n_steps, drive, po, stream);
  h->io_pos = nullptr;
  return rc;
}

int rod_set_input(rod_handle h, const float* drive, void* stream) {
  if (int rc = check_handle(h)) return rc;
  if (!drive) return fail(CORDE_ERR_ARG, "drive is NULL");
  CK(cudaMemcpyAsync(h->d_drive, drive, h->n_rods * 2 * sizeof(float4), cudaMemcpyDefault, (cudaStream_t)stream));
  return CORDE_OK;
}

int rod_get_state(rod_handle h, float* pos4, float* quat4, float* vel4, float* omega4, void* stream) {
  if (int rc = check_handle(h)) return rc;
  const size_t b = (size_t)h->n_elem * sizeof(float4);
  cudaStream_t s = (cudaStream_t)stream;
  if (pos4) CK(cudaMemcpyAsync(pos4, h->d_x, b, cudaMemcpyDefault, s));
  if (quat4) CK(cudaMemcpyAsync(quat4, h->d_q, b, cudaMemcpyDefault, s));
  if (vel4) CK(cudaMemcpyAsync(vel4, h->d_v, b, cudaMemcpyDefault, s));
  if (omega4) CK(cudaMemcpyAsync(omega4, h->d_o, b, cudaMemcpyDefault, s));
  return CORDE_OK;
}

int rod_set_state(rod_handle h, const float* pos4, const float* quat4, const float* vel4, const float* omega4,
                  void* stream) {
  if (int rc = check_handle(h)) return rc;
  const size_t b = (size_t)h->n_elem * sizeof(float4);
  cudaStream_t s = (cudaStream_t)stream;
  // positions: copy x, y, z only (12 of every 16 bytes) so that the masses in .w stay
  if (pos4)
    CK(cudaMemcpy2DAsync(h->d_x, sizeof(float4), pos4, sizeof(float4), 3 * sizeof(float), h->n_elem,
                         cudaMemcpyDefault, s));
  if (quat4) CK(cudaMemcpyAsync(h->d_q, quat4, b, cudaMemcpyDefault, s));
  if (vel4) CK(cudaMemcpyAsync(h->d_v, vel4, b, cudaMemcpyDefault, s));
  if (omega4) CK(cudaMemcpyAsync(h->d_o, omega4, b, cudaMemcpyDefault, s));
  return CORDE_OK;
}

int rod_info(rod_handle h, int* n_rods, int64_t* n_elements) {
  if (!h) return fail(CORDE_ERR_ARG, "NULL rod handle");
  if (n_rods) *n_rods = h->n_rods;
  if (n_elements) *n_elements = h->n_elem;
  return CORDE_OK;
}

int rod_get_derived(rod_handle h, double* per_rod, float* per_joint) {
  if (int rc = check_handle(h)) return rc;
  if (per_rod) std::memcpy(per_rod, h->derived.data(), h->derived.size() * sizeof(double));
  if (per_joint) {
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy2D(per_joint, 2 * sizeof(float4), h->d_k, sizeof(float4), sizeof(float4), h->n_elem,
                    cudaMemcpyDefault));
    CK(cudaMemcpy2D(per_joint + 4, 2 * sizeof(float4), h->d_u, sizeof(float4), sizeof(float4), h->n_elem,
                    cudaMemcpyDefault));
  }
  return CORDE_OK;
}

int rod_set_material(rod_handle h, const float* per_joint, void* stream) {
  if (int rc = check_handle(h)) return rc;
  if (!per_joint) return fail(CORDE_ERR_ARG, "per_joint is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpy2DAsync(h->d_k, sizeof(float4), per_joint, 2 * sizeof(float4), sizeof(float4), h->n_elem,
                       cudaMemcpyDefault, s));
  CK(cudaMemcpy2DAsync(h->d_u, sizeof(float4), per_joint + 4, 2 * sizeof(float4), sizeof(float4), h->n_elem,
                       cudaMemcpyDefault, s));
  return CORDE_OK;
}

int rod_diagnostics(rod_handle h, double* out) {
  if (int rc = check_handle(h)) return rc;
  if (!out) return fail(CORDE_ERR_ARG, "out is NULL");
  double* d_out = nullptr;
  CK(cudaMalloc(&d_out, 4 * h->n_rods * sizeof(double)));
  diag_kernel<<<h->n_rods, 256>>>(h->d_rods, h->d_derived, h->d_x, h->d_q, h->d_v, h->d_o, h->d_u, h->d_k, d_out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, 4 * h->n_rods * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d_out);
  if (e != cudaSuccess) return fail(CORDE_ERR_CUDA, std::string("diagnostics: ") + cudaGetErrorString(e));
  for (int r = 0; r < h->n_rods; ++r)
    if (out[4 * r + 2] > 0) return fail(CORDE_ERR_NONFINITE, "rod " + std::to_string(r) + " has non-finite state");
  return CORDE_OK;
}

int rod_set_plan(rod_handle h, int ept, int nt) {
  if (int rc = check_handle(h)) return rc;
  if (ept == 0) {
    for (int r = 0; r < h->n_rods; ++r) {
      if (h->self[r]) continue;
      h->plan_cluster[r] = 0;
      h->plan_grid[r] = 0;
      if (h->n_nodes[r] <= max_block_capacity()) {
        h->plan[r] = default_variant(h->n_nodes[r]);
      } else if (h->n_nodes[r] <= max_capacity()) {
        default_cluster_plan(h->n_nodes[r], &h->plan[r], &h->plan_cluster[r]);
      } else {
        if (h->mb_period > 0) return fail(CORDE_ERR_UNSUPPORTED, "rod_set_plan: a rod on a grid runs without the mailbox");
        default_grid_plan(h->n_nodes[r], &h->plan[r], &h->plan_cluster[r]);
        h->plan_grid[r] = 1;
      }
    }
    return build_bins(h);
  }
  const int v = find_variant(ept, nt);
  if (v < 0) return fail(CORDE_ERR_ARG, "no compiled variant with ept=" + std::to_string(ept) + ", nt=" + std::to_string(nt));
  for (int r = 0; r < h->n_rods; ++r)
    if (!h->self[r] && variants()[v].capacity() >= h->n_nodes[r]) {
      h->plan[r] = v;
      h->plan_cluster[r] = 0;
      h->plan_grid[r] = 0;
    }
  return build_bins(h);
}

int rod_set_plan_grid(rod_handle h, int ept, int nt, int blocks) {
  if (int rc = check_handle(h)) return rc;
  const int v = find_cluster_variant(ept, nt);
  if (v < 0 || blocks < 2)
    return fail(CORDE_ERR_ARG, "no grid variant with ept=" + std::to_string(ept) + ", nt=" + std::to_string(nt) +
                                   ", blocks=" + std::to_string(blocks));
  if (h->mb_period > 0) return fail(CORDE_ERR_UNSUPPORTED, "rod_set_plan_grid: a rod on a grid runs without the mailbox");
  int rods = 0;
  for (int r = 0; r < h->n_rods; ++r)
    if (!h->self[r] && !(r < (int)h->paired.size() && h->paired[r]) && kClusterVariants[v].capacity(blocks) >= h->n_nodes[r])
      ++rods;
  if ((int64_t)rods * blocks > kClusterVariants[v].grid_blocks())
    return fail(CORDE_ERR_UNSUPPORTED, "rod_set_plan_grid: " + std::to_string(rods) + " rods x " +
                                           std::to_string(blocks) + " blocks are more than the " +
                                           std::to_string(kClusterVariants[v].grid_blocks()) +
                                           " blocks the device holds at once");
  for (int r = 0; r < h->n_rods; ++r)
    if (!h->self[r] && !(r < (int)h->paired.size() && h->paired[r]) && kClusterVariants[v].capacity(blocks) >= h->n_nodes[r]) {
      h->plan[r] = v;
      h->plan_cluster[r] = blocks;
      h->plan_grid[r] = 1;
    }
  return build_bins(h);
}

int rod_set_adjoint_pipeline(rod_handle h, int enable) {
  if (int rc = check_handle(h)) return rc;
  h->adj_pipe = enable ? 1 : 0;
  return CORDE_OK;
}

int rod_set_adjoint_record_budget(rod_handle h, long long bytes) {
  if (int rc = check_handle(h)) return rc;
  if (bytes < 0) return fail(CORDE_ERR_ARG, "rod_set_adjoint_record_budget: bytes must be >= 0");
  h->adj_record_budget = bytes;
  return CORDE_OK;
}

int rod_set_launch_overlap(rod_handle h, int enable) {
  if (int rc = check_handle(h)) return rc;
  if (enable != 0 && enable != 1) return fail(CORDE_ERR_ARG, "rod_set_launch_overlap: enable must be 0 or 1");
  if (h->pdl != enable) invalidate_graph(h);
  h->pdl = enable;
  return CORDE_OK;
}

int rod_set_plan_cluster(rod_handle h, int ept, int nt, int cluster) {
  if (int rc = check_handle(h)) return rc;
  const int v = find_cluster_variant(ept, nt);
  if (v < 0 || cluster < 2 || cluster > kMaxCluster)
    return fail(CORDE_ERR_ARG, "no cluster variant with ept=" + std::to_string(ept) + ", nt=" + std::to_string(nt) +
                                   ", cluster=" + std::to_string(cluster));
  for (int r = 0; r < h->n_rods; ++r)
    if (!h->self[r] && kClusterVariants[v].capacity(cluster) >= h->n_nodes[r]) {
      h->plan[r] = v;
      h->plan_cluster[r] = cluster;
      h->plan_grid[r] = 0;
    }
  return build_bins(h);
}

int rod_autotune_steps(rod_handle h, const int* candidates, int n_candidates, int min_steps, int* best,
                       void* stream) {
  if (int rc = check_handle(h)) return rc;
  if (!candidates || n_candidates < 1 || !best || min_steps < 1)
    return fail(CORDE_ERR_ARG, "rod_autotune_steps: need candidates, min_steps >= 1 and best");
  for (int k = 0; k < n_candidates; ++k)
    if (candidates[k] < 1) return fail(CORDE_ERR_ARG, "rod_autotune_steps: candidates must be >= 1");
  if (h->mb_period > 0) return fail(CORDE_ERR_UNSUPPORTED, "rod_autotune_steps: not with a mailbox enabled");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b = (size_t)h->n_elem * sizeof(float4);
  float4 *sx = nullptr, *sv = nullptr, *sq = nullptr, *so = nullptr;
  CK(cudaMalloc(&sx, b));
  CK(cudaMalloc(&sv, b));
  CK(cudaMalloc(&sq, b));
  CK(cudaMalloc(&so, b));
  CK(cudaMemcpyAsync(sx, h->d_x, b, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(sv, h->d_v, b, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(sq, h->d_q, b, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(so, h->d_o, b, cudaMemcpyDeviceToDevice, s));
  auto restore = [&]() {
    cudaMemcpyAsync(h->d_x, sx, b, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->d_v, sv, b, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->d_q, sq, b, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->d_o, so, b, cudaMemcpyDeviceToDevice, s);
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const long long steps0 = h->steps_done;
  int rc = CORDE_OK;
  float best_us = 1e30f;
  int best_n = candidates[0];
  // two passes, the second one counts (clock ramp-up, graph capture per candidate)
  for (int pass = 0; pass < 2 && rc == CORDE_OK; ++pass) {
    best_us = 1e30f;
    for (int k = 0; k < n_candidates && rc == CORDE_OK; ++k) {
      const int S = candidates[k];
      const int launches = (min_steps + S - 1) / S;
      restore();
      if ((rc = step_impl(h, S, nullptr, nullptr, s)) != CORDE_OK) break;  // warm-up (and graph capture)
      restore();
      cudaEventRecord(e0, s);
      for (int l = 0; l < launches && rc == CORDE_OK; ++l) rc = step_impl(h, S, nullptr, nullptr, s);
      cudaEventRecord(e1, s);
      if (rc != CORDE_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = fail(CORDE_ERR_CUDA, "rod_autotune_steps: timing");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const float us_per_step = ms * 1e3f / (float)(launches * S);
      if (us_per_step < best_us) {
        best_us = us_per_step;
        best_n = S;
      }
    }
  }
  restore();
  cudaStreamSynchronize(s);
  h->steps_done = steps0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sx); cudaFree(sv); cudaFree(sq); cudaFree(so);
  if (rc != CORDE_OK) return rc;
  *best = best_n;
  return CORDE_OK;
}

int rod_get_plan(rod_handle h, int* plan) {
  if (!h || !plan) return fail(CORDE_ERR_ARG, "NULL argument");
  for (int r = 0; r < h->n_rods; ++r) {
    const int C = h->plan_cluster[r];
    const int ept = C > 0 ? kClusterVariants[h->plan[r]].ept
                          : (C < 0 ? kSelfVariants[h->plan[r]].ept : variants()[h->plan[r]].ept);
    const int nt = C > 0 ? kClusterVariants[h->plan[r]].nt
                         : (C < 0 ? kSelfVariants[h->plan[r]].nt : variants()[h->plan[r]].nt);
    plan[3 * r] = ept;
    plan[3 * r + 1] = nt;
    plan[3 * r + 2] = C > 0 ? (h->plan_grid[r] ? -C : C) : 0;
  }
  return CORDE_OK;
}

int rod_last_launch_count(rod_handle h) { return h ? h->last_launches : 0; }

int rod_autotune(rod_handle h, int n_steps, void* stream) {
  if (int rc = check_handle(h)) return rc;
  if (n_steps < 1) return fail(CORDE_ERR_ARG, "n_steps must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b = (size_t)h->n_elem * sizeof(float4);
  float4 *sx = nullptr, *sv = nullptr, *sq = nullptr, *so = nullptr;
  CK(cudaMalloc(&sx, b));
  CK(cudaMalloc(&sv, b));
  CK(cudaMalloc(&sq, b));
  CK(cudaMalloc(&so, b));
  CK(cudaMemcpyAsync(sx, h->d_x, b, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(sv, h->d_v, b, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(sq, h->d_q, b, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(so, h->d_o, b, cudaMemcpyDeviceToDevice, s));
  auto restore = [&]() {
    cudaMemcpyAsync(h->d_x, sx, b, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->d_v, sv, b, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->d_q, sq, b, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->d_o, so, b, cudaMemcpyDeviceToDevice, s);
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // Length classes: powers of two (rods in (2^(k-1), 2^k]).
  std::vector<int> cls(h->n_rods);
  int max_cls = 0;
  for (int r = 0; r < h->n_rods; ++r) {
    int c = 5;
    while ((1 << c) < h->n_nodes[r]) ++c;
    cls[r] = c;
    if (h->plan_cluster[r] == 0) max_cls = std::max(max_cls, c);
  }
  int rc = CORDE_OK;
  for (int c = 5; c <= max_cls && rc == CORDE_OK; ++c) {
    std::vector<int> rods;
    int nmax = 0;
    for (int r = 0; r < h->n_rods; ++r)
      if (cls[r] == c && h->plan_cluster[r] == 0 && !(r < (int)h->paired.size() && h->paired[r])) {
        rods.push_back(r);
        nmax = std::max(nmax, h->n_nodes[r]);
      }
    if (rods.empty()) continue;
    std::stable_sort(rods.begin(), rods.end(), [&](int a, int bb) {
      return (int64_t)h->n_nodes[a] * (7 + h->n_iters[a]) > (int64_t)h->n_nodes[bb] * (7 + h->n_iters[bb]);
    });
    int* d_work = nullptr;
    if (cudaMalloc(&d_work, rods.size() * sizeof(int)) != cudaSuccess) { rc = fail(CORDE_ERR_OOM, "autotune work list"); break; }
    cudaMemcpy(d_work, rods.data(), rods.size() * sizeof(int), cudaMemcpyHostToDevice);
    float best_ms = 1e30f;
    int best_v = -1;
    // Each candidate: one warm-up launch, then the best of three timed launches from the same
    // state.  The whole sweep runs twice and only the second pass counts, so that the first
    // candidates are not measured while the clocks still ramp up from idle.
    for (int pass = 0; pass < 2 && rc == CORDE_OK; ++pass) {
      best_ms = 1e30f;
      best_v = -1;
      for (size_t vi = 0; vi < variants().size(); ++vi) {
        const StepVariant& v = variants()[vi];
        if (v.capacity() < nmax) continue;
        if (v.capacity() >= 8 * nmax && v.nt > 32) continue;  // mostly idle threads
        std::vector<Bin> one{Bin{(int)vi, (int)rods.size(), d_work}};
        restore();
        if ((rc = launch_bins(h, one, n_steps, h->d_drive, s)) != CORDE_OK) break;  // warm-up
        float best_rep = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          float ms = 0.f;
          restore();
          cudaEventRecord(e0, s);
          if ((rc = launch_bins(h, one, n_steps, h->d_drive, s)) != CORDE_OK) break;
          cudaEventRecord(e1, s);
          if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(CORDE_ERR_CUDA, "autotune timing"); break; }
          cudaEventElapsedTime(&ms, e0, e1);
          best_rep = std::min(best_rep, ms);
        }
        if (rc != CORDE_OK) break;
        if (best_rep < best_ms) { best_ms = best_rep; best_v = (int)vi; }
      }
    }
    cudaFree(d_work);
    if (best_v >= 0)
      for (int r : rods) h->plan[r] = best_v;
  }
  restore();
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sx); cudaFree(sv); cudaFree(sq); cudaFree(so);
  if (rc != CORDE_OK) return rc;
  return build_bins(h);
}

__global__ void set_tube_kernel(RodDev* rods, int r, float cx, float cy, float cz, float rc, float allow, float mu,
                                int enable) {
  RodDev& R = rods[r];
  R.tube_cx = cx;
  R.tube_cy = cy;
  R.tube_cz = cz;
  R.tube_rc = rc;
  R.tube_allow = allow;
  R.tube_mu = mu;
  R.flags = enable ? (R.flags | F_TUBE) : (R.flags & ~F_TUBE);
}

int rod_set_tube(rod_handle h, int rod, const double* tube) {
  if (int rc = check_handle(h)) return rc;
  if (rod < 0 || rod >= h->n_rods || !tube) return fail(CORDE_ERR_ARG, "rod_set_tube: bad rod or NULL tube");
  const double radius = h->derived[16 * (size_t)rod + 1] > 0 ? std::sqrt(h->derived[16 * (size_t)rod + 1] / kPi) : 0;
  const int enable = tube[6] != 0.0;
  if (enable && !(tube[3] > 0 && tube[4] > radius && tube[5] >= 0))
    return fail(CORDE_ERR_ARG, "rod_set_tube: need rc > 0, inner radius > rod radius, mu >= 0");
  if (enable && h->n_iters[rod] == 0)
    return fail(CORDE_ERR_UNSUPPORTED, "rod_set_tube: contact runs in the constraint iterations of an inextensible rod");
  if (enable && !h->paired.empty() && h->paired[rod])
    return fail(CORDE_ERR_UNSUPPORTED, "rod_set_tube: not for a rod bound in a pair");
  set_tube_kernel<<<1, 1>>>(h->d_rods, rod, (float)tube[0], (float)tube[1], (float)tube[2], (float)tube[3],
                            (float)(tube[4] - radius), (float)tube[5], enable);
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  if (enable) h->tube[rod] = 1;
  else h->tube[rod] = 0;
  return CORDE_OK;
}

__global__ void set_self_kernel(RodDev* rods, int r, float dist, float reach, float mu, float sep, int enable) {
  RodDev& R = rods[r];
  R.self_dist = dist;
  R.self_reach = reach;
  R.self_mu = mu;
  R.self_sep = sep;
  R.flags = enable ? (R.flags | F_SELF) : (R.flags & ~F_SELF);
}

int rod_set_self_collision(rod_handle h, int rod, const double* p) {
  if (int rc = check_handle(h)) return rc;
  if (rod < 0 || rod >= h->n_rods || !p) return fail(CORDE_ERR_ARG, "rod_set_self_collision: bad rod or NULL params");
  const int enable = p[1] != 0.0;
  if (enable) {
    if (!(p[0] >= 0)) return fail(CORDE_ERR_ARG, "rod_set_self_collision: mu must be >= 0");
    if (h->n_iters[rod] == 0)
      return fail(CORDE_ERR_UNSUPPORTED, "rod_set_self_collision: contact runs in the constraint iterations of an "
                                         "inextensible rod");
    if (!h->paired.empty() && h->paired[rod])
      return fail(CORDE_ERR_UNSUPPORTED, "rod_set_self_collision: not for a rod bound in a pair");
    if (h->mb_period > 0) return fail(CORDE_ERR_UNSUPPORTED, "rod_set_self_collision: not with a mailbox enabled");
    if (h->n_nodes[rod] > kSelfMaxNodes)
      return fail(CORDE_ERR_UNSUPPORTED, "rod_set_self_collision: rods of at most " + std::to_string(kSelfMaxNodes) +
                                             " nodes");
  }
  if (!h->d_self_stats) {
    CK(cudaMalloc(&h->d_self_stats, 2 * h->n_rods * sizeof(int4)));
    CK(cudaMemset(h->d_self_stats, 0, 2 * h->n_rods * sizeof(int4)));
  }
  if (!h->d_self_skin) {
    CK(cudaMalloc(&h->d_self_skin, (size_t)h->n_rods * kSelfSkinBytes));
    CK(cudaMemset(h->d_self_skin, 0, (size_t)h->n_rods * kSelfSkinBytes));
  }
  // a kept skin list was built with the old settings: discard it
  CK(cudaMemset(h->d_self_skin + (size_t)rod * kSelfSkinBytes, 0, 16));
  const double* dr = &h->derived[16 * (size_t)rod];
  const double radius = std::sqrt(dr[1] / kPi), l0 = dr[0];
  const int sep = std::max(2, (int)std::floor(2.0 * radius / l0) + 1);
  set_self_kernel<<<1, 1>>>(h->d_rods, rod, (float)(2.0 * radius), (float)(3.0 * radius), (float)p[0], (float)sep,
                            enable);
  CK(cudaGetLastError());
  CK(cudaMemset(h->d_self_stats + 2 * rod, 0, 2 * sizeof(int4)));
  CK(cudaDeviceSynchronize());
  h->self[rod] = (char)enable;
  if (enable) {
    // the first block of the list that holds the rod (two elements per thread up to 512
    // nodes, four beyond)
    int v = 0;
    while (v + 1 < kNumSelfVariants && kSelfVariants[v].capacity() < h->n_nodes[rod]) ++v;
    h->plan[rod] = v;
    h->plan_cluster[rod] = -1;
    h->plan_grid[rod] = 0;
  } else if (h->plan_cluster[rod] < 0) {
    h->plan[rod] = default_variant(h->n_nodes[rod]);
    h->plan_cluster[rod] = 0;
    h->plan_grid[rod] = 0;
  }
  return build_bins(h);
}

int rod_self_collision_stats(rod_handle h, int rod, int* out) {
  if (int rc = check_handle(h)) return rc;
  if (rod < 0 || rod >= h->n_rods || !out) return fail(CORDE_ERR_ARG, "rod_self_collision_stats: bad rod or NULL out");
  int4 st[2] = {make_int4(0, 0, 0, 0), make_int4(0, 0, 0, 0)};
  if (h->d_self_stats) CK(cudaMemcpy(st, h->d_self_stats + 2 * rod, 2 * sizeof(int4), cudaMemcpyDeviceToHost));
  out[0] = st[0].x;
  out[1] = st[0].y;
  out[2] = st[0].z;
  out[3] = st[0].w;
  out[4] = st[1].x;
  return CORDE_OK;
}

// Pair kernel layout: two elements per thread up to 512 nodes per rod, four up to 1024,
// the smallest power-of-two group (>= 32 threads) holding the longer rod.
static int pair_layout(int n, int* ept, int* nt) {
  *ept = n <= 512 ? 2 : 4;
  *nt = 32;
  while (*nt * *ept < n) *nt *= 2;
  return *nt <= 256 ? CORDE_OK : CORDE_ERR_UNSUPPORTED;
}

static int build_pair_bins(rod_handle h) {
  invalidate_graph(h);
  for (auto& pb : h->pair_bins) cudaFree(pb.d_pairs);
  h->pair_bins.clear();
  for (int ept : {2, 4})
    for (int nt = 32; nt <= 256; nt *= 2) {
      std::vector<int4> ps;
      for (const int4& p : h->pairs) {
        int e = 0, t = 0;
        pair_layout(std::max(h->n_nodes[p.x], h->n_nodes[p.y]), &e, &t);
        if (e == ept && t == nt) ps.push_back(p);
      }
      if (ps.empty()) continue;
      corde_rods::PairBin pb{ept, nt, (int)ps.size(), nullptr};
      CK(cudaMalloc(&pb.d_pairs, ps.size() * sizeof(int4)));
      CK(cudaMemcpy(pb.d_pairs, ps.data(), ps.size() * sizeof(int4), cudaMemcpyHostToDevice));
      h->pair_bins.push_back(pb);
    }
  return CORDE_OK;
}

int rod_bind(rod_handle h, int outer, int inner, int mode) {
  if (int rc = check_handle(h)) return rc;
  if (outer < 0 || inner < 0 || outer >= h->n_rods || inner >= h->n_rods || outer == inner)
    return fail(CORDE_ERR_ARG, "rod_bind: bad rod indices");
  if (mode < 0 || mode > 2) return fail(CORDE_ERR_ARG, "rod_bind: mode must be 0, 1 or 2");
  if (h->mb_period > 0) return fail(CORDE_ERR_UNSUPPORTED, "rod_bind: not with a mailbox enabled");
  if (h->paired.empty()) h->paired.assign(h->n_rods, 0);
  if (h->paired[outer] || h->paired[inner]) return fail(CORDE_ERR_ARG, "rod_bind: rod already in a pair");
  if (h->tube[outer] || h->tube[inner]) return fail(CORDE_ERR_UNSUPPORTED, "rod_bind: not for a rod inside a vessel");
  if (h->self[outer] || h->self[inner]) return fail(CORDE_ERR_UNSUPPORTED, "rod_bind: not for a self-colliding rod");
  const double* a = &h->derived[16 * (size_t)outer];
  const double* b = &h->derived[16 * (size_t)inner];
  if (h->n_iters[outer] != h->n_iters[inner] || h->n_iters[outer] == 0)
    return fail(CORDE_ERR_ARG, "rod_bind: both rods must be inextensible with the same n_iters");
  if (h->dt[outer] != h->dt[inner]) return fail(CORDE_ERR_ARG, "rod_bind: both rods must share dt");
  if (std::fabs(a[0] - b[0]) > 1e-9 * a[0]) return fail(CORDE_ERR_ARG, "rod_bind: both rods must share l0");
  int e = 0, t = 0;
  if (pair_layout(std::max(h->n_nodes[outer], h->n_nodes[inner]), &e, &t) != CORDE_OK)
    return fail(CORDE_ERR_UNSUPPORTED, "rod_bind: rods of at most 1024 nodes");
  h->pairs.push_back(make_int4(outer, inner, mode, 0));
  h->paired[outer] = h->paired[inner] = 1;
  if (int rc = build_bins(h)) return rc;
  return build_pair_bins(h);
}

// Bins of the adjoint layout: two elements per thread, the smallest power-of-two block
// (>= 32 threads) holding the rod.  Bin.variant is the index of the matching <2, nt> step
// variant, so that rod_rollout and the adjoint's recomputation run the same kernel code.
static int build_adjoint_bins(rod_handle h) {
  if (!h->adj_bins.empty()) return CORDE_OK;
  for (int nt = 32; nt <= kAdjointMaxNodes / 2; nt *= 2) {
    std::vector<int> rods;
    for (int r = 0; r < h->n_rods; ++r) {
      int need = 32;
      while (2 * need < h->n_nodes[r]) need *= 2;
      if (need == nt) rods.push_back(r);
    }
    if (rods.empty()) continue;
    const int v = find_variant(2, nt);
    if (v < 0) return fail(CORDE_ERR_UNSUPPORTED, "no <2, " + std::to_string(nt) + "> step variant");
    Bin b{v, (int)rods.size(), nullptr};
    CK(cudaMalloc(&b.d_work, rods.size() * sizeof(int)));
    CK(cudaMemcpy(b.d_work, rods.data(), rods.size() * sizeof(int), cudaMemcpyHostToDevice));
    h->adj_bins.push_back(b);
  }
  return CORDE_OK;
}

static bool adjoint_capable(rod_handle h) {
  for (int r = 0; r < h->n_rods; ++r)
    if (h->n_nodes[r] > kAdjointMaxNodes) return false;
  return true;
}

int rod_rollout(rod_handle h, int n_steps, int ckpt_every, float* pos_traj, void* stream) {
  if (int rc = check_handle(h)) return rc;
  if (n_steps < 1 || ckpt_every < 1) return fail(CORDE_ERR_ARG, "n_steps and ckpt_every must be >= 1");
  if (!h->pairs.empty()) return fail(CORDE_ERR_UNSUPPORTED, "rod_rollout: bound pairs are not supported");
  for (int r = 0; r < h->n_rods; ++r)
    if (h->self[r]) return fail(CORDE_ERR_UNSUPPORTED, "rod_rollout: not with self-collision");
  float4* traj = nullptr;
  if (pos_traj) {
    const void* dp = nullptr;
    if (!device_accessible(pos_traj, &dp))
      return fail(CORDE_ERR_ARG, "pos_traj must be 16-byte aligned device memory");
    traj = reinterpret_cast<float4*>(const_cast<void*>(dp));
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t E = h->n_elem;
  const int n_seg = (n_steps + ckpt_every - 1) / ckpt_every;
  if (int rc = ensure_capacity(&h->d_ckpt, &h->ckpt_cap, (size_t)n_seg * 4 * E)) return rc;
  const size_t b = (size_t)E * sizeof(float4);
  const bool adj = adjoint_capable(h);
  if (adj)
    if (int rc = build_adjoint_bins(h)) return rc;
  const std::vector<Bin>& bins = adj ? h->adj_bins : h->bins;
  int launches = 0;
  for (int seg = 0; seg < n_seg; ++seg) {
    float4* ck = h->d_ckpt + (size_t)seg * 4 * E;
    CK(cudaMemcpyAsync(ck, h->d_x, b, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(ck + E, h->d_v, b, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(ck + 2 * E, h->d_q, b, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(ck + 3 * E, h->d_o, b, cudaMemcpyDeviceToDevice, s));
    const int t0 = seg * ckpt_every;
    const int cnt = std::min(ckpt_every, n_steps - t0);
    if (int rc = launch_bins(h, bins, cnt, h->d_drive, s, traj ? traj + (size_t)t0 * E : nullptr)) return rc;
    launches += h->last_launches;
  }
  h->last_launches = launches;
  h->ro_steps = n_steps;
  h->ro_every = ckpt_every;
  return CORDE_OK;
}

int rod_adjoint(rod_handle h, const float* dL_dpos_traj, float* dL_dK, float* dL_duhat, float* dL_dvel0,
                float* dL_dpos0, float* dL_dquat0, float* dL_domega0, void* stream) {
  if (int rc = check_handle(h)) return rc;
  if (h->ro_steps < 1) return fail(CORDE_ERR_ARG, "rod_adjoint needs a preceding rod_rollout");
  if (!h->pairs.empty()) return fail(CORDE_ERR_UNSUPPORTED, "rod_adjoint: bound pairs are not supported");
  for (int r = 0; r < h->n_rods; ++r)
    if (h->tube[r] || h->self[r])
      return fail(CORDE_ERR_UNSUPPORTED, "rod_adjoint: contact (vessel or self) is not differentiated");
  for (int r = 0; r < h->n_rods; ++r)
    if (h->n_nodes[r] > kAdjointMaxNodes)
      return fail(CORDE_ERR_UNSUPPORTED, "the adjoint kernel holds rods of at most " +
                                             std::to_string(kAdjointMaxNodes) + " nodes");
  const float* ptrs_in[1] = {dL_dpos_traj};
  float* ptrs_out[6] = {dL_dK, dL_duhat, dL_dvel0, dL_dpos0, dL_dquat0, dL_domega0};
  const void* dev_in = nullptr;
  if (ptrs_in[0] && !device_accessible(ptrs_in[0], &dev_in))
    return fail(CORDE_ERR_ARG, "dL_dpos_traj must be 16-byte aligned device memory");
  float4* dev_out[6];
  for (int k = 0; k < 6; ++k) {
    dev_out[k] = nullptr;
    if (ptrs_out[k]) {
      const void* dp = nullptr;
      if (!device_accessible(ptrs_out[k], &dp)) return fail(CORDE_ERR_ARG, "gradient outputs must be device memory");
      dev_out[k] = reinterpret_cast<float4*>(const_cast<void*>(dp));
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t E = h->n_elem;
  if (int rc = build_adjoint_bins(h)) return rc;
  int dev = 0, smem_max = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  int smem_sm = 0;
  CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  int iters = 0;
  for (int r = 0; r < h->n_rods; ++r) iters = std::max(iters, h->n_iters[r]);
  const int rec_iters = iters > 0 ? iters : 1;
  // record mode per launch when its scratch fits the budget, recompute mode otherwise.
  // Record layout: compact where the launch has more rods than the GPU has SMs (blocks
  // share SMs, throughput and so the records' memory traffic decide), full otherwise (each
  // rod's latency decides, and rebuilding the even half-sweeps' inputs lengthens it), or
  // compact when only that fits.  Two sweep buffers in shared memory (the copy of a step's
  // records overlaps the reverse of the step after it), or one when two do not fit or when
  // one lets the launch run in fewer waves (more resident blocks per SM).
  const size_t K = (size_t)h->ro_every;
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  std::vector<int> mode(h->adj_bins.size(), 0);
  std::vector<char> compact(h->adj_bins.size(), 0);
  std::vector<char> pipe(h->adj_bins.size(), 0);
  size_t sweep_need = 0;
  for (size_t i = 0; i < h->adj_bins.size(); ++i) {
    const Bin& b = h->adj_bins[i];
    const int nt = variants()[b.variant].nt;
    const bool prefer_compact = b.count > sms;
    for (int pass = 0; pass < 2 && mode[i] == 0; ++pass) {
      const bool cpt = pass == 0 ? prefer_compact : true;
      if (pass == 1 && prefer_compact) break;
      // float4 entries: 12 B per node and slot
      const size_t sw = K * b.count * (cpt ? rec_iters + 1 : 2 * rec_iters) * 3 * 2 * nt / 4;
      if ((long long)(sw * sizeof(float4)) > h->adj_record_budget) continue;
      const int smem1 = adjoint_smem_bytes(nt, iters, 1, cpt), smem2 = adjoint_smem_bytes(nt, iters, 2, cpt);
      if (smem1 > smem_max) continue;
      int m = 1;
      if (smem2 <= smem_max) {
        int occ1 = 0, occ2 = 0;
        CK(adjoint_occupancy(nt, 1, cpt, smem1, &occ1));
        CK(adjoint_occupancy(nt, 2, cpt, smem2, &occ2));
        auto waves = [&](int occ) { return occ > 0 ? (b.count + occ * sms - 1) / (occ * sms) : INT_MAX; };
        m = waves(occ2) <= waves(occ1) ? 2 : 1;
      }
      mode[i] = m;
      compact[i] = cpt;
      sweep_need = std::max(sweep_need, sw);
    }
    // recompute mode keeps the step's records in shared memory only: the full layout
    // unless only the compact one fits the block
    if (mode[i] == 0) compact[i] = adjoint_smem_bytes(nt, iters, 0, false) > smem_max;
    // a rod's reverse pipelined over two SMs (a cluster of two blocks: one records the
    // segments, the other reverses them one segment behind) when every rod of the launch
    // gets its own two SMs and the doubled scratch fits the budget
    if (h->adj_pipe && mode[i] == 2 && !compact[i] && 2 * b.count <= sms) {
      const size_t sw = K * b.count * (2 * rec_iters) * 3 * 2 * nt / 4;
      if ((long long)(2 * sw * sizeof(float4)) <= h->adj_record_budget) {
        pipe[i] = 1;
        sweep_need = std::max(sweep_need, 2 * sw);
      }
    }
  }
  const bool any_record = sweep_need > 0;
  const bool any_pipe = std::find(pipe.begin(), pipe.end(), 1) != pipe.end();
  if (int rc = ensure_capacity(&h->d_seg, &h->seg_cap, (K + (any_record ? 1 : 0)) * (any_pipe ? 2 : 1) * 4 * E))
    return rc;
  if (any_record) {
    if (int rc = ensure_capacity(&h->d_sweep_rec, &h->sweep_rec_cap, sweep_need)) return rc;
  }
  AdjointArgs a;
  a.rods = h->d_rods;
  a.ckpt = h->d_ckpt;
  a.seg_states = h->d_seg;
  a.u4 = h->d_u;
  a.k4 = h->d_k;
  a.drive = h->d_drive;
  a.dLdpos = reinterpret_cast<const float4*>(dev_in);
  a.n_steps = h->ro_steps;
  a.ckpt_every = h->ro_every;
  a.n_elem = E;
  a.dK = dev_out[0];
  a.duhat = dev_out[1];
  a.dvel0 = dev_out[2];
  a.dpos0 = dev_out[3];
  a.dquat0 = dev_out[4];
  a.domega0 = dev_out[5];
  int launches = 0;
  std::fill(h->adj_info, h->adj_info + 7, 0);
  for (size_t i = 0; i < h->adj_bins.size(); ++i) {
    const Bin& b = h->adj_bins[i];
    const int nt = variants()[b.variant].nt;
    int smem = adjoint_smem_bytes(nt, iters, mode[i], compact[i] != 0);
    // pipelined: shared memory of more than half an SM keeps the cluster's two blocks on
    // two SMs
    if (pipe[i]) smem = std::min(smem_max, std::max(smem, smem_sm / 2));
    a.sweep_rec = mode[i] ? h->d_sweep_rec : nullptr;
    a.rec_iters = rec_iters;
    if (smem > smem_max)
      return fail(CORDE_ERR_UNSUPPORTED, "adjoint needs " + std::to_string(smem) + " B of shared memory per block; " +
                                             std::to_string(smem_max) + " available (fewer constraint iterations " +
                                             "or shorter rods)");
    a.work = b.d_work;
    const int n_blocks = pipe[i] ? 2 * b.count : b.count;
    if (n_blocks >= h->adj_info[3]) {
      int per_sm = 1;
      if (!pipe[i]) CK(adjoint_occupancy(nt, mode[i], compact[i] != 0, smem, &per_sm));
      const int info[7] = {mode[i], nt, per_sm, n_blocks, sms, compact[i] ? 1 : 0, pipe[i] ? 1 : 0};
      std::copy(info, info + 7, h->adj_info);
    }
    cudaError_t e = pipe[i] ? launch_adjoint_pipe(nt, a, b.count, smem, s)
                            : launch_adjoint(nt, mode[i], compact[i] != 0, a, b.count, smem, s);
    if (e != cudaSuccess) return fail(CORDE_ERR_CUDA, std::string("adjoint launch: ") + cudaGetErrorString(e));
    ++launches;
  }
  h->last_launches = launches;
  return CORDE_OK;
}

int rod_adjoint_info(rod_handle h, int* out) {
  if (!h || !out) return fail(CORDE_ERR_ARG, "rod_adjoint_info: NULL argument");
  std::copy(h->adj_info, h->adj_info + 7, out);
  return CORDE_OK;
}

static void mailbox_free(rod_handle h) {
  if (h->mb_in_host) cudaFreeHost(h->mb_in_host);
  if (h->mb_out_host) cudaFreeHost(h->mb_out_host);
  if (h->mb_pos_host) cudaFreeHost(h->mb_pos_host);
  h->mb_pos_host = nullptr;
  cudaFree(h->mb_dev.log);
  cudaFree(h->mb_dev.log_count);
  h->mb_in_host = h->mb_out_host = nullptr;
  h->mb_dev = MailboxDev{};
  h->mb_period = 0;
}

int rod_mailbox_enable(rod_handle h, int period, int log_capacity) {
  if (int rc = check_handle(h)) return rc;
  if (period < 1 || log_capacity < 1) return fail(CORDE_ERR_ARG, "rod_mailbox_enable: period and log_capacity >= 1");
  for (int r = 0; r < h->n_rods; ++r)
    if (h->self[r]) return fail(CORDE_ERR_UNSUPPORTED, "rod_mailbox_enable: not with self-collision");
  for (int r = 0; r < h->n_rods; ++r)
    if (h->plan_grid[r]) return fail(CORDE_ERR_UNSUPPORTED, "rod_mailbox_enable: not with a rod on a cooperative grid");
  CK(cudaDeviceSynchronize());
  mailbox_free(h);
  const size_t in_bytes = 16 + (size_t)h->n_rods * 8 * sizeof(float);
  const size_t out_bytes = (size_t)h->n_rods * 16 * sizeof(unsigned) + 16;  // records, then the status word
  CK(cudaHostAlloc(&h->mb_in_host, in_bytes, cudaHostAllocMapped | cudaHostAllocPortable));
  CK(cudaHostAlloc(&h->mb_out_host, out_bytes, cudaHostAllocMapped | cudaHostAllocPortable));
  std::memset(h->mb_in_host, 0, in_bytes);
  std::memset(h->mb_out_host, 0, out_bytes);
  void *din = nullptr, *dout = nullptr;
  CK(cudaHostGetDevicePointer(&din, h->mb_in_host, 0));
  CK(cudaHostGetDevicePointer(&dout, h->mb_out_host, 0));
  h->mb_dev.in_seq = reinterpret_cast<const unsigned*>(din);
  h->mb_dev.in_drive = reinterpret_cast<const float*>(static_cast<char*>(din) + 16);
  h->mb_dev.out = reinterpret_cast<unsigned*>(dout);
  h->mb_dev.status = reinterpret_cast<unsigned*>(dout) + (size_t)h->n_rods * 16;
  CK(cudaMalloc(&h->mb_dev.log, (size_t)log_capacity * sizeof(int2)));
  CK(cudaMalloc(&h->mb_dev.log_count, sizeof(int)));
  CK(cudaMemset(h->mb_dev.log_count, 0, sizeof(int)));
  h->mb_dev.log_cap = log_capacity;
  h->mb_dev.period = period;
  h->mb_period = period;
  h->mb_host_seq = 0;
  invalidate_graph(h);
  return CORDE_OK;
}

int rod_mailbox_lockstep(rod_handle h, int enable, int timeout_us) {
  if (int rc = check_handle(h)) return rc;
  if (h->mb_period <= 0) return fail(CORDE_ERR_ARG, "rod_mailbox_lockstep: mailbox not enabled");
  if (enable && timeout_us < 1) return fail(CORDE_ERR_ARG, "rod_mailbox_lockstep: timeout_us >= 1");
  CK(cudaDeviceSynchronize());
  h->mb_dev.lockstep = enable ? 1 : 0;
  h->mb_dev.wait_ns = enable ? (unsigned long long)timeout_us * 1000ull : 0ull;
  return CORDE_OK;
}

int rod_mailbox_status(rod_handle h, unsigned* status) {
  if (!h || !status) return fail(CORDE_ERR_ARG, "rod_mailbox_status: NULL argument");
  if (h->mb_period <= 0) return fail(CORDE_ERR_ARG, "rod_mailbox_status: mailbox not enabled");
  unsigned* st = static_cast<unsigned*>(h->mb_out_host) + (size_t)h->n_rods * 16;
  *status = __atomic_exchange_n(st, 0u, __ATOMIC_ACQ_REL);
  return CORDE_OK;
}

int rod_mailbox_positions_enable(rod_handle h, int enable) {
  if (int rc = check_handle(h)) return rc;
  if (h->mb_period <= 0) return fail(CORDE_ERR_ARG, "rod_mailbox_positions_enable: mailbox not enabled");
  CK(cudaDeviceSynchronize());
  if (h->mb_pos_host) cudaFreeHost(h->mb_pos_host);
  h->mb_pos_host = nullptr;
  h->mb_dev.pos_seq = nullptr;
  h->mb_dev.pos = nullptr;
  if (!enable) return CORDE_OK;
  const size_t hdr = (size_t)h->n_rods * 32 * sizeof(unsigned);
  const size_t bytes = hdr + (size_t)kPosSlots * h->n_elem * sizeof(float4);
  CK(cudaHostAlloc(&h->mb_pos_host, bytes, cudaHostAllocMapped | cudaHostAllocPortable));
  std::memset(h->mb_pos_host, 0, bytes);
  void* d = nullptr;
  CK(cudaHostGetDevicePointer(&d, h->mb_pos_host, 0));
  h->mb_dev.pos_seq = reinterpret_cast<unsigned*>(d);
  h->mb_dev.pos = reinterpret_cast<float4*>(static_cast<char*>(d) + hdr);
  h->mb_dev.n_elem = h->n_elem;
  return CORDE_OK;
}

int rod_mailbox_positions(rod_handle h, int rod, float* out, long long* step) {
  if (!h || !step) return fail(CORDE_ERR_ARG, "rod_mailbox_positions: NULL argument");
  if (!h->mb_pos_host) return fail(CORDE_ERR_ARG, "rod_mailbox_positions: position snapshots not enabled");
  if (rod < 0 || rod >= h->n_rods) return fail(CORDE_ERR_ARG, "rod_mailbox_positions: bad rod");
  const unsigned* hdr = static_cast<const unsigned*>(h->mb_pos_host) + 32 * (size_t)rod;
  const size_t hbytes = (size_t)h->n_rods * 32 * sizeof(unsigned);
  const size_t nf = 4 * (size_t)h->n_nodes[rod];
  for (int attempt = 0; attempt < 10000; ++attempt) {
    // the newest publication p (count p + 1) lives in slot p % kPosSlots; the kernel
    // rewrites that slot only after count p + kPosSlots is visible, so the copy is whole
    // if the count, read again after it, has not reached p + kPosSlots
    const unsigned pubs = __atomic_load_n(&hdr[0], __ATOMIC_ACQUIRE);
    if (pubs == 0u) {
      *step = -1;
      return CORDE_OK;
    }
    const unsigned p = pubs - 1u;
    const unsigned* sh = hdr + 4 + 4 * (p % kPosSlots);
    const unsigned lo = __atomic_load_n(&sh[1], __ATOMIC_RELAXED), hi = __atomic_load_n(&sh[2], __ATOMIC_RELAXED);
    const float* src = reinterpret_cast<const float*>(static_cast<const char*>(h->mb_pos_host) + hbytes) +
                       4 * ((size_t)(p % kPosSlots) * h->n_elem + h->off[rod]);
    if (out) std::memcpy(out, src, nf * sizeof(float));  // out NULL: the step only
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
    if (__atomic_load_n(&hdr[0], __ATOMIC_RELAXED) - pubs <= (unsigned)(kPosSlots - 2)) {
      *step = (long long)(((unsigned long long)hi << 32) | lo);
      return CORDE_OK;
    }
  }
  return fail(CORDE_ERR_BUSY, "rod_mailbox_positions: no consistent snapshot after 10000 attempts");
}

constexpr long long kExchangePollNs = 300;  // host poll interval of the snapshot waits

// Spins until rod `rod`'s newest position snapshot was taken after a global step >=
// target_step, polling only the rod's publication count and that slot's step.
static int await_snapshot(rod_handle h, int rod, long long target_step, long long timeout_us, const char* who) {
  const unsigned* hdr = static_cast<const unsigned*>(h->mb_pos_host) + 32 * (size_t)rod;
  const unsigned* status = static_cast<const unsigned*>(h->mb_out_host) + (size_t)h->n_rods * 16;
  const auto t0 = std::chrono::steady_clock::now();
  for (unsigned long long k = 0;; ++k) {
    const unsigned pubs = __atomic_load_n(&hdr[0], __ATOMIC_ACQUIRE);
    if (pubs > 0u) {
      const unsigned p = pubs - 1u;
      const unsigned* sh = hdr + 4 + 4 * (p % kPosSlots);
      const unsigned lo = __atomic_load_n(&sh[1], __ATOMIC_RELAXED), hi = __atomic_load_n(&sh[2], __ATOMIC_RELAXED);
      if ((long long)(((unsigned long long)hi << 32) | lo) >= target_step) return CORDE_OK;
    }
    if ((k & 63u) == 63u) {
      if (__atomic_load_n(status, __ATOMIC_ACQUIRE) != 0u)
        return fail(CORDE_ERR_BUSY, std::string(who) + ": a lock-step wait of the kernel ran out");
      const long long us =
          std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
      if (us > timeout_us) return fail(CORDE_ERR_BUSY, std::string(who) + ": no snapshot of the target step in time");
    }
    // back off between polls without touching the shared lines
    const auto tp = std::chrono::steady_clock::now();
    while (std::chrono::steady_clock::now() - tp < std::chrono::nanoseconds(kExchangePollNs)) {
    }
  }
}

static int check_snapshot_call(rod_handle h, int rod, long long timeout_us, const void* step, const char* who) {
  if (!h || !step) return fail(CORDE_ERR_ARG, std::string(who) + ": NULL argument");
  if (!h->mb_pos_host) return fail(CORDE_ERR_ARG, std::string(who) + ": position snapshots not enabled");
  if (rod < 0 || rod >= h->n_rods) return fail(CORDE_ERR_ARG, std::string(who) + ": bad rod");
  if (timeout_us < 0) return fail(CORDE_ERR_ARG, std::string(who) + ": timeout_us must be >= 0");
  return CORDE_OK;
}

int rod_mailbox_exchange(rod_handle h, const float* drive, int rod, long long target_step, float* out,
                         long long timeout_us, long long* step) {
  if (!out) return fail(CORDE_ERR_ARG, "rod_mailbox_exchange: NULL argument");
  if (int rc = check_snapshot_call(h, rod, timeout_us, step, "rod_mailbox_exchange")) return rc;
  if (drive)
    if (int rc = rod_mailbox_write(h, drive)) return rc;
  if (int rc = await_snapshot(h, rod, target_step, timeout_us, "rod_mailbox_exchange")) return rc;
  return rod_mailbox_positions(h, rod, out, step);
}

int rod_mailbox_tick(rod_handle h, int rod, long long target_step, const float* next_drive, float* out,
                     long long timeout_us, long long* step) {
  if (int rc = check_snapshot_call(h, rod, timeout_us, step, "rod_mailbox_tick")) return rc;
  if (int rc = await_snapshot(h, rod, target_step, timeout_us, "rod_mailbox_tick")) return rc;
  // the next drive goes out before the copy, so the kernel steps while the host copies
  if (next_drive)
    if (int rc = rod_mailbox_write(h, next_drive)) return rc;
  return rod_mailbox_positions(h, rod, out, step);
}

int rod_mailbox_disable(rod_handle h) {
  if (int rc = check_handle(h)) return rc;
  CK(cudaDeviceSynchronize());
  mailbox_free(h);
  return CORDE_OK;
}

int rod_mailbox_write(rod_handle h, const float* drive) {
  if (!h || !drive) return fail(CORDE_ERR_ARG, "rod_mailbox_write: NULL argument");
  if (h->mb_period <= 0) return fail(CORDE_ERR_ARG, "rod_mailbox_write: mailbox not enabled");
  unsigned* seq = static_cast<unsigned*>(h->mb_in_host);
  unsigned* payload = reinterpret_cast<unsigned*>(static_cast<char*>(h->mb_in_host) + 16);
  const unsigned s0 = h->mb_host_seq;
  __atomic_store_n(seq, s0 + 1u, __ATOMIC_RELAXED);  // odd: the payload is being written
  __atomic_thread_fence(__ATOMIC_SEQ_CST);
  for (int k = 0; k < h->n_rods * 8; ++k) {
    unsigned bits;
    std::memcpy(&bits, &drive[k], sizeof(bits));
    __atomic_store_n(&payload[k], bits, __ATOMIC_RELAXED);
  }
  __atomic_thread_fence(__ATOMIC_SEQ_CST);
  __atomic_store_n(seq, s0 + 2u, __ATOMIC_RELEASE);
  h->mb_host_seq = s0 + 2u;
  return CORDE_OK;
}

int rod_mailbox_read(rod_handle h, unsigned* out) {
  if (!h || !out) return fail(CORDE_ERR_ARG, "rod_mailbox_read: NULL argument");
  if (h->mb_period <= 0) return fail(CORDE_ERR_ARG, "rod_mailbox_read: mailbox not enabled");
  const unsigned* rec = static_cast<const unsigned*>(h->mb_out_host);
  for (int k = 0; k < 2 * h->n_rods; ++k) {
    const unsigned* r = rec + 8 * k;
    unsigned* o = out + 8 * k;
    bool ok = false;
    for (int attempt = 0; attempt < 10000 && !ok; ++attempt) {
      const unsigned s1 = __atomic_load_n(&r[0], __ATOMIC_ACQUIRE);
      if (s1 & 1u) continue;
      for (int j = 1; j < 8; ++j) o[j] = __atomic_load_n(&r[j], __ATOMIC_RELAXED);
      __atomic_thread_fence(__ATOMIC_SEQ_CST);
      const unsigned s2 = __atomic_load_n(&r[0], __ATOMIC_RELAXED);
      if (s1 == s2) {
        o[0] = s1;
        ok = true;
      }
    }
    if (!ok) return fail(CORDE_ERR_CUDA, "rod_mailbox_read: no consistent record after 10000 attempts");
  }
  return CORDE_OK;
}

int rod_mailbox_log(rod_handle h, int* out, int capacity, int* count) {
  if (int rc = check_handle(h)) return rc;
  if (!count || (capacity > 0 && !out)) return fail(CORDE_ERR_ARG, "rod_mailbox_log: NULL argument");
  if (h->mb_period <= 0) return fail(CORDE_ERR_ARG, "rod_mailbox_log: mailbox not enabled");
  CK(cudaDeviceSynchronize());
  int n = 0;
  CK(cudaMemcpy(&n, h->mb_dev.log_count, sizeof(int), cudaMemcpyDeviceToHost));
  *count = n;
  const int m = std::min(std::min(n, capacity), h->mb_dev.log_cap);
  if (m > 0) CK(cudaMemcpy(out, h->mb_dev.log, (size_t)m * sizeof(int2), cudaMemcpyDeviceToHost));
  CK(cudaMemset(h->mb_dev.log_count, 0, sizeof(int)));
  return CORDE_OK;
}

int64_t rod_steps_done(rod_handle h) { return h ? h->steps_done : -1; }

void rod_destroy(rod_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  free_bins(h);
  cudaFree(h->d_rods); cudaFree(h->d_derived);
  cudaFree(h->d_x); cudaFree(h->d_v); cudaFree(h->d_q); cudaFree(h->d_o); cudaFree(h->d_u); cudaFree(h->d_k);
  cudaFree(h->d_drive); cudaFree(h->d_elem_rod); cudaFree(h->d_drive_graph);
  cudaFree(h->d_ckpt); cudaFree(h->d_seg); cudaFree(h->d_self_stats); cudaFree(h->d_self_skin);
  cudaFree(h->d_sweep_rec);
  for (auto& b : h->adj_bins) cudaFree(b.d_work);
  for (auto& pb : h->pair_bins) cudaFree(pb.d_pairs);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  for (auto st : h->side) cudaStreamDestroy(st);
  for (auto ev : h->join_ev) cudaEventDestroy(ev);
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  mailbox_free(h);
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Gradient entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc at the point where they need a gradient: a haptic or
// control loop running under a real-time budget (an allocation can stall for milliseconds
// and may synchronise the device), an application whose device memory is owned by its own
// pool or arena, or code that must not change the process's allocation state.  For them,
// rod_adjoint_noalloc runs the recorded rollout and the reverse pass of one rod with every
// intermediate (derived constants, packed state, checkpoints, per-segment states) in the
// file-scope array below, which is part of the library image: every GPU that loads the
// library holds these 16 MiB until the process exits.  The caller passes inputs and
// outputs as device memory.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
constexpr int kMaxDevices = 64;
// Device address of the array, per device; set once, by the first call on that device.
std::atomic<void*> g_noalloc_base[kMaxDevices];
std::mutex g_noalloc_init_mutex;

__global__ void noalloc_setup_kernel(RodParams p, int n, RodParams* P, int* off, int* work, int* elem_rod,
                                     const float* drive_in, float4* drive) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *P = p;
    off[0] = 0;
    work[0] = 0;
    drive[0] = drive_in ? make_float4(drive_in[0], drive_in[1], drive_in[2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    drive[1] = drive_in ? make_float4(drive_in[4], drive_in[5], drive_in[6], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (i < n) elem_rod[i] = 0;
}

bool device_readable(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int rod_adjoint_noalloc(const RodParams* params, const float* pos, const float* quat,
                                   const float* rest_quat, const float* vel, const float* omega,
                                   const float* stiff_mul, const float* drive, int n_steps, int ckpt_every,
                                   const float* dL_dpos_traj, float* pos_traj, float* dL_dK, float* dL_duhat,
                                   float* dL_dvel0, float* dL_dpos0, void* stream) {
  if (!params || !pos || !quat) return fail(CORDE_ERR_ARG, "rod_adjoint_noalloc: need params, pos and quat");
  std::string why;
  if (!params_valid(*params, why)) return fail(CORDE_ERR_ARG, "rod_adjoint_noalloc: " + why);
  const int N = params->n_nodes;
  if (N > kAdjointMaxNodes)
    return fail(CORDE_ERR_ARG, "rod_adjoint_noalloc: at most " + std::to_string(kAdjointMaxNodes) + " nodes");
  if (n_steps < 1 || ckpt_every < 1) return fail(CORDE_ERR_ARG, "rod_adjoint_noalloc: n_steps, ckpt_every >= 1");
  const float* ins[7] = {pos, quat, rest_quat, vel, omega, stiff_mul, drive};
  for (const float* p : ins)
    if (p && !device_readable(p)) return fail(CORDE_ERR_ARG, "rod_adjoint_noalloc: inputs must be device memory");
  const void* dev_traj_in = nullptr;
  if (dL_dpos_traj && !device_accessible(dL_dpos_traj, &dev_traj_in))
    return fail(CORDE_ERR_ARG, "rod_adjoint_noalloc: dL_dpos_traj must be 16-byte aligned device memory");
  float* outs[5] = {pos_traj, dL_dK, dL_duhat, dL_dvel0, dL_dpos0};
  float4* dev_out[5];
  for (int k = 0; k < 5; ++k) {
    dev_out[k] = nullptr;
    if (outs[k]) {
      const void* dp = nullptr;
      if (!device_accessible(outs[k], &dp))
        return fail(CORDE_ERR_ARG, "rod_adjoint_noalloc: outputs must be 16-byte aligned device memory");
      dev_out[k] = reinterpret_cast<float4*>(const_cast<void*>(dp));
    }
  }

  // scratch layout
  const int n_seg = (n_steps + ckpt_every - 1) / ckpt_every;
  const int K = std::min(ckpt_every, n_steps);
  size_t o = 0;
  const size_t o_P = o; o = align256(o + sizeof(RodParams));
  const size_t o_off = o; o = align256(o + sizeof(int));
  const size_t o_work = o; o = align256(o + sizeof(int));
  const size_t o_der = o; o = align256(o + 16 * sizeof(double));
  const size_t o_rod = o; o = align256(o + sizeof(RodDev));
  const size_t o_drv = o; o = align256(o + 2 * sizeof(float4));
  const size_t o_er = o; o = align256(o + (size_t)N * sizeof(int));
  const size_t o_state = o; o = align256(o + 6 * (size_t)N * sizeof(float4));
  const size_t o_ckpt = o; o = align256(o + (size_t)n_seg * 4 * N * sizeof(float4));
  const size_t o_seg = o; o = align256(o + (size_t)K * 4 * N * sizeof(float4));
  if (o > kNoAllocScratchBytes)
    return fail(CORDE_ERR_ARG, "rod_adjoint_noalloc: needs " + std::to_string(o) + " bytes of scratch, above the " +
                                   std::to_string(kNoAllocScratchBytes) +
                                   "-byte static limit (fewer steps, a smaller ckpt_every or a shorter rod)");

  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(CORDE_ERR_UNSUPPORTED, "rod_adjoint_noalloc: device index");
  void* base_addr = g_noalloc_base[dev].load(std::memory_order_acquire);
  if (!base_addr) {
    // First call on this device: look up the array's device address, and load every
    // kernel this entry point can launch, so that no later call loads a module (with
    // lazy module loading, the CUDA default, a kernel's first launch would otherwise
    // load it, which takes device memory and can block).
    std::lock_guard<std::mutex> lock(g_noalloc_init_mutex);
    base_addr = g_noalloc_base[dev].load(std::memory_order_acquire);
    if (!base_addr) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return fail(CORDE_ERR_CUDA, std::string("rod_adjoint_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      cudaFuncAttributes at;
      e = cudaFuncGetAttributes(&at, noalloc_setup_kernel);
      if (e == cudaSuccess) e = cudaFuncGetAttributes(&at, derive_kernel);
      if (e == cudaSuccess) e = cudaFuncGetAttributes(&at, pack_kernel);
      for (int nt = 32; e == cudaSuccess && nt <= 256; nt *= 2) {
        const int v = find_variant(2, nt);
        e = v < 0 ? cudaErrorInvalidValue : variants()[v].preload();
        if (e == cudaSuccess) e = preload_adjoint(nt);
      }
      if (e != cudaSuccess)
        return fail(CORDE_ERR_CUDA, std::string("rod_adjoint_noalloc: loading kernels: ") + cudaGetErrorString(e));
      g_noalloc_base[dev].store(p, std::memory_order_release);
      base_addr = p;
    }
  }
  unsigned char* base = static_cast<unsigned char*>(base_addr);
  RodParams* d_P = reinterpret_cast<RodParams*>(base + o_P);
  int* d_off = reinterpret_cast<int*>(base + o_off);
  int* d_work = reinterpret_cast<int*>(base + o_work);
  double* d_der = reinterpret_cast<double*>(base + o_der);
  RodDev* d_rod = reinterpret_cast<RodDev*>(base + o_rod);
  float4* d_drv = reinterpret_cast<float4*>(base + o_drv);
  int* d_er = reinterpret_cast<int*>(base + o_er);
  float4* st = reinterpret_cast<float4*>(base + o_state);
  float4 *x4 = st, *v4 = st + N, *q4 = st + 2 * N, *o4 = st + 3 * N, *u4 = st + 4 * N, *k4 = st + 5 * N;
  float4* ckpt = reinterpret_cast<float4*>(base + o_ckpt);
  float4* seg = reinterpret_cast<float4*>(base + o_seg);
  cudaStream_t s = (cudaStream_t)stream;

  noalloc_setup_kernel<<<(N + 255) / 256, 256, 0, s>>>(*params, N, d_P, d_off, d_work, d_er, drive, d_drv);
  derive_kernel<<<1, 32, 0, s>>>(1, d_P, d_off, d_rod, d_der);
  pack_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, d_er, d_rod, d_P, d_der, pos, quat, rest_quat, vel, omega, stiff_mul,
                                               x4, v4, q4, o4, u4, k4);
  CK(cudaGetLastError());

  // forward rollout in the adjoint's layout: two elements per thread
  int nt = 32;
  while (2 * nt < N) nt *= 2;
  const int v = find_variant(2, nt);
  if (v < 0) return fail(CORDE_ERR_UNSUPPORTED, "rod_adjoint_noalloc: no step variant");
  StepArgs a = {};
  // ordinary launches: a device-to-device copy of the checkpoint sits between
  // consecutive step launches, so overlapped launch would change nothing here
  a.pdl = 0;
  a.rods = d_rod;
  a.work = d_work;
  a.x4 = x4;
  a.v4 = v4;
  a.q4 = q4;
  a.o4 = o4;
  a.u4 = u4;
  a.k4 = k4;
  a.drive = d_drv;
  a.n_elem = N;
  const size_t b = (size_t)N * sizeof(float4);
  for (int sg = 0; sg < n_seg; ++sg) {
    float4* ck = ckpt + (size_t)sg * 4 * N;
    CK(cudaMemcpyAsync(ck, x4, b, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(ck + N, v4, b, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(ck + 2 * N, q4, b, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(ck + 3 * N, o4, b, cudaMemcpyDeviceToDevice, s));
    const int t0 = sg * ckpt_every;
    a.n_steps = std::min(ckpt_every, n_steps - t0);
    a.traj = dev_out[0] ? dev_out[0] + (size_t)t0 * N : nullptr;
    cudaError_t e = variants()[v].launch(a, 1, s);
    if (e != cudaSuccess) return fail(CORDE_ERR_CUDA, std::string("rod_adjoint_noalloc: step: ") + cudaGetErrorString(e));
  }

  // reverse pass
  const int iters = params->inextensible ? params->n_iters : 0;
  int smem_max = 0;
  CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // the compact record layout where the full one does not fit the block
  const bool cpt = adjoint_smem_bytes(nt, iters, 0, false) > smem_max;
  const int smem = adjoint_smem_bytes(nt, iters, 0, cpt);
  if (smem > smem_max) return fail(CORDE_ERR_UNSUPPORTED, "rod_adjoint_noalloc: shared memory");
  AdjointArgs ad;
  ad.rods = d_rod;
  ad.work = d_work;
  ad.ckpt = ckpt;
  ad.seg_states = seg;
  ad.u4 = u4;
  ad.k4 = k4;
  ad.drive = d_drv;
  ad.dLdpos = reinterpret_cast<const float4*>(dev_traj_in);
  ad.n_steps = n_steps;
  ad.ckpt_every = ckpt_every;
  ad.n_elem = N;
  ad.dK = dev_out[1];
  ad.duhat = dev_out[2];
  ad.dvel0 = dev_out[3];
  ad.dpos0 = dev_out[4];
  ad.dquat0 = nullptr;
  ad.domega0 = nullptr;
  cudaError_t e = launch_adjoint(nt, 0, cpt, ad, 1, smem, s);
  if (e != cudaSuccess) return fail(CORDE_ERR_CUDA, std::string("rod_adjoint_noalloc: adjoint: ") + cudaGetErrorString(e));
  return CORDE_OK;
}
