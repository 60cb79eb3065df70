// FP64 CPU oracle of the CoRdE Cosserat-rod time step and its inextensible variant.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
// baseline may load this library.  It shares no code with the CUDA path.
//
// It is deliberately plain: serial loops over nodes, frames and constraints in the
// order the paper states them, double precision, no blocking, fusion or reordering.
// Every function is templated on the scalar type T so that the same code runs with
//   * double  - the oracle proper,
//   * Dual    - forward-mode derivatives (dual numbers, value + one tangent), used to
//               produce exact directional derivatives of rollouts for gradient checks,
//   * Counted - a double that counts floating-point operations (algorithmic work).
//
// Paper sections followed (Korzeniowski, Hald, Bello, "Massively-Parallel
// Implementation of Inextensible Elastic Rods Using Inter-block GPU Synchronization"):
//   Section 2.1, "Cosserat Rod": centreline r_i (N points), N-1 frames as unit
//     quaternions q_j; tangent Eq. 4; stretch energy Eq. 2; bend/twist energy Eq. 3;
//     Darboux vector from adjacent quaternions Eq. 5-6 (Eq. 1 in the continuum);
//     parallel-constraint penalty Eq. 7-8; internal friction as dissipation.
//   Section 2.1, "Constraints": inextensibility as distance constraints solved locally
//     and iteratively by impulses (J M^-1 J^T projection); binding constraints are
//     distance constraints of rest length zero.
//   Section 2.1 (end) and Fig. 5: per time step - external forces and torques; elastic
//     forces and torques by differentiating the energies; force integration (points as
//     particles, quaternions as rigid-body orientations); j iterations of constraint
//     impulses; integration of linear and angular velocity (semi-implicit Euler).
//
// Readings where the paper is silent or garbled (each one a documented design reading):
//   * Eq. 3 prints K1 = K2 = E pi r^2/4 and K3 = G pi r^2/2; bending and torsional
//     stiffness need the second moments, so K1 = K2 = E pi r^4/4, K3 = G pi r^4/2.
//   * B_k of Eq. 6 (given only in the paper's reference [17]) are chosen so that
//     2 (B_k q_j) . q'_j = (2/l_j) Im(conj(q_j) q_{j+1})_k, the discrete body-frame
//     Darboux vector; with skew-symmetric B_k, q_j and the midpoint give the same u.
//   * Masses m_i = rho A (l0_{i-1} + l0_i)/2, frame inertia rho l0 diag(I, I, 2I); the
//     inertial (not gravitational) masses and inertias are scaled so that the
//     explicit step stays stable (default rule in derive()).
//   * Internal friction is mass-proportional Rayleigh damping, applied implicitly.
//   * Constraint impulses are predictive (they make C(r + dt v) = 0 per constraint),
//     swept red-black: even segments, then odd segments, per iteration.
//   * "Clamped" / driven base: node 0 and frame 0 are kinematic (inverse mass 0); their
//     velocities come from the drive input.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

// ------------------------------------------------------------------ scalar types

struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
static inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
static inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
static inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
static inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
static inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
static inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
static inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
static inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
static inline double val(double x) { return x; }
static inline double val(Dual x) { return x.v; }

// Operation counter: every +, -, *, / and sqrt on a Counted value is one operation.
static uint64_t g_flops = 0;
struct Counted {
  double v;
  Counted() : v(0) {}
  Counted(double x) : v(x) {}
};
static inline Counted operator+(Counted a, Counted b) { ++g_flops; return Counted(a.v + b.v); }
static inline Counted operator-(Counted a, Counted b) { ++g_flops; return Counted(a.v - b.v); }
static inline Counted operator-(Counted a) { return Counted(-a.v); }
static inline Counted operator*(Counted a, Counted b) { ++g_flops; return Counted(a.v * b.v); }
static inline Counted operator/(Counted a, Counted b) { ++g_flops; return Counted(a.v / b.v); }
static inline Counted& operator+=(Counted& a, Counted b) { a = a + b; return a; }
static inline Counted& operator-=(Counted& a, Counted b) { a = a - b; return a; }
static inline Counted sqrt(Counted a) { ++g_flops; return Counted(std::sqrt(a.v)); }
static inline double val(Counted x) { return x.v; }

// ------------------------------------------------------------------ small vector algebra

template <class T> struct V3 { T x, y, z; };
template <class T> struct Q4 { T w, x, y, z; };  // Hamilton quaternion, w real part

template <class T> static inline V3<T> v3(T x, T y, T z) { return V3<T>{x, y, z}; }
template <class T> static inline V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> static inline V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T, class S> static inline V3<T> operator*(S s, V3<T> a) { return {T(s) * a.x, T(s) * a.y, T(s) * a.z}; }
template <class T> static inline T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> static inline V3<T> cross(V3<T> a, V3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T> static inline T norm(V3<T> a) { return sqrt(dot(a, a)); }

template <class T> static inline Q4<T> qadd(Q4<T> a, Q4<T> b) { return {a.w + b.w, a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> static inline Q4<T> qsub(Q4<T> a, Q4<T> b) { return {a.w - b.w, a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T, class S> static inline Q4<T> qscale(S s, Q4<T> a) { return {T(s) * a.w, T(s) * a.x, T(s) * a.y, T(s) * a.z}; }
template <class T> static inline T qdot(Q4<T> a, Q4<T> b) { return a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> static inline Q4<T> qconj(Q4<T> a) { return {a.w, -a.x, -a.y, -a.z}; }
// Hamilton product a (x) b.
template <class T> static inline Q4<T> qmul(Q4<T> a, Q4<T> b) {
  return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
          a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
          a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
          a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
template <class T> static inline V3<T> qim(Q4<T> a) { return {a.x, a.y, a.z}; }
template <class T> static inline Q4<T> qpure(V3<T> v) { return {T(0.0), v.x, v.y, v.z}; }

// The three constant skew-symmetric 4x4 matrices B_k of Eq. 6, acting on (w, x, y, z):
// (B_k a) . b = Im(conj(a) (x) b)_k.
template <class T> static inline Q4<T> Bk(int k, Q4<T> a) {
  if (k == 0) return {-a.x, a.w, a.z, -a.y};
  if (k == 1) return {-a.y, -a.z, a.w, a.x};
  return {-a.z, a.y, -a.x, a.w};
}

// Third director d3 = R(q) e_z (the frame's tangent direction), homogeneous quadratic form.
template <class T> static inline V3<T> director3(Q4<T> q) {
  return {T(2.0) * (q.x * q.z + q.w * q.y), T(2.0) * (q.y * q.z - q.w * q.x),
          q.w * q.w - q.x * q.x - q.y * q.y + q.z * q.z};
}
// Transposed Jacobian of director3: (d d3 / d q)^T a, a 4-vector.
template <class T> static inline Q4<T> director3_vjp(Q4<T> q, V3<T> a) {
  T two(2.0);
  return {two * (q.y * a.x - q.x * a.y + q.w * a.z),
          two * (q.z * a.x - q.w * a.y - q.x * a.z),
          two * (q.w * a.x + q.z * a.y - q.y * a.z),
          two * (q.x * a.x + q.y * a.y + q.z * a.z)};
}

// ------------------------------------------------------------------ parameters

extern "C" {
// Rod material, geometry and stepping parameters (SI units).  Kp, mass_scale and
// inertia_scale <= 0 select the default rules of derive().
typedef struct {
  double length, radius, E_bend, E_stretch, G, density, Kp, damping_alpha;
  double mass_scale, inertia_scale, dt;
  double gravity[3];
  int n_nodes, n_iters, inextensible, clamp;
} OracleParams;
}

struct Derived {
  int N, M;          // nodes, frames
  double l0;         // rest segment length (uniform)
  double A, I;       // area, second moment of area
  double K1, K2, K3; // bend, bend, twist stiffness (N m^2)
  double Ks, Kp;     // stretch stiffness (N), penalty constant (N)
  double mass_scale, inertia_scale;
  std::vector<double> m;  // physical lumped node mass
  std::vector<double> w;  // inverse inertial node mass (0: kinematic)
  double J[3];            // inertial frame inertia (body diagonal)
  double Jinv[3];
  bool frame0_kinematic;
};

static const double kPi = 3.14159265358979323846;

// Section 2.1: stiffness constants of Eq. 2-3 (with the r^4 reading), lumped masses,
// frame inertias, and the default rules for the penalty constant and the inertial
// scaling.  Default rules:
//   Kp = 100 * 4 K1 / L^2   (shear compliance of the penalty 1 % of bending compliance)
//   mass_scale    = max(1, (dt^2 * 4 k_node / m) / 0.25),   k_node = max(Kp, Ks*[extensible]) / l0,
//                   m = rho A l0
//   inertia_scale = max(1, (dt^2 * k_rot / J) / 0.25),      k_rot = 4 max(K1, K3) / l0 + Kp l0,
//                   J = rho l0 I
// i.e. the smallest scaling that puts the estimated highest mode at omega dt <= 0.5.
static Derived derive(const OracleParams& p) {
  Derived d;
  d.N = p.n_nodes;
  d.M = p.n_nodes - 1;
  d.l0 = p.length / d.M;
  d.A = kPi * p.radius * p.radius;
  d.I = kPi * p.radius * p.radius * p.radius * p.radius / 4.0;
  d.K1 = p.E_bend * d.I;
  d.K2 = p.E_bend * d.I;
  d.K3 = p.G * 2.0 * d.I;
  d.Ks = p.E_stretch * d.A;
  d.Kp = p.Kp > 0 ? p.Kp : 100.0 * 4.0 * d.K1 / (p.length * p.length);
  const double m_el = p.density * d.A * d.l0;
  const double J_el = p.density * d.l0 * d.I;
  if (p.mass_scale > 0) {
    d.mass_scale = p.mass_scale;
  } else {
    double k_node = d.Kp / d.l0;
    if (!p.inextensible && d.Ks / d.l0 > k_node) k_node = d.Ks / d.l0;
    double w2dt2 = p.dt * p.dt * 4.0 * k_node / m_el;
    d.mass_scale = w2dt2 / 0.25 > 1.0 ? w2dt2 / 0.25 : 1.0;
  }
  if (p.inertia_scale > 0) {
    d.inertia_scale = p.inertia_scale;
  } else {
    double kb = d.K1 > d.K3 ? d.K1 : d.K3;
    double k_rot = 4.0 * kb / d.l0 + d.Kp * d.l0;
    double w2dt2 = p.dt * p.dt * k_rot / J_el;
    d.inertia_scale = w2dt2 / 0.25 > 1.0 ? w2dt2 / 0.25 : 1.0;
  }
  d.m.assign(d.N, 0.0);
  d.w.assign(d.N, 0.0);
  for (int i = 0; i < d.N; ++i) {
    double left = i > 0 ? d.l0 : 0.0;
    double right = i < d.N - 1 ? d.l0 : 0.0;
    d.m[i] = p.density * d.A * (left + right) / 2.0;
    d.w[i] = 1.0 / (d.mass_scale * d.m[i]);
  }
  d.frame0_kinematic = p.clamp != 0;
  if (p.clamp) d.w[0] = 0.0;
  d.J[0] = d.inertia_scale * J_el;
  d.J[1] = d.inertia_scale * J_el;
  d.J[2] = d.inertia_scale * 2.0 * J_el;
  for (int k = 0; k < 3; ++k) d.Jinv[k] = 1.0 / d.J[k];
  return d;
}

// ------------------------------------------------------------------ state containers

template <class T> struct State {
  std::vector<V3<T>> r, v;   // N nodes
  std::vector<Q4<T>> q;      // M frames
  std::vector<V3<T>> om;     // M frames, body-frame angular velocity
};

template <class T> struct Material {
  std::vector<V3<T>> K;     // per joint (M-1): (K1, K2, K3)
  std::vector<V3<T>> uhat;  // per joint: intrinsic Darboux vector
};

// Discrete Darboux vector of joint j between frames j and j+1 (Eq. 5-6):
// q'_j = (q_{j+1} - q_j) / l_j and u_k = 2 (B_k q_j) . q'_j.
template <class T> static inline V3<T> darboux(Q4<T> qj, Q4<T> qn, double lj) {
  Q4<T> qp = qscale(1.0 / lj, qsub(qn, qj));
  return {T(2.0) * qdot(Bk(0, qj), qp), T(2.0) * qdot(Bk(1, qj), qp), T(2.0) * qdot(Bk(2, qj), qp)};
}

// Rest Darboux vectors from rest frames (u-hat of Eq. 3): the rest shape carries no force.
static void rest_darboux(const Derived& d, const double* rest_xyzw, std::vector<V3<double>>& uhat) {
  uhat.assign(d.M > 1 ? d.M - 1 : 0, V3<double>{0, 0, 0});
  if (!rest_xyzw) return;
  for (int j = 0; j + 1 < d.M; ++j) {
    Q4<double> a{rest_xyzw[4 * j + 3], rest_xyzw[4 * j + 0], rest_xyzw[4 * j + 1], rest_xyzw[4 * j + 2]};
    Q4<double> b{rest_xyzw[4 * j + 7], rest_xyzw[4 * j + 4], rest_xyzw[4 * j + 5], rest_xyzw[4 * j + 6]};
    uhat[j] = darboux(a, b, d.l0);
  }
}

// ------------------------------------------------------------------ energies (Eq. 2, 3, 8)

template <class T> struct Energies { T bend, penalty, stretch, gravity, kin_lin, kin_ang; };

template <class T>
static Energies<T> energies(const OracleParams& p, const Derived& d, const Material<T>& mat, const State<T>& s) {
  Energies<T> e{T(0.0), T(0.0), T(0.0), T(0.0), T(0.0), T(0.0)};
  // Eq. 3, discretised: sum_j 1/2 l_j sum_k K_k (u_k - uhat_k)^2, l_j = l0 (uniform).
  for (int j = 0; j + 1 < d.M; ++j) {
    V3<T> u = darboux(s.q[j], s.q[j + 1], d.l0);
    V3<T> du = u - mat.uhat[j];
    e.bend += T(0.5 * d.l0) * (mat.K[j].x * du.x * du.x + mat.K[j].y * du.y * du.y + mat.K[j].z * du.z * du.z);
  }
  for (int j = 0; j < d.M; ++j) {
    V3<T> seg = s.r[j + 1] - s.r[j];
    T len = norm(seg);
    V3<T> t = (T(1.0) / len) * seg;  // Eq. 4
    V3<T> a = t - director3(s.q[j]);
    e.penalty += T(0.5 * d.l0 * d.Kp) * dot(a, a);  // Eq. 8
    if (!p.inextensible) {
      T str = len / T(d.l0) - T(1.0);  // v3 - 1 (Eq. 2)
      e.stretch += T(0.5 * d.l0 * d.Ks) * str * str;
    }
  }
  V3<T> g{T(p.gravity[0]), T(p.gravity[1]), T(p.gravity[2])};
  for (int i = 0; i < d.N; ++i) {
    e.gravity -= T(d.m[i]) * dot(g, s.r[i]);
    if (d.w[i] > 0) e.kin_lin += T(0.5 * d.mass_scale * d.m[i]) * dot(s.v[i], s.v[i]);
  }
  for (int j = 0; j < d.M; ++j) {
    if (j == 0 && d.frame0_kinematic) continue;
    const V3<T>& w = s.om[j];
    e.kin_ang += T(0.5) * (T(d.J[0]) * w.x * w.x + T(d.J[1]) * w.y * w.y + T(d.J[2]) * w.z * w.z);
  }
  return e;
}

// ------------------------------------------------------------------ forces and torques

// Elastic forces F_i = -dV/dr_i and quaternion gradients g_j = dV/dq_j of
// V = V_b + E_p (+ V_s for the extensible rod), by hand differentiation of Eq. 2, 3, 8.
template <class T>
static void elastic_gradients(const OracleParams& p, const Derived& d, const Material<T>& mat,
                              const State<T>& s, std::vector<V3<T>>& F, std::vector<Q4<T>>& g) {
  const T zero(0.0);
  F.assign(d.N, V3<T>{zero, zero, zero});
  g.assign(d.M, Q4<T>{zero, zero, zero, zero});
  // Bend / twist (Eq. 3 with Eq. 5-6).  dV/du_k = l_j K_k (u_k - uhat_k), and
  // du_k/dq_{j+1} = (2/l_j) B_k q_j,  du_k/dq_j = -(2/l_j) B_k q_{j+1}  (B_k skew).
  for (int j = 0; j + 1 < d.M; ++j) {
    V3<T> u = darboux(s.q[j], s.q[j + 1], d.l0);
    V3<T> du = u - mat.uhat[j];
    T c[3] = {T(2.0) * mat.K[j].x * du.x, T(2.0) * mat.K[j].y * du.y, T(2.0) * mat.K[j].z * du.z};
    for (int k = 0; k < 3; ++k) {
      g[j + 1] = qadd(g[j + 1], qscale(c[k], Bk(k, s.q[j])));
      g[j] = qsub(g[j], qscale(c[k], Bk(k, s.q[j + 1])));
    }
  }
  for (int j = 0; j < d.M; ++j) {
    V3<T> seg = s.r[j + 1] - s.r[j];
    T len = norm(seg);
    V3<T> t = (T(1.0) / len) * seg;
    V3<T> d3 = director3(s.q[j]);
    // Penalty (Eq. 8): E = 1/2 l0 Kp |t - d3|^2.
    //   dE/dseg = l0 Kp (I - t t^T)(t - d3) / |seg|,  dE/dd3 = -l0 Kp (t - d3).
    V3<T> a = t - d3;
    V3<T> proj = a - dot(t, a) * t;
    V3<T> dEdseg = (T(d.l0 * d.Kp) / len) * proj;
    F[j] = F[j] + dEdseg;
    F[j + 1] = F[j + 1] - dEdseg;
    g[j] = qadd(g[j], director3_vjp(s.q[j], (T(-d.l0 * d.Kp)) * a));
    // Stretch (Eq. 2), extensible rod only: E = 1/2 l0 Ks (|seg|/l0 - 1)^2.
    if (!p.inextensible) {
      V3<T> dSdseg = (T(d.Ks) * (len / T(d.l0) - T(1.0))) * t;
      F[j] = F[j] + dSdseg;
      F[j + 1] = F[j + 1] - dSdseg;
    }
  }
}

// Body-frame torque from a quaternion gradient: with dq/dt = 1/2 q (x) (0, omega) the
// power is -g . dq/dt = tau . omega, so tau = -1/2 Im(conj(q) (x) g).
template <class T> static inline V3<T> torque_from_gradient(Q4<T> q, Q4<T> g) {
  return T(-0.5) * qim(qmul(qconj(q), g));
}

// ------------------------------------------------------------------ the time step

// Fig. 5, first lines: external forces and torques (gravity with the physical mass,
// optional loads), Cosserat elastic forces and torques, and their integration into
// velocities (points as particles, frames as rigid bodies), with Rayleigh damping applied
// implicitly: x <- (x + dt a) / (1 + alpha dt).  drive = [v_x v_y v_z . w_x w_y w_z .]
// of the kinematic base (node 0, frame 0).  f_ext (N x 3, world) and tau_ext (M x 3,
// body) are optional external loads.
template <class T>
static void integrate_forces(const OracleParams& p, const Derived& d, const Material<T>& mat, State<T>& s,
                             const double* drive, const double* f_ext, const double* tau_ext) {
  const double dt = p.dt;
  std::vector<V3<T>> Fext(d.N), F;
  std::vector<Q4<T>> g;
  for (int i = 0; i < d.N; ++i) {
    Fext[i] = v3(T(d.m[i] * p.gravity[0]), T(d.m[i] * p.gravity[1]), T(d.m[i] * p.gravity[2]));
    if (f_ext) Fext[i] = Fext[i] + v3(T(f_ext[3 * i]), T(f_ext[3 * i + 1]), T(f_ext[3 * i + 2]));
  }
  elastic_gradients(p, d, mat, s, F, g);
  const double damp = 1.0 / (1.0 + p.damping_alpha * dt);
  for (int i = 0; i < d.N; ++i) {
    if (d.w[i] == 0.0) continue;
    V3<T> Ftot = F[i] + Fext[i];
    s.v[i] = damp * (s.v[i] + (dt * d.w[i]) * Ftot);
  }
  for (int j = 0; j < d.M; ++j) {
    if (j == 0 && d.frame0_kinematic) continue;
    V3<T> tau = torque_from_gradient(s.q[j], g[j]);
    if (tau_ext) tau = tau + v3(T(tau_ext[3 * j]), T(tau_ext[3 * j + 1]), T(tau_ext[3 * j + 2]));
    const V3<T>& w = s.om[j];
    V3<T> Jw{T(d.J[0]) * w.x, T(d.J[1]) * w.y, T(d.J[2]) * w.z};
    V3<T> rhs = tau - cross(w, Jw);
    V3<T> wn{w.x + T(dt * d.Jinv[0]) * rhs.x, w.y + T(dt * d.Jinv[1]) * rhs.y, w.z + T(dt * d.Jinv[2]) * rhs.z};
    s.om[j] = damp * wn;
  }
  if (p.clamp) {
    s.v[0] = v3(T(drive ? drive[0] : 0.0), T(drive ? drive[1] : 0.0), T(drive ? drive[2] : 0.0));
    if (d.M > 0) s.om[0] = v3(T(drive ? drive[4] : 0.0), T(drive ? drive[5] : 0.0), T(drive ? drive[6] : 0.0));
  }
}

// One half-sweep of the distance constraints C_d (inextensible rod, Section 2.1
// "Constraints"): every segment j with j % 2 == parity gets a predictive impulse,
// lambda = -C / (dt (w_a + w_b)) with C = |d| - l0, d = (r_b + dt v_b) - (r_a + dt v_a),
// n = d / |d|, v_a -= w_a lambda n, v_b += w_b lambda n.
template <class T>
static void distance_sweep(const OracleParams& p, const Derived& d, State<T>& s, int parity) {
  const double dt = p.dt;
  for (int j = parity; j < d.M; j += 2) {
    const int a = j, b = j + 1;
    const double W = d.w[a] + d.w[b];
    if (W == 0.0) continue;
    V3<T> pa = s.r[a] + dt * s.v[a];
    V3<T> pb = s.r[b] + dt * s.v[b];
    V3<T> dd = pb - pa;
    T len = norm(dd);
    T C = len - T(d.l0);
    V3<T> n = (T(1.0) / len) * dd;
    T lam = -C / T(dt * W);
    s.v[a] = s.v[a] - (T(d.w[a]) * lam) * n;
    s.v[b] = s.v[b] + (T(d.w[b]) * lam) * n;
  }
}

// Fig. 5, last line: semi-implicit Euler integration of linear and angular velocity.
template <class T>
static void integrate_positions(const OracleParams& p, const Derived& d, State<T>& s) {
  const double dt = p.dt;
  for (int i = 0; i < d.N; ++i) s.r[i] = s.r[i] + dt * s.v[i];
  for (int j = 0; j < d.M; ++j) {
    Q4<T> dq = qmul(s.q[j], qpure(s.om[j]));
    Q4<T> qn = qadd(s.q[j], qscale(0.5 * dt, dq));
    T nn = sqrt(qdot(qn, qn));
    s.q[j] = qscale(T(1.0) / nn, qn);
  }
}

// Collision response against an analytic vessel (contact constraints C_c with Coulomb
// friction, Section 2.1 "Constraints"; iterated with the distance constraints, Section
// 3.3).  tube = [cx, cy, cz, Rc, Rt, mu]: the vessel centreline is the circle of radius Rc
// about (cx, cy) in the plane z = cz, its inner radius Rt.  A dynamic node must keep its
// predicted position p = r + dt v within Rt - r of the centreline.  With c the centreline
// point nearest to p and delta = p - c, a violation |delta| > Rt - r changes the
// normal velocity by dvn = -(|delta| - (Rt - r)) / dt along n = delta / |delta| and cuts
// the tangential velocity v_t by at most mu |dvn| (Coulomb).
template <class T>
static void contact_sweep(const OracleParams& p, const Derived& d, State<T>& s, const double* tube) {
  const double dt = p.dt;
  const double allow = tube[4] - p.radius;
  for (int i = 0; i < d.N; ++i) {
    if (d.w[i] == 0.0) continue;
    const V3<T> pr = s.r[i] + dt * s.v[i];
    const T dx = pr.x - T(tube[0]), dy = pr.y - T(tube[1]);
    const T rho = sqrt(dx * dx + dy * dy);
    if (val(rho) == 0.0) continue;
    const V3<T> c{T(tube[0]) + T(tube[3]) * dx / rho, T(tube[1]) + T(tube[3]) * dy / rho, T(tube[2])};
    const V3<T> delta = pr - c;
    const T dist = norm(delta);
    if (!(val(dist) > allow)) continue;
    const V3<T> n = (T(1.0) / dist) * delta;
    const T dvn = -(dist - T(allow)) / T(dt);
    const V3<T> vt = s.v[i] - dot(s.v[i], n) * n;
    const T vtn = norm(vt);
    T keep(1.0);
    if (val(vtn) > 0.0) {
      const T f = T(1.0) - T(tube[5]) * (val(dvn) < 0 ? -dvn : dvn) / vtn;
      keep = val(f) > 0.0 ? f : T(0.0);
    }
    s.v[i] = (s.v[i] + dvn * n) - (T(1.0) - keep) * vt;
  }
}

// Self-collision ("Collisions and self-collisions" and Section 2.1 "Constraints": contact
// constraints C_c for self-collisions with Coulomb friction).  Every mass point carries a
// sphere of the rod radius r; two mass points i, j at least min_sep apart along the rod
// collide when their spheres overlap.  Detection runs once per step, on the positions the
// constraint stage starts from: the candidate pairs are all pairs with |i - j| >= min_sep
// and |r_i - r_j| < reach (reach = 3r: contact distance 2r plus a skin of r, so a pair
// that comes into contact during the step is a candidate).  This is the definition the
// GPU's bounding-sphere broad phase and sphere-sphere narrow phase must reproduce.
//   min_sep = max(2, floor(2r / l0) + 1): the smallest index gap whose rest distance
//   exceeds the contact distance (mass points closer along a straight rod always overlap).
struct SelfContact {
  double mu;       // Coulomb friction coefficient between strands
  double contact;  // contact distance 2r
  double reach;    // candidate distance 3r
  int min_sep;     // smallest index gap considered
};

static SelfContact self_contact_of(const OracleParams& p, const Derived& d, double mu) {
  SelfContact sc;
  sc.mu = mu;
  sc.contact = 2.0 * p.radius;
  sc.reach = 3.0 * p.radius;
  const int m = (int)std::floor(sc.contact / d.l0) + 1;
  sc.min_sep = m > 2 ? m : 2;
  return sc;
}

// Candidate partners of every mass point, ascending, by brute force over all pairs.
template <class T>
static void self_candidates(const SelfContact& sc, const Derived& d, const State<T>& s,
                            std::vector<std::vector<int>>& cand) {
  cand.assign(d.N, std::vector<int>());
  for (int i = 0; i < d.N; ++i)
    for (int j = i + sc.min_sep; j < d.N; ++j) {
      const double dx = val(s.r[j].x) - val(s.r[i].x);
      const double dy = val(s.r[j].y) - val(s.r[i].y);
      const double dz = val(s.r[j].z) - val(s.r[i].z);
      if (dx * dx + dy * dy + dz * dz < sc.reach * sc.reach) {
        cand[i].push_back(j);
        cand[j].push_back(i);
      }
    }
  for (auto& c : cand) std::sort(c.begin(), c.end());
}

// One pass of the self-contact constraints (Jacobi: every impulse from the velocities the
// pass starts with).  For a candidate pair (i, j) with predicted offset
// delta = (r_j - r_i) + dt (v_j - v_i) shorter than the contact distance, the pair's
// impulse J (applied +J to j, -J to i) makes the relative normal velocity separate the
// predicted spheres exactly and cuts the relative tangential velocity u_t by at most
// mu times that normal change (Coulomb):
//   phi = 2r - |delta|,  n = delta / |delta|,  du_n = phi / dt,
//   J = (du_n n - min(1, mu du_n / |u_t|) u_t) / (w_i + w_j).
// A mass point touching several others takes the average of its pairs' velocity changes,
// weighted by penetration depth (as the paper weights its collision response vectors):
//   dv_i = -w_i sum_j phi_ij J_ij / sum_j phi_ij.
template <class T>
static void self_contact_sweep(const OracleParams& p, const Derived& d, State<T>& s, const SelfContact& sc,
                               const std::vector<std::vector<int>>& cand) {
  const double dt = p.dt;
  std::vector<V3<T>> dv(d.N, V3<T>{T(0.0), T(0.0), T(0.0)});
  for (int i = 0; i < d.N; ++i) {
    if (d.w[i] == 0.0 || cand[i].empty()) continue;
    V3<T> acc{T(0.0), T(0.0), T(0.0)};
    T wphi(0.0);
    for (int j : cand[i]) {
      const double wsum = d.w[i] + d.w[j];
      const V3<T> u = s.v[j] - s.v[i];
      const V3<T> delta = (s.r[j] - s.r[i]) + dt * u;
      const T dist = norm(delta);
      if (!(val(dist) < sc.contact) || val(dist) == 0.0) continue;
      const T phi = T(sc.contact) - dist;
      const V3<T> n = (T(1.0) / dist) * delta;
      const T dun = phi / T(dt);
      const V3<T> ut = u - dot(u, n) * n;
      const T utn = norm(ut);
      T cut(0.0);
      if (val(utn) > 0.0) {
        const T f = T(sc.mu) * dun / utn;
        cut = val(f) < 1.0 ? f : T(1.0);
      }
      const V3<T> J = (T(1.0) / T(wsum)) * (dun * n - cut * ut);
      acc = acc + phi * J;
      wphi = wphi + phi;
    }
    if (val(wphi) > 0.0) dv[i] = (-d.w[i] / wphi) * acc;
  }
  for (int i = 0; i < d.N; ++i) s.v[i] = s.v[i] + dv[i];
}

// One time step of one rod, Fig. 5 order: forces, then n_iters iterations of the
// red-black distance sweeps (even segments, then odd) followed by the collision
// responses (the vessel when given, then self-contact when given), then the position
// update.
template <class T>
static void step(const OracleParams& p, const Derived& d, const Material<T>& mat, State<T>& s,
                 const double* drive, const double* f_ext, const double* tau_ext, const double* tube = nullptr,
                 const SelfContact* sc = nullptr) {
  integrate_forces(p, d, mat, s, drive, f_ext, tau_ext);
  if (p.inextensible) {
    std::vector<std::vector<int>> cand;
    if (sc) self_candidates(*sc, d, s, cand);
    for (int it = 0; it < p.n_iters; ++it) {
      distance_sweep(p, d, s, 0);
      distance_sweep(p, d, s, 1);
      if (tube) contact_sweep(p, d, s, tube);
      if (sc) self_contact_sweep(p, d, s, *sc, cand);
    }
  }
  integrate_positions(p, d, s);
}

// One color of the binding constraints C_b (Section 2.1 "Constraints": distance
// constraints of rest length zero that keep two rods together; Section 3.4: v1 one-way,
// the outer rod is not moved; v2 two-way).  Inner node i with i % 2 == color is bound to
// the outer rod's centreline point at arclength (i + beta) l0 (both rods share l0):
// segment k = floor(i + beta), fraction a = (i + beta) - k, point p = (1-a) r_k + a r_{k+1}.
// Predictive vector impulse making (r_i + dt v_i) - (p + dt v_p) vanish:
// lambda = -d / (dt w_eff), w_eff = w_i (+ (1-a)^2 w_k + a^2 w_{k+1} in v2).
template <class T>
static void binding_color(const OracleParams& po, const Derived& dout, State<T>& so, const Derived& din,
                          State<T>& si, int mode, double beta, int color) {
  const double dt = po.dt;
  const double kb = std::floor(beta);
  const double a = beta - kb;
  for (int i = color; i < din.N; i += 2) {
    const double kk = (double)i + kb;
    if (kk < 0.0 || kk > (double)(dout.N - 2)) continue;
    const int k = (int)kk;
    const double wi = din.w[i];
    const double wk = mode == 2 ? dout.w[k] : 0.0, wk1 = mode == 2 ? dout.w[k + 1] : 0.0;
    const double weff = wi + (1.0 - a) * (1.0 - a) * wk + a * a * wk1;
    if (weff == 0.0) continue;
    V3<T> pc = (1.0 - a) * so.r[k] + a * so.r[k + 1];
    V3<T> vc = (1.0 - a) * so.v[k] + a * so.v[k + 1];
    V3<T> dd = (si.r[i] + dt * si.v[i]) - (pc + dt * vc);
    V3<T> lam = (-1.0 / (dt * weff)) * dd;
    si.v[i] = si.v[i] + wi * lam;
    if (mode == 2) {
      so.v[k] = so.v[k] - ((1.0 - a) * wk) * lam;
      so.v[k + 1] = so.v[k + 1] - (a * wk1) * lam;
    }
  }
}

// One time step of an outer/inner rod pair (catheter and guidewire, Section 3.4): both
// rods' forces, then per constraint iteration both rods' distance sweeps followed by the
// two binding colors (mode 0: none), then both position updates.
template <class T>
static void step_pair(const OracleParams& po, const Derived& dout, const Material<T>& mo, State<T>& so,
                      const double* drive_o, const OracleParams& pi, const Derived& din, const Material<T>& mi,
                      State<T>& si, const double* drive_i, int mode, double beta) {
  integrate_forces(po, dout, mo, so, drive_o, nullptr, nullptr);
  integrate_forces(pi, din, mi, si, drive_i, nullptr, nullptr);
  for (int it = 0; it < po.n_iters; ++it) {
    distance_sweep(po, dout, so, 0);
    distance_sweep(po, dout, so, 1);
    distance_sweep(pi, din, si, 0);
    distance_sweep(pi, din, si, 1);
    if (mode != 0) {
      binding_color(po, dout, so, din, si, mode, beta, 0);
      binding_color(po, dout, so, din, si, mode, beta, 1);
    }
  }
  integrate_positions(po, dout, so);
  integrate_positions(pi, din, si);
}

// ------------------------------------------------------------------ marshalling

template <class T>
static void load_state(const Derived& d, const double* pos, const double* quat, const double* vel,
                       const double* omega, State<T>& s) {
  s.r.resize(d.N);
  s.v.resize(d.N);
  s.q.resize(d.M);
  s.om.resize(d.M);
  for (int i = 0; i < d.N; ++i) {
    s.r[i] = v3(T(pos[3 * i]), T(pos[3 * i + 1]), T(pos[3 * i + 2]));
    s.v[i] = vel ? v3(T(vel[3 * i]), T(vel[3 * i + 1]), T(vel[3 * i + 2])) : v3(T(0.0), T(0.0), T(0.0));
  }
  for (int j = 0; j < d.M; ++j) {
    s.q[j] = quat ? Q4<T>{T(quat[4 * j + 3]), T(quat[4 * j]), T(quat[4 * j + 1]), T(quat[4 * j + 2])}
                  : Q4<T>{T(1.0), T(0.0), T(0.0), T(0.0)};
    s.om[j] = omega ? v3(T(omega[3 * j]), T(omega[3 * j + 1]), T(omega[3 * j + 2])) : v3(T(0.0), T(0.0), T(0.0));
  }
}

static void store_state(const Derived& d, const State<double>& s, double* pos, double* quat, double* vel,
                        double* omega) {
  for (int i = 0; i < d.N; ++i) {
    if (pos) { pos[3 * i] = s.r[i].x; pos[3 * i + 1] = s.r[i].y; pos[3 * i + 2] = s.r[i].z; }
    if (vel) { vel[3 * i] = s.v[i].x; vel[3 * i + 1] = s.v[i].y; vel[3 * i + 2] = s.v[i].z; }
  }
  for (int j = 0; j < d.M; ++j) {
    if (quat) { quat[4 * j] = s.q[j].x; quat[4 * j + 1] = s.q[j].y; quat[4 * j + 2] = s.q[j].z; quat[4 * j + 3] = s.q[j].w; }
    if (omega) { omega[3 * j] = s.om[j].x; omega[3 * j + 1] = s.om[j].y; omega[3 * j + 2] = s.om[j].z; }
  }
}

// Per-joint stiffness: base (K1, K2, K3) times optional multipliers (M-1 x 3); intrinsic
// Darboux vectors from the rest frames (or zero).
template <class T>
static void load_material(const Derived& d, const double* rest_quat, const double* stiff_mul, Material<T>& mat,
                          const double* K_abs = nullptr, const double* uhat_abs = nullptr) {
  std::vector<V3<double>> uh;
  rest_darboux(d, rest_quat, uh);
  int J = d.M > 1 ? d.M - 1 : 0;
  mat.K.resize(J);
  mat.uhat.resize(J);
  for (int j = 0; j < J; ++j) {
    double m1 = stiff_mul ? stiff_mul[3 * j] : 1.0, m2 = stiff_mul ? stiff_mul[3 * j + 1] : 1.0,
           m3 = stiff_mul ? stiff_mul[3 * j + 2] : 1.0;
    mat.K[j] = v3(T(d.K1 * m1), T(d.K2 * m2), T(d.K3 * m3));
    mat.uhat[j] = v3(T(uh[j].x), T(uh[j].y), T(uh[j].z));
    if (K_abs) mat.K[j] = v3(T(K_abs[3 * j]), T(K_abs[3 * j + 1]), T(K_abs[3 * j + 2]));
    if (uhat_abs) mat.uhat[j] = v3(T(uhat_abs[3 * j]), T(uhat_abs[3 * j + 1]), T(uhat_abs[3 * j + 2]));
  }
}

static bool valid(const OracleParams* p) {
  return p && p->n_nodes >= 2 && p->length > 0 && p->radius > 0 && p->density > 0 && p->dt > 0 && p->n_iters >= 0;
}

// ------------------------------------------------------------------ C interface

extern "C" {

// Derived quantities: out[16] = l0, A, I, K1, K2, K3, Ks, Kp, mass_scale, inertia_scale,
// m_interior (physical), J1, J2, J3 (inertial), w_interior (inverse inertial), 0.
int oracle_derive(const OracleParams* p, double* out) {
  if (!valid(p) || !out) return -1;
  Derived d = derive(*p);
  double m_int = p->density * d.A * d.l0;
  double v[16] = {d.l0, d.A, d.I, d.K1, d.K2, d.K3, d.Ks, d.Kp, d.mass_scale, d.inertia_scale,
                  m_int, d.J[0], d.J[1], d.J[2], 1.0 / (d.mass_scale * m_int), 0.0};
  std::memcpy(out, v, sizeof(v));
  return 0;
}

// Darboux vectors (Eq. 5-6) of frames quat (M x 4, xyzw) -> u ((M-1) x 3).
int oracle_darboux(const OracleParams* p, const double* quat, double* u_out) {
  if (!valid(p) || !quat || !u_out) return -1;
  Derived d = derive(*p);
  for (int j = 0; j + 1 < d.M; ++j) {
    Q4<double> a{quat[4 * j + 3], quat[4 * j], quat[4 * j + 1], quat[4 * j + 2]};
    Q4<double> b{quat[4 * j + 7], quat[4 * j + 4], quat[4 * j + 5], quat[4 * j + 6]};
    V3<double> u = darboux(a, b, d.l0);
    u_out[3 * j] = u.x; u_out[3 * j + 1] = u.y; u_out[3 * j + 2] = u.z;
  }
  return 0;
}

// Energies: out[6] = V_bend, E_penalty, V_stretch, V_gravity, T_linear, T_angular.
int oracle_energy(const OracleParams* p, const double* rest_quat, const double* stiff_mul, const double* pos,
                  const double* quat, const double* vel, const double* omega, double* out) {
  if (!valid(p) || !pos || !quat || !out) return -1;
  Derived d = derive(*p);
  Material<double> mat;
  load_material(d, rest_quat, stiff_mul, mat);
  State<double> s;
  load_state(d, pos, quat, vel, omega, s);
  Energies<double> e = energies(*p, d, mat, s);
  out[0] = e.bend; out[1] = e.penalty; out[2] = e.stretch; out[3] = e.gravity; out[4] = e.kin_lin; out[5] = e.kin_ang;
  return 0;
}

// Elastic forces F (N x 3), body torques tau (M x 3) and quaternion gradients g (M x 4,
// xyzw order) of the current configuration (no gravity, no damping).
int oracle_forces(const OracleParams* p, const double* rest_quat, const double* stiff_mul, const double* pos,
                  const double* quat, double* F_out, double* tau_out, double* g_out) {
  if (!valid(p) || !pos || !quat) return -1;
  Derived d = derive(*p);
  Material<double> mat;
  load_material(d, rest_quat, stiff_mul, mat);
  State<double> s;
  load_state(d, pos, quat, nullptr, nullptr, s);
  std::vector<V3<double>> F;
  std::vector<Q4<double>> g;
  elastic_gradients(*p, d, mat, s, F, g);
  for (int i = 0; i < d.N; ++i)
    if (F_out) { F_out[3 * i] = F[i].x; F_out[3 * i + 1] = F[i].y; F_out[3 * i + 2] = F[i].z; }
  for (int j = 0; j < d.M; ++j) {
    V3<double> t = torque_from_gradient(s.q[j], g[j]);
    if (tau_out) { tau_out[3 * j] = t.x; tau_out[3 * j + 1] = t.y; tau_out[3 * j + 2] = t.z; }
    if (g_out) { g_out[4 * j] = g[j].x; g_out[4 * j + 1] = g[j].y; g_out[4 * j + 2] = g[j].z; g_out[4 * j + 3] = g[j].w; }
  }
  return 0;
}

// n_steps time steps in place.  drive: 8 doubles (constant over the call) or NULL.
int oracle_step(const OracleParams* p, const double* rest_quat, const double* stiff_mul, double* pos, double* quat,
                double* vel, double* omega, const double* drive, const double* f_ext, const double* tau_ext,
                int n_steps) {
  if (!valid(p) || !pos || !quat || !vel || !omega || n_steps < 0) return -1;
  Derived d = derive(*p);
  Material<double> mat;
  load_material(d, rest_quat, stiff_mul, mat);
  State<double> s;
  load_state(d, pos, quat, vel, omega, s);
  for (int k = 0; k < n_steps; ++k) step(*p, d, mat, s, drive, f_ext, tau_ext);
  store_state(d, s, pos, quat, vel, omega);
  return 0;
}

// Rollout of n_steps with a per-step drive table (n_steps x 8, or NULL) recording the
// node positions after every step: traj (n_steps x N x 3).  Optionally advances the
// state arrays in place (when update_state != 0).  K_abs / uhat_abs ((M-1) x 3, or
// NULL) override the per-joint stiffness and intrinsic Darboux vectors.
int oracle_rollout(const OracleParams* p, const double* rest_quat, const double* stiff_mul, const double* K_abs,
                   const double* uhat_abs, double* pos, double* quat, double* vel, double* omega,
                   const double* drive_table, int n_steps, double* traj, int update_state) {
  if (!valid(p) || !pos || !quat || n_steps < 0) return -1;
  Derived d = derive(*p);
  Material<double> mat;
  load_material(d, rest_quat, stiff_mul, mat, K_abs, uhat_abs);
  State<double> s;
  load_state(d, pos, quat, vel, omega, s);
  for (int k = 0; k < n_steps; ++k) {
    step(*p, d, mat, s, drive_table ? drive_table + 8 * k : nullptr, nullptr, nullptr);
    if (traj)
      for (int i = 0; i < d.N; ++i) {
        double* o = traj + ((size_t)k * d.N + i) * 3;
        o[0] = s.r[i].x; o[1] = s.r[i].y; o[2] = s.r[i].z;
      }
  }
  if (update_state) store_state(d, s, pos, quat, vel, omega);
  return 0;
}

// Forward-mode derivative of a rollout (dual numbers): perturbs the initial positions
// (d_pos, N x 3), initial velocities (d_vel, N x 3), per-joint stiffness (d_K, absolute,
// (M-1) x 3), intrinsic Darboux vectors (d_uhat, (M-1) x 3), initial frames (d_quat,
// M x 4, tangents of the four quaternion components x, y, z, w) and initial body angular
// velocities (d_omega, M x 3); any may be NULL.  The state the method evolves is the
// centreline, the frames and their velocities (Section 2.1), so each is an input here.
// Writes the position trajectory (traj, n_steps x N x 3) and its tangent (dtraj).
int oracle_rollout_jvp(const OracleParams* p, const double* rest_quat, const double* stiff_mul, const double* K_abs,
                       const double* uhat_abs, const double* pos, const double* quat, const double* vel,
                       const double* omega, const double* drive_table, int n_steps, const double* d_pos,
                       const double* d_vel, const double* d_K, const double* d_uhat, const double* d_quat,
                       const double* d_omega, double* traj, double* dtraj) {
  if (!valid(p) || !pos || !quat || n_steps < 0) return -1;
  Derived d = derive(*p);
  Material<double> base;
  load_material(d, rest_quat, stiff_mul, base, K_abs, uhat_abs);
  Material<Dual> mat;
  int J = d.M > 1 ? d.M - 1 : 0;
  mat.K.resize(J);
  mat.uhat.resize(J);
  for (int j = 0; j < J; ++j) {
    mat.K[j] = v3(Dual(base.K[j].x, d_K ? d_K[3 * j] : 0.0), Dual(base.K[j].y, d_K ? d_K[3 * j + 1] : 0.0),
                  Dual(base.K[j].z, d_K ? d_K[3 * j + 2] : 0.0));
    mat.uhat[j] = v3(Dual(base.uhat[j].x, d_uhat ? d_uhat[3 * j] : 0.0), Dual(base.uhat[j].y, d_uhat ? d_uhat[3 * j + 1] : 0.0),
                     Dual(base.uhat[j].z, d_uhat ? d_uhat[3 * j + 2] : 0.0));
  }
  State<Dual> s;
  load_state(d, pos, quat, vel, omega, s);
  for (int i = 0; i < d.N; ++i) {
    if (d_pos) { s.r[i].x.d = d_pos[3 * i]; s.r[i].y.d = d_pos[3 * i + 1]; s.r[i].z.d = d_pos[3 * i + 2]; }
    if (d_vel) { s.v[i].x.d = d_vel[3 * i]; s.v[i].y.d = d_vel[3 * i + 1]; s.v[i].z.d = d_vel[3 * i + 2]; }
  }
  for (int j = 0; j < d.M; ++j) {
    if (d_quat) {
      s.q[j].x.d = d_quat[4 * j]; s.q[j].y.d = d_quat[4 * j + 1];
      s.q[j].z.d = d_quat[4 * j + 2]; s.q[j].w.d = d_quat[4 * j + 3];
    }
    if (d_omega) { s.om[j].x.d = d_omega[3 * j]; s.om[j].y.d = d_omega[3 * j + 1]; s.om[j].z.d = d_omega[3 * j + 2]; }
  }
  for (int k = 0; k < n_steps; ++k) {
    step(*p, d, mat, s, drive_table ? drive_table + 8 * k : nullptr, nullptr, nullptr);
    for (int i = 0; i < d.N; ++i) {
      size_t o = ((size_t)k * d.N + i) * 3;
      if (traj) { traj[o] = s.r[i].x.v; traj[o + 1] = s.r[i].y.v; traj[o + 2] = s.r[i].z.v; }
      if (dtraj) { dtraj[o] = s.r[i].x.d; dtraj[o + 1] = s.r[i].y.d; dtraj[o + 2] = s.r[i].z.d; }
    }
  }
  return 0;
}

// n_steps time steps of one rod inside an analytic vessel tube = [cx, cy, cz, Rc, Rt, mu]
// (see contact_sweep); otherwise as oracle_step.
int oracle_step_tube(const OracleParams* p, const double* rest_quat, double* pos, double* quat, double* vel,
                     double* omega, const double* drive, const double* tube, int n_steps) {
  if (!valid(p) || !pos || !quat || !vel || !omega || !tube || n_steps < 0) return -1;
  if (!(tube[3] > 0) || !(tube[4] > p->radius) || !(tube[5] >= 0)) return -1;
  Derived d = derive(*p);
  Material<double> mat;
  load_material(d, rest_quat, nullptr, mat);
  State<double> s;
  load_state(d, pos, quat, vel, omega, s);
  for (int k = 0; k < n_steps; ++k) step(*p, d, mat, s, drive, nullptr, nullptr, tube);
  store_state(d, s, pos, quat, vel, omega);
  return 0;
}

// n_steps time steps of one rod with contact: the vessel tube = [cx, cy, cz, Rc, Rt, mu]
// (NULL: none) and self-collision self = [mu] (NULL: none); otherwise as oracle_step.
int oracle_step_contact(const OracleParams* p, const double* rest_quat, double* pos, double* quat, double* vel,
                        double* omega, const double* drive, const double* tube, const double* self, int n_steps) {
  if (!valid(p) || !pos || !quat || !vel || !omega || n_steps < 0 || !p->inextensible) return -1;
  if (tube && (!(tube[3] > 0) || !(tube[4] > p->radius) || !(tube[5] >= 0))) return -1;
  if (self && !(self[0] >= 0)) return -1;
  Derived d = derive(*p);
  Material<double> mat;
  load_material(d, rest_quat, nullptr, mat);
  State<double> s;
  load_state(d, pos, quat, vel, omega, s);
  SelfContact sc;
  if (self) sc = self_contact_of(*p, d, self[0]);
  for (int k = 0; k < n_steps; ++k) step(*p, d, mat, s, drive, nullptr, nullptr, tube, self ? &sc : nullptr);
  store_state(d, s, pos, quat, vel, omega);
  return 0;
}

// Self-collision candidates of the positions pos: counts[i] partners of node i, listed
// ascending in list[i * cap ...] (at most cap kept); returns the number of pairs, or -1.
int oracle_self_candidates(const OracleParams* p, const double* pos, int* counts, int* list, int cap) {
  if (!valid(p) || !pos || !counts || cap < 0) return -1;
  Derived d = derive(*p);
  State<double> s;
  load_state(d, pos, nullptr, nullptr, nullptr, s);
  const SelfContact sc = self_contact_of(*p, d, 0.0);
  std::vector<std::vector<int>> cand;
  self_candidates(sc, d, s, cand);
  int pairs = 0;
  for (int i = 0; i < d.N; ++i) {
    counts[i] = (int)cand[i].size();
    pairs += counts[i];
    for (int k = 0; k < counts[i] && k < cap; ++k) list[(size_t)i * cap + k] = cand[i][k];
  }
  return pairs / 2;
}

// One Jacobi pass of the self-contact constraints on (pos, vel) with friction mu (vel is
// updated in place); the candidates are detected on pos.
int oracle_self_contact_pass(const OracleParams* p, const double* pos, double* vel, double mu) {
  if (!valid(p) || !pos || !vel || !(mu >= 0)) return -1;
  Derived d = derive(*p);
  State<double> s;
  load_state(d, pos, nullptr, vel, nullptr, s);
  const SelfContact sc = self_contact_of(*p, d, mu);
  std::vector<std::vector<int>> cand;
  self_candidates(sc, d, s, cand);
  self_contact_sweep(*p, d, s, sc, cand);
  for (int i = 0; i < d.N; ++i) {
    vel[3 * i] = s.v[i].x;
    vel[3 * i + 1] = s.v[i].y;
    vel[3 * i + 2] = s.v[i].z;
  }
  return 0;
}

// n_steps time steps of an outer/inner rod pair with binding mode 0, 1 or 2 (v0/v1/v2 of
// Section 3.4) and binding offset beta (inner node i sits at outer arclength (i + beta) l0).
// Both rods must be inextensible with the same l0, dt and n_iters.  State arrays of both
// rods are advanced in place; drives are 8 doubles each or NULL.
int oracle_step_pair(const OracleParams* po, const double* rest_o, double* pos_o, double* quat_o, double* vel_o,
                     double* om_o, const double* drive_o, const OracleParams* pi, const double* rest_i,
                     double* pos_i, double* quat_i, double* vel_i, double* om_i, const double* drive_i, int mode,
                     double beta, int n_steps) {
  if (!valid(po) || !valid(pi) || mode < 0 || mode > 2 || n_steps < 0) return -1;
  if (!po->inextensible || !pi->inextensible || po->n_iters != pi->n_iters || po->dt != pi->dt) return -1;
  Derived dout = derive(*po), din = derive(*pi);
  if (std::fabs(dout.l0 - din.l0) > 1e-12 * dout.l0) return -1;
  Material<double> mo, mi;
  load_material(dout, rest_o, nullptr, mo);
  load_material(din, rest_i, nullptr, mi);
  State<double> so, si;
  load_state(dout, pos_o, quat_o, vel_o, om_o, so);
  load_state(din, pos_i, quat_i, vel_i, om_i, si);
  for (int k = 0; k < n_steps; ++k) step_pair(*po, dout, mo, so, drive_o, *pi, din, mi, si, drive_i, mode, beta);
  store_state(dout, so, pos_o, quat_o, vel_o, om_o);
  store_state(din, si, pos_i, quat_i, vel_i, om_i);
  return 0;
}

// Floating-point operations of n_steps steps of this rod (counted, not estimated).
int64_t oracle_count_flops(const OracleParams* p, const double* rest_quat, const double* pos, const double* quat,
                           int n_steps) {
  if (!valid(p) || !pos || !quat) return -1;
  Derived d = derive(*p);
  Material<Counted> mat;
  load_material(d, rest_quat, nullptr, mat);
  State<Counted> s;
  load_state(d, pos, quat, nullptr, nullptr, s);
  double drive[8] = {0};
  g_flops = 0;
  for (int k = 0; k < n_steps; ++k) step(*p, d, mat, s, drive, nullptr, nullptr);
  return (int64_t)g_flops;
}

// Many independent rods (concatenated arrays, node offsets from params[r].n_nodes,
// frame offsets from n_nodes - 1) stepped n_steps each; OpenMP over rods when built
// with it.  Returns the number of threads used.
int oracle_step_batch(int n_rods, const OracleParams* params, const double* rest_quat, double* pos, double* quat,
                      double* vel, double* omega, int n_steps) {
  if (n_rods < 0 || !params) return -1;
  std::vector<size_t> no(n_rods + 1, 0), fo(n_rods + 1, 0);
  for (int r = 0; r < n_rods; ++r) {
    if (!valid(&params[r])) return -1;
    no[r + 1] = no[r] + params[r].n_nodes;
    fo[r + 1] = fo[r] + params[r].n_nodes - 1;
  }
  int threads = 1;
#ifdef _OPENMP
#pragma omp parallel
  {
#pragma omp single
    threads = omp_get_num_threads();
  }
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int r = 0; r < n_rods; ++r) {
    oracle_step(&params[r], rest_quat ? rest_quat + 4 * fo[r] : nullptr, nullptr, pos + 3 * no[r], quat + 4 * fo[r],
                vel + 3 * no[r], omega + 3 * fo[r], nullptr, nullptr, nullptr, n_steps);
  }
  return threads;
}

}  // extern "C"
