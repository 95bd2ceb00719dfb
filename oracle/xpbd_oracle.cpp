/*
 * FP64 CPU oracle of the differentiable XPBD step (DiffXPBD, Stuyck & Chen).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg load it.  It shares no code
 * with the CUDA library (no headers, helpers or generated tables).
 *
 * What it computes, in the paper's order:
 *   forward step (Sec. 3.1, Eq. xpbdUpdateRule):
 *     p = x_n + dt v_n + dt^2 M^-1 f_ext                         (inertial prediction)
 *     lambda = 0; contact set detected at p                      (Sec. 4.6 collisions)
 *     for each iteration, for each color in input order, for each constraint j of the
 *     color: the XPBD multiplier update of Eq. xpbd solved for that one constraint
 *       (grad C^T M^-1 grad C + alpha~) dlambda = -C - alpha~ lambda,  alpha~ = alpha/dt^2
 *     followed by dx = M^-1 grad C dlambda; then one collision pass over the contacts.
 *     v_{n+1} = (x_{n+1} - x_n) / dt
 *   reverse sweep: the exact reverse-mode derivative of that program (the adjoint states
 *     of Eq. adjointRule / Eq. rawAdjoint in discrete form) giving dL/dalpha, dL/dx0,
 *     dL/dv0, dL/dG_n (per-step global force), dL/dW (per-vertex force) and dL/d(plane h,
 *     sphere centre, sphere radius) (Eq. gradientRule, Sec. 5.5-5.6).
 *   tangent mode: the same forward program run on dual numbers (exact directional
 *     derivative, independent of the reverse sweep).
 *
 * Constraints are defined only by their function C(x); every derivative (gradient and
 * Hessian-vector product) is taken by forward-mode automatic differentiation of that
 * definition, never by a hand-derived formula:
 *   distance  C = |x_a - x_b| - L                                 (springs, Sec. 4.6)
 *   bending   C = theta - theta0, theta the signed dihedral angle atan2 form (Sec. 5.1)
 *   tet       C_H = det F - gamma,  C_D = sqrt(tr F^T F)          (Sec. 5.2)
 *   plane     C = y - h - thickness;  sphere  C = |x - c| - r - thickness   (Sec. 4.6)
 *   membrane  C = (E_uu, E_vv, 2 E_uv), E = (F^T F - I)/2 the Green strain of a triangle,
 *             F = Ds Dm^-1 (3x2) from the warp/weft (u, v) rest coordinates, with the 3x3
 *             compliance block (A K)^-1, K = [C00 C01 .; C01 C11 .; . . C22]
 *             (Sec. "Cloth Material Parameter Estimation", orthotropic StVK); its three
 *             multipliers are solved together (3x3 system)
 * Readings where the paper is silent (lambda reset per step, Gauss-Seidel over colors,
 * contact set fixed per step at the predicted positions, degenerate-constraint skip) are
 * listed in the design notes of the repository.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ------------------------------------------------------------------ dual numbers
template <class T>
struct Dual {
  T v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double c) : v(c), d(0.0) {}
  Dual(const T& a, const T& b) : v(a), d(b) {}
};

inline double val(double a) { return a; }
template <class T> inline double val(const Dual<T>& a) { return val(a.v); }

template <class T> Dual<T> operator+(const Dual<T>& a, const Dual<T>& b) { return {a.v + b.v, a.d + b.d}; }
template <class T> Dual<T> operator-(const Dual<T>& a, const Dual<T>& b) { return {a.v - b.v, a.d - b.d}; }
template <class T> Dual<T> operator-(const Dual<T>& a) { return {-a.v, -a.d}; }
template <class T> Dual<T> operator*(const Dual<T>& a, const Dual<T>& b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
template <class T> Dual<T> operator/(const Dual<T>& a, const Dual<T>& b) {
  T q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
template <class T> Dual<T> operator+(const Dual<T>& a, double b) { return {a.v + b, a.d}; }
template <class T> Dual<T> operator+(double a, const Dual<T>& b) { return {a + b.v, b.d}; }
template <class T> Dual<T> operator-(const Dual<T>& a, double b) { return {a.v - b, a.d}; }
template <class T> Dual<T> operator-(double a, const Dual<T>& b) { return {a - b.v, -b.d}; }
template <class T> Dual<T> operator*(const Dual<T>& a, double b) { return {a.v * b, a.d * b}; }
template <class T> Dual<T> operator*(double a, const Dual<T>& b) { return {a * b.v, a * b.d}; }
template <class T> Dual<T> operator/(const Dual<T>& a, double b) { return {a.v / b, a.d / b}; }
template <class T> Dual<T> operator/(double a, const Dual<T>& b) { return Dual<T>(a) / b; }
template <class T> Dual<T>& operator+=(Dual<T>& a, const Dual<T>& b) { a = a + b; return a; }
template <class T> Dual<T>& operator-=(Dual<T>& a, const Dual<T>& b) { a = a - b; return a; }

using std::atan2;
using std::sqrt;
template <class T> Dual<T> sqrt(const Dual<T>& a) {
  T s = sqrt(a.v);
  return {s, a.d / (2.0 * s)};
}
// d atan2(y, x) = (x dy - y dx) / (x^2 + y^2)
template <class T> Dual<T> atan2(const Dual<T>& y, const Dual<T>& x) {
  return {atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / (x.v * x.v + y.v * y.v)};
}

template <class S> struct V3 { S x, y, z; };
template <class S> V3<S> sub(const V3<S>& a, const V3<S>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class S> S dot(const V3<S>& a, const V3<S>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class S> V3<S> cross(const V3<S>& a, const V3<S>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class S> V3<S> load3(const S* p) { return {p[0], p[1], p[2]}; }

const double kPi = 3.14159265358979323846;

// FP32-rounding emulation (off by default): when on, every position, velocity and
// multiplier the FP64 forward program produces is rounded to the nearest float, as the
// float32 GPU state is.  Comparing the two FP64 runs measures how far float32 state
// rounding alone moves a result: the attainable agreement between a float32 and a
// float64 implementation.  It changes nothing when off.
bool g_round32 = false;

template <class T>
inline void round32(T& v) {
  if constexpr (std::is_same<T, double>::value) {
    if (g_round32) v = (double)(float)v;
  }
}

// ------------------------------------------------------------------ constraint definitions
enum Kind { K_DIST = 0, K_BEND = 1, K_TETH = 2, K_TETD = 3, K_PLANE = 4, K_SPHERE = 5,
            K_MEMB0 = 6, K_MEMB1 = 7, K_MEMB2 = 8 };   // membrane components E_uu, E_vv, 2 E_uv

// Constant (non-differentiated) rest data of one constraint.
struct Rest {
  double L = 0.0;        // distance rest length
  double theta0 = 0.0;   // bending rest angle
  double B[9] = {0};     // tet Dm^-1, row-major (membrane: the 2x2 Dm^-1 in B[0..3])
  double gamma = 1.0;    // tet hydrostatic rest offset
  double vol = 0.0;      // tet rest volume (membrane: rest area)
  double thickness = 0.0;
};

// Number of differentiated inputs of each kind: vertex coordinates, then collider
// parameters (plane: h; sphere: cx, cy, cz, r) which the projection does not move.
inline int n_inputs(int kind) {
  switch (kind) {
    case K_DIST: return 6;
    case K_BEND: case K_TETH: case K_TETD: return 12;
    case K_PLANE: return 4;
    case K_SPHERE: return 7;
    case K_MEMB0: case K_MEMB1: case K_MEMB2: return 9;
  }
  return 0;
}
inline int n_verts(int kind) {
  switch (kind) {
    case K_DIST: return 2;
    case K_BEND: case K_TETH: case K_TETD: return 4;
    case K_MEMB0: case K_MEMB1: case K_MEMB2: return 3;
    default: return 1;
  }
}

// C(x) for every kind, on any scalar type.
template <class S>
S constraint_C(int kind, const S* q, const Rest& r) {
  switch (kind) {
    case K_DIST: {
      V3<S> d = sub(load3(q), load3(q + 3));
      return sqrt(dot(d, d)) - r.L;
    }
    case K_BEND: {
      // signed dihedral angle about the hinge edge e = x1 - x0 between the triangle
      // normals nA = e x (x2 - x0) and nB = (x3 - x0) x e; theta = 0 for a flat hinge.
      V3<S> x0 = load3(q), x1 = load3(q + 3), x2 = load3(q + 6), x3 = load3(q + 9);
      V3<S> e = sub(x1, x0);
      V3<S> nA = cross(e, sub(x2, x0));
      V3<S> nB = cross(sub(x3, x0), e);
      S sn = dot(cross(nA, nB), e) / sqrt(dot(e, e));
      S cs = dot(nA, nB);
      S c = atan2(sn, cs) - r.theta0;
      if (val(c) > kPi) c = c - 2.0 * kPi;
      if (val(c) <= -kPi) c = c + 2.0 * kPi;
      return c;
    }
    case K_TETH:
    case K_TETD: {
      // F = Ds Dm^-1, Ds = [x1-x0, x2-x0, x3-x0] as columns
      S Ds[9];
      for (int c = 0; c < 3; ++c)
        for (int row = 0; row < 3; ++row) Ds[row * 3 + c] = q[3 * (c + 1) + row] - q[row];
      S F[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          S s = Ds[i * 3 + 0] * r.B[0 * 3 + j];
          s = s + Ds[i * 3 + 1] * r.B[1 * 3 + j];
          s = s + Ds[i * 3 + 2] * r.B[2 * 3 + j];
          F[i * 3 + j] = s;
        }
      if (kind == K_TETH) {
        S det = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                F[2] * (F[3] * F[7] - F[4] * F[6]);
        return det - r.gamma;
      }
      S ss = F[0] * F[0];
      for (int i = 1; i < 9; ++i) ss = ss + F[i] * F[i];
      return sqrt(ss);
    }
    case K_PLANE:
      return q[1] - q[3] - r.thickness;
    case K_SPHERE: {
      V3<S> d = sub(load3(q), load3(q + 3));
      return sqrt(dot(d, d)) - q[6] - r.thickness;
    }
    case K_MEMB0:
    case K_MEMB1:
    case K_MEMB2: {
      // F = [x1-x0, x2-x0] Dm^-1 (3x2); columns f_u, f_v; Green strain E = (F^T F - I)/2
      V3<S> x0 = load3(q), d1 = sub(load3(q + 3), x0), d2 = sub(load3(q + 6), x0);
      V3<S> fu = {d1.x * r.B[0] + d2.x * r.B[2], d1.y * r.B[0] + d2.y * r.B[2], d1.z * r.B[0] + d2.z * r.B[2]};
      V3<S> fv = {d1.x * r.B[1] + d2.x * r.B[3], d1.y * r.B[1] + d2.y * r.B[3], d1.z * r.B[1] + d2.z * r.B[3]};
      if (kind == K_MEMB0) return 0.5 * (dot(fu, fu) - 1.0);
      if (kind == K_MEMB1) return 0.5 * (dot(fv, fv) - 1.0);
      return dot(fu, fv);
    }
  }
  return S(0.0);
}

// A constraint is skipped when it is degenerate at the current positions (the paper is
// silent; the skip keeps the update finite): zero-length spring, collapsed hinge
// triangle or edge, vanishing deformation gradient for C_D.
template <class S>
bool degenerate(int kind, const S* q, const Rest& r) {
  const double eps = 1e-12;
  switch (kind) {
    case K_DIST: case K_SPHERE: {
      double d0 = val(q[0]) - val(q[3]), d1 = val(q[1]) - val(q[4]), d2 = val(q[2]) - val(q[5]);
      return std::sqrt(d0 * d0 + d1 * d1 + d2 * d2) < eps;
    }
    case K_BEND: {
      V3<double> x0{val(q[0]), val(q[1]), val(q[2])}, x1{val(q[3]), val(q[4]), val(q[5])};
      V3<double> x2{val(q[6]), val(q[7]), val(q[8])}, x3{val(q[9]), val(q[10]), val(q[11])};
      V3<double> e = sub(x1, x0);
      V3<double> nA = cross(e, sub(x2, x0)), nB = cross(sub(x3, x0), e);
      return std::sqrt(dot(e, e)) < eps || std::sqrt(dot(nA, nA)) < eps ||
             std::sqrt(dot(nB, nB)) < eps;
    }
    case K_TETD: {
      double v = val(constraint_C<S>(kind, q, r));
      return v < eps;
    }
    default:
      return false;
  }
}

// Gradient of C by forward-mode AD: one dual evaluation per input.
template <class T>
void constraint_grad(int kind, const T* q, const Rest& r, T* g) {
  int n = n_inputs(kind);
  Dual<T> qd[12];
  for (int k = 0; k < n; ++k) {
    for (int i = 0; i < n; ++i) qd[i] = Dual<T>(q[i], T(i == k ? 1.0 : 0.0));
    g[k] = constraint_C<Dual<T>>(kind, qd, r).d;
  }
}

// Hessian-vector product (d^2 C/dq^2) u by nested forward-mode AD: the outer seed picks
// the row k, the inner seed is the direction u.
void constraint_hvp(int kind, const double* q, const Rest& r, const double* u, double* hu) {
  int n = n_inputs(kind);
  using DD = Dual<Dual<double>>;
  DD qd[12];
  for (int k = 0; k < n; ++k) {
    for (int i = 0; i < n; ++i)
      qd[i] = DD(Dual<double>(q[i], u[i]), Dual<double>(i == k ? 1.0 : 0.0, 0.0));
    hu[k] = constraint_C<DD>(kind, qd, r).d.d;
  }
}

// ------------------------------------------------------------------ model
struct Model {
  int V = 0;
  std::vector<double> rest_x, w;
  int nd = 0, nb = 0, nt = 0;
  std::vector<int> dist_idx, bend_idx, tet_idx;
  std::vector<double> tet_gamma;
  int K = 0;
  std::vector<int> offsets, order;
  std::vector<Rest> rest;   // per constraint id
  bool coupled = false;     // a tet's two constraints are projected together (its C_H id in the coloring)
  // membrane triangles: coloring ids m() + t; vertices, warp/weft rest coordinates, rest data
  int nm = 0;
  std::vector<int> memb_idx;      // [nm*3]
  std::vector<double> memb_uv;    // [nm*6] (u, v) of each triangle's three vertices
  std::vector<Rest> mrest;        // [nm] Dm^-1 in B[0..3], area in vol
  int m() const { return nd + nb + 2 * nt; }
  int kind(int j) const {
    if (j < nd) return K_DIST;
    if (j < nd + nb) return K_BEND;
    if (j < nd + nb + nt) return K_TETH;
    if (j < nd + nb + 2 * nt) return K_TETD;
    return K_MEMB0;
  }
  void verts(int j, int* out) const {
    if (j >= m()) { for (int i = 0; i < 3; ++i) out[i] = memb_idx[3 * (j - m()) + i]; return; }
    if (j < nd) { out[0] = dist_idx[2 * j]; out[1] = dist_idx[2 * j + 1]; return; }
    j -= nd;
    if (j < nb) { for (int i = 0; i < 4; ++i) out[i] = bend_idx[4 * j + i]; return; }
    j -= nb;
    int t = j % nt;
    for (int i = 0; i < 4; ++i) out[i] = tet_idx[4 * t + i];
  }
};

// Rest data from the rest positions: spring length, hinge angle (the bending constraint
// evaluated with theta0 = 0), Dm^-1 and |det Dm|/6.
void build_rest(Model& M) {
  M.rest.assign(M.m(), Rest());
  for (int j = 0; j < M.m(); ++j) {
    int k = M.kind(j);
    int vs[4];
    M.verts(j, vs);
    double q[12];
    for (int a = 0; a < n_verts(k); ++a)
      for (int c = 0; c < 3; ++c) q[3 * a + c] = M.rest_x[3 * vs[a] + c];
    Rest& r = M.rest[j];
    if (k == K_DIST) {
      Rest z;
      r.L = constraint_C<double>(K_DIST, q, z);
    } else if (k == K_BEND) {
      Rest z;
      r.theta0 = constraint_C<double>(K_BEND, q, z);
    } else {
      double Dm[9];
      for (int c = 0; c < 3; ++c)
        for (int row = 0; row < 3; ++row) Dm[row * 3 + c] = q[3 * (c + 1) + row] - q[row];
      double det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
                   Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
      // inverse by the adjugate
      r.B[0] = (Dm[4] * Dm[8] - Dm[5] * Dm[7]) / det;
      r.B[1] = (Dm[2] * Dm[7] - Dm[1] * Dm[8]) / det;
      r.B[2] = (Dm[1] * Dm[5] - Dm[2] * Dm[4]) / det;
      r.B[3] = (Dm[5] * Dm[6] - Dm[3] * Dm[8]) / det;
      r.B[4] = (Dm[0] * Dm[8] - Dm[2] * Dm[6]) / det;
      r.B[5] = (Dm[2] * Dm[3] - Dm[0] * Dm[5]) / det;
      r.B[6] = (Dm[3] * Dm[7] - Dm[4] * Dm[6]) / det;
      r.B[7] = (Dm[1] * Dm[6] - Dm[0] * Dm[7]) / det;
      r.B[8] = (Dm[0] * Dm[4] - Dm[1] * Dm[3]) / det;
      r.vol = std::fabs(det) / 6.0;
      int t = (j - M.nd - M.nb) % M.nt;
      r.gamma = M.tet_gamma.empty() ? 1.0 : M.tet_gamma[t];
    }
  }
}

// Membrane rest data from the warp/weft coordinates: Dm = [uv1 - uv0, uv2 - uv0] (columns),
// B = Dm^-1, area = |det Dm| / 2.
void build_memb_rest(Model& M) {
  M.mrest.assign(M.nm, Rest());
  for (int t = 0; t < M.nm; ++t) {
    const double* uv = &M.memb_uv[6 * (size_t)t];
    double a = uv[2] - uv[0], b = uv[4] - uv[0];   // first row (u) of Dm
    double c = uv[3] - uv[1], d = uv[5] - uv[1];   // second row (v)
    double det = a * d - b * c;
    Rest& r = M.mrest[t];
    r.B[0] = d / det;
    r.B[1] = -b / det;
    r.B[2] = -c / det;
    r.B[3] = a / det;
    r.vol = std::fabs(det) / 2.0;
  }
}

// ------------------------------------------------------------------ parameters (generic)
template <class T>
struct Params {
  double dt = 0.0;
  double g[3] = {0, 0, 0};
  std::vector<T> compliance;     // [m]
  std::vector<T> f_global;       // [steps*3] (may be empty)
  std::vector<T> f_vertex;       // [V*3]    (may be empty)
  std::vector<T> f_vertex_steps; // [steps*V*3] force on vertex i at step n (may be empty)
  int flags = 0;                 // bit0 plane, bit1 sphere
  T plane_h = T(0.0);
  T sphere[4] = {T(0.0), T(0.0), T(0.0), T(0.0)};
  double contact_alpha = 0.0;
  double thickness = 0.0;
  std::vector<T> memb_k;         // [nm*4] (C00, C11, C01, C22) per membrane triangle
};

// alpha~ = alpha / dt^2, with the tet compliance alpha = alpha_hat / V_e.
template <class T>
T alpha_tilde(const Model& M, const Params<T>& P, int j) {
  int k = M.kind(j);
  T a = P.compliance[j];
  if (k == K_TETH || k == K_TETD) a = a / M.rest[j].vol;
  return a / (P.dt * P.dt);
}

// The membrane's 3x3 alpha~ = (A K)^-1 / dt^2, row-major, from K = [C00 C01 0; C01 C11 0;
// 0 0 C22] of triangle t.
template <class T>
void memb_alpha_tilde(const Model& M, const Params<T>& P, int t, T* at) {
  const T c00 = P.memb_k[4 * (size_t)t + 0], c11 = P.memb_k[4 * (size_t)t + 1];
  const T c01 = P.memb_k[4 * (size_t)t + 2], c22 = P.memb_k[4 * (size_t)t + 3];
  const double s = 1.0 / (M.mrest[t].vol * P.dt * P.dt);
  const T det = c00 * c11 - c01 * c01;
  for (int i = 0; i < 9; ++i) at[i] = T(0.0);
  at[0] = s * c11 / det;
  at[1] = -(s * c01) / det;
  at[3] = at[1];
  at[4] = s * c00 / det;
  at[8] = s / c22;
}

// State of one solve: positions p [V*3], multipliers lambda [m], per-vertex contact
// multipliers and activity (plane, sphere), membrane multipliers [nm*3].
template <class T>
struct Work {
  std::vector<T> p, lam, lam_c;   // lam_c [V*2]
  std::vector<uint8_t> active;    // [V*2]
  std::vector<T> lam_m;           // [nm*3]
};

// Gather the differentiated inputs of constraint j (vertex coordinates) or of a contact.
template <class T>
int gather(const Model& M, int j, const std::vector<T>& p, T* q, int* vs) {
  int k = M.kind(j);
  M.verts(j, vs);
  for (int a = 0; a < n_verts(k); ++a)
    for (int c = 0; c < 3; ++c) q[3 * a + c] = p[3 * vs[a] + c];
  return k;
}

template <class T>
void contact_inputs(int kind, int i, const std::vector<T>& p, const Params<T>& P, T* q) {
  for (int c = 0; c < 3; ++c) q[c] = p[3 * i + c];
  if (kind == K_PLANE) {
    q[3] = P.plane_h;
  } else {
    for (int c = 0; c < 4; ++c) q[3 + c] = P.sphere[c];
  }
}

// One XPBD multiplier/position update of a single constraint (Eq. xpbd, the position
// update after it):  D = sum_i w_i |g_i|^2 + alpha~;  dlambda = (-C - alpha~ lambda) / D;
// lambda += dlambda;  x_i += w_i g_i dlambda.  Inputs beyond the vertices (collider
// parameters) carry w = 0.
template <class T>
void project_one(int kind, T* q, const double* wv, const Rest& r, T& lam, const T& at) {
  if (degenerate<T>(kind, q, r)) return;
  int n = n_inputs(kind);
  T g[12];
  constraint_grad<T>(kind, q, r, g);
  T C = constraint_C<T>(kind, q, r);
  T D = at;
  for (int a = 0; a < n_verts(kind); ++a)
    for (int c = 0; c < 3; ++c) D = D + wv[a] * g[3 * a + c] * g[3 * a + c];
  (void)n;
  if (!(val(D) > 0.0)) return;
  T dl = (-C - at * lam) / D;
  lam = lam + dl;
  round32(lam);
  for (int a = 0; a < n_verts(kind); ++a)
    for (int c = 0; c < 3; ++c) {
      q[3 * a + c] = q[3 * a + c] + wv[a] * g[3 * a + c] * dl;
      round32(q[3 * a + c]);
    }
}

// Coupled update of a tet's hydrostatic (h) and deviatoric (d) constraints, the
// formulation the paper's volumetric model follows (Macklin and Mueller 2021): both
// multipliers from one 2x2 system,
//   S dlambda = -C - A~ lambda,  S = G W G^T + A~ (G: the two gradients as rows),
// then x += W G^T dlambda.  When C_D is degenerate only C_H is projected.
template <class T>
void project_pair(T* q, const double* wv, const Rest& rh, const Rest& rd, T& lh, T& ld, const T& ath,
                  const T& atd) {
  if (degenerate<T>(K_TETD, q, rd)) {
    project_one<T>(K_TETH, q, wv, rh, lh, ath);
    return;
  }
  T gh[12], gd[12];
  constraint_grad<T>(K_TETH, q, rh, gh);
  constraint_grad<T>(K_TETD, q, rd, gd);
  const T Ch = constraint_C<T>(K_TETH, q, rh), Cd = constraint_C<T>(K_TETD, q, rd);
  T s11 = ath, s22 = atd, s12 = T(0.0);
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 3; ++c) {
      const int i = 3 * a + c;
      s11 = s11 + wv[a] * gh[i] * gh[i];
      s22 = s22 + wv[a] * gd[i] * gd[i];
      s12 = s12 + wv[a] * gh[i] * gd[i];
    }
  const T det = s11 * s22 - s12 * s12;
  if (!(val(det) > 0.0)) return;
  const T rhh = -Ch - ath * lh, rdd = -Cd - atd * ld;
  const T dlh = (s22 * rhh - s12 * rdd) / det, dld = (s11 * rdd - s12 * rhh) / det;
  lh = lh + dlh;
  ld = ld + dld;
  round32(lh);
  round32(ld);
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 3; ++c) {
      const int i = 3 * a + c;
      q[i] = q[i] + wv[a] * (gh[i] * dlh + gd[i] * dld);
      round32(q[i]);
    }
}

// Solve the 3x3 system S x = r by Cramer's rule (S symmetric positive definite here).
template <class T>
bool solve3(const T* S, const T* r, T* x) {
  const T c0 = S[4] * S[8] - S[5] * S[7], c1 = S[5] * S[6] - S[3] * S[8], c2 = S[3] * S[7] - S[4] * S[6];
  const T det = S[0] * c0 + S[1] * c1 + S[2] * c2;
  if (!(val(det) > 0.0)) return false;
  // x = adj(S) r / det
  x[0] = (c0 * r[0] + (S[2] * S[7] - S[1] * S[8]) * r[1] + (S[1] * S[5] - S[2] * S[4]) * r[2]) / det;
  x[1] = (c1 * r[0] + (S[0] * S[8] - S[2] * S[6]) * r[1] + (S[2] * S[3] - S[0] * S[5]) * r[2]) / det;
  x[2] = (c2 * r[0] + (S[1] * S[6] - S[0] * S[7]) * r[1] + (S[0] * S[4] - S[1] * S[3]) * r[2]) / det;
  return true;
}

// XPBD update of one membrane (Eq. xpbd for a vector constraint): the three multipliers
// from S dlambda = -C - A~ lambda with S = G W G^T + A~ (G: the three component gradients
// as rows), then x += W G^T dlambda.
template <class T>
void project_memb(T* q, const double* wv, const Rest& r, T* lam, const T* at) {
  T g[3][9], C[3];
  for (int k = 0; k < 3; ++k) {
    constraint_grad<T>(K_MEMB0 + k, q, r, g[k]);
    C[k] = constraint_C<T>(K_MEMB0 + k, q, r);
  }
  T S[9], rhs[3], dl[3];
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      T s = at[3 * k + l];
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) s = s + wv[a] * g[k][3 * a + c] * g[l][3 * a + c];
      S[3 * k + l] = s;
    }
  for (int k = 0; k < 3; ++k) rhs[k] = -C[k] - (at[3 * k] * lam[0] + at[3 * k + 1] * lam[1] + at[3 * k + 2] * lam[2]);
  if (!solve3(S, rhs, dl)) return;
  for (int k = 0; k < 3; ++k) {
    lam[k] = lam[k] + dl[k];
    round32(lam[k]);
  }
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      const int i = 3 * a + c;
      q[i] = q[i] + wv[a] * (g[0][i] * dl[0] + g[1][i] * dl[1] + g[2][i] * dl[2]);
      round32(q[i]);
    }
}

template <class T>
void project_constraint(const Model& M, const Params<T>& P, int j, Work<T>& W) {
  if (j >= M.m()) {   // membrane triangle
    const int t = j - M.m();
    T q[9], at[9];
    int vs[3];
    double wv[3];
    M.verts(j, vs);
    for (int a = 0; a < 3; ++a) {
      wv[a] = M.w[vs[a]];
      for (int c = 0; c < 3; ++c) q[3 * a + c] = W.p[3 * vs[a] + c];
    }
    memb_alpha_tilde(M, P, t, at);
    project_memb<T>(q, wv, M.mrest[t], &W.lam_m[3 * (size_t)t], at);
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) W.p[3 * vs[a] + c] = q[3 * a + c];
    return;
  }
  T q[12];
  int vs[4];
  int k = gather(M, j, W.p, q, vs);
  double wv[4];
  for (int a = 0; a < n_verts(k); ++a) wv[a] = M.w[vs[a]];
  T at = alpha_tilde(M, P, j);
  if (M.coupled && k == K_TETH) {
    const int jd = j + M.nt;
    project_pair<T>(q, wv, M.rest[j], M.rest[jd], W.lam[j], W.lam[jd], at, alpha_tilde(M, P, jd));
  } else {
    project_one<T>(k, q, wv, M.rest[j], W.lam[j], at);
  }
  for (int a = 0; a < n_verts(k); ++a)
    for (int c = 0; c < 3; ++c) W.p[3 * vs[a] + c] = q[3 * a + c];
}

template <class T>
void project_contact(const Model& M, const Params<T>& P, int i, int which, Work<T>& W) {
  int kind = which == 0 ? K_PLANE : K_SPHERE;
  T q[7];
  contact_inputs(kind, i, W.p, P, q);
  Rest r;
  r.thickness = P.thickness;
  double wv[1] = {M.w[i]};
  T at = T(P.contact_alpha / (P.dt * P.dt));
  project_one<T>(kind, q, wv, r, W.lam_c[2 * i + which], at);
  for (int c = 0; c < 3; ++c) W.p[3 * i + c] = q[c];
}

// Contact detection at the predicted positions: a contact is active for the whole step
// when its constraint is violated (C < 0) at p.
template <class T>
void detect_contacts(const Model& M, const Params<T>& P, Work<T>& W) {
  Rest r;
  r.thickness = P.thickness;
  for (int i = 0; i < M.V; ++i) {
    for (int which = 0; which < 2; ++which) {
      W.active[2 * i + which] = 0;
      if (!(P.flags & (1 << which))) continue;
      int kind = which == 0 ? K_PLANE : K_SPHERE;
      T q[7];
      contact_inputs(kind, i, W.p, P, q);
      W.active[2 * i + which] = val(constraint_C<T>(kind, q, r)) < 0.0 ? 1 : 0;
    }
  }
}

// Inertial prediction p = x + dt v + dt^2 w (m g + G_n + W_i + F_{n,i})  (Eq. xpbdUpdateRule).
// w m g = g for free vertices and 0 for pinned ones.  F_{n,i} is a force per vertex per step,
// the control variables of the keyframe example (Sec. "Keyframe Simulation").
template <class T>
void predict(const Model& M, const Params<T>& P, int n, const std::vector<T>& x,
             const std::vector<T>& v, std::vector<T>& p) {
  double dt = P.dt;
  for (int i = 0; i < M.V; ++i) {
    double w = M.w[i];
    for (int c = 0; c < 3; ++c) {
      T f = T(0.0);
      if (!P.f_global.empty()) f = f + P.f_global[3 * n + c];
      if (!P.f_vertex.empty()) f = f + P.f_vertex[3 * i + c];
      if (!P.f_vertex_steps.empty()) f = f + P.f_vertex_steps[3 * ((size_t)M.V * n + i) + c];
      T acc = w * f + (w > 0.0 ? P.g[c] : 0.0);
      p[3 * i + c] = x[3 * i + c] + dt * v[3 * i + c] + dt * dt * acc;
      round32(p[3 * i + c]);
    }
  }
}

template <class T>
void solve_iteration(const Model& M, const Params<T>& P, Work<T>& W) {
  for (int c = 0; c < M.K; ++c) {
    int b = M.offsets[c], e = M.offsets[c + 1];
    // constraints of one color share no vertex: they are independent
#pragma omp parallel for schedule(static) if (e - b >= 1024)
    for (int t = b; t < e; ++t) project_constraint(M, P, M.order[t], W);
  }
  if (P.flags) {
#pragma omp parallel for schedule(static) if (M.V > 4096)
    for (int i = 0; i < M.V; ++i) {
      if (W.active[2 * i + 0]) project_contact(M, P, i, 0, W);
      if (W.active[2 * i + 1]) project_contact(M, P, i, 1, W);
    }
  }
}

// Forward simulation over `steps` steps; xs/vs receive x_0..x_N and v_0..v_N.
template <class T>
void forward(const Model& M, const Params<T>& P, int steps, int iters, const std::vector<T>& x0,
             const std::vector<T>& v0, std::vector<T>& xs, std::vector<T>& vs,
             std::vector<T>* lam_steps = nullptr, std::vector<T>* lamc_steps = nullptr,
             std::vector<uint8_t>* active_steps = nullptr, std::vector<T>* lam_m_steps = nullptr) {
  size_t V3n = (size_t)M.V * 3;
  xs.assign(V3n * (steps + 1), T(0.0));
  vs.assign(V3n * (steps + 1), T(0.0));
  std::copy(x0.begin(), x0.end(), xs.begin());
  std::copy(v0.begin(), v0.end(), vs.begin());
  Work<T> W;
  W.p.assign(V3n, T(0.0));
  W.lam.assign(M.m(), T(0.0));
  W.lam_c.assign(2 * M.V, T(0.0));
  W.active.assign(2 * M.V, 0);
  W.lam_m.assign(3 * (size_t)M.nm, T(0.0));
  std::vector<T> x(V3n), v(V3n);
  for (int n = 0; n < steps; ++n) {
    std::copy(xs.begin() + V3n * n, xs.begin() + V3n * (n + 1), x.begin());
    std::copy(vs.begin() + V3n * n, vs.begin() + V3n * (n + 1), v.begin());
    predict(M, P, n, x, v, W.p);
    std::fill(W.lam.begin(), W.lam.end(), T(0.0));
    std::fill(W.lam_c.begin(), W.lam_c.end(), T(0.0));
    std::fill(W.lam_m.begin(), W.lam_m.end(), T(0.0));
    detect_contacts(M, P, W);
    for (int k = 0; k < iters; ++k) solve_iteration(M, P, W);
    // the multipliers and contact set the step ended with
    if (lam_steps) lam_steps->insert(lam_steps->end(), W.lam.begin(), W.lam.end());
    if (lamc_steps) lamc_steps->insert(lamc_steps->end(), W.lam_c.begin(), W.lam_c.end());
    if (active_steps) active_steps->insert(active_steps->end(), W.active.begin(), W.active.end());
    if (lam_m_steps) lam_m_steps->insert(lam_m_steps->end(), W.lam_m.begin(), W.lam_m.end());
    for (size_t i = 0; i < V3n; ++i) {
      xs[V3n * (n + 1) + i] = W.p[i];
      vs[V3n * (n + 1) + i] = (W.p[i] - x[i]) / P.dt;
      round32(vs[V3n * (n + 1) + i]);
    }
  }
}

// ------------------------------------------------------------------ reverse sweep
// Adjoint of one projection.  Pre-projection inputs q, lambda; post-projection adjoints
// qbar (in: adjoint of the updated inputs; out: adjoint of the inputs), lambar likewise;
// abar accumulates the adjoint of alpha~.  With g = grad C, D, dlambda recomputed:
//   s    = lambar' + sum_i w_i g_i . qbar'_i               (adjoint of dlambda)
//   u_i  = dlambda w_i qbar'_i - 2 (s dlambda / D) w_i g_i  (adjoint of g_i)
//   qbar = qbar' - (s/D) g + H u,   lambar = lambar' - (alpha~/D) s,
//   abar += -s (lambda + dlambda) / D.
void vjp_one(int kind, const double* q, const double* wv, const Rest& r, double lam, double at,
             double* qbar, double& lambar, double& abar) {
  if (degenerate<double>(kind, q, r)) return;
  int n = n_inputs(kind);
  double g[12];
  constraint_grad<double>(kind, q, r, g);
  double C = constraint_C<double>(kind, q, r);
  double D = at;
  for (int a = 0; a < n_verts(kind); ++a)
    for (int c = 0; c < 3; ++c) D += wv[a] * g[3 * a + c] * g[3 * a + c];
  if (!(D > 0.0)) return;
  double dl = (-C - at * lam) / D;
  double s = lambar;
  for (int a = 0; a < n_verts(kind); ++a)
    for (int c = 0; c < 3; ++c) s += wv[a] * g[3 * a + c] * qbar[3 * a + c];
  double u[12] = {0};
  for (int a = 0; a < n_verts(kind); ++a)
    for (int c = 0; c < 3; ++c)
      u[3 * a + c] = dl * wv[a] * qbar[3 * a + c] - 2.0 * (s * dl / D) * wv[a] * g[3 * a + c];
  double hu[12];
  constraint_hvp(kind, q, r, u, hu);
  for (int i = 0; i < n; ++i) qbar[i] += -(s / D) * g[i] + hu[i];
  abar += -s * (lam + dl) / D;
  lambar -= (at / D) * s;
}

// Adjoint of project_pair.  With S, dlambda recomputed and the adjoints qbar', lambar' of
// the updated values:  sbar = lambar' + G W qbar',  q = S^-1 sbar,
//   Gbar_k = dlambda_k W qbar' - sum_l (q_k dlambda_l + dlambda_k q_l) W g_l,
//   qbar = qbar' - sum_k q_k g_k + sum_k hess C_k Gbar_k,
//   lambar_k = lambar'_k - alpha~_k q_k,  alphabar~_k += -q_k (lambda_k + dlambda_k).
void vjp_pair(const double* q, const double* wv, const Rest& rh, const Rest& rd, double lh, double ld, double ath,
              double atd, double* qbar, double& lbh, double& lbd, double& abh, double& abd) {
  if (degenerate<double>(K_TETD, q, rd)) {
    vjp_one(K_TETH, q, wv, rh, lh, ath, qbar, lbh, abh);
    return;
  }
  double gh[12], gd[12];
  constraint_grad<double>(K_TETH, q, rh, gh);
  constraint_grad<double>(K_TETD, q, rd, gd);
  const double Ch = constraint_C<double>(K_TETH, q, rh), Cd = constraint_C<double>(K_TETD, q, rd);
  double s11 = ath, s22 = atd, s12 = 0.0;
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 3; ++c) {
      const int i = 3 * a + c;
      s11 += wv[a] * gh[i] * gh[i];
      s22 += wv[a] * gd[i] * gd[i];
      s12 += wv[a] * gh[i] * gd[i];
    }
  const double det = s11 * s22 - s12 * s12;
  if (!(det > 0.0)) return;
  const double rhh = -Ch - ath * lh, rdd = -Cd - atd * ld;
  const double dlh = (s22 * rhh - s12 * rdd) / det, dld = (s11 * rdd - s12 * rhh) / det;
  double sh = lbh, sd = lbd;
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 3; ++c) {
      const int i = 3 * a + c;
      sh += wv[a] * gh[i] * qbar[i];
      sd += wv[a] * gd[i] * qbar[i];
    }
  const double qh = (s22 * sh - s12 * sd) / det, qd = (s11 * sd - s12 * sh) / det;
  double uh[12], ud[12];
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 3; ++c) {
      const int i = 3 * a + c;
      uh[i] = dlh * wv[a] * qbar[i] - (2.0 * qh * dlh) * wv[a] * gh[i] - (qh * dld + dlh * qd) * wv[a] * gd[i];
      ud[i] = dld * wv[a] * qbar[i] - (qd * dlh + dld * qh) * wv[a] * gh[i] - (2.0 * qd * dld) * wv[a] * gd[i];
    }
  double huh[12], hud[12];
  constraint_hvp(K_TETH, q, rh, uh, huh);
  constraint_hvp(K_TETD, q, rd, ud, hud);
  for (int i = 0; i < 12; ++i) qbar[i] += -qh * gh[i] - qd * gd[i] + huh[i] + hud[i];
  abh += -qh * (lh + dlh);
  abd += -qd * (ld + dld);
  lbh -= ath * qh;
  lbd -= atd * qd;
}

// Adjoint of project_memb (3x3 generalisation of vjp_pair).  With S, dlambda recomputed:
//   sbar = lambar' + G W qbar',  q = S^-1 sbar,
//   Gbar_k = dlambda_k W qbar' - sum_l (q_k dlambda_l + dlambda_k q_l) W g_l,
//   qbar = qbar' - G^T q + sum_k H_k Gbar_k,  lambar = lambar' - A~ q,
//   Abar~ += -q (lambda + dlambda)^T, kept on the entries A~ depends on:
//   abar4 += (a00, a11, a01 + a10, a22).
void vjp_memb(const double* q, const double* wv, const Rest& r, const double* lam, const double* at,
              double* qbar, double* lambar, double* abar4) {
  double g[3][9], C[3];
  for (int k = 0; k < 3; ++k) {
    constraint_grad<double>(K_MEMB0 + k, q, r, g[k]);
    C[k] = constraint_C<double>(K_MEMB0 + k, q, r);
  }
  double S[9], rhs[3], dl[3];
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      double sv = at[3 * k + l];
      for (int i = 0; i < 9; ++i) sv += wv[i / 3] * g[k][i] * g[l][i];
      S[3 * k + l] = sv;
    }
  for (int k = 0; k < 3; ++k) rhs[k] = -C[k] - (at[3 * k] * lam[0] + at[3 * k + 1] * lam[1] + at[3 * k + 2] * lam[2]);
  if (!solve3(S, rhs, dl)) return;
  double sb[3], qv[3];
  for (int k = 0; k < 3; ++k) {
    sb[k] = lambar[k];
    for (int i = 0; i < 9; ++i) sb[k] += wv[i / 3] * g[k][i] * qbar[i];
  }
  solve3(S, sb, qv);   // S symmetric: S^-T = S^-1
  double out[9];
  for (int i = 0; i < 9; ++i) out[i] = qbar[i] - (g[0][i] * qv[0] + g[1][i] * qv[1] + g[2][i] * qv[2]);
  for (int k = 0; k < 3; ++k) {
    double u[9], hu[9];
    for (int i = 0; i < 9; ++i) {
      double t = dl[k] * wv[i / 3] * qbar[i];
      for (int l = 0; l < 3; ++l) t -= (qv[k] * dl[l] + dl[k] * qv[l]) * wv[i / 3] * g[l][i];
      u[i] = t;
    }
    constraint_hvp(K_MEMB0 + k, q, r, u, hu);
    for (int i = 0; i < 9; ++i) out[i] += hu[i];
  }
  for (int i = 0; i < 9; ++i) qbar[i] = out[i];
  double mm[3] = {lam[0] + dl[0], lam[1] + dl[1], lam[2] + dl[2]};
  abar4[0] += -qv[0] * mm[0];
  abar4[1] += -qv[1] * mm[1];
  abar4[2] += -(qv[0] * mm[1] + qv[1] * mm[0]);
  abar4[3] += -qv[2] * mm[2];
  for (int k = 0; k < 3; ++k) lambar[k] -= at[3 * k] * qv[0] + at[3 * k + 1] * qv[1] + at[3 * k + 2] * qv[2];
}

struct Grads {
  std::vector<double> d_memb;   // [nm*4] dL/d(C00, C11, C01, C22)
  std::vector<double> d_alpha, d_x0, d_v0, d_fg, d_fv, d_fvs;
  double d_coll[5] = {0, 0, 0, 0, 0};   // plane h, sphere cx, cy, cz, r
};

void adjoint(const Model& M, const Params<double>& P, int steps, int iters,
             const std::vector<double>& x0, const std::vector<double>& v0, int n_seed,
             const int* seed_steps, const double* seed_dx, const double* seed_dv_T, Grads& G) {
  size_t V3n = (size_t)M.V * 3;
  std::vector<double> xs, vs;
  forward(M, P, steps, iters, x0, v0, xs, vs);
  double dt = P.dt;
  std::vector<double> xbar(V3n, 0.0), vbar(V3n, 0.0);
  auto add_seed = [&](int n) {
    for (int s = 0; s < n_seed; ++s)
      if (seed_steps[s] == n)
        for (size_t i = 0; i < V3n; ++i) xbar[i] += seed_dx[V3n * s + i];
  };
  add_seed(steps);
  if (seed_dv_T)
    for (size_t i = 0; i < V3n; ++i) vbar[i] += seed_dv_T[i];
  G.d_alpha.assign(M.m(), 0.0);
  G.d_fg.assign(3 * (size_t)steps, 0.0);
  G.d_fv.assign(V3n, 0.0);
  G.d_fvs.assign(V3n * (size_t)steps, 0.0);
  std::vector<double> abar_t(M.m(), 0.0);   // adjoint of alpha~ (converted at the end)
  Work<double> W;
  W.p.assign(V3n, 0.0);
  W.lam.assign(M.m(), 0.0);
  W.lam_c.assign(2 * M.V, 0.0);
  W.active.assign(2 * M.V, 0);
  W.lam_m.assign(3 * (size_t)M.nm, 0.0);
  std::vector<double> lambar(M.m()), lambar_c(2 * M.V);
  std::vector<double> lambar_m(3 * (size_t)M.nm), abar_m(4 * (size_t)M.nm, 0.0), lam_before_m((size_t)iters * 3 * M.nm);
  // per-step replay records: positions before every color pass and before the
  // collision pass, multipliers before every iteration
  int passes = M.K + 1;
  std::vector<double> p_before((size_t)iters * passes * V3n);
  std::vector<double> lam_before((size_t)iters * M.m()), lamc_before((size_t)iters * 2 * M.V);
  std::vector<double> x(V3n), v(V3n), pbar(V3n);
  Rest cr;
  cr.thickness = P.thickness;
  double at_c = P.contact_alpha / (dt * dt);
  for (int n = steps - 1; n >= 0; --n) {
    // adjoint of v_{n+1} = (x_{n+1} - x_n)/dt with x_{n+1} = p
    for (size_t i = 0; i < V3n; ++i) {
      pbar[i] = xbar[i] + vbar[i] / dt;
      xbar[i] = -vbar[i] / dt;
    }
    // replay step n from its checkpoint
    std::copy(xs.begin() + V3n * n, xs.begin() + V3n * (n + 1), x.begin());
    std::copy(vs.begin() + V3n * n, vs.begin() + V3n * (n + 1), v.begin());
    predict(M, P, n, x, v, W.p);
    std::fill(W.lam.begin(), W.lam.end(), 0.0);
    std::fill(W.lam_c.begin(), W.lam_c.end(), 0.0);
    std::fill(W.lam_m.begin(), W.lam_m.end(), 0.0);
    detect_contacts(M, P, W);
    for (int k = 0; k < iters; ++k) {
      std::copy(W.lam.begin(), W.lam.end(), lam_before.begin() + (size_t)k * M.m());
      std::copy(W.lam_m.begin(), W.lam_m.end(), lam_before_m.begin() + (size_t)k * 3 * M.nm);
      std::copy(W.lam_c.begin(), W.lam_c.end(), lamc_before.begin() + (size_t)k * 2 * M.V);
      for (int c = 0; c < M.K; ++c) {
        std::copy(W.p.begin(), W.p.end(), p_before.begin() + ((size_t)k * passes + c) * V3n);
        int b = M.offsets[c], e = M.offsets[c + 1];
        for (int t = b; t < e; ++t) project_constraint(M, P, M.order[t], W);
      }
      std::copy(W.p.begin(), W.p.end(), p_before.begin() + ((size_t)k * passes + M.K) * V3n);
      if (P.flags)
        for (int i = 0; i < M.V; ++i) {
          if (W.active[2 * i + 0]) project_contact(M, P, i, 0, W);
          if (W.active[2 * i + 1]) project_contact(M, P, i, 1, W);
        }
    }
    // reverse the iterations
    std::fill(lambar.begin(), lambar.end(), 0.0);
    std::fill(lambar_c.begin(), lambar_c.end(), 0.0);
    std::fill(lambar_m.begin(), lambar_m.end(), 0.0);
    for (int k = iters - 1; k >= 0; --k) {
      if (P.flags) {
        const double* pb = &p_before[((size_t)k * passes + M.K) * V3n];
        for (int i = 0; i < M.V; ++i) {
          double lp = lamc_before[(size_t)k * 2 * M.V + 2 * i + 0];
          double ls = lamc_before[(size_t)k * 2 * M.V + 2 * i + 1];
          // pre-states: plane sees pb; sphere sees pb after the plane projection
          double q_plane[4] = {pb[3 * i], pb[3 * i + 1], pb[3 * i + 2], P.plane_h};
          double q_mid[3] = {pb[3 * i], pb[3 * i + 1], pb[3 * i + 2]};
          double wv[1] = {M.w[i]};
          if (W.active[2 * i + 0]) {
            double qq[4] = {q_plane[0], q_plane[1], q_plane[2], q_plane[3]};
            double l = lp;
            project_one<double>(K_PLANE, qq, wv, cr, l, at_c);
            q_mid[0] = qq[0]; q_mid[1] = qq[1]; q_mid[2] = qq[2];
          }
          double dummy = 0.0;
          if (W.active[2 * i + 1]) {
            double qs[7] = {q_mid[0], q_mid[1], q_mid[2], P.sphere[0], P.sphere[1], P.sphere[2], P.sphere[3]};
            double qb[7] = {pbar[3 * i], pbar[3 * i + 1], pbar[3 * i + 2], 0, 0, 0, 0};
            vjp_one(K_SPHERE, qs, wv, cr, ls, at_c, qb, lambar_c[2 * i + 1], dummy);
            for (int c = 0; c < 3; ++c) pbar[3 * i + c] = qb[c];
            for (int c = 0; c < 4; ++c) G.d_coll[1 + c] += qb[3 + c];
          }
          if (W.active[2 * i + 0]) {
            double qb[4] = {pbar[3 * i], pbar[3 * i + 1], pbar[3 * i + 2], 0};
            vjp_one(K_PLANE, q_plane, wv, cr, lp, at_c, qb, lambar_c[2 * i + 0], dummy);
            for (int c = 0; c < 3; ++c) pbar[3 * i + c] = qb[c];
            G.d_coll[0] += qb[3];
          }
        }
      }
      for (int c = M.K - 1; c >= 0; --c) {
        const double* pb = &p_before[((size_t)k * passes + c) * V3n];
        int b = M.offsets[c], e = M.offsets[c + 1];
        for (int t = b; t < e; ++t) {
          int j = M.order[t];
          if (j >= M.m()) {   // membrane triangle
            const int tm = j - M.m();
            int vs3[3];
            M.verts(j, vs3);
            double q[9], qb[9], wv[3], at[9];
            for (int a = 0; a < 3; ++a) {
              wv[a] = M.w[vs3[a]];
              for (int cc = 0; cc < 3; ++cc) {
                q[3 * a + cc] = pb[3 * vs3[a] + cc];
                qb[3 * a + cc] = pbar[3 * vs3[a] + cc];
              }
            }
            memb_alpha_tilde(M, P, tm, at);
            vjp_memb(q, wv, M.mrest[tm], &lam_before_m[(size_t)k * 3 * M.nm + 3 * (size_t)tm], at, qb,
                     &lambar_m[3 * (size_t)tm], &abar_m[4 * (size_t)tm]);
            for (int a = 0; a < 3; ++a)
              for (int cc = 0; cc < 3; ++cc) pbar[3 * vs3[a] + cc] = qb[3 * a + cc];
            continue;
          }
          int kind = M.kind(j);
          int vs4[4];
          M.verts(j, vs4);
          double q[12], qb[12], wv[4];
          for (int a = 0; a < n_verts(kind); ++a) {
            wv[a] = M.w[vs4[a]];
            for (int cc = 0; cc < 3; ++cc) {
              q[3 * a + cc] = pb[3 * vs4[a] + cc];
              qb[3 * a + cc] = pbar[3 * vs4[a] + cc];
            }
          }
          double at = alpha_tilde(M, P, j);
          if (M.coupled && kind == K_TETH) {
            const int jd = j + M.nt;
            vjp_pair(q, wv, M.rest[j], M.rest[jd], lam_before[(size_t)k * M.m() + j],
                     lam_before[(size_t)k * M.m() + jd], at, alpha_tilde(M, P, jd), qb, lambar[j], lambar[jd],
                     abar_t[j], abar_t[jd]);
          } else {
            vjp_one(kind, q, wv, M.rest[j], lam_before[(size_t)k * M.m() + j], at, qb, lambar[j],
                    abar_t[j]);
          }
          for (int a = 0; a < n_verts(kind); ++a)
            for (int cc = 0; cc < 3; ++cc) pbar[3 * vs4[a] + cc] = qb[3 * a + cc];
        }
      }
    }
    // adjoint of the prediction p = x + dt v + dt^2 w (G_n + W_i + F_{n,i}) + dt^2 [w>0] g
    for (int i = 0; i < M.V; ++i) {
      double w = M.w[i];
      for (int c = 0; c < 3; ++c) {
        double pb = pbar[3 * i + c];
        xbar[3 * i + c] += pb;
        vbar[3 * i + c] = dt * pb;
        double fb = dt * dt * w * pb;
        G.d_fg[3 * n + c] += fb;
        G.d_fv[3 * i + c] += fb;
        G.d_fvs[V3n * n + 3 * i + c] = fb;
      }
    }
    add_seed(n);
  }
  for (int j = 0; j < M.m(); ++j) {
    int k = M.kind(j);
    double scale = 1.0 / (dt * dt);
    if (k == K_TETH || k == K_TETD) scale /= M.rest[j].vol;
    G.d_alpha[j] = abar_t[j] * scale;
  }
  // membranes: chain rule from the entries of alpha~ to (C00, C11, C01, C22), the
  // derivative of memb_alpha_tilde taken by forward-mode AD, one parameter at a time
  G.d_memb.assign(4 * (size_t)M.nm, 0.0);
  {
    using D1 = Dual<double>;
    Params<D1> PD;
    PD.dt = P.dt;
    PD.memb_k.resize(P.memb_k.size());
    for (int t = 0; t < M.nm; ++t)
      for (int pi = 0; pi < 4; ++pi) {
        for (int qi = 0; qi < 4; ++qi)
          PD.memb_k[4 * (size_t)t + qi] = D1(P.memb_k[4 * (size_t)t + qi], qi == pi ? 1.0 : 0.0);
        D1 at[9];
        memb_alpha_tilde(M, PD, t, at);
        const double* ab = &abar_m[4 * (size_t)t];
        G.d_memb[4 * (size_t)t + pi] = ab[0] * at[0].d + ab[1] * at[4].d + ab[2] * at[1].d + ab[3] * at[8].d;
      }
  }
  G.d_x0 = xbar;
  G.d_v0 = vbar;
}

}  // namespace

// ======================================================================== C interface

typedef struct {
  int32_t V;
  const double* rest_x;     // [V*3]
  const double* inv_mass;   // [V]
  int32_t n_dist;
  const int32_t* dist_idx;  // [n_dist*2]
  int32_t n_bend;
  const int32_t* bend_idx;  // [n_bend*4]
  int32_t n_tet;
  const int32_t* tet_idx;   // [n_tet*4]
  const double* tet_gamma;  // [n_tet] or NULL (1.0)
  int32_t n_colors;
  const int32_t* color_offsets;   // [n_colors+1]
  const int32_t* color_order;     // [offsets[n_colors]]
  int32_t tet_coupled;            // 1: a tet's C_H and C_D are projected together; the
                                  // coloring then lists its C_H id only
  int32_t n_memb;                 // membrane triangles (coloring ids m + t)
  const int32_t* memb_idx;        // [n_memb*3]
  const double* memb_uv;          // [n_memb*6] warp/weft rest coordinates per triangle vertex
} om_model;

typedef struct {
  double dt;
  double gravity[3];
  const double* compliance;   // [m]
  const double* f_global;     // [steps*3] or NULL
  const double* f_vertex;     // [V*3] or NULL
  int32_t collider_flags;     // bit0 plane (y = h), bit1 sphere
  double plane_h;
  double sphere[4];           // cx, cy, cz, r
  double contact_compliance;
  double thickness;
  const double* f_vertex_steps;  // [steps*V*3] or NULL
  const double* memb_stiffness;  // [n_memb*4] (C00, C11, C01, C22) or NULL when n_memb = 0
} om_params;

typedef struct {              // tangent directions (NULL = zero)
  const double* d_compliance; // [m]
  const double* d_x0;         // [V*3]
  const double* d_v0;         // [V*3]
  const double* d_f_global;   // [steps*3]
  const double* d_f_vertex;   // [V*3]
  const double* d_collider;   // [5] plane h, cx, cy, cz, r
  const double* d_f_vertex_steps;  // [steps*V*3]
  const double* d_memb_stiffness;  // [n_memb*4]
} om_direction;

static Model make_model(const om_model* in) {
  Model M;
  M.V = in->V;
  M.rest_x.assign(in->rest_x, in->rest_x + 3 * (size_t)in->V);
  M.w.assign(in->inv_mass, in->inv_mass + in->V);
  M.nd = in->n_dist;
  M.nb = in->n_bend;
  M.nt = in->n_tet;
  if (M.nd) M.dist_idx.assign(in->dist_idx, in->dist_idx + 2 * (size_t)M.nd);
  if (M.nb) M.bend_idx.assign(in->bend_idx, in->bend_idx + 4 * (size_t)M.nb);
  if (M.nt) {
    M.tet_idx.assign(in->tet_idx, in->tet_idx + 4 * (size_t)M.nt);
    if (in->tet_gamma) M.tet_gamma.assign(in->tet_gamma, in->tet_gamma + M.nt);
  }
  M.K = in->n_colors;
  M.offsets.assign(in->color_offsets, in->color_offsets + M.K + 1);
  M.order.assign(in->color_order, in->color_order + M.offsets[M.K]);
  M.coupled = in->tet_coupled != 0;
  M.nm = in->n_memb;
  if (M.nm) {
    M.memb_idx.assign(in->memb_idx, in->memb_idx + 3 * (size_t)M.nm);
    M.memb_uv.assign(in->memb_uv, in->memb_uv + 6 * (size_t)M.nm);
  }
  build_rest(M);
  build_memb_rest(M);
  return M;
}

template <class T>
static Params<T> make_params(const Model& M, const om_params* in, int steps) {
  Params<T> P;
  P.dt = in->dt;
  for (int c = 0; c < 3; ++c) P.g[c] = in->gravity[c];
  P.compliance.assign(M.m(), T(0.0));
  for (int j = 0; j < M.m(); ++j) P.compliance[j] = T(in->compliance[j]);
  if (in->f_global) {
    P.f_global.resize(3 * (size_t)steps);
    for (size_t i = 0; i < P.f_global.size(); ++i) P.f_global[i] = T(in->f_global[i]);
  }
  if (in->f_vertex) {
    P.f_vertex.resize(3 * (size_t)M.V);
    for (size_t i = 0; i < P.f_vertex.size(); ++i) P.f_vertex[i] = T(in->f_vertex[i]);
  }
  if (in->f_vertex_steps) {
    P.f_vertex_steps.resize(3 * (size_t)M.V * steps);
    for (size_t i = 0; i < P.f_vertex_steps.size(); ++i) P.f_vertex_steps[i] = T(in->f_vertex_steps[i]);
  }
  P.flags = in->collider_flags;
  P.plane_h = T(in->plane_h);
  for (int c = 0; c < 4; ++c) P.sphere[c] = T(in->sphere[c]);
  P.contact_alpha = in->contact_compliance;
  P.thickness = in->thickness;
  P.memb_k.assign(4 * (size_t)M.nm, T(0.0));
  for (size_t i = 0; i < P.memb_k.size(); ++i) P.memb_k[i] = T(in->memb_stiffness[i]);
  return P;
}

extern "C" {

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Turn the FP32-rounding emulation on (1) or off (0); see g_round32.
void oracle_set_fp32_rounding(int on) { g_round32 = on != 0; }

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

// Rest data the oracle derives from the rest positions: per constraint id
// out[j*12 + 0..11] = (L, theta0, B[0..8], vol) (unused entries 0).
int oracle_rest_data(const om_model* in, double* out) {
  Model M = make_model(in);
  for (int j = 0; j < M.m(); ++j) {
    const Rest& r = M.rest[j];
    double* o = out + 12 * (size_t)j;
    o[0] = r.L;
    o[1] = r.theta0;
    for (int i = 0; i < 9; ++i) o[2 + i] = r.B[i];
    o[11] = r.vol;
  }
  return 0;
}

// Forward simulation: xs, vs receive [(steps+1)*V*3].
int oracle_forward(const om_model* in, const om_params* pin, int32_t steps, int32_t iters,
                   const double* x0, const double* v0, double* xs_out, double* vs_out) {
  Model M = make_model(in);
  Params<double> P = make_params<double>(M, pin, steps);
  std::vector<double> x(x0, x0 + 3 * (size_t)M.V), v(v0, v0 + 3 * (size_t)M.V), xs, vs;
  forward(M, P, steps, iters, x, v, xs, vs);
  std::copy(xs.begin(), xs.end(), xs_out);
  if (vs_out) std::copy(vs.begin(), vs.end(), vs_out);
  return 0;
}

// Forward simulation that also returns, per step, the multipliers the step ended with:
// lam_out [steps*m] (constraint id order), lamc_out [steps*V*2] (plane, sphere contact of
// each vertex) and active_out [steps*V*2] (1 where that contact was active).  Any output
// may be NULL.
int oracle_forward_multipliers(const om_model* in, const om_params* pin, int32_t steps, int32_t iters,
                               const double* x0, const double* v0, double* xs_out, double* vs_out,
                               double* lam_out, double* lamc_out, uint8_t* active_out) {
  Model M = make_model(in);
  Params<double> P = make_params<double>(M, pin, steps);
  std::vector<double> x(x0, x0 + 3 * (size_t)M.V), v(v0, v0 + 3 * (size_t)M.V), xs, vs, lam, lamc;
  std::vector<uint8_t> act;
  forward(M, P, steps, iters, x, v, xs, vs, &lam, &lamc, &act);
  if (xs_out) std::copy(xs.begin(), xs.end(), xs_out);
  if (vs_out) std::copy(vs.begin(), vs.end(), vs_out);
  if (lam_out) std::copy(lam.begin(), lam.end(), lam_out);
  if (lamc_out) std::copy(lamc.begin(), lamc.end(), lamc_out);
  if (active_out) std::copy(act.begin(), act.end(), active_out);
  return 0;
}

// The membranes' multipliers each step ended with: lam_m_out [steps*n_memb*3].
int oracle_forward_memb_multipliers(const om_model* in, const om_params* pin, int32_t steps, int32_t iters,
                                    const double* x0, const double* v0, double* lam_m_out) {
  Model M = make_model(in);
  Params<double> P = make_params<double>(M, pin, steps);
  std::vector<double> x(x0, x0 + 3 * (size_t)M.V), v(v0, v0 + 3 * (size_t)M.V), xs, vs, lm;
  forward<double>(M, P, steps, iters, x, v, xs, vs, nullptr, nullptr, nullptr, &lm);
  std::copy(lm.begin(), lm.end(), lam_m_out);
  return 0;
}

// Reverse sweep.  Seeds: dL/dx_n for n = seed_steps[s] in seed_dx[s*V*3..], and
// optionally dL/dv_N.  Outputs (NULL = not wanted): d_compliance [m], d_x0, d_v0 [V*3],
// d_f_global [steps*3], d_f_vertex [V*3], d_collider [5], d_f_vertex_steps [steps*V*3],
// d_memb_stiffness [n_memb*4].
int oracle_adjoint(const om_model* in, const om_params* pin, int32_t steps, int32_t iters,
                   const double* x0, const double* v0, int32_t n_seed, const int32_t* seed_steps,
                   const double* seed_dx, const double* seed_dv_T, double* d_compliance,
                   double* d_x0, double* d_v0, double* d_f_global, double* d_f_vertex,
                   double* d_collider, double* d_f_vertex_steps, double* d_memb_stiffness) {
  Model M = make_model(in);
  Params<double> P = make_params<double>(M, pin, steps);
  std::vector<double> x(x0, x0 + 3 * (size_t)M.V), v(v0, v0 + 3 * (size_t)M.V);
  std::vector<int> ss(seed_steps, seed_steps + n_seed);
  Grads G;
  adjoint(M, P, steps, iters, x, v, n_seed, ss.data(), seed_dx, seed_dv_T, G);
  if (d_compliance) std::copy(G.d_alpha.begin(), G.d_alpha.end(), d_compliance);
  if (d_x0) std::copy(G.d_x0.begin(), G.d_x0.end(), d_x0);
  if (d_v0) std::copy(G.d_v0.begin(), G.d_v0.end(), d_v0);
  if (d_f_global) std::copy(G.d_fg.begin(), G.d_fg.end(), d_f_global);
  if (d_f_vertex) std::copy(G.d_fv.begin(), G.d_fv.end(), d_f_vertex);
  if (d_collider) std::copy(G.d_coll, G.d_coll + 5, d_collider);
  if (d_f_vertex_steps) std::copy(G.d_fvs.begin(), G.d_fvs.end(), d_f_vertex_steps);
  if (d_memb_stiffness) std::copy(G.d_memb.begin(), G.d_memb.end(), d_memb_stiffness);
  return 0;
}

// Tangent (forward-mode) sweep along a parameter direction: dxs, dvs receive the exact
// directional derivative of x_0..x_N and v_0..v_N.
int oracle_tangent(const om_model* in, const om_params* pin, int32_t steps, int32_t iters,
                   const double* x0, const double* v0, const om_direction* dir, double* dxs_out,
                   double* dvs_out) {
  using D1 = Dual<double>;
  Model M = make_model(in);
  Params<D1> P = make_params<D1>(M, pin, steps);
  if (dir->d_compliance)
    for (int j = 0; j < M.m(); ++j) P.compliance[j].d = dir->d_compliance[j];
  if (dir->d_f_global) {
    if (P.f_global.empty()) P.f_global.assign(3 * (size_t)steps, D1(0.0));
    for (size_t i = 0; i < P.f_global.size(); ++i) P.f_global[i].d = dir->d_f_global[i];
  }
  if (dir->d_f_vertex) {
    if (P.f_vertex.empty()) P.f_vertex.assign(3 * (size_t)M.V, D1(0.0));
    for (size_t i = 0; i < P.f_vertex.size(); ++i) P.f_vertex[i].d = dir->d_f_vertex[i];
  }
  if (dir->d_f_vertex_steps) {
    if (P.f_vertex_steps.empty()) P.f_vertex_steps.assign(3 * (size_t)M.V * steps, D1(0.0));
    for (size_t i = 0; i < P.f_vertex_steps.size(); ++i) P.f_vertex_steps[i].d = dir->d_f_vertex_steps[i];
  }
  if (dir->d_collider) {
    P.plane_h.d = dir->d_collider[0];
    for (int c = 0; c < 4; ++c) P.sphere[c].d = dir->d_collider[1 + c];
  }
  if (dir->d_memb_stiffness)
    for (size_t i = 0; i < P.memb_k.size(); ++i) P.memb_k[i].d = dir->d_memb_stiffness[i];
  size_t V3n = 3 * (size_t)M.V;
  std::vector<D1> x(V3n), v(V3n), xs, vs;
  for (size_t i = 0; i < V3n; ++i) {
    x[i] = D1(x0[i], dir->d_x0 ? dir->d_x0[i] : 0.0);
    v[i] = D1(v0[i], dir->d_v0 ? dir->d_v0[i] : 0.0);
  }
  forward(M, P, steps, iters, x, v, xs, vs);
  for (size_t i = 0; i < xs.size(); ++i) {
    dxs_out[i] = xs[i].d;
    if (dvs_out) dvs_out[i] = vs[i].d;
  }
  return 0;
}

// One constraint in isolation: value, AD gradient and AD Hessian-vector product.
// kind: 0 distance, 1 bending, 2 tet C_H, 3 tet C_D, 4 plane, 5 sphere.  rest12 holds
// (L, theta0, B[9], gamma) and thickness comes from rest12[11] for contacts.
int oracle_constraint(int32_t kind, const double* q, const double* rest12, const double* u,
                      double* C_out, double* grad_out, double* hu_out) {
  Rest r;
  r.L = rest12[0];
  r.theta0 = rest12[1];
  for (int i = 0; i < 9; ++i) r.B[i] = rest12[2 + i];
  r.gamma = rest12[11];
  r.thickness = (kind == K_PLANE || kind == K_SPHERE) ? rest12[11] : 0.0;
  *C_out = constraint_C<double>(kind, q, r);
  if (grad_out) constraint_grad<double>(kind, q, r, grad_out);
  if (hu_out && u) constraint_hvp(kind, q, r, u, hu_out);
  return n_inputs(kind);
}

// One projection and its reverse, for unit tests of the per-constraint map.
// inputs q [n_inputs], w per vertex, lambda, alpha~; outputs the projected q and lambda.
int oracle_project_one(int32_t kind, double* q, const double* wv, const double* rest12,
                       double* lam, double at) {
  Rest r;
  r.L = rest12[0];
  r.theta0 = rest12[1];
  for (int i = 0; i < 9; ++i) r.B[i] = rest12[2 + i];
  r.gamma = rest12[11];
  r.thickness = (kind == K_PLANE || kind == K_SPHERE) ? rest12[11] : 0.0;
  project_one<double>(kind, q, wv, r, *lam, at);
  return 0;
}

int oracle_vjp_one(int32_t kind, const double* q, const double* wv, const double* rest12,
                   double lam, double at, double* qbar, double* lambar, double* abar) {
  Rest r;
  r.L = rest12[0];
  r.theta0 = rest12[1];
  for (int i = 0; i < 9; ++i) r.B[i] = rest12[2 + i];
  r.gamma = rest12[11];
  r.thickness = (kind == K_PLANE || kind == K_SPHERE) ? rest12[11] : 0.0;
  vjp_one(kind, q, wv, r, lam, at, qbar, *lambar, *abar);
  return 0;
}

// The coupled tet update and its reverse in isolation.  q [12] the tet's vertices,
// rest12 (B[9] at 2..10, gamma at 11) shared by both constraints, lam[2] and at[2] the
// (C_H, C_D) multipliers and alpha~; the reverse accumulates lambar[2] and abar[2].
int oracle_project_pair(double* q, const double* wv, const double* rest12, double* lam, const double* at) {
  Rest r;
  for (int i = 0; i < 9; ++i) r.B[i] = rest12[2 + i];
  r.gamma = rest12[11];
  project_pair<double>(q, wv, r, r, lam[0], lam[1], at[0], at[1]);
  return 0;
}

int oracle_vjp_pair(const double* q, const double* wv, const double* rest12, const double* lam, const double* at,
                    double* qbar, double* lambar, double* abar) {
  Rest r;
  for (int i = 0; i < 9; ++i) r.B[i] = rest12[2 + i];
  r.gamma = rest12[11];
  vjp_pair(q, wv, r, r, lam[0], lam[1], at[0], at[1], qbar, lambar[0], lambar[1], abar[0], abar[1]);
  return 0;
}

// One membrane update and its reverse in isolation.  q [9] the triangle's vertices,
// B2 the 2x2 Dm^-1 (row-major), at [9] the 3x3 alpha~ (row-major), lam [3]; the reverse
// accumulates lambar [3] and abar4 [4] (alpha~ entries 00, 11, 01 + 10, 22).
int oracle_project_memb(double* q, const double* wv, const double* B2, double* lam, const double* at) {
  Rest r;
  for (int i = 0; i < 4; ++i) r.B[i] = B2[i];
  project_memb<double>(q, wv, r, lam, at);
  return 0;
}

int oracle_vjp_memb(const double* q, const double* wv, const double* B2, const double* lam, const double* at,
                    double* qbar, double* lambar, double* abar4) {
  Rest r;
  for (int i = 0; i < 4; ++i) r.B[i] = B2[i];
  vjp_memb(q, wv, r, lam, at, qbar, lambar, abar4);
  return 0;
}

}  // extern "C"
