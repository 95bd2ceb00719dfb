// Per-constraint math of the XPBD step and of its reverse, in float32.
//
// Every function is __host__ __device__ so the same code runs in the kernels.  Gradients
// are analytic; Hessian-vector products (needed by the reverse of one update) are written
// out in closed form for the distance and bending constraints, and come from one
// forward-mode dual evaluation of the analytic gradient for tets.
//
// Constraint functions (Sec. 4.6, Sec. 5.1, Sec. 5.2 of DiffXPBD):
//   distance  C = |x_a - x_b| - L
//   bending   C = theta - theta0, theta = atan2(((nA x nB) . e)/|e|, nA . nB),
//             e = x1 - x0, nA = e x (x2 - x0), nB = (x3 - x0) x e   (wrapped to (-pi, pi])
//   tet       F = Ds Dm^-1, C_H = det F - gamma, C_D = ||F||_F
//   plane     C = y - h - thickness;  sphere  C = |x - c| - r - thickness
#pragma once

#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define XHD __host__ __device__ __forceinline__
#else
#define XHD inline
#endif

namespace xpbd {

// ------------------------------------------------------------------ scalar types
struct df {            // float dual number v + d eps
  float v, d;
  df() = default;
  XHD df(float v_, float d_ = 0.f) : v(v_), d(d_) {}
};
XHD df mkd(float v, float d = 0.f) { return df{v, d}; }
XHD df operator+(df a, df b) { return {a.v + b.v, a.d + b.d}; }
XHD df operator-(df a, df b) { return {a.v - b.v, a.d - b.d}; }
XHD df operator-(df a) { return {-a.v, -a.d}; }
XHD df operator*(df a, df b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
XHD df operator*(float a, df b) { return {a * b.v, a * b.d}; }
XHD df operator*(df a, float b) { return {a.v * b, a.d * b}; }
XHD df operator/(df a, df b) {
  float q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
XHD df operator+(df a, float b) { return {a.v + b, a.d}; }
XHD df operator-(df a, float b) { return {a.v - b, a.d}; }
XHD df sqrt_(df a) {
  float s = sqrtf(a.v);
  return {s, a.d / (2.f * s)};
}
XHD float sqrt_(float a) { return sqrtf(a); }
XHD float val(float a) { return a; }
XHD float val(df a) { return a.v; }
XHD df inv_(df a) {
  float r = 1.f / a.v;
  return {r, -a.d * r * r};
}
XHD float inv_(float a) { return 1.f / a; }

template <class S>
struct v3 {
  S x, y, z;
};
template <class S> XHD v3<S> operator+(v3<S> a, v3<S> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class S> XHD v3<S> operator-(v3<S> a, v3<S> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class S> XHD v3<S> operator-(v3<S> a) { return {-a.x, -a.y, -a.z}; }
template <class S> XHD v3<S> operator*(S s, v3<S> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class S> XHD v3<S> operator*(v3<S> a, S s) { return {a.x * s, a.y * s, a.z * s}; }
template <class S> XHD S dot(v3<S> a, v3<S> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class S> XHD v3<S> cross(v3<S> a, v3<S> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
typedef v3<float> f3;
typedef v3<df> d3;
XHD d3 mkd3(f3 v, f3 d) { return {mkd(v.x, d.x), mkd(v.y, d.y), mkd(v.z, d.z)}; }
XHD f3 dpart(d3 a) { return {a.x.d, a.y.d, a.z.d}; }
XHD f3 vpart(d3 a) { return {a.x.v, a.y.v, a.z.v}; }
XHD f3 mk3(float x, float y, float z) { return {x, y, z}; }

// Squared-length threshold below which a constraint is treated as degenerate and skipped
// (zero-length spring, collapsed hinge triangle or edge, vanishing F for C_D): lengths
// under 1e-12 m.
#define XPBD_DEGEN2 1e-24f

constexpr float kPi = 3.14159265358979323846f;

// ------------------------------------------------------------------ records
// Constraint records as stored on the device, grouped by color.  `at` is alpha~ =
// alpha / dt^2 (tets: alpha_hat / (V_e dt^2)), written at the start of every call.
struct __align__(16) DistRec {
  int a, b;
  float L, at;
};
struct __align__(16) BendRec {
  int v[4];
  float theta0, at, pad0, pad1;
};
struct __align__(16) TetRec {
  int v[4];
  float B[9];     // Dm^-1 row-major
  float at, gamma, vol;
};
// Orthotropic StVK membrane triangle: vertices, Dm^-1 (2x2, row-major) of the warp/weft
// rest coordinates, rest area, and the entries of its 3x3 alpha~ = (A K)^-1 / dt^2 that K
// reaches (00, 11, 01 = 10, 22; the others are 0).
struct __align__(16) MembRec {
  int v[3];
  float B[4];
  float A;
  float a00, a11, a01, a22;
};
// The phase kernels keep their bending records as two arrays: the four vertex indices
// (int4) and this tail (rest angle, alpha~), 24 bytes per record instead of 32, staged as
// two contiguous blocks (16-byte and 8-byte reads per thread, free of bank conflicts).
struct __align__(8) BendTail {
  float theta0, at;
};
static_assert(sizeof(MembRec) == 48, "MembRec");
static_assert(sizeof(DistRec) == 16, "DistRec");
static_assert(sizeof(BendRec) == 32, "BendRec");
static_assert(sizeof(TetRec) == 64, "TetRec");

// ------------------------------------------------------------------ bending
// Gradient of the signed dihedral angle (Bridson et al. 2003 form, sign matched to the
// atan2 convention above): with qA = nA/|nA|^2, qB = nB/|nB|^2,
//   g2 = -|e| qA,  g3 = -|e| qB,
//   g0 = -(((x2-x1).e) qA + ((x3-x1).e) qB)/|e|,  g1 = (((x2-x0).e) qA + ((x3-x0).e) qB)/|e|.
template <class S>
XHD void bend_grad(const v3<S> x[4], v3<S> g[4]) {
  v3<S> e = x[1] - x[0];
  v3<S> a = x[2] - x[0];
  v3<S> b = x[3] - x[0];
  v3<S> nA = cross(e, a);
  v3<S> nB = cross(b, e);
  S le = sqrt_(dot(e, e));
  S ile = inv_(le);
  v3<S> qA = nA * inv_(dot(nA, nA));
  v3<S> qB = nB * inv_(dot(nB, nB));
  g[2] = -(le * qA);
  g[3] = -(le * qB);
  S tA1 = dot(x[2] - x[1], e) * ile, tB1 = dot(x[3] - x[1], e) * ile;
  S tA0 = dot(a, e) * ile, tB0 = dot(b, e) * ile;
  g[0] = -(tA1 * qA + tB1 * qB);
  g[1] = tA0 * qA + tB0 * qB;
}

// The same gradient in relative coordinates e = x1 - x0, a = x2 - x0, b = x3 - x0 (the
// constraint is translation invariant): returns g1, g2, g3; g0 = -(g1 + g2 + g3).  With
// dual inputs whose derivative parts are u_k - u_0, the derivative parts of the result are
// (H u)_1..3, and (H u)_0 = -((H u)_1 + (H u)_2 + (H u)_3) (rows of H sum to zero).
template <class S>
XHD void bend_grad_rel(const v3<S>& e, const v3<S>& a, const v3<S>& b, v3<S>& g1, v3<S>& g2,
                       v3<S>& g3) {
  v3<S> nA = cross(e, a);
  v3<S> nB = cross(b, e);
  S le = sqrt_(dot(e, e));
  S ile = inv_(le);
  v3<S> qA = nA * inv_(dot(nA, nA));
  v3<S> qB = nB * inv_(dot(nB, nB));
  g2 = -(le * qA);
  g3 = -(le * qB);
  g1 = (dot(a, e) * ile) * qA + (dot(b, e) * ile) * qB;
}

// Hessian-vector product of the signed dihedral angle in the same relative coordinates:
// the directional derivative of (g1, g2, g3) = bend_grad_rel(e, a, b) along (de, da, db),
// written out by the chain rule (no dual numbers).  With nA = e x a, nB = b x e,
// qA = nA/|nA|^2, cA = (a.e)/|e| (likewise B):
//   dnA = de x a + e x da,              dnB = db x e + b x de
//   dqA = dnA/|nA|^2 - 2 (qA.dnA) qA,   d|e| = (e.de)/|e|
//   dcA = ((da.e) + (a.de) - cA d|e|)/|e|
//   dg1 = dcA qA + cA dqA + dcB qB + cB dqB,   dg2 = -(d|e| qA + |e| dqA),   dg3 likewise.
XHD void bend_hvp_rel(const f3& e, const f3& a, const f3& b, const f3& de, const f3& da, const f3& db, f3& h1,
                      f3& h2, f3& h3) {
  const f3 nA = cross(e, a);
  const f3 nB = cross(b, e);
  const float iA = 1.f / dot(nA, nA), iB = 1.f / dot(nB, nB);
  const f3 qA = nA * iA, qB = nB * iB;
  const float le = sqrtf(dot(e, e));
  const float ile = 1.f / le;
  const float cA = dot(a, e) * ile, cB = dot(b, e) * ile;
  const f3 dnA = cross(de, a) + cross(e, da);
  const f3 dnB = cross(db, e) + cross(b, de);
  const f3 dqA = dnA * iA - qA * (2.f * dot(qA, dnA));
  const f3 dqB = dnB * iB - qB * (2.f * dot(qB, dnB));
  const float dle = dot(e, de) * ile;
  const float dcA = (dot(da, e) + dot(a, de) - cA * dle) * ile;
  const float dcB = (dot(db, e) + dot(b, de) - cB * dle) * ile;
  h1 = qA * dcA + dqA * cA + qB * dcB + dqB * cB;
  h2 = -(qA * dle + dqA * le);
  h3 = -(qB * dle + dqB * le);
}

XHD bool bend_degenerate_rel(const f3& e, const f3& a, const f3& b) {
  f3 nA = cross(e, a);
  f3 nB = cross(b, e);
  return dot(e, e) < XPBD_DEGEN2 || dot(nA, nA) < XPBD_DEGEN2 || dot(nB, nB) < XPBD_DEGEN2;
}

XHD float bend_C_rel(const f3& e, const f3& a, const f3& b, float theta0) {
  f3 nA = cross(e, a);
  f3 nB = cross(b, e);
  float sn = dot(cross(nA, nB), e) * (1.f / sqrtf(dot(e, e)));
  float cs = dot(nA, nB);
  float c = atan2f(sn, cs) - theta0;
  if (c > kPi) c -= 2.f * kPi;
  if (c <= -kPi) c += 2.f * kPi;
  return c;
}

XHD bool bend_degenerate(const f3 x[4]) {
  f3 e = x[1] - x[0];
  f3 nA = cross(e, x[2] - x[0]);
  f3 nB = cross(x[3] - x[0], e);
  return dot(e, e) < XPBD_DEGEN2 || dot(nA, nA) < XPBD_DEGEN2 || dot(nB, nB) < XPBD_DEGEN2;
}

XHD float bend_C(const f3 x[4], float theta0) {
  f3 e = x[1] - x[0];
  f3 nA = cross(e, x[2] - x[0]);
  f3 nB = cross(x[3] - x[0], e);
  float sn = dot(cross(nA, nB), e) * (1.f / sqrtf(dot(e, e)));
  float cs = dot(nA, nB);
  float c = atan2f(sn, cs) - theta0;
  if (c > kPi) c -= 2.f * kPi;
  if (c <= -kPi) c += 2.f * kPi;
  return c;
}

// ------------------------------------------------------------------ tets
// F = Ds B with Ds = [x1-x0, x2-x0, x3-x0] (columns) and B = Dm^-1.  dC/dF = P:
//   C_H = det F - gamma:  P = cof F = [f1 x f2, f2 x f0, f0 x f1] (columns f_j of F)
//   C_D = ||F||_F:        P = F / ||F||
// dC/dDs = P B^T, whose columns are g1..g3; g0 = -(g1 + g2 + g3).
template <class S>
XHD void tet_F(const v3<S> x[4], const float* B, v3<S> f[3]) {
  v3<S> d1 = x[1] - x[0], d2 = x[2] - x[0], d3 = x[3] - x[0];
  for (int j = 0; j < 3; ++j) f[j] = d1 * S(B[0 * 3 + j]) + d2 * S(B[1 * 3 + j]) + d3 * S(B[2 * 3 + j]);
}

// Relative form: Ds columns d1, d2, d3 in, g1..g3 out (g0 = -(g1 + g2 + g3)).
template <bool HYDRO, class S>
XHD void tet_grad_rel(const v3<S>& d1, const v3<S>& d2, const v3<S>& d3, const float* B, v3<S>& g1,
                      v3<S>& g2, v3<S>& g3, S* C_out, float gamma) {
  v3<S> f[3];
  for (int j = 0; j < 3; ++j) f[j] = d1 * S(B[0 * 3 + j]) + d2 * S(B[1 * 3 + j]) + d3 * S(B[2 * 3 + j]);
  v3<S> p[3];
  if (HYDRO) {
    p[0] = cross(f[1], f[2]);
    p[1] = cross(f[2], f[0]);
    p[2] = cross(f[0], f[1]);
    if (C_out) *C_out = dot(f[0], p[0]) - gamma;
  } else {
    S nrm = sqrt_(dot(f[0], f[0]) + dot(f[1], f[1]) + dot(f[2], f[2]));
    S in = inv_(nrm);
    p[0] = f[0] * in;
    p[1] = f[1] * in;
    p[2] = f[2] * in;
    if (C_out) *C_out = nrm;
  }
  g1 = p[0] * S(B[0]) + p[1] * S(B[1]) + p[2] * S(B[2]);
  g2 = p[0] * S(B[3]) + p[1] * S(B[4]) + p[2] * S(B[5]);
  g3 = p[0] * S(B[6]) + p[1] * S(B[7]) + p[2] * S(B[8]);
}

template <bool HYDRO, class S>
XHD void tet_grad(const v3<S> x[4], const float* B, v3<S> g[4], S* C_out, float gamma) {
  v3<S> f[3];
  tet_F<S>(x, B, f);
  v3<S> p[3];
  if (HYDRO) {
    p[0] = cross(f[1], f[2]);
    p[1] = cross(f[2], f[0]);
    p[2] = cross(f[0], f[1]);
    if (C_out) *C_out = dot(f[0], p[0]) - gamma;
  } else {
    S nrm = sqrt_(dot(f[0], f[0]) + dot(f[1], f[1]) + dot(f[2], f[2]));
    S in = inv_(nrm);
    p[0] = f[0] * in;
    p[1] = f[1] * in;
    p[2] = f[2] * in;
    if (C_out) *C_out = nrm;
  }
  for (int k = 0; k < 3; ++k)
    g[k + 1] = p[0] * S(B[k * 3 + 0]) + p[1] * S(B[k * 3 + 1]) + p[2] * S(B[k * 3 + 2]);
  g[0] = -(g[1] + g[2] + g[3]);
}

}  // namespace xpbd
