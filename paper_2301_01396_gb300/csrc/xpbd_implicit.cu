// Implicit adjoint of the paper (Sec. "Adjoint State Computation", Eq. adjointXPBD;
// "Positive Definite Projection"; "Linear System Filtering"), derived in reverse mode.
//
// Step n ends at x_{n+1} with multipliers lambda.  At the step's exact solution
// x_{n+1} = p_n + M^-1 grad C^T lambda and C + alpha~ lambda = 0; linearising both and
// eliminating d lambda gives
//     A dx_{n+1} = M dp_n - sum_j grad C_j^T (lambda_j / alpha~_j) d alpha~_j,
//     A = M + sum_j B_j,  B_j = grad C_j^T grad C_j / alpha~_j - lambda_j hess C_j
// over the constraints and the step's active contacts.  Every constraint is translation
// invariant, so B_j = T^T B_rel T in the relative coordinates of its vertices (positions
// relative to its first vertex); with projection, B_rel's negative eigenvalues are clamped
// to 0.  The reverse step solves A y = xbar on the free vertices by preconditioned
// conjugate gradients (pinned vertices filtered out), then pbar = M y on free vertices and
// pbar = xbar - (A y) on pinned ones, and alphabar~_j += -(lambda_j / alpha~_j) grad C_j . y.
//
// Blocks: distance and contact blocks are applied analytically (B_rel = nn^T / alpha~ +
// c P with P = I - nn^T, c = -lambda / l, clamped at 0 under projection); a bending or tet
// block is formed once per step from the analytic gradient and nine Hessian-vector
// products, projected with cyclic Jacobi rotations and stored packed (45 float64).
// Matrix-vector products run color by color (a color's constraints share no vertex), so
// every sum has a fixed order and the solve is deterministic.
#include "xpbd_elems.cuh"

namespace xpbd {

namespace {

__device__ __forceinline__ int pk9(int i, int j) {   // packed upper triangle of a 9x9
  if (i > j) { int t = i; i = j; j = t; }
  return i * 9 - (i * (i - 1)) / 2 + (j - i);
}

__device__ __forceinline__ int pk6(int i, int j) {   // packed upper triangle of a 6x6
  if (i > j) { int t = i; i = j; j = t; }
  return i * 6 - (i * (i - 1)) / 2 + (j - i);
}

// Positive semi-definite part of a symmetric N x N matrix (row-major in a), by cyclic
// Jacobi rotations: a = V D V^T, then sum over max(d_i, 0) v_i v_i^T.  In float64: the
// projected block must stay semi-definite to well below a vertex mass, which float32
// round-off of a stiff bending block (entries ~1e3) does not guarantee.
template <int N>
__device__ void psd_part(double* a) {
  double v[N * N];
  for (int i = 0; i < N * N; ++i) v[i] = (i % (N + 1) == 0) ? 1.0 : 0.0;
  double scale = 0.0;
  for (int i = 0; i < N * N; ++i) scale = fmax(scale, fabs(a[i]));
  if (scale == 0.0) return;
  for (int sweep = 0; sweep < 20; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < N; ++p)
      for (int q = p + 1; q < N; ++q) off += a[p * N + q] * a[p * N + q];
    if (off <= 1e-28 * scale * scale) break;
    for (int p = 0; p < N; ++p)
      for (int q = p + 1; q < N; ++q) {
        const double apq = a[p * N + q];
        if (fabs(apq) <= 1e-30 * scale) continue;
        const double theta = (a[q * N + q] - a[p * N + p]) / (2.0 * apq);
        const double t = copysign(1.0, theta) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < N; ++k) {   // columns p, q
          const double akp = a[k * N + p], akq = a[k * N + q];
          a[k * N + p] = c * akp - s * akq;
          a[k * N + q] = s * akp + c * akq;
        }
        for (int k = 0; k < N; ++k) {   // rows p, q
          const double apk = a[p * N + k], aqk = a[q * N + k];
          a[p * N + k] = c * apk - s * aqk;
          a[q * N + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < N; ++k) {
          const double vkp = v[k * N + p], vkq = v[k * N + q];
          v[k * N + p] = c * vkp - s * vkq;
          v[k * N + q] = s * vkp + c * vkq;
        }
      }
  }
  double d[N];
  for (int i = 0; i < N; ++i) d[i] = fmax(a[i * N + i], 0.0);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
      for (int k = 0; k < N; ++k) s += v[i * N + k] * d[k] * v[j * N + k];
      a[i * N + j] = s;
    }
}

struct D3 {
  double x, y, z;
};
__device__ __forceinline__ D3 ld3(const double* a, int v) { return {a[3 * v], a[3 * v + 1], a[3 * v + 2]}; }
__device__ __forceinline__ void add3(double* a, int v, double x, double y, double z) {
  a[3 * v] += x;
  a[3 * v + 1] += y;
  a[3 * v + 2] += z;
}

// Distance block in relative coordinates at x: B_rel u = n (n.u) / alpha~ + c (u - n (n.u)).
struct DistBlock {
  float nx, ny, nz, inv_at, c;
  bool ok;
  __device__ DistBlock(const DistRec& r, const float4* X, float lam, bool pd) {
    const float4 xa = X[r.a], xb = X[r.b];
    const float dx = xa.x - xb.x, dy = xa.y - xb.y, dz = xa.z - xb.z;
    const float l2 = dx * dx + dy * dy + dz * dz;
    ok = l2 >= XPBD_DEGEN2 && r.at > 0.f;
    const float il = ok ? rsqrtf(l2) : 0.f;
    nx = dx * il;
    ny = dy * il;
    nz = dz * il;
    inv_at = ok ? 1.f / r.at : 0.f;
    c = -lam * il;
    if (pd) c = fmaxf(c, 0.f);
  }
  __device__ D3 apply(D3 u) const {
    const double nu = (double)nx * u.x + (double)ny * u.y + (double)nz * u.z;
    const double a = nu * (double)inv_at - (double)c * nu;
    return {a * nx + (double)c * u.x, a * ny + (double)c * u.y, a * nz + (double)c * u.z};
  }
};

// Contact block of vertex i (plane then sphere), B u accumulated; the matrix itself for
// the preconditioner.
__device__ __forceinline__ void contact_block(int i, const float4* X, uint8_t f, float2 lam, const Collide& c,
                                              bool pd, float B[9]) {
  for (int k = 0; k < 9; ++k) B[k] = 0.f;
  if (c.at <= 0.f) return;
  const float inv_at = 1.f / c.at;
  if (f & 1) B[4] += inv_at;   // n = e_y, hess C = 0
  if (f & 2) {
    const float4 x = X[i];
    const float dx = x.x - c.cx, dy = x.y - c.cy, dz = x.z - c.cz;
    const float l2 = dx * dx + dy * dy + dz * dz;
    if (l2 >= XPBD_DEGEN2) {
      const float il = rsqrtf(l2);
      const float n[3] = {dx * il, dy * il, dz * il};
      float cc = -lam.y * il;   // -lambda hess C = -lambda P / l
      if (pd) cc = fmaxf(cc, 0.f);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) B[3 * a + b] += n[a] * n[b] * inv_at + cc * ((a == b ? 1.f : 0.f) - n[a] * n[b]);
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(kBlock) k_quad_blocks(const typename Quad<KIND>::Rec* __restrict__ rec, int n,
                                                        const float4* __restrict__ X, const float* __restrict__ lam,
                                                        double* __restrict__ blocks, bool pd) {
  XPBD_TID_OR_RETURN(n);
  const typename Quad<KIND>::Rec r = rec[i];
  double* out = blocks + 45 * (size_t)i;
  const f3 x0 = xyz(X[r.v[0]]);
  const f3 e1 = xyz(X[r.v[1]]) - x0, e2 = xyz(X[r.v[2]]) - x0, e3 = xyz(X[r.v[3]]) - x0;
  f3 g1, g2, g3;
  float C;
  if (r.at <= 0.f || !Quad<KIND>::eval(r, e1, e2, e3, g1, g2, g3, C)) {
    for (int k = 0; k < 45; ++k) out[k] = 0.0;
    return;
  }
  const double g[9] = {g1.x, g1.y, g1.z, g2.x, g2.y, g2.z, g3.x, g3.y, g3.z};
  double a[81];
  const f3 zero = mk3(0.f, 0.f, 0.f);
  for (int col = 0; col < 9; ++col) {
    const int vtx = col / 3, comp = col % 3;
    const f3 u = mk3(comp == 0 ? 1.f : 0.f, comp == 1 ? 1.f : 0.f, comp == 2 ? 1.f : 0.f);
    d3 h1, h2, h3;
    Quad<KIND>::hvp(r, e1, e2, e3, vtx == 0 ? u : zero, vtx == 1 ? u : zero, vtx == 2 ? u : zero, h1, h2, h3);
    const f3 c1 = dpart(h1), c2 = dpart(h2), c3 = dpart(h3);
    const float hc[9] = {c1.x, c1.y, c1.z, c2.x, c2.y, c2.z, c3.x, c3.y, c3.z};
    for (int row = 0; row < 9; ++row) a[row * 9 + col] = hc[row];
  }
  const double inv_at = 1.0 / (double)r.at, l = lam[i];
  for (int row = 0; row < 9; ++row)
    for (int col = row; col < 9; ++col) {
      const double h = 0.5 * (a[row * 9 + col] + a[col * 9 + row]);
      const double b = g[row] * g[col] * inv_at - l * h;
      a[row * 9 + col] = b;
      a[col * 9 + row] = b;
    }
  if (pd) psd_part<9>(a);
  for (int row = 0; row < 9; ++row)
    for (int col = row; col < 9; ++col) out[pk9(row, col)] = a[row * 9 + col];
}

// q = M p + (contact blocks) p over all vertices; pinned vertices have no mass term.
__global__ void __launch_bounds__(kBlock) k_apply_mass_contacts(const float4* __restrict__ X, const uint8_t* __restrict__ cflags,
                                                                const float2* __restrict__ lamc, Collide c, bool pd,
                                                                const double* __restrict__ p, double* __restrict__ q, int V) {
  XPBD_TID_OR_RETURN(V);
  const float w = X[i].w;
  const double m = w > 0.f ? 1.0 / (double)w : 0.0;
  const D3 u = ld3(p, i);
  double y[3] = {m * u.x, m * u.y, m * u.z};
  const uint8_t f = cflags ? cflags[i] : 0;
  if (f) {
    float B[9];
    contact_block(i, X, f, lamc[i], c, pd, B);
    const double uu[3] = {u.x, u.y, u.z};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) y[a] += (double)B[3 * a + b] * uu[b];
  }
  q[3 * i] = y[0];
  q[3 * i + 1] = y[1];
  q[3 * i + 2] = y[2];
}

__global__ void __launch_bounds__(kBlock) k_apply_dist(const DistRec* __restrict__ rec, int n, const float4* __restrict__ X,
                                                       const float* __restrict__ lam, bool pd,
                                                       const double* __restrict__ p, double* __restrict__ q) {
  XPBD_TID_OR_RETURN(n);
  const DistRec r = rec[i];
  const DistBlock B(r, X, lam[i], pd);
  if (!B.ok) return;
  const D3 pa = ld3(p, r.a), pb = ld3(p, r.b);
  const D3 t = B.apply({pa.x - pb.x, pa.y - pb.y, pa.z - pb.z});
  add3(q, r.a, t.x, t.y, t.z);
  add3(q, r.b, -t.x, -t.y, -t.z);
}

template <class Rec>
__global__ void __launch_bounds__(kBlock) k_apply_quad(const Rec* __restrict__ rec, int n, const double* __restrict__ blocks,
                                                       const double* __restrict__ p, double* __restrict__ q) {
  XPBD_TID_OR_RETURN(n);
  const Rec r = rec[i];
  const double* B = blocks + 45 * (size_t)i;
  const D3 p0 = ld3(p, r.v[0]);
  double u[9];
  for (int k = 0; k < 3; ++k) {
    const D3 pk = ld3(p, r.v[k + 1]);
    u[3 * k] = pk.x - p0.x;
    u[3 * k + 1] = pk.y - p0.y;
    u[3 * k + 2] = pk.z - p0.z;
  }
  double s[3] = {0.0, 0.0, 0.0};
  for (int row = 0; row < 9; ++row) {
    double t = 0.0;
    for (int col = 0; col < 9; ++col) t += B[pk9(row, col)] * u[col];
    const int k = row / 3;
    q[3 * r.v[k + 1] + row % 3] += t;
    s[row % 3] += t;
  }
  add3(q, r.v[0], -s[0], -s[1], -s[2]);
}

// Diagonal 3x3 blocks of A (the block-Jacobi preconditioner), in dinv[9 i] before inversion.
__global__ void __launch_bounds__(kBlock) k_diag_mass_contacts(const float4* __restrict__ X, const uint8_t* __restrict__ cflags,
                                                               const float2* __restrict__ lamc, Collide c, bool pd,
                                                               double* __restrict__ dg, int V) {
  XPBD_TID_OR_RETURN(V);
  const float w = X[i].w;
  const double m = w > 0.f ? 1.0 / (double)w : 0.0;
  float B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const uint8_t f = cflags ? cflags[i] : 0;
  if (f) contact_block(i, X, f, lamc[i], c, pd, B);
  for (int k = 0; k < 9; ++k) dg[9 * i + k] = (double)B[k] + (k % 4 == 0 ? m : 0.0);
}

__global__ void __launch_bounds__(kBlock) k_diag_dist(const DistRec* __restrict__ rec, int n, const float4* __restrict__ X,
                                                      const float* __restrict__ lam, bool pd, double* __restrict__ dg) {
  XPBD_TID_OR_RETURN(n);
  const DistRec r = rec[i];
  const DistBlock B(r, X, lam[i], pd);
  if (!B.ok) return;
  const float nn[3] = {B.nx, B.ny, B.nz};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const double v = (double)nn[a] * nn[b] * (B.inv_at - B.c) + (a == b ? (double)B.c : 0.0);
      dg[9 * r.a + 3 * a + b] += v;
      dg[9 * r.b + 3 * a + b] += v;
    }
}

template <class Rec>
__global__ void __launch_bounds__(kBlock) k_diag_quad(const Rec* __restrict__ rec, int n, const double* __restrict__ blocks,
                                                      double* __restrict__ dg) {
  XPBD_TID_OR_RETURN(n);
  const Rec r = rec[i];
  const double* B = blocks + 45 * (size_t)i;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s0 = 0.0;
      for (int k = 0; k < 3; ++k) {
        for (int l = 0; l < 3; ++l) s0 += B[pk9(3 * k + a, 3 * l + b)];
        dg[9 * r.v[k + 1] + 3 * a + b] += B[pk9(3 * k + a, 3 * k + b)];
      }
      dg[9 * r.v[0] + 3 * a + b] += s0;
    }
}

__global__ void __launch_bounds__(kBlock) k_diag_invert(const float4* __restrict__ X, double* __restrict__ dg, int V) {
  XPBD_TID_OR_RETURN(V);
  double* m = dg + 9 * (size_t)i;
  if (!(X[i].w > 0.f)) {
    for (int k = 0; k < 9; ++k) m[k] = 0.0;
    return;
  }
  const double a = m[0], b = m[1], c = m[2], d = m[3], e = m[4], f = m[5], g = m[6], h = m[7], k = m[8];
  const double A = e * k - f * h, B = -(d * k - f * g), Cc = d * h - e * g;
  const double det = a * A + b * B + c * Cc;
  if (!(fabs(det) > 0.0)) {   // singular block: plain diagonal scaling
    for (int t = 0; t < 9; ++t) m[t] = 0.0;
    m[0] = a != 0.0 ? 1.0 / a : 0.0;
    m[4] = e != 0.0 ? 1.0 / e : 0.0;
    m[8] = k != 0.0 ? 1.0 / k : 0.0;
    return;
  }
  const double id = 1.0 / det;
  m[0] = A * id;
  m[1] = -(b * k - c * h) * id;
  m[2] = (b * f - c * e) * id;
  m[3] = B * id;
  m[4] = (a * k - c * g) * id;
  m[5] = -(a * f - c * d) * id;
  m[6] = Cc * id;
  m[7] = -(a * h - b * g) * id;
  m[8] = (a * e - b * d) * id;
}

__device__ __forceinline__ void precond(const double* dinv, int i, const double r[3], double z[3]) {
  const double* m = dinv + 9 * (size_t)i;
  for (int a = 0; a < 3; ++a) z[a] = m[3 * a] * r[0] + m[3 * a + 1] * r[1] + m[3 * a + 2] * r[2];
}

// Start: y = 0, r = b (free vertices), z = P^-1 r, p = z; partial sums of (r.z, r.r, b.b).
__global__ void __launch_bounds__(kBlock) k_cg_start(const float4* __restrict__ X, const double* __restrict__ b,
                                                     const double* __restrict__ dinv, double* __restrict__ y,
                                                     double* __restrict__ r, double* __restrict__ z,
                                                     double* __restrict__ p, double* __restrict__ partials, int V) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const bool fr = X[i].w > 0.f;
    double rr[3], zz[3];
    for (int a = 0; a < 3; ++a) rr[a] = fr ? b[3 * i + a] : 0.0;
    precond(dinv, i, rr, zz);
    for (int a = 0; a < 3; ++a) {
      y[3 * i + a] = 0.0;
      r[3 * i + a] = rr[a];
      z[3 * i + a] = zz[a];
      p[3 * i + a] = zz[a];
      acc[0] += rr[a] * zz[a];
      acc[1] += rr[a] * rr[a];
      acc[2] += rr[a] * rr[a];
    }
  }
  block_sum_store<3>(acc, partials + 3 * blockIdx.x);
}

// Pinned rows of q are filtered out; partial sums of p.q.
__global__ void __launch_bounds__(kBlock) k_cg_pq(const float4* __restrict__ X, const double* __restrict__ p,
                                                  double* __restrict__ q, double* __restrict__ partials, int V) {
  double acc[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    if (!(X[i].w > 0.f)) {
      q[3 * i] = q[3 * i + 1] = q[3 * i + 2] = 0.0;
      continue;
    }
    for (int a = 0; a < 3; ++a) acc[0] += p[3 * i + a] * q[3 * i + a];
  }
  block_sum_store<1>(acc, partials + blockIdx.x);
}

// Scalars of the solve: sc[0] = p.q, (sc[1], sc[2]) and (sc[4], sc[5]) = (r.z, r.r) of
// alternate iterations, sc[3] = b.b.
// alpha = rz / pq; y += alpha p; r -= alpha q; z = P^-1 r; partial sums of (r.z, r.r).
__global__ void __launch_bounds__(kBlock) k_cg_step(const double* __restrict__ sc, int rz_slot, const double* __restrict__ p,
                                                    const double* __restrict__ q, const double* __restrict__ dinv,
                                                    double* __restrict__ y, double* __restrict__ r, double* __restrict__ z,
                                                    double* __restrict__ partials, int V) {
  const double pq = sc[0];
  const double alpha = pq != 0.0 ? sc[rz_slot] / pq : 0.0;
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    double rr[3], zz[3];
    for (int a = 0; a < 3; ++a) {
      y[3 * i + a] += alpha * p[3 * i + a];
      rr[a] = r[3 * i + a] - alpha * q[3 * i + a];
      r[3 * i + a] = rr[a];
    }
    precond(dinv, i, rr, zz);
    for (int a = 0; a < 3; ++a) {
      z[3 * i + a] = zz[a];
      acc[0] += rr[a] * zz[a];
      acc[1] += rr[a] * rr[a];
    }
  }
  block_sum_store<2>(acc, partials + 2 * blockIdx.x);
}

// beta = rz_new / rz_old; p = z + beta p.
__global__ void __launch_bounds__(kBlock) k_cg_dir(const double* __restrict__ sc, int old_slot, int new_slot,
                                                   const double* __restrict__ z, double* __restrict__ p, int V) {
  const double ro = sc[old_slot];
  const double beta = ro != 0.0 ? sc[new_slot] / ro : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * V; i += gridDim.x * blockDim.x) p[i] = z[i] + beta * p[i];
}

// pbar into xbar: M y on free vertices, b - (A y) on pinned ones.
__global__ void __launch_bounds__(kBlock) k_finish(const float4* __restrict__ X, const double* __restrict__ b,
                                                   const double* __restrict__ y, const double* __restrict__ ay,
                                                   float4* __restrict__ xbar, int V) {
  XPBD_TID_OR_RETURN(V);
  const float w = X[i].w;
  double o[3];
  for (int a = 0; a < 3; ++a) o[a] = w > 0.f ? y[3 * i + a] / (double)w : b[3 * i + a] - ay[3 * i + a];
  xbar[i] = make_float4((float)o[0], (float)o[1], (float)o[2], 0.f);
}

__global__ void __launch_bounds__(kBlock) k_xbar_to_b(const float4* __restrict__ xbar, double* __restrict__ b, int V) {
  XPBD_TID_OR_RETURN(V);
  const float4 v = xbar[i];
  b[3 * i] = v.x;
  b[3 * i + 1] = v.y;
  b[3 * i + 2] = v.z;
}

// alphabar~_j += -(lambda_j / alpha~_j) grad C_j . y (relative coordinates).
__global__ void __launch_bounds__(kBlock) k_abar_dist(const DistRec* __restrict__ rec, int n, const float4* __restrict__ X,
                                                      const float* __restrict__ lam, const double* __restrict__ y,
                                                      double* __restrict__ acc) {
  XPBD_TID_OR_RETURN(n);
  const DistRec r = rec[i];
  const float4 xa = X[r.a], xb = X[r.b];
  const float dx = xa.x - xb.x, dy = xa.y - xb.y, dz = xa.z - xb.z;
  const float l2 = dx * dx + dy * dy + dz * dz;
  if (!(l2 >= XPBD_DEGEN2) || !(r.at > 0.f)) return;
  const float il = rsqrtf(l2);
  const D3 ya = ld3(y, r.a), yb = ld3(y, r.b);
  const double gy = (double)(dx * il) * (ya.x - yb.x) + (double)(dy * il) * (ya.y - yb.y) + (double)(dz * il) * (ya.z - yb.z);
  acc[i] += -((double)lam[i] / (double)r.at) * gy;
}

template <int KIND>
__global__ void __launch_bounds__(kBlock) k_abar_quad(const typename Quad<KIND>::Rec* __restrict__ rec, int n,
                                                      const float4* __restrict__ X, const float* __restrict__ lam,
                                                      const double* __restrict__ y, double* __restrict__ acc) {
  XPBD_TID_OR_RETURN(n);
  const typename Quad<KIND>::Rec r = rec[i];
  if (!(r.at > 0.f)) return;
  const f3 x0 = xyz(X[r.v[0]]);
  const f3 e1 = xyz(X[r.v[1]]) - x0, e2 = xyz(X[r.v[2]]) - x0, e3 = xyz(X[r.v[3]]) - x0;
  f3 g[3];
  float C;
  if (!Quad<KIND>::eval(r, e1, e2, e3, g[0], g[1], g[2], C)) return;
  const D3 y0 = ld3(y, r.v[0]);
  double gy = 0.0;
  for (int k = 0; k < 3; ++k) {
    const D3 yk = ld3(y, r.v[k + 1]);
    gy += (double)g[k].x * (yk.x - y0.x) + (double)g[k].y * (yk.y - y0.y) + (double)g[k].z * (yk.z - y0.z);
  }
  acc[i] += -((double)lam[i] / (double)r.at) * gy;
}

// ---- membranes (three rows, 3x3 compliance block), in relative coordinates of vertices 1, 2
// (e_a = x_a - x_0): the rows' gradients are b_u,a f_u | b_v,a f_v | b_u,a f_v + b_v,a f_u
// per vertex a, their Hessians (b b^T) (x) I3 with the per-vertex weights b of f_u, f_v.
struct MembRows {
  double G[3][6];       // row k, relative coordinate 3 (a-1) + c
  double Ai[3][3];      // alpha~^-1
  double bu[2], bv[2];  // weights of vertices 1, 2
  bool ok;
  __device__ MembRows(const MembRec& r, const float4* X) {
    const double det2 = (double)r.a00 * r.a11 - (double)r.a01 * r.a01;
    ok = r.a00 > 0.f && r.a22 > 0.f && det2 > 0.0;
    const float4 p0 = X[r.v[0]], p1 = X[r.v[1]], p2 = X[r.v[2]];
    const double d1[3] = {(double)p1.x - p0.x, (double)p1.y - p0.y, (double)p1.z - p0.z};
    const double d2[3] = {(double)p2.x - p0.x, (double)p2.y - p0.y, (double)p2.z - p0.z};
    bu[0] = r.B[0];
    bu[1] = r.B[2];
    bv[0] = r.B[1];
    bv[1] = r.B[3];
    double fu[3], fv[3];
    for (int c = 0; c < 3; ++c) {
      fu[c] = d1[c] * bu[0] + d2[c] * bu[1];
      fv[c] = d1[c] * bv[0] + d2[c] * bv[1];
    }
    for (int a = 0; a < 2; ++a)
      for (int c = 0; c < 3; ++c) {
        G[0][3 * a + c] = bu[a] * fu[c];
        G[1][3 * a + c] = bv[a] * fv[c];
        G[2][3 * a + c] = bu[a] * fv[c] + bv[a] * fu[c];
      }
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) Ai[k][l] = 0.0;
    if (ok) {
      Ai[0][0] = r.a11 / det2;
      Ai[1][1] = r.a00 / det2;
      Ai[0][1] = Ai[1][0] = -r.a01 / det2;
      Ai[2][2] = 1.0 / r.a22;
    }
  }
};

// B_rel = G^T alpha~^-1 G - (lambda_0 b_u b_u^T + lambda_1 b_v b_v^T + lambda_2 (b_u b_v^T + b_v b_u^T)) (x) I3,
// projected when pd, stored packed (21 float64).
__global__ void __launch_bounds__(kBlock) k_memb_blocks(const MembRec* __restrict__ rec, int n, const float4* __restrict__ X,
                                                        const float* __restrict__ lam, int stride,
                                                        double* __restrict__ blocks, bool pd) {
  XPBD_TID_OR_RETURN(n);
  const MembRec r = rec[i];
  double* out = blocks + 21 * (size_t)i;
  const MembRows M(r, X);
  if (!M.ok) {
    for (int k = 0; k < 21; ++k) out[k] = 0.0;
    return;
  }
  const double l0 = lam[i], l1 = lam[i + stride], l2 = lam[i + 2 * stride];
  double a[36];
  for (int row = 0; row < 6; ++row)
    for (int col = 0; col < 6; ++col) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s += M.G[k][row] * M.Ai[k][l] * M.G[l][col];
      if (row % 3 == col % 3) {
        const int va = row / 3, vb = col / 3;
        s -= l0 * M.bu[va] * M.bu[vb] + l1 * M.bv[va] * M.bv[vb] + l2 * (M.bu[va] * M.bv[vb] + M.bv[va] * M.bu[vb]);
      }
      a[row * 6 + col] = s;
    }
  for (int row = 0; row < 6; ++row)
    for (int col = row + 1; col < 6; ++col) {
      const double h = 0.5 * (a[row * 6 + col] + a[col * 6 + row]);
      a[row * 6 + col] = a[col * 6 + row] = h;
    }
  if (pd) psd_part<6>(a);
  for (int row = 0; row < 6; ++row)
    for (int col = row; col < 6; ++col) out[pk6(row, col)] = a[row * 6 + col];
}

__global__ void __launch_bounds__(kBlock) k_apply_memb(const MembRec* __restrict__ rec, int n, const double* __restrict__ blocks,
                                                       const double* __restrict__ p, double* __restrict__ q) {
  XPBD_TID_OR_RETURN(n);
  const MembRec r = rec[i];
  const double* B = blocks + 21 * (size_t)i;
  const D3 p0 = ld3(p, r.v[0]);
  double u[6];
  for (int k = 0; k < 2; ++k) {
    const D3 pk = ld3(p, r.v[k + 1]);
    u[3 * k] = pk.x - p0.x;
    u[3 * k + 1] = pk.y - p0.y;
    u[3 * k + 2] = pk.z - p0.z;
  }
  double s[3] = {0.0, 0.0, 0.0};
  for (int row = 0; row < 6; ++row) {
    double t = 0.0;
    for (int col = 0; col < 6; ++col) t += B[pk6(row, col)] * u[col];
    q[3 * r.v[row / 3 + 1] + row % 3] += t;
    s[row % 3] += t;
  }
  add3(q, r.v[0], -s[0], -s[1], -s[2]);
}

__global__ void __launch_bounds__(kBlock) k_diag_memb(const MembRec* __restrict__ rec, int n, const double* __restrict__ blocks,
                                                      double* __restrict__ dg) {
  XPBD_TID_OR_RETURN(n);
  const MembRec r = rec[i];
  const double* B = blocks + 21 * (size_t)i;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s0 = 0.0;
      for (int k = 0; k < 2; ++k) {
        for (int l = 0; l < 2; ++l) s0 += B[pk6(3 * k + a, 3 * l + b)];
        dg[9 * r.v[k + 1] + 3 * a + b] += B[pk6(3 * k + a, 3 * k + b)];
      }
      dg[9 * r.v[0] + 3 * a + b] += s0;
    }
}

// alphabar~ += -(alpha~^-1 G y) lambda^T on the entries (00, 11, 01 + 10, 22).
__global__ void __launch_bounds__(kBlock) k_abar_memb(const MembRec* __restrict__ rec, int n, const float4* __restrict__ X,
                                                      const float* __restrict__ lam, int stride, const double* __restrict__ y,
                                                      double* __restrict__ acc) {
  XPBD_TID_OR_RETURN(n);
  const MembRec r = rec[i];
  const MembRows M(r, X);
  if (!M.ok) return;
  const D3 y0 = ld3(y, r.v[0]);
  double u[6];
  for (int k = 0; k < 2; ++k) {
    const D3 yk = ld3(y, r.v[k + 1]);
    u[3 * k] = yk.x - y0.x;
    u[3 * k + 1] = yk.y - y0.y;
    u[3 * k + 2] = yk.z - y0.z;
  }
  double gy[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 6; ++c) gy[k] += M.G[k][c] * u[c];
  double z[3];
  for (int k = 0; k < 3; ++k) z[k] = M.Ai[k][0] * gy[0] + M.Ai[k][1] * gy[1] + M.Ai[k][2] * gy[2];
  const double l0 = lam[i], l1 = lam[i + stride], l2 = lam[i + 2 * stride];
  acc[i] += -z[0] * l0;
  acc[i + stride] += -z[1] * l1;
  acc[i + 2 * stride] += -(z[0] * l1 + z[1] * l0);
  acc[i + 3 * stride] += -z[2] * l2;
}

}  // namespace

void launch_memb_blocks(const MembRec* rec, int n, const float4* X, const float* lam, int stride, double* blocks, bool pd,
                        cudaStream_t s) {
  if (n > 0) k_memb_blocks<<<grid_for(n), kBlock, 0, s>>>(rec, n, X, lam, stride, blocks, pd);
}

void launch_apply_memb(const MembRec* rec, int n, const double* blocks, const double* p, double* q, cudaStream_t s) {
  if (n > 0) k_apply_memb<<<grid_for(n), kBlock, 0, s>>>(rec, n, blocks, p, q);
}

void launch_diag_memb(const MembRec* rec, int n, const double* blocks, double* dg, cudaStream_t s) {
  if (n > 0) k_diag_memb<<<grid_for(n), kBlock, 0, s>>>(rec, n, blocks, dg);
}

void launch_abar_memb(const MembRec* rec, int n, const float4* X, const float* lam, int stride, const double* y,
                      double* acc, cudaStream_t s) {
  if (n > 0) k_abar_memb<<<grid_for(n), kBlock, 0, s>>>(rec, n, X, lam, stride, y, acc);
}

void launch_quad_blocks(SegType t, const void* rec, int n, const float4* X, const float* lam, double* blocks, bool pd,
                        cudaStream_t s) {
  if (n <= 0) return;
  switch (t) {
    case SEG_BEND: k_quad_blocks<1><<<grid_for(n), kBlock, 0, s>>>((const BendRec*)rec, n, X, lam, blocks, pd); break;
    case SEG_TETH: k_quad_blocks<2><<<grid_for(n), kBlock, 0, s>>>((const TetRec*)rec, n, X, lam, blocks, pd); break;
    case SEG_TETD: k_quad_blocks<3><<<grid_for(n), kBlock, 0, s>>>((const TetRec*)rec, n, X, lam, blocks, pd); break;
    default: break;
  }
}

void launch_apply_mass_contacts(const float4* X, const uint8_t* cflags, const float2* lamc, Collide c, bool pd,
                                const double* p, double* q, int V, cudaStream_t s) {
  if (V > 0) k_apply_mass_contacts<<<grid_for(V), kBlock, 0, s>>>(X, cflags, lamc, c, pd, p, q, V);
}

void launch_apply_block(SegType t, const void* rec, int n, const float4* X, const float* lam, const double* blocks,
                        bool pd, const double* p, double* q, cudaStream_t s) {
  if (n <= 0) return;
  if (t == SEG_DIST)
    k_apply_dist<<<grid_for(n), kBlock, 0, s>>>((const DistRec*)rec, n, X, lam, pd, p, q);
  else if (t == SEG_BEND)
    k_apply_quad<BendRec><<<grid_for(n), kBlock, 0, s>>>((const BendRec*)rec, n, blocks, p, q);
  else
    k_apply_quad<TetRec><<<grid_for(n), kBlock, 0, s>>>((const TetRec*)rec, n, blocks, p, q);
}

void launch_diag_mass_contacts(const float4* X, const uint8_t* cflags, const float2* lamc, Collide c, bool pd,
                               double* dg, int V, cudaStream_t s) {
  if (V > 0) k_diag_mass_contacts<<<grid_for(V), kBlock, 0, s>>>(X, cflags, lamc, c, pd, dg, V);
}

void launch_diag_block(SegType t, const void* rec, int n, const float4* X, const float* lam, const double* blocks,
                       bool pd, double* dg, cudaStream_t s) {
  if (n <= 0) return;
  if (t == SEG_DIST)
    k_diag_dist<<<grid_for(n), kBlock, 0, s>>>((const DistRec*)rec, n, X, lam, pd, dg);
  else if (t == SEG_BEND)
    k_diag_quad<BendRec><<<grid_for(n), kBlock, 0, s>>>((const BendRec*)rec, n, blocks, dg);
  else
    k_diag_quad<TetRec><<<grid_for(n), kBlock, 0, s>>>((const TetRec*)rec, n, blocks, dg);
}

void launch_diag_invert(const float4* X, double* dg, int V, cudaStream_t s) {
  if (V > 0) k_diag_invert<<<grid_for(V), kBlock, 0, s>>>(X, dg, V);
}

void launch_cg_start(const float4* X, const double* b, const double* dinv, double* y, double* r, double* z, double* p,
                     double* partials, int V, cudaStream_t s) {
  k_cg_start<<<partial_blocks(V), kBlock, 0, s>>>(X, b, dinv, y, r, z, p, partials, V);
}

void launch_cg_pq(const float4* X, const double* p, double* q, double* partials, int V, cudaStream_t s) {
  k_cg_pq<<<partial_blocks(V), kBlock, 0, s>>>(X, p, q, partials, V);
}

void launch_cg_step(const double* sc, int rz_slot, const double* p, const double* q, const double* dinv, double* y,
                    double* r, double* z, double* partials, int V, cudaStream_t s) {
  k_cg_step<<<partial_blocks(V), kBlock, 0, s>>>(sc, rz_slot, p, q, dinv, y, r, z, partials, V);
}

void launch_cg_dir(const double* sc, int old_slot, int new_slot, const double* z, double* p, int V, cudaStream_t s) {
  if (V > 0) k_cg_dir<<<grid_for(3 * V), kBlock, 0, s>>>(sc, old_slot, new_slot, z, p, V);
}

void launch_implicit_finish(const float4* X, const double* b, const double* y, const double* ay, float4* xbar, int V,
                            cudaStream_t s) {
  if (V > 0) k_finish<<<grid_for(V), kBlock, 0, s>>>(X, b, y, ay, xbar, V);
}

void launch_xbar_to_b(const float4* xbar, double* b, int V, cudaStream_t s) {
  if (V > 0) k_xbar_to_b<<<grid_for(V), kBlock, 0, s>>>(xbar, b, V);
}

void launch_abar(SegType t, const void* rec, int n, const float4* X, const float* lam, const double* y, double* acc,
                 cudaStream_t s) {
  if (n <= 0) return;
  switch (t) {
    case SEG_DIST: k_abar_dist<<<grid_for(n), kBlock, 0, s>>>((const DistRec*)rec, n, X, lam, y, acc); break;
    case SEG_BEND: k_abar_quad<1><<<grid_for(n), kBlock, 0, s>>>((const BendRec*)rec, n, X, lam, y, acc); break;
    case SEG_TETH: k_abar_quad<2><<<grid_for(n), kBlock, 0, s>>>((const TetRec*)rec, n, X, lam, y, acc); break;
    default: k_abar_quad<3><<<grid_for(n), kBlock, 0, s>>>((const TetRec*)rec, n, X, lam, y, acc);
  }
}

}  // namespace xpbd
