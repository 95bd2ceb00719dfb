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
#include "xpbd_multigrid.cuh"

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

// ============================================================================ multigrid
// Grid multigrid preconditioner (declared in xpbd_multigrid.cuh, which states the method).

namespace {

__device__ __forceinline__ bool mg_inv3(const double* m, double* o) {
  const double a = m[0], b = m[1], c = m[2], d = m[3], e = m[4], f = m[5], g = m[6], h = m[7], k = m[8];
  const double A = e * k - f * h, B = -(d * k - f * g), Cc = d * h - e * g;
  const double det = a * A + b * B + c * Cc;
  if (!(fabs(det) > 0.0) || !isfinite(det)) {
    for (int t = 0; t < 9; ++t) o[t] = 0.0;
    return false;
  }
  const double id = 1.0 / det;
  o[0] = A * id;
  o[1] = -(b * k - c * h) * id;
  o[2] = (b * f - c * e) * id;
  o[3] = B * id;
  o[4] = (a * k - c * g) * id;
  o[5] = -(a * f - c * d) * id;
  o[6] = Cc * id;
  o[7] = -(a * h - b * g) * id;
  o[8] = (a * e - b * d) * id;
  return true;
}

// o = a b (3x3), o = a b^T, o -= a b^T
__device__ __forceinline__ void mm3(const double* a, const double* b, double* o) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) o[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}
__device__ __forceinline__ void mm3_sub_bt(const double* a, const double* b, double* o) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) o[3 * i + j] -= a[3 * i] * b[3 * j] + a[3 * i + 1] * b[3 * j + 1] + a[3 * i + 2] * b[3 * j + 2];
}

__device__ __forceinline__ bool mg_pinned(const float4* X, int v) { return X && !(X[v].w > 0.f); }

// out += (A x)_v over the 5 x 5 stencil.
__device__ __forceinline__ void mg_row_apply(const double* __restrict__ A, const double* __restrict__ x, int v, int nx,
                                             int ny, double out[3]) {
  const int vx = v % nx, vy = v / nx;
  const double* a = A + (size_t)v * kMgBlock;
#pragma unroll 5
  for (int sl = 0; sl < kMgSlots; ++sl) {
    const int xx = vx + sl % 5 - 2, yy = vy + sl / 5 - 2;
    if (xx < 0 || xx >= nx || yy < 0 || yy >= ny) continue;
    const double* xj = x + 3 * ((size_t)yy * nx + xx);
    const double x0 = xj[0], x1 = xj[1], x2 = xj[2];
    const double* m = a + 9 * sl;
    out[0] += m[0] * x0 + m[1] * x1 + m[2] * x2;
    out[1] += m[3] * x0 + m[4] * x1 + m[5] * x2;
    out[2] += m[6] * x0 + m[7] * x1 + m[8] * x2;
  }
}

// The same product with a warp per row: lane s < 25 takes stencil slot s, and the three
// sums are reduced over the warp in a fixed order (every lane gets them).  float64 issues
// at 1/64 of the float32 rate on this GPU, so a thread that sums a whole row (225
// multiply-adds) costs ~7 us however few rows a launch has; a warp per row costs ~1 us.
__device__ __forceinline__ void mg_row_apply_warp(const double* __restrict__ A, const double* __restrict__ x, int v,
                                                  int nx, int ny, double out[3]) {
  const int lane = threadIdx.x & 31;
  double o0 = 0.0, o1 = 0.0, o2 = 0.0;
  if (lane < kMgSlots) {
    const int xx = v % nx + lane % 5 - 2, yy = v / nx + lane / 5 - 2;
    if (xx >= 0 && xx < nx && yy >= 0 && yy < ny) {
      const double* xj = x + 3 * ((size_t)yy * nx + xx);
      const double x0 = xj[0], x1 = xj[1], x2 = xj[2];
      const double* m = A + (size_t)v * kMgBlock + 9 * lane;
      o0 = m[0] * x0 + m[1] * x1 + m[2] * x2;
      o1 = m[3] * x0 + m[4] * x1 + m[5] * x2;
      o2 = m[6] * x0 + m[7] * x1 + m[8] * x2;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    o0 += __shfl_xor_sync(0xffffffffu, o0, off);
    o1 += __shfl_xor_sync(0xffffffffu, o1, off);
    o2 += __shfl_xor_sync(0xffffffffu, o2, off);
  }
  out[0] += o0;
  out[1] += o1;
  out[2] += o2;
}

// Item (row) index of this thread (WARP = false) or of this thread's warp (WARP = true);
// with WARP every lane of a warp gets the same item, so early returns are warp-uniform.
template <bool WARP>
__device__ __forceinline__ int mg_item() {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  return WARP ? (t >> 5) : t;
}

template <bool WARP>
__device__ __forceinline__ void mg_apply(const double* __restrict__ A, const double* __restrict__ x, int v, int nx, int ny,
                                         double out[3]) {
  if (WARP)
    mg_row_apply_warp(A, x, v, nx, ny, out);
  else
    mg_row_apply(A, x, v, nx, ny, out);
}

__device__ __forceinline__ void mg_add(double* A0, int vi, int vj, int nx, int V, const double* B, double* flag) {
  if (vi < 0 || vj < 0 || vi >= V || vj >= V) {
    *flag = 1.0;
    return;
  }
  const int dx = vj % nx - vi % nx, dy = vj / nx - vi / nx;
  if (dx < -2 || dx > 2 || dy < -2 || dy > 2) {
    *flag = 1.0;
    return;
  }
  double* a = A0 + (size_t)vi * kMgBlock + 9 * ((dy + 2) * 5 + dx + 2);
  for (int k = 0; k < 9; ++k) a[k] += B[k];
}

__global__ void __launch_bounds__(kBlock) k_mg_mass_contacts(const float4* __restrict__ X, const uint8_t* __restrict__ cflags,
                                                             const float2* __restrict__ lamc, Collide c, bool pd,
                                                             double* __restrict__ A0, int V) {
  XPBD_TID_OR_RETURN(V);
  const float w = X[i].w;
  const double m = w > 0.f ? 1.0 / (double)w : 0.0;
  float B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const uint8_t f = cflags ? cflags[i] : 0;
  if (f) contact_block(i, X, f, lamc[i], c, pd, B);
  double* a = A0 + (size_t)i * kMgBlock + 9 * 12;
  for (int k = 0; k < 9; ++k) a[k] += (double)B[k] + (k % 4 == 0 ? m : 0.0);
}

__global__ void __launch_bounds__(kBlock) k_mg_asm_dist(const DistRec* __restrict__ rec, int n, const float4* __restrict__ X,
                                                        const float* __restrict__ lam, bool pd, double* __restrict__ A0,
                                                        int nx, int V, double* flag) {
  XPBD_TID_OR_RETURN(n);
  const DistRec r = rec[i];
  const DistBlock B(r, X, lam[i], pd);
  if (!B.ok) return;
  const float nn[3] = {B.nx, B.ny, B.nz};
  double P[9], N[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      P[3 * a + b] = (double)nn[a] * nn[b] * ((double)B.inv_at - (double)B.c) + (a == b ? (double)B.c : 0.0);
      N[3 * a + b] = -P[3 * a + b];
    }
  mg_add(A0, r.a, r.a, nx, V, P, flag);
  mg_add(A0, r.b, r.b, nx, V, P, flag);
  mg_add(A0, r.a, r.b, nx, V, N, flag);
  mg_add(A0, r.b, r.a, nx, V, N, flag);
}

// A block stored in the relative coordinates of vertices 1..NR (packed upper triangle of
// a (3 NR)^2 matrix), scattered into the vertex-pair blocks T^T B T.
template <int NR>
__device__ __forceinline__ double rel_entry(const double* B, int row, int col) {
  return NR == 3 ? B[pk9(row, col)] : B[pk6(row, col)];
}

template <int NR>
__device__ void mg_scatter_rel(const int* v, const double* __restrict__ B, double* __restrict__ A0, int nx, int V,
                               double* flag) {
  for (int a = 0; a <= NR; ++a)
    for (int b = 0; b <= NR; ++b) {
      double M[9];
      for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be) {
          double s = 0.0;
          if (a > 0 && b > 0) {
            s = rel_entry<NR>(B, 3 * (a - 1) + al, 3 * (b - 1) + be);
          } else if (a > 0) {
            for (int l = 0; l < NR; ++l) s -= rel_entry<NR>(B, 3 * (a - 1) + al, 3 * l + be);
          } else if (b > 0) {
            for (int k = 0; k < NR; ++k) s -= rel_entry<NR>(B, 3 * k + al, 3 * (b - 1) + be);
          } else {
            for (int k = 0; k < NR; ++k)
              for (int l = 0; l < NR; ++l) s += rel_entry<NR>(B, 3 * k + al, 3 * l + be);
          }
          M[3 * al + be] = s;
        }
      mg_add(A0, v[a], v[b], nx, V, M, flag);
    }
}

template <class Rec>
__global__ void __launch_bounds__(kBlock) k_mg_asm_quad(const Rec* __restrict__ rec, int n, const double* __restrict__ blocks,
                                                        double* __restrict__ A0, int nx, int V, double* flag) {
  XPBD_TID_OR_RETURN(n);
  const Rec r = rec[i];
  const int v[4] = {r.v[0], r.v[1], r.v[2], r.v[3]};
  mg_scatter_rel<3>(v, blocks + 45 * (size_t)i, A0, nx, V, flag);
}

__global__ void __launch_bounds__(kBlock) k_mg_asm_memb(const MembRec* __restrict__ rec, int n, const double* __restrict__ blocks,
                                                        double* __restrict__ A0, int nx, int V, double* flag) {
  XPBD_TID_OR_RETURN(n);
  const MembRec r = rec[i];
  const int v[3] = {r.v[0], r.v[1], r.v[2]};
  mg_scatter_rel<2>(v, blocks + 21 * (size_t)i, A0, nx, V, flag);
}

// Galerkin coarse operator: one thread per (coarse vertex, stencil offset).
__global__ void __launch_bounds__(kBlock) k_mg_rap(const double* __restrict__ Af, int nxf, int nyf,
                                                   const float4* __restrict__ X, double* __restrict__ Ac, int nxc,
                                                   int nyc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nxc * nyc * kMgSlots) return;
  const int I = t / kMgSlots, sl = t % kMgSlots;
  const int IX = I % nxc, IY = I / nxc;
  const int JX = IX + sl % 5 - 2, JY = IY + sl / 5 - 2;
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (JX >= 0 && JX < nxc && JY >= 0 && JY < nyc) {
    for (int iy = max(2 * IY - 1, 0); iy <= min(2 * IY + 1, nyf - 1); ++iy) {
      const double wy = mg_w(iy, IY, nyc);
      if (wy == 0.0) continue;
      for (int ix = max(2 * IX - 1, 0); ix <= min(2 * IX + 1, nxf - 1); ++ix) {
        const double wi = wy * mg_w(ix, IX, nxc);
        const int i = iy * nxf + ix;
        if (wi == 0.0 || mg_pinned(X, i)) continue;
        const double* ai = Af + (size_t)i * kMgBlock;
        for (int jy = max(2 * JY - 1, max(iy - 2, 0)); jy <= min(2 * JY + 1, min(iy + 2, nyf - 1)); ++jy) {
          const double wjy = mg_w(jy, JY, nyc);
          if (wjy == 0.0) continue;
          for (int jx = max(2 * JX - 1, max(ix - 2, 0)); jx <= min(2 * JX + 1, min(ix + 2, nxf - 1)); ++jx) {
            const double w = wi * wjy * mg_w(jx, JX, nxc);
            if (w == 0.0 || mg_pinned(X, jy * nxf + jx)) continue;
            const double* m = ai + 9 * ((jy - iy + 2) * 5 + (jx - ix + 2));
            for (int k = 0; k < 9; ++k) acc[k] += w * m[k];
          }
        }
      }
    }
  }
  double* o = Ac + (size_t)t * 9;
  for (int k = 0; k < 9; ++k) o[k] = acc[k];
}

__global__ void __launch_bounds__(kBlock) k_mg_dinv(const double* __restrict__ A, const float4* __restrict__ X,
                                                    double* __restrict__ dinv, int n) {
  XPBD_TID_OR_RETURN(n);
  double* o = dinv + 9 * (size_t)i;
  if (mg_pinned(X, i)) {
    for (int k = 0; k < 9; ++k) o[k] = 0.0;
    return;
  }
  mg_inv3(A + (size_t)i * kMgBlock + 9 * 12, o);
}

// Dense inverse of the coarsest level by in-place Gauss-Jordan elimination (the matrix is
// symmetric positive definite on its nonempty rows; empty rows get a unit diagonal).
__global__ void __launch_bounds__(256) k_mg_coarse_inverse(const double* __restrict__ A, const float4* __restrict__ X,
                                                           int nx, int ny, double* __restrict__ cinv) {
  constexpr int NM = 3 * kMgCoarseMax;
  __shared__ double M[NM * NM];
  __shared__ double col[NM];
  const int n = nx * ny, N = 3 * n;
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) M[t] = 0.0;
  __syncthreads();
  for (int t = threadIdx.x; t < n * kMgSlots; t += blockDim.x) {
    const int v = t / kMgSlots, sl = t % kMgSlots;
    const int xx = v % nx + sl % 5 - 2, yy = v / nx + sl / 5 - 2;
    if (xx < 0 || xx >= nx || yy < 0 || yy >= ny) continue;
    const int j = yy * nx + xx;
    if (mg_pinned(X, v) || mg_pinned(X, j)) continue;
    const double* m = A + (size_t)v * kMgBlock + 9 * sl;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) M[(3 * v + a) * N + 3 * j + b] = m[3 * a + b];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N; t += blockDim.x)
    if (M[t * N + t] == 0.0) M[t * N + t] = 1.0;
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    for (int t = threadIdx.x; t < N; t += blockDim.x) col[t] = M[t * N + k];
    __syncthreads();
    double p = col[k];
    if (!(fabs(p) > 0.0)) p = 1.0;
    const double ip = 1.0 / p;
    for (int j = threadIdx.x; j < N; j += blockDim.x) M[k * N + j] = (j == k ? 1.0 : M[k * N + j]) * ip;
    __syncthreads();
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
      const int i = t / N, j = t % N;
      if (i == k) continue;
      M[t] = (j == k ? 0.0 : M[t]) - col[i] * M[k * N + j];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) cinv[t] = M[t];
}

__global__ void __launch_bounds__(256) k_mg_coarse_solve(const double* __restrict__ cinv, const double* __restrict__ b,
                                                         double* __restrict__ x, int N) {
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < N; ++j) s += cinv[(size_t)r * N + j] * b[j];
    x[r] = s;
  }
}

// Block LDL^T of every line's pentadiagonal block matrix (its vertices' couplings along the
// line); pinned vertices are left out (zero inverse pivot, no coupling).  Per vertex:
// [L(k, k-1) | L(k, k-2) | D_k^-1].
__global__ void __launch_bounds__(kBlock) k_mg_line_factor(const double* __restrict__ A, const float4* __restrict__ X,
                                                           int nx, int ny, int dir, float* __restrict__ F) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nx + ny - 1) return;
  int x0, y0;
  const int len = mg_line(l, nx, ny, dir, x0, y0);
  const int s1 = 5 + (2 - dir), s2 = 2 - 2 * dir;   // in-line offsets -1 and -2
  double Dm1[9], Dm2[9], L2m1[9];
  for (int k = 0; k < 9; ++k) Dm1[k] = Dm2[k] = L2m1[k] = 0.0;
  for (int k = 0; k < len; ++k) {
    const int v = (y0 + k) * nx + x0 + dir * k;
    float* f = F + (size_t)v * kMgLineFactor;
    double L1[9], L2[9], D[9], W1[9], W2[9];
    if (mg_pinned(X, v)) {
      for (int t = 0; t < 27; ++t) f[t] = 0.f;
      for (int t = 0; t < 9; ++t) {
        Dm2[t] = Dm1[t];
        Dm1[t] = 0.0;
        L2m1[t] = 0.0;
      }
      continue;
    }
    const double* a = A + (size_t)v * kMgBlock;
    for (int t = 0; t < 9; ++t) {
      W2[t] = k >= 2 ? a[9 * s2 + t] : 0.0;
      W1[t] = k >= 1 ? a[9 * s1 + t] : 0.0;
      D[t] = a[9 * 12 + t];
    }
    mm3(W2, Dm2, L2);          // L(k, k-2) = W2 D_{k-2}^-1
    mm3_sub_bt(W2, L2m1, W1);  // W1 = A(k, k-1) - W2 L(k-1, k-2)^T
    mm3(W1, Dm1, L1);          // L(k, k-1) = W1 D_{k-1}^-1
    mm3_sub_bt(W2, L2, D);     // D_k = A(k, k) - W2 L2^T - W1 L1^T
    mm3_sub_bt(W1, L1, D);
    double Di[9];
    mg_inv3(D, Di);
    for (int t = 0; t < 9; ++t) {
      f[t] = (float)L1[t];
      f[9 + t] = (float)L2[t];
      f[18 + t] = (float)Di[t];
      Dm2[t] = Dm1[t];
      Dm1[t] = Di[t];
      L2m1[t] = L2[t];
    }
  }
}

// Residual of the colour's line vertices (items as mg_line_item numbers them).
template <bool WARP>
__global__ void __launch_bounds__(kBlock) k_mg_line_resid(const double* __restrict__ A, const float4* __restrict__ X,
                                                          const double* __restrict__ b, const double* __restrict__ x,
                                                          double* __restrict__ r, int nx, int ny, int dir, int color,
                                                          int items) {
  const int t = mg_item<WARP>();
  int i;
  if (t >= items || !mg_line_item(t, nx, ny, dir, color, i)) return;
  double o[3] = {0.0, 0.0, 0.0};
  const bool pin = mg_pinned(X, i);
  if (!pin) mg_apply<WARP>(A, x, i, nx, ny, o);
  if (WARP && (threadIdx.x & 31) != 0) return;
  for (int a = 0; a < 3; ++a) r[3 * i + a] = pin ? 0.0 : b[3 * i + a] - o[a];
}

// One block per line of the colour: solve the line's block system for the residual in r
// and add the solution to x.  The recurrences are sequential along the line, so the block
// stages the line's factors in chunks into shared memory and one thread runs them there
// (forward substitution writes z over r; backward substitution adds u to x).  The factors
// and the substitutions are float32: a dependent float64 chain costs ~1.6 us per line
// vertex on this GPU (float64 issues at 1/64 of the float32 rate), and a smoother needs no
// more than float32 accuracy; residuals, corrections and the CG stay float64.
constexpr int kLineChunk = 128;

__global__ void __launch_bounds__(256) k_mg_line_solve(const float* __restrict__ F, double* __restrict__ r,
                                                      double* __restrict__ x, int nx, int ny, int dir, int color) {
  __shared__ float sf[kLineChunk * kMgLineFactor];
  __shared__ float sv[kLineChunk * 3];
  const int l = color + 5 * blockIdx.x;
  if (l >= nx + ny - 1) return;
  int x0, y0;
  const int len = mg_line(l, nx, ny, dir, x0, y0);
  auto vert = [&](int k) { return (y0 + k) * nx + x0 + dir * k; };
  float z1[3] = {0.f, 0.f, 0.f}, z2[3] = {0.f, 0.f, 0.f};
  for (int c0 = 0; c0 < len; c0 += kLineChunk) {   // forward: z_k = r_k - L(k,k-1) z_{k-1} - L(k,k-2) z_{k-2}
    const int cn = min(kLineChunk, len - c0);
    for (int t = threadIdx.x; t < cn * 18; t += blockDim.x)
      sf[(t / 18) * kMgLineFactor + t % 18] = F[(size_t)vert(c0 + t / 18) * kMgLineFactor + t % 18];
    for (int t = threadIdx.x; t < cn * 3; t += blockDim.x) sv[t] = (float)r[3 * (size_t)vert(c0 + t / 3) + t % 3];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll 4
      for (int k = 0; k < cn; ++k) {
        const float* f = sf + k * kMgLineFactor;
        float z[3];
        for (int a = 0; a < 3; ++a)
          z[a] = sv[3 * k + a] - (f[3 * a] * z1[0] + f[3 * a + 1] * z1[1] + f[3 * a + 2] * z1[2]) -
                 (f[9 + 3 * a] * z2[0] + f[9 + 3 * a + 1] * z2[1] + f[9 + 3 * a + 2] * z2[2]);
        for (int a = 0; a < 3; ++a) {
          sv[3 * k + a] = z[a];
          z2[a] = z1[a];
          z1[a] = z[a];
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < cn * 3; t += blockDim.x) r[3 * (size_t)vert(c0 + t / 3) + t % 3] = (double)sv[t];
    __syncthreads();
  }
  // backward: u_k = D_k^-1 z_k - L(k+1,k)^T u_{k+1} - L(k+2,k)^T u_{k+2}
  float u1[3] = {0.f, 0.f, 0.f}, u2[3] = {0.f, 0.f, 0.f};
  float L1n[9], L2n[9], L2nn[9];   // L(k+1, k), L(k+1, k-1), L(k+2, k)
  for (int t = 0; t < 9; ++t) L1n[t] = L2n[t] = L2nn[t] = 0.f;
  for (int c1 = len; c1 > 0; c1 -= kLineChunk) {
    const int c0 = max(0, c1 - kLineChunk), cn = c1 - c0;
    for (int t = threadIdx.x; t < cn * kMgLineFactor; t += blockDim.x)
      sf[t] = F[(size_t)vert(c0 + t / kMgLineFactor) * kMgLineFactor + t % kMgLineFactor];
    for (int t = threadIdx.x; t < cn * 3; t += blockDim.x) sv[t] = (float)r[3 * (size_t)vert(c0 + t / 3) + t % 3];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll 4
      for (int k = cn - 1; k >= 0; --k) {
        const float* f = sf + k * kMgLineFactor;
        float u[3];
        for (int a = 0; a < 3; ++a) {
          const float w = f[18 + 3 * a] * sv[3 * k] + f[18 + 3 * a + 1] * sv[3 * k + 1] + f[18 + 3 * a + 2] * sv[3 * k + 2];
          u[a] = w - (L1n[a] * u1[0] + L1n[3 + a] * u1[1] + L1n[6 + a] * u1[2]) -
                 (L2nn[a] * u2[0] + L2nn[3 + a] * u2[1] + L2nn[6 + a] * u2[2]);
        }
        for (int a = 0; a < 3; ++a) {
          sv[3 * k + a] = u[a];
          u2[a] = u1[a];
          u1[a] = u[a];
        }
        for (int t = 0; t < 9; ++t) {
          L2nn[t] = L2n[t];
          L1n[t] = f[t];
          L2n[t] = f[9 + t];
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < cn * 3; t += blockDim.x) x[3 * (size_t)vert(c0 + t / 3) + t % 3] += (double)sv[t];
    __syncthreads();
  }
}

template <bool WARP>
__global__ void __launch_bounds__(kBlock) k_mg_point_gs(const double* __restrict__ A, const double* __restrict__ dinv,
                                                        const double* __restrict__ b, double* __restrict__ x, int nx,
                                                        int ny, int cx, int cy) {
  const int t = mg_item<WARP>();
  if (t >= mg_color_points(nx, ny, 3 * cy + cx)) return;
  const int v = mg_color_point(t, nx, 3 * cy + cx);
  double o[3] = {0.0, 0.0, 0.0};
  mg_apply<WARP>(A, x, v, nx, ny, o);
  if (WARP && (threadIdx.x & 31) != 0) return;
  double r[3];
  for (int a = 0; a < 3; ++a) r[a] = b[3 * v + a] - o[a];
  const double* m = dinv + 9 * (size_t)v;
  for (int a = 0; a < 3; ++a) x[3 * v + a] += m[3 * a] * r[0] + m[3 * a + 1] * r[1] + m[3 * a + 2] * r[2];
}

template <bool WARP>
__global__ void __launch_bounds__(kBlock) k_mg_resid(const double* __restrict__ A, const float4* __restrict__ X,
                                                     const double* __restrict__ b, const double* __restrict__ x,
                                                     double* __restrict__ r, int nx, int ny) {
  const int i = mg_item<WARP>();
  if (i >= nx * ny) return;
  double o[3] = {0.0, 0.0, 0.0};
  const bool pin = mg_pinned(X, i);
  if (!pin) mg_apply<WARP>(A, x, i, nx, ny, o);
  if (WARP && (threadIdx.x & 31) != 0) return;
  for (int a = 0; a < 3; ++a) r[3 * i + a] = pin ? 0.0 : b[3 * i + a] - o[a];
}

__global__ void __launch_bounds__(kBlock) k_mg_restrict(const double* __restrict__ r, int nxf, int nyf,
                                                        double* __restrict__ bc, int nxc, int nyc) {
  XPBD_TID_OR_RETURN(nxc * nyc);
  const int IX = i % nxc, IY = i / nxc;
  double s[3] = {0.0, 0.0, 0.0};
  for (int iy = max(2 * IY - 1, 0); iy <= min(2 * IY + 1, nyf - 1); ++iy) {
    const double wy = mg_w(iy, IY, nyc);
    for (int ix = max(2 * IX - 1, 0); ix <= min(2 * IX + 1, nxf - 1); ++ix) {
      const double w = wy * mg_w(ix, IX, nxc);
      const double* rf = r + 3 * ((size_t)iy * nxf + ix);
      for (int a = 0; a < 3; ++a) s[a] += w * rf[a];
    }
  }
  for (int a = 0; a < 3; ++a) bc[3 * i + a] = s[a];
}

__global__ void __launch_bounds__(kBlock) k_mg_prolong(const double* __restrict__ xc, int nxc, int nyc,
                                                       const float4* __restrict__ X, double* __restrict__ x, int nxf,
                                                       int nyf) {
  XPBD_TID_OR_RETURN(nxf * nyf);
  if (mg_pinned(X, i)) return;
  const int ix = i % nxf, iy = i / nxf;
  double s[3] = {0.0, 0.0, 0.0};
  for (int Y = (iy - 1) / 2; Y <= min((iy + 1) / 2, nyc - 1); ++Y) {
    const double wy = mg_w(iy, Y, nyc);
    for (int Xc = (ix - 1) / 2; Xc <= min((ix + 1) / 2, nxc - 1); ++Xc) {
      const double w = wy * mg_w(ix, Xc, nxc);
      const double* c = xc + 3 * ((size_t)Y * nxc + Xc);
      for (int a = 0; a < 3; ++a) s[a] += w * c[a];
    }
  }
  for (int a = 0; a < 3; ++a) x[3 * i + a] += s[a];
}

// CG with an external preconditioner.
__global__ void __launch_bounds__(kBlock) k_cg_init(const float4* __restrict__ X, const double* __restrict__ b,
                                                    double* __restrict__ y, double* __restrict__ r, int V) {
  XPBD_TID_OR_RETURN(V);
  const bool fr = X[i].w > 0.f;
  for (int a = 0; a < 3; ++a) {
    y[3 * i + a] = 0.0;
    r[3 * i + a] = fr ? b[3 * i + a] : 0.0;
  }
}

template <int NC>
__global__ void __launch_bounds__(kBlock) k_cg_rz(const double* __restrict__ r, const double* __restrict__ z,
                                                  double* __restrict__ p, double* __restrict__ partials, int V) {
  double acc[NC];
  for (int k = 0; k < NC; ++k) acc[k] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      const double rr = r[3 * i + a], zz = z[3 * i + a];
      if (p) p[3 * i + a] = zz;
      acc[0] += rr * zz;
      acc[1] += rr * rr;
      if (NC == 3) acc[NC - 1] += rr * rr;
    }
  }
  block_sum_store<NC>(acc, partials + NC * blockIdx.x);
}

__global__ void __launch_bounds__(kBlock) k_cg_update(const double* __restrict__ sc, int rz_slot, const double* __restrict__ p,
                                                      const double* __restrict__ q, double* __restrict__ y,
                                                      double* __restrict__ r, int V) {
  const double pq = sc[0];
  const double alpha = pq != 0.0 ? sc[rz_slot] / pq : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * V; i += gridDim.x * blockDim.x) {
    y[i] += alpha * p[i];
    r[i] -= alpha * q[i];
  }
}

}  // namespace

void launch_mg_asm_mass_contacts(const float4* X, const uint8_t* cflags, const float2* lamc, Collide c, bool pd,
                                 double* A0, int V, cudaStream_t s) {
  if (V > 0) k_mg_mass_contacts<<<grid_for(V), kBlock, 0, s>>>(X, cflags, lamc, c, pd, A0, V);
}

void launch_mg_asm_block(SegType t, const void* rec, int n, const float4* X, const float* lam, const double* blocks,
                         bool pd, double* A0, int nx, int V, double* flag, cudaStream_t s) {
  if (n <= 0) return;
  if (t == SEG_DIST)
    k_mg_asm_dist<<<grid_for(n), kBlock, 0, s>>>((const DistRec*)rec, n, X, lam, pd, A0, nx, V, flag);
  else if (t == SEG_BEND)
    k_mg_asm_quad<BendRec><<<grid_for(n), kBlock, 0, s>>>((const BendRec*)rec, n, blocks, A0, nx, V, flag);
  else
    k_mg_asm_quad<TetRec><<<grid_for(n), kBlock, 0, s>>>((const TetRec*)rec, n, blocks, A0, nx, V, flag);
}

void launch_mg_asm_memb(const MembRec* rec, int n, const double* blocks, double* A0, int nx, int V, double* flag,
                        cudaStream_t s) {
  if (n > 0) k_mg_asm_memb<<<grid_for(n), kBlock, 0, s>>>(rec, n, blocks, A0, nx, V, flag);
}

void launch_mg_rap(const MgLevel& f, const MgLevel& c, const float4* X, cudaStream_t s) {
  const int n = c.nx * c.ny * kMgSlots;
  k_mg_rap<<<grid_for(n), kBlock, 0, s>>>(f.A, f.nx, f.ny, X, c.A, c.nx, c.ny);
}

void launch_mg_dinv(const MgLevel& l, const float4* X, cudaStream_t s) {
  const int n = l.nx * l.ny;
  k_mg_dinv<<<grid_for(n), kBlock, 0, s>>>(l.A, X, l.dinv, n);
}

void launch_mg_coarse_inverse(const MgLevel& l, const float4* X, double* cinv, cudaStream_t s) {
  k_mg_coarse_inverse<<<1, 256, 0, s>>>(l.A, X, l.nx, l.ny, cinv);
}

void launch_mg_line_factor(const MgLevel& l, const float4* X, int dir, float* lfac, cudaStream_t s) {
  const int lines = l.nx + l.ny - 1;
  k_mg_line_factor<<<grid_for(lines), kBlock, 0, s>>>(l.A, X, l.nx, l.ny, dir, lfac);
}

// Rows per launch up to which a warp per row beats a thread per row (one warp per row
// keeps at most ~7 warps per SM sub-partition busy; beyond that the thread form's fewer
// instructions win).
constexpr int kMgWarpRows = 4096;

void launch_mg_point_gs(const MgLevel& l, const double* b, double* x, int color, cudaStream_t s) {
  const int cx = color % 3, cy = color / 3;
  const int n = mg_color_points(l.nx, l.ny, color);
  if (n <= 0) return;
  if (n <= kMgWarpRows)
    k_mg_point_gs<true><<<(n * 32 + kBlock - 1) / kBlock, kBlock, 0, s>>>(l.A, l.dinv, b, x, l.nx, l.ny, cx, cy);
  else
    k_mg_point_gs<false><<<grid_for(n), kBlock, 0, s>>>(l.A, l.dinv, b, x, l.nx, l.ny, cx, cy);
}

void launch_mg_line_resid(const MgLevel& l, const float4* X, const double* b, const double* x, double* r, int dir,
                          int color, cudaStream_t s) {
  const int n = mg_line_items(l.nx, l.ny, color);
  if (n <= 0) return;
  if (n <= kMgWarpRows)
    k_mg_line_resid<true><<<(n * 32 + kBlock - 1) / kBlock, kBlock, 0, s>>>(l.A, X, b, x, r, l.nx, l.ny, dir, color, n);
  else
    k_mg_line_resid<false><<<grid_for(n), kBlock, 0, s>>>(l.A, X, b, x, r, l.nx, l.ny, dir, color, n);
}

void launch_mg_line_solve(const MgLevel& l, const float* lfac, double* r, double* x, int dir, int color,
                          cudaStream_t s) {
  const int lines = mg_color_lines(l.nx, l.ny, color);
  if (lines > 0) k_mg_line_solve<<<lines, 256, 0, s>>>(lfac, r, x, l.nx, l.ny, dir, color);
}

void launch_mg_resid(const MgLevel& l, const float4* X, const double* b, const double* x, double* r, cudaStream_t s) {
  const int n = l.nx * l.ny;
  if (n <= kMgWarpRows)
    k_mg_resid<true><<<(n * 32 + kBlock - 1) / kBlock, kBlock, 0, s>>>(l.A, X, b, x, r, l.nx, l.ny);
  else
    k_mg_resid<false><<<grid_for(n), kBlock, 0, s>>>(l.A, X, b, x, r, l.nx, l.ny);
}

void launch_mg_restrict(const MgLevel& f, const double* r, const MgLevel& c, double* bc, cudaStream_t s) {
  const int n = c.nx * c.ny;
  k_mg_restrict<<<grid_for(n), kBlock, 0, s>>>(r, f.nx, f.ny, bc, c.nx, c.ny);
}

void launch_mg_prolong(const MgLevel& c, const double* xc, const MgLevel& f, const float4* X, double* x,
                       cudaStream_t s) {
  const int n = f.nx * f.ny;
  k_mg_prolong<<<grid_for(n), kBlock, 0, s>>>(xc, c.nx, c.ny, X, x, f.nx, f.ny);
}

void launch_mg_coarse_solve(const MgLevel& l, const double* cinv, const double* b, double* x, cudaStream_t s) {
  k_mg_coarse_solve<<<1, 256, 0, s>>>(cinv, b, x, 3 * l.nx * l.ny);
}

void launch_cg_init(const float4* X, const double* b, double* y, double* r, int V, cudaStream_t s) {
  if (V > 0) k_cg_init<<<grid_for(V), kBlock, 0, s>>>(X, b, y, r, V);
}

void launch_cg_rz(const double* r, const double* z, double* p, double* partials, int ncomp, int V, cudaStream_t s) {
  if (ncomp == 3)
    k_cg_rz<3><<<partial_blocks(V), kBlock, 0, s>>>(r, z, p, partials, V);
  else
    k_cg_rz<2><<<partial_blocks(V), kBlock, 0, s>>>(r, z, p, partials, V);
}

void launch_cg_update(const double* sc, int rz_slot, const double* p, const double* q, double* y, double* r, int V,
                      cudaStream_t s) {
  k_cg_update<<<partial_blocks(V), kBlock, 0, s>>>(sc, rz_slot, p, q, y, r, V);
}

}  // namespace xpbd
