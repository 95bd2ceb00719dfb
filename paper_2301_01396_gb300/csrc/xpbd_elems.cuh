// Per-element device functions of the XPBD step and of its discrete adjoint.
//
// Every kernel of the library is one of these functions applied to an index range: the
// one-request kernels (xpbd_kernels.cu) launch them over a whole color or vertex array,
// and the batched serving kernel (xpbd_serve.cu) dispatches them from a work table.  Both
// call exactly this code, so a request computes the same values in either path.
//
// Layout in HBM: vertices as float4 (x, y, z, inverse mass); constraint records of one
// color contiguous and sorted by first vertex (coalesced gathers along grid rows);
// multipliers lambda as float in record order; the reverse sweep's per-iteration tape
// holds the pre-projection float4 of every vertex of every constraint, in record order.
//
// One thread updates one constraint of the current color: a color's constraints are
// vertex-disjoint (Sec. 3.1, graph coloring), so the Jacobi update inside a color equals
// the sequential Gauss-Seidel order.  The path is gather/scatter bound (no dense
// contraction): 128-bit vertex and record accesses, streaming (evict-first) hints on
// single-use data, evict-last on the vertex arrays that every color pass re-reads.
#pragma once

#include "xpbd_kernels.cuh"

namespace xpbd {

__device__ __forceinline__ f3 xyz(float4 a) { return mk3(a.x, a.y, a.z); }
__device__ __forceinline__ float4 with_w(f3 a, float w) { return make_float4(a.x, a.y, a.z, w); }

__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldcs(p); }
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }

// ------------------------------------------------------------------ cache policy
// XPBD_L2_VERTEX_HINT marks vertex traffic L2 evict-last (a fraction
// XPBD_L2_VERTEX_FRACTION of the lines) so the streams evict it last; XPBD_REC_STREAM
// loads records with the streaming (evict-first) hint.  Both are on by default: on the
// 2950^2 cloth they cut the forward and replay passes by 7-13% (CUDA events per class).
#ifndef XPBD_L2_VERTEX_HINT
#define XPBD_L2_VERTEX_HINT 1
#endif
#ifndef XPBD_L2_VERTEX_FRACTION
#define XPBD_L2_VERTEX_FRACTION 1.0
#endif
#ifndef XPBD_REC_STREAM
#define XPBD_REC_STREAM 1
#endif
#define XPBD_STR2(x) #x
#define XPBD_STR(x) XPBD_STR2(x)

__device__ __forceinline__ uint64_t vtx_policy() {
#if XPBD_L2_VERTEX_HINT
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, " XPBD_STR(XPBD_L2_VERTEX_FRACTION) ";" : "=l"(p));
  return p;
#else
  return 0;
#endif
}

__device__ __forceinline__ float4 ld_vtx(const float4* a, uint64_t pol) {
#if XPBD_L2_VERTEX_HINT
  float4 v;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(a), "l"(pol));
  return v;
#else
  (void)pol;
  return *a;
#endif
}

__device__ __forceinline__ void st_vtx(float4* a, float4 v, uint64_t pol) {
#if XPBD_L2_VERTEX_HINT
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w), "l"(pol)
               : "memory");
#else
  (void)pol;
  *a = v;
#endif
}

// Vertex access of the element functions: global memory with the L2 hint (SH = false), or a
// shared-memory copy of a group's vertices addressed by local index (SH = true).
template <bool SH>
__device__ __forceinline__ float4 vload(const float4* a, uint64_t pol) {
  if constexpr (SH) {
    (void)pol;
    return *a;
  } else {
    return ld_vtx(a, pol);
  }
}
template <bool SH>
__device__ __forceinline__ void vstore(float4* a, float4 v, uint64_t pol) {
  if constexpr (SH) {
    (void)pol;
    *a = v;
  } else {
    st_vtx(a, v, pol);
  }
}

// A record of 16, 32 or 64 bytes as 128-bit loads (streaming hint when XPBD_REC_STREAM).
template <class Rec>
__device__ __forceinline__ Rec ld_rec(const Rec* p) {
#if XPBD_REC_STREAM
  static_assert(sizeof(Rec) % 16 == 0, "records are 16-byte multiples");
  union {
    int4 v[sizeof(Rec) / 16];
    Rec r;
  } u;
  const int4* q = reinterpret_cast<const int4*>(p);
#pragma unroll
  for (int k = 0; k < (int)(sizeof(Rec) / 16); ++k) u.v[k] = __ldcs(q + k);
  return u.r;
#else
  return *p;
#endif
}

// ------------------------------------------------------------------ deterministic reductions
// Block-wide sum of NC doubles; thread 0 writes the block's partial sums.  The order of
// additions depends only on the launch shape, so results are bitwise reproducible.  Every
// thread of the block must call it.
template <int NC>
__device__ __forceinline__ void block_sum_store(double v[NC], double* out) {
  __shared__ double sh[NC][kBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double x = v[c];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[c][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double t = 0.0;
      for (int w = 0; w < kBlock / 32; ++w) t += sh[c][w];
      out[c] = t;
    }
  }
  __syncthreads();
}

// One block sums nblocks x ncomp partials (row-major) in a fixed order into out[0..ncomp).
__device__ __forceinline__ void reduce_partials_block(const double* __restrict__ partials, int nblocks,
                                                      int ncomp, double* __restrict__ out, bool accumulate) {
  __shared__ double sh[kBlock];
  for (int c = 0; c < ncomp; ++c) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) t += partials[ncomp * b + c];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = accumulate ? out[c] + sh[0] : sh[0];
    __syncthreads();
  }
}

// ======================================================================== forward

__device__ __forceinline__ void init_ckpt_elem(int i, const float* __restrict__ x0, const float* __restrict__ v0,
                                               const float* __restrict__ w, float4* __restrict__ ckx,
                                               float4* __restrict__ ckv) {
  ckx[i] = make_float4(x0[3 * i], x0[3 * i + 1], x0[3 * i + 2], w[i]);
  ckv[i] = make_float4(v0[3 * i], v0[3 * i + 1], v0[3 * i + 2], 0.f);
}

// alpha~ of record i from the caller's per-constraint compliance (caller order).  A
// compliance that is negative or not finite sets bit 1 of the error word.  Padding records
// (perm -1) keep alpha~ = 0.
template <class Rec, bool VOL>
__device__ __forceinline__ void set_alpha_elem(int i, Rec* __restrict__ rec, const int* __restrict__ perm,
                                               const float* __restrict__ compliance, float inv_dt2,
                                               int* __restrict__ err) {
  const int j = perm[i];
  if (j < 0) return;
  float c = compliance[j];
  if (!(c >= 0.f) || isinf(c)) atomicOr(err, 2);
  float a = c * inv_dt2;
  if constexpr (VOL) a = a / rec[i].vol;
  rec[i].at = a;
}

// Inertial prediction (Eq. xpbdUpdateRule): p = x + dt v + dt^2 (w (G_n + W_i + F_{n,i}) + [w > 0] g),
// and contact detection at p: a contact is active for the whole step when C(p) < 0.
// fvs_n: step n's force per vertex F_{n,i} (the keyframe example's controls), or NULL.
__device__ __forceinline__ void predict_elem(int i, const float4* __restrict__ ckx, const float4* __restrict__ ckv,
                                             float4* __restrict__ P, const float* __restrict__ fg_n,
                                             const float* __restrict__ fv, const float* __restrict__ fvs_n,
                                             float dt, float gx, float gy, float gz, const Collide& c,
                                             uint8_t* __restrict__ cflags) {
  float4 x = ckx[i];
  float4 v = ckv[i];
  float w = x.w;
  float fx = 0.f, fy = 0.f, fz = 0.f;
  if (fg_n) { fx = fg_n[0]; fy = fg_n[1]; fz = fg_n[2]; }
  if (fv) { fx += fv[3 * i]; fy += fv[3 * i + 1]; fz += fv[3 * i + 2]; }
  if (fvs_n) { fx += fvs_n[3 * i]; fy += fvs_n[3 * i + 1]; fz += fvs_n[3 * i + 2]; }
  float free_ = w > 0.f ? 1.f : 0.f;
  float dt2 = dt * dt;
  float4 p;
  p.x = x.x + dt * v.x + dt2 * (w * fx + free_ * gx);
  p.y = x.y + dt * v.y + dt2 * (w * fy + free_ * gy);
  p.z = x.z + dt * v.z + dt2 * (w * fz + free_ * gz);
  p.w = w;
  P[i] = p;
  if (c.flags) {
    uint8_t f = 0;
    if ((c.flags & 1) && (p.y - c.h - c.thick < 0.f)) f |= 1;
    if (c.flags & 2) {
      float dx = p.x - c.cx, dy = p.y - c.cy, dz = p.z - c.cz;
      if (sqrtf(dx * dx + dy * dy + dz * dz) - c.r - c.thick < 0.f) f |= 2;
    }
    cflags[i] = f;
  }
}

// ---- distance: C = |x_a - x_b| - L, grad_a = n = (x_a - x_b)/l, grad_b = -n.
// One update on values in registers: returns false (nothing changes) for a degenerate
// constraint, else updates pa, pb and lam.
__device__ __forceinline__ bool dist_step(const DistRec& r, float4& pa, float4& pb, float& lam) {
  f3 d = xyz(pa) - xyz(pb);
  float l2 = dot(d, d);
  float D = pa.w + pb.w + r.at;
  if (!(l2 >= XPBD_DEGEN2 && D > 0.f)) return false;
  float il = rsqrtf(l2);
  float l = l2 * il;
  f3 nrm = d * il;
  float dl = (-(l - r.L) - r.at * lam) / D;
  lam += dl;
  pa = with_w(xyz(pa) + nrm * (pa.w * dl), pa.w);
  pb = with_w(xyz(pb) - nrm * (pb.w * dl), pb.w);
  return true;
}

// lam_in and lam_out may alias (in-place forward), so they are not __restrict__.
template <bool SH = false>
__device__ __forceinline__ float proj_dist_core(const DistRec& r, float4* __restrict__ P, float lam,
                                                float4* __restrict__ tape2, int ts = 1) {
  const uint64_t pol = SH ? 0 : vtx_policy();
  float4 pa = vload<SH>(P + r.a, pol);
  float4 pb = vload<SH>(P + r.b, pol);
  if (tape2) {   // the two pre-projection positions, ts float4 apart
    __stcs(tape2, pa);
    __stcs(tape2 + ts, pb);
  }
  if (dist_step(r, pa, pb, lam)) {
    vstore<SH>(P + r.a, pa, pol);
    vstore<SH>(P + r.b, pb, pol);
  }
  return lam;
}

template <bool SH = false>
__device__ __forceinline__ void proj_dist_elem(int i, const DistRec* __restrict__ rec, float4* __restrict__ P,
                                               const float* lam_in, float* lam_out, float4* __restrict__ tape) {
  const DistRec r = ld_rec(rec + i);
  const float lam = lam_in ? ld_stream(lam_in + i) : 0.f;
  __stcs(lam_out + i, proj_dist_core<SH>(r, P, lam, tape ? tape + 2 * i : nullptr));
}

// ---- 4-vertex constraints (bending, tet C_H, tet C_D), in relative coordinates
// e1 = x1 - x0, e2 = x2 - x0, e3 = x3 - x0 (all three constraints are translation
// invariant): grad_0 = -(grad_1 + grad_2 + grad_3) and (H u)_0 = -sum_k (H u)_k.
template <int KIND>   // 1 bending, 2 hydrostatic, 3 deviatoric
struct Quad;

template <>
struct Quad<1> {
  typedef BendRec Rec;
  // value and gradient (g1..g3); false if degenerate
  __device__ static bool eval(const Rec& r, const f3& e1, const f3& e2, const f3& e3, f3& g1, f3& g2,
                              f3& g3, float& C) {
    if (bend_degenerate_rel(e1, e2, e3)) return false;
    bend_grad_rel<float>(e1, e2, e3, g1, g2, g3);
    C = bend_C_rel(e1, e2, e3, r.theta0);
    return true;
  }
  // gradient (value parts) and H u (derivative parts) for relative directions du1..du3
  __device__ static void hvp(const Rec& r, const f3& e1, const f3& e2, const f3& e3, const f3& du1,
                             const f3& du2, const f3& du3, d3& g1, d3& g2, d3& g3) {
    bend_grad_rel<df>(mkd3(e1, du1), mkd3(e2, du2), mkd3(e3, du3), g1, g2, g3);
  }
  // H u alone (relative rows 1..3), in closed form
  __device__ static void hvp_f(const Rec& r, const f3& e1, const f3& e2, const f3& e3, const f3& du1,
                               const f3& du2, const f3& du3, f3& h1, f3& h2, f3& h3) {
    bend_hvp_rel(e1, e2, e3, du1, du2, du3, h1, h2, h3);
  }
};

template <bool HYDRO>
struct TetQuad {
  typedef TetRec Rec;
  __device__ static bool eval(const Rec& r, const f3& e1, const f3& e2, const f3& e3, f3& g1, f3& g2,
                              f3& g3, float& C) {
    tet_grad_rel<HYDRO, float>(e1, e2, e3, r.B, g1, g2, g3, &C, r.gamma);
    if (!HYDRO && C * C < XPBD_DEGEN2) return false;
    return true;
  }
  __device__ static void hvp(const Rec& r, const f3& e1, const f3& e2, const f3& e3, const f3& du1,
                             const f3& du2, const f3& du3, d3& g1, d3& g2, d3& g3) {
    tet_grad_rel<HYDRO, df>(mkd3(e1, du1), mkd3(e2, du2), mkd3(e3, du3), r.B, g1, g2, g3, nullptr,
                            r.gamma);
  }
  __device__ static void hvp_f(const Rec& r, const f3& e1, const f3& e2, const f3& e3, const f3& du1,
                               const f3& du2, const f3& du3, f3& h1, f3& h2, f3& h3) {
    d3 g1, g2, g3;
    hvp(r, e1, e2, e3, du1, du2, du3, g1, g2, g3);
    h1 = dpart(g1);
    h2 = dpart(g2);
    h3 = dpart(g3);
  }
};
template <> struct Quad<2> : TetQuad<true> {};
template <> struct Quad<3> : TetQuad<false> {};

template <int KIND, bool SH = false>
__device__ __forceinline__ float proj_quad_core(const typename Quad<KIND>::Rec& r, float4* __restrict__ P,
                                                float lam, float4* __restrict__ tape4, int ts = 1) {
  const uint64_t pol = SH ? 0 : vtx_policy();
  float4 p[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) p[k] = vload<SH>(P + r.v[k], pol);
  if (tape4) {
#pragma unroll
    for (int k = 0; k < 4; ++k) __stcs(tape4 + k * ts, p[k]);
  }
  const f3 x0 = xyz(p[0]);
  const f3 e1 = xyz(p[1]) - x0, e2 = xyz(p[2]) - x0, e3 = xyz(p[3]) - x0;
  f3 g1, g2, g3;
  float C;
  if (Quad<KIND>::eval(r, e1, e2, e3, g1, g2, g3, C)) {
    const f3 g0 = -(g1 + g2 + g3);
    float D = r.at + p[0].w * dot(g0, g0) + p[1].w * dot(g1, g1) + p[2].w * dot(g2, g2) +
              p[3].w * dot(g3, g3);
    if (D > 0.f) {
      float dl = (-C - r.at * lam) / D;
      lam += dl;
      vstore<SH>(P + r.v[0], with_w(x0 + g0 * (p[0].w * dl), p[0].w), pol);
      vstore<SH>(P + r.v[1], with_w(xyz(p[1]) + g1 * (p[1].w * dl), p[1].w), pol);
      vstore<SH>(P + r.v[2], with_w(xyz(p[2]) + g2 * (p[2].w * dl), p[2].w), pol);
      vstore<SH>(P + r.v[3], with_w(xyz(p[3]) + g3 * (p[3].w * dl), p[3].w), pol);
    }
  }
  return lam;
}

template <int KIND, bool SH = false>
__device__ __forceinline__ void proj_quad_elem(int i, const typename Quad<KIND>::Rec* __restrict__ rec,
                                               float4* __restrict__ P, const float* lam_in, float* lam_out,
                                               float4* __restrict__ tape) {
  const typename Quad<KIND>::Rec r = ld_rec(rec + i);
  const float lam = lam_in ? ld_stream(lam_in + i) : 0.f;
  __stcs(lam_out + i, proj_quad_core<KIND, SH>(r, P, lam, tape ? tape + 4 * i : nullptr));
}

// ---- contacts (Sec. 4.6): plane then sphere on the same vertex, equality springs for the
// step in which they were detected
__device__ __forceinline__ void plane_project(f3& p, float w, float& lam, const Collide& c) {
  float C = p.y - c.h - c.thick;
  float D = w + c.at;
  if (D > 0.f) {
    float dl = (-C - c.at * lam) / D;
    lam += dl;
    p.y += w * dl;
  }
}

__device__ __forceinline__ void sphere_project(f3& p, float w, float& lam, const Collide& c) {
  f3 d = p - mk3(c.cx, c.cy, c.cz);
  float l2 = dot(d, d);
  float D = w + c.at;
  if (l2 >= XPBD_DEGEN2 && D > 0.f) {
    float il = rsqrtf(l2);
    float l = l2 * il;
    f3 nrm = d * il;
    float dl = (-(l - c.r - c.thick) - c.at * lam) / D;
    lam += dl;
    p = p + nrm * (w * dl);
  }
}

__device__ __forceinline__ void contact_elem(int i, float4* __restrict__ P, const uint8_t* __restrict__ cflags,
                                             const float2* lam_in, float2* lam_out, float4* __restrict__ tape,
                                             const Collide& c) {
  uint8_t f = cflags[i];
  if (!f) return;
  float4 p4 = P[i];
  if (tape) __stcs(tape + i, p4);
  float2 lam = lam_in ? lam_in[i] : make_float2(0.f, 0.f);
  f3 p = xyz(p4);
  if (f & 1) plane_project(p, p4.w, lam.x, c);
  if (f & 2) sphere_project(p, p4.w, lam.y, c);
  P[i] = with_w(p, p4.w);
  lam_out[i] = lam;
}

// Velocity update (Eq. xpbdUpdateRule): v_{n+1} = (x_{n+1} - x_n)/dt; flags non-finite state.
__device__ __forceinline__ void velocity_elem(int i, const float4* __restrict__ P, const float4* __restrict__ ckx_n,
                                              float4* __restrict__ ckx_next, float4* __restrict__ ckv_next,
                                              float inv_dt, int* __restrict__ err) {
  float4 p = P[i];
  float4 x = ckx_n[i];
  float4 v = make_float4((p.x - x.x) * inv_dt, (p.y - x.y) * inv_dt, (p.z - x.z) * inv_dt, 0.f);
  ckx_next[i] = p;
  ckv_next[i] = v;
  if (!isfinite(p.x + p.y + p.z + v.x + v.y + v.z)) atomicOr(err, 1);
}

// ======================================================================== reverse

__device__ __forceinline__ void seed_adjoint_elem(int i, const float* __restrict__ sx, const float* __restrict__ sv,
                                                  float4* __restrict__ xbar, float4* __restrict__ vbar) {
  xbar[i] = sx ? make_float4(sx[3 * i], sx[3 * i + 1], sx[3 * i + 2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
  vbar[i] = sv ? make_float4(sv[3 * i], sv[3 * i + 1], sv[3 * i + 2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Adjoint of v_{n+1} = (p - x_n)/dt, x_{n+1} = p:  pbar = xbar + vbar/dt, xbar_n = -vbar/dt.
// In place: xbar <- pbar, vbar <- the partial xbar_n.
__device__ __forceinline__ void adj_begin_elem(int i, float4* __restrict__ xbar, float4* __restrict__ vbar,
                                               float inv_dt) {
  float4 xb = xbar[i], vb = vbar[i];
  xbar[i] = make_float4(xb.x + vb.x * inv_dt, xb.y + vb.y * inv_dt, xb.z + vb.z * inv_dt, 0.f);
  vbar[i] = make_float4(-vb.x * inv_dt, -vb.y * inv_dt, -vb.z * inv_dt, 0.f);
}

// Reverse of one XPBD update.  With the pre-projection state from the tape, g = grad C,
// D = sum w|g|^2 + alpha~, dlambda = (-C - alpha~ lambda)/D recomputed, and the adjoints
// xbar', lambar' of the updated values:
//   s = lambar' + sum_i w_i g_i . xbar'_i                 (adjoint of dlambda)
//   u_i = dlambda w_i xbar'_i - 2 (s dlambda / D) w_i g_i (adjoint of g_i)
//   xbar_i = xbar'_i - (s/D) g_i + (H u)_i,  lambar = lambar' - (alpha~/D) s,
//   alphabar~ += -s (lambda + dlambda) / D.
// These are the terms of Sec. 4.4 (J = D, dJ/dx dlambda, db/dx = -grad C - alpha~ ...)
// applied in reverse mode to the sequence of single-constraint updates.  `first`: the
// first reverse iteration of a step (lambar', alphabar' start at 0); `last`: fold the step's
// alphabar into the float64 accumulator.
__device__ __forceinline__ void lb_finish(int i, float lambar, float abar, float2* __restrict__ lb,
                                          double* __restrict__ acc, bool last) {
  if (last)
    acc[i] += (double)abar;
  else
    lb[i] = make_float2(lambar, abar);
}

// Reverse of one distance update from its tape (pa, pb), multiplier before the update and
// (lambar', alphabar'); updates the two vertex adjoints and returns (lambar, alphabar).
template <bool SH = false>
__device__ __forceinline__ float2 vjp_dist_core(const DistRec& r, float4 pa, float4 pb, float lam, float2 l,
                                                float4* __restrict__ xbar) {
  const uint64_t pol = SH ? 0 : vtx_policy();
  f3 d = xyz(pa) - xyz(pb);
  float l2 = dot(d, d);
  float D = pa.w + pb.w + r.at;
  if (l2 >= XPBD_DEGEN2 && D > 0.f) {
    float il = rsqrtf(l2);
    float len = l2 * il;
    f3 nrm = d * il;
    float dl = (-(len - r.L) - r.at * lam) / D;
    float4 xa4 = vload<SH>(xbar + r.a, pol), xb4 = vload<SH>(xbar + r.b, pol);
    f3 xa = xyz(xa4), xb = xyz(xb4);
    float s = l.x + pa.w * dot(nrm, xa) - pb.w * dot(nrm, xb);
    // H u for the distance constraint: (P (u_a - u_b))/l on a, the negative on b, with
    // P = I - n n^T; the n-parallel part of u drops out.
    f3 t = (xa * pa.w - xb * pb.w) * dl;
    f3 hv = (t - nrm * dot(nrm, t)) * il;
    float sD = s / D;
    xa = xa - nrm * sD + hv;
    xb = xb + nrm * sD - hv;
    vstore<SH>(xbar + r.a, with_w(xa, 0.f), pol);
    vstore<SH>(xbar + r.b, with_w(xb, 0.f), pol);
    l.y += -sD * (lam + dl);
    l.x -= r.at * sD;
  }
  return l;
}

template <bool SH = false>
__device__ __forceinline__ void vjp_dist_elem(int i, const DistRec* __restrict__ rec, const float4* __restrict__ tape,
                                              const float* __restrict__ lam_pre, float4* __restrict__ xbar,
                                              float2* __restrict__ lb, double* __restrict__ acc, bool first,
                                              bool last) {
  const DistRec r = ld_rec(rec + i);
  float4 pa = ld_stream(tape + 2 * i), pb = ld_stream(tape + 2 * i + 1);
  float lam = lam_pre ? ld_stream(lam_pre + i) : 0.f;
  float2 l = first ? make_float2(0.f, 0.f) : lb[i];
  l = vjp_dist_core<SH>(r, pa, pb, lam, l, xbar);
  lb_finish(i, l.x, l.y, lb, acc, last);
}

// Reverse of one 4-vertex update from its tape p[0..3]; see vjp_dist_core.
template <int KIND, bool SH = false>
__device__ __forceinline__ float2 vjp_quad_core(const typename Quad<KIND>::Rec& r, const float4 (&p)[4], float lam,
                                                float2 l, float4* __restrict__ xbar) {
  const uint64_t pol = SH ? 0 : vtx_policy();
  float4 xb4[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) xb4[k] = vload<SH>(xbar + r.v[k], pol);
  const f3 x0 = xyz(p[0]);
  const f3 e1 = xyz(p[1]) - x0, e2 = xyz(p[2]) - x0, e3 = xyz(p[3]) - x0;
  f3 g1, g2, g3;
  float C;
  if (Quad<KIND>::eval(r, e1, e2, e3, g1, g2, g3, C)) {
    const f3 g0 = -(g1 + g2 + g3);
    const float w0 = p[0].w, w1 = p[1].w, w2 = p[2].w, w3 = p[3].w;
    float D = r.at + w0 * dot(g0, g0) + w1 * dot(g1, g1) + w2 * dot(g2, g2) + w3 * dot(g3, g3);
    if (D > 0.f) {
      float dl = (-C - r.at * lam) / D;
      const f3 xb0 = xyz(xb4[0]), xb1 = xyz(xb4[1]), xb2 = xyz(xb4[2]), xb3 = xyz(xb4[3]);
      float s = l.x + w0 * dot(g0, xb0) + w1 * dot(g1, xb1) + w2 * dot(g2, xb2) + w3 * dot(g3, xb3);
      float sD = s / D;
      float c2 = 2.f * sD * dl;
      const f3 u0 = (xb0 * dl - g0 * c2) * w0;
      const f3 du1 = (xb1 * dl - g1 * c2) * w1 - u0;
      const f3 du2 = (xb2 * dl - g2 * c2) * w2 - u0;
      const f3 du3 = (xb3 * dl - g3 * c2) * w3 - u0;
      f3 hu1, hu2, hu3;
      Quad<KIND>::hvp_f(r, e1, e2, e3, du1, du2, du3, hu1, hu2, hu3);
      const f3 hu0 = -(hu1 + hu2 + hu3);
      vstore<SH>(xbar + r.v[0], with_w(xb0 - g0 * sD + hu0, 0.f), pol);
      vstore<SH>(xbar + r.v[1], with_w(xb1 - g1 * sD + hu1, 0.f), pol);
      vstore<SH>(xbar + r.v[2], with_w(xb2 - g2 * sD + hu2, 0.f), pol);
      vstore<SH>(xbar + r.v[3], with_w(xb3 - g3 * sD + hu3, 0.f), pol);
      l.y += -sD * (lam + dl);
      l.x -= r.at * sD;
    }
  }
  return l;
}

template <int KIND, bool SH = false>
__device__ __forceinline__ void vjp_quad_elem(int i, const typename Quad<KIND>::Rec* __restrict__ rec,
                                              const float4* __restrict__ tape, const float* __restrict__ lam_pre,
                                              float4* __restrict__ xbar, float2* __restrict__ lb,
                                              double* __restrict__ acc, bool first, bool last) {
  const typename Quad<KIND>::Rec r = ld_rec(rec + i);
  // every global read is independent of the arithmetic: issue them all first
  float4 p[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) p[k] = ld_stream(tape + 4 * i + k);
  float lam = lam_pre ? ld_stream(lam_pre + i) : 0.f;
  float2 l = first ? make_float2(0.f, 0.f) : lb[i];
  l = vjp_quad_core<KIND, SH>(r, p, lam, l, xbar);
  lb_finish(i, l.x, l.y, lb, acc, last);
}

// ---- coupled tet update: a tet's C_H and C_D from one 2x2 system (the update of the
// neo-Hookean constraint pair that the volumetric model of Sec. 3.2 follows, Macklin and
// Mueller 2021):  S dlambda = -C - A~ lambda,  S = G W G^T + A~,  x += W G^T dlambda.
// det S is formed as a (b_perp + at_D) + at_H (b + at_D), a = |g_H|^2_W, b = |g_D|^2_W and
// b_perp the W-norm of the part of g_D orthogonal to g_H: non-negative terms only, free of
// the cancellation in s11 s22 - s12^2 when the gradients are nearly parallel (at the rest
// shape they are parallel).  When C_D is degenerate only C_H is projected.
struct TetPair {
  f3 h[4], d[4];   // per-vertex gradients of C_H and C_D (d unset unless `both`)
  float Ch, Cd, s11, s12, s22, det;
  bool both;       // false: C_D degenerate, C_H alone with D = s11
};

__device__ __forceinline__ void tet_pair_eval(const TetRec& r, float atd, const float4 (&p)[4], TetPair& T) {
  const f3 x0 = xyz(p[0]);
  const f3 e1 = xyz(p[1]) - x0, e2 = xyz(p[2]) - x0, e3 = xyz(p[3]) - x0;
  tet_grad_rel<true, float>(e1, e2, e3, r.B, T.h[1], T.h[2], T.h[3], &T.Ch, r.gamma);
  T.h[0] = -(T.h[1] + T.h[2] + T.h[3]);
  float a = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) a += p[k].w * dot(T.h[k], T.h[k]);
  T.s11 = r.at + a;
  tet_grad_rel<false, float>(e1, e2, e3, r.B, T.d[1], T.d[2], T.d[3], &T.Cd, r.gamma);
  T.both = !(T.Cd * T.Cd < XPBD_DEGEN2);
  if (!T.both) return;
  T.d[0] = -(T.d[1] + T.d[2] + T.d[3]);
  float b = 0.f, c = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    b += p[k].w * dot(T.d[k], T.d[k]);
    c += p[k].w * dot(T.h[k], T.d[k]);
  }
  float bp = b;
  if (a > 0.f) {
    const float beta = c / a;
    bp = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const f3 o = T.d[k] - T.h[k] * beta;
      bp += p[k].w * dot(o, o);
    }
  }
  T.s12 = c;
  T.s22 = atd + b;
  T.det = a * (bp + atd) + r.at * (b + atd);
}

// Multiplier increments of the pair (dlambda_D = 0 when C_D is degenerate); false when
// the system is singular and nothing moves.
__device__ __forceinline__ bool tet_pair_solve(const TetPair& T, float ath, float atd, float2 lam, float& dlh,
                                               float& dld) {
  if (!T.both) {
    if (!(T.s11 > 0.f)) return false;
    dlh = (-T.Ch - ath * lam.x) / T.s11;
    dld = 0.f;
    return true;
  }
  if (!(T.det > 0.f)) return false;
  const float rh = -T.Ch - ath * lam.x, rd = -T.Cd - atd * lam.y;
  const float inv = 1.f / T.det;
  dlh = (T.s22 * rh - T.s12 * rd) * inv;
  dld = (T.s11 * rd - T.s12 * rh) * inv;
  return true;
}

template <bool SH = false>
__device__ __forceinline__ float2 proj_pair_core(const TetRec& r, float atd, float4* __restrict__ P, float2 lam,
                                                 float4* __restrict__ tape4, int ts = 1) {
  const uint64_t pol = SH ? 0 : vtx_policy();
  float4 p[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) p[k] = vload<SH>(P + r.v[k], pol);
  if (tape4) {
#pragma unroll
    for (int k = 0; k < 4; ++k) __stcs(tape4 + k * ts, p[k]);
  }
  TetPair T;
  tet_pair_eval(r, atd, p, T);
  float dlh, dld;
  if (!tet_pair_solve(T, r.at, atd, lam, dlh, dld)) return lam;
  lam.x += dlh;
  lam.y += dld;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const f3 dx = T.both ? T.h[k] * dlh + T.d[k] * dld : T.h[k] * dlh;
    vstore<SH>(P + r.v[k], with_w(xyz(p[k]) + dx * p[k].w, p[k].w), pol);
  }
  return lam;
}

// rh / rd: the C_H records of a color segment and their C_D shadows (same tets, same
// order); the C_D multipliers sit doff slots after the C_H ones.
__device__ __forceinline__ void proj_pair_elem(int i, const TetRec* __restrict__ rh, const TetRec* __restrict__ rd,
                                               float4* __restrict__ P, const float* lam_in, float* lam_out, int doff,
                                               float4* __restrict__ tape) {
  const TetRec r = ld_rec(rh + i);
  const float atd = ld_stream(&rd[i].at);
  float2 lam = lam_in ? make_float2(ld_stream(lam_in + i), ld_stream(lam_in + i + doff)) : make_float2(0.f, 0.f);
  lam = proj_pair_core(r, atd, P, lam, tape ? tape + 4 * i : nullptr);
  __stcs(lam_out + i, lam.x);
  __stcs(lam_out + i + doff, lam.y);
}

// Reverse of the coupled update.  With S, dlambda recomputed from the tape and the adjoints
// xbar', lambar' of the updated values:  sbar = lambar' + G W xbar',  q = S^-1 sbar,
//   Gbar_k = dlambda_k W xbar' - sum_l (q_k dlambda_l + dlambda_k q_l) W g_l,
//   xbar = xbar' - sum_k q_k g_k + sum_k H_k Gbar_k,
//   lambar_k = lambar'_k - alpha~_k q_k,  alphabar~_k += -q_k (lambda_k + dlambda_k).
// With one constraint this is vjp_quad_core's update (q = s/D).  lh, ld: (lambar, alphabar)
// of C_H and C_D.
template <bool SH = false>
__device__ __forceinline__ void vjp_pair_core(const TetRec& r, float atd, const float4 (&p)[4], float2 lam,
                                              float2& lh, float2& ld, float4* __restrict__ xbar) {
  const uint64_t pol = SH ? 0 : vtx_policy();
  float4 xb4[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) xb4[k] = vload<SH>(xbar + r.v[k], pol);
  TetPair T;
  tet_pair_eval(r, atd, p, T);
  float dlh, dld;
  if (!tet_pair_solve(T, r.at, atd, lam, dlh, dld)) return;
  f3 xb[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) xb[k] = xyz(xb4[k]);
  float sh = lh.x, sd = ld.x;
#pragma unroll
  for (int k = 0; k < 4; ++k) sh += p[k].w * dot(T.h[k], xb[k]);
  float qh, qd = 0.f;
  if (T.both) {
#pragma unroll
    for (int k = 0; k < 4; ++k) sd += p[k].w * dot(T.d[k], xb[k]);
    const float inv = 1.f / T.det;
    qh = (T.s22 * sh - T.s12 * sd) * inv;
    qd = (T.s11 * sd - T.s12 * sh) * inv;
  } else {
    qh = sh / T.s11;
  }
  const f3 x0 = xyz(p[0]);
  const f3 e1 = xyz(p[1]) - x0, e2 = xyz(p[2]) - x0, e3 = xyz(p[3]) - x0;
  f3 out[4];
  {   // C_H: u_H = W (dlambda_H xbar' - 2 q_H dlambda_H g_H - (q_H dlambda_D + dlambda_H q_D) g_D)
    const float chh = 2.f * qh * dlh, chd = qh * dld + dlh * qd;
    f3 u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      f3 t = xb[k] * dlh - T.h[k] * chh;
      if (T.both) t = t - T.d[k] * chd;
      u[k] = t * p[k].w;
    }
    d3 g1, g2, g3;
    Quad<2>::hvp(r, e1, e2, e3, u[1] - u[0], u[2] - u[0], u[3] - u[0], g1, g2, g3);
    const f3 hu1 = dpart(g1), hu2 = dpart(g2), hu3 = dpart(g3);
    out[0] = xb[0] - T.h[0] * qh - (hu1 + hu2 + hu3);
    out[1] = xb[1] - T.h[1] * qh + hu1;
    out[2] = xb[2] - T.h[2] * qh + hu2;
    out[3] = xb[3] - T.h[3] * qh + hu3;
  }
  if (T.both) {   // C_D: u_D = W (dlambda_D xbar' - (q_D dlambda_H + dlambda_D q_H) g_H - 2 q_D dlambda_D g_D)
    const float cdh = qd * dlh + dld * qh, cdd = 2.f * qd * dld;
    f3 u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = (xb[k] * dld - T.h[k] * cdh - T.d[k] * cdd) * p[k].w;
    d3 g1, g2, g3;
    Quad<3>::hvp(r, e1, e2, e3, u[1] - u[0], u[2] - u[0], u[3] - u[0], g1, g2, g3);
    const f3 hu1 = dpart(g1), hu2 = dpart(g2), hu3 = dpart(g3);
    out[0] = out[0] - T.d[0] * qd - (hu1 + hu2 + hu3);
    out[1] = out[1] - T.d[1] * qd + hu1;
    out[2] = out[2] - T.d[2] * qd + hu2;
    out[3] = out[3] - T.d[3] * qd + hu3;
    ld.y += -qd * (lam.y + dld);
    ld.x -= atd * qd;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) vstore<SH>(xbar + r.v[k], with_w(out[k], 0.f), pol);
  lh.y += -qh * (lam.x + dlh);
  lh.x -= r.at * qh;
}

__device__ __forceinline__ void vjp_pair_elem(int i, const TetRec* __restrict__ rh, const TetRec* __restrict__ rd,
                                              const float4* __restrict__ tape, const float* __restrict__ lam_pre,
                                              int doff, float4* __restrict__ xbar, float2* __restrict__ lb,
                                              double* __restrict__ acc, bool first, bool last) {
  const TetRec r = ld_rec(rh + i);
  const float atd = ld_stream(&rd[i].at);
  float4 p[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) p[k] = ld_stream(tape + 4 * i + k);
  const float2 lam = lam_pre ? make_float2(ld_stream(lam_pre + i), ld_stream(lam_pre + i + doff)) : make_float2(0.f, 0.f);
  float2 lh = first ? make_float2(0.f, 0.f) : lb[i];
  float2 ld = first ? make_float2(0.f, 0.f) : lb[i + doff];
  vjp_pair_core(r, atd, p, lam, lh, ld, xbar);
  lb_finish(i, lh.x, lh.y, lb, acc, last);
  lb_finish(i + doff, ld.x, ld.y, lb, acc, last);
}

// ---- orthotropic StVK membrane (Sec. "Cloth Material Parameter Estimation"):
// C = (E_uu, E_vv, 2 E_uv), E = (F^T F - I)/2, F = [x1-x0, x2-x0] Dm^-1 = [f_u f_v].  With
// b_u = (-(B00+B10), B00, B10), b_v = (-(B01+B11), B01, B11) the per-vertex weights of f_u
// and f_v:  grad_i E_uu = b_u,i f_u,  grad_i E_vv = b_v,i f_v,
// grad_i 2E_uv = b_u,i f_v + b_v,i f_u, and the Hessians are constant:
// (H_uu y)_i = b_u,i Y_u, (H_vv y)_i = b_v,i Y_v, (H_uv y)_i = b_u,i Y_v + b_v,i Y_u with
// Y_u = sum_j b_u,j y_j, Y_v = sum_j b_v,j y_j.  The three multipliers come from
// S dlambda = -C - A~ lambda, S = G W G^T + A~ (3x3 SPD, Cholesky), x += W G^T dlambda.
struct MembEval {
  float bu[3], bv[3];
  f3 fu, fv;
  float C[3];
  float Wuu, Wvv, Wuv;   // sum_i w_i b_u,i^2, w_i b_v,i^2, w_i b_u,i b_v,i
  float L[6];            // Cholesky factor of S: L00, L11, L22 (inverses), L10, L20, L21
};

// Fills M and factors S; false when S is not positive definite (nothing moves).
__device__ __forceinline__ bool memb_eval(const MembRec& r, const float4 (&p)[3], MembEval& M) {
  M.bu[1] = r.B[0];
  M.bu[2] = r.B[2];
  M.bu[0] = -(r.B[0] + r.B[2]);
  M.bv[1] = r.B[1];
  M.bv[2] = r.B[3];
  M.bv[0] = -(r.B[1] + r.B[3]);
  const f3 x0 = xyz(p[0]);
  const f3 d1 = xyz(p[1]) - x0, d2 = xyz(p[2]) - x0;
  M.fu = d1 * r.B[0] + d2 * r.B[2];
  M.fv = d1 * r.B[1] + d2 * r.B[3];
  const float uu = dot(M.fu, M.fu), vv = dot(M.fv, M.fv), uv = dot(M.fu, M.fv);
  M.C[0] = 0.5f * (uu - 1.f);
  M.C[1] = 0.5f * (vv - 1.f);
  M.C[2] = uv;
  float Wuu = 0.f, Wvv = 0.f, Wuv = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Wuu += p[k].w * M.bu[k] * M.bu[k];
    Wvv += p[k].w * M.bv[k] * M.bv[k];
    Wuv += p[k].w * M.bu[k] * M.bv[k];
  }
  M.Wuu = Wuu;
  M.Wvv = Wvv;
  M.Wuv = Wuv;
  const float S00 = Wuu * uu + r.a00, S11 = Wvv * vv + r.a11, S01 = Wuv * uv + r.a01;
  const float S22 = Wuu * vv + 2.f * Wuv * uv + Wvv * uu + r.a22;
  const float S02 = Wuu * uv + Wuv * uu, S12 = Wuv * vv + Wvv * uv;
  if (!(S00 > 0.f)) return false;
  const float i00 = rsqrtf(S00);
  const float l10 = S01 * i00, l20 = S02 * i00;
  const float d11 = S11 - l10 * l10;
  if (!(d11 > 0.f)) return false;
  const float i11 = rsqrtf(d11);
  const float l21 = (S12 - l20 * l10) * i11;
  const float d22 = S22 - l20 * l20 - l21 * l21;
  if (!(d22 > 0.f)) return false;
  M.L[0] = i00;
  M.L[1] = i11;
  M.L[2] = rsqrtf(d22);
  M.L[3] = l10;
  M.L[4] = l20;
  M.L[5] = l21;
  return true;
}

__device__ __forceinline__ void memb_solve(const MembEval& M, const float (&b)[3], float (&x)[3]) {
  const float y0 = b[0] * M.L[0];
  const float y1 = (b[1] - M.L[3] * y0) * M.L[1];
  const float y2 = (b[2] - M.L[4] * y0 - M.L[5] * y1) * M.L[2];
  x[2] = y2 * M.L[2];
  x[1] = (y1 - M.L[5] * x[2]) * M.L[1];
  x[0] = (y0 - M.L[3] * x[1] - M.L[4] * x[2]) * M.L[0];
}

__device__ __forceinline__ void memb_dlambda(const MembRec& r, const MembEval& M, const float (&lam)[3],
                                             float (&dl)[3]) {
  const float rhs[3] = {-M.C[0] - (r.a00 * lam[0] + r.a01 * lam[1]), -M.C[1] - (r.a01 * lam[0] + r.a11 * lam[1]),
                        -M.C[2] - r.a22 * lam[2]};
  memb_solve(M, rhs, dl);
}

template <bool SH = false>
__device__ __forceinline__ void proj_memb_core(const MembRec& r, float4* __restrict__ P, float (&lam)[3],
                                               float4* __restrict__ tape3, int ts = 1) {
  const uint64_t pol = SH ? 0 : vtx_policy();
  float4 p[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) p[k] = vload<SH>(P + r.v[k], pol);
  if (tape3) {
#pragma unroll
    for (int k = 0; k < 3; ++k) __stcs(tape3 + k * ts, p[k]);
  }
  MembEval M;
  if (!memb_eval(r, p, M)) return;
  float dl[3];
  memb_dlambda(r, M, lam, dl);
#pragma unroll
  for (int k = 0; k < 3; ++k) lam[k] += dl[k];
  const f3 Pu = M.fu * dl[0] + M.fv * dl[2], Pv = M.fv * dl[1] + M.fu * dl[2];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    vstore<SH>(P + r.v[k], with_w(xyz(p[k]) + (Pu * M.bu[k] + Pv * M.bv[k]) * p[k].w, p[k].w), pol);
}

// Record i's multipliers sit at slots i, i + stride, i + 2 stride (lam_in / lam_out may
// alias); its tape entries at tape[3i .. 3i+2].
__device__ __forceinline__ void proj_memb_elem(int i, const MembRec* __restrict__ rec, float4* __restrict__ P,
                                               const float* lam_in, float* lam_out, int stride,
                                               float4* __restrict__ tape) {
  const MembRec r = ld_rec(rec + i);
  float lam[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) lam[k] = lam_in ? ld_stream(lam_in + i + k * stride) : 0.f;
  proj_memb_core(r, P, lam, tape ? tape + 3 * i : nullptr);
#pragma unroll
  for (int k = 0; k < 3; ++k) __stcs(lam_out + i + k * stride, lam[k]);
}

// Reverse of one membrane update (the 3x3 form of vjp_pair_core):
//   sbar = lambar' + G W xbar',  q = S^-1 sbar,
//   Gbar_k = dlambda_k W xbar' - sum_l (q_k dlambda_l + dlambda_k q_l) W g_l,
//   xbar = xbar' - G^T q + sum_k H_k Gbar_k,  lambar = lambar' - A~ q,
//   alphabar~ += -q (lambda + dlambda)^T on the entries (00, 11, 01 + 10, 22).
// With the constant Hessians, sum_k H_k Gbar_k and G^T q both reduce to
// b_u,i A_u + b_v,i A_v for two vectors A_u, A_v.
template <bool SH = false>
__device__ __forceinline__ void vjp_memb_core(const MembRec& r, const float4 (&p)[3], const float (&lam)[3],
                                              float (&lb)[3], float (&ab)[4], float4* __restrict__ xbar) {
  const uint64_t pol = SH ? 0 : vtx_policy();
  float4 xb4[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) xb4[k] = vload<SH>(xbar + r.v[k], pol);
  MembEval M;
  if (!memb_eval(r, p, M)) return;
  float dl[3];
  memb_dlambda(r, M, lam, dl);
  f3 Xu = {0.f, 0.f, 0.f}, Xv = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const f3 x = xyz(xb4[k]) * p[k].w;
    Xu = Xu + x * M.bu[k];
    Xv = Xv + x * M.bv[k];
  }
  const float sb[3] = {lb[0] + dot(M.fu, Xu), lb[1] + dot(M.fv, Xv), lb[2] + dot(M.fv, Xu) + dot(M.fu, Xv)};
  float q[3];
  memb_solve(M, sb, q);
  const float c00 = 2.f * q[0] * dl[0], c11 = 2.f * q[1] * dl[1], c22 = 2.f * q[2] * dl[2];
  const float c01 = q[0] * dl[1] + dl[0] * q[1], c02 = q[0] * dl[2] + dl[0] * q[2], c12 = q[1] * dl[2] + dl[1] * q[2];
  // sum_j b_u,j w_j g_l,j and sum_j b_v,j w_j g_l,j for l = uu, vv, uv
  const f3 Gu0 = M.fu * M.Wuu, Gu1 = M.fv * M.Wuv, Gu2 = M.fv * M.Wuu + M.fu * M.Wuv;
  const f3 Gv0 = M.fu * M.Wuv, Gv1 = M.fv * M.Wvv, Gv2 = M.fv * M.Wuv + M.fu * M.Wvv;
  const f3 P0 = Xu * dl[0] - (Gu0 * c00 + Gu1 * c01 + Gu2 * c02);
  const f3 P1 = Xv * dl[1] - (Gv0 * c01 + Gv1 * c11 + Gv2 * c12);
  const f3 Q0 = Xu * dl[2] - (Gu0 * c02 + Gu1 * c12 + Gu2 * c22);
  const f3 Q1 = Xv * dl[2] - (Gv0 * c02 + Gv1 * c12 + Gv2 * c22);
  const f3 Au = P0 + Q1 - (M.fu * q[0] + M.fv * q[2]);
  const f3 Av = P1 + Q0 - (M.fv * q[1] + M.fu * q[2]);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    vstore<SH>(xbar + r.v[k], with_w(xyz(xb4[k]) + Au * M.bu[k] + Av * M.bv[k], 0.f), pol);
  const float m0 = lam[0] + dl[0], m1 = lam[1] + dl[1], m2 = lam[2] + dl[2];
  ab[0] -= q[0] * m0;
  ab[1] -= q[1] * m1;
  ab[2] -= q[0] * m1 + q[1] * m0;
  ab[3] -= q[2] * m2;
  lb[0] -= r.a00 * q[0] + r.a01 * q[1];
  lb[1] -= r.a01 * q[0] + r.a11 * q[1];
  lb[2] -= r.a22 * q[2];
}

// Slots i + k stride (k = 0..3) carry (lambar_k, alphabar partial k) within a step and the
// float64 alphabar accumulators (00, 11, 01, 22) across steps.
__device__ __forceinline__ void vjp_memb_elem(int i, const MembRec* __restrict__ rec, const float4* __restrict__ tape,
                                              const float* __restrict__ lam_pre, int stride, float4* __restrict__ xbar,
                                              float2* __restrict__ lb, double* __restrict__ acc, bool first,
                                              bool last) {
  const MembRec r = ld_rec(rec + i);
  float4 p[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) p[k] = ld_stream(tape + 3 * i + k);
  float lam[3], lbv[3], ab[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) lam[k] = lam_pre ? ld_stream(lam_pre + i + k * stride) : 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 l = first ? make_float2(0.f, 0.f) : lb[i + k * stride];
    if (k < 3) lbv[k] = l.x;
    ab[k] = l.y;
  }
  vjp_memb_core(r, p, lam, lbv, ab, xbar);
#pragma unroll
  for (int k = 0; k < 4; ++k) lb_finish(i + k * stride, k < 3 ? lbv[k] : 0.f, ab[k], lb, acc, last);
}

// alpha~ entries of record i from the caller's (C00, C11, C01, C22) of its triangle:
// alpha~ = (A K)^-1 / dt^2.  K not positive definite or not finite sets bit 1 of the error
// word and leaves the record's alpha~ unchanged.
__device__ __forceinline__ void memb_set_alpha_elem(int i, MembRec* __restrict__ rec, const int* __restrict__ perm,
                                                    const float* __restrict__ K, float inv_dt2,
                                                    int* __restrict__ err) {
  const int t = perm[i];
  if (t < 0) return;   // padding record of the phase layout (alpha~ stays 0)
  const float c00 = K[4 * t], c11 = K[4 * t + 1], c01 = K[4 * t + 2], c22 = K[4 * t + 3];
  const float det = c00 * c11 - c01 * c01;
  if (!(c00 > 0.f) || !(det > 0.f) || !(c22 > 0.f) || isinf(c00) || isinf(c11) || isinf(c22) || isinf(det)) {
    atomicOr(err, 2);
    return;
  }
  const float s = inv_dt2 / rec[i].A;
  const float sd = s / det;
  rec[i].a00 = c11 * sd;
  rec[i].a11 = c00 * sd;
  rec[i].a01 = -c01 * sd;
  rec[i].a22 = s / c22;
}

// dL/d(C00, C11, C01, C22) of record i's triangle from the float64 accumulated adjoints
// g = (g00, g11, g01, g22) of its alpha~ entries: with alpha~_2x2 = s K2^-1,
// Kbar2 = -s K2^-1 Gbar K2^-1 (Gbar = [g00 g01/2; g01/2 g11]), and d alpha~_22 / d C22 =
// -s / C22^2.  Written (not accumulated) in the caller's triangle order, in float64.
__device__ __forceinline__ void memb_gradient_elem(int i, const MembRec* __restrict__ rec, const int* __restrict__ perm,
                                                   const float* __restrict__ K, double inv_dt2,
                                                   const double* __restrict__ acc, int stride,
                                                   double* __restrict__ out) {
  const int t = perm[i];
  if (t < 0) return;
  const double c00 = K[4 * t], c11 = K[4 * t + 1], c01 = K[4 * t + 2], c22 = K[4 * t + 3];
  const double s = inv_dt2 / (double)rec[i].A;
  const double det = c00 * c11 - c01 * c01;
  const double i00 = c11 / det, i11 = c00 / det, i01 = -c01 / det;
  const double g00 = acc[i], g11 = acc[i + stride], g01 = 0.5 * acc[i + 2 * stride], g22 = acc[i + 3 * stride];
  // M = Gbar K2^-1, Kbar2 = -s K2^-1 M
  const double m00 = g00 * i00 + g01 * i01, m01 = g00 * i01 + g01 * i11;
  const double m10 = g01 * i00 + g11 * i01, m11 = g01 * i01 + g11 * i11;
  const double k00 = -s * (i00 * m00 + i01 * m10), k11 = -s * (i01 * m01 + i11 * m11);
  const double k01 = -s * (i00 * m01 + i01 * m11);
  out[4 * t] = k00;
  out[4 * t + 1] = k11;
  out[4 * t + 2] = 2.0 * k01;
  out[4 * t + 3] = -s * g22 / (c22 * c22);
}

// Reverse of the collision pass.  Plane (inputs p, h; grad_p = e_y, grad_h = -1, H = 0) and
// sphere (inputs p, c, r; grad_p = n, grad_c = -n, grad_r = -1, H_pp = P/l, H_pc = -P/l;
// the centre and radius are not moved, so u_c = 0).  Collider adjoints accumulate in the
// per-vertex float32 scratch cgrad = (hbar, cbar_x, cbar_y, cbar_z, rbar) over the step.
__device__ __forceinline__ void vjp_contact_elem(int i, const float4* __restrict__ tape,
                                                 const uint8_t* __restrict__ cflags, const float2* __restrict__ lam_pre,
                                                 float4* __restrict__ xbar, float2* __restrict__ lbc,
                                                 float* __restrict__ cgrad, bool first, const Collide& c) {
  uint8_t f = cflags[i];
  if (!f) return;
  float4 p4 = tape[i];
  float w = p4.w;
  float2 lam = lam_pre ? lam_pre[i] : make_float2(0.f, 0.f);
  float2 lb = first ? make_float2(0.f, 0.f) : lbc[i];
  float cg[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  if (cgrad && !first)
    for (int k = 0; k < 5; ++k) cg[k] = cgrad[5 * i + k];
  f3 xb = xyz(xbar[i]);
  f3 pre = xyz(p4);
  f3 mid = pre;
  if ((f & 1) && (f & 2)) {
    float lp = lam.x;
    plane_project(mid, w, lp, c);
  }
  float D = w + c.at;
  if ((f & 2) && D > 0.f) {
    f3 d = mid - mk3(c.cx, c.cy, c.cz);
    float l2 = dot(d, d);
    if (l2 >= XPBD_DEGEN2) {
      float il = rsqrtf(l2);
      float len = l2 * il;
      f3 nrm = d * il;
      float dl = (-(len - c.r - c.thick) - c.at * lam.y) / D;
      float s = lb.y + w * dot(nrm, xb);
      float sD = s / D;
      f3 t = xb * (w * dl);
      f3 hv = (t - nrm * dot(nrm, t)) * il;
      xb = xb - nrm * sD + hv;
      // centre: -(s/D) grad_c + (H u)_c = (s/D) n - hv ; radius: -(s/D) grad_r = s/D
      cg[1] += nrm.x * sD - hv.x;
      cg[2] += nrm.y * sD - hv.y;
      cg[3] += nrm.z * sD - hv.z;
      cg[4] += sD;
      lb.y -= c.at * sD;
    }
  }
  if ((f & 1) && D > 0.f) {
    float s = lb.x + w * xb.y;
    float sD = s / D;
    xb.y -= sD;
    cg[0] += sD;
    lb.x -= c.at * sD;
  }
  xbar[i] = with_w(xb, 0.f);
  lbc[i] = lb;
  if (cgrad)
    for (int k = 0; k < 5; ++k) cgrad[5 * i + k] = cg[k];
}

// Per-vertex collider adjoints of this step (contact vertices only: cgrad of the other
// vertices is stale), added to v.
__device__ __forceinline__ void collider_contrib(int i, const float* __restrict__ cgrad,
                                                 const uint8_t* __restrict__ cflags, double v[5]) {
  if (cflags[i])
    for (int k = 0; k < 5; ++k) v[k] += (double)cgrad[5 * i + k];
}

// Adjoint of the prediction p = x_n + dt v_n + dt^2 (w (G_n + W_i) + [w>0] g):
//   xbar_n = xbar_partial + pbar (+ dL/dx_n seed),  vbar_n = dt pbar,
//   fbar_i = dt^2 w_i pbar_i  (Sec. 5.6: force gradients from the adjoint velocities),
//   dL/dW_i += fbar_i (float64); fbar_i is added to fs for dL/dG_n.
// fvs_out: step n's per-vertex force gradient dt^2 w pbar (written, float64), or NULL.
__device__ __forceinline__ void adj_predict_elem(int i, float4* __restrict__ xbar, float4* __restrict__ vbar,
                                                 const float4* __restrict__ ckx_n, const float* __restrict__ seed,
                                                 float dt, double* __restrict__ fv_acc, double fs[3],
                                                 double* __restrict__ fvs_out = nullptr) {
  float dt2 = dt * dt;
  float4 pb = xbar[i];
  float4 xp = vbar[i];
  float w = ckx_n[i].w;
  float4 xn = make_float4(xp.x + pb.x, xp.y + pb.y, xp.z + pb.z, 0.f);
  if (seed) {
    xn.x += seed[3 * i];
    xn.y += seed[3 * i + 1];
    xn.z += seed[3 * i + 2];
  }
  xbar[i] = xn;
  vbar[i] = make_float4(dt * pb.x, dt * pb.y, dt * pb.z, 0.f);
  double fx = (double)(dt2 * w) * (double)pb.x;
  double fy = (double)(dt2 * w) * (double)pb.y;
  double fz = (double)(dt2 * w) * (double)pb.z;
  if (fv_acc) {
    fv_acc[3 * i] += fx;
    fv_acc[3 * i + 1] += fy;
    fv_acc[3 * i + 2] += fz;
  }
  if (fvs_out) {
    fvs_out[3 * i] = fx;
    fvs_out[3 * i + 1] = fy;
    fvs_out[3 * i + 2] = fz;
  }
  fs[0] += fx;
  fs[1] += fy;
  fs[2] += fz;
}

// dL/d compliance in the caller's constraint order: alpha~ = compliance / dt^2 (tets:
// / (V_e dt^2)), so dL/dcompliance = alphabar~ / dt^2 (/ V_e).
template <class Rec, bool VOL>
__device__ __forceinline__ void finalize_elem(int i, const Rec* __restrict__ rec, const int* __restrict__ perm,
                                              const double* __restrict__ acc, float inv_dt2,
                                              double* __restrict__ out) {
  const int j = perm[i];
  if (j < 0) return;   // padding record
  double a = acc[i] * (double)inv_dt2;
  if constexpr (VOL) a = a / (double)rec[i].vol;
  out[j] = a;
}

__device__ __forceinline__ void to_double_elem(int i, const float4* __restrict__ a, double* __restrict__ out) {
  float4 v = a[i];
  out[3 * i] = v.x;
  out[3 * i + 1] = v.y;
  out[3 * i + 2] = v.z;
}

// Goal function of Sec. 4.1 on one keyframe: seed = x - x*, accumulates |x - x*|^2 / 2.
__device__ __forceinline__ void loss_elem(int i, const float4* __restrict__ ckx, const float* __restrict__ target,
                                          float* __restrict__ seed_out, double& acc) {
  float4 x = ckx[i];
  float dx = x.x - target[3 * i], dy = x.y - target[3 * i + 1], dz = x.z - target[3 * i + 2];
  if (seed_out) {
    seed_out[3 * i] = dx;
    seed_out[3 * i + 1] = dy;
    seed_out[3 * i + 2] = dz;
  }
  acc += 0.5 * ((double)dx * dx + (double)dy * dy + (double)dz * dz);
}

__device__ __forceinline__ void read_state_elem(int i, const float4* __restrict__ ckx, const float4* __restrict__ ckv,
                                                float* __restrict__ x_out, float* __restrict__ v_out) {
  if (x_out) {
    float4 x = ckx[i];
    x_out[3 * i] = x.x;
    x_out[3 * i + 1] = x.y;
    x_out[3 * i + 2] = x.z;
  }
  if (v_out) {
    float4 v = ckv[i];
    v_out[3 * i] = v.x;
    v_out[3 * i + 1] = v.y;
    v_out[3 * i + 2] = v.z;
  }
}

}  // namespace xpbd
