// sm_103a kernels of the XPBD step (Sec. 3.1 of DiffXPBD) and of its discrete adjoint for
// one request: each kernel applies one element function of xpbd_elems.cuh to a whole
// color (one thread per constraint) or to every vertex.
#include "xpbd_elems.cuh"

namespace xpbd {

namespace {

constexpr int kMaxPartialBlocks = 1024;

}  // namespace

int partial_blocks(int V) {
  int b = grid_for(V);
  return b < 1 ? 1 : (b > kMaxPartialBlocks ? kMaxPartialBlocks : b);
}

// ======================================================================== forward

__global__ void k_init_ckpt(const float* __restrict__ x0, const float* __restrict__ v0,
                            const float* __restrict__ w, float4* __restrict__ ckx,
                            float4* __restrict__ ckv, int V) {
  XPBD_TID_OR_RETURN(V);
  init_ckpt_elem(i, x0, v0, w, ckx, ckv);
}

void launch_init_ckpt(const float* x0, const float* v0, const float* w, float4* ckx, float4* ckv,
                      int V, cudaStream_t s) {
  if (V > 0) k_init_ckpt<<<grid_for(V), kBlock, 0, s>>>(x0, v0, w, ckx, ckv, V);
}

template <class Rec, bool VOL>
__global__ void k_set_alpha(Rec* __restrict__ rec, const int* __restrict__ perm, int n,
                            const float* __restrict__ compliance, float inv_dt2, int* __restrict__ err) {
  XPBD_TID_OR_RETURN(n);
  set_alpha_elem<Rec, VOL>(i, rec, perm, compliance, inv_dt2, err);
}

void launch_set_alpha_btail(BendTail* tail, const int* perm, int n, const float* compliance, float inv_dt2, int* err,
                            cudaStream_t s) {
  if (n <= 0) return;
  k_set_alpha<BendTail, false><<<grid_for(n), kBlock, 0, s>>>(tail, perm, n, compliance, inv_dt2, err);
}

void launch_set_alpha(SegType t, void* rec, const int* perm, int n, const float* compliance,
                      float inv_dt2, int* err, cudaStream_t s) {
  if (n <= 0) return;
  switch (t) {
    case SEG_DIST:
      k_set_alpha<DistRec, false><<<grid_for(n), kBlock, 0, s>>>((DistRec*)rec, perm, n, compliance, inv_dt2, err);
      break;
    case SEG_BEND:
      k_set_alpha<BendRec, false><<<grid_for(n), kBlock, 0, s>>>((BendRec*)rec, perm, n, compliance, inv_dt2, err);
      break;
    default:
      k_set_alpha<TetRec, true><<<grid_for(n), kBlock, 0, s>>>((TetRec*)rec, perm, n, compliance, inv_dt2, err);
  }
}

__global__ void k_predict(const float4* __restrict__ ckx, const float4* __restrict__ ckv,
                          float4* __restrict__ P, const float* __restrict__ fg_n,
                          const float* __restrict__ fv, const float* __restrict__ fvs_n, float dt, float gx,
                          float gy, float gz, Collide c, uint8_t* __restrict__ cflags, int V) {
  XPBD_TID_OR_RETURN(V);
  predict_elem(i, ckx, ckv, P, fg_n, fv, fvs_n, dt, gx, gy, gz, c, cflags);
}

void launch_predict(const float4* ckx, const float4* ckv, float4* P, const float* fg_n,
                    const float* fv, const float* fvs_n, float dt, float gx, float gy, float gz, Collide c,
                    uint8_t* cflags, int V, cudaStream_t s) {
  if (V > 0)
    k_predict<<<grid_for(V), kBlock, 0, s>>>(ckx, ckv, P, fg_n, fv, fvs_n, dt, gx, gy, gz, c, cflags, V);
}

__global__ void k_proj_dist(const DistRec* __restrict__ rec, int n, float4* __restrict__ P,
                            const float* lam_in, float* lam_out, float4* __restrict__ tape) {
  XPBD_TID_OR_RETURN(n);
  proj_dist_elem(i, rec, P, lam_in, lam_out, tape);
}

#ifndef XPBD_PROJ_QUAD_MIN_BLOCKS
#define XPBD_PROJ_QUAD_MIN_BLOCKS 1
#endif
template <int KIND>
__global__ void __launch_bounds__(kBlock, XPBD_PROJ_QUAD_MIN_BLOCKS)
k_proj_quad(const typename Quad<KIND>::Rec* __restrict__ rec, int n, float4* __restrict__ P,
            const float* lam_in, float* lam_out, float4* __restrict__ tape) {
  XPBD_TID_OR_RETURN(n);
  proj_quad_elem<KIND>(i, rec, P, lam_in, lam_out, tape);
}

void launch_project(SegType t, const void* rec, int n, float4* P, const float* lam_in,
                    float* lam_out, float4* tape, cudaStream_t s) {
  if (n <= 0) return;
  switch (t) {
    case SEG_DIST:
      k_proj_dist<<<grid_for(n), kBlock, 0, s>>>((const DistRec*)rec, n, P, lam_in, lam_out, tape);
      break;
    case SEG_BEND:
      k_proj_quad<1><<<grid_for(n), kBlock, 0, s>>>((const BendRec*)rec, n, P, lam_in, lam_out, tape);
      break;
    case SEG_TETH:
      k_proj_quad<2><<<grid_for(n), kBlock, 0, s>>>((const TetRec*)rec, n, P, lam_in, lam_out, tape);
      break;
    case SEG_TETD:
      k_proj_quad<3><<<grid_for(n), kBlock, 0, s>>>((const TetRec*)rec, n, P, lam_in, lam_out, tape);
      break;
  }
}

__global__ void __launch_bounds__(kBlock, XPBD_PROJ_QUAD_MIN_BLOCKS)
k_proj_tet_pair(const TetRec* __restrict__ rh, const TetRec* __restrict__ rd, int n, float4* __restrict__ P,
                const float* lam_in, float* lam_out, int doff, float4* __restrict__ tape) {
  XPBD_TID_OR_RETURN(n);
  proj_pair_elem(i, rh, rd, P, lam_in, lam_out, doff, tape);
}

void launch_project_tet_pair(const TetRec* rh, const TetRec* rd, int n, float4* P, const float* lam_in,
                             float* lam_out, int doff, float4* tape, cudaStream_t s) {
  if (n > 0) k_proj_tet_pair<<<grid_for(n), kBlock, 0, s>>>(rh, rd, n, P, lam_in, lam_out, doff, tape);
}

__global__ void k_memb_set_alpha(MembRec* __restrict__ rec, const int* __restrict__ perm, int n,
                                 const float* __restrict__ K, float inv_dt2, int* __restrict__ err) {
  XPBD_TID_OR_RETURN(n);
  memb_set_alpha_elem(i, rec, perm, K, inv_dt2, err);
}

void launch_memb_set_alpha(MembRec* rec, const int* perm, int n, const float* stiffness, float inv_dt2, int* err,
                           cudaStream_t s) {
  if (n > 0) k_memb_set_alpha<<<grid_for(n), kBlock, 0, s>>>(rec, perm, n, stiffness, inv_dt2, err);
}

__global__ void k_proj_memb(const MembRec* __restrict__ rec, int n, float4* __restrict__ P, const float* lam_in,
                            float* lam_out, int stride, float4* __restrict__ tape) {
  XPBD_TID_OR_RETURN(n);
  proj_memb_elem(i, rec, P, lam_in, lam_out, stride, tape);
}

void launch_project_memb(const MembRec* rec, int n, float4* P, const float* lam_in, float* lam_out, int stride,
                         float4* tape, cudaStream_t s) {
  if (n > 0) k_proj_memb<<<grid_for(n), kBlock, 0, s>>>(rec, n, P, lam_in, lam_out, stride, tape);
}

__global__ void k_contact(float4* __restrict__ P, const uint8_t* __restrict__ cflags, int V,
                          const float2* lam_in, float2* lam_out, float4* __restrict__ tape, Collide c) {
  XPBD_TID_OR_RETURN(V);
  contact_elem(i, P, cflags, lam_in, lam_out, tape, c);
}

void launch_contact(float4* P, const uint8_t* cflags, int V, const float2* lam_in,
                    float2* lam_out, float4* tape, Collide c, cudaStream_t s) {
  if (V > 0 && c.flags) k_contact<<<grid_for(V), kBlock, 0, s>>>(P, cflags, V, lam_in, lam_out, tape, c);
}

__global__ void k_velocity(const float4* __restrict__ P, const float4* __restrict__ ckx_n,
                           float4* __restrict__ ckx_next, float4* __restrict__ ckv_next,
                           float inv_dt, int V, int* __restrict__ err) {
  XPBD_TID_OR_RETURN(V);
  velocity_elem(i, P, ckx_n, ckx_next, ckv_next, inv_dt, err);
}

void launch_velocity(const float4* P, const float4* ckx_n, float4* ckx_next, float4* ckv_next,
                     float inv_dt, int V, int* err, cudaStream_t s) {
  if (V > 0) k_velocity<<<grid_for(V), kBlock, 0, s>>>(P, ckx_n, ckx_next, ckv_next, inv_dt, V, err);
}

// ======================================================================== reverse

__global__ void k_seed_adjoint(const float* __restrict__ sx, const float* __restrict__ sv,
                               float4* __restrict__ xbar, float4* __restrict__ vbar, int V) {
  XPBD_TID_OR_RETURN(V);
  seed_adjoint_elem(i, sx, sv, xbar, vbar);
}

void launch_seed_adjoint(const float* seed_x, const float* seed_v, float4* xbar, float4* vbar,
                         int V, cudaStream_t s) {
  if (V > 0) k_seed_adjoint<<<grid_for(V), kBlock, 0, s>>>(seed_x, seed_v, xbar, vbar, V);
}

__global__ void k_adj_begin(float4* __restrict__ xbar, float4* __restrict__ vbar, float inv_dt, int V) {
  XPBD_TID_OR_RETURN(V);
  adj_begin_elem(i, xbar, vbar, inv_dt);
}

void launch_adj_begin(float4* xbar, float4* vbar, float inv_dt, int V, cudaStream_t s) {
  if (V > 0) k_adj_begin<<<grid_for(V), kBlock, 0, s>>>(xbar, vbar, inv_dt, V);
}

__global__ void k_vjp_dist(const DistRec* __restrict__ rec, int n, const float4* __restrict__ tape,
                           const float* __restrict__ lam_pre, float4* __restrict__ xbar,
                           float2* __restrict__ lb, double* __restrict__ acc, bool first, bool last) {
  XPBD_TID_OR_RETURN(n);
  vjp_dist_elem(i, rec, tape, lam_pre, xbar, lb, acc, first, last);
}

// 3 resident blocks of 256 threads for the 4-vertex reverse passes (<= 85 registers; the
// compiler spills 24-48 bytes): 11% faster than 2 blocks at 96-107 registers on the
// bending reverse pass.
#ifndef XPBD_VJP_QUAD_MIN_BLOCKS
#define XPBD_VJP_QUAD_MIN_BLOCKS 3
#endif
template <int KIND>
__global__ void __launch_bounds__(kBlock, XPBD_VJP_QUAD_MIN_BLOCKS)
k_vjp_quad(const typename Quad<KIND>::Rec* __restrict__ rec, int n, const float4* __restrict__ tape,
           const float* __restrict__ lam_pre, float4* __restrict__ xbar, float2* __restrict__ lb,
           double* __restrict__ acc, bool first, bool last) {
  XPBD_TID_OR_RETURN(n);
  vjp_quad_elem<KIND>(i, rec, tape, lam_pre, xbar, lb, acc, first, last);
}

void launch_vjp(SegType t, const void* rec, int n, const float4* tape, const float* lam_pre,
                float4* xbar, float2* lb, double* acc, bool first, bool last, cudaStream_t s) {
  if (n <= 0) return;
  switch (t) {
    case SEG_DIST:
      k_vjp_dist<<<grid_for(n), kBlock, 0, s>>>((const DistRec*)rec, n, tape, lam_pre, xbar, lb, acc, first, last);
      break;
    case SEG_BEND:
      k_vjp_quad<1><<<grid_for(n), kBlock, 0, s>>>((const BendRec*)rec, n, tape, lam_pre, xbar, lb, acc, first, last);
      break;
    case SEG_TETH:
      k_vjp_quad<2><<<grid_for(n), kBlock, 0, s>>>((const TetRec*)rec, n, tape, lam_pre, xbar, lb, acc, first, last);
      break;
    case SEG_TETD:
      k_vjp_quad<3><<<grid_for(n), kBlock, 0, s>>>((const TetRec*)rec, n, tape, lam_pre, xbar, lb, acc, first, last);
      break;
  }
}

// Two resident blocks: the pair reverse holds both gradients and both Hessian products
// (84 bytes of spills at the 85-register cap of three blocks).
__global__ void __launch_bounds__(kBlock, 2)
k_vjp_tet_pair(const TetRec* __restrict__ rh, const TetRec* __restrict__ rd, int n, const float4* __restrict__ tape,
               const float* __restrict__ lam_pre, int doff, float4* __restrict__ xbar, float2* __restrict__ lb,
               double* __restrict__ acc, bool first, bool last) {
  XPBD_TID_OR_RETURN(n);
  vjp_pair_elem(i, rh, rd, tape, lam_pre, doff, xbar, lb, acc, first, last);
}

void launch_vjp_tet_pair(const TetRec* rh, const TetRec* rd, int n, const float4* tape, const float* lam_pre,
                         int doff, float4* xbar, float2* lb, double* acc, bool first, bool last, cudaStream_t s) {
  if (n > 0)
    k_vjp_tet_pair<<<grid_for(n), kBlock, 0, s>>>(rh, rd, n, tape, lam_pre, doff, xbar, lb, acc, first, last);
}

__global__ void __launch_bounds__(kBlock, 2)
k_vjp_memb(const MembRec* __restrict__ rec, int n, const float4* __restrict__ tape, const float* __restrict__ lam_pre,
           int stride, float4* __restrict__ xbar, float2* __restrict__ lb, double* __restrict__ acc, bool first,
           bool last) {
  XPBD_TID_OR_RETURN(n);
  vjp_memb_elem(i, rec, tape, lam_pre, stride, xbar, lb, acc, first, last);
}

void launch_vjp_memb(const MembRec* rec, int n, const float4* tape, const float* lam_pre, int stride, float4* xbar,
                     float2* lb, double* acc, bool first, bool last, cudaStream_t s) {
  if (n > 0) k_vjp_memb<<<grid_for(n), kBlock, 0, s>>>(rec, n, tape, lam_pre, stride, xbar, lb, acc, first, last);
}

__global__ void k_memb_gradient(const MembRec* __restrict__ rec, const int* __restrict__ perm, int n,
                                const float* __restrict__ K, double inv_dt2, const double* __restrict__ acc,
                                int stride, double* __restrict__ out) {
  XPBD_TID_OR_RETURN(n);
  memb_gradient_elem(i, rec, perm, K, inv_dt2, acc, stride, out);
}

void launch_memb_gradient(const MembRec* rec, const int* perm, int n, const float* stiffness, float inv_dt2,
                          const double* acc, int stride, double* out, cudaStream_t s) {
  if (n > 0) k_memb_gradient<<<grid_for(n), kBlock, 0, s>>>(rec, perm, n, stiffness, (double)inv_dt2, acc, stride, out);
}

__global__ void k_vjp_contact(const float4* __restrict__ tape, const uint8_t* __restrict__ cflags,
                              int V, const float2* __restrict__ lam_pre, float4* __restrict__ xbar,
                              float2* __restrict__ lbc, float* __restrict__ cgrad, bool first, Collide c) {
  XPBD_TID_OR_RETURN(V);
  vjp_contact_elem(i, tape, cflags, lam_pre, xbar, lbc, cgrad, first, c);
}

void launch_vjp_contact(const float4* tape, const uint8_t* cflags, int V, const float2* lam_pre,
                        float4* xbar, float2* lbc, float* cgrad, bool first, Collide c,
                        cudaStream_t s) {
  if (V > 0 && c.flags)
    k_vjp_contact<<<grid_for(V), kBlock, 0, s>>>(tape, cflags, V, lam_pre, xbar, lbc, cgrad, first, c);
}

// Per-block float64 sums of the per-vertex collider adjoints of this step.
__global__ void k_collider_partials(const float* __restrict__ cgrad, const uint8_t* __restrict__ cflags,
                                    int V, double* __restrict__ partials) {
  double v[5] = {0, 0, 0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x)
    collider_contrib(i, cgrad, cflags, v);
  block_sum_store<5>(v, partials + 5 * blockIdx.x);
}

void launch_collider_partials(const float* cgrad, const uint8_t* cflags, int V, double* partials,
                              cudaStream_t s) {
  k_collider_partials<<<partial_blocks(V), kBlock, 0, s>>>(cgrad, cflags, V, partials);
}

// Adjoint of the prediction, with per-block float64 partial sums of the force adjoint
// (dL/dG_n = sum_i fbar_i, reduced in a fixed order afterwards).
__global__ void k_adj_predict(float4* __restrict__ xbar, float4* __restrict__ vbar,
                              const float4* __restrict__ ckx_n, const float* __restrict__ seed,
                              float dt, double* __restrict__ fv_acc, double* __restrict__ fg_partials,
                              double* __restrict__ fvs_out, int V) {
  double fs[3] = {0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x)
    adj_predict_elem(i, xbar, vbar, ckx_n, seed, dt, fv_acc, fs, fvs_out);
  if (fg_partials) block_sum_store<3>(fs, fg_partials + 3 * blockIdx.x);
}

void launch_adj_predict(float4* xbar, float4* vbar, const float4* ckx_n, const float* seed,
                        float dt, double* fv_acc, double* fg_partials, double* fvs_out, int V, cudaStream_t s) {
  k_adj_predict<<<partial_blocks(V), kBlock, 0, s>>>(xbar, vbar, ckx_n, seed, dt, fv_acc, fg_partials, fvs_out, V);
}

__global__ void k_reduce_partials(const double* __restrict__ partials, int nblocks, int ncomp,
                                  double* __restrict__ out, bool accumulate) {
  reduce_partials_block(partials, nblocks, ncomp, out, accumulate);
}

void launch_reduce_partials(const double* partials, int nblocks, int ncomp, double* out,
                            bool accumulate, cudaStream_t s) {
  k_reduce_partials<<<1, kBlock, 0, s>>>(partials, nblocks, ncomp, out, accumulate);
}

template <class Rec, bool VOL>
__global__ void k_finalize_compliance(const Rec* __restrict__ rec, const int* __restrict__ perm,
                                      int n, const double* __restrict__ acc, float inv_dt2,
                                      double* __restrict__ out) {
  XPBD_TID_OR_RETURN(n);
  finalize_elem<Rec, VOL>(i, rec, perm, acc, inv_dt2, out);
}

void launch_finalize_compliance(SegType t, const void* rec, const int* perm, int n,
                                const double* acc, float inv_dt2, double* out, cudaStream_t s) {
  if (n <= 0) return;
  switch (t) {
    case SEG_DIST:
      k_finalize_compliance<DistRec, false><<<grid_for(n), kBlock, 0, s>>>((const DistRec*)rec, perm, n, acc, inv_dt2, out);
      break;
    case SEG_BEND:
      k_finalize_compliance<BendRec, false><<<grid_for(n), kBlock, 0, s>>>((const BendRec*)rec, perm, n, acc, inv_dt2, out);
      break;
    default:
      k_finalize_compliance<TetRec, true><<<grid_for(n), kBlock, 0, s>>>((const TetRec*)rec, perm, n, acc, inv_dt2, out);
  }
}

__global__ void k_to_double(const float4* __restrict__ a, double* __restrict__ out, int V) {
  XPBD_TID_OR_RETURN(V);
  to_double_elem(i, a, out);
}

void launch_to_double(const float4* a, double* out, int V, cudaStream_t s) {
  if (V > 0) k_to_double<<<grid_for(V), kBlock, 0, s>>>(a, out, V);
}

// ======================================================================== utilities

__global__ void k_loss(const float4* __restrict__ ckx, const float* __restrict__ target,
                       float* __restrict__ seed_out, double* __restrict__ partials, int V) {
  double acc[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x)
    loss_elem(i, ckx, target, seed_out, acc[0]);
  block_sum_store<1>(acc, partials + blockIdx.x);
}

void launch_loss(const float4* ckx, const float* target, float* seed_out, double* partials,
                 int V, cudaStream_t s) {
  k_loss<<<partial_blocks(V), kBlock, 0, s>>>(ckx, target, seed_out, partials, V);
}

__global__ void k_read_state(const float4* __restrict__ ckx, const float4* __restrict__ ckv,
                             float* __restrict__ x_out, float* __restrict__ v_out, int V) {
  XPBD_TID_OR_RETURN(V);
  read_state_elem(i, ckx, ckv, x_out, v_out);
}

void launch_read_state(const float4* ckx, const float4* ckv, float* x_out, float* v_out, int V,
                       cudaStream_t s) {
  if (V > 0) k_read_state<<<grid_for(V), kBlock, 0, s>>>(ckx, ckv, x_out, v_out, V);
}

}  // namespace xpbd

// ======================================================================== materials
// Tet materials (Sec. "Volumetric Material Parameter Estimation"): material k has Lame
// parameters mu = a_k^2 and lambda = b_k^2, so the inverse moduli of a tet of material k
// are alpha_hat_D = 1/a_k^2 (deviatoric) and alpha_hat_H = 1/b_k^2 (hydrostatic).
namespace xpbd {

namespace {

__global__ void k_material_compliance(const int* __restrict__ mat, const float* __restrict__ a,
                                      const float* __restrict__ b, int nt, int n_mat, float* __restrict__ comp_h,
                                      float* __restrict__ comp_d, int* __restrict__ err) {
  XPBD_TID_OR_RETURN(nt);
  const int k = mat[i];
  if (k < 0 || k >= n_mat) {
    atomicOr(err, 8);
    return;
  }
  const float ak = a[k], bk = b[k];
  comp_h[i] = 1.f / (bk * bk);
  comp_d[i] = 1.f / (ak * ak);
}

// dL/da_k = sum over the tets of material k of dL/dalpha_hat_D * (-2 / a_k^3), and b_k with
// the hydrostatic entries.  One block per material sums its tets in a fixed order.
__global__ void __launch_bounds__(kBlock) k_material_gradient(const int* __restrict__ mat, const float* __restrict__ a,
                                                              const float* __restrict__ b, int nt,
                                                              const double* __restrict__ g_h,
                                                              const double* __restrict__ g_d, double* __restrict__ da,
                                                              double* __restrict__ db) {
  __shared__ double sh[2][kBlock / 32];
  const int k = blockIdx.x;
  double sd = 0.0, sh_ = 0.0;
  for (int t = threadIdx.x; t < nt; t += blockDim.x)
    if (mat[t] == k) {
      sd += g_d[t];
      sh_ += g_h[t];
    }
  for (int o = 16; o > 0; o >>= 1) {
    sd += __shfl_down_sync(0xffffffffu, sd, o);
    sh_ += __shfl_down_sync(0xffffffffu, sh_, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = sd;
    sh[1][threadIdx.x >> 5] = sh_;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double td = 0.0, th = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) {
      td += sh[0][w];
      th += sh[1][w];
    }
    const double ak = a[k], bk = b[k];
    if (da) da[k] = td * (-2.0 / (ak * ak * ak));
    if (db) db[k] = th * (-2.0 / (bk * bk * bk));
  }
}

}  // namespace

void launch_material_compliance(const int* mat, const float* a, const float* b, int nt, int n_mat, float* comp_h,
                                float* comp_d, int* err, cudaStream_t s) {
  if (nt > 0) k_material_compliance<<<grid_for(nt), kBlock, 0, s>>>(mat, a, b, nt, n_mat, comp_h, comp_d, err);
}

void launch_material_gradient(const int* mat, const float* a, const float* b, int nt, int n_mat, const double* g_h,
                              const double* g_d, double* da, double* db, cudaStream_t s) {
  if (n_mat > 0) k_material_gradient<<<n_mat, kBlock, 0, s>>>(mat, a, b, nt, g_h, g_d, da, db);
}

}  // namespace xpbd
