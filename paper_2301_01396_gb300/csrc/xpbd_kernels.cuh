// Internal launch interface of the XPBD kernels (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "xpbd_math.cuh"

namespace xpbd {

constexpr int kBlock = 256;

// Collider description passed by value to the kernels.
struct Collide {
  int flags;          // bit0 plane, bit1 sphere
  float h;            // plane y = h
  float cx, cy, cz, r;
  float at;           // contact alpha~ = contact compliance / dt^2
  float thick;
};

// Types of constraint records (segments of a color).
enum SegType { SEG_DIST = 0, SEG_BEND = 1, SEG_TETH = 2, SEG_TETD = 3 };
constexpr int kVerts[4] = {2, 4, 4, 4};

// ---- forward
void launch_init_ckpt(const float* x0, const float* v0, const float* w, float4* ckx, float4* ckv,
                      int V, cudaStream_t s);
void launch_set_alpha(SegType t, void* rec, const int* perm, int n, const float* compliance,
                      float inv_dt2, int* err, cudaStream_t s);
void launch_predict(const float4* ckx, const float4* ckv, float4* P, const float* fg_n,
                    const float* fv, float dt, float gx, float gy, float gz, Collide c,
                    uint8_t* cflags, int V, cudaStream_t s);
// lam_in == nullptr means lambda = 0 (first iteration of a step); tape == nullptr skips the
// record of pre-projection positions (forward only)
void launch_project(SegType t, const void* rec, int n, float4* P, const float* lam_in,
                    float* lam_out, float4* tape, cudaStream_t s);
void launch_contact(float4* P, const uint8_t* cflags, int V, const float2* lam_in,
                    float2* lam_out, float4* tape, Collide c, cudaStream_t s);
void launch_velocity(const float4* P, const float4* ckx_n, float4* ckx_next, float4* ckv_next,
                     float inv_dt, int V, int* err, cudaStream_t s);

// ---- reverse
void launch_seed_adjoint(const float* seed_x, const float* seed_v, float4* xbar, float4* vbar,
                         int V, cudaStream_t s);
void launch_adj_begin(float4* xbar, float4* vbar, float inv_dt, int V, cudaStream_t s);
// first: the first reverse iteration of a step (lambda-bar, alpha-bar start at 0);
// last: the final one (fold the step's alpha-bar into the float64 accumulator)
void launch_vjp(SegType t, const void* rec, int n, const float4* tape, const float* lam_pre,
                float4* xbar, float2* lb, double* acc, bool first, bool last, cudaStream_t s);
void launch_vjp_contact(const float4* tape, const uint8_t* cflags, int V, const float2* lam_pre,
                        float4* xbar, float2* lbc, float* cgrad, bool first, Collide c,
                        cudaStream_t s);
int partial_blocks(int V);
void launch_collider_partials(const float* cgrad, const uint8_t* cflags, int V, double* partials,
                              cudaStream_t s);
void launch_adj_predict(float4* xbar, float4* vbar, const float4* ckx_n, const float* seed,
                        float dt, double* fv_acc, double* fg_partials, int V, cudaStream_t s);
void launch_reduce_partials(const double* partials, int nblocks, int ncomp, double* out,
                            bool accumulate, cudaStream_t s);
void launch_finalize_compliance(SegType t, const void* rec, const int* perm, int n,
                                const double* acc, float inv_dt2, double* out, cudaStream_t s);
void launch_to_double(const float4* a, double* out, int V, cudaStream_t s);

// ---- utilities
void launch_loss(const float4* ckx, const float* target, float* seed_out, double* partials,
                 int V, cudaStream_t s);
void launch_read_state(const float4* ckx, const float4* ckv, float* x_out, float* v_out, int V,
                       cudaStream_t s);

}  // namespace xpbd
