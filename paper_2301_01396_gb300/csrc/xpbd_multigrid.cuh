// Geometric multigrid preconditioner of the implicit adjoint's conjugate gradients, for a
// model whose vertices form an nx x ny grid (vertex (i, j) = j * nx + i) and whose
// constraints couple only vertices at most two grid cells apart in each direction (the
// stretch, shear and bending stencils of a grid cloth).
//
// Every level stores its matrix as a 5 x 5 stencil of 3x3 float64 blocks per vertex:
// A[v][(dy + 2) * 5 + (dx + 2)] is the block between vertex v and its neighbour at offset
// (dx, dy).  Level 0 is assembled from the per-constraint blocks of A = M + sum_j B_j (the
// operator of "Adjoint State Computation"); level l + 1 is the Galerkin product P^T A_l P
// with bilinear prolongation P from a coarse grid of ((nx + 1) / 2) x ((ny + 1) / 2)
// vertices (coarse vertex (I, J) sits on fine vertex (2I, 2J); an odd fine vertex takes the
// mean of its two coarse neighbours, or the one it has at a boundary).  Bilinear P
// reproduces linear displacement fields, so rigid translations and infinitesimal rotations
// stay in every coarse space; pinned vertices have zero rows of P ("Linear System
// Filtering").  The coarsest level (at most 4 x 4 vertices) is inverted densely.
//
// Smoothing is symmetric Gauss-Seidel: forward sweeps before the coarse correction,
// backward sweeps after, so the V-cycle is a symmetric positive definite preconditioner
// for a symmetric positive definite A.  Coarse levels use 9-colour point Gauss-Seidel with
// 3x3 block diagonals (vertices of one colour are three cells apart).  On level 0 the
// smoother can instead solve whole grid diagonals (lines x - y = c, or x + y = c) exactly:
// a cloth triangulated along one diagonal with hinges only on its axis-aligned edges folds
// along that diagonal at no bending cost, so while it is slack every out-of-plane field
// constant along those lines, w = f(x - y), has only its mass as stiffness; no point
// smoother or smooth coarse space reduces such modes, and a line smoother contains them.
// Lines more than four apart do not interact, so 5 line colours run in parallel.
#pragma once

#include "xpbd_kernels.cuh"
#include "xpbd_mg_index.h"

namespace xpbd {

// Level-0 assembly (A0 zeroed by the caller): mass and contact blocks, then the blocks of
// one colour's records at a time (records of one colour share no vertex, so their rows
// are disjoint).  A pair of vertices outside the stencil or the grid sets *flag = 1.
void launch_mg_asm_mass_contacts(const float4* X, const uint8_t* cflags, const float2* lamc, Collide c, bool pd,
                                 double* A0, int V, cudaStream_t s);
void launch_mg_asm_block(SegType t, const void* rec, int n, const float4* X, const float* lam, const double* blocks,
                         bool pd, double* A0, int nx, int V, double* flag, cudaStream_t s);
void launch_mg_asm_memb(const MembRec* rec, int n, const double* blocks, double* A0, int nx, int V, double* flag,
                        cudaStream_t s);

// Setup pieces (X: level-0 pin mask, null on coarse levels).
void launch_mg_rap(const MgLevel& f, const MgLevel& c, const float4* X, cudaStream_t s);
void launch_mg_dinv(const MgLevel& l, const float4* X, cudaStream_t s);
void launch_mg_coarse_inverse(const MgLevel& l, const float4* X, double* cinv, cudaStream_t s);
void launch_mg_line_factor(const MgLevel& l, const float4* X, int dir, float* lfac, cudaStream_t s);

// V-cycle pieces.
void launch_mg_point_gs(const MgLevel& l, const double* b, double* x, int color, cudaStream_t s);
void launch_mg_line_resid(const MgLevel& l, const float4* X, const double* b, const double* x, double* r, int dir,
                          int color, cudaStream_t s);
void launch_mg_line_solve(const MgLevel& l, const float* lfac, double* r, double* x, int dir, int color,
                          cudaStream_t s);
void launch_mg_resid(const MgLevel& l, const float4* X, const double* b, const double* x, double* r, cudaStream_t s);
void launch_mg_restrict(const MgLevel& f, const double* r, const MgLevel& c, double* bc, cudaStream_t s);
void launch_mg_prolong(const MgLevel& c, const double* xc, const MgLevel& f, const float4* X, double* x,
                       cudaStream_t s);
void launch_mg_coarse_solve(const MgLevel& l, const double* cinv, const double* b, double* x, cudaStream_t s);

// Conjugate-gradient pieces for an external preconditioner z = P^-1 r.
void launch_cg_init(const float4* X, const double* b, double* y, double* r, int V, cudaStream_t s);
// p = z (when p is non-null); partial sums of (r.z, r.r[, r.r]) (ncomp 2 or 3).
void launch_cg_rz(const double* r, const double* z, double* p, double* partials, int ncomp, int V, cudaStream_t s);
// alpha = rz / pq; y += alpha p; r -= alpha q.
void launch_cg_update(const double* sc, int rz_slot, const double* p, const double* q, double* y, double* r, int V,
                      cudaStream_t s);

}  // namespace xpbd
