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

// Blocks of kBlock threads covering n items; a kernel's thread index i, returning past n.
inline int grid_for(int n) { return (n + kBlock - 1) / kBlock; }
#define XPBD_TID_OR_RETURN(n)                          \
  const int i = blockIdx.x * blockDim.x + threadIdx.x; \
  if (i >= (n)) return

// Types of constraint records (segments of a color).
// SEG_MEMB segments hold membrane records, which sit outside the four per-type arrays
// (their own record array, multiplier block and tape range).
enum SegType { SEG_DIST = 0, SEG_BEND = 1, SEG_TETH = 2, SEG_TETD = 3, SEG_MEMB = 4 };
constexpr int kVerts[5] = {2, 4, 4, 4, 3};
constexpr int kSegTypes = 5;

// ---- forward
void launch_init_ckpt(const float* x0, const float* v0, const float* w, float4* ckx, float4* ckv,
                      int V, cudaStream_t s);
void launch_set_alpha(SegType t, void* rec, const int* perm, int n, const float* compliance,
                      float inv_dt2, int* err, cudaStream_t s);
// alpha~ of the phase bending records' tails (BendTail array)
void launch_set_alpha_btail(BendTail* tail, const int* perm, int n, const float* compliance, float inv_dt2, int* err,
                            cudaStream_t s);
void launch_predict(const float4* ckx, const float4* ckv, float4* P, const float* fg_n,
                    const float* fv, const float* fvs_n, float dt, float gx, float gy, float gz, Collide c,
                    uint8_t* cflags, int V, cudaStream_t s);
// lam_in == nullptr means lambda = 0 (first iteration of a step); tape == nullptr skips the
// record of pre-projection positions (forward only)
void launch_project(SegType t, const void* rec, int n, float4* P, const float* lam_in,
                    float* lam_out, float4* tape, cudaStream_t s);
// Coupled tets: the C_H records rh of a color segment with their C_D shadows rd; the C_D
// multipliers are doff slots after the C_H ones, the tape holds the C_H layout.
void launch_project_tet_pair(const TetRec* rh, const TetRec* rd, int n, float4* P, const float* lam_in,
                             float* lam_out, int doff, float4* tape, cudaStream_t s);
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
// Membranes: `stride` separates the per-component multiplier / adjoint slots of one
// record (slot k of record i at i + k * stride), the tape holds 3 float4 per record.
void launch_memb_set_alpha(MembRec* rec, const int* perm, int n, const float* stiffness, float inv_dt2, int* err,
                           cudaStream_t s);
void launch_project_memb(const MembRec* rec, int n, float4* P, const float* lam_in, float* lam_out, int stride,
                         float4* tape, cudaStream_t s);
void launch_vjp_memb(const MembRec* rec, int n, const float4* tape, const float* lam_pre, int stride, float4* xbar,
                     float2* lb, double* acc, bool first, bool last, cudaStream_t s);
void launch_memb_gradient(const MembRec* rec, const int* perm, int n, const float* stiffness, float inv_dt2,
                          const double* acc, int stride, double* out, cudaStream_t s);
void launch_vjp_tet_pair(const TetRec* rh, const TetRec* rd, int n, const float4* tape, const float* lam_pre,
                         int doff, float4* xbar, float2* lb, double* acc, bool first, bool last, cudaStream_t s);
void launch_vjp_contact(const float4* tape, const uint8_t* cflags, int V, const float2* lam_pre,
                        float4* xbar, float2* lbc, float* cgrad, bool first, Collide c,
                        cudaStream_t s);
int partial_blocks(int V);
void launch_collider_partials(const float* cgrad, const uint8_t* cflags, int V, double* partials,
                              cudaStream_t s);
void launch_adj_predict(float4* xbar, float4* vbar, const float4* ckx_n, const float* seed,
                        float dt, double* fv_acc, double* fg_partials, double* fvs_out, int V, cudaStream_t s);
void launch_reduce_partials(const double* partials, int nblocks, int ncomp, double* out,
                            bool accumulate, cudaStream_t s);
void launch_finalize_compliance(SegType t, const void* rec, const int* perm, int n,
                                const double* acc, float inv_dt2, double* out, cudaStream_t s);
void launch_to_double(const float4* a, double* out, int V, cudaStream_t s);

// ---- phase execution (xpbd_phase.cu): several consecutive colors per launch
constexpr int kPhaseBlock = 256;                 // consumer threads per CTA = constraints per chunk
constexpr int kPhaseChunk = kPhaseBlock;
constexpr int kPhaseThreads = kPhaseBlock + 32;  // + one producer warp
constexpr int kPhaseMaxVerts = 6144;             // largest component a phase may hold
constexpr int kPhaseGroupVerts = 1536;           // small components are packed up to this
constexpr int kPhaseTargetGroups = 304;          // CTAs a phase should keep (2 per SM) before packing
constexpr int kPhaseMaxStages = 8;
constexpr int kPhaseSmemLimit = 226 * 1024;      // dynamic shared memory per CTA (below the 227 KB opt-in
                                                 // maximum, leaving room for static shared memory)

struct PhaseGroup {   // one CTA: a set of components of one phase
  int vert_begin;     // first entry of its vertex list (global vertex ids, ascending)
  int vert_count;     // local vertex vert_count is a zero-mass dummy that padding records use
  int chunk_begin;    // its chunks, in forward execution order
  int chunk_count;
};
struct PhaseChunk {   // up to kPhaseChunk constraints of one type and one color of a group
  int type;           // SegType, or kChunkPair
  int begin;          // first record in the phase record array of its type (multiple of 4)
  int count;          // multiple of 4
  int flags;          // kChunkColorFirst / kChunkColorLast: first / last chunk of its color
};
constexpr int kChunkColorFirst = 1, kChunkColorLast = 2;
// Chunk type of coupled tets: C_H records with their C_D shadows (same phase index in the
// type-3 array, multipliers in the type-3 slots), updated by one 2x2 solve each.
constexpr int kChunkPair = 5;
struct PhaseLaunch {
  const PhaseGroup* groups;
  // CTA b's vertex list at pverts + b * vstride (padded with -1) and its chunks at
  // chunks + b * cstride in execution order (chunks_rev: reverse order; padded with empty
  // chunks), so a CTA finds them without first reading its PhaseGroup
  const PhaseChunk* chunks;
  const PhaseChunk* chunks_rev;
  const int* pverts;
  int vstride, cstride;
  int slot_off[5];         // offset of each type in the multiplier slot space (multiples of 4)
  const void* prec[5];     // phase records (vertex indices local to the group); bending:
                           // the int4 vertex indices, with their tails in prec_btail
  const BendTail* prec_btail;
  size_t tape_off[5];      // float4 offset of each type within one iteration's tape
  int memb_stride;         // membranes: slot k of phase record i at slot_off[4] + i + k * memb_stride
  float4* P;               // positions (forward / replay) or vertex adjoints (reverse)
  const float* lam_in;     // multipliers before the iteration (NULL: zero)
  float* lam_out;
  float4* tape;            // this iteration's tape (written by replay, read by reverse)
  float2* lb;              // reverse: (lambar, alphabar) per constraint
  double* acc;             // reverse: float64 compliance-adjoint accumulator
  int* err;                // device error word (bit 4: a bounded wait gave up)
  long long wait_cycles;   // limit of every wait (SM clock cycles)
  int no_issue;            // self-test of the bounded waits: the producer issues no copies
  // shared-memory layout, filled by the launcher: vertices (float4, then their global
  // indices), chunk table, stage ring
  int vert_bytes;
  int chunk_bytes;
  int slot_bytes;          // bytes of one stage
  int stages;              // stages in flight
  unsigned stage_magic;    // ceil(2^32 / stages): k / stages = __umulhi(k, stage_magic) for the
                           // chunk counts of a group (exact for k < 2^32 / stages)
};
// Sizes of one phase: its groups, the largest group's vertex and chunk counts and the
// constraint types present (bit t set when type t occurs; selects the kernel).
struct PhaseShape {
  int n_groups, max_verts, max_chunks, type_mask;
  int max_chunk_size;   // the largest chunk's constraint count (a stage holds one such chunk)
};
cudaError_t phase_kernel_setup();
// Shared memory a launch of this phase needs (0 if it cannot fit).
size_t phase_smem_bytes(const PhaseShape& sh, bool reverse);
void launch_phase_fwd(PhaseLaunch a, const PhaseShape& sh, bool record, cudaStream_t s);
void launch_phase_vjp(PhaseLaunch a, const PhaseShape& sh, bool first, bool last, cudaStream_t s);

// ---- implicit adjoint (xpbd_implicit.cu): blocks, matrix-free products, PCG pieces
void launch_quad_blocks(SegType t, const void* rec, int n, const float4* X, const float* lam, double* blocks, bool pd,
                        cudaStream_t s);
// membranes: 21 packed float64 per block (6x6 in the relative coordinates of vertices 1, 2);
// multiplier and accumulator slots k of record i at i + k * stride
void launch_memb_blocks(const MembRec* rec, int n, const float4* X, const float* lam, int stride, double* blocks, bool pd,
                        cudaStream_t s);
void launch_apply_memb(const MembRec* rec, int n, const double* blocks, const double* p, double* q, cudaStream_t s);
void launch_diag_memb(const MembRec* rec, int n, const double* blocks, double* dg, cudaStream_t s);
void launch_abar_memb(const MembRec* rec, int n, const float4* X, const float* lam, int stride, const double* y,
                      double* acc, cudaStream_t s);
void launch_apply_mass_contacts(const float4* X, const uint8_t* cflags, const float2* lamc, Collide c, bool pd,
                                const double* p, double* q, int V, cudaStream_t s);
void launch_apply_block(SegType t, const void* rec, int n, const float4* X, const float* lam, const double* blocks,
                        bool pd, const double* p, double* q, cudaStream_t s);
void launch_diag_mass_contacts(const float4* X, const uint8_t* cflags, const float2* lamc, Collide c, bool pd,
                               double* dg, int V, cudaStream_t s);
void launch_diag_block(SegType t, const void* rec, int n, const float4* X, const float* lam, const double* blocks,
                       bool pd, double* dg, cudaStream_t s);
void launch_diag_invert(const float4* X, double* dg, int V, cudaStream_t s);
void launch_cg_start(const float4* X, const double* b, const double* dinv, double* y, double* r, double* z, double* p,
                     double* partials, int V, cudaStream_t s);
void launch_cg_pq(const float4* X, const double* p, double* q, double* partials, int V, cudaStream_t s);
void launch_cg_step(const double* sc, int rz_slot, const double* p, const double* q, const double* dinv, double* y,
                    double* r, double* z, double* partials, int V, cudaStream_t s);
void launch_cg_dir(const double* sc, int old_slot, int new_slot, const double* z, double* p, int V, cudaStream_t s);
void launch_implicit_finish(const float4* X, const double* b, const double* y, const double* ay, float4* xbar, int V,
                            cudaStream_t s);
void launch_xbar_to_b(const float4* xbar, double* b, int V, cudaStream_t s);
void launch_abar(SegType t, const void* rec, int n, const float4* X, const float* lam, const double* y, double* acc,
                 cudaStream_t s);

// ---- tet materials (mu = a^2, lambda = b^2)
void launch_material_compliance(const int* mat, const float* a, const float* b, int nt, int n_mat, float* comp_h,
                                float* comp_d, int* err, cudaStream_t s);
void launch_material_gradient(const int* mat, const float* a, const float* b, int nt, int n_mat, const double* g_h,
                              const double* g_d, double* da, double* db, cudaStream_t s);

// ---- utilities
void launch_loss(const float4* ckx, const float* target, float* seed_out, double* partials,
                 int V, cudaStream_t s);
void launch_read_state(const float4* ckx, const float4* ckv, float* x_out, float* v_out, int V,
                       cudaStream_t s);

}  // namespace xpbd
