// Internal definitions shared by the C-ABI runtime (xpbd_api.cu) and the batched serving
// runtime (xpbd_serve.cu): the solver handle, its per-color segments and workspace, error
// reporting and the counted/timed launch helper.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/diffxpbd.h"
#include "xpbd_kernels.cuh"

using namespace xpbd;

inline thread_local std::string g_err;

// A named NVTX range around an entry point's host work (what it enqueues shows up under it
// in a timeline profiler; without a profiler attached the calls do nothing).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

inline xpbd_status fail(xpbd_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define CU_TRY(expr)                                                                    \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? XPBD_ERR_OOM : XPBD_ERR_CUDA,       \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

#define LAUNCH_CHECK()                                                                  \
  do {                                                                                  \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess)                                                              \
      return fail(XPBD_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

struct Seg {
  SegType type;
  int begin;   // first record of the type array
  int count;
};

// Device buffer that grows on demand and is freed with the handle.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, need ? need : 16);
    if (e == cudaSuccess) bytes = need;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

struct xpbd_solver {
  int V = 0, nd = 0, nb = 0, nt = 0, m = 0, K = 0;
  // Coupled tets: the colors hold C_H segments only, and the C_D records (type 3) are
  // shadows of the C_H records in the same order, updated with them by one 2x2 solve.
  bool coupled = false;
  // Membranes (segments of type SEG_MEMB): records in color-segment order, record ->
  // triangle id, and the slot block they use: record i's slot k at mslot + i + k * nm
  // (k < 3 multipliers; k < 4 adjoint pairs and float64 accumulators); their tape follows
  // the four types' in each iteration, 3 float4 per record from mtape.
  int nm = 0;
  MembRec* d_mrec = nullptr;
  int* d_mperm = nullptr;
  int mslot = 0;
  size_t mtape = 0;
  std::vector<std::vector<Seg>> colors;
  // type arrays in record order; rec_off[t] = offset of type t in the m-long record space
  int n_rec[4] = {0, 0, 0, 0};
  int rec_off[4] = {0, 0, 0, 0};
  void* d_rec[4] = {nullptr, nullptr, nullptr, nullptr};
  int* d_perm = nullptr;        // [m] record index -> global constraint id
  float* d_w = nullptr;         // [V] inverse masses
  int* d_err = nullptr;
  // workspace
  DevBuf P, lam, cflags, lamc;                       // forward
  DevBuf tape, lam_tape, tape_c, lamc_tape;          // replay tapes
  DevBuf xbar, vbar, lb, acc, lbc, cgrad, partials;  // reverse
  DevBuf roll, seg;                                  // sparse checkpoints: rolling / segment states
  DevBuf imp_blocks, imp_vec, imp_dinv, imp_sc;      // implicit adjoint: blocks, CG vectors, scalars
  DevBuf imp_mg;                                     // implicit adjoint: multigrid levels
  // launch statistics per kernel class (always counted; timed with CUDA events on the
  // launching stream while profiling is enabled)
  bool prof_on = false;
  int64_t launches[XPBD_KERNEL_CLASSES] = {0};
  int64_t units[XPBD_KERNEL_CLASSES] = {0};
  double alg_bytes[XPBD_KERNEL_CLASSES] = {0};
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Timed { int cls; cudaEvent_t a, b; };
  std::vector<Timed> timed;
  // phase execution plan: runs of consecutive colors launched together (see xpbd_phase.cu)
  bool use_phases = false;
  struct PhaseHost {
    int first_group = 0, n_groups = 0, c0 = 0, ncolors = 0, max_verts = 0, max_chunks = 0;
    int type_mask = 0;                      // bit t: constraint type t occurs
    int max_chunk_size = 0;
    // padded per-group tables: group g's vertex list at vbase + g * vstride (padding -1),
    // its chunks at cbase + g * cstride (padding: empty chunks), forward and reverse order
    int64_t vbase = 0, cbase = 0;
    int vstride = 0, cstride = 0;
    PhaseShape shape() const { return PhaseShape{n_groups, max_verts, max_chunks, type_mask, max_chunk_size}; }
    int64_t units = 0;                      // constraints updated by one launch
    double bytes_fwd = 0, bytes_replay = 0, bytes_vjp = 0;   // algorithmic bytes per launch
  };
  std::vector<PhaseHost> phases;
  // per type (membranes last: 4 slots per record, component-major)
  void* d_prec[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // phase-ordered records (padded);
                                                                     // bending: int4 vertex indices
  BendTail* d_prec_btail = nullptr;                                  // bending: (theta0, alpha~)
  int n_prec[5] = {0, 0, 0, 0, 0};                                   // phase records per type
  int pslot_off[5] = {0, 0, 0, 0, 0};                                // their offsets in the slot space
  size_t ptape_off[5] = {0, 0, 0, 0, 0};                             // float4 offsets in an iteration's tape
  int* d_pperm = nullptr;                                     // phase record -> constraint id (-1: pad)
  PhaseGroup* d_groups = nullptr;
  PhaseChunk* d_chunks = nullptr;
  PhaseChunk* d_chunks_rev = nullptr;
  int* d_pverts = nullptr;
  // Per-constraint slot space of the multiplier / adjoint buffers and float4 entries of
  // one iteration's tape: large enough for the per-color layout and the padded phase layout.
  size_t slots = 0, tape_slots = 0;
  // Multiplier slots of the one-launch-per-color layout alone (no phase padding).
  size_t color_slots() const { return (size_t)mslot + ((size_t)4 * nm + 3) / 4 * 4; }
  // Device address of the allocation-free forward's fixed working array on the device this
  // handle was created on (looked up by xpbd_create).
  void* static_base = nullptr;
  size_t tape_per_iter() const {  // float4 entries per iteration, per-color layout
    return (size_t)2 * nd + (size_t)4 * nb + (size_t)8 * nt + (size_t)3 * nm;
  }
};

inline cudaEvent_t next_event(xpbd_solver* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

// Algorithmic bytes per constraint of the one-color launches (steady-state iteration):
//   forward  distance: record 16 + lambda r/w 8 + two vertices read and written 64 = 88;
//            bending / tet: record 32 / 64 + lambda 8 + four vertices r/w 128 = 168 / 200
//   replay   forward + the pre-projection tape write (16 B per vertex): 120 / 232 / 264
//   reverse  distance: record 16 + tape 32 + lambda 4 + vertex adjoints r/w 64 +
//            (lambar, alphabar) r/w 16 = 132; bending 244; tets 276
inline double unit_bytes(int cls) {
  switch (cls) {
    case XPBD_K_FWD_DIST: return 88;
    case XPBD_K_FWD_BEND: return 168;
    case XPBD_K_FWD_TETH: case XPBD_K_FWD_TETD: return 200;
    case XPBD_K_REPLAY_DIST: return 120;
    case XPBD_K_REPLAY_BEND: return 232;
    case XPBD_K_REPLAY_TETH: case XPBD_K_REPLAY_TETD: return 264;
    case XPBD_K_VJP_DIST: return 132;
    case XPBD_K_VJP_BEND: return 244;
    case XPBD_K_VJP_TETH: case XPBD_K_VJP_TETD: return 276;
    // membrane: record 48 + three multipliers r/w 24 + three vertices r/w 96 (+ tape 48);
    // reverse: record 48, tape 48, multipliers 12, vertex adjoints r/w 96, four
    // (lambar, alphabar) pairs r/w 64
    case XPBD_K_FWD_MEMB: return 168;
    case XPBD_K_REPLAY_MEMB: return 216;
    case XPBD_K_VJP_MEMB: return 268;
    default: return 0;
  }
}

// Counts (and, while profiling, times) one kernel launch of class `cls` covering `units`
// constraints or vertices and moving `bytes` algorithmic bytes (< 0: units x unit_bytes).
// Launches with no work are skipped by the launchers and not counted.
template <class F>
inline void launch(xpbd_solver* h, int cls, int64_t units, cudaStream_t s, F&& f, double bytes = -1.0) {
  if (units <= 0) return;
  h->alg_bytes[cls] += bytes >= 0 ? bytes : (double)units * unit_bytes(cls);
  cudaEvent_t a = nullptr, b = nullptr;
  if (h->prof_on) {
    a = next_event(h);
    b = next_event(h);
    if (a) cudaEventRecord(a, s);
  }
  f();
  h->launches[cls] += 1;
  h->units[cls] += units;
  if (h->prof_on && a && b) {
    cudaEventRecord(b, s);
    h->timed.push_back({cls, a, b});
  }
}

inline size_t tape_offset(const xpbd_solver* h, SegType t) {   // float4 offset of type t in one iteration
  size_t o = 0;
  for (int k = 0; k < (int)t; ++k) o += (size_t)h->n_rec[k] * kVerts[k];
  return o;
}

inline void* rec_ptr(const xpbd_solver* h, SegType t, int begin) {
  static const size_t sz[4] = {sizeof(DistRec), sizeof(BendRec), sizeof(TetRec), sizeof(TetRec)};
  return (char*)h->d_rec[t] + sz[t] * (size_t)begin;
}

// The record segments a color segment stands for: itself, and for coupled tets the C_D
// shadow of a C_H segment as well (launched after it: same vertices, so the two launches
// of an assembly pass over one color never write the same vertex at once).
template <class F>
inline void for_each_record_seg(const xpbd_solver* h, const Seg& g, F&& f) {
  f(g);
  if (h->coupled && g.type == SEG_TETH) f(Seg{SEG_TETD, g.begin, g.count});
}

inline Collide make_collide(const xpbd_params* p) {
  Collide c;
  c.flags = p->collider_flags & 3;
  c.h = p->plane_h;
  c.cx = p->sphere[0];
  c.cy = p->sphere[1];
  c.cz = p->sphere[2];
  c.r = p->sphere[3];
  c.at = p->contact_compliance / (p->dt * p->dt);
  c.thick = p->thickness;
  return c;
}

inline xpbd_status check_params(const xpbd_solver* h, const xpbd_params* p, int steps, int iters) {
  if (!h || !p) return fail(XPBD_ERR_INVALID, "null handle or params");
  if (steps < 0 || iters < 1) return fail(XPBD_ERR_INVALID, "steps must be >= 0 and iters >= 1");
  if (!(p->dt > 0.f) || !std::isfinite(p->dt)) return fail(XPBD_ERR_INVALID, "dt must be positive");
  if (h->m > 0 && !p->compliance) return fail(XPBD_ERR_INVALID, "compliance is NULL");
  if (h->nm > 0 && !p->memb_stiffness) return fail(XPBD_ERR_INVALID, "memb_stiffness is NULL");
  if (p->collider_flags & ~3) return fail(XPBD_ERR_INVALID, "unknown collider flag");
  if ((p->collider_flags & XPBD_COLLIDE_SPHERE) && !(p->sphere[3] > 0.f))
    return fail(XPBD_ERR_INVALID, "sphere radius must be positive");
  if (p->collider_flags && !(p->contact_compliance >= 0.f))
    return fail(XPBD_ERR_INVALID, "contact compliance must be >= 0");
  return XPBD_OK;
}

inline const float4* ck_x(const float* ck, int V, int n) {
  return reinterpret_cast<const float4*>(ck) + (size_t)2 * V * n;
}
inline const float4* ck_v(const float* ck, int V, int n) { return ck_x(ck, V, n) + V; }

