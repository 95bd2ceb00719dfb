// Batched serving runtime: continuous batching of forward + gradient requests on one GPU.
//
// Every admitted request is a fixed program of passes (the same sequence xpbd_forward,
// xpbd_loss and xpbd_adjoint launch for it).  A tick runs the next pass of every resident
// request: its blocks are the concatenation of those passes' blocks, and each block looks
// up its pass in a table built on the host.  A batch of up to kMaxTicksPerRun ticks is one
// cooperative launch of k_ticks (a grid no larger than the GPU holds at once): its blocks
// walk the first tick's blocks, meet at a grid-wide barrier, walk the next tick's, and so
// on.  Consecutive passes of one request are ordered by those barriers; passes of
// different requests touch disjoint memory, so they share a tick freely.  Each element of
// a pass runs the element function of xpbd_elems.cuh that the one-request kernels run,
// and a pass is split into blocks the same way whatever shares its tick, so a request's
// results do not depend on the mix.  The barrier's waits are bounded: a wait that runs out
// latches an error and every block leaves the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "xpbd_elems.cuh"
#include "xpbd_solver.cuh"

namespace xpbd {

enum ItemKind : int32_t {
  IK_SET_ALPHA = 0,
  IK_INIT_CKPT,
  IK_PREDICT,
  IK_PROJ,
  IK_CONTACT,
  IK_VELOCITY,
  IK_LOSS,
  IK_REDUCE,
  IK_SEED_ADJ,
  IK_ADJ_BEGIN,
  IK_VJP,
  IK_VJP_CONTACT,
  IK_ADJ_PREDICT,
  IK_COLLIDER_PARTIALS,
  IK_FINALIZE,
  IK_TO_DOUBLE
};

// One pass of one request inside a dispatch launch.
struct __align__(16) TickItem {
  int32_t kind;
  int32_t sub;      // constraint type (SET_ALPHA, PROJ, VJP, FINALIZE); components (REDUCE)
  int32_t n;        // elements; REDUCE: number of partial blocks
  int32_t block0;   // first block of this pass in the launch
  int32_t flags;    // bit0 first reverse iteration, bit1 last, bit2 accumulate (REDUCE)
  int32_t pad[3];
  const void* rec;
  void* p[7];
  float f[4];
  Collide col;
};
static_assert(sizeof(TickItem) % 16 == 0, "TickItem alignment");

__host__ __device__ inline int item_blocks(const TickItem& it) {
  return it.kind == IK_REDUCE ? 1 : (it.n + kBlock - 1) / kBlock;
}

// The ticks of one batch: tick t's passes are items [first, first + count) of the batch
// table, and its blocks number `blocks`.
struct __align__(16) TickHead {
  int32_t first, count, blocks, pad;
};

// Block b of a tick: runs block (b - block0) of the pass whose block range holds b.
__device__ __forceinline__ void tick_block(const TickItem* __restrict__ items, int n_items, int b, TickItem& it) {
  if (threadIdx.x == 0) {
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (items[mid].block0 <= b)
        lo = mid;
      else
        hi = mid - 1;
    }
    it = items[lo];
  }
  __syncthreads();
  const int lb = b - it.block0;
  const int i = lb * kBlock + threadIdx.x;
  const bool ok = i < it.n;
  const bool first = (it.flags & 1) != 0, last = (it.flags & 2) != 0;
  switch (it.kind) {
    case IK_SET_ALPHA:
      if (ok) {
        if (it.sub == SEG_DIST)
          set_alpha_elem<DistRec, false>(i, (DistRec*)it.rec, (const int*)it.p[0], (const float*)it.p[1], it.f[0], (int*)it.p[2]);
        else if (it.sub == SEG_BEND)
          set_alpha_elem<BendRec, false>(i, (BendRec*)it.rec, (const int*)it.p[0], (const float*)it.p[1], it.f[0], (int*)it.p[2]);
        else
          set_alpha_elem<TetRec, true>(i, (TetRec*)it.rec, (const int*)it.p[0], (const float*)it.p[1], it.f[0], (int*)it.p[2]);
      }
      break;
    case IK_INIT_CKPT:
      if (ok) init_ckpt_elem(i, (const float*)it.p[0], (const float*)it.p[1], (const float*)it.p[2], (float4*)it.p[3], (float4*)it.p[4]);
      break;
    case IK_PREDICT:
      if (ok)
        predict_elem(i, (const float4*)it.p[0], (const float4*)it.p[1], (float4*)it.p[2], (const float*)it.p[3],
                     (const float*)it.p[4], nullptr, it.f[0], it.f[1], it.f[2], it.f[3], it.col, (uint8_t*)it.p[5]);
      break;
    case IK_PROJ:
      if (ok) {
        float4* P = (float4*)it.p[0];
        const float* li = (const float*)it.p[1];
        float* lo = (float*)it.p[2];
        float4* tp = (float4*)it.p[3];
        if (it.sub == SEG_DIST)
          proj_dist_elem(i, (const DistRec*)it.rec, P, li, lo, tp);
        else if (it.sub == SEG_BEND)
          proj_quad_elem<1>(i, (const BendRec*)it.rec, P, li, lo, tp);
        else if (it.sub == SEG_TETH)
          proj_quad_elem<2>(i, (const TetRec*)it.rec, P, li, lo, tp);
        else
          proj_quad_elem<3>(i, (const TetRec*)it.rec, P, li, lo, tp);
      }
      break;
    case IK_CONTACT:
      if (ok) contact_elem(i, (float4*)it.p[0], (const uint8_t*)it.p[1], (const float2*)it.p[2], (float2*)it.p[3], (float4*)it.p[4], it.col);
      break;
    case IK_VELOCITY:
      if (ok) velocity_elem(i, (const float4*)it.p[0], (const float4*)it.p[1], (float4*)it.p[2], (float4*)it.p[3], it.f[0], (int*)it.p[4]);
      break;
    case IK_LOSS: {
      double acc[1] = {0.0};
      if (ok) loss_elem(i, (const float4*)it.p[0], (const float*)it.p[1], (float*)it.p[2], acc[0]);
      block_sum_store<1>(acc, (double*)it.p[3] + lb);
      break;
    }
    case IK_REDUCE:
      reduce_partials_block((const double*)it.p[0], it.n, it.sub, (double*)it.p[1], (it.flags & 4) != 0);
      break;
    case IK_SEED_ADJ:
      if (ok) seed_adjoint_elem(i, (const float*)it.p[0], (const float*)it.p[1], (float4*)it.p[2], (float4*)it.p[3]);
      break;
    case IK_ADJ_BEGIN:
      if (ok) adj_begin_elem(i, (float4*)it.p[0], (float4*)it.p[1], it.f[0]);
      break;
    case IK_VJP:
      if (ok) {
        const float4* tp = (const float4*)it.p[0];
        const float* lp = (const float*)it.p[1];
        float4* xb = (float4*)it.p[2];
        float2* lbp = (float2*)it.p[3];
        double* ac = (double*)it.p[4];
        if (it.sub == SEG_DIST)
          vjp_dist_elem(i, (const DistRec*)it.rec, tp, lp, xb, lbp, ac, first, last);
        else if (it.sub == SEG_BEND)
          vjp_quad_elem<1>(i, (const BendRec*)it.rec, tp, lp, xb, lbp, ac, first, last);
        else if (it.sub == SEG_TETH)
          vjp_quad_elem<2>(i, (const TetRec*)it.rec, tp, lp, xb, lbp, ac, first, last);
        else
          vjp_quad_elem<3>(i, (const TetRec*)it.rec, tp, lp, xb, lbp, ac, first, last);
      }
      break;
    case IK_VJP_CONTACT:
      if (ok)
        vjp_contact_elem(i, (const float4*)it.p[0], (const uint8_t*)it.p[1], (const float2*)it.p[2], (float4*)it.p[3],
                         (float2*)it.p[4], (float*)it.p[5], first, it.col);
      break;
    case IK_ADJ_PREDICT: {
      double fs[3] = {0.0, 0.0, 0.0};
      if (ok) adj_predict_elem(i, (float4*)it.p[0], (float4*)it.p[1], (const float4*)it.p[2], (const float*)it.p[3], it.f[0], (double*)it.p[4], fs);
      if (it.p[5]) block_sum_store<3>(fs, (double*)it.p[5] + 3 * lb);
      break;
    }
    case IK_COLLIDER_PARTIALS: {
      double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      if (ok) collider_contrib(i, (const float*)it.p[0], (const uint8_t*)it.p[1], v);
      block_sum_store<5>(v, (double*)it.p[2] + 5 * lb);
      break;
    }
    case IK_FINALIZE:
      if (ok) {
        if (it.sub == SEG_DIST)
          finalize_elem<DistRec, false>(i, (const DistRec*)it.rec, (const int*)it.p[0], (const double*)it.p[1], it.f[0], (double*)it.p[2]);
        else if (it.sub == SEG_BEND)
          finalize_elem<BendRec, false>(i, (const BendRec*)it.rec, (const int*)it.p[0], (const double*)it.p[1], it.f[0], (double*)it.p[2]);
        else
          finalize_elem<TetRec, true>(i, (const TetRec*)it.rec, (const int*)it.p[0], (const double*)it.p[1], it.f[0], (double*)it.p[2]);
      }
      break;
    case IK_TO_DOUBLE:
      if (ok) to_double_elem(i, (const float4*)it.p[0], (double*)it.p[1]);
      break;
    default:
      break;
  }
  __syncthreads();   // `it` is rewritten by the next block this thread block runs
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_gpu(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch: bar[0] counts arrivals, bar[1] is the
// generation.  The last block to arrive resets the count and advances the generation
// (release); the others wait for the generation to change (acquire), at most `limit`
// cycles, after which they latch bit 0 of *err and return false.  Writes of every block
// before the barrier are visible to every block after it (release / acquire at GPU scope,
// ordered within a block by __syncthreads).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, long long limit, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = ld_acquire_gpu(bar + 1);
    ok = 1;
    if (atom_add_acq_rel_gpu(bar, 1u) == nblocks - 1) {
      st_relaxed_gpu(bar, 0u);
      st_release_gpu(bar + 1, g + 1);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_gpu(bar + 1) == g) {
        if (clock64() - t0 > limit) {
          atomicOr(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

// One batch of ticks in one cooperative launch (gridDim.x blocks, all resident at once).
__global__ void __launch_bounds__(kBlock, 3)
    k_ticks(const TickItem* __restrict__ items, const TickHead* __restrict__ heads, int n_ticks, unsigned* bar,
            long long limit, int* err) {
  __shared__ TickItem it;
  for (int t = 0; t < n_ticks; ++t) {
    const TickHead h = heads[t];
    for (int b = blockIdx.x; b < h.blocks; b += gridDim.x) tick_block(items + h.first, h.count, b, it);
    if (t + 1 < n_ticks && !grid_barrier(bar, gridDim.x, limit, err)) return;
  }
}

}  // namespace xpbd

namespace {

constexpr int kMaxTicksPerRun = 256;

enum Phase {
  PH_ALPHA, PH_INIT, PH_PRED, PH_PASS, PH_CONTACT, PH_VEL, PH_LOSS, PH_LOSS_RED, PH_SEED,
  PH_ADJ_BEGIN, PH_REP_PRED, PH_REP_PASS, PH_REP_CONTACT, PH_VJP_CONTACT, PH_VJP_PASS,
  PH_COLL, PH_COLL_RED, PH_ADJ_PRED, PH_FG_RED, PH_NEXT_N, PH_FIN, PH_TOX, PH_TOV, PH_DONE
};

enum ReqState { RQ_QUEUED, RQ_RESIDENT, RQ_ALL_QUEUED, RQ_DONE };

struct Request {
  uint64_t ticket = 0;
  xpbd_request r{};
  xpbd_solver* h = nullptr;
  int V = 0, m = 0, N = 0, I = 0;
  bool contacts = false;
  size_t ws_bytes = 0;
  char* ws = nullptr;
  float* ck = nullptr;
  float4 *P = nullptr, *tape = nullptr, *tape_c = nullptr, *xbar = nullptr, *vbar = nullptr;
  float *lam = nullptr, *lam_tape = nullptr, *seed = nullptr, *cgrad = nullptr;
  uint8_t* cflags = nullptr;
  float2 *lamc = nullptr, *lamc_tape = nullptr, *lb = nullptr, *lbc = nullptr;
  double *acc = nullptr, *partials = nullptr;
  int pb = 1;   // partial blocks of a per-vertex pass
  // program cursor
  int phase = PH_ALPHA, n = 0, k = 0, col = 0, seg = 0, t = 0;
  int state = RQ_QUEUED;
  int last_tick = -1;   // tick (within the current batch) of the last queued pass
  cudaEvent_t ev = nullptr;
  bool ev_recorded = false;
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout of a request; with base == nullptr only sizes it.
size_t layout(Request& q, char* base) {
  const size_t V = q.V, m = std::max(q.m, 1), N = q.N, I = q.I;
  const size_t tpi = q.h->tape_per_iter();
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += align256(std::max<size_t>(bytes, 16));
    return p;
  };
  q.ck = (float*)take((N + 1) * V * 2 * sizeof(float4));
  q.P = (float4*)take(V * sizeof(float4));
  q.lam = (float*)take(m * sizeof(float));
  q.cflags = (uint8_t*)take(V);
  q.lamc = (float2*)take(V * sizeof(float2));
  q.tape = (float4*)take(I * tpi * sizeof(float4));
  q.lam_tape = (float*)take(I * m * sizeof(float));
  if (q.contacts) {
    q.tape_c = (float4*)take(I * V * sizeof(float4));
    q.lamc_tape = (float2*)take(I * V * sizeof(float2));
    q.lbc = (float2*)take(V * sizeof(float2));
    q.cgrad = (float*)take(V * 5 * sizeof(float));
  }
  q.xbar = (float4*)take(V * sizeof(float4));
  q.vbar = (float4*)take(V * sizeof(float4));
  q.lb = (float2*)take(m * sizeof(float2));
  q.acc = (double*)take(m * sizeof(double));
  q.pb = (int)((V + kBlock - 1) / kBlock);
  q.partials = (double*)take((size_t)std::max(q.pb, 1) * 5 * sizeof(double));
  q.seed = (float*)take(V * 3 * sizeof(float));
  return off;
}

void fill_proj(Request& q, TickItem& it, bool record) {
  const Seg& g = q.h->colors[q.col][q.seg];
  const size_t ro = (size_t)q.h->rec_off[g.type] + g.begin;
  it.kind = IK_PROJ;
  it.sub = g.type;
  it.n = g.count;
  it.rec = rec_ptr(q.h, g.type, g.begin);
  it.p[0] = q.P;
  if (record) {
    it.p[1] = q.k == 0 ? nullptr : q.lam_tape + (size_t)(q.k - 1) * q.m + ro;
    it.p[2] = q.lam_tape + (size_t)q.k * q.m + ro;
    it.p[3] = q.tape + (size_t)q.k * q.h->tape_per_iter() + tape_offset(q.h, g.type) + (size_t)g.begin * kVerts[g.type];
  } else {
    it.p[1] = q.k == 0 ? nullptr : q.lam + ro;
    it.p[2] = q.lam + ro;
    it.p[3] = nullptr;
  }
}

void fill_predict(Request& q, TickItem& it) {
  const xpbd_params& p = q.r.params;
  it.kind = IK_PREDICT;
  it.n = q.V;
  it.p[0] = (void*)ck_x(q.ck, q.V, q.n);
  it.p[1] = (void*)ck_v(q.ck, q.V, q.n);
  it.p[2] = q.P;
  it.p[3] = p.f_global ? (void*)(p.f_global + 3 * (size_t)q.n) : nullptr;
  it.p[4] = (void*)p.f_vertex;
  it.p[5] = q.cflags;
  it.f[0] = p.dt;
  it.f[1] = p.gravity[0];
  it.f[2] = p.gravity[1];
  it.f[3] = p.gravity[2];
}

void fill_contact(Request& q, TickItem& it, bool record) {
  it.kind = IK_CONTACT;
  it.n = q.V;
  it.p[0] = q.P;
  it.p[1] = q.cflags;
  if (record) {
    it.p[2] = q.k == 0 ? nullptr : q.lamc_tape + (size_t)(q.k - 1) * q.V;
    it.p[3] = q.lamc_tape + (size_t)q.k * q.V;
    it.p[4] = q.tape_c + (size_t)q.k * q.V;
  } else {
    it.p[2] = q.k == 0 ? nullptr : q.lamc;
    it.p[3] = q.lamc;
    it.p[4] = nullptr;
  }
}

// Next pass of a request's program; false once the program has ended.
bool emit(Request& q, TickItem& it) {
  std::memset(&it, 0, sizeof(it));
  xpbd_solver* h = q.h;
  const xpbd_params& p = q.r.params;
  it.col = make_collide(&p);
  const float inv_dt = 1.f / p.dt;
  const float inv_dt2 = 1.f / (p.dt * p.dt);
  for (;;) {
    switch (q.phase) {
      case PH_ALPHA:
        while (q.t < 4 && h->n_rec[q.t] == 0) ++q.t;
        if (q.t < 4) {
          it.kind = IK_SET_ALPHA;
          it.sub = q.t;
          it.n = h->n_rec[q.t];
          it.rec = h->d_rec[q.t];
          it.p[0] = h->d_perm + h->rec_off[q.t];
          it.p[1] = (void*)p.compliance;
          it.p[2] = h->d_err;
          it.f[0] = inv_dt2;
          ++q.t;
          return true;
        }
        q.phase = PH_INIT;
        continue;
      case PH_INIT:
        it.kind = IK_INIT_CKPT;
        it.n = q.V;
        it.p[0] = (void*)q.r.x0;
        it.p[1] = (void*)q.r.v0;
        it.p[2] = h->d_w;
        it.p[3] = q.ck;
        it.p[4] = (float4*)q.ck + q.V;
        q.n = 0;
        q.phase = q.N > 0 ? PH_PRED : PH_LOSS;
        return true;
      case PH_PRED:
      case PH_REP_PRED:
        fill_predict(q, it);
        q.k = 0;
        q.col = 0;
        q.seg = 0;
        q.phase = q.phase == PH_PRED ? PH_PASS : PH_REP_PASS;
        return true;
      case PH_PASS:
      case PH_REP_PASS: {
        while (q.col < h->K && q.seg >= (int)h->colors[q.col].size()) {
          ++q.col;
          q.seg = 0;
        }
        if (q.col < h->K) {
          fill_proj(q, it, q.phase == PH_REP_PASS);
          ++q.seg;
          return true;
        }
        q.phase = q.phase == PH_PASS ? PH_CONTACT : PH_REP_CONTACT;
        continue;
      }
      case PH_CONTACT:
      case PH_REP_CONTACT: {
        const bool rec = q.phase == PH_REP_CONTACT;
        bool emitted = false;
        if (q.contacts) {
          fill_contact(q, it, rec);
          emitted = true;
        }
        ++q.k;
        q.col = 0;
        q.seg = 0;
        if (q.k < q.I) {
          q.phase = rec ? PH_REP_PASS : PH_PASS;
        } else if (!rec) {
          q.phase = PH_VEL;
        } else {
          q.k = q.I - 1;
          q.phase = PH_VJP_CONTACT;
        }
        if (emitted) return true;
        continue;
      }
      case PH_VEL: {
        it.kind = IK_VELOCITY;
        it.n = q.V;
        float4* nx = (float4*)q.ck + (size_t)2 * q.V * (q.n + 1);
        it.p[0] = q.P;
        it.p[1] = (void*)ck_x(q.ck, q.V, q.n);
        it.p[2] = nx;
        it.p[3] = nx + q.V;
        it.p[4] = h->d_err;
        it.f[0] = inv_dt;
        ++q.n;
        q.phase = q.n < q.N ? PH_PRED : PH_LOSS;
        return true;
      }
      case PH_LOSS:
        it.kind = IK_LOSS;
        it.n = q.V;
        it.p[0] = (void*)ck_x(q.ck, q.V, q.N);
        it.p[1] = (void*)q.r.target;
        it.p[2] = q.seed;
        it.p[3] = q.partials;
        q.phase = q.r.loss_out ? PH_LOSS_RED : PH_SEED;
        return true;
      case PH_LOSS_RED:
        it.kind = IK_REDUCE;
        it.sub = 1;
        it.n = q.pb;
        it.p[0] = q.partials;
        it.p[1] = q.r.loss_out;
        q.phase = PH_SEED;
        return true;
      case PH_SEED:
        it.kind = IK_SEED_ADJ;
        it.n = q.V;
        it.p[0] = q.seed;
        it.p[1] = nullptr;
        it.p[2] = q.xbar;
        it.p[3] = q.vbar;
        q.n = q.N - 1;
        q.phase = q.N > 0 ? PH_ADJ_BEGIN : PH_FIN;
        q.t = 0;
        return true;
      case PH_ADJ_BEGIN:
        it.kind = IK_ADJ_BEGIN;
        it.n = q.V;
        it.p[0] = q.xbar;
        it.p[1] = q.vbar;
        it.f[0] = inv_dt;
        q.phase = PH_REP_PRED;
        return true;
      case PH_VJP_CONTACT: {
        bool emitted = false;
        if (q.contacts) {
          it.kind = IK_VJP_CONTACT;
          it.n = q.V;
          it.flags = q.k == q.I - 1 ? 1 : 0;
          it.p[0] = q.tape_c + (size_t)q.k * q.V;
          it.p[1] = q.cflags;
          it.p[2] = q.k == 0 ? nullptr : q.lamc_tape + (size_t)(q.k - 1) * q.V;
          it.p[3] = q.xbar;
          it.p[4] = q.lbc;
          it.p[5] = q.r.grads.d_collider ? q.cgrad : nullptr;
          emitted = true;
        }
        q.col = h->K - 1;
        q.seg = q.col >= 0 ? (int)h->colors[q.col].size() - 1 : -1;
        q.phase = PH_VJP_PASS;
        if (emitted) return true;
        continue;
      }
      case PH_VJP_PASS: {
        while (q.col >= 0 && q.seg < 0) {
          --q.col;
          if (q.col >= 0) q.seg = (int)h->colors[q.col].size() - 1;
        }
        if (q.col >= 0) {
          const Seg& g = h->colors[q.col][q.seg];
          const size_t ro = (size_t)h->rec_off[g.type] + g.begin;
          it.kind = IK_VJP;
          it.sub = g.type;
          it.n = g.count;
          it.flags = (q.k == q.I - 1 ? 1 : 0) | (q.k == 0 ? 2 : 0);
          it.rec = rec_ptr(h, g.type, g.begin);
          it.p[0] = q.tape + (size_t)q.k * h->tape_per_iter() + tape_offset(h, g.type) + (size_t)g.begin * kVerts[g.type];
          it.p[1] = q.k == 0 ? nullptr : q.lam_tape + (size_t)(q.k - 1) * q.m + ro;
          it.p[2] = q.xbar;
          it.p[3] = q.lb + ro;
          it.p[4] = q.acc + ro;
          --q.seg;
          return true;
        }
        --q.k;
        q.phase = q.k >= 0 ? PH_VJP_CONTACT : PH_COLL;
        continue;
      }
      case PH_COLL:
        if (q.contacts && q.r.grads.d_collider) {
          it.kind = IK_COLLIDER_PARTIALS;
          it.n = q.V;
          it.p[0] = q.cgrad;
          it.p[1] = q.cflags;
          it.p[2] = q.partials;
          q.phase = PH_COLL_RED;
          return true;
        }
        q.phase = PH_ADJ_PRED;
        continue;
      case PH_COLL_RED:
        it.kind = IK_REDUCE;
        it.sub = 5;
        it.n = q.pb;
        it.flags = 4;
        it.p[0] = q.partials;
        it.p[1] = q.r.grads.d_collider;
        q.phase = PH_ADJ_PRED;
        return true;
      case PH_ADJ_PRED:
        it.kind = IK_ADJ_PREDICT;
        it.n = q.V;
        it.p[0] = q.xbar;
        it.p[1] = q.vbar;
        it.p[2] = (void*)ck_x(q.ck, q.V, q.n);
        it.p[3] = nullptr;
        it.p[4] = q.r.grads.d_f_vertex;
        it.p[5] = q.r.grads.d_f_global ? q.partials : nullptr;
        it.f[0] = p.dt;
        q.phase = q.r.grads.d_f_global ? PH_FG_RED : PH_NEXT_N;
        return true;
      case PH_FG_RED:
        it.kind = IK_REDUCE;
        it.sub = 3;
        it.n = q.pb;
        it.p[0] = q.partials;
        it.p[1] = q.r.grads.d_f_global + 3 * (size_t)q.n;
        q.phase = PH_NEXT_N;
        return true;
      case PH_NEXT_N:
        --q.n;
        q.phase = q.n >= 0 ? PH_ADJ_BEGIN : PH_FIN;
        q.t = 0;
        continue;
      case PH_FIN:
        while (q.t < 4 && h->n_rec[q.t] == 0) ++q.t;
        if (q.t < 4 && q.r.grads.d_compliance) {
          it.kind = IK_FINALIZE;
          it.sub = q.t;
          it.n = h->n_rec[q.t];
          it.rec = h->d_rec[q.t];
          it.p[0] = h->d_perm + h->rec_off[q.t];
          it.p[1] = q.acc + h->rec_off[q.t];
          it.p[2] = q.r.grads.d_compliance;
          it.f[0] = inv_dt2;
          ++q.t;
          return true;
        }
        q.phase = PH_TOX;
        continue;
      case PH_TOX:
        q.phase = PH_TOV;
        if (q.r.grads.d_x0) {
          it.kind = IK_TO_DOUBLE;
          it.n = q.V;
          it.p[0] = q.xbar;
          it.p[1] = q.r.grads.d_x0;
          return true;
        }
        continue;
      case PH_TOV:
        q.phase = PH_DONE;
        if (q.r.grads.d_v0) {
          it.kind = IK_TO_DOUBLE;
          it.n = q.V;
          it.p[0] = q.vbar;
          it.p[1] = q.r.grads.d_v0;
          return true;
        }
        continue;
      default:
        return false;
    }
  }
}

size_t request_bytes(xpbd_solver* h, int steps, int iters, int flags) {
  Request q;
  q.h = h;
  q.V = h->V;
  q.m = h->m;
  q.N = steps;
  q.I = iters;
  q.contacts = (flags & 3) != 0;
  return layout(q, nullptr);
}

}  // namespace

struct xpbd_server_t {
  cudaStream_t stream = nullptr;
  size_t budget = 0, in_use = 0;
  int max_slots = 1;
  uint64_t next_ticket = 1;
  std::deque<Request*> queued;
  std::vector<Request*> resident;                       // admission order
  std::map<uint64_t, std::unique_ptr<Request>> all;
  // double-buffered dispatch tables: pass items, then the batch's tick heads
  size_t cap_items = 0;
  char* host_tab[2] = {nullptr, nullptr};
  char* dev_tab[2] = {nullptr, nullptr};
  cudaEvent_t tab_ev[2] = {nullptr, nullptr};
  bool tab_used[2] = {false, false};
  // the batch kernel's grid barrier (arrival count, generation) and error word; the error
  // word is copied to pinned memory after every batch and checked when its buffer is reused
  unsigned* d_bar = nullptr;
  int* d_err = nullptr;
  int* h_err = nullptr;   // [2], pinned
  int grid = 1;           // blocks of a batch launch (all resident at once)
  int run_count = 0;
  xpbd_server_stats stats{};
};

namespace {

void retire(xpbd_server_t* s, Request* q) {
  if (q->ws) cudaFreeAsync(q->ws, s->stream);
  q->ws = nullptr;
  s->in_use -= q->ws_bytes;
  if (q->ev) cudaEventDestroy(q->ev);
  q->ev = nullptr;
  q->state = RQ_DONE;
  s->stats.completed += 1;
}

// Retire resident requests whose last pass has finished on the GPU.
xpbd_status sweep(xpbd_server_t* s) {
  std::vector<Request*> keep;
  for (Request* q : s->resident) {
    if (q->state == RQ_ALL_QUEUED && q->ev_recorded) {
      cudaError_t e = cudaEventQuery(q->ev);
      if (e == cudaSuccess) {
        retire(s, q);
        continue;
      }
      if (e != cudaErrorNotReady) return fail(XPBD_ERR_CUDA, std::string("server event: ") + cudaGetErrorString(e));
    }
    keep.push_back(q);
  }
  s->resident.swap(keep);
  return XPBD_OK;
}

xpbd_status admit(xpbd_server_t* s) {
  while (!s->queued.empty() && (int)s->resident.size() < s->max_slots) {
    Request* q = s->queued.front();
    if (s->in_use + q->ws_bytes > s->budget) break;
    void* ws = nullptr;
    cudaError_t e = cudaMallocAsync(&ws, q->ws_bytes, s->stream);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      break;   // stays queued until memory frees up
    }
    if (e != cudaSuccess) return fail(XPBD_ERR_CUDA, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    q->ws = (char*)ws;
    layout(*q, q->ws);
    if (q->m > 0) CU_TRY(cudaMemsetAsync(q->acc, 0, sizeof(double) * (size_t)q->m, s->stream));
    if (q->r.grads.d_f_vertex)
      CU_TRY(cudaMemsetAsync(q->r.grads.d_f_vertex, 0, sizeof(double) * 3 * (size_t)q->V, s->stream));
    if (q->r.grads.d_collider) CU_TRY(cudaMemsetAsync(q->r.grads.d_collider, 0, sizeof(double) * 5, s->stream));
    if (q->r.grads.d_f_global && q->N > 0)
      CU_TRY(cudaMemsetAsync(q->r.grads.d_f_global, 0, sizeof(double) * 3 * (size_t)q->N, s->stream));
    CU_TRY(cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming));
    s->in_use += q->ws_bytes;
    q->state = RQ_RESIDENT;
    s->queued.pop_front();
    s->resident.push_back(q);
    s->stats.admitted += 1;
  }
  return XPBD_OK;
}

}  // namespace

extern "C" {

size_t xpbd_request_bytes(xpbd_handle h, int32_t steps, int32_t iters, int32_t collider_flags) {
  if (!h || steps < 0 || iters < 1) return 0;
  return request_bytes(h, steps, iters, collider_flags);
}

xpbd_status xpbd_server_create(size_t hbm_budget, int32_t max_slots, void* stream, xpbd_server* out) {
  g_err.clear();
  if (!out || max_slots < 1) return fail(XPBD_ERR_INVALID, "bad argument");
  *out = nullptr;
  std::unique_ptr<xpbd_server_t> s(new xpbd_server_t());
  s->stream = (cudaStream_t)stream;
  s->max_slots = max_slots;
  if (hbm_budget == 0) {
    size_t free_b = 0, total_b = 0;
    CU_TRY(cudaMemGetInfo(&free_b, &total_b));
    hbm_budget = (size_t)(0.9 * (double)free_b);
  }
  s->budget = hbm_budget;
  s->cap_items = (size_t)kMaxTicksPerRun * (size_t)max_slots;
  const size_t tab_bytes = s->cap_items * sizeof(TickItem) + kMaxTicksPerRun * sizeof(TickHead);
  for (int b = 0; b < 2; ++b) {
    CU_TRY(cudaHostAlloc((void**)&s->host_tab[b], tab_bytes, cudaHostAllocDefault));
    CU_TRY(cudaMalloc((void**)&s->dev_tab[b], tab_bytes));
    CU_TRY(cudaEventCreateWithFlags(&s->tab_ev[b], cudaEventDisableTiming));
  }
  CU_TRY(cudaMalloc((void**)&s->d_bar, 2 * sizeof(unsigned)));
  CU_TRY(cudaMemset(s->d_bar, 0, 2 * sizeof(unsigned)));
  CU_TRY(cudaMalloc((void**)&s->d_err, sizeof(int)));
  CU_TRY(cudaMemset(s->d_err, 0, sizeof(int)));
  CU_TRY(cudaHostAlloc((void**)&s->h_err, 2 * sizeof(int), cudaHostAllocDefault));
  s->h_err[0] = s->h_err[1] = 0;
  // a cooperative launch must fit on the GPU at once: the grid is the number of k_ticks
  // blocks every SM holds together
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  CU_TRY(cudaGetDevice(&dev));
  CU_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CU_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  CU_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ticks, kBlock, 0));
  if (!coop || per_sm < 1) return fail(XPBD_ERR_CUDA, "the device cannot run the cooperative serving kernel");
  s->grid = sms * per_sm;
  s->stats.budget = s->budget;
  *out = s.release();
  return XPBD_OK;
}

xpbd_status xpbd_server_destroy(xpbd_server s) {
  if (!s) return XPBD_OK;
  cudaStreamSynchronize(s->stream);
  for (auto& kv : s->all) {
    Request* q = kv.second.get();
    if (q->ws) cudaFreeAsync(q->ws, s->stream);
    if (q->ev) cudaEventDestroy(q->ev);
  }
  cudaStreamSynchronize(s->stream);
  for (int b = 0; b < 2; ++b) {
    if (s->host_tab[b]) cudaFreeHost(s->host_tab[b]);
    if (s->dev_tab[b]) cudaFree(s->dev_tab[b]);
    if (s->tab_ev[b]) cudaEventDestroy(s->tab_ev[b]);
  }
  if (s->d_bar) cudaFree(s->d_bar);
  if (s->d_err) cudaFree(s->d_err);
  if (s->h_err) cudaFreeHost(s->h_err);
  delete s;
  return XPBD_OK;
}

xpbd_status xpbd_server_submit(xpbd_server s, const xpbd_request* r, uint64_t* ticket) {
  g_err.clear();
  if (!s || !r || !ticket) return fail(XPBD_ERR_INVALID, "bad argument");
  xpbd_status st = check_params(r->handle, &r->params, r->steps, r->iters);
  if (st != XPBD_OK) return st;
  if (r->handle->V > 0 && (!r->x0 || !r->v0 || !r->target))
    return fail(XPBD_ERR_INVALID, "x0/v0/target NULL");
  if (r->params.f_vertex_steps || r->grads.d_f_vertex_steps)
    return fail(XPBD_ERR_INVALID, "per-step per-vertex forces are not served (use xpbd_forward/xpbd_adjoint)");
  if (r->handle->coupled || r->handle->nm > 0)
    return fail(XPBD_ERR_INVALID, "models with coupled tets or membranes are not served (use xpbd_forward/xpbd_adjoint)");
  std::unique_ptr<Request> q(new Request());
  q->r = *r;
  q->h = r->handle;
  q->V = q->h->V;
  q->m = q->h->m;
  q->N = r->steps;
  q->I = r->iters;
  q->contacts = (r->params.collider_flags & 3) != 0;
  q->ws_bytes = layout(*q, nullptr);
  if (q->ws_bytes > s->budget)
    return fail(XPBD_ERR_OOM, "request workspace (" + std::to_string(q->ws_bytes) + " bytes) exceeds the server budget");
  q->ticket = s->next_ticket++;
  *ticket = q->ticket;
  s->queued.push_back(q.get());
  s->all[q->ticket] = std::move(q);
  s->stats.submitted += 1;
  return XPBD_OK;
}

xpbd_status xpbd_server_run(xpbd_server s, int32_t max_ticks, int32_t* active_out) {
  g_err.clear();
  NvtxRange nvtx_range("xpbd_server_run");
  if (!s) return fail(XPBD_ERR_INVALID, "null server");
  xpbd_status st = sweep(s);
  if (st != XPBD_OK) return st;
  st = admit(s);
  if (st != XPBD_OK) return st;
  const int T = std::max(1, std::min<int>(max_ticks, kMaxTicksPerRun));
  const int b = s->run_count & 1;
  using clk = std::chrono::steady_clock;
  const auto t_wait = clk::now();
  if (s->tab_used[b]) {   // at most two batches in flight
    CU_TRY(cudaEventSynchronize(s->tab_ev[b]));
    s->stats.host_wait_s += std::chrono::duration<double>(clk::now() - t_wait).count();
    if (s->h_err[b]) {
      s->h_err[b] = 0;
      return fail(XPBD_ERR_TIMEOUT, "a grid barrier of the serving kernel gave up waiting");
    }
  }
  const auto t_build = clk::now();
  TickItem* tab = reinterpret_cast<TickItem*>(s->host_tab[b]);
  TickHead* heads = reinterpret_cast<TickHead*>(s->host_tab[b] + s->cap_items * sizeof(TickItem));
  int n_ticks = 0, max_blocks = 0;
  std::vector<Request*> finished;   // programs whose last pass is in this batch (or earlier)
  size_t used = 0;
  for (int t = 0; t < T; ++t) {
    const size_t first = used;
    int nb = 0;
    for (Request* q : s->resident) {
      if (q->state != RQ_RESIDENT) continue;
      TickItem& it = tab[used];
      if (emit(*q, it)) {
        it.block0 = nb;
        nb += item_blocks(it);
        ++used;
      } else {
        q->state = RQ_ALL_QUEUED;
        finished.push_back(q);
      }
    }
    if (used == first) break;
    heads[n_ticks++] = TickHead{(int)first, (int)(used - first), nb, 0};
    max_blocks = std::max(max_blocks, nb);
  }
  if (n_ticks > 0) {
    char* dev = s->dev_tab[b];
    const TickItem* d_items = reinterpret_cast<const TickItem*>(dev);
    const TickHead* d_heads = reinterpret_cast<const TickHead*>(dev + s->cap_items * sizeof(TickItem));
    CU_TRY(cudaMemcpyAsync(dev, tab, used * sizeof(TickItem), cudaMemcpyHostToDevice, s->stream));
    CU_TRY(cudaMemcpyAsync((void*)d_heads, heads, n_ticks * sizeof(TickHead), cudaMemcpyHostToDevice, s->stream));
    CU_TRY(cudaMemsetAsync(s->d_bar, 0, sizeof(unsigned), s->stream));   // arrival count
    int grid = std::min(s->grid, max_blocks);
    long long limit = 1ll << 31;   // ~1 s at 2 GHz, far beyond any tick
    int nt = n_ticks;
    void* args[] = {(void*)&d_items, (void*)&d_heads, (void*)&nt, (void*)&s->d_bar, (void*)&limit, (void*)&s->d_err};
    CU_TRY(cudaLaunchCooperativeKernel((const void*)k_ticks, dim3(grid), dim3(kBlock), args, 0, s->stream));
    s->stats.ticks += n_ticks;
    s->stats.items += (int64_t)used;
    s->stats.batches += 1;
  }
  for (Request* q : finished) {
    CU_TRY(cudaEventRecord(q->ev, s->stream));
    q->ev_recorded = true;
  }
  CU_TRY(cudaMemcpyAsync(&s->h_err[b], s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CU_TRY(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
  CU_TRY(cudaEventRecord(s->tab_ev[b], s->stream));
  s->tab_used[b] = true;
  s->run_count += 1;
  s->stats.host_build_s += std::chrono::duration<double>(clk::now() - t_build).count();
  if (active_out) *active_out = (int)s->resident.size();
  return XPBD_OK;
}

xpbd_status xpbd_server_poll(xpbd_server s, uint64_t ticket, int32_t* done) {
  g_err.clear();
  if (!s || !done) return fail(XPBD_ERR_INVALID, "bad argument");
  auto itr = s->all.find(ticket);
  if (itr == s->all.end()) return fail(XPBD_ERR_INVALID, "unknown or already completed ticket");
  Request* q = itr->second.get();
  *done = 0;
  if (q->state == RQ_ALL_QUEUED && q->ev_recorded) {
    cudaError_t e = cudaEventQuery(q->ev);
    if (e == cudaSuccess) {
      s->resident.erase(std::remove(s->resident.begin(), s->resident.end(), q), s->resident.end());
      retire(s, q);
    } else if (e != cudaErrorNotReady) {
      return fail(XPBD_ERR_CUDA, std::string("server event: ") + cudaGetErrorString(e));
    }
  }
  if (q->state == RQ_DONE) {
    *done = 1;
    s->all.erase(itr);
  }
  return XPBD_OK;
}

xpbd_status xpbd_server_get_stats(xpbd_server s, xpbd_server_stats* out) {
  if (!s || !out) return fail(XPBD_ERR_INVALID, "bad argument");
  *out = s->stats;
  out->pending = (int32_t)s->queued.size();
  out->active = (int32_t)s->resident.size();
  out->bytes_in_use = s->in_use;
  out->budget = s->budget;
  return XPBD_OK;
}

}  // extern "C"
