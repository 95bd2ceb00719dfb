// Phase kernels: several consecutive colors in one launch.
//
// A phase is a run of consecutive colors whose constraints, taken together, split into
// small connected components (constraints linked through shared vertices).  A component's
// vertices are touched by no constraint of another component within the phase, so one
// CTA can run all of the phase's colors on a group of components on its own: it stages the
// group's vertices (forward) or vertex adjoints (reverse) in shared memory, runs the
// colors in order (reverse order for the adjoint) with a barrier between colors, and
// writes the vertices back once.  Every constraint sees exactly the values the color-by-
// color launches would give it, in the same order, so results are those of the colored
// Gauss-Seidel sweep; only the vertex traffic changes: one load and one store per vertex
// per phase instead of one per color.
//
// The per-constraint streams (records, multipliers, tape, adjoint slots) are read once
// each.  A group's constraints are cut into chunks of kPhaseChunk constraints of one type
// and one color; a producer thread copies the streams of the next `stages` chunks into a ring of
// shared-memory stages with bulk asynchronous copies (cp.async.bulk, completion counted on
// one mbarrier per stage), so DRAM latency is hidden by copies in flight rather than by
// resident threads, and the element code reads its record, multiplier and tape from
// shared memory.  Each consumer thread updates one constraint of a chunk; a producer warp
// issues the copies, so no consumer carries that work on its critical path.
//
// Padding: every chunk's count and start are multiples of 4 so that each stream starts on
// a 16-byte boundary.  Padding constraints reference the group's dummy vertex (zero mass,
// zero position, never written back) with alpha~ = 0, so they never move anything.
//
// Waits are bounded: a stage that has not arrived after about a second (far beyond any
// copy) sets bit 4 of the error word; the consumers return at the next color end and the
// producer waits, again bounded, for the copies it has in flight.  xpbd_selftest_wait_timeout
// exercises this path with a launch whose producer issues nothing.
#include "xpbd_elems.cuh"

// Tape layout of a chunk: struct of arrays (vertex k of constraint i at k * count + i, so
// the staged reads of the reverse sweep are free of shared-memory bank conflicts) or one
// constraint's vertices side by side.
#ifndef XPBD_PHASE_TAPE_SOA
#define XPBD_PHASE_TAPE_SOA 1
#endif

namespace xpbd {

namespace {


__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of parity `parity` of barrier b to complete: false once
// `limit` SM clock cycles have passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, long long limit) {
  if (mbar_try_wait(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(b, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned);
// completion is counted in bytes on barrier b.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_u32(b))
      : "memory");
}

// Record bytes staged per constraint (a coupled pair stages its C_H and its C_D record).
__host__ __device__ constexpr unsigned rec_size(int t) {
  return t == SEG_DIST ? (unsigned)sizeof(DistRec)
                       : (t == SEG_BEND ? (unsigned)(sizeof(int4) + sizeof(BendTail))
                                        : (t == SEG_MEMB ? (unsigned)sizeof(MembRec)
                                                         : (t == kChunkPair ? 2u : 1u) * (unsigned)sizeof(TetRec)));
}
__host__ __device__ constexpr unsigned nverts(int t) { return t == SEG_DIST ? 2u : (t == SEG_MEMB ? 3u : 4u); }
// multiplier components (a membrane has three, a pair two) and adjoint slots (four for a
// membrane: three multiplier adjoints and four alpha~ adjoints in the float2 pairs' halves)
__host__ __device__ constexpr unsigned nlam(int t) { return t == SEG_MEMB ? 3u : (t == kChunkPair ? 2u : 1u); }
__host__ __device__ constexpr unsigned nadj(int t) { return t == SEG_MEMB ? 4u : (t == kChunkPair ? 2u : 1u); }
// The record array, slot block and tape range a chunk type uses (pairs: the C_H ones).
__host__ __device__ constexpr int home(int t) { return t == kChunkPair ? (int)SEG_TETH : t; }

template <int TM>
__device__ __forceinline__ constexpr bool has(int t) {
  return (TM >> t) & 1;
}

// The same sizes in a kernel of type set TM: the types it cannot meet fold away, so a
// cloth kernel computes its stage layout exactly as if membranes and pairs did not exist.
template <int TM>
struct TypeSet {
  static __device__ __forceinline__ bool memb(int t) { return has<TM>(SEG_MEMB) && t == SEG_MEMB; }
  static __device__ __forceinline__ bool pair(int t) { return has<TM>(kChunkPair) && t == kChunkPair; }
  static __device__ __forceinline__ unsigned rec(int t) {
    if (memb(t)) return (unsigned)sizeof(MembRec);
    if (pair(t)) return 2u * (unsigned)sizeof(TetRec);
    return t == SEG_DIST ? (unsigned)sizeof(DistRec)
                         : (t == SEG_BEND ? (unsigned)(sizeof(int4) + sizeof(BendTail)) : (unsigned)sizeof(TetRec));
  }
  static __device__ __forceinline__ unsigned nv(int t) { return memb(t) ? 3u : (t == SEG_DIST ? 2u : 4u); }
  static __device__ __forceinline__ unsigned nl(int t) { return memb(t) ? 3u : (pair(t) ? 2u : 1u); }
  static __device__ __forceinline__ unsigned na(int t) { return memb(t) ? 4u : (pair(t) ? 2u : 1u); }
  static __device__ __forceinline__ int home(int t) { return pair(t) ? (int)SEG_TETH : t; }
};

// Stage layout of a chunk of n constraints of type t: records (n R), multipliers in
// (4 n per component, component-major), and for the reverse sweep the tape (16 nv n) and
// (lambar, alphabar) pairs (8 n per slot).  Every part starts on a 16-byte boundary because
// n is a multiple of 4.  The last reverse iteration of a step folds alphabar into the float64
// accumulators with one atomic add per slot (fire and forget; a slot is added to once per
// launch, so the sums are deterministic).
template <int TM>
struct StageLayout {
  unsigned lam, tape, lb;
  __device__ StageLayout(int t, unsigned n) {
    using TS = TypeSet<TM>;
    lam = n * TS::rec(t);
    tape = lam + 4 * TS::nl(t) * n;
    lb = tape + 16 * TS::nv(t) * n;
  }
};

// Issued by the producer: copies of chunk c's streams into stage `st`, counted on barrier b.
template <bool REVERSE, int TM>
__device__ __forceinline__ void issue_chunk(const PhaseLaunch& a, const PhaseChunk& c, unsigned char* st,
                                            uint64_t* b, bool first, bool last) {
  using TS = TypeSet<TM>;
  const int t = c.type, h = TS::home(t);
  const unsigned n = (unsigned)c.count, R = TS::rec(t), nv = TS::nv(t), nl = TS::nl(t), na = TS::na(t);
  const StageLayout<TM> L(t, n);
  const size_t so = (size_t)a.slot_off[h] + c.begin;
  // component stride in the slot space: membrane blocks, or C_H -> C_D slots of a pair
  const size_t cs = TS::memb(t) ? (size_t)a.memb_stride
                                 : (TS::pair(t) ? (size_t)(a.slot_off[SEG_TETD] - a.slot_off[SEG_TETH]) : 0);
  unsigned total = n * R + (a.lam_in ? 4 * nl * n : 0);
  if (REVERSE) total += 16 * nv * n + (first ? 0 : 8 * na * n);
  mbar_expect_tx(b, total);
  if (n == 0) return;   // a padding entry of the chunk table: the arrival completes the stage
  if (TS::pair(t)) {
    const unsigned R1 = (unsigned)sizeof(TetRec);
    bulk_g2s(st, (const char*)a.prec[SEG_TETH] + (size_t)c.begin * R1, n * R1, b);
    bulk_g2s(st + n * R1, (const char*)a.prec[SEG_TETD] + (size_t)c.begin * R1, n * R1, b);
  } else if (t == SEG_BEND) {   // vertex indices, then the tails
    bulk_g2s(st, (const int4*)a.prec[SEG_BEND] + c.begin, n * (unsigned)sizeof(int4), b);
    bulk_g2s(st + n * sizeof(int4), a.prec_btail + c.begin, n * (unsigned)sizeof(BendTail), b);
  } else {
    bulk_g2s(st, (const char*)a.prec[h] + (size_t)c.begin * R, n * R, b);
  }
  if (a.lam_in)
    for (unsigned k = 0; k < nl; ++k) bulk_g2s(st + L.lam + 4 * n * k, a.lam_in + so + k * cs, 4 * n, b);
  if (REVERSE) {
    bulk_g2s(st + L.tape, a.tape + a.tape_off[h] + (size_t)c.begin * nv, 16 * nv * n, b);
    for (unsigned k = 0; k < na; ++k) {
      if (!first) bulk_g2s(st + L.lb + 8 * n * k, a.lb + so + k * cs, 8 * n, b);
    }
  }
}

// Bending record i of a stage holding n of them (vertex indices, then tails).
__device__ __forceinline__ BendRec staged_bend(const unsigned char* st, int n, int i) {
  const int4 v = reinterpret_cast<const int4*>(st)[i];
  const BendTail tl = reinterpret_cast<const BendTail*>(st + (size_t)n * sizeof(int4))[i];
  BendRec r;
  r.v[0] = v.x;
  r.v[1] = v.y;
  r.v[2] = v.z;
  r.v[3] = v.w;
  r.theta0 = tl.theta0;
  r.at = tl.at;
  r.pad0 = r.pad1 = 0.f;
  return r;
}

// Forward / replay update of constraint `tid` of chunk c from stage st.  `release` hands the
// stage back to the producer (every thread of the warp calls it once).  In the cloth kernel
// a thread first reads what its update needs from the stage into registers and releases
// before the arithmetic, so the next copy into the stage overlaps it.
template <bool RECORD, int TM, class Release>
__device__ __forceinline__ void fwd_chunk(const PhaseLaunch& a, const PhaseChunk& c, const unsigned char* st,
                                          float4* sv, Release&& release) {
  using TS = TypeSet<TM>;
  const int t = c.type, tid = threadIdx.x, n = c.count;
  const bool act = tid < n;
  const StageLayout<TM> L(t, (unsigned)n);
  const float* sl = reinterpret_cast<const float*>(st + L.lam);
  const size_t gi = (size_t)a.slot_off[TS::home(t)] + c.begin + tid;
#if XPBD_PHASE_TAPE_SOA
  float4* tp = RECORD ? a.tape + a.tape_off[TS::home(t)] + (size_t)c.begin * TS::nv(t) + tid : nullptr;
  const int ts = n;
#else
  float4* tp = RECORD ? a.tape + a.tape_off[TS::home(t)] + (size_t)(c.begin + tid) * TS::nv(t) : nullptr;
  const int ts = 1;
#endif
  // coupled pairs, membranes and tets read the stage as they go and release it at the end
  // (holding their larger records in registers across the release spills them)
  if (has<TM>(kChunkPair) && t == kChunkPair) {
    if (act) {
      const float atd = reinterpret_cast<const TetRec*>(st + (size_t)n * sizeof(TetRec))[tid].at;
      const float2 l2 = a.lam_in ? make_float2(sl[tid], sl[n + tid]) : make_float2(0.f, 0.f);
      const float2 lo2 = proj_pair_core<true>(reinterpret_cast<const TetRec*>(st)[tid], atd, sv, l2, tp, ts);
      __stcs(a.lam_out + gi, lo2.x);
      __stcs(a.lam_out + gi + (a.slot_off[SEG_TETD] - a.slot_off[SEG_TETH]), lo2.y);
    }
    release();
    return;
  }
  if (has<TM>(SEG_MEMB) && t == SEG_MEMB) {
    if (act) {
      float lm[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) lm[k] = a.lam_in ? sl[k * n + tid] : 0.f;
      proj_memb_core<true>(reinterpret_cast<const MembRec*>(st)[tid], sv, lm, tp, ts);
#pragma unroll
      for (int k = 0; k < 3; ++k) __stcs(a.lam_out + gi + (size_t)k * a.memb_stride, lm[k]);
    }
    release();
    return;
  }
  const float lam = act && a.lam_in ? sl[tid] : 0.f;
  float lo = lam;
  // the cloth kernel (distance and bending only) releases before its arithmetic; kernels
  // that also carry tets or membranes keep their registers for those and release after
  constexpr bool early = TM == 0x3;
  if (has<TM>(SEG_DIST) && t == SEG_DIST) {
    if constexpr (early) {
      DistRec r;
      if (act) r = reinterpret_cast<const DistRec*>(st)[tid];
      release();
      if (!act) return;
      lo = proj_dist_core<true>(r, sv, lam, tp, ts);
    } else {
      if (act) lo = proj_dist_core<true>(reinterpret_cast<const DistRec*>(st)[tid], sv, lam, tp, ts);
      release();
      if (!act) return;
    }
  } else if (has<TM>(SEG_BEND) && t == SEG_BEND) {
    if constexpr (early) {
      BendRec r;
      if (act) r = staged_bend(st, n, tid);
      release();
      if (!act) return;
      lo = proj_quad_core<1, true>(r, sv, lam, tp, ts);
    } else {
      if (act) lo = proj_quad_core<1, true>(staged_bend(st, n, tid), sv, lam, tp, ts);
      release();
      if (!act) return;
    }
  } else if ((has<TM>(SEG_TETH) && t == SEG_TETH) || (has<TM>(SEG_TETD) && t == SEG_TETD)) {
    if (act) {
      const TetRec* r = reinterpret_cast<const TetRec*>(st) + tid;
      lo = t == SEG_TETH ? proj_quad_core<2, true>(*r, sv, lam, tp, ts) : proj_quad_core<3, true>(*r, sv, lam, tp, ts);
    }
    release();
    if (!act) return;
  } else {
    release();
    return;
  }
  __stcs(a.lam_out + gi, lo);
}

// Reverse update of constraint `tid` of chunk c from stage st.  The reverse holds more
// state per update (tape, adjoint slots); it reads the stage as it goes and the caller
// releases the stage afterwards.
template <int TM>
__device__ __forceinline__ void vjp_chunk(const PhaseLaunch& a, const PhaseChunk& c, const unsigned char* st,
                                          float4* sx, bool first, bool last) {
  using TS = TypeSet<TM>;
  const int t = c.type, tid = threadIdx.x;
  if (tid >= c.count) return;
  const StageLayout<TM> L(t, (unsigned)c.count);
  const float lam = a.lam_in ? reinterpret_cast<const float*>(st + L.lam)[tid] : 0.f;
  float2 l = first ? make_float2(0.f, 0.f) : reinterpret_cast<const float2*>(st + L.lb)[tid];
  const size_t gi = (size_t)a.slot_off[TS::home(t)] + c.begin + tid;
#if XPBD_PHASE_TAPE_SOA
  const float4* tp = reinterpret_cast<const float4*>(st + L.tape) + tid;
  const int ts = c.count;
#else
  const float4* tp = reinterpret_cast<const float4*>(st + L.tape) + (size_t)tid * TS::nv(t);
  const int ts = 1;
#endif
  if (has<TM>(kChunkPair) && t == kChunkPair) {
    const int n = c.count;
    const float* sl = reinterpret_cast<const float*>(st + L.lam);
    const float2* slb = reinterpret_cast<const float2*>(st + L.lb);
    const float atd = reinterpret_cast<const TetRec*>(st + (size_t)n * sizeof(TetRec))[tid].at;
    const float2 l2 = a.lam_in ? make_float2(sl[tid], sl[n + tid]) : make_float2(0.f, 0.f);
    float2 lh = first ? make_float2(0.f, 0.f) : slb[tid];
    float2 ld = first ? make_float2(0.f, 0.f) : slb[n + tid];
    const float4 p[4] = {tp[0], tp[ts], tp[2 * ts], tp[3 * ts]};
    vjp_pair_core<true>(reinterpret_cast<const TetRec*>(st)[tid], atd, p, l2, lh, ld, sx);
    const size_t gd = gi + (a.slot_off[SEG_TETD] - a.slot_off[SEG_TETH]);
    if (last) {
      atomicAdd(a.acc + gi, (double)lh.y);
      atomicAdd(a.acc + gd, (double)ld.y);
    } else {
      a.lb[gi] = lh;
      a.lb[gd] = ld;
    }
    return;
  }
  if (has<TM>(SEG_MEMB) && t == SEG_MEMB) {
    const int n = c.count;
    const float* sl = reinterpret_cast<const float*>(st + L.lam);
    const float2* slb = reinterpret_cast<const float2*>(st + L.lb);
    float lm[3], lbv[3], ab[4];
#pragma unroll
    for (int k = 0; k < 3; ++k) lm[k] = a.lam_in ? sl[k * n + tid] : 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 q = first ? make_float2(0.f, 0.f) : slb[k * n + tid];
      if (k < 3) lbv[k] = q.x;
      ab[k] = q.y;
    }
    const float4 p[3] = {tp[0], tp[ts], tp[2 * ts]};
    vjp_memb_core<true>(reinterpret_cast<const MembRec*>(st)[tid], p, lm, lbv, ab, sx);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const size_t g = gi + (size_t)k * a.memb_stride;
      if (last)
        atomicAdd(a.acc + g, (double)ab[k]);
      else
        a.lb[g] = make_float2(k < 3 ? lbv[k] : 0.f, ab[k]);
    }
    return;
  }
  if (has<TM>(SEG_DIST) && t == SEG_DIST) {
    l = vjp_dist_core<true>(reinterpret_cast<const DistRec*>(st)[tid], tp[0], tp[ts], lam, l, sx);
  } else {
    const float4 p[4] = {tp[0], tp[ts], tp[2 * ts], tp[3 * ts]};
    if (has<TM>(SEG_BEND) && t == SEG_BEND)
      l = vjp_quad_core<1, true>(staged_bend(st, c.count, tid), p, lam, l, sx);
    else if (has<TM>(SEG_TETH) && t == SEG_TETH)
      l = vjp_quad_core<2, true>(reinterpret_cast<const TetRec*>(st)[tid], p, lam, l, sx);
    else if (has<TM>(SEG_TETD) && t == SEG_TETD)
      l = vjp_quad_core<3, true>(reinterpret_cast<const TetRec*>(st)[tid], p, lam, l, sx);
  }
  if (last)
    atomicAdd(a.acc + gi, (double)l.y);
  else
    a.lb[gi] = l;
}

}  // namespace

// Resident CTAs per SM each kernel is compiled for; the stage ring is sized so that the
// shared memory of that many CTAs fits in one SM.
#ifndef XPBD_PHASE_FWD_MIN_BLOCKS
#define XPBD_PHASE_FWD_MIN_BLOCKS 4
#endif
#ifndef XPBD_PHASE_VJP_MIN_BLOCKS
#define XPBD_PHASE_VJP_MIN_BLOCKS 2
#endif

// Gathers the group's vertices (or vertex adjoints) into shared memory, 6 independent
// loads in flight per thread, and (svl not NULL) keeps their global indices there for the
// write-back.  The list is the group's padded one (`stride` entries, -1 for the padding
// between row halves and past the group's vertices), so this needs nothing from the
// group's record.
__device__ __forceinline__ void gather_vertices(const float4* __restrict__ P, const int* __restrict__ vlist,
                                                int stride, float4* sv, int* svl) {
  constexpr int U = 6;
  for (int v0 = threadIdx.x; v0 < stride; v0 += U * blockDim.x) {
    int idx[U];
    float4 val[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int v = v0 + u * (int)blockDim.x;
      idx[u] = v < stride ? __ldg(vlist + v) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (idx[u] >= 0) val[u] = P[idx[u]];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int v = v0 + u * (int)blockDim.x;
      if (idx[u] >= 0) sv[v] = val[u];
      if (svl && v < stride) svl[v] = idx[u];
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// Barrier among the consumer warps only (named barrier 1; the producer warp is not part).
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(kPhaseBlock) : "memory");
}

// MODE 0 forward, 1 replay (forward + tape), 2 reverse.  One CTA per group: kPhaseBlock
// consumer threads (one constraint of a chunk each) and one producer warp whose first lane
// keeps the stage ring filled.  A stage is refilled once all consumer warps have released
// it (`empty`, one arrival per warp); the consumers synchronise with each other only where
// a color ends.
template <int MODE, int TM>
__global__ void __launch_bounds__(kPhaseThreads, MODE == 2 ? XPBD_PHASE_VJP_MIN_BLOCKS : XPBD_PHASE_FWD_MIN_BLOCKS)
    k_phase(PhaseLaunch a, bool first, bool last) {
  constexpr bool REV = MODE == 2;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[kPhaseMaxStages], empty[kPhaseMaxStages];
  __shared__ int abort_run;
  float4* sv = reinterpret_cast<float4*>(smem);
  // the reverse keeps the vertex indices in shared memory for its write-back; the forward
  // re-reads them (still in L2) and spends that shared memory on another stage
  int* svl = REV ? reinterpret_cast<int*>(smem + (size_t)(a.vstride + 1) * sizeof(float4)) : nullptr;
  PhaseChunk* sch = reinterpret_cast<PhaseChunk*>(smem + a.vert_bytes);
  unsigned char* stage = smem + a.vert_bytes + a.chunk_bytes;
  // the chunk table (in execution order) and vertex list of this CTA, and its record, are
  // read at once: none of the three addresses depends on another load
  const PhaseChunk* ch = (REV ? a.chunks_rev : a.chunks) + (size_t)blockIdx.x * a.cstride;
  const int S = a.stages;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kPhaseBlock / 32);
    }
    abort_run = 0;
    mbar_fence_init();
  }
  __syncthreads();
  // lanes of the producer warp start the first stages (one chunk each, empty padding chunks
  // only arrive); everyone else copies the table to shared memory and gathers the vertices
  const int lane_p = (int)threadIdx.x - kPhaseBlock;
  if (lane_p >= 0 && lane_p < S && lane_p < a.cstride && !a.no_issue)
    issue_chunk<REV, TM>(a, ch[lane_p], stage + (size_t)lane_p * a.slot_bytes, &full[lane_p], first, last);
  for (int i = threadIdx.x; i < a.cstride; i += blockDim.x) sch[i] = ch[i];
  const PhaseGroup G = a.groups[blockIdx.x];
  gather_vertices(a.P, a.pverts + (size_t)blockIdx.x * a.vstride, a.vstride, sv, svl);
  if (threadIdx.x == 0) sv[G.vert_count] = make_float4(0.f, 0.f, 0.f, 0.f);   // the dummy vertex
  const int nch = G.chunk_count;
  __syncthreads();
  if (threadIdx.x >= kPhaseBlock) {   // producer warp
    if (threadIdx.x == kPhaseBlock && !a.no_issue) {
      // stages [0, S) were issued above (chunks past nch are empty); refill from chunk S on
      int issued = S < a.cstride ? S : a.cstride;
      for (; issued < nch; ++issued) {
        // stage issued mod S, whose previous use was phase (issued / S - 1) mod 2; the
        // quotient by multiplication (a division by the runtime S costs ~20 instructions)
        const unsigned q = __umulhi((unsigned)issued, a.stage_magic);
        const int s = issued - (int)q * S;
        if (!mbar_wait(&empty[s], (q - 1u) & 1u, a.wait_cycles)) break;   // the consumers stopped
        issue_chunk<REV, TM>(a, sch[issued], stage + (size_t)s * a.slot_bytes, &full[s], first, last);
      }
      // Whether it issued every chunk or gave up, the CTA must not end while a copy into its
      // shared memory is in flight (the consumers may have stopped early): wait for the last
      // stages issued.  A drain that runs out latches bit 5: the context may be unusable.
      for (int j = issued > S ? issued - S : 0; j < issued; ++j)
        if (!mbar_wait(&full[j % S], (unsigned)(j / S) & 1u, a.wait_cycles)) {
          atomicOr(a.err, 16);
          break;
        }
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < nch; ++k) {
    // stage s = k mod S and par = (k / S) mod 2, the phase of stage s that chunk k fills
    // (the quotient by multiplication, as in the producer)
    const unsigned q = __umulhi((unsigned)k, a.stage_magic);
    const int s = k - (int)q * S;
    const unsigned par = q & 1u;
    const unsigned char* st = stage + (size_t)s * a.slot_bytes;
    const PhaseChunk c = sch[k];
    // a warp hands the stage back once all its threads have read what they need from it
    uint64_t* const emp = &empty[s];
    auto release = [emp, lane]() {
      __syncwarp();
      if (lane == 0) mbar_arrive(emp);
    };
    if (mbar_wait(&full[s], par, a.wait_cycles)) {
      if (REV) {
        vjp_chunk<TM>(a, c, st, sv, first, last);
        release();
      } else {
        fwd_chunk<MODE == 1, TM>(a, c, st, sv, release);
      }
    } else {
      abort_run = 1;
      release();
    }
    if ((c.flags & (REV ? kChunkColorFirst : kChunkColorLast)) || k + 1 == nch) {
      consumer_sync();
      if (abort_run) {
        if (threadIdx.x == 0) atomicOr(a.err, 4);
        return;
      }
    }
  }
  const int* vlist = a.pverts + (size_t)blockIdx.x * a.vstride;
  for (int v = threadIdx.x; v < G.vert_count; v += kPhaseBlock) {
    const int gv = REV ? svl[v] : __ldg(vlist + v);
    if (gv >= 0) a.P[gv] = sv[v];
  }
}

namespace {

// Type sets with their own kernels: cloth (distance + bending), solids (the two tet
// constraints, with or without distance constraints), membrane cloth (membranes with
// bending and distance constraints) and everything.
// Coupled tets (pair chunks, bit kChunkPair) have a kernel of their own (with distance
// constraints); they never share a model with one-at-a-time tets.
constexpr int kMaskCloth = 0x3, kMaskSolid = 0xD, kMaskMemb = 0x13, kMaskPair = 0x21, kMaskAll = 0x3F;

int kernel_mask(int type_mask) {
  if ((type_mask & ~kMaskCloth) == 0) return kMaskCloth;
  if ((type_mask & ~kMaskSolid) == 0) return kMaskSolid;
  if ((type_mask & ~kMaskMemb) == 0) return kMaskMemb;
  if ((type_mask & ~kMaskPair) == 0) return kMaskPair;
  return kMaskAll;
}

unsigned elem_stage_bytes(int t, bool rev) {
  return rec_size(t) + 4 * nlam(t) + (rev ? 16 * nverts(t) + 8 * nadj(t) : 0);
}

struct Plan {
  int vert_bytes = 0, chunk_bytes = 0, slot_bytes = 0, stages = 0;
  size_t smem() const { return (size_t)vert_bytes + chunk_bytes + (size_t)stages * slot_bytes; }
};

// Shared memory of a launch: the largest group's vertices (+ the dummy), its chunk table and
// as many stages (2..kPhaseMaxStages) as fit in the shared memory of 3 (forward) or 2
// (reverse) resident CTAs per SM.
Plan stage_plan(const PhaseShape& sh, bool rev) {
  Plan p;
  p.vert_bytes = ((sh.max_verts + 1) * (rev ? 20 : 16) + 127) / 128 * 128;
  p.chunk_bytes = (std::max(sh.max_chunks, 1) * (int)sizeof(PhaseChunk) + 127) / 128 * 128;
  unsigned e = 0;
  for (int t = 0; t <= kChunkPair; ++t)
    if ((sh.type_mask >> t) & 1) e = std::max(e, elem_stage_bytes(t, rev));
  // a stage holds the phase's largest chunk: phases of small groups (small models) get
  // stages of their chunk size and so more of them in flight
  const int csz = sh.max_chunk_size > 0 ? (sh.max_chunk_size + 3) / 4 * 4 : kPhaseChunk;
  p.slot_bytes = (int)(e * (unsigned)std::min(csz, kPhaseChunk));
  if (p.slot_bytes == 0) return p;
  const int per_sm = 228 * 1024, ctas = rev ? XPBD_PHASE_VJP_MIN_BLOCKS : XPBD_PHASE_FWD_MIN_BLOCKS;
  const int fixed = p.vert_bytes + p.chunk_bytes;
  const int budget = per_sm / ctas - 1024 - 256;   // per-CTA reservation, static shared memory
  int S = (budget - fixed) / p.slot_bytes;
  S = std::min(std::max(S, 2), kPhaseMaxStages);
  while (S >= 2 && fixed + S * p.slot_bytes > kPhaseSmemLimit) --S;
  p.stages = S >= 2 ? S : 0;
  return p;
}

template <int MODE, int TM>
cudaError_t setup_one() {
  cudaError_t e = cudaFuncSetAttribute(k_phase<MODE, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPhaseSmemLimit);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_phase<MODE, TM>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}

template <int TM>
cudaError_t setup_mask() {
  cudaError_t e = setup_one<0, TM>();
  if (e == cudaSuccess) e = setup_one<1, TM>();
  if (e == cudaSuccess) e = setup_one<2, TM>();
  return e;
}

template <int MODE>
void launch_mode(PhaseLaunch a, const PhaseShape& sh, bool first, bool last, cudaStream_t s) {
  if (sh.n_groups <= 0) return;
  const Plan p = stage_plan(sh, MODE == 2);
  a.vert_bytes = p.vert_bytes;
  a.chunk_bytes = p.chunk_bytes;
  a.slot_bytes = p.slot_bytes;
  a.stages = p.stages;
  a.stage_magic = p.stages > 0 ? (unsigned)((0x100000000ull + (unsigned)p.stages - 1) / (unsigned)p.stages) : 0u;
  const size_t smem = p.smem();
  switch (kernel_mask(sh.type_mask)) {
    case kMaskCloth: k_phase<MODE, kMaskCloth><<<sh.n_groups, kPhaseThreads, smem, s>>>(a, first, last); break;
    case kMaskSolid: k_phase<MODE, kMaskSolid><<<sh.n_groups, kPhaseThreads, smem, s>>>(a, first, last); break;
    case kMaskMemb: k_phase<MODE, kMaskMemb><<<sh.n_groups, kPhaseThreads, smem, s>>>(a, first, last); break;
    case kMaskPair: k_phase<MODE, kMaskPair><<<sh.n_groups, kPhaseThreads, smem, s>>>(a, first, last); break;
    default: k_phase<MODE, kMaskAll><<<sh.n_groups, kPhaseThreads, smem, s>>>(a, first, last);
  }
}

}  // namespace

cudaError_t phase_kernel_setup() {
  cudaError_t e = setup_mask<kMaskCloth>();
  if (e == cudaSuccess) e = setup_mask<kMaskSolid>();
  if (e == cudaSuccess) e = setup_mask<kMaskMemb>();
  if (e == cudaSuccess) e = setup_mask<kMaskPair>();
  if (e == cudaSuccess) e = setup_mask<kMaskAll>();
  return e;
}

size_t phase_smem_bytes(const PhaseShape& sh, bool reverse) {
  const Plan p = stage_plan(sh, reverse);
  return p.stages < 2 ? 0 : p.smem();
}

void launch_phase_fwd(PhaseLaunch a, const PhaseShape& sh, bool record, cudaStream_t s) {
  if (record)
    launch_mode<1>(a, sh, false, false, s);
  else
    launch_mode<0>(a, sh, false, false, s);
}

void launch_phase_vjp(PhaseLaunch a, const PhaseShape& sh, bool first, bool last, cudaStream_t s) {
  launch_mode<2>(a, sh, first, last, s);
}

}  // namespace xpbd
