// Host runtime of the C ABI declared in include/diffxpbd.h.
//
// xpbd_create validates the model, derives rest data (spring lengths, hinge angles,
// Dm^-1, tet volumes) from the rest positions, regroups every color by constraint type and
// first vertex and uploads the records.  xpbd_forward / xpbd_adjoint queue the per-color
// kernels of xpbd_kernels.cu on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/diffxpbd.h"
#include "xpbd_kernels.cuh"
#include "xpbd_multigrid.cuh"
#include "xpbd_solver.cuh"

using namespace xpbd;

namespace {

// Forward workspace (no tapes).
xpbd_status ensure_forward_ws(xpbd_solver* h) {
  CU_TRY(h->P.ensure(sizeof(float4) * (size_t)h->V));
  CU_TRY(h->lam.ensure(sizeof(float) * h->slots));
  CU_TRY(h->cflags.ensure((size_t)std::max(h->V, 1)));
  CU_TRY(h->lamc.ensure(sizeof(float2) * (size_t)std::max(h->V, 1)));
  return XPBD_OK;
}

xpbd_status ensure_adjoint_ws(xpbd_solver* h, int iters, bool contacts) {
  xpbd_status st = ensure_forward_ws(h);
  if (st != XPBD_OK) return st;
  size_t V = (size_t)h->V, m = h->slots;
  CU_TRY(h->tape.ensure(sizeof(float4) * std::max(h->tape_slots, (size_t)1) * iters));
  CU_TRY(h->lam_tape.ensure(sizeof(float) * m * iters));
  if (contacts) {
    CU_TRY(h->tape_c.ensure(sizeof(float4) * V * iters));
    CU_TRY(h->lamc_tape.ensure(sizeof(float2) * V * iters));
    CU_TRY(h->lbc.ensure(sizeof(float2) * V));
    CU_TRY(h->cgrad.ensure(sizeof(float) * 5 * V));
  }
  CU_TRY(h->xbar.ensure(sizeof(float4) * V));
  CU_TRY(h->vbar.ensure(sizeof(float4) * V));
  CU_TRY(h->lb.ensure(sizeof(float2) * m));
  CU_TRY(h->acc.ensure(sizeof(double) * m));
  CU_TRY(h->partials.ensure(sizeof(double) * 5 * (size_t)partial_blocks(std::max(h->V, 1))));
  return XPBD_OK;
}

PhaseLaunch phase_args(const xpbd_solver* h, const xpbd_solver::PhaseHost& ph);
xpbd_status forward_step(xpbd_solver* h, const xpbd_params* p, int n, int32_t iters, const float4* ckx_n,
                         const float4* ckv_n, float4* nx, cudaStream_t s);

// alpha~ into the records a call will use: the phase-ordered copy when the phase plan runs
// the sweep (`phase`), else the per-color records.
xpbd_status set_alpha(xpbd_solver* h, const xpbd_params* p, cudaStream_t s, bool phase = false) {
  float inv_dt2 = 1.f / (p->dt * p->dt);
  void* const* rec = phase ? h->d_prec : h->d_rec;
  const int* perm = phase ? h->d_pperm : h->d_perm;
  const int* off = phase ? h->pslot_off : h->rec_off;
  const int* cnt = phase ? h->n_prec : h->n_rec;
  for (int t = 0; t < 4; ++t)
    launch(h, XPBD_K_OTHER, cnt[t], s, [&] {
      if (phase && t == SEG_BEND)
        launch_set_alpha_btail(h->d_prec_btail, perm + off[t], cnt[t], p->compliance, inv_dt2, h->d_err, s);
      else
        launch_set_alpha((SegType)t, rec[t], perm + off[t], cnt[t], p->compliance, inv_dt2, h->d_err, s);
    });
  const int nmr = phase ? h->n_prec[SEG_MEMB] : h->nm;
  launch(h, XPBD_K_OTHER, nmr, s, [&] {
    launch_memb_set_alpha(phase ? (MembRec*)h->d_prec[SEG_MEMB] : h->d_mrec,
                          phase ? h->d_pperm + h->pslot_off[SEG_MEMB] : h->d_mperm, nmr, p->memb_stiffness, inv_dt2,
                          h->d_err, s);
  });
  LAUNCH_CHECK();
  return XPBD_OK;
}

// Forward update of one color segment; `tape_k` (replay) receives the pre-projection
// positions.  With coupled tets a C_H segment updates its tets' C_D constraints too.
void project_segment(xpbd_solver* h, const Seg& g, float4* P, const float* lam_in, float* lam_out,
                     float4* tape_k, cudaStream_t s) {
  const bool record = tape_k != nullptr;
  if (g.type == SEG_MEMB) {
    const size_t mo = (size_t)h->mslot + g.begin;
    float4* tp = tape_k ? tape_k + h->mtape + 3 * (size_t)g.begin : nullptr;
    launch(h, record ? XPBD_K_REPLAY_MEMB : XPBD_K_FWD_MEMB, g.count, s, [&] {
      launch_project_memb(h->d_mrec + g.begin, g.count, P, lam_in ? lam_in + mo : nullptr, lam_out + mo, h->nm, tp, s);
    });
    return;
  }
  const size_t ro = (size_t)h->rec_off[g.type] + g.begin;
  float4* tp = tape_k ? tape_k + tape_offset(h, g.type) + (size_t)g.begin * kVerts[g.type] : nullptr;
  if (h->coupled && g.type == SEG_TETH) {
    // per tet: C_H record 64 + C_D alpha~ 4 + two multipliers r/w 16 + four vertices r/w 128
    // (+ 64 tape)
    launch(h, record ? XPBD_K_REPLAY_TETH : XPBD_K_FWD_TETH, 2 * (int64_t)g.count, s, [&] {
      launch_project_tet_pair((const TetRec*)rec_ptr(h, SEG_TETH, g.begin),
                              (const TetRec*)rec_ptr(h, SEG_TETD, g.begin), g.count, P,
                              lam_in ? lam_in + ro : nullptr, lam_out + ro, h->rec_off[3] - h->rec_off[2], tp, s);
    }, (double)g.count * (record ? 276 : 212));
    return;
  }
  launch(h, (record ? XPBD_K_REPLAY_DIST : XPBD_K_FWD_DIST) + (int)g.type, g.count, s, [&] {
    launch_project(g.type, rec_ptr(h, g.type, g.begin), g.count, P, lam_in ? lam_in + ro : nullptr,
                   lam_out + ro, tp, s);
  });
}

// Reverse of project_segment from iteration k's tape and multipliers before it.
void vjp_segment(xpbd_solver* h, const Seg& g, const float4* tape_k, const float* lam_pre, float4* xbar,
                 bool first, bool last, cudaStream_t s) {
  if (g.type == SEG_MEMB) {
    const size_t mo = (size_t)h->mslot + g.begin;
    launch(h, XPBD_K_VJP_MEMB, g.count, s, [&] {
      launch_vjp_memb(h->d_mrec + g.begin, g.count, tape_k + h->mtape + 3 * (size_t)g.begin,
                      lam_pre ? lam_pre + mo : nullptr, h->nm, xbar, h->lb.as<float2>() + mo,
                      h->acc.as<double>() + mo, first, last, s);
    });
    return;
  }
  const size_t ro = (size_t)h->rec_off[g.type] + g.begin;
  const float4* tp = tape_k + tape_offset(h, g.type) + (size_t)g.begin * kVerts[g.type];
  if (h->coupled && g.type == SEG_TETH) {
    // per tet: record 64 + 4, tape 64, multipliers 8, vertex adjoints r/w 128, two
    // (lambar, alphabar) r/w 32
    launch(h, XPBD_K_VJP_TETH, 2 * (int64_t)g.count, s, [&] {
      launch_vjp_tet_pair((const TetRec*)rec_ptr(h, SEG_TETH, g.begin), (const TetRec*)rec_ptr(h, SEG_TETD, g.begin),
                          g.count, tp, lam_pre ? lam_pre + ro : nullptr, h->rec_off[3] - h->rec_off[2], xbar,
                          h->lb.as<float2>() + ro, h->acc.as<double>() + ro, first, last, s);
    }, (double)g.count * 300);
    return;
  }
  launch(h, XPBD_K_VJP_DIST + (int)g.type, g.count, s, [&] {
    launch_vjp(g.type, rec_ptr(h, g.type, g.begin), g.count, tp, lam_pre ? lam_pre + ro : nullptr, xbar,
               h->lb.as<float2>() + ro, h->acc.as<double>() + ro, first, last, s);
  });
}

// One step: prediction from checkpoint n, `iters` colored iterations, collision passes.
// With `record`, the multipliers of iteration k go to lam_tape[k] and the pre-projection
// positions to tape[k] (replay for the reverse sweep); otherwise lambda is updated in place.
xpbd_status run_step(xpbd_solver* h, const xpbd_params* p, int n, int iters, const float4* ckx_n,
                     const float4* ckv_n, bool record, cudaStream_t s, bool per_color = false) {
  const bool phases = h->use_phases && !per_color;
  Collide c = make_collide(p);
  float4* P = h->P.as<float4>();
  uint8_t* cf = h->cflags.as<uint8_t>();
  launch(h, XPBD_K_PREDICT, h->V, s, [&] {
    launch_predict(ckx_n, ckv_n, P, p->f_global ? p->f_global + 3 * (size_t)n : nullptr, p->f_vertex,
                   p->f_vertex_steps ? p->f_vertex_steps + 3 * (size_t)h->V * n : nullptr,
                   p->dt, p->gravity[0], p->gravity[1], p->gravity[2], c, cf, h->V, s);
  });
  LAUNCH_CHECK();
  const size_t tpi = h->tape_slots;
  for (int k = 0; k < iters; ++k) {
    float* lam_in;
    float* lam_out;
    float4* tape_k = nullptr;
    if (record) {
      lam_in = k == 0 ? nullptr : h->lam_tape.as<float>() + (size_t)(k - 1) * h->slots;
      lam_out = h->lam_tape.as<float>() + (size_t)k * h->slots;
      tape_k = h->tape.as<float4>() + (size_t)k * tpi;
    } else {
      lam_in = k == 0 ? nullptr : h->lam.as<float>();
      lam_out = h->lam.as<float>();
    }
    if (phases) {
      for (const auto& ph : h->phases) {
        PhaseLaunch a = phase_args(h, ph);
        a.P = P;
        a.lam_in = lam_in;
        a.lam_out = lam_out;
        a.tape = tape_k;
        launch(h, record ? XPBD_K_REPLAY_PHASE : XPBD_K_FWD_PHASE, ph.units, s,
               [&] { launch_phase_fwd(a, ph.shape(), record, s); },
               record ? ph.bytes_replay : ph.bytes_fwd);
      }
    } else {
      for (int col = 0; col < h->K; ++col)
        for (const Seg& g : h->colors[col]) project_segment(h, g, P, lam_in, lam_out, tape_k, s);
    }
    if (c.flags) {
      float2* li;
      float2* lo;
      float4* tc = nullptr;
      if (record) {
        li = k == 0 ? nullptr : h->lamc_tape.as<float2>() + (size_t)(k - 1) * h->V;
        lo = h->lamc_tape.as<float2>() + (size_t)k * h->V;
        tc = h->tape_c.as<float4>() + (size_t)k * h->V;
      } else {
        li = k == 0 ? nullptr : h->lamc.as<float2>();
        lo = h->lamc.as<float2>();
      }
      launch(h, record ? XPBD_K_REPLAY_CONTACT : XPBD_K_FWD_CONTACT, h->V, s,
             [&] { launch_contact(P, cf, h->V, li, lo, tc, c, s); });
    }
    LAUNCH_CHECK();
  }
  return XPBD_OK;
}


double rest_angle(const double* x0, const double* x1, const double* x2, const double* x3) {
  double e[3], a[3], b[3];
  for (int c = 0; c < 3; ++c) {
    e[c] = x1[c] - x0[c];
    a[c] = x2[c] - x0[c];
    b[c] = x3[c] - x0[c];
  }
  auto cr = [](const double* u, const double* v, double* o) {
    o[0] = u[1] * v[2] - u[2] * v[1];
    o[1] = u[2] * v[0] - u[0] * v[2];
    o[2] = u[0] * v[1] - u[1] * v[0];
  };
  double nA[3], nB[3], nn[3];
  cr(e, a, nA);
  cr(b, e, nB);
  cr(nA, nB, nn);
  double le = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
  double sn = (nn[0] * e[0] + nn[1] * e[1] + nn[2] * e[2]) / le;
  double cs = nA[0] * nB[0] + nA[1] * nB[1] + nA[2] * nB[2];
  return std::atan2(sn, cs);
}

}  // namespace


// ---------------------------------------------------------------- allocation-free forward
// Working state of xpbd_forward_static in one file-scope device array, so that entry point
// needs no device allocation: predicted positions, multipliers, contact multipliers and
// contact flags of meshes up to XPBD_STATIC_MAX_VERTICES / XPBD_STATIC_MAX_CONSTRAINTS.
// Every GPU that loads this library holds the array (about 3.1 MiB) until the process exits.
namespace {
constexpr size_t kStaticPosBytes = sizeof(float4) * XPBD_STATIC_MAX_VERTICES;      // 1 MiB
constexpr size_t kStaticLamBytes = sizeof(float) * XPBD_STATIC_MAX_CONSTRAINTS;    // 1.5 MiB
constexpr size_t kStaticLamcBytes = sizeof(float2) * XPBD_STATIC_MAX_VERTICES;     // 512 KiB
constexpr size_t kStaticFlagBytes = XPBD_STATIC_MAX_VERTICES;                      // 64 KiB
constexpr size_t kStaticBytes = kStaticPosBytes + kStaticLamBytes + kStaticLamcBytes + kStaticFlagBytes;
static_assert(kStaticPosBytes % 256 == 0 && kStaticLamBytes % 256 == 0 && kStaticLamcBytes % 256 == 0,
              "sub-arrays stay 256-byte aligned");
}  // namespace

static __device__ __align__(256) unsigned char g_forward_scratch[kStaticBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {nullptr};

// Device address of g_forward_scratch on the current device, looked up once per device.
// In host code the symbol itself is only a host-side stand-in, never a device address.
xpbd_status static_scratch_address(void** out) {
  int dev = 0;
  CU_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(XPBD_ERR_BOUNDS, "device ordinal beyond 64");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    CU_TRY(cudaGetSymbolAddress(&p, g_forward_scratch));
    if (!p) return fail(XPBD_ERR_CUDA, "cudaGetSymbolAddress returned NULL");
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return XPBD_OK;
}

// Frees every growable workspace buffer of a handle (the caller has synchronised).
void release_workspace(xpbd_solver* h) {
  DevBuf* bufs[] = {&h->P, &h->lam, &h->cflags, &h->lamc, &h->tape, &h->lam_tape, &h->tape_c,
                    &h->lamc_tape, &h->xbar, &h->vbar, &h->lb, &h->acc, &h->lbc, &h->cgrad,
                    &h->partials, &h->roll, &h->seg, &h->imp_blocks, &h->imp_vec, &h->imp_dinv,
                    &h->imp_sc, &h->imp_mg};
  for (DevBuf* b : bufs) b->release();
}

// ---------------------------------------------------------------- phase plan
// Runs of consecutive colors whose constraints, taken together, split into connected
// components of at most kPhaseMaxVerts vertices are launched as one phase kernel
// (xpbd_phase.cu).  Components are packed into CTA groups; records are copied into a phase
// order (phase, group, color, type, first vertex) with vertex indices local to the group.
// The plan is used when it needs fewer launches per iteration than there are colors.
template <class Rec>
Rec localize(Rec r, const std::vector<int>& loc);
template <>
DistRec localize(DistRec r, const std::vector<int>& loc) {
  r.a = loc[r.a];
  r.b = loc[r.b];
  return r;
}
template <>
BendRec localize(BendRec r, const std::vector<int>& loc) {
  for (int k = 0; k < 4; ++k) r.v[k] = loc[r.v[k]];
  return r;
}
template <>
TetRec localize(TetRec r, const std::vector<int>& loc) {
  for (int k = 0; k < 4; ++k) r.v[k] = loc[r.v[k]];
  return r;
}
template <>
MembRec localize(MembRec r, const std::vector<int>& loc) {
  for (int k = 0; k < 3; ++k) r.v[k] = loc[r.v[k]];
  return r;
}

// Local order of a group's vertices in shared memory.  A run of consecutive vertex ids (a
// grid row) is stored as its even offsets followed by its odd offsets.  A color's
// constraints are sorted by the local index of their first vertex, so a grid color whose
// constraints step by two columns (one parity class) then touches consecutive local
// vertices instead of every other one: the 128-bit accesses of 8 threads cover 128
// contiguous bytes, free of shared-memory bank conflicts.
std::vector<int> shared_memory_order(const std::vector<int>& list) {
  std::vector<int> out;
  out.reserve(list.size());
  size_t i = 0;
  while (i < list.size()) {
    size_t j = i;
    while (j + 1 < list.size() && list[j + 1] == list[j] + 1) ++j;
    for (size_t k = i; k <= j; k += 2) out.push_back(list[k]);
    for (size_t k = i + 1; k <= j; k += 2) out.push_back(list[k]);
    i = j + 1;
  }
  return out;
}

xpbd_status build_phases(xpbd_solver* h, const int* offsets, const int* order, const std::vector<DistRec>& rd,
                         const std::vector<BendRec>& rb, const std::vector<TetRec>& rh,
                         const std::vector<TetRec>& rdv, const std::vector<int>& perm,
                         const std::vector<MembRec>& rmb, const std::vector<int>& mperm, int min_cut) {
  const int V = h->V, K = h->K;
  if (K == 0 || V == 0) return XPBD_OK;
  // constraint id (membranes: m + triangle) -> (type, index in its type's record array)
  std::vector<int> type_of(h->m + h->nm), idx_of(h->m + h->nm);
  for (int t = 0; t < 4; ++t)
    for (int i = 0; i < h->n_rec[t]; ++i) {
      int j = perm[h->rec_off[t] + i];
      type_of[j] = t;
      idx_of[j] = i;
    }
  for (int i = 0; i < h->nm; ++i) {
    type_of[h->m + mperm[i]] = SEG_MEMB;
    idx_of[h->m + mperm[i]] = i;
  }
  auto verts_of = [&](int j, int* vs) -> int {
    int t = type_of[j], i = idx_of[j];
    if (t == 0) {
      vs[0] = rd[i].a;
      vs[1] = rd[i].b;
      return 2;
    }
    if (t == SEG_MEMB) {
      for (int k = 0; k < 3; ++k) vs[k] = rmb[i].v[k];
      return 3;
    }
    const int* v = t == 1 ? rb[i].v : (t == 2 ? rh[i].v : rdv[i].v);
    for (int k = 0; k < 4; ++k) vs[k] = v[k];
    return 4;
  };
  std::vector<int> parent(V), csz(V, 1);
  std::iota(parent.begin(), parent.end(), 0);
  std::vector<char> in(V, 0);
  std::vector<int> touched;
  int maxc = 1;
  auto find = [&](int x) {
    while (parent[x] != x) {
      parent[x] = parent[parent[x]];
      x = parent[x];
    }
    return x;
  };
  auto reset = [&]() {
    for (int v : touched) {
      parent[v] = v;
      csz[v] = 1;
      in[v] = 0;
    }
    touched.clear();
    maxc = 1;
  };
  auto add_color = [&](int c) {
    int vs[4];
    for (int t = offsets[c]; t < offsets[c + 1]; ++t) {
      int nv = verts_of(order[t], vs);
      for (int k = 0; k < nv; ++k)
        if (!in[vs[k]]) {
          in[vs[k]] = 1;
          touched.push_back(vs[k]);
        }
      for (int k = 1; k < nv; ++k) {
        int a = find(vs[0]), b = find(vs[k]);
        if (a == b) continue;
        if (csz[a] < csz[b]) std::swap(a, b);
        parent[b] = a;
        csz[a] += csz[b];
        maxc = std::max(maxc, csz[a]);
      }
    }
  };
  // 1. runs of colors.  Greedy: extend each run until the next color would make a
  // component larger than the limit.  Smaller components mean less shared memory per CTA
  // and more resident CTAs, so the smallest limit that needs no more runs than
  // kPhaseMaxVerts does is taken.  If even that leaves a one-color run, take the fewest runs
  // at kPhaseMaxVerts instead (dynamic program over each start's longest feasible run: an
  // interval that is too large stays too large when extended).
  auto greedy = [&](int limit, bool& single) {
    std::vector<std::pair<int, int>> rr;
    single = false;
    for (int c = 0; c < K;) {
      reset();
      const int c0 = c;
      while (c < K) {
        add_color(c);
        if (maxc > limit) break;
        ++c;
      }
      if (c == c0) ++c;
      single |= (c - c0) < 2;
      rr.push_back({c0, c});
    }
    return rr;
  };
  bool single = false;
  std::vector<std::pair<int, int>> runs = greedy(kPhaseMaxVerts, single);
  for (int limit : {kPhaseGroupVerts, 2 * kPhaseGroupVerts}) {
    bool s2 = false;
    std::vector<std::pair<int, int>> r2 = greedy(limit, s2);
    if (!s2 && r2.size() <= runs.size()) {
      runs = r2;
      single = false;
      break;
    }
  }
  if (single) {
    std::vector<int> reach(K);
    for (int a = 0; a < K; ++a) {
      reset();
      int b = a;
      while (b < K) {
        add_color(b);
        if (maxc > kPhaseMaxVerts) break;
        ++b;
      }
      reach[a] = std::max(b, a + 1);
    }
    std::vector<int> best(K + 1, 1 << 30), from(K + 1, -1);
    best[0] = 0;
    for (int a = 0; a < K; ++a) {
      if (best[a] == (1 << 30)) continue;
      for (int b = a + 1; b <= reach[a]; ++b)
        if (best[a] + 1 < best[b]) {
          best[b] = best[a] + 1;
          from[b] = a;
        }
    }
    runs.clear();
    for (int b = K; b > 0; b = from[b]) runs.push_back({from[b], b});
    std::reverse(runs.begin(), runs.end());
  }
  // keep one launch per color unless the runs cut the launches per iteration min_cut-fold
  if ((int)runs.size() >= K || (int64_t)runs.size() * min_cut > K) return XPBD_OK;
  // 2. groups, chunks and the padded phase records
  std::vector<DistRec> pd;
  std::vector<BendRec> pb;
  std::vector<TetRec> ph, pdv;
  std::vector<MembRec> pm;
  std::vector<int> pperm_t[kSegTypes];
  std::vector<PhaseGroup> groups;
  std::vector<PhaseChunk> chunks;
  std::vector<int> pverts;
  std::vector<int> loc(V, -1), comp_of_root(V, -1), group_of_vertex(V, -1);
  const double rec_bytes[kSegTypes] = {sizeof(DistRec), sizeof(int4) + sizeof(BendTail), sizeof(TetRec), sizeof(TetRec),
                                       sizeof(MembRec)};
  auto type_size = [&](int t) -> size_t {
    return t == 0 ? pd.size() : (t == 1 ? pb.size() : (t == 2 ? ph.size() : (t == 3 ? pdv.size() : pm.size())));
  };
  // a padding record: every vertex is the group's dummy vertex, alpha~ = 0
  auto push_pad = [&](int t, int dummy) {
    if (t == 0) {
      DistRec r{dummy, dummy, 0.f, 0.f};
      pd.push_back(r);
    } else if (t == 1) {
      BendRec r{{dummy, dummy, dummy, dummy}, 0.f, 0.f, 0.f, 0.f};
      pb.push_back(r);
    } else if (t == SEG_MEMB) {   // Dm^-1 = 0: S = 0 is not positive definite, so it never moves
      MembRec r;
      std::memset(&r, 0, sizeof(r));
      for (int k = 0; k < 3; ++k) r.v[k] = dummy;
      r.A = 1.f;
      pm.push_back(r);
    } else {
      TetRec r;
      std::memset(&r, 0, sizeof(r));
      for (int k = 0; k < 4; ++k) r.v[k] = dummy;
      r.gamma = 1.f;
      r.vol = 1.f;
      (t == 2 ? ph : pdv).push_back(r);
    }
    pperm_t[t].push_back(-1);
  };
  for (auto& run : runs) {
    reset();
    for (int c = run.first; c < run.second; ++c) add_color(c);
    const int ncol = run.second - run.first;
    std::vector<int> tv(touched.begin(), touched.end());
    std::sort(tv.begin(), tv.end());
    // components in order of their smallest vertex
    std::vector<std::vector<int>> comps;
    for (int v : tv) {
      int r = find(v);
      if (comp_of_root[r] < 0) {
        comp_of_root[r] = (int)comps.size();
        comps.emplace_back();
      }
      comps[comp_of_root[r]].push_back(v);
    }
    xpbd_solver::PhaseHost ph_info;
    ph_info.first_group = (int)groups.size();
    ph_info.c0 = run.first;
    ph_info.ncolors = ncol;
    // groups: consecutive components packed up to kPhaseGroupVerts vertices (a larger
    // component is a group of its own).  A small model packs less, down to one component
    // per group, so that a phase still has about kPhaseTargetGroups CTAs.
    std::vector<int> real_verts;   // per group of this phase: vertices without padding
    {
      const int pack = std::max(1, std::min(kPhaseGroupVerts, (int)(tv.size() / kPhaseTargetGroups)));
      std::vector<std::vector<int>> gv;
      int cur_n = 0;
      for (size_t k = 0; k < comps.size(); ++k) {
        int sz = (int)comps[k].size();
        if (gv.empty() || cur_n + sz > pack) {
          gv.emplace_back();
          cur_n = 0;
        }
        gv.back().insert(gv.back().end(), comps[k].begin(), comps[k].end());
        cur_n += sz;
      }
      for (const std::vector<int>& list : gv) {
        PhaseGroup g;
        g.vert_begin = (int)pverts.size();
        g.chunk_begin = 0;
        g.chunk_count = 0;
        const std::vector<int> order = shared_memory_order(list);
        g.vert_count = (int)order.size();
        groups.push_back(g);
        const int cur = (int)groups.size() - 1;
        for (int k = 0; k < (int)order.size(); ++k) {
          pverts.push_back(order[k]);
          if (order[k] < 0) continue;
          loc[order[k]] = k;
          group_of_vertex[order[k]] = cur;
        }
        real_verts.push_back((int)list.size());
      }
    }
    ph_info.n_groups = (int)groups.size() - ph_info.first_group;
    // bucket the run's constraints by (group, color, type), keeping color order
    std::vector<std::vector<int>> bucket((size_t)ph_info.n_groups * ncol * kSegTypes);
    for (int c = run.first; c < run.second; ++c)
      for (int t = offsets[c]; t < offsets[c + 1]; ++t) {
        int j = order[t], vs[4];
        verts_of(j, vs);
        int g = group_of_vertex[vs[0]] - ph_info.first_group;
        bucket[((size_t)g * ncol + (c - run.first)) * kSegTypes + type_of[j]].push_back(j);
      }
    double vbytes = 0;
    int64_t units = 0;
    double rbytes_f = 0, rbytes_r = 0, rbytes_v = 0;
    for (int g = 0; g < ph_info.n_groups; ++g) {
      PhaseGroup& G = groups[ph_info.first_group + g];
      G.chunk_begin = (int)chunks.size();
      ph_info.max_verts = std::max(ph_info.max_verts, G.vert_count);
      vbytes += 36.0 * real_verts[g];   // vertex index + one float4 read + one write
      for (int ci = 0; ci < ncol; ++ci) {
        const size_t color_first = chunks.size();
        for (int t = 0; t < kSegTypes; ++t) {
          std::vector<int>& b = bucket[((size_t)g * ncol + ci) * kSegTypes + t];
          if (b.empty()) continue;
          int vs0[4], vs1[4];
          std::stable_sort(b.begin(), b.end(), [&](int x, int y) {
            verts_of(x, vs0);
            verts_of(y, vs1);
            return loc[vs0[0]] < loc[vs1[0]];
          });
          const int begin = (int)type_size(t);   // a multiple of 4: every bucket is padded
          for (int j : b) {
            int i = idx_of[j];
            if (t == 0) pd.push_back(localize(rd[i], loc));
            else if (t == 1) pb.push_back(localize(rb[i], loc));
            else if (t == 2) ph.push_back(localize(rh[i], loc));
            else if (t == 3) pdv.push_back(localize(rdv[i], loc));
            else pm.push_back(localize(rmb[i], loc));
            pperm_t[t].push_back(t == SEG_MEMB ? j - h->m : j);
            if (h->coupled && t == SEG_TETH) {   // the C_D shadow at the same phase index
              pdv.push_back(localize(rdv[i], loc));
              pperm_t[SEG_TETD].push_back(j + h->nt);
            }
          }
          while (type_size(t) % 4) {
            push_pad(t, G.vert_count);
            if (h->coupled && t == SEG_TETH) push_pad(SEG_TETD, G.vert_count);
          }
          const bool pair = h->coupled && t == SEG_TETH;
          const int total = (int)type_size(t) - begin;
          for (int off = 0; off < total; off += kPhaseChunk) {
            PhaseChunk ck;
            ck.type = pair ? kChunkPair : t;
            ck.begin = begin + off;
            ck.count = std::min(kPhaseChunk, total - off);
            ck.flags = 0;
            chunks.push_back(ck);
            ph_info.max_chunk_size = std::max(ph_info.max_chunk_size, ck.count);
          }
          ph_info.type_mask |= 1 << (pair ? kChunkPair : t);
          const double n = (double)b.size(), nv = kVerts[t];
          const double nl = t == SEG_MEMB ? 3.0 : (pair ? 2.0 : 1.0), na = t == SEG_MEMB ? 4.0 : (pair ? 2.0 : 1.0);
          const double rb_ = pair ? 2.0 * rec_bytes[t] : rec_bytes[t];
          units += (int64_t)b.size() * (pair ? 2 : 1);
          rbytes_f += n * (rb_ + 8.0 * nl);
          rbytes_r += n * (rb_ + 8.0 * nl + 16.0 * nv);
          rbytes_v += n * (rb_ + 16.0 * nv + 4.0 * nl + 16.0 * na);
        }
        if (chunks.size() > color_first) {
          chunks[color_first].flags |= kChunkColorFirst;
          chunks.back().flags |= kChunkColorLast;
        }
      }
      G.chunk_count = (int)chunks.size() - G.chunk_begin;
      ph_info.max_chunks = std::max(ph_info.max_chunks, G.chunk_count);
    }
    ph_info.units = units;
    ph_info.bytes_fwd = rbytes_f + vbytes;
    ph_info.bytes_replay = rbytes_r + vbytes;
    ph_info.bytes_vjp = rbytes_v + vbytes;
    if (!phase_smem_bytes(ph_info.shape(), true) || !phase_smem_bytes(ph_info.shape(), false)) {
      h->phases.clear();   // cannot happen with kPhaseMaxVerts components; keep per-color launches
      return XPBD_OK;
    }
    h->phases.push_back(ph_info);
    for (int v : tv) {
      comp_of_root[v] = -1;
      comp_of_root[find(v)] = -1;
    }
  }
  // padded per-group vertex lists and chunk tables (fixed strides per phase), so a CTA
  // addresses its own from its index alone; chunk tables in forward and reverse order
  std::vector<int> pv_pad;
  std::vector<PhaseChunk> ch_pad, ch_rev;
  for (auto& ph : h->phases) {
    ph.vstride = ph.max_verts;
    ph.cstride = std::max(ph.max_chunks, 1);
    ph.vbase = (int64_t)pv_pad.size();
    ph.cbase = (int64_t)ch_pad.size();
    pv_pad.resize(pv_pad.size() + (size_t)ph.n_groups * ph.vstride, -1);
    PhaseChunk empty;
    std::memset(&empty, 0, sizeof(empty));
    ch_pad.resize(ch_pad.size() + (size_t)ph.n_groups * ph.cstride, empty);
    ch_rev.resize(ch_pad.size(), empty);
    for (int g = 0; g < ph.n_groups; ++g) {
      PhaseGroup& G = groups[ph.first_group + g];
      const int64_t vb = ph.vbase + (int64_t)g * ph.vstride, cb = ph.cbase + (int64_t)g * ph.cstride;
      std::copy(pverts.begin() + G.vert_begin, pverts.begin() + G.vert_begin + G.vert_count, pv_pad.begin() + vb);
      for (int k = 0; k < G.chunk_count; ++k) {
        ch_pad[cb + k] = chunks[G.chunk_begin + k];
        ch_rev[cb + k] = chunks[G.chunk_begin + G.chunk_count - 1 - k];
      }
      G.vert_begin = (int)vb;
      G.chunk_begin = (int)cb;
    }
  }
  pverts.swap(pv_pad);
  chunks.swap(ch_pad);
  // slot space and tape layout of the phase records
  size_t nslots = 0, ntape = 0;
  std::vector<int> pperm;
  for (int t = 0; t < kSegTypes; ++t) {   // membranes last, 4 slots per record
    h->n_prec[t] = (int)type_size(t);
    h->pslot_off[t] = (int)nslots;
    h->ptape_off[t] = ntape;
    nslots += (size_t)h->n_prec[t] * (t == SEG_MEMB ? 4 : 1);
    ntape += (size_t)h->n_prec[t] * kVerts[t];
    pperm.insert(pperm.end(), pperm_t[t].begin(), pperm_t[t].end());
  }
  // upload
  auto up = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
    *dst = nullptr;
    if (!bytes) return cudaSuccess;
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  cudaError_t e = up(&h->d_prec[0], pd.data(), pd.size() * sizeof(DistRec));
  {   // bending records as vertex indices and tails
    std::vector<int4> bv(pb.size());
    std::vector<BendTail> bt(pb.size());
    for (size_t i = 0; i < pb.size(); ++i) {
      bv[i] = make_int4(pb[i].v[0], pb[i].v[1], pb[i].v[2], pb[i].v[3]);
      bt[i] = BendTail{pb[i].theta0, pb[i].at};
    }
    if (e == cudaSuccess) e = up(&h->d_prec[1], bv.data(), bv.size() * sizeof(int4));
    if (e == cudaSuccess) e = up((void**)&h->d_prec_btail, bt.data(), bt.size() * sizeof(BendTail));
  }
  if (e == cudaSuccess) e = up(&h->d_prec[2], ph.data(), ph.size() * sizeof(TetRec));
  if (e == cudaSuccess) e = up(&h->d_prec[3], pdv.data(), pdv.size() * sizeof(TetRec));
  if (e == cudaSuccess) e = up(&h->d_prec[4], pm.data(), pm.size() * sizeof(MembRec));
  if (e == cudaSuccess) e = up((void**)&h->d_pperm, pperm.data(), pperm.size() * sizeof(int));
  if (e == cudaSuccess) e = up((void**)&h->d_groups, groups.data(), groups.size() * sizeof(PhaseGroup));
  if (e == cudaSuccess) e = up((void**)&h->d_chunks, chunks.data(), chunks.size() * sizeof(PhaseChunk));
  if (e == cudaSuccess) e = up((void**)&h->d_chunks_rev, ch_rev.data(), ch_rev.size() * sizeof(PhaseChunk));
  if (e == cudaSuccess) e = up((void**)&h->d_pverts, pverts.data(), pverts.size() * sizeof(int));
  if (e == cudaSuccess) e = phase_kernel_setup();
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? XPBD_ERR_OOM : XPBD_ERR_CUDA,
                std::string("phase plan upload: ") + cudaGetErrorString(e));
  h->slots = std::max(h->slots, (nslots + 3) / 4 * 4);
  h->tape_slots = std::max(h->tape_slots, ntape);
  h->use_phases = true;
  return XPBD_OK;
}

PhaseLaunch phase_args(const xpbd_solver* h, const xpbd_solver::PhaseHost& ph) {
  PhaseLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.groups = h->d_groups + ph.first_group;
  a.chunks = h->d_chunks + ph.cbase;
  a.chunks_rev = h->d_chunks_rev + ph.cbase;
  a.pverts = h->d_pverts + ph.vbase;
  a.vstride = ph.vstride;
  a.cstride = ph.cstride;
  for (int t = 0; t < kSegTypes; ++t) {
    a.slot_off[t] = h->pslot_off[t];
    a.prec[t] = h->d_prec[t];
    a.tape_off[t] = h->ptape_off[t];
  }
  a.prec_btail = h->d_prec_btail;
  a.memb_stride = h->n_prec[SEG_MEMB];
  a.err = h->d_err;
  a.wait_cycles = 1ll << 31;   // ~1 s at 2 GHz, far beyond any copy
  a.no_issue = 0;
  return a;
}

}  // namespace

extern "C" {

const char* xpbd_last_error(void) { return g_err.c_str(); }

xpbd_status xpbd_create(const xpbd_model* md, xpbd_handle* out) {
  g_err.clear();
  NvtxRange nvtx_range("xpbd_create");
  if (!md || !out) return fail(XPBD_ERR_INVALID, "null argument");
  *out = nullptr;
  const int V = md->n_vertices, nd = md->n_dist, nb = md->n_bend, nt = md->n_tet, K = md->n_colors;
  const int nm = md->n_memb;
  if (V < 0 || nd < 0 || nb < 0 || nt < 0 || K < 0 || nm < 0) return fail(XPBD_ERR_INVALID, "negative size");
  const long long mll = (long long)nd + nb + 2LL * nt;
  if (mll + 4LL * nm + 8 > 0x7fffffffLL) return fail(XPBD_ERR_INVALID, "too many constraints");
  const int m = (int)mll;
  if (nm && (!md->memb_idx || !md->memb_uv)) return fail(XPBD_ERR_INVALID, "membrane arrays NULL");
  if (V > 0 && (!md->rest_x || !md->inv_mass)) return fail(XPBD_ERR_INVALID, "rest_x/inv_mass NULL");
  if ((nd && !md->dist_idx) || (nb && !md->bend_idx) || (nt && !md->tet_idx))
    return fail(XPBD_ERR_INVALID, "index array NULL");
  if (!md->color_offsets || (m > 0 && !md->color_order)) return fail(XPBD_ERR_INVALID, "coloring NULL");
  for (int i = 0; i < 3 * V; ++i)
    if (!std::isfinite(md->rest_x[i])) return fail(XPBD_ERR_INVALID, "non-finite rest position");
  for (int i = 0; i < V; ++i)
    if (!(md->inv_mass[i] >= 0.f) || !std::isfinite(md->inv_mass[i]))
      return fail(XPBD_ERR_INVALID, "inverse mass must be finite and >= 0");
  auto verts_of = [&](int j, int* vs) -> int {
    if (j >= m) { for (int k = 0; k < 3; ++k) vs[k] = md->memb_idx[3 * (size_t)(j - m) + k]; return 3; }
    if (j < nd) { vs[0] = md->dist_idx[2 * (size_t)j]; vs[1] = md->dist_idx[2 * (size_t)j + 1]; return 2; }
    j -= nd;
    if (j < nb) { for (int k = 0; k < 4; ++k) vs[k] = md->bend_idx[4 * (size_t)j + k]; return 4; }
    j -= nb;
    int t = j % nt;
    for (int k = 0; k < 4; ++k) vs[k] = md->tet_idx[4 * (size_t)t + k];
    return 4;
  };
  for (int j = 0; j < m + nm; ++j) {
    int vs[4];
    int nv = verts_of(j, vs);
    for (int k = 0; k < nv; ++k) {
      if (vs[k] < 0 || vs[k] >= V) return fail(XPBD_ERR_INVALID, "vertex index out of range in constraint " + std::to_string(j));
      for (int q = 0; q < k; ++q)
        if (vs[q] == vs[k]) return fail(XPBD_ERR_INVALID, "constraint " + std::to_string(j) + " repeats a vertex");
    }
  }
  // coloring: offsets monotone, a permutation of the colored ids, vertex-disjoint colors.
  // Coupled tets: the C_D ids (nd + nb + nt ...) are not colored; each C_H id stands for
  // its tet's pair.
  if (md->tet_coupled != 0 && md->tet_coupled != 1) return fail(XPBD_ERR_INVALID, "tet_coupled must be 0 or 1");
  const bool coupled = md->tet_coupled == 1 && nt > 0;
  const int mc = coupled ? m - nt : m;
  // colored ids: [0, mc) and the membranes' [m, m + nm)
  auto colored = [&](int j) { return (j >= 0 && j < mc) || (j >= m && j < m + nm); };
  for (int t = 0; t < nm; ++t) {
    const float* uv = md->memb_uv + 6 * (size_t)t;
    for (int k = 0; k < 6; ++k)
      if (!std::isfinite(uv[k])) return fail(XPBD_ERR_INVALID, "non-finite membrane rest coordinate");
    const double det = ((double)uv[2] - uv[0]) * ((double)uv[5] - uv[1]) - ((double)uv[4] - uv[0]) * ((double)uv[3] - uv[1]);
    if (!(std::fabs(det) > 1e-30)) return fail(XPBD_ERR_INVALID, "membrane " + std::to_string(t) + " has zero rest area");
  }
  if (md->color_offsets[0] != 0 || md->color_offsets[K] != mc + nm)
    return fail(XPBD_ERR_COLORING, coupled ? "color offsets must start at 0 and end at m - n_tet + n_memb (coupled tets)"
                                           : "color offsets must start at 0 and end at m + n_memb");
  std::vector<char> seen(m + nm, 0);
  std::vector<int> stamp(V, -1);
  for (int c = 0; c < K; ++c) {
    int b = md->color_offsets[c], e = md->color_offsets[c + 1];
    if (e < b) return fail(XPBD_ERR_COLORING, "color offsets decrease");
    for (int t = b; t < e; ++t) {
      int j = md->color_order[t];
      if (!colored(j)) return fail(XPBD_ERR_COLORING, "constraint id out of range in coloring");
      if (seen[j]) return fail(XPBD_ERR_COLORING, "constraint " + std::to_string(j) + " appears twice");
      seen[j] = 1;
      int vs[4];
      int nv = verts_of(j, vs);
      for (int k = 0; k < nv; ++k) {
        if (stamp[vs[k]] == c)
          return fail(XPBD_ERR_COLORING, "color " + std::to_string(c) + " has two constraints on vertex " + std::to_string(vs[k]));
        stamp[vs[k]] = c;
      }
    }
  }
  for (int j = 0; j < m + nm; ++j)
    if (colored(j) && !seen[j]) return fail(XPBD_ERR_COLORING, "constraint " + std::to_string(j) + " has no color");

  // records, grouped by color, then type, then first vertex
  xpbd_solver* h = new xpbd_solver();
  h->V = V; h->nd = nd; h->nb = nb; h->nt = nt; h->m = m; h->K = K;
  h->coupled = coupled;
  h->nm = nm;
  h->mslot = (int)(((size_t)std::max(m, 1) + 3) / 4 * 4);
  h->slots = h->color_slots();
  h->mtape = (size_t)2 * nd + (size_t)4 * nb + (size_t)8 * nt;
  h->tape_slots = h->tape_per_iter();
  h->n_rec[0] = nd; h->n_rec[1] = nb; h->n_rec[2] = nt; h->n_rec[3] = nt;
  h->rec_off[0] = 0; h->rec_off[1] = nd; h->rec_off[2] = nd + nb; h->rec_off[3] = nd + nb + nt;
  std::vector<DistRec> rd; rd.reserve(nd);
  std::vector<BendRec> rb; rb.reserve(nb);
  std::vector<TetRec> rh, rdv; rh.reserve(nt); rdv.reserve(nt);
  std::vector<MembRec> rmb; rmb.reserve(nm);
  std::vector<int> perm(m), mperm(nm);
  auto X = [&](int v, double* o) { for (int c = 0; c < 3; ++c) o[c] = md->rest_x[3 * (size_t)v + c]; };
  h->colors.resize(K);
  for (int c = 0; c < K; ++c) {
    int b = md->color_offsets[c], e = md->color_offsets[c + 1];
    std::vector<int> ids[5];
    for (int t = b; t < e; ++t) {
      int j = md->color_order[t];
      int type = j >= m ? 4 : (j < nd ? 0 : (j < nd + nb ? 1 : (j < nd + nb + nt ? 2 : 3)));
      ids[type].push_back(j);
    }
    for (int type = 0; type < 5; ++type) {
      if (ids[type].empty()) continue;
      auto by_first_vertex = [&](int a, int bb) {
        int va[4], vb[4];
        verts_of(a, va);
        verts_of(bb, vb);
        return va[0] < vb[0];
      };
      if (!std::is_sorted(ids[type].begin(), ids[type].end(), by_first_vertex))
        std::stable_sort(ids[type].begin(), ids[type].end(), by_first_vertex);
      Seg sg;
      sg.type = (SegType)type;
      sg.count = (int)ids[type].size();
      sg.begin = type == 0 ? (int)rd.size() : type == 1 ? (int)rb.size() : type == 2 ? (int)rh.size()
                 : type == 3 ? (int)rdv.size() : (int)rmb.size();
      for (int j : ids[type]) {
        int vs[4];
        verts_of(j, vs);
        if (type == 4) {
          // Dm = [uv1 - uv0, uv2 - uv0] (columns), B = Dm^-1 row-major, A = |det Dm| / 2
          const float* uv = md->memb_uv + 6 * (size_t)(j - m);
          const double a = (double)uv[2] - uv[0], bb = (double)uv[4] - uv[0];
          const double c = (double)uv[3] - uv[1], d = (double)uv[5] - uv[1];
          const double det = a * d - bb * c;
          MembRec r;
          for (int k = 0; k < 3; ++k) r.v[k] = vs[k];
          r.B[0] = (float)(d / det);
          r.B[1] = (float)(-bb / det);
          r.B[2] = (float)(-c / det);
          r.B[3] = (float)(a / det);
          r.A = (float)(std::fabs(det) / 2.0);
          r.a00 = r.a11 = r.a01 = r.a22 = 0.f;
          mperm[rmb.size()] = j - m;
          rmb.push_back(r);
          continue;
        }
        if (type == 0) {
          double a[3], bb[3];
          X(vs[0], a);
          X(vs[1], bb);
          DistRec r;
          r.a = vs[0];
          r.b = vs[1];
          r.L = (float)std::sqrt((a[0] - bb[0]) * (a[0] - bb[0]) + (a[1] - bb[1]) * (a[1] - bb[1]) + (a[2] - bb[2]) * (a[2] - bb[2]));
          r.at = 0.f;
          perm[h->rec_off[0] + rd.size()] = j;
          rd.push_back(r);
        } else if (type == 1) {
          double x[4][3];
          for (int k = 0; k < 4; ++k) X(vs[k], x[k]);
          BendRec r;
          for (int k = 0; k < 4; ++k) r.v[k] = vs[k];
          r.theta0 = (float)rest_angle(x[0], x[1], x[2], x[3]);
          r.at = 0.f;
          r.pad0 = r.pad1 = 0.f;
          perm[h->rec_off[1] + rb.size()] = j;
          rb.push_back(r);
        } else {
          double x[4][3];
          for (int k = 0; k < 4; ++k) X(vs[k], x[k]);
          double Dm[9];
          for (int col = 0; col < 3; ++col)
            for (int row = 0; row < 3; ++row) Dm[row * 3 + col] = x[col + 1][row] - x[0][row];
          double det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
                       Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
          if (!(std::fabs(det) > 1e-30) || !std::isfinite(det)) {
            delete h;
            return fail(XPBD_ERR_INVALID, "degenerate rest tetrahedron " + std::to_string(j));
          }
          double inv[9] = {Dm[4] * Dm[8] - Dm[5] * Dm[7], Dm[2] * Dm[7] - Dm[1] * Dm[8], Dm[1] * Dm[5] - Dm[2] * Dm[4],
                           Dm[5] * Dm[6] - Dm[3] * Dm[8], Dm[0] * Dm[8] - Dm[2] * Dm[6], Dm[2] * Dm[3] - Dm[0] * Dm[5],
                           Dm[3] * Dm[7] - Dm[4] * Dm[6], Dm[1] * Dm[6] - Dm[0] * Dm[7], Dm[0] * Dm[4] - Dm[1] * Dm[3]};
          TetRec r;
          for (int k = 0; k < 4; ++k) r.v[k] = vs[k];
          for (int k = 0; k < 9; ++k) r.B[k] = (float)(inv[k] / det);
          r.at = 0.f;
          int t = (j - nd - nb) % nt;
          r.gamma = md->tet_gamma ? md->tet_gamma[t] : 1.f;
          r.vol = (float)(std::fabs(det) / 6.0);
          if (type == 2) {
            perm[h->rec_off[2] + rh.size()] = j;
            rh.push_back(r);
            if (coupled) {   // the C_D shadow: same tet, same slot index
              perm[h->rec_off[3] + rdv.size()] = j + nt;
              rdv.push_back(r);
            }
          } else {
            perm[h->rec_off[3] + rdv.size()] = j;
            rdv.push_back(r);
          }
        }
      }
      h->colors[c].push_back(sg);
    }
  }
  // upload
  auto up = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
    *dst = nullptr;
    if (!bytes) return cudaSuccess;
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = up(&h->d_rec[0], rd.data(), rd.size() * sizeof(DistRec));
  if (e == cudaSuccess) e = up(&h->d_rec[1], rb.data(), rb.size() * sizeof(BendRec));
  if (e == cudaSuccess) e = up(&h->d_rec[2], rh.data(), rh.size() * sizeof(TetRec));
  if (e == cudaSuccess) e = up(&h->d_rec[3], rdv.data(), rdv.size() * sizeof(TetRec));
  if (e == cudaSuccess) e = up((void**)&h->d_perm, perm.data(), perm.size() * sizeof(int));
  if (e == cudaSuccess) e = up((void**)&h->d_mrec, rmb.data(), rmb.size() * sizeof(MembRec));
  if (e == cudaSuccess) e = up((void**)&h->d_mperm, mperm.data(), mperm.size() * sizeof(int));
  if (e == cudaSuccess) e = up((void**)&h->d_w, md->inv_mass, (size_t)V * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    xpbd_destroy(h);
    return fail(e == cudaErrorMemoryAllocation ? XPBD_ERR_OOM : XPBD_ERR_CUDA,
                std::string("xpbd_create upload: ") + cudaGetErrorString(e));
  }
  if (md->exec_mode < 0 || md->exec_mode > 2) {
    xpbd_destroy(h);
    return fail(XPBD_ERR_INVALID, "exec_mode must be 0, 1 or 2");
  }
  if (md->exec_mode != 1) {
    // Automatic mode: on GB300 the phase plan was faster than per-color launches of the
    // same coloring by 1.7-3.4x where it cut launches per iteration 16x (cloth tiles), and
    // slower (0.5-0.8x) where it cut them 1.8x (row-shaped components serialise many chunks
    // per CTA), so it is used when it needs at most a quarter of the launches.
    const int min_cut = md->exec_mode == 0 ? 4 : 1;
    xpbd_status pst = build_phases(h, md->color_offsets, md->color_order, rd, rb, rh, rdv, perm, rmb, mperm, min_cut);
    if (pst != XPBD_OK) {
      xpbd_destroy(h);
      return pst;
    }
  }
  // The allocation-free forward's working array lives in this file's device module.  With
  // CUDA's lazy module loading that module (and the array's memory) is loaded on first use,
  // so it is looked up here, at set-up, where allocating is allowed: xpbd_forward_static
  // then only reads the stored address.
  xpbd_status sst = static_scratch_address(&h->static_base);
  if (sst != XPBD_OK) {
    xpbd_destroy(h);
    return sst;
  }
  *out = h;
  return XPBD_OK;
}

xpbd_status xpbd_release_workspace(xpbd_handle h) {
  if (!h) return fail(XPBD_ERR_INVALID, "null handle");
  CU_TRY(cudaDeviceSynchronize());
  release_workspace(h);
  return XPBD_OK;
}

xpbd_status xpbd_destroy(xpbd_handle h) {
  if (!h) return XPBD_OK;
  cudaDeviceSynchronize();
  for (int t = 0; t < 4; ++t)
    if (h->d_rec[t]) cudaFree(h->d_rec[t]);
  if (h->d_perm) cudaFree(h->d_perm);
  if (h->d_mrec) cudaFree(h->d_mrec);
  if (h->d_mperm) cudaFree(h->d_mperm);
  if (h->d_w) cudaFree(h->d_w);
  if (h->d_err) cudaFree(h->d_err);
  for (int t = 0; t < kSegTypes; ++t)
    if (h->d_prec[t]) cudaFree(h->d_prec[t]);
  if (h->d_prec_btail) cudaFree(h->d_prec_btail);
  void* plan[] = {h->d_pperm, h->d_groups, h->d_chunks, h->d_chunks_rev, h->d_pverts};
  for (void* q : plan)
    if (q) cudaFree(q);
  release_workspace(h);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
  return XPBD_OK;
}

xpbd_status xpbd_sizes(xpbd_handle h, int32_t* nv, int32_t* nc, int32_t* ncol) {
  if (!h) return fail(XPBD_ERR_INVALID, "null handle");
  if (nv) *nv = h->V;
  if (nc) *nc = h->m;
  if (ncol) *ncol = h->K;
  return XPBD_OK;
}

size_t xpbd_checkpoint_bytes(xpbd_handle h, int32_t steps) {
  if (!h || steps < 0) return 0;
  return (size_t)(steps + 1) * (size_t)h->V * 2 * sizeof(float4);
}

size_t xpbd_workspace_bytes(xpbd_handle h, int32_t iters) {
  if (!h || iters < 1) return 0;
  size_t V = h->V, m = h->slots;
  size_t b = 16 * V + 4 * m + V + 8 * V;                          // forward
  b += 16 * std::max(h->tape_slots, (size_t)1) * iters + 4 * m * iters;            // replay tapes
  b += (16 + 8) * V * iters + 8 * V + 20 * V;                      // contact tapes and scratch
  b += 32 * V + 8 * m + 8 * m + 40 * (size_t)partial_blocks(std::max(h->V, 1));
  return b;
}

xpbd_status xpbd_forward(xpbd_handle h, const xpbd_params* p, int32_t steps, int32_t iters,
                         const float* x0, const float* v0, float* ck, void* stream) {
  g_err.clear();
  NvtxRange nvtx_range("xpbd_forward");
  xpbd_status st = check_params(h, p, steps, iters);
  if (st != XPBD_OK) return st;
  if (h->V > 0 && (!x0 || !v0 || !ck)) return fail(XPBD_ERR_INVALID, "x0/v0/checkpoints NULL");
  if (h->V == 0) return XPBD_OK;
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_forward_ws(h);
  if (st != XPBD_OK) return st;
  st = set_alpha(h, p, s, h->use_phases);
  if (st != XPBD_OK) return st;
  float4* ck4 = reinterpret_cast<float4*>(ck);
  launch(h, XPBD_K_OTHER, h->V, s, [&] { launch_init_ckpt(x0, v0, h->d_w, ck4, ck4 + h->V, h->V, s); });
  LAUNCH_CHECK();
  for (int n = 0; n < steps; ++n) {
    st = forward_step(h, p, n, iters, ck_x(ck, h->V, n), ck_v(ck, h->V, n), ck4 + (size_t)2 * h->V * (n + 1), s);
    if (st != XPBD_OK) return st;
  }
  return XPBD_OK;
}

xpbd_status xpbd_read_state(xpbd_handle h, const float* ck, int32_t step, float* x_out, float* v_out,
                            void* stream) {
  if (!h || !ck || step < 0) return fail(XPBD_ERR_INVALID, "bad argument");
  launch(h, XPBD_K_OTHER, h->V, (cudaStream_t)stream, [&] {
    launch_read_state(ck_x(ck, h->V, step), ck_v(ck, h->V, step), x_out, v_out, h->V, (cudaStream_t)stream);
  });
  LAUNCH_CHECK();
  return XPBD_OK;
}

xpbd_status xpbd_loss(xpbd_handle h, const float* ck, int32_t n_keys, const int32_t* key_steps,
                      const float* targets, double* loss_out, float* seeds_out, void* stream) {
  g_err.clear();
  NvtxRange nvtx_range("xpbd_loss");
  if (!h || !ck || n_keys < 0 || (n_keys > 0 && (!key_steps || !targets)))
    return fail(XPBD_ERR_INVALID, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  int pb = partial_blocks(std::max(h->V, 1));
  CU_TRY(h->partials.ensure(sizeof(double) * 5 * (size_t)pb));
  if (loss_out) CU_TRY(cudaMemsetAsync(loss_out, 0, sizeof(double), s));
  for (int k = 0; k < n_keys; ++k) {
    if (key_steps[k] < 0) return fail(XPBD_ERR_INVALID, "negative key step");
    launch(h, XPBD_K_OTHER, h->V, s, [&] {
      launch_loss(ck_x(ck, h->V, key_steps[k]), targets + 3 * (size_t)h->V * k,
                  seeds_out ? seeds_out + 3 * (size_t)h->V * k : nullptr, h->partials.as<double>(), h->V, s);
    });
    if (loss_out)
      launch(h, XPBD_K_OTHER, 1, s, [&] { launch_reduce_partials(h->partials.as<double>(), pb, 1, loss_out, true, s); });
    LAUNCH_CHECK();
  }
  return XPBD_OK;
}

}  // extern "C"

namespace {

// State of one reverse sweep shared by its steps.
struct AdjointSweep {
  std::vector<int> seed_of;   // step -> index of its dL/dx seed, or -1
  const float* seed_dx = nullptr;
  const xpbd_grads* out = nullptr;
  bool contacts = false;
  int pb = 0;
};

// Validation, workspace, alpha~, zeroed outputs and the seeds at the last step.
xpbd_status adjoint_begin(xpbd_solver* h, const xpbd_params* p, int32_t steps, int32_t iters, int32_t n_seeds,
                          const int32_t* seed_steps, const float* seed_dx, const float* seed_dv_T,
                          const xpbd_grads* out, cudaStream_t s, AdjointSweep& A) {
  A.seed_of.assign(steps + 1, -1);
  for (int k = 0; k < n_seeds; ++k) {
    int n = seed_steps[k];
    if (n < 0 || n > steps) return fail(XPBD_ERR_INVALID, "seed step out of range");
    if (A.seed_of[n] >= 0) return fail(XPBD_ERR_INVALID, "two seeds for one step");
    A.seed_of[n] = k;
  }
  A.seed_dx = seed_dx;
  A.out = out;
  const int V = h->V;
  A.contacts = (p->collider_flags & 3) != 0;
  xpbd_status st = ensure_adjoint_ws(h, iters, A.contacts);
  if (st != XPBD_OK) return st;
  st = set_alpha(h, p, s, h->use_phases);
  if (st != XPBD_OK) return st;
  A.pb = partial_blocks(std::max(V, 1));
  CU_TRY(cudaMemsetAsync(h->acc.p, 0, sizeof(double) * h->slots, s));
  if (out->d_f_vertex) CU_TRY(cudaMemsetAsync(out->d_f_vertex, 0, sizeof(double) * 3 * (size_t)V, s));
  if (out->d_collider) CU_TRY(cudaMemsetAsync(out->d_collider, 0, sizeof(double) * 5, s));
  if (out->d_f_global && steps > 0) CU_TRY(cudaMemsetAsync(out->d_f_global, 0, sizeof(double) * 3 * (size_t)steps, s));
  launch(h, XPBD_K_ADJ_OTHER, V, s, [&] {
    launch_seed_adjoint(A.seed_of[steps] >= 0 ? seed_dx + 3 * (size_t)V * A.seed_of[steps] : nullptr, seed_dv_T,
                        h->xbar.as<float4>(), h->vbar.as<float4>(), V, s);
  });
  LAUNCH_CHECK();
  return XPBD_OK;
}

xpbd_status adjoint_predict(xpbd_solver* h, const xpbd_params* p, int n, const float4* ckx_n, const AdjointSweep& A,
                            cudaStream_t s);

// Reverse of step n from its state (x_n, v_n): replay with tapes, then the reverse
// iterations, then the adjoint of the prediction.
xpbd_status adjoint_step(xpbd_solver* h, const xpbd_params* p, int n, int32_t iters, const float4* ckx_n,
                         const float4* ckv_n, const AdjointSweep& A, cudaStream_t s) {
  const int V = h->V;
  const xpbd_grads* out = A.out;
  float4* xbar = h->xbar.as<float4>();
  float4* vbar = h->vbar.as<float4>();
  double* partials = h->partials.as<double>();
  const size_t tpi = h->tape_slots;
  const Collide c = make_collide(p);
  launch(h, XPBD_K_ADJ_OTHER, V, s, [&] { launch_adj_begin(xbar, vbar, 1.f / p->dt, V, s); });
  xpbd_status st = run_step(h, p, n, iters, ckx_n, ckv_n, true, s);
  if (st != XPBD_OK) return st;
  for (int k = iters - 1; k >= 0; --k) {
    const bool first = k == iters - 1, last = k == 0;
    if (A.contacts) {
      launch(h, XPBD_K_VJP_CONTACT, V, s, [&] {
        launch_vjp_contact(h->tape_c.as<float4>() + (size_t)k * V, h->cflags.as<uint8_t>(), V,
                           k == 0 ? nullptr : h->lamc_tape.as<float2>() + (size_t)(k - 1) * V, xbar,
                           h->lbc.as<float2>(), out->d_collider ? h->cgrad.as<float>() : nullptr, first, c, s);
      });
    }
    const float4* tape_k = h->tape.as<float4>() + (size_t)k * tpi;
    const float* lam_pre = k == 0 ? nullptr : h->lam_tape.as<float>() + (size_t)(k - 1) * h->slots;
    for (int q = h->use_phases ? (int)h->phases.size() - 1 : -1; q >= 0; --q) {
      const auto& ph = h->phases[q];
      PhaseLaunch a = phase_args(h, ph);
      a.P = xbar;
      a.lam_in = lam_pre;
      a.tape = const_cast<float4*>(tape_k);
      a.lb = h->lb.as<float2>();
      a.acc = h->acc.as<double>();
      launch(h, XPBD_K_VJP_PHASE, ph.units, s,
             [&] { launch_phase_vjp(a, ph.shape(), first, last, s); }, ph.bytes_vjp);
    }
    for (int col = h->use_phases ? -1 : h->K - 1; col >= 0; --col) {
      const std::vector<Seg>& segs = h->colors[col];
      for (int q = (int)segs.size() - 1; q >= 0; --q) vjp_segment(h, segs[q], tape_k, lam_pre, xbar, first, last, s);
    }
    LAUNCH_CHECK();
  }
  if (A.contacts && out->d_collider) {
    launch(h, XPBD_K_ADJ_OTHER, V, s,
           [&] { launch_collider_partials(h->cgrad.as<float>(), h->cflags.as<uint8_t>(), V, partials, s); });
    launch(h, XPBD_K_ADJ_OTHER, 1, s, [&] { launch_reduce_partials(partials, A.pb, 5, out->d_collider, true, s); });
  }
  return adjoint_predict(h, p, n, ckx_n, A, s);
}

// Adjoint of step n's prediction, xbar holding pbar: dL/dx_n, dL/dv_n, the seed at step n
// and the force gradients.
xpbd_status adjoint_predict(xpbd_solver* h, const xpbd_params* p, int n, const float4* ckx_n, const AdjointSweep& A,
                            cudaStream_t s) {
  const int V = h->V;
  const xpbd_grads* out = A.out;
  double* partials = h->partials.as<double>();
  const float* seed = A.seed_of[n] >= 0 ? A.seed_dx + 3 * (size_t)V * A.seed_of[n] : nullptr;
  launch(h, XPBD_K_ADJ_OTHER, V, s, [&] {
    launch_adj_predict(h->xbar.as<float4>(), h->vbar.as<float4>(), ckx_n, seed, p->dt, out->d_f_vertex,
                       out->d_f_global ? partials : nullptr,
                       out->d_f_vertex_steps ? out->d_f_vertex_steps + 3 * (size_t)V * n : nullptr, V, s);
  });
  if (out->d_f_global)
    launch(h, XPBD_K_ADJ_OTHER, 1, s,
           [&] { launch_reduce_partials(partials, A.pb, 3, out->d_f_global + 3 * (size_t)n, false, s); });
  LAUNCH_CHECK();
  return XPBD_OK;
}

// dL/dx0, dL/dv0 and the compliance gradient in caller order (the accumulators in the
// phase-plan slot order when `phase_layout`, else in the per-color one).
xpbd_status adjoint_end(xpbd_solver* h, const xpbd_params* p, const xpbd_grads* out, cudaStream_t s,
                        bool phase_layout) {
  const int V = h->V;
  if (out->d_x0) launch(h, XPBD_K_ADJ_OTHER, V, s, [&] { launch_to_double(h->xbar.as<float4>(), out->d_x0, V, s); });
  if (out->d_v0) launch(h, XPBD_K_ADJ_OTHER, V, s, [&] { launch_to_double(h->vbar.as<float4>(), out->d_v0, V, s); });
  if (out->d_compliance) {
    float inv_dt2 = 1.f / (p->dt * p->dt);
    const bool ph = phase_layout;
    for (int t = 0; t < 4; ++t) {
      const int off = ph ? h->pslot_off[t] : h->rec_off[t], cnt = ph ? h->n_prec[t] : h->n_rec[t];
      launch(h, XPBD_K_ADJ_OTHER, cnt, s, [&] {
        launch_finalize_compliance((SegType)t, ph ? h->d_prec[t] : h->d_rec[t], (ph ? h->d_pperm : h->d_perm) + off,
                                   cnt, h->acc.as<double>() + off, inv_dt2, out->d_compliance, s);
      });
    }
  }
  if (out->d_memb_stiffness) {
    const bool ph = phase_layout;
    const int nmr = ph ? h->n_prec[SEG_MEMB] : h->nm;
    launch(h, XPBD_K_ADJ_OTHER, nmr, s, [&] {
      launch_memb_gradient(ph ? (const MembRec*)h->d_prec[SEG_MEMB] : h->d_mrec,
                           ph ? h->d_pperm + h->pslot_off[SEG_MEMB] : h->d_mperm, nmr, p->memb_stiffness,
                           1.f / (p->dt * p->dt), h->acc.as<double>() + (ph ? h->pslot_off[SEG_MEMB] : h->mslot),
                           nmr, out->d_memb_stiffness, s);
    });
  }
  LAUNCH_CHECK();
  return XPBD_OK;
}

// Forward step n from state (x_n, v_n) to (x_{n+1}, v_{n+1}) at nx (positions; velocities follow).
xpbd_status forward_step(xpbd_solver* h, const xpbd_params* p, int n, int32_t iters, const float4* ckx_n,
                         const float4* ckv_n, float4* nx, cudaStream_t s) {
  xpbd_status st = run_step(h, p, n, iters, ckx_n, ckv_n, false, s);
  if (st != XPBD_OK) return st;
  const float inv_dt = 1.f / p->dt;
  launch(h, XPBD_K_VELOCITY, h->V, s, [&] {
    launch_velocity(h->P.as<float4>(), ckx_n, nx, nx + h->V, inv_dt, h->V, h->d_err, s);
  });
  LAUNCH_CHECK();
  return XPBD_OK;
}

}  // namespace

extern "C" {

int32_t xpbd_sparse_slots(int32_t steps, int32_t stride) {
  if (steps < 0 || stride < 1) return -1;
  return steps / stride + 1 + (steps % stride ? 1 : 0);
}

int32_t xpbd_sparse_slot(int32_t steps, int32_t stride, int32_t step) {
  if (steps < 0 || stride < 1 || step < 0 || step > steps) return -1;
  if (step % stride == 0) return step / stride;
  return step == steps ? steps / stride + 1 : -1;
}

xpbd_status xpbd_forward_sparse(xpbd_handle h, const xpbd_params* p, int32_t steps, int32_t iters,
                                const float* x0, const float* v0, int32_t stride, float* ck, void* stream) {
  g_err.clear();
  NvtxRange nvtx_range("xpbd_forward_sparse");
  xpbd_status st = check_params(h, p, steps, iters);
  if (st != XPBD_OK) return st;
  if (stride < 1) return fail(XPBD_ERR_INVALID, "stride must be >= 1");
  if (h->V > 0 && (!x0 || !v0 || !ck)) return fail(XPBD_ERR_INVALID, "x0/v0/checkpoints NULL");
  if (h->V == 0) return XPBD_OK;
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_forward_ws(h);
  if (st != XPBD_OK) return st;
  CU_TRY(h->roll.ensure(sizeof(float4) * 4 * (size_t)h->V));
  st = set_alpha(h, p, s, h->use_phases);
  if (st != XPBD_OK) return st;
  const size_t V = (size_t)h->V;
  float4* ck4 = reinterpret_cast<float4*>(ck);
  float4* roll = h->roll.as<float4>();
  launch(h, XPBD_K_OTHER, h->V, s, [&] { launch_init_ckpt(x0, v0, h->d_w, ck4, ck4 + V, h->V, s); });
  LAUNCH_CHECK();
  const float4* cur = ck4;   // state n: a stored slot or the rolling buffer
  for (int n = 0; n < steps; ++n) {
    const int slot = xpbd_sparse_slot(steps, stride, n + 1);
    float4* nx = slot >= 0 ? ck4 + 2 * V * slot : roll + 2 * V * ((n + 1) & 1);
    st = forward_step(h, p, n, iters, cur, cur + V, nx, s);
    if (st != XPBD_OK) return st;
    cur = nx;
  }
  return XPBD_OK;
}

xpbd_status xpbd_adjoint_sparse(xpbd_handle h, const xpbd_params* p, int32_t steps, int32_t iters,
                                const float* ck, int32_t stride, int32_t n_seeds, const int32_t* seed_steps,
                                const float* seed_dx, const float* seed_dv_T, const xpbd_grads* out,
                                void* stream) {
  g_err.clear();
  NvtxRange nvtx_range("xpbd_adjoint_sparse");
  xpbd_status st = check_params(h, p, steps, iters);
  if (st != XPBD_OK) return st;
  if (stride < 1) return fail(XPBD_ERR_INVALID, "stride must be >= 1");
  if (!ck || !out || n_seeds < 0 || (n_seeds > 0 && (!seed_steps || !seed_dx)))
    return fail(XPBD_ERR_INVALID, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  AdjointSweep A;
  st = adjoint_begin(h, p, steps, iters, n_seeds, seed_steps, seed_dx, seed_dv_T, out, s, A);
  if (st != XPBD_OK) return st;
  const size_t V = (size_t)h->V;
  if (steps > 0 && V > 0) {
    CU_TRY(h->seg.ensure(sizeof(float4) * 2 * V * (size_t)std::max(stride - 1, 1)));
    const float4* ck4 = reinterpret_cast<const float4*>(ck);
    float4* seg = h->seg.as<float4>();
    // segments [s0, s0 + len) from the last to the first: recompute the states inside a
    // segment from its stored first state, then reverse its steps
    for (int s0 = ((steps - 1) / stride) * stride; s0 >= 0; s0 -= stride) {
      const int len = std::min(stride, steps - s0);
      const float4* first = ck4 + 2 * V * (size_t)(s0 / stride);
      const float4* cur = first;
      for (int j = 0; j + 1 < len; ++j) {
        float4* nx = seg + 2 * V * (size_t)j;
        st = forward_step(h, p, s0 + j, iters, cur, cur + V, nx, s);
        if (st != XPBD_OK) return st;
        cur = nx;
      }
      for (int n = s0 + len - 1; n >= s0; --n) {
        const float4* x_n = n == s0 ? first : seg + 2 * V * (size_t)(n - s0 - 1);
        st = adjoint_step(h, p, n, iters, x_n, x_n + V, A, s);
        if (st != XPBD_OK) return st;
      }
    }
  }
  return adjoint_end(h, p, out, s, h->use_phases);
}

// z = V-cycle(r) of the grid multigrid preconditioner (xpbd_multigrid.cuh); X is the
// level-0 pin mask.  Level 0's right-hand side and correction are r and z themselves.
static void mg_vcycle(xpbd_solver* h, const MgPlan& g, const float4* X, const double* r, double* z, cudaStream_t s) {
  const int L = g.levels;
  auto rhs = [&](int l) { return l == 0 ? r : (const double*)g.lv[l].b; };
  auto sol = [&](int l) { return l == 0 ? z : g.lv[l].x; };
  auto smooth = [&](int l, bool forward) {
    const MgLevel& lv = g.lv[l];
    const int n = lv.nx * lv.ny;
    for (int sweep = 0; sweep < g.sweeps; ++sweep) {
      if (l == 0 && g.line_dir) {
        for (int k = 0; k < 5; ++k) {
          const int col = forward ? k : 4 - k;
          launch(h, XPBD_K_ADJ_OTHER, n, s, [&] { launch_mg_line_resid(lv, X, rhs(l), sol(l), lv.r, g.line_dir, col, s); });
          launch(h, XPBD_K_ADJ_OTHER, n, s, [&] { launch_mg_line_solve(lv, g.lfac, lv.r, sol(l), g.line_dir, col, s); });
        }
      } else {
        for (int k = 0; k < 9; ++k) {
          const int col = forward ? k : 8 - k;
          launch(h, XPBD_K_ADJ_OTHER, n, s, [&] { launch_mg_point_gs(lv, rhs(l), sol(l), col, s); });
        }
      }
    }
  };
  for (int l = 0; l + 1 < L; ++l) {
    const MgLevel& lv = g.lv[l];
    const int n = lv.nx * lv.ny;
    cudaMemsetAsync(sol(l), 0, sizeof(double) * 3 * (size_t)n, s);
    smooth(l, true);
    launch(h, XPBD_K_ADJ_OTHER, n, s, [&] { launch_mg_resid(lv, l == 0 ? X : nullptr, rhs(l), sol(l), lv.r, s); });
    launch(h, XPBD_K_ADJ_OTHER, n, s, [&] { launch_mg_restrict(lv, lv.r, g.lv[l + 1], g.lv[l + 1].b, s); });
  }
  const MgLevel& lc = g.lv[L - 1];
  launch(h, XPBD_K_ADJ_OTHER, lc.nx * lc.ny, s, [&] { launch_mg_coarse_solve(lc, g.cinv, rhs(L - 1), sol(L - 1), s); });
  for (int l = L - 2; l >= 0; --l) {
    const MgLevel& lv = g.lv[l];
    launch(h, XPBD_K_ADJ_OTHER, lv.nx * lv.ny, s,
           [&] { launch_mg_prolong(g.lv[l + 1], g.lv[l + 1].x, lv, l == 0 ? X : nullptr, sol(l), s); });
    smooth(l, false);
  }
}

// The V-cycle's launches are the same in every CG iteration of a call (same buffers; the
// level-0 pin mask reads only the inverse masses, which every checkpointed state holds),
// so they are captured once per call into a CUDA graph and replayed: the ~135 small
// launches of a V-cycle otherwise cost more in launch overhead than in work.  Capture
// runs on a private stream (the caller's may be the legacy default stream, which cannot
// capture); the replay is ordered on the caller's stream.  If capture fails the V-cycle
// is launched directly.
struct VcycleGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
  cudaStream_t cs = nullptr;
  mutable cudaStream_t replayed_on = nullptr;   // waited for before the graph is destroyed
  mutable bool replayed = false;
  int64_t launches = 0, units = 0;
  double bytes = 0.0;
  VcycleGraph() = default;
  VcycleGraph(const VcycleGraph&) = delete;
  VcycleGraph& operator=(const VcycleGraph&) = delete;
  ~VcycleGraph() {
    // Every step's CG loop ends with a stream synchronisation, so on the normal path no
    // replay is in flight here; on an early error return one may be.
    if (replayed) cudaStreamSynchronize(replayed_on);
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
    if (cs) cudaStreamDestroy(cs);
  }
  bool capture(xpbd_solver* h, const MgPlan& mg, const float4* X, const double* r, double* z) {
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      cs = nullptr;
      cudaGetLastError();
      return false;
    }
    const int k = XPBD_K_ADJ_OTHER;
    const bool prof = h->prof_on;
    const int64_t l0 = h->launches[k], u0 = h->units[k];
    const double b0 = h->alg_bytes[k];
    h->prof_on = false;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      mg_vcycle(h, mg, X, r, z, cs);
      ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && g != nullptr;
    }
    h->prof_on = prof;
    launches = h->launches[k] - l0;
    units = h->units[k] - u0;
    bytes = h->alg_bytes[k] - b0;
    h->launches[k] = l0;
    h->units[k] = u0;
    h->alg_bytes[k] = b0;
    if (ok) ok = cudaGraphInstantiate(&e, g, 0) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      if (e) cudaGraphExecDestroy(e);
      if (g) cudaGraphDestroy(g);
      e = nullptr;
      g = nullptr;
    }
    return ok;
  }
  cudaError_t run(xpbd_solver* h, cudaStream_t s) const {
    replayed = true;
    replayed_on = s;
    h->launches[XPBD_K_ADJ_OTHER] += launches;
    h->units[XPBD_K_ADJ_OTHER] += units;
    h->alg_bytes[XPBD_K_ADJ_OTHER] += bytes;
    return cudaGraphLaunch(e, s);
  }
};

xpbd_status xpbd_adjoint_implicit(xpbd_handle h, const xpbd_params* p, int32_t steps, int32_t iters,
                                  const float* ck, int32_t n_seeds, const int32_t* seed_steps, const float* seed_dx,
                                  const float* seed_dv_T, const xpbd_grads* out, const xpbd_implicit_opts* o,
                                  void* stream) {
  g_err.clear();
  NvtxRange nvtx_range("xpbd_adjoint_implicit");
  xpbd_status st = check_params(h, p, steps, iters);
  if (st != XPBD_OK) return st;
  if (!ck || !out || !o || n_seeds < 0 || (n_seeds > 0 && (!seed_steps || !seed_dx)))
    return fail(XPBD_ERR_INVALID, "bad argument");
  if (out->d_collider)
    return fail(XPBD_ERR_INVALID, "the implicit adjoint forms no collider-parameter gradient (d_collider must be NULL)");
  if (!(o->cg_tol > 0.0) || o->cg_max_iters < 1) return fail(XPBD_ERR_INVALID, "cg_tol must be > 0 and cg_max_iters >= 1");
  const bool use_mg = o->mg_nx != 0 || o->mg_ny != 0;
  if (use_mg && (o->mg_nx < 1 || o->mg_ny < 1 || (int64_t)o->mg_nx * o->mg_ny != h->V))
    return fail(XPBD_ERR_INVALID, "multigrid: mg_nx * mg_ny must equal the vertex count");
  if (use_mg && (o->mg_lines < -1 || o->mg_lines > 1 || o->mg_sweeps < 0))
    return fail(XPBD_ERR_INVALID, "multigrid: mg_lines must be -1, 0 or 1 and mg_sweeps >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  AdjointSweep A;
  st = adjoint_begin(h, p, steps, iters, n_seeds, seed_steps, seed_dx, seed_dv_T, out, s, A);
  if (st != XPBD_OK) return st;
  if (h->use_phases) {   // the solve runs on the per-color records (global vertex indices)
    st = set_alpha(h, p, s, false);
    if (st != XPBD_OK) return st;
  }
  const int V = h->V;
  const size_t V3 = 3 * (size_t)V;
  const int64_t nq = (int64_t)h->n_rec[1] + h->n_rec[2] + h->n_rec[3];
  CU_TRY(h->imp_blocks.ensure(sizeof(double) * (45 * (size_t)nq + 21 * (size_t)h->nm + 1)));
  CU_TRY(h->imp_vec.ensure(sizeof(double) * 6 * std::max<size_t>(V3, 1)));
  CU_TRY(h->imp_dinv.ensure(sizeof(double) * 9 * (size_t)std::max(V, 1)));
  CU_TRY(h->imp_sc.ensure(sizeof(double) * 8));
  double* vb = h->imp_vec.as<double>();
  double *b = vb, *y = vb + V3, *r = vb + 2 * V3, *z = vb + 3 * V3, *pd_dir = vb + 4 * V3, *q = vb + 5 * V3;
  double* dinv = h->imp_dinv.as<double>();
  double* sc = h->imp_sc.as<double>();
  double* partials = h->partials.as<double>();
  double* blocks = h->imp_blocks.as<double>();
  double* mblocks = blocks + 45 * (size_t)nq;   // membranes: 21 per record
  MgPlan mg;
  VcycleGraph vgraph;
  bool use_graph = false;
  if (use_mg) {
    CU_TRY(h->imp_mg.ensure(sizeof(double) * mg_workspace_doubles(o->mg_nx, o->mg_ny, o->mg_lines != 0)));
    mg_carve(mg, h->imp_mg.as<double>(), o->mg_nx, o->mg_ny, o->mg_lines, std::max(o->mg_sweeps, 1));
    use_graph = vgraph.capture(h, mg, ck_x(ck, V, 0), vb + 2 * V3, vb + 3 * V3);   // r -> z
  }
  auto vcycle = [&](const float4* Xm) -> cudaError_t {
    if (use_graph) return vgraph.run(h, s);
    mg_vcycle(h, mg, Xm, r, z, s);
    return cudaSuccess;
  };
  const int64_t boff[4] = {0, 0, h->n_rec[1], (int64_t)h->n_rec[1] + h->n_rec[2]};
  const float* lam = h->lam.as<float>();
  const Collide c = make_collide(p);
  const bool pd = o->pd_project != 0;
  const double tol2 = o->cg_tol * o->cg_tol;
  float4* xbar = h->xbar.as<float4>();
  float4* vbar = h->vbar.as<float4>();
  for (int n = steps - 1; n >= 0 && V > 0; --n) {
    const float4* X = ck_x(ck, V, n + 1);
    const uint8_t* cf = c.flags ? h->cflags.as<uint8_t>() : nullptr;
    const float2* lamc = h->lamc.as<float2>();
    auto spmv = [&](const double* pin, double* qout) {   // q = A pin, color by color
      launch(h, XPBD_K_ADJ_OTHER, V, s, [&] { launch_apply_mass_contacts(X, cf, lamc, c, pd, pin, qout, V, s); });
      for (int col = 0; col < h->K; ++col)
        for (const Seg& cg : h->colors[col])
          for_each_record_seg(h, cg, [&](const Seg& g) {
            if (g.type == SEG_MEMB) {
              launch(h, XPBD_K_ADJ_OTHER, g.count, s, [&] {
                launch_apply_memb(h->d_mrec + g.begin, g.count, mblocks + 21 * (size_t)g.begin, pin, qout, s);
              });
              return;
            }
            const size_t ro = (size_t)h->rec_off[g.type] + g.begin;
            launch(h, XPBD_K_ADJ_OTHER, g.count, s, [&] {
              launch_apply_block(g.type, rec_ptr(h, g.type, g.begin), g.count, X, lam + ro,
                                 blocks + 45 * (size_t)(boff[g.type] + g.begin), pd, pin, qout, s);
            });
          });
    };
    launch(h, XPBD_K_ADJ_OTHER, V, s, [&] { launch_adj_begin(xbar, vbar, 1.f / p->dt, V, s); });
    st = run_step(h, p, n, iters, ck_x(ck, V, n), ck_v(ck, V, n), false, s, true);   // lambda, contacts
    if (st != XPBD_OK) return st;
    launch(h, XPBD_K_ADJ_OTHER, V, s, [&] { launch_xbar_to_b(xbar, b, V, s); });
    for (int t = 1; t < 4; ++t)
      launch(h, XPBD_K_ADJ_OTHER, h->n_rec[t], s, [&] {
        launch_quad_blocks((SegType)t, h->d_rec[t], h->n_rec[t], X, lam + h->rec_off[t],
                           blocks + 45 * (size_t)boff[t], pd, s);
      });
    launch(h, XPBD_K_ADJ_OTHER, h->nm, s, [&] {
      launch_memb_blocks(h->d_mrec, h->nm, X, lam + h->mslot, h->nm, mblocks, pd, s);
    });
    if (use_mg) {   // level-0 stencil, colour by colour, then the coarse levels
      double* A0 = mg.lv[0].A;
      CU_TRY(cudaMemsetAsync(A0, 0, sizeof(double) * kMgBlock * (size_t)V, s));
      CU_TRY(cudaMemsetAsync(sc + 6, 0, sizeof(double), s));
      launch(h, XPBD_K_ADJ_OTHER, V, s, [&] { launch_mg_asm_mass_contacts(X, cf, lamc, c, pd, A0, V, s); });
      for (int col = 0; col < h->K; ++col)
        for (const Seg& cg : h->colors[col])
          for_each_record_seg(h, cg, [&](const Seg& g) {
            if (g.type == SEG_MEMB) {
              launch(h, XPBD_K_ADJ_OTHER, g.count, s, [&] {
                launch_mg_asm_memb(h->d_mrec + g.begin, g.count, mblocks + 21 * (size_t)g.begin, A0, o->mg_nx, V,
                                   sc + 6, s);
              });
              return;
            }
            const size_t ro = (size_t)h->rec_off[g.type] + g.begin;
            launch(h, XPBD_K_ADJ_OTHER, g.count, s, [&] {
              launch_mg_asm_block(g.type, rec_ptr(h, g.type, g.begin), g.count, X, lam + ro,
                                  blocks + 45 * (size_t)(boff[g.type] + g.begin), pd, A0, o->mg_nx, V, sc + 6, s);
            });
          });
      for (int l = 0; l + 1 < mg.levels; ++l)
        launch(h, XPBD_K_ADJ_OTHER, (int64_t)mg.lv[l + 1].nx * mg.lv[l + 1].ny * kMgSlots, s,
               [&] { launch_mg_rap(mg.lv[l], mg.lv[l + 1], l == 0 ? X : nullptr, s); });
      for (int l = 0; l < mg.levels; ++l)
        launch(h, XPBD_K_ADJ_OTHER, (int64_t)mg.lv[l].nx * mg.lv[l].ny, s,
               [&] { launch_mg_dinv(mg.lv[l], l == 0 ? X : nullptr, s); });
      const MgLevel& lc = mg.lv[mg.levels - 1];
      launch(h, XPBD_K_ADJ_OTHER, lc.nx * lc.ny, s,
             [&] { launch_mg_coarse_inverse(lc, mg.levels == 1 ? X : nullptr, mg.cinv, s); });
      if (mg.line_dir)
        launch(h, XPBD_K_ADJ_OTHER, V, s, [&] { launch_mg_line_factor(mg.lv[0], X, mg.line_dir, mg.lfac, s); });
    } else {
      launch(h, XPBD_K_ADJ_OTHER, V, s, [&] { launch_diag_mass_contacts(X, cf, lamc, c, pd, dinv, V, s); });
      for (int col = 0; col < h->K; ++col)
        for (const Seg& cg : h->colors[col])
          for_each_record_seg(h, cg, [&](const Seg& g) {
            if (g.type == SEG_MEMB) {
              launch(h, XPBD_K_ADJ_OTHER, g.count, s, [&] {
                launch_diag_memb(h->d_mrec + g.begin, g.count, mblocks + 21 * (size_t)g.begin, dinv, s);
              });
              return;
            }
            const size_t ro = (size_t)h->rec_off[g.type] + g.begin;
            launch(h, XPBD_K_ADJ_OTHER, g.count, s, [&] {
              launch_diag_block(g.type, rec_ptr(h, g.type, g.begin), g.count, X, lam + ro,
                                blocks + 45 * (size_t)(boff[g.type] + g.begin), pd, dinv, s);
            });
          });
      launch(h, XPBD_K_ADJ_OTHER, V, s, [&] { launch_diag_invert(X, dinv, V, s); });
    }
    LAUNCH_CHECK();
    // preconditioned conjugate gradients on the free vertices
    const int pb = partial_blocks(V);
    if (use_mg) {
      launch(h, XPBD_K_ADJ_OTHER, V, s, [&] { launch_cg_init(X, b, y, r, V, s); });
      CU_TRY(vcycle(X));
      launch_cg_rz(r, z, pd_dir, partials, 3, V, s);
    } else {
      launch_cg_start(X, b, dinv, y, r, z, pd_dir, partials, V, s);
    }
    launch_reduce_partials(partials, pb, 3, sc + 1, false, s);
    double host[4];
    CU_TRY(cudaMemcpyAsync(host, sc + 3, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    if (use_mg && host[3] != 0.0)
      return fail(XPBD_ERR_INVALID, "multigrid: a constraint couples vertices more than two grid cells apart");
    const double bb = host[0];
    int used = 0;
    if (bb > 0.0) {
      for (int it = 0; it < o->cg_max_iters; ++it) {
        const int old_slot = (it & 1) ? 4 : 1, new_slot = (it & 1) ? 1 : 4;
        spmv(pd_dir, q);
        launch_cg_pq(X, pd_dir, q, partials, V, s);
        launch_reduce_partials(partials, pb, 1, sc, false, s);
        if (use_mg) {
          launch_cg_update(sc, old_slot, pd_dir, q, y, r, V, s);
          CU_TRY(vcycle(X));
          launch_cg_rz(r, z, nullptr, partials, 2, V, s);
        } else {
          launch_cg_step(sc, old_slot, pd_dir, q, dinv, y, r, z, partials, V, s);
        }
        launch_reduce_partials(partials, pb, 2, sc + new_slot, false, s);
        launch_cg_dir(sc, old_slot, new_slot, z, pd_dir, V, s);
        used = it + 1;
        if ((it & 3) == 3 || it + 1 == o->cg_max_iters) {
          LAUNCH_CHECK();
          CU_TRY(cudaMemcpyAsync(host, sc + new_slot + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
          CU_TRY(cudaStreamSynchronize(s));
          if (host[0] <= tol2 * bb) break;
        }
      }
    } else {
      CU_TRY(cudaMemsetAsync(y, 0, sizeof(double) * V3, s));
    }
    if (o->cg_iters_out) o->cg_iters_out[n] = used;
    spmv(y, q);   // A y, pinned rows included
    launch(h, XPBD_K_ADJ_OTHER, V, s, [&] { launch_implicit_finish(X, b, y, q, xbar, V, s); });
    for (int t = 0; t < 4; ++t)
      launch(h, XPBD_K_ADJ_OTHER, h->n_rec[t], s, [&] {
        launch_abar((SegType)t, h->d_rec[t], h->n_rec[t], X, lam + h->rec_off[t], y,
                    h->acc.as<double>() + h->rec_off[t], s);
      });
    launch(h, XPBD_K_ADJ_OTHER, h->nm, s, [&] {
      launch_abar_memb(h->d_mrec, h->nm, X, lam + h->mslot, h->nm, y, h->acc.as<double>() + h->mslot, s);
    });
    LAUNCH_CHECK();
    st = adjoint_predict(h, p, n, ck_x(ck, V, n), A, s);
    if (st != XPBD_OK) return st;
  }
  return adjoint_end(h, p, out, s, false);
}

xpbd_status xpbd_adjoint(xpbd_handle h, const xpbd_params* p, int32_t steps, int32_t iters,
                         const float* ck, int32_t n_seeds, const int32_t* seed_steps,
                         const float* seed_dx, const float* seed_dv_T, const xpbd_grads* out,
                         void* stream) {
  g_err.clear();
  NvtxRange nvtx_range("xpbd_adjoint");
  xpbd_status st = check_params(h, p, steps, iters);
  if (st != XPBD_OK) return st;
  if (!ck || !out || n_seeds < 0 || (n_seeds > 0 && (!seed_steps || !seed_dx)))
    return fail(XPBD_ERR_INVALID, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  AdjointSweep A;
  st = adjoint_begin(h, p, steps, iters, n_seeds, seed_steps, seed_dx, seed_dv_T, out, s, A);
  if (st != XPBD_OK) return st;
  for (int n = steps - 1; n >= 0; --n) {
    st = adjoint_step(h, p, n, iters, ck_x(ck, h->V, n), ck_v(ck, h->V, n), A, s);
    if (st != XPBD_OK) return st;
  }
  return adjoint_end(h, p, out, s, h->use_phases);
}

static const char* kClassNames[] = {
    "fwd_dist", "fwd_bend", "fwd_tet_h", "fwd_tet_d", "fwd_contact",
    "replay_dist", "replay_bend", "replay_tet_h", "replay_tet_d", "replay_contact",
    "vjp_dist", "vjp_bend", "vjp_tet_h", "vjp_tet_d", "vjp_contact",
    "predict", "velocity", "adjoint_other", "other", "fwd_phase", "replay_phase", "vjp_phase",
    "fwd_memb", "replay_memb", "vjp_memb"};
static_assert(sizeof(kClassNames) / sizeof(kClassNames[0]) == XPBD_KERNEL_CLASSES, "one name per kernel class");

const char* xpbd_kernel_class_name(int32_t cls) {
  return (cls >= 0 && cls < XPBD_KERNEL_CLASSES) ? kClassNames[cls] : "";
}

xpbd_status xpbd_profile(xpbd_handle h, int32_t enable) {
  if (!h) return fail(XPBD_ERR_INVALID, "null handle");
  CU_TRY(cudaDeviceSynchronize());
  h->prof_on = enable != 0;
  h->timed.clear();
  h->ev_used = 0;
  for (int c = 0; c < XPBD_KERNEL_CLASSES; ++c) {
    h->launches[c] = h->units[c] = 0;
    h->alg_bytes[c] = 0.0;
  }
  return XPBD_OK;
}

xpbd_status xpbd_profile_read(xpbd_handle h, xpbd_kernel_stat* out) {
  if (!h || !out) return fail(XPBD_ERR_INVALID, "null argument");
  CU_TRY(cudaDeviceSynchronize());
  for (int c = 0; c < XPBD_KERNEL_CLASSES; ++c) {
    out[c].launches = h->launches[c];
    out[c].units = h->units[c];
    out[c].ms = 0.0;
    out[c].timed_launches = 0;
    out[c].alg_bytes = h->alg_bytes[c];
  }
  for (const auto& t : h->timed) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      out[t.cls].ms += ms;
      out[t.cls].timed_launches += 1;
    }
  }
  return XPBD_OK;
}


// Same steps and kernels as xpbd_forward, with the working state in g_forward_scratch.
// Nothing there needs clearing between calls: prediction overwrites the positions and the
// contact flags every step, and the first iteration of a step reads no multiplier (it
// starts from lambda = 0), so a call never sees what the previous call left behind.
xpbd_status xpbd_forward_static(xpbd_handle h, const xpbd_params* p, int32_t steps, int32_t iters,
                                const float* x0, const float* v0, float* ck, void* stream) {
  g_err.clear();
  NvtxRange nvtx_range("xpbd_forward_static");
  xpbd_status st = check_params(h, p, steps, iters);
  if (st != XPBD_OK) return st;
  // the one-launch-per-color sweep this entry point runs needs one multiplier slot per
  // constraint and four per membrane (rounded up to a multiple of 4 per block)
  const size_t need = h->color_slots();
  if (h->V > XPBD_STATIC_MAX_VERTICES || need > (size_t)XPBD_STATIC_MAX_CONSTRAINTS)
    return fail(XPBD_ERR_BOUNDS, "xpbd_forward_static supports at most " + std::to_string(XPBD_STATIC_MAX_VERTICES) +
                                     " vertices and " + std::to_string(XPBD_STATIC_MAX_CONSTRAINTS) +
                                     " multiplier slots (one per constraint, four per membrane); this model has " +
                                     std::to_string(h->V) + " vertices and needs " + std::to_string(need) + " slots");
  if (h->V > 0 && (!x0 || !v0 || !ck)) return fail(XPBD_ERR_INVALID, "x0/v0/checkpoints NULL");
  if (h->V == 0) return XPBD_OK;
  void* base = h->static_base;
  if (!base) return fail(XPBD_ERR_CUDA, "the fixed working array has no device address");
  float4* P = reinterpret_cast<float4*>(base);
  float* lam = reinterpret_cast<float*>(static_cast<char*>(base) + kStaticPosBytes);
  float2* lamc = reinterpret_cast<float2*>(static_cast<char*>(base) + kStaticPosBytes + kStaticLamBytes);
  uint8_t* cf = reinterpret_cast<uint8_t*>(static_cast<char*>(base) + kStaticPosBytes + kStaticLamBytes +
                                           kStaticLamcBytes);
  cudaStream_t s = (cudaStream_t)stream;
  st = set_alpha(h, p, s);
  if (st != XPBD_OK) return st;
  float4* ck4 = reinterpret_cast<float4*>(ck);
  launch(h, XPBD_K_OTHER, h->V, s, [&] { launch_init_ckpt(x0, v0, h->d_w, ck4, ck4 + h->V, h->V, s); });
  LAUNCH_CHECK();
  const Collide c = make_collide(p);
  const float inv_dt = 1.f / p->dt;
  for (int n = 0; n < steps; ++n) {
    const float4* xn = ck_x(ck, h->V, n);
    const float4* vn = ck_v(ck, h->V, n);
    launch(h, XPBD_K_PREDICT, h->V, s, [&] {
      launch_predict(xn, vn, P, p->f_global ? p->f_global + 3 * (size_t)n : nullptr, p->f_vertex,
                     p->f_vertex_steps ? p->f_vertex_steps + 3 * (size_t)h->V * n : nullptr, p->dt,
                     p->gravity[0], p->gravity[1], p->gravity[2], c, cf, h->V, s);
    });
    for (int k = 0; k < iters; ++k) {
      for (int col = 0; col < h->K; ++col)
        for (const Seg& g : h->colors[col]) project_segment(h, g, P, k == 0 ? nullptr : lam, lam, nullptr, s);
      if (c.flags)
        launch(h, XPBD_K_FWD_CONTACT, h->V, s,
               [&] { launch_contact(P, cf, h->V, k == 0 ? nullptr : lamc, lamc, nullptr, c, s); });
      LAUNCH_CHECK();
    }
    float4* nx = ck4 + (size_t)2 * h->V * (n + 1);
    launch(h, XPBD_K_VELOCITY, h->V, s,
           [&] { launch_velocity(P, xn, nx, nx + h->V, inv_dt, h->V, h->d_err, s); });
    LAUNCH_CHECK();
  }
  return XPBD_OK;
}

xpbd_status xpbd_exec_info(xpbd_handle h, int32_t* uses_phases, int32_t* n_phases) {
  if (!h) return fail(XPBD_ERR_INVALID, "null handle");
  if (uses_phases) *uses_phases = h->use_phases ? 1 : 0;
  if (n_phases) *n_phases = h->use_phases ? (int32_t)h->phases.size() : h->K;
  return XPBD_OK;
}

xpbd_status xpbd_selftest_wait_timeout(xpbd_handle h, void* stream) {
  g_err.clear();
  if (!h) return fail(XPBD_ERR_INVALID, "null handle");
  if (!h->use_phases || h->phases.empty())
    return fail(XPBD_ERR_INVALID, "the handle runs no phase kernels (exec_mode 1 or a coloring without phases)");
  xpbd_status st = ensure_forward_ws(h);
  if (st != XPBD_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const auto& ph = h->phases[0];
  PhaseLaunch a = phase_args(h, ph);
  a.P = h->P.as<float4>();
  a.lam_in = nullptr;
  a.lam_out = h->lam.as<float>();
  a.wait_cycles = 1ll << 22;   // ~2 ms
  a.no_issue = 1;
  PhaseShape one = ph.shape();
  one.n_groups = 1;            // one CTA: its waits run out one after another
  launch_phase_fwd(a, one, false, s);
  LAUNCH_CHECK();
  return XPBD_OK;
}

xpbd_status xpbd_material_compliance(xpbd_handle h, int32_t n_materials, const int32_t* tet_material,
                                     const float* a, const float* b, float* compliance, void* stream) {
  g_err.clear();
  if (!h || n_materials < 1 || !a || !b || !compliance || (h->nt > 0 && !tet_material))
    return fail(XPBD_ERR_INVALID, "bad argument");
  const size_t off = (size_t)h->nd + h->nb;
  launch(h, XPBD_K_OTHER, h->nt, (cudaStream_t)stream, [&] {
    launch_material_compliance(tet_material, a, b, h->nt, n_materials, compliance + off, compliance + off + h->nt,
                               h->d_err, (cudaStream_t)stream);
  });
  LAUNCH_CHECK();
  return XPBD_OK;
}

xpbd_status xpbd_material_gradient(xpbd_handle h, int32_t n_materials, const int32_t* tet_material, const float* a,
                                   const float* b, const double* d_compliance, double* d_a, double* d_b,
                                   void* stream) {
  g_err.clear();
  if (!h || n_materials < 1 || !a || !b || !d_compliance || (h->nt > 0 && !tet_material))
    return fail(XPBD_ERR_INVALID, "bad argument");
  const size_t off = (size_t)h->nd + h->nb;
  launch(h, XPBD_K_OTHER, n_materials, (cudaStream_t)stream, [&] {
    launch_material_gradient(tet_material, a, b, h->nt, n_materials, d_compliance + off, d_compliance + off + h->nt,
                             d_a, d_b, (cudaStream_t)stream);
  });
  LAUNCH_CHECK();
  return XPBD_OK;
}

xpbd_status xpbd_sync_status(xpbd_handle h, void* stream) {
  if (!h) return fail(XPBD_ERR_INVALID, "null handle");
  CU_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int err = 0;
  CU_TRY(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  CU_TRY(cudaMemset(h->d_err, 0, sizeof(int)));
  if (err & 16)
    return fail(XPBD_ERR_TIMEOUT, "a phase kernel gave up waiting for its own copies in flight before it returned; "
                                  "the CUDA context may be unusable");
  if (err & 4) return fail(XPBD_ERR_TIMEOUT, "a phase kernel gave up waiting for its staged copies");
  if (err & 8) return fail(XPBD_ERR_INVALID, "a tet material id is out of range");
  if (err & 2)
    return fail(XPBD_ERR_NONFINITE, "a compliance value is negative or not finite, or a membrane stiffness is not "
                                    "finite and positive definite");
  if (err & 1) return fail(XPBD_ERR_NONFINITE, "a step produced a non-finite position or velocity");
  return XPBD_OK;
}

}  // extern "C"
