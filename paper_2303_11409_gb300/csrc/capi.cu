// C ABI of the GB300 symmetric-MPS library (U(1), Z_n and several U(1) charges): handles,
// the device arena, and the batched two-site update executor.
//
// One update (Sec. II of arXiv:2303.11409) runs as
//   host planner (K0) -> theta_kernel (K1: Theta'(c) for all middle charges)
//   -> jacobi_svd_kernel (K2: one CTA per sector) -> select_kernel (K3: global
//   top-chi) -> one device-to-host copy of the kept counts -> host layout of the
//   new blocks -> gemm/scatter/lambda kernels (K4/K5: reassembly, renormalisation).
// Any number of independent updates (disjoint site pairs, possibly of different
// handles) share each launch, which is how a whole Trotter layer is one set of
// launches with one host round trip.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mps_internal.h"

using namespace mps;

namespace mps {

cudaError_t DevBuf::reserve(size_t want) {
  if (want <= bytes) return cudaSuccess;
  if (p) { cudaFree(p); p = nullptr; bytes = 0; }
  size_t sz = want + want / 4 + (1 << 20);
  cudaError_t e = cudaMalloc(&p, sz);
  if (e != cudaSuccess) { p = nullptr; return e; }
  bytes = sz;
  return cudaSuccess;
}
void DevBuf::release() { if (p) cudaFree(p); p = nullptr; bytes = 0; }

cudaError_t PinnedBuf::reserve(size_t want) {
  if (want <= bytes) return cudaSuccess;
  if (p) { cudaFreeHost(p); p = nullptr; bytes = 0; }
  size_t sz = want + want / 4 + (1 << 16);
  cudaError_t e = cudaMallocHost(&p, sz);
  if (e != cudaSuccess) { p = nullptr; return e; }
  bytes = sz;
  return cudaSuccess;
}
void PinnedBuf::release() { if (p) cudaFreeHost(p); p = nullptr; bytes = 0; }

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace mps

namespace {

// NVTX range over a scope (no-op unless a profiler is attached): the phases of an update call
// (plan, launch phase 1, host layout, launch phase 2) show up by name in a timeline.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

int fail(mps_s* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

#define CUDA_OR_FAIL(h, x)                                                            \
  do {                                                                                \
    cudaError_t _e = (x);                                                             \
    if (_e != cudaSuccess)                                                            \
      return fail(h, MPS_ECUDA, std::string(#x) + ": " + cudaGetErrorString(_e));     \
  } while (0)

inline int64_t a256(int64_t x) { return (x + 255) & ~int64_t(255); }
inline int cdiv(int a, int b) { return (a + b - 1) / b; }
inline int64_t ldt_of(int Dr) { return (Dr + 3) & ~3; }   // row stride of a product T_m (32-byte rows)

// ---- per-kernel device timing and algorithmic work ------------------------------------
cudaEvent_t pool_event(mps_s* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Adds the device time of completed event pairs; call only when they have completed.
void resolve_pending(mps_s* h) {
  for (auto& p : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) h->kstat[p.kind].ms += ms;
    if (p.pooled) {
      h->event_pool.push_back(p.a);
      h->event_pool.push_back(p.b);
    }
  }
  cudaGetLastError();
  h->pending.clear();
}

// Inside a stream capture a timing event must be an external event-record node of the
// graph; those use one fixed event pair per kernel kind, so that the graph's event nodes
// stay the same from one update call to the next (each kind is timed at most once per
// phase, and pending pairs are read back before the phase that records them again).
cudaError_t ensure_kind_events(mps_s* h) {
  for (int k = 0; k < MPS_K_COUNT; ++k)
    for (int j = 0; j < 2; ++j)
      if (!h->kind_ev[k][j]) {
        cudaError_t e = cudaEventCreate(&h->kind_ev[k][j]);
        if (e != cudaSuccess) return e;
      }
  return cudaSuccess;
}

template <class F>
cudaError_t timed(mps_s* h, int kind, bool nonempty, double flops, double bytes, F&& launch) {
  const bool prof = h->profiling && nonempty;
  cudaEvent_t a = nullptr, b = nullptr;
  const bool pooled = !h->capturing;
  if (prof) {
    if (pooled) {
      a = pool_event(h);
      b = pool_event(h);
      cudaEventRecord(a, h->stream);
    } else {
      a = h->kind_ev[kind][0];
      b = h->kind_ev[kind][1];
      cudaEventRecordWithFlags(a, h->stream, cudaEventRecordExternal);
    }
  }
  cudaError_t e = launch();
  if (prof) {
    if (pooled) cudaEventRecord(b, h->stream);
    else cudaEventRecordWithFlags(b, h->stream, cudaEventRecordExternal);
    h->pending.push_back(PendingTiming{kind, a, b, pooled});
  }
  if (nonempty) {
    KStat& k = h->kstat[kind];
    k.launches++;
    k.flops += flops;
    k.bytes += bytes;
  }
  return e;
}

// Runs one launch phase of an update call.  With graphs on (and a stream that can be
// captured), the phase's copies and kernels are captured into a CUDA graph and replayed
// through the handle's executable graph for that phase, updated in place
// (cudaGraphExecUpdate) when only parameters changed and re-instantiated when the
// topology changed (for example a different number of SVD kernel groups).
template <class F>
cudaError_t run_phase(mps_s* o, int slot, F&& body) {
  Range range(slot == 0 ? "mps.phase1 theta-svd-select" : "mps.phase2 reassembly");
  cudaStream_t st = o->stream;
  if (!o->graphs || st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) return body();
  if (o->profiling) {
    cudaError_t e = ensure_kind_events(o);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  o->capturing = true;
  const cudaError_t eb = body();
  o->capturing = false;
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(st, &g);
  if (eb != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return eb != cudaSuccess ? eb : ee;
  }
  bool updated = false;
  if (o->gexec[slot]) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(o->gexec[slot], g, &info) == cudaSuccess) {
      updated = true;
      o->graph_updates++;
    } else {
      cudaGetLastError();
      cudaGraphExecDestroy(o->gexec[slot]);
      o->gexec[slot] = nullptr;
    }
  }
  if (!updated) {
    e = cudaGraphInstantiate(&o->gexec[slot], g, 0);
    if (e != cudaSuccess) {
      o->gexec[slot] = nullptr;
      cudaGraphDestroy(g);
      return e;
    }
    o->graph_instantiations++;
  }
  cudaGraphDestroy(g);
  o->graph_launches++;
  return cudaGraphLaunch(o->gexec[slot], st);
}

// ---- SVD tile-shape autotuner ----------------------------------------------------------
// Key: the histogram of the batch's cluster-mode sectors over octaves of K = min(m, n),
// counts rounded to powers of two, leaving out octaves that hold under 5% of the batch's
// nominal SVD work (so that a few edge sectors do not split otherwise equal batches).
// On the first batch with a new key (enough SVD work, tuning not frozen) every candidate
// tile shape runs the batch's SVD phase on the same inputs (the phase reads Theta' and
// writes only its own outputs and scratch, so it can be repeated), timed with CUDA
// events, and the default shape runs once more at the end; a candidate replaces the
// default only if it beats the faster of the default's two runs by more than 3%.  The
// choice is stored and used for every later batch with that key.  The table is shared by
// all handles of the process.
struct TuneEntry {
  int best = -1;
  float ms[kTuneCands] = {};
  int64_t hits = 0;
};
std::mutex g_tune_mu;
std::map<std::vector<int>, TuneEntry> g_tune;
int64_t g_tune_runs = 0;
double g_tune_min_flops = 2e10;   // below this an SVD phase is too short to be worth tuning
bool g_tune_frozen = false;       // frozen: unseen keys use the default shape without tuning
int g_tune_force = -1;            // >= 0: every batch uses this candidate (tests, experiments)
constexpr int kTuneDefault = 1;   // svd_tune_candidate(1) is the default shape (bw 6, clusters from 2)

std::vector<int> tune_key(const std::vector<SvdSector>& secs) {
  std::map<int, std::pair<int, double>> hist;   // octave -> (count, nominal work)
  double tot = 0.0;
  for (const SvdSector& S : secs) {
    if (S.mode == kSvdSmem) continue;
    const double a = std::max(S.m, S.n), b = std::min(S.m, S.n);
    const double w = 6.0 * a * b * b + 20.0 * b * b * b;
    auto& e = hist[(int)std::floor(std::log2(b))];
    e.first++;
    e.second += w;
    tot += w;
  }
  std::vector<int> key;
  for (const auto& kv : hist) {
    if (kv.second.second < 0.05 * tot) continue;
    int q = 0;
    for (int c = kv.second.first; c; c >>= 1) ++q;     // floor(log2(count)) + 1
    key.push_back(kv.first);
    key.push_back(q);
  }
  return key;
}

// Number of occupation strings of n sites (0..d-1 each) summing to q, saturated.
std::vector<std::vector<double>> config_counts(int L, int d, int N) {
  std::vector<std::vector<double>> W(L + 1, std::vector<double>(N + 1, 0.0));
  W[0][0] = 1.0;
  for (int n = 1; n <= L; ++n)
    for (int q = 0; q <= N; ++q) {
      double s = 0.0;
      for (int i = 0; i < d && i <= q; ++i) s += W[n - 1][q - i];
      W[n][q] = std::min(s, 1e30);
    }
  return W;
}

// A host-side bump allocator over a staging buffer plus the matching device offsets.
struct Stager {
  char* host; int64_t size = 0;
  template <typename T> int64_t put(const T* src, int64_t count) {
    int64_t off = size;
    std::memcpy(host + off, src, sizeof(T) * count);
    size = a256(off + (int64_t)sizeof(T) * count);
    return off;
  }
};

struct Req {
  mps_s* h; int site; const double* gate; int chi; double cutoff;
  int status = MPS_OK; double trunc = 0.0;
};

// Per-update scratch bookkeeping of one batch.
struct UpdWork {
  UpdatePlan plan;
  std::vector<int64_t> theta_off, y_off, sig_off;   // byte offsets into the workspace per sector
  int sel_first = 0;                                // index of the first sector in the select arrays
  int64_t gate_off = 0;                             // byte offset of this update's staged gate
  double cut_est = 0.0;                             // the bond's previous relative cut (0: none)
  double chi_level = 0.0;                           // the deflation level applied to it
};

int run_batch(std::vector<Req>& reqs, mps_s* owner) {
  if (reqs.empty()) return MPS_OK;
  cudaStream_t st = owner->stream;
  const int nreq = (int)reqs.size();
  std::vector<UpdWork> W(nreq);
  {   // one more update call on every handle of the batch
    std::vector<mps_s*> seen;
    for (const Req& r : reqs)
      if (std::find(seen.begin(), seen.end(), r.h) == seen.end()) {
        seen.push_back(r.h);
        r.h->calls++;
      }
  }

  Range batch_range("mps.update_call");
  // ---- K0: plan every update and size the workspace --------------------------------
  int64_t ws = 0;
  int n_sec_total = 0, n_tiles = 0, n_tasks = 0, max_tri = 0;
  // reduced-precision updates ([0] TF32, [1] BF16x3): shadow slots, shadow tiles, products,
  // gate-mix tasks, and the complex64 buffer of the products T_m
  int64_t tc_slots[2] = {0, 0}, tc_shtiles[2] = {0, 0}, tc_jobs[2] = {0, 0}, tc_mix[2] = {0, 0};
  int64_t tc_shtasks[2] = {0, 0}, tc_slots2[2] = {0, 0}, tc_shtiles2[2] = {0, 0}, tc_jobs2[2] = {0, 0};
  int64_t tc_shtasks2[2] = {0, 0};
  int64_t tbuf_bytes = 0;
  bool any_tc = false;
  int64_t theta_bytes_begin = 0, theta_bytes_end = 0;
  int64_t scatter_bound = 0, gemm_tiles_bound = 0, gemm_tasks_bound = 0, lam_bound = 0;
  for (int u = 0; u < nreq; ++u) {
    mps_s* h = reqs[u].h;
    const int s = reqs[u].site;
    plan_update(h->bonds[s], h->bonds[s + 1], h->bonds[s + 2], h->rule, W[u].plan);
    if (h->chi_deflate > 0.0 && (int)h->cut_est.size() == h->L + 1) {
      W[u].cut_est = h->cut_est[s + 1];
      // a cut recorded by the previous update call on this handle (the same layer kind in a row,
      // as the two odd half-step layers of consecutive Strang steps) is a close estimate; an
      // older one has seen the neighbouring bonds change in between, so its level is 30x lower
      // (a redo then needs a 30x larger drop of the cut)
      const bool fresh = (int)h->cut_call.size() == h->L + 1 && h->calls - h->cut_call[s + 1] <= 1;
      W[u].chi_level = fresh ? h->chi_deflate : h->chi_deflate / 30.0;
    }
    max_tri = std::max<int>(max_tri, (int)W[u].plan.triple_l.size());
    n_sec_total += (int)W[u].plan.sectors.size();
    if (W[u].plan.sectors.empty()) return fail(owner, MPS_EINVAL, "update has no charge sectors");
  }
  // Theta' region first (one memset), then Y, sigma, Jacobi scratch, gates.
  theta_bytes_begin = 0;
  for (int u = 0; u < nreq; ++u)
    for (auto& e : W[u].plan.sectors) {
      W[u].theta_off.push_back(ws);
      ws = a256(ws + 16LL * e.rows * e.cols);
    }
  theta_bytes_end = ws;
  for (int u = 0; u < nreq; ++u)
    for (auto& e : W[u].plan.sectors) {
      const int k = std::min(e.rows, e.cols);
      W[u].y_off.push_back(ws);
      ws = a256(ws + 16LL * e.cols * k);
      W[u].sig_off.push_back(ws);
      ws = a256(ws + 8LL * k);
      scatter_bound += (int64_t)e.ri.size();
      gemm_tasks_bound += (int64_t)e.li.size();
      lam_bound += 1 + (e.contiguous ? 0 : (int64_t)e.li.size());
      for (int i : e.li) {
        const int Dl = reqs[u].h->bonds[reqs[u].site].dim[i];
        gemm_tiles_bound += (int64_t)((Dl + kTile - 1) / kTile) * ((k + kTile - 1) / kTile);
      }
    }
  // Jacobi scratch: one-CTA sectors live in shared memory, cluster sectors in L2
  SvdScratchLayout JL;
  {
    std::vector<int> sm, sn;
    for (int u = 0; u < nreq; ++u)
      for (auto& e : W[u].plan.sectors) { sm.push_back(e.rows); sn.push_back(e.cols); }
    svd_layout((int)sm.size(), sm.data(), sn.data(), JL);
  }
  const int64_t jac_base = ws;
  ws = a256(ws + JL.total);
  int64_t gates_bytes = 0;                      // gate blocks of every update (d may differ)
  for (int u = 0; u < nreq; ++u) gates_bytes += a256(16LL * reqs[u].h->rule.gate_len());
  const int64_t kept_off = ws; ws = a256(ws + 4LL * n_sec_total);
  const int64_t status_off = ws; ws = a256(ws + 4LL * n_sec_total);
  const int64_t res_off = ws; ws = a256(ws + (int64_t)sizeof(SelectResult) * nreq);
  // the left lambdas of sectors whose rows are not one run of the bond table (several-U(1)
  // handles), gathered so that the SVD reads its row scale contiguously
  int64_t gather_rows = 0, n_gather = 0;
  for (int u = 0; u < nreq; ++u)
    for (auto& e : W[u].plan.sectors)
      if (!e.contiguous) { gather_rows += e.rows; n_gather += (int64_t)e.li.size(); }
  const int64_t gath_off = ws; ws = a256(ws + 8LL * gather_rows);
  const int64_t desc_off = ws;   // phase-1 descriptors start here; phase-2 reuses the same region

  // count theta tasks to size descriptors
  for (int u = 0; u < nreq; ++u) {
    mps_s* h = reqs[u].h;
    const int s = reqs[u].site, d = h->d;
    const bool tc = h->precision != MPS_FP64;
    any_tc = any_tc || tc;
    const BondTable &Lb = h->bonds[s], &Mb = h->bonds[s + 1], &Rb = h->bonds[s + 2];
    const ChargeRule& rule = h->rule;
    for (int li = 0; li < Lb.size(); ++li)
      for (int ri = 0; ri < Rb.size(); ++ri) {
        const int l = Lb.charge[li], r = Rb.charge[ri];
        if (rule.pair(l, r) < 0) continue;
        int nm = 0;
        for (int mi = 0; mi < Mb.size(); ++mi) {
          const int m = Mb.charge[mi];
          if (rule.phys(l, m) >= 0 && rule.phys(m, r) >= 0) ++nm;
        }
        if (nm == 0) continue;
        if (tc) {   // one product T_m per middle charge m, then the gate mix over m
          const int p = h->precision == MPS_BF16X3;
          tc_jobs[p] += (int64_t)nm * cdiv(Lb.dim[li], kShRows) * cdiv(Rb.dim[ri], kShTileN);
          tbuf_bytes += (int64_t)nm * a256(8LL * Lb.dim[li] * ldt_of(Rb.dim[ri]));
          tc_mix[p] += 1;
          continue;
        }
        n_tasks++;
        n_tiles += ((Lb.dim[li] + kTile - 1) / kTile) * ((Rb.dim[ri] + kTile - 1) / kTile);
      }
    if (tc) {   // shadow tiles: site s as A operand, site s+1 as B operand, Theta' as reassembly A
      const int p = h->precision == MPS_BF16X3, KC = sh_kc(h->precision), TPK = sh_tiles_per_k(h->precision);
      for (const SiteBlock& b : h->sites[s].blocks) {
        const int64_t t = (int64_t)cdiv(b.Dl, kShRows) * cdiv(b.Dm, KC);
        tc_shtiles[p] += t; tc_slots[p] += t * TPK; tc_shtasks[p] += 1;
      }
      for (const SiteBlock& b : h->sites[s + 1].blocks) {
        const int64_t t = (int64_t)cdiv(b.Dm, kShTileN) * cdiv(b.Dl, KC);
        tc_shtiles[p] += t; tc_slots[p] += t * TPK; tc_shtasks[p] += 1;
      }
      for (const SectorPlanEntry& e : W[u].plan.sectors) {
        const int k = std::min(e.rows, e.cols), ktn = cdiv(e.cols, KC);
        for (int i : e.li) {
          tc_slots[p] += (int64_t)cdiv(Lb.dim[i], kShRows) * ktn * TPK;
          tc_jobs2[p] += (int64_t)cdiv(Lb.dim[i], kShRows) * cdiv(k, kShTileN);
        }
        const int64_t ty = (int64_t)cdiv(k, kShTileN) * ktn;   // Y(c) as reassembly B operand
        tc_slots2[p] += ty * TPK; tc_shtiles2[p] += ty; tc_shtasks2[p] += 1;
      }
    }
  }
  const int64_t phase1_desc = a256((int64_t)sizeof(ThetaTask) * n_tasks) + a256(sizeof(TileRef) * (int64_t)n_tiles) +
                              (owner->autotune ? kTuneCands : 1) * a256((int64_t)sizeof(SvdSector) * n_sec_total) +
                              a256((int64_t)sizeof(SelectSector) * n_sec_total) +
                              a256((int64_t)sizeof(SelectTask) * nreq) + gates_bytes +
                              a256((int64_t)sizeof(ShadowTask) * (tc_shtasks[0] + tc_shtasks[1])) +
                              a256((int64_t)sizeof(ShadowTile) * (tc_shtiles[0] + tc_shtiles[1])) +
                              a256((int64_t)sizeof(TmaJob) * (tc_jobs[0] + tc_jobs[1])) +
                              a256((int64_t)sizeof(MixTask) * (tc_mix[0] + tc_mix[1])) +
                              a256((int64_t)sizeof(LambdaTask) * n_gather) + 4 * 256;
  const int64_t phase2_desc = a256((int64_t)sizeof(LambdaTask) * lam_bound) +
                              a256((int64_t)sizeof(ScatterTask) * scatter_bound) +
                              a256((int64_t)sizeof(GemmTask) * gemm_tasks_bound) +
                              a256((int64_t)sizeof(TileRef) * gemm_tiles_bound) +
                              a256((int64_t)sizeof(ShadowTask) * (tc_shtasks2[0] + tc_shtasks2[1])) +
                              a256((int64_t)sizeof(ShadowTile) * (tc_shtiles2[0] + tc_shtiles2[1])) +
                              a256((int64_t)sizeof(TmaJob) * (tc_jobs2[0] + tc_jobs2[1])) + 4 * 256;
  const int64_t desc_bytes = std::max(phase1_desc, phase2_desc);
  ws = desc_off + desc_bytes;
  // the products T_m, then the shadow slots of each precision (1024-byte aligned once the
  // workspace base is known: 1 KB of slack each); phase 2 appends Y's slots to phase 1's
  const int64_t tbuf_off = ws;
  ws = a256(ws + tbuf_bytes);
  int64_t slot_off[2];
  for (int p = 0; p < 2; ++p) {
    slot_off[p] = ws;
    if (tc_slots[p] + tc_slots2[p] > 0) ws = a256(ws + (tc_slots[p] + tc_slots2[p]) * kShTileBytes + 1024);
  }

  CUDA_OR_FAIL(owner, cudaEventSynchronize(owner->staged));   // pin_in free again
  {
    cudaError_t e = owner->work.reserve((size_t)ws);
    if (e != cudaSuccess) return fail(owner, MPS_ENOMEM, std::string("workspace: ") + cudaGetErrorString(e));
    e = owner->pin_in.reserve((size_t)std::max<int64_t>(desc_bytes, 1) + 4096);
    if (e != cudaSuccess) return fail(owner, MPS_ENOMEM, "pinned staging");
    e = owner->pin_out.reserve((size_t)a256(res_off + (int64_t)sizeof(SelectResult) * nreq - kept_off) + 4096);
    if (e != cudaSuccess) return fail(owner, MPS_ENOMEM, "pinned staging");
    if (any_tc && !owner->tc_flag) {
      e = cudaMalloc(&owner->tc_flag, 256);
      if (e == cudaSuccess) e = cudaMemsetAsync(owner->tc_flag, 0, 256, st);
      if (e != cudaSuccess) return fail(owner, MPS_ENOMEM, "tensor-core error flag");
    }
  }
  char* base = (char*)owner->work.p;
  auto dptr = [&](int64_t off) { return base + off; };
  // gates go first into the staging area; tasks point at their device copies
  Stager sg{(char*)owner->pin_in.p};
  for (int u = 0; u < nreq; ++u) W[u].gate_off = desc_off + sg.put(reqs[u].gate, 2 * reqs[u].h->rule.gate_len());

  // ---- build phase-1 descriptors ------------------------------------------------------
  std::vector<ThetaTask> tasks; tasks.reserve(n_tasks);
  std::vector<TileRef> tiles; tiles.reserve(n_tiles);
  // reduced-precision updates, per precision ([0] TF32, [1] BF16x3)
  std::vector<ShadowTask> shtask[2];
  std::vector<ShadowTile> shtile[2];
  std::vector<TmaJob> tjobs[2];
  std::vector<MixTask> mixes[2];
  int64_t slot_next[2] = {0, 0}, tbuf_next = 0;
  std::vector<std::vector<std::vector<int64_t>>> ra_slot(nreq);   // [u][sector][l - l0]: reassembly A slots
  char* slot_base[2];
  for (int p = 0; p < 2; ++p)
    slot_base[p] = reinterpret_cast<char*>(((uintptr_t)(base + slot_off[p]) + 1023) & ~(uintptr_t)1023);
  double tc_th_flops = 0, tc_prod_flops = 0;
  std::vector<SvdSector> svd; svd.reserve(n_sec_total);
  std::vector<SelectSector> selsec; selsec.reserve(n_sec_total);
  std::vector<SelectTask> seltask; seltask.reserve(nreq);
  std::vector<LambdaTask> gath;
  int64_t gath_next = 0;
  int sec_global = 0;
  for (int u = 0; u < nreq; ++u) {
    mps_s* h = reqs[u].h;
    const int s = reqs[u].site, d = h->d;
    const BondTable &Lb = h->bonds[s], &Mb = h->bonds[s + 1], &Rb = h->bonds[s + 2];
    const SiteTable &SL = h->sites[s], &SR = h->sites[s + 1];
    const double2* slotL = h->slot_ptr(s, h->cur[s]);
    const double2* slotR = h->slot_ptr(s + 1, h->cur[s + 1]);
    const UpdatePlan& P = W[u].plan;
    // sector index by charge
    auto sector_of = [&](int c) -> int {
      int lo = 0, hi = (int)P.sectors.size() - 1;
      while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (P.sectors[mid].c == c) return mid;
        if (P.sectors[mid].c < c) lo = mid + 1; else hi = mid - 1;
      }
      return -1;
    };
    const bool tc = h->precision != MPS_FP64;
    const int tp = h->precision == MPS_BF16X3;
    const int KC = sh_kc(h->precision), TPK = sh_tiles_per_k(h->precision);
    const ChargeRule& rule = h->rule;
    std::vector<int64_t> a_slot, b_slot;
    if (tc) {
      // site s as A tiles (rows of l, K over m), site s+1 as B tiles (columns of r, K over m)
      for (const SiteBlock& b : SL.blocks) {
        a_slot.push_back(slot_next[tp]);
        ShadowTask Tk{slotL + b.off, b.Dm, 1, b.Dl, b.Dm, slot_next[tp], cdiv(b.Dm, KC), 0};
        const int id = (int)shtask[tp].size();
        shtask[tp].push_back(Tk);
        for (int it = 0; it < cdiv(b.Dl, kShRows); ++it)
          for (int kt = 0; kt < Tk.kt_n; ++kt) shtile[tp].push_back(ShadowTile{id, it, kt});
        slot_next[tp] += (int64_t)cdiv(b.Dl, kShRows) * Tk.kt_n * TPK;
      }
      for (const SiteBlock& b : SR.blocks) {
        b_slot.push_back(slot_next[tp]);
        ShadowTask Tk{slotR + b.off, 1, b.Dm, b.Dm, b.Dl, slot_next[tp], cdiv(b.Dl, KC), 1};
        const int id = (int)shtask[tp].size();
        shtask[tp].push_back(Tk);
        for (int it = 0; it < cdiv(b.Dm, kShTileN); ++it)
          for (int kt = 0; kt < Tk.kt_n; ++kt) shtile[tp].push_back(ShadowTile{id, it, kt});
        slot_next[tp] += (int64_t)cdiv(b.Dm, kShTileN) * Tk.kt_n * TPK;
      }
      // Theta'(c) as the reassembly's A operand: block (l, c) = its rows of l, K = its columns
      ra_slot[u].resize(P.sectors.size());
      for (size_t si = 0; si < P.sectors.size(); ++si) {
        const SectorPlanEntry& E = P.sectors[si];
        for (int i : E.li) {
          ra_slot[u][si].push_back(slot_next[tp]);
          slot_next[tp] += (int64_t)cdiv(Lb.dim[i], kShRows) * cdiv(E.cols, KC) * TPK;
        }
      }
    }
    for (int li = 0; li < Lb.size(); ++li)
      for (int ri = 0; ri < Rb.size(); ++ri) {
        const int l = Lb.charge[li], r = Rb.charge[ri];
        const int n = rule.pair(l, r);           // the gate block of this pair
        if (n < 0) continue;
        ThetaTask T;
        std::memset(&T, 0, sizeof(T));
        T.nm = 0;
        for (int mi = 0; mi < Mb.size(); ++mi) {
          const int m = Mb.charge[mi];
          if (rule.phys(l, m) < 0 || rule.phys(m, r) < 0) continue;
          const int bl = SL.find(l, m), br = SR.find(m, r);
          if (bl < 0 || br < 0) return fail(owner, MPS_EINVAL, "internal: missing block");
          T.A[T.nm] = slotL + SL.blocks[bl].off;
          T.B[T.nm] = slotR + SR.blocks[br].off;
          T.Dm[T.nm] = Mb.dim[mi];
          T.gi[T.nm] = rule.gpos(n, rule.phys(l, m));
          T.nm++;
        }
        if (T.nm == 0) continue;
        T.nc = 0;
        int cs[MPS_MAX_D];
        const int ncs = rule.mids(l, r, cs);
        for (int ci = 0; ci < ncs; ++ci) {
          const int c = cs[ci];
          const int si = sector_of(c);
          if (si < 0) return fail(owner, MPS_EINVAL, "internal: missing sector");
          const SectorPlanEntry& E = P.sectors[si];
          const int roff = E.row_off(li);
          const int coff = E.col_off(ri);
          if (roff < 0 || coff < 0) return fail(owner, MPS_EINVAL, "internal: sector layout");
          T.out[T.nc] = reinterpret_cast<double2*>(dptr(W[u].theta_off[si])) + (int64_t)roff * E.cols + coff;
          T.ldo[T.nc] = E.cols;
          T.go[T.nc] = rule.gpos(n, rule.phys(l, c));
          T.nc++;
        }
        T.gate = reinterpret_cast<const double2*>(dptr(W[u].gate_off)) + rule.block_off(n);
        T.sn = rule.sn(n);
        T.Dl = Lb.dim[li];
        T.Dr = Rb.dim[ri];
        if (tc) {
          // T_i = B[s][l, m_i] . B[s+1][m_i, r] on the tensor cores (one product per middle
          // charge), then Theta'(c)[l, r] = sum_i G_n[c, m_i] T_i in mix_kernel
          MixTask X;
          std::memset(&X, 0, sizeof(X));
          X.nm = T.nm; X.nc = T.nc; X.gate = T.gate; X.sn = T.sn; X.Dl = T.Dl; X.Dr = T.Dr;
          X.ldt = (int)ldt_of(T.Dr);
          int i = 0;
          for (int mi = 0; mi < Mb.size(); ++mi) {
            const int m = Mb.charge[mi];
            if (rule.phys(l, m) < 0 || rule.phys(m, r) < 0) continue;
            const int bl = SL.find(l, m), br = SR.find(m, r);
            float2* Tm = reinterpret_cast<float2*>(dptr(tbuf_off + tbuf_next));
            tbuf_next += a256(8LL * T.Dl * X.ldt);
            X.T[i] = Tm;
            X.gi[i] = T.gi[i];
            const int ktn = cdiv(T.Dm[i], KC);
            for (int rt = 0; rt < cdiv(T.Dl, kShRows); ++rt)
              for (int ct = 0; ct < cdiv(T.Dr, kShTileN); ++ct) {
                TmaJob J;
                J.a0 = a_slot[bl] + (int64_t)rt * ktn * TPK;
                J.b0 = b_slot[br] + (int64_t)ct * ktn * TPK;
                J.kt_n = ktn;
                J.M = std::min(kShRows, T.Dl - rt * kShRows);
                J.N = std::min(kShTileN, T.Dr - ct * kShTileN);
                J.mode = 0;
                J.alpha = 1.0f;
                J.C = Tm + (int64_t)rt * kShRows * X.ldt + ct * kShTileN;
                J.ldc = X.ldt;
                tjobs[tp].push_back(J);
              }
            tc_prod_flops += 8.0 * T.Dl * T.Dm[i] * T.Dr;
            ++i;
          }
          for (int k = 0; k < T.nc; ++k) {
            const int c = cs[k];
            const int si = sector_of(c);
            const SectorPlanEntry& E = P.sectors[si];
            X.out[k] = T.out[k];
            X.ldo[k] = T.ldo[k];
            X.go[k] = T.go[k];
            int pos = 0;
            while (E.li[pos] != li) ++pos;
            X.sh0[k] = ra_slot[u][si][pos];
            X.sh_ktn[k] = cdiv(E.cols, KC);
            X.coff[k] = E.col_off(ri);
          }
          mixes[tp].push_back(X);
          tc_th_flops += 8.0 * T.nm * T.nc * T.Dl * T.Dr;
          continue;
        }
        const int task_id = (int)tasks.size();
        tasks.push_back(T);
        for (int ti = 0; ti < (T.Dl + kTile - 1) / kTile; ++ti)
          for (int tj = 0; tj < (T.Dr + kTile - 1) / kTile; ++tj) tiles.push_back(TileRef{task_id, ti, tj});
      }
    W[u].sel_first = (int)selsec.size();
    for (size_t si = 0; si < P.sectors.size(); ++si, ++sec_global) {
      const SectorPlanEntry& E = P.sectors[si];
      SvdSector S = {};
      S.theta = reinterpret_cast<const double2*>(dptr(W[u].theta_off[si]));
      if (E.contiguous) {
        S.rowscale = h->lambda_ptr(s) + Lb.off[E.li.front()];
      } else {
        double* g = reinterpret_cast<double*>(dptr(gath_off)) + gath_next;
        for (size_t a = 0; a < E.li.size(); ++a)
          gath.push_back(LambdaTask{h->lambda_ptr(s) + Lb.off[E.li[a]], g + E.loff[a], Lb.dim[E.li[a]], 1.0});
        gath_next += E.rows;
        S.rowscale = g;
      }
      S.m = E.rows;
      S.n = E.cols;
      S.floor_rel = kDeflateRel * reqs[u].cutoff;
      S.floor_abs = W[u].chi_level * W[u].cut_est;
      svd_fill_scratch(S, JL, sec_global, dptr(jac_base));
      S.sigma = reinterpret_cast<double*>(dptr(W[u].sig_off[si]));
      S.Y = reinterpret_cast<double2*>(dptr(W[u].y_off[si]));
      S.status = reinterpret_cast<int*>(dptr(status_off)) + sec_global;
      svd.push_back(S);
      selsec.push_back(SelectSector{S.sigma, std::min(E.rows, E.cols)});
    }
    seltask.push_back(SelectTask{W[u].sel_first, (int)selsec.size(), reqs[u].chi, reqs[u].cutoff});
  }
  // ---- SVD tile shape: the tuned choice for this sector-size histogram, or a tuning run ---
  // group the sectors by SVD kernel and cluster size, most expensive first inside a group
  double svd_flops = 0, svd_bytes = 0, sel_bytes = 0;
  for (const SvdSector& S : svd) {
    const double a = std::max(S.m, S.n), b = std::min(S.m, S.n);
    svd_flops += 4.0 * (6.0 * a * b * b + 20.0 * b * b * b);
    svd_bytes += 16.0 * S.m * S.n + 16.0 * S.n * b + 8.0 * b + 8.0 * S.m;
    sel_bytes += 8.0 * b;
  }
  std::vector<int> tkey;
  int n_cand = 1, chosen = -1;       // n_cand > 1: this batch runs every candidate
  int forced;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    forced = g_tune_force;
  }
  if (forced >= 0) {
    chosen = forced;
  } else if (owner->autotune) {
    tkey = tune_key(svd);
    if (!tkey.empty()) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(tkey);
      if (it != g_tune.end() && it->second.best >= 0) {
        chosen = it->second.best;
        it->second.hits++;
      } else if (!g_tune_frozen && svd_flops >= g_tune_min_flops) {
        n_cand = kTuneCands;
      }
    }
  }
  std::vector<std::vector<SvdSector>> svd_sorted(n_cand, svd);
  std::vector<std::vector<SvdGroup>> svd_groups(n_cand);
  for (int c = 0; c < n_cand; ++c) {
    const SvdTune tune = n_cand > 1 ? svd_tune_candidate(c) : (chosen >= 0 ? svd_tune_candidate(chosen) : SvdTune());
    CUDA_OR_FAIL(owner, svd_group(svd_sorted[c], svd_groups[c], tune));
  }

  // ---- descriptors into the staging buffer (uploaded in one copy) ---------------------
  const int64_t o_tasks = sg.put(tasks.data(), (int64_t)tasks.size());
  const int64_t o_tiles = sg.put(tiles.data(), (int64_t)tiles.size());
  std::vector<int64_t> o_svd(n_cand);
  for (int c = 0; c < n_cand; ++c) o_svd[c] = sg.put(svd_sorted[c].data(), (int64_t)svd_sorted[c].size());
  const int64_t o_selsec = sg.put(selsec.data(), (int64_t)selsec.size());
  const int64_t o_seltask = sg.put(seltask.data(), (int64_t)seltask.size());
  const int64_t o_gath = sg.put(gath.data(), (int64_t)gath.size());
  int64_t o_shtask[2], o_shtile[2], o_tjobs[2], o_mix[2];
  double sh_bytes = 0, prod_bytes = 0;
  for (int p = 0; p < 2; ++p) {
    // the longest K first: a static round-robin over the persistent CTAs then balances
    std::stable_sort(tjobs[p].begin(), tjobs[p].end(),
                     [](const TmaJob& a, const TmaJob& b) { return a.kt_n > b.kt_n; });
    // every slot a job or a shadow tile touches lies inside the buffer its tensor map covers
    const int64_t tpk = p ? 2 : 1, lim = tc_slots[p] + tc_slots2[p];
    if (slot_next[p] > tc_slots[p]) return fail(owner, MPS_EINVAL, "internal: shadow slot bound exceeded");
    for (const TmaJob& j : tjobs[p])
      if (j.a0 < 0 || j.b0 < 0 || j.a0 + j.kt_n * tpk > lim || j.b0 + j.kt_n * tpk > lim)
        return fail(owner, MPS_EINVAL, "internal: tensor-core job outside the shadow buffer");
    o_shtask[p] = sg.put(shtask[p].data(), (int64_t)shtask[p].size());
    o_shtile[p] = sg.put(shtile[p].data(), (int64_t)shtile[p].size());
    o_tjobs[p] = sg.put(tjobs[p].data(), (int64_t)tjobs[p].size());
    o_mix[p] = sg.put(mixes[p].data(), (int64_t)mixes[p].size());
    for (const ShadowTask& t : shtask[p]) sh_bytes += 16.0 * t.n_i * t.K;   // FP64 operands read
    sh_bytes += (double)slot_next[p] * kShTileBytes;                       // slots written (and zeroed)
    for (const TmaJob& j : tjobs[p]) prod_bytes += 8.0 * j.M * j.N;        // T_m written
  }
  if (sg.size > desc_bytes) return fail(owner, MPS_EINVAL, "internal: descriptor bound exceeded");

  // ---- algorithmic work of the three kernels (flops: complex multiply-add = 8) -------
  double th_flops = 0, th_bytes = (double)(theta_bytes_end - theta_bytes_begin);   // Theta' written
  for (const ThetaTask& T : tasks) {
    for (int i = 0; i < T.nm; ++i) th_flops += 8.0 * T.Dl * T.Dm[i] * T.Dr;
    th_flops += 8.0 * T.nm * T.nc * T.Dl * T.Dr;
  }
  th_flops += tc_th_flops;
  for (int p = 0; p < 2; ++p)
    for (const MixTask& x : mixes[p]) th_bytes += 8.0 * x.nm * x.Dl * x.Dr;    // T_m read by the mix
  for (int u = 0; u < nreq; ++u) {
    const int s = reqs[u].site;
    th_bytes += 16.0 * (double)(reqs[u].h->sites[s].nnz + reqs[u].h->sites[s + 1].nnz);
  }
  const int64_t out_bytes = res_off + (int64_t)sizeof(SelectResult) * nreq - kept_off;
  int* tc_err_host = reinterpret_cast<int*>((char*)owner->pin_out.p + a256(out_bytes));
  *tc_err_host = 0;

  // ---- phase 1: upload, K1 (Theta'), K2 (SVD), K3 (top-chi), read-back ------------------
  auto upload_and_theta = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(dptr(desc_off), owner->pin_in.p, sg.size, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(dptr(theta_bytes_begin), 0, theta_bytes_end - theta_bytes_begin, st);
    if (e != cudaSuccess) return e;
    const int precs[2] = {MPS_TF32, MPS_BF16X3};
    const bool any_tc_work = !tjobs[0].empty() || !tjobs[1].empty();
    for (int p = 0; p < 2 && e == cudaSuccess; ++p)   // padding rows and K of every slot are zero
      if (slot_next[p] > 0) e = cudaMemsetAsync(slot_base[p], 0, (size_t)(slot_next[p] * kShTileBytes), st);
    // products a failed (timed-out) GEMM leaves unwritten read as zero, not as stale memory
    if (e == cudaSuccess && tbuf_next > 0) e = cudaMemsetAsync(dptr(tbuf_off), 0, (size_t)tbuf_next, st);
    if (e == cudaSuccess)
      e = timed(owner, MPS_K_SHADOW, any_tc_work, 0.0, sh_bytes, [&] {
        cudaError_t e2 = cudaSuccess;
        for (int p = 0; p < 2 && e2 == cudaSuccess; ++p)
          e2 = launch_shadow(precs[p], reinterpret_cast<ShadowTask*>(dptr(desc_off + o_shtask[p])),
                             reinterpret_cast<ShadowTile*>(dptr(desc_off + o_shtile[p])), (int)shtile[p].size(),
                             slot_base[p], st);
        return e2;
      });
    if (e == cudaSuccess)
      e = timed(owner, MPS_K_TCGEMM, any_tc_work, tc_prod_flops, sh_bytes + prod_bytes, [&] {
        cudaError_t e2 = cudaSuccess;
        for (int p = 0; p < 2 && e2 == cudaSuccess; ++p)
          e2 = launch_tma_zgemm(precs[p], reinterpret_cast<TmaJob*>(dptr(desc_off + o_tjobs[p])),
                                (int)tjobs[p].size(), slot_base[p], tc_slots[p] + tc_slots2[p], owner->tc_flag, st);
        return e2;
      });
    if (e != cudaSuccess) return e;
    if (!gath.empty())
      e = timed(owner, MPS_K_LAMBDA, true, 0.0, 16.0 * (double)gather_rows, [&] {
        return launch_lambda(reinterpret_cast<LambdaTask*>(dptr(desc_off + o_gath)), (int)gath.size(), st);
      });
    if (e != cudaSuccess) return e;
    const bool any_theta = !tiles.empty() || !mixes[0].empty() || !mixes[1].empty();
    return timed(owner, MPS_K_THETA, any_theta, th_flops, th_bytes, [&] {
      cudaError_t e2 = launch_theta(reinterpret_cast<ThetaTask*>(dptr(desc_off + o_tasks)),
                                    reinterpret_cast<TileRef*>(dptr(desc_off + o_tiles)), (int)tiles.size(), st);
      for (int p = 0; p < 2 && e2 == cudaSuccess; ++p)
        e2 = launch_mix(precs[p], reinterpret_cast<MixTask*>(dptr(desc_off + o_mix[p])), (int)mixes[p].size(),
                        slot_base[p], st);
      return e2;
    });
  };
  auto svd_launch = [&](int c) -> cudaError_t {   // one or more kernels
    const SvdSector* d_svd = reinterpret_cast<SvdSector*>(dptr(desc_off + o_svd[c]));
    return launch_svd_groups(d_svd, svd_groups[c], st, owner->side, kSvdSideStreams, owner->fork, owner->join,
                             owner->sweep_limit);
  };
  auto select_and_readback = [&]() -> cudaError_t {
    cudaError_t e = timed(owner, MPS_K_SELECT, nreq > 0, 0.0, sel_bytes, [&] {
      return launch_select(reinterpret_cast<SelectSector*>(dptr(desc_off + o_selsec)),
                           reinterpret_cast<SelectTask*>(dptr(desc_off + o_seltask)), nreq,
                           reinterpret_cast<int*>(dptr(kept_off)), reinterpret_cast<SelectResult*>(dptr(res_off)), st);
    });
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(owner->pin_out.p, dptr(kept_off), out_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && owner->tc_flag)   // this update's Theta' GEMM, or the previous reassembly GEMM
      e = cudaMemcpyAsync(tc_err_host, owner->tc_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    return e;
  };
  int c_used = 0;                    // the tile shape whose outputs the batch keeps
  if (n_cand == 1) {
    CUDA_OR_FAIL(owner, run_phase(owner, 0, [&]() -> cudaError_t {
      cudaError_t e = upload_and_theta();
      if (e == cudaSuccess)
        e = timed(owner, MPS_K_SVD, !svd.empty(), svd_flops, svd_bytes, [&] { return svd_launch(0); });
      if (e == cudaSuccess) e = select_and_readback();
      return e;
    }));
  } else {
    // tuning run: every candidate tile shape on the same inputs, timed on the stream
    CUDA_OR_FAIL(owner, upload_and_theta());
    std::vector<cudaEvent_t> ev(2 * (n_cand + 1));
    for (auto& x : ev) x = pool_event(owner);
    for (int r = 0; r <= n_cand; ++r) {         // every candidate, then the default once more
      const int c = r < n_cand ? r : kTuneDefault;
      CUDA_OR_FAIL(owner, cudaEventRecord(ev[2 * r], st));
      CUDA_OR_FAIL(owner, svd_launch(c));
      CUDA_OR_FAIL(owner, cudaEventRecord(ev[2 * r + 1], st));
    }
    CUDA_OR_FAIL(owner, cudaStreamSynchronize(st));
    float ms[kTuneCands + 1] = {};
    for (int r = 0; r <= n_cand; ++r) CUDA_OR_FAIL(owner, cudaEventElapsedTime(&ms[r], ev[2 * r], ev[2 * r + 1]));
    ms[kTuneDefault] = std::min(ms[kTuneDefault], ms[n_cand]);
    int best = kTuneDefault;
    for (int c = 0; c < n_cand; ++c)
      if (ms[c] < 0.97f * ms[kTuneDefault] && ms[c] < ms[best]) best = c;
    for (auto& x : ev) owner->event_pool.push_back(x);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      TuneEntry& te = g_tune[tkey];
      te.best = best;
      for (int c = 0; c < n_cand; ++c) te.ms[c] = ms[c];
      g_tune_runs++;
    }
    // the outputs must come from the chosen shape: rerun it unless it ran last
    if (best != kTuneDefault) CUDA_OR_FAIL(owner, svd_launch(best));
    c_used = best;
    KStat& k = owner->kstat[MPS_K_SVD];
    k.launches++;
    k.flops += svd_flops;
    k.bytes += svd_bytes;
    if (owner->profiling) k.ms += ms[best];
    CUDA_OR_FAIL(owner, select_and_readback());
  }
  CUDA_OR_FAIL(owner, cudaEventRecord(owner->staged, st));
  CUDA_OR_FAIL(owner, cudaStreamSynchronize(st));
  resolve_pending(owner);
  if (*tc_err_host) {
    CUDA_OR_FAIL(owner, cudaMemsetAsync(owner->tc_flag, 0, sizeof(int), st));
    return fail(owner, MPS_ETIMEOUT, "a bounded wait inside the tensor-core GEMM expired");
  }
  const int* kept = (const int*)owner->pin_out.p;
  const int* sstat = (const int*)((char*)owner->pin_out.p + (status_off - kept_off));
  const SelectResult* res = (const SelectResult*)((char*)owner->pin_out.p + (res_off - kept_off));

  // ---- deflation check: an update whose new cut fell below level / kChiGuard x the estimate its
  // SVDs were deflated with has its own SVDs redone without that level, then the selection
  // of the batch is repeated (the other updates' spectra are unchanged, so their selections
  // are too).  Redoing only the failing updates keeps every result independent of which
  // other updates share the batch. ----
  {
    std::vector<char> redo_upd(nreq, 0);
    bool redo = false;
    for (int u = 0; u < nreq; ++u) {
      if (W[u].cut_est <= 0.0) continue;
      reqs[u].h->stats.deflated_updates++;
      if (res[u].status == 0 && res[u].cut * kChiGuard < W[u].chi_level * W[u].cut_est) redo = redo_upd[u] = 1;
    }
    if (redo) {
      // the update of each sector, from the position of its status word
      const int* status0 = reinterpret_cast<const int*>(dptr(status_off));
      std::vector<int> upd_of(n_sec_total, 0);
      for (int u = 0; u < nreq; ++u)
        for (size_t si = 0; si < W[u].plan.sectors.size(); ++si) upd_of[W[u].sel_first + si] = u;
      std::vector<SvdSector> sub;
      double sub_flops = 0, sub_bytes = 0;
      for (const SvdSector& S : svd_sorted[c_used]) {
        if (!redo_upd[upd_of[S.status - status0]]) continue;
        SvdSector T = S;
        // when chi set the first pass's cut, that cut bounds the redo's from below (resolving
        // more values can only raise the chi-th largest candidate), so values under kChiGuard
        // times it stay unresolved within the same guard; otherwise everything is resolved
        const int uu = upd_of[S.status - status0];
        const SelectResult& R1 = res[uu];
        T.floor_abs = (R1.n_candidates > reqs[uu].chi && R1.norm_all > 0.0) ? kChiGuard * R1.cut / R1.norm_all : 0.0;
        sub.push_back(T);
        const double a = std::max(S.m, S.n), b = std::min(S.m, S.n);
        sub_flops += 4.0 * (6.0 * a * b * b + 20.0 * b * b * b);
        sub_bytes += 16.0 * S.m * S.n + 16.0 * S.n * b + 8.0 * b + 8.0 * S.m;
      }
      std::vector<SvdGroup> sub_groups;
      // the tile shape the first run used for these sectors
      const SvdTune tune = n_cand > 1 ? svd_tune_candidate(c_used) : (chosen >= 0 ? svd_tune_candidate(chosen) : SvdTune());
      CUDA_OR_FAIL(owner, svd_group(sub, sub_groups, tune));
      // the phase-1 SVD descriptors are no longer read (the stream is synchronised): reuse them
      char* hsrc = (char*)owner->pin_in.p + o_svd[c_used];
      std::memcpy(hsrc, sub.data(), sizeof(SvdSector) * sub.size());
      CUDA_OR_FAIL(owner, cudaMemcpyAsync(dptr(desc_off + o_svd[c_used]), hsrc, sizeof(SvdSector) * sub.size(),
                                          cudaMemcpyHostToDevice, st));
      const SvdSector* d_sub = reinterpret_cast<SvdSector*>(dptr(desc_off + o_svd[c_used]));
      CUDA_OR_FAIL(owner, timed(owner, MPS_K_SVD, !sub.empty(), sub_flops, sub_bytes, [&] {
        return launch_svd_groups(d_sub, sub_groups, st, owner->side, kSvdSideStreams, owner->fork, owner->join,
                                 owner->sweep_limit);
      }));
      CUDA_OR_FAIL(owner, select_and_readback());
      CUDA_OR_FAIL(owner, cudaStreamSynchronize(st));
      resolve_pending(owner);
      for (int u = 0; u < nreq; ++u)
        if (redo_upd[u]) reqs[u].h->stats.deflation_redos++;
    }
  }

  // ---- host: new bond tables and block layouts; phase-2 descriptors -------------------
  std::vector<LambdaTask> lam;
  std::vector<ScatterTask> sc;
  std::vector<GemmTask> gm;
  std::vector<TileRef> gt;
  // reduced-precision reassembly ([0] TF32, [1] BF16x3): Y(c)[:, :k] as B tiles, appended to the
  // phase-1 slots (the reassembly A tiles of Theta' written by the mix are still there)
  std::vector<ShadowTask> yshtask[2];
  std::vector<ShadowTile> yshtile[2];
  std::vector<TmaJob> gjobs[2];
  int64_t yslot_next[2] = {slot_next[0], slot_next[1]};
  double tc_gm_flops = 0, tc_gm_bytes = 0, ysh_bytes = 0;
  int64_t sc_elems = 0;
  std::vector<char> apply(nreq, 0);
  {
    int bmax = 0;
    int64_t bsum = 0;
    for (int k = 0; k < n_sec_total; ++k) {
      bmax = std::max(bmax, sstat[k]);
      bsum += std::max(sstat[k], 0);
    }
    owner->stats.batch_sectors = n_sec_total;
    owner->stats.batch_sweeps_sum = bsum;
    owner->stats.batch_sweeps_max = bmax;
  }
  std::vector<BondTable> newmid(nreq);
  std::vector<SiteTable> newL(nreq), newR(nreq);
  sec_global = 0;
  for (int u = 0; u < nreq; ++u) {
    mps_s* h = reqs[u].h;
    const int s = reqs[u].site;
    const UpdatePlan& P = W[u].plan;
    const SelectResult R = res[u];
    int max_sweeps = 0;
    bool noconv = false;
    for (size_t si = 0; si < P.sectors.size(); ++si) {
      const int sw = sstat[W[u].sel_first + si];
      if (sw < 0) noconv = true; else max_sweeps = std::max(max_sweeps, sw);
    }
    if (R.status != 0) {
      reqs[u].status = MPS_EINVAL;
      h->err = "all singular values vanish (the gate annihilated the state)";
      continue;
    }
    reqs[u].status = noconv ? MPS_ENOCONV : MPS_OK;
    if (noconv) h->err = "Jacobi SVD hit its sweep limit; state updated with the last iterate";
    reqs[u].trunc = R.trunc_err;
    const BondTable &Lb = h->bonds[s], &Rb = h->bonds[s + 2];
    BondTable& M = newmid[u];
    for (size_t si = 0; si < P.sectors.size(); ++si) {
      const int k = kept[W[u].sel_first + si];
      if (k > 0) { M.charge.push_back(P.sectors[si].c); M.dim.push_back(k); }
    }
    M.rebuild_offsets();
    if (M.size() == 0) {
      reqs[u].status = MPS_EINVAL;
      h->err = "the cutoff discards every singular value";
      continue;
    }
    if (M.total() > h->bond_cap[s + 1]) {
      reqs[u].status = MPS_ENOMEM;
      h->err = "new bond exceeds its capacity";
      continue;
    }
    layout_site(Lb, M, h->rule, newL[u]);
    layout_site(M, Rb, h->rule, newR[u]);
    if (newL[u].nnz > h->site_cap[s] || newR[u].nnz > h->site_cap[s + 1]) {
      reqs[u].status = MPS_ENOMEM;
      h->err = "new site tensor exceeds its capacity";
      continue;
    }
    apply[u] = 1;
    const double scale = 1.0 / R.norm_kept;
    double2* dstL = h->slot_ptr(s, h->cur[s] ^ 1);
    double2* dstR = h->slot_ptr(s + 1, h->cur[s + 1] ^ 1);
    int mi = 0;
    for (size_t si = 0; si < P.sectors.size(); ++si) {
      const int k = kept[W[u].sel_first + si];
      if (k == 0) continue;
      const SectorPlanEntry& E = P.sectors[si];
      const double* sig = reinterpret_cast<const double*>(dptr(W[u].sig_off[si]));
      const double2* Y = reinterpret_cast<const double2*>(dptr(W[u].y_off[si]));
      const double2* th = reinterpret_cast<const double2*>(dptr(W[u].theta_off[si]));
      lam.push_back(LambdaTask{sig, h->lambda_ptr(s + 1) + M.off[mi], k, scale});
      for (size_t ra = 0; ra < E.ri.size(); ++ra) {
        const int ri = E.ri[ra];
        const int b = newR[u].find(E.c, Rb.charge[ri]);
        ScatterTask T;
        T.Y = Y;
        T.out = dstR + newR[u].blocks[b].off;
        T.n = E.cols;
        T.coff = E.coff[ra];
        T.k = k;
        T.Dr = Rb.dim[ri];
        T.first = sc_elems;
        sc_elems += (int64_t)k * T.Dr;
        sc.push_back(T);
      }
      const bool tc = h->precision != MPS_FP64;
      const int tp = h->precision == MPS_BF16X3;
      const int KC = sh_kc(h->precision), TPK = sh_tiles_per_k(h->precision), ktn = cdiv(E.cols, KC);
      int64_t y0 = 0;
      if (tc) {   // Y(c)[:, :k] (column-major, n x k) as B tiles: column j of Y is output column j
        y0 = yslot_next[tp];
        ShadowTask Tk{Y, E.cols, 1, k, E.cols, y0, ktn, 1};
        const int id = (int)yshtask[tp].size();
        yshtask[tp].push_back(Tk);
        for (int it = 0; it < cdiv(k, kShTileN); ++it)
          for (int kt = 0; kt < ktn; ++kt) yshtile[tp].push_back(ShadowTile{id, it, kt});
        yslot_next[tp] += (int64_t)cdiv(k, kShTileN) * ktn * TPK;
        ysh_bytes += 16.0 * k * E.cols + (double)cdiv(k, kShTileN) * ktn * TPK * kShTileBytes;
      }
      for (size_t la = 0; la < E.li.size(); ++la) {
        const int li = E.li[la];
        const int b = newL[u].find(Lb.charge[li], E.c);
        if (tc) {   // B^[s][l, c] = (Theta'(c)[rows of l] . Y(c)[:, :k]) / |S_kept| on the tensor cores
          const int Dl = Lb.dim[li];
          const int64_t a0 = ra_slot[u][si][la];
          for (int rt = 0; rt < cdiv(Dl, kShRows); ++rt)
            for (int ct = 0; ct < cdiv(k, kShTileN); ++ct) {
              TmaJob J;
              J.a0 = a0 + (int64_t)rt * ktn * TPK;
              J.b0 = y0 + (int64_t)ct * ktn * TPK;
              J.kt_n = ktn;
              J.M = std::min(kShRows, Dl - rt * kShRows);
              J.N = std::min(kShTileN, k - ct * kShTileN);
              J.mode = 1;
              J.alpha = (float)scale;
              J.C = dstL + newL[u].blocks[b].off + (int64_t)rt * kShRows * k + ct * kShTileN;
              J.ldc = k;
              gjobs[tp].push_back(J);
            }
          tc_gm_flops += 8.0 * Dl * k * E.cols;
          tc_gm_bytes += 16.0 * (double)Dl * k + 8.0 * (double)Dl * E.cols;   // B^[s] written, Theta' tiles read
          continue;
        }
        GemmTask G;
        G.A = th + (int64_t)E.loff[la] * E.cols;
        G.sar = E.cols; G.sac = 1;
        G.B = Y; G.sbr = 1; G.sbc = E.cols;
        G.C = dstL + newL[u].blocks[b].off;
        G.ldc = k;
        G.M = Lb.dim[li]; G.N = k; G.K = E.cols;
        G.alpha = scale;
        const int tid = (int)gm.size();
        gm.push_back(G);
        for (int ti = 0; ti < (G.M + kTile - 1) / kTile; ++ti)
          for (int tj = 0; tj < (G.N + kTile - 1) / kTile; ++tj) gt.push_back(TileRef{tid, ti, tj});
      }
      ++mi;
    }
    Stats& S = h->stats;
    S.n_sectors = (int)P.sectors.size();
    S.n_triples = (int)P.triple_l.size();
    S.max_sweeps = max_sweeps;
    S.tie_band = R.band;
    S.norm_all = R.norm_all;
    S.norm_kept = R.norm_kept;
  }
  if (!lam.empty()) {
    // phase-1 kernels are complete (stream synchronised), so the descriptor region is free
    Stager s2{(char*)owner->pin_in.p};
    const int64_t o_lam = s2.put(lam.data(), (int64_t)lam.size());
    const int64_t o_sc = s2.put(sc.data(), (int64_t)sc.size());
    const int64_t o_gm = s2.put(gm.data(), (int64_t)gm.size());
    const int64_t o_gt = s2.put(gt.data(), (int64_t)gt.size());
    int64_t o_ysh[2], o_ytile[2], o_gjobs[2];
    for (int p = 0; p < 2; ++p) {
      std::stable_sort(gjobs[p].begin(), gjobs[p].end(),
                       [](const TmaJob& a, const TmaJob& b) { return a.kt_n > b.kt_n; });
      const int64_t tpk = p ? 2 : 1, lim = tc_slots[p] + tc_slots2[p];
      for (const TmaJob& j : gjobs[p])
        if (j.a0 < 0 || j.b0 < 0 || j.a0 + j.kt_n * tpk > lim || j.b0 + j.kt_n * tpk > lim)
          return fail(owner, MPS_EINVAL, "internal: tensor-core job outside the shadow buffer");
      o_ysh[p] = s2.put(yshtask[p].data(), (int64_t)yshtask[p].size());
      o_ytile[p] = s2.put(yshtile[p].data(), (int64_t)yshtile[p].size());
      o_gjobs[p] = s2.put(gjobs[p].data(), (int64_t)gjobs[p].size());
      if (yslot_next[p] > tc_slots[p] + tc_slots2[p])
        return fail(owner, MPS_EINVAL, "internal: shadow slot bound exceeded");
    }
    if (s2.size > desc_bytes) return fail(owner, MPS_EINVAL, "internal: descriptor bound exceeded");
    double lam_bytes = 0, gm_flops = 0, gm_bytes = 0;
    for (const LambdaTask& T : lam) lam_bytes += 16.0 * T.k;
    for (const GemmTask& T : gm) {
      gm_flops += 8.0 * T.M * T.N * T.K;
      gm_bytes += 16.0 * ((double)T.M * T.K + (double)T.K * T.N + (double)T.M * T.N);
    }
    // ---- phase 2: upload, K4/K5 (lambda, B^[s+1] scatter, B^[s] product) ----------------
    CUDA_OR_FAIL(owner, run_phase(owner, 1, [&]() -> cudaError_t {
      cudaError_t e = cudaMemcpyAsync(dptr(desc_off), owner->pin_in.p, s2.size, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = timed(owner, MPS_K_LAMBDA, true, 0.0, lam_bytes, [&] {
          return launch_lambda(reinterpret_cast<LambdaTask*>(dptr(desc_off + o_lam)), (int)lam.size(), st);
        });
      if (e == cudaSuccess)
        e = timed(owner, MPS_K_SCATTER, sc_elems > 0, 0.0, 32.0 * (double)sc_elems, [&] {
          return launch_scatter(reinterpret_cast<ScatterTask*>(dptr(desc_off + o_sc)), (int)sc.size(), sc_elems, st);
        });
      if (e == cudaSuccess)
        e = timed(owner, MPS_K_GEMM, !gt.empty(), gm_flops, gm_bytes, [&] {
          return launch_gemm(reinterpret_cast<GemmTask*>(dptr(desc_off + o_gm)),
                             reinterpret_cast<TileRef*>(dptr(desc_off + o_gt)), (int)gt.size(), st);
        });
      const int precs[2] = {MPS_TF32, MPS_BF16X3};
      const bool any_tc_gemm = !gjobs[0].empty() || !gjobs[1].empty();
      if (e == cudaSuccess)
        e = timed(owner, MPS_K_SHADOW, any_tc_gemm, 0.0, ysh_bytes, [&] {
          cudaError_t e2 = cudaSuccess;
          for (int p = 0; p < 2 && e2 == cudaSuccess; ++p)
            e2 = launch_shadow(precs[p], reinterpret_cast<ShadowTask*>(dptr(desc_off + o_ysh[p])),
                               reinterpret_cast<ShadowTile*>(dptr(desc_off + o_ytile[p])), (int)yshtile[p].size(),
                               slot_base[p], st);
          return e2;
        });
      if (e == cudaSuccess)
        e = timed(owner, MPS_K_TCGEMM, any_tc_gemm, tc_gm_flops, tc_gm_bytes, [&] {
          cudaError_t e2 = cudaSuccess;
          for (int p = 0; p < 2 && e2 == cudaSuccess; ++p)
            e2 = launch_tma_zgemm(precs[p], reinterpret_cast<TmaJob*>(dptr(desc_off + o_gjobs[p])),
                                  (int)gjobs[p].size(), slot_base[p], tc_slots[p] + tc_slots2[p], owner->tc_flag, st);
          return e2;
        });
      return e;
    }));
    CUDA_OR_FAIL(owner, cudaEventRecord(owner->staged, st));
  }
  for (int u = 0; u < nreq; ++u) {
    if (!apply[u]) continue;
    mps_s* h = reqs[u].h;
    const int s = reqs[u].site;
    h->bonds[s + 1] = newmid[u];
    h->sites[s] = newL[u];
    h->sites[s + 1] = newR[u];
    // the next update of this bond deflates from this cut when chi set it (more candidates
    // than kept); a cut set by the cutoff lies under the cutoff deflation level anyway
    if ((int)h->cut_est.size() == h->L + 1) {
      h->cut_est[s + 1] = (res[u].n_candidates > reqs[u].chi && res[u].norm_all > 0.0)
                              ? res[u].cut / res[u].norm_all : 0.0;
      if ((int)h->cut_call.size() == h->L + 1) h->cut_call[s + 1] = h->calls;
    }
    h->cur[s] ^= 1;
    h->cur[s + 1] ^= 1;
  }
  return MPS_OK;
}

int check_handle(mps_s* h) { return h ? MPS_OK : MPS_EINVAL; }

int check_site_ready(mps_s* h, int s) {
  if (h->dirty[s]) return fail(h, MPS_EINVAL, "site " + std::to_string(s) + " needs mps_set_site");
  return MPS_OK;
}

int check_gate_args(mps_s* h, int site, const double* gate, int chi, double cutoff) {
  if (site < 0 || site >= h->L - 1) return fail(h, MPS_EINVAL, "site out of range");
  if (!gate) return fail(h, MPS_EINVAL, "gate_blocks is NULL");
  if (chi < 1 || chi > h->chi_max) return fail(h, MPS_EINVAL, "chi outside [1, chi_max]");
  if (!(cutoff >= 0.0) || !std::isfinite(cutoff)) return fail(h, MPS_EINVAL, "cutoff must be finite and >= 0");
  int rc = check_site_ready(h, site);
  if (rc) return rc;
  return check_site_ready(h, site + 1);
}

}  // namespace

namespace mps {
bool svd_forced_tune(SvdTune& t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune_force < 0) return false;
  t = svd_tune_candidate(g_tune_force);
  return true;
}
}  // namespace mps

// ======================================================================================
extern "C" {

static int create_handle(mps_t* out, int L, int d, const int32_t* site_charges, int site_lo, int site_hi,
                         int precision, int chi_max, void* cuda_stream, int zn = 0,
                         const ChargeRule* multi = nullptr);

int mps_create(mps_t* out, int L, int d, const int32_t* site_charges, int precision, int chi_max,
               void* cuda_stream) {
  return create_handle(out, L, d, site_charges, 0, L, precision, chi_max, cuda_stream);
}

int mps_create_segment(mps_t* out, int L, int d, const int32_t* site_charges, int site_lo, int site_hi,
                       int precision, int chi_max, void* cuda_stream) {
  if (site_lo < 0 || site_hi > L || site_hi - site_lo < 1) {
    if (out) *out = nullptr;
    return MPS_EINVAL;
  }
  return create_handle(out, L, d, site_charges, site_lo, site_hi, precision, chi_max, cuda_stream);
}

int mps_create_zn(mps_t* out, int L, int n, const int32_t* site_charges, int precision, int chi_max,
                  void* cuda_stream) {
  if (n < 2) {
    if (out) *out = nullptr;
    return MPS_EINVAL;
  }
  return create_handle(out, L, n, site_charges, 0, L, precision, chi_max, cuda_stream, n);
}

int mps_create_cyclic(mps_t* out, int L, int d, int n, const int32_t* site_charges, int precision, int chi_max,
                      void* cuda_stream) {
  if (out) *out = nullptr;
  if (!out || d < 2 || d > MPS_MAX_D || n < d || n > kMaxZn) return MPS_EINVAL;
  if (n == d) return create_handle(out, L, n, site_charges, 0, L, precision, chi_max, cuda_stream, n);
  ChargeRule r;
  r.d = d;
  r.zn = n;
  r.init_zn();
  return create_handle(out, L, d, site_charges, 0, L, precision, chi_max, cuda_stream, n, &r);
}

int mps_create_multi(mps_t* out, int L, int d, int ncomp, const int32_t* phys_charges, const int32_t* site_indices,
                     int precision, int chi_max, void* cuda_stream) {
  if (out) *out = nullptr;
  if (!out || L < 2 || d < 2 || d > MPS_MAX_D || ncomp < 1 || ncomp > 4 || !phys_charges) return MPS_EINVAL;
  ChargeRule r;
  r.d = d;
  r.multi = 1;
  r.ncomp = ncomp;
  // radix per component: more than twice the largest bond value (L * max charge), so that every
  // difference of two charges decodes uniquely
  int64_t w = 1;
  std::vector<int64_t> weight(ncomp);
  for (int k = ncomp - 1; k >= 0; --k) {
    int mx = 0;
    for (int i = 0; i < d; ++i) {
      const int v = phys_charges[i * ncomp + k];
      if (v < 0) return MPS_ECHARGE;
      mx = std::max(mx, v);
    }
    r.radix[k] = (int)std::min<int64_t>(INT32_MAX, 2LL * L * mx + 3);
    weight[k] = w;
    w *= r.radix[k];
    if (w > (int64_t)1 << 30) return MPS_EINVAL;     // encoded charges must fit in int32
  }
  for (int i = 0; i < d; ++i) {
    int64_t e = 0;
    for (int k = 0; k < ncomp; ++k) e += phys_charges[i * ncomp + k] * weight[k];
    r.q[i] = (int)e;
    if (i && r.q[i] <= r.q[i - 1]) return MPS_ECHARGE;   // distinct, in ascending order
  }
  r.init_multi();
  return create_handle(out, L, d, site_indices, 0, L, precision, chi_max, cuda_stream, 0, &r);
}

int mps_charge_rule(mps_t h, int* zn, int* ncomp, int32_t* phys_charges) {
  if (!h) return MPS_EINVAL;
  const ChargeRule& R = h->rule;
  if (zn) *zn = R.zn;
  if (ncomp) *ncomp = R.multi ? R.ncomp : 0;
  if (phys_charges && R.multi)
    for (int i = 0; i < h->d; ++i) {   // decode q_i, first component most significant
      int64_t v = R.q[i];
      for (int k = R.ncomp - 1; k >= 0; --k) {
        phys_charges[i * R.ncomp + k] = (int32_t)(v % R.radix[k]);
        v /= R.radix[k];
      }
    }
  return MPS_OK;
}

int mps_charge_radix(mps_t h, int* ncomp, int32_t* radix) {
  if (!h || !ncomp) return MPS_EINVAL;
  *ncomp = h->rule.multi ? h->rule.ncomp : 1;
  if (radix)
    for (int k = 0; k < *ncomp; ++k) radix[k] = h->rule.multi ? h->rule.radix[k] : 0;
  return MPS_OK;
}

static int create_handle(mps_t* out, int L, int d, const int32_t* site_charges, int site_lo, int site_hi,
                         int precision, int chi_max, void* cuda_stream, int zn, const ChargeRule* multi) {
  if (!out) return MPS_EINVAL;
  *out = nullptr;
  if (L < 2 || d < 2 || d > MPS_MAX_D || chi_max < 1 || !site_charges) return MPS_EINVAL;
  if (precision != MPS_FP64 && precision != MPS_TF32 && precision != MPS_BF16X3) return MPS_EINVAL;
  for (int s = 0; s < L; ++s)
    if (site_charges[s] < 0 || site_charges[s] > d - 1) return MPS_ECHARGE;
  mps_s* h = new mps_s();
  h->L = L; h->d = d; h->chi_max = chi_max; h->precision = precision;
  if (multi) h->rule = *multi;
  h->rule.d = d;
  h->rule.zn = zn;
  h->stream = (cudaStream_t)cuda_stream;
  std::vector<int> c(L + 1, 0);
  for (int b = L - 1; b >= 0; --b) c[b] = h->rule.wrap(c[b + 1] + h->rule.charge_of(site_charges[b]));
  h->N = c[0];
  const int N = h->N;
  auto Wc = (zn || multi) ? std::vector<std::vector<double>>() : config_counts(L, d, N);
  h->bonds.resize(L + 1);
  h->bond_cap.resize(L + 1);
  h->lam_base.resize(L + 1);
  int64_t lam_total = 0;
  for (int b = 0; b <= L; ++b) {
    BondTable& t = h->bonds[b];
    t.charge = {c[b]};
    t.dim = {1};
    t.rebuild_offsets();
    double hb = 0.0;
    if (zn || multi) {   // d^k strings of k sites: the smaller side bounds the Schmidt rank
      hb = std::pow((double)d, (double)std::min(b, L - b));
    } else {
      const int lo = std::max(0, N - (d - 1) * b), hi = std::min(N, (d - 1) * (L - b));
      for (int q = lo; q <= hi; ++q) hb += std::min(Wc[b][N - q], Wc[L - b][q]);
    }
    h->bond_cap[b] = (int64_t)std::max(1.0, std::min((double)chi_max, hb));
    h->lam_base[b] = lam_total;
    lam_total += (h->bond_cap[b] + 31) / 32 * 32;
  }
  h->sites.resize(L);
  h->cur.assign(L, 0);
  h->cut_est.assign(L + 1, 0.0);
  h->cut_call.assign(L + 1, 0);
  h->dirty.assign(L, 0);
  h->site_cap.resize(L);
  h->site_base.resize(L);
  int64_t site_total = 0;
  for (int s = 0; s < L; ++s) {
    layout_site(h->bonds[s], h->bonds[s + 1], h->rule, h->sites[s]);
    // sites outside [site_lo, site_hi) keep their one product-state element and never grow
    h->site_cap[s] = (s >= site_lo && s < site_hi) ? std::max<int64_t>(1, h->bond_cap[s] * h->bond_cap[s + 1]) : 1;
    h->site_base[s] = site_total;
    site_total += 2 * ((h->site_cap[s] + 15) / 16 * 16);
  }
  cudaError_t e = cudaMalloc(&h->d_lambda, sizeof(double) * lam_total);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_sites, sizeof(double2) * site_total);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->staged, cudaEventDisableTiming);
  for (int i = 0; i < kSvdSideStreams && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&h->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (h->d_lambda) cudaFree(h->d_lambda);
    if (h->d_sites) cudaFree(h->d_sites);
    delete h;
    return MPS_ENOMEM;
  }
  std::vector<double> lam(lam_total, 0.0);
  for (int b = 0; b <= L; ++b) lam[h->lam_base[b]] = 1.0;
  e = cudaMemcpyAsync(h->d_lambda, lam.data(), sizeof(double) * lam_total, cudaMemcpyHostToDevice, h->stream);
  const double2 one = make_double2(1.0, 0.0);
  for (int s = 0; s < L && e == cudaSuccess; ++s)
    e = cudaMemcpyAsync(h->slot_ptr(s, 0), &one, sizeof(double2), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    mps_destroy(h);
    return MPS_ECUDA;
  }
  *out = h;
  return MPS_OK;
}

int mps_destroy(mps_t h) {
  if (!h) return MPS_EINVAL;
  cudaStreamSynchronize(h->stream);
  if (h->d_lambda) cudaFree(h->d_lambda);
  if (h->d_sites) cudaFree(h->d_sites);
  if (h->staged) cudaEventDestroy(h->staged);
  for (int i = 0; i < kSvdSideStreams; ++i) {
    if (h->side[i]) { cudaStreamSynchronize(h->side[i]); cudaStreamDestroy(h->side[i]); }
    if (h->join[i]) cudaEventDestroy(h->join[i]);
  }
  if (h->fork) cudaEventDestroy(h->fork);
  for (auto& p : h->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
  if (h->tc_flag) cudaFree(h->tc_flag);
  for (auto& g : h->gexec)
    if (g) cudaGraphExecDestroy(g);
  for (auto& kk : h->kind_ev)
    for (auto& e : kk)
      if (e) cudaEventDestroy(e);
  h->work.release();
  h->pin_in.release();
  h->pin_out.release();
  delete h;
  return MPS_OK;
}

const char* mps_last_error(mps_t h) { return h ? h->err.c_str() : "null handle"; }

int mps_info(mps_t h, int* L, int* d, int* N, int* chi_max, int* precision) {
  if (!h) return MPS_EINVAL;
  if (L) *L = h->L;
  if (d) *d = h->d;
  if (N) *N = h->N;
  if (chi_max) *chi_max = h->chi_max;
  if (precision) *precision = h->precision;
  return MPS_OK;
}

int mps_apply_gate2(mps_t h, int site, const double* gate_blocks, int chi, double cutoff,
                    double* trunc_err_out) {
  if (check_handle(h)) return MPS_EINVAL;
  int rc = check_gate_args(h, site, gate_blocks, chi, cutoff);
  if (rc) return rc;
  std::vector<Req> r(1);
  r[0].h = h; r[0].site = site; r[0].gate = gate_blocks; r[0].chi = chi; r[0].cutoff = cutoff;
  rc = run_batch(r, h);
  if (rc) return rc;
  if (trunc_err_out) *trunc_err_out = r[0].trunc;
  return r[0].status;
}

int mps_apply_layer(mps_t h, int n, const int* sites, const double* const* gate_blocks, int chi,
                    double cutoff, double* trunc_err_out) {
  if (check_handle(h)) return MPS_EINVAL;
  if (n < 0 || (n > 0 && (!sites || !gate_blocks))) return fail(h, MPS_EINVAL, "bad layer arguments");
  if (n == 0) return MPS_OK;
  std::vector<int> sorted(sites, sites + n);
  std::sort(sorted.begin(), sorted.end());
  for (int k = 1; k < n; ++k)
    if (sorted[k] - sorted[k - 1] < 2) return fail(h, MPS_EINVAL, "layer site pairs overlap");
  std::vector<Req> r(n);
  for (int k = 0; k < n; ++k) {
    int rc = check_gate_args(h, sites[k], gate_blocks[k], chi, cutoff);
    if (rc) return rc;
    r[k].h = h; r[k].site = sites[k]; r[k].gate = gate_blocks[k]; r[k].chi = chi; r[k].cutoff = cutoff;
  }
  int rc = run_batch(r, h);
  if (rc) return rc;
  int first = MPS_OK;
  for (int k = 0; k < n; ++k) {
    if (trunc_err_out) trunc_err_out[k] = r[k].trunc;
    if (first == MPS_OK && r[k].status != MPS_OK) first = r[k].status;
  }
  return first;
}

static int batch_on(mps_s* owner, int n, mps_t* hs, const int* sites, const double* const* gates,
                    const int* chis, const double* cutoffs, double* trunc_err_out, int* status_out);

int mps_apply_gate2_batch(int n, mps_t* hs, const int* sites, const double* const* gates, const int* chis,
                          const double* cutoffs, double* trunc_err_out, int* status_out) {
  if (n < 0 || (n > 0 && (!hs || !sites || !gates || !chis || !cutoffs))) return MPS_EINVAL;
  if (n == 0) return MPS_OK;
  if (!hs[0]) return MPS_EINVAL;
  return batch_on(hs[0], n, hs, sites, gates, chis, cutoffs, trunc_err_out, status_out);
}

int mps_exec_create(mps_exec_t* out, void* cuda_stream) {
  if (!out) return MPS_EINVAL;
  *out = nullptr;
  mps_s* h = new mps_s();
  h->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaEventCreateWithFlags(&h->staged, cudaEventDisableTiming);
  for (int i = 0; i < kSvdSideStreams && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&h->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    mps_destroy(h);
    return MPS_ECUDA;
  }
  *out = h;
  return MPS_OK;
}

int mps_exec_destroy(mps_exec_t ex) { return mps_destroy(ex); }

int mps_exec_apply(mps_exec_t ex, int n, mps_t* hs, const int* sites, const double* const* gates, const int* chis,
                   const double* cutoffs, double* trunc_err_out, int* status_out) {
  if (!ex || n < 0 || (n > 0 && (!hs || !sites || !gates || !chis || !cutoffs))) return MPS_EINVAL;
  if (n == 0) return MPS_OK;
  return batch_on(ex, n, hs, sites, gates, chis, cutoffs, trunc_err_out, status_out);
}

int mps_footprint_bytes(int L, int d, int N, int chi_max, int64_t* arena_bytes, int64_t* layer_workspace_bytes) {
  if (L < 2 || d < 2 || d > MPS_MAX_D || N < 0 || N > L * (d - 1) || chi_max < 1) return MPS_EINVAL;
  auto Wc = config_counts(L, d, N);
  std::vector<int64_t> cap(L + 1);
  int64_t lam = 0, sites = 0;
  for (int b = 0; b <= L; ++b) {
    double hb = 0.0;
    const int lo = std::max(0, N - (d - 1) * b), hi = std::min(N, (d - 1) * (L - b));
    for (int q = lo; q <= hi; ++q) hb += std::min(Wc[b][N - q], Wc[L - b][q]);
    cap[b] = (int64_t)std::max(1.0, std::min((double)chi_max, hb));
    lam += (cap[b] + 31) / 32 * 32;
  }
  int64_t ws = 0;
  for (int s = 0; s < L; ++s) {
    const int64_t c = std::max<int64_t>(1, cap[s] * cap[s + 1]);
    sites += 2 * ((c + 15) / 16 * 16);
    if (s + 1 < L) ws = std::max<int64_t>(ws, 64LL * d * std::max(cap[s], cap[s + 2]) * std::max(cap[s], cap[s + 2]));
  }
  if (arena_bytes) *arena_bytes = 8 * lam + 16 * sites;
  if (layer_workspace_bytes) *layer_workspace_bytes = ws * (L / 2);
  return MPS_OK;
}

static int batch_on(mps_s* owner, int n, mps_t* hs, const int* sites, const double* const* gates,
                    const int* chis, const double* cutoffs, double* trunc_err_out, int* status_out) {
  std::vector<Req> r(n);
  std::vector<mps_s*> others;
  for (int k = 0; k < n; ++k) {
    mps_s* h = hs[k];
    if (!h) return MPS_EINVAL;
    int rc = check_gate_args(h, sites[k], gates[k], chis[k], cutoffs[k]);
    if (rc) { if (status_out) status_out[k] = rc; return rc; }
    for (int j = 0; j < k; ++j)
      if (hs[j] == h && std::abs(sites[j] - sites[k]) < 2) return fail(owner, MPS_EINVAL, "overlapping pairs in batch");
    r[k].h = h; r[k].site = sites[k]; r[k].gate = gates[k]; r[k].chi = chis[k]; r[k].cutoff = cutoffs[k];
    if (h != owner && h->stream != owner->stream &&
        std::find(others.begin(), others.end(), h) == others.end())
      others.push_back(h);
  }
  // join the other handles' streams into the owner's stream, and back afterwards
  cudaEvent_t ev;
  CUDA_OR_FAIL(owner, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  for (mps_s* h : others) {
    cudaEventRecord(ev, h->stream);
    cudaStreamWaitEvent(owner->stream, ev, 0);
  }
  int rc = run_batch(r, owner);
  cudaEventRecord(ev, owner->stream);
  for (mps_s* h : others) cudaStreamWaitEvent(h->stream, ev, 0);
  cudaEventDestroy(ev);
  if (rc) return rc;
  int first = MPS_OK;
  for (int k = 0; k < n; ++k) {
    if (trunc_err_out) trunc_err_out[k] = r[k].trunc;
    if (status_out) status_out[k] = r[k].status;
    if (first == MPS_OK && r[k].status != MPS_OK) first = r[k].status;
  }
  return first;
}

int mps_expect(mps_t h, int site, const double* diag_op, double* out) {
  if (check_handle(h)) return MPS_EINVAL;
  if (site < 0 || site >= h->L || !diag_op || !out) return fail(h, MPS_EINVAL, "bad expect arguments");
  int rc = check_site_ready(h, site);
  if (rc) return rc;
  const SiteTable& S = h->sites[site];
  const BondTable& Lb = h->bonds[site];
  const double2* slot = h->slot_ptr(site, h->cur[site]);
  std::vector<ExpectTask> t;
  for (const SiteBlock& b : S.blocks)
    t.push_back(ExpectTask{slot + b.off, h->lambda_ptr(site) + Lb.off[b.il], b.Dl, b.Dm,
                           diag_op[h->rule.phys(b.l, b.m)]});
  const int nt = (int)t.size();
  const int64_t bytes_t = a256(sizeof(ExpectTask) * (int64_t)nt);
  CUDA_OR_FAIL(h, cudaEventSynchronize(h->staged));
  if (h->work.reserve(bytes_t + 8 * (int64_t)nt + 512) != cudaSuccess) return fail(h, MPS_ENOMEM, "workspace");
  if (h->pin_in.reserve(bytes_t + 512) != cudaSuccess || h->pin_out.reserve(8 * (size_t)nt + 512) != cudaSuccess)
    return fail(h, MPS_ENOMEM, "pinned staging");
  std::memcpy(h->pin_in.p, t.data(), sizeof(ExpectTask) * nt);
  char* base = (char*)h->work.p;
  CUDA_OR_FAIL(h, cudaMemcpyAsync(base, h->pin_in.p, sizeof(ExpectTask) * nt, cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaEventRecord(h->staged, h->stream));
  double ex_bytes = 0;
  for (const ExpectTask& T : t) ex_bytes += 16.0 * T.Dl * T.Dm + 8.0 * T.Dl;
  CUDA_OR_FAIL(h, timed(h, MPS_K_EXPECT, nt > 0, 0.0, ex_bytes,
                        [&] { return launch_expect((ExpectTask*)base, nt, (double*)(base + bytes_t), h->stream); }));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->pin_out.p, base + bytes_t, 8 * (size_t)nt, cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  double acc = 0.0;
  for (int k = 0; k < nt; ++k) acc += ((double*)h->pin_out.p)[k];
  *out = acc;
  return MPS_OK;
}

int mps_amplitude_batch(mps_t h, int n, const int32_t* configs, double* out) {
  if (check_handle(h)) return MPS_EINVAL;
  if (n < 0 || (n > 0 && (!configs || !out))) return fail(h, MPS_EINVAL, "bad amplitude arguments");
  if (n == 0) return MPS_OK;
  for (int s = 0; s < h->L; ++s)
    if (h->dirty[s]) return check_site_ready(h, s);
  const int L = h->L;
  std::vector<AmpStep> steps((size_t)n * L);
  std::vector<int> c(L + 1);
  int cap = 1;
  for (int b = 0; b <= L; ++b) cap = std::max(cap, h->bonds[b].total());
  for (int k = 0; k < n; ++k) {
    const int32_t* cfg = configs + (size_t)k * L;
    bool ok = true;
    c[L] = 0;
    for (int b = L - 1; b >= 0; --b) {
      if (cfg[b] < 0 || cfg[b] > h->d - 1) { ok = false; continue; }
      c[b] = h->rule.wrap(c[b + 1] + h->rule.charge_of(cfg[b]));
    }
    if (c[0] != h->N) ok = false;
    for (int s = 0; s < L; ++s) {
      AmpStep a{nullptr, 0, 0};
      if (ok) {
        const int bi = h->sites[s].find(c[s], c[s + 1]);
        if (bi >= 0) {
          const SiteBlock& B = h->sites[s].blocks[bi];
          a.blk = h->slot_ptr(s, h->cur[s]) + B.off;
          a.Dl = B.Dl; a.Dm = B.Dm;
        }
      }
      steps[(size_t)k * L + s] = a;
    }
  }
  const int64_t bytes_s = a256(sizeof(AmpStep) * (int64_t)steps.size());
  CUDA_OR_FAIL(h, cudaEventSynchronize(h->staged));
  if (h->work.reserve(bytes_s + 16 * (int64_t)n + 512) != cudaSuccess) return fail(h, MPS_ENOMEM, "workspace");
  if (h->pin_in.reserve(bytes_s + 512) != cudaSuccess || h->pin_out.reserve(16 * (size_t)n + 512) != cudaSuccess)
    return fail(h, MPS_ENOMEM, "pinned staging");
  std::memcpy(h->pin_in.p, steps.data(), sizeof(AmpStep) * steps.size());
  char* base = (char*)h->work.p;
  CUDA_OR_FAIL(h, cudaMemcpyAsync(base, h->pin_in.p, sizeof(AmpStep) * steps.size(), cudaMemcpyHostToDevice,
                                  h->stream));
  CUDA_OR_FAIL(h, cudaEventRecord(h->staged, h->stream));
  double amp_flops = 0;
  for (const AmpStep& a : steps) amp_flops += 8.0 * a.Dl * a.Dm;
  CUDA_OR_FAIL(h, timed(h, MPS_K_AMPLITUDE, n > 0, amp_flops, 16.0 * amp_flops / 8.0, [&] {
    return launch_amplitude((AmpStep*)base, L, n, (double2*)(base + bytes_s), cap, h->stream);
  }));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->pin_out.p, base + bytes_s, 16 * (size_t)n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  std::memcpy(out, h->pin_out.p, 16 * (size_t)n);
  return MPS_OK;
}

int mps_sample(mps_t h, int n, const double* uniforms, int32_t* configs_out, double* probs_out) {
  if (check_handle(h)) return MPS_EINVAL;
  if (n < 0 || (n > 0 && (!uniforms || !configs_out))) return fail(h, MPS_EINVAL, "bad sample arguments");
  if (n == 0) return MPS_OK;
  for (int s = 0; s < h->L; ++s)
    if (h->dirty[s]) return check_site_ready(h, s);
  const int L = h->L, d = h->d;
  for (int64_t k = 0; k < (int64_t)n * L; ++k)
    if (!(uniforms[k] >= 0.0 && uniforms[k] < 1.0)) return fail(h, MPS_EINVAL, "uniforms must lie in [0, 1)");
  // per site, per charge of its left bond, per occupation: the block and the next charge's index
  std::vector<int> site_off(L);
  std::vector<SampleEntry> table;
  int cap = 1;
  for (int s = 0; s < L; ++s) {
    const BondTable &Lb = h->bonds[s], &Rb = h->bonds[s + 1];
    cap = std::max(cap, std::max(Lb.total(), Rb.total()));
    site_off[s] = (int)table.size();
    const double2* slot = h->slot_ptr(s, h->cur[s]);
    for (int li = 0; li < Lb.size(); ++li)
      for (int i = 0; i < d; ++i) {
        SampleEntry e{nullptr, 0, 0, -1, 0};
        const int bi = h->sites[s].find(Lb.charge[li], h->rule.wrap(Lb.charge[li] - h->rule.charge_of(i)));
        if (bi >= 0) {
          const SiteBlock& B = h->sites[s].blocks[bi];
          e.blk = slot + B.off;
          e.Dl = B.Dl;
          e.Dm = B.Dm;
          e.next = B.im;
        }
        table.push_back(e);
      }
  }
  const int64_t b_table = a256(sizeof(SampleEntry) * (int64_t)table.size());
  const int64_t b_off = a256(sizeof(int) * (int64_t)L);
  const int64_t b_u = a256(8 * (int64_t)n * L);
  const int64_t b_cfg = a256(4 * (int64_t)n * L);
  const int64_t b_prob = a256(8 * (int64_t)n);
  const int64_t in_bytes = b_table + b_off + b_u;
  CUDA_OR_FAIL(h, cudaEventSynchronize(h->staged));
  if (h->work.reserve(in_bytes + b_cfg + b_prob) != cudaSuccess) return fail(h, MPS_ENOMEM, "workspace");
  if (h->pin_in.reserve(in_bytes) != cudaSuccess || h->pin_out.reserve(b_cfg + b_prob) != cudaSuccess)
    return fail(h, MPS_ENOMEM, "pinned staging");
  char* hp = (char*)h->pin_in.p;
  std::memcpy(hp, table.data(), sizeof(SampleEntry) * table.size());
  std::memcpy(hp + b_table, site_off.data(), sizeof(int) * L);
  std::memcpy(hp + b_table + b_off, uniforms, 8 * (size_t)n * L);
  char* base = (char*)h->work.p;
  CUDA_OR_FAIL(h, cudaMemcpyAsync(base, hp, in_bytes, cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaEventRecord(h->staged, h->stream));
  int* d_cfg = reinterpret_cast<int*>(base + in_bytes);
  double* d_prob = reinterpret_cast<double*>(base + in_bytes + b_cfg);
  // the work depends on the drawn patterns (the blocks visited), so none is counted
  CUDA_OR_FAIL(h, timed(h, MPS_K_SAMPLE, true, 0.0, 0.0, [&] {
    return launch_sample(reinterpret_cast<SampleEntry*>(base), reinterpret_cast<int*>(base + b_table), L, d, cap,
                         reinterpret_cast<double*>(base + b_table + b_off), n, d_cfg, d_prob, h->stream);
  }));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->pin_out.p, d_cfg, b_cfg + b_prob, cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  std::memcpy(configs_out, h->pin_out.p, 4 * (size_t)n * L);
  const double* pr = reinterpret_cast<const double*>((char*)h->pin_out.p + b_cfg);
  if (probs_out) std::memcpy(probs_out, pr, 8 * (size_t)n);
  for (int k = 0; k < n; ++k)
    if (pr[k] == 0.0) return fail(h, MPS_EINVAL, "a sample reached a prefix whose continuations have zero weight");
  return MPS_OK;
}

int mps_amplitude(mps_t h, const int32_t* config, double out_complex[2]) {
  return mps_amplitude_batch(h, 1, config, out_complex);
}

int mps_bond_spectrum(mps_t h, int bond, int32_t* charges, int32_t* dims, double* lambda, int cap, int* n_out) {
  if (check_handle(h)) return MPS_EINVAL;
  if (bond < 0 || bond > h->L || !n_out) return fail(h, MPS_EINVAL, "bad bond");
  const BondTable& t = h->bonds[bond];
  *n_out = t.size();
  if (cap < t.size() || !charges || !dims || !lambda) return fail(h, MPS_EINVAL, "capacity too small");
  for (int i = 0; i < t.size(); ++i) { charges[i] = t.charge[i]; dims[i] = t.dim[i]; }
  CUDA_OR_FAIL(h, cudaMemcpyAsync(lambda, h->lambda_ptr(bond), sizeof(double) * t.total(), cudaMemcpyDeviceToHost,
                                  h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return MPS_OK;
}

int mps_bond_entropy(mps_t h, int bond, double* out) {
  if (check_handle(h)) return MPS_EINVAL;
  if (bond < 0 || bond > h->L || !out) return fail(h, MPS_EINVAL, "bad bond");
  CUDA_OR_FAIL(h, cudaEventSynchronize(h->staged));
  if (h->work.reserve(256) != cudaSuccess) return fail(h, MPS_ENOMEM, "workspace");
  if (h->pin_out.reserve(256) != cudaSuccess) return fail(h, MPS_ENOMEM, "pinned staging");
  double* d_out = reinterpret_cast<double*>(h->work.p);
  CUDA_OR_FAIL(h, launch_entropy(h->lambda_ptr(bond), h->bonds[bond].total(), d_out, h->stream));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->pin_out.p, d_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  *out = *reinterpret_cast<const double*>(h->pin_out.p);
  return MPS_OK;
}

int mps_get_site(mps_t h, int site, int32_t* lcharges, int32_t* mcharges, int cap_blocks, double* data,
                 int64_t cap_values, int* n_blocks, int64_t* n_values) {
  if (check_handle(h)) return MPS_EINVAL;
  if (site < 0 || site >= h->L || !n_blocks || !n_values) return fail(h, MPS_EINVAL, "bad site");
  const SiteTable& S = h->sites[site];
  *n_blocks = (int)S.blocks.size();
  *n_values = S.nnz;
  if (cap_blocks < *n_blocks || cap_values < S.nnz || !lcharges || !mcharges || (!data && S.nnz))
    return fail(h, MPS_EINVAL, "capacity too small");
  for (size_t i = 0; i < S.blocks.size(); ++i) { lcharges[i] = S.blocks[i].l; mcharges[i] = S.blocks[i].m; }
  if (S.nnz) {
    CUDA_OR_FAIL(h, cudaMemcpyAsync(data, h->slot_ptr(site, h->cur[site]), sizeof(double2) * S.nnz,
                                    cudaMemcpyDeviceToHost, h->stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  }
  return MPS_OK;
}

int mps_set_bond(mps_t h, int bond, int n_sectors, const int32_t* charges, const int32_t* dims,
                 const double* lambda) {
  if (check_handle(h)) return MPS_EINVAL;
  if (bond < 1 || bond > h->L - 1) return fail(h, MPS_EINVAL, "only inner bonds 1..L-1 can be set");
  if (n_sectors < 1 || !charges || !dims || !lambda) return fail(h, MPS_EINVAL, "bad bond table");
  BondTable t;
  t.charge.assign(charges, charges + n_sectors);
  t.dim.assign(dims, dims + n_sectors);
  const int d = h->d, L = h->L, N = h->N;
  // several-U(1) handles: any encoded charge (the site layout keeps only blocks whose charge
  // difference is a physical charge)
  const int lo = h->rule.multi ? INT32_MIN : (h->rule.zn ? 0 : std::max(0, N - (d - 1) * bond));
  const int hi = h->rule.multi ? INT32_MAX : (h->rule.zn ? h->rule.zn - 1 : std::min(N, (d - 1) * (L - bond)));
  for (int i = 0; i < n_sectors; ++i) {
    if (t.dim[i] < 1) return fail(h, MPS_EINVAL, "sector dimension < 1");
    if (i && t.charge[i] <= t.charge[i - 1]) return fail(h, MPS_EINVAL, "charges not ascending");
    if (t.charge[i] < lo || t.charge[i] > hi) return fail(h, MPS_ECHARGE, "charge outside the bond's range");
  }
  t.rebuild_offsets();
  if (t.total() > h->bond_cap[bond]) return fail(h, MPS_ENOMEM, "bond dimension exceeds capacity");
  CUDA_OR_FAIL(h, cudaEventSynchronize(h->staged));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  CUDA_OR_FAIL(h, cudaMemcpy(h->lambda_ptr(bond), lambda, sizeof(double) * t.total(), cudaMemcpyHostToDevice));
  h->bonds[bond] = t;
  h->dirty[bond - 1] = 1;
  h->dirty[bond] = 1;
  h->cut_est[bond] = 0.0;   // a loaded bond has no deflation history (the other bonds keep theirs)
  return MPS_OK;
}

int mps_set_site(mps_t h, int site, int n_blocks, const int32_t* lcharges, const int32_t* mcharges,
                 const double* data) {
  if (check_handle(h)) return MPS_EINVAL;
  if (site < 0 || site >= h->L) return fail(h, MPS_EINVAL, "bad site");
  SiteTable t;
  layout_site(h->bonds[site], h->bonds[site + 1], h->rule, t);
  if (n_blocks != (int)t.blocks.size() || (n_blocks && (!lcharges || !mcharges)))
    return fail(h, MPS_ECHARGE, "block list does not match the allowed (l, m) pairs");
  for (int i = 0; i < n_blocks; ++i)
    if (lcharges[i] != t.blocks[i].l || mcharges[i] != t.blocks[i].m)
      return fail(h, MPS_ECHARGE, "block list does not match the allowed (l, m) pairs");
  if (t.nnz > h->site_cap[site]) return fail(h, MPS_ENOMEM, "site exceeds capacity");
  if (t.nnz && !data) return fail(h, MPS_EINVAL, "data is NULL");
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  if (t.nnz)
    CUDA_OR_FAIL(h, cudaMemcpy(h->slot_ptr(site, h->cur[site]), data, sizeof(double2) * t.nnz,
                               cudaMemcpyHostToDevice));
  h->sites[site] = t;
  h->dirty[site] = 0;
  return MPS_OK;
}

int mps_set_profiling(mps_t h, int on) {
  if (!h) return MPS_EINVAL;
  h->profiling = on != 0;
  return MPS_OK;
}

int mps_kernel_stats(mps_t h, int kind, int64_t* launches, double* ms, double* flops, double* bytes) {
  if (!h || kind < 0 || kind >= MPS_K_COUNT) return MPS_EINVAL;
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  resolve_pending(h);
  const KStat& k = h->kstat[kind];
  if (launches) *launches = k.launches;
  if (ms) *ms = k.ms;
  if (flops) *flops = k.flops;
  if (bytes) *bytes = k.bytes;
  return MPS_OK;
}

int mps_reset_kernel_stats(mps_t h) {
  if (!h) return MPS_EINVAL;
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  resolve_pending(h);
  for (auto& k : h->kstat) k = KStat();
  return MPS_OK;
}

int64_t mps_launch_count(void) { return g_launches.load(); }

int mps_set_chi_deflation(mps_t h, double level) {
  if (!h || !(level >= 0.0 && level <= kChiGuard)) return MPS_EINVAL;
  h->chi_deflate = level;
  return MPS_OK;
}

int mps_set_sweep_limit(mps_t h, int max_sweeps) {
  if (!h || max_sweeps < 1 || max_sweeps > kJacobiMaxSweeps) return MPS_EINVAL;
  h->sweep_limit = max_sweeps;
  return MPS_OK;
}

int mps_set_graphs(mps_t h, int on) {
  if (!h) return MPS_EINVAL;
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  h->graphs = on != 0;
  if (!h->graphs)
    for (auto& g : h->gexec)
      if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  return MPS_OK;
}

int mps_graph_stats(mps_t h, int64_t* launches, int64_t* updates, int64_t* instantiations) {
  if (!h) return MPS_EINVAL;
  if (launches) *launches = h->graph_launches;
  if (updates) *updates = h->graph_updates;
  if (instantiations) *instantiations = h->graph_instantiations;
  return MPS_OK;
}

int mps_set_autotune(mps_t h, int on) {
  if (!h) return MPS_EINVAL;
  h->autotune = on != 0;
  return MPS_OK;
}

int mps_autotune_stats(int64_t* keys, int64_t* tuning_runs, int64_t* hits) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int64_t nh = 0;
  for (const auto& kv : g_tune) nh += kv.second.hits;
  if (keys) *keys = (int64_t)g_tune.size();
  if (tuning_runs) *tuning_runs = g_tune_runs;
  if (hits) *hits = nh;
  return MPS_OK;
}

int mps_autotune_table(char* buf, int cap, int* len) {
  std::string t;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    char line[256];
    for (const auto& kv : g_tune) {
      std::string key;
      for (size_t i = 0; i + 1 < kv.first.size(); i += 2) {
        std::snprintf(line, sizeof(line), "%sK~2^%d:%d", key.empty() ? "" : ",", kv.first[i],
                      kv.first[i + 1] ? 1 << (kv.first[i + 1] - 1) : 0);
        key += line;
      }
      const TuneEntry& e = kv.second;
      if (e.best < 0) continue;
      const SvdTune b = svd_tune_candidate(e.best);
      if (b.rr_min_k < (1 << 30))
        std::snprintf(line, sizeof(line), "%s -> round-robin from K=%d hits=%lld ms=", key.c_str(), b.rr_min_k,
                      (long long)e.hits);
      else if (b.c16_min_k < (1 << 30))
        std::snprintf(line, sizeof(line), "%s -> 16-CTA clusters from K=%d hits=%lld ms=", key.c_str(), b.c16_min_k,
                      (long long)e.hits);
      else
        std::snprintf(line, sizeof(line), "%s -> bw=%d cl_min=%d hits=%lld ms=", key.c_str(), b.bw, b.cl_min,
                      (long long)e.hits);
      t += line;
      for (int c = 0; c < kTuneCands; ++c) {
        std::snprintf(line, sizeof(line), "%s%.2f", c ? "/" : "", e.ms[c]);
        t += line;
      }
      t += "\n";
    }
  }
  if (len) *len = (int)t.size();
  if (!buf || cap <= (int)t.size()) return buf ? MPS_EINVAL : MPS_OK;
  std::memcpy(buf, t.c_str(), t.size() + 1);
  return MPS_OK;
}

int mps_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  g_tune_runs = 0;
  return MPS_OK;
}

int mps_autotune_force(int candidate) {
  if (candidate < -1 || candidate >= kTuneCands) return MPS_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_force = candidate;
  return MPS_OK;
}

int mps_autotune_freeze(int frozen) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_frozen = frozen != 0;
  return MPS_OK;
}

int mps_autotune_min_flops(double flops) {
  if (!(flops >= 0.0) || !std::isfinite(flops)) return MPS_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_min_flops = flops;
  return MPS_OK;
}

int mps_last_batch_sweeps(mps_t h, int* n_sectors, int64_t* sweeps_sum, int* sweeps_max) {
  if (!h) return MPS_EINVAL;
  if (n_sectors) *n_sectors = h->stats.batch_sectors;
  if (sweeps_sum) *sweeps_sum = h->stats.batch_sweeps_sum;
  if (sweeps_max) *sweeps_max = h->stats.batch_sweeps_max;
  return MPS_OK;
}

int mps_deflation_stats(mps_t h, int64_t* deflated_updates, int64_t* redos) {
  if (!h) return MPS_EINVAL;
  if (deflated_updates) *deflated_updates = h->stats.deflated_updates;
  if (redos) *redos = h->stats.deflation_redos;
  return MPS_OK;
}

int mps_last_update_stats(mps_t h, int* n_sectors, int* n_triples, int* max_sweeps, int* tie_band,
                          double* norm_all, double* norm_kept) {
  if (!h) return MPS_EINVAL;
  if (n_sectors) *n_sectors = h->stats.n_sectors;
  if (n_triples) *n_triples = h->stats.n_triples;
  if (max_sweeps) *max_sweeps = h->stats.max_sweeps;
  if (tie_band) *tie_band = h->stats.tie_band;
  if (norm_all) *norm_all = h->stats.norm_all;
  if (norm_kept) *norm_kept = h->stats.norm_kept;
  return MPS_OK;
}

}  // extern "C"
