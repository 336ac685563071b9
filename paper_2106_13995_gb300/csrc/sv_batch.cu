// C ABI: batched execution of many circuits on many states (uneven widths)
// in one persistent launch, optionally replayed from a CUDA graph; the
// autotuner that picks fusion width and tile size per circuit shape; and the
// self-test of the bounded device wait.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "sv_internal.h"

namespace sv {

// ---------------------------------------------------------------------------
// autotune cache: (n, dtype, op-count bucket, widest op) -> (fusion_k, tile_m)
// ---------------------------------------------------------------------------
using TuneKey = std::tuple<int, int, int, int>;
static std::map<TuneKey, std::pair<int, int>> g_tune;
static std::mutex g_tune_mu;
static bool g_tune_loaded = false;

static TuneKey tune_key(int n, sv_dtype dt, const sv_circuit *c) {
  int arity = 0;
  for (int i = 0; i < c->n_ops; i++) arity = std::max(arity, c->ops[i].n_targets + c->ops[i].n_controls);
  // op counts within ~12% share a bucket
  int bucket = 0;
  for (int x = std::max(1, c->n_ops); x > 1; x = (x * 8) / 9) bucket++;
  return TuneKey(n, (int)dt, bucket, arity);
}

static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *path = std::getenv("SV_TUNE_CACHE");
  if (!path) return;
  FILE *f = std::fopen(path, "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    int n, dt, b, a, k, m;
    if (std::sscanf(line, " {\"n\": %d, \"dtype\": %d, \"ops_bucket\": %d, \"arity\": %d, \"fusion_k\": %d, \"tile_m\": %d",
                    &n, &dt, &b, &a, &k, &m) == 6)
      g_tune[TuneKey(n, dt, b, a)] = {k, m};
  }
  std::fclose(f);
}

static void tune_save_locked() {
  const char *path = std::getenv("SV_TUNE_CACHE");
  if (!path) return;
  FILE *f = std::fopen(path, "w");
  if (!f) return;
  std::fprintf(f, "[\n");
  size_t i = 0;
  for (auto &kv : g_tune) {
    std::fprintf(f, "  {\"n\": %d, \"dtype\": %d, \"ops_bucket\": %d, \"arity\": %d, \"fusion_k\": %d, \"tile_m\": %d}%s\n",
                 std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first),
                 kv.second.first, kv.second.second, ++i < g_tune.size() ? "," : "");
  }
  std::fprintf(f, "]\n");
  std::fclose(f);
}

void tuned_options(const sv_state *s, const sv_circuit *c, const sv_options *opt, Opts &o) {
  // the tuner times CUDA-core configurations: tensor-core modes keep their
  // own defaults (5-qubit blocks, 12-qubit tiles)
  if (o.prec != SV_PREC_PLAIN) return;
  const bool want_k = !opt || opt->fusion_k == 0, want_m = !opt || opt->tile_m == 0;
  if (!want_k && !want_m) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  auto it = g_tune.find(tune_key(s->n, s->dt, c));
  if (it == g_tune.end()) return;
  if (want_k) o.fusion_k = it->second.first;
  if (want_m) o.tile_m = std::min(it->second.second, s->n);
}

// ---------------------------------------------------------------------------
// persistent batch
// ---------------------------------------------------------------------------
struct BatchGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};
// key: the first state and, per state, (program serial, amplitudes,
// workspace, wide flag), plus the wait budget -- everything the recorded
// launches depend on
using GraphKey = std::pair<const sv_state *, std::vector<uint64_t>>;
static std::map<GraphKey, BatchGraph> g_graphs;
static std::mutex g_graphs_mu;
constexpr size_t kMaxGraphs = 64;

constexpr uint64_t kDefaultSpin = 1ull << 23;   // ~1 s of 128 ns polls

static sv_status run_batch(sv_state *const *states, int B, const sv_circuit *const *circs,
                           const double *const *params, const sv_options *opt) {
  sv_state *s0 = states[0];
  // the programs stay alive for the whole call even if the cache evicts them
  std::vector<ProgramRef> cps(B);
  std::vector<Opts> os(B);
  int maxP = 0, m_max = 1;
  for (int b = 0; b < B; b++) {
    SV_TRY(get_program(states[b], circs[b], params ? params[b] : nullptr, opt, &cps[b], &os[b]));
    if (os[b].mode == SV_MODE_PER_GATE) return set_error(SV_EINVAL, "per-gate mode has no batched form");
    maxP = std::max(maxP, (int)cps[b]->prog.passes.size());
    for (const TilePass &tp : cps[b]->prog.passes) m_max = std::max(m_max, tp.m);
  }
  for (int b = 0; b < B; b++) SV_TRY(upload_program(states[b], *cps[b]));
  // States whose passes have at least one tile per SM fill the GPU with one
  // ordinary launch per pass (measured on 256 uneven circuits: 21-qubit
  // states, 256 tiles a pass, take 15.6 ms as launches against 23.7 ms in
  // the queue); the persistent queue is for the rest, whose passes alone
  // would leave most SMs idle.
  std::vector<char> wide(B, 0);
  for (int b = 0; b < B; b++) {
    uint64_t min_tiles = ~0ull;
    for (const TilePass &tp : cps[b]->prog.passes) min_tiles = std::min<uint64_t>(min_tiles, (uint64_t)1 << (tp.n - tp.m));
    bool has_tc = false;
    // (tensor-core and permutation passes have kernels of their own, which
    // the persistent queue does not run)
    for (const TilePass &tp : cps[b]->prog.passes) has_tc |= (tp.flags & (kPassTC | kPassHasTC | kPassTable)) != 0;
    wide[b] = !cps[b]->prog.passes.empty() && (has_tc || min_tiles >= (uint64_t)s0->sm_count);
  }
  // descriptors in wave order: pass 0 of every state, then pass 1, ...
  std::vector<TilePass> desc;
  std::vector<unsigned long long> first;
  std::vector<int32_t> dep;
  std::vector<uint32_t> ntiles, chunk;
  std::vector<int> last_desc(B, -1);
  unsigned long long items = 0;
  for (int p = 0; p < maxP; p++)
    for (int b = 0; b < B; b++) {
      const CachedProgram &cp = *cps[b];
      if (wide[b] || p >= (int)cp.prog.passes.size()) continue;
      TilePass tp = cp.prog.passes[p];
      char *base = states[b]->ws + kWsProg;
      tp.ops = reinterpret_cast<const TileOp *>(base + cp.lay.ops_off) + cp.op0s[p];
      tp.mats = base + cp.lay.mats_off;
      tp.coeffs = reinterpret_cast<const double *>(base + cp.lay.coeffs_off);
      tp.v0 = states[b]->amps;
      tp.nvec = 1;
      desc.push_back(tp);
      first.push_back(items);
      dep.push_back(last_desc[b]);
      const uint32_t nt = 1u << (tp.n - tp.m);
      // tiles per queue item: big passes hand out up to 16 tiles at a time
      const uint32_t ch = std::max(1u, std::min(16u, nt / 64u));
      ntiles.push_back(nt);
      chunk.push_back(ch);
      last_desc[b] = (int)desc.size() - 1;
      items += (nt + ch - 1) / ch;
    }
  const uint32_t nd = (uint32_t)desc.size();
  // The wide states' passes, as ordinary launches.  The states are
  // independent, so with two or more of them they are spread over the
  // library's fan-out streams (longest first onto the least-loaded stream,
  // load = tiles x passes), forked from st and joined back into it: one
  // state's passes fill the waves another leaves partly empty, and a stream
  // launches while another's kernel runs.  Recorded in a graph, the streams
  // become parallel branches.
  std::vector<int> wb;
  std::vector<double> work(B, 0.0);
  for (int b = 0; b < B; b++)
    if (wide[b]) {
      wb.push_back(b);
      for (const TilePass &tp : cps[b]->prog.passes) work[b] += std::ldexp(1.0, tp.n - tp.m);
    }
  const int K = std::min<int>(kFanStreams, (int)wb.size());
  std::vector<int> lane(B, 0);
  if (K >= 2) {
    for (int k = 0; k < K; k++)
      if (!s0->fan[k]) SV_CUDA(cudaStreamCreateWithFlags(&s0->fan[k], cudaStreamNonBlocking));
    if (!s0->fan_fork) SV_CUDA(cudaEventCreateWithFlags(&s0->fan_fork, cudaEventDisableTiming));
    for (int k = 0; k < K; k++)
      if (!s0->fan_join[k]) SV_CUDA(cudaEventCreateWithFlags(&s0->fan_join[k], cudaEventDisableTiming));
    std::vector<int> order = wb;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return work[a] > work[c]; });
    std::vector<double> load(K, 0.0);
    for (int b : order) {
      const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      lane[b] = k;
      load[k] += work[b];
    }
  }
  auto launch_state = [&](int b, cudaStream_t st) -> sv_status {
    const CachedProgram &cp = *cps[b];
    char *base = states[b]->ws + kWsProg;
    for (size_t p = 0; p < cp.prog.passes.size(); p++) {
      TilePass tp = cp.prog.passes[p];
      tp.ops = reinterpret_cast<const TileOp *>(base + cp.lay.ops_off) + cp.op0s[p];
      tp.mats = base + cp.lay.mats_off;
      tp.coeffs = reinterpret_cast<const double *>(base + cp.lay.coeffs_off);
      tp.v0 = states[b]->amps;
      tp.nvec = 1;
      tp.err = reinterpret_cast<uint32_t *>(states[b]->ws + kWsCtrl + kWsErrFlag);
      const HostPass hp{cp.prog.ops.data() + cp.op0s[p], cp.prog.mats.data()};
      SV_TRY(launch_any_pass(states[b], tp, 1, st, &hp));
    }
    return SV_OK;
  };
  auto launch_wide = [&](cudaStream_t st) -> sv_status {
    if (K < 2) {
      for (int b : wb) SV_TRY(launch_state(b, st));
      return SV_OK;
    }
    SV_CUDA(cudaEventRecord(s0->fan_fork, st));
    for (int k = 0; k < K; k++) SV_CUDA(cudaStreamWaitEvent(s0->fan[k], s0->fan_fork, 0));
    sv_status rc = SV_OK;
    for (int b : wb)
      if (rc == SV_OK) rc = launch_state(b, s0->fan[lane[b]]);
    // join every stream back even after an error, so none is left forked
    for (int k = 0; k < K; k++) {
      SV_CUDA(cudaEventRecord(s0->fan_join[k], s0->fan[k]));
      SV_CUDA(cudaStreamWaitEvent(st, s0->fan_join[k], 0));
    }
    return rc;
  };
  const bool use_graph = opt && opt->mode == SV_MODE_TILED_GRAPH;
  if (nd == 0) {
    if (!use_graph) return launch_wide(s0->stream);
  }
  // table layout at the start of the first state's reduction area
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = (off + bytes + 255) & ~(size_t)255;
    return at;
  };
  const size_t o_desc = take(sizeof(TilePass) * nd), o_first = take(sizeof(unsigned long long) * nd);
  const size_t o_dep = take(sizeof(int32_t) * nd), o_nt = take(sizeof(uint32_t) * nd);
  const size_t o_ch = take(sizeof(uint32_t) * nd);
  const size_t o_done = take(sizeof(uint32_t) * nd + 2 * sizeof(unsigned long long));
  const size_t total = off;
  if (total > red_bytes(s0->n)) return set_error(SV_ENOMEM, "batch too large for the first state's workspace");
  char *tb = s0->ws + kWsRed;
  SV_TRY(stage_upload_to(s0, tb,
                         {{desc.data(), sizeof(TilePass) * nd}, {first.data(), sizeof(unsigned long long) * nd},
                          {dep.data(), sizeof(int32_t) * nd}, {ntiles.data(), sizeof(uint32_t) * nd},
                          {chunk.data(), sizeof(uint32_t) * nd}},
                         {o_desc, o_first, o_dep, o_nt, o_ch}, o_done));
  PersistArgs A;
  std::memset(&A, 0, sizeof(A));
  A.passes = reinterpret_cast<const TilePass *>(tb + o_desc);
  A.first_item = reinterpret_cast<const unsigned long long *>(tb + o_first);
  A.dep = reinterpret_cast<const int32_t *>(tb + o_dep);
  A.ntiles = reinterpret_cast<const uint32_t *>(tb + o_nt);
  A.chunk = reinterpret_cast<const uint32_t *>(tb + o_ch);
  A.done = reinterpret_cast<uint32_t *>(tb + o_done);
  A.next_item = reinterpret_cast<unsigned long long *>(tb + o_done + ((sizeof(uint32_t) * nd + 7) & ~(size_t)7));
  A.err = reinterpret_cast<uint32_t *>(s0->ws + kWsCtrl + kWsErrFlag);
  A.total_items = items;
  A.ndesc = nd;
  A.spin_limit = (opt && opt->timeout_cycles) ? opt->timeout_cycles : kDefaultSpin;
  const size_t zero_bytes = total - o_done;
  auto record = [&](cudaStream_t st) -> sv_status {
    if (nd > 0) {
      SV_CUDA(cudaMemsetAsync(tb + o_done, 0, zero_bytes, st));
      SV_TRY(launch_tile_persist(s0, A, m_max, nullptr, st));
    }
    return launch_wide(st);
  };
  if (!use_graph) return record(s0->stream);
  // graph: capture the counter reset and the cooperative launch once per
  // batch layout, then replay
  GraphKey gk;
  gk.first = s0;
  gk.second.reserve(4 * (size_t)B + 1);
  for (int b = 0; b < B; b++) {
    gk.second.push_back(cps[b]->serial);
    gk.second.push_back((uint64_t)(uintptr_t)states[b]->amps);
    gk.second.push_back((uint64_t)(uintptr_t)states[b]->ws);
    gk.second.push_back((uint64_t)wide[b]);
  }
  gk.second.push_back(A.spin_limit);
  std::lock_guard<std::mutex> lk(g_graphs_mu);
  auto it = g_graphs.find(gk);
  if (it == g_graphs.end()) {
    BatchGraph g;
    // record on a library-owned stream (the caller's may be the legacy
    // default stream, which cannot be captured); replay on the caller's
    if (!s0->capture) SV_CUDA(cudaStreamCreateWithFlags(&s0->capture, cudaStreamNonBlocking));
    SV_CUDA(cudaStreamBeginCapture(s0->capture, cudaStreamCaptureModeThreadLocal));
    sv_status st = record(s0->capture);
    cudaError_t e2 = cudaStreamEndCapture(s0->capture, &g.graph);
    if (st != SV_OK) {
      if (g.graph) cudaGraphDestroy(g.graph);
      return st;
    }
    if (e2 != cudaSuccess) return cuda_error(e2, "cudaStreamEndCapture");
    SV_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
    if (g_graphs.size() >= kMaxGraphs) {
      // earlier replays may still be running on this stream: let them finish
      // before their executable graphs go
      SV_CUDA(cudaStreamSynchronize(s0->stream));
      for (auto &kv : g_graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
      }
      g_graphs.clear();
    }
    it = g_graphs.emplace(std::move(gk), g).first;
  }
  SV_CUDA(cudaGraphLaunch(it->second.exec, s0->stream));
  g_launches++;
  return SV_OK;
}

void drop_graphs(const sv_state *s) {
  std::lock_guard<std::mutex> lk(g_graphs_mu);
  for (auto it = g_graphs.begin(); it != g_graphs.end();) {
    if (it->first.first == s) {
      cudaGraphExecDestroy(it->second.exec);
      cudaGraphDestroy(it->second.graph);
      it = g_graphs.erase(it);
    } else {
      ++it;
    }
  }
}

}  // namespace sv

using namespace sv;

extern "C" {

sv_status sv_apply_circuit_batch(sv_state *const *states, int B, const sv_circuit *const *circs,
                                 const double *const *params, const sv_options *opt) {
  if (!states || !circs || B < 1) return set_error(SV_EINVAL, "null argument");
  for (int b = 0; b < B; b++) {
    if (!states[b] || !circs[b]) return set_error(SV_EINVAL, "null state or circuit in batch");
    if (states[b]->stream != states[0]->stream || states[b]->device != states[0]->device)
      return set_error(SV_EINVAL, "batch states must share one stream and device");
    for (int j = 0; j < b; j++)
      if (states[j]->amps == states[b]->amps) return set_error(SV_EINVAL, "a state appears twice in the batch");
  }
  if (opt && opt->mode == SV_MODE_PER_GATE) {
    for (int b = 0; b < B; b++) SV_TRY(sv_apply_circuit(states[b], circs[b], params ? params[b] : nullptr, opt));
    return SV_OK;
  }
  for (int b = 0; b < B; b++) states[b]->basis_known = false;
  return run_batch(states, B, circs, params, opt);
}

sv_status sv_autotune(sv_state *s, const sv_circuit *c, sv_options *inout) {
  if (!s || !c || !inout) return set_error(SV_EINVAL, "null argument");
  if (c->n_qubits != s->n) return set_error(SV_EINVAL, "circuit width does not match the scratch state");
  if (c->n_params > 0) return set_error(SV_EUNSUPPORTED, "autotune a circuit with fixed angles");
  s->basis_known = false;
  cudaEvent_t e0, e1;
  SV_CUDA(cudaEventCreate(&e0));
  SV_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bk = 3, bm = std::min(12, s->n);
  for (int k = 2; k <= 6; k++)
    for (int m = std::min(10, s->n); m <= std::min(13, s->n); m++) {
      sv_options o = *inout;
      o.fusion_k = k;
      o.tile_m = m;
      o.mode = SV_MODE_TILED;
      sv_status st = sv_apply_circuit(s, c, nullptr, &o);   // plans, uploads, warms up
      if (st == SV_EUNSUPPORTED) continue;
      if (st != SV_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
      }
      SV_CUDA(cudaEventRecord(e0, s->stream));
      for (int r = 0; r < 2; r++) SV_TRY(sv_apply_circuit(s, c, nullptr, &o));
      SV_CUDA(cudaEventRecord(e1, s->stream));
      SV_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      SV_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        bk = k;
        bm = m;
      }
      if (m == s->n) break;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  inout->fusion_k = bk;
  inout->tile_m = bm;
  if (inout->prec != SV_PREC_PLAIN) return SV_OK;   // the cache serves CUDA-core defaults only
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  g_tune[tune_key(s->n, s->dt, c)] = {bk, bm};
  tune_save_locked();
  return SV_OK;
}

sv_status sv_wait_selftest(void *stream, uint64_t polls) {
  // a counter nothing increments and an error flag, in one small buffer the
  // caller's stream owns for the duration of the call
  uint32_t *buf = nullptr;
  SV_CUDA(cudaMallocAsync((void **)&buf, 2 * sizeof(uint32_t), (cudaStream_t)stream));
  cudaError_t e = cudaMemsetAsync(buf, 0, 2 * sizeof(uint32_t), (cudaStream_t)stream);
  sv_status st = e == cudaSuccess ? launch_wait_selftest((cudaStream_t)stream, buf, buf + 1, polls)
                                  : cuda_error(e, "cudaMemsetAsync");
  uint32_t err = 0;
  if (st == SV_OK) {
    e = cudaMemcpyAsync(&err, buf + 1, sizeof(err), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) st = cuda_error(e, "sv_wait_selftest");
  }
  cudaFreeAsync(buf, (cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  if (st != SV_OK) return st;
  return err ? set_error(SV_ETIMEOUT, "bounded device wait ran out (as the self-test intends)") : SV_OK;
}

}  // extern "C"
