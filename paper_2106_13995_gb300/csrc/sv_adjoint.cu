// C ABI: adjoint-method gradients (plain and batched) and batched circuit
// application.
//
// One "adjoint program" is a single list of tile passes:
//   forward   : the circuit on psi (1 vector per tile);
//   lambda    : lambda = H psi from Pauli strings, <H> = Re<psi|lambda>
//               (2 vectors: psi read-only, lambda written);
//   reverse   : for j = G..1, Im<lambda|G_j|psi> for parametric gates, then
//               U_j^dagger on both vectors (2 vectors).
// Parametric gates are kept as separate ops whose 2x2 matrices come from a
// per-batch table (forward U(theta_b) and reverse U(theta_b)^dagger), so one
// program serves every parameter set; fixed gates are fused as usual.  The
// batched form launches each pass once for all B states (grid.y = B).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "sv_internal.h"

namespace sv {

struct AdjointProgram {
  uint64_t serial = 0;            // unique per built program (graph cache key)
  DeviceProgram prog;
  std::vector<uint32_t> op0s;
  std::vector<int> inst_param;   // parameter index of each parametric instance
  std::vector<int> inst_gate;    // sv_gate of each parametric instance
  int n_params = 0;
  int n_inst = 0;
};

static ProgCache<AdjointProgram> g_adj_cache(64);

// Recorded launch sequences of batched gradients (SV_MODE_TILED_GRAPH): the
// accumulator reset and every pass, per (first state, program, batch layout).
struct AdjGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};
using AdjGraphKey = std::pair<const sv_state *, std::vector<uint64_t>>;
static std::map<AdjGraphKey, AdjGraph> g_adj_graphs;
static std::mutex g_adj_graphs_mu;
constexpr size_t kMaxAdjGraphs = 32;

static void destroy_graph(AdjGraph &g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
}

void drop_adjoint_programs(const sv_state *s) {
  g_adj_cache.drop_owner(s);
  std::lock_guard<std::mutex> lk(g_adj_graphs_mu);
  for (auto it = g_adj_graphs.begin(); it != g_adj_graphs.end();) {
    if (it->first.first == s) {
      destroy_graph(it->second);
      it = g_adj_graphs.erase(it);
    } else {
      ++it;
    }
  }
}

static void append_passes(DeviceProgram &prog, std::vector<uint32_t> &op0s, const std::vector<PassPlan> &passes,
                          const BuildCtx &b, const std::vector<int> &bmo, sv_status &st) {
  for (const PassPlan &P : passes) {
    if (st != SV_OK) return;
    st = emit_pass(prog, P, b, op0s, bmo);
  }
}

static sv_status build_adjoint(sv_state *s, const sv_circuit *c, const double *params0,
                               const sv_pauli_term *terms, int nt, const Opts &o1, const Opts &o2,
                               AdjointProgram &A) {
  std::vector<Gate> gates;
  SV_TRY(circuit_to_gates(c, params0, s->n, gates, true));
  A.n_params = c->n_params;
  for (Gate &g : gates) {
    if (g.param < 0) continue;
    if (g.targets.size() != 1 || !g.controls.empty() || gate_generator(g.param_gate) == 0)
      return set_error(SV_EUNSUPPORTED,
                       "parametric gates must be uncontrolled single-qubit RX/RY/RZ/PHASE for gradients");
    g.inst = A.n_inst++;
    A.inst_param.push_back(g.param);
    A.inst_gate.push_back(g.param_gate);
  }
  const int G = (int)gates.size();
  std::vector<int> fwd_off(A.n_inst), rev_off(A.n_inst);
  for (int i = 0; i < A.n_inst; i++) {
    fwd_off[i] = 4 * i;
    rev_off[i] = 4 * (A.n_inst + i);
  }
  sv_status st = SV_OK;
  // forward
  {
    std::vector<Block> blocks = fuse(gates, o1.fusion_k);
    int m = o1.tile_m, L = o1.L;
    if (!fit_tile(blocks, s->n, lmin(s->dt), mmax(s->dt, 1), m, L))
      return set_error(SV_EUNSUPPORTED, "a fused block does not fit a shared-memory tile");
    std::vector<PassPlan> passes = plan_passes(blocks, s->n, m, L, 256, 1 << 16);
    if (passes.empty() && !blocks.empty()) return set_error(SV_EINVAL, "internal: pass planning failed");
    BuildCtx b{s->dt, s->n, m, L, 1, 0};
    append_passes(A.prog, A.op0s, passes, b, fwd_off, st);
  }
  // lambda = H psi
  {
    std::vector<Block> blocks;
    for (int t = 0; t < nt; t++) {
      Block b;
      b.kind = TOP_PAULI;
      for (int q = 0; q < s->n; q++)
        if ((terms[t].x_mask >> q) & 1) b.qubits.push_back(q);
      b.xmask = terms[t].x_mask;
      b.zmask = terms[t].z_mask;
      b.coeff = terms[t].coeff;
      b.fusable = false;
      blocks.push_back(b);
    }
    int m = o2.tile_m, L = o2.L;
    if (!fit_tile(blocks, s->n, lmin(s->dt), mmax(s->dt, 2), m, L))
      return set_error(SV_EUNSUPPORTED, "a Pauli string's X support does not fit a shared-memory tile");
    std::vector<PassPlan> passes = plan_passes(blocks, s->n, m, L, 256, 1 << 16);
    if (passes.empty() && !blocks.empty()) return set_error(SV_EINVAL, "internal: pass planning failed");
    if (passes.empty()) {
      PassPlan P;
      for (int q = 0; q < std::min(m, s->n); q++) P.S.push_back(q);
      passes.push_back(P);
    }
    Block zero;
    zero.kind = TOP_ZERO;
    passes.front().ops.insert(passes.front().ops.begin(), zero);
    Block dot;
    dot.kind = TOP_DOT;
    dot.slot = A.n_params;
    passes.back().ops.push_back(dot);
    for (size_t i = 0; i < passes.size() && st == SV_OK; i++) {
      BuildCtx b{s->dt, s->n, m, L, 2, (i == 0 ? 1u : 0u) | 2u};
      st = emit_pass(A.prog, passes[i], b, A.op0s, {});
    }
  }
  // reverse sweep
  {
    std::vector<Gate> rev;
    rev.reserve(2 * G);
    for (int j = G - 1; j >= 0; j--) {
      const Gate &g = gates[j];
      if (g.param >= 0) {
        Gate probe;
        probe.targets = g.targets;
        probe.grad_gen = gate_generator(g.param_gate);
        probe.grad_slot = g.param;
        rev.push_back(probe);
      }
      Gate u = g;
      u.U = adjoint_of(g.U, (int)g.targets.size());
      rev.push_back(u);
    }
    std::vector<Block> blocks = fuse(rev, o2.fusion_k);
    for (Block &b : blocks)
      if (b.kind == TOP_DENSE) b.vmask = 3;
    int m = o2.tile_m, L = o2.L;
    if (!fit_tile(blocks, s->n, lmin(s->dt), mmax(s->dt, 2), m, L))
      return set_error(SV_EUNSUPPORTED, "a fused block does not fit a shared-memory tile");
    std::vector<PassPlan> passes = plan_passes(blocks, s->n, m, L, 256, 1 << 16);
    if (passes.empty() && !blocks.empty()) return set_error(SV_EINVAL, "internal: pass planning failed");
    BuildCtx b{s->dt, s->n, m, L, 2, 0};
    append_passes(A.prog, A.op0s, passes, b, rev_off, st);
  }
  return st;
}

template <typename R>
static void put_mats(std::vector<uint8_t> &pool, const AdjointProgram &A, const double *theta) {
  // forward matrices for every instance, then their adjoints
  std::vector<cd> U;
  for (int pass = 0; pass < 2; pass++)
    for (int i = 0; i < A.n_inst; i++) {
      const double ang[3] = {theta[A.inst_param[i]], 0, 0};
      gate_matrix(A.inst_gate[i], ang, U);
      if (pass == 1) U = adjoint_of(U, 1);
      if constexpr (sizeof(R) == 4) {
        put_pairs_c64(pool, U.data(), 1);   // the layout complex64 tile ops read
      } else {
        for (int e = 0; e < 4; e++) {
          R v[2] = {(R)U[e].real(), (R)U[e].imag()};
          const uint8_t *p = (const uint8_t *)v;
          pool.insert(pool.end(), p, p + sizeof(v));
        }
      }
    }
}

static sv_status check_batch(sv_state *const *psi, int B, int n, sv_dtype dt, cudaStream_t st) {
  for (int b = 0; b < B; b++) {
    if (!psi[b]) return set_error(SV_EINVAL, "null state in batch");
    if (psi[b]->n != n || psi[b]->dt != dt) return set_error(SV_EINVAL, "batch states differ in width or dtype");
    if (psi[b]->stream != st) return set_error(SV_EINVAL, "batch states must share one stream");
  }
  return SV_OK;
}

static sv_status adjoint_batch(sv_state *const *psi, sv_state *const *lam, int B, const sv_circuit *c,
                               const double *params, const sv_pauli_term *terms, int nt, const sv_options *opt,
                               double *ev_out, double *grad_out) {
  if (!psi || !lam || B < 1 || !c || !ev_out || (c->n_params > 0 && (!params || !grad_out)))
    return set_error(SV_EINVAL, "null argument");
  sv_state *s = psi[0];
  if (!s) return set_error(SV_EINVAL, "null state");
  SV_TRY(check_batch(psi, B, s->n, s->dt, s->stream));
  SV_TRY(check_batch(lam, B, s->n, s->dt, s->stream));
  for (int b = 0; b < B; b++) psi[b]->basis_known = lam[b]->basis_known = false;
  if (nt < 0 || (nt > 0 && !terms)) return set_error(SV_EINVAL, "bad term list");
  const uint64_t lim = (1ull << s->n) - 1;
  for (int t = 0; t < nt; t++)
    if ((terms[t].x_mask & ~lim) || (terms[t].z_mask & ~lim))
      return set_error(SV_EINVAL, "Pauli mask references a qubit >= n");
  Opts o1 = resolve(s, opt, 1), o2 = resolve(s, opt, 2);
  // defaults for the gradient program (measured on the 20-qubit, 64-set
  // ansatz): fusion width 2 and 12-qubit tiles for both sweeps
  if (!opt || opt->fusion_k == 0) o1.fusion_k = o2.fusion_k = 2;
  if (!opt || opt->tile_m == 0) {
    o1.tile_m = o2.tile_m = std::min(12, s->n);
    o1.L = o2.L = std::min(o1.L, o1.tile_m);
  }
  // cache key: circuit structure, terms, options (parameters enter only the
  // per-batch matrices, uploaded every call)
  KeyBytes k;
  k.val((int)0xad);
  circuit_key(k, c);
  if (nt) k.bytes(terms, sizeof(sv_pauli_term) * nt);
  k.val(o1);
  k.val(o2);
  k.val(s->dt);
  const uint64_t kh = k.hash();
  std::shared_ptr<const AdjointProgram> Ap = g_adj_cache.find(s, k, kh);
  if (!Ap) {
    auto built = std::make_shared<AdjointProgram>();
    SV_TRY(build_adjoint(s, c, params, terms, nt, o1, o2, *built));
    built->serial = next_program_serial();
    Ap = g_adj_cache.insert(s, k, kh, std::move(built));
  }
  const AdjointProgram &A = *Ap;
  const int np = c->n_params;
  // per-batch matrices, state pointer tables
  std::vector<uint8_t> pm;
  for (int b = 0; b < B; b++) {
    if (s->dt == SV_C64) put_mats<float>(pm, A, params + (size_t)b * np);
    else put_mats<double>(pm, A, params + (size_t)b * np);
  }
  std::vector<void *> tbl(2 * (size_t)B);
  for (int b = 0; b < B; b++) {
    tbl[b] = psi[b]->amps;
    tbl[B + b] = lam[b]->amps;
  }
  const ProgLayout L = layout_of(A.prog, tbl.size() * sizeof(void *), pm.size());
  SV_TRY(stage_upload(s,
                      {{A.prog.ops.data(), A.prog.ops.size() * sizeof(TileOp)},
                       {A.prog.mats.data(), A.prog.mats.size()},
                       {A.prog.coeffs.data(), A.prog.coeffs.size() * sizeof(double)},
                       {tbl.data(), tbl.size() * sizeof(void *)},
                       {pm.data(), pm.size()}},
                      {L.ops_off, L.mats_off, L.coeffs_off, L.tbl_off, L.pmats_off}, L.end));
  const size_t acc_stride = (size_t)np + 1;
  const size_t acc_bytes = acc_stride * B * sizeof(double);
  if (acc_bytes > red_bytes(s->n)) return set_error(SV_ENOMEM, "workspace too small for the gradient batch");
  double *acc = reinterpret_cast<double *>(s->ws + kWsRed);
  char *base = s->ws + kWsProg;
  LaunchEnv E;
  E.batch = B;
  E.tbl0 = reinterpret_cast<void *const *>(base + L.tbl_off);
  E.tbl1 = E.tbl0 + B;
  E.pmats = base + L.pmats_off;
  E.pmats_stride = (uint64_t)8 * A.n_inst;
  E.acc = acc;
  E.acc_stride = acc_stride;
  if (opt && opt->mode == SV_MODE_TILED_GRAPH) {
    // the reset and all passes as one recorded launch sequence; the tables
    // and per-set matrices were uploaded above, in stream order, so a
    // replay reads this call's parameters
    std::lock_guard<std::mutex> lk(g_adj_graphs_mu);
    AdjGraphKey gk{s, {Ap->serial, (uint64_t)B, (uint64_t)L.end, (uint64_t)acc_bytes}};
    auto it = g_adj_graphs.find(gk);
    if (it == g_adj_graphs.end()) {
      AdjGraph g;
      if (!s->capture) SV_CUDA(cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking));
      SV_CUDA(cudaStreamBeginCapture(s->capture, cudaStreamCaptureModeThreadLocal));
      cudaError_t e1 = cudaMemsetAsync(acc, 0, acc_bytes, s->capture);
      sv_status st = e1 == cudaSuccess ? launch_program(s, A.prog, L, A.op0s, E, s->capture)
                                       : cuda_error(e1, "cudaMemsetAsync");
      cudaError_t e2 = cudaStreamEndCapture(s->capture, &g.graph);
      if (st != SV_OK) {
        destroy_graph(g);
        return st;
      }
      if (e2 != cudaSuccess) return cuda_error(e2, "cudaStreamEndCapture");
      cudaError_t e3 = cudaGraphInstantiate(&g.exec, g.graph, 0);
      if (e3 != cudaSuccess) {
        destroy_graph(g);
        return cuda_error(e3, "cudaGraphInstantiate");
      }
      if (g_adj_graphs.size() >= kMaxAdjGraphs) {
        SV_CUDA(cudaStreamSynchronize(s->stream));   // replays in flight finish first
        for (auto &kv : g_adj_graphs) destroy_graph(kv.second);
        g_adj_graphs.clear();
      }
      it = g_adj_graphs.emplace(std::move(gk), g).first;
    }
    SV_CUDA(cudaGraphLaunch(it->second.exec, s->stream));
    g_launches++;
  } else {
    SV_CUDA(cudaMemsetAsync(acc, 0, acc_bytes, s->stream));
    SV_TRY(launch_program(s, A.prog, L, A.op0s, E));
  }
  std::vector<double> h(acc_stride * B);
  SV_CUDA(cudaMemcpyAsync(h.data(), acc, acc_bytes, cudaMemcpyDeviceToHost, s->stream));
  SV_CUDA(cudaStreamSynchronize(s->stream));
  for (int b = 0; b < B; b++) {
    ev_out[b] = h[(size_t)b * acc_stride + np];
    for (int p = 0; p < np; p++) grad_out[(size_t)b * np + p] = h[(size_t)b * acc_stride + p];
  }
  return SV_OK;
}

}  // namespace sv

using namespace sv;

extern "C" {

sv_status sv_adjoint_grad(sv_state *psi, sv_state *lam, const sv_circuit *c, const double *params,
                          const sv_pauli_term *terms, int nt, const sv_options *opt, double *ev, double *grad) {
  if (!psi || !lam) return set_error(SV_EINVAL, "null state");
  if (psi == lam || psi->amps == lam->amps) return set_error(SV_EINVAL, "psi and lambda must be distinct buffers");
  return adjoint_batch(&psi, &lam, 1, c, params, terms, nt, opt, ev, grad);
}

sv_status sv_adjoint_grad_batch(sv_state *const *psi, sv_state *const *lam, int B, const sv_circuit *c,
                                const double *params, const sv_pauli_term *terms, int nt, const sv_options *opt,
                                double *ev, double *grad) {
  return adjoint_batch(psi, lam, B, c, params, terms, nt, opt, ev, grad);
}

}  // extern "C"
