// C ABI implementation: state handles, argument validation, program building
// (fusion + tile passes), upload, and orchestration of every entry point.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "sv_internal.h"

namespace sv {

std::atomic<uint64_t> g_launches{0};
static thread_local std::string g_err;

sv_status set_error(sv_status st, const std::string &msg) {
  g_err = msg;
  return st;
}
sv_status cuda_error(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return SV_ECUDA;
}

size_t amp_bytes(sv_dtype dt) { return dt == SV_C64 ? 8 : 16; }
int lmin(sv_dtype dt) { return dt == SV_C64 ? 1 : 0; }
int mmax(sv_dtype dt, int nvec) {
  // largest tile whose vectors fit the 200 KB dynamic shared-memory budget
  int m = 1;
  while (tile_smem(dt, m + 1, nvec) <= (200u << 10)) m++;
  return m;
}

size_t red_bytes(int n) {
  const int cb = n < 10 ? n : 10;
  const size_t chunks = (size_t)1 << (n - cb);
  // CDF chunks (256-byte aligned) + shot buffer + the prefix scan's scratch
  size_t need = ((chunks * sizeof(double) + 255) & ~(size_t)255) + (1 << 20) + scan_scratch_bytes(n);
  return std::max<size_t>(need, 2 << 20);
}

// ---------------------------------------------------------------------------
// defaults
// ---------------------------------------------------------------------------
Opts resolve(const sv_state *s, const sv_options *o, int nvec) {
  Opts r;
  r.fusion_k = (o && o->fusion_k > 0) ? o->fusion_k : (o && o->prec != SV_PREC_PLAIN ? 5 : 3);
  // default tiles: 13 qubits for single-vector CUDA-core passes on complex64
  // (fewer passes; 32 amplitudes per thread at 256 threads), 12 otherwise
  // (tensor-core tile passes need 12; two-vector and complex128 tiles would
  // crowd shared memory)
  const bool plain64 = s->dt == SV_C64 && nvec == 1 && !(o && o->prec != SV_PREC_PLAIN);
  r.tile_m = (o && o->tile_m > 0) ? o->tile_m : (plain64 ? 13 : 12 - (nvec - 1));
  // contiguous low qubits in every tile: 64-byte runs for complex64 (three
  // rather than four fixed qubits leave the planner more choice: the
  // 30-qubit grid circuit takes 23 instead of 26 passes, 209 vs 216 ms; two
  // give 32-byte runs and cost DRAM efficiency), 128-byte runs for complex128
  r.L = 3;
  r.prec = o ? o->prec : SV_PREC_PLAIN;
  r.mode = o ? o->mode : SV_MODE_TILED;
  r.fusion_k = std::min(r.fusion_k, 6);
  r.tile_m = std::max(1, std::min(r.tile_m, s->n));
  // tensor-core blocks run inside 12-qubit tile passes for split-BF16 (four
  // CTAs per SM fit) unless another tile size is asked for, and for split-TF32
  // only when 12-qubit tiles are asked for explicitly (its operands admit two
  // CTAs per SM, and passes of their own measure faster)
  const bool explicit12 = o && o->tile_m == kTcTileM;
  const bool default_m = !(o && o->tile_m > 0);
  r.tc_in_tile = r.prec != SV_PREC_PLAIN && (explicit12 || (r.prec == SV_PREC_TC_BF16X3 && default_m));
  r.L = std::min(r.L, r.tile_m);
  if (s->dt == SV_C64 && r.L < 1) r.L = 1;
  return r;
}

// ---------------------------------------------------------------------------
// program cache keys
// ---------------------------------------------------------------------------
uint64_t KeyBytes::hash() const {
  // 8 bytes per step, each word mixed by a multiply-xorshift (splitmix64's
  // finaliser); only a bucket index: equal hashes are compared byte for byte
  uint64_t h = 0x243F6A8885A308D3ull ^ (uint64_t)b.size();
  size_t i = 0;
  for (; i + 8 <= b.size(); i += 8) {
    uint64_t w;
    std::memcpy(&w, b.data() + i, 8);
    h = (h ^ w) * 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
  }
  uint64_t w = 0;
  std::memcpy(&w, b.data() + i, b.size() - i);
  h = (h ^ w) * 0xBF58476D1CE4E5B9ull;
  return h ^ (h >> 31);
}

void circuit_key(KeyBytes &k, const sv_circuit *c) {
  k.val(c->n_qubits);
  k.val(c->n_ops);
  k.val(c->n_params);
  if (c->n_ops > 0) k.bytes(c->ops, sizeof(sv_op) * (size_t)c->n_ops);
  for (int i = 0; i < c->n_ops; i++)
    if (c->ops[i].gate == SV_GATE_MATRIX && c->matrices && c->ops[i].matrix_offset >= 0) {
      const int d = 1 << c->ops[i].n_targets;
      k.bytes(c->matrices + 2 * c->ops[i].matrix_offset, sizeof(double) * 2 * d * d);
    }
}

static std::atomic<uint64_t> g_serial{0};
uint64_t next_program_serial() { return ++g_serial; }

// kernel attributes, once per (kernel, device, attribute, value)
static std::mutex g_attr_mu;
static std::vector<std::tuple<const void *, int, int, int>> g_attr_done;
sv_status func_attr_once(const void *fn, int device, cudaFuncAttribute attr, int value) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  const auto key = std::make_tuple(fn, device, (int)attr, value);
  for (const auto &t : g_attr_done)
    if (t == key) return SV_OK;
  SV_CUDA(cudaFuncSetAttribute(fn, attr, value));
  g_attr_done.push_back(key);
  return SV_OK;
}

// ---------------------------------------------------------------------------
// program building
// ---------------------------------------------------------------------------
template <typename R> static void put_c(std::vector<uint8_t> &pool, cd v) {
  R t[2] = {(R)v.real(), (R)v.imag()};
  const uint8_t *p = (const uint8_t *)t;
  pool.insert(pool.end(), p, p + sizeof(t));
}

// Positions of a tile op's thread-index bits.  The groups of an op are the
// local indices with zeros at its fixed positions (targets, local controls);
// thread bit i takes the i-th lowest free position, except that lane bit j
// (j < NB) takes position j or j + NB when one of them is among the first
// log2(T) free positions: the swizzle folds both onto slot bit j, so the
// 2^NB lanes of one shared-memory wavefront reach different bank rows.  Only
// the first log2(T) positions are permuted (T = the fewest threads a pass of
// this tile size runs with), so larger blocks keep the same trip positions.
static void set_thread_positions(TileOp &op, uint32_t fixed, int m, sv_dtype dt) {
  const int NB = dt == SV_C64 ? 4 : 3;
  int ntb = 0;
  while ((1 << (ntb + 1)) <= tile_threads(m, dt)) ntb++;
  int pos[9], nf = 0;
  for (int p = 0; p < m && nf < 9; p++)
    if (!((fixed >> p) & 1u)) pos[nf++] = p;
  const int nlim = std::min(ntb, nf);
  int P[9];
  uint32_t used = 0;
  for (int i = 0; i < 9; i++) P[i] = -1;
  for (int j = 0; j < std::min(NB, nlim); j++)
    for (int c : {j, j + NB}) {
      bool among = false;
      for (int i = 0; i < nlim; i++) among |= pos[i] == c;
      if (among && !((used >> c) & 1u)) {
        P[j] = c;
        used |= 1u << c;
        break;
      }
    }
  int r = 0;
  for (int i = 0; i < nlim; i++)
    if (P[i] < 0) {
      while ((used >> pos[r]) & 1u) r++;
      P[i] = pos[r];
      used |= 1u << pos[r];
    }
  for (int i = nlim; i < nf; i++) P[i] = pos[i];
  std::memset(op.tbpos, 0, sizeof(op.tbpos));
  for (int i = 0; i < nf; i++) op.tbpos[i >> 1] |= (uint8_t)(P[i] << (4 * (i & 1)));
}

// perm[c] = the row of the single entry 1 in column c, if U (2^k x 2^k) is a
// permutation matrix with exact 0/1 entries
bool permutation_of(const std::vector<cd> &U, int k, int *perm) {
  const int d = 1 << k;
  if (k > 6) return false;
  uint64_t rows = 0;
  for (int c = 0; c < d; c++) {
    int r1 = -1;
    for (int r = 0; r < d; r++) {
      const cd u = U[(size_t)r * d + c];
      if (u == cd(0.0)) continue;
      if (u != cd(1.0) || r1 >= 0) return false;
      r1 = r;
    }
    if (r1 < 0 || ((rows >> r1) & 1ull)) return false;
    rows |= 1ull << r1;
    perm[c] = r1;
  }
  return true;
}

void put_pairs_c64(std::vector<uint8_t> &pool, const cd *U, int k) {
  const int d = 1 << k;
  for (int p = 0; p < d / 2; p++)
    for (int y = 0; y < d; y++) {
      const cd a = U[(size_t)(2 * p) * d + y], b = U[(size_t)(2 * p + 1) * d + y];
      const float v[4] = {(float)a.real(), (float)b.real(), (float)a.imag(), (float)b.imag()};
      const uint8_t *q = reinterpret_cast<const uint8_t *>(v);
      pool.insert(pool.end(), q, q + sizeof(v));
    }
}

// Convert one planned pass into TilePass + TileOps (+ matrices).
// A pass whose every block only moves amplitudes (0/1 permutation blocks:
// X, CNOT, Toffoli, multi-controlled X and their products, paper Sec. III's
// multipliers) is composed on the host into one gather table per setting of
// the pass's global control qubits: the tile kernel then reads each
// amplitude from its source slot (out[y] = in[table[y]]), one move per
// amplitude for the whole pass instead of a complex matrix product per
// block.  Table block in the matrix pool (16-byte aligned): uint32 g, int8
// global qubit positions[8], 4 bytes padding, then 2^g tables of 2^m uint16
// (table v serves the tiles whose global control qubits read v's bits).
// Returns false (nothing appended) if the pass does not qualify.
static bool table_pass(const PassPlan &P, const BuildCtx &b, const int *loc, int m, std::vector<uint8_t> &pool,
                       uint32_t &mat0) {
  if (b.nvec != 1 || m > 16 || P.ops.empty()) return false;
  struct PB {
    uint32_t lc = 0, tmask = 0;
    uint64_t gc = 0;
    int k = 0;
    int t[6];
    int perm[64];
  };
  std::vector<PB> pbs;
  uint64_t gall = 0;
  for (const Block &blk : P.ops) {
    if ((blk.kind != TOP_DENSE && blk.kind != TOP_TC) || blk.inst >= 0 || blk.param >= 0 || blk.vmask != 1 ||
        blk.xmask || blk.qubits.size() > 6)
      return false;
    PB pb;
    pb.k = (int)blk.qubits.size();
    if (!permutation_of(blk.U, pb.k, pb.perm)) return false;
    for (int j = 0; j < pb.k; j++) {
      if (loc[blk.qubits[j]] < 0) return false;
      pb.t[j] = loc[blk.qubits[j]];
      pb.tmask |= 1u << pb.t[j];
    }
    for (int q : blk.controls) {
      if (loc[q] >= 0) pb.lc |= 1u << loc[q];
      else pb.gc |= 1ull << q;
    }
    gall |= pb.gc;
    pbs.push_back(pb);
  }
  const int g = __builtin_popcountll(gall);
  const uint32_t N = 1u << m;
  const size_t bytes = 16 + ((size_t)N << g) * sizeof(uint16_t);
  // at most 5 global control qubits, and tables take at most half the
  // workspace's program area
  if (g > 5 || pool.size() + bytes > kWsProgBytes / 2) return false;
  int gq[8] = {0};
  {
    int i = 0;
    for (uint64_t x = gall; x; x &= x - 1) gq[i++] = __builtin_ctzll(x);
  }
  std::vector<uint32_t> x(N);
  std::vector<uint16_t> tab((size_t)N << g);
  for (uint32_t v = 0; v < (1u << g); v++) {
    uint64_t gset = 0;
    for (int i = 0; i < g; i++)
      if ((v >> i) & 1u) gset |= 1ull << gq[i];
    for (uint32_t l = 0; l < N; l++) x[l] = l;
    for (const PB &pb : pbs) {
      if (pb.gc & ~gset) continue;   // a global control reads 0 in these tiles
      for (uint32_t l = 0; l < N; l++) {
        const uint32_t xv = x[l];
        if ((xv & pb.lc) != pb.lc) continue;
        int c = 0;
        for (int j = 0; j < pb.k; j++) c |= (int)((xv >> pb.t[j]) & 1u) << j;
        const int r = pb.perm[c];
        if (r == c) continue;
        uint32_t nv = xv & ~pb.tmask;
        for (int j = 0; j < pb.k; j++) nv |= (uint32_t)((r >> j) & 1) << pb.t[j];
        x[l] = nv;
      }
    }
    // the amplitude at tile slot l ends at x[l]: gather out[x[l]] = in[l]
    uint16_t *t = tab.data() + (size_t)v * N;
    for (uint32_t l = 0; l < N; l++) t[x[l]] = (uint16_t)l;
  }
  while (pool.size() % 16) pool.push_back(0);
  mat0 = (uint32_t)(pool.size() / 16);
  uint8_t hdr[16] = {0};
  const uint32_t g32 = (uint32_t)g;
  std::memcpy(hdr, &g32, 4);
  for (int i = 0; i < g; i++) hdr[4 + i] = (uint8_t)gq[i];
  pool.insert(pool.end(), hdr, hdr + 16);
  const uint8_t *tb = reinterpret_cast<const uint8_t *>(tab.data());
  pool.insert(pool.end(), tb, tb + tab.size() * sizeof(uint16_t));
  return true;
}

// First targets (tile positions) of the blocks of a pass the pipelined
// tensor-core kernel runs.  Block j > 0 is gathered under a layout whose
// pair bit is its first target c_j; it scatters in 16-byte pairs when
// c_j = c_{j+1} (the last block and the store: when c_j = 0), and block 0
// gathers in pairs when c_0 = 0.  Pick c_j among each block's targets to
// maximise those cases (dynamic programming over at most 6 x 5 choices;
// ties go to the lowest tile position).
static std::vector<int> tcp_first_targets(const std::vector<std::vector<int>> &T) {
  const int n = (int)T.size();
  std::vector<std::vector<int>> score(n), from(n);
  for (int j = 0; j < n; j++) {
    score[j].assign(T[j].size(), 0);
    from[j].assign(T[j].size(), -1);
    for (size_t a = 0; a < T[j].size(); a++) {
      int best = j == 0 ? (T[0][a] == 0 ? 1 : 0) : -1;
      if (j > 0)
        for (size_t c = 0; c < T[j - 1].size(); c++) {
          const int v = score[j - 1][c] + (T[j - 1][c] == T[j][a] ? 1 : 0);
          if (v > best) {
            best = v;
            from[j][a] = (int)c;
          }
        }
      score[j][a] = best + (j == n - 1 && T[j][a] == 0 ? 1 : 0);
    }
  }
  std::vector<int> c(n);
  int a = 0;
  for (size_t x = 1; x < T[n - 1].size(); x++)
    if (score[n - 1][x] > score[n - 1][a]) a = (int)x;
  for (int j = n - 1; j >= 0; j--) {
    c[j] = T[j][a];
    a = from[j][a];
  }
  return c;
}

sv_status emit_pass(DeviceProgram &prog, const PassPlan &P, const BuildCtx &b,
                           std::vector<uint32_t> &op0s, const std::vector<int> &batch_mat_off) {
  TilePass tp;
  std::memset(&tp, 0, sizeof(tp));
  tp.n = b.n;
  tp.m = (int)P.S.size();
  tp.L = std::min(b.L, tp.m);
  tp.nvec = b.nvec;
  tp.flags = b.flags;
  int loc[64];
  for (int q = 0; q < 64; q++) loc[q] = -1;
  for (size_t i = 0; i < P.S.size(); i++) loc[P.S[i]] = (int)i;
  for (int j = tp.L; j < tp.m; j++) tp.hi_pos[j - tp.L] = (int8_t)P.S[j];
  int no = 0;
  for (int q = 0; q < b.n; q++)
    if (loc[q] < 0) tp.out_pos[no++] = (int8_t)q;
  op0s.push_back((uint32_t)prog.ops.size());
  const size_t ab = amp_bytes(b.dt);
  if (batch_mat_off.empty() && table_pass(P, b, loc, tp.m, prog.mats, tp.mat0)) {
    tp.nops = 0;
    tp.flags |= kPassTable;
    prog.passes.push_back(tp);
    return SV_OK;
  }
  // a pass for the pipelined tensor-core kernel: its blocks' first targets
  std::vector<int> tc_first;
  {
    bool pure = tp.m == kTcTileM && !P.ops.empty() && P.ops.size() <= (size_t)kTcpMaxBlocks;
    std::vector<std::vector<int>> T;
    for (const Block &blk : P.ops) {
      pure = pure && blk.kind == TOP_TC && blk.qubits.size() == 5;
      if (!pure) break;
      std::vector<int> t;
      for (int q : blk.qubits) t.push_back(loc[q]);
      std::sort(t.begin(), t.end());
      T.push_back(t);
    }
    if (pure) tc_first = tcp_first_targets(T);
  }
  for (size_t bi = 0; bi < P.ops.size(); bi++) {
    const Block &blk = P.ops[bi];
    // the adjoint sweep's probe of a parametric gate directly followed by
    // that gate's U^dagger on both vectors: one fused op
    if (blk.kind == TOP_GRAD && bi + 1 < P.ops.size() && !batch_mat_off.empty()) {
      const Block &u = P.ops[bi + 1];
      if (u.kind == TOP_DENSE && u.inst >= 0 && u.qubits.size() == 1 && u.qubits == blk.qubits &&
          u.controls.empty() && u.vmask == 3 && loc[blk.qubits[0]] >= 0) {
        TileOp op;
        std::memset(&op, 0, sizeof(op));
        op.kind = TOP_GRADU;
        op.k = 1;
        op.vmask = 3;
        op.t[0] = (uint8_t)loc[blk.qubits[0]];
        op.gen = (uint8_t)(blk.gen | kGenBatchMat);
        op.slot = (int16_t)blk.slot;
        op.mat = (uint32_t)batch_mat_off[u.inst];
        prog.ops.push_back(op);
        bi++;
        continue;
      }
    }
    TileOp op;
    std::memset(&op, 0, sizeof(op));
    op.kind = (uint8_t)blk.kind;
    op.k = (uint8_t)blk.qubits.size();
    op.vmask = (uint8_t)blk.vmask;
    for (size_t j = 0; j < blk.qubits.size(); j++) {
      if (loc[blk.qubits[j]] < 0) return set_error(SV_EINVAL, "internal: target outside tile");
      op.t[j] = (uint8_t)loc[blk.qubits[j]];
    }
    uint64_t gcm = 0;
    for (int q : blk.controls) {
      if (loc[q] >= 0) op.lcmask |= 1u << loc[q];
      else gcm |= 1ull << q;
    }
    if (blk.kind == TOP_DENSE && blk.diag) op.kind = TOP_DIAG;
    // 0/1 permutation blocks of complex128 states move amplitudes instead of
    // multiplying by 0 and 1 at the GB300's low FP64 rate (complex64 dense
    // blocks are exact for such matrices and as fast)
    int perm[8];
    if (op.kind == TOP_DENSE && b.dt == SV_C128 && blk.inst < 0 && op.k <= 3 && permutation_of(blk.U, op.k, perm))
      op.kind = TOP_PERM;
    if (op.kind == TOP_PERM) {
      uint32_t fixed = op.lcmask;
      for (int j = 0; j < op.k; j++) fixed |= 1u << op.t[j];
      set_thread_positions(op, fixed, tp.m, b.dt);
      while (prog.mats.size() % 16) prog.mats.push_back(0);
      op.mat = (uint32_t)(prog.mats.size() / ab);
      for (int y = 0; y < (1 << op.k); y++) prog.mats.push_back((uint8_t)perm[y]);
    } else if (op.kind == TOP_DENSE || op.kind == TOP_DIAG) {
      uint32_t fixed = op.lcmask;
      if (op.kind == TOP_DENSE)
        for (int j = 0; j < op.k; j++) fixed |= 1u << op.t[j];
      set_thread_positions(op, fixed, tp.m, b.dt);
      if (blk.inst >= 0 && !batch_mat_off.empty()) {
        op.gen = kGenBatchMat;
        op.mat = (uint32_t)batch_mat_off[blk.inst];
      } else {
        while (prog.mats.size() % 16) prog.mats.push_back(0);   // rows are read 16 bytes at a time
        op.mat = (uint32_t)(prog.mats.size() / ab);
        const int d = 1 << op.k;
        if (op.kind == TOP_DIAG) {
          for (int r = 0; r < d; r++)
            b.dt == SV_C64 ? put_c<float>(prog.mats, blk.U[(size_t)r * d + r])
                           : put_c<double>(prog.mats, blk.U[(size_t)r * d + r]);
        } else if (b.dt == SV_C64 && op.k <= 3) {
          put_pairs_c64(prog.mats, blk.U.data(), op.k);
        } else {
          for (int e = 0; e < d * d; e++)
            b.dt == SV_C64 ? put_c<float>(prog.mats, blk.U[e]) : put_c<double>(prog.mats, blk.U[e]);
        }
      }
    } else if (op.kind == TOP_TC) {
      // targets in increasing tile position, except that in a pipelined
      // pass the block's chosen first target leads (member pairs (y, y+1)
      // then differ in it); U permuted to match; rows of the GEMM on the
      // free tile bits, lane bits chosen to spread a warp's gathers over the
      // banks of the layout the block is gathered under
      const int jop = (int)(prog.ops.size() - op0s.back());
      const int first = tc_first.empty() ? -1 : tc_first[jop];
      int ord[6] = {0, 1, 2, 3, 4, 5};
      std::sort(ord, ord + op.k, [&](int a, int c) {
        if ((op.t[a] == first) != (op.t[c] == first)) return op.t[a] == first;
        return op.t[a] < op.t[c];
      });
      uint8_t tsorted[6];
      for (int j = 0; j < op.k; j++) tsorted[j] = op.t[ord[j]];
      for (int j = 0; j < op.k; j++) op.t[j] = tsorted[j];
      const int d = 1 << op.k;
      std::vector<cd> Up((size_t)d * d);
      auto from_sorted = [&](int x) {
        int y = 0;
        for (int j = 0; j < op.k; j++) y |= ((x >> j) & 1) << ord[j];
        return y;
      };
      for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) Up[(size_t)r * d + c] = blk.U[(size_t)from_sorted(r) * d + from_sorted(c)];
      const int next_pair = tc_first.empty() || jop + 1 >= (int)tc_first.size() ? 0 : tc_first[jop + 1];
      tcp_row_positions(op, tc_first.empty() || jop == 0 ? 0 : first, next_pair);
      while (prog.mats.size() % 16) prog.mats.push_back(0);
      op.mat = (uint32_t)(prog.mats.size() / ab);
      std::vector<uint32_t> packed;
      tc_pack_matrix(Up, (sv_prec)b.prec, packed);
      const uint8_t *pb = reinterpret_cast<const uint8_t *>(packed.data());
      prog.mats.insert(prog.mats.end(), pb, pb + packed.size() * 4);
      tp.flags |= kPassHasTC | ((uint32_t)b.prec << 9);
    } else if (op.kind == TOP_GRAD) {
      op.gen = (uint8_t)blk.gen;
      op.slot = (int16_t)blk.slot;
    } else if (op.kind == TOP_PAULI) {
      uint32_t xl = 0, zl = 0;
      gcm = 0;
      for (int q = 0; q < b.n; q++) {
        if ((blk.xmask >> q) & 1) xl |= 1u << loc[q];
        if ((blk.zmask >> q) & 1) {
          if (loc[q] >= 0) zl |= 1u << loc[q];
          else gcm |= 1ull << q;
        }
      }
      op.slot = (int16_t)xl;
      op.lcmask = zl;
      op.gen = (uint8_t)(__builtin_popcountll(blk.xmask & blk.zmask) & 3);
      op.mat = (uint32_t)prog.coeffs.size();
      prog.coeffs.push_back(blk.coeff);
    } else if (op.kind == TOP_DOT) {
      op.slot = (int16_t)blk.slot;
    }
    op.gcmask_lo = (uint32_t)gcm;
    op.gcmask_hi = (uint16_t)(gcm >> 32);
    prog.ops.push_back(op);
  }
  tp.nops = (int)(prog.ops.size() - op0s.back());
  prog.passes.push_back(tp);
  return SV_OK;
}

static constexpr int kMaxOpsPerPass = 256;
static constexpr int kMaxMatPerPass = 1 << 16;


static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

ProgLayout layout_of(const DeviceProgram &p, size_t tbl_bytes, size_t pmats_bytes) {
  ProgLayout L;
  L.ops_off = 0;
  L.mats_off = align256(p.ops.size() * sizeof(TileOp));
  L.coeffs_off = align256(L.mats_off + p.mats.size());
  L.tbl_off = align256(L.coeffs_off + p.coeffs.size() * sizeof(double));
  L.pmats_off = align256(L.tbl_off + tbl_bytes);
  L.end = align256(L.pmats_off + pmats_bytes);
  return L;
}

// Copy host bytes to device memory `dst` through the state's pinned buffer
// (at most kWsProgBytes per call), ordered on the state's stream.
sv_status stage_upload_to(sv_state *s, void *dst, const std::vector<std::pair<const void *, size_t>> &parts,
                          const std::vector<size_t> &offs, size_t total) {
  if (total > kWsProgBytes) return set_error(SV_ENOMEM, "upload exceeds the staging buffer");
  SV_CUDA(cudaEventSynchronize(s->staged));
  for (size_t i = 0; i < parts.size(); i++)
    if (parts[i].second) std::memcpy(s->pinned + offs[i], parts[i].first, parts[i].second);
  SV_CUDA(cudaMemcpyAsync(dst, s->pinned, total, cudaMemcpyHostToDevice, s->stream));
  SV_CUDA(cudaEventRecord(s->staged, s->stream));
  return SV_OK;
}

// Copy host bytes into the workspace program area.
sv_status stage_upload(sv_state *s, const std::vector<std::pair<const void *, size_t>> &parts,
                       const std::vector<size_t> &offs, size_t total) {
  if (total > kWsProgBytes) return set_error(SV_ENOMEM, "gate program exceeds the workspace program area");
  SV_TRY(stage_upload_to(s, s->ws + kWsProg, parts, offs, total));
  s->resident = 0;
  return SV_OK;
}

sv_status launch_any_pass(sv_state *s, const TilePass &tp, int batch, cudaStream_t st, const HostPass *host) {
  if (!(tp.flags & kPassTC)) return launch_tile_pass_on(s, tp, batch, st, host);
  int t[6];
  for (int j = 0; j < 6; j++) t[j] = tp.hi_pos[j];
  const uint32_t *b = reinterpret_cast<const uint32_t *>(static_cast<const char *>(tp.mats) + 16 * (size_t)tp.mat0);
  if (tp.L == 6) return launch_dense_tc6(s, tp.v0, t, b, 0, st);
  return launch_dense_tc(s, tp.v0, t, b, (sv_prec)((tp.flags >> 9) & 3), 0, st);
}

// Launch every pass of a program.
sv_status launch_program(sv_state *s, const DeviceProgram &p, const ProgLayout &L,
                                const std::vector<uint32_t> &op0s, const LaunchEnv &E, cudaStream_t st) {
  if (!st) st = s->stream;
  char *base = s->ws + kWsProg;
  for (size_t i = 0; i < p.passes.size(); i++) {
    TilePass tp = p.passes[i];
    tp.ops = reinterpret_cast<const TileOp *>(base + L.ops_off) + op0s[i];
    tp.mats = base + L.mats_off;
    tp.coeffs = reinterpret_cast<const double *>(base + L.coeffs_off);
    tp.pmats = E.pmats;
    tp.pmats_stride = E.pmats_stride;
    tp.acc = E.acc;
    tp.acc_stride = E.acc_stride;
    tp.tbl0 = E.tbl0;
    tp.tbl1 = E.tbl1;
    tp.v0 = E.v0;
    tp.v1 = E.v1;
    tp.err = reinterpret_cast<uint32_t *>(s->ws + kWsCtrl + kWsErrFlag);
    const HostPass hp{p.ops.data() + op0s[i], p.mats.data()};
    SV_TRY(launch_any_pass(s, tp, E.batch, st, &hp));
  }
  return SV_OK;
}

static ProgCache<CachedProgram> g_cache(kProgramCacheDefault);

// Pad a block of k < 5 qubits to a 5-qubit block U' = I (x) U over idle
// qubits of its pass's tile (tile qubits S, tile position p <-> S[p]): tile
// positions 7 and 11, which do not steer the pipelined kernel's bank
// mapping, first, then the highest free ones.
static void pad_in_tile(Block &blk, const std::vector<int> &S) {
  static const int kOrder[12] = {7, 11, 10, 9, 8, 6, 5, 4, 3, 2, 1, 0};
  const int k = (int)blk.qubits.size(), d = 1 << k;
  for (int p : kOrder) {
    if ((int)blk.qubits.size() == 5) break;
    if (p >= (int)S.size()) continue;
    if (std::find(blk.qubits.begin(), blk.qubits.end(), S[p]) == blk.qubits.end()) blk.qubits.push_back(S[p]);
  }
  std::vector<cd> U5(32 * 32, 0.0);
  for (int r = 0; r < 32; r++)
    for (int c = 0; c < 32; c++)
      if ((r >> k) == (c >> k)) U5[(size_t)r * 32 + c] = blk.U[(size_t)(r & (d - 1)) * d + (c & (d - 1))];
  blk.U = std::move(U5);
  blk.diag = false;
}

// One dense block of 5 or 6 qubits as a tensor-core pass of its own.
static sv_status emit_tc_pass(CachedProgram &out, const Block &blk, int n, int prec) {
  TilePass tp;
  std::memset(&tp, 0, sizeof(tp));
  tp.n = n;
  tp.m = n;
  tp.L = (int)blk.qubits.size();
  tp.nvec = 1;
  tp.flags = kPassTC | ((uint32_t)prec << 9);
  for (int j = 0; j < tp.L; j++) tp.hi_pos[j] = (int8_t)blk.qubits[j];
  while (out.prog.mats.size() % 16) out.prog.mats.push_back(0);
  tp.mat0 = (uint32_t)(out.prog.mats.size() / 16);
  std::vector<uint32_t> packed;
  tc_pack_matrix(blk.U, (sv_prec)prec, packed);
  const uint8_t *pb = reinterpret_cast<const uint8_t *>(packed.data());
  out.prog.mats.insert(out.prog.mats.end(), pb, pb + packed.size() * 4);
  out.op0s.push_back((uint32_t)out.prog.ops.size());
  out.prog.passes.push_back(tp);
  return SV_OK;
}

static sv_status build_circuit_program(sv_state *s, const std::vector<Gate> &gates, const Opts &o,
                                       CachedProgram &out) {
  out.blocks = fuse(gates, o.fusion_k);
  if (o.mode == SV_MODE_PER_GATE) return SV_OK;
  int m = o.tile_m, L = o.L;
  if (!fit_tile(out.blocks, s->n, lmin(s->dt), mmax(s->dt, 1), m, L))
    return set_error(SV_EUNSUPPORTED, "a fused block does not fit a shared-memory tile");
  if (o.fusion_k >= 2 && m < s->n) {
    // blocks that meet inside a pass merge (one pass-sized op instead of two)
    const std::vector<PassPlan> first = plan_passes(out.blocks, s->n, m, L, kMaxOpsPerPass, kMaxMatPerPass);
    if (!first.empty()) {
      std::vector<Block> merged = merge_in_passes(first, o.fusion_k);
      int m2 = m, L2 = L;
      if (merged.size() < out.blocks.size() && fit_tile(merged, s->n, lmin(s->dt), mmax(s->dt, 1), m2, L2)) {
        out.blocks = std::move(merged);
        m = m2;
        L = L2;
      }
    }
  }
  BuildCtx b{s->dt, s->n, m, L, 1, 0, o.prec};
  // With a tensor-core precision mode, dense 5-qubit blocks run on the tensor
  // cores: inside 12-qubit tile passes (TOP_TC ops) when the tile size is
  // 12, otherwise as passes of their own between the tile passes.
  const bool tc = o.prec != SV_PREC_PLAIN && s->dt == SV_C64 && s->n >= 12;
  // a dense 4-qubit block would be the slowest op of a tile pass on CUDA
  // cores: pad it with an idle qubit (U x I) and run it on the tensor cores
  auto pad4 = [](Block &blk) {
    if (!(blk.kind == TOP_DENSE && blk.qubits.size() == 4 && blk.controls.empty() && !blk.diag)) return;
    int extra = 0;
    while (std::find(blk.qubits.begin(), blk.qubits.end(), extra) != blk.qubits.end()) extra++;
    std::vector<cd> U5(32 * 32, 0.0);
    for (int r = 0; r < 32; r++)
      for (int c = 0; c < 32; c++)
        if ((r >> 4) == (c >> 4)) U5[(size_t)r * 32 + c] = blk.U[(size_t)(r & 15) * 16 + (c & 15)];
    blk.U = U5;
    blk.qubits.push_back(extra);
  };
  if (tc && m == kTcTileM && o.tc_in_tile) {
    // Split-BF16: every uncontrolled dense or diagonal block of at most 5
    // qubits runs on the tensor cores (padded to 5 qubits with idle tile
    // qubits once its pass is known), so most passes hold tensor-core blocks
    // only and take the pipelined kernel; at most kTcpMaxBlocks per pass,
    // whose operands stay in shared memory (each counts 1024 entries).
    // Split-TF32: dense 4- and 5-qubit blocks only.
    const bool bf16 = o.prec == SV_PREC_TC_BF16X3;
    for (Block &blk : out.blocks) {
      if (bf16) {
        if (blk.kind == TOP_DENSE && blk.controls.empty() && blk.qubits.size() <= 5) blk.kind = TOP_TC;
      } else {
        pad4(blk);
        if (blk.kind == TOP_DENSE && blk.qubits.size() == 5 && blk.controls.empty() && !blk.diag) blk.kind = TOP_TC;
      }
    }
    const int mat_cap = bf16 ? kTcpMaxBlocks * 1024 + 1023 : kMaxMatPerPass;
    std::vector<Block> seg;
    auto flush_tc = [&]() -> sv_status {
      if (seg.empty()) return SV_OK;
      std::vector<PassPlan> passes = plan_passes(seg, s->n, m, L, kMaxOpsPerPass, mat_cap);
      if (passes.empty()) return set_error(SV_EINVAL, "internal: pass planning failed");
      for (PassPlan &P : passes) {
        for (Block &blk : P.ops)
          if (blk.kind == TOP_TC && blk.qubits.size() < 5) pad_in_tile(blk, P.S);
        SV_TRY(emit_pass(out.prog, P, b, out.op0s, {}));
      }
      seg.clear();
      return SV_OK;
    };
    for (const Block &blk : out.blocks) {
      // split-BF16: an uncontrolled dense 6-qubit block (fusion width 6) is
      // a tensor-core pass of its own, between the tile passes
      const bool six = bf16 && s->n >= 13 && blk.kind == TOP_DENSE && blk.qubits.size() == 6 &&
                       blk.controls.empty() && !blk.diag;
      if (!six) {
        seg.push_back(blk);
        continue;
      }
      SV_TRY(flush_tc());
      SV_TRY(emit_tc_pass(out, blk, s->n, o.prec));
    }
    SV_TRY(flush_tc());
    out.lay = layout_of(out.prog, 0, 0);
    return SV_OK;
  }
  std::vector<Block> seg;
  auto flush = [&]() -> sv_status {
    if (seg.empty()) return SV_OK;
    std::vector<PassPlan> passes = plan_passes(seg, s->n, m, L, kMaxOpsPerPass, kMaxMatPerPass);
    if (passes.empty()) return set_error(SV_EINVAL, "internal: pass planning failed");
    for (const PassPlan &P : passes) SV_TRY(emit_pass(out.prog, P, b, out.op0s, {}));
    seg.clear();
    return SV_OK;
  };
  for (const Block &blk0 : out.blocks) {
    Block blk = blk0;
    if (tc) pad4(blk);
    const bool is_tc = tc && blk.kind == TOP_DENSE && blk.qubits.size() == 5 && blk.controls.empty() && !blk.diag;
    if (!is_tc) {
      seg.push_back(blk);
      continue;
    }
    SV_TRY(flush());
    SV_TRY(emit_tc_pass(out, blk, s->n, o.prec));
  }
  SV_TRY(flush());
  out.lay = layout_of(out.prog, 0, 0);
  return SV_OK;
}

static sv_status run_blocks_per_gate(sv_state *s, const std::vector<Block> &blocks) {
  for (const Block &b : blocks) {
    if (b.diag && b.qubits.size() + b.controls.size() <= 8) {
      const int d = 1 << (int)b.qubits.size();
      std::vector<cd> dg(d);
      for (int r = 0; r < d; r++) dg[r] = b.U[(size_t)r * d + r];
      SV_TRY(launch_diag_gate(s, b.qubits, b.controls, dg));
    } else {
      SV_TRY(launch_dense_gate(s, b.qubits, b.controls, b.U));
    }
  }
  return SV_OK;
}

sv_status upload_program(sv_state *s, const CachedProgram &cp) {
  if (s->resident == cp.serial && cp.serial != 0) return SV_OK;
  const DeviceProgram &p = cp.prog;
  std::vector<std::pair<const void *, size_t>> parts = {
      {p.ops.data(), p.ops.size() * sizeof(TileOp)},
      {p.mats.data(), p.mats.size()},
      {p.coeffs.data(), p.coeffs.size() * sizeof(double)}};
  std::vector<size_t> offs = {cp.lay.ops_off, cp.lay.mats_off, cp.lay.coeffs_off};
  SV_TRY(stage_upload(s, parts, offs, cp.lay.end));
  s->resident = cp.serial;
  return SV_OK;
}

sv_status get_program(sv_state *s, const sv_circuit *c, const double *params, const sv_options *opt,
                      ProgramRef *out, Opts *o_out) {
  if (!s) return set_error(SV_EINVAL, "null state");
  if (!c) return set_error(SV_EINVAL, "null circuit");
  Opts o = resolve(s, opt, 1);
  tuned_options(s, c, opt, o);
  KeyBytes k;
  k.val((int)0x51);
  circuit_key(k, c);
  k.val(o.fusion_k);
  k.val(o.tile_m);
  k.val(o.L);
  k.val(o.mode);
  k.val(o.prec);
  k.val(o.tc_in_tile);
  k.val((int)s->dt);
  if (params && c->n_params > 0) k.bytes(params, sizeof(double) * c->n_params);
  const uint64_t h = k.hash();
  ProgramRef cp = g_cache.find(s, k, h);
  if (!cp) {
    std::vector<Gate> gates;
    SV_TRY(circuit_to_gates(c, params, s->n, gates, false));
    auto built = std::make_shared<CachedProgram>();
    SV_TRY(build_circuit_program(s, gates, o, *built));
    built->serial = next_program_serial();
    cp = g_cache.insert(s, k, h, std::move(built));
  }
  *out = std::move(cp);
  *o_out = o;
  return SV_OK;
}

}  // namespace sv

using namespace sv;
static_assert(sizeof(sv_op) == 104, "sv_op layout is part of the ABI");
static_assert(sizeof(sv_pauli_term) == 24, "sv_pauli_term layout is part of the ABI");
static_assert(sizeof(sv_options) == 24, "sv_options layout is part of the ABI");

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *sv_last_error(void) { return g_err.c_str(); }

const char *sv_status_string(sv_status st) {
  switch (st) {
    case SV_OK: return "SV_OK";
    case SV_EINVAL: return "SV_EINVAL";
    case SV_ENOMEM: return "SV_ENOMEM";
    case SV_ECUDA: return "SV_ECUDA";
    case SV_ETIMEOUT: return "SV_ETIMEOUT";
    case SV_EUNSUPPORTED: return "SV_EUNSUPPORTED";
    default: return "unknown";
  }
}

uint64_t sv_kernel_launch_count(void) { return g_launches.load(); }

int64_t sv_program_cache_limit(int64_t max_programs) {
  return (int64_t)g_cache.set_limit(max_programs > 0 ? (size_t)max_programs : 0);
}

size_t sv_workspace_bytes(int n, sv_dtype dt) {
  (void)dt;
  if (n < 1 || n > 34) return 0;
  return kWsRed + red_bytes(n);
}

sv_status sv_create(int n, sv_dtype dt, void *amps, size_t amps_bytes, void *ws, size_t ws_bytes,
                    void *stream, sv_state **out) {
  if (!out) return set_error(SV_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > 34) return set_error(SV_EINVAL, "n_qubits must be in [1, 34]");
  if (dt != SV_C64 && dt != SV_C128) return set_error(SV_EINVAL, "unknown dtype");
  if (!amps || !ws) return set_error(SV_EINVAL, "null device pointer");
  if (((uintptr_t)amps & 255) || ((uintptr_t)ws & 255))
    return set_error(SV_EINVAL, "device buffers must be 256-byte aligned");
  if (amps_bytes < ((size_t)1 << n) * amp_bytes(dt)) return set_error(SV_EINVAL, "amplitude buffer too small");
  if (ws_bytes < sv_workspace_bytes(n, dt))
    return set_error(SV_ENOMEM, "workspace smaller than sv_workspace_bytes()");
  cudaPointerAttributes attr;
  SV_CUDA(cudaPointerGetAttributes(&attr, amps));
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return set_error(SV_EINVAL, "amplitudes must be device memory");
  sv_state *s = new (std::nothrow) sv_state();
  if (!s) return set_error(SV_ENOMEM, "host allocation failed");
  s->n = n;
  s->dt = dt;
  s->amps = amps;
  s->amps_bytes = amps_bytes;
  s->ws = (char *)ws;
  s->ws_bytes = ws_bytes;
  s->stream = (cudaStream_t)stream;
  s->device = attr.device;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != s->device) cudaSetDevice(s->device);
  cudaError_t e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&s->pinned, kPinnedBytes);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->staged, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(s->staged, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->ws + kWsCtrl + kWsErrFlag, 0, sizeof(uint32_t), s->stream);
  if (e != cudaSuccess) {
    if (s->pinned) cudaFreeHost(s->pinned);
    delete s;
    return cuda_error(e, "sv_create");
  }
  s->pinned_bytes = kPinnedBytes;
  *out = s;
  return SV_OK;
}

sv_status sv_destroy(sv_state *s) {
  if (!s) return SV_OK;
  cudaStreamSynchronize(s->stream);
  g_cache.drop_owner(s);
  drop_adjoint_programs(s);
  drop_graphs(s);
  if (s->capture) cudaStreamDestroy(s->capture);
  for (int k = 0; k < kFanStreams; k++) {
    if (s->fan[k]) cudaStreamDestroy(s->fan[k]);
    if (s->fan_join[k]) cudaEventDestroy(s->fan_join[k]);
  }
  if (s->fan_fork) cudaEventDestroy(s->fan_fork);
  if (s->staged) cudaEventDestroy(s->staged);
  if (s->pinned) cudaFreeHost(s->pinned);
  delete s;
  return SV_OK;
}

sv_status sv_set_basis(sv_state *s, uint64_t index) {
  if (!s) return set_error(SV_EINVAL, "null state");
  if (index >= (1ull << s->n)) return set_error(SV_EINVAL, "basis index out of range");
  s->basis_known = false;
  SV_TRY(launch_set_basis(s, index));
  s->basis_known = true;
  s->basis_index = index;
  s->basis_amp = 1.0;
  return SV_OK;
}

sv_status sv_mark_modified(sv_state *s) {
  if (!s) return set_error(SV_EINVAL, "null state");
  s->basis_known = false;
  return SV_OK;
}

// The device address of page-locked host memory (16-byte aligned), or null
// for any other host pointer.
static const void *mapped_host(const void *host) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, host) != cudaSuccess) {
    cudaGetLastError();   // unregistered memory on older runtimes: not an error
    return nullptr;
  }
  if (attr.type != cudaMemoryTypeHost || !attr.devicePointer || (uintptr_t)attr.devicePointer % 16) return nullptr;
  return attr.devicePointer;
}

sv_status sv_upload(sv_state *s, const void *host, size_t bytes) {
  if (!s || !host) return set_error(SV_EINVAL, "null argument");
  if (bytes != ((size_t)1 << s->n) * amp_bytes(s->dt)) return set_error(SV_EINVAL, "size mismatch");
  s->basis_known = false;
  if (const void *dev = mapped_host(host); dev && bytes % 16 == 0)
    SV_TRY(launch_copy16(s, dev, s->amps, bytes));
  else
    SV_CUDA(cudaMemcpyAsync(s->amps, host, bytes, cudaMemcpyHostToDevice, s->stream));
  SV_CUDA(cudaStreamSynchronize(s->stream));
  return SV_OK;
}

sv_status sv_download(sv_state *s, void *host, size_t bytes) {
  if (!s || !host) return set_error(SV_EINVAL, "null argument");
  if (bytes != ((size_t)1 << s->n) * amp_bytes(s->dt)) return set_error(SV_EINVAL, "size mismatch");
  if (const void *dev = mapped_host(host); dev && bytes % 16 == 0)
    SV_TRY(launch_copy16(s, s->amps, const_cast<void *>(dev), bytes));
  else
    SV_CUDA(cudaMemcpyAsync(host, s->amps, bytes, cudaMemcpyDeviceToHost, s->stream));
  SV_CUDA(cudaStreamSynchronize(s->stream));
  return SV_OK;
}

sv_status sv_synchronize(sv_state *s) {
  if (!s) return set_error(SV_EINVAL, "null state");
  uint32_t *flag = reinterpret_cast<uint32_t *>(s->ws + kWsCtrl + kWsErrFlag);
  uint32_t *host = reinterpret_cast<uint32_t *>(s->pinned + kWsProgBytes + 4096);
  SV_CUDA(cudaMemcpyAsync(host, flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream));
  SV_CUDA(cudaStreamSynchronize(s->stream));
  if (*host) {
    const uint32_t bits = *host;
    SV_CUDA(cudaMemsetAsync(flag, 0, sizeof(uint32_t), s->stream));
    SV_CUDA(cudaStreamSynchronize(s->stream));
    if (bits & kErrNoInlineBlock)
      return set_error(SV_EUNSUPPORTED, "internal: a tile pass met a block missing from its parameter block");
    return set_error(SV_ETIMEOUT, "a bounded device wait ran out; the last batch is incomplete");
  }
  return SV_OK;
}

sv_status sv_apply_gate(sv_state *s, const int32_t *targets, int k, const int32_t *controls, int nctrl,
                        const double *matrix, int adjoint) {
  if (!s || !targets || !matrix) return set_error(SV_EINVAL, "null argument");
  if (k < 1 || k > 6) return set_error(SV_EINVAL, "k must be in [1, 6]");
  if (nctrl < 0 || nctrl > 8 || (nctrl > 0 && !controls)) return set_error(SV_EINVAL, "bad controls");
  uint64_t seen = 0;
  std::vector<int> t(k), c(nctrl);
  for (int j = 0; j < k + nctrl; j++) {
    const int q = j < k ? targets[j] : controls[j - k];
    if (q < 0 || q >= s->n) return set_error(SV_EINVAL, "qubit out of range");
    if ((seen >> q) & 1) return set_error(SV_EINVAL, "duplicate qubit (or control overlaps a target)");
    seen |= 1ull << q;
    (j < k ? t[j] : c[j - k]) = q;
  }
  const int d = 1 << k;
  std::vector<cd> U((size_t)d * d);
  for (int e = 0; e < d * d; e++) U[e] = cd(matrix[2 * e], matrix[2 * e + 1]);
  if (unitarity_checks() && unitarity_error(U, k) > kUnitaryTol)
    return set_error(SV_EINVAL, "matrix is not unitary");
  s->basis_known = false;
  if (adjoint) U = adjoint_of(U, k);
  bool diag = true;
  for (int r = 0; r < d && diag; r++)
    for (int cc = 0; cc < d; cc++)
      if (r != cc && U[(size_t)r * d + cc] != cd(0.0)) {
        diag = false;
        break;
      }
  if (diag && k + nctrl <= 8) {
    std::vector<cd> dg(d);
    for (int r = 0; r < d; r++) dg[r] = U[(size_t)r * d + r];
    return launch_diag_gate(s, t, c, dg);
  }
  return launch_dense_gate(s, t, c, U);
}


sv_status sv_apply_circuit(sv_state *s, const sv_circuit *c, const double *params, const sv_options *opt) {
  if (s && c && s->basis_known) {
    // a basis state through permutation and phase gates stays a basis
    // state: follow it on the host and rewrite two amplitudes, with no pass
    // over the state (exact: only the FP64 phases are rounded, once)
    std::vector<Gate> gates;
    SV_TRY(circuit_to_gates(c, params, s->n, gates, false));
    uint64_t idx = s->basis_index;
    cd amp = s->basis_amp;
    if (propagate_basis(gates, idx, amp)) {
      SV_TRY(launch_move_basis(s, s->basis_index, idx, amp));
      s->basis_index = idx;
      s->basis_amp = amp;
      return SV_OK;
    }
  }
  ProgramRef cp;
  Opts o;
  SV_TRY(get_program(s, c, params, opt, &cp, &o));
  s->basis_known = false;
  if (o.mode == SV_MODE_PER_GATE) return run_blocks_per_gate(s, cp->blocks);
  SV_TRY(upload_program(s, *cp));
  LaunchEnv E;
  E.v0 = s->amps;
  return launch_program(s, cp->prog, cp->lay, cp->op0s, E);
}

sv_status sv_plan_info(sv_state *s, const sv_circuit *c, const double *params, const sv_options *opt,
                       int64_t *n_blocks, int64_t *n_passes) {
  ProgramRef cp;
  Opts o;
  SV_TRY(get_program(s, c, params, opt, &cp, &o));
  if (n_blocks) *n_blocks = (int64_t)cp->blocks.size();
  if (n_passes) *n_passes = o.mode == SV_MODE_PER_GATE ? (int64_t)cp->blocks.size() : (int64_t)cp->prog.passes.size();
  return SV_OK;
}

sv_status sv_plan_fmas(sv_state *s, const sv_circuit *c, const double *params, const sv_options *opt,
                       double *fma_per_amp) {
  if (!fma_per_amp) return set_error(SV_EINVAL, "null argument");
  ProgramRef cp;
  Opts o;
  SV_TRY(get_program(s, c, params, opt, &cp, &o));
  double f = 0;
  for (const Block &b : cp->blocks) {
    // split-BF16 tile passes run every tensor-core block as a 5-qubit block
    if (b.kind == TOP_TC) {
      f += 4.0 * 32.0;
      continue;
    }
    if (b.kind != TOP_DENSE) continue;
    const double share = std::ldexp(1.0, -(int)b.controls.size());
    f += b.diag ? 4.0 * share : 4.0 * std::ldexp(1.0, (int)b.qubits.size()) * share;
  }
  *fma_per_amp = f;
  return SV_OK;
}

}  // extern "C"
