// Host interpreter of the tile-pass programs the library builds (test only).
//
// Runs the library's own fusion planner, pass planner and program emitter
// (linked from its object files) on a circuit, then executes the emitted
// TilePass / TileOp lists on the CPU in complex128 exactly as the tile
// kernels define them: per tile, gather the 2^m amplitudes of the pass's
// qubit set, apply the ops in order, scatter.  The tests compare the result
// with the FP64 oracle, which checks the planning and emission logic without
// a GPU.
#include <complex>
#include <cstdio>
#include <cstring>
#include <set>
#include <vector>

#include "../../paper_2106_13995_gb300/csrc/sv_internal.h"

using namespace sv;

static uint32_t ins0_h(uint32_t x, int p) {
  const uint32_t lo = x & ((1u << p) - 1);
  return ((x ^ lo) << 1) | lo;
}
static uint32_t ins0_mask_h(uint32_t x, uint32_t f) {
  while (f) {
    const int p = __builtin_ctz(f);
    f &= f - 1;
    x = ins0_h(x, p);
  }
  return x;
}

// permutation passes met by plan_emulate so far (read and reset by
// table_pass_count)
static int g_table_passes = 0;
extern "C" int table_pass_count() {
  const int n = g_table_passes;
  g_table_passes = 0;
  return n;
}

// A permutation pass (kPassTable): the tile's amplitudes moved through the
// gather table for the tile's global control values, out[y] = in[table[y]].
template <typename V>
static void apply_table_pass(const DeviceProgram &prog, const TilePass &tp, uint64_t base, V &v) {
  const uint8_t *blk = prog.mats.data() + 16 * (size_t)tp.mat0;
  uint32_t g;
  std::memcpy(&g, blk, 4);
  uint32_t var = 0;
  for (uint32_t i = 0; i < g; i++) var |= (uint32_t)((base >> blk[4 + i]) & 1ull) << i;
  const uint32_t TS = 1u << tp.m;
  const uint16_t *tab = reinterpret_cast<const uint16_t *>(blk + 16) + (size_t)var * TS;
  V w(v.size());
  for (uint32_t y = 0; y < TS; y++) w[y] = v[tab[y]];
  v.swap(w);
}

// returns the number of passes, or -1 (message printed)
extern "C" int plan_emulate(const sv_circuit *c, double *psi_, int fusion_k, int m, int L, int *n_blocks,
                            int merge) {
  std::vector<Gate> gates;
  if (circuit_to_gates(c, nullptr, c->n_qubits, gates, false) != SV_OK) {
    std::printf("circuit rejected: %s\n", sv_last_error());
    return -1;
  }
  const int n = c->n_qubits;
  std::vector<Block> blocks = fuse(gates, fusion_k);
  if (n_blocks) *n_blocks = (int)blocks.size();
  if (!fit_tile(blocks, n, 0, 16, m, L)) {
    std::printf("blocks do not fit a tile\n");
    return -1;
  }
  std::vector<PassPlan> passes = plan_passes(blocks, n, m, L, 256, 1 << 16);
  if (merge && fusion_k >= 2 && !passes.empty()) {
    // the library's merging of blocks that meet inside a pass, then a new plan
    blocks = merge_in_passes(passes, fusion_k);
    if (n_blocks) *n_blocks = (int)blocks.size();
    if (!fit_tile(blocks, n, 0, 16, m, L)) {
      std::printf("merged blocks do not fit a tile\n");
      return -1;
    }
    passes = plan_passes(blocks, n, m, L, 256, 1 << 16);
  }
  if (passes.empty() && !blocks.empty()) {
    std::printf("planning failed\n");
    return -1;
  }
  DeviceProgram prog;
  std::vector<uint32_t> op0s;
  BuildCtx bc{SV_C128, n, m, L, 1, 0};
  for (const PassPlan &P : passes)
    if (emit_pass(prog, P, bc, op0s, {}) != SV_OK) {
      std::printf("emit failed: %s\n", sv_last_error());
      return -1;
    }
  typedef std::complex<double> cx;
  cx *psi = reinterpret_cast<cx *>(psi_);
  const cx *mats = reinterpret_cast<const cx *>(prog.mats.data());
  for (size_t pi = 0; pi < prog.passes.size(); pi++) {
    const TilePass &tp = prog.passes[pi];
    const uint32_t TS = 1u << tp.m;
    g_table_passes += (tp.flags & kPassTable) ? 1 : 0;
    for (uint64_t t = 0; t < (1ull << (n - tp.m)); t++) {
      uint64_t base = 0;
      for (int j = 0; j < n - tp.m; j++) base |= ((t >> j) & 1ull) << tp.out_pos[j];
      std::vector<uint64_t> gi(TS);
      for (uint32_t l = 0; l < TS; l++) {
        uint64_t g = l & ((1u << tp.L) - 1);
        for (int b = tp.L; b < tp.m; b++) g |= (uint64_t)((l >> b) & 1u) << tp.hi_pos[b - tp.L];
        gi[l] = base | g;
      }
      std::vector<cx> v(TS);
      for (uint32_t l = 0; l < TS; l++) v[l] = psi[gi[l]];
      if (tp.flags & kPassTable) apply_table_pass(prog, tp, base, v);
      for (int oi = 0; oi < tp.nops; oi++) {
        const TileOp &op = prog.ops[op0s[pi] + oi];
        const uint64_t gcm = (uint64_t)op.gcmask_lo | ((uint64_t)op.gcmask_hi << 32);
        if ((base & gcm) != gcm) continue;
        const cx *U = mats + op.mat;
        const int K = op.k, D = 1 << K;
        if (op.kind == TOP_DIAG) {
          for (uint32_t g = 0; g < (TS >> __builtin_popcount(op.lcmask)); g++) {
            const uint32_t l = ins0_mask_h(g, op.lcmask) | op.lcmask;
            uint32_t r = 0;
            for (int j = 0; j < K; j++) r |= ((l >> op.t[j]) & 1u) << j;
            v[l] = U[r] * v[l];
          }
        } else if (op.kind == TOP_DENSE || op.kind == TOP_PERM) {
          std::vector<cx> Up;
          if (op.kind == TOP_PERM) {   // table perm[c] = row of column c's 1
            const uint8_t *perm = prog.mats.data() + (size_t)op.mat * sizeof(cx);
            Up.assign((size_t)D * D, 0.0);
            for (int q = 0; q < D; q++) Up[(size_t)perm[q] * D + q] = 1.0;
            U = Up.data();
          }
          std::vector<uint32_t> off(D);
          for (int y = 0; y < D; y++) {
            uint32_t o = 0;
            for (int j = 0; j < K; j++) o |= (uint32_t)((y >> j) & 1) << op.t[j];
            off[y] = o;
          }
          const uint32_t fixed = off[D - 1] | op.lcmask;
          for (uint32_t g = 0; g < (TS >> __builtin_popcount(fixed)); g++) {
            const uint32_t i0 = ins0_mask_h(g, fixed) | op.lcmask;
            std::vector<cx> x(D);
            for (int y = 0; y < D; y++) x[y] = v[i0 + off[y]];
            for (int r = 0; r < D; r++) {
              cx a = 0;
              for (int y = 0; y < D; y++) a += U[(size_t)r * D + y] * x[y];
              v[i0 + off[r]] = a;
            }
          }
        } else {
          std::printf("unexpected op kind %d\n", op.kind);
          return -1;
        }
      }
      for (uint32_t l = 0; l < TS; l++) psi[gi[l]] = v[l];
    }
  }
  return (int)prog.passes.size();
}

// The complex64 program of a circuit, checked op by op against the device's
// group enumeration: thread t's first group sits at l(t) = OR over bits i of t
// of 1 << (TileOp.tbpos nibble i), trip c adds ins0_mask(c << shift, hi) with
// the trip map of the thread count T (fixed positions up to the trip region
// shift it, those above are inserted).  For T = the tile pass's thread count
// and 512 (the persistent kernel) every op's groups must come out exactly
// once.  Returns the number of ops checked, or -1 (message printed);
// *spread counts ops whose lanes 0..15 reach 16 different bank rows of the
// swizzled layout (slot l ^ ((l >> 4) & 15), modulo 16).
extern "C" int check_thread_positions(const sv_circuit *c, int fusion_k, int m, int L, int *spread) {
  std::vector<Gate> gates;
  if (circuit_to_gates(c, nullptr, c->n_qubits, gates, false) != SV_OK) return -1;
  const int n = c->n_qubits;
  std::vector<Block> blocks = fuse(gates, fusion_k);
  if (!fit_tile(blocks, n, 1, 14, m, L)) return -1;
  std::vector<PassPlan> passes = plan_passes(blocks, n, m, L, 256, 1 << 16);
  DeviceProgram prog;
  std::vector<uint32_t> op0s;
  BuildCtx bc{SV_C64, n, m, L, 1, 0};
  for (const PassPlan &P : passes)
    if (emit_pass(prog, P, bc, op0s, {}) != SV_OK) return -1;
  int checked = 0, good = 0;
  for (size_t pi = 0; pi < prog.passes.size(); pi++) {
    const TilePass &tp = prog.passes[pi];
    for (int oi = 0; oi < tp.nops; oi++) {
      const TileOp &op = prog.ops[op0s[pi] + oi];
      if (op.kind != TOP_DENSE && op.kind != TOP_DIAG && op.kind != TOP_PERM) continue;
      uint32_t fixed = op.lcmask;
      if (op.kind == TOP_DENSE || op.kind == TOP_PERM)
        for (int j = 0; j < op.k; j++) fixed |= 1u << op.t[j];
      const uint32_t ngroups = 1u << (tp.m - __builtin_popcount(fixed));
      auto thread_l = [&](uint32_t t) {
        uint32_t l = 0;
        for (int i = 0; i < 9; i++) l |= ((t >> i) & 1u) << ((op.tbpos[i >> 1] >> (4 * (i & 1))) & 15u);
        return l;
      };
      for (int T : {tile_threads(tp.m, SV_C64), 512}) {
        uint32_t low = (uint32_t)__builtin_ctz((uint32_t)T), f = fixed;
        while (f) {
          const uint32_t q = (uint32_t)__builtin_ctz(f);
          if (q > low) break;
          f &= f - 1;
          low++;
        }
        const uint32_t nthr = ngroups < (uint32_t)T ? ngroups : (uint32_t)T;
        const uint32_t ntrips = ngroups > (uint32_t)T ? ngroups / (uint32_t)T : 1u;
        std::multiset<uint32_t> got, want;
        for (uint32_t t = 0; t < nthr; t++)
          for (uint32_t cc = 0; cc < ntrips; cc++) got.insert(thread_l(t) ^ ins0_mask_h(cc << low, f));
        for (uint32_t g = 0; g < ngroups; g++) want.insert(ins0_mask_h(g, fixed));
        if (got != want) {
          std::printf("pass %zu op %d (k %d, fixed %x, T %d): groups differ\n", pi, oi, op.k, fixed, T);
          return -1;
        }
      }
      if (ngroups >= 16) {
        uint32_t rows = 0;
        for (uint32_t t = 0; t < 16; t++) {
          const uint32_t l = thread_l(t) | op.lcmask;
          rows |= 1u << ((l ^ ((l >> 4) & 15u)) & 15u);
        }
        good += rows == 0xffffu;
      }
      checked++;
    }
  }
  if (spread) *spread = good;
  return checked;
}

// The host-computed set-up of parameter-block ops (OpPre), against slots
// computed directly: for every dense 1-3 qubit op of the complex64 program,
// thread t, trip it < 4, group h of the trip and member y, the device's
// slot swb(l(t) | lcmask) ^ tc[it] ^ dh[h] ^ soff[y] must be the swizzled
// byte offset of that amplitude (group base l(t) ^ trip part, plus the
// member's target bits).  Returns the number of ops checked, or -1.
extern "C" int check_op_pre(const sv_circuit *c, int m, int L) {
  std::vector<Gate> gates;
  if (circuit_to_gates(c, nullptr, c->n_qubits, gates, false) != SV_OK) return -1;
  const int n = c->n_qubits;
  std::vector<Block> blocks = fuse(gates, 3);
  if (!fit_tile(blocks, n, 1, 14, m, L)) return -1;
  std::vector<PassPlan> passes = plan_passes(blocks, n, m, L, 256, 1 << 16);
  DeviceProgram prog;
  std::vector<uint32_t> op0s;
  BuildCtx bc{SV_C64, n, m, L, 1, 0};
  for (const PassPlan &P : passes)
    if (emit_pass(prog, P, bc, op0s, {}) != SV_OK) return -1;
  auto swb = [](uint32_t l) { return (l ^ ((l >> 4) & 15u)) * 8u; };
  int checked = 0;
  for (size_t pi = 0; pi < prog.passes.size(); pi++) {
    const TilePass &tp = prog.passes[pi];
    const int T = tile_threads(tp.m, SV_C64);
    for (int oi = 0; oi < tp.nops; oi++) {
      const TileOp &op = prog.ops[op0s[pi] + oi];
      if (op.kind != TOP_DENSE || op.k > 3) continue;
      OpPre pre;
      fill_op_pre(op, T, pre);
      uint32_t fixed = op.lcmask;
      for (int j = 0; j < op.k; j++) fixed |= 1u << op.t[j];
      const uint32_t ngroups = 1u << (tp.m - __builtin_popcount(fixed));
      const uint32_t ntrips = ngroups > (uint32_t)T ? ngroups / (uint32_t)T : 1u;
      const int G = pairs_groups(op.k);
      const uint32_t nthr = ngroups < (uint32_t)T ? ngroups : (uint32_t)T;
      for (uint32_t t = 0; t < nthr; t++) {
        uint32_t lt = 0;
        for (int i = 0; i < 9; i++) lt |= ((t >> i) & 1u) << ((op.tbpos[i >> 1] >> (4 * (i & 1))) & 15u);
        for (uint32_t it = 0; it < 4 && it * (uint32_t)G < ntrips; it++)
          for (int h = 0; h < G && it * G + h < ntrips; h++) {
            const uint32_t cc = it * G + h;
            const uint32_t lg = lt ^ ins0_mask_h(cc * (uint32_t)T, fixed);   // the group's base index
            for (int y = 0; y < (1 << op.k); y++) {
              uint32_t off = 0;
              for (int j = 0; j < op.k; j++) off |= (uint32_t)((y >> j) & 1) << op.t[j];
              const uint32_t want = swb(lg | op.lcmask | off);
              const uint32_t got = swb(lt | op.lcmask) ^ pre.tc[it] ^ pre.dh[h] ^ pre.soff[y];
              if (got != want) {
                std::printf("pass %zu op %d t %u trip %u h %d y %d: %x != %x\n", pi, oi, t, it, h, y, got, want);
                return -1;
              }
            }
          }
      }
      checked++;
    }
  }
  return checked;
}

// The library's program cache, driven past its bound on a host-only state
// handle (planning touches no device): with the bound at `limit`, the first
// circuit's program is held while `nc` circuits are planned in turn (as one
// batched call does); the held program must stay intact after its entry is
// evicted, every lookup must return the program of its own circuit (same
// blocks as a fresh plan), a repeated lookup must hit the cache, and the
// cache must stay within its bound.  Returns 0, or the number of the failed
// check.
static bool same_program(const CachedProgram &a, const CachedProgram &b) {
  if (a.prog.ops.size() != b.prog.ops.size() || a.prog.mats != b.prog.mats) return false;
  if (std::memcmp(a.prog.ops.data(), b.prog.ops.data(), a.prog.ops.size() * sizeof(TileOp)) != 0) return false;
  return a.blocks.size() == b.blocks.size();
}
extern "C" int cache_selftest(const sv_circuit *const *cs, int nc, int limit) {
  sv_state st;
  st.n = cs[0]->n_qubits;
  st.dt = SV_C64;
  const int64_t old = sv_program_cache_limit(limit);
  int rc = 0;
  {
    ProgramRef held;
    Opts o;
    if (get_program(&st, cs[0], nullptr, nullptr, &held, &o) != SV_OK) rc = 1;
    const CachedProgram snapshot = rc ? CachedProgram() : *held;
    ProgramRef again;
    if (!rc && (get_program(&st, cs[0], nullptr, nullptr, &again, &o) != SV_OK || again != held)) rc = 2;
    for (int i = 1; i < nc && !rc; i++) {
      ProgramRef p;
      if (get_program(&st, cs[i], nullptr, nullptr, &p, &o) != SV_OK) { rc = 3; break; }
      // a fresh plan of the same circuit, outside the cache
      std::vector<Gate> gates;
      circuit_to_gates(cs[i], nullptr, st.n, gates, false);
      const std::vector<Block> blocks = fuse(gates, o.fusion_k);
      if (p->blocks.size() != blocks.size()) rc = 4;
      if (p->serial == held->serial) rc = 5;
    }
    if (!rc && !same_program(snapshot, *held)) rc = 6;   // evicted but still held, intact
    ProgramRef back;
    if (!rc && get_program(&st, cs[0], nullptr, nullptr, &back, &o) != SV_OK) rc = 7;
    if (!rc && nc > limit && back->serial == held->serial) rc = 8;   // it was evicted: rebuilt
    if (!rc && !same_program(*back, *held)) rc = 9;
  }
  sv_program_cache_limit(old);
  return rc;
}

// The split-BF16 tensor-core program the library builds for a circuit
// (through its own cache and planner on a host-only state handle), run on
// the CPU in complex128: every tensor-core block's packed operand (BF16 hi
// and lo parts of the real embedding, in the tensor cores' core-matrix
// layout) is unpacked back to its complex 32 x 32 matrix and applied on the
// block's 5 tile positions; CUDA-core blocks use their stored matrices.
// Also checks what the pipelined kernel relies on: 5 targets in increasing
// tile position, a row map that is a bijection onto the free tile bits,
// lane bits on distinct bank classes.  Returns the number of passes and sets
// *npure to the passes the pipelined kernel takes, or -1 (message printed).
static float bf16_at(const uint8_t *part, int n, int k) {
  // canonical K-major layout without swizzle, 2-byte elements, 64 rows:
  // core matrices of 8 rows x 16 bytes, 64 * 16 bytes apart along K and 128
  // bytes apart along the rows
  const uint32_t o = (uint32_t)(k / 8) * 64 * 16 + (uint32_t)(n / 8) * 128 + (uint32_t)(n % 8) * 16 +
                     (uint32_t)(k % 8) * 2;
  uint16_t h;
  std::memcpy(&h, part + o, 2);
  const uint32_t bits = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &bits, 4);
  return f;
}
static std::vector<std::complex<double>> unpack_embedding(const uint8_t *base, int k) {
  // B hi then lo parts (BF16, N x N, N = 2^(k+1)); U[r][q] = R[2r][2q] + i R[2r+1][2q]
  const int D = 1 << k, N = 2 * D;
  auto at = [&](const uint8_t *part, int nn, int kk) {
    const uint32_t o = (uint32_t)(kk / 8) * N * 16 + (uint32_t)(nn / 8) * 128 + (uint32_t)(nn % 8) * 16 +
                       (uint32_t)(kk % 8) * 2;
    uint16_t h;
    std::memcpy(&h, part + o, 2);
    const uint32_t bits = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &bits, 4);
    return (double)f;
  };
  const uint8_t *hi = base, *lo = base + (size_t)N * N * 2;
  std::vector<std::complex<double>> U((size_t)D * D);
  for (int r = 0; r < D; r++)
    for (int q = 0; q < D; q++)
      U[(size_t)r * D + q] = std::complex<double>(at(hi, 2 * r, 2 * q) + at(lo, 2 * r, 2 * q),
                                                  at(hi, 2 * r + 1, 2 * q) + at(lo, 2 * r + 1, 2 * q));
  return U;
}

// blocks of the pipelined passes emulated so far that move 16-byte pairs
static int g_pair_gathers = 0, g_pair_scatters = 0;
extern "C" void tc_pair_counts(int *gathers, int *scatters) {
  *gathers = g_pair_gathers;
  *scatters = g_pair_scatters;
  g_pair_gathers = g_pair_scatters = 0;
}

extern "C" int tc_program_emulate(const sv_circuit *c, double *psi_, int *npure, int fusion_k, int *nsix) {
  typedef std::complex<double> cx;
  sv_state st;
  st.n = c->n_qubits;
  st.dt = SV_C64;
  sv_options opt{fusion_k, 0, SV_PREC_TC_BF16X3, SV_MODE_TILED, 0};
  *nsix = 0;
  ProgramRef cp;
  Opts o;
  if (get_program(&st, c, nullptr, &opt, &cp, &o) != SV_OK) {
    std::printf("get_program: %s\n", sv_last_error());
    return -1;
  }
  const DeviceProgram &prog = cp->prog;
  const int n = c->n_qubits;
  cx *psi = reinterpret_cast<cx *>(psi_);
  *npure = 0;
  for (size_t pi = 0; pi < prog.passes.size(); pi++) {
    const TilePass &tp = prog.passes[pi];
    if (tp.flags & kPassTC) {   // one block of tp.L qubits over the whole state
      const int K = tp.L, D = 1 << K;
      if (K != 6) { std::printf("unexpected %d-qubit tensor-core pass\n", K); return -1; }
      (*nsix)++;
      const std::vector<cx> U = unpack_embedding(prog.mats.data() + 16 * (size_t)tp.mat0, K);
      uint64_t tmask = 0;
      std::vector<uint64_t> off(D);
      for (int y = 0; y < D; y++) {
        uint64_t o = 0;
        for (int j = 0; j < K; j++) o |= (uint64_t)((y >> j) & 1) << tp.hi_pos[j];
        off[y] = o;
      }
      tmask = off[D - 1];
      std::vector<cx> x(D);
      for (uint64_t base = 0; base < (1ull << n); base++) {
        if (base & tmask) continue;
        for (int y = 0; y < D; y++) x[y] = psi[base + off[y]];
        for (int r = 0; r < D; r++) {
          cx a = 0;
          for (int y = 0; y < D; y++) a += U[(size_t)r * D + y] * x[y];
          psi[base + off[r]] = a;
        }
      }
      continue;
    }
    const HostPass hp{prog.ops.data() + cp->op0s[pi], prog.mats.data()};
    if (tcp_pass_ok(tp, hp)) {
      (*npure)++;
      const std::string why = tcp_layout_selftest(tp, hp, &g_pair_gathers, &g_pair_scatters);
      if (!why.empty()) {
        std::printf("pass %zu layouts: %s\n", pi, why.c_str());
        return -1;
      }
    }
    const uint32_t TS = 1u << tp.m;
    // decode every op's matrix once
    std::vector<std::vector<cx>> Us(tp.nops);
    for (int oi = 0; oi < tp.nops; oi++) {
      const TileOp &op = prog.ops[cp->op0s[pi] + oi];
      const int D = 1 << op.k;
      std::vector<cx> &U = Us[oi];
      const uint8_t *base = prog.mats.data() + (size_t)op.mat * 8;
      if (op.kind == TOP_TC) {
        if (op.k != 5) { std::printf("tensor-core block with %d targets\n", op.k); return -1; }
        uint32_t tmask = 0;
        for (int j = 0; j < 5; j++) {
          // the first target may be any (the pass's layout chain picks it), the rest increase
          if (j > 1 && op.t[j] <= op.t[j - 1]) { std::printf("targets not increasing\n"); return -1; }
          if ((tmask >> op.t[j]) & 1u) { std::printf("repeated target\n"); return -1; }
          tmask |= 1u << op.t[j];
        }
        uint32_t rows = 0;
        for (int i = 0; i < 7; i++) rows |= 1u << ((op.tbpos[i >> 1] >> (4 * (i & 1))) & 15u);
        if ((rows | tmask) != (1u << tp.m) - 1 || (rows & tmask)) { std::printf("row map not a bijection\n"); return -1; }
        U.assign(32 * 32, 0.0);
        const uint8_t *hi = base, *lo = base + 64 * 64 * 2;
        for (int r = 0; r < 32; r++)
          for (int q = 0; q < 32; q++) {
            const double re = (double)bf16_at(hi, 2 * r, 2 * q) + (double)bf16_at(lo, 2 * r, 2 * q);
            const double im = (double)bf16_at(hi, 2 * r + 1, 2 * q) + (double)bf16_at(lo, 2 * r + 1, 2 * q);
            U[(size_t)r * 32 + q] = cx(re, im);
          }
      } else if (op.kind == TOP_PERM) {
        U.assign((size_t)D * D, 0.0);
        for (int q = 0; q < D; q++) U[(size_t)base[q] * D + q] = 1.0;
      } else if (op.kind == TOP_DIAG) {
        const float *f = reinterpret_cast<const float *>(base);
        U.resize(D);
        for (int r = 0; r < D; r++) U[r] = cx(f[2 * r], f[2 * r + 1]);
      } else if (op.kind == TOP_DENSE) {
        const float *f = reinterpret_cast<const float *>(base);
        U.assign((size_t)D * D, 0.0);
        if (op.k <= 3) {   // row pairs
          for (int p = 0; p < D / 2; p++)
            for (int y = 0; y < D; y++) {
              const float *q = f + 4 * ((size_t)p * D + y);
              U[(size_t)(2 * p) * D + y] = cx(q[0], q[2]);
              U[(size_t)(2 * p + 1) * D + y] = cx(q[1], q[3]);
            }
        } else {
          for (int e = 0; e < D * D; e++) U[e] = cx(f[2 * e], f[2 * e + 1]);
        }
      } else {
        std::printf("unexpected op kind %d\n", op.kind);
        return -1;
      }
    }
    for (uint64_t t = 0; t < (1ull << (n - tp.m)); t++) {
      uint64_t gbase = 0;
      for (int j = 0; j < n - tp.m; j++) gbase |= ((t >> j) & 1ull) << tp.out_pos[j];
      std::vector<uint64_t> gi(TS);
      for (uint32_t l = 0; l < TS; l++) {
        uint64_t g = l & ((1u << tp.L) - 1);
        for (int b = tp.L; b < tp.m; b++) g |= (uint64_t)((l >> b) & 1u) << tp.hi_pos[b - tp.L];
        gi[l] = gbase | g;
      }
      std::vector<cx> v(TS);
      for (uint32_t l = 0; l < TS; l++) v[l] = psi[gi[l]];
      if (tp.flags & kPassTable) apply_table_pass(prog, tp, gbase, v);
      for (int oi = 0; oi < tp.nops; oi++) {
        const TileOp &op = prog.ops[cp->op0s[pi] + oi];
        const uint64_t gcm = (uint64_t)op.gcmask_lo | ((uint64_t)op.gcmask_hi << 32);
        if ((gbase & gcm) != gcm) continue;
        const std::vector<cx> &U = Us[oi];
        const int K = op.k, D = 1 << K;
        if (op.kind == TOP_DIAG) {
          for (uint32_t g = 0; g < (TS >> __builtin_popcount(op.lcmask)); g++) {
            const uint32_t l = ins0_mask_h(g, op.lcmask) | op.lcmask;
            uint32_t r = 0;
            for (int j = 0; j < K; j++) r |= ((l >> op.t[j]) & 1u) << j;
            v[l] = U[r] * v[l];
          }
          continue;
        }
        std::vector<uint32_t> off(D);
        for (int y = 0; y < D; y++) {
          uint32_t ofs = 0;
          for (int j = 0; j < K; j++) ofs |= (uint32_t)((y >> j) & 1) << op.t[j];
          off[y] = ofs;
        }
        const uint32_t fixed = off[D - 1] | op.lcmask;
        for (uint32_t g = 0; g < (TS >> __builtin_popcount(fixed)); g++) {
          const uint32_t i0 = ins0_mask_h(g, fixed) | op.lcmask;
          std::vector<cx> x(D);
          for (int y = 0; y < D; y++) x[y] = v[i0 + off[y]];
          for (int r = 0; r < D; r++) {
            cx a = 0;
            for (int y = 0; y < D; y++) a += U[(size_t)r * D + y] * x[y];
            v[i0 + off[r]] = a;
          }
        }
      }
      for (uint32_t l = 0; l < TS; l++) psi[gi[l]] = v[l];
    }
  }
  return (int)prog.passes.size();
}

// The library's basis-state propagation (sv_apply_circuit's fast path) on
// the host: follows |index> through the circuit's gates.  Returns 1 and the
// final index and amplitude, or 0 when some gate does not keep a basis
// state a basis state.
extern "C" int basis_propagate(const sv_circuit *c, uint64_t index, uint64_t *out_index, double *amp_re_im) {
  std::vector<Gate> gates;
  if (circuit_to_gates(c, nullptr, c->n_qubits, gates, false) != SV_OK) return -1;
  cd amp = 1.0;
  if (!propagate_basis(gates, index, amp)) return 0;
  *out_index = index;
  amp_re_im[0] = amp.real();
  amp_re_im[1] = amp.imag();
  return 1;
}

// Build a circuit's program through the library's cache on a host-only
// state (no device work): returns the status, for argument checks.
extern "C" int build_status(const sv_circuit *c) {
  sv_state st;
  st.n = c->n_qubits;
  st.dt = SV_C64;
  ProgramRef cp;
  Opts o;
  return (int)get_program(&st, c, nullptr, nullptr, &cp, &o);
}
