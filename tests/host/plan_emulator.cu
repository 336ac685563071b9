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
        } else if (op.kind == TOP_DENSE) {
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
