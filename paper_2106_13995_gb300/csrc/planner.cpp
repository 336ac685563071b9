// Gate fusion and tile-pass planning (host, FP64).
//
// Fusion: consecutive gates acting on at most K qubits are multiplied into one
// 2^K x 2^K block.  A gate joins the latest block that touches any of its
// qubits, so it only ever moves past blocks on disjoint qubits (which commute
// with it).  Products are formed in FP64 and cast to the state's type later.
//
// Pass planning: each pass holds a set S of tile qubits (the L lowest qubits
// plus chosen high ones, |S| = m).  Blocks whose targets lie in S are applied
// to 2^m-amplitude tiles in shared memory, so the pass reads and writes the
// state once.  A block that cannot join blocks every qubit it touches for the
// rest of the scan, which keeps every reordering between commuting blocks.
#include <algorithm>

#include "sv_internal.h"

namespace sv {

static int index_of(const std::vector<int> &v, int q) {
  for (size_t i = 0; i < v.size(); i++)
    if (v[i] == q) return (int)i;
  return -1;
}

// Embed a (controlled) gate on `targets`/`controls` into a dense matrix over
// the qubit list `Q` (which contains all of them).
static std::vector<cd> embed(const std::vector<cd> &U, const std::vector<int> &targets,
                             const std::vector<int> &controls, const std::vector<int> &Q) {
  const int kq = (int)Q.size();
  const int D = 1 << kq;
  const int d = 1 << (int)targets.size();
  std::vector<int> tpos(targets.size()), cpos(controls.size());
  for (size_t j = 0; j < targets.size(); j++) tpos[j] = index_of(Q, targets[j]);
  for (size_t j = 0; j < controls.size(); j++) cpos[j] = index_of(Q, controls[j]);
  int tmask = 0, cmask = 0;
  for (int p : tpos) tmask |= 1 << p;
  for (int p : cpos) cmask |= 1 << p;
  std::vector<cd> E((size_t)D * D, 0.0);
  for (int col = 0; col < D; col++) {
    if ((col & cmask) != cmask) {
      E[(size_t)col * D + col] = 1.0;
      continue;
    }
    int ct = 0;
    for (size_t j = 0; j < tpos.size(); j++) ct |= ((col >> tpos[j]) & 1) << j;
    for (int rt = 0; rt < d; rt++) {
      int row = col & ~tmask;
      for (size_t j = 0; j < tpos.size(); j++) row |= ((rt >> j) & 1) << tpos[j];
      E[(size_t)row * D + col] = U[(size_t)rt * d + ct];
    }
  }
  return E;
}

static std::vector<cd> matmul(const std::vector<cd> &A, const std::vector<cd> &B, int D) {
  std::vector<cd> C((size_t)D * D, 0.0);
  for (int i = 0; i < D; i++)
    for (int k = 0; k < D; k++) {
      cd a = A[(size_t)i * D + k];
      if (a == cd(0.0)) continue;
      for (int j = 0; j < D; j++) C[(size_t)i * D + j] += a * B[(size_t)k * D + j];
    }
  return C;
}

static bool is_diagonal(const std::vector<cd> &U, int k) {
  const int d = 1 << k;
  for (int r = 0; r < d; r++)
    for (int c = 0; c < d; c++)
      if (r != c && U[(size_t)r * d + c] != cd(0.0)) return false;
  return true;
}

std::vector<Block> fuse(const std::vector<Gate> &gates, int K) {
  std::vector<Block> blocks;
  blocks.reserve(gates.size());
  std::vector<int> last(64, -1);
  for (const Gate &g : gates) {
    std::vector<int> Q = g.targets;
    Q.insert(Q.end(), g.controls.begin(), g.controls.end());
    const bool standalone = K <= 1 || g.fixed_structure || g.grad_gen > 0 ||
                            g.controls.size() >= 2 || (int)Q.size() > K;
    int bstar = -1;
    for (int q : Q) bstar = std::max(bstar, last[q]);
    if (!standalone && bstar >= 0 && blocks[bstar].fusable) {
      Block &b = blocks[bstar];
      std::vector<int> uni = b.qubits;
      for (int q : Q)
        if (index_of(uni, q) < 0) uni.push_back(q);
      if ((int)uni.size() <= K) {
        const int D = 1 << (int)uni.size();
        std::vector<cd> Ub = embed(b.U, b.qubits, {}, uni);
        std::vector<cd> Ug = embed(g.U, g.targets, g.controls, uni);
        b.U = matmul(Ug, Ub, D);
        b.qubits = uni;
        // the block's older qubits may already have later blocks: keep those
        for (int q : uni) last[q] = std::max(last[q], bstar);
        continue;
      }
    }
    Block nb;
    if (g.grad_gen > 0) {
      nb.kind = TOP_GRAD;
      nb.qubits = g.targets;
      nb.gen = g.grad_gen;
      nb.slot = g.grad_slot;
      nb.fusable = false;
      nb.vmask = 3;
    } else if (standalone) {
      nb.qubits = g.targets;
      nb.controls = g.controls;
      nb.U = g.U;
      // a block that keeps explicit controls cannot absorb more gates
      nb.fusable = !g.fixed_structure && g.controls.empty() && K > 1;
      nb.param = g.fixed_structure ? g.param : -1;
      nb.param_gate = g.fixed_structure ? g.param_gate : -1;
      nb.inst = g.fixed_structure ? g.inst : -1;
      if (K <= 1) nb.fusable = false;
    } else {
      nb.qubits = Q;
      nb.U = embed(g.U, g.targets, g.controls, Q);
    }
    blocks.push_back(std::move(nb));
    const int idx = (int)blocks.size() - 1;
    for (int q : Q) last[q] = idx;
  }
  for (Block &b : blocks)
    if (b.kind == TOP_DENSE) b.diag = b.inst < 0 && is_diagonal(b.U, (int)b.qubits.size());
  return blocks;
}

static uint64_t qmask(const std::vector<int> &v) {
  uint64_t m = 0;
  for (int q : v) m |= 1ull << q;
  return m;
}

static int mat_entries(const Block &b) {
  if (b.kind == TOP_TC) return 1024;   // a 5-qubit block (its packed operand is counted as 32 x 32)
  if (b.kind != TOP_DENSE && b.kind != TOP_DIAG) return 0;
  const int d = 1 << (int)b.qubits.size();
  return b.diag ? d : d * d;
}

int max_targets(const std::vector<Block> &blocks) {
  int k = 0;
  for (const Block &b : blocks) k = std::max(k, (int)b.qubits.size());
  return k;
}

bool fit_tile(const std::vector<Block> &blocks, int n, int lmin, int mmax, int &m, int &L) {
  const int kmax = max_targets(blocks);
  m = std::min(m, n);
  if (m >= n) {
    L = std::min(L, n);
    return true;
  }
  if (m - kmax < lmin) m = std::min(n, std::min(mmax, kmax + lmin));
  if (m >= n) {
    m = n;
    L = std::min(L, n);
    return true;
  }
  L = std::min(L, m - kmax);
  return L >= lmin;
}

std::vector<PassPlan> plan_passes(const std::vector<Block> &blocks, int n, int m, int L,
                                  int max_ops, int max_mat_entries) {
  std::vector<PassPlan> passes;
  m = std::min(m, n);
  L = std::min(L, m);
  // every block must fit next to the L fixed low qubits
  if (m < n && max_targets(blocks) > m - L) return passes;
  const uint64_t low = (L >= 64) ? ~0ull : ((1ull << L) - 1);
  const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
  std::vector<char> done(blocks.size(), 0);
  size_t remaining = blocks.size(), first = 0;
  while (remaining > 0) {
    while (first < blocks.size() && done[first]) first++;
    uint64_t S = low, blocked = 0;
    int nops = 0, nmat = 0;
    PassPlan P;
    for (size_t i = first; i < blocks.size(); i++) {
      if (done[i]) continue;
      const Block &b = blocks[i];
      const uint64_t need = qmask(b.qubits);
      const uint64_t touch = need | qmask(b.controls) | b.xmask;
      if (touch & blocked) {
        blocked |= touch;
      } else if (__builtin_popcountll(S | need) <= m && nops < max_ops &&
                 nmat + mat_entries(b) <= max_mat_entries) {
        S |= need;
        nops++;
        nmat += mat_entries(b);
        P.ops.push_back(b);
        done[i] = 1;
        remaining--;
      } else {
        blocked |= touch;
      }
      if ((blocked & all) == all) break;
    }
    if (P.ops.empty()) return {};     // nothing fits: the caller reports it
    // fill the tile up to m qubits with the lowest unused qubits
    for (int q = 0; q < n && __builtin_popcountll(S) < m; q++) S |= 1ull << q;
    for (int q = 0; q < n; q++)
      if ((S >> q) & 1) P.S.push_back(q);
    passes.push_back(std::move(P));
  }
  return passes;
}

// Merge small blocks inside each pass: a block joins an earlier block of the
// same pass when every block between them acts on other qubits (so it may
// move back next to it) and the two together touch at most K qubits.  The
// product is formed in FP64 as in fuse().  Blocks with controls, parameters
// or non-dense kinds neither merge nor move past blocks sharing a qubit.
static bool mergeable(const Block &b) {
  return b.kind == TOP_DENSE && b.controls.empty() && b.param < 0 && b.inst < 0 && b.fusable;
}
std::vector<Block> merge_in_passes(const std::vector<PassPlan> &passes, int K) {
  std::vector<Block> out;
  for (const PassPlan &P : passes) {
    std::vector<Block> ops = P.ops;
    std::vector<char> alive(ops.size(), 1);
    for (size_t j = 0; j < ops.size(); j++) {
      if (!mergeable(ops[j])) continue;
      const uint64_t tj = qmask(ops[j].qubits);
      for (size_t i = j; i-- > 0;) {
        if (!alive[i]) continue;
        const uint64_t ti = qmask(ops[i].qubits) | qmask(ops[i].controls) | ops[i].xmask;
        if (mergeable(ops[i]) && __builtin_popcountll(qmask(ops[i].qubits) | tj) <= K) {
          Block &A = ops[i];
          std::vector<int> uni = A.qubits;
          for (int q : ops[j].qubits)
            if (index_of(uni, q) < 0) uni.push_back(q);
          const int D = 1 << (int)uni.size();
          const std::vector<cd> Ua = embed(A.U, A.qubits, {}, uni);
          const std::vector<cd> Ub = embed(ops[j].U, ops[j].qubits, {}, uni);
          A.U = matmul(Ub, Ua, D);   // ops[j] acts after ops[i]
          A.qubits = uni;
          A.diag = is_diagonal(A.U, (int)uni.size());
          alive[j] = 0;
          break;
        }
        if (ti & tj) break;   // ops[j] cannot move past a block on its qubits
      }
    }
    for (size_t k = 0; k < ops.size(); k++)
      if (alive[k]) out.push_back(std::move(ops[k]));
  }
  return out;
}

}  // namespace sv
