// K9: pipelined tile passes of tensor-core blocks (complex64, 12-qubit
// tiles, split-BF16).
//
// Every block of such a pass is a dense 5-qubit block (smaller uncontrolled
// blocks are padded to 5 qubits with idle tile qubits on the host): on a
// 4096-amplitude tile it is one M = 128, N = 64, K = 64 real GEMM against the
// embedding of U, done as A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32
// accumulation in TMEM (paper Sec. II: a circuit moment is a matrix applied
// to the state vector).  The kernel is arranged so that HBM, the tensor
// cores and the CUDA cores work at the same time:
//   - one persistent CTA per SM runs four independent groups of four
//     warps; each group owns 128 TMEM columns (A_hi, A_lo, D), one
//     shared-memory tile buffer, and walks its own sequence of tiles;
//   - a group loads its tile, runs the pass's blocks on it and stores it;
//     while it waits for its loads or its MMAs the other three groups
//     gather, split and scatter (16 warps per SM: the register file allows
//     no more, and shared memory no more tile buffers next to the B
//     operands); when a group starts a tile it asks L2 for its next one, so
//     that load waits on L2 rather than HBM;
//   - the B operands of all blocks of the pass are copied into shared memory
//     once per CTA and stay there for all its tiles.
// The tile's shared-memory layout keeps each even/odd amplitude pair
// together (16-byte units) and XORs slot bits 1..3 with tile bits 4..6 and
// 8..10, so unit loads and stores are conflict-free.  Each block after the
// first sees the tile through its own layout, tile bit 0 swapped with its
// first target, so the members of a row move as 16-byte pairs; a block
// scatters into the next block's layout (in pairs when the two share that
// first target; the last one into the store's layout), and the host picks
// the first targets and which tile bits the lane bits address
// (TileOp.tbpos) so that gathers and scatters spread over the banks.
//
// Every wait is bounded: a wait that runs out raises the error flag, the
// group stops, and before the CTA exits it waits (bounded) for its MMAs and
// copies and frees its TMEM.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "tile_ops.cuh"

namespace sv {

constexpr int kPGroups = 4;                          // tile groups per CTA
constexpr uint32_t kPGroupThreads = 128;             // group thread t <-> TMEM lane t
constexpr int kPThreads = kPGroups * (int)kPGroupThreads;
constexpr uint32_t kPTileBytes = (1u << kTcTileM) * 8;   // 32 KB
constexpr uint32_t kPBBytes = 2 * 64 * 64 * 2;       // B_hi + B_lo, BF16: 16 KB per block
constexpr uint32_t kPUnits = (1u << kTcTileM) / 2 / kPGroupThreads;   // 16-byte units per thread
constexpr uint32_t kPTmemCols = 512;                 // 128 per group, allocated as a power of two
constexpr uint32_t kPSpin = 1u << 22;

// shared memory: [tile buffers][B: ntc blocks][mbarriers][TMEM address, flags]
__host__ __device__ constexpr uint32_t tcp_bars_off(int ntc) {
  return kPGroups * kPTileBytes + (uint32_t)ntc * kPBBytes;
}
__host__ __device__ constexpr uint32_t tcp_smem_bytes(int ntc) {
  return tcp_bars_off(ntc) + 8 * (1 + kPGroups) + 4 * (1 + kPGroups) + 4;
}
static_assert(tcp_smem_bytes(kTcpMaxBlocks) + 8 * kPUnits <= 227u * 1024u, "shared memory of a CTA");
static_assert(kPGroups * 128u <= kPTmemCols, "TMEM columns of a CTA");

// Byte offset of tile amplitude l: pairs (2j, 2j+1) stay together, slot bits
// 1..3 are XORed with tile bits 4..6 and 8..10 (linear over GF(2)).
__host__ __device__ constexpr uint32_t tcp_swz(uint32_t l) {
  return (l ^ ((((l >> 4) ^ (l >> 8)) & 7u) << 1)) * 8u;
}

// Per-block set-up, computed on the host and passed in the launch's
// parameter block (warp-uniform reads): each block's member offsets
// tcp_swz(layout(target bits of y)) and the offset contributed by each row
// bit, under the block's own layout (gather) and the next one's (scatter).
struct TcpTable {
  uint32_t soff[kTcpMaxBlocks][32];   // gather: the block's own layout
  uint32_t rbit[kTcpMaxBlocks][8];
  uint32_t doff[kTcpMaxBlocks][32];   // scatter: the next block's layout (the store's after the last)
  uint32_t dbit[kTcpMaxBlocks][8];
  uint32_t flags[kTcpMaxBlocks];      // bit 0: gather member pairs, bit 1: scatter member pairs
};

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(g + 1), "r"(kPGroupThreads) : "memory");
}
// group barrier that also ORs a predicate over the group's threads
__device__ __forceinline__ bool group_sync_or(int g, bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, %2, %3, pi;\n"
      " selp.u32 %0, 1, 0, po;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(g + 1), "r"(kPGroupThreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}
__device__ __forceinline__ void sts128(uint32_t a, int4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ int4 lds128(uint32_t a) {
  int4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];\n" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ void tmem_st16x(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
// D (TMEM) += A (TMEM) x B (shared memory), BF16 inputs, FP32 accumulation
__device__ __forceinline__ void mma_bf16_ta(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(idesc), "r"(acc));
}

// Global offsets of a thread's units: unit i of group thread t is tile
// amplitude l = 2 (t + 128 i); its offset is the tile's base | the thread's
// part | the trip's part, the trip parts shared by all threads (a table in
// shared memory).
struct TcpAddr {
  uint64_t thr;                 // thread part of the offset
  const uint64_t *trip;         // kPUnits trip parts
};

struct TcpGroup {
  int g;              // group index in the CTA
  uint32_t tid;       // thread index in the group (= TMEM lane)
  uint32_t tmem;      // TMEM address of the group's first column (lane 0)
  uint32_t bar_b;     // mbarrier: every B operand has landed
  uint32_t bar_mma;   // mbarrier of this group's MMAs
  volatile uint32_t *flag;   // shared: the elected thread could not issue (B never landed)
  bool b_ready;       // (elected thread) bar_b has been observed
  uint32_t done;      // this group's blocks so far (mbarrier parity)
  bool pend_mma;      // (elected thread) MMAs committed but not observed
};

// Split 16 amplitudes into BF16 hi/lo pairs and store them in this thread's
// TMEM lane at taddr (hi) and taddr + 32 columns (lo).
__device__ __forceinline__ void tcp_split_store(const float2 (&x)[16], uint32_t taddr) {
  uint32_t hi[16], lo[16];
  const uint64_t neg1 = pk2(-1.0f, -1.0f);
#pragma unroll
  for (int y = 0; y < 16; y++) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(x[y].x, x[y].y);
    hi[y] = *reinterpret_cast<const uint32_t *>(&hb);
    // the hi parts back in FP32 (a BF16 is the top half of an FP32), then
    // x - hi in one packed FMA
    const uint64_t hf = pk2(__uint_as_float(hi[y] << 16), __uint_as_float(hi[y] & 0xFFFF0000u));
    const float2 l = upk2(fma2(hf, neg1, pk2(x[y].x, x[y].y)));
    const __nv_bfloat162 lb = __floats2bfloat162_rn(l.x, l.y);
    lo[y] = *reinterpret_cast<const uint32_t *>(&lb);
  }
  tmem_st16x(taddr, hi);
  tmem_st16x(taddr + 32, lo);
}

// One tensor-core block (op i of table T) on the tile at shared address
// `ts`, its B operand at shared address `bs`: gathered from the tile in the
// block's layout, scattered back in the next one's.  Returns false in a
// thread whose wait ran out.
__device__ __forceinline__ bool tcp_block(const TcpTable &T, int i, uint32_t ts, uint32_t bs, TcpGroup &G) {
  const uint32_t *soff = T.soff[i], *rbit = T.rbit[i];
  uint32_t s0 = 0;   // this thread's row (group of 32 amplitudes)
#pragma unroll
  for (int b = 0; b < 7; b++) s0 ^= ((G.tid >> b) & 1u) ? rbit[b] : 0u;
  const uint32_t lane = (G.tid & ~31u) << 16;         // the warp's TMEM lane quadrant
  const uint32_t flags = T.flags[i];
  bool pairs = flags & 1u;                            // member pairs (y, y + 1) share a 16-byte unit
#pragma unroll
  for (int h = 0; h < 2; h++) {
    float2 x[16];
    if (pairs) {
#pragma unroll
      for (int y = 0; y < 16; y += 2) {
        const int4 v = lds128(ts + (s0 ^ soff[16 * h + y]));
        x[y] = make_float2(__int_as_float(v.x), __int_as_float(v.y));
        x[y + 1] = make_float2(__int_as_float(v.z), __int_as_float(v.w));
      }
    } else {
#pragma unroll
      for (int y = 0; y < 16; y++) x[y] = lds_c(ts + (s0 ^ soff[16 * h + y]), (const float2 *)nullptr);
    }
    tcp_split_store(x, G.tmem + lane + 16 * h);
  }
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  tc_fence_before();
  group_sync(G.g);
  if (G.tid == 0) {
    tc_fence_after();
    const bool ok = G.b_ready || mbar_wait(G.bar_b, 0, kPSpin);
    G.b_ready = ok;
    if (ok) {
      const uint32_t idesc = instr_desc(1u);   // BF16 A and B, FP32 D, M = 128, N = 64
      const uint32_t as[3] = {0, 0, 32}, bo[3] = {0, kPBBytes / 2, 0};
#pragma unroll
      for (int t = 0; t < 3; t++)
#pragma unroll
        for (uint32_t k = 0; k < 4; k++)
          mma_bf16_ta(G.tmem + 64, G.tmem + as[t] + 8 * k, smem_desc(bs + bo[t] + k * 2048, 1024, 128), idesc,
                      (t > 0 || k > 0) ? 1u : 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(G.bar_mma)
                   : "memory");
      G.pend_mma = true;
    } else {
      *G.flag = 1u;   // nothing committed: the group's waits below fail
    }
  }
  // every thread waits for the MMAs itself (no second barrier); a failed
  // wait reaches the whole group through the next barrier's OR
  const bool ok = !*G.flag && mbar_wait(G.bar_mma, G.done & 1, kPSpin);
  if (!ok) return false;
  if (G.tid == 0) G.pend_mma = false;
  G.done++;
  tc_fence_after();
  {
    const uint32_t *dbit = T.dbit[i];
    soff = T.doff[i];
    s0 = 0;
#pragma unroll
    for (int b = 0; b < 7; b++) s0 ^= ((G.tid >> b) & 1u) ? dbit[b] : 0u;
    pairs = flags & 2u;
  }
#pragma unroll
  for (int h = 0; h < 2; h++) {
    uint32_t r[32];
    tmem_ld32(G.tmem + lane + 64 + 32 * h, r);
    if (pairs) {
#pragma unroll
      for (int y = 0; y < 16; y += 2)
        sts128(ts + (s0 ^ soff[16 * h + y]),
               make_int4((int)r[2 * y], (int)r[2 * y + 1], (int)r[2 * y + 2], (int)r[2 * y + 3]));
    } else {
#pragma unroll
      for (int y = 0; y < 16; y++)
        sts_c(ts + (s0 ^ soff[16 * h + y]), make_float2(__uint_as_float(r[2 * y]), __uint_as_float(r[2 * y + 1])));
    }
  }
  tc_fence_before();   // the next block's A stores and MMAs come after a group barrier
  return true;
}

__global__ void __launch_bounds__(kPThreads, 1)
    k_tile_tcp(const __grid_constant__ TilePass P, const __grid_constant__ TcpTable T) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t s_trip[kPUnits];
  const int g = (int)(threadIdx.x / kPGroupThreads);
  const int ntc = P.nops;   // every op of the pass is a tensor-core block
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bbase = sbase + kPGroups * kPTileBytes;
  const uint32_t bars = sbase + tcp_bars_off(ntc);
  uint32_t *slots = reinterpret_cast<uint32_t *>(smem + tcp_bars_off(ntc) + 8 * (1 + kPGroups));
  TcpGroup G;
  G.g = g;
  G.tid = threadIdx.x % kPGroupThreads;
  G.bar_b = bars;
  G.bar_mma = bars + 8 * (1 + g);
  G.flag = slots + 1 + g;
  G.b_ready = false;
  G.done = 0;
  G.pend_mma = false;
  const uint32_t segmask = (1u << P.L) - 1;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 1 + kPGroups; i++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bars + 8 * i));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (threadIdx.x < kPGroups) slots[1 + threadIdx.x] = 0u;
  if (threadIdx.x < kPUnits) {
    const uint32_t lt = threadIdx.x * kPGroupThreads * 2;
    s_trip[threadIdx.x] = (lt & segmask) | spread_hi(P, lt & ~segmask);
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slots)),
                 "r"(kPTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  G.tmem = slots[0] + 128u * (uint32_t)g;
  const uint64_t ntiles = 1ull << (P.n - P.m);
  const uint64_t stride = (uint64_t)gridDim.x * kPGroups;
  uint64_t t = (uint64_t)blockIdx.x * kPGroups + g;
  // the B operands of every block of the pass, once per CTA
  if (threadIdx.x == 0 && ntc > 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bars), "r"(ntc * kPBBytes)
                 : "memory");
    for (int j = 0; j < ntc; j++) {
      const char *src = static_cast<const char *>(P.mats) + (size_t)P.ops[j].mat * sizeof(float2);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
              bbase + (uint32_t)j * kPBBytes),
          "l"(src), "r"(kPBBytes), "r"(bars)
          : "memory");
    }
  }
  const uint32_t ts = sbase + (uint32_t)g * kPTileBytes;
  const uint32_t lthr = G.tid * 2;
  const TcpAddr A{(lthr & segmask) | spread_hi(P, lthr & ~segmask), s_trip};
  bool failed = false;
  uint64_t cur = t < ntiles ? tile_base(P, t) : 0;
  for (; t < ntiles && !failed; t += stride) {
    // the tile into the buffer (its last tile was stored before the barrier
    // that ended the previous iteration); the other groups work meanwhile
    const int4 *g0 = reinterpret_cast<const int4 *>(P.v0);
    {
      int4 v[kPUnits];
#pragma unroll
      for (uint32_t i = 0; i < kPUnits; i++) v[i] = __ldcs(g0 + ((cur | A.thr | A.trip[i]) >> 1));
#pragma unroll
      for (uint32_t i = 0; i < kPUnits; i++) sts128(ts + tcp_swz((G.tid + i * kPGroupThreads) * 2), v[i]);
    }
    // the group's next tile towards L2 while this one's blocks run, so its
    // load waits on L2 rather than on HBM
    uint64_t nxt = 0;
    if (t + stride < ntiles) {
      nxt = tile_base(P, t + stride);
#pragma unroll
      for (uint32_t i = 0; i < kPUnits; i++) prefetch_l2(g0 + ((nxt | A.thr | A.trip[i]) >> 1));
    }
    bool ok = true;
    for (int oi = 0; oi < P.nops; oi++) {
      if (group_sync_or(g, !ok)) break;
      ok = tcp_block(T, oi, ts, bbase + (uint32_t)oi * kPBBytes, G);
    }
    if (group_sync_or(g, !ok)) {
      failed = true;
      break;
    }
    int4 *o0 = reinterpret_cast<int4 *>(P.v0);
#pragma unroll
    for (uint32_t i = 0; i < kPUnits; i++)
      __stcs(o0 + ((cur | A.thr | A.trip[i]) >> 1), lds128(ts + tcp_swz((G.tid + i * kPGroupThreads) * 2)));
    cur = nxt;
    group_sync(g);
  }
  // no copy or MMA may outlive the CTA
  if (failed && G.tid == 0) atomicExch(P.err, 1u);
  if (G.tid == 0) {
    if (G.pend_mma) mbar_wait(G.bar_mma, G.done & 1, kPSpin);
    if (g == 0 && ntc > 0) mbar_wait(G.bar_b, 0, kPSpin);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(slots[0]), "r"(kPTmemCols));
}

// Tile position p under the layout with pair bit pb: bits 0 and pb swapped.
static inline uint32_t tcp_layout_pos(uint32_t p, uint32_t pb) { return p == pb ? 0u : (p == 0 ? pb : p); }
static inline uint32_t tcp_layout(uint32_t l, uint32_t pb) {
  if (pb == 0) return l;
  const uint32_t b0 = l & 1u, bp = (l >> pb) & 1u;
  return (l & ~(1u | (1u << pb))) | bp | (b0 << pb);
}

// Thread-index bits of a block's rows (host).  A warp's shared-memory
// accesses are conflict-free when its lanes reach distinct banks: under
// tcp_swz the bank of slot s (8-byte granule) is given by slot bits 0..3
// after bits 1..3 take the XOR of bits 4..6 and 8..10, so slot bit p
// contributes the vector e0 (p = 0), e1 (p in {1,4,8}), e2 ({2,5,9}),
// e3 ({3,6,10}) or nothing (7, 11).  8-byte moves want lane bits 0..3 to
// contribute four independent vectors (16 lanes per wavefront), 16-byte
// pair moves lane bits 0..2 three independent ones among e1..e3.  The
// block gathers under the layout with pair bit pg and scatters under the
// one with pair bit ps; the lane bits are picked among its row bits so that
// both are conflict-free where possible (gather first), then the remaining
// row bits follow in increasing order.
static uint32_t tcp_bank_vec(uint32_t slot) {
  static const uint32_t kVec[12] = {1u, 2u, 4u, 8u, 2u, 4u, 8u, 0u, 2u, 4u, 8u, 0u};
  return slot < 12 ? kVec[slot] : 0u;
}
// true when the k vectors (restricted to mask) are linearly independent over GF(2)
static bool tcp_independent(const uint32_t *v, int k, uint32_t mask) {
  uint32_t basis[4] = {0, 0, 0, 0};   // basis[b]: a kept vector whose top bit is b
  for (int i = 0; i < k; i++) {
    uint32_t x = v[i] & mask;
    for (int b = 3; b >= 0; b--) {
      if (!((x >> b) & 1u)) continue;
      if (!basis[b]) {
        basis[b] = x;
        break;
      }
      x ^= basis[b];
    }
    if (x == 0) return false;
  }
  return true;
}
void tcp_row_positions(TileOp &op, int pair_gather, int pair_scatter) {
  const uint32_t pg = (uint32_t)pair_gather, ps = (uint32_t)pair_scatter;
  uint32_t targets = 0;
  for (int j = 0; j < op.k; j++) targets |= 1u << op.t[j];
  int rows[12], nr = 0;
  for (int p = 0; p < kTcTileM; p++)
    if (!((targets >> p) & 1u)) rows[nr++] = p;
  const bool gpair = tcp_layout_pos(op.t[0], pg) == 0, spair = tcp_layout_pos(op.t[0], ps) == 0;
  const int kg = gpair ? 3 : 4, ks = spair ? 3 : 4;
  const uint32_t mg = gpair ? 0xEu : 0xFu, ms = spair ? 0xEu : 0xFu;
  int best[4] = {0, 1, 2, 3}, best_score = -1;
  const int K = nr < 4 ? nr : 4;
  int sel[4];
  // ordered choices of K lane positions among the row bits
  for (sel[0] = 0; sel[0] < nr; sel[0]++)
    for (sel[1] = 0; sel[1] < nr; sel[1]++)
      for (sel[2] = 0; sel[2] < nr; sel[2]++)
        for (sel[3] = 0; sel[3] < nr; sel[3]++) {
          bool distinct = true;
          for (int x = 0; x < K; x++)
            for (int y = 0; y < x; y++) distinct &= sel[x] != sel[y];
          if (!distinct) continue;
          uint32_t vg[4], vs[4];
          for (int x = 0; x < K; x++) {
            vg[x] = tcp_bank_vec(tcp_layout_pos((uint32_t)rows[sel[x]], pg));
            vs[x] = tcp_bank_vec(tcp_layout_pos((uint32_t)rows[sel[x]], ps));
          }
          const int score = (tcp_independent(vg, std::min(kg, K), mg) ? 2 : 0) +
                            (tcp_independent(vs, std::min(ks, K), ms) ? 1 : 0);
          if (score > best_score) {
            best_score = score;
            for (int x = 0; x < K; x++) best[x] = sel[x];
          }
        }
  int P[12], np = 0;
  uint32_t used = 0;
  for (int x = 0; x < K; x++) {
    P[np++] = rows[best[x]];
    used |= 1u << rows[best[x]];
  }
  for (int i = 0; i < nr; i++)
    if (!((used >> rows[i]) & 1u)) P[np++] = rows[i];
  std::memset(op.tbpos, 0, sizeof(op.tbpos));
  for (int i = 0; i < np && i < 9; i++) op.tbpos[i >> 1] |= (uint8_t)(P[i] << (4 * (i & 1)));
}

// Host replay of a pipelined pass's shared-memory addressing (the tables
// launch_tile_tcp builds): tile amplitudes carry their own index as a
// label; the load, every block's gather and scatter, and the store follow
// the kernel's offsets.  Returns "" when every gathered member is the
// amplitude the block's row and member index name, every scatter fills
// all 4096 slots, pair moves are 16-byte aligned units, and the store
// finds each amplitude at its place; else what failed.  Adds the pass's
// blocks that gather / scatter in 16-byte pairs to the counters given.
static void tcp_build_table(const TilePass &p, const HostPass &host, TcpTable &tab);
std::string tcp_layout_selftest(const TilePass &p, const HostPass &host, int *pair_gathers, int *pair_scatters) {
  if (!tcp_pass_ok(p, host)) return "not a pure tensor-core pass";
  TcpTable T;
  tcp_build_table(p, host, T);
  for (int i = 0; i < p.nops; i++) {
    if (pair_gathers) *pair_gathers += (int)(T.flags[i] & 1u);
    if (pair_scatters) *pair_scatters += (int)((T.flags[i] >> 1) & 1u);
  }
  const uint32_t NT = 1u << kTcTileM;
  std::vector<int32_t> slot(NT, -1), next(NT);
  for (uint32_t l = 0; l < NT; l++) slot[tcp_swz(l) / 8] = (int32_t)l;
  for (int i = 0; i < p.nops; i++) {
    const TileOp &op = host.ops[i];
    std::fill(next.begin(), next.end(), -1);
    for (uint32_t tid = 0; tid < kPGroupThreads; tid++) {
      uint32_t s0 = 0, d0 = 0, row = 0;
      for (int b = 0; b < 7; b++)
        if ((tid >> b) & 1u) {
          s0 ^= T.rbit[i][b];
          d0 ^= T.dbit[i][b];
          row |= 1u << ((op.tbpos[b >> 1] >> (4 * (b & 1))) & 15u);
        }
      for (int y = 0; y < 32; y++) {
        uint32_t l = row;
        for (int j = 0; j < 5; j++) l |= (uint32_t)((y >> j) & 1) << op.t[j];
        const uint32_t ga = s0 ^ T.soff[i][y], sa = d0 ^ T.doff[i][y];
        if (ga >= NT * 8 || sa >= NT * 8) return "offset outside the tile";
        if ((T.flags[i] & 1u) && (y & 1) == 0 && (ga % 16 != 0 || T.soff[i][y + 1] != T.soff[i][y] + 8))
          return "gather pair not a 16-byte unit";
        if ((T.flags[i] & 2u) && (y & 1) == 0 && (sa % 16 != 0 || T.doff[i][y + 1] != T.doff[i][y] + 8))
          return "scatter pair not a 16-byte unit";
        if (slot[ga / 8] != (int32_t)l) return "block " + std::to_string(i) + " gathers the wrong amplitude";
        if (next[sa / 8] != -1) return "block " + std::to_string(i) + " scatters twice to one slot";
        next[sa / 8] = (int32_t)l;
      }
    }
    slot.swap(next);
  }
  for (uint32_t l = 0; l < NT; l++)
    if (slot[tcp_swz(l) / 8] != (int32_t)l) return "the store finds the wrong amplitude";
  return "";
}

bool tcp_pass_ok(const TilePass &p, const HostPass &host) {
  if (p.m != kTcTileM || p.nops < 1 || p.nops > kTcpMaxBlocks) return false;
  for (int i = 0; i < p.nops; i++)
    if (host.ops[i].kind != TOP_TC || host.ops[i].k != 5) return false;
  return true;
}

sv_status launch_tile_tcp(sv_state *s, const TilePass &p, const HostPass &host, cudaStream_t stream) {
  if (!tcp_pass_ok(p, host)) return set_error(SV_EINVAL, "internal: not a pure tensor-core tile pass");
  SV_TRY(func_attr_once((const void *)k_tile_tcp, s->device, cudaFuncAttributeMaxDynamicSharedMemorySize,
                        (int)tcp_smem_bytes(kTcpMaxBlocks)));
  const uint64_t ntiles = 1ull << (p.n - p.m);
  const uint64_t per_cta = (uint64_t)kPGroups;
  const int grid = (int)std::min<uint64_t>((ntiles + per_cta - 1) / per_cta, (uint64_t)s->sm_count);
  TcpTable tab;
  tcp_build_table(p, host, tab);
  k_tile_tcp<<<grid, kPThreads, tcp_smem_bytes(p.nops), stream>>>(p, tab);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

// The per-block tables of a pass: member and row-bit offsets under the
// block's layout (gather) and the next block's (scatter), and pair flags.
static void tcp_build_table(const TilePass &p, const HostPass &host, TcpTable &tab) {
  std::memset(&tab, 0, sizeof(tab));
  for (int i = 0; i < p.nops; i++) {
    const TileOp &op = host.ops[i];
    const uint32_t pg = (uint32_t)tcp_pair_bit(host.ops, p.nops, i);       // this block's layout
    const uint32_t ps = (uint32_t)tcp_pair_bit(host.ops, p.nops, i + 1);   // the next one's
    for (int y = 0; y < 32; y++) {
      uint32_t l = 0;
      for (int j = 0; j < 5; j++) l |= (uint32_t)((y >> j) & 1) << op.t[j];
      tab.soff[i][y] = tcp_swz(tcp_layout(l, pg));
      tab.doff[i][y] = tcp_swz(tcp_layout(l, ps));
    }
    for (int b = 0; b < 7; b++) {
      const uint32_t r = 1u << ((op.tbpos[b >> 1] >> (4 * (b & 1))) & 15u);
      tab.rbit[i][b] = tcp_swz(tcp_layout(r, pg));
      tab.dbit[i][b] = tcp_swz(tcp_layout(r, ps));
    }
    tab.flags[i] = (tcp_layout_pos(op.t[0], pg) == 0 ? 1u : 0u) | (tcp_layout_pos(op.t[0], ps) == 0 ? 2u : 0u);
  }
}

}  // namespace sv
