// K8: tile passes with tensor-core blocks (complex64, 12-qubit tiles).
#include <algorithm>

#include "tile_ops.cuh"

namespace sv {

// ---------------------------------------------------------------------------
// Tile passes with tensor-core blocks (complex64, 12-qubit tiles).
//
// A fused dense 5-qubit block acting on a 4096-amplitude tile is the product
// of the tile's 128 groups of 32 amplitudes (rows, as 64 reals each) with the
// real 64 x 64 embedding [[Re U, Im U], [-Im U, Re U]]^T of U: one
// M = 128, N = 64, K = 64 GEMM, done in split precision as
// A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation.
//
// Data flow per op and tile: thread t of the CTA's four warps reads row t's
// 32 amplitudes from the shared-memory tile, splits them into hi/lo parts and
// writes them straight into its own TMEM lane (tcgen05.st), where the MMAs
// read A; B (the packed matrix) comes from shared memory, loaded by one bulk
// copy per op and prefetched one op ahead; D lands in TMEM and thread t
// reads its row back (tcgen05.ld) and scatters it into the tile.  Shared
// memory therefore carries only the gather, the scatter and B, and four CTAs
// (split-BF16; two with split-TF32 operands) share an SM, so one CTA's MMAs
// overlap the others' gathers, scatters and HBM traffic.  While a tile is
// stored, the next tile's units are copied asynchronously into the slots just
// read.  Dense blocks of 1-3 qubits and diagonal blocks of the same pass run
// on the CUDA cores in the same tile.
//
// Every wait is bounded; a wait that runs out raises the error flag, the CTA
// stops storing tiles, waits (bounded) for its own copies and MMAs, frees
// its TMEM and returns.
// ---------------------------------------------------------------------------
constexpr int kTcThreads = 128;   // thread t <-> TMEM lane (row) t
constexpr uint32_t kTcSpin = 1u << 22;
// BF16 operands: one B buffer, 48 KB of shared memory and 128 TMEM columns
// per CTA, four CTAs per SM; TF32: two B buffers, 96 KB and 256 columns,
// two CTAs per SM (TMEM admits no more)
__host__ __device__ constexpr uint32_t tc_bufs(sv_prec mode) {
  return mode == SV_PREC_TC_TF32X3 ? 2u : 1u;
}
constexpr int kTcMinBlocks = 4;

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31]), "r"(r[32])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// D (TMEM) = A (TMEM) x B (shared memory, descriptor)
__device__ __forceinline__ void mma_tmem_a(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc,
                                           bool tf32) {
  if (tf32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ uint32_t tf32_hi(float x) { return __float_as_uint(x) & 0xFFFFE000u; }

// next TOP_TC op after op index `oi` (wrapping to the pass's first one), -1 if none
__device__ __forceinline__ int next_tc_op(const TilePass &P, int oi) {
  for (int k = 1; k <= P.nops; k++) {
    const int j = (oi + k) % P.nops;
    if (P.ops[j].kind == TOP_TC) return j;
  }
  return -1;
}

// 16-byte units of a 12-qubit tile (one vector) <-> registers / the swizzled
// shared-memory tile (all of a thread's loads in flight at once).
constexpr int kTcUnits = (1 << kTcTileM) / 2 / kTcThreads;

__device__ __forceinline__ uint64_t tc_unit(const TilePass &P, uint64_t gthr, int j) {
  const uint32_t lt = (uint32_t)j * kTcThreads * 2;
  const uint32_t segmask = (1u << P.L) - 1;
  return gthr | (lt & segmask) | spread_hi(P, lt & ~segmask);
}
__device__ __forceinline__ uint64_t tc_thread_base(const TilePass &P, uint64_t tile) {
  const uint32_t segmask = (1u << P.L) - 1;
  const uint32_t lthr = threadIdx.x * 2;
  return tile_base(P, tile) | (lthr & segmask) | spread_hi(P, lthr & ~segmask);
}
__device__ __forceinline__ void tc_load_regs(const TilePass &P, uint64_t tile, int4 (&r)[kTcUnits]) {
  const float2 *g0 = reinterpret_cast<const float2 *>(P.v0);
  const uint64_t gthr = tc_thread_base(P, tile);
#pragma unroll
  for (int j = 0; j < kTcUnits; j++) r[j] = __ldcs(reinterpret_cast<const int4 *>(&g0[tc_unit(P, gthr, j)]));
}
__device__ __forceinline__ void tc_put_regs(float2 *v, const int4 (&r)[kTcUnits]) {
#pragma unroll
  for (int j = 0; j < kTcUnits; j++) Unit<float>::put(v, (j * kTcThreads + threadIdx.x) * 2, r[j]);
}
__device__ __forceinline__ void cp_async8(uint32_t smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem), "l"(gmem) : "memory");
}

// Store the tile; if `next` is a valid tile index, each thread then issues
// asynchronous copies of its own units of the next tile into the very slots
// it has just read (no other thread touches them), so the next tile's loads
// are in flight during the stores and the first op's wait is short.
__device__ __forceinline__ void tc_store_then_fetch(const TilePass &P, uint64_t tile, float2 *v, bool fetch,
                                                    uint64_t next) {
  float2 *g0 = reinterpret_cast<float2 *>(P.v0);
  const uint64_t gthr = tc_thread_base(P, tile);
  const uint64_t gnext = fetch ? tc_thread_base(P, next) : 0;
  const uint32_t vs = smem_u32(v);
#pragma unroll 2
  for (int j = 0; j < kTcUnits; j++) {
    const uint32_t l = (j * kTcThreads + threadIdx.x) * 2;
    __stcs(reinterpret_cast<int4 *>(&g0[tc_unit(P, gthr, j)]), Unit<float>::get(v, l));
    if (fetch) {
      const float2 *src = &g0[tc_unit(P, gnext, j)];
      cp_async8(vs + swb<float>(l), src);
      cp_async8(vs + swb<float>(l + 1), src + 1);
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

struct TcCta {
  uint32_t tmem;       // TMEM base (lane 0, first allocated column)
  uint32_t bufs;       // shared address of the B buffers
  uint32_t bar_b;      // two mbarriers: B buffer 0 / 1 loaded
  uint32_t bar_mma;    // mbarrier: the op's MMAs completed
  uint32_t *flag;      // shared: the last wait succeeded
  bool tf32;
  uint32_t nbufs;      // B buffers (1 or 2)
  uint32_t bbytes;     // B hi + lo
  uint32_t a_lo, d;    // TMEM column offsets of A_lo and D (A_hi at 0)
};

// One TOP_TC op on the tile; j = this CTA's count of TC ops so far.
// Returns false if a wait ran out.
// Thread 0 tracks what it has in flight: pend_b = the TC op index whose B
// load has not been waited for, pend_mma = the op whose MMAs have not (or
// kNone).
constexpr uint32_t kNone = 0xFFFFFFFFu;

__device__ __forceinline__ bool tc_tile_op(const TilePass &P, const TileOp &op, float2 *v, const TcCta &c,
                                           uint32_t j, int next_op, bool more, uint32_t &pend_b,
                                           uint32_t &pend_mma) {
  const uint32_t vs = smem_u32(v);
  const int tid = threadIdx.x, warp = tid >> 5;
  uint32_t soff[32], tmask = 0;
  soff[0] = 0;
#pragma unroll
  for (int q = 0; q < 5; q++) {
    const uint32_t bit = 1u << op.t[q];
    tmask |= bit;
    const uint32_t e = swb<float>(bit);
#pragma unroll
    for (int y = 0; y < (1 << q); y++) soff[y + (1 << q)] = soff[y] ^ e;
  }
  const uint32_t s0 = swb<float>(ins0_mask((uint32_t)tid, tmask));   // row tid
  const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
  // gather + split, straight into this thread's TMEM lane
#pragma unroll
  for (int h = 0; h < 2; h++) {
    if (c.tf32) {
#pragma unroll
      for (int hh = 0; hh < 2; hh++) {
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int y = 0; y < 8; y++) {
          const float2 a = lds_c(vs + (s0 ^ soff[16 * h + 8 * hh + y]), (const float2 *)nullptr);
          hi[2 * y] = tf32_hi(a.x);
          hi[2 * y + 1] = tf32_hi(a.y);
          lo[2 * y] = __float_as_uint(a.x - __uint_as_float(hi[2 * y]));
          lo[2 * y + 1] = __float_as_uint(a.y - __uint_as_float(hi[2 * y + 1]));
        }
        tmem_st16(c.tmem + lane_base + 32 * h + 16 * hh, hi);
        tmem_st16(c.tmem + lane_base + c.a_lo + 32 * h + 16 * hh, lo);
      }
    } else {
      uint32_t hi[16], lo[16];
#pragma unroll
      for (int y = 0; y < 16; y++) {
        const float2 a = lds_c(vs + (s0 ^ soff[16 * h + y]), (const float2 *)nullptr);
        const __nv_bfloat162 hb = __floats2bfloat162_rn(a.x, a.y);
        const float2 hf = __bfloat1622float2(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(a.x - hf.x, a.y - hf.y);
        hi[y] = *reinterpret_cast<const uint32_t *>(&hb);
        lo[y] = *reinterpret_cast<const uint32_t *>(&lb);
      }
      tmem_st16(c.tmem + lane_base + 16 * h, hi);
      tmem_st16(c.tmem + lane_base + c.a_lo + 16 * h, lo);
    }
  }
  tmem_wait_st();
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    tc_fence_after();
    // B buffer of op j and the parity of its load's completion
    const uint32_t nb = c.nbufs, buf = j % nb;
    bool ok = mbar_wait(c.bar_b + 8 * buf, (j / nb) & 1, kTcSpin);
    if (ok) {
      pend_b = kNone;
      const uint32_t idesc = instr_desc(c.tf32 ? 2u : 1u);
      const uint32_t ksteps = c.tf32 ? 8 : 4;
      const uint32_t half = c.bbytes / 2, b_lbo = 64 * 16;
      const uint32_t bh = c.bufs + buf * c.bbytes;
      const uint32_t as[3] = {0, 0, c.a_lo}, bs[3] = {bh, bh + half, bh};
      for (int t = 0; t < 3; t++)
        for (uint32_t k = 0; k < ksteps; k++)
          mma_tmem_a(c.tmem + c.d, c.tmem + as[t] + 8 * k, smem_desc(bs[t] + k * 2 * b_lbo, b_lbo, 128), idesc,
                     (t > 0 || k > 0) ? 1u : 0u, c.tf32);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       c.bar_mma)
                   : "memory");
      pend_mma = j;
      const float2 *mats = reinterpret_cast<const float2 *>(P.mats);
      const uint32_t nbuf = (j + 1) % nb;
      // two buffers: prefetch the next TC op's B now (the other buffer's last
      // reader, op j - 1, has completed); one buffer: once op j's MMAs are done
      if (nb == 2 && more && next_op >= 0) {
        bulk_load(c.bufs + nbuf * c.bbytes, mats + P.ops[next_op].mat, c.bbytes, c.bar_b + 8 * nbuf);
        pend_b = j + 1;
      }
      ok = mbar_wait(c.bar_mma, j & 1, kTcSpin);
      if (ok) {
        pend_mma = kNone;
        if (nb == 1 && more && next_op >= 0) {
          bulk_load(c.bufs, mats + P.ops[next_op].mat, c.bbytes, c.bar_b);
          pend_b = j + 1;
        }
      }
    }
    if (!ok) atomicExch(P.err, 1u);
    *c.flag = ok ? 1u : 0u;
  }
  __syncthreads();
  if (!*c.flag) return false;
  tc_fence_after();
#pragma unroll
  for (int h = 0; h < 2; h++) {
    uint32_t r[32];
    tmem_ld32(c.tmem + lane_base + c.d + 32 * h, r);
#pragma unroll
    for (int y = 0; y < 16; y++)
      sts_c(vs + (s0 ^ soff[16 * h + y]), make_float2(__uint_as_float(r[2 * y]), __uint_as_float(r[2 * y + 1])));
  }
  tc_fence_before();
  return true;
}

__global__ void __launch_bounds__(kTcThreads, kTcMinBlocks) k_tile_tc(const __grid_constant__ TilePass P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t TS = 1u << P.m;
  float2 *tile = reinterpret_cast<float2 *>(smem_raw);
  TcCta c;
  c.tf32 = ((P.flags >> 9) & 3) == SV_PREC_TC_TF32X3;
  c.bbytes = 2 * 64 * 64 * (c.tf32 ? 4 : 2);
  c.a_lo = c.tf32 ? 64 : 32;
  c.d = c.tf32 ? 128 : 64;
  const uint32_t ncols = c.tf32 ? 256 : 128;
  c.nbufs = tc_bufs((sv_prec)((P.flags >> 9) & 3));
  c.bufs = smem_u32(smem_raw) + TS * (uint32_t)sizeof(float2);
  c.bar_b = c.bufs + c.nbufs * c.bbytes;
  c.bar_mma = c.bar_b + 16;
  uint32_t *slots = reinterpret_cast<uint32_t *>(smem_raw + (c.bar_mma + 8 - smem_u32(smem_raw)));
  c.flag = slots + 1;
  const uint64_t ntiles = 1ull << (P.n - P.m);
  const int first_tc = next_tc_op(P, P.nops - 1);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(c.bar_b));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(c.bar_b + 8));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(c.bar_mma));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slots)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  c.tmem = slots[0];
  // B of the first TC op
  uint32_t pend_b = kNone, pend_mma = kNone;
  if (threadIdx.x == 0 && first_tc >= 0 && blockIdx.x < ntiles) {
    bulk_load(c.bufs, reinterpret_cast<const float2 *>(P.mats) + P.ops[first_tc].mat, c.bbytes, c.bar_b);
    pend_b = 0;
  }
  const float2 *mats = reinterpret_cast<const float2 *>(P.mats);
  uint32_t j = 0;   // TC ops done by this CTA
  bool failed = false;
  for (uint64_t t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
    if (t == blockIdx.x) {
      int4 r[kTcUnits];
      tc_load_regs(P, t, r);
      tc_put_regs(tile, r);
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // this tile's units, fetched during the last store
    }
    const uint64_t base = tile_base(P, t);
    const bool more_tiles = t + gridDim.x < ntiles;
    for (int oi = 0; oi < P.nops && !failed; oi++) {
      __syncthreads();
      const TileOp op = P.ops[oi];
      if (op.kind == TOP_TC) {
        const int nx = next_tc_op(P, oi);
        const bool more = nx > oi || more_tiles;   // a later TC op in this tile, or a next tile
        if (!tc_tile_op(P, op, tile, c, j, nx, more, pend_b, pend_mma)) failed = true;
        j++;
      } else {
        const uint64_t gcm = (uint64_t)op.gcmask_lo | ((uint64_t)op.gcmask_hi << 32);
        if ((base & gcm) != gcm) {
        } else if (op.kind == TOP_PERM) {
          perm_op<float>(tile, P.m, P.ops + oi, op.k, reinterpret_cast<const uint8_t *>(mats + op.mat), threadIdx.x,
                         blockDim.x);
        } else {
          apply_op<float, false, true>(tile, P.m, op, P.ops + oi, mats + op.mat, threadIdx.x, blockDim.x);
        }
      }
    }
    __syncthreads();
    if (failed) break;
    tc_store_then_fetch(P, t, tile, more_tiles, t + gridDim.x);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  // no copy or MMA may outlive the CTA
  if (threadIdx.x == 0) {
    if (pend_mma != kNone) mbar_wait(c.bar_mma, pend_mma & 1, kTcSpin);
    if (pend_b != kNone) mbar_wait(c.bar_b + 8 * (pend_b % c.nbufs), (pend_b / c.nbufs) & 1, kTcSpin);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(c.tmem), "r"(ncols));
}

size_t tc_tile_smem(sv_prec mode) {
  const size_t bbytes = 2 * 64 * 64 * (mode == SV_PREC_TC_TF32X3 ? 4 : 2);
  return ((size_t)1 << kTcTileM) * 8 + tc_bufs(mode) * bbytes + 64;
}

sv_status launch_tile_tc(sv_state *s, const TilePass &p, cudaStream_t stream) {
  const sv_prec mode = (sv_prec)((p.flags >> 9) & 3);
  const size_t smem = tc_tile_smem(mode);
  SV_TRY(func_attr_once((const void *)k_tile_tc, s->device, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10));
  SV_TRY(func_attr_once((const void *)k_tile_tc, s->device, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  // CTAs per SM as shared memory and TMEM admit them (see tc_bufs); the
  // grid strides over the tiles, so CTAs that do not fit at once start later
  const uint64_t per_sm = mode == SV_PREC_TC_TF32X3 ? 2 : (uint64_t)kTcMinBlocks;
  const uint64_t ntiles = 1ull << (p.n - p.m);
  const int grid = (int)std::min<uint64_t>(ntiles, per_sm * (uint64_t)s->sm_count);
  k_tile_tc<<<grid, kTcThreads, smem, stream>>>(p);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

}  // namespace sv
