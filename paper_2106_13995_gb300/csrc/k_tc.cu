// K7: fused 5-qubit dense block on the tensor cores (tcgen05, TMEM).
//
// A k-qubit block U acts on 2^{n-k} groups of 2^k amplitudes; with the
// amplitudes of group g interleaved as a real row x_g = (re_0, im_0, re_1, ...)
// the update is x_g <- x_g R^T with the real embedding
//   R[2r][2c] = Re U[r][c],  R[2r][2c+1] = -Im U[r][c],
//   R[2r+1][2c] = Im U[r][c], R[2r+1][2c+1] = Re U[r][c],
// a dense (2^{n-k} x 2^{k+1}) x (2^{k+1} x 2^{k+1}) real GEMM -- the only
// step of the method that is a real contraction, so it goes to the tensor
// cores.  For k = 5 each CTA takes 128 groups (M = 128, N = K = 64).
//
// Precision: FP32 inputs are split x = x_hi + x_lo (TF32 or BF16 parts) and
// the three products hi*hi + hi*lo + lo*hi are accumulated in FP32 in TMEM.
//
// Per tile: every thread gathers one group's 32 amplitudes from HBM, writes
// the hi/lo rows into shared memory in the canonical no-swizzle K-major
// layout (core matrices of 8 rows x 16 bytes), one thread issues the MMAs
// and commits them to an mbarrier, every warp reads its 32 TMEM lanes back
// and scatters the new amplitudes.  All waits are bounded; on timeout the
// CTA raises the error flag, waits (bounded) for its own MMAs, frees its TMEM
// and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "sv_device.cuh"
#include "sv_internal.h"

namespace sv {

constexpr int kTcK = 5;              // qubits per block
constexpr int kTcRows = 128;         // groups per tile (MMA M)
constexpr int kTcCols = 64;          // 2^{k+1} real columns (MMA N and K)
constexpr int kTcThreads = 128;
constexpr uint32_t kTmemCols = 64;

struct TcArgs {
  float2 *amps;
  uint64_t ngroups;          // 2^{n-5}
  uint64_t tmask;            // target bits
  uint64_t off[32];          // index offset of local basis state y
  const uint32_t *bmat;      // device: B_hi then B_lo, each 64 x 64 words in core-matrix layout
  uint32_t *err;             // error flag (set on a timed-out wait)
  uint32_t mode;             // 1 = TF32 x3, 2 = BF16 x3
  uint32_t spin_limit;       // mbarrier polls per wait
};

// shared-memory layout (bytes)
constexpr uint32_t kABytes = kTcRows * kTcCols * 4;   // one fp32 operand copy (32 KB)
constexpr uint32_t kBBytes = kTcCols * kTcCols * 4;   // 16 KB
constexpr uint32_t kSmA = 0;                          // A_hi, A_lo
constexpr uint32_t kSmB = 2 * kABytes;                // B_hi, B_lo
constexpr uint32_t kSmBar = kSmB + 2 * kBBytes;       // mbarrier (8 B) + TMEM address (4 B)
constexpr uint32_t kSmTotal = kSmBar + 16;

// TF32 part: FP32 bits with the low 13 mantissa bits cleared (exact split)
__device__ __forceinline__ uint32_t tf32_hi(float x) { return __float_as_uint(x) & 0xFFFFE000u; }

__global__ void __launch_bounds__(kTcThreads, 1) k_dense_tc(const __grid_constant__ TcArgs A) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const uint32_t sbase = smem_u32(sm);
  const uint32_t bar = sbase + kSmBar;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kSmBar + 8);
  const int tid = threadIdx.x, warp = tid >> 5;

  const uint32_t elem = A.mode == 1 ? 4 : 2;
  const uint32_t a_bytes = kTcRows * kTcCols * elem, b_bytes = kTcCols * kTcCols * elem;
  // B operand (hi and lo parts, 2 * b_bytes) into shared memory, once per CTA
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(A.bmat);
    uint4 *dst = reinterpret_cast<uint4 *>(sm + kSmB);
    for (uint32_t i = tid; i < 2 * b_bytes / 16; i += kTcThreads) dst[i] = src[i];
  }
  __shared__ uint32_t s_ok;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = instr_desc(A.mode == 1 ? 2u : 1u);
  const uint32_t a_lbo = kTcRows * 16, b_lbo = kTcCols * 16;   // bytes between K core matrices
  // bytes of K per MMA instruction: 8 TF32 or 16 BF16 = 32 bytes = 2 core matrices
  const uint32_t ksteps = A.mode == 1 ? kTcCols / 8 : kTcCols / 16;

  uint32_t phase = 0;
  const uint64_t ntiles = A.ngroups / kTcRows;
  // software pipeline: the next tile's amplitudes are loaded into registers
  // while the current tile's MMAs run and its results are written back
  uint64_t tile = blockIdx.x;
  float2 x[32];
  uint64_t base = 0;
  if (tile < ntiles) {
    base = ins0_mask64(tile * kTcRows + tid, A.tmask);
#pragma unroll
    for (int y = 0; y < 32; y++) x[y] = __ldcs(A.amps + base + A.off[y]);
  }
  for (; tile < ntiles; tile += gridDim.x) {
    if (A.mode == 1) {
#pragma unroll
      for (int c = 0; c < 16; c++) {   // 16-byte chunk c = columns 4c .. 4c+3 = amplitudes 2c, 2c+1
        const float f[4] = {x[2 * c].x, x[2 * c].y, x[2 * c + 1].x, x[2 * c + 1].y};
        uint4 hi, lo;
        hi.x = tf32_hi(f[0]); hi.y = tf32_hi(f[1]); hi.z = tf32_hi(f[2]); hi.w = tf32_hi(f[3]);
        lo.x = __float_as_uint(f[0] - __uint_as_float(hi.x));
        lo.y = __float_as_uint(f[1] - __uint_as_float(hi.y));
        lo.z = __float_as_uint(f[2] - __uint_as_float(hi.z));
        lo.w = __float_as_uint(f[3] - __uint_as_float(hi.w));
        const uint32_t o = cm_offset(tid, c, kTcRows);
        *reinterpret_cast<uint4 *>(sm + kSmA + o) = hi;
        *reinterpret_cast<uint4 *>(sm + kSmA + a_bytes + o) = lo;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 8; c++) {    // 16-byte chunk c = 8 BF16 columns = amplitudes 4c .. 4c+3
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const float2 a = x[4 * c + e];
          const __nv_bfloat16 hr = __float2bfloat16_rn(a.x), hi_ = __float2bfloat16_rn(a.y);
          const __nv_bfloat16 lr = __float2bfloat16_rn(a.x - __bfloat162float(hr));
          const __nv_bfloat16 li = __float2bfloat16_rn(a.y - __bfloat162float(hi_));
          hw[e] = (uint32_t)__bfloat16_as_ushort(hr) | ((uint32_t)__bfloat16_as_ushort(hi_) << 16);
          lw[e] = (uint32_t)__bfloat16_as_ushort(lr) | ((uint32_t)__bfloat16_as_ushort(li) << 16);
        }
        const uint32_t o = cm_offset(tid, c, kTcRows);
        *reinterpret_cast<uint4 *>(sm + kSmA + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(sm + kSmA + a_bytes + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0) {
      const uint32_t a_hi = sbase + kSmA, a_lo = a_hi + a_bytes;
      const uint32_t b_hi = sbase + kSmB, b_lo = b_hi + b_bytes;
      // D = A_hi B_hi + A_hi B_lo + A_lo B_hi
      const uint32_t as[3] = {a_hi, a_hi, a_lo}, bs[3] = {b_hi, b_lo, b_hi};
      for (int t = 0; t < 3; t++)
        for (uint32_t s = 0; s < ksteps; s++) {
          const uint64_t ad = smem_desc(as[t] + s * 2 * a_lbo, a_lbo, 128);
          const uint64_t bd = smem_desc(bs[t] + s * 2 * b_lbo, b_lbo, 128);
          mma_issue(tmem, ad, bd, idesc, (t > 0 || s > 0) ? 1u : 0u, A.mode);
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                   : "memory");
    }
    // prefetch the next tile while the MMAs run
    const uint64_t cur_base = base;
    const uint64_t next = tile + gridDim.x;
    float2 xn[32];
    if (next < ntiles) {
      base = ins0_mask64(next * kTcRows + tid, A.tmask);
#pragma unroll
      for (int y = 0; y < 32; y++) xn[y] = __ldcs(A.amps + base + A.off[y]);
    }
    // thread 0 waits (bounded) and tells the others, so all take one branch
    if (tid == 0) {
      s_ok = mbar_wait(bar, phase, A.spin_limit) ? 1u : 0u;
      if (!s_ok) {
        atomicExch(A.err, 1u);
        mbar_wait(bar, phase, A.spin_limit);   // give the MMAs a last bounded chance to drain
      }
    }
    __syncthreads();
    if (!s_ok) break;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    uint32_t r[64];
    tmem_ld64(tmem + ((uint32_t)(warp * 32) << 16), r);
#pragma unroll
    for (int y = 0; y < 32; y++)
      __stcs(A.amps + cur_base + A.off[y], make_float2(__uint_as_float(r[2 * y]), __uint_as_float(r[2 * y + 1])));
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();   // TMEM and shared rows are free for the next tile
#pragma unroll
    for (int y = 0; y < 32; y++) x[y] = xn[y];
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

// Host: real embedding R of U (64 x 64 for 5 qubits, 128 x 128 for 6), split
// into hi/lo parts and laid out as the K-major B operand (B[n][k] = R[n][k]).
static void build_b(const std::vector<cd> &U, uint32_t mode, std::vector<uint32_t> &out) {
  const int D = U.size() == 64 * 64 ? 64 : 32, N = 2 * D;   // 5- or 6-qubit block
  std::vector<float> R((size_t)N * N);
  for (int r = 0; r < D; r++)
    for (int c = 0; c < D; c++) {
      const float ur = (float)U[(size_t)r * D + c].real(), ui = (float)U[(size_t)r * D + c].imag();
      R[(size_t)(2 * r) * N + 2 * c] = ur;
      R[(size_t)(2 * r) * N + 2 * c + 1] = -ui;
      R[(size_t)(2 * r + 1) * N + 2 * c] = ui;
      R[(size_t)(2 * r + 1) * N + 2 * c + 1] = ur;
    }
  const size_t words = (size_t)N * N * (mode == 1 ? 1 : 2) / 2;   // per part, in 32-bit words
  out.assign(2 * (mode == 1 ? (size_t)N * N : (size_t)N * N / 2), 0u);
  unsigned char *hi = reinterpret_cast<unsigned char *>(out.data());
  unsigned char *lo = hi + (mode == 1 ? (size_t)N * N * 4 : (size_t)N * N * 2);
  (void)words;
  for (int n = 0; n < N; n++)
    for (int k = 0; k < N; k++) {
      const float v = R[(size_t)n * N + k];
      if (mode == 1) {
        uint32_t bits;
        std::memcpy(&bits, &v, 4);
        const uint32_t h = bits & 0xFFFFE000u;
        float hf;
        std::memcpy(&hf, &h, 4);
        const float l = v - hf;
        const uint32_t o = cm_offset(n, k / 4, N) + (k % 4) * 4;
        std::memcpy(hi + o, &h, 4);
        std::memcpy(lo + o, &l, 4);
      } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        const uint32_t o = cm_offset(n, k / 8, N) + (k % 8) * 2;
        std::memcpy(hi + o, &h, 2);
        std::memcpy(lo + o, &l, 2);
      }
    }
}

size_t tc_matrix_words(sv_prec mode, int k) {
  const size_t N = (size_t)2 << k;
  return mode == SV_PREC_TC_TF32X3 ? 2 * N * N : N * N;
}

void tc_pack_matrix(const std::vector<cd> &U, sv_prec mode, std::vector<uint32_t> &out) {
  build_b(U, mode == SV_PREC_TC_TF32X3 ? 1u : 2u, out);
}

sv_status launch_dense_tc(sv_state *s, void *amps, const int *targets, const uint32_t *bmat_dev, sv_prec mode,
                          uint64_t spin_limit, cudaStream_t stream) {
  if (s->dt != SV_C64) return set_error(SV_EUNSUPPORTED, "tensor-core blocks need a complex64 state");
  if (s->n < kTcK + 7) return set_error(SV_EUNSUPPORTED, "tensor-core blocks need at least 12 qubits");
  if (((uintptr_t)bmat_dev) & 15) return set_error(SV_EINVAL, "internal: tensor-core operand misaligned");
  TcArgs A;
  std::memset(&A, 0, sizeof(A));
  A.amps = reinterpret_cast<float2 *>(amps);
  A.ngroups = 1ull << (s->n - kTcK);
  for (int y = 0; y < 32; y++) {
    uint64_t o = 0;
    for (int j = 0; j < kTcK; j++) o |= (uint64_t)((y >> j) & 1) << targets[j];
    A.off[y] = o;
  }
  A.tmask = A.off[31];
  A.bmat = bmat_dev;
  A.err = reinterpret_cast<uint32_t *>(s->ws + kWsCtrl + kWsErrFlag);
  A.mode = mode == SV_PREC_TC_TF32X3 ? 1u : 2u;
  A.spin_limit = (uint32_t)std::min<uint64_t>(spin_limit ? spin_limit : (1u << 22), 0xFFFFFFFFu);
  SV_TRY(func_attr_once((const void *)k_dense_tc, s->device, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmTotal));
  const uint64_t ntiles = A.ngroups / kTcRows;
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)s->sm_count * 2);
  k_dense_tc<<<grid, kTcThreads, kSmTotal, stream>>>(A);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

// ---------------------------------------------------------------------------
// K10: a fused 6-qubit dense block on the tensor cores (split-BF16).
//
// The block's real embedding is 128 x 128; a CTA takes 128 groups of 64
// amplitudes (M = 128, N = K = 128), two threads per group: thread t gathers
// amplitudes 32h .. 32h + 31 (h = t / 128) of group t % 128 from HBM, splits
// them into BF16 hi/lo parts and writes them into the A operand in shared
// memory (canonical K-major layout); one thread issues the 3 x 8 MMAs, and
// while they run every thread loads its share of the next tile into
// registers; the warps then read their TMEM lanes back (warps w and w + 4
// share a lane quadrant, each reading its half of the columns) and scatter.
// Shared memory: A hi/lo 64 KB + B hi/lo 64 KB, one CTA per SM.
// ---------------------------------------------------------------------------
constexpr int kTc6Threads = 256;
constexpr uint32_t kTc6ABytes = 128 * 128 * 2;      // one BF16 part of A (32 KB)
constexpr uint32_t kTc6BBytes = 128 * 128 * 2;      // one BF16 part of B
constexpr uint32_t kTc6SmA = 0, kTc6SmB = 2 * kTc6ABytes, kTc6SmBar = kTc6SmB + 2 * kTc6BBytes;
constexpr uint32_t kTc6Smem = kTc6SmBar + 16;

struct Tc6Args {
  float2 *amps;
  uint64_t ngroups;          // 2^{n-6}
  uint64_t tmask;            // target bits
  uint64_t off[64];          // index offset of local basis state y
  const uint32_t *bmat;      // device: B_hi then B_lo, 128 x 128 BF16 each, core-matrix layout
  uint32_t *err;
  uint32_t spin_limit;
};

__global__ void __launch_bounds__(kTc6Threads, 1) k_dense_tc6(const __grid_constant__ Tc6Args A) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const uint32_t sbase = smem_u32(sm);
  const uint32_t bar = sbase + kTc6SmBar;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kTc6SmBar + 8);
  __shared__ uint32_t s_ok;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & 127, half = tid >> 7;
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(A.bmat);
    uint4 *dst = reinterpret_cast<uint4 *>(sm + kTc6SmB);
    for (uint32_t i = tid; i < 2 * kTc6BBytes / 16; i += kTc6Threads) dst[i] = src[i];
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = instr_desc(1u, 128, 128);   // BF16, M = 128, N = 128
  uint32_t phase = 0;
  const uint64_t ntiles = A.ngroups / 128;
  uint64_t tile = blockIdx.x;
  float2 x[32];
  uint64_t base = 0;
  if (tile < ntiles) {
    base = ins0_mask64(tile * 128 + row, A.tmask);
#pragma unroll
    for (int y = 0; y < 32; y++) x[y] = __ldcs(A.amps + base + A.off[32 * half + y]);
  }
  for (; tile < ntiles; tile += gridDim.x) {
    // this thread's 32 amplitudes = K columns 64 half .. 64 half + 63 of its
    // row = core-matrix chunks 8 half .. 8 half + 7 (8 BF16 = 4 amplitudes each)
#pragma unroll
    for (int c = 0; c < 8; c++) {
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const float2 a = x[4 * c + e];
        const __nv_bfloat162 hb = __floats2bfloat162_rn(a.x, a.y);
        const float2 hf = __bfloat1622float2(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(a.x - hf.x, a.y - hf.y);
        hw[e] = *reinterpret_cast<const uint32_t *>(&hb);
        lw[e] = *reinterpret_cast<const uint32_t *>(&lb);
      }
      const uint32_t o = cm_offset(row, 8 * half + c, 128);
      *reinterpret_cast<uint4 *>(sm + kTc6SmA + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4 *>(sm + kTc6SmA + kTc6ABytes + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0) {
      const uint32_t a_hi = sbase + kTc6SmA, a_lo = a_hi + kTc6ABytes;
      const uint32_t b_hi = sbase + kTc6SmB, b_lo = b_hi + kTc6BBytes;
      const uint32_t as[3] = {a_hi, a_hi, a_lo}, bs[3] = {b_hi, b_lo, b_hi};
      for (int t = 0; t < 3; t++)
        for (uint32_t k = 0; k < 8; k++)   // K = 16 per MMA: two core matrices of 128 x 16 bytes
          mma_issue(tmem, smem_desc(as[t] + k * 2 * 2048, 2048, 128), smem_desc(bs[t] + k * 2 * 2048, 2048, 128),
                    idesc, (t > 0 || k > 0) ? 1u : 0u, 2u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                   : "memory");
    }
    // the next tile's amplitudes while the MMAs run
    const uint64_t cur_base = base;
    const uint64_t next = tile + gridDim.x;
    float2 xn[32];
    if (next < ntiles) {
      base = ins0_mask64(next * 128 + row, A.tmask);
#pragma unroll
      for (int y = 0; y < 32; y++) xn[y] = __ldcs(A.amps + base + A.off[32 * half + y]);
    }
    if (tid == 0) {
      s_ok = mbar_wait(bar, phase, A.spin_limit) ? 1u : 0u;
      if (!s_ok) {
        atomicExch(A.err, 1u);
        mbar_wait(bar, phase, A.spin_limit);   // a last bounded chance for the MMAs to drain
      }
    }
    __syncthreads();
    if (!s_ok) break;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    uint32_t r[64];
    tmem_ld64(tmem + ((uint32_t)((warp & 3) * 32) << 16) + 64 * half, r);
#pragma unroll
    for (int y = 0; y < 32; y++)
      __stcs(A.amps + cur_base + A.off[32 * half + y],
             make_float2(__uint_as_float(r[2 * y]), __uint_as_float(r[2 * y + 1])));
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();   // TMEM and the A operand are free for the next tile
#pragma unroll
    for (int y = 0; y < 32; y++) x[y] = xn[y];
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(128));
}

sv_status launch_dense_tc6(sv_state *s, void *amps, const int *targets, const uint32_t *bmat_dev,
                           uint64_t spin_limit, cudaStream_t stream) {
  if (s->dt != SV_C64) return set_error(SV_EUNSUPPORTED, "tensor-core blocks need a complex64 state");
  if (s->n < 13) return set_error(SV_EUNSUPPORTED, "6-qubit tensor-core blocks need at least 13 qubits");
  if (((uintptr_t)bmat_dev) & 15) return set_error(SV_EINVAL, "internal: tensor-core operand misaligned");
  Tc6Args A;
  std::memset(&A, 0, sizeof(A));
  A.amps = reinterpret_cast<float2 *>(amps);
  A.ngroups = 1ull << (s->n - 6);
  for (int y = 0; y < 64; y++) {
    uint64_t o = 0;
    for (int j = 0; j < 6; j++) o |= (uint64_t)((y >> j) & 1) << targets[j];
    A.off[y] = o;
  }
  A.tmask = A.off[63];
  A.bmat = bmat_dev;
  A.err = reinterpret_cast<uint32_t *>(s->ws + kWsCtrl + kWsErrFlag);
  A.spin_limit = (uint32_t)std::min<uint64_t>(spin_limit ? spin_limit : (1u << 22), 0xFFFFFFFFu);
  SV_TRY(func_attr_once((const void *)k_dense_tc6, s->device, cudaFuncAttributeMaxDynamicSharedMemorySize,
                        (int)kTc6Smem));
  const uint64_t ntiles = A.ngroups / 128;
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)s->sm_count);
  k_dense_tc6<<<grid, kTc6Threads, kTc6Smem, stream>>>(A);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

}  // namespace sv
