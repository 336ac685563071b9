// K6: tile-pass kernel.
//
// One CTA owns one tile: the 2^m amplitudes whose indices agree outside the
// pass's qubit set S (the L lowest qubits, contiguous in memory, plus m - L
// chosen high qubits).  The CTA reads the tile (one or two vectors) from HBM
// with 16-byte loads into shared memory, applies the pass's op list there,
// and writes the tile back, so a whole run of gates costs one read and one
// write of the state -- the HBM-bound core of the matrix-vector method (paper
// Sec. II, assumption (a)).  Ops: dense k-qubit blocks with local and
// out-of-tile controls, diagonal blocks, and the reductions used by the
// adjoint gradient (Im<lambda|G|psi>, Re<psi|lambda>) and by building
// lambda = H psi from Pauli strings.
//
// Shared-memory layout: amplitude l of the tile lives at sw(l), an XOR
// swizzle of its low bits by the next bits up.  A gate on low local qubits
// makes a warp's 32 groups stride through the tile; without the swizzle
// those strides land on a few banks (up to 8-way conflicts for three low
// targets), with it every access pattern of the op list spreads over all
// banks.
#include <cuda_bf16.h>

#include <algorithm>

#include "sv_device.cuh"
#include "sv_internal.h"

namespace sv {

constexpr int kTileMaxThreads = 512;

// swizzled shared-memory slot of tile amplitude l (a bijection on [0, 2^m))
template <typename R> __device__ __forceinline__ uint32_t sw(uint32_t l);
template <> __device__ __forceinline__ uint32_t sw<float>(uint32_t l) { return l ^ ((l >> 4) & 15u); }
template <> __device__ __forceinline__ uint32_t sw<double>(uint32_t l) { return l ^ ((l >> 3) & 7u); }

__device__ __forceinline__ uint64_t tile_base(const TilePass &P, uint64_t t) {
  uint64_t base = 0;
  const int nout = P.n - P.m;
  for (int j = 0; j < nout; j++) base |= ((t >> j) & 1ull) << P.out_pos[j];
  return base;
}

__device__ __forceinline__ uint64_t spread_hi(const TilePass &P, uint32_t l) {
  uint64_t g = 0;
  for (int b = P.L; b < P.m; b++) g |= (uint64_t)((l >> b) & 1u) << P.hi_pos[b - P.L];
  return g;
}

// Dense block on K local targets (U row-major complex in global memory,
// read through L1).  Matrices of 1-2 qubits are held in registers for the
// whole op; larger ones are read per use, each load serving G groups.
template <typename R, int K, int G>
__device__ __forceinline__ void dense_op(typename Cx<R>::T *__restrict__ v, int m, const TileOp &op,
                                         const typename Cx<R>::T *__restrict__ U) {
  using C = typename Cx<R>::T;
  constexpr int D = 1 << K;
  constexpr bool kRegU = K <= 2;
  uint32_t off[D];
#pragma unroll
  for (int y = 0; y < D; y++) {
    uint32_t o = 0;
#pragma unroll
    for (int j = 0; j < K; j++) o |= (uint32_t)((y >> j) & 1) << op.t[j];
    off[y] = o;
  }
  C ur[kRegU ? D * D : 1];
  if constexpr (kRegU) {
#pragma unroll
    for (int e = 0; e < D * D; e++) ur[e] = __ldg(&U[e]);
  }
  const uint32_t fixed = off[D - 1] | op.lcmask;
  const uint32_t ngroups = 1u << (m - __popc(fixed));
  const uint32_t step = blockDim.x * G;
  for (uint32_t g0 = threadIdx.x; g0 < ngroups; g0 += step) {
    uint32_t i0[G];
    bool ok[G];
    C x[G][D];
#pragma unroll
    for (int h = 0; h < G; h++) {
      const uint32_t g = g0 + h * blockDim.x;
      ok[h] = g < ngroups;
      i0[h] = ins0_mask(ok[h] ? g : 0, fixed) | op.lcmask;
#pragma unroll
      for (int y = 0; y < D; y++) x[h][y] = v[sw<R>(i0[h] + off[y])];
    }
#pragma unroll(kRegU ? D : 1)
    for (int r = 0; r < D; r++) {
      C a[G];
#pragma unroll
      for (int h = 0; h < G; h++) a[h] = czero<C>();
#pragma unroll
      for (int y = 0; y < D; y++) {
        const C u = kRegU ? ur[(r * D + y) % (kRegU ? D * D : 1)] : __ldg(&U[r * D + y]);
#pragma unroll
        for (int h = 0; h < G; h++) a[h] = cfma(u, x[h][y], a[h]);
      }
#pragma unroll
      for (int h = 0; h < G; h++)
        if (ok[h]) v[sw<R>(i0[h] + off[r])] = a[h];
    }
  }
}

// Dense blocks of 4..6 qubits keep 2^k amplitudes per thread; they live in
// separate functions so their register pressure does not spill the k <= 3
// paths that make up most passes.
template <typename R, int K>
__device__ __noinline__ void dense_op_big(typename Cx<R>::T *__restrict__ v, int m, const TileOp &op,
                                          const typename Cx<R>::T *__restrict__ U) {
  dense_op<R, K, 1>(v, m, op, U);
}

template <typename R>
__device__ __forceinline__ void diag_op(typename Cx<R>::T *__restrict__ v, int m, const TileOp &op,
                                        const typename Cx<R>::T *__restrict__ d) {
  const uint32_t ngroups = 1u << (m - __popc(op.lcmask));
  for (uint32_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
    const uint32_t l = ins0_mask(g, op.lcmask) | op.lcmask;
    uint32_t r = 0;
    for (int j = 0; j < op.k; j++) r |= ((l >> op.t[j]) & 1u) << j;
    const uint32_t p = sw<R>(l);
    v[p] = cmul(__ldg(&d[r]), v[p]);
  }
}

template <typename R>
__device__ __forceinline__ void apply_op(typename Cx<R>::T *v, int m, const TileOp &op,
                                         const typename Cx<R>::T *U) {
  if (op.kind == TOP_DIAG) {
    diag_op<R>(v, m, op, U);
    return;
  }
  switch (op.k) {
    case 1: dense_op<R, 1, 2>(v, m, op, U); break;
    case 2: dense_op<R, 2, 1>(v, m, op, U); break;
    case 3: dense_op<R, 3, sizeof(R) == 4 ? 2 : 1>(v, m, op, U); break;
    case 4: dense_op_big<R, 4>(v, m, op, U); break;
    case 5: dense_op_big<R, 5>(v, m, op, U); break;
    default: dense_op_big<R, 6>(v, m, op, U); break;
  }
}

// Im(conj(b) a)
template <typename C> __device__ __forceinline__ auto imdot(C b, C a) -> decltype(a.x) {
  return b.x * a.y - b.y * a.x;
}

template <typename R>
__device__ __forceinline__ void block_acc(R part, double *dst) {
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) atomicAdd(dst, (double)part);
}

template <typename R>
__device__ void grad_op(const typename Cx<R>::T *__restrict__ psi,
                        const typename Cx<R>::T *__restrict__ lam, int m, const TileOp &op,
                        double *acc) {
  using C = typename Cx<R>::T;
  const int t = op.t[0];
  const uint32_t bit = 1u << t;
  const uint32_t ngroups = 1u << (m - 1);
  R part = 0;
  for (uint32_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
    const uint32_t l0 = ins0(g, t), l1 = l0 | bit;
    const uint32_t p0 = sw<R>(l0), p1 = sw<R>(l1);
    const C a0 = psi[p0], a1 = psi[p1], b0 = lam[p0], b1 = lam[p1];
    switch (op.gen) {
      case 1:  // X
        part += imdot(b0, a1) + imdot(b1, a0);
        break;
      case 2: {  // Y: (Y psi)[l0] = -i a1, (Y psi)[l1] = i a0
        C ma1 = cmake(a1.y, -a1.x), pa0 = cmake(-a0.y, a0.x);
        part += imdot(b0, ma1) + imdot(b1, pa0);
        break;
      }
      case 3:  // Z
        part += imdot(b0, a0) - imdot(b1, a1);
        break;
      default:  // diag(0, -2)
        part += R(-2) * imdot(b1, a1);
        break;
    }
  }
  block_acc<R>(part, acc + op.slot);
}

// ---- TOP_TC: 5-qubit block on the tensor cores inside a 12-qubit tile -----
// The tile's 128 groups of 32 amplitudes form the A operand (hi/lo parts of
// every real column, canonical K-major layout), the packed real embedding of
// U is the B operand (staged from global memory per op), D (128 x 64 FP32)
// lives in TMEM.  See k_tc.cu for the operand formats.
struct TcShared {
  uint32_t a;        // shared address of A_hi (A_lo follows)
  uint32_t b;        // shared address of B_hi (B_lo follows)
  uint32_t bar;      // mbarrier
  uint32_t tmem;     // TMEM base address
  uint32_t mode;     // 1 = TF32 x3, 2 = BF16 x3
  uint32_t *ok;      // shared flag: the MMAs completed
};

__device__ __forceinline__ uint32_t tf32_part(float x) { return __float_as_uint(x) & 0xFFFFE000u; }

// returns false if the MMA wait ran out (error flag raised)
__device__ __noinline__ bool tc_op(float2 *__restrict__ v, const TileOp &op, const uint4 *__restrict__ bglob,
                                   const TcShared &T, uint32_t &phase, uint32_t *err, unsigned char *smem) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const uint32_t elem = T.mode == 1 ? 4 : 2;
  const uint32_t a_bytes = 128 * 64 * elem, b_bytes = 64 * 64 * elem;
  unsigned char *sm_a = smem + (T.a - smem_u32(smem));
  unsigned char *sm_b = smem + (T.b - smem_u32(smem));
  // B operand
  for (uint32_t i = tid; i < 2 * b_bytes / 16; i += nthr) reinterpret_cast<uint4 *>(sm_b)[i] = __ldg(bglob + i);
  uint32_t offs[32], tmask = 0;
#pragma unroll
  for (int y = 0; y < 32; y++) {
    uint32_t o = 0;
#pragma unroll
    for (int j = 0; j < 5; j++) o |= (uint32_t)((y >> j) & 1) << op.t[j];
    offs[y] = o;
  }
  tmask = offs[31];
  // A operand: item = (row, quarter of its 32 amplitudes)
  for (int item = tid; item < 512; item += nthr) {
    const uint32_t row = item >> 2, q = item & 3;
    const uint32_t i0 = ins0_mask(row, tmask);
    float2 x[8];
#pragma unroll
    for (int e = 0; e < 8; e++) x[e] = v[sw<float>(i0 + offs[8 * q + e])];
    if (T.mode == 1) {
#pragma unroll
      for (int c = 0; c < 4; c++) {          // 16-byte chunk (4q + c): amplitudes 8q + 2c, +1
        const float f[4] = {x[2 * c].x, x[2 * c].y, x[2 * c + 1].x, x[2 * c + 1].y};
        uint4 hi, lo;
        hi.x = tf32_part(f[0]); hi.y = tf32_part(f[1]); hi.z = tf32_part(f[2]); hi.w = tf32_part(f[3]);
        lo.x = __float_as_uint(f[0] - __uint_as_float(hi.x));
        lo.y = __float_as_uint(f[1] - __uint_as_float(hi.y));
        lo.z = __float_as_uint(f[2] - __uint_as_float(hi.z));
        lo.w = __float_as_uint(f[3] - __uint_as_float(hi.w));
        const uint32_t o = cm_offset(row, 4 * q + c, 128);
        *reinterpret_cast<uint4 *>(sm_a + o) = hi;
        *reinterpret_cast<uint4 *>(sm_a + a_bytes + o) = lo;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 2; c++) {          // 16-byte chunk (2q + c): amplitudes 8q + 4c .. +3
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
        const uint32_t o = cm_offset(row, 2 * q + c, 128);
        *reinterpret_cast<uint4 *>(sm_a + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(sm_a + a_bytes + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    const uint32_t idesc = instr_desc(T.mode == 1 ? 2u : 1u);
    const uint32_t ksteps = T.mode == 1 ? 8 : 4;
    const uint32_t a_lbo = 128 * 16, b_lbo = 64 * 16;
    const uint32_t as[3] = {T.a, T.a, T.a + a_bytes}, bs[3] = {T.b, T.b + b_bytes, T.b};
    for (int t = 0; t < 3; t++)
      for (uint32_t k = 0; k < ksteps; k++)
        mma_issue(T.tmem, smem_desc(as[t] + k * 2 * a_lbo, a_lbo, 128), smem_desc(bs[t] + k * 2 * b_lbo, b_lbo, 128),
                  idesc, (t > 0 || k > 0) ? 1u : 0u, T.mode);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(T.bar)
                 : "memory");
    const bool ok = mbar_wait(T.bar, phase, 1u << 22);
    if (!ok) {
      atomicExch(err, 1u);
      mbar_wait(T.bar, phase, 1u << 22);
    }
    *T.ok = ok ? 1u : 0u;
  }
  __syncthreads();
  phase ^= 1u;
  if (!*T.ok) return false;
  tc_fence_after();
  // epilogue: warp w reads lanes 32 (w % 4) .. +31 (rows) and a share of the
  // 64 columns; 16 columns = 8 amplitudes per read
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  const int lq = warp & 3, cgroups = nwarps >> 2;
  const uint32_t row = 32 * lq + lane;
  const uint32_t i0 = ins0_mask(row, tmask);
  for (int cg = warp >> 2; cg < 4; cg += cgroups) {
    uint32_t r[16];
    tmem_ld16(T.tmem + ((uint32_t)(32 * lq) << 16) + 16 * cg, r);
#pragma unroll
    for (int e = 0; e < 8; e++)
      v[sw<float>(i0 + offs[8 * cg + e])] = make_float2(__uint_as_float(r[2 * e]), __uint_as_float(r[2 * e + 1]));
  }
  tc_fence_before();
  return true;
}

// 16-byte unit u of the tile <-> shared memory (swizzled amplitude slots)
template <typename R> struct Unit;
template <> struct Unit<float> {
  static constexpr uint32_t APU = 2;
  __device__ static void put(float2 *v, uint32_t l, int4 raw) {
    const float4 f = *reinterpret_cast<const float4 *>(&raw);
    v[sw<float>(l)] = make_float2(f.x, f.y);
    v[sw<float>(l + 1)] = make_float2(f.z, f.w);
  }
  __device__ static int4 get(const float2 *v, uint32_t l) {
    const float2 a = v[sw<float>(l)], b = v[sw<float>(l + 1)];
    const float4 f = make_float4(a.x, a.y, b.x, b.y);
    return *reinterpret_cast<const int4 *>(&f);
  }
};
template <> struct Unit<double> {
  static constexpr uint32_t APU = 1;
  __device__ static void put(double2 *v, uint32_t l, int4 raw) {
    v[sw<double>(l)] = *reinterpret_cast<const double2 *>(&raw);
  }
  __device__ static int4 get(const double2 *v, uint32_t l) {
    const double2 a = v[sw<double>(l)];
    return *reinterpret_cast<const int4 *>(&a);
  }
};

// The work of one CTA on one tile.  COH selects L2-coherent loads and stores
// (bypassing L1), needed when other CTAs of the same launch wrote the tile
// earlier (the persistent batch kernel); otherwise streaming hints are used.
struct TcState {
  TcShared T;
  uint32_t phase;
  bool failed;
};

template <typename R, bool COH, bool TC = false>
__device__ __forceinline__ void tile_body(const TilePass &P, uint64_t tile, int b, unsigned char *smem_raw,
                                          TcState *tcs = nullptr) {
  using C = typename Cx<R>::T;
  const uint32_t TS = 1u << P.m;
  C *v0 = reinterpret_cast<C *>(smem_raw);
  C *v1 = v0 + TS;
  const uint64_t base = tile_base(P, tile);
  C *g0 = reinterpret_cast<C *>(P.tbl0 ? P.tbl0[b] : P.v0);
  C *g1 = P.nvec > 1 ? reinterpret_cast<C *>(P.tbl1 ? P.tbl1[b] : P.v1) : nullptr;

  using UN = Unit<R>;
  const uint32_t nunits = TS / UN::APU;
  const uint32_t segmask = (1u << P.L) - 1;
  const bool load1 = P.nvec > 1 && !(P.flags & 1u);
  // Global offset of unit u = threadIdx.x + i * blockDim.x: the thread's bits
  // and the trip's bits of the local index are disjoint, so their spreads
  // are computed separately (the thread part once per tile).
  const uint32_t lthr = threadIdx.x * UN::APU;
  const uint64_t gthr = base | (lthr & segmask) | spread_hi(P, lthr & ~segmask);
  const uint32_t tstep = blockDim.x * UN::APU;
  auto goff = [&](uint32_t i) -> uint64_t {
    const uint32_t lt = i * tstep;     // bits above the thread bits
    return gthr | (lt & segmask) | spread_hi(P, lt & ~segmask);
  };
  // loads: four 16-byte units in flight per thread before any shared store
  constexpr int BATCH = 4;
  for (uint32_t i0 = 0; i0 * blockDim.x + threadIdx.x < nunits; i0 += BATCH) {
    int4 r0[BATCH], r1[BATCH];
#pragma unroll
    for (int j = 0; j < BATCH; j++) {
      const uint32_t u = (i0 + j) * blockDim.x + threadIdx.x;
      if (u < nunits) {
        const uint64_t g = goff(i0 + j);
        const int4 *p0 = reinterpret_cast<const int4 *>(&g0[g]);
        r0[j] = COH ? __ldcg(p0) : __ldcs(p0);
        if (load1) {
          const int4 *p1 = reinterpret_cast<const int4 *>(&g1[g]);
          r1[j] = COH ? __ldcg(p1) : __ldcs(p1);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < BATCH; j++) {
      const uint32_t u = (i0 + j) * blockDim.x + threadIdx.x;
      if (u < nunits) {
        UN::put(v0, u * UN::APU, r0[j]);
        if (load1) UN::put(v1, u * UN::APU, r1[j]);
      }
    }
  }

  const C *mats = reinterpret_cast<const C *>(P.mats);
  const C *pmats = P.pmats ? reinterpret_cast<const C *>(P.pmats) + (size_t)b * P.pmats_stride : nullptr;
  double *acc = P.acc ? P.acc + (size_t)b * P.acc_stride : nullptr;

  for (int oi = 0; oi < P.nops; oi++) {
    __syncthreads();
    const TileOp op = P.ops[oi];
    const uint64_t gcm = (uint64_t)op.gcmask_lo | ((uint64_t)op.gcmask_hi << 32);
    switch (op.kind) {
      case TOP_DENSE:
      case TOP_DIAG: {
        if ((base & gcm) != gcm) break;
        const C *U = ((op.gen & kGenBatchMat) ? pmats : mats) + op.mat;
        if (op.vmask & 1) apply_op<R>(v0, P.m, op, U);
        if (op.vmask & 2) apply_op<R>(v1, P.m, op, U);
        break;
      }
      case TOP_GRAD:
        grad_op<R>(v0, v1, P.m, op, acc);
        break;
      case TOP_TC:
        if constexpr (TC && sizeof(R) == 4) {
          if (!tcs->failed && !tc_op(reinterpret_cast<float2 *>(v0), op,
                                     reinterpret_cast<const uint4 *>(mats + op.mat), tcs->T, tcs->phase, P.err,
                                     smem_raw))
            tcs->failed = true;
        }
        break;
      case TOP_PAULI: {
        const uint32_t xm = (uint16_t)op.slot;
        const uint32_t zl = op.lcmask;
        const int tsign = __popcll(base & gcm) & 1;
        const double c = P.coeffs[op.mat];
        // c * i^k
        R fr = 0, fi = 0;
        switch (op.gen & 3) {
          case 0: fr = (R)c; break;
          case 1: fi = (R)c; break;
          case 2: fr = (R)-c; break;
          default: fi = (R)-c; break;
        }
        for (uint32_t l = threadIdx.x; l < TS; l += blockDim.x) {
          const int s = (__popc(l & zl) + tsign) & 1;
          const R sr = s ? -fr : fr, si = s ? -fi : fi;
          const C a = v0[sw<R>(l)];
          C &dst = v1[sw<R>(l ^ xm)];
          dst.x += sr * a.x - si * a.y;
          dst.y += sr * a.y + si * a.x;
        }
        break;
      }
      case TOP_ZERO:
        for (uint32_t l = threadIdx.x; l < TS; l += blockDim.x) v1[l] = czero<C>();
        break;
      case TOP_DOT: {
        R part = 0;
        for (uint32_t l = threadIdx.x; l < TS; l += blockDim.x) {
          const C a = v0[l], c = v1[l];   // same slot in both vectors: the swizzle cancels
          part += a.x * c.x + a.y * c.y;
        }
        block_acc<R>(part, acc + op.slot);
        break;
      }
      default:
        break;
    }
  }
  __syncthreads();
  if constexpr (TC) {
    if (tcs->failed) return;   // the tile is incomplete: leave HBM as it was
  }
  const bool store0 = !(P.flags & 2u), store1 = P.nvec > 1 && !(P.flags & 4u);
  for (uint32_t i = 0; i * blockDim.x + threadIdx.x < nunits; i++) {
    const uint32_t l = (i * blockDim.x + threadIdx.x) * UN::APU;
    const uint64_t g = goff(i);
    if (store0) {
      if (COH) __stcg(reinterpret_cast<int4 *>(&g0[g]), UN::get(v0, l));
      else __stcs(reinterpret_cast<int4 *>(&g0[g]), UN::get(v0, l));
    }
    if (store1) {
      if (COH) __stcg(reinterpret_cast<int4 *>(&g1[g]), UN::get(v1, l));
      else __stcs(reinterpret_cast<int4 *>(&g1[g]), UN::get(v1, l));
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kTileMaxThreads, 2) k_tile(const __grid_constant__ TilePass P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tile_body<R, false>(P, blockIdx.x, blockIdx.y, smem_raw);
}

// Tile passes that contain tensor-core ops (one vector; dense, diagonal and
// TC ops).  Each CTA allocates its TMEM columns and mbarrier once and walks
// over tiles with two tile buffers: while it applies the ops of one tile,
// 8-byte cp.async copies bring the next tile into the other buffer (into the
// same swizzled slots), so HBM reads overlap the MMAs.
constexpr int kTcTileThreads = 256;

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}

__device__ __forceinline__ void tc_issue_loads(const TilePass &P, uint64_t tile, float2 *buf) {
  const uint32_t TS = 1u << P.m, nunits = TS / 2;
  const uint64_t base = tile_base(P, tile);
  const uint32_t segmask = (1u << P.L) - 1;
  const float2 *g0 = reinterpret_cast<const float2 *>(P.v0);
  const uint32_t lthr = threadIdx.x * 2;
  const uint64_t gthr = base | (lthr & segmask) | spread_hi(P, lthr & ~segmask);
  const uint32_t tstep = blockDim.x * 2;
  for (uint32_t i = 0; i * blockDim.x + threadIdx.x < nunits; i++) {
    const uint32_t lt = i * tstep;
    const uint64_t g = gthr | (lt & segmask) | spread_hi(P, lt & ~segmask);
    const uint32_t l = (i * blockDim.x + threadIdx.x) * 2;
    cp_async8(&buf[sw<float>(l)], &g0[g]);
    cp_async8(&buf[sw<float>(l + 1)], &g0[g + 1]);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void tc_store(const TilePass &P, uint64_t tile, const float2 *buf) {
  const uint32_t TS = 1u << P.m, nunits = TS / 2;
  const uint64_t base = tile_base(P, tile);
  const uint32_t segmask = (1u << P.L) - 1;
  float2 *g0 = reinterpret_cast<float2 *>(P.v0);
  const uint32_t lthr = threadIdx.x * 2;
  const uint64_t gthr = base | (lthr & segmask) | spread_hi(P, lthr & ~segmask);
  const uint32_t tstep = blockDim.x * 2;
  for (uint32_t i = 0; i * blockDim.x + threadIdx.x < nunits; i++) {
    const uint32_t lt = i * tstep;
    const uint64_t g = gthr | (lt & segmask) | spread_hi(P, lt & ~segmask);
    const uint32_t l = (i * blockDim.x + threadIdx.x) * 2;
    __stcs(reinterpret_cast<int4 *>(&g0[g]), Unit<float>::get(buf, l));
  }
}

__global__ void __launch_bounds__(kTcTileThreads, 2) k_tile_tc(const __grid_constant__ TilePass P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t TS = 1u << P.m;
  const uint32_t mode = (P.flags >> 9) & 3;
  const uint32_t elem = mode == SV_PREC_TC_TF32X3 ? 4 : 2;
  float2 *buf[2] = {reinterpret_cast<float2 *>(smem_raw), reinterpret_cast<float2 *>(smem_raw) + TS};
  TcState st;
  st.phase = 0;
  st.failed = false;
  st.T.mode = mode == SV_PREC_TC_TF32X3 ? 1u : 2u;
  st.T.a = smem_u32(smem_raw) + (uint32_t)(2 * TS * sizeof(float2));
  st.T.b = st.T.a + 2 * 128 * 64 * elem;
  st.T.bar = st.T.b + 2 * 64 * 64 * elem;
  uint32_t *slots = reinterpret_cast<uint32_t *>(smem_raw + (st.T.bar + 8 - smem_u32(smem_raw)));
  st.T.ok = slots + 1;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(st.T.bar));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slots)),
                 "r"(64u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  st.T.tmem = slots[0];
  const float2 *mats = reinterpret_cast<const float2 *>(P.mats);
  const uint64_t ntiles = 1ull << (P.n - P.m);
  uint64_t t = blockIdx.x;
  if (t < ntiles) tc_issue_loads(P, t, buf[0]);
  for (uint32_t it = 0; t < ntiles; t += gridDim.x, it++) {
    float2 *cur = buf[it & 1];
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const uint64_t tn = t + gridDim.x;
    if (tn < ntiles) tc_issue_loads(P, tn, buf[(it + 1) & 1]);   // overlaps with the ops below
    const uint64_t base = tile_base(P, t);
    for (int oi = 0; oi < P.nops; oi++) {
      __syncthreads();
      const TileOp op = P.ops[oi];
      if (op.kind == TOP_TC) {
        if (!st.failed && !tc_op(cur, op, reinterpret_cast<const uint4 *>(mats + op.mat), st.T, st.phase, P.err,
                                 smem_raw))
          st.failed = true;
      } else {
        const uint64_t gcm = (uint64_t)op.gcmask_lo | ((uint64_t)op.gcmask_hi << 32);
        if ((base & gcm) == gcm) apply_op<float>(cur, P.m, op, mats + op.mat);
      }
    }
    __syncthreads();
    if (st.failed) break;
    tc_store(P, t, cur);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");   // no copy may outlive the CTA
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(st.T.tmem), "r"(64u));
}

// ---------------------------------------------------------------------------
// Persistent batch kernel: one cooperative launch works through a queue of
// (pass, tile) items of many independent states, pass by pass in wave order.
// An item of pass p of a state waits (bounded) until every tile of pass p-1
// of that state is done; all CTAs are co-resident (cooperative launch) and
// items are handed out in queue order, so every awaited item is already held
// by a running CTA.  A wait that runs out sets *err and the CTA stops.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Poll *ctr until it reaches target; at most `limit` polls ~128 ns apart.
__device__ __forceinline__ bool bounded_wait(const uint32_t *ctr, uint32_t target, uint64_t limit) {
  for (uint64_t i = 0; i < limit; i++) {
    if (ld_acquire(ctr) >= target) return true;
    __nanosleep(128);
  }
  return ld_acquire(ctr) >= target;
}

// the tile body out of line, so the queue loop's registers do not crowd it
template <typename R>
__device__ __noinline__ void tile_body_coherent(const TilePass &P, uint64_t tile, unsigned char *smem_raw) {
  tile_body<R, true>(P, tile, 0, smem_raw);
}

template <typename R>
__global__ void __launch_bounds__(kTileMaxThreads, 2) k_tile_persist(const __grid_constant__ PersistArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ TilePass sP;
  __shared__ unsigned long long s_chunk;
  __shared__ int s_desc, s_stop;
  for (;;) {
    if (threadIdx.x == 0) {
      s_chunk = atomicAdd(A.next_item, 1ull);
      s_stop = 0;
      if (s_chunk < A.total_items) {
        // last descriptor whose first chunk is <= s_chunk
        uint32_t lo = 0, hi = A.ndesc - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (A.first_item[mid] <= s_chunk) lo = mid; else hi = mid - 1;
        }
        s_desc = (int)lo;
        const int dep = A.dep[lo];
        if (dep >= 0 && !bounded_wait(A.done + dep, A.ntiles[dep], A.spin_limit)) {
          atomicExch(A.err, 1u);
          s_stop = 1;
        }
        if (!s_stop) {
          __threadfence();
          sP = A.passes[lo];
        }
      } else {
        s_stop = 1;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int d = s_desc;
    const uint32_t nt = A.ntiles[d], ch = A.chunk[d];
    const uint64_t t0 = (s_chunk - A.first_item[d]) * ch;
    const uint64_t left = (uint64_t)nt - t0;
    const uint32_t cnt = left < ch ? (uint32_t)left : ch;
    for (uint32_t j = 0; j < cnt; j++) {
      tile_body_coherent<R>(sP, t0 + j, smem_raw);
      __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(A.done + d, cnt);
  }
}

// Self-test of the bounded wait: waits on a counter nothing increments and
// reports the timeout through *err (status read by the host).
__global__ void k_wait_selftest(const uint32_t *never, uint32_t *err, uint64_t limit) {
  if (threadIdx.x == 0 && !bounded_wait(never, 1u, limit)) atomicExch(err, 1u);
}

int tile_threads(int m, sv_dtype dt) {
  const int units = (1 << m) / (dt == SV_C64 ? 2 : 1);
  int t = units / 8;
  if (t < 32) t = 32;
  if (t > kTileMaxThreads) t = kTileMaxThreads;
  return t;
}

size_t tile_smem(sv_dtype dt, int m, int nvec) { return (size_t)nvec * ((size_t)1 << m) * amp_bytes(dt); }
size_t tc_smem_bytes(sv_prec mode) {
  const size_t elem = mode == SV_PREC_TC_TF32X3 ? 4 : 2;
  return 2 * 128 * 64 * elem + 2 * 64 * 64 * elem + 16;
}


sv_status launch_tile_pass(sv_state *s, const TilePass &p, int batch) {
  return launch_tile_pass_on(s, p, batch, s->stream);
}

sv_status launch_tile_pass_on(sv_state *s, const TilePass &p, int batch, cudaStream_t stream) {
  static bool attr_set[2][64] = {};
  if (p.flags & kPassHasTC) {
    if (s->dt != SV_C64 || p.m != kTcTileM || batch != 1)
      return set_error(SV_EINVAL, "internal: tensor-core ops need a single complex64 state and 12-qubit tiles");
    if (p.nvec != 1) return set_error(SV_EINVAL, "internal: tensor-core ops act on one vector");
    const size_t smem = 2 * tile_smem(s->dt, p.m, 1) + tc_smem_bytes((sv_prec)((p.flags >> 9) & 3));
    static bool attr = false;
    if (!attr) {
      SV_CUDA(cudaFuncSetAttribute(k_tile_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10));
      attr = true;
    }
    int per_sm = 0;
    SV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_tc, kTcTileThreads, smem));
    const uint64_t ntiles = 1ull << (p.n - p.m);
    const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)std::max(1, per_sm) * s->sm_count);
    k_tile_tc<<<grid, kTcTileThreads, smem, stream>>>(p);
    g_launches++;
    SV_CUDA(cudaGetLastError());
    return SV_OK;
  }
  const size_t smem = tile_smem(s->dt, p.m, (int)p.nvec);
  const int dev = s->device & 63;
  const int di = s->dt == SV_C64 ? 0 : 1;
  if (!attr_set[di][dev]) {
    if (s->dt == SV_C64)
      SV_CUDA(cudaFuncSetAttribute(k_tile<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10));
    else
      SV_CUDA(cudaFuncSetAttribute(k_tile<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10));
    attr_set[di][dev] = true;
  }
  if (smem > (200u << 10)) return set_error(SV_EINVAL, "tile too large for shared memory");
  dim3 grid((unsigned)(1ull << (p.n - p.m)), (unsigned)batch);
  const int threads = tile_threads(p.m, s->dt);
  if (s->dt == SV_C64)
    k_tile<float><<<grid, threads, smem, stream>>>(p);
  else
    k_tile<double><<<grid, threads, smem, stream>>>(p);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

sv_status launch_tile_persist(sv_state *s, const PersistArgs &A, int m_max, int *grid_out, cudaStream_t st) {
  const size_t smem = tile_smem(s->dt, m_max, 1);
  if (smem > (200u << 10)) return set_error(SV_EINVAL, "tile too large for shared memory");
  const void *fn = s->dt == SV_C64 ? (const void *)k_tile_persist<float> : (const void *)k_tile_persist<double>;
  SV_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10));
  int per_sm = 0;
  SV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTileMaxThreads, smem));
  if (per_sm < 1) return set_error(SV_EUNSUPPORTED, "persistent tile kernel does not fit on an SM");
  const int grid = per_sm * s->sm_count;
  PersistArgs a = A;
  void *args[] = {&a};
  SV_CUDA(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kTileMaxThreads), args, smem, st));
  g_launches++;
  if (grid_out) *grid_out = grid;
  return SV_OK;
}

sv_status launch_wait_selftest(cudaStream_t st, const uint32_t *never, uint32_t *err, uint64_t limit) {
  k_wait_selftest<<<1, 32, 0, st>>>(never, err, limit);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

}  // namespace sv
