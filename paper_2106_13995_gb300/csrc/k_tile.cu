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

constexpr int kTileMaxThreads = 512;    // persistent batch kernel
// tile passes: at most 256 threads (larger tiles give each thread more
// amplitudes), four CTAs per SM (64 registers a thread)
constexpr int kTilePassThreads = 256;
constexpr int kTilePassMinBlocks = 4;

// swizzled shared-memory slot of tile amplitude l (a bijection on [0, 2^m))
template <typename R> __device__ __forceinline__ uint32_t sw(uint32_t l);
template <> __device__ __forceinline__ uint32_t sw<float>(uint32_t l) { return l ^ ((l >> 4) & 15u); }
template <> __device__ __forceinline__ uint32_t sw<double>(uint32_t l) { return l ^ ((l >> 3) & 7u); }

// byte offset of tile amplitude l in the swizzled layout.  The swizzle is
// linear over GF(2), so swb(a ^ b) = swb(a) ^ swb(b): the offset of a group
// member is the group base's offset XOR a per-op constant.
template <typename R> __device__ __forceinline__ uint32_t swb(uint32_t l) {
  return sw<R>(l) * (uint32_t)sizeof(typename Cx<R>::T);
}

// shared-memory access by 32-bit address (the tile's slots)
__device__ __forceinline__ float2 lds_c(uint32_t a, const float2 *) {
  float2 r;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(r.x), "=f"(r.y) : "r"(a));
  return r;
}
__device__ __forceinline__ double2 lds_c(uint32_t a, const double2 *) {
  double2 r;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(r.x), "=d"(r.y) : "r"(a));
  return r;
}
__device__ __forceinline__ void sts_c(uint32_t a, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void sts_c(uint32_t a, double2 v) {
  asm volatile("st.shared.v2.f64 [%0], {%1, %2};\n" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}

// State index of tile t's amplitude 0 and of local bits above the L
// contiguous qubits; only set bits cost work.
__device__ __forceinline__ uint64_t tile_base(const TilePass &P, uint64_t t) {
  uint64_t base = 0;
  for (; t; t &= t - 1) base |= 1ull << P.out_pos[__ffsll((long long)t) - 1];
  return base;
}

__device__ __forceinline__ uint64_t spread_hi(const TilePass &P, uint32_t l) {
  uint64_t g = 0;
  for (uint32_t x = l >> P.L; x; x &= x - 1) g |= 1ull << P.hi_pos[__ffs(x) - 1];
  return g;
}

// two consecutive complex entries of a matrix row (16-byte aligned for c64)
__device__ __forceinline__ void ld_pair(const float2 *p, float2 &a, float2 &b) {
  const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
  a = make_float2(q.x, q.y);
  b = make_float2(q.z, q.w);
}
__device__ __forceinline__ void ld_pair(const double2 *p, double2 &a, double2 &b) {
  a = __ldg(p);
  b = __ldg(p + 1);
}

// Dense block on K local targets (U row-major complex in global memory,
// read through L1).  Group g's members sit at swb(base(g)) ^ soff[y]; with a
// power-of-two block size the thread's part of base(g) is computed once per
// op and each trip adds a warp-uniform part.  Matrices of 1-2 qubits stay in
// registers for the whole op; larger ones are read per row, each 16-byte load
// serving G groups.
template <typename R, int K, int G>
__device__ __forceinline__ void dense_op(typename Cx<R>::T *__restrict__ v, int m, const TileOp &op,
                                         const typename Cx<R>::T *__restrict__ U) {
  using C = typename Cx<R>::T;
  constexpr int D = 1 << K;
  constexpr bool kRegU = K <= 2;
  constexpr bool kUnrollRows = K <= 3;
  const uint32_t vs = smem_u32(v);
  uint32_t soff[D], e[K], tmask = 0;
  soff[0] = 0;
#pragma unroll
  for (int j = 0; j < K; j++) {
    const uint32_t bit = 1u << op.t[j];
    tmask |= bit;
    e[j] = swb<R>(bit);
#pragma unroll
    for (int y = 0; y < (1 << j); y++) soff[y + (1 << j)] = soff[y] ^ e[j];
  }
  C ur[kRegU ? D * D : 1];
  if constexpr (kRegU) {
#pragma unroll
    for (int q = 0; q < D * D; q += 2) ld_pair(U + q, ur[q], ur[q + 1]);
  }
  const uint32_t fixed = tmask | op.lcmask;
  const uint32_t ngroups = 1u << (m - __popc(fixed));
  const uint32_t T = blockDim.x;
  if (threadIdx.x >= ngroups) return;
  // thread t's groups are t + c T, c < ntrips; base(t + c T) = base(t) ^ D(c)
  // with D linear in c: D(c) = XOR of f[j] over the set bits j of c
  const uint32_t ntrips = ngroups > T ? ngroups / T : 1u;
  const uint32_t sthr = swb<R>(ins0_mask(threadIdx.x, fixed) | op.lcmask);
  for (uint32_t c0 = 0; c0 < ntrips; c0 += G) {
    uint32_t s[G];
    bool ok[G];
    C x[G][D];
#pragma unroll
    for (int h = 0; h < G; h++) {
      const uint32_t cc = c0 + h;
      ok[h] = cc < ntrips;
      s[h] = sthr ^ swb<R>(ins0_mask(ok[h] ? cc * T : 0u, fixed));
#pragma unroll
      for (int y = 0; y < D; y++) {
        x[h][y] = lds_c(vs + (s[h] ^ soff[y]), (const C *)nullptr);
      }
    }
#pragma unroll(kUnrollRows ? D : 1)
    for (int r = 0; r < D; r++) {
      C a[G];
#pragma unroll
      for (int h = 0; h < G; h++) a[h] = czero<C>();
#pragma unroll
      for (int y = 0; y < D; y += 2) {
        C u0, u1;
        if constexpr (kRegU) {
          u0 = ur[(r * D + y) % (kRegU ? D * D : 1)];
          u1 = ur[(r * D + y + 1) % (kRegU ? D * D : 1)];
        } else {
          ld_pair(U + r * D + y, u0, u1);
        }
#pragma unroll
        for (int h = 0; h < G; h++) {
          a[h] = cfma(u0, x[h][y], a[h]);
          a[h] = cfma(u1, x[h][y + 1], a[h]);
        }
      }
      uint32_t so;
      if constexpr (kUnrollRows) {
        so = soff[r % D];
      } else {
        so = 0;
#pragma unroll
        for (int j = 0; j < K; j++) so ^= ((r >> j) & 1) ? e[j] : 0u;
      }
#pragma unroll
      for (int h = 0; h < G; h++)
        if (ok[h]) {
          sts_c(vs + (s[h] ^ so), a[h]);
        }
    }
  }
}

// Dense blocks of 4..6 qubits keep 2^k amplitudes per thread; they live in
// separate functions so their register pressure does not spill the k <= 3
// paths that make up most passes.
// Dense blocks of 4..6 qubits keep 2^k amplitudes per thread; they run as
// functions of their own so their registers do not crowd the k <= 3 paths
// that make up most passes.  The op is read from global memory here, so no
// caller keeps an addressable (local-memory) copy of it.
template <typename R, int K>
__device__ __noinline__ void dense_op_big(typename Cx<R>::T *__restrict__ v, int m, const TileOp *gop,
                                          const typename Cx<R>::T *__restrict__ U) {
  const TileOp op = *gop;
  dense_op<R, K, 1>(v, m, op, U);
}

// Diagonal block: amplitude l is multiplied by d[r(l)], r(l) the target bits
// of l.  Both the slot and r are linear in l, so each splits into a thread
// part and a warp-uniform trip part.
template <typename R>
__device__ __forceinline__ void diag_op(typename Cx<R>::T *__restrict__ v, int m, const TileOp &op,
                                        const typename Cx<R>::T *__restrict__ d) {
  using C = typename Cx<R>::T;
  unsigned char *vb = reinterpret_cast<unsigned char *>(v);
  const uint32_t ngroups = 1u << (m - __popc(op.lcmask));
  const uint32_t T = blockDim.x;
  if (threadIdx.x >= ngroups) return;
  uint32_t tpos[6];
#pragma unroll
  for (int j = 0; j < 6; j++) tpos[j] = op.t[j];
  const int k = op.k;
  auto rows = [&](uint32_t l) {
    uint32_t r = 0;
#pragma unroll
    for (int j = 0; j < 6; j++)
      if (j < k) r |= ((l >> tpos[j]) & 1u) << j;
    return r;
  };
  const uint32_t lthr = ins0_mask(threadIdx.x, op.lcmask) | op.lcmask;
  const uint32_t sthr = swb<R>(lthr), rthr = rows(lthr);
  for (uint32_t g0 = 0; g0 < ngroups; g0 += T) {
    const uint32_t lg = ins0_mask(g0, op.lcmask);
    C *p = reinterpret_cast<C *>(vb + (sthr ^ swb<R>(lg)));
    *p = cmul(__ldg(&d[rthr ^ rows(lg)]), *p);
  }
}

template <typename R>
__device__ __forceinline__ void apply_op(typename Cx<R>::T *v, int m, const TileOp &op, const TileOp *gop,
                                         const typename Cx<R>::T *U) {
  if (op.kind == TOP_DIAG) {
    diag_op<R>(v, m, op, U);
    return;
  }
  switch (op.k) {
    case 1: dense_op<R, 1, 2>(v, m, op, U); break;
    case 2: dense_op<R, 2, 1>(v, m, op, U); break;
    case 3: dense_op<R, 3, sizeof(R) == 4 ? 2 : 1>(v, m, op, U); break;
    case 4: dense_op_big<R, 4>(v, m, gop, U); break;
    case 5: dense_op_big<R, 5>(v, m, gop, U); break;
    default: dense_op_big<R, 6>(v, m, gop, U); break;
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
template <typename R, bool COH>
__device__ __forceinline__ void tile_body(const TilePass &P, uint64_t tile, int b, unsigned char *smem_raw) {
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
        if (op.vmask & 1) apply_op<R>(v0, P.m, op, P.ops + oi, U);
        if (op.vmask & 2) apply_op<R>(v1, P.m, op, P.ops + oi, U);
        break;
      }
      case TOP_GRAD:
        grad_op<R>(v0, v1, P.m, op, acc);
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
__global__ void __launch_bounds__(kTilePassThreads, kTilePassMinBlocks) k_tile(const __grid_constant__ TilePass P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tile_body<R, false>(P, blockIdx.x, blockIdx.y, smem_raw);
}

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
// memory therefore carries only the gather, the scatter and B, and three
// CTAs share an SM, so one CTA's MMAs overlap the others' gathers, scatters
// and HBM traffic.  Dense blocks of 1-3 qubits and diagonal blocks of the
// same pass run on the CUDA cores in the same tile.
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
        if ((base & gcm) == gcm) apply_op<float>(tile, P.m, op, P.ops + oi, mats + op.mat);
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
  if (t > kTilePassThreads) t = kTilePassThreads;
  return t;
}

size_t tile_smem(sv_dtype dt, int m, int nvec) { return (size_t)nvec * ((size_t)1 << m) * amp_bytes(dt); }


sv_status launch_tile_pass(sv_state *s, const TilePass &p, int batch) {
  return launch_tile_pass_on(s, p, batch, s->stream);
}

sv_status launch_tile_pass_on(sv_state *s, const TilePass &p, int batch, cudaStream_t stream) {
  static bool attr_set[2][64] = {};
  if (p.flags & kPassHasTC) {
    if (s->dt != SV_C64 || p.m != kTcTileM || batch != 1 || p.nvec != 1)
      return set_error(SV_EINVAL, "internal: tensor-core tile pass needs one complex64 vector and 12-qubit tiles");
    const sv_prec mode = (sv_prec)((p.flags >> 9) & 3);
    const size_t smem = tc_tile_smem(mode);
    static bool attr = false;
    if (!attr) {
      SV_CUDA(cudaFuncSetAttribute(k_tile_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10));
      SV_CUDA(cudaFuncSetAttribute(k_tile_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
      attr = true;
    }
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
