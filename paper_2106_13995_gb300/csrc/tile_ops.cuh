// Tile operations shared by the tile-pass kernels: the swizzled shared-memory
// layout of a tile, index spreading between tile-local and state indices, and
// the ops a pass applies to a tile (dense blocks with local controls, diagonal
// blocks, gradient probes, the 16-byte unit moves of tile loads and stores).
//
// Shared-memory layout: amplitude l of the tile lives at sw(l), an XOR
// swizzle of its low bits by the next bits up.  A gate on low local qubits
// makes a warp's 32 groups stride through the tile; without the swizzle
// those strides land on a few banks (up to 8-way conflicts for three low
// targets), with it every access pattern of the op list spreads over all
// banks.
#pragma once

#include <cuda_bf16.h>

#include "sv_device.cuh"
#include "sv_internal.h"

namespace sv {

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

// Trip part of a group's local index.  A thread's groups are g = t + c T
// (t < T, T a power of two), and the local index inserts zeros at the op's
// fixed bit positions: l(g) = l(t) ^ l(c T), both maps linear over GF(2).
// For l(c T) the fixed positions below the trip bits only shift them up,
// the same for every c; only fixed positions above need a per-trip insert.
struct TripMap {
  uint32_t shift;  // log2(T) + fixed bits below the trip region
  uint32_t hi;     // fixed bits above it
};
__device__ __forceinline__ TripMap trip_map(uint32_t T, uint32_t fixed) {
  uint32_t low = __ffs(T) - 1, f = fixed;
  while (f) {
    const uint32_t p = __ffs(f) - 1;
    if (p > low) break;
    f &= f - 1;
    low++;
  }
  return {low, f};
}
__device__ __forceinline__ uint32_t trip_l(uint32_t c, const TripMap &tm) {
  return ins0_mask(c << tm.shift, tm.hi);
}

// Local index of thread t's first group: thread bit i goes to the position
// the plan stored for it (the free positions of the op, with the lane bits
// arranged so that one shared-memory wavefront spans all bank rows).
__device__ __forceinline__ uint32_t thread_l(uint32_t t, const TileOp &op) {
  uint32_t l = 0;
#pragma unroll
  for (int i = 0; i < 9; i++) l |= ((t >> i) & 1u) << ((op.tbpos[i >> 1] >> (4 * (i & 1))) & 15u);
  return l;
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
                                         const typename Cx<R>::T *__restrict__ U,
                                         uint32_t tid, uint32_t T) {
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
  if (tid >= ngroups) return;
  // thread t's groups are t + c T, c < ntrips; slot(t + c T) = slot(t) ^
  // slot(c T), and a trip's G groups c0 + h share slot(c0 T)
  const uint32_t ntrips = ngroups > T ? ngroups / T : 1u;
  const uint32_t sthr = swb<R>(thread_l(tid, op) | op.lcmask);
  const TripMap tm = trip_map(T, fixed);
  uint32_t dh[G];
#pragma unroll
  for (int h = 0; h < G; h++) dh[h] = swb<R>(trip_l(h, tm));
  for (uint32_t c0 = 0; c0 < ntrips; c0 += G) {
    uint32_t s[G];
    bool ok[G];
    C x[G][D];
    const uint32_t sc = sthr ^ swb<R>(trip_l(c0, tm));
#pragma unroll
    for (int h = 0; h < G; h++) {
      ok[h] = c0 + h < ntrips;
      s[h] = ok[h] ? sc ^ dh[h] : sthr;
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

// Packed FP32 pairs: one f32x2 instruction performs two FMAs.
__device__ __forceinline__ uint64_t pk2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 upk2(uint64_t r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t lds_b64(uint32_t a) {
  uint64_t r;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(r) : "r"(a));
  return r;
}

// complex64 dense blocks of 1-3 qubits in packed FP32 arithmetic, columns
// outermost.  For output rows (2p, 2p+1) the packed accumulators hold
//   re = sum_y (Re U[2p][y], Re U[2p+1][y]) * (Re x_y, Re x_y)
//   tt = sum_y (Im U[2p][y], Im U[2p+1][y]) * (Im x_y, Im x_y)
//   im = sum_y (Re U .. ) * (Im x_y, Im x_y) + (Im U .. ) * (Re x_y, Re x_y)
// and the outputs are (re - tt, im) per row.  Each input amplitude is read
// once and broadcast into two pairs that feed every row pair; a group's
// outputs are written after its last column.  The matrix arrives as the
// row pairs (Re U[2p][y], Re U[2p+1][y]), (Im U[2p][y], Im U[2p+1][y]),
// the layout the host stores complex64 blocks of 1-3 qubits in: read from
// the launch's parameter block (warp-uniform reads take the uniform
// datapath) or from global memory through L1, with the same arithmetic, so
// every kernel that applies these blocks produces the same bits.
struct ParamPairs {
  static constexpr bool kPre = true;   // set-up from the host (OpPre)
  const TileInline &I;
  uint32_t base;
  uint32_t oi;
  template <int D>
  __device__ __forceinline__ void pair(int p, int y, uint64_t &ur, uint64_t &ui) const {
    const uint64_t *M = reinterpret_cast<const uint64_t *>(&I.mats[base]);
    ur = M[(p * D + y) * 2];
    ui = M[(p * D + y) * 2 + 1];
  }
};
struct GlobalPairs {
  static constexpr bool kPre = false;
  const float2 *U;   // row pairs, 16-byte aligned
  template <int D>
  __device__ __forceinline__ void pair(int p, int y, uint64_t &ur, uint64_t &ui) const {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(U + (p * D + y) * 2));
    ur = pk2(q.x, q.y);
    ui = pk2(q.z, q.w);
  }
};
template <int K, int G, class Src>
__device__ __forceinline__ void dense_pairs(float2 *__restrict__ v, int m, const TileOp &op, const Src &src,
                                            uint32_t tid, uint32_t T) {
  constexpr int D = 1 << K, NP = D / 2;
  const uint32_t vs = smem_u32(v);
  uint32_t soff[D], tmask = 0;
#pragma unroll
  for (int j = 0; j < K; j++) tmask |= 1u << op.t[j];
  if constexpr (Src::kPre) {
#pragma unroll
    for (int y = 0; y < D; y++) soff[y] = src.I.pre[src.oi].soff[y];
  } else {
    soff[0] = 0;
#pragma unroll
    for (int j = 0; j < K; j++) {
      const uint32_t e = swb<float>(1u << op.t[j]);
#pragma unroll
      for (int y = 0; y < (1 << j); y++) soff[y + (1 << j)] = soff[y] ^ e;
    }
  }
  const uint32_t fixed = tmask | op.lcmask;
  const uint32_t ngroups = 1u << (m - __popc(fixed));
  if (tid >= ngroups) return;
  // thread t's groups are t + c T, c < ntrips; slot(t + c T) = slot(t) ^
  // slot(c T), and a trip's G groups c0 + h share slot(c0 T)
  const uint32_t ntrips = ngroups > T ? ngroups / T : 1u;
  const uint32_t sthr = swb<float>(thread_l(tid, op) | op.lcmask);
  TripMap tm;
  uint32_t dh[G];
  if constexpr (Src::kPre) {
    const OpPre &pre = src.I.pre[src.oi];
    tm = TripMap{pre.tm_shift, pre.tm_hi};
#pragma unroll
    for (int h = 0; h < G; h++) dh[h] = pre.dh[h];
  } else {
    tm = trip_map(T, fixed);
#pragma unroll
    for (int h = 0; h < G; h++) dh[h] = swb<float>(trip_l(h, tm));
  }
  for (uint32_t c0 = 0, it = 0; c0 < ntrips; c0 += G, it++) {
    uint32_t s[G];
    bool ok[G];
    uint32_t sct;
    if constexpr (Src::kPre) sct = it < 4 ? src.I.pre[src.oi].tc[it] : swb<float>(trip_l(c0, tm));
    else sct = swb<float>(trip_l(c0, tm));
    const uint32_t sc = sthr ^ sct;
#pragma unroll
    for (int h = 0; h < G; h++) {
      ok[h] = c0 + h < ntrips;
      s[h] = ok[h] ? sc ^ dh[h] : sthr;
    }
    uint64_t re[NP][G], tt[NP][G], im[NP][G];
#pragma unroll
    for (int p = 0; p < NP; p++)
#pragma unroll
      for (int h = 0; h < G; h++) re[p][h] = tt[p][h] = im[p][h] = 0ull;
#pragma unroll
    for (int y = 0; y < D; y++) {
      uint64_t xr[G], xi[G];
#pragma unroll
      for (int h = 0; h < G; h++) {
        const float2 x = upk2(lds_b64(vs + (s[h] ^ soff[y])));
        xr[h] = pk2(x.x, x.x);
        xi[h] = pk2(x.y, x.y);
      }
#pragma unroll
      for (int p = 0; p < NP; p++) {
        uint64_t ur, ui;
        src.template pair<D>(p, y, ur, ui);
#pragma unroll
        for (int h = 0; h < G; h++) {
          re[p][h] = fma2(ur, xr[h], re[p][h]);
          tt[p][h] = fma2(ui, xi[h], tt[p][h]);
          im[p][h] = fma2(ur, xi[h], im[p][h]);
          im[p][h] = fma2(ui, xr[h], im[p][h]);
        }
      }
    }
#pragma unroll
    for (int p = 0; p < NP; p++)
#pragma unroll
      for (int h = 0; h < G; h++)
        if (ok[h]) {
          const float2 a = upk2(re[p][h]), b = upk2(tt[p][h]), c = upk2(im[p][h]);
          sts_c(vs + (s[h] ^ soff[2 * p]), make_float2(a.x - b.x, c.x));
          sts_c(vs + (s[h] ^ soff[2 * p + 1]), make_float2(a.y - b.y, c.y));
        }
  }
}

// groups per trip of the packed blocks (registers: three packed
// accumulators per row pair and group); the grouping does not change the
// arithmetic
template <int K> constexpr int kPairsG = pairs_groups(K);

// groups per trip with matrices in global memory (batched, two-vector and
// tensor-core passes, ops beyond a parameter block): the loaded pairs take
// ordinary registers, so 3-qubit blocks run one group per trip
template <int K> constexpr int kPairsGlobalG = K == 1 ? 4 : (K == 2 ? 2 : 1);

// WIDE: the kernel has registers to spare (128 a thread): two groups per
// trip for 3-qubit blocks
template <bool WIDE = false>
__device__ __forceinline__ void dense_pairs_global(float2 *v, int m, const TileOp &op, const float2 *U,
                                                   uint32_t tid, uint32_t T) {
  const GlobalPairs src{U};
  switch (op.k) {
    case 1: dense_pairs<1, kPairsGlobalG<1>>(v, m, op, src, tid, T); break;
    case 2: dense_pairs<2, kPairsGlobalG<2>>(v, m, op, src, tid, T); break;
    default: dense_pairs<3, WIDE ? 2 : kPairsGlobalG<3>>(v, m, op, src, tid, T); break;
  }
}

// Dense complex64 block of 1-3 qubits whose matrix is in the launch's
// parameter block (op.mat indexes TileInline::mats, stored as row pairs).
__device__ __forceinline__ void apply_op_inl(float2 *v, int m, const TileOp &op, const TileInline &I, int oi,
                                             uint32_t tid, uint32_t T) {
  const ParamPairs src{I, op.mat, (uint32_t)oi};
  switch (op.k) {
    case 1: dense_pairs<1, kPairsG<1>>(v, m, op, src, tid, T); break;
    case 2: dense_pairs<2, kPairsG<2>>(v, m, op, src, tid, T); break;
    default: dense_pairs<3, kPairsG<3>>(v, m, op, src, tid, T); break;
  }
}

// Dense blocks of 4..6 qubits keep 2^k amplitudes per thread; they run as
// functions of their own so their registers do not crowd the k <= 3 paths
// that make up most passes.  The op is read from global memory here, so no
// caller keeps an addressable (local-memory) copy of it.
template <typename R, int K>
__device__ __noinline__ void dense_op_big(typename Cx<R>::T *__restrict__ v, int m, const TileOp *gop,
                                          const typename Cx<R>::T *__restrict__ U, uint32_t tid,
                                          uint32_t T) {
  const TileOp op = *gop;
  dense_op<R, K, 1>(v, m, op, U, tid, T);
}

// Diagonal block: amplitude l is multiplied by d[r(l)], r(l) the target bits
// of l.  Both the slot and r are linear in l, so each splits into a thread
// part and a warp-uniform trip part.
template <typename R>
__device__ __forceinline__ void diag_op(typename Cx<R>::T *__restrict__ v, int m, const TileOp &op,
                                        const typename Cx<R>::T *__restrict__ d, uint32_t tid,
                                        uint32_t T) {
  using C = typename Cx<R>::T;
  unsigned char *vb = reinterpret_cast<unsigned char *>(v);
  const uint32_t ngroups = 1u << (m - __popc(op.lcmask));
  if (tid >= ngroups) return;
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
  const uint32_t lthr = thread_l(tid, op) | op.lcmask;
  const uint32_t sthr = swb<R>(lthr), rthr = rows(lthr);
  const TripMap tm = trip_map(T, op.lcmask);
  for (uint32_t g0 = 0, c = 0; g0 < ngroups; g0 += T, c++) {
    const uint32_t lg = trip_l(c, tm);
    C *p = reinterpret_cast<C *>(vb + (sthr ^ swb<R>(lg)));
    *p = cmul(__ldg(&d[rthr ^ rows(lg)]), *p);
  }
}

// kSmallInParams: the kernel takes complex64 dense blocks of 1-3 qubits from
// its parameter block and never here (leaving that code out keeps its
// registers off the hot path)
template <typename R, bool kSmallInParams = false, bool kWideRegs = false>
__device__ __forceinline__ void apply_op(typename Cx<R>::T *v, int m, const TileOp &op, const TileOp *gop,
                                         const typename Cx<R>::T *U, uint32_t tid, uint32_t T) {
  if (op.kind == TOP_DIAG) {
    diag_op<R>(v, m, op, U, tid, T);
    return;
  }
  if constexpr (sizeof(R) == 4) {
    if constexpr (!kSmallInParams) {
      if (op.k <= 3) {
        dense_pairs_global<kWideRegs>(v, m, op, U, tid, T);
        return;
      }
    }
  }
  switch (op.k) {
    // groups per trip: as many as the registers allow next to a thread's
    // amplitudes (complex128 needs twice the registers per amplitude)
    case 1: dense_op<R, 1, sizeof(R) == 4 ? 4 : 2>(v, m, op, U, tid, T); break;
    case 2: dense_op<R, 2, sizeof(R) == 4 ? 2 : 1>(v, m, op, U, tid, T); break;
    case 3: dense_op<R, 3, sizeof(R) == 4 ? 2 : 1>(v, m, op, U, tid, T); break;
    case 4: dense_op_big<R, 4>(v, m, gop, U, tid, T); break;
    case 5: dense_op_big<R, 5>(v, m, gop, U, tid, T); break;
    default: dense_op_big<R, 6>(v, m, gop, U, tid, T); break;
  }
}

// Permutation block: a dense block whose matrix has one entry 1 in every
// row and column (X, CNOT, Toffoli, C^3X and their products) only moves
// amplitudes: member y of each control-satisfied group goes to member
// perm[y] (perm: 2^K bytes).  No arithmetic, so the result is exact.  Out of
// line, like the large dense blocks, so its registers stay off the hot path;
// the op is read from global memory.
template <typename R, int K>
__device__ __noinline__ void perm_op_k(typename Cx<R>::T *__restrict__ v, int m, const TileOp *gop,
                                       const uint8_t *__restrict__ perm, uint32_t tid, uint32_t T) {
  using C = typename Cx<R>::T;
  constexpr int D = 1 << K;
  const TileOp op = *gop;
  const uint32_t vs = smem_u32(v);
  uint32_t soff[D], dst[D], tmask = 0;
  soff[0] = 0;
#pragma unroll
  for (int j = 0; j < K; j++) {
    const uint32_t bit = 1u << op.t[j];
    tmask |= bit;
    const uint32_t e = swb<R>(bit);
#pragma unroll
    for (int y = 0; y < (1 << j); y++) soff[y + (1 << j)] = soff[y] ^ e;
  }
#pragma unroll
  for (int y = 0; y < D; y++) {
    const uint32_t r = __ldg(perm + y) & (D - 1);
    uint32_t so = 0;
#pragma unroll
    for (int j = 0; j < K; j++) so ^= ((r >> j) & 1u) ? swb<R>(1u << op.t[j]) : 0u;
    dst[y] = so;
  }
  const uint32_t fixed = tmask | op.lcmask;
  const uint32_t ngroups = 1u << (m - __popc(fixed));
  if (tid >= ngroups) return;
  const uint32_t ntrips = ngroups > T ? ngroups / T : 1u;
  const uint32_t sthr = swb<R>(thread_l(tid, op) | op.lcmask);
  const TripMap tm = trip_map(T, fixed);
  for (uint32_t c = 0; c < ntrips; c++) {
    const uint32_t s = sthr ^ swb<R>(trip_l(c, tm));
    C x[D];
#pragma unroll
    for (int y = 0; y < D; y++) x[y] = lds_c(vs + (s ^ soff[y]), (const C *)nullptr);
#pragma unroll
    for (int y = 0; y < D; y++) sts_c(vs + (s ^ dst[y]), x[y]);
  }
}
template <typename R>
__device__ __forceinline__ void perm_op(typename Cx<R>::T *v, int m, const TileOp *gop, int k, const uint8_t *perm,
                                        uint32_t tid, uint32_t T) {
  switch (k) {
    case 1: perm_op_k<R, 1>(v, m, gop, perm, tid, T); break;
    case 2: perm_op_k<R, 2>(v, m, gop, perm, tid, T); break;
    default: perm_op_k<R, 3>(v, m, gop, perm, tid, T); break;
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

// The adjoint sweep's step for one parametric gate, in one pass over the
// pairs of both vectors: acc[slot] += Im <lambda | G | psi> (as grad_op,
// on the vectors after the gate), then both vectors <- U^dagger (the 1-qubit
// matrix at U: row pairs for complex64, row-major for complex128).
__device__ __forceinline__ void load_u2(const float2 *U, float2 &u00, float2 &u01, float2 &u10, float2 &u11) {
  const float4 q0 = __ldg(reinterpret_cast<const float4 *>(U));
  const float4 q1 = __ldg(reinterpret_cast<const float4 *>(U) + 1);
  u00 = make_float2(q0.x, q0.z);
  u10 = make_float2(q0.y, q0.w);
  u01 = make_float2(q1.x, q1.z);
  u11 = make_float2(q1.y, q1.w);
}
__device__ __forceinline__ void load_u2(const double2 *U, double2 &u00, double2 &u01, double2 &u10, double2 &u11) {
  u00 = __ldg(U);
  u01 = __ldg(U + 1);
  u10 = __ldg(U + 2);
  u11 = __ldg(U + 3);
}

template <typename R>
__device__ void grad_u_op(typename Cx<R>::T *__restrict__ psi, typename Cx<R>::T *__restrict__ lam, int m,
                          const TileOp &op, const typename Cx<R>::T *__restrict__ U, double *acc) {
  using C = typename Cx<R>::T;
  const int t = op.t[0];
  const uint32_t bit = 1u << t;
  const uint32_t ngroups = 1u << (m - 1);
  C u00, u01, u10, u11;
  load_u2(U, u00, u01, u10, u11);
  const int gen = op.gen & 0x7;
  R part = 0;
  for (uint32_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
    const uint32_t l0 = ins0(g, t), l1 = l0 | bit;
    const uint32_t p0 = sw<R>(l0), p1 = sw<R>(l1);
    const C a0 = psi[p0], a1 = psi[p1], b0 = lam[p0], b1 = lam[p1];
    switch (gen) {
      case 1: part += imdot(b0, a1) + imdot(b1, a0); break;                       // X
      case 2: part += imdot(b0, cmake(a1.y, -a1.x)) + imdot(b1, cmake(-a0.y, a0.x)); break;   // Y
      case 3: part += imdot(b0, a0) - imdot(b1, a1); break;                       // Z
      default: part += R(-2) * imdot(b1, a1); break;                              // diag(0, -2)
    }
    psi[p0] = cfma(u01, a1, cmul(u00, a0));
    psi[p1] = cfma(u11, a1, cmul(u10, a0));
    lam[p0] = cfma(u01, b1, cmul(u00, b0));
    lam[p1] = cfma(u11, b1, cmul(u10, b0));
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

}  // namespace sv
