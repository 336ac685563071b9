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
        if (op.vmask & 1) apply_op<R>(v0, P.m, op, U);
        if (op.vmask & 2) apply_op<R>(v1, P.m, op, U);
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
__global__ void __launch_bounds__(kTileMaxThreads, 2) k_tile(const __grid_constant__ TilePass P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tile_body<R, false>(P, blockIdx.x, blockIdx.y, smem_raw);
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


sv_status launch_tile_pass(sv_state *s, const TilePass &p, int batch) {
  return launch_tile_pass_on(s, p, batch, s->stream);
}

sv_status launch_tile_pass_on(sv_state *s, const TilePass &p, int batch, cudaStream_t stream) {
  static bool attr_set[2][64] = {};
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
