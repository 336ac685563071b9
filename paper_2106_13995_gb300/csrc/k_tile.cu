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
// The ops themselves and the tile's shared-memory layout are in
// tile_ops.cuh; tile passes with tensor-core blocks are in k_tile_tc.cu.
#include <algorithm>
#include <cstring>

#include "tile_ops.cuh"

namespace sv {

constexpr int kTileMaxThreads = 512;    // persistent batch kernel
// tile passes: 32 amplitudes per thread (each op's set-up is paid for that
// many), at most 256 threads, up to 80 registers a thread
constexpr int kTilePassThreads = 256;
constexpr int kTilePassMinBlocks = 3;

__device__ __forceinline__ void cp_async8(uint32_t smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem), "l"(gmem) : "memory");
}

// The work of one CTA on one tile.  COH selects L2-coherent loads and stores
// (bypassing L1), needed when other CTAs of the same launch wrote the tile
// earlier (the persistent batch kernel); otherwise streaming hints are used.
template <typename R, bool COH, bool INL = false>
__device__ __forceinline__ void tile_body(const TilePass &P, uint64_t tile, int b, unsigned char *smem_raw,
                                          const TileInline *I = nullptr) {
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
  if constexpr (!COH) {
    // loads: asynchronous copies straight into the swizzled slots (8 bytes
    // per complex64 amplitude: a unit's two slots may be swapped), all of a
    // thread's copies in flight at once
    const uint32_t vs0 = smem_u32(v0), vs1 = smem_u32(v1);
    for (uint32_t i = 0; i * blockDim.x + threadIdx.x < nunits; i++) {
      const uint64_t g = goff(i);
      const uint32_t l = (i * blockDim.x + threadIdx.x) * UN::APU;
      if (sizeof(C) == 8) {
        cp_async8(vs0 + swb<R>(l), &g0[g]);
        cp_async8(vs0 + swb<R>(l + 1), &g0[g + 1]);
        if (load1) {
          cp_async8(vs1 + swb<R>(l), &g1[g]);
          cp_async8(vs1 + swb<R>(l + 1), &g1[g + 1]);
        }
      } else {
        cp_async16(vs0 + swb<R>(l), &g0[g]);
        if (load1) cp_async16(vs1 + swb<R>(l), &g1[g]);
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  } else {
    // loads through L2 only (other CTAs of the launch wrote the tile): four
    // 16-byte units in flight per thread before any shared store
    constexpr int BATCH = 4;
    for (uint32_t i0 = 0; i0 * blockDim.x + threadIdx.x < nunits; i0 += BATCH) {
      int4 r0[BATCH], r1[BATCH];
#pragma unroll
      for (int j = 0; j < BATCH; j++) {
        const uint32_t u = (i0 + j) * blockDim.x + threadIdx.x;
        if (u < nunits) {
          const uint64_t g = goff(i0 + j);
          r0[j] = __ldcg(reinterpret_cast<const int4 *>(&g0[g]));
          if (load1) r1[j] = __ldcg(reinterpret_cast<const int4 *>(&g1[g]));
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
  }

  const C *mats = reinterpret_cast<const C *>(P.mats);
  const C *pmats = P.pmats ? reinterpret_cast<const C *>(P.pmats) + (size_t)b * P.pmats_stride : nullptr;
  double *acc = P.acc ? P.acc + (size_t)b * P.acc_stride : nullptr;

  for (int oi = 0; oi < P.nops; oi++) {
    __syncthreads();
    TileOp op;
    if constexpr (INL) op = I->ops[oi];
    else op = P.ops[oi];
    const uint64_t gcm = (uint64_t)op.gcmask_lo | ((uint64_t)op.gcmask_hi << 32);
    switch (op.kind) {
      case TOP_DENSE:
      case TOP_DIAG: {
        if ((base & gcm) != gcm) break;
        if constexpr (INL && sizeof(R) == 4) {
          if (op.gen & kGenInline) {   // single vector: vmask is 1
            apply_op_inl(reinterpret_cast<float2 *>(v0), P.m, op, *I, oi, threadIdx.x, blockDim.x);
            break;
          }
          if (op.kind == TOP_DENSE && op.k <= 3) {
            // the host launches this kernel only when every such block is in
            // the parameter block; report a broken invariant instead of
            // computing without the block
            if (threadIdx.x == 0) atomicOr(P.err, kErrNoInlineBlock);
            break;
          }
        }
        const C *U = ((op.gen & kGenBatchMat) ? pmats : mats) + op.mat;
        if (op.vmask & 1) apply_op<R, INL>(v0, P.m, op, P.ops + oi, U, threadIdx.x, blockDim.x);
        if (op.vmask & 2) apply_op<R, INL>(v1, P.m, op, P.ops + oi, U, threadIdx.x, blockDim.x);
        break;
      }
      case TOP_PERM: {
        if ((base & gcm) != gcm) break;
        const uint8_t *perm = static_cast<const uint8_t *>(P.mats) + (size_t)op.mat * sizeof(C);
        if (op.vmask & 1) perm_op<R>(v0, P.m, P.ops + oi, op.k, perm, threadIdx.x, blockDim.x);
        if (op.vmask & 2) perm_op<R>(v1, P.m, P.ops + oi, op.k, perm, threadIdx.x, blockDim.x);
        break;
      }
      case TOP_GRAD:
        grad_op<R>(v0, v1, P.m, op, acc);
        break;
      case TOP_GRADU: {
        const C *U = ((op.gen & kGenBatchMat) ? pmats : mats) + op.mat;
        grad_u_op<R>(v0, v1, P.m, op, U, acc);
        break;
      }
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

// The same pass with its op list and small dense matrices in the parameter
// block (complex64, one vector, one state).
__global__ void __launch_bounds__(kTilePassThreads, kTilePassMinBlocks)
    k_tile_inl(const __grid_constant__ TilePass P, const __grid_constant__ TileInline I) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tile_body<float, false, true>(P, blockIdx.x, 0, smem_raw, &I);
}
static_assert(sizeof(TilePass) + sizeof(TileInline) <= 32000, "kernel parameters exceed 32 KB");

// Fill a parameter block from the host copy of a pass: all ops, and the
// matrices of its 1-3 qubit dense blocks (already in the row-pair layout).
// False unless every such block fits (the kernel has no other path for
// them).
// host copies of the device's index maps (tile_ops.cuh), for OpPre
static uint32_t h_swb(uint32_t l) { return (l ^ ((l >> 4) & 15u)) * (uint32_t)sizeof(float2); }
static uint32_t h_ins0_mask(uint32_t x, uint32_t fixed) {
  for (; fixed; fixed &= fixed - 1) {
    const int p = __builtin_ctz(fixed);
    const uint32_t low = x & ((1u << p) - 1);
    x = ((x ^ low) << 1) | low;
  }
  return x;
}

void fill_op_pre(const TileOp &op, int threads, OpPre &pre) {
  std::memset(&pre, 0, sizeof(pre));
  uint32_t fixed = op.lcmask;
  pre.soff[0] = 0;
  for (int j = 0; j < op.k; j++) {
    const uint32_t bit = 1u << op.t[j];
    fixed |= bit;
    for (int y = 0; y < (1 << j); y++) pre.soff[y + (1 << j)] = pre.soff[y] ^ h_swb(bit);
  }
  // trip map for T = threads (a power of two): fixed bits up to the trip
  // region shift it, the ones above are inserted per trip
  uint32_t low = (uint32_t)__builtin_ctz((uint32_t)threads), f = fixed;
  while (f) {
    const uint32_t q = (uint32_t)__builtin_ctz(f);
    if (q > low) break;
    f &= f - 1;
    low++;
  }
  pre.tm_shift = low;
  pre.tm_hi = f;
  const int G = pairs_groups(op.k);
  for (int hh = 0; hh < G; hh++) pre.dh[hh] = h_swb(h_ins0_mask((uint32_t)hh << low, f));
  for (int it = 0; it < 4; it++) pre.tc[it] = h_swb(h_ins0_mask((uint32_t)(it * G) << low, f));
}

static bool build_inline(const TilePass &p, const HostPass &h, TileInline &I, int threads) {
  if (p.nops > kInlOps) return false;
  I.nops = (uint32_t)p.nops;
  I.nmat = 0;
  for (int i = 0; i < p.nops; i++) {
    TileOp op = h.ops[i];
    if (op.kind == TOP_DENSE && op.k <= 3) {
      const uint32_t cnt = 1u << (2 * op.k);
      const uint32_t at = I.nmat;
      if (op.gen != 0 || op.vmask != 1 || at + cnt > (uint32_t)kInlMat) return false;
      std::memcpy(&I.mats[at], h.mats + (size_t)op.mat * sizeof(float2), cnt * sizeof(float2));
      op.mat = at;
      op.gen = kGenInline;
      I.nmat = at + cnt;
      fill_op_pre(op, threads, I.pre[i]);
    }
    I.ops[i] = op;
  }
  return true;
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
  int t = units / 16;
  if (t < 32) t = 32;
  if (t > kTilePassThreads) t = kTilePassThreads;
  return t;
}

size_t tile_smem(sv_dtype dt, int m, int nvec) { return (size_t)nvec * ((size_t)1 << m) * amp_bytes(dt); }


sv_status launch_tile_pass(sv_state *s, const TilePass &p, int batch) {
  return launch_tile_pass_on(s, p, batch, s->stream);
}

// K11: a permutation pass (kPassTable; paper Sec. III's reversible
// multipliers).  One CTA per tile (and per state of a batch): the tile is
// loaded into shared memory, then every output amplitude is read from the
// slot the pass's gather table names and stored -- one move per amplitude
// for all the pass's blocks, no arithmetic.  The table is the one for the
// values the pass's global control qubits take in this tile.
template <typename R>
__global__ void __launch_bounds__(kTilePassThreads) k_tile_tperm(const __grid_constant__ TilePass P) {
  using C = typename Cx<R>::T;
  using UN = Unit<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *v = reinterpret_cast<C *>(smem_raw);
  const uint32_t TS = 1u << P.m;
  const uint64_t base = tile_base(P, blockIdx.x);
  C *g0 = reinterpret_cast<C *>(P.tbl0 ? P.tbl0[blockIdx.y] : P.v0);
  const unsigned char *blk = static_cast<const unsigned char *>(P.mats) + 16 * (size_t)P.mat0;
  const uint32_t g = *reinterpret_cast<const uint32_t *>(blk);
  uint32_t var = 0;
  for (uint32_t i = 0; i < g; i++) var |= (uint32_t)((base >> blk[4 + i]) & 1ull) << i;
  const uint16_t *tab = reinterpret_cast<const uint16_t *>(blk + 16) + (size_t)var * TS;
  const uint32_t nunits = TS / UN::APU;
  const uint32_t segmask = (1u << P.L) - 1;
  const uint32_t lthr = threadIdx.x * UN::APU;
  const uint64_t gthr = base | (lthr & segmask) | spread_hi(P, lthr & ~segmask);
  const uint32_t tstep = blockDim.x * UN::APU;
  auto goff = [&](uint32_t i) -> uint64_t {
    const uint32_t lt = i * tstep;
    return gthr | (lt & segmask) | spread_hi(P, lt & ~segmask);
  };
  // sixteen units per thread and batch, so sixteen loads (and table reads)
  // are in flight at a time
  constexpr uint32_t kBatch = 16;
  for (uint32_t i0 = 0; i0 * blockDim.x + threadIdx.x < nunits; i0 += kBatch) {
    int4 r[kBatch];
#pragma unroll
    for (uint32_t j = 0; j < kBatch; j++)
      if ((i0 + j) * blockDim.x + threadIdx.x < nunits) r[j] = __ldcs(reinterpret_cast<const int4 *>(&g0[goff(i0 + j)]));
#pragma unroll
    for (uint32_t j = 0; j < kBatch; j++) {
      const uint32_t u = (i0 + j) * blockDim.x + threadIdx.x;
      if (u < nunits) UN::put(v, u * UN::APU, r[j]);
    }
  }
  __syncthreads();
  for (uint32_t i0 = 0; i0 * blockDim.x + threadIdx.x < nunits; i0 += kBatch) {
    uint16_t src[kBatch][UN::APU];
#pragma unroll
    for (uint32_t j = 0; j < kBatch; j++) {
      const uint32_t u = (i0 + j) * blockDim.x + threadIdx.x;
      if (u < nunits) {
#pragma unroll
        for (uint32_t a = 0; a < UN::APU; a++) src[j][a] = __ldg(tab + u * UN::APU + a);
      }
    }
#pragma unroll
    for (uint32_t j = 0; j < kBatch; j++) {
      const uint32_t u = (i0 + j) * blockDim.x + threadIdx.x;
      if (u < nunits) {
        C out[UN::APU];
#pragma unroll
        for (uint32_t a = 0; a < UN::APU; a++) out[a] = v[sw<R>(src[j][a])];
        __stcs(reinterpret_cast<int4 *>(&g0[goff(i0 + j)]), *reinterpret_cast<const int4 *>(out));
      }
    }
  }
}

static sv_status launch_tile_tperm(sv_state *s, const TilePass &p, int batch, cudaStream_t stream) {
  if (p.nvec != 1 || p.m > 16) return set_error(SV_EINVAL, "internal: permutation pass needs one vector and m <= 16");
  const size_t smem = tile_smem(s->dt, p.m, 1);
  if (smem > (200u << 10)) return set_error(SV_EINVAL, "tile too large for shared memory");
  const void *fn = s->dt == SV_C64 ? (const void *)k_tile_tperm<float> : (const void *)k_tile_tperm<double>;
  SV_TRY(func_attr_once(fn, s->device, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10));
  dim3 grid((unsigned)(1ull << (p.n - p.m)), (unsigned)batch);
  const int threads = tile_threads(p.m, s->dt);
  if (s->dt == SV_C64)
    k_tile_tperm<float><<<grid, threads, smem, stream>>>(p);
  else
    k_tile_tperm<double><<<grid, threads, smem, stream>>>(p);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

sv_status launch_tile_pass_on(sv_state *s, const TilePass &p, int batch, cudaStream_t stream,
                              const HostPass *host) {
  if (p.flags & kPassTable) return launch_tile_tperm(s, p, batch, stream);
  if (p.flags & kPassHasTC) {
    if (s->dt != SV_C64 || p.m != kTcTileM || batch != 1 || p.nvec != 1)
      return set_error(SV_EINVAL, "internal: tensor-core tile pass needs one complex64 vector and 12-qubit tiles");
    // passes of split-BF16 tensor-core blocks only: the pipelined kernel
    if (host && ((p.flags >> 9) & 3) == SV_PREC_TC_BF16X3 && tcp_pass_ok(p, *host))
      return launch_tile_tcp(s, p, *host, stream);
    return launch_tile_tc(s, p, stream);
  }
  const size_t smem = tile_smem(s->dt, p.m, (int)p.nvec);
  const cudaFuncAttribute kSmemAttr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (s->dt == SV_C64) {
    SV_TRY(func_attr_once((const void *)k_tile<float>, s->device, kSmemAttr, 200 << 10));
    SV_TRY(func_attr_once((const void *)k_tile_inl, s->device, kSmemAttr, 200 << 10));
  } else {
    SV_TRY(func_attr_once((const void *)k_tile<double>, s->device, kSmemAttr, 200 << 10));
  }
  if (smem > (200u << 10)) return set_error(SV_EINVAL, "tile too large for shared memory");
  dim3 grid((unsigned)(1ull << (p.n - p.m)), (unsigned)batch);
  const int threads = tile_threads(p.m, s->dt);
  TileInline inl;   // copied into the launch
  if (host && s->dt == SV_C64 && batch == 1 && p.nvec == 1 && build_inline(p, *host, inl, threads))
    k_tile_inl<<<grid, threads, smem, stream>>>(p, inl);
  else if (s->dt == SV_C64)
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
  SV_TRY(func_attr_once(fn, s->device, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10));
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
