// K8-K10 and state set-up: basis initialisation, scaling, norm, Pauli-string
// expectations, all-qubit <Z_q>, and inverse-CDF sampling.
//
// Reductions form products in the state's precision and accumulate short
// runs (8-16 amplitudes) in that precision before adding into FP64; block and
// grid levels are FP64 throughout.  Sampling locates a draw's 1024-amplitude
// chunk from such chunk totals and then walks the chunk with |psi_x|^2 in
// FP64, so the chosen index is the one an FP64 reference would pick from the
// same amplitudes (up to draws within ~1e-12 of a chunk boundary).
#include <algorithm>
#include <mutex>
#include <vector>

#include "sv_device.cuh"
#include "sv_internal.h"

namespace sv {

constexpr int kRedThreads = 256;

static int red_grid(sv_state *s, uint64_t work) {
  const uint64_t want = (work + kRedThreads - 1) / kRedThreads;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)s->sm_count * 4));
}
int red_blocks_max(sv_state *s) { return s->sm_count * 4; }

// ---- basis state / scaling -----------------------------------------------
template <typename R>
__global__ void k_set_basis(int4 *__restrict__ a, uint64_t nunits, uint64_t index) {
  using C = typename Cx<R>::T;
  constexpr uint64_t APU = 16 / sizeof(C);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t hit = index / APU;
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nunits; u += stride) {
    int4 z = make_int4(0, 0, 0, 0);
    if (u == hit) {
      C v[APU];
      for (uint64_t j = 0; j < APU; j++) v[j] = czero<C>();
      v[index % APU].x = R(1);
      z = *reinterpret_cast<int4 *>(v);
    }
    __stcs(a + u, z);
  }
}

template <typename R>
__global__ void k_scale(typename Cx<R>::T *__restrict__ a, uint64_t namps, R f) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < namps; i += stride) {
    auto v = a[i];
    v.x *= f;
    v.y *= f;
    a[i] = v;
  }
}

sv_status launch_set_basis(sv_state *s, uint64_t index) {
  const uint64_t nunits = ((1ull << s->n) * amp_bytes(s->dt) + 15) / 16;
  const int g = std::min<uint64_t>((nunits + kRedThreads - 1) / kRedThreads, (uint64_t)s->sm_count * 8);
  if (s->dt == SV_C64)
    k_set_basis<float><<<std::max(g, 1), kRedThreads, 0, s->stream>>>((int4 *)s->amps, nunits, index);
  else
    k_set_basis<double><<<std::max(g, 1), kRedThreads, 0, s->stream>>>((int4 *)s->amps, nunits, index);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

template <typename R>
__global__ void k_move_basis(typename Cx<R>::T *a, uint64_t from, uint64_t to, R re, R im) {
  if (from != to) a[from] = czero<typename Cx<R>::T>();
  a[to] = cmake(re, im);
}

// Bulk copy by the SMs, 16 bytes per thread and trip, four trips in flight:
// used for host <-> device moves of page-locked host memory, which the GPU
// reads and writes directly over its host link (the copy engines are not
// involved, so their other traffic does not slow it).
__global__ void __launch_bounds__(256) k_copy16(const int4 *__restrict__ src, int4 *__restrict__ dst, size_t n16) {
  const size_t st = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * st < n16; i += 4 * st) {
    const int4 a = src[i], b = src[i + st], c = src[i + 2 * st], d = src[i + 3 * st];
    dst[i] = a;
    dst[i + st] = b;
    dst[i + 2 * st] = c;
    dst[i + 3 * st] = d;
  }
  for (; i < n16; i += st) dst[i] = src[i];
}

sv_status launch_copy16(sv_state *s, const void *src, void *dst, size_t bytes) {
  if (bytes % 16 || ((uintptr_t)src | (uintptr_t)dst) % 16) return set_error(SV_EINVAL, "internal: unaligned copy");
  if (bytes == 0) return SV_OK;
  const size_t n16 = bytes / 16;
  const size_t want = (n16 + 255) / 256;
  const int grid = (int)std::max<size_t>(1, std::min<size_t>(want, (size_t)s->sm_count * 4));
  k_copy16<<<grid, 256, 0, s->stream>>>(reinterpret_cast<const int4 *>(src), reinterpret_cast<int4 *>(dst), n16);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

sv_status launch_move_basis(sv_state *s, uint64_t from, uint64_t to, cd amp) {
  if (s->dt == SV_C64)
    k_move_basis<float><<<1, 1, 0, s->stream>>>((float2 *)s->amps, from, to, (float)amp.real(), (float)amp.imag());
  else
    k_move_basis<double><<<1, 1, 0, s->stream>>>((double2 *)s->amps, from, to, amp.real(), amp.imag());
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

sv_status launch_scale(sv_state *s, double f) {
  const uint64_t na = 1ull << s->n;
  const int g = red_grid(s, na);
  if (s->dt == SV_C64)
    k_scale<float><<<g, kRedThreads, 0, s->stream>>>((float2 *)s->amps, na, (float)f);
  else
    k_scale<double><<<g, kRedThreads, 0, s->stream>>>((double2 *)s->amps, na, f);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

// ---- block reduction helpers ---------------------------------------------
__device__ __forceinline__ void block_sum_to(double v, double *dst) {
  __shared__ double red[32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
    t = warp_sum(t);
    if (l == 0) *dst = t;
  }
}

// out[j] = sum_b partial[b * nvals + j]  (+ optional add into out)
__global__ void k_finalize(const double *__restrict__ partial, int nblocks, int nvals, double *out) {
  for (int j = threadIdx.x; j < nvals; j += blockDim.x) {
    double s = 0;
    for (int b = 0; b < nblocks; b++) s += partial[(size_t)b * nvals + j];
    out[j] = s;
  }
}

// ---- norm -----------------------------------------------------------------
template <typename R>
__global__ void k_norm(const int4 *__restrict__ a, uint64_t nunits, double *partial) {
  using C = typename Cx<R>::T;
  constexpr int APU = 16 / sizeof(C);
  constexpr int RUN = 8;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double acc = 0;
  for (uint64_t u0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u0 < nunits; u0 += RUN * stride) {
    R run = 0;
#pragma unroll
    for (int j = 0; j < RUN; j++) {
      const uint64_t u = u0 + j * stride;
      if (u < nunits) {
        int4 raw = __ldcs(a + u);
        const C *v = reinterpret_cast<const C *>(&raw);
#pragma unroll
        for (int e = 0; e < APU; e++) run += v[e].x * v[e].x + v[e].y * v[e].y;
      }
    }
    acc += (double)run;
  }
  block_sum_to(acc, partial + blockIdx.x);
}

sv_status launch_norm(sv_state *s, double *out_dev) {
  const uint64_t nunits = ((1ull << s->n) * amp_bytes(s->dt) + 15) / 16;
  double *partial = reinterpret_cast<double *>(s->ws + kWsRed);
  const int g = red_grid(s, nunits / 8 + 1);
  if (s->dt == SV_C64)
    k_norm<float><<<g, kRedThreads, 0, s->stream>>>((const int4 *)s->amps, nunits, partial);
  else
    k_norm<double><<<g, kRedThreads, 0, s->stream>>>((const int4 *)s->amps, nunits, partial);
  k_finalize<<<1, 32, 0, s->stream>>>(partial, g, 1, out_dev);
  g_launches += 2;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

// ---- Pauli-string group expectation --------------------------------------
// For one x_mask: sum_x Re( conj(psi[x ^ xm]) * F(x) * psi[x] ),
// F(x) = sum_t c_t i^{k_t} (-1)^{popcount(x & zm_t)}.
constexpr int kMaxGroupTerms = 64;
// Coefficients are stored in the state's precision: converting FP64 to FP32
// per amplitude would run on the (slow) FP64 pipe.
template <typename R> struct ExpectArgs {
  uint64_t xm;
  int nt;
  uint64_t zm[kMaxGroupTerms];
  R fr[kMaxGroupTerms], fi[kMaxGroupTerms];
};

// Term t's sign at index x is (-1)^{Y_t(x)}, Y_t(x) = parity(x & z_t).  The
// map x -> Y(x) (one bit per term) is linear over GF(2), so Y(x) is the XOR of
// five per-byte tables of x; the group's factor f(x) = sum_t f_t (-1)^{Y_t}
// is the sum of per-byte tables of Y.  A warp sweeps runs of 256 consecutive
// amplitudes: the high bytes of x are fixed over a run, so each amplitude
// costs one x-table lookup and one lookup per 8 terms instead of a parity and
// a select per term.
constexpr int kExpectXBytes = 5;   // n <= 40

template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_expect(const typename Cx<R>::T *__restrict__ a, uint64_t namps,
                                                        const __grid_constant__ ExpectArgs<R> A, double *partial) {
  using C = typename Cx<R>::T;
  __shared__ uint64_t sCol[8 * kExpectXBytes];
  __shared__ uint64_t sT[kExpectXBytes][256];
  __shared__ C sW[kMaxGroupTerms / 8][256];
  const int tid = threadIdx.x;
  // column of qubit q: the terms whose z mask contains q
  for (int q = tid; q < 8 * kExpectXBytes; q += blockDim.x) {
    uint64_t col = 0;
    for (int t = 0; t < A.nt; t++) col |= ((A.zm[t] >> q) & 1ull) << t;
    sCol[q] = col;
  }
  // signed coefficient sums of each byte value of Y (bit set: -f_t, clear: +f_t)
  const int nyb = (A.nt + 7) >> 3;
  for (int e = tid; e < nyb * 256; e += blockDim.x) {
    const int j = e >> 8, v = e & 255;
    R wr = 0, wi = 0;
    for (int b = 0; b < 8; b++) {
      const int t = 8 * j + b;
      if (t >= A.nt) break;
      const R sg = ((v >> b) & 1) ? R(-1) : R(1);
      wr += sg * A.fr[t];
      wi += sg * A.fi[t];
    }
    sW[j][v] = cmake(wr, wi);
  }
  __syncthreads();
  for (int e = tid; e < kExpectXBytes * 256; e += blockDim.x) {
    const int k = e >> 8, v = e & 255;
    uint64_t y = 0;
    for (int b = 0; b < 8; b++)
      if ((v >> b) & 1) y ^= sCol[8 * k + b];
    sT[k][v] = y;
  }
  __syncthreads();

  const int lane = tid & 31;
  const uint64_t nruns = (namps + 255) >> 8;
  const uint64_t wstride = (uint64_t)gridDim.x * (blockDim.x >> 5);
  double acc = 0;
  for (uint64_t run = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (tid >> 5); run < nruns; run += wstride) {
    const uint64_t x0 = run << 8;
    uint64_t yhi = 0;
#pragma unroll
    for (int k = 1; k < kExpectXBytes; k++) yhi ^= sT[k][(x0 >> (8 * k)) & 255];
    R part = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const uint32_t lo = 32 * j + lane;
      const uint64_t x = x0 + lo;
      if (x < namps) {
        const uint64_t y = yhi ^ sT[0][lo];
        R fr = 0, fi = 0;
#pragma unroll
        for (int q = 0; q < kMaxGroupTerms / 8; q++) {
          if (q < nyb) {
            const C w8 = sW[q][(y >> (8 * q)) & 255];
            fr += w8.x;
            fi += w8.y;
          }
        }
        const C v = a[x], w = a[x ^ A.xm];
        // Re(conj(w) * (f * v))
        const R pr = fr * v.x - fi * v.y, pi = fr * v.y + fi * v.x;
        part += w.x * pr + w.y * pi;
      }
    }
    acc += (double)part;
  }
  block_sum_to(acc, partial + blockIdx.x);
}

// ---- diagonal groups (x mask 0) ---------------------------------------------
// E = sum_x |psi_x|^2 f(x), f(x) = sum_t c_t (-1)^{popcount(x & z_t)} (real c_t:
// the imaginary parts cancel for a diagonal group).  A warp sweeps chunks of
// 32 lanes x kDiagTrips 16-byte units; index bits below LB + 5 + log2(trips)
// (unit, lane and trip bits) vary inside a chunk, the bits above are fixed.
// With x = h + l and z_t = (high part, low part L_t):
//   chunk sum = sum_t c_t (-1)^{popcount(h & z_t)} P(L_t),
//   P(L) = sum_l |psi_{h+l}|^2 (-1)^{popcount(l & L)},
// a Walsh coefficient of the chunk's probabilities.  Each lane transforms
// its 2^LB x trips probabilities over the unit and trip bits (the pattern
// bits) in registers and parks the coefficients in shared memory; P(L) is
// the sum over lanes of the lane's coefficient for L's pattern with the sign
// of L's lane bits, so each lane accumulates its signed coefficients and
// the block sums once at the end.  Terms sharing a low part form a group
// whose chunk coefficient sums their high-part signs.  The group loop reads
// the coefficients from shared memory, which keeps the code small (unrolled
// over all patterns it missed the instruction cache).
constexpr int kDiagTrips = 32;
template <typename R> struct DiagArgs {
  uint32_t ng;                              // groups (terms sharing a low part)
  uint32_t gpat[kMaxGroupTerms];            // each group's pattern (unit and trip bits)
  uint32_t lm[kMaxGroupTerms];              // each group's lane mask
  uint32_t tstart[kMaxGroupTerms + 1];      // terms of each group
  uint64_t zm[kMaxGroupTerms];              // terms, ordered by group
  R c[kMaxGroupTerms];
};
constexpr int kDiagThreads = 128;

template <typename R>
__global__ void __launch_bounds__(kDiagThreads) k_expect_diag(const int4 *__restrict__ a, uint64_t nchunks,
                                                              const __grid_constant__ DiagArgs<R> A,
                                                              double *partial) {
  using C = typename Cx<R>::T;
  constexpr int APU = 16 / sizeof(C);
  constexpr int TRIPS = kDiagTrips;
  constexpr int NPAT = APU * TRIPS;
  __shared__ R sq[kDiagThreads / 32][NPAT][32];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  double acc = 0;
  for (uint64_t ch = warp; ch < nchunks; ch += nwarps) {
    const uint64_t ubase = ch * (32 * TRIPS);
    const uint64_t x0 = ubase * APU;
    R q[NPAT];
#pragma unroll
    for (int j = 0; j < TRIPS; j++) {
      int4 raw = __ldcs(a + ubase + j * 32 + lane);
      const C *v = reinterpret_cast<const C *>(&raw);
#pragma unroll
      for (int e = 0; e < APU; e++) q[e + APU * j] = v[e].x * v[e].x + v[e].y * v[e].y;
    }
#pragma unroll
    for (int st = 1; st < NPAT; st <<= 1)
#pragma unroll
      for (int i = 0; i < NPAT; i++)
        if (!(i & st)) {
          const R u = q[i], w = q[i | st];
          q[i] = u + w;
          q[i | st] = u - w;
        }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < NPAT; i++) sq[wi][i][lane] = q[i];
    __syncwarp();
    // two accumulators each, so the sums are not one serial chain
    R part0 = 0, part1 = 0;
    for (uint32_t g = 0; g < A.ng; g++) {
      R ck0 = 0, ck1 = 0;
      uint32_t t = A.tstart[g];
      const uint32_t te = A.tstart[g + 1];
      for (; t + 1 < te; t += 2) {
        ck0 += (__popcll(x0 & A.zm[t]) & 1) ? -A.c[t] : A.c[t];
        ck1 += (__popcll(x0 & A.zm[t + 1]) & 1) ? -A.c[t + 1] : A.c[t + 1];
      }
      if (t < te) ck0 += (__popcll(x0 & A.zm[t]) & 1) ? -A.c[t] : A.c[t];
      const R ck = ck0 + ck1;
      const R qv = sq[wi][A.gpat[g]][lane];
      const R term = (__popc((uint32_t)lane & A.lm[g]) & 1) ? -ck * qv : ck * qv;
      if (g & 1) part1 += term;
      else part0 += term;
    }
    acc += (double)part0 + (double)part1;
  }
  block_sum_to(acc, partial + blockIdx.x);
}

// Launch the diagonal kernel for a group of Z strings; false (nothing
// launched) when the state is smaller than one chunk.
template <typename R>
static bool expect_diag_launch(sv_state *s, const uint64_t *zm, const double *cf, const int *ipow, int nt,
                               double *out_dev, sv_status &st) {
  constexpr int APU = 16 / (2 * (int)sizeof(R));
  constexpr int LB = APU == 2 ? 1 : 0;
  constexpr int TB = 5;   // log2(kDiagTrips)
  constexpr int NPAT = APU * kDiagTrips;
  if (s->n < LB + 5 + TB) return false;
  struct T {
    int pat;
    uint32_t lm;
    uint64_t z;
    double c;
  };
  std::vector<T> ts;
  for (int t = 0; t < nt; t++) {
    const uint64_t lo = zm[t] & ((1ull << (LB + 5 + TB)) - 1);
    const int pat = (int)((lo & ((1u << LB) - 1)) | (((lo >> (LB + 5)) & (kDiagTrips - 1)) << LB));
    const uint32_t lm = (uint32_t)((lo >> LB) & 31);
    const double c = (ipow[t] & 2) ? -cf[t] : cf[t];   // i^k, k even
    ts.push_back({pat, lm, zm[t], c});
  }
  std::stable_sort(ts.begin(), ts.end(), [](const T &x, const T &y) {
    return x.pat != y.pat ? x.pat < y.pat : x.lm < y.lm;
  });
  DiagArgs<R> A{};
  int ng = 0;
  for (int t = 0; t < nt; t++) {
    if (t == 0 || ts[t].pat != ts[t - 1].pat || ts[t].lm != ts[t - 1].lm) {
      A.gpat[ng] = (uint32_t)ts[t].pat;
      A.lm[ng] = ts[t].lm;
      A.tstart[ng] = (uint32_t)t;
      ng++;
    }
    A.zm[t] = ts[t].z;
    A.c[t] = (R)ts[t].c;
  }
  A.tstart[ng] = (uint32_t)nt;
  A.ng = (uint32_t)ng;
  (void)NPAT;
  const uint64_t nchunks = (1ull << s->n) / ((uint64_t)APU * 32 * kDiagTrips);
  double *partial = reinterpret_cast<double *>(s->ws + kWsRed);
  // a warp per chunk, up to eight blocks per SM (the partial-sum area holds them)
  const uint64_t want = (nchunks * 32 + kDiagThreads - 1) / kDiagThreads;
  const int g = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)s->sm_count * 8));
  k_expect_diag<R><<<g, kDiagThreads, 0, s->stream>>>(reinterpret_cast<const int4 *>(s->amps), nchunks, A,
                                                       partial);
  k_finalize<<<1, 32, 0, s->stream>>>(partial, g, 1, out_dev);
  g_launches += 2;
  const cudaError_t e = cudaGetLastError();
  st = e == cudaSuccess ? SV_OK : cuda_error(e, "k_expect_diag");
  return true;
}

template <typename R>
static sv_status expect_launch(sv_state *s, uint64_t xm, const uint64_t *zm, const double *cf, const int *ipow,
                               int nt, double *out_dev) {
  if (xm == 0) {
    bool odd = false;   // an odd power of i would make a term imaginary
    for (int t = 0; t < nt; t++) odd |= (ipow[t] & 1) != 0;
    sv_status st = SV_OK;
    if (!odd && expect_diag_launch<R>(s, zm, cf, ipow, nt, out_dev, st)) return st;
  }
  ExpectArgs<R> A{};
  A.xm = xm;
  A.nt = nt;
  for (int t = 0; t < nt; t++) {
    A.zm[t] = zm[t];
    switch (ipow[t] & 3) {
      case 0: A.fr[t] = (R)cf[t]; break;
      case 1: A.fi[t] = (R)cf[t]; break;
      case 2: A.fr[t] = (R)-cf[t]; break;
      default: A.fi[t] = (R)-cf[t]; break;
    }
  }
  const uint64_t na = 1ull << s->n;
  double *partial = reinterpret_cast<double *>(s->ws + kWsRed);
  const int g = red_grid(s, na / 64 + 1);
  k_expect<R><<<g, kRedThreads, 0, s->stream>>>(reinterpret_cast<const typename Cx<R>::T *>(s->amps), na, A,
                                                partial);
  k_finalize<<<1, 32, 0, s->stream>>>(partial, g, 1, out_dev);
  g_launches += 2;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

sv_status launch_expect_group(sv_state *s, uint64_t xm, const uint64_t *zm, const double *cf,
                              const int *ipow, int nt, double *out_dev) {
  if (nt > kMaxGroupTerms) return set_error(SV_EINVAL, "too many terms in one group");
  return s->dt == SV_C64 ? expect_launch<float>(s, xm, zm, cf, ipow, nt, out_dev)
                         : expect_launch<double>(s, xm, zm, cf, ipow, nt, out_dev);
}

// ---- <Z_q> for every qubit in one pass -----------------------------------
// A warp sweeps chunks of 8 x 32 16-byte units.  Index bits inside a unit,
// the 5 lane bits and the 3 trip bits are resolved with FP32 warp sums; the
// bits above are constant over a chunk.  Lane q keeps the FP64 running sum
// S_q = sum over amplitudes with bit q set (lanes 0..31 and, for n > 32,
// a second register for q + 32).  <Z_q> = total - 2 S_q.
template <typename R>
__global__ void k_zall(const int4 *__restrict__ a, int n, uint64_t nchunks, double *partial) {
  using C = typename Cx<R>::T;
  constexpr int APU = 16 / sizeof(C);
  constexpr int LB = APU == 2 ? 1 : 0;  // index bits inside a unit
  constexpr int TRIPS = 8;
  const int lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  double S0 = 0, S1 = 0, T = 0;
  for (uint64_t ch = warp; ch < nchunks; ch += nwarps) {
    const uint64_t ubase = ch * (32 * TRIPS);
    R tot = 0, b0 = 0, bj[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < TRIPS; j++) {
      int4 raw = __ldcs(a + ubase + j * 32 + lane);
      const C *v = reinterpret_cast<const C *>(&raw);
      R ps = 0;
#pragma unroll
      for (int e = 0; e < APU; e++) {
        const R p = v[e].x * v[e].x + v[e].y * v[e].y;
        ps += p;
        if (LB == 1 && e == 1) b0 += p;
      }
      tot += ps;
#pragma unroll
      for (int b = 0; b < 3; b++)
        if ((j >> b) & 1) bj[b] += ps;
    }
    // warp-level sums
    R lanebit[5];
#pragma unroll
    for (int b = 0; b < 5; b++) lanebit[b] = warp_sum(((lane >> b) & 1) ? tot : R(0));
    const R wtot = warp_sum(tot);
    const R wb0 = LB ? warp_sum(b0) : R(0);
    R wbj[3];
#pragma unroll
    for (int b = 0; b < 3; b++) wbj[b] = warp_sum(bj[b]);
    const uint64_t abase = ubase * APU;  // first amplitude index of the chunk
    auto bitsum = [&](int q) -> R {
      if (q < LB) return wb0;
      if (q < LB + 5) return lanebit[q - LB];
      if (q < LB + 8) return wbj[q - LB - 5];
      return ((abase >> q) & 1) ? wtot : R(0);
    };
    if (lane < n) S0 += (double)bitsum(lane);
    if (lane + 32 < n) S1 += (double)bitsum(lane + 32);
    T += (double)wtot;
  }
  // block reduction: partial[block][q] for q < n, partial[block][n] = total
  __shared__ double sm[64 + 1];
  for (int i = threadIdx.x; i < 65; i += blockDim.x) sm[i] = 0;
  __syncthreads();
  if (lane < n) atomicAdd(&sm[lane], S0);
  if (lane + 32 < n) atomicAdd(&sm[lane + 32], S1);
  if (lane == 0) atomicAdd(&sm[64], T);
  __syncthreads();
  for (int q = threadIdx.x; q <= n; q += blockDim.x)
    partial[(size_t)blockIdx.x * (n + 1) + q] = q < n ? sm[q] : sm[64];
}

// small states: one thread per amplitude, FP64 per bit
template <typename R>
__global__ void k_zall_small(const typename Cx<R>::T *__restrict__ a, int n, double *out) {
  __shared__ double sm[65];
  for (int i = threadIdx.x; i < 65; i += blockDim.x) sm[i] = 0;
  __syncthreads();
  for (uint64_t x = threadIdx.x; x < (1ull << n); x += blockDim.x) {
    const double p = (double)a[x].x * a[x].x + (double)a[x].y * a[x].y;
    for (int q = 0; q < n; q++)
      if ((x >> q) & 1) atomicAdd(&sm[q], p);
    atomicAdd(&sm[64], p);
  }
  __syncthreads();
  for (int q = threadIdx.x; q <= n; q += blockDim.x) out[q] = q < n ? sm[q] : sm[64];
}

// z[q] = total - 2 S_q from the reduced S_q (in place: buf[0..n] -> z[0..n-1])
__global__ void k_zall_finish(const double *__restrict__ partial, int nblocks, int n, double *out) {
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double t = 0;
    for (int b = 0; b < nblocks; b++) t += partial[(size_t)b * (n + 1) + n];
    tot = t;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    double s = 0;
    for (int b = 0; b < nblocks; b++) s += partial[(size_t)b * (n + 1) + q];
    out[q] = tot - 2.0 * s;
  }
}

sv_status launch_z_all(sv_state *s, double *out_dev) {
  double *partial = reinterpret_cast<double *>(s->ws + kWsRed);
  const int apu = s->dt == SV_C64 ? 2 : 1;
  const uint64_t namps = 1ull << s->n;
  const uint64_t chunk_amps = 32ull * 8 * apu;
  if (namps < chunk_amps) {
    if (s->dt == SV_C64)
      k_zall_small<float><<<1, 256, 0, s->stream>>>((const float2 *)s->amps, s->n, partial);
    else
      k_zall_small<double><<<1, 256, 0, s->stream>>>((const double2 *)s->amps, s->n, partial);
    k_zall_finish<<<1, 64, 0, s->stream>>>(partial, 1, s->n, out_dev);
  } else {
    const uint64_t nchunks = namps / chunk_amps;
    const uint64_t warps_per_block = kRedThreads / 32;
    const int g = (int)std::max<uint64_t>(
        1, std::min<uint64_t>((nchunks + warps_per_block - 1) / warps_per_block, (uint64_t)s->sm_count * 4));
    if (s->dt == SV_C64)
      k_zall<float><<<g, kRedThreads, 0, s->stream>>>((const int4 *)s->amps, s->n, nchunks, partial);
    else
      k_zall<double><<<g, kRedThreads, 0, s->stream>>>((const int4 *)s->amps, s->n, nchunks, partial);
    k_zall_finish<<<1, 64, 0, s->stream>>>(partial, g, s->n, out_dev);
  }
  g_launches += 2;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

// ---- <Z_q> without any allocation ------------------------------------------
// Callers that cannot allocate device memory (code running while a CUDA graph
// is being captured, hosts whose device allocator belongs to someone else,
// latency-critical loops where an allocation's implicit synchronisation is
// not allowed) use sv_expect_z_all_noalloc.  Its per-block partial sums live
// in the fixed array below, which every GPU that loads this library keeps
// for the life of the process: kNoAllocBlocks blocks x (kNoAllocMaxQ + 1)
// doubles = 143,360 bytes.
constexpr int kNoAllocBlocks = 512;
constexpr int kNoAllocMaxQ = 34;
static __device__ __align__(256) double g_zall_scratch[kNoAllocBlocks * (kNoAllocMaxQ + 1)];
struct NoAllocDev {
  double *scratch = nullptr;   // device address of g_zall_scratch on this device
  int sms = 0;
};
static NoAllocDev g_noalloc_dev[64];
static std::mutex g_noalloc_mu;

sv_status zall_noalloc(const void *amps, int n, sv_dtype dt, double *out, cudaStream_t stream) {
  int dev = 0;
  SV_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(SV_EUNSUPPORTED, "device ordinal above 63");
  NoAllocDev d;
  {
    // once per device, under a lock (host threads may call concurrently):
    // the array's name is only a host-side handle, so ask the runtime for
    // its address on the current device; the SM count sizes the grid
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_dev[dev].scratch) {
      void *p = nullptr;
      int sms = 0;
      SV_CUDA(cudaGetSymbolAddress(&p, g_zall_scratch));
      SV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      g_noalloc_dev[dev].sms = sms;
      g_noalloc_dev[dev].scratch = static_cast<double *>(p);
    }
    d = g_noalloc_dev[dev];
  }
  double *partial = d.scratch;
  const int sms = d.sms;
  const int apu = dt == SV_C64 ? 2 : 1;
  const uint64_t namps = 1ull << n;
  const uint64_t chunk_amps = 32ull * 8 * apu;
  if (namps < chunk_amps) {
    if (dt == SV_C64)
      k_zall_small<float><<<1, 256, 0, stream>>>((const float2 *)amps, n, partial);
    else
      k_zall_small<double><<<1, 256, 0, stream>>>((const double2 *)amps, n, partial);
    k_zall_finish<<<1, 64, 0, stream>>>(partial, 1, n, out);
  } else {
    const uint64_t nchunks = namps / chunk_amps;
    const uint64_t wpb = kRedThreads / 32;
    const uint64_t cap = std::min<uint64_t>((uint64_t)kNoAllocBlocks, (uint64_t)sms * 4);
    const int g = (int)std::max<uint64_t>(1, std::min<uint64_t>((nchunks + wpb - 1) / wpb, cap));
    // every block writes all n + 1 of its partial sums, so nothing needs zeroing
    if (dt == SV_C64)
      k_zall<float><<<g, kRedThreads, 0, stream>>>((const int4 *)amps, n, nchunks, partial);
    else
      k_zall<double><<<g, kRedThreads, 0, stream>>>((const int4 *)amps, n, nchunks, partial);
    k_zall_finish<<<1, 64, 0, stream>>>(partial, g, n, out);
  }
  g_launches += 2;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

// ---- sampling --------------------------------------------------------------
constexpr int kChunkBits = 10;  // 1024 amplitudes per CDF chunk

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t j) {
  // the j-th output of SplitMix64 seeded with `seed` (Steele, Lea, Flood 2014)
  uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename R>
__device__ __forceinline__ double prob64(const typename Cx<R>::T v) {
  const double re = (double)v.x, im = (double)v.y;
  return re * re + im * im;
}

// chunk sums of |psi|^2: one warp per chunk; products and runs of 8
// amplitudes per lane in the state's precision, FP64 above that (the shot
// search recomputes the FP64 prefix inside the chosen chunk, so a chunk total
// that is off in its last bits only matters for a draw within ~1e-12 of a
// chunk boundary)
template <typename R>
__global__ void k_chunk_sums(const typename Cx<R>::T *__restrict__ a, int n, uint64_t nchunks,
                             double *csum) {
  using C = typename Cx<R>::T;
  const uint64_t camps = 1ull << (n < kChunkBits ? n : kChunkBits);
  const int lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t c = warp; c < nchunks; c += nwarps) {
    const C *ac = a + c * camps;
    double acc = 0;
    for (uint64_t i0 = 0; i0 < camps; i0 += 256) {
      R run = 0;
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const uint64_t i = i0 + 32 * j + lane;
        if (i < camps) {
          const C v = ac[i];
          run = fma(v.x, v.x, fma(v.y, v.y, run));
        }
      }
      acc += (double)run;
    }
    acc = warp_sum(acc);
    if (lane == 0) csum[c] = acc;
  }
}

// Inclusive FP64 prefix sums of the chunk totals, coalesced: k_scan_seg
// scans segments of kScanSeg values in place (warp shuffles, then the warps'
// totals) and writes each segment's total; the totals are scanned the same
// way, level by level, and k_scan_add adds segment b's offset (the scanned
// total of segments 0..b-1) to its values.
constexpr int kScanSeg = 1024;
__global__ void __launch_bounds__(kScanSeg) k_scan_seg(double *x, uint64_t len, double *tops) {
  __shared__ double wsum[kScanSeg / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t i = (uint64_t)blockIdx.x * kScanSeg + threadIdx.x;
  double v = i < len ? x[i] : 0.0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) wsum[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    wsum[lane] = t;
  }
  __syncthreads();
  if (w > 0) v += wsum[w - 1];
  if (i < len) x[i] = v;
  if (tops && threadIdx.x == kScanSeg - 1) tops[blockIdx.x] = v;
}
__global__ void __launch_bounds__(kScanSeg) k_scan_add(double *x, uint64_t len, const double *tops) {
  const uint64_t b = (uint64_t)blockIdx.x + 1;   // segment 0 has no offset
  const uint64_t i = b * kScanSeg + threadIdx.x;
  if (i < len) x[i] += tops[b - 1];
}
// scan x[0, len); tops: scratch for the segment totals of every level
static void scan_levels(double *x, uint64_t len, double *tops, cudaStream_t st) {
  if (len <= (uint64_t)kScanSeg) {
    k_scan_seg<<<1, kScanSeg, 0, st>>>(x, len, nullptr);
    g_launches++;
    return;
  }
  const uint64_t nseg = (len + kScanSeg - 1) / kScanSeg;
  k_scan_seg<<<(unsigned)nseg, kScanSeg, 0, st>>>(x, len, tops);
  scan_levels(tops, nseg, tops + ((nseg + 31) & ~(uint64_t)31), st);
  k_scan_add<<<(unsigned)(nseg - 1), kScanSeg, 0, st>>>(x, len, tops);
  g_launches += 2;
}
size_t scan_scratch_bytes(int n) {
  const int cb = n < 10 ? n : 10;
  uint64_t len = 1ull << (n - cb), total = 0;
  while (len > (uint64_t)kScanSeg) {
    len = (len + kScanSeg - 1) / kScanSeg;
    total += (len + 31) & ~(uint64_t)31;
  }
  return (size_t)total * sizeof(double);
}

// one warp per shot: binary search over chunk prefixes, then a warp scan
// inside the chunk.  Shot j of this launch is global shot shot0 + j.
template <typename R>
__global__ void k_sample(const typename Cx<R>::T *__restrict__ a, int n, const double *__restrict__ pref,
                         uint64_t nchunks, int64_t shot0, int64_t shots, uint64_t seed, uint64_t *out) {
  const int lane = threadIdx.x & 31;
  const uint64_t camps = 1ull << (n < kChunkBits ? n : kChunkBits);
  const double total = pref[nchunks - 1];
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t sh = warp; sh < (uint64_t)shots; sh += nwarps) {
    const double u = (double)(splitmix64(seed, (uint64_t)shot0 + sh) >> 11) * 0x1.0p-53;
    const double target = u * total;
    // smallest chunk c with pref[c] > target
    uint64_t lo = 0, hi = nchunks - 1;
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if (pref[mid] > target) hi = mid; else lo = mid + 1;
    }
    const uint64_t c = lo;
    double run = c > 0 ? pref[c - 1] : 0.0;
    uint64_t ans = c * camps + camps - 1;
    for (uint64_t i0 = 0; i0 < camps; i0 += 32) {
      const uint64_t x = c * camps + i0 + lane;
      double p = (i0 + lane < camps) ? prob64<R>(a[x]) : 0.0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, p, o);
        if (lane >= o) p += t;
      }
      const unsigned hit = __ballot_sync(0xffffffffu, (run + p > target) && (i0 + lane < camps));
      if (hit) {
        ans = c * camps + i0 + (__ffs(hit) - 1);
        break;
      }
      run += __shfl_sync(0xffffffffu, p, 31);
    }
    if (lane == 0) out[sh] = ans;
  }
}

static uint64_t n_chunks(int n) { return 1ull << (n - (n < kChunkBits ? n : kChunkBits)); }
size_t sample_shot_offset(int n) { return (n_chunks(n) * sizeof(double) + 255) & ~(size_t)255; }
int64_t sample_shot_capacity() { return (1 << 20) / sizeof(uint64_t); }

sv_status launch_sample_prepare(sv_state *s) {
  const uint64_t nchunks = n_chunks(s->n);
  double *csum = reinterpret_cast<double *>(s->ws + kWsRed);
  const int g = (int)std::min<uint64_t>(nchunks, (uint64_t)s->sm_count * 8);
  if (s->dt == SV_C64)
    k_chunk_sums<float><<<g, kRedThreads, 0, s->stream>>>((const float2 *)s->amps, s->n, nchunks, csum);
  else
    k_chunk_sums<double><<<g, kRedThreads, 0, s->stream>>>((const double2 *)s->amps, s->n, nchunks, csum);
  g_launches++;
  // the scan's scratch follows the shot buffer
  scan_levels(csum, nchunks,
              reinterpret_cast<double *>(s->ws + kWsRed + sample_shot_offset(s->n) +
                                         sample_shot_capacity() * sizeof(uint64_t)),
              s->stream);
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

sv_status launch_sample_shots(sv_state *s, int64_t shot0, int64_t count, uint64_t seed, uint64_t *out_dev) {
  const uint64_t nchunks = n_chunks(s->n);
  const double *csum = reinterpret_cast<const double *>(s->ws + kWsRed);
  const int sg = (int)std::max<int64_t>(1, std::min<int64_t>((count + 7) / 8, (int64_t)s->sm_count * 16));
  if (s->dt == SV_C64)
    k_sample<float><<<sg, 256, 0, s->stream>>>((const float2 *)s->amps, s->n, csum, nchunks, shot0, count,
                                               seed, out_dev);
  else
    k_sample<double><<<sg, 256, 0, s->stream>>>((const double2 *)s->amps, s->n, csum, nchunks, shot0, count,
                                                seed, out_dev);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

}  // namespace sv
