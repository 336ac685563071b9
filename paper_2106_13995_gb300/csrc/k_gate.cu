// K1-K5: single-gate global-memory passes.
//
// Each kernel streams the state once (read + write 2 * 2^n * bytes/amp):
//   K1  1q gate on qubit 0, complex64: both amplitudes of a pair sit in one
//       16-byte float4, updated in registers;
//   K2  1q gate on a low qubit: the partner amplitude lives in another lane
//       of the same warp and is exchanged with __shfl_xor_sync, so every load
//       and store is a fully coalesced 16-byte access;
//   K3  1q gate on a high qubit: each thread loads 16 bytes at i0 and at
//       i0 | 2^q, two independent coalesced streams;
//   K4  controlled dense gates (only the 2^{n-c} amplitudes whose control
//       bits are 1 are visited) and diagonal gates (elementwise phases);
//   K5  dense k-qubit gates, k <= 6: gather 2^k amplitudes, multiply,
//       scatter.
// Permutation gates (X, CNOT, Toffoli, SWAP) multiply by exact 0/1 entries,
// so they move amplitudes bit-exactly.
#include <algorithm>

#include "sv_device.cuh"
#include "sv_internal.h"

namespace sv {

template <typename R> struct M1 { typename Cx<R>::T u[4]; };

static int grid_for(sv_state *s, uint64_t work, int threads) {
  const uint64_t want = (work + threads - 1) / threads;
  const uint64_t cap = (uint64_t)s->sm_count * 8;
  return (int)std::max<uint64_t>(1, std::min(want, cap));
}

// ---- K1: complex64, target 0 --------------------------------------------
__global__ void k_1q_q0_c64(float4 *__restrict__ a, uint64_t nunits, M1<float> U) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nunits; u += stride) {
    const float4 x = __ldcs(a + u);
    const float2 a0 = make_float2(x.x, x.y), a1 = make_float2(x.z, x.w);
    const float2 o0 = cfma(U.u[1], a1, cmul(U.u[0], a0));
    const float2 o1 = cfma(U.u[3], a1, cmul(U.u[2], a0));
    __stcs(a + u, make_float4(o0.x, o0.y, o1.x, o1.y));
  }
}

// ---- K2: low target via warp shuffles -----------------------------------
// complex64: lane holds amplitudes 2u, 2u+1 (one float4); target q in 1..5,
// partner lane = lane ^ 2^(q-1).  complex128: lane holds amplitude u; target
// q in 0..4, partner lane = lane ^ 2^q.
__global__ void k_1q_shfl_c64(float4 *__restrict__ a, uint64_t nunits, int q, M1<float> U) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const int lm = 1 << (q - 1);
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nunits; u += stride) {
    const float4 x = __ldcs(a + u);
    float4 y;
    y.x = __shfl_xor_sync(0xffffffffu, x.x, lm);
    y.y = __shfl_xor_sync(0xffffffffu, x.y, lm);
    y.z = __shfl_xor_sync(0xffffffffu, x.z, lm);
    y.w = __shfl_xor_sync(0xffffffffu, x.w, lm);
    const bool one = (u >> (q - 1)) & 1;  // this lane's amplitudes have bit q = 1
    const float2 m0 = make_float2(x.x, x.y), m1 = make_float2(x.z, x.w);
    const float2 p0 = make_float2(y.x, y.y), p1 = make_float2(y.z, y.w);
    float2 o0, o1;
    if (!one) {
      o0 = cfma(U.u[1], p0, cmul(U.u[0], m0));
      o1 = cfma(U.u[1], p1, cmul(U.u[0], m1));
    } else {
      o0 = cfma(U.u[3], m0, cmul(U.u[2], p0));
      o1 = cfma(U.u[3], m1, cmul(U.u[2], p1));
    }
    __stcs(a + u, make_float4(o0.x, o0.y, o1.x, o1.y));
  }
}

__global__ void k_1q_shfl_c128(double2 *__restrict__ a, uint64_t namps, int q, M1<double> U) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const int lm = 1 << q;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < namps; i += stride) {
    const double2 x = __ldcs(a + i);
    double2 y;
    y.x = __shfl_xor_sync(0xffffffffu, x.x, lm);
    y.y = __shfl_xor_sync(0xffffffffu, x.y, lm);
    const bool one = (i >> q) & 1;
    const double2 o = one ? cfma(U.u[3], x, cmul(U.u[2], y)) : cfma(U.u[1], y, cmul(U.u[0], x));
    __stcs(a + i, o);
  }
}

// ---- K3: high target -----------------------------------------------------
// complex64: unit u covers amplitudes {i0, i0+1} and {i0 + 2^q, i0 + 2^q + 1},
// i0 = ins0(2u, q), q >= 1.  Four units per thread per trip keep 128 bytes
// in flight per thread.
__global__ void k_1q_hi_c64(float2 *__restrict__ a, uint64_t nunits, int q, M1<float> U) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t hb = 1ull << q;
  constexpr int UN = 4;
  for (uint64_t u0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u0 < nunits; u0 += UN * stride) {
    float4 x0[UN], x1[UN];
    uint64_t i0[UN];
#pragma unroll
    for (int j = 0; j < UN; j++) {
      const uint64_t u = u0 + j * stride;
      i0[j] = ins0(2 * u, q);
      if (u < nunits) {
        x0[j] = __ldcs(reinterpret_cast<const float4 *>(a + i0[j]));
        x1[j] = __ldcs(reinterpret_cast<const float4 *>(a + (i0[j] | hb)));
      }
    }
#pragma unroll
    for (int j = 0; j < UN; j++) {
      if (u0 + j * stride >= nunits) break;
      const float2 a0 = make_float2(x0[j].x, x0[j].y), b0 = make_float2(x0[j].z, x0[j].w);
      const float2 a1 = make_float2(x1[j].x, x1[j].y), b1 = make_float2(x1[j].z, x1[j].w);
      const float2 ya0 = cfma(U.u[1], a1, cmul(U.u[0], a0)), yb0 = cfma(U.u[1], b1, cmul(U.u[0], b0));
      const float2 ya1 = cfma(U.u[3], a1, cmul(U.u[2], a0)), yb1 = cfma(U.u[3], b1, cmul(U.u[2], b0));
      __stcs(reinterpret_cast<float4 *>(a + i0[j]), make_float4(ya0.x, ya0.y, yb0.x, yb0.y));
      __stcs(reinterpret_cast<float4 *>(a + (i0[j] | hb)), make_float4(ya1.x, ya1.y, yb1.x, yb1.y));
    }
  }
}

__global__ void k_1q_hi_c128(double2 *__restrict__ a, uint64_t npairs, int q, M1<double> U) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t hb = 1ull << q;
  constexpr int UN = 4;
  for (uint64_t u0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u0 < npairs; u0 += UN * stride) {
    double2 x0[UN], x1[UN];
    uint64_t i0[UN];
#pragma unroll
    for (int j = 0; j < UN; j++) {
      const uint64_t u = u0 + j * stride;
      i0[j] = ins0(u, q);
      if (u < npairs) {
        x0[j] = __ldcs(a + i0[j]);
        x1[j] = __ldcs(a + (i0[j] | hb));
      }
    }
#pragma unroll
    for (int j = 0; j < UN; j++) {
      if (u0 + j * stride >= npairs) break;
      __stcs(a + i0[j], cfma(U.u[1], x1[j], cmul(U.u[0], x0[j])));
      __stcs(a + (i0[j] | hb), cfma(U.u[3], x1[j], cmul(U.u[2], x0[j])));
    }
  }
}

// ---- K4/K5: dense k-qubit gate with controls -----------------------------
template <typename R, int K> struct DenseArgs {
  uint64_t off[1 << K];                 // index offset of local basis state y
  typename Cx<R>::T u[K <= 3 ? (1 << (2 * K)) : 1];   // matrix (k <= 3)
  const typename Cx<R>::T *ug;          // matrix in device memory (k >= 4)
};

template <typename R, int K>
__global__ void k_dense(typename Cx<R>::T *__restrict__ a, uint64_t ngroups, uint64_t fixed,
                        uint64_t cmask, const __grid_constant__ DenseArgs<R, K> A) {
  using C = typename Cx<R>::T;
  constexpr int D = 1 << K;
  const C *U = K <= 3 ? A.u : A.ug;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
    const uint64_t i0 = ins0_mask64(g, fixed) | cmask;
    C x[D];
#pragma unroll
    for (int y = 0; y < D; y++) x[y] = a[i0 + A.off[y]];
#pragma unroll (K <= 3 ? D : 1)
    for (int r = 0; r < D; r++) {
      C acc = czero<C>();
#pragma unroll
      for (int y = 0; y < D; y++) acc = cfma(U[r * D + y], x[y], acc);
      a[i0 + A.off[r]] = acc;
    }
  }
}

// ---- K4: diagonal gate (targets and controls folded into one table) ------
template <typename R> struct DiagArgs {
  int npos;
  int pos[14];                  // qubit of table bit j
  typename Cx<R>::T d[256];     // 2^npos entries, 1 where controls are not all set
};

template <typename R>
__global__ void k_diag(typename Cx<R>::T *__restrict__ a, uint64_t namps, const __grid_constant__ DiagArgs<R> A) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < namps; x += stride) {
    uint32_t r = 0;
    for (int j = 0; j < A.npos; j++) r |= (uint32_t)((x >> A.pos[j]) & 1ull) << j;
    a[x] = cmul(A.d[r], a[x]);
  }
}

// ---------------------------------------------------------------------------
template <typename R>
static M1<R> pack1(const std::vector<cd> &U) {
  M1<R> m;
  for (int e = 0; e < 4; e++) {
    m.u[e].x = (R)U[e].real();
    m.u[e].y = (R)U[e].imag();
  }
  return m;
}

template <typename R, int K>
static sv_status dense_k(sv_state *s, const std::vector<int> &t, const std::vector<int> &c,
                         const std::vector<cd> &U) {
  constexpr int D = 1 << K;
  DenseArgs<R, K> A{};
  uint64_t fixed = 0, cmask = 0;
  for (int y = 0; y < D; y++) {
    uint64_t o = 0;
    for (int j = 0; j < K; j++) o |= (uint64_t)((y >> j) & 1) << t[j];
    A.off[y] = o;
  }
  fixed = A.off[D - 1];
  for (int q : c) cmask |= 1ull << q;
  fixed |= cmask;
  if (K <= 3) {
    for (int e = 0; e < D * D; e++) {
      A.u[e].x = (R)U[e].real();
      A.u[e].y = (R)U[e].imag();
    }
    A.ug = nullptr;
  } else {
    // stage the matrix into the workspace gate-matrix scratch
    const size_t bytes = (size_t)D * D * 2 * sizeof(R);
    SV_CUDA(cudaEventSynchronize(s->staged));
    R *h = reinterpret_cast<R *>(s->pinned);
    for (int e = 0; e < D * D; e++) {
      h[2 * e] = (R)U[e].real();
      h[2 * e + 1] = (R)U[e].imag();
    }
    void *dst = s->ws + kWsGateMat;
    SV_CUDA(cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, s->stream));
    SV_CUDA(cudaEventRecord(s->staged, s->stream));
    A.ug = reinterpret_cast<const typename Cx<R>::T *>(dst);
  }
  const uint64_t ngroups = 1ull << (s->n - __builtin_popcountll(fixed));
  const int threads = 256;
  k_dense<R, K><<<grid_for(s, ngroups, threads), threads, 0, s->stream>>>(
      reinterpret_cast<typename Cx<R>::T *>(s->amps), ngroups, fixed, cmask, A);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

template <typename R>
static sv_status dense_any(sv_state *s, const std::vector<int> &t, const std::vector<int> &c,
                           const std::vector<cd> &U) {
  switch (t.size()) {
    case 1: return dense_k<R, 1>(s, t, c, U);
    case 2: return dense_k<R, 2>(s, t, c, U);
    case 3: return dense_k<R, 3>(s, t, c, U);
    case 4: return dense_k<R, 4>(s, t, c, U);
    case 5: return dense_k<R, 5>(s, t, c, U);
    case 6: return dense_k<R, 6>(s, t, c, U);
    default: return set_error(SV_EINVAL, "gate must have 1..6 targets");
  }
}

sv_status launch_dense_gate(sv_state *s, const std::vector<int> &t, const std::vector<int> &c,
                            const std::vector<cd> &U) {
  const int threads = 256;
  // uncontrolled single-qubit gates take the specialised streaming kernels
  if (t.size() == 1 && c.empty()) {
    const int q = t[0];
    if (s->dt == SV_C64 && s->n >= 6) {
      const M1<float> m = pack1<float>(U);
      float4 *a4 = reinterpret_cast<float4 *>(s->amps);
      const uint64_t nunits = 1ull << (s->n - 1);
      if (q == 0) {
        k_1q_q0_c64<<<grid_for(s, nunits, threads), threads, 0, s->stream>>>(a4, nunits, m);
      } else if (q <= 5) {
        k_1q_shfl_c64<<<grid_for(s, nunits, threads), threads, 0, s->stream>>>(a4, nunits, q, m);
      } else {
        const uint64_t np = 1ull << (s->n - 2);
        k_1q_hi_c64<<<grid_for(s, np / 4, threads), threads, 0, s->stream>>>(
            reinterpret_cast<float2 *>(s->amps), np, q, m);
      }
      g_launches++;
      SV_CUDA(cudaGetLastError());
      return SV_OK;
    }
    if (s->dt == SV_C128 && s->n >= 5) {
      const M1<double> m = pack1<double>(U);
      double2 *a2 = reinterpret_cast<double2 *>(s->amps);
      if (q <= 4) {
        const uint64_t na = 1ull << s->n;
        k_1q_shfl_c128<<<grid_for(s, na, threads), threads, 0, s->stream>>>(a2, na, q, m);
      } else {
        const uint64_t np = 1ull << (s->n - 1);
        k_1q_hi_c128<<<grid_for(s, np / 4, threads), threads, 0, s->stream>>>(a2, np, q, m);
      }
      g_launches++;
      SV_CUDA(cudaGetLastError());
      return SV_OK;
    }
  }
  return s->dt == SV_C64 ? dense_any<float>(s, t, c, U) : dense_any<double>(s, t, c, U);
}

template <typename R>
static sv_status diag_launch(sv_state *s, const std::vector<int> &t, const std::vector<int> &c,
                             const std::vector<cd> &d) {
  DiagArgs<R> A{};
  const int k = (int)t.size(), nc = (int)c.size();
  A.npos = k + nc;
  if (A.npos > 8) return set_error(SV_EUNSUPPORTED, "diagonal gate with more than 8 qubits");
  for (int j = 0; j < k; j++) A.pos[j] = t[j];
  for (int j = 0; j < nc; j++) A.pos[k + j] = c[j];
  const int cm = ((1 << nc) - 1) << k;
  for (int r = 0; r < (1 << A.npos); r++) {
    cd v = ((r & cm) == cm) ? d[r & ((1 << k) - 1)] : cd(1.0);
    A.d[r].x = (R)v.real();
    A.d[r].y = (R)v.imag();
  }
  const uint64_t na = 1ull << s->n;
  const int threads = 256;
  k_diag<R><<<grid_for(s, na, threads), threads, 0, s->stream>>>(
      reinterpret_cast<typename Cx<R>::T *>(s->amps), na, A);
  g_launches++;
  SV_CUDA(cudaGetLastError());
  return SV_OK;
}

sv_status launch_diag_gate(sv_state *s, const std::vector<int> &t, const std::vector<int> &c,
                           const std::vector<cd> &d) {
  return s->dt == SV_C64 ? diag_launch<float>(s, t, c, d) : diag_launch<double>(s, t, c, d);
}

}  // namespace sv
