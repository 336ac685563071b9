// C ABI: expectations, norms and sampling (host orchestration of K8-K10).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "sv_internal.h"

using namespace sv;

static double *scalars_dev(sv_state *s) { return reinterpret_cast<double *>(s->ws + kWsCtrl + kWsScalars); }
static double *scalars_host(sv_state *s) { return reinterpret_cast<double *>(s->pinned + kWsProgBytes); }
constexpr int kMaxSlots = 256;  // 2 KB of FP64 result slots

static sv_status fetch(sv_state *s, int count) {
  SV_CUDA(cudaMemcpyAsync(scalars_host(s), scalars_dev(s), sizeof(double) * count, cudaMemcpyDeviceToHost,
                          s->stream));
  SV_CUDA(cudaStreamSynchronize(s->stream));
  return SV_OK;
}

static sv_status check_terms(const sv_state *s, const sv_pauli_term *terms, int nt) {
  if (nt < 0 || (nt > 0 && !terms)) return set_error(SV_EINVAL, "bad term list");
  const uint64_t lim = s->n >= 64 ? ~0ull : ((1ull << s->n) - 1);
  for (int t = 0; t < nt; t++)
    if ((terms[t].x_mask & ~lim) || (terms[t].z_mask & ~lim))
      return set_error(SV_EINVAL, "Pauli mask references a qubit >= n");
  return SV_OK;
}

extern "C" {

sv_status sv_expect(sv_state *s, const sv_pauli_term *terms, int nt, double *out) {
  if (!s || !out) return set_error(SV_EINVAL, "null argument");
  SV_TRY(check_terms(s, terms, nt));
  // group by x mask: each group is one read pass
  std::map<uint64_t, std::vector<int>> groups;
  for (int t = 0; t < nt; t++) groups[terms[t].x_mask].push_back(t);
  std::vector<std::vector<int>> chunks;
  for (auto &g : groups)
    for (size_t i = 0; i < g.second.size(); i += 64)
      chunks.emplace_back(g.second.begin() + i, g.second.begin() + std::min(g.second.size(), i + 64));
  double total = 0;
  for (size_t c0 = 0; c0 < chunks.size(); c0 += kMaxSlots) {
    const size_t c1 = std::min(chunks.size(), c0 + kMaxSlots);
    for (size_t c = c0; c < c1; c++) {
      std::vector<uint64_t> zm;
      std::vector<double> cf;
      std::vector<int> ip;
      for (int t : chunks[c]) {
        zm.push_back(terms[t].z_mask);
        cf.push_back(terms[t].coeff);
        ip.push_back(__builtin_popcountll(terms[t].x_mask & terms[t].z_mask) & 3);
      }
      SV_TRY(launch_expect_group(s, terms[chunks[c][0]].x_mask, zm.data(), cf.data(), ip.data(),
                                 (int)zm.size(), scalars_dev(s) + (c - c0)));
    }
    SV_TRY(fetch(s, (int)(c1 - c0)));
    for (size_t c = c0; c < c1; c++) total += scalars_host(s)[c - c0];
  }
  *out = total;
  return SV_OK;
}

sv_status sv_expect_z_all(sv_state *s, double *out) {
  if (!s || !out) return set_error(SV_EINVAL, "null argument");
  SV_TRY(launch_z_all(s, scalars_dev(s)));
  SV_TRY(fetch(s, s->n));
  std::memcpy(out, scalars_host(s), sizeof(double) * s->n);
  return SV_OK;
}

sv_status sv_expect_z_all_noalloc(const void *amps_dev, int n_qubits, sv_dtype dtype, double *out_dev,
                                  void *stream) {
  if (!amps_dev || !out_dev) return set_error(SV_EINVAL, "null device pointer");
  if (n_qubits < 1 || n_qubits > 34)
    return set_error(SV_EINVAL, "sv_expect_z_all_noalloc handles 1 to 34 qubits");
  if (dtype != SV_C64 && dtype != SV_C128) return set_error(SV_EINVAL, "unknown dtype");
  if ((uintptr_t)amps_dev & 255) return set_error(SV_EINVAL, "amplitudes must be 256-byte aligned");
  if ((uintptr_t)out_dev & 7) return set_error(SV_EINVAL, "output must be 8-byte aligned");
  // both buffers must be memory the current device can address: a host
  // pointer or another device's memory would make the kernels fault
  int cur = 0;
  SV_CUDA(cudaGetDevice(&cur));
  for (const void *p : {amps_dev, static_cast<const void *>(out_dev)}) {
    cudaPointerAttributes attr;
    SV_CUDA(cudaPointerGetAttributes(&attr, p));
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
      return set_error(SV_EINVAL, "amplitudes and output must be device memory");
    if (attr.type == cudaMemoryTypeDevice && attr.device != cur)
      return set_error(SV_EINVAL, "amplitudes and output must be on the current device");
  }
  return zall_noalloc(amps_dev, n_qubits, dtype, out_dev, (cudaStream_t)stream);
}

sv_status sv_norm(sv_state *s, double *out) {
  if (!s || !out) return set_error(SV_EINVAL, "null argument");
  SV_TRY(launch_norm(s, scalars_dev(s)));
  SV_TRY(fetch(s, 1));
  *out = scalars_host(s)[0];
  return SV_OK;
}

sv_status sv_renormalize(sv_state *s, double *out) {
  double nrm = 0;
  SV_TRY(sv_norm(s, &nrm));
  if (out) *out = nrm;
  if (!(nrm > 0) || !std::isfinite(nrm)) return set_error(SV_EINVAL, "state has zero or non-finite norm");
  s->basis_known = false;
  return launch_scale(s, 1.0 / std::sqrt(nrm));
}

sv_status sv_sample(sv_state *s, int64_t shots, uint64_t seed, uint64_t *out) {
  if (!s) return set_error(SV_EINVAL, "null state");
  if (shots < 0 || (shots > 0 && !out)) return set_error(SV_EINVAL, "bad shot buffer");
  if (shots == 0) return SV_OK;
  SV_TRY(launch_sample_prepare(s));
  uint64_t *dev = reinterpret_cast<uint64_t *>(s->ws + kWsRed + sample_shot_offset(s->n));
  const int64_t cap = sample_shot_capacity();
  for (int64_t s0 = 0; s0 < shots; s0 += cap) {
    const int64_t cnt = std::min(cap, shots - s0);
    SV_TRY(launch_sample_shots(s, s0, cnt, seed, dev));
    SV_CUDA(cudaMemcpyAsync(out + s0, dev, sizeof(uint64_t) * cnt, cudaMemcpyDeviceToHost, s->stream));
    SV_CUDA(cudaStreamSynchronize(s->stream));
  }
  return SV_OK;
}

}  // extern "C"
