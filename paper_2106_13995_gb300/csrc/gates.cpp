// Host-side gate matrices in FP64 and circuit validation.
//
// Each named gate is written out entry by entry.  The paper fixes no gate
// convention (its circuits come from Cirq and QUANTIFY, Sec. II); the library
// uses: OpenQASM's U3; RX/RY/RZ = exp(-i theta P / 2); PHASE = diag(1, e^{i l});
// SX/SY/SW = ((1+i)/2)(I - iP) for P = X, Y, W = (X+Y)/sqrt(2); fSim with
// cos/sin snapped to 0 below 1e-15 so that fSim(pi/2, .) has exact zeros.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>

#include "sv_internal.h"

namespace sv {

static const cd kI(0.0, 1.0);

int gate_arity(int g) {
  switch (g) {
    case SV_GATE_H: case SV_GATE_X: case SV_GATE_Y: case SV_GATE_Z: case SV_GATE_S:
    case SV_GATE_SDG: case SV_GATE_T: case SV_GATE_TDG: case SV_GATE_SX: case SV_GATE_SY:
    case SV_GATE_SW: case SV_GATE_ID: case SV_GATE_RX: case SV_GATE_RY: case SV_GATE_RZ:
    case SV_GATE_PHASE: case SV_GATE_U3:
      return 1;
    case SV_GATE_CZ: case SV_GATE_SWAP: case SV_GATE_FSIM:
      return 2;
    case SV_GATE_MATRIX:
      return 0;
    default:
      return -1;
  }
}

static double snap0(double v) { return std::fabs(v) < 1e-15 ? 0.0 : v; }

bool gate_matrix(int g, const double *a, std::vector<cd> &U) {
  const double r2 = 1.0 / std::sqrt(2.0);
  const cd h(0.5, 0.5);  // (1+i)/2
  switch (g) {
    case SV_GATE_H: U = {r2, r2, r2, -r2}; return true;
    case SV_GATE_X: U = {0.0, 1.0, 1.0, 0.0}; return true;
    case SV_GATE_Y: U = {0.0, -kI, kI, 0.0}; return true;
    case SV_GATE_Z: U = {1.0, 0.0, 0.0, -1.0}; return true;
    case SV_GATE_ID: U = {1.0, 0.0, 0.0, 1.0}; return true;
    case SV_GATE_S: U = {1.0, 0.0, 0.0, kI}; return true;
    case SV_GATE_SDG: U = {1.0, 0.0, 0.0, -kI}; return true;
    case SV_GATE_T: U = {1.0, 0.0, 0.0, cd(r2, r2)}; return true;
    case SV_GATE_TDG: U = {1.0, 0.0, 0.0, cd(r2, -r2)}; return true;
    case SV_GATE_SX: U = {h, std::conj(h), std::conj(h), h}; return true;
    case SV_GATE_SY: U = {h, -h, h, h}; return true;
    case SV_GATE_SW: U = {h, cd(0.0, -r2), cd(r2, 0.0), h}; return true;
    case SV_GATE_RX: {
      double c = std::cos(a[0] / 2), s = std::sin(a[0] / 2);
      U = {c, cd(0, -s), cd(0, -s), c};
      return true;
    }
    case SV_GATE_RY: {
      double c = std::cos(a[0] / 2), s = std::sin(a[0] / 2);
      U = {c, -s, s, c};
      return true;
    }
    case SV_GATE_RZ: {
      double c = std::cos(a[0] / 2), s = std::sin(a[0] / 2);
      U = {cd(c, -s), 0.0, 0.0, cd(c, s)};
      return true;
    }
    case SV_GATE_PHASE:
      U = {1.0, 0.0, 0.0, cd(std::cos(a[0]), std::sin(a[0]))};
      return true;
    case SV_GATE_U3: {
      double c = std::cos(a[0] / 2), s = std::sin(a[0] / 2);
      cd el(std::cos(a[2]), std::sin(a[2])), ep(std::cos(a[1]), std::sin(a[1]));
      cd epl(std::cos(a[1] + a[2]), std::sin(a[1] + a[2]));
      U = {c, -el * s, ep * s, epl * c};
      return true;
    }
    case SV_GATE_CZ:
      U.assign(16, 0.0);
      U[0] = U[5] = U[10] = 1.0;
      U[15] = -1.0;
      return true;
    case SV_GATE_SWAP:
      U.assign(16, 0.0);
      U[0] = U[6] = U[9] = U[15] = 1.0;
      return true;
    case SV_GATE_FSIM: {
      double c = snap0(std::cos(a[0])), s = snap0(std::sin(a[0]));
      U.assign(16, 0.0);
      U[0] = 1.0;
      U[5] = c;
      U[6] = cd(0, -s);
      U[9] = cd(0, -s);
      U[10] = c;
      U[15] = cd(std::cos(a[1]), -std::sin(a[1]));
      return true;
    }
    default:
      return false;
  }
}

int gate_generator(int g) {
  switch (g) {
    case SV_GATE_RX: return 1;
    case SV_GATE_RY: return 2;
    case SV_GATE_RZ: return 3;
    case SV_GATE_PHASE: return 4;
    default: return 0;
  }
}

std::vector<cd> adjoint_of(const std::vector<cd> &U, int k) {
  const int d = 1 << k;
  std::vector<cd> A(U.size());
  for (int r = 0; r < d; r++)
    for (int c = 0; c < d; c++) A[r * d + c] = std::conj(U[c * d + r]);
  return A;
}

sv_status circuit_to_gates(const sv_circuit *c, const double *params, int n,
                           std::vector<Gate> &out, bool keep_params_unfused) {
  if (!c || (c->n_ops > 0 && !c->ops)) return set_error(SV_EINVAL, "null circuit");
  if (c->n_qubits != n)
    return set_error(SV_EINVAL, "circuit width " + std::to_string(c->n_qubits) +
                                    " does not match the state's " + std::to_string(n));
  out.clear();
  out.reserve(c->n_ops);
  for (int i = 0; i < c->n_ops; i++) {
    const sv_op &op = c->ops[i];
    const std::string where = "op " + std::to_string(i) + ": ";
    int ar = gate_arity(op.gate);
    if (ar < 0) return set_error(SV_EINVAL, where + "unknown gate id " + std::to_string(op.gate));
    int k = op.n_targets;
    if (ar == 0 ? (k < 1 || k > 6) : k != ar)
      return set_error(SV_EINVAL, where + "wrong number of targets");
    if (op.n_controls < 0 || op.n_controls > 8)
      return set_error(SV_EINVAL, where + "0..8 controls allowed");
    uint64_t seen = 0;
    Gate g;
    for (int j = 0; j < k + op.n_controls; j++) {
      int q = j < k ? op.targets[j] : op.controls[j - k];
      if (q < 0 || q >= n) return set_error(SV_EINVAL, where + "qubit out of range");
      if ((seen >> q) & 1) return set_error(SV_EINVAL, where + "duplicate qubit");
      seen |= 1ull << q;
      (j < k ? g.targets : g.controls).push_back(q);
    }
    if (op.gate == SV_GATE_MATRIX) {
      if (!c->matrices || op.matrix_offset < 0)
        return set_error(SV_EINVAL, where + "MATRIX op without a matrix");
      const int d = 1 << k;
      g.U.resize(d * d);
      const double *m = c->matrices + 2 * op.matrix_offset;
      for (int e = 0; e < d * d; e++) g.U[e] = cd(m[2 * e], m[2 * e + 1]);
      if (unitarity_checks() && unitarity_error(g.U, k) > kUnitaryTol)
        return set_error(SV_EINVAL, where + "matrix is not unitary (max |U^dagger U - I| = " +
                                        std::to_string(unitarity_error(g.U, k)) + ")");
    } else {
      double ang[3] = {op.angles[0], op.angles[1], op.angles[2]};
      if (op.param >= 0) {
        if (op.param >= c->n_params) return set_error(SV_EINVAL, where + "param index out of range");
        if (!params) return set_error(SV_EINVAL, where + "parametric op but params is NULL");
        ang[0] = params[op.param];
        g.param = op.param;
        g.param_gate = op.gate;
        g.fixed_structure = keep_params_unfused;
      }
      gate_matrix(op.gate, ang, g.U);
    }
    out.push_back(std::move(g));
  }
  return SV_OK;
}

// max over entries of |U^dagger U - I|
double unitarity_error(const std::vector<cd> &U, int k) {
  const int d = 1 << k;
  double worst = 0;
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) {
      cd a = 0;
      for (int r = 0; r < d; r++) a += std::conj(U[(size_t)r * d + i]) * U[(size_t)r * d + j];
      worst = std::max(worst, std::abs(a - (i == j ? cd(1.0) : cd(0.0))));
    }
  return worst;
}

// on in SV_DEBUG builds, or when the environment sets SV_CHECK_UNITARY=1
bool unitarity_checks() {
#ifdef SV_DEBUG
  return true;
#else
  const char *e = std::getenv("SV_CHECK_UNITARY");
  return e && e[0] == '1';
#endif
}

bool propagate_basis(const std::vector<Gate> &gates, uint64_t &index, cd &amp) {
  for (const Gate &g : gates) {
    if (g.grad_gen > 0) return false;
    bool on = true;
    for (int q : g.controls) on = on && ((index >> q) & 1ull);
    if (!on) continue;
    const int k = (int)g.targets.size(), d = 1 << k;
    int c = 0;
    for (int j = 0; j < k; j++) c |= (int)((index >> g.targets[j]) & 1ull) << j;
    // column c of U must hold exactly one nonzero entry
    int r1 = -1;
    for (int r = 0; r < d; r++)
      if (g.U[(size_t)r * d + c] != cd(0.0)) {
        if (r1 >= 0) return false;
        r1 = r;
      }
    if (r1 < 0) return false;
    amp *= g.U[(size_t)r1 * d + c];
    for (int j = 0; j < k; j++) {
      const uint64_t bit = 1ull << g.targets[j];
      index = ((r1 >> j) & 1) ? (index | bit) : (index & ~bit);
    }
  }
  return true;
}

}  // namespace sv
