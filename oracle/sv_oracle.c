/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see sv_oracle.h).
 *
 * Every routine is the plain definition, in complex128, looped over the
 * amplitude index.  OpenMP only splits those loops across host cores; no
 * blocking, fusion or reordering of the arithmetic is done.
 */
#define _GNU_SOURCE
#include "sv_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* thread count of later parallel loops (timing on one core vs all cores) */
void or_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* ------------------------------------------------------------------------ */
/* gate matrices (the paper names no convention; readings stated per gate)  */
/* ------------------------------------------------------------------------ */

static const char *const k_names[OR_NGATES] = {
  "MATRIX", "I", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG",
  "SX", "SY", "SW", "RX", "RY", "RZ", "PHASE", "U3", "CZ", "SWAP", "FSIM"};

int or_gate_id(const char *name) {
  for (int g = 0; g < OR_NGATES; g++)
    if (strcmp(name, k_names[g]) == 0) return g;
  return -1;
}

int or_gate_targets(int gate) {
  if (gate == OR_MATRIX) return 0;
  if (gate == OR_CZ || gate == OR_SWAP || gate == OR_FSIM) return 2;
  if (gate > 0 && gate < OR_NGATES) return 1;
  return -1;
}

/* single-qubit Pauli matrices, row-major */
static void pauli(int which, cplx P[4]) {
  switch (which) {
    case 0: P[0] = 1; P[1] = 0; P[2] = 0; P[3] = 1; break;       /* I */
    case 1: P[0] = 0; P[1] = 1; P[2] = 1; P[3] = 0; break;       /* X */
    case 2: P[0] = 0; P[1] = -I; P[2] = I; P[3] = 0; break;      /* Y */
    default: P[0] = 1; P[1] = 0; P[2] = 0; P[3] = -1; break;     /* Z */
  }
}

/* exp(-i theta P / 2) = cos(theta/2) I - i sin(theta/2) P for a Pauli P */
static void pauli_rotation(int which, double theta, cplx U[4]) {
  cplx P[4];
  pauli(which, P);
  double c = cos(theta / 2), s = sin(theta / 2);
  for (int i = 0; i < 4; i++) U[i] = (i == 0 || i == 3 ? c : 0.0) - I * s * P[i];
}

/* square root of a Pauli-like involution P with Cirq's phase:
 * P^(1/2) = ((1+i)/2) (I - i P) */
static void sqrt_involution(const cplx P[4], cplx U[4]) {
  const cplx f = (1.0 + I) / 2.0;
  for (int i = 0; i < 4; i++) U[i] = f * ((i == 0 || i == 3 ? 1.0 : 0.0) - I * P[i]);
}

static double snap(double v) { return fabs(v) < 1e-15 ? 0.0 : v; }

static void store(const cplx *U, int dim, double *out) {
  for (int i = 0; i < dim * dim; i++) {
    out[2 * i] = creal(U[i]);
    out[2 * i + 1] = cimag(U[i]);
  }
}

int or_gate_matrix(int gate, const double *a, double *out) {
  cplx U[16];
  memset(U, 0, sizeof U);
  cplx P[4];
  switch (gate) {
    case OR_I: case OR_X: case OR_Y: case OR_Z:
      pauli(gate == OR_I ? 0 : gate == OR_X ? 1 : gate == OR_Y ? 2 : 3, U);
      store(U, 2, out);
      return 1;
    case OR_H: {
      double r = 1.0 / sqrt(2.0);
      U[0] = r; U[1] = r; U[2] = r; U[3] = -r;
      store(U, 2, out);
      return 1;
    }
    case OR_S: U[0] = 1; U[3] = I; store(U, 2, out); return 1;
    case OR_SDG: U[0] = 1; U[3] = -I; store(U, 2, out); return 1;
    case OR_T: U[0] = 1; U[3] = cexp(I * M_PI / 4); store(U, 2, out); return 1;
    case OR_TDG: U[0] = 1; U[3] = cexp(-I * M_PI / 4); store(U, 2, out); return 1;
    case OR_SX: pauli(1, P); sqrt_involution(P, U); store(U, 2, out); return 1;
    case OR_SY: pauli(2, P); sqrt_involution(P, U); store(U, 2, out); return 1;
    case OR_SW: {
      /* W = (X + Y) / sqrt(2) */
      cplx X[4], Y[4];
      pauli(1, X);
      pauli(2, Y);
      for (int i = 0; i < 4; i++) P[i] = (X[i] + Y[i]) / sqrt(2.0);
      sqrt_involution(P, U);
      store(U, 2, out);
      return 1;
    }
    case OR_RX: pauli_rotation(1, a[0], U); store(U, 2, out); return 1;
    case OR_RY: pauli_rotation(2, a[0], U); store(U, 2, out); return 1;
    case OR_RZ: pauli_rotation(3, a[0], U); store(U, 2, out); return 1;
    case OR_PHASE: U[0] = 1; U[3] = cexp(I * a[0]); store(U, 2, out); return 1;
    case OR_U3: {
      /* OpenQASM U3(theta, phi, lambda) */
      double c = cos(a[0] / 2), s = sin(a[0] / 2);
      U[0] = c;
      U[1] = -cexp(I * a[2]) * s;
      U[2] = cexp(I * a[1]) * s;
      U[3] = cexp(I * (a[1] + a[2])) * c;
      store(U, 2, out);
      return 1;
    }
    case OR_CZ:
      U[0] = 1; U[5] = 1; U[10] = 1; U[15] = -1;
      store(U, 4, out);
      return 2;
    case OR_SWAP:
      U[0] = 1; U[1 * 4 + 2] = 1; U[2 * 4 + 1] = 1; U[15] = 1;
      store(U, 4, out);
      return 2;
    case OR_FSIM: {
      /* basis (t1 t0) = 00, 01, 10, 11; cos/sin below 1e-15 taken as 0 */
      double c = snap(cos(a[0])), s = snap(sin(a[0]));
      U[0] = 1;
      U[1 * 4 + 1] = c;
      U[1 * 4 + 2] = -I * s;
      U[2 * 4 + 1] = -I * s;
      U[2 * 4 + 2] = c;
      U[15] = cexp(-I * a[1]);
      store(U, 4, out);
      return 2;
    }
    default:
      return -1;
  }
}

int or_op_matrix(const or_op *op, const double *params, double *out) {
  if (op->gate == OR_MATRIX) {
    if (!op->matrix || op->k < 1 || op->k > 6) return -1;
    int d = 1 << op->k;
    memcpy(out, op->matrix, sizeof(double) * 2 * d * d);
    return op->k;
  }
  double ang[3] = {op->angles[0], op->angles[1], op->angles[2]};
  if (op->param >= 0) {
    if (!params) return -1;
    ang[0] = params[op->param];
  }
  int k = or_gate_matrix(op->gate, ang, out);
  if (k != op->k) return -1;
  return k;
}

/* ------------------------------------------------------------------------ */
/* gate application                                                          */
/* ------------------------------------------------------------------------ */

static uint64_t target_offset(uint64_t y, const int32_t *t, int k) {
  uint64_t off = 0;
  for (int j = 0; j < k; j++) off |= ((y >> j) & 1ULL) << t[j];
  return off;
}

void or_apply(double *psi_, int n, const int32_t *t, int k, const int32_t *c, int nc,
              const double *U_) {
  cplx *psi = (cplx *)psi_;
  const cplx *U = (const cplx *)U_;
  const int64_t N = (int64_t)1 << n;
  const int dim = 1 << k;
  uint64_t tmask = 0, cmask = 0;
  for (int j = 0; j < k; j++) tmask |= 1ULL << t[j];
  for (int j = 0; j < nc; j++) cmask |= 1ULL << c[j];
  uint64_t off[64];
  for (int y = 0; y < dim; y++) off[y] = target_offset((uint64_t)y, t, k);
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < N; x++) {
    if ((uint64_t)x & tmask) continue;              /* x must be a group base */
    if (((uint64_t)x & cmask) != cmask) continue;   /* controls not all 1 */
    cplx v[64], w[64];
    for (int y = 0; y < dim; y++) v[y] = psi[(uint64_t)x | off[y]];
    for (int r = 0; r < dim; r++) {
      cplx acc = 0;
      for (int y = 0; y < dim; y++) acc += U[r * dim + y] * v[y];
      w[r] = acc;
    }
    for (int r = 0; r < dim; r++) psi[(uint64_t)x | off[r]] = w[r];
  }
}

static uint64_t local_index(uint64_t x, const int32_t *t, int k) {
  uint64_t r = 0;
  for (int j = 0; j < k; j++) r |= ((x >> t[j]) & 1ULL) << j;
  return r;
}

int or_full_matrix(int n, const int32_t *t, int k, const int32_t *c, int nc, const double *U_,
                   double *M_) {
  if (n > 12) return -1;
  const cplx *U = (const cplx *)U_;
  cplx *M = (cplx *)M_;
  const uint64_t N = 1ULL << n;
  const int dim = 1 << k;
  uint64_t tmask = 0, cmask = 0;
  for (int j = 0; j < k; j++) tmask |= 1ULL << t[j];
  for (int j = 0; j < nc; j++) cmask |= 1ULL << c[j];
  for (uint64_t r = 0; r < N; r++)
    for (uint64_t col = 0; col < N; col++) {
      cplx v = 0;
      if ((r & ~tmask) == (col & ~tmask)) {
        uint64_t rt = local_index(r, t, k), ct = local_index(col, t, k);
        if ((col & cmask) == cmask)
          v = U[rt * dim + ct];
        else
          v = (rt == ct) ? 1.0 : 0.0;
      }
      M[r * N + col] = v;
    }
  return 0;
}

void or_matvec(int n, const double *M_, const double *x_, double *y_) {
  const cplx *M = (const cplx *)M_, *x = (const cplx *)x_;
  cplx *y = (cplx *)y_;
  const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < N; r++) {
    cplx acc = 0;
    for (int64_t col = 0; col < N; col++) acc += M[r * N + col] * x[col];
    y[r] = acc;
  }
}

static int op_ok(const or_op *op, int n) {
  if (op->k < 1 || op->k > 6 || op->nctrl < 0 || op->nctrl > 8) return 0;
  uint64_t seen = 0;
  for (int j = 0; j < op->k; j++) {
    int q = op->targets[j];
    if (q < 0 || q >= n || (seen >> q) & 1) return 0;
    seen |= 1ULL << q;
  }
  for (int j = 0; j < op->nctrl; j++) {
    int q = op->controls[j];
    if (q < 0 || q >= n || (seen >> q) & 1) return 0;
    seen |= 1ULL << q;
  }
  return 1;
}

int or_run(double *psi, int n, const or_op *ops, int nops, const double *params) {
  double U[2 * 64 * 64];
  for (int i = 0; i < nops; i++) {
    if (!op_ok(&ops[i], n)) return -1;
    if (or_op_matrix(&ops[i], params, U) < 0) return -1;
    or_apply(psi, n, ops[i].targets, ops[i].k, ops[i].controls, ops[i].nctrl, U);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* observables                                                              */
/* ------------------------------------------------------------------------ */

/* (P psi)[x ^ xm] = i^{popcount(xm & zm)} (-1)^{popcount(x & zm)} psi[x] */
static cplx y_phase(uint64_t xm, uint64_t zm) {
  static const cplx ipow[4] = {1, I, -1, -I};
  return ipow[__builtin_popcountll(xm & zm) & 3];
}

double or_expect(const double *psi_, int n, const uint64_t *xm, const uint64_t *zm,
                 const double *coeff, int nterms) {
  const cplx *psi = (const cplx *)psi_;
  const int64_t N = (int64_t)1 << n;
  double total = 0;
  for (int t = 0; t < nterms; t++) {
    const cplx ph = y_phase(xm[t], zm[t]);
    double re = 0;
#pragma omp parallel for reduction(+ : re) schedule(static)
    for (int64_t x = 0; x < N; x++) {
      double sgn = (__builtin_popcountll((uint64_t)x & zm[t]) & 1) ? -1.0 : 1.0;
      cplx p = ph * sgn * psi[x];                        /* component of P psi at x ^ xm */
      re += creal(conj(psi[(uint64_t)x ^ xm[t]]) * p);
    }
    total += coeff[t] * re;
  }
  return total;
}

void or_apply_pauli_sum(const double *psi_, double *out_, int n, const uint64_t *xm,
                        const uint64_t *zm, const double *coeff, int nterms) {
  const cplx *psi = (const cplx *)psi_;
  cplx *out = (cplx *)out_;
  const int64_t N = (int64_t)1 << n;
  memset(out, 0, sizeof(cplx) * (size_t)N);
  for (int t = 0; t < nterms; t++) {
    const cplx ph = y_phase(xm[t], zm[t]) * coeff[t];
    /* x -> x ^ xm is a bijection, so each output index is written once per term */
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; x++) {
      double sgn = (__builtin_popcountll((uint64_t)x & zm[t]) & 1) ? -1.0 : 1.0;
      out[(uint64_t)x ^ xm[t]] += ph * sgn * psi[x];
    }
  }
}

void or_z_all(const double *psi_, int n, double *out) {
  const cplx *psi = (const cplx *)psi_;
  const int64_t N = (int64_t)1 << n;
  for (int q = 0; q < n; q++) {
    double acc = 0;
#pragma omp parallel for reduction(+ : acc) schedule(static)
    for (int64_t x = 0; x < N; x++) {
      double p = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
      acc += ((x >> q) & 1) ? -p : p;
    }
    out[q] = acc;
  }
}

double or_norm2(const double *psi_, int n) {
  const cplx *psi = (const cplx *)psi_;
  const int64_t N = (int64_t)1 << n;
  double acc = 0;
#pragma omp parallel for reduction(+ : acc) schedule(static)
  for (int64_t x = 0; x < N; x++) acc += creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
  return acc;
}

/* ------------------------------------------------------------------------ */
/* sampling                                                                 */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea, Flood 2014): state advances by the golden-ratio
 * increment, output is the 64-bit finaliser of the state. */
uint64_t or_splitmix64(uint64_t seed, uint64_t s) {
  uint64_t z = seed + (s + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct { double target; int64_t shot; } shot_t;

static int cmp_shot(const void *a, const void *b) {
  double x = ((const shot_t *)a)->target, y = ((const shot_t *)b)->target;
  return x < y ? -1 : x > y ? 1 : 0;
}

void or_sample(const double *psi_, int n, int64_t shots, uint64_t seed, uint64_t *out) {
  const cplx *psi = (const cplx *)psi_;
  const uint64_t N = 1ULL << n;
  /* total probability: the CDF's last entry, summed in index order */
  double total = 0;
  for (uint64_t x = 0; x < N; x++) total += creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
  shot_t *sh = (shot_t *)malloc(sizeof(shot_t) * (size_t)(shots > 0 ? shots : 1));
  for (int64_t s = 0; s < shots; s++) {
    double u = (double)(or_splitmix64(seed, (uint64_t)s) >> 11) * 0x1.0p-53;
    sh[s].target = u * total;
    sh[s].shot = s;
  }
  qsort(sh, (size_t)shots, sizeof(shot_t), cmp_shot);
  /* one sweep of the inclusive prefix sum: smallest x with CDF(x) > target */
  double cdf = 0;
  uint64_t x = 0;
  int64_t i = 0;
  while (i < shots) {
    double p = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
    double next = cdf + p;
    while (i < shots && next > sh[i].target) out[sh[i++].shot] = x;
    if (x == N - 1) {               /* rounding left targets at the top: last index */
      while (i < shots) out[sh[i++].shot] = N - 1;
      break;
    }
    cdf = next;
    x++;
  }
  free(sh);
}

/* ------------------------------------------------------------------------ */
/* adjoint differentiation                                                   */
/* ------------------------------------------------------------------------ */

/* U(theta) = exp(-i theta G / 2): generator G for the supported gates */
static int generator(int gate, cplx G[4]) {
  memset(G, 0, sizeof(cplx) * 4);
  switch (gate) {
    case OR_RX: pauli(1, G); return 0;
    case OR_RY: pauli(2, G); return 0;
    case OR_RZ: pauli(3, G); return 0;
    case OR_PHASE: G[3] = -2.0; return 0;   /* diag(1, e^{i t}) = exp(-i t diag(0,-2) / 2) */
    default: return -1;
  }
}

/* phi = (projector onto controls = 1) (G on target) psi */
static void apply_generator(const cplx *psi, cplx *phi, int n, const or_op *op, const cplx G[4]) {
  const int64_t N = (int64_t)1 << n;
  uint64_t cmask = 0, tb = 1ULL << op->targets[0];
  for (int j = 0; j < op->nctrl; j++) cmask |= 1ULL << op->controls[j];
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < N; x++) {
    if (((uint64_t)x & cmask) != cmask) { phi[x] = 0; continue; }
    int r = ((uint64_t)x & tb) ? 1 : 0;
    cplx v0 = psi[(uint64_t)x & ~tb], v1 = psi[(uint64_t)x | tb];
    phi[x] = G[r * 2 + 0] * v0 + G[r * 2 + 1] * v1;
  }
}

static void adjoint_matrix(const double *U_, int k, double *Ud_) {
  const cplx *U = (const cplx *)U_;
  cplx *Ud = (cplx *)Ud_;
  int d = 1 << k;
  for (int r = 0; r < d; r++)
    for (int c = 0; c < d; c++) Ud[r * d + c] = conj(U[c * d + r]);
}

int or_adjoint_grad(double *psi_, int n, const or_op *ops, int nops, const double *params,
                    int n_params, const uint64_t *xm, const uint64_t *zm, const double *coeff,
                    int nterms, double *expval, double *grad) {
  const int64_t N = (int64_t)1 << n;
  for (int i = 0; i < nops; i++) {
    if (!op_ok(&ops[i], n)) return -1;
    cplx G[4];
    if (ops[i].param >= 0 && (ops[i].k != 1 || generator(ops[i].gate, G) != 0)) return -2;
    if (ops[i].param >= n_params) return -1;
  }
  /* forward sweep */
  if (or_run(psi_, n, ops, nops, params) != 0) return -1;
  const cplx *out = (const cplx *)psi_;
  cplx *lam = (cplx *)malloc(sizeof(cplx) * (size_t)N);
  cplx *phi = (cplx *)malloc(sizeof(cplx) * (size_t)N);
  cplx *psi = (cplx *)malloc(sizeof(cplx) * (size_t)N);
  if (!lam || !phi || !psi) { free(lam); free(phi); free(psi); return -3; }
  memcpy(psi, out, sizeof(cplx) * (size_t)N);      /* psi_ keeps the forward result */
  /* lambda = H psi, <H> = Re <psi | lambda> */
  or_apply_pauli_sum(psi_, (double *)lam, n, xm, zm, coeff, nterms);
  double e = 0;
#pragma omp parallel for reduction(+ : e) schedule(static)
  for (int64_t x = 0; x < N; x++) e += creal(conj(psi[x]) * lam[x]);
  *expval = e;
  for (int p = 0; p < n_params; p++) grad[p] = 0;
  /* backward sweep: psi, lambda are the states just after gate j */
  double U[2 * 64 * 64], Ud[2 * 64 * 64];
  for (int j = nops - 1; j >= 0; j--) {
    const or_op *op = &ops[j];
    if (op->param >= 0) {
      cplx G[4];
      generator(op->gate, G);
      apply_generator(psi, phi, n, op, G);
      double im = 0;
#pragma omp parallel for reduction(+ : im) schedule(static)
      for (int64_t x = 0; x < N; x++) im += cimag(conj(lam[x]) * phi[x]);
      grad[op->param] += im;     /* d<H>/dtheta = Im <lambda | G | psi> */
    }
    int k = or_op_matrix(op, params, U);
    adjoint_matrix(U, k, Ud);
    or_apply((double *)psi, n, op->targets, k, op->controls, op->nctrl, Ud);
    or_apply((double *)lam, n, op->targets, k, op->controls, op->nctrl, Ud);
  }
  free(psi);
  free(lam);
  free(phi);
  return 0;
}
