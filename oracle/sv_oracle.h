/*
 * FP64 CPU oracle for Schroedinger state-vector simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, obviously
 * correct statement of what the GPU library computes.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no source with the CUDA library.
 *
 * Method (paper, Sec. I-A and Sec. II): the 2^n complex amplitudes are kept
 * in full and every gate is a matrix-vector product on them, so a circuit's
 * output is  psi_out = U_G ... U_1 psi_in.
 *
 * Conventions: qubit q is bit q of the amplitude index; a k-qubit gate's
 * local row/column bit j belongs to targets[j]; all controls must be 1.
 * States are complex128, stored as interleaved (re, im) doubles.
 *
 * Pins (tests/test_oracle_*.py): index loop == materialised 2^n x 2^n matrix
 * for n <= 10; that matrix == numpy Kronecker / tensor contractions;
 * GHZ, QFT, H^n closed forms; multiplier outputs a*b; Pauli expectations vs
 * explicit Hamiltonian matrices; adjoint gradient vs the exact
 * parameter-shift rule and sin(h)/h-corrected central differences;
 * SplitMix64 vs its published output for seed 0; sampling vs basis, GHZ
 * and chi-square cases.
 */
#ifndef SV_ORACLE_H
#define SV_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  OR_MATRIX = 0, OR_I, OR_X, OR_Y, OR_Z, OR_H, OR_S, OR_SDG, OR_T, OR_TDG,
  OR_SX, OR_SY, OR_SW, OR_RX, OR_RY, OR_RZ, OR_PHASE, OR_U3,
  OR_CZ, OR_SWAP, OR_FSIM, OR_NGATES
};

typedef struct {
  int32_t gate;          /* OR_* */
  int32_t k;             /* number of targets */
  int32_t nctrl;         /* number of controls */
  int32_t param;         /* -1, or index into params replacing angles[0] */
  int32_t targets[8];
  int32_t controls[8];
  double angles[3];
  const double *matrix;  /* OR_MATRIX: 2^k x 2^k complex, row-major, interleaved */
} or_op;

/* gate table */
int or_gate_id(const char *name);          /* -1 if unknown */
int or_gate_targets(int gate);             /* 0 for OR_MATRIX (any k) */
/* Writes the 2^k x 2^k matrix of a named gate (complex, interleaved).
 * Returns k, or -1 for OR_MATRIX / unknown gates. */
int or_gate_matrix(int gate, const double *angles, double *out);

/* c-1 (i): in-place index loop.  psi' [x] = sum_y U[r(x), y] psi[x|y on targets]
 * where every control bit of x is 1; other amplitudes unchanged. */
void or_apply(double *psi, int n, const int32_t *targets, int k,
              const int32_t *controls, int nctrl, const double *U);
/* c-1 (ii): the same gate as an explicit 2^n x 2^n matrix (n <= 12). */
int or_full_matrix(int n, const int32_t *targets, int k, const int32_t *controls,
                   int nctrl, const double *U, double *M);
/* dense y = M x for a 2^n x 2^n matrix */
void or_matvec(int n, const double *M, const double *x, double *y);

/* run a circuit in place; params may be NULL when no op is parametric.
 * Returns 0, or -1 on a malformed op. */
int or_run(double *psi, int n, const or_op *ops, int nops, const double *params);
/* the op's matrix after substituting params (k returned, -1 on error) */
int or_op_matrix(const or_op *op, const double *params, double *out);

/* Pauli strings: X on bits of x_mask, Z on bits of z_mask, Y where both. */
double or_expect(const double *psi, int n, const uint64_t *x_mask, const uint64_t *z_mask,
                 const double *coeff, int nterms);
void or_apply_pauli_sum(const double *psi, double *out, int n, const uint64_t *x_mask,
                        const uint64_t *z_mask, const double *coeff, int nterms);
void or_z_all(const double *psi, int n, double *out);
double or_norm2(const double *psi, int n);

/* counter-based SplitMix64: the s-th (0-based) output of the sequential
 * generator seeded with `seed` */
uint64_t or_splitmix64(uint64_t seed, uint64_t s);
/* shot s -> smallest x with CDF(x) > u_s * sum|psi|^2, u_s = (splitmix >> 11) 2^-53 */
void or_sample(const double *psi, int n, int64_t shots, uint64_t seed, uint64_t *out);

/* Adjoint gradient of <psi_out|H|psi_out>, psi_out = circuit(params) psi_in.
 * psi: in = psi_in, out = psi_out (forward result).  Parametric ops must be
 * RX, RY, RZ or PHASE (any controls).  grad has n_params entries.
 * Returns 0, -1 on malformed op, -2 on unsupported parametric gate, -3 on
 * allocation failure. */
int or_adjoint_grad(double *psi, int n, const or_op *ops, int nops, const double *params,
                    int n_params, const uint64_t *x_mask, const uint64_t *z_mask,
                    const double *coeff, int nterms, double *expval, double *grad);

int or_num_threads(void);
void or_set_num_threads(int t);

#ifdef __cplusplus
}
#endif
#endif
