/*
 * FP64 CPU oracle for the cut-CZ partition scheme (arXiv 1802.06952).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and used by
 * tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py.  It shares
 * no code, header or table with the CUDA library, and the library never calls it.
 *
 * What it computes, each step written plainly in the paper's order:
 *   - or_evolve: the state-vector update of Supplementary A, Eq. (4), applied one
 *     gate at a time to a complex128 vector, little-endian (qubit q = bit q of the
 *     index).  No gate fusion and no combining of diagonal gates.
 *   - or_cut_sum: the reconstruction of Supplementary A, Eq. (8) / Section 2.1:
 *     for each copy k of the 2^c copies, evolve the upper and lower half-circuits
 *     separately and add U_k[x_u] * L_k[x_l] into every requested amplitude, in
 *     k order, in FP64.
 *
 * Gate matrices (principal square roots; the paper names X, Y, T and gives
 * T_11 = (1+i)/sqrt 2 in Section 2.4):
 *   H   = 1/sqrt2 [[1, 1], [1, -1]]
 *   X2  = X^1/2 = 1/2 [[1+i, 1-i], [1-i, 1+i]]
 *   Y2  = Y^1/2 = 1/2 [[1+i, -1-i], [1+i, 1+i]]
 *   T   = diag(1, (1+i)/sqrt2)
 *   CZ  = diag(1, 1, 1, -1)                                    (Eq. 1 left side)
 *   P0  = diag(1, 0), P1 = diag(0, 1), Z = diag(1, -1)         (Eq. 1 right side)
 *   CX  = controlled X, control q1, target q2; X = [[0, 1], [1, 0]]
 *         (Supplementary A, Eq. 1 with U = X: CX = P0 (x) I + P1 (x) X)
 *   CT, CY2 = controlled T and controlled Y^1/2, control q1, target q2
 *         (Supplementary A, Eq. 1: P0 (x) I + P1 (x) U with U = T or Y^1/2)
 *
 * Gate encoding (three int32 per gate): {code, q1, q2}; q2 is used by CZ and CX.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_H = 0, OR_X2 = 1, OR_Y2 = 2, OR_T = 3, OR_CZ = 4, OR_P0 = 5, OR_P1 = 6, OR_Z = 7, OR_CX = 8, OR_X = 9,
       OR_CT = 10, OR_CY2 = 11 };

typedef double complex cplx;

static void gate_matrix(int code, cplx m[4]) {
  const double s = 1.0 / sqrt(2.0);
  switch (code) {
    case OR_H:
      m[0] = s; m[1] = s; m[2] = s; m[3] = -s;
      break;
    case OR_X2:
      m[0] = 0.5 * (1 + I); m[1] = 0.5 * (1 - I);
      m[2] = 0.5 * (1 - I); m[3] = 0.5 * (1 + I);
      break;
    case OR_Y2:
      m[0] = 0.5 * (1 + I); m[1] = 0.5 * (-1 - I);
      m[2] = 0.5 * (1 + I); m[3] = 0.5 * (1 + I);
      break;
    case OR_T:
      m[0] = 1; m[1] = 0; m[2] = 0; m[3] = s * (1 + I);
      break;
    case OR_P0:
      m[0] = 1; m[1] = 0; m[2] = 0; m[3] = 0;
      break;
    case OR_P1:
      m[0] = 0; m[1] = 0; m[2] = 0; m[3] = 1;
      break;
    case OR_Z:
      m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -1;
      break;
    case OR_X:
      m[0] = 0; m[1] = 1; m[2] = 1; m[3] = 0;
      break;
    default:
      m[0] = 1; m[1] = 0; m[2] = 0; m[3] = 1;
  }
}

/* psi'_{..i_q..} = sum_j U_{i_q j} psi_{..j..}  (Eq. 4 for one single-qubit gate). */
static void apply_1q(cplx* psi, int n, int q, const cplx m[4]) {
  const int64_t dim = (int64_t)1 << n;
  const int64_t bit = (int64_t)1 << q;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < dim; ++i) {
    if (i & bit) continue;
    cplx a0 = psi[i], a1 = psi[i | bit];
    psi[i] = m[0] * a0 + m[1] * a1;
    psi[i | bit] = m[2] * a0 + m[3] * a1;
  }
}

/* CZ on (q1, q2): amplitude negated where both bits are 1 (Eq. 6 for one gate). */
static void apply_cz(cplx* psi, int n, int q1, int q2) {
  const int64_t dim = (int64_t)1 << n;
  const int64_t m = ((int64_t)1 << q1) | ((int64_t)1 << q2);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < dim; ++i)
    if ((i & m) == m) psi[i] = -psi[i];
}

/* CX with control qc and target qt: amplitudes with bit qc set exchange the target
 * bit (Eq. 4 for the two-qubit gate). */
static void apply_cx(cplx* psi, int n, int qc, int qt) {
  const int64_t dim = (int64_t)1 << n;
  const int64_t c = (int64_t)1 << qc, t = (int64_t)1 << qt;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < dim; ++i) {
    if (!(i & c) || (i & t)) continue;
    const cplx a = psi[i];
    psi[i] = psi[i | t];
    psi[i | t] = a;
  }
}

/* P0 (x) I + P1 (x) U on (qc, qt): the pairs of the target with the control bit
 * set get U, the others are left alone (Supplementary A, Eq. 1). */
static void apply_cu(cplx* psi, int n, int qc, int qt, const cplx m[4]) {
  const int64_t dim = (int64_t)1 << n;
  const int64_t c = (int64_t)1 << qc, t = (int64_t)1 << qt;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < dim; ++i) {
    if (!(i & c) || (i & t)) continue;
    cplx a0 = psi[i], a1 = psi[i | t];
    psi[i] = m[0] * a0 + m[1] * a1;
    psi[i | t] = m[2] * a0 + m[3] * a1;
  }
}

void or_evolve(int n, const int32_t* ops, int nops, double* psi_d, int init_zero) {
  cplx* psi = (cplx*)psi_d;
  const int64_t dim = (int64_t)1 << n;
  if (init_zero) {
    memset(psi, 0, sizeof(cplx) * dim);
    psi[0] = 1.0;
  }
  for (int g = 0; g < nops; ++g) {
    int code = ops[3 * g], q1 = ops[3 * g + 1], q2 = ops[3 * g + 2];
    if (code == OR_CZ) {
      apply_cz(psi, n, q1, q2);
    } else if (code == OR_CX) {
      apply_cx(psi, n, q1, q2);
    } else if (code == OR_CT || code == OR_CY2) {
      cplx m[4];
      gate_matrix(code == OR_CT ? OR_T : OR_Y2, m);
      apply_cu(psi, n, q1, q2, m);
    } else {
      cplx m[4];
      gate_matrix(code, m);
      apply_1q(psi, n, q1, m);
    }
  }
}

/*
 * Reconstruction over copies k in [k_begin, k_end):
 *   out[i_l * n_sel_u + i_u] (+)= sum_k U_k[sel_u[i_u]] * L_k[sel_l[i_l]]
 * The half gate lists carry cut slots: code -1 means "P_{l_m} on q1" (the control
 * side, m = q2), code -2 means "Z^{l_m} on q1" and code -3 "X^{l_m} on q1" (the
 * target side of a cut CZ or CX), code -100 - u "U^{l_m} on q1" with U the gate of
 * code u (the target side of a cut controlled T or Y^1/2), with l_m = bit m of k
 * (Supplementary A, Eqs. 1, 7-8).  If accumulate is 0 the output is
 * cleared first.  The sum over k is taken in ascending k for every output.
 */
static int resolve(const int32_t* tmpl, int ntmpl, uint64_t k, int32_t* out) {
  int n = 0;
  for (int g = 0; g < ntmpl; ++g) {
    int code = tmpl[3 * g], q1 = tmpl[3 * g + 1], q2 = tmpl[3 * g + 2];
    if (code == -1) {
      int bitv = (int)((k >> q2) & 1u);
      out[3 * n] = bitv ? OR_P1 : OR_P0; out[3 * n + 1] = q1; out[3 * n + 2] = 0; ++n;
    } else if (code == -2) {
      if ((k >> q2) & 1u) { out[3 * n] = OR_Z; out[3 * n + 1] = q1; out[3 * n + 2] = 0; ++n; }
    } else if (code == -3) {
      if ((k >> q2) & 1u) { out[3 * n] = OR_X; out[3 * n + 1] = q1; out[3 * n + 2] = 0; ++n; }
    } else if (code <= -100) {
      if ((k >> q2) & 1u) { out[3 * n] = -100 - code; out[3 * n + 1] = q1; out[3 * n + 2] = 0; ++n; }
    } else {
      out[3 * n] = code; out[3 * n + 1] = q1; out[3 * n + 2] = q2; ++n;
    }
  }
  return n;
}

int or_cut_sum(int n_u, const int32_t* up_tmpl, int n_up,
               int n_l, const int32_t* lo_tmpl, int n_lo,
               uint64_t k_begin, uint64_t k_end,
               const uint64_t* sel_u, int64_t n_sel_u,
               const uint64_t* sel_l, int64_t n_sel_l,
               int accumulate, double* out_d) {
  cplx* out = (cplx*)out_d;
  const int64_t nout = n_sel_u * n_sel_l;
  if (!accumulate) memset(out, 0, sizeof(cplx) * nout);
  cplx* U = (cplx*)malloc(sizeof(cplx) * ((size_t)1 << n_u));
  cplx* L = (cplx*)malloc(sizeof(cplx) * ((size_t)1 << n_l));
  cplx* us = (cplx*)malloc(sizeof(cplx) * (size_t)n_sel_u);
  cplx* ls = (cplx*)malloc(sizeof(cplx) * (size_t)n_sel_l);
  int32_t* up = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(n_up + 1));
  int32_t* lo = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(n_lo + 1));
  if (!U || !L || !us || !ls || !up || !lo) {
    free(U); free(L); free(us); free(ls); free(up); free(lo);
    return -1;
  }
  for (uint64_t k = k_begin; k < k_end; ++k) {
    int nu = resolve(up_tmpl, n_up, k, up);
    int nl = resolve(lo_tmpl, n_lo, k, lo);
    or_evolve(n_u, up, nu, (double*)U, 1);
    or_evolve(n_l, lo, nl, (double*)L, 1);
    for (int64_t i = 0; i < n_sel_u; ++i) us[i] = U[sel_u[i]];
    for (int64_t i = 0; i < n_sel_l; ++i) ls[i] = L[sel_l[i]];
#pragma omp parallel for schedule(static)
    for (int64_t il = 0; il < n_sel_l; ++il)
      for (int64_t iu = 0; iu < n_sel_u; ++iu)
        out[il * n_sel_u + iu] += us[iu] * ls[il];
  }
  free(U); free(L); free(us); free(ls); free(up); free(lo);
  return 0;
}

/* One half-state of copy k (for per-copy checks of the GPU half-states). */
int or_half_state(int n_h, const int32_t* tmpl, int ntmpl, uint64_t k, double* psi_d) {
  int32_t* ops = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(ntmpl + 1));
  if (!ops) return -1;
  int nops = resolve(tmpl, ntmpl, k, ops);
  or_evolve(n_h, ops, nops, psi_d, 1);
  free(ops);
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
