/*
 * Plain FP64 state-vector executor for the oracle.  Test infrastructure only:
 * only tests, the smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * State: 2^n complex amplitudes, interleaved (re, im) doubles; qubit q is bit q
 * of the basis index.  Each op is applied on its own, one full pass per op, in
 * the order given (the circuit of Sec. III.A with the noise of Eqs. 1-2 and the
 * coherent terms, unrolled into unitaries and measurements by circuit.py).
 * Measurement follows the Born rule: P(1) = sum over bit q = 1 of |a|^2 divided
 * by the total, outcome 1 iff u < P(1); the kept half is renormalised, the
 * other half zeroed, and a reset moves the kept half to bit q = 0 (Sec. II.B:
 * the measured qubit is reused).  Probability sums are taken over fixed chunks
 * and the chunk sums added in order, so results do not depend on thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int32_t type;   /* 1: one-qubit unitary, 2: two-qubit unitary, 3: measurement */
  int32_t q0;     /* qubit (type 1, 3) or first-listed qubit (type 2) */
  int32_t q1;     /* second qubit (type 2); reset flag (type 3) */
  int32_t flag;   /* type 3: forced outcome (0/1) or -1 to sample with u */
  double u;       /* type 3: uniform in [0, 1) */
  double m[32];   /* row-major complex matrix, (re, im) pairs */
} sv_op;

#define CHUNK 4096

void sv_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

int sv_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* index with a zero bit inserted at position q */
static inline int64_t ins0(int64_t k, int q) {
  int64_t lo = k & ((1LL << q) - 1);
  return ((k >> q) << (q + 1)) | lo;
}

void sv_apply1(double* psi, int n, int q, const double* m) {
  int64_t half = 1LL << (n - 1);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < half; ++k) {
    int64_t i0 = ins0(k, q), i1 = i0 | (1LL << q);
    double ar = psi[2 * i0], ai = psi[2 * i0 + 1];
    double br = psi[2 * i1], bi = psi[2 * i1 + 1];
    psi[2 * i0] = m[0] * ar - m[1] * ai + m[2] * br - m[3] * bi;
    psi[2 * i0 + 1] = m[0] * ai + m[1] * ar + m[2] * bi + m[3] * br;
    psi[2 * i1] = m[4] * ar - m[5] * ai + m[6] * br - m[7] * bi;
    psi[2 * i1 + 1] = m[4] * ai + m[5] * ar + m[6] * bi + m[7] * br;
  }
}

void sv_apply2(double* psi, int n, int qa, int qb, const double* m) {
  int lo = qa < qb ? qa : qb, hi = qa < qb ? qb : qa;
  int64_t quarter = 1LL << (n - 2);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < quarter; ++k) {
    int64_t base = ins0(ins0(k, lo), hi);
    int64_t idx[4];
    double xr[4], xi[4];
    for (int l = 0; l < 4; ++l) {   /* local index l = 2*bit(qa) + bit(qb) */
      idx[l] = base | ((int64_t)(l >> 1) << qa) | ((int64_t)(l & 1) << qb);
      xr[l] = psi[2 * idx[l]];
      xi[l] = psi[2 * idx[l] + 1];
    }
    for (int r = 0; r < 4; ++r) {
      double sr = 0.0, si = 0.0;
      for (int c = 0; c < 4; ++c) {
        double mr = m[2 * (4 * r + c)], mi = m[2 * (4 * r + c) + 1];
        sr += mr * xr[c] - mi * xi[c];
        si += mr * xi[c] + mi * xr[c];
      }
      psi[2 * idx[r]] = sr;
      psi[2 * idx[r] + 1] = si;
    }
  }
}

/* Returns the outcome, or -1 if the kept branch has zero probability. */
int sv_measure(double* psi, int n, int q, double u, int forced, int reset, double* probs) {
  int64_t half = 1LL << (n - 1);
  int64_t nchunk = (half + CHUNK - 1) / CHUNK;
  double* part = (double*)malloc(sizeof(double) * 2 * (size_t)nchunk);
  if (!part) return -2;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nchunk; ++c) {
    double s0 = 0.0, s1 = 0.0;
    int64_t end = (c + 1) * CHUNK < half ? (c + 1) * CHUNK : half;
    for (int64_t k = c * CHUNK; k < end; ++k) {
      int64_t i0 = ins0(k, q), i1 = i0 | (1LL << q);
      s0 += psi[2 * i0] * psi[2 * i0] + psi[2 * i0 + 1] * psi[2 * i0 + 1];
      s1 += psi[2 * i1] * psi[2 * i1] + psi[2 * i1 + 1] * psi[2 * i1 + 1];
    }
    part[2 * c] = s0;
    part[2 * c + 1] = s1;
  }
  double p0 = 0.0, p1 = 0.0;
  for (int64_t c = 0; c < nchunk; ++c) { p0 += part[2 * c]; p1 += part[2 * c + 1]; }
  free(part);
  double prob1 = p1 / (p0 + p1);
  probs[0] = p0;
  probs[1] = p1;
  probs[2] = prob1;
  int out = forced >= 0 ? forced : (u < prob1 ? 1 : 0);
  double keep = out ? p1 : p0;
  if (!(keep > 0.0)) return -1;
  double s = 1.0 / sqrt(keep);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < half; ++k) {
    int64_t i0 = ins0(k, q), i1 = i0 | (1LL << q);
    int64_t ik = out ? i1 : i0, iz = out ? i0 : i1;
    double kr = psi[2 * ik] * s, ki = psi[2 * ik + 1] * s;
    psi[2 * iz] = 0.0;
    psi[2 * iz + 1] = 0.0;
    psi[2 * ik] = kr;
    psi[2 * ik + 1] = ki;
    if (reset && out) {           /* X on the measured qubit: move the kept half to bit q = 0 */
      psi[2 * i0] = kr;
      psi[2 * i0 + 1] = ki;
      psi[2 * i1] = 0.0;
      psi[2 * i1 + 1] = 0.0;
    }
  }
  return out;
}

/* Run ops in order.  For every measurement op, writes its outcome and P(1)
 * into outcomes[] / p1s[] (in op order).  Returns the number of measurements,
 * or -(index+1) of the first measurement whose kept branch had zero weight. */
int64_t sv_run(double* psi, int n, const sv_op* ops, int64_t nops, int32_t* outcomes, double* p1s) {
  int64_t nm = 0;
  for (int64_t i = 0; i < nops; ++i) {
    const sv_op* o = &ops[i];
    if (o->type == 1) {
      sv_apply1(psi, n, o->q0, o->m);
    } else if (o->type == 2) {
      sv_apply2(psi, n, o->q0, o->q1, o->m);
    } else if (o->type == 3) {
      double pr[3];
      int r = sv_measure(psi, n, o->q0, o->u, o->flag, o->q1, pr);
      if (r < 0) return -(i + 1);
      outcomes[nm] = r;
      p1s[nm] = pr[2];
      ++nm;
    }
  }
  return nm;
}
