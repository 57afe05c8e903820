// Shared host/device pieces: Philox4x64-10, the per-trajectory noise draws,
// and the fusion of one block's ops into its Kraus pair.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "program.hpp"

namespace qec {

#if defined(__CUDACC__)
#define QEC_HD __host__ __device__ __forceinline__
#else
#define QEC_HD inline
#endif

// ---- Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3) -------------------------
struct U64x4 { uint64_t v[4]; };

QEC_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
#endif
}

QEC_HD U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    uint64_t hi0 = mulhi64(M0, c0), lo0 = M0 * c0;
    uint64_t hi1 = mulhi64(M1, c2), lo1 = M1 * c2;
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  U64x4 o;
  o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

enum : uint64_t { TAG_NOISE = 0, TAG_MEASURE = 1, TAG_READOUT = 3, TAG_TWIRL = 4 };

// Counter (trajectory, round, step << 32 | site, tag), key (seed, 0).
QEC_HD U64x4 draw(uint64_t seed, uint64_t traj, uint64_t rnd, uint32_t step, uint32_t site, uint64_t tag) {
  return philox4x64_10(traj, rnd, ((uint64_t)step << 32) | site, tag, seed, 0);
}

QEC_HD double uniform53(uint64_t w) { return (double)(w >> 11) * (1.0 / 9007199254740992.0); }

// Noise draw at one site: 0 = none; N1: 1..3 = X, Y, Z; N2: k = 1..15, ancilla Pauli k>>2, data Pauli k&3.
QEC_HD int noise_code(const ProgOp& op, double p, uint64_t seed, uint64_t traj, uint64_t rnd) {
  U64x4 w = draw(seed, traj, rnd, op.step, op.site, TAG_NOISE);
  if (!(uniform53(w.v[0]) < p)) return 0;
  uint64_t hi = w.v[1] >> 32;
  if (op.kind == OP_N1) return (int)((hi * 3ull) >> 32) + 1;
  return (int)((hi * 15ull) >> 32) + 1;
}

// Twirled coherent term (OP_T1 / OP_T2): fires with probability p (site field factor << 24 | site).
QEC_HD bool twirl_fires(const ProgOp& op, double p, uint64_t seed, uint64_t traj, uint64_t rnd) {
  U64x4 w = draw(seed, traj, rnd, op.step, op.site, TAG_TWIRL);
  return uniform53(w.v[0]) < p;
}

// ---- block fusion -----------------------------------------------------------------------
// U holds the block unitary restricted to ancilla-|0> inputs: rows r in [0, 2^(w+1)),
// columns c in [0, 2^w), row stride 16, local bit w = ancilla.
QEC_HD int64_t ins0(int64_t k, int b) { return ((k >> b) << (b + 1)) | (k & ((1ll << b) - 1)); }

QEC_HD int items_1q(int w) { return (1 << w) * (1 << w); }
QEC_HD int items_2q(int w) { return (1 << (w - 1)) * (1 << w); }

QEC_HD void apply1_item(double2* U, int w, int b, const double (*m)[2], int item) {
  const int C = 1 << w;
  int c = item % C, pr = item / C;
  int r0 = (int)ins0(pr, b), r1 = r0 | (1 << b);
  double2 x = U[r0 * 16 + c], y = U[r1 * 16 + c];
  double2 o0, o1;
  o0.x = m[0][0] * x.x - m[0][1] * x.y + m[1][0] * y.x - m[1][1] * y.y;
  o0.y = m[0][0] * x.y + m[0][1] * x.x + m[1][0] * y.y + m[1][1] * y.x;
  o1.x = m[4][0] * x.x - m[4][1] * x.y + m[5][0] * y.x - m[5][1] * y.y;
  o1.y = m[4][0] * x.y + m[4][1] * x.x + m[5][0] * y.y + m[5][1] * y.x;
  U[r0 * 16 + c] = o0;
  U[r1 * 16 + c] = o1;
}

// Two-qubit matrix on local index 2*bit(a) + bit(b).
QEC_HD void apply2_item(double2* U, int w, int a, int b, const double (*m)[2], int item) {
  const int C = 1 << w;
  int c = item % C, qd = item / C;
  int lo = a < b ? a : b, hi = a < b ? b : a;
  int base = (int)ins0(ins0(qd, lo), hi);
  int idx[4];
  double2 x[4];
  for (int l = 0; l < 4; ++l) {
    idx[l] = base | ((l >> 1) << a) | ((l & 1) << b);
    x[l] = U[idx[l] * 16 + c];
  }
  for (int r = 0; r < 4; ++r) {
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < 4; ++k) {
      double mr = m[4 * r + k][0], mi = m[4 * r + k][1];
      sr += mr * x[k].x - mi * x[k].y;
      si += mr * x[k].y + mi * x[k].x;
    }
    U[idx[r] * 16 + c] = make_double2(sr, si);
  }
}

}  // namespace qec
