// Batched form: many small-register trajectories in one persistent launch.
//
// One warp simulates one trajectory of the d = 3 delayed-measurement register
// (9 data qubits + the reused ancilla, Sec. II.B) entirely in shared memory:
// per stabilizer block it draws the trajectory's noise, fuses the block's ops
// into its Kraus pair (as k_instantiate does), measures the ancilla (FP64
// accumulated probability, on-warp outcome), collapses and renormalises, and
// at the end samples the final Z readout.  Warps take trajectories from a
// global work counter, so complex128 and complex64 trajectories and
// different noise parameters mix freely in one launch.  Each trajectory's
// noise (p, angles) is an input array; the circuit program is built once with
// every noise and coherent slot present (a zero angle or probability then
// acts as the identity / never fires).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/qecsv.h"
#include "common.cuh"
#include "kernels.hpp"
#include "program.hpp"

using namespace qec;

namespace {

constexpr int kD = 3;                    // register of the batched form: d = 3
constexpr int kND = kD * kD;             // 9 data qubits
constexpr int kNAmp = 1 << kND;          // 512 amplitudes
constexpr int kNStab = kND - 1;          // 8 stabilizers
constexpr int kWarpSmem = 32 * 16 * 16 + kNAmp * 16 + M_COUNT * 16 * 16 + 16 * 16 + 64;   // U, psi, mats, pending factor, misc (c128)
constexpr int kUMaxFusionDecl = 6;       // widest pass of the unreduced engine (slab bits)

template <typename T> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float> { using t = float2; };

struct BatchCtl {
  uint64_t seed;
  uint32_t n;                 // reduced-register (10-qubit) trajectories in this run
  unsigned int counter;       // their work queue head (zeroed before every run)
  uint32_t n_u;               // unreduced-register (17-qubit) trajectories in this run
  unsigned int counter_u;     // their work queue head
  uint32_t snap_item;         // item whose final data-register state goes to snap (~0u = none)
};

// One pass of the unreduced engine over the slab: kind 0 applies the units punits[u0, u1) (disjoint
// slab bits, together `nbits` bits listed in bits[]); kind 1 measures the ancilla of items[item].
struct UPass {
  int32_t kind;
  int32_t item;
  int32_t u0, u1;
  int32_t nbits;
  int32_t bits[kUMaxFusionDecl];
};

// A unit inside a pass: items[item] on slab bits qa (, qb), and the pass's other bits.  A two-qubit
// unit also carries the one-qubit units folded into its matrix: entries abs0 .. abs0 + nabs - 1 of
// the program's UAbs list.
struct UPassUnit {
  int32_t item;
  int32_t nq, qa, qb;
  int32_t nother;
  int32_t other[kUMaxFusionDecl];
  int32_t abs0, nabs;
};

// A one-qubit unit folded into a two-qubit unit's matrix: item1's matrix on the unit's local bit
// (mode bit 1: 1 = qa, 0 = qb), multiplied from the left (mode bit 0 = 1: it follows the unit) or
// from the right (it precedes).  A unit's entries list the right factors latest first, then the
// left factors in program order.
struct UAbs {
  int32_t item1;
  int32_t mode;
};

struct BatchArgs {
  const ProgOp* ops;          // noisy program (all slots present)
  const BlockInfo* blocks;
  const ProgOp* iops;         // init program
  const BlockInfo* iblocks;
  const double* mats;         // static matrices [M_COUNT][16][2] (coherent entries overwritten per trajectory)
  const qec_noise* noise;     // [n]
  const int32_t* kind;        // [n]: bit 0 = complex64 (else complex128), bit 1 = unreduced register
  const uint32_t* idx;        // reduced-register items of this run
  const uint32_t* idx_u;      // unreduced-register items of this run
  const ProgOp* uops;         // unreduced time-ordered program (one round)
  const UItem* uitems;
  int n_uitems;
  const ProgOp* iuops;        // its noise-free init round
  const UItem* iuitems;
  int n_iuitems;
  const void* psi0_u[2];      // unreduced init slab per precision
  const UPass* upasses;       // its passes for one round (fusion width of the batch)
  int n_upasses;
  const UPassUnit* upunits;
  const UPass* iupasses;      // the init round's passes
  int n_iupasses;
  const UPassUnit* iupunits;
  int n_upunits, n_iupunits;
  const UAbs* uabs;           // one-qubit units folded into two-qubit units (noisy round, init round)
  const UAbs* iuabs;
  const uint64_t* traj;       // [n]
  BatchCtl* ctl;
  int rounds;
  const void* psi0[2];        // init code state per precision
  uint8_t* syn;               // [n][rounds+1][8]
  uint8_t* bits;              // [n][9]
  uint8_t* logical;           // [n]
  double2* snap;              // [512] data-register state of ctl->snap_item after its last round
  int init_mode;              // 1: compute the init state of precision init_prec into init_out
  int init_prec;
  void* init_out;
};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T2>
__device__ __forceinline__ T2 mk(double re, double im) {
  T2 r;
  r.x = (decltype(r.x))re;
  r.y = (decltype(r.y))im;
  return r;
}

template <typename T, typename T2>
__device__ __forceinline__ T2 cmul_add(T2 acc, T2 a, T2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}

// Per-trajectory coherent matrices (same conventions as the program builder).
// Per-trajectory probabilities: p1, p2, p_idle and the twirl probabilities (0 unless twirled).
__device__ void traj_probs(const qec_noise& nz, double* prob) {
  const bool on = nz.twirl != 0.0;
  prob[PR_P1] = nz.p1;
  prob[PR_P2] = nz.p2;
  prob[PR_IDLE] = nz.p_idle;
  auto half = [&](double th) { const double s = sin(th / 2); return on ? s * s : 0.0; };
  prob[PR_TW_RX] = half(nz.theta_rx);
  prob[PR_TW_RZ] = half(nz.theta_rz);
  prob[PR_TW_RZX] = half(nz.theta_rzx);
  prob[PR_TW_ZZ] = on ? sin(nz.phi_zz) * sin(nz.phi_zz) : 0.0;
  prob[PR_TW_ROUND_RZ] = half(nz.round_rz);
  prob[PR_TW_ROUND_RX] = half(nz.round_rx);
}

// Per-trajectory coherent matrices; identities when the trajectory's coherent terms are twirled
// (the program holds both forms of every term).
template <typename T2>
__device__ void coherent_mats(T2 (*m)[16], qec_noise nz, int lane) {
  if (lane != 0) return;
  if (nz.twirl != 0.0) nz.theta_rx = nz.theta_rz = nz.theta_rzx = nz.phi_zz = nz.round_rz = nz.round_rx = 0.0;
  auto clear = [&](int id) { for (int i = 0; i < 16; ++i) m[id][i] = mk<T2>(0, 0); };
  auto rot1 = [&](int id, bool x, double th) {
    clear(id);
    const double c = cos(th / 2), s = sin(th / 2);
    if (x) { m[id][0] = mk<T2>(c, 0); m[id][1] = mk<T2>(0, -s); m[id][4] = mk<T2>(0, -s); m[id][5] = mk<T2>(c, 0); }
    else { m[id][0] = mk<T2>(c, -s); m[id][5] = mk<T2>(c, s); }
  };
  rot1(M_ROT_RX, true, nz.theta_rx);
  rot1(M_ROT_RXP, true, nz.overrot_follows != 0.0 ? -nz.theta_rx : nz.theta_rx);
  rot1(M_ROT_RZ, false, nz.theta_rz);
  rot1(M_ROUND_RZ, false, nz.round_rz);
  rot1(M_ROUND_RX, true, nz.round_rx);
  clear(M_ROT_RZX);
  {
    const double c = cos(nz.theta_rzx / 2), s = sin(nz.theta_rzx / 2);
    for (int r = 0; r < 4; ++r) {
      m[M_ROT_RZX][5 * r] = mk<T2>(c, 0);
      const int a = r >> 1, b = r & 1, col = (a << 1) | (b ^ 1);
      m[M_ROT_RZX][4 * r + col] = mk<T2>(0, -s * (a ? -1.0 : 1.0));
    }
  }
  clear(M_ZZ);
  for (int r = 0; r < 4; ++r) {
    const double zz = ((r >> 1) ^ (r & 1)) ? -1.0 : 1.0, ph = -nz.phi_zz * zz;
    m[M_ZZ][5 * r] = mk<T2>(cos(ph), sin(ph));
  }
}

template <typename T, typename T2>
__device__ void apply1_w(T2* U, int w, int b, const T2* m, int lane) {
  const int C = 1 << w;
  for (int it = lane; it < C * C; it += 32) {
    const int c = it % C, pr = it / C;
    const int r0 = (int)ins0(pr, b), r1 = r0 | (1 << b);
    const T2 x = U[r0 * 16 + c], y = U[r1 * 16 + c];
    T2 o0 = mk<T2>(0, 0), o1 = mk<T2>(0, 0);
    o0 = cmul_add<T>(o0, m[0], x); o0 = cmul_add<T>(o0, m[1], y);
    o1 = cmul_add<T>(o1, m[4], x); o1 = cmul_add<T>(o1, m[5], y);
    U[r0 * 16 + c] = o0;
    U[r1 * 16 + c] = o1;
  }
  __syncwarp();
}

template <typename T, typename T2>
__device__ void apply2_w(T2* U, int w, int a, int b, const T2* m, int lane) {
  const int C = 1 << w;
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  for (int it = lane; it < (C / 2) * C; it += 32) {
    const int c = it % C, qd = it / C;
    const int base = (int)ins0(ins0(qd, lo), hi);
    int idx[4];
    T2 x[4];
    for (int l = 0; l < 4; ++l) {
      idx[l] = base | ((l >> 1) << a) | ((l & 1) << b);
      x[l] = U[idx[l] * 16 + c];
    }
    for (int r = 0; r < 4; ++r) {
      T2 acc = mk<T2>(0, 0);
      for (int k = 0; k < 4; ++k) acc = cmul_add<T>(acc, m[4 * r + k], x[k]);
      U[idx[r] * 16 + c] = acc;
    }
  }
  __syncwarp();
}

// Ancilla measurement of one block on the warp's register: A = sum |K1 v|^2, N = sum |v|^2
// (FP64 accumulated), outcome u < A / N (forced to the offset in the init round), then
// v <- K_m v / sqrt(N) in place.  Returns the raw outcome.
template <typename T, int W>
__device__ int measure_block(typename C2<T>::t* psi, const typename C2<T>::t* U, const BlockInfo& bi, bool init,
                             uint64_t seed, uint64_t traj, int rnd, int k, int lane) {
  using T2 = typename C2<T>::t;
  constexpr int C = 1 << W, G = kNAmp >> W;
  int q[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) q[j] = j < W ? bi.q[j] : 0;
  uint32_t off[C];
#pragma unroll
  for (int l = 0; l < C; ++l) {
    uint32_t o = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) o |= (uint32_t)((l >> j) & 1) << q[j];
    off[l] = o;
  }
  double A = 0.0, N = 0.0;
  for (int g = lane; g < G; g += 32) {
    uint32_t base = g;
#pragma unroll
    for (int j = 0; j < W; ++j) base = (uint32_t)ins0(base, q[j]);
    T2 v[C];
#pragma unroll
    for (int l = 0; l < C; ++l) {
      v[l] = psi[base + off[l]];
      N += (double)v[l].x * v[l].x + (double)v[l].y * v[l].y;
    }
#pragma unroll
    for (int r = 0; r < C; ++r) {
      T2 acc = mk<T2>(0, 0);
#pragma unroll
      for (int c = 0; c < C; ++c) acc = cmul_add<T>(acc, U[(C + r) * 16 + c], v[c]);
      A += (double)acc.x * acc.x + (double)acc.y * acc.y;
    }
  }
  A = wsum(A);
  N = wsum(N);
  int m;
  if (init) {
    m = bi.offset;
  } else {
    const double u = uniform53(draw(seed, traj, (uint64_t)rnd, 0u, (uint32_t)(kND + k), TAG_MEASURE).v[0]);
    m = u < A / N ? 1 : 0;
  }
  const double scale = 1.0 / sqrt(N);
  for (int g = lane; g < G; g += 32) {
    uint32_t base = g;
#pragma unroll
    for (int j = 0; j < W; ++j) base = (uint32_t)ins0(base, q[j]);
    T2 v[C];
#pragma unroll
    for (int l = 0; l < C; ++l) v[l] = psi[base + off[l]];
#pragma unroll
    for (int r = 0; r < C; ++r) {
      T2 acc = mk<T2>(0, 0);
#pragma unroll
      for (int c = 0; c < C; ++c) acc = cmul_add<T>(acc, U[(m * C + r) * 16 + c], v[c]);
      psi[base + off[r]] = mk<T2>((double)acc.x * scale, (double)acc.y * scale);
    }
  }
  __syncwarp();
  return m;
}

// A block's compile folds consecutive ops on the same qubits into one pending factor before it
// touches the 32 x 16 block matrix U: a 2x2 on one qubit (pb < 0; entries 0, 1, 4, 5 of P) or a 4x4
// on a qubit pair (local index 2 bit(pa) + bit(pb)).  An op on other qubits first applies the
// pending factor to U.  The product is the same operator as the ops applied one at a time.
template <typename T>
struct PendingOp {
  using T2 = typename C2<T>::t;
  T2* P;        // [16], the warp's pending factor
  int pa = -1, pb = -1;
  int lane;
  static __device__ __forceinline__ int sw(int i) { return ((i & 1) << 1) | (i >> 1); }
  // P <- G P for a 4x4 G (qubit order of G swapped against P's when swap)
  __device__ void lmul2(const T2* g, bool swap) {
    T2 acc = mk<T2>(0, 0);
    if (lane < 16) {
      const int r = lane >> 2, c = lane & 3;
#pragma unroll
      for (int k = 0; k < 4; ++k) acc = cmul_add<T>(acc, g[4 * (swap ? sw(r) : r) + (swap ? sw(k) : k)], P[4 * k + c]);
    }
    __syncwarp();
    if (lane < 16) P[lane] = acc;
    __syncwarp();
  }
  // P <- (g on local bit) P for a 2x2 g (entries 0, 1, 4, 5), P a 4x4 (dim 4) or a 2x2 (dim 2)
  __device__ void lmul1(const T2* g, int bit, int dim) {
    T2 acc = mk<T2>(0, 0);
    const int r = lane >> 2, c = lane & 3;
    const bool on = dim == 4 ? lane < 16 : (r < 2 && c < 2);
    if (on) {
      const int rb = (r >> bit) & 1, r0 = r & ~(1 << bit), r1 = r | (1 << bit);
      acc = cmul_add<T>(acc, g[4 * rb], P[4 * r0 + c]);
      acc = cmul_add<T>(acc, g[4 * rb + 1], P[4 * r1 + c]);
    }
    __syncwarp();
    if (on) P[lane] = acc;
    __syncwarp();
  }
  __device__ void flush(T2* U, int w) {
    if (pa < 0) return;
    if (pb < 0) apply1_w<T>(U, w, pa, P, lane);
    else apply2_w<T>(U, w, pa, pb, P, lane);
    pa = pb = -1;
  }
  __device__ void start(const T2* g, int x, int y) {   // P <- g (a 4x4 on (x, y), or a 2x2 on x when y < 0)
    if (lane < 16) P[lane] = g[lane];
    __syncwarp();
    pa = x;
    pb = y;
  }
  __device__ void one(T2* U, int w, int x, const T2* g) {
    if (pa == x && pb < 0) {
      lmul1(g, 0, 2);
    } else if (pb >= 0 && (x == pa || x == pb)) {
      lmul1(g, x == pa ? 1 : 0, 4);
    } else {
      flush(U, w);
      start(g, x, -1);
    }
  }
  __device__ void two(T2* U, int w, int x, int y, const T2* g) {
    if (pb >= 0 && ((x == pa && y == pb) || (x == pb && y == pa))) {
      lmul2(g, x != pa);
      return;
    }
    if (pb < 0 && pa >= 0 && (x == pa || y == pa)) {
      // the pending one-qubit factor becomes a 4x4 on (x, y): Q on its bit, the identity on the other
      const int bit = x == pa ? 1 : 0;
      T2 q00 = P[0], q01 = P[1], q10 = P[4], q11 = P[5];
      __syncwarp();
      if (lane < 16) {
        const int r = lane >> 2, c = lane & 3;
        const int ob = 1 - bit;
        T2 v = mk<T2>(0, 0);
        if (((r >> ob) & 1) == ((c >> ob) & 1)) {
          const int rb = (r >> bit) & 1, cb = (c >> bit) & 1;
          v = rb ? (cb ? q11 : q10) : (cb ? q01 : q00);
        }
        P[lane] = v;
      }
      __syncwarp();
      pa = x;
      pb = y;
      lmul2(g, false);
      return;
    }
    flush(U, w);
    start(g, x, y);
  }
};

// One trajectory (or, in init mode, the noise-free init round) on one warp.
template <typename T>
__device__ void run_warp(const BatchArgs& a, unsigned char* wsm, uint32_t item) {
  using T2 = typename C2<T>::t;
  const int lane = threadIdx.x & 31;
  T2* U = reinterpret_cast<T2*>(wsm);
  T2* psi = U + 32 * 16;
  T2 (*mats)[16] = reinterpret_cast<T2 (*)[16]>(psi + kNAmp);
  PendingOp<T> pend;
  pend.P = reinterpret_cast<T2*>(mats + M_COUNT);
  pend.lane = lane;
  const bool init = a.init_mode != 0;
  const qec_noise nz = init ? qec_noise{} : a.noise[item];
  const uint64_t traj = init ? 0ull : a.traj[item];
  const ProgOp* ops = init ? a.iops : a.ops;
  const BlockInfo* blocks = init ? a.iblocks : a.blocks;
  for (int i = lane; i < M_COUNT * 16; i += 32) {
    const int id = i / 16, e = i % 16;
    mats[id][e] = mk<T2>(a.mats[(id * 16 + e) * 2], a.mats[(id * 16 + e) * 2 + 1]);
  }
  __syncwarp();
  if (!init) coherent_mats(mats, nz, lane);
  double prob[PR_COUNT];
  traj_probs(nz, prob);
  if (init) {
    for (int i = lane; i < kNAmp; i += 32) psi[i] = mk<T2>(i == 0 ? 1.0 : 0.0, 0.0);
  } else {
    const T2* p0 = reinterpret_cast<const T2*>(a.psi0[a.kind[item] & 1]);
    for (int i = lane; i < kNAmp; i += 32) psi[i] = p0[i];
  }
  __syncwarp();
  const int r_first = init ? 0 : 1, r_last = init ? 0 : a.rounds;
  uint8_t* syn = init ? nullptr : a.syn + (size_t)item * (a.rounds + 1) * kNStab;
  if (syn)
    for (int k = lane; k < kNStab; k += 32) syn[k] = 0;
  for (int rnd = r_first; rnd <= r_last; ++rnd) {
    for (int k = 0; k < kNStab; ++k) {
      const BlockInfo bi = blocks[k];
      const int w = bi.w, C = 1 << w;
      for (int i = lane; i < 32 * 16; i += 32) U[i] = mk<T2>((i / 16 < C && i / 16 == i % 16) ? 1.0 : 0.0, 0.0);
      __syncwarp();
      for (int oi = bi.op_begin; oi < bi.op_end; ++oi) {
        const ProgOp op = ops[oi];
        if (op.kind == OP_T1 || op.kind == OP_T2) {
          int fire = 0;
          if (lane == 0) fire = twirl_fires(op, prob[op.pidx], a.ctl->seed, traj, (uint64_t)rnd) ? 1 : 0;
          fire = __shfl_sync(0xffffffffu, fire, 0);
          if (!fire) continue;
          if (op.kind == OP_T1) pend.one(U, w, op.q0, mats[op.mat]);
          else pend.two(U, w, op.q0, op.q1, mats[op.mat]);
          continue;
        }
        if (op.kind == OP_N1 || op.kind == OP_N2) {
          int code = 0;
          if (lane == 0) code = noise_code(op, prob[op.pidx], a.ctl->seed, traj, (uint64_t)rnd);
          code = __shfl_sync(0xffffffffu, code, 0);
          if (!code) continue;
          if (op.kind == OP_N1) {
            pend.one(U, w, op.q0, mats[code]);
          } else {
            if (code >> 2) pend.one(U, w, op.q0, mats[code >> 2]);
            if (code & 3) pend.one(U, w, op.q1, mats[code & 3]);
          }
        } else if (op.kind == OP_U1) {
          pend.one(U, w, op.q0, mats[op.mat]);
        } else {
          pend.two(U, w, op.q0, op.q1, mats[op.mat]);
        }
      }
      pend.flush(U, w);
      int m;
      if (w == 4) m = measure_block<T, 4>(psi, U, bi, init, a.ctl->seed, traj, rnd, k, lane);
      else m = measure_block<T, 2>(psi, U, bi, init, a.ctl->seed, traj, rnd, k, lane);
      if (syn && lane == 0) syn[rnd * kNStab + k] = (uint8_t)(m ^ bi.offset);
    }
  }
  if (init) {
    T2* out = reinterpret_cast<T2*>(a.init_out);
    for (int i = lane; i < kNAmp; i += 32) out[i] = psi[i];
    return;
  }
  if (item == a.ctl->snap_item)
    for (int i = lane; i < kNAmp; i += 32) a.snap[i] = make_double2((double)psi[i].x, (double)psi[i].y);
  // final Z readout: qubit j gets [u_j < P(q_j = 1 | earlier outcomes)]
  uint8_t* bits = a.bits + (size_t)item * kND;
  uint32_t prefix = 0;
  for (int j = 0; j < kND; ++j) {
    const uint32_t mask = (1u << j) - 1u;
    double s_all = 0.0, s_one = 0.0;
    for (int x = lane; x < kNAmp; x += 32) {
      if ((x & mask) == prefix) {
        const double p = (double)psi[x].x * psi[x].x + (double)psi[x].y * psi[x].y;
        s_all += p;
        if ((x >> j) & 1) s_one += p;
      }
    }
    s_all = wsum(s_all);
    s_one = wsum(s_one);
    const double u = uniform53(draw(a.ctl->seed, traj, (uint64_t)a.rounds + 1, 0u, (uint32_t)j, TAG_READOUT).v[0]);
    const int b = u < s_one / s_all ? 1 : 0;
    prefix |= (uint32_t)b << j;
    if (lane == 0) bits[j] = (uint8_t)b;
  }
  if (lane == 0) {
    int par = 0;
    for (int c = 0; c < kD; ++c) par ^= (int)((prefix >> c) & 1u);
    a.logical[item] = (uint8_t)par;
  }
}

__global__ void k_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char bsm[];
  const int warp = threadIdx.x >> 5;
  unsigned char* wsm = bsm + (size_t)warp * kWarpSmem;
  if (a.init_mode) {
    if (blockIdx.x == 0 && warp == 0) {
      if (a.init_prec == 0) run_warp<double>(a, wsm, 0);
      else run_warp<float>(a, wsm, 0);
    }
    return;
  }
  for (;;) {
    uint32_t pos = 0;
    if ((threadIdx.x & 31) == 0) pos = atomicAdd(&a.ctl->counter, 1u);
    pos = __shfl_sync(0xffffffffu, pos, 0);
    if (pos >= a.ctl->n) return;
    const uint32_t item = a.idx[pos];
    if ((a.kind[item] & 1) == 0) run_warp<double>(a, wsm, item);
    else run_warp<float>(a, wsm, item);
  }
}

// ---- unreduced register: one CTA per 17-qubit trajectory --------------------------------
// Each round's gate units (a gate with its coherent terms and sampled Paulis on 1 or 2 slab bits)
// are fused into their matrices at the start of the round, one thread per unit: the noise draws
// depend only on (seed, trajectory, round, step, site), not on the state.  The slab is then
// updated in passes: a pass holds consecutive units on disjoint slab bits (which commute), at most
// `fusion width` bits in all, and each thread applies every unit of the pass to whole groups of
// amplitudes (all combinations of the pass's bits) that it alone touches, so a pass needs one
// barrier however many units it holds.  Measurements are passes of their own.
constexpr int kUBits = kND + kNStab / 2;      // 13 slab bits: 9 data + the active part's 4 ancillas
constexpr int kUAmp = 1 << kUBits;            // 8192 amplitudes
constexpr int kUMaxItems = 192;               // items of one round (units and measurements)
// slab, mats, unit matrices (FP64) and flags, reduction, flag
constexpr int kUChunks = 256;                 // complex64 measurement: chunks of the 4096 amplitude pairs
constexpr int kUSmem = kUAmp * 16 + M_COUNT * 16 * 16 + kUMaxItems * 16 * 16 + kUMaxItems * 4 + 64 * 8 +
                       2 * kUChunks * 8 + 16;

template <typename T>
__device__ void block_sum2_u(double& x, double& y, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  x = wsum(x);
  y = wsum(y);
  __syncthreads();
  if (lane == 0) { sh[w] = x; sh[32 + w] = y; }
  __syncthreads();
  x = 0.0;
  y = 0.0;
  for (int i = 0; i < nw; ++i) { x += sh[i]; y += sh[32 + i]; }   // fixed order, same in every thread
  __syncthreads();
}

// Left-multiplies the DIM x DIM unit matrix M (row stride 4) by a one-qubit gate g on local bit BIT.
template <int DIM, int BIT, typename T2>
__device__ __forceinline__ void left1(double2 (&M)[16], const T2* g) {
  const double2 g00 = make_double2((double)g[0].x, (double)g[0].y), g01 = make_double2((double)g[1].x, (double)g[1].y);
  const double2 g10 = make_double2((double)g[4].x, (double)g[4].y), g11 = make_double2((double)g[5].x, (double)g[5].y);
#pragma unroll
  for (int r0 = 0; r0 < DIM; ++r0) {
    if (r0 & (1 << BIT)) continue;
    const int r1 = r0 | (1 << BIT);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const double2 x = M[r0 * 4 + c], y = M[r1 * 4 + c];
      M[r0 * 4 + c] = make_double2(g00.x * x.x - g00.y * x.y + g01.x * y.x - g01.y * y.y,
                                   g00.x * x.y + g00.y * x.x + g01.x * y.y + g01.y * y.x);
      M[r1 * 4 + c] = make_double2(g10.x * x.x - g10.y * x.y + g11.x * y.x - g11.y * y.y,
                                   g10.x * x.y + g10.y * x.x + g11.x * y.y + g11.y * y.x);
    }
  }
}

// Left-multiplies the 4x4 unit matrix M by a two-qubit gate g (local index 2 bit(qa) + bit(qb)).
template <typename T2>
__device__ __forceinline__ void left2(double2 (&M)[16], const T2* g) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double2 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = M[k * 4 + c];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double gx = (double)g[r * 4 + k].x, gy = (double)g[r * 4 + k].y;
        re += gx * v[k].x - gy * v[k].y;
        im += gx * v[k].y + gy * v[k].x;
      }
      M[r * 4 + c] = make_double2(re, im);
    }
  }
}

// Right-multiplies the DIM x DIM unit matrix M (row stride 4) by a one-qubit gate g on local bit BIT:
// M <- M (g on BIT), the gate applied before M.
template <int DIM, int BIT, typename T2>
__device__ __forceinline__ void right1(double2 (&M)[16], const T2* g) {
  const double2 g00 = make_double2((double)g[0].x, (double)g[0].y), g01 = make_double2((double)g[1].x, (double)g[1].y);
  const double2 g10 = make_double2((double)g[4].x, (double)g[4].y), g11 = make_double2((double)g[5].x, (double)g[5].y);
#pragma unroll
  for (int r = 0; r < DIM; ++r) {
#pragma unroll
    for (int c0 = 0; c0 < DIM; ++c0) {
      if (c0 & (1 << BIT)) continue;
      const int c1 = c0 | (1 << BIT);
      const double2 x = M[r * 4 + c0], y = M[r * 4 + c1];
      M[r * 4 + c0] = make_double2(x.x * g00.x - x.y * g00.y + y.x * g10.x - y.y * g10.y,
                                   x.x * g00.y + x.y * g00.x + y.x * g10.y + y.y * g10.x);
      M[r * 4 + c1] = make_double2(x.x * g01.x - x.y * g01.y + y.x * g11.x - y.y * g11.y,
                                   x.x * g01.y + x.y * g01.x + y.x * g11.y + y.y * g11.x);
    }
  }
}

// The fused matrix of one unit: the product, in op order, of its gate, coherent terms and the
// Paulis its noise sites draw (DIM 2 or 4; local index 2 bit(qa) + bit(qb), qa the only bit of a
// one-qubit unit), built in place by left multiplications.  Returns 0 when no op of the unit acts
// (every draw came up empty and no gate): the unit is then the identity.
template <int DIM, typename T2>
__device__ int fuse_unit(const UItem& u, const ProgOp* ops, const T2 (*mats)[16], const double* prob,
                         uint64_t seed, uint64_t traj, int rnd, double2* F) {
  double2 M[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) M[i] = make_double2((i / 4 == i % 4) ? 1.0 : 0.0, 0.0);
  int any = 0;
  auto one = [&](int id, bool on_qa) {   // one-qubit matrix id on qa (local bit 1) or qb (bit 0)
    if (id == M_I) return;
    if (DIM == 2) left1<DIM, 0>(M, mats[id]);
    else if (on_qa) left1<DIM, 1>(M, mats[id]);
    else left1<DIM, 0>(M, mats[id]);
  };
  for (int oi = u.op_begin; oi < u.op_end; ++oi) {
    const ProgOp op = ops[oi];
    int code = 0;
    if (op.kind == OP_N1 || op.kind == OP_N2) {
      code = noise_code(op, prob[op.pidx], seed, traj, (uint64_t)rnd);
      if (!code) continue;
    }
    if ((op.kind == OP_T1 || op.kind == OP_T2) && !twirl_fires(op, prob[op.pidx], seed, traj, (uint64_t)rnd))
      continue;
    any = 1;
    if (DIM == 4 && (op.kind == OP_U2 || op.kind == OP_T2)) {
      left2(M, mats[op.mat]);
    } else if (op.kind == OP_N2) {   // Pauli code >> 2 on op.q0, code & 3 on op.q1
      one(code >> 2, op.q0 == u.qa);
      one(code & 3, op.q1 == u.qa);
    } else {
      one((op.kind == OP_U1 || op.kind == OP_T1) ? op.mat : code, op.q0 == u.qa);
    }
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) F[i] = M[i];
  return any;
}

// Offset of pass-local combination s over the `n` slab bits in b[] (bit j of s -> slab bit b[j]).
__device__ __forceinline__ int deposit_bits(int s, const int* b, int n) {
  int o = 0;
  for (int j = 0; j < n; ++j) o |= ((s >> j) & 1) << b[j];
  return o;
}

// Slab index of group g of a pass: g's bits spread over the slab bits outside the pass
// (insert a zero at each pass bit, ascending).
__device__ __forceinline__ int group_base_u(int g, const int* bits, int nbits) {
  for (int j = 0; j < nbits; ++j) g = ((g >> bits[j]) << (bits[j] + 1)) | (g & ((1 << bits[j]) - 1));
  return g;
}

// One trajectory (or the noise-free init round) of the unreduced register on one CTA.
template <typename T>
__device__ void run_cta_u(const BatchArgs& a, unsigned char* sm, uint32_t item) {
  using T2 = typename C2<T>::t;
  const int tid = threadIdx.x, nt = blockDim.x;
  T2* slab = reinterpret_cast<T2*>(sm);
  T2 (*mats)[16] = reinterpret_cast<T2 (*)[16]>(slab + kUAmp);
  double2* Ft = reinterpret_cast<double2*>(sm + kUAmp * 16 + M_COUNT * 16 * 16);   // [kUMaxItems][16]
  int* Fon = reinterpret_cast<int*>(Ft + kUMaxItems * 16);                           // [kUMaxItems]
  double* sh = reinterpret_cast<double*>(Fon + kUMaxItems);                          // 64 doubles
  double* csum = sh + 64;                                                            // [2][kUChunks]
  const bool init = a.init_mode != 0;
  const qec_noise nz = init ? qec_noise{} : a.noise[item];
  const uint64_t traj = init ? 0ull : a.traj[item];
  const uint64_t seed = a.ctl->seed;
  const ProgOp* ops = init ? a.iuops : a.uops;
  const UItem* items = init ? a.iuitems : a.uitems;
  const int nitems = init ? a.n_iuitems : a.n_uitems;
  const UPass* passes = init ? a.iupasses : a.upasses;
  const int npass = init ? a.n_iupasses : a.n_upasses;
  const UPassUnit* punits = init ? a.iupunits : a.upunits;
  const int npunits = init ? a.n_iupunits : a.n_upunits;
  const UAbs* uabs = init ? a.iuabs : a.uabs;
  double prob[PR_COUNT];
  traj_probs(nz, prob);
  for (int i = tid; i < M_COUNT * 16; i += nt) {
    const int id = i / 16, e = i % 16;
    mats[id][e] = mk<T2>(a.mats[(id * 16 + e) * 2], a.mats[(id * 16 + e) * 2 + 1]);
  }
  __syncthreads();
  if (!init && tid < 32) coherent_mats(mats, nz, tid & 31);
  if (init) {
    for (int i = tid; i < kUAmp; i += nt) slab[i] = mk<T2>(i == 0 ? 1.0 : 0.0, 0.0);
  } else {
    const T2* p0 = reinterpret_cast<const T2*>(a.psi0_u[a.kind[item] & 1]);
    for (int i = tid; i < kUAmp; i += nt) slab[i] = p0[i];
  }
  __syncthreads();
  uint8_t* syn = init ? nullptr : a.syn + (size_t)item * (a.rounds + 1) * kNStab;
  if (syn)
    for (int k = tid; k < kNStab; k += nt) syn[k] = 0;
  const int r_first = init ? 0 : 1, r_last = init ? 0 : a.rounds;
  for (int rnd = r_first; rnd <= r_last; ++rnd) {
    // every unit of the round, one thread each
    for (int it = tid; it < nitems; it += nt) {
      const UItem u = items[it];
      Fon[it] = u.kind != 0 ? 0
                : u.nq == 1 ? fuse_unit<2, T2>(u, ops, mats, prob, seed, traj, rnd, Ft + 16 * it)
                            : fuse_unit<4, T2>(u, ops, mats, prob, seed, traj, rnd, Ft + 16 * it);
    }
    __syncthreads();
    // the one-qubit units next to a two-qubit unit on the same qubit, folded into its matrix (one
    // thread per two-qubit unit; each one-qubit unit belongs to at most one); the passes skip them.
    // Then the unit's shape, from exact zeros: Fon = 2 when the matrix is block-diagonal in its first
    // qubit (local bit 1: the two-qubit gates act on the second qubit conditioned on the first), 3
    // when block-antidiagonal (an X or Y drawn on the first qubit), else 1 (dense).
    for (int pu = tid; pu < npunits; pu += nt) {
      const UPassUnit U = punits[pu];
      if (U.nq != 2) continue;
      double2 M[16];
      double2* F = Ft + 16 * U.item;
#pragma unroll
      for (int i = 0; i < 16; ++i) M[i] = F[i];
      for (int e = U.abs0; e < U.abs0 + U.nabs; ++e) {
        const UAbs A = uabs[e];
        if (!Fon[A.item1]) continue;   // the identity
        const double2* g = Ft + 16 * A.item1;
        if (A.mode & 1) {
          if (A.mode & 2) left1<4, 1>(M, g);
          else left1<4, 0>(M, g);
        } else {
          if (A.mode & 2) right1<4, 1>(M, g);
          else right1<4, 0>(M, g);
        }
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) F[i] = M[i];
      bool bd = true, ad = true;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const bool z = M[i].x == 0.0 && M[i].y == 0.0;
        if (((i >> 3) & 1) != ((i >> 1) & 1)) bd = bd && z;   // row bit 1 != column bit 1
        else ad = ad && z;
      }
      if (Fon[U.item]) Fon[U.item] = bd ? 2 : ad ? 3 : 1;
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      // complex64: each unit's matrix converted once, in place (the first half of its slot), instead of
      // by every thread of every pass
      for (int it = tid; it < nitems; it += nt) {
        if (!Fon[it]) continue;
        double2 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = Ft[16 * it + i];
        T2* o = reinterpret_cast<T2*>(Ft + 16 * it);
#pragma unroll
        for (int i = 0; i < 16; ++i) o[i] = mk<T2>(v[i].x, v[i].y);
      }
      __syncthreads();
    }
    for (int pi = 0; pi < npass; ++pi) {
      const UPass P = passes[pi];
      if (P.kind == 1) {
        // measurement of the ancilla at slab bit u.qa: Born rule, collapse, renormalise, reset
        const UItem u = items[P.item];
        const int b = u.qa;
        double s0 = 0.0, s1 = 0.0;
        if constexpr (sizeof(T) == 4) {
          // complex64: the squares summed in FP32 over fixed chunks (chunk c: pairs c, c + 256, ..., 16 of
          // them), the chunk sums in FP64 in a fixed order by one warp, so that the sums, like the rest of
          // the run, do not depend on the CTA size
          for (int c = tid; c < kUChunks; c += nt) {
            float f0 = 0.f, f1 = 0.f;
            for (int pr = c; pr < kUAmp / 2; pr += kUChunks) {
              const int i0 = (int)ins0(pr, b), i1 = i0 | (1 << b);
              f0 = fmaf(slab[i0].x, slab[i0].x, fmaf(slab[i0].y, slab[i0].y, f0));
              f1 = fmaf(slab[i1].x, slab[i1].x, fmaf(slab[i1].y, slab[i1].y, f1));
            }
            csum[c] = (double)f0;
            csum[kUChunks + c] = (double)f1;
          }
          __syncthreads();
          if (tid < 32) {
            double a0 = 0.0, a1 = 0.0;
            for (int c = tid; c < kUChunks; c += 32) {
              a0 += csum[c];
              a1 += csum[kUChunks + c];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              a0 += __shfl_xor_sync(0xffffffffu, a0, o);
              a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            }
            if (tid == 0) {
              csum[0] = a0;
              csum[1] = a1;
            }
          }
          __syncthreads();
          s0 = csum[0];
          s1 = csum[1];
        } else {
          for (int pr = tid; pr < kUAmp / 2; pr += nt) {
            const int i0 = (int)ins0(pr, b), i1 = i0 | (1 << b);
            s0 += (double)slab[i0].x * slab[i0].x + (double)slab[i0].y * slab[i0].y;
            s1 += (double)slab[i1].x * slab[i1].x + (double)slab[i1].y * slab[i1].y;
          }
          block_sum2_u<T>(s0, s1, sh);
        }
        int m;
        if (init) {
          m = u.offset;
        } else {
          const double uu = uniform53(draw(seed, traj, (uint64_t)rnd, 0u, (uint32_t)(kND + u.stab), TAG_MEASURE).v[0]);
          m = uu < s1 / (s0 + s1) ? 1 : 0;
        }
        const double sc = 1.0 / sqrt(m ? s1 : s0);   // the renormalisation factor in FP64
        const T scT = (T)sc;                            // applied in the state's precision
        for (int pr = tid; pr < kUAmp / 2; pr += nt) {
          const int i0 = (int)ins0(pr, b), i1 = i0 | (1 << b);
          const T2 kept = m ? slab[i1] : slab[i0];
          T2 v;
          v.x = kept.x * scT;
          v.y = kept.y * scT;
          slab[i0] = v;
          slab[i1] = mk<T2>(0, 0);
        }
        __syncthreads();
        if (syn && tid == 0) syn[rnd * kNStab + u.stab] = (uint8_t)(m ^ u.offset);
        continue;
      }
      // apply: thread-local groups over the pass's bits, every unit of the pass in turn
      const int G = kUAmp >> P.nbits;
      for (int pu = P.u0; pu < P.u1; ++pu) {
        const UPassUnit U = punits[pu];
        if (!Fon[U.item]) continue;
        const T2* Fg = reinterpret_cast<const T2*>(Ft + 16 * U.item);   // the unit's matrix in the state's precision
        const int nsub = 1 << U.nother;
        if (U.nq == 1) {
          const T2 f0 = Fg[0], f1 = Fg[1], f4 = Fg[4], f5 = Fg[5];
          for (int g = tid; g < G; g += nt) {
            const int base = group_base_u(g, P.bits, P.nbits);
            for (int sub = 0; sub < nsub; ++sub) {
              const int i0 = base | deposit_bits(sub, U.other, U.nother), i1 = i0 | (1 << U.qa);
              const T2 x = slab[i0], y = slab[i1];
              T2 o0 = mk<T2>(0, 0), o1 = mk<T2>(0, 0);
              o0 = cmul_add<T>(o0, f0, x); o0 = cmul_add<T>(o0, f1, y);
              o1 = cmul_add<T>(o1, f4, x); o1 = cmul_add<T>(o1, f5, y);
              slab[i0] = o0;
              slab[i1] = o1;
            }
          }
        } else {
          T2 f[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) f[i] = Fg[i];
          const int shape = Fon[U.item];
          if (shape != 1) {
            // block-(anti)diagonal in the first qubit: rows 0, 1 from one column pair, rows 2, 3 from the
            // other (the nonzero terms of the dense sum, in the same order); selects keep every index
            // a constant
            const bool bd = shape == 2;
            T2 h[8];   // row r, term j: f[r][c(r) + j]
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
              for (int j = 0; j < 2; ++j) h[2 * r + j] = ((r < 2) == bd) ? f[r * 4 + j] : f[r * 4 + 2 + j];
            for (int g = tid; g < G; g += nt) {
              const int base = group_base_u(g, P.bits, P.nbits);
              for (int sub = 0; sub < nsub; ++sub) {
                const int b0 = base | deposit_bits(sub, U.other, U.nother);
                int idx[4];
                T2 x[4];
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                  idx[l] = b0 | ((l >> 1) << U.qa) | ((l & 1) << U.qb);
                  x[l] = slab[idx[l]];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                  const bool low = (r < 2) == bd;   // this row reads columns 0, 1
                  T2 acc = mk<T2>(0, 0);
                  acc = cmul_add<T>(acc, h[2 * r], low ? x[0] : x[2]);
                  acc = cmul_add<T>(acc, h[2 * r + 1], low ? x[1] : x[3]);
                  slab[idx[r]] = acc;
                }
              }
            }
            continue;
          }
          for (int g = tid; g < G; g += nt) {
            const int base = group_base_u(g, P.bits, P.nbits);
            for (int sub = 0; sub < nsub; ++sub) {
              const int b0 = base | deposit_bits(sub, U.other, U.nother);
              int idx[4];
              T2 x[4];
#pragma unroll
              for (int l = 0; l < 4; ++l) {
                idx[l] = b0 | ((l >> 1) << U.qa) | ((l & 1) << U.qb);
                x[l] = slab[idx[l]];
              }
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                T2 acc = mk<T2>(0, 0);
#pragma unroll
                for (int k = 0; k < 4; ++k) acc = cmul_add<T>(acc, f[r * 4 + k], x[k]);
                slab[idx[r]] = acc;
              }
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (init) {
    T2* out = reinterpret_cast<T2*>(a.init_out);
    for (int i = tid; i < kUAmp; i += nt) out[i] = slab[i];
    return;
  }
  if (item == a.ctl->snap_item)   // slab entries 0..511: the data qubits with every ancilla |0>
    for (int i = tid; i < kNAmp; i += nt) a.snap[i] = make_double2((double)slab[i].x, (double)slab[i].y);
  // final Z readout of the data qubits (the ancillas are all |0>: slab entries 0..511)
  uint8_t* bits = a.bits + (size_t)item * kND;
  uint32_t prefix = 0;
  for (int j = 0; j < kND; ++j) {
    const uint32_t mask = (1u << j) - 1u;
    double s_all = 0.0, s_one = 0.0;
    for (int x = tid; x < kNAmp; x += nt) {
      if ((x & mask) == prefix) {
        const double pp = (double)slab[x].x * slab[x].x + (double)slab[x].y * slab[x].y;
        s_all += pp;
        if ((x >> j) & 1) s_one += pp;
      }
    }
    block_sum2_u<T>(s_all, s_one, sh);
    const double uu = uniform53(draw(seed, traj, (uint64_t)a.rounds + 1, 0u, (uint32_t)j, TAG_READOUT).v[0]);
    const int bb = uu < s_one / s_all ? 1 : 0;
    prefix |= (uint32_t)bb << j;
    if (tid == 0) bits[j] = (uint8_t)bb;
  }
  if (tid == 0) {
    int par = 0;
    for (int c = 0; c < kD; ++c) par ^= (int)((prefix >> c) & 1u);
    a.logical[item] = (uint8_t)par;
  }
}

__global__ void __launch_bounds__(256) k_batch_u(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char usm[];
  __shared__ uint32_t s_pos;
  if (a.init_mode) {
    if (blockIdx.x == 0) {
      if (a.init_prec == 0) run_cta_u<double>(a, usm, 0);
      else run_cta_u<float>(a, usm, 0);
    }
    return;
  }
  for (;;) {
    if (threadIdx.x == 0) s_pos = atomicAdd(&a.ctl->counter_u, 1u);
    __syncthreads();
    const uint32_t pos = s_pos;
    __syncthreads();
    if (pos >= a.ctl->n_u) return;
    const uint32_t item = a.idx_u[pos];
    if ((a.kind[item] & 1) == 0) run_cta_u<double>(a, usm, item);
    else run_cta_u<float>(a, usm, item);
    __syncthreads();
  }
}

}  // namespace

struct qec_batch {
  int rounds = 0, gates = 0, num_sms = 0;
  uint32_t cap = 0;
  cudaStream_t work = nullptr;
  cudaStream_t user = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
  Program prog, iprog;
  ProgOp* d_ops = nullptr;
  BlockInfo* d_blocks = nullptr;
  ProgOp* d_iops = nullptr;
  BlockInfo* d_iblocks = nullptr;
  double* d_mats = nullptr;
  void* d_psi0[2] = {nullptr, nullptr};
  UProgram uprog, iuprog;
  ProgOp* d_uops = nullptr;
  UItem* d_uitems = nullptr;
  ProgOp* d_iuops = nullptr;
  UItem* d_iuitems = nullptr;
  void* d_psi0_u[2] = {nullptr, nullptr};
  uint32_t* d_idx = nullptr;
  uint32_t* d_idx_u = nullptr;
  std::vector<uint32_t> h_idx, h_idx_u;
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  int u_ctas_per_sm = 1;
  qec_noise* d_noise = nullptr;
  int32_t* d_kind = nullptr;
  uint64_t* d_traj = nullptr;
  BatchCtl* d_ctl = nullptr;
  BatchCtl* h_ctl = nullptr;   // pinned
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  uint8_t* d_syn = nullptr;
  uint8_t* d_bits = nullptr;
  uint8_t* d_log = nullptr;
  int warps_per_cta = 8;
  int ctas_per_sm = 1;
  float last_ms = 0.f;
  double2* d_snap = nullptr;
  int64_t snap_item = -1;   // for the next run
  bool snap_valid = false;  // a completed run recorded a snapshot
  int fusion_k = 4;         // unreduced engine: widest pass (slab bits)
  int u_threads = 256;      // unreduced engine: threads per CTA
  UPass* d_upasses[2] = {nullptr, nullptr};        // [0] noisy round, [1] init round
  UPassUnit* d_upunits[2] = {nullptr, nullptr};
  int n_upasses[2] = {0, 0};
  int n_upunits[2] = {0, 0};
  UAbs* d_uabs[2] = {nullptr, nullptr};           // one-qubit units folded into two-qubit units
};

namespace {

qec_status bfail(qec_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

#define QEC_BCUDA(call)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bfail(e_ == cudaErrorMemoryAllocation ? QEC_ENOMEM : QEC_ECUDA,              \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

void drop_batch_graph(qec_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
}

void batch_free(qec_batch* b) {
  drop_batch_graph(b);
  void* ptrs[] = {b->d_ops, b->d_blocks, b->d_iops, b->d_iblocks, b->d_mats, b->d_psi0[0], b->d_psi0[1],
                  b->d_noise, b->d_kind, b->d_traj, b->d_ctl, b->d_syn, b->d_bits, b->d_log,
                  b->d_uops, b->d_uitems, b->d_iuops, b->d_iuitems, b->d_psi0_u[0], b->d_psi0_u[1],
                  b->d_idx, b->d_idx_u, b->d_snap, b->d_upasses[0], b->d_upasses[1], b->d_upunits[0],
                  b->d_upunits[1], b->d_uabs[0], b->d_uabs[1]};
  for (void* p : ptrs) if (p) cudaFree(p);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  cudaEvent_t evs[] = {b->ev_in, b->ev_out, b->t0, b->t1};
  for (cudaEvent_t e : evs) if (e) cudaEventDestroy(e);
  if (b->work) cudaStreamDestroy(b->work);
}

BatchArgs batch_args(const qec_batch* b) {
  BatchArgs a;
  a.ops = b->d_ops;
  a.blocks = b->d_blocks;
  a.iops = b->d_iops;
  a.iblocks = b->d_iblocks;
  a.mats = b->d_mats;
  a.noise = b->d_noise;
  a.kind = b->d_kind;
  a.traj = b->d_traj;
  a.ctl = b->d_ctl;
  a.rounds = b->rounds;
  a.psi0[0] = b->d_psi0[0];
  a.psi0[1] = b->d_psi0[1];
  a.idx = b->d_idx;
  a.idx_u = b->d_idx_u;
  a.uops = b->d_uops;
  a.uitems = b->d_uitems;
  a.n_uitems = (int)b->uprog.items.size();
  a.iuops = b->d_iuops;
  a.iuitems = b->d_iuitems;
  a.n_iuitems = (int)b->iuprog.items.size();
  a.psi0_u[0] = b->d_psi0_u[0];
  a.psi0_u[1] = b->d_psi0_u[1];
  a.syn = b->d_syn;
  a.bits = b->d_bits;
  a.logical = b->d_log;
  a.snap = b->d_snap;
  a.upasses = b->d_upasses[0];
  a.n_upasses = b->n_upasses[0];
  a.upunits = b->d_upunits[0];
  a.iupasses = b->d_upasses[1];
  a.n_iupasses = b->n_upasses[1];
  a.iupunits = b->d_upunits[1];
  a.n_upunits = b->n_upunits[0];
  a.n_iupunits = b->n_upunits[1];
  a.uabs = b->d_uabs[0];
  a.iuabs = b->d_uabs[1];
  a.init_mode = 0;
  a.init_prec = 0;
  a.init_out = nullptr;
  return a;
}

size_t smem_for(int warps) { return (size_t)warps * kWarpSmem; }

// The persistent launch, captured once per kernel shape: one CTA wave, warps pull trajectories
// from the control word's counter (reset by the H2D copy of the control word before each run).
qec_status ensure_batch_graph(qec_batch* b) {
  if (b->gexec) return QEC_OK;
  QEC_BCUDA(cudaStreamBeginCapture(b->work, cudaStreamCaptureModeThreadLocal));
  BatchArgs a = batch_args(b);
  // reduced-register warps on the main branch, unreduced-register CTAs on a parallel branch
  cudaError_t le = cudaEventRecord(b->fork, b->work);
  if (le == cudaSuccess) le = cudaStreamWaitEvent(b->side, b->fork, 0);
  if (le == cudaSuccess) {
    k_batch<<<b->num_sms * b->ctas_per_sm, 32 * b->warps_per_cta, smem_for(b->warps_per_cta), b->work>>>(a);
    le = cudaGetLastError();
  }
  if (le == cudaSuccess) {
    k_batch_u<<<b->num_sms * b->u_ctas_per_sm, b->u_threads, kUSmem, b->side>>>(a);
    le = cudaGetLastError();
  }
  if (le == cudaSuccess) le = cudaEventRecord(b->join, b->side);
  if (le == cudaSuccess) le = cudaStreamWaitEvent(b->work, b->join, 0);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->work, &g);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(QEC_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(le != cudaSuccess ? le : e));
  }
  b->graph = g;
  QEC_BCUDA(cudaGraphInstantiate(&b->gexec, g, 0));
  return QEC_OK;
}

// Passes of one round of the unreduced engine for fusion width k: consecutive units whose slab bits
// are disjoint from those already in the pass (they commute with them) join it while the pass has at
// most k bits; a unit on a bit already in the pass, or a measurement, closes it.
// One-qubit units folded into two-qubit units: on each slab bit, a run of consecutive one-qubit units
// (nothing else on that bit between them) directly before a two-qubit unit on the bit goes into that
// unit's matrix from the right, a run directly after one from the left (between two, into the one
// whose second qubit is the bit).  Moving the run next to the unit is exact: the run acts on its bit alone, and nothing else
// acts on that bit in between.  absorbed[it] marks the folded units; pre/post list them per
// two-qubit unit in program order.
void plan_absorb(const UProgram& U, std::vector<char>& absorbed, std::vector<std::vector<UAbs>>& pre,
                 std::vector<std::vector<UAbs>>& post) {
  const int n = (int)U.items.size();
  absorbed.assign(n, 0);
  pre.assign(n, {});
  post.assign(n, {});
  auto is1 = [&](int it) { return U.items[it].kind == 0 && U.items[it].nq == 1; };
  auto is2 = [&](int it) { return U.items[it].kind == 0 && U.items[it].nq == 2; };
  for (int b = 0; b < U.nbits; ++b) {
    std::vector<int> seq;   // items acting on bit b, in order
    for (int it = 0; it < n; ++it) {
      const UItem& u = U.items[it];
      if (u.qa == b || (u.kind == 0 && u.nq == 2 && u.qb == b)) seq.push_back(it);
    }
    for (size_t i = 0; i < seq.size();) {
      if (!is1(seq[i])) { ++i; continue; }
      size_t j = i;
      while (j < seq.size() && is1(seq[j])) ++j;
      int target = -1;
      bool after = false;
      const bool next2 = j < seq.size() && is2(seq[j]), prev2 = i > 0 && is2(seq[i - 1]);
      // between two two-qubit units, the one in which b is the second qubit (the gate's target) takes
      // the run: a one-qubit matrix there keeps that unit block-diagonal in its first qubit
      if (next2 && (!prev2 || U.items[seq[j]].qb == b || U.items[seq[i - 1]].qb != b)) {
        target = seq[j];
      } else if (prev2) {
        target = seq[i - 1];
        after = true;
      }
      if (target >= 0) {
        const int bit = U.items[target].qa == b ? 2 : 0;
        for (size_t r = i; r < j; ++r) {
          absorbed[seq[r]] = 1;
          (after ? post : pre)[target].push_back({seq[r], bit | (after ? 1 : 0)});
        }
      }
      i = j;
    }
  }
}

void build_passes(const UProgram& U, int k, std::vector<UPass>& passes, std::vector<UPassUnit>& punits,
                  std::vector<UAbs>& uabs) {
  passes.clear();
  punits.clear();
  uabs.clear();
  std::vector<char> absorbed;
  std::vector<std::vector<UAbs>> pre, post;
  plan_absorb(U, absorbed, pre, post);
  UPass cur{};
  uint32_t mask = 0;
  auto close = [&]() {
    if (cur.u1 == cur.u0) return;
    cur.nbits = 0;
    for (int q = 0; q < 32; ++q)
      if (mask & (1u << q)) cur.bits[cur.nbits++] = q;
    for (int i = cur.u0; i < cur.u1; ++i) {
      UPassUnit& pu = punits[i];
      const uint32_t um = (1u << pu.qa) | (pu.nq == 2 ? (1u << pu.qb) : 0u);
      pu.nother = 0;
      for (int j = 0; j < cur.nbits; ++j)
        if (!(um & (1u << cur.bits[j]))) pu.other[pu.nother++] = cur.bits[j];
    }
    passes.push_back(cur);
  };
  auto open = [&]() {
    cur = UPass{};
    cur.kind = 0;
    cur.u0 = cur.u1 = (int32_t)punits.size();
    mask = 0;
  };
  open();
  for (int it = 0; it < (int)U.items.size(); ++it) {
    const UItem& u = U.items[it];
    if (u.kind == 1) {
      close();
      UPass m{};
      m.kind = 1;
      m.item = it;
      passes.push_back(m);
      open();
      continue;
    }
    if (absorbed[it]) continue;
    const uint32_t um = (1u << u.qa) | (u.nq == 2 ? (1u << u.qb) : 0u);
    if ((mask & um) || __builtin_popcount(mask | um) > k) {
      close();
      open();
    }
    UPassUnit pu{};
    pu.item = it;
    pu.nq = u.nq;
    pu.qa = u.qa;
    pu.qb = u.nq == 2 ? u.qb : 0;
    pu.abs0 = (int32_t)uabs.size();
    for (auto r = pre[it].rbegin(); r != pre[it].rend(); ++r) uabs.push_back(*r);   // right factors, latest first
    for (const UAbs& x : post[it]) uabs.push_back(x);                              // left factors, in order
    pu.nabs = (int32_t)uabs.size() - pu.abs0;
    punits.push_back(pu);
    cur.u1 = (int32_t)punits.size();
    mask |= um;
  }
  close();
}

// Fusion width (2..6 slab bits per pass) and threads per CTA (128..512) of the unreduced engine.
qec_status set_fusion(qec_batch* b, int k, int threads) {
  if (k < 2 || k > kUMaxFusionDecl || (threads != 128 && threads != 256 && threads != 512))
    return bfail(QEC_EINVAL, "fusion width must be in [2, 6] and threads 128, 256 or 512");
  const UProgram* progs[2] = {&b->uprog, &b->iuprog};
  for (int w = 0; w < 2; ++w) {
    std::vector<UPass> passes;
    std::vector<UPassUnit> punits;
    std::vector<UAbs> uabs;
    build_passes(*progs[w], k, passes, punits, uabs);
    QEC_BCUDA(cudaMemcpy(b->d_upasses[w], passes.data(), sizeof(UPass) * passes.size(), cudaMemcpyHostToDevice));
    if (!punits.empty())
      QEC_BCUDA(cudaMemcpy(b->d_upunits[w], punits.data(), sizeof(UPassUnit) * punits.size(), cudaMemcpyHostToDevice));
    if (!uabs.empty())
      QEC_BCUDA(cudaMemcpy(b->d_uabs[w], uabs.data(), sizeof(UAbs) * uabs.size(), cudaMemcpyHostToDevice));
    b->n_upasses[w] = (int)passes.size();
    b->n_upunits[w] = (int)punits.size();
  }
  int occ = 0;
  QEC_BCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_u, threads, kUSmem));
  if (occ < 1) return bfail(QEC_EUNSUPPORTED, "unreduced batched kernel does not fit an SM with this shape");
  drop_batch_graph(b);
  b->fusion_k = k;
  b->u_threads = threads;
  b->u_ctas_per_sm = occ;
  return QEC_OK;
}

qec_status set_shape(qec_batch* b, int warps) {
  QEC_BCUDA(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_for(warps)));
  int occ = 0;
  QEC_BCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch, 32 * warps, smem_for(warps)));
  if (occ < 1) return bfail(QEC_EUNSUPPORTED, "batched kernel does not fit an SM with this shape");
  if (warps != b->warps_per_cta || occ != b->ctas_per_sm) drop_batch_graph(b);
  b->warps_per_cta = warps;
  b->ctas_per_sm = occ;
  return QEC_OK;
}

}  // namespace

extern "C" {

qec_status qec_debug_unreduced_plan(int32_t gates, int32_t k, int32_t* items, uint32_t cap, uint32_t* n_items,
                                    int32_t* pass_units, uint32_t* n_pass_units, int32_t* absorbs, uint32_t* n_absorbs) {
  if (!items || !n_items || !pass_units || !n_pass_units || !absorbs || !n_absorbs)
    return bfail(QEC_EINVAL, "null argument");
  if (k < 2 || k > kUMaxFusionDecl) return bfail(QEC_EINVAL, "fusion width must be in [2, 6]");
  try {
    qec_params p{};
    p.d = kD;
    p.rounds = 1;
    p.layout = QEC_LAYOUT_REDUCED;   // the parameters qec_batch_create builds both programs from
    p.gates = gates;
    p.precision = QEC_C128;
    p.noise = qec_noise{1, 1, 1, 1, 1, 1, 1, 1, 1, 0};   // every site and coherent op present
    std::string err;
    UProgram U;
    if (!build_unreduced_program(p, true, U, err, true)) return bfail(QEC_EINVAL, err);
    std::vector<UPass> passes;
    std::vector<UPassUnit> punits;
    std::vector<UAbs> uabs;
    build_passes(U, k, passes, punits, uabs);
    *n_items = (uint32_t)U.items.size();
    if (U.items.size() > cap || punits.size() > cap || uabs.size() > cap)
      return bfail(QEC_EINVAL, "capacity too small");
    for (size_t i = 0; i < U.items.size(); ++i) {
      const UItem& u = U.items[i];
      items[4 * i] = u.kind;
      items[4 * i + 1] = u.nq;
      items[4 * i + 2] = u.qa;
      items[4 * i + 3] = u.kind == 0 && u.nq == 2 ? u.qb : -1;
    }
    uint32_t na = 0;
    for (size_t i = 0; i < punits.size(); ++i) {
      pass_units[i] = punits[i].item;
      for (int e = punits[i].abs0; e < punits[i].abs0 + punits[i].nabs; ++e) {
        absorbs[3 * na] = uabs[e].item1;
        absorbs[3 * na + 1] = punits[i].item;
        absorbs[3 * na + 2] = uabs[e].mode;
        ++na;
      }
    }
    *n_pass_units = (uint32_t)punits.size();
    *n_absorbs = na;
    return QEC_OK;
  } catch (...) {
    return bfail(QEC_ENOMEM, "host allocation failed");
  }
}

qec_status qec_batch_create(int32_t d, int32_t rounds, int32_t gates, uint32_t max_traj, void* cuda_stream,
                            qec_batch** out) {
  if (!out) return bfail(QEC_EINVAL, "null output handle");
  *out = nullptr;
  if (d != kD) return bfail(QEC_EUNSUPPORTED, "the batched form runs the d = 3 reduced register");
  if (rounds < 0 || rounds > 64 || max_traj == 0 || max_traj > (1u << 24))
    return bfail(QEC_EINVAL, "rounds must be in [0, 64] and max_traj in [1, 2^24]");
  qec_params p{};
  p.d = d;
  p.rounds = rounds;
  p.layout = QEC_LAYOUT_REDUCED;
  p.gates = gates;
  p.precision = QEC_C128;
  // every noise site and coherent op present; the per-trajectory values decide what they do
  p.noise = qec_noise{1, 1, 1, 1, 1, 1, 1, 1, 1, 0};
  std::string err;
  qec_batch* b = new (std::nothrow) qec_batch();
  if (!b) return bfail(QEC_ENOMEM, "host allocation failed");
  auto bail = [&](qec_status s) { batch_free(b); delete b; return s; };
  b->rounds = rounds;
  b->gates = gates;
  b->cap = max_traj;
  b->user = static_cast<cudaStream_t>(cuda_stream);
  if (!build_program(p, true, b->prog, err, true) || !build_program(p, false, b->iprog, err) ||
      !build_unreduced_program(p, true, b->uprog, err, true) || !build_unreduced_program(p, false, b->iuprog, err))
    return bail(bfail(QEC_EINVAL, err));
  if (b->uprog.items.size() > (size_t)kUMaxItems || b->iuprog.items.size() > (size_t)kUMaxItems)
    return bail(bfail(QEC_EUNSUPPORTED, "unreduced round has more items than the engine's unit table"));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->work, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&b->t0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->t1);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(bfail(QEC_ECUDA, std::string("CUDA setup: ") + cudaGetErrorString(e)));
  const size_t syn_bytes = (size_t)max_traj * (rounds + 1) * kNStab;
  void** allocs[] = {(void**)&b->d_ops, (void**)&b->d_blocks, (void**)&b->d_iops, (void**)&b->d_iblocks,
                     (void**)&b->d_mats, &b->d_psi0[0], &b->d_psi0[1], (void**)&b->d_noise, (void**)&b->d_kind,
                     (void**)&b->d_traj, (void**)&b->d_ctl, (void**)&b->d_syn, (void**)&b->d_bits,
                     (void**)&b->d_log, (void**)&b->d_uops, (void**)&b->d_uitems, (void**)&b->d_iuops,
                     (void**)&b->d_iuitems, &b->d_psi0_u[0], &b->d_psi0_u[1], (void**)&b->d_idx,
                     (void**)&b->d_idx_u, (void**)&b->d_snap, (void**)&b->d_upasses[0], (void**)&b->d_upasses[1],
                     (void**)&b->d_upunits[0], (void**)&b->d_upunits[1], (void**)&b->d_uabs[0],
                     (void**)&b->d_uabs[1]};
  const size_t sizes[] = {sizeof(ProgOp) * (b->prog.ops.size() + 1), sizeof(BlockInfo) * kNStab,
                          sizeof(ProgOp) * (b->iprog.ops.size() + 1), sizeof(BlockInfo) * kNStab,
                          sizeof(b->prog.mats), (size_t)kNAmp * 16, (size_t)kNAmp * 8,
                          sizeof(qec_noise) * max_traj, sizeof(int32_t) * max_traj, sizeof(uint64_t) * max_traj,
                          sizeof(BatchCtl), syn_bytes, (size_t)max_traj * kND, (size_t)max_traj,
                          sizeof(ProgOp) * (b->uprog.ops.size() + 1), sizeof(UItem) * (b->uprog.items.size() + 1),
                          sizeof(ProgOp) * (b->iuprog.ops.size() + 1), sizeof(UItem) * (b->iuprog.items.size() + 1),
                          (size_t)kUAmp * 16, (size_t)kUAmp * 8, sizeof(uint32_t) * max_traj,
                          sizeof(uint32_t) * max_traj, sizeof(double2) * kNAmp,
                          sizeof(UPass) * (b->uprog.items.size() + 1), sizeof(UPass) * (b->iuprog.items.size() + 1),
                          sizeof(UPassUnit) * (b->uprog.items.size() + 1),
                          sizeof(UPassUnit) * (b->iuprog.items.size() + 1),
                          sizeof(UAbs) * (b->uprog.items.size() + 1), sizeof(UAbs) * (b->iuprog.items.size() + 1)};
  for (size_t i = 0; i < sizeof(sizes) / sizeof(sizes[0]); ++i) {
    e = cudaMalloc(allocs[i], sizes[i]);
    if (e != cudaSuccess) return bail(bfail(QEC_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)));
  }
  e = cudaMemcpy(b->d_ops, b->prog.ops.data(), sizeof(ProgOp) * b->prog.ops.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_blocks, b->prog.blocks.data(), sizeof(BlockInfo) * kNStab, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b->iprog.ops.empty())
    e = cudaMemcpy(b->d_iops, b->iprog.ops.data(), sizeof(ProgOp) * b->iprog.ops.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_iblocks, b->iprog.blocks.data(), sizeof(BlockInfo) * kNStab, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_mats, b->prog.mats, sizeof(b->prog.mats), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b->uprog.ops.empty())
    e = cudaMemcpy(b->d_uops, b->uprog.ops.data(), sizeof(ProgOp) * b->uprog.ops.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_uitems, b->uprog.items.data(), sizeof(UItem) * b->uprog.items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b->iuprog.ops.empty())
    e = cudaMemcpy(b->d_iuops, b->iuprog.ops.data(), sizeof(ProgOp) * b->iuprog.ops.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_iuitems, b->iuprog.items.data(), sizeof(UItem) * b->iuprog.items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(bfail(QEC_ECUDA, std::string("upload: ") + cudaGetErrorString(e)));
  e = cudaMallocHost((void**)&b->h_ctl, sizeof(BatchCtl));
  if (e != cudaSuccess) return bail(bfail(QEC_ENOMEM, "pinned allocation failed"));
  std::memset(b->h_ctl, 0, sizeof(BatchCtl));
  e = cudaMemcpy(b->d_ctl, b->h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(bfail(QEC_ECUDA, cudaGetErrorString(e)));
  qec_status st = set_shape(b, 8);
  if (st) return bail(st);
  e = cudaFuncSetAttribute(k_batch_u, cudaFuncAttributeMaxDynamicSharedMemorySize, kUSmem);
  if (e != cudaSuccess) return bail(bfail(QEC_ECUDA, "unreduced batched kernel does not fit an SM"));
  if ((st = set_fusion(b, 4, 256))) return bail(st);
  for (int prec = 0; prec < 2; ++prec) {   // the noise-free init round, once per precision
    BatchArgs a = batch_args(b);
    a.init_mode = 1;
    a.init_prec = prec;
    a.init_out = b->d_psi0[prec];
    k_batch<<<1, 32, smem_for(1), b->work>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bail(bfail(QEC_ECUDA, std::string("init round: ") + cudaGetErrorString(e)));
    a.init_out = b->d_psi0_u[prec];   // and of the unreduced register
    k_batch_u<<<1, 256, kUSmem, b->work>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bail(bfail(QEC_ECUDA, std::string("init round: ") + cudaGetErrorString(e)));
  }
  e = cudaStreamSynchronize(b->work);
  if (e != cudaSuccess) return bail(bfail(QEC_ECUDA, std::string("init round: ") + cudaGetErrorString(e)));
  *out = b;
  return QEC_OK;
}

qec_status qec_batch_run(qec_batch* b, uint64_t seed, uint32_t n, const uint64_t* traj, const int32_t* kind,
                         const qec_noise* noise, uint8_t* syndromes, uint8_t* data_bits, uint8_t* raw_logical) {
  if (!b) return bfail(QEC_EINVAL, "null handle");
  if (n > b->cap) return bfail(QEC_EINVAL, "n exceeds the batch capacity given at creation");
  if (n == 0) return QEC_OK;
  if (!traj || !kind || !noise) return bfail(QEC_EINVAL, "null input array");
  for (uint32_t i = 0; i < n; ++i) {
    if (kind[i] < 0 || kind[i] > 3)
      return bfail(QEC_EINVAL, "kind must be precision (QEC_C128 or QEC_C64) | 2 * layout (QEC_LAYOUT_*)");
    const qec_noise& z = noise[i];
    const double pr[3] = {z.p1, z.p2, z.p_idle};
    for (double v : pr)
      if (!(v >= 0.0 && v <= 1.0)) return bfail(QEC_EINVAL, "noise probabilities must be in [0, 1]");
    const double an[6] = {z.theta_rx, z.theta_rz, z.theta_rzx, z.phi_zz, z.round_rz, z.round_rx};
    for (double v : an)
      if (!(std::fabs(v) <= 4.0)) return bfail(QEC_EINVAL, "angles must be finite with |angle| <= 4");
    if (z.twirl != 0.0 && z.twirl != 1.0) return bfail(QEC_EINVAL, "twirl must be 0 or 1");
    if (z.overrot_follows != 0.0 && z.overrot_follows != 1.0) return bfail(QEC_EINVAL, "overrot_follows must be 0 or 1");
  }
  if (b->user) {
    QEC_BCUDA(cudaEventRecord(b->ev_in, b->user));
    QEC_BCUDA(cudaStreamWaitEvent(b->work, b->ev_in, 0));
  }
  QEC_BCUDA(cudaMemcpyAsync(b->d_traj, traj, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, b->work));
  QEC_BCUDA(cudaMemcpyAsync(b->d_kind, kind, sizeof(int32_t) * n, cudaMemcpyHostToDevice, b->work));
  QEC_BCUDA(cudaMemcpyAsync(b->d_noise, noise, sizeof(qec_noise) * n, cudaMemcpyHostToDevice, b->work));
  b->h_idx.clear();
  b->h_idx_u.clear();
  // each engine's items complex128 first, then complex64: the warps (CTAs) then run one precision's
  // code at a time instead of interleaving both instantiations, and the longer items start first.
  // Every trajectory's result is independent of the order.
  for (int prec = 0; prec < 2; ++prec)
    for (uint32_t i = 0; i < n; ++i)
      if ((kind[i] & 1) == prec) ((kind[i] & 2) ? b->h_idx_u : b->h_idx).push_back(i);
  if (!b->h_idx.empty())
    QEC_BCUDA(cudaMemcpyAsync(b->d_idx, b->h_idx.data(), sizeof(uint32_t) * b->h_idx.size(), cudaMemcpyHostToDevice, b->work));
  if (!b->h_idx_u.empty())
    QEC_BCUDA(cudaMemcpyAsync(b->d_idx_u, b->h_idx_u.data(), sizeof(uint32_t) * b->h_idx_u.size(),
                              cudaMemcpyHostToDevice, b->work));
  qec_status st = ensure_batch_graph(b);
  if (st) return st;
  QEC_BCUDA(cudaStreamSynchronize(b->work));   // h_ctl is reused
  b->h_ctl->seed = seed;
  b->h_ctl->n = (uint32_t)b->h_idx.size();
  b->h_ctl->counter = 0;
  b->h_ctl->n_u = (uint32_t)b->h_idx_u.size();
  b->h_ctl->counter_u = 0;
  const bool snap = b->snap_item >= 0 && b->snap_item < (int64_t)n;
  b->h_ctl->snap_item = snap ? (uint32_t)b->snap_item : ~0u;
  b->snap_valid = false;
  QEC_BCUDA(cudaMemcpyAsync(b->d_ctl, b->h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, b->work));
  QEC_BCUDA(cudaEventRecord(b->t0, b->work));
  QEC_BCUDA(cudaGraphLaunch(b->gexec, b->work));
  QEC_BCUDA(cudaEventRecord(b->t1, b->work));
  const size_t ss = (size_t)(b->rounds + 1) * kNStab;
  if (syndromes) QEC_BCUDA(cudaMemcpyAsync(syndromes, b->d_syn, n * ss, cudaMemcpyDeviceToHost, b->work));
  if (data_bits) QEC_BCUDA(cudaMemcpyAsync(data_bits, b->d_bits, (size_t)n * kND, cudaMemcpyDeviceToHost, b->work));
  if (raw_logical) QEC_BCUDA(cudaMemcpyAsync(raw_logical, b->d_log, n, cudaMemcpyDeviceToHost, b->work));
  if (b->user) {
    QEC_BCUDA(cudaEventRecord(b->ev_out, b->work));
    QEC_BCUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
  }
  QEC_BCUDA(cudaStreamSynchronize(b->work));
  QEC_BCUDA(cudaEventElapsedTime(&b->last_ms, b->t0, b->t1));
  b->snap_valid = snap;
  return QEC_OK;
}

qec_status qec_batch_autotune(qec_batch* b, uint64_t seed, uint32_t n, const uint64_t* traj, const int32_t* kind,
                              const qec_noise* noise, int32_t* chosen_warps, float* best_ms) {
  if (!b || !chosen_warps || !best_ms || !traj || !kind || !noise) return bfail(QEC_EINVAL, "null argument");
  // the sample split by register: each engine is tuned on its own trajectories
  std::vector<uint64_t> tr[2];
  std::vector<int32_t> kd[2];
  std::vector<qec_noise> nz[2];
  for (uint32_t i = 0; i < n; ++i) {
    const int u = (kind[i] & 2) ? 1 : 0;
    tr[u].push_back(traj[i]);
    kd[u].push_back(kind[i]);
    nz[u].push_back(noise[i]);
  }
  auto time_run = [&](int u, float& t) -> qec_status {
    t = 1e30f;
    if (tr[u].empty()) return QEC_OK;
    for (int rep = 0; rep < 2; ++rep) {   // first run warms up
      qec_status st = qec_batch_run(b, seed, (uint32_t)tr[u].size(), tr[u].data(), kd[u].data(), nz[u].data(),
                                    nullptr, nullptr, nullptr);
      if (st) return st;
      if (rep) t = b->last_ms;
    }
    return QEC_OK;
  };
  // reduced register: warps per CTA
  const int cand[] = {2, 4, 6, 8, 10};
  int best = -1;
  float best_t = 0.f;
  for (int w : cand) {
    if (set_shape(b, w) != QEC_OK) continue;
    float t;
    qec_status st = time_run(0, t);
    if (st) return st;
    if (best < 0 || t < best_t) {
      best = w;
      best_t = t;
    }
  }
  if (best < 0) return bfail(QEC_EUNSUPPORTED, "no batched kernel shape fits");
  qec_status st = set_shape(b, best);
  if (st) return st;
  // unreduced register: fusion width (slab bits per pass) x threads per CTA
  int bk = -1, bthr = 256;
  float bu = 0.f;
  for (int k = 2; k <= kUMaxFusionDecl; ++k)
    for (int thr : {128, 256}) {
      if (set_fusion(b, k, thr) != QEC_OK) continue;
      float t;
      if ((st = time_run(1, t))) return st;
      if (bk < 0 || t < bu) {
        bk = k;
        bthr = thr;
        bu = t;
      }
    }
  if (bk < 0) return bfail(QEC_EUNSUPPORTED, "no unreduced engine shape fits");
  if ((st = set_fusion(b, bk, bthr))) return st;
  float t_all = 0.f;   // the whole sample with the chosen configuration
  for (int rep = 0; rep < 2; ++rep) {
    if ((st = qec_batch_run(b, seed, n, traj, kind, noise, nullptr, nullptr, nullptr))) return st;
    t_all = b->last_ms;
  }
  *chosen_warps = best;
  *best_ms = t_all;
  return QEC_OK;
}

qec_status qec_batch_config(const qec_batch* b, int32_t* warps_per_cta, int32_t* fusion_width, int32_t* u_threads) {
  if (!b || !warps_per_cta || !fusion_width || !u_threads) return bfail(QEC_EINVAL, "null argument");
  *warps_per_cta = b->warps_per_cta;
  *fusion_width = b->fusion_k;
  *u_threads = b->u_threads;
  return QEC_OK;
}

qec_status qec_batch_set_config(qec_batch* b, int32_t warps_per_cta, int32_t fusion_width, int32_t u_threads) {
  if (!b) return bfail(QEC_EINVAL, "null handle");
  qec_status st = set_shape(b, warps_per_cta);
  if (st) return st;
  return set_fusion(b, fusion_width, u_threads);
}

qec_status qec_batch_snapshot(qec_batch* b, int64_t item) {
  if (!b || item < -1) return bfail(QEC_EINVAL, "null handle or item < -1");
  b->snap_item = item;
  return QEC_OK;
}

qec_status qec_batch_get_state(qec_batch* b, void* host_buf, size_t bytes) {
  if (!b || !host_buf) return bfail(QEC_EINVAL, "null argument");
  if (bytes < sizeof(double2) * kNAmp) return bfail(QEC_EINVAL, "host buffer too small");
  if (!b->snap_valid) return bfail(QEC_EINVAL, "no completed run recorded a snapshot");
  double* out = static_cast<double*>(host_buf);
  QEC_BCUDA(cudaMemcpy(out, b->d_snap, sizeof(double2) * kNAmp, cudaMemcpyDeviceToHost));
  double nrm = 0.0;   // the reduced register keeps the norm P(m) of the last outcome; report unit norm
  for (int i = 0; i < 2 * kNAmp; ++i) nrm += out[i] * out[i];
  const double sc = nrm > 0.0 ? 1.0 / std::sqrt(nrm) : 1.0;
  for (int i = 0; i < 2 * kNAmp; ++i) out[i] *= sc;
  return QEC_OK;
}

qec_status qec_batch_last_ms(const qec_batch* b, float* ms) {
  if (!b || !ms) return bfail(QEC_EINVAL, "null argument");
  *ms = b->last_ms;
  return QEC_OK;
}

qec_status qec_batch_destroy(qec_batch* b) {
  if (!b) return QEC_OK;
  if (b->work) cudaStreamSynchronize(b->work);
  batch_free(b);
  delete b;
  return QEC_OK;
}

}  // extern "C"
