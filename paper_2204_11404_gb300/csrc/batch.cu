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
constexpr int kWarpSmem = 32 * 16 * 16 + kNAmp * 16 + M_COUNT * 16 * 16 + 64;   // U, psi, mats, misc (c128)

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

// One trajectory (or, in init mode, the noise-free init round) on one warp.
template <typename T>
__device__ void run_warp(const BatchArgs& a, unsigned char* wsm, uint32_t item) {
  using T2 = typename C2<T>::t;
  const int lane = threadIdx.x & 31;
  T2* U = reinterpret_cast<T2*>(wsm);
  T2* psi = U + 32 * 16;
  T2 (*mats)[16] = reinterpret_cast<T2 (*)[16]>(psi + kNAmp);
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
          if (op.kind == OP_T1) apply1_w<T>(U, w, op.q0, mats[op.mat], lane);
          else apply2_w<T>(U, w, op.q0, op.q1, mats[op.mat], lane);
          continue;
        }
        if (op.kind == OP_N1 || op.kind == OP_N2) {
          int code = 0;
          if (lane == 0) code = noise_code(op, prob[op.pidx], a.ctl->seed, traj, (uint64_t)rnd);
          code = __shfl_sync(0xffffffffu, code, 0);
          if (!code) continue;
          if (op.kind == OP_N1) {
            apply1_w<T>(U, w, op.q0, mats[code], lane);
          } else {
            if (code >> 2) apply1_w<T>(U, w, op.q0, mats[code >> 2], lane);
            if (code & 3) apply1_w<T>(U, w, op.q1, mats[code & 3], lane);
          }
        } else if (op.kind == OP_U1) {
          apply1_w<T>(U, w, op.q0, mats[op.mat], lane);
        } else {
          apply2_w<T>(U, w, op.q0, op.q1, mats[op.mat], lane);
        }
      }
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
constexpr int kUBits = kND + kNStab / 2;      // 13 slab bits: 9 data + the active part's 4 ancillas
constexpr int kUAmp = 1 << kUBits;            // 8192 amplitudes
constexpr int kUSmem = kUAmp * 16 + M_COUNT * 16 * 16 + 16 * 16 + 64 * 8 + 16;   // slab, mats, F, reduction, flag

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

// One trajectory (or the noise-free init round) of the unreduced register on one CTA.
template <typename T>
__device__ void run_cta_u(const BatchArgs& a, unsigned char* sm, uint32_t item) {
  using T2 = typename C2<T>::t;
  const int tid = threadIdx.x, nt = blockDim.x;
  T2* slab = reinterpret_cast<T2*>(sm);
  T2 (*mats)[16] = reinterpret_cast<T2 (*)[16]>(slab + kUAmp);
  double2* F = reinterpret_cast<double2*>(mats + M_COUNT);         // fused unit matrix (FP64, 16 entries)
  double* sh = reinterpret_cast<double*>(F + 16);                  // 64 doubles
  int* sflag = reinterpret_cast<int*>(sh + 64);
  const bool init = a.init_mode != 0;
  const qec_noise nz = init ? qec_noise{} : a.noise[item];
  const uint64_t traj = init ? 0ull : a.traj[item];
  const uint64_t seed = a.ctl->seed;
  const ProgOp* ops = init ? a.iuops : a.uops;
  const UItem* items = init ? a.iuitems : a.uitems;
  const int nitems = init ? a.n_iuitems : a.n_uitems;
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
    for (int it = 0; it < nitems; ++it) {
      const UItem u = items[it];
      if (u.kind == 0) {
        // thread 0 fuses the unit: F = (Pauli) (coherent) (gate), applied in op order
        if (tid == 0) {
          const int dim = u.nq == 1 ? 2 : 4;
          double2 M[16];
          for (int i = 0; i < 16; ++i) M[i] = make_double2((i / 4 == i % 4) ? 1.0 : 0.0, 0.0);
          int any = 0;
          for (int oi = u.op_begin; oi < u.op_end; ++oi) {
            const ProgOp op = ops[oi];
            int code = 0;
            if (op.kind == OP_N1 || op.kind == OP_N2) {
              code = noise_code(op, prob[op.pidx], seed, traj, (uint64_t)rnd);
              if (!code) continue;
            }
            if ((op.kind == OP_T1 || op.kind == OP_T2) && !twirl_fires(op, prob[op.pidx], seed, traj, (uint64_t)rnd))
              continue;
            // left-multiply M by this op's matrix G (dim x dim, embedded in the unit's local qubits)
            double2 G[16];
            for (int i = 0; i < 16; ++i) G[i] = make_double2(0.0, 0.0);
            auto from_tab = [&](int id, int r, int c) {
              return make_double2((double)mats[id][r * 4 + c].x, (double)mats[id][r * 4 + c].y);
            };
            if (dim == 2) {
              const int id = (op.kind == OP_U1 || op.kind == OP_T1) ? op.mat : code;
              for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) G[r * 4 + c] = from_tab(id, r, c);
            } else if (op.kind == OP_U2 || op.kind == OP_T2) {
              for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c) G[r * 4 + c] = from_tab(op.mat, r, c);
            } else {
              // one-qubit op or Pauli pair on a 2-qubit unit: local index 2*bit(qa) + bit(qb)
              int ida = 0, idb = 0;
              if (op.kind == OP_N2) { ida = code >> 2; idb = code & 3; }
              else {
                const int id = op.kind == OP_U1 ? op.mat : code;
                if (op.q0 == u.qa) ida = id; else idb = id;
              }
              if (op.kind == OP_N2 && op.q0 != u.qa) { const int t = ida; ida = idb; idb = t; }
              for (int ra = 0; ra < 2; ++ra)
                for (int rb = 0; rb < 2; ++rb)
                  for (int ca = 0; ca < 2; ++ca)
                    for (int cb = 0; cb < 2; ++cb) {
                      const double2 x = from_tab(ida, ra, ca), y = from_tab(idb, rb, cb);
                      G[(2 * ra + rb) * 4 + 2 * ca + cb] = make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
                    }
            }
            double2 R[16];
            for (int r = 0; r < dim; ++r)
              for (int c = 0; c < dim; ++c) {
                double re = 0.0, im = 0.0;
                for (int k = 0; k < dim; ++k) {
                  const double2 g = G[r * 4 + k], m = M[k * 4 + c];
                  re += g.x * m.x - g.y * m.y;
                  im += g.x * m.y + g.y * m.x;
                }
                R[r * 4 + c] = make_double2(re, im);
              }
            for (int r = 0; r < dim; ++r)
              for (int c = 0; c < dim; ++c) M[r * 4 + c] = R[r * 4 + c];
            any = 1;
          }
          for (int i = 0; i < 16; ++i) F[i] = M[i];
          *sflag = any;
        }
        __syncthreads();
        if (*sflag) {
          T2 f[16];
          for (int i = 0; i < 16; ++i) f[i] = mk<T2>(F[i].x, F[i].y);
          if (u.nq == 1) {
            const int b = u.qa;
            for (int pr = tid; pr < kUAmp / 2; pr += nt) {
              const int i0 = (int)ins0(pr, b), i1 = i0 | (1 << b);
              const T2 x = slab[i0], y = slab[i1];
              T2 o0 = mk<T2>(0, 0), o1 = mk<T2>(0, 0);
              o0 = cmul_add<T>(o0, f[0], x); o0 = cmul_add<T>(o0, f[1], y);
              o1 = cmul_add<T>(o1, f[4], x); o1 = cmul_add<T>(o1, f[5], y);
              slab[i0] = o0;
              slab[i1] = o1;
            }
          } else {
            const int qa = u.qa, qb = u.qb, lo = qa < qb ? qa : qb, hi = qa < qb ? qb : qa;
            for (int qd = tid; qd < kUAmp / 4; qd += nt) {
              const int base = (int)ins0(ins0(qd, lo), hi);
              int idx[4];
              T2 x[4];
              for (int l = 0; l < 4; ++l) {
                idx[l] = base | ((l >> 1) << qa) | ((l & 1) << qb);
                x[l] = slab[idx[l]];
              }
              for (int r = 0; r < 4; ++r) {
                T2 acc = mk<T2>(0, 0);
                for (int k = 0; k < 4; ++k) acc = cmul_add<T>(acc, f[r * 4 + k], x[k]);
                slab[idx[r]] = acc;
              }
            }
          }
        }
        __syncthreads();
      } else {
        // measurement of the ancilla at slab bit u.qa: Born rule, collapse, renormalise, reset
        const int b = u.qa;
        double s0 = 0.0, s1 = 0.0;
        for (int pr = tid; pr < kUAmp / 2; pr += nt) {
          const int i0 = (int)ins0(pr, b), i1 = i0 | (1 << b);
          s0 += (double)slab[i0].x * slab[i0].x + (double)slab[i0].y * slab[i0].y;
          s1 += (double)slab[i1].x * slab[i1].x + (double)slab[i1].y * slab[i1].y;
        }
        block_sum2_u<T>(s0, s1, sh);
        int m;
        if (init) {
          m = u.offset;
        } else {
          const double uu = uniform53(draw(seed, traj, (uint64_t)rnd, 0u, (uint32_t)(kND + u.stab), TAG_MEASURE).v[0]);
          m = uu < s1 / (s0 + s1) ? 1 : 0;
        }
        const double sc = 1.0 / sqrt(m ? s1 : s0);
        for (int pr = tid; pr < kUAmp / 2; pr += nt) {
          const int i0 = (int)ins0(pr, b), i1 = i0 | (1 << b);
          const T2 kept = m ? slab[i1] : slab[i0];
          slab[i0] = mk<T2>((double)kept.x * sc, (double)kept.y * sc);
          slab[i1] = mk<T2>(0, 0);
        }
        __syncthreads();
        if (syn && tid == 0) syn[rnd * kNStab + u.stab] = (uint8_t)(m ^ u.offset);
      }
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
                  b->d_idx, b->d_idx_u, b->d_snap};
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
    k_batch_u<<<b->num_sms * b->u_ctas_per_sm, 256, kUSmem, b->side>>>(a);
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
                     (void**)&b->d_idx_u, (void**)&b->d_snap};
  const size_t sizes[] = {sizeof(ProgOp) * (b->prog.ops.size() + 1), sizeof(BlockInfo) * kNStab,
                          sizeof(ProgOp) * (b->iprog.ops.size() + 1), sizeof(BlockInfo) * kNStab,
                          sizeof(b->prog.mats), (size_t)kNAmp * 16, (size_t)kNAmp * 8,
                          sizeof(qec_noise) * max_traj, sizeof(int32_t) * max_traj, sizeof(uint64_t) * max_traj,
                          sizeof(BatchCtl), syn_bytes, (size_t)max_traj * kND, (size_t)max_traj,
                          sizeof(ProgOp) * (b->uprog.ops.size() + 1), sizeof(UItem) * (b->uprog.items.size() + 1),
                          sizeof(ProgOp) * (b->iuprog.ops.size() + 1), sizeof(UItem) * (b->iuprog.items.size() + 1),
                          (size_t)kUAmp * 16, (size_t)kUAmp * 8, sizeof(uint32_t) * max_traj,
                          sizeof(uint32_t) * max_traj, sizeof(double2) * kNAmp};
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
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->u_ctas_per_sm, k_batch_u, 256, kUSmem);
  if (e != cudaSuccess || b->u_ctas_per_sm < 1)
    return bail(bfail(QEC_ECUDA, "unreduced batched kernel does not fit an SM"));
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
  for (uint32_t i = 0; i < n; ++i) ((kind[i] & 2) ? b->h_idx_u : b->h_idx).push_back(i);
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
  if (!b || !chosen_warps || !best_ms) return bfail(QEC_EINVAL, "null argument");
  const int cand[] = {2, 4, 6, 8, 10};
  int best = -1;
  float best_t = 0.f;
  for (int w : cand) {
    if (set_shape(b, w) != QEC_OK) continue;
    float t = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {   // first run warms up
      qec_status st = qec_batch_run(b, seed, n, traj, kind, noise, nullptr, nullptr, nullptr);
      if (st) return st;
      if (rep) t = b->last_ms;
    }
    if (best < 0 || t < best_t) {
      best = w;
      best_t = t;
    }
  }
  if (best < 0) return bfail(QEC_EUNSUPPORTED, "no batched kernel shape fits");
  qec_status st = set_shape(b, best);
  if (st) return st;
  *chosen_warps = best;
  *best_ms = best_t;
  return QEC_OK;
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
