// Trajectory kernels for GB300 (sm_103a).
//
// Per stabilizer of a round (Sec. II.B: one stabilizer circuit at a time on the
// reused ancilla) the ancilla starts in |0>, so the block's unitary U acts on
// the data register through two Kraus matrices K_m = <m|U|0> (16x16 on its <= 4
// data qubits).  A measurement is then one FP64-accumulated probability pass
// P(1) = <psi|K1^dag K1|psi> / <psi|psi> over the register (warp shuffle ->
// block -> last-CTA reduction in a fixed order), an on-device outcome
// u < P(1), and one pass psi <- K_m psi / sqrt(<psi|psi>) that collapses,
// renormalises and resets in one go.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.hpp"
#include "ozaki.cuh"

namespace qec {

template <typename T> struct V2;
template <> struct V2<double> { using t = double2; };
template <> struct V2<float> { using t = float2; };

__device__ __forceinline__ double2 to_v2(double2 v, double*) { return v; }

// Shared-memory loads the compiler may not hoist out of the group loop (hoisting all
// 256 matrix entries into registers would spill).
__device__ __forceinline__ double2 lds_v2(const double2* p) {
  double2 r;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return r;
}
// Two consecutive complex entries p[0], p[1]: one 16-byte load for float (p 16-byte aligned),
// two for double.
__device__ __forceinline__ void lds_pair(const float2* p, float2& a, float2& b) {
  float4 r;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"((unsigned)__cvta_generic_to_shared(p)));
  a = make_float2(r.x, r.y);
  b = make_float2(r.z, r.w);
}
__device__ __forceinline__ double2 lds_v2(const double2* p);
__device__ __forceinline__ void lds_pair(const double2* p, double2& a, double2& b) {
  a = lds_v2(p);
  b = lds_v2(p + 1);
}

__device__ __forceinline__ float2 lds_v2(const float2* p) {
  float2 r;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return r;
}
__device__ __forceinline__ float2 to_v2(double2 v, float*) { return make_float2((float)v.x, (float)v.y); }

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of two values (fixed shuffle tree, then warp 0); result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh /* >= 2*32 */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) { sh[wid] = a; sh[32 + wid] = b; }
  __syncthreads();
  if (wid == 0) {
    a = lane < nw ? sh[lane] : 0.0;
    b = lane < nw ? sh[32 + lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
  __syncthreads();
}

// ---- instantiate: draw this trajectory's noise and fuse every block -----------------------
__device__ void inst_block(const InstArgs& a, double2* U, double (*sm)[16][2], int* scode,
                           int blk, uint64_t seed, uint64_t traj) {
  const int k = blk % a.nstab;
  const int rnd = a.round_base + blk / a.nstab;
  const BlockInfo bi = a.blocks[k];
  const int w = bi.w, C = 1 << w;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < 32 * 16; i += nt) {
    int r = i / 16, c = i % 16;
    U[i] = make_double2((r < C && r == c) ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int oi = bi.op_begin; oi < bi.op_end; ++oi) {
    const ProgOp op = a.ops[oi];
    if (op.kind == OP_T1 || op.kind == OP_T2) {
      if (tid == 0) *scode = twirl_fires(op, a.prob[op.pidx], seed, traj, rnd) ? 1 : 0;
      __syncthreads();
      const int fire = *scode;
      __syncthreads();
      if (!fire) continue;
      if (op.kind == OP_T1) {
        for (int it = tid; it < items_1q(w); it += nt) apply1_item(U, w, op.q0, sm[op.mat], it);
      } else {
        for (int it = tid; it < items_2q(w); it += nt) apply2_item(U, w, op.q0, op.q1, sm[op.mat], it);
      }
      __syncthreads();
      continue;
    }
    if (op.kind == OP_N1 || op.kind == OP_N2) {
      if (tid == 0) {
        int code = noise_code(op, a.prob[op.pidx], seed, traj, rnd);
        *scode = code;
        if (code && a.events && a.ctl) {
          unsigned int e = atomicAdd(&a.ctl->n_events, 1u);
          if (e < a.ctl->ev_cap) {
            int32_t* ev = a.events + 5 * (size_t)e;
            ev[0] = (int32_t)traj; ev[1] = rnd; ev[2] = op.step; ev[3] = (int32_t)op.site;
            ev[4] = code;
          }
        }
      }
      __syncthreads();
      const int code = *scode;
      __syncthreads();
      if (code == 0) continue;
      if (op.kind == OP_N1) {
        for (int it = tid; it < items_1q(w); it += nt) apply1_item(U, w, op.q0, sm[code], it);
      } else {
        const int pa = code >> 2, pd = code & 3;
        if (pa) for (int it = tid; it < items_1q(w); it += nt) apply1_item(U, w, op.q0, sm[pa], it);
        __syncthreads();
        if (pd) for (int it = tid; it < items_1q(w); it += nt) apply1_item(U, w, op.q1, sm[pd], it);
      }
    } else if (op.kind == OP_U1) {
      for (int it = tid; it < items_1q(w); it += nt) apply1_item(U, w, op.q0, sm[op.mat], it);
    } else {
      for (int it = tid; it < items_2q(w); it += nt) apply2_item(U, w, op.q0, op.q1, sm[op.mat], it);
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_instantiate(InstArgs a) {
  using T2 = typename V2<T>::t;
  __shared__ double2 U[32 * 16];
  __shared__ double sm[M_COUNT][16][2];
  __shared__ int scode;
  for (int i = threadIdx.x; i < M_COUNT * 32; i += blockDim.x) (&sm[0][0][0])[i] = a.mats[i];
  __syncthreads();
  const uint64_t seed = a.ctl ? a.ctl->seed : 0ull;
  const uint64_t traj = a.ctl ? a.ctl->traj : 0ull;
  const int blk = blockIdx.x;
  inst_block(a, U, sm, &scode, blk, seed, traj);
  const int k = blk % a.nstab;
  const int C = 1 << a.blocks[k].w;
  T2* out = reinterpret_cast<T2*>(a.kraus) + (size_t)blk * KRAUS_STRIDE;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    const int r = i / 16, c = i % 16;
    double2 k0 = make_double2(0, 0), k1 = make_double2(0, 0), mm = make_double2(0, 0);
    if (r < C && c < C) {
      k0 = U[r * 16 + c];
      k1 = U[(C + r) * 16 + c];
      for (int x = 0; x < C; ++x) {           // M_rc = sum_x conj(K1_xr) K1_xc
        double2 p = U[(C + x) * 16 + r], q = U[(C + x) * 16 + c];
        mm.x += p.x * q.x + p.y * q.y;
        mm.y += p.x * q.y - p.y * q.x;
      }
    }
    out[i] = to_v2(k0, (T*)nullptr);
    out[256 + i] = to_v2(k1, (T*)nullptr);
    out[512 + i] = to_v2(mm, (T*)nullptr);
  }
  if (threadIdx.x == 0) {
    const int rnd = a.round_base + blk / a.nstab;
    a.u[blk] = uniform53(draw(seed, traj, (uint64_t)rnd, 0u, (uint32_t)(a.nd + k), TAG_MEASURE).v[0]);
  }
}

// ---- probability pass: A = <psi|M|psi>, N = <psi|psi>, then the outcome ----------------
// Register index of member 0 of group g: insert a zero bit at each block qubit (ascending).
template <int W>
__device__ __forceinline__ uint32_t group_base(uint32_t g, const int (&q)[4]) {
#pragma unroll
  for (int j = 0; j < W; ++j) g = ((g >> q[j]) << (q[j] + 1)) | (g & ((1u << q[j]) - 1u));
  return g;
}

template <int W>
__device__ __forceinline__ void load_q(const PassArgs& a, int (&q)[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) q[j] = j < W ? a.q[j] : 0;
}

// Offset of member l of a group (bit j of l -> register bit q[j]).
template <int W>
__device__ __forceinline__ uint32_t member_off(int l, const int (&q)[4]) {
  uint32_t o = 0;
#pragma unroll
  for (int j = 0; j < W; ++j) o |= (uint32_t)((l >> j) & 1) << q[j];
  return o;
}

// Register offset of tile tix in a tiled pass: bit j of tix goes to register bit obits[j], j < nout
// (nout <= 25 < 32).  Lane j deposits bit j (obit = obits[lane], loaded once per thread) and the warp
// ORs the lanes' bits: one step per thread instead of a loop over nout bits.  Every lane of the warp
// must call it with the same tix.
__device__ __forceinline__ uint32_t tile_base_warp(uint32_t tix, int nout, int obit) {
  const int lane = threadIdx.x & 31;
  return __reduce_or_sync(0xffffffffu, lane < nout ? ((tix >> lane) & 1u) << obit : 0u);
}

// End of a probability pass: block sums of (A, N) into per-CTA partials; the last CTA to finish
// (ticket) sums the partials in a fixed order, draws the outcome m (u < A/N, or the forced value),
// stores A, N, m and the syndrome bit, and resets the ticket.  Deterministic for a fixed grid.
__device__ void prob_finish(const PassArgs& a, double accA, double accN, double* sred, int* s_last) {
  block_sum2(accA, accN, sred);
  if (threadIdx.x == 0) {
    a.partials[2 * blockIdx.x] = accA;
    a.partials[2 * blockIdx.x + 1] = accN;
    __threadfence();
    const unsigned int t = atomicAdd(&a.ctl->ticket, 1u);
    *s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  double sA = 0.0, sN = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    sA += __ldcg(&a.partials[2 * i]);
    sN += __ldcg(&a.partials[2 * i + 1]);
  }
  block_sum2(sA, sN, sred);
  if (threadIdx.x == 0) {
    const double p1 = sA / sN;
    const int m = a.forced >= 0 ? a.forced : (*a.u < p1 ? 1 : 0);
    *a.A = sA;
    if (a.store_n) *a.N = sN;
    *a.m = m;
    if (a.syn) {
      const unsigned long long t = a.ctl->traj - a.ctl->first;
      a.syn[t * (unsigned long long)a.syn_stride + a.syn_idx] = (uint8_t)(m ^ a.offset);
    }
    a.ctl->ticket = 0u;
  }
}

// The bounded probability pass's end: block sums of (A^, N, bound) into 3 partials per CTA; the last
// CTA sums them in a fixed order and decides the outcome only if |u N - A^| exceeds twice the bound
// plus 1e-10 (A^ + N) (the exact pass's own rounding, with room), where the exact pass must decide
// the same way; it then stores A^, N (bit-identical to the exact pass's N), m and the syndrome bit.
// Otherwise (or with ctl->prob_force_exact) it sets ctl->prob_uncertain and stores nothing.
__device__ void prob_finish_bounded(const PassArgs& a, double accA, double accN, double accE, double* sred,
                                    int* s_last, bool n_always = false) {
  double dummy = 0.0;
  block_sum2(accA, accN, sred);
  __syncthreads();
  block_sum2(accE, dummy, sred);
  if (threadIdx.x == 0) {
    a.partials[3 * blockIdx.x] = accA;
    a.partials[3 * blockIdx.x + 1] = accN;
    a.partials[3 * blockIdx.x + 2] = accE;
    __threadfence();
    const unsigned int t = atomicAdd(&a.ctl->ticket, 1u);
    *s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  double sA = 0.0, sN = 0.0, sE = 0.0, d2 = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    sA += __ldcg(&a.partials[3 * i]);
    sN += __ldcg(&a.partials[3 * i + 1]);
    sE += __ldcg(&a.partials[3 * i + 2]);
  }
  block_sum2(sA, sN, sred);
  __syncthreads();
  block_sum2(sE, d2, sred);
  if (threadIdx.x == 0) {
    bool decided = true;
    int m = a.forced;
    if (m < 0) {
      const double u = *a.u;
      decided = !a.ctl->prob_force_exact && fabs(u * sN - sA) > 2.0 * sE + 1e-10 * (sA + sN);
      m = u < sA / sN ? 1 : 0;
    }
    a.ctl->prob_uncertain = decided ? 0u : 1u;
    if (n_always) *a.N = sN;   // the fused pass's norm estimate renormalises whichever pass decides
    if (decided) {
      *a.A = sA;
      if (!n_always) *a.N = sN;
      *a.m = m;
      if (a.syn) {
        const unsigned long long t = a.ctl->traj - a.ctl->first;
        a.syn[t * (unsigned long long)a.syn_stride + a.syn_idx] = (uint8_t)(m ^ a.offset);
      }
    }
    a.ctl->ticket = 0u;
  }
}

template <typename T, int W>
__global__ void __launch_bounds__(256) k_prob(PassArgs a) {
  using T2 = typename V2<T>::t;
  constexpr int C = 1 << W;
  __shared__ T2 sM[C * C];
  __shared__ double sred[64];
  __shared__ int s_last;
  const T2* Mg = reinterpret_cast<const T2*>(a.kraus) + 512;
  for (int i = threadIdx.x; i < C * C; i += blockDim.x) sM[i] = Mg[(i / C) * 16 + (i % C)];
  __syncthreads();
  int q[4];
  load_q<W>(a, q);
  uint32_t off[C];
#pragma unroll
  for (int l = 0; l < C; ++l) off[l] = member_off<W>(l, q);
  const T2* src = reinterpret_cast<const T2*>(a.src);
  const uint32_t G = 1u << (a.D - W);
  double accA = 0.0, accN = 0.0;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const uint32_t base = group_base<W>(g, q);
    T2 v[C];
#pragma unroll
    for (int l = 0; l < C; ++l) v[l] = src[base + off[l]];
    // <v|M|v> = sum_i M_ii |v_i|^2 + 2 Re sum_i conj(v_i) sum_{j>i} M_ij v_j  (M Hermitian);
    // every product is an FMA into its accumulator.
    T cross = 0, diag = 0, sn = 0;
#pragma unroll
    for (int i = 0; i < C; ++i) {
      T tr = 0, ti = 0;
#pragma unroll
      for (int j = i + 1; j < C; ++j) {
        const T2 m = lds_v2(&sM[i * C + j]);
        tr = fma_t(m.x, v[j].x, tr);
        tr = fma_t(-m.y, v[j].y, tr);
        ti = fma_t(m.x, v[j].y, ti);
        ti = fma_t(m.y, v[j].x, ti);
      }
      cross = fma_t(v[i].x, tr, cross);
      cross = fma_t(v[i].y, ti, cross);
      const T nv = fma_t(v[i].x, v[i].x, v[i].y * v[i].y);
      diag = fma_t(lds_v2(&sM[i * C + i]).x, nv, diag);
      sn += nv;
    }
    accA += (double)(2 * cross + diag);
    accN += (double)sn;
  }
  prob_finish(a, accA, accN, sred, &s_last);
}

// ---- apply pass: psi <- K_m psi / sqrt(N) ---------------------------------------------
template <typename T, int W>
__global__ void __launch_bounds__(256) k_apply(PassArgs a) {
  using T2 = typename V2<T>::t;
  constexpr int C = 1 << W;
  __shared__ T2 sK[C * C];
  const int m = *a.m;
  const double scale = 1.0 / sqrt(*a.N);
  const T2* Kg = reinterpret_cast<const T2*>(a.kraus) + (m ? 256 : 0);
  for (int i = threadIdx.x; i < C * C; i += blockDim.x) {
    T2 kv = Kg[(i / C) * 16 + (i % C)];
    kv.x = (T)((double)kv.x * scale);
    kv.y = (T)((double)kv.y * scale);
    sK[i] = kv;
  }
  __syncthreads();
  int q[4];
  load_q<W>(a, q);
  uint32_t off[C];
#pragma unroll
  for (int l = 0; l < C; ++l) off[l] = member_off<W>(l, q);
  const T2* src = reinterpret_cast<const T2*>(a.src);
  T2* dst = reinterpret_cast<T2*>(a.dst);
  const uint32_t G = 1u << (a.D - W);
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const uint32_t base = group_base<W>(g, q);
    T2 v[C];
#pragma unroll
    for (int l = 0; l < C; ++l) v[l] = src[base + off[l]];
#pragma unroll
    for (int r = 0; r < C; ++r) {
      T sr = 0, si = 0;
#pragma unroll
      for (int c = 0; c < C; ++c) {   // 4 FMAs per complex multiply-add
        const T2 k = lds_v2(&sK[r * C + c]);
        sr = fma_t(k.x, v[c].x, sr);
        sr = fma_t(-k.y, v[c].y, sr);
        si = fma_t(k.x, v[c].y, si);
        si = fma_t(k.y, v[c].x, si);
      }
      T2 o;
      o.x = sr;
      o.y = si;
      dst[base + off[r]] = o;
    }
  }
}

// The guessed raw outcome of block a: the forced one, else the same stabilizer's raw outcome one round
// earlier (the init round's, forced to offset, for the first noisy round).
__device__ __forceinline__ int spec_guess(const PassArgs& a) {
  if (a.forced >= 0) return a.forced;
  if (a.spec_prev < 0 || !a.syn) return a.offset;
  const unsigned long long t = a.ctl->traj - a.ctl->first;
  return (int)(a.syn[t * (unsigned long long)a.syn_stride + a.spec_prev] & 1u) ^ a.offset;
}

// End of a speculative (FIX = false) or corrective (FIX = true) pass (Sec. II.B, evaluated as the
// tensor-core k_ozs below describes): block sums of (Nin^ = |input|^2, its bound) and (Y^ = |output|^2,
// its bound) into 4 partials per CTA; the last CTA sums them in a fixed order and stores Y^ as the
// next block's N.  The speculative pass then decides where |u N' - P(1) N'| exceeds twice the summed
// bounds plus 1e-10 (N' + Y^), N' = Nin^ / N, P(1) N' = Y^ for g = 1 and N' - Y^ for g = 0, and
// otherwise flags the exact pass.  exact: the sums are FP64 sums of the FP64 values themselves (the
// CUDA-core pass) and decide every outcome directly, as the FP64 probability pass does.
template <bool FIX>
__device__ void spec_finish(const FusedArgs& f, int g, double nI, double rI, double nO, double rO, double* sred,
                            int* s_last, bool exact = false) {
  const PassArgs& a = f.ap;
  block_sum2(nI, rI, sred);
  block_sum2(nO, rO, sred);
  if (threadIdx.x == 0) {
    double* p = a.partials + 4 * blockIdx.x;
    p[0] = nI;
    p[1] = rI;
    p[2] = nO;
    p[3] = rO;
    __threadfence();
    const unsigned int t = atomicAdd(&a.ctl->ticket, 1u);
    *s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  double sI = 0.0, sRI = 0.0, sO = 0.0, sRO = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    sI += __ldcg(&a.partials[4 * i]);
    sRI += __ldcg(&a.partials[4 * i + 1]);
    sO += __ldcg(&a.partials[4 * i + 2]);
    sRO += __ldcg(&a.partials[4 * i + 3]);
  }
  block_sum2(sI, sRI, sred);
  block_sum2(sO, sRO, sred);
  if (threadIdx.x == 0) {
    if (f.n_next) *f.n_next = sO;
    if (FIX) {
      atomicAdd(&a.ctl->spec_misses, 1ull);
    } else {
      const double inv = f.spec_unit ? 1.0 : 1.0 / *a.N;   // the inputs' scale squared
      const double Np = sI * inv, rNp = sRI * inv;
      const double A1 = g ? sO : Np - sO;                  // P(1) N'
      bool decided = true;
      int m = a.forced;
      if (m < 0) {
        const double u = *a.u;
        decided = exact || (!a.ctl->prob_force_exact && fabs(u * Np - A1) > 2.0 * (rNp + sRO) + 1e-10 * (Np + sO));
        m = u * Np < A1 ? 1 : 0;
      }
      a.ctl->prob_uncertain = decided ? 0u : 1u;
      if (decided) {
        *a.A = A1;
        *a.m = m;
        if (a.syn) {
          const unsigned long long t = a.ctl->traj - a.ctl->first;
          a.syn[t * (unsigned long long)a.syn_stride + a.syn_idx] = (uint8_t)(m ^ a.offset);
        }
      }
    }
    a.ctl->ticket = 0u;
  }
}

// ---- speculative FP64 pass (QEC_C128, and QEC_C128_TC where the tensor-core tile does not fit) ----
// The order of evaluation of the tensor-core k_ozs (Sec. II.B; guess = the same stabilizer's outcome
// one round earlier): y = K_g psi / sqrt(N) out of place, with Nin = sum |psi|^2 and Y = sum |y|^2
// summed in FP64 per thread; the last CTA decides u N' < P(1) N' (N' = Nin / N; P(1) N' = Y for
// g = 1, N' - Y for g = 0) and stores Y as the next block's N.  FIX: the corrective apply of the
// decided K_m from the untouched input, only where m != g.  Grid-stride over groups as k_apply, so
// every sum and outcome is the same in every run for a fixed grid.
template <int W, bool FIX>
__global__ void __launch_bounds__(256) k_apply_spec(FusedArgs f) {
  const PassArgs& a = f.ap;
  const int gs = spec_guess(a);
  const int m = FIX ? *a.m : gs;
  if (FIX && m == gs) return;
  constexpr int C = 1 << W;
  __shared__ double2 sK[C * C];
  __shared__ double sred[64];
  __shared__ int s_last;
  const double scale = f.spec_unit ? 1.0 : 1.0 / sqrt(*a.N);
  const double2* Kg = reinterpret_cast<const double2*>(a.kraus) + (m ? 256 : 0);
  for (int i = threadIdx.x; i < C * C; i += blockDim.x) {
    double2 kv = Kg[(i / C) * 16 + (i % C)];
    kv.x *= scale;
    kv.y *= scale;
    sK[i] = kv;
  }
  __syncthreads();
  int q[4];
  load_q<W>(a, q);
  uint32_t off[C];
#pragma unroll
  for (int l = 0; l < C; ++l) off[l] = member_off<W>(l, q);
  const double2* src = reinterpret_cast<const double2*>(a.src);
  double2* dst = reinterpret_cast<double2*>(a.dst);
  const uint32_t G = 1u << (a.D - W);
  double accI = 0.0, accO = 0.0;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const uint32_t base = group_base<W>(g, q);
    double2 v[C];
#pragma unroll
    for (int l = 0; l < C; ++l) {
      v[l] = src[base + off[l]];
      accI = fma(v[l].x, v[l].x, fma(v[l].y, v[l].y, accI));
    }
#pragma unroll
    for (int r = 0; r < C; ++r) {
      double sr = 0, si = 0;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const double2 k = lds_v2(&sK[r * C + c]);
        sr = fma(k.x, v[c].x, sr);
        sr = fma(-k.y, v[c].y, sr);
        si = fma(k.x, v[c].y, si);
        si = fma(k.y, v[c].x, si);
      }
      dst[base + off[r]] = make_double2(sr, si);
      accO = fma(sr, sr, fma(si, si, accO));
    }
  }
  spec_finish<FIX>(f, gs, accI, 0.0, accO, 0.0, sred, &s_last, true);
}

// ---- fused pass: apply block s, then probability of block s+1, per shared-memory tile ----
template <int W>
__device__ __forceinline__ uint32_t local_base(uint32_t g, const int (&q)[4]) {
#pragma unroll
  for (int j = 0; j < W; ++j) g = ((g >> q[j]) << (q[j] + 1)) | (g & ((1u << q[j]) - 1u));
  return g;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Tiles stream through two shared-memory buffers: while tile i is computed, tile i+1 arrives by
// 16-byte asynchronous copies (runs of 2^lb contiguous amplitudes, >= 128 bytes, 16-byte aligned).
template <typename T, int W, int W2>
__global__ void __launch_bounds__(256) k_fused(FusedArgs f) {
  using T2 = typename V2<T>::t;
  constexpr int C = 1 << W, C2 = 1 << W2;
  constexpr int CH = 16 / sizeof(T2);   // amplitudes per 16-byte copy
  extern __shared__ __align__(16) unsigned char fsm[];
  const uint32_t tsz = 1u << f.nt, lmask = (1u << f.lb) - 1u;
  T2* buf0 = reinterpret_cast<T2*>(fsm);
  T2* buf1 = buf0 + tsz;
  uint32_t* hoff = reinterpret_cast<uint32_t*>(buf1 + tsz);
  __shared__ __align__(16) T2 sK[C * C];
  __shared__ __align__(16) T2 sM[C2 * C2];
  __shared__ double sred[64];
  __shared__ int s_last;
  {
    const int m = *f.ap.m;
    const double scale = 1.0 / sqrt(*f.ap.N);
    const T2* Kg = reinterpret_cast<const T2*>(f.ap.kraus) + (m ? 256 : 0);
    for (int i = threadIdx.x; i < C * C; i += blockDim.x) {
      T2 kv = Kg[(i / C) * 16 + (i % C)];
      kv.x = (T)((double)kv.x * scale);
      kv.y = (T)((double)kv.y * scale);
      sK[i] = kv;
    }
    const T2* Mg = reinterpret_cast<const T2*>(f.pr.kraus) + 512;
    for (int i = threadIdx.x; i < C2 * C2; i += blockDim.x) sM[i] = Mg[(i / C2) * 16 + (i % C2)];
    const int nh = f.nt - f.lb;
    for (int h = threadIdx.x; h < (1 << nh); h += blockDim.x) {
      uint32_t o = 0;
      for (int j = 0; j < nh; ++j) o |= (uint32_t)((h >> j) & 1) << f.hbits[j];
      hoff[h] = o;
    }
  }
  __syncthreads();
  int qa[4], qp[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    qa[j] = j < W ? f.qa[j] : 0;
    qp[j] = j < W2 ? f.qp[j] : 0;
  }
  uint32_t offa[C], offp[C2];
#pragma unroll
  for (int l = 0; l < C; ++l) offa[l] = member_off<W>(l, qa);
#pragma unroll
  for (int l = 0; l < C2; ++l) offp[l] = member_off<W2>(l, qp);
  const T2* src = reinterpret_cast<const T2*>(f.ap.src);
  T2* dst = reinterpret_cast<T2*>(f.ap.dst);
  const uint32_t ntile = 1u << f.nout;
  const int obit = (threadIdx.x & 31) < (unsigned)f.nout ? f.obits[threadIdx.x & 31] : 0;
  auto tile_base = [&](uint32_t tix) { return tile_base_warp(tix, f.nout, obit); };
  auto issue = [&](uint32_t tix, T2* buf) {
    const uint32_t tb = tile_base(tix);
    for (uint32_t e = threadIdx.x * CH; e < tsz; e += blockDim.x * CH)
      cp_async16(buf + e, src + (tb | hoff[e >> f.lb] | (e & lmask)));
    cp_async_commit();
  };
  double accA = 0.0, accN = 0.0;
  uint32_t tix = blockIdx.x;
  if (tix < ntile) issue(tix, buf0);
  int cur = 0;
  for (; tix < ntile; tix += gridDim.x) {
    T2* tile = cur ? buf1 : buf0;
    const uint32_t nxt = tix + gridDim.x;
    if (nxt < ntile) issue(nxt, cur ? buf0 : buf1);
    else cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    for (uint32_t g = threadIdx.x; g < (tsz >> W); g += blockDim.x) {
      const uint32_t b = local_base<W>(g, qa);
      T2 v[C];
#pragma unroll
      for (int l = 0; l < C; ++l) v[l] = tile[b + offa[l]];
#pragma unroll
      for (int r = 0; r < C; ++r) {
        T sr = 0, si = 0;
#pragma unroll
        for (int c = 0; c < C; c += 2) {
          T2 k0, k1;
          lds_pair(&sK[r * C + c], k0, k1);
          sr = fma_t(k0.x, v[c].x, sr);
          sr = fma_t(-k0.y, v[c].y, sr);
          si = fma_t(k0.x, v[c].y, si);
          si = fma_t(k0.y, v[c].x, si);
          sr = fma_t(k1.x, v[c + 1].x, sr);
          sr = fma_t(-k1.y, v[c + 1].y, sr);
          si = fma_t(k1.x, v[c + 1].y, si);
          si = fma_t(k1.y, v[c + 1].x, si);
        }
        T2 o;
        o.x = sr;
        o.y = si;
        tile[b + offa[r]] = o;
      }
    }
    __syncthreads();
    T tA = 0, tN = 0;   // this thread's sums over its groups of the tile (complex64: added in FP64 once per tile)
    for (uint32_t g = threadIdx.x; g < (tsz >> W2); g += blockDim.x) {
      const uint32_t b = local_base<W2>(g, qp);
      T2 v[C2];
#pragma unroll
      for (int l = 0; l < C2; ++l) v[l] = tile[b + offp[l]];
      T cross = 0, diag = 0, sn = 0;
#pragma unroll
      for (int i = 0; i < C2; ++i) {
        T tr = 0, ti = 0;
        int j = i + 1;
        if (j & 1) {               // reach an even column, then take pairs
          if (j < C2) {
            const T2 m = lds_v2(&sM[i * C2 + j]);
            tr = fma_t(m.x, v[j].x, tr);
            tr = fma_t(-m.y, v[j].y, tr);
            ti = fma_t(m.x, v[j].y, ti);
            ti = fma_t(m.y, v[j].x, ti);
          }
          ++j;
        }
#pragma unroll
        for (; j < C2; j += 2) {
          T2 m0, m1;
          lds_pair(&sM[i * C2 + j], m0, m1);
          tr = fma_t(m0.x, v[j].x, tr);
          tr = fma_t(-m0.y, v[j].y, tr);
          ti = fma_t(m0.x, v[j].y, ti);
          ti = fma_t(m0.y, v[j].x, ti);
          tr = fma_t(m1.x, v[j + 1].x, tr);
          tr = fma_t(-m1.y, v[j + 1].y, tr);
          ti = fma_t(m1.x, v[j + 1].y, ti);
          ti = fma_t(m1.y, v[j + 1].x, ti);
        }
        cross = fma_t(v[i].x, tr, cross);
        cross = fma_t(v[i].y, ti, cross);
        const T nv = fma_t(v[i].x, v[i].x, v[i].y * v[i].y);
        diag = fma_t(lds_v2(&sM[i * C2 + i]).x, nv, diag);
        sn += nv;
      }
      if constexpr (sizeof(T) == 4) {
        tA += 2 * cross + diag;
        tN += sn;
      } else {
        accA += (double)(2 * cross + diag);
        accN += (double)sn;
      }
    }
    if constexpr (sizeof(T) == 4) {
      accA += (double)tA;
      accN += (double)tN;
    }
    const uint32_t tb = tile_base(tix);
    for (uint32_t e = threadIdx.x * CH; e < tsz; e += blockDim.x * CH)
      *reinterpret_cast<float4*>(dst + (tb | hoff[e >> f.lb] | (e & lmask))) = *reinterpret_cast<const float4*>(tile + e);
    __syncthreads();
    cur ^= 1;
  }
  cp_async_wait<0>();
  prob_finish(f.pr, accA, accN, sred, &s_last);
}

// ---- speculative complex64 pass (QEC_C64), per shared-memory tile -------------------------------
// The order of evaluation of k_apply_spec (Sec. II.B; guess = the same stabilizer's outcome one round
// earlier) on k_fused's double-buffered tiles of block a's qubits and the low register bits: the
// tile's groups are multiplied by K_g / sqrt(N) in FP32, in shared memory, with |in|^2 and |out|^2
// summed per thread in FP32 over the tile and in FP64 across tiles (as k_fused sums its
// probabilities); the tile is stored to the other working state.  The last CTA decides
// u N' < P(1) N' directly, as the complex64 probability pass does.  FIX: the corrective apply where
// the drawn outcome differs from g.
template <int W, bool FIX>
__global__ void __launch_bounds__(256) k_fused_spec(FusedArgs f) {
  const int gs = spec_guess(f.ap);
  const int m = FIX ? *f.ap.m : gs;
  if (FIX && m == gs) return;
  constexpr int C = 1 << W;
  constexpr int CH = 2;   // complex64 amplitudes per 16-byte copy
  extern __shared__ __align__(16) unsigned char fsm[];
  const uint32_t tsz = 1u << f.nt, lmask = (1u << f.lb) - 1u;
  float2* buf0 = reinterpret_cast<float2*>(fsm);
  float2* buf1 = buf0 + tsz;
  uint32_t* hoff = reinterpret_cast<uint32_t*>(buf1 + tsz);
  __shared__ __align__(16) float2 sK[C * C];
  __shared__ double sred[64];
  __shared__ int s_last;
  {
    const double scale = f.spec_unit ? 1.0 : 1.0 / sqrt(*f.ap.N);
    const float2* Kg = reinterpret_cast<const float2*>(f.ap.kraus) + (m ? 256 : 0);
    for (int i = threadIdx.x; i < C * C; i += blockDim.x) {
      float2 kv = Kg[(i / C) * 16 + (i % C)];
      kv.x = (float)((double)kv.x * scale);
      kv.y = (float)((double)kv.y * scale);
      sK[i] = kv;
    }
    const int nh = f.nt - f.lb;
    for (int h = threadIdx.x; h < (1 << nh); h += blockDim.x) {
      uint32_t o = 0;
      for (int j = 0; j < nh; ++j) o |= (uint32_t)((h >> j) & 1) << f.hbits[j];
      hoff[h] = o;
    }
  }
  __syncthreads();
  int qa[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) qa[j] = j < W ? f.qa[j] : 0;
  uint32_t offa[C];
#pragma unroll
  for (int l = 0; l < C; ++l) offa[l] = member_off<W>(l, qa);
  const float2* src = reinterpret_cast<const float2*>(f.ap.src);
  float2* dst = reinterpret_cast<float2*>(f.ap.dst);
  const uint32_t ntile = 1u << f.nout;
  const int obit = (threadIdx.x & 31) < (unsigned)f.nout ? f.obits[threadIdx.x & 31] : 0;
  auto tile_base = [&](uint32_t tix) { return tile_base_warp(tix, f.nout, obit); };
  auto issue = [&](uint32_t tix, float2* buf) {
    const uint32_t tb = tile_base(tix);
    for (uint32_t e = threadIdx.x * CH; e < tsz; e += blockDim.x * CH)
      cp_async16(buf + e, src + (tb | hoff[e >> f.lb] | (e & lmask)));
    cp_async_commit();
  };
  double accI = 0.0, accO = 0.0;
  uint32_t tix = blockIdx.x;
  if (tix < ntile) issue(tix, buf0);
  int cur = 0;
  for (; tix < ntile; tix += gridDim.x) {
    float2* tile = cur ? buf1 : buf0;
    const uint32_t nxt = tix + gridDim.x;
    if (nxt < ntile) issue(nxt, cur ? buf0 : buf1);
    else cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    float tI = 0.f, tO = 0.f;   // this thread's sums over its groups of the tile
    for (uint32_t g = threadIdx.x; g < (tsz >> W); g += blockDim.x) {
      const uint32_t b = local_base<W>(g, qa);
      float2 v[C];
#pragma unroll
      for (int l = 0; l < C; ++l) {
        v[l] = tile[b + offa[l]];
        tI = fmaf(v[l].x, v[l].x, fmaf(v[l].y, v[l].y, tI));
      }
#pragma unroll
      for (int r = 0; r < C; ++r) {
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int c = 0; c < C; c += 2) {
          float2 k0, k1;
          lds_pair(&sK[r * C + c], k0, k1);
          sr = fmaf(k0.x, v[c].x, sr);
          sr = fmaf(-k0.y, v[c].y, sr);
          si = fmaf(k0.x, v[c].y, si);
          si = fmaf(k0.y, v[c].x, si);
          sr = fmaf(k1.x, v[c + 1].x, sr);
          sr = fmaf(-k1.y, v[c + 1].y, sr);
          si = fmaf(k1.x, v[c + 1].y, si);
          si = fmaf(k1.y, v[c + 1].x, si);
        }
        tile[b + offa[r]] = make_float2(sr, si);
        tO = fmaf(sr, sr, fmaf(si, si, tO));
      }
    }
    accI += (double)tI;
    accO += (double)tO;
    __syncthreads();
    const uint32_t tb = tile_base(tix);
    for (uint32_t e = threadIdx.x * CH; e < tsz; e += blockDim.x * CH)
      *reinterpret_cast<float4*>(dst + (tb | hoff[e >> f.lb] | (e & lmask))) = *reinterpret_cast<const float4*>(tile + e);
    __syncthreads();
    cur ^= 1;
  }
  cp_async_wait<0>();
  spec_finish<FIX>(f, gs, accI, 0.0, accO, 0.0, sred, &s_last, true);
}

// ---- tensor-core complex64 fused pass (tcgen05, 3xTF32, FP32 accumulation in TMEM) --------
// A weight-4 block's 16x16 complex matrix acts on every 16-amplitude group of a tile as a real
// GEMM: rows = groups (M = 256 per tile, two M = 128 MMAs), K = 32 input reals (re, im
// interleaved), N = 32 output reals, B[n][k] = real embedding of the matrix.  Operands are
// split x = hi + lo in TF32 and D = Ahi.Bhi + Ahi.Blo + Alo.Bhi, accumulated in FP32 in
// tensor memory.  The probability pass of the next block is the same GEMM with its K1 on
// the regrouped tile, reduced as sum |D|^2.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle, 8-row x 16-byte core matrices.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= 1ull << 46;   // descriptor version of sm_100-class tensor cores
  return d;
}

// Float index of element (row r, k) of a K = 32 operand: core matrix (r/8, k/4) of 32 floats.
__device__ __forceinline__ int core_off32(int r, int k) { return ((r >> 3) * 8 + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3); }

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// TF32 MMA M = 128, N = 32, D = F32, A and B K-major.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(kIdescTf32), "r"(acc));
}

// Bounded wait for an mbarrier phase; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long limit = 40000000) {
  for (long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// Self-test of the bounded-wait path: waits on an mbarrier that nothing arrives on, gives up
// after `limit` polls and records the timeout in *status (bit 0), as the tensor-core pass does.
__global__ void k_wait_selftest(unsigned int* status, long limit) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (!mbar_wait(smem_u32(&mbar), 0, limit) && threadIdx.x == 0) atomicOr(status, 1u);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                 "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                 "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Writes the 3xTF32-split real embedding of a 16x16 complex matrix (times scale) as B operands.  A
// weight-2 block (w2) has its 4x4 matrix K in rows and columns 0..3; it is embedded as K (x) I on
// groups whose index bits 0..1 are its qubits and bits 2..3 two spectator qubits.
__device__ void build_b(const float2* Kg, double scale, float* Bhi, float* Blo, bool w2) {
  for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
    const int n = idx >> 5, k = idx & 31, r = n >> 1, c = k >> 1;
    const float2 kv = !w2 ? Kg[r * 16 + c] : ((r >> 2) == (c >> 2) ? Kg[(r & 3) * 16 + (c & 3)] : make_float2(0.f, 0.f));
    const double re = (double)kv.x * scale, im = (double)kv.y * scale;
    const float v = (float)((n & 1) ? ((k & 1) ? re : im) : ((k & 1) ? -im : re));
    const float hi = tf32_rna(v);
    Bhi[core_off32(n, k)] = hi;
    Blo[core_off32(n, k)] = tf32_rna(v - hi);
  }
}

// Two complex amplitudes = reals k .. k+3 of one row (k % 4 == 0): one 16-byte store per operand.
__device__ __forceinline__ void put_a4(float* Ahi, float* Alo, int row, int k, float2 a, float2 b) {
  float4 h, l;
  h.x = tf32_rna(a.x); l.x = tf32_rna(a.x - h.x);
  h.y = tf32_rna(a.y); l.y = tf32_rna(a.y - h.y);
  h.z = tf32_rna(b.x); l.z = tf32_rna(b.x - h.z);
  h.w = tf32_rna(b.y); l.w = tf32_rna(b.y - h.w);
  *reinterpret_cast<float4*>(Ahi + core_off32(row, k)) = h;
  *reinterpret_cast<float4*>(Alo + core_off32(row, k)) = l;
}

// 2 M-halves x 4 K-steps x 3 split terms; commit arrives on mbar.
__device__ __forceinline__ void issue_gemm(uint32_t tmem, const float* Ahi, const float* Alo, const float* Bhi,
                                           const float* Blo, uint32_t mbar) {
  const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint32_t d = tmem + 32u * h;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const uint32_t ko = 256u * s, mo = 16384u * h;
      umma_tf32(d, umma_desc(ah + mo + ko, 128, 1024), umma_desc(bh + ko, 128, 1024), s > 0);
      umma_tf32(d, umma_desc(ah + mo + ko, 128, 1024), umma_desc(bl + ko, 128, 1024), 1);
      umma_tf32(d, umma_desc(al + mo + ko, 128, 1024), umma_desc(bh + ko, 128, 1024), 1);
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// TF32 MMA M = 128, N = 32, D = F32, with A in tensor memory (row m in lane m, its K = 8 elements
// in 8 consecutive 32-bit columns from a_tmem) and B K-major in shared memory.
__device__ __forceinline__ void umma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bd, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
               ::"r"(d_tmem), "r"(a_tmem), "l"(bd), "r"(kIdescTf32), "r"(acc));
}

// Stores v[0..7] into 8 consecutive columns of this thread's lane (warp quarter rule as tcgen05.ld).
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}

// The probability GEMM of a regrouped tile whose 3xTF32 A operands are in tensor memory: M-half h
// has A_hi at columns ca + 64h .. + 31 and A_lo at ca + 64h + 32 .. + 63; D at column dc + 32h.
// 2 M-halves x 4 K-steps x 3 split terms, in the order of issue_gemm; commit arrives on mbar.
__device__ __forceinline__ void issue_gemm_ts(uint32_t tmem, uint32_t dc, uint32_t ca, const float* Bhi,
                                              const float* Blo, uint32_t mbar) {
  const uint64_t bh = umma_desc(smem_u32(Bhi), 128, 1024), bl = umma_desc(smem_u32(Blo), 128, 1024);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint32_t d = tmem + dc + 32u * h;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const uint32_t ah = tmem + ca + 64u * h + 8u * s, ko = (256u * s) >> 4;
      umma_tf32_ts(d, ah, bh + ko, s > 0);
      umma_tf32_ts(d, ah, bl + ko, 1);
      umma_tf32_ts(d, ah + 32u, bh + ko, 1);
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// Shared memory: the input tile (32 KiB), the first GEMM's 3xTF32 A operands (2 x 32 KiB; the
// updated tile takes their place once that GEMM has read them) and four 4 KiB B operands: 112 KiB,
// so two CTAs share an SM.  Tensor memory, 256 columns per CTA (two CTAs fill an SM's 512): D of
// the apply GEMM (columns 0..63), D of the probability GEMM (64..127) and that GEMM's A operands,
// the regrouped updated tile in TF32 hi and lo (128..255).  Tile addresses are computed from the
// bit lists (no offset table).
constexpr int kTcSmem = 8 * 4096 + 2 * 4 * 256 * 32 + 4 * 4 * 32 * 32;
constexpr uint32_t kTcColD2 = 64, kTcColA2 = 128;

// Per 4096-amplitude tile (256 groups of 16 amplitudes, one per thread):
//  1. gather each group of block s from the input tile as a row of K = 32 reals, split hi + lo in
//     TF32 into the A operands; the input buffer then takes the next tile's copy at once;
//  2. the apply GEMM (24 MMAs into TMEM); under it, the previous tile's probability sums;
//  3. its outputs, the updated tile, go where the A operands were;
//  4. regroup the updated tile by block s+1 (sum |psi|^2 for N), split it into tensor memory as the
//     probability GEMM's A, and store the updated tile to the register;
//  5. the probability GEMM (A from tensor memory), left running under the next tile's gather.
// Per-thread sums are taken in tile order, as one thread's tiles are fixed (b, b + grid, ...).
__global__ void __launch_bounds__(256, 2) k_fused_tc(FusedArgs f) {
  constexpr int C = 16;
  extern __shared__ __align__(128) unsigned char tsm[];
  const uint32_t tsz = 1u << f.nt, lmask = (1u << f.lb) - 1u;     // tsz = 4096 (checked by the launcher)
  float2* tile = reinterpret_cast<float2*>(tsm);
  float* Ahi = reinterpret_cast<float*>(tile + tsz);
  float* Alo = Ahi + 256 * 32;
  float2* outt = reinterpret_cast<float2*>(Ahi);                  // the updated tile (tile slots)
  float* Bahi = Alo + 256 * 32;
  float* Balo = Bahi + 32 * 32;
  float* Bphi = Balo + 32 * 32;
  float* Bplo = Bphi + 32 * 32;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_err;
  __shared__ double sred[64];
  __shared__ int s_last;
  const int tid = threadIdx.x, warp = tid >> 5;
  {
    const int m = *f.ap.m;
    const double scale = 1.0 / sqrt(*f.ap.N);
    build_b(reinterpret_cast<const float2*>(f.ap.kraus) + (m ? 256 : 0), scale, Bahi, Balo, f.ap.w == 2);
    build_b(reinterpret_cast<const float2*>(f.pr.kraus) + 256, 1.0, Bphi, Bplo, f.pr.w == 2);
    if (tid == 0) {
      s_err = 0;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_base)));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t mb1 = smem_u32(&mbar[0]), mb2 = smem_u32(&mbar[1]);
  int qa[4], qp[4], qas[4], qps[4];   // member bits (a weight-2 block's qubits, then spectators) and sorted
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    qa[j] = f.qa[j];
    qp[j] = f.qp[j];
    qas[j] = f.qa_s[j];
    qps[j] = f.qp_s[j];
  }
  // Tile slot of float2 e in shared memory: bits 1..3 (the 8-byte bank pair within a 16-byte
  // chunk's position) XOR a fold of the chunk index's higher bits, so group gathers spread over
  // the banks whichever tile bits a block occupies; bit 0 is kept, so 16-byte chunks stay whole.
  // The map is linear over XOR: slot(base + member) = slot(base) ^ slot(member) (disjoint bits).
  auto slot = [](uint32_t e) { return e ^ ((((e >> 4) ^ (e >> 7) ^ (e >> 10)) & 7u) << 1); };
  uint32_t offa[C], offp[C];
#pragma unroll
  for (int l = 0; l < C; ++l) {
    offa[l] = slot(member_off<4>(l, qa));
    offp[l] = slot(member_off<4>(l, qp));
  }
  // this thread's 16-byte chunks of a tile: chunk e = tid*2 + 512*i, i < 8; register offsets of their
  // high tile bits are the same for every tile
  uint32_t coff[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t e = (uint32_t)tid * 2 + 512u * i, h = e >> f.lb;
    uint32_t o = 0;
    for (int j = 0; j < f.nt - f.lb; ++j) o |= ((h >> j) & 1u) << f.hbits[j];
    coff[i] = o | (e & lmask);
  }
  // Thread tid owns row tid of both GEMMs: M-half tid / 128, TMEM lane tid % 128, which is in its
  // warp's lane quarter (32 (warp % 4) ..).
  const uint32_t sba = slot(local_base<4>((uint32_t)tid, qas)), sbp = slot(local_base<4>((uint32_t)tid, qps));
  uint32_t cd[8];   // slots of this thread's 16-byte chunks
#pragma unroll
  for (int i = 0; i < 8; ++i) cd[i] = slot((uint32_t)tid * 2 + 512u * i);
  const uint32_t tq = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t taddr = tq + 32u * (warp >> 2);                      // D of the apply GEMM, this row
  const uint32_t taddr2 = tq + kTcColD2 + 32u * (warp >> 2);          // D of the probability GEMM
  const uint32_t tA2 = tq + kTcColA2 + 64u * (warp >> 2);             // this row of its A (hi; lo at +32)
  const float2* src = reinterpret_cast<const float2*>(f.ap.src);
  float2* dst = reinterpret_cast<float2*>(f.ap.dst);
  const uint32_t ntile = 1u << f.nout;
  double accA = 0.0, accN = 0.0;
  uint32_t ph1 = 0, ph2 = 0;
  bool pending = false;   // a probability GEMM whose sums are not taken yet
  const int obit = (threadIdx.x & 31) < (unsigned)f.nout ? f.obits[threadIdx.x & 31] : 0;
  auto tile_base = [&](uint32_t tix) { return tile_base_warp(tix, f.nout, obit); };
  auto load_tile = [&](uint32_t tix) {
    const uint32_t tb = tile_base(tix);
#pragma unroll
    for (int i = 0; i < 8; ++i) cp_async16(tile + cd[i], src + (tb | coff[i]));
    cp_async_commit();
  };
  // sum of |y|^2 over this row's outputs of the probability GEMM (every thread waits on its barrier)
  auto take_sums = [&]() {
    if (!mbar_wait(mb2, ph2 & 1)) s_err = 1;
    ++ph2;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float d[32];
    tmem_ld32(taddr2, d);
    float sa = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) sa = fmaf(d[j], d[j], sa);
    accA += (double)sa;
  };
  if (blockIdx.x < ntile) load_tile(blockIdx.x);
  for (uint32_t tix = blockIdx.x; tix < ntile; tix += gridDim.x) {
    const uint32_t tb = tile_base(tix);
    cp_async_wait<0>();
    __syncthreads();   // the input tile is in; the previous tile's readers of the updated tile are done
#pragma unroll
    for (int l = 0; l < C; l += 2) put_a4(Ahi, Alo, tid, 2 * l, tile[sba ^ offa[l]], tile[sba ^ offa[l + 1]]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    // every thread has read the input tile: it takes the next tile's copy
    if (tix + gridDim.x < ntile) load_tile(tix + gridDim.x);
    if (tid == 0) issue_gemm(tmem, Ahi, Alo, Bahi, Balo, mb1);
    if (pending) take_sums();   // the previous tile's probability GEMM, under this tile's apply GEMM
    pending = false;
    if (!mbar_wait(mb1, ph1 & 1)) s_err = 1;
    ++ph1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (s_err) break;
    {
      float d[32];
      tmem_ld32(taddr, d);
#pragma unroll
      for (int r = 0; r < C; ++r) outt[sba ^ offa[r]] = make_float2(d[2 * r], d[2 * r + 1]);
    }
    __syncthreads();
    {
      // regroup by block s+1 into the probability GEMM's A (tensor memory), 4 members at a time
      float sn = 0.f;
#pragma unroll
      for (int l = 0; l < C; l += 4) {
        float hv[8], lv[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 v = outt[sbp ^ offp[l + q]];
          sn = fmaf(v.x, v.x, fmaf(v.y, v.y, sn));
          hv[2 * q] = tf32_rna(v.x);
          lv[2 * q] = tf32_rna(v.x - hv[2 * q]);
          hv[2 * q + 1] = tf32_rna(v.y);
          lv[2 * q + 1] = tf32_rna(v.y - hv[2 * q + 1]);
        }
        tmem_st8(tA2 + 2u * l, hv);
        tmem_st8(tA2 + 32u + 2u * l, lv);
      }
      accN += (double)sn;
    }
    // the updated tile to the register
#pragma unroll
    for (int i = 0; i < 8; ++i)
      *reinterpret_cast<float4*>(dst + (tb | coff[i])) = *reinterpret_cast<const float4*>(outt + cd[i]);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_sync();
    if (tid == 0) issue_gemm_ts(tmem, kTcColD2, kTcColA2, Bphi, Bplo, mb2);
    pending = true;
  }
  if (pending && !s_err) take_sums();
  cp_async_wait<0>();
  tc_sync();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  if (s_err && tid == 0) atomicOr(&f.pr.ctl->status, 1u);
  prob_finish(f.pr, accA, accN, sred, &s_last);
}

// Speculative complex64 pass on the tensor cores (QEC_C64_TC, weight-4 blocks): the order of
// evaluation of k_apply_spec (Sec. II.B; guess = the same stabilizer's outcome one round earlier)
// with k_fused_tc's 3xTF32 apply.  Per 4096-amplitude tile (256 groups of 16, one per thread):
//  1. gather the thread's group from the input tile, split hi + lo in TF32 straight into tensor memory
//     as the GEMM's A operand (the layout of k_fused_tc's probability GEMM), summing |in|^2;
//  2. the input buffer takes the copy of the tile two ahead (two input buffers, so that two tile
//     copies are in flight while one tile is computed);
//  3. the apply GEMM, A from tensor memory, B (K_g / sqrt(N)) from shared memory, D in columns 0..63;
//  4. its outputs into the updated tile in shared memory, summing |out|^2, then stored to the other
//     working state in whole 16-byte chunks.
// Sums in FP32 per tile, FP64 across tiles; the last CTA decides directly, as the complex64
// probability pass does.  FIX: the corrective apply where the drawn outcome differs from g.
// Shared memory: two input tiles and the updated tile (3 x 32 KiB) and B (8 KiB): 104 KiB, two CTAs
// per SM; tensor memory: 256 columns per CTA.
template <bool FIX>
__global__ void __launch_bounds__(256, 2) k_fused_tc_spec(FusedArgs f) {
  const int gs = spec_guess(f.ap);
  const int m = FIX ? *f.ap.m : gs;
  if (FIX && m == gs) return;
  constexpr int C = 16;
  extern __shared__ __align__(128) unsigned char tsm[];
  const uint32_t tsz = 1u << f.nt, lmask = (1u << f.lb) - 1u;     // tsz = 4096 (checked by the launcher)
  float2* tiles = reinterpret_cast<float2*>(tsm);                 // input tiles i even / odd
  float2* outt = tiles + 2 * tsz;                                 // the updated tile (tile slots)
  float* Bahi = reinterpret_cast<float*>(outt + tsz);
  float* Balo = Bahi + 32 * 32;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_err;
  __shared__ double sred[64];
  __shared__ int s_last;
  const int tid = threadIdx.x, warp = tid >> 5;
  {
    const double scale = f.spec_unit ? 1.0 : 1.0 / sqrt(*f.ap.N);
    build_b(reinterpret_cast<const float2*>(f.ap.kraus) + (m ? 256 : 0), scale, Bahi, Balo, f.ap.w == 2);
    if (tid == 0) {
      s_err = 0;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_base)));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t mb = smem_u32(&mbar);
  int qa[4], qas[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    qa[j] = f.qa[j];
    qas[j] = f.qa_s[j];
  }
  // tile slots and chunk offsets as in k_fused_tc
  auto slot = [](uint32_t e) { return e ^ ((((e >> 4) ^ (e >> 7) ^ (e >> 10)) & 7u) << 1); };
  uint32_t offa[C];
#pragma unroll
  for (int l = 0; l < C; ++l) offa[l] = slot(member_off<4>(l, qa));
  uint32_t coff[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t e = (uint32_t)tid * 2 + 512u * i, h = e >> f.lb;
    uint32_t o = 0;
    for (int j = 0; j < f.nt - f.lb; ++j) o |= ((h >> j) & 1u) << f.hbits[j];
    coff[i] = o | (e & lmask);
  }
  const uint32_t sba = slot(local_base<4>((uint32_t)tid, qas));
  uint32_t cd[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) cd[i] = slot((uint32_t)tid * 2 + 512u * i);
  // Thread tid owns row tid: M-half tid / 128, TMEM lane tid % 128 (its warp's lane quarter).
  const uint32_t tq = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t taddr = tq + 32u * (warp >> 2);                 // D, this row
  const uint32_t tA = tq + kTcColA2 + 64u * (warp >> 2);         // A of this row (hi; lo at +32)
  const float2* src = reinterpret_cast<const float2*>(f.ap.src);
  float2* dst = reinterpret_cast<float2*>(f.ap.dst);
  const uint32_t ntile = 1u << f.nout;
  double accI = 0.0, accO = 0.0;
  uint32_t ph = 0;
  const int obit = (threadIdx.x & 31) < (unsigned)f.nout ? f.obits[threadIdx.x & 31] : 0;
  auto tile_base = [&](uint32_t tix) { return tile_base_warp(tix, f.nout, obit); };
  // one commit group per call, empty past the last tile, so that wait_group<1> always means "all but
  // the newest copy are in"
  auto load_tile = [&](uint32_t tix, float2* buf) {
    if (tix < ntile) {
      const uint32_t tb = tile_base(tix);
#pragma unroll
      for (int i = 0; i < 8; ++i) cp_async16(buf + cd[i], src + (tb | coff[i]));
    }
    cp_async_commit();
  };
  load_tile(blockIdx.x, tiles);
  load_tile(blockIdx.x + gridDim.x, tiles + tsz);
  int cur = 0;
  for (uint32_t tix = blockIdx.x; tix < ntile; tix += gridDim.x) {
    const uint32_t tb = tile_base(tix);
    float2* tile = tiles + (cur ? tsz : 0u);
    cp_async_wait<1>();
    __syncthreads();   // this tile is in; the previous tile's readers of the updated tile are done
    float sI = 0.f;
#pragma unroll
    for (int l = 0; l < C; l += 4) {
      float hv[8], lv[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 v = tile[sba ^ offa[l + q]];
        sI = fmaf(v.x, v.x, fmaf(v.y, v.y, sI));
        hv[2 * q] = tf32_rna(v.x);
        lv[2 * q] = tf32_rna(v.x - hv[2 * q]);
        hv[2 * q + 1] = tf32_rna(v.y);
        lv[2 * q + 1] = tf32_rna(v.y - hv[2 * q + 1]);
      }
      tmem_st8(tA + 2u * l, hv);
      tmem_st8(tA + 32u + 2u * l, lv);
    }
    accI += (double)sI;
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_sync();
    load_tile(tix + 2 * gridDim.x, tile);   // every thread has read this tile: the copy two ahead
    if (tid == 0) issue_gemm_ts(tmem, 0u, kTcColA2, Bahi, Balo, mb);
    if (!mbar_wait(mb, ph & 1)) s_err = 1;
    ++ph;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (s_err) break;
    {
      float d[32];
      tmem_ld32(taddr, d);
      float sO = 0.f;
#pragma unroll
      for (int r = 0; r < C; ++r) {
        outt[sba ^ offa[r]] = make_float2(d[2 * r], d[2 * r + 1]);
        sO = fmaf(d[2 * r], d[2 * r], fmaf(d[2 * r + 1], d[2 * r + 1], sO));
      }
      accO += (double)sO;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i)
      *reinterpret_cast<float4*>(dst + (tb | coff[i])) = *reinterpret_cast<const float4*>(outt + cd[i]);
    cur ^= 1;
  }
  cp_async_wait<0>();
  tc_sync();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  if (s_err && tid == 0) atomicOr(&f.ap.ctl->status, 1u);
  spec_finish<FIX>(f, gs, accI, 0.0, accO, 0.0, sred, &s_last, true);
}

// ---- complex128 passes, FP64-exact on the FP16 tensor cores (Ozaki slices) ---------------------
enum OzMode { OZ_APPLY = 0, OZ_PROB = 1, OZ_PROB_BOUND = 2 };
// A weight-4 block's 16x16 complex matrix (times 1/sqrt(N)) on the 128 groups of a 2048-amplitude
// tile is a real product y = x . B^T (x: 128 x 32 reals, B: 32 x 32).  A weight-2 block's 4x4
// matrix K runs as K (x) I on 16-amplitude groups made of its two qubits and two spectator qubits
// of the tile: the same product with a block-diagonal B.  Each row of x and of B is split into 7
// signed 8-bit slices under its own exponent (ozaki.cuh); the 28 slice products with p + q <= 6 run
// as 14 FP16 MMAs (M = 128, K = 16, N = 32(7-p) for A slice p against the stacked B slices) that
// accumulate each diagonal p + q = t exactly in its own FP32 TMEM columns; the epilogue recombines
// the 7 diagonals in integers and rounds once to FP64.  Two CTAs per SM (103 KiB of shared memory
// and 256 TMEM columns each) overlap one tile's copies with the other's slicing, MMAs and
// recombination; the next tile's copy is issued as soon as the current one is sliced.
// FP16 inputs, FP32 accumulator, K-major A and B, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t n) { return (1u << 4) | ((n >> 3) << 17) | ((128u >> 4) << 24); }
constexpr int kOzTileBits = 11;
constexpr int kOzSlab = 128 * 32;                    // fp16 elements per A slice
constexpr int kOzSmem = 16 * (1 << kOzTileBits) + 2 * oz::kSlices * kOzSlab + 2 * oz::kSlices * 32 * 32 + 4 * 256 + 4 * 32;

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// Element offset of (row r, k) of a K = 32 16-bit operand: core matrix (r/8, k/8) of 64 elements.
__device__ __forceinline__ int core_off16(int r, int k) { return ((r >> 3) * 4 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Orders every later use of r after the preceding tcgen05.wait::ld.
__device__ __forceinline__ void reg_fence8(uint32_t (&r)[8]) {
  asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// FP16x2 of (digit P of a, digit P of b): the byte is placed in the mantissa of 1024 (0x6400),
// and one fma with (+-1, -+1024) removes the offset and applies each value's sign, exactly.
template <int P>
__device__ __forceinline__ uint32_t digit_pair(uint64_t Xa, uint64_t Xb, uint32_t sg, uint32_t nsg) {
  constexpr int j = P < 3 ? 2 - P : 6 - P;           // byte of the 32-bit word holding bits 48-8P..55-8P
  const uint32_t wa = P < 3 ? (uint32_t)(Xa >> 32) : (uint32_t)Xa;
  const uint32_t wb = P < 3 ? (uint32_t)(Xb >> 32) : (uint32_t)Xb;
  const uint32_t t = (__byte_perm(wa, wb, j | (j << 4) | ((4 + j) << 8) | ((4 + j) << 12)) & 0x00FF00FFu) | 0x64006400u;
  uint32_t r;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(t), "r"(sg), "r"(nsg));
  return r;
}

// Writes the first NS FP16 slices of 8 consecutive reals (row `row`, k0 % 8 == 0) given their
// magnitudes X[0..7] (digit P = byte 6 - P of the 56-bit value) and the high words of the reals
// (for their signs).
template <int NS = oz::kSlices>
__device__ __forceinline__ void put_digits8(uint16_t* S, int slab, int row, int k0, const uint64_t (&X)[8],
                                            const uint32_t (&hw)[8]) {
  uint32_t sg[4], nsg[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t sb = ((hw[2 * i] >> 16) & 0x8000u) | (hw[2 * i + 1] & 0x80000000u);
    sg[i] = 0x3C003C00u | sb;
    nsg[i] = 0xE400E400u ^ sb;
  }
  uint16_t* base = S + core_off16(row, k0);
#define QEC_OZ_SLICE(P)                                                                    \
  if ((P) < NS)                                                                          \
  *reinterpret_cast<uint4*>(base + (P) * slab) =                                         \
      make_uint4(digit_pair<P>(X[0], X[1], sg[0], nsg[0]), digit_pair<P>(X[2], X[3], sg[1], nsg[1]), \
                 digit_pair<P>(X[4], X[5], sg[2], nsg[2]), digit_pair<P>(X[6], X[7], sg[3], nsg[3]));
  QEC_OZ_SLICE(0) QEC_OZ_SLICE(1) QEC_OZ_SLICE(2) QEC_OZ_SLICE(3) QEC_OZ_SLICE(4) QEC_OZ_SLICE(5) QEC_OZ_SLICE(6)
#undef QEC_OZ_SLICE
}

// Writes the first NS FP16 slices of 8 consecutive reals x[0..7] (row `row`, k0 % 8 == 0) under
// exponent E; X[0..7] receives their 56-bit magnitudes.
template <int NS = oz::kSlices>
__device__ __forceinline__ void put_slices8(uint16_t* S, int slab, int row, int k0, const double* x, int E,
                                            uint64_t (&X)[8]) {
  uint32_t hw[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    X[j] = E ? oz::mag56(x[j], E) : 0ull;
    hw[j] = (uint32_t)(oz::d2u(x[j]) >> 32);
  }
  put_digits8<NS>(S, slab, row, k0, X, hw);
}

// MODE 0 (OZ_APPLY): psi <- K_m psi / sqrt(N).  MODE 1 (OZ_PROB): A = sum |K_1 psi_g|^2 and
// N = sum |psi|^2 over all groups, then the outcome (K_1^dagger K_1 is the operator M of the FP64
// pass, so A is the same quantity).  MODE 2 (OZ_PROB_BOUND): the same N exactly, A from the top 3
// slices only with a rigorous bound on its error; the outcome is decided only where the bound
// shows the exact pass would decide the same way, else the ctl flag calls the exact pass.
// f.skip_unless_uncertain (MODE 1): return at once unless that flag is set.
template <int MODE>
__global__ void __launch_bounds__(256, 2) k_oz(FusedArgs f) {
  constexpr bool PROB = MODE != OZ_APPLY;
  constexpr int NS = MODE == OZ_PROB_BOUND ? 3 : oz::kSlices;       // slices of each operand
  constexpr int ND = MODE == OZ_PROB_BOUND ? 2 * NS - 1 : oz::kSlices;   // diagonals accumulated
  if (MODE == OZ_PROB && f.skip_unless_uncertain) {
    if (*(volatile unsigned int*)&f.ap.ctl->prob_uncertain == 0u) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&f.ap.ctl->prob_fallbacks, 1ull);
  }
  constexpr int TS = 1 << kOzTileBits;
  extern __shared__ __align__(128) unsigned char osm[];
  const uint32_t lmask = (1u << f.lb) - 1u;
  double2* tile = reinterpret_cast<double2*>(osm);
  uint16_t* A = reinterpret_cast<uint16_t*>(tile + TS);            // 7 slices x 128 rows x 32
  uint16_t* B = A + oz::kSlices * kOzSlab;                         // 7 slices x 32 rows x 32
  int* rowE = reinterpret_cast<int*>(B + oz::kSlices * 32 * 32);   // [128]: row exponents ([256] reserved)
  int* colE = rowE + 256;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_err;
  __shared__ double sred[64];
  __shared__ int s_last;
  __shared__ int s_eb[4];
  __shared__ uint32_t s_next;   // the tile this CTA takes after the current one
  const int tid = threadIdx.x, warp = tid >> 5;
  int qa[4], qs[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    qa[j] = f.qa[j];
    qs[j] = f.qp[j];
  }
  // recombination: thread = (row r, half hf), outputs 16hf..16hf+15 = amplitudes 8hf..8hf+7 of group r
  // (warp w reads TMEM lanes 32 (w % 4) ..); the slicing maps rows to threads differently (below)
  const int r = tid & 127, hf = tid >> 7;
  const uint32_t gbase = local_base<4>((uint32_t)r, qs);
  uint32_t offa[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) offa[l] = gbase + member_off<4>(8 * hf + l, qa);
  // Tile slot of amplitude e in shared memory: the low 3 bits (the 16-byte bank slot) XOR a fold
  // of the higher bits, so a warp's 32 group gathers spread over all 8 slots whichever tile bits
  // the block occupies (a bijection: only the low bits change, and only as a function of the rest).
  auto slot = [](uint32_t e) { return e ^ (((e >> 3) ^ (e >> 6) ^ (e >> 9)) & 7u); };
  // The slicing maps lanes l and l ^ 16 of a warp to the two halves of one row, so that the row's
  // exponent is one shuffle away: row sr = 16 warp + l % 16, half sh = l / 16.  (The
  // recombination keeps row r = 32 (warp % 4) + l, the TMEM lane its warp may read.)
  const int sr = 16 * warp + (tid & 15), sh = (tid >> 4) & 1;
  uint32_t rda[8];
  {
    const uint32_t sbase = local_base<4>((uint32_t)sr, qs);
#pragma unroll
    for (int l = 0; l < 8; ++l) rda[l] = slot(sbase + member_off<4>(8 * sh + l, qa));
  }
  auto t2g = [&](uint32_t e) {   // tile index -> offset within the register (tile bits)
    const uint32_t h = e >> f.lb;
    uint32_t o = 0;
    for (int j = 0; j < f.nt - f.lb; ++j) o |= ((h >> j) & 1u) << f.hbits[j];
    return o | (e & lmask);
  };
  uint32_t coff[TS / 256], cdst[TS / 256];   // this thread's copies: amplitude e = tid + 256 i, its slot
#pragma unroll
  for (int i = 0; i < TS / 256; ++i) {
    coff[i] = t2g((uint32_t)tid + 256u * i);
    cdst[i] = slot((uint32_t)tid + 256u * i);
  }
  const double2* src = reinterpret_cast<const double2*>(f.ap.src);
  double2* dst = reinterpret_cast<double2*>(f.ap.dst);
  const uint32_t ntile = 1u << f.nout;
  const int obit = (threadIdx.x & 31) < (unsigned)f.nout ? f.obits[threadIdx.x & 31] : 0;
  auto tile_base = [&](uint32_t tix) { return tile_base_warp(tix, f.nout, obit); };
  auto load_tile = [&](uint32_t tb) {
#pragma unroll
    for (int i = 0; i < TS / 256; ++i) cp_async16(tile + cdst[i], src + (tb | coff[i]));
    cp_async_commit();
  };
  // Tiles: CTA b starts with tile b.  Apply: every further tile comes from a device counter, drawn
  // one tile ahead, so that the CTAs sharing an SM finish together whichever started first.  The
  // probability passes keep the fixed tiles b, b + grid, ...: their per-CTA sums, and so A and N,
  // are then the same in every run.  The first copy is issued before the operand setup below,
  // which it overlaps.
  constexpr bool DYN = MODE == OZ_APPLY;
  uint32_t tix = blockIdx.x;
  uint32_t tb = tix < ntile ? tile_base(tix) : 0u;
  if (tix < ntile) load_tile(tb);
  if (tid == 0) s_next = gridDim.x + (DYN ? atomicAdd(&f.ap.ctl->tile_next, 1u) : blockIdx.x);
  // B: real embedding of K_m / sqrt(N) (apply) or K_1 (probability), sliced; 128 threads, thread =
  // (row bn of B, reals 8 bkc .. 8 bkc + 7)
  const int bn = tid >> 2, bkc = tid & 3;
  double bv[8];
  int bE = 0;
  if (tid < 128) {
    const int br = bn >> 1;
    const int m = PROB ? 1 : *f.ap.m;
    const double scale = PROB ? 1.0 : 1.0 / sqrt(*f.ap.N);
    const double2* Kg = reinterpret_cast<const double2*>(f.ap.kraus) + (m ? 256 : 0);
    const bool w2 = f.ap.w == 2;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int l = 4 * bkc + j;
      const double2 kv = !w2 ? Kg[br * 16 + l] : ((br >> 2) == (l >> 2) ? Kg[(br & 3) * 16 + (l & 3)] : make_double2(0.0, 0.0));
      const double re = kv.x * scale, im = kv.y * scale;
      bv[2 * j] = (bn & 1) ? im : re;
      bv[2 * j + 1] = (bn & 1) ? re : -im;
      bE = max(bE, max(oz::bexp(bv[2 * j]), oz::bexp(bv[2 * j + 1])));
    }
    bE = max(bE, __shfl_xor_sync(0xffffffffu, bE, 1));   // the row's 4 threads
    bE = max(bE, __shfl_xor_sync(0xffffffffu, bE, 2));
    if (PROB) {   // one exponent for all of K_1: the outputs share a scale
      const int w = __reduce_max_sync(0xffffffffu, bE);
      if ((tid & 31) == 0) s_eb[warp] = w;
    }
  }
  if (MODE == OZ_PROB_BOUND) {   // B slices 3 and 4 = 0: the first MMA then clears diagonals 3 and 4 too
    uint4* z = reinterpret_cast<uint4*>(B + NS * 32 * 32);
    for (int i = tid; i < 2 * 32 * 32 / 8; i += 256) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    s_err = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  if (tid < 128) {
    const int E = PROB ? max(max(s_eb[0], s_eb[1]), max(s_eb[2], s_eb[3])) : bE;
    if (bkc == 0) colE[bn] = E;
    uint64_t Xb[8];
    put_slices8<NS>(B, 32 * 32, bn, 8 * bkc, bv, E, Xb);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t mb = smem_u32(&mbar);
  uint32_t goff[8];          // this thread's 8 outputs (apply): written straight to the register
#pragma unroll
  for (int l = 0; l < 8; ++l) goff[l] = t2g(offa[l]);
  const uint32_t tlane = (uint32_t)(32 * (warp & 3)) << 16;
  int cmin = 4095, cmax = 0;   // exponents of this thread's 16 outputs' B rows (nonzero rows for cmin)
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int e = colE[16 * hf + j];
    if (e) cmin = min(cmin, e);
    cmax = max(cmax, e);
  }
  uint32_t phase = 0;
  double accA = 0.0, accN = 0.0, accE = 0.0;   // accE: error bound of accA (MODE 2)
  oz::SqAcc sq;    // probability pass: integer sums of squares, one FP64 conversion per tile and sum
  oz::SqAccS sqs;  // the bounded pass's outputs: signed, squared without taking magnitudes
  while (tix < ntile) {
    cp_async_wait<0>();
    __syncthreads();
    const uint32_t tnext = s_next;
    uint32_t tfar = ntile;   // the tile after tnext (thread 0 draws it; published at the end)
    if (tid == 0 && tnext < ntile) tfar = DYN ? gridDim.x + atomicAdd(&f.ap.ctl->tile_next, 1u) : tnext + gridDim.x;
    double x[16];
    int E = 0;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const double2 v = tile[rda[l]];
      x[2 * l] = v.x;
      x[2 * l + 1] = v.y;
      E = max(E, max(oz::bexp(v.x), oz::bexp(v.y)));
    }
    E = max(E, __shfl_xor_sync(0xffffffffu, E, 16));   // the row's other half
    if (sh == 0) rowE[sr] = E;   // for the recombination
    {
      uint64_t X0[8], X1[8];
      put_slices8<NS>(A, kOzSlab, sr, 16 * sh, x, E, X0);
      put_slices8<NS>(A, kOzSlab, sr, 16 * sh + 8, x + 8, E, X1);
      if (PROB) {   // N: sum of x^2 with x = X 2^(E - 1078)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          sq.add(X0[j]);
          sq.add(X1[j]);
        }
        accN += sq.take(2 * (E - 1078));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    // every thread has read its inputs: the tile buffer takes the next tile's copy
    const uint32_t tbn = tnext < ntile ? tile_base(tnext) : 0u;
    if (tnext < ntile) load_tile(tbn);
    if (tid == 0) {
      // 14 MMAs.  The B slices are contiguous 32-row blocks with one row-group stride, so slices
      // 0..6-p form a single N = 32(7-p) operand; written at TMEM column 32p, its product (p, q)
      // lands in the columns of diagonal t = p + q.  Slice 0 (p = 0, first K step) initialises
      // every diagonal; the rest accumulate.  Descriptors: constant offsets (address field:
      // bytes / 16) from two bases.
      const uint64_t da = umma_desc(smem_u32(A), 128, 512), db = umma_desc(smem_u32(B), 128, 512);
      // (MODE 2: 3 slices each side, every product, diagonals 0..4; slice 0 of A runs against
      // B slices 0..4, the last two zero, so that it clears all five diagonals.)
#pragma unroll
      for (int p = 0; p < NS; ++p)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
          umma_f16(tmem + 32u * p, da + ((2u * kOzSlab * p + 256u * ks) >> 4), db + ((256u * ks) >> 4),
                   idesc_f16(32u * (MODE == OZ_PROB_BOUND ? (p == 0 ? ND : NS) : oz::kSlices - p)),
                   (p > 0 || ks > 0) ? 1u : 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
    }
    if (!mbar_wait(mb, phase & 1)) s_err = 1;
    ++phase;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (s_err) break;
    E = rowE[r];
    // outputs 16hf..16hf+15 of row r: amplitudes 8hf..8hf+7; in range: no output can leave the
    // normal FP64 range, so the recombination skips its range checks
    const bool in_range = E == 0 || (E + cmin >= 1076 && E + cmax <= 2980);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      uint32_t R[ND][8];
#pragma unroll
      for (int t = 0; t < ND; ++t) tmem_ld8_nowait(tmem + tlane + 32u * t + 16u * hf + 8u * c, R[t]);
      tmem_wait_ld();
#pragma unroll
      for (int t = 0; t < ND; ++t) reg_fence8(R[t]);
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        float d0[oz::kSlices], d1[oz::kSlices];
#pragma unroll
        for (int t = 0; t < ND; ++t) {
          d0[t] = __uint_as_float(R[t][j]);
          d1[t] = __uint_as_float(R[t][j + 1]);
        }
        const int n = 16 * hf + 8 * c + j;
        if (MODE == OZ_PROB_BOUND) {   // y^ = Z 2^(E + E_B - 2092), Z = sum_t D_t 2^(8(4-t)) exactly
          sqs.add(oz::combine5(d0));
          sqs.add(oz::combine5(d1));
        } else if (PROB) {   // A: sum of y^2 with y = Z 2^(E + E_B - 2098)
          const int64_t z0 = oz::combine7(d0), z1 = oz::combine7(d1);
          sq.add((uint64_t)(z0 < 0 ? -z0 : z0));
          sq.add((uint64_t)(z1 < 0 ? -z1 : z1));
        } else {
          const double y0 = in_range ? oz::assemble7_cvt_inrange(d0, E, colE[n]) : oz::assemble7_cvt(d0, E, colE[n]);
          const double y1 = in_range ? oz::assemble7_cvt_inrange(d1, E, colE[n + 1]) : oz::assemble7_cvt(d1, E, colE[n + 1]);
          dst[tb | goff[4 * c + j / 2]] = make_double2(y0, y1);
        }
      }
    }
    if (MODE == OZ_PROB_BOUND) {
      const double ah = (E && colE[0]) ? sqs.take(2 * (E + colE[0] - 2092)) : sqs.take(-4000);
      accA += ah;
      if (E && colE[0]) accE += oz::part_bound(ah, E + colE[0]);
    } else if (PROB) {
      accA += (E && colE[0]) ? sq.take(2 * (E + colE[0] - 2098)) : sq.take(-4000);
    }
    if (tid == 0) s_next = tfar;   // every thread read s_next before this tile's MMAs
    // No barrier here: the next tile's MMAs are issued after its slicing barrier (tc_sync, with the
    // tcgen05 fences), which every thread reaches only after this recombination's TMEM loads have
    // completed; the loop-top barrier keeps rowE and s_next from being overwritten early.
    tb = tbn;
    tix = tnext;
  }
  cp_async_wait<0>();  // a copy still in flight after an early exit
  // The last CTA to finish returns the tile counter to 0: every CTA drew its last tile before.
  if (DYN && tid == 0 && atomicAdd(&f.ap.ctl->tile_done, 1u) == gridDim.x - 1) {
    f.ap.ctl->tile_next = 0u;
    f.ap.ctl->tile_done = 0u;
  }
  tc_sync();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  if (s_err && tid == 0) atomicOr(&f.ap.ctl->status, 1u);
  if (MODE == OZ_PROB) prob_finish(f.ap, accA, accN, sred, &s_last);
  if (MODE == OZ_PROB_BOUND) prob_finish_bounded(f.ap, accA, accN, accE, sred, &s_last);
}

// ---- fused complex128 pass on the tensor cores: apply block s, then block s+1's probability ----------
// The tile holds both blocks' qubits (at most 8) and the lowest register bits: 2^11 amplitudes.  Per
// tile, on 256 threads, two CTAs per SM:
//  1. Apply block s exactly as k_oz<OZ_APPLY> does (7 slices under each group's exponent, 14 MMAs,
//     integer recombination, one rounding to FP64).  The results go, on chip, into the A-operand
//     slices 3..6 (free once the MMAs have read them), so that the tile buffer takes the next tile's
//     copy as soon as this tile's digits are written; from there they are stored to the register
//     in whole 128-byte runs.
//  2. Probability of block s+1 on the updated tile (Sec. II.B: the ancilla is |0> again, so the
//     next measurement is a quadratic form of this state).  Every real is cut to its top 24 bits
//     under the tile's largest exponent (3 slices); 6 MMAs against the 3 slices of K_1 (one
//     exponent) accumulate the diagonals 0..2; A^ = sum of the squared outputs and N^ = sum of the
//     squared 24-bit inputs, each summed exactly in 64-bit integers per thread, each with a rigorous
//     bound on its error (oz::part_bound with the per-output error 2^(Et + EP - 2060) and the
//     per-input error 2^(Et - 1046)).  The last CTA decides the outcome where |u N^ - A^| exceeds
//     twice the summed bound plus 1e-10 (A^ + N^), where the exact pass must decide the same way;
//     otherwise it flags the exact pass.  N^ (within 2^-22 of the norm) renormalises block s+1's
//     apply whichever pass decides: it scales the whole state, which no outcome depends on (every
//     probability is a ratio of two sums over one state) and which the readout removes.
// Tiles are fixed per CTA (b, b + grid, ...), so every per-thread sum, and so A^, N^ and the
// outcome, are the same in every run.
constexpr int kOzfOut = 3 * kOzSlab;   // outputs: A slices 3..6 (4 x 8 KiB = 2048 complex128)
constexpr int kOzfSmem = 16 * (1 << kOzTileBits) + 2 * oz::kSlices * kOzSlab + 2 * oz::kSlices * 32 * 32 +
                         2 * 3 * 32 * 32 + 4 * 128 + 4 * 32;

__global__ void __launch_bounds__(256, 2) k_ozf(FusedArgs f) {
  constexpr int TS = 1 << kOzTileBits;
  extern __shared__ __align__(128) unsigned char osm[];
  const uint32_t lmask = (1u << f.lb) - 1u;
  double2* tile = reinterpret_cast<double2*>(osm);
  uint16_t* A = reinterpret_cast<uint16_t*>(tile + TS);            // 7 slices x 128 rows x 32
  double2* outb = reinterpret_cast<double2*>(A + kOzfOut);         // updated tile (slots as the tile)
  uint16_t* BA = A + oz::kSlices * kOzSlab;                        // K_m / sqrt(N) of block s, 7 slices
  uint16_t* BP = BA + oz::kSlices * 32 * 32;                       // K_1 of block s+1, 3 slices
  int* rowE = reinterpret_cast<int*>(BP + 3 * 32 * 32);            // [128]
  int* colE = rowE + 128;                                          // [32]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_err;
  __shared__ double sred[64];
  __shared__ int s_last;
  __shared__ int s_eb[4];
  __shared__ uint32_t s_emax[8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int qa[4], qas[4], qp[4], qps[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    qa[j] = f.qa[j];
    qas[j] = f.qa_s[j];
    qp[j] = f.qp[j];
    qps[j] = f.qp_s[j];
  }
  // Tile slot of amplitude e (as in k_oz): linear over XOR, so slot(base | member) = slot(base) ^
  // slot(member) for disjoint bits, and the 8 addresses of a half row are one base and 3 generators.
  auto slot = [](uint32_t e) { return e ^ (((e >> 3) ^ (e >> 6) ^ (e >> 9)) & 7u); };
  auto t2g = [&](uint32_t e) {   // tile index -> offset within the register (also linear over XOR)
    const uint32_t h = e >> f.lb;
    uint32_t o = 0;
    for (int j = 0; j < f.nt - f.lb; ++j) o |= ((h >> j) & 1u) << f.hbits[j];
    return o | (e & lmask);
  };
  // recombination: thread = (b-group r = its TMEM lane, half hf: amplitudes 8hf..8hf+7)
  const int r = tid & 127, hf = tid >> 7;
  // slicing: row sr, half sh; lanes l and l ^ 16 hold the two halves of a row
  const int sr = 16 * warp + (tid & 15), sh = (tid >> 4) & 1;
  uint32_t sa[3], spb[3];   // generators: member bits 0..2 of block s and of block s+1 (tile slots)
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    sa[j] = slot(1u << qa[j]);
    spb[j] = slot(1u << qp[j]);
  }
  const uint32_t rda0 = slot(local_base<4>((uint32_t)sr, qas)) ^ (sh ? slot(1u << qa[3]) : 0u);
  const uint32_t rdp0 = slot(local_base<4>((uint32_t)sr, qps)) ^ (sh ? slot(1u << qp[3]) : 0u);
  const uint32_t gb = local_base<4>((uint32_t)r, qas) | (hf ? (1u << qa[3]) : 0u);
  const uint32_t sd0 = slot(gb);
  auto gen = [](uint32_t b0, const uint32_t (&g)[3], int l) {
    return b0 ^ ((l & 1) ? g[0] : 0u) ^ ((l & 2) ? g[1] : 0u) ^ ((l & 4) ? g[2] : 0u);
  };
  // This thread's copies in and out: amplitudes e = tid + 256 i, i < 8, whose low bits run along the
  // register, so that each quarter warp moves one whole 128-byte run.  Both maps are linear over XOR
  // and tid, 256 i have disjoint bits: a base and 3 generators (slot(256 i) is a constant).
  const uint32_t cb = t2g((uint32_t)tid), cs = slot((uint32_t)tid);
  uint32_t cg[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) cg[j] = t2g(256u << j);
  auto coff = [&](int i) { return cb ^ ((i & 1) ? cg[0] : 0u) ^ ((i & 2) ? cg[1] : 0u) ^ ((i & 4) ? cg[2] : 0u); };
  auto cdst = [&](int i) { return cs ^ slot(256u * (uint32_t)i); };
  const double2* src = reinterpret_cast<const double2*>(f.ap.src);
  double2* dst = reinterpret_cast<double2*>(f.ap.dst);
  const uint32_t ntile = 1u << f.nout;
  const int obit = (threadIdx.x & 31) < (unsigned)f.nout ? f.obits[threadIdx.x & 31] : 0;
  auto tile_base = [&](uint32_t tix) { return tile_base_warp(tix, f.nout, obit); };
  auto load_tile = [&](uint32_t tb) {
#pragma unroll
    for (int i = 0; i < TS / 256; ++i) cp_async16(tile + cdst(i), src + (tb | coff(i)));
    cp_async_commit();
  };
  uint32_t tix = blockIdx.x;
  uint32_t tb = tix < ntile ? tile_base(tix) : 0u;
  if (tix < ntile) load_tile(tb);
  // B operands, overlapping the first copy: threads 0..127 the real embedding of K_m / sqrt(N) of
  // block s (7 slices, each row under its own exponent), threads 128..255 that of K_1 of block s+1
  // (3 slices, one exponent for all of it).  Thread = (row bn, reals 8 bkc .. 8 bkc + 7).
  const bool isP = tid >= 128;
  const int bn = (tid & 127) >> 2, bkc = tid & 3;
  double bv[8];
  int bE = 0;
  {
    const int br = bn >> 1;
    const int m = isP ? 1 : *f.ap.m;
    const double scale = isP ? 1.0 : 1.0 / sqrt(*f.ap.N);
    const double2* Kg = reinterpret_cast<const double2*>(isP ? f.pr.kraus : f.ap.kraus) + (m ? 256 : 0);
    const bool w2 = (isP ? f.pr.w : f.ap.w) == 2;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int l = 4 * bkc + j;
      const double2 kv = !w2 ? Kg[br * 16 + l] : ((br >> 2) == (l >> 2) ? Kg[(br & 3) * 16 + (l & 3)] : make_double2(0.0, 0.0));
      const double re = kv.x * scale, im = kv.y * scale;
      bv[2 * j] = (bn & 1) ? im : re;
      bv[2 * j + 1] = (bn & 1) ? re : -im;
      bE = max(bE, max(oz::bexp(bv[2 * j]), oz::bexp(bv[2 * j + 1])));
    }
    bE = max(bE, __shfl_xor_sync(0xffffffffu, bE, 1));
    bE = max(bE, __shfl_xor_sync(0xffffffffu, bE, 2));
    if (isP) {
      const int w = __reduce_max_sync(0xffffffffu, bE);
      if (lane == 0) s_eb[warp - 4] = w;
    }
  }
  if (tid == 0) {
    s_err = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  const int EP = max(max(s_eb[0], s_eb[1]), max(s_eb[2], s_eb[3]));
  {
    uint64_t Xb[8];
    if (!isP) {
      if (bkc == 0) colE[bn] = bE;
      put_slices8<oz::kSlices>(BA, 32 * 32, bn, 8 * bkc, bv, bE, Xb);
    } else {
      put_slices8<3>(BP, 32 * 32, bn, 8 * bkc, bv, EP, Xb);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t mb = smem_u32(&mbar);
  const uint32_t tlane = (uint32_t)(32 * (warp & 3)) << 16;
  int cmin = 4095, cmax = 0;   // exponents of this thread's 16 outputs' B rows (nonzero rows for cmin)
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int e = colE[16 * hf + j];
    if (e) cmin = min(cmin, e);
    cmax = max(cmax, e);
  }
  uint32_t phase = 0;
  oz::FusedSums sums;
  while (tix < ntile) {
    cp_async_wait<0>();
    __syncthreads();
    const uint32_t tnext = tix + gridDim.x;
    // ---- 1. apply block s: digits of this thread's half row under the row's exponent
    {
      double x[16];
      int E = 0;
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        const double2 v = tile[gen(rda0, sa, l)];
        x[2 * l] = v.x;
        x[2 * l + 1] = v.y;
        E = max(E, max(oz::bexp(v.x), oz::bexp(v.y)));
      }
      E = max(E, __shfl_xor_sync(0xffffffffu, E, 16));
      if (sh == 0) rowE[sr] = E;
      uint64_t X0[8], X1[8];
      put_slices8(A, kOzSlab, sr, 16 * sh, x, E, X0);
      put_slices8(A, kOzSlab, sr, 16 * sh + 8, x + 8, E, X1);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    // every thread has read its inputs: the tile buffer takes the next tile's copy
    const uint32_t tbn = tnext < ntile ? tile_base(tnext) : 0u;
    if (tnext < ntile) load_tile(tbn);
    if (tid == 0) {   // the 14 MMAs of k_oz<OZ_APPLY>
      const uint64_t da = umma_desc(smem_u32(A), 128, 512), db = umma_desc(smem_u32(BA), 128, 512);
#pragma unroll
      for (int p = 0; p < oz::kSlices; ++p)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
          umma_f16(tmem + 32u * p, da + ((2u * kOzSlab * p + 256u * ks) >> 4), db + ((256u * ks) >> 4),
                   idesc_f16(32u * (oz::kSlices - p)), (p > 0 || ks > 0) ? 1u : 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
    }
    if (!mbar_wait(mb, phase & 1)) s_err = 1;
    ++phase;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (s_err) break;
    {
      const int E = rowE[r];
      const bool in_range = E == 0 || (E + cmin >= 1076 && E + cmax <= 2980);
      uint32_t emax = 0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        uint32_t R[oz::kSlices][8];
#pragma unroll
        for (int t = 0; t < oz::kSlices; ++t) tmem_ld8_nowait(tmem + tlane + 32u * t + 16u * hf + 8u * c, R[t]);
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < oz::kSlices; ++t) reg_fence8(R[t]);
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          float d0[oz::kSlices], d1[oz::kSlices];
#pragma unroll
          for (int t = 0; t < oz::kSlices; ++t) {
            d0[t] = __uint_as_float(R[t][j]);
            d1[t] = __uint_as_float(R[t][j + 1]);
          }
          const int n = 16 * hf + 8 * c + j, l = 4 * c + j / 2;
          const double y0 = in_range ? oz::assemble7_cvt_inrange(d0, E, colE[n]) : oz::assemble7_cvt(d0, E, colE[n]);
          const double y1 = in_range ? oz::assemble7_cvt_inrange(d1, E, colE[n + 1]) : oz::assemble7_cvt(d1, E, colE[n + 1]);
          const double2 yv = make_double2(y0, y1);
          outb[gen(sd0, sa, l)] = yv;
          emax = max(emax, max((uint32_t)(oz::d2u(y0) >> 32) & 0x7FF00000u, (uint32_t)(oz::d2u(y1) >> 32) & 0x7FF00000u));
        }
      }
      emax = __reduce_max_sync(0xffffffffu, emax);
      if (lane == 0) s_emax[warp] = emax;
    }
    __syncthreads();   // the updated tile and its exponent are in shared memory
    // the updated tile to the register, with the copy-in mapping (whole 128-byte runs per quarter
    // warp whatever qubits the block acts on; stores straight from the recombination threads
    // scatter when the block holds low register bits)
#pragma unroll
    for (int i = 0; i < TS / 256; ++i) dst[tb | coff(i)] = outb[cdst(i)];
    // ---- 2. probability of block s+1: 24-bit digits under the tile's largest exponent
    uint32_t em = s_emax[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) em = max(em, s_emax[w]);
    const int Et = max((int)(em >> 20), 24);   // >= 24: zero and subnormal reals give 0 digits
    uint64_t nacc = 0;                         // sum of a^2 over this thread's 16 reals (< 2^52)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      uint64_t X[8];
      uint32_t hw[8];
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const double2 v = outb[gen(rdp0, spb, 4 * hh + l)];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const uint64_t u = oz::d2u(c ? v.y : v.x);
          const uint32_t a = oz::top24(u, Et);   // < 2^24
          X[2 * l + c] = (uint64_t)a << 32;
          hw[2 * l + c] = (uint32_t)(u >> 32);
          nacc += (uint64_t)a * a;
        }
      }
      put_digits8<3>(A, kOzSlab, sr, 16 * sh + 8 * hh, X, hw);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    if (tid == 0) {   // 6 MMAs: A slice p at TMEM column 32p against the stacked K_1 slices 0..2-p
      const uint64_t da = umma_desc(smem_u32(A), 128, 512), db = umma_desc(smem_u32(BP), 128, 512);
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
          umma_f16(tmem + 32u * p, da + ((2u * kOzSlab * p + 256u * ks) >> 4), db + ((256u * ks) >> 4),
                   idesc_f16(32u * (3 - p)), (p > 0 || ks > 0) ? 1u : 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
    }
    if (!mbar_wait(mb, phase & 1)) s_err = 1;
    ++phase;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (s_err) break;
    uint64_t aacc = 0;   // sum of Zt^2 over this thread's 16 outputs of K_1 (< 2^62)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      uint32_t R[3][8];
#pragma unroll
      for (int t = 0; t < 3; ++t) tmem_ld8_nowait(tmem + tlane + 32u * t + 16u * hf + 8u * c, R[t]);
      tmem_wait_ld();
#pragma unroll
      for (int t = 0; t < 3; ++t) reg_fence8(R[t]);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float D[3] = {__uint_as_float(R[0][j]), __uint_as_float(R[1][j]), __uint_as_float(R[2][j])};
        const int64_t z = oz::combine3(D);
        aacc += (uint64_t)(z * z);
      }
    }
    // this tile's per-thread sums and their truncation bounds, as FP32 intervals (no FP64 work)
    sums.add_tile(nacc, aacc, Et, EP);
    // no barrier here: the next tile's MMAs are issued after its slicing barrier (tc_sync), which
    // every thread reaches after these TMEM loads; the loop-top barrier protects rowE and s_emax
    tb = tbn;
    tix = tnext;
  }
  cp_async_wait<0>();   // a copy still in flight after an early exit
  tc_sync();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  if (s_err && tid == 0) atomicOr(&f.pr.ctl->status, 1u);
  double accN, rN, accA, rA;
  sums.finish(accN, rN, accA, rA);
  prob_finish_bounded(f.pr, accA, accN, rN + rA, sred, &s_last, true);
}

// ---- speculative complex128 pass on the tensor cores ------------------------------------------------
// Block b's outcome is drawn from the state that block b's own apply reads, so a pass that applies it
// and decides it together must apply before it knows it.  The outcome usually repeats the same
// stabilizer's outcome one round earlier (it changes only at a detection event, Sec. II.B), so the
// pass applies K_g / sqrt(N) for that guess g at once, from the input register into the other buffer,
// and sums on the same tiles, per thread, as FP32 intervals with directed rounding (oz::SqSum24):
//   Nin^ = sum |psi|^2 from each input real's top 24 bits under its group's exponent,
//   Y^   = sum |y|^2 of the FP64 outputs y = K_g psi / sqrt(N), top 24 bits under the tile's largest.
// With N' = Nin^ / N: P(g) = Y^ / N', and P(1) N' = Y^ for g = 1, N' - Y^ for g = 0
// (K_0^dagger K_0 + K_1^dagger K_1 = I).  The last CTA decides the outcome where |u N' - P(1) N'|
// exceeds twice the summed bounds plus 1e-10 (N' + Y^), where the exact pass must decide the same
// way; otherwise the exact pass runs on the input, which the pass left untouched.  If the outcome is
// not g, the corrective launch (FIX) applies K_m from the same input over the speculative output.
// Either way |output|^2 of the apply that stands is stored for the next block's scale (the state's
// scale is free: every probability is a ratio of two sums over one state, and the readout removes
// it).  Tiles are fixed per CTA (b, b + grid, ...), so the sums and outcomes repeat in every run.
constexpr int kOzsSmem = 16 * (1 << kOzTileBits) + 2 * oz::kSlices * kOzSlab + 2 * oz::kSlices * 32 * 32 +
                         4 * 128 + 4 * 32;

template <bool FIX>
__global__ void __launch_bounds__(256, 2) k_ozs(FusedArgs f) {
  const int g = spec_guess(f.ap);
  const int m = FIX ? *f.ap.m : g;   // the corrective pass applies the decided outcome ...
  if (FIX && m == g) return;         // ... only where the guess was wrong
  constexpr int TS = 1 << kOzTileBits;
  extern __shared__ __align__(128) unsigned char osm[];
  const uint32_t lmask = (1u << f.lb) - 1u;
  double2* tile = reinterpret_cast<double2*>(osm);
  uint16_t* A = reinterpret_cast<uint16_t*>(tile + TS);            // 7 slices x 128 rows x 32
  double2* outb = reinterpret_cast<double2*>(A + kOzfOut);         // updated tile (slots as the tile)
  uint16_t* BA = A + oz::kSlices * kOzSlab;                        // K_m / sqrt(N), 7 slices
  int* rowE = reinterpret_cast<int*>(BA + oz::kSlices * 32 * 32);  // [128]
  int* colE = rowE + 128;                                          // [32]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_err;
  __shared__ double sred[64];
  __shared__ int s_last;
  __shared__ uint32_t s_emax[8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int qa[4], qas[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    qa[j] = f.qa[j];
    qas[j] = f.qa_s[j];
  }
  // tile slots, tile-to-register map and thread roles as in k_ozf
  auto slot = [](uint32_t e) { return e ^ (((e >> 3) ^ (e >> 6) ^ (e >> 9)) & 7u); };
  auto t2g = [&](uint32_t e) {
    const uint32_t h = e >> f.lb;
    uint32_t o = 0;
    for (int j = 0; j < f.nt - f.lb; ++j) o |= ((h >> j) & 1u) << f.hbits[j];
    return o | (e & lmask);
  };
  const int r = tid & 127, hf = tid >> 7;                     // recombination: group r, half hf
  const int sr = 16 * warp + (tid & 15), sh = (tid >> 4) & 1;   // slicing: row sr, half sh
  uint32_t sa[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) sa[j] = slot(1u << qa[j]);
  const uint32_t rda0 = slot(local_base<4>((uint32_t)sr, qas)) ^ (sh ? slot(1u << qa[3]) : 0u);
  const uint32_t gb = local_base<4>((uint32_t)r, qas) | (hf ? (1u << qa[3]) : 0u);
  const uint32_t sd0 = slot(gb);
  auto gen = [](uint32_t b0, const uint32_t (&gg)[3], int l) {
    return b0 ^ ((l & 1) ? gg[0] : 0u) ^ ((l & 2) ? gg[1] : 0u) ^ ((l & 4) ? gg[2] : 0u);
  };
  const uint32_t cb = t2g((uint32_t)tid), cs = slot((uint32_t)tid);
  uint32_t cg[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) cg[j] = t2g(256u << j);
  auto coff = [&](int i) { return cb ^ ((i & 1) ? cg[0] : 0u) ^ ((i & 2) ? cg[1] : 0u) ^ ((i & 4) ? cg[2] : 0u); };
  auto cdst = [&](int i) { return cs ^ slot(256u * (uint32_t)i); };
  const double2* src = reinterpret_cast<const double2*>(f.ap.src);
  double2* dst = reinterpret_cast<double2*>(f.ap.dst);
  const uint32_t ntile = 1u << f.nout;
  const int obit = lane < f.nout ? f.obits[lane] : 0;
  auto tile_base = [&](uint32_t tix) { return tile_base_warp(tix, f.nout, obit); };
  auto load_tile = [&](uint32_t tb) {
#pragma unroll
    for (int i = 0; i < TS / 256; ++i) cp_async16(tile + cdst(i), src + (tb | coff(i)));
    cp_async_commit();
  };
  uint32_t tix = blockIdx.x;
  uint32_t tb = tix < ntile ? tile_base(tix) : 0u;
  if (tix < ntile) load_tile(tb);
  // B, overlapping the first copy: threads 0..127 the real embedding of K_m / sqrt(N) (7 slices,
  // each row under its own exponent); thread = (row bn, reals 8 bkc .. 8 bkc + 7)
  const int bn = (tid & 127) >> 2, bkc = tid & 3;
  double bv[8];
  int bE = 0;
  if (tid < 128) {
    const int br = bn >> 1;
    const double scale = f.spec_unit ? 1.0 : 1.0 / sqrt(*f.ap.N);
    const double2* Kg = reinterpret_cast<const double2*>(f.ap.kraus) + (m ? 256 : 0);
    const bool w2 = f.ap.w == 2;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int l = 4 * bkc + j;
      const double2 kv = !w2 ? Kg[br * 16 + l] : ((br >> 2) == (l >> 2) ? Kg[(br & 3) * 16 + (l & 3)] : make_double2(0.0, 0.0));
      const double re = kv.x * scale, im = kv.y * scale;
      bv[2 * j] = (bn & 1) ? im : re;
      bv[2 * j + 1] = (bn & 1) ? re : -im;
      bE = max(bE, max(oz::bexp(bv[2 * j]), oz::bexp(bv[2 * j + 1])));
    }
    bE = max(bE, __shfl_xor_sync(0xffffffffu, bE, 1));
    bE = max(bE, __shfl_xor_sync(0xffffffffu, bE, 2));
  }
  if (tid == 0) {
    s_err = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  if (tid < 128) {
    uint64_t Xb[8];
    if (bkc == 0) colE[bn] = bE;
    put_slices8<oz::kSlices>(BA, 32 * 32, bn, 8 * bkc, bv, bE, Xb);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t mb = smem_u32(&mbar);
  const uint32_t tlane = (uint32_t)(32 * (warp & 3)) << 16;
  int cmin = 4095, cmax = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int e = colE[16 * hf + j];
    if (e) cmin = min(cmin, e);
    cmax = max(cmax, e);
  }
  uint32_t phase = 0;
  oz::SqSum24 sin_, sout;
  while (tix < ntile) {
    cp_async_wait<0>();
    __syncthreads();
    const uint32_t tnext = tix + gridDim.x;
    // ---- digits of this thread's half row under the row's exponent; Nin^ from their top 24 bits
    {
      double x[16];
      int E = 0;
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        const double2 v = tile[gen(rda0, sa, l)];
        x[2 * l] = v.x;
        x[2 * l + 1] = v.y;
        E = max(E, max(oz::bexp(v.x), oz::bexp(v.y)));
      }
      E = max(E, __shfl_xor_sync(0xffffffffu, E, 16));
      if (sh == 0) rowE[sr] = E;
      uint64_t X0[8], X1[8];
      put_slices8(A, kOzSlab, sr, 16 * sh, x, E, X0);
      put_slices8(A, kOzSlab, sr, 16 * sh + 8, x + 8, E, X1);
      uint64_t nacc = 0;   // |x| = 2^(E - 1078) X = 2^(E - 1046) (X / 2^32): top 24 bits X >> 32
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint64_t a0 = X0[j] >> 32, a1 = X1[j] >> 32;
        nacc += a0 * a0 + a1 * a1;
      }
      sin_.add(nacc, E);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    const uint32_t tbn = tnext < ntile ? tile_base(tnext) : 0u;
    if (tnext < ntile) load_tile(tbn);
    if (tid == 0) {   // the 14 MMAs of k_oz<OZ_APPLY>
      const uint64_t da = umma_desc(smem_u32(A), 128, 512), db = umma_desc(smem_u32(BA), 128, 512);
#pragma unroll
      for (int p = 0; p < oz::kSlices; ++p)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
          umma_f16(tmem + 32u * p, da + ((2u * kOzSlab * p + 256u * ks) >> 4), db + ((256u * ks) >> 4),
                   idesc_f16(32u * (oz::kSlices - p)), (p > 0 || ks > 0) ? 1u : 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
    }
    if (!mbar_wait(mb, phase & 1)) s_err = 1;
    ++phase;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (s_err) break;
    {
      const int E = rowE[r];
      const bool in_range = E == 0 || (E + cmin >= 1076 && E + cmax <= 2980);
      uint32_t emax = 0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        uint32_t R[oz::kSlices][8];
#pragma unroll
        for (int t = 0; t < oz::kSlices; ++t) tmem_ld8_nowait(tmem + tlane + 32u * t + 16u * hf + 8u * c, R[t]);
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < oz::kSlices; ++t) reg_fence8(R[t]);
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          float d0[oz::kSlices], d1[oz::kSlices];
#pragma unroll
          for (int t = 0; t < oz::kSlices; ++t) {
            d0[t] = __uint_as_float(R[t][j]);
            d1[t] = __uint_as_float(R[t][j + 1]);
          }
          const int n = 16 * hf + 8 * c + j, l = 4 * c + j / 2;
          const double y0 = in_range ? oz::assemble7_cvt_inrange(d0, E, colE[n]) : oz::assemble7_cvt(d0, E, colE[n]);
          const double y1 = in_range ? oz::assemble7_cvt_inrange(d1, E, colE[n + 1]) : oz::assemble7_cvt(d1, E, colE[n + 1]);
          outb[gen(sd0, sa, l)] = make_double2(y0, y1);
          emax = max(emax, max((uint32_t)(oz::d2u(y0) >> 32) & 0x7FF00000u, (uint32_t)(oz::d2u(y1) >> 32) & 0x7FF00000u));
        }
      }
      emax = __reduce_max_sync(0xffffffffu, emax);
      if (lane == 0) s_emax[warp] = emax;
    }
    __syncthreads();   // the updated tile and its exponent are in shared memory
    // ---- the updated tile to the register (whole 128-byte runs per quarter warp, as in k_ozf); Y^
    // from the stored values' top 24 bits under the tile's largest exponent
    uint32_t em = s_emax[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) em = max(em, s_emax[w]);
    const int Et = max((int)(em >> 20), 24);   // >= 24: zero and subnormal reals give 0
    uint64_t yacc = 0;
#pragma unroll
    for (int i = 0; i < TS / 256; ++i) {
      const double2 v = outb[cdst(i)];
      dst[tb | coff(i)] = v;
      const uint64_t a0 = oz::top24(oz::d2u(v.x), Et), a1 = oz::top24(oz::d2u(v.y), Et);
      yacc += a0 * a0 + a1 * a1;
    }
    sout.add(yacc, Et);
    // no barrier here: the loop-top barrier keeps outb (A slices 3..6), rowE and s_emax until every
    // thread is past this tile; the next tile's MMAs follow its slicing barrier
    tb = tbn;
    tix = tnext;
  }
  cp_async_wait<0>();   // a copy still in flight after an early exit
  tc_sync();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  if (s_err && tid == 0) atomicOr(&f.ap.ctl->status, 1u);
  double nI, rI, nO, rO;
  sin_.finish(nI, rI);
  sout.finish(nO, rO);
  spec_finish<FIX>(f, g, nI, rI, nO, rO, sred, &s_last);
}

// ---- final Z readout (Sec. III.B): sequential per-qubit sampling -------------------------
// Qubit j gets outcome [u_j < P(q_j = 1 | outcomes of qubits < j)].  The conditional
// marginals of the low k1 qubits come from one histogram pass over the register; the
// remaining qubits from the 2^(D-k1) amplitudes that carry the sampled low bits.
template <typename T>
__global__ void __launch_bounds__(256) k_hist(ReadArgs a) {
  using T2 = typename V2<T>::t;
  const int B = 1 << a.k1;
  const int nb = B >> 8;                 // bins per thread (B >= 256)
  const int64_t nchunk = 1ll << (a.D - a.k1);
  const T2* src = reinterpret_cast<const T2*>(a.src);
  double acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.0;
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const int64_t base = ch << a.k1;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j < nb) {
        const T2 v = src[base + threadIdx.x + 256 * j];
        acc[j] += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (j < nb) a.hist_part[(size_t)blockIdx.x * B + threadIdx.x + 256 * j] = acc[j];
}

__global__ void __launch_bounds__(256) k_hist_reduce(ReadArgs a) {
  const int B = 1 << a.k1;
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= B) return;
  double s = 0.0;
  for (int c = 0; c < a.grid_hist; ++c) s += a.hist_part[(size_t)c * B + bin];
  a.hist[bin] = s;
}

// Samples the bits [0, nbits) of the index over the weights w[0, n) (n = 2^nbits),
// qubit-by-qubit; bit j of the result goes to out_bits[bit_base + j].
__device__ int sample_bits(const double* w, int nbits, int bit_base, uint64_t seed, uint64_t traj,
                           uint64_t rnd, uint8_t* out_bits, double* sred, int* sbit) {
  const int n = 1 << nbits;
  int prefix = 0;
  for (int j = 0; j < nbits; ++j) {
    const int mask = (1 << j) - 1;
    double s_all = 0.0, s_one = 0.0;
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
      if ((x & mask) == prefix) {
        s_all += w[x];
        if ((x >> j) & 1) s_one += w[x];
      }
    }
    block_sum2(s_all, s_one, sred);
    if (threadIdx.x == 0) {
      const double u = uniform53(draw(seed, traj, rnd, 0u, (uint32_t)(bit_base + j), TAG_READOUT).v[0]);
      const int b = (u < s_one / s_all) ? 1 : 0;
      *sbit = b;
      out_bits[bit_base + j] = (uint8_t)b;
    }
    __syncthreads();
    prefix |= (*sbit) << j;
    __syncthreads();
  }
  return prefix;
}

template <typename T>
__global__ void __launch_bounds__(256) k_sample(ReadArgs a) {
  using T2 = typename V2<T>::t;
  extern __shared__ double sh[];
  __shared__ double sred[64];
  __shared__ int sbit;
  const int B = 1 << a.k1;
  const uint64_t seed = a.ctl->seed, traj = a.ctl->traj;
  const unsigned long long t = traj - a.ctl->first;
  const uint64_t rnd = (uint64_t)a.rounds + 1;
  const int nd = a.D;   // data qubits = resident register bits
  uint8_t* bits = a.bits + t * (unsigned long long)nd;
  double tot = 0.0, dummy = 0.0;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    sh[i] = a.hist[i];
    tot += sh[i];
  }
  block_sum2(tot, dummy, sred);
  if (threadIdx.x == 0) a.ctl->final_norm = tot;
  const int low = sample_bits(sh, a.k1, 0, seed, traj, rnd, bits, sred, &sbit);
  if (a.D > a.k1) {
    const int H = 1 << (a.D - a.k1);
    const T2* src = reinterpret_cast<const T2*>(a.src);
    __syncthreads();
    for (int y = threadIdx.x; y < H; y += blockDim.x) {
      const T2 v = src[((int64_t)y << a.k1) | low];
      sh[y] = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    }
    __syncthreads();
    sample_bits(sh, a.D - a.k1, a.k1, seed, traj, rnd, bits, sred, &sbit);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int par = 0;
    for (int c = 0; c < a.d; ++c) par ^= bits[c];   // Z_L: the first row (surface), the whole line (repetition)
    a.logical[t] = (uint8_t)par;
    for (int k = 0; k < a.nstab; ++k) a.syn[t * (unsigned long long)a.syn_stride + k] = 0;
    a.ctl->traj = traj + 1;
  }
}

template <typename T>
__global__ void k_set_basis0(void* psi, int64_t n) {
  using T2 = typename V2<T>::t;
  T2* p = reinterpret_cast<T2*>(psi);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T2 z;
    z.x = (i == 0) ? (T)1 : (T)0;
    z.y = 0;
    p[i] = z;
  }
}

constexpr int kFusedSmemMax = 160 * 1024;

// Resident CTAs of 256 threads per SM for this kernel and dynamic shared memory.
static int blocks_per_sm(const void* fn, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 256, smem) != cudaSuccess || n < 1) n = 1;
  return n;
}

// One wave of resident CTAs (grid-stride loops cover the rest), capped by the work and the partials.
static int wave_grid(const void* fn, size_t smem, int num_sms, int64_t work) {
  int64_t g = (int64_t)num_sms * blocks_per_sm(fn, smem);
  if (g > work) g = work;
  if (g > MAX_PASS_GRID) g = MAX_PASS_GRID;
  return (int)(g < 1 ? 1 : g);
}

// ---- launchers --------------------------------------------------------------------------
int pass_grid(int D, int w, int num_sms) {
  const int64_t G = 1ll << (D - w);
  int64_t g = (G + 255) / 256;
  int64_t cap = (int64_t)num_sms * 4;
  if (g > cap) g = cap;
  if (g > MAX_PASS_GRID) g = MAX_PASS_GRID;
  return (int)(g < 1 ? 1 : g);
}

int hist_k1(int D) { return D < 12 ? D : 12; }

int hist_grid(int D, int num_sms) {
  const int64_t nchunk = 1ll << (D - hist_k1(D));
  int64_t g = nchunk < (int64_t)num_sms * 2 ? nchunk : (int64_t)num_sms * 2;
  return (int)g;
}

cudaError_t launch_instantiate(int precision, const InstArgs& a, cudaStream_t s) {
  if (is_f64(precision)) k_instantiate<double><<<a.nblk, 256, 0, s>>>(a);
  else k_instantiate<float><<<a.nblk, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
static void prob_t(const PassArgs& a, int grid, cudaStream_t s) {
  if (a.w == 4) k_prob<T, 4><<<grid, 256, 0, s>>>(a);
  else k_prob<T, 2><<<grid, 256, 0, s>>>(a);
}

template <typename T>
static void apply_t(const PassArgs& a, int grid, cudaStream_t s) {
  if (a.w == 4) k_apply<T, 4><<<grid, 256, 0, s>>>(a);
  else k_apply<T, 2><<<grid, 256, 0, s>>>(a);
}

int pass_grid_for(int precision, bool prob, int D, int w, int num_sms) {
  const void* fn;
  if (is_f64(precision))
    fn = prob ? (w == 4 ? (const void*)k_prob<double, 4> : (const void*)k_prob<double, 2>)
              : (w == 4 ? (const void*)k_apply<double, 4> : (const void*)k_apply<double, 2>);
  else
    fn = prob ? (w == 4 ? (const void*)k_prob<float, 4> : (const void*)k_prob<float, 2>)
              : (w == 4 ? (const void*)k_apply<float, 4> : (const void*)k_apply<float, 2>);
  return wave_grid(fn, 0, num_sms, ((1ll << (D - w)) + 255) / 256);
}

cudaError_t launch_prob(int precision, const PassArgs& a, int grid, cudaStream_t s) {
  if (a.w != 2 && a.w != 4) return cudaErrorInvalidValue;
  if (is_f64(precision)) prob_t<double>(a, grid, s);
  else prob_t<float>(a, grid, s);
  return cudaGetLastError();
}

cudaError_t launch_apply(int precision, const PassArgs& a, int grid, cudaStream_t s) {
  if (a.w != 2 && a.w != 4) return cudaErrorInvalidValue;
  if (is_f64(precision)) apply_t<double>(a, grid, s);
  else apply_t<float>(a, grid, s);
  return cudaGetLastError();
}

static size_t sample_smem(int D) {
  const int k1 = hist_k1(D);
  const size_t B = (size_t)1 << k1, H = D > k1 ? ((size_t)1 << (D - k1)) : 0;
  return sizeof(double) * (B > H ? B : H);
}

cudaError_t launch_readout(int precision, const ReadArgs& a, cudaStream_t s) {
  const int B = 1 << a.k1;
  const size_t smem = sample_smem(a.D);
  if (is_f64(precision)) {
    k_hist<double><<<a.grid_hist, 256, 0, s>>>(a);
    k_hist_reduce<<<(B + 255) / 256, 256, 0, s>>>(a);
    k_sample<double><<<1, 256, smem, s>>>(a);
  } else {
    k_hist<float><<<a.grid_hist, 256, 0, s>>>(a);
    k_hist_reduce<<<(B + 255) / 256, 256, 0, s>>>(a);
    k_sample<float><<<1, 256, smem, s>>>(a);
  }
  return cudaGetLastError();
}

static int tile_pos(int q, int lb, const int* hb, int nh) {
  if (q < lb) return q;
  for (int j = 0; j < nh; ++j)
    if (hb[j] == q) return lb + j;
  return -1;
}

template <typename T, int W, int W2>
static cudaError_t fused_t(FusedArgs f, size_t smem, int num_sms, cudaStream_t s) {
  f.grid = wave_grid((const void*)k_fused<T, W, W2>, smem, num_sms, 1ll << f.nout);
  k_fused<T, W, W2><<<f.grid, 256, smem, s>>>(f);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t fused_attrs() {
  const void* fns[4] = {(const void*)k_fused<T, 2, 2>, (const void*)k_fused<T, 2, 4>, (const void*)k_fused<T, 4, 2>,
                        (const void*)k_fused<T, 4, 4>};
  for (const void* fn : fns) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmemMax);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static void oz_block_bits(int w, int* q, int* qs, int nt);

cudaError_t launch_fused(int precision, const PassArgs& ap, const PassArgs& pr, int num_sms, cudaStream_t s) {
  if ((ap.w != 2 && ap.w != 4) || (pr.w != 2 && pr.w != 4)) return cudaErrorInvalidValue;
  const size_t amp = is_f64(precision) ? 16 : 8;
  FusedArgs f;
  f.ap = ap;
  f.pr = pr;
  // Tile bits: both blocks' qubits plus the low bits [0, lb), lb chosen for >= 128-byte runs
  // and then raised until the tile has >= 2^12 amplitudes (or the register ends), so that a
  // weight-4 block has one 16-amplitude group per thread.
  uint32_t mask = 0;
  for (int j = 0; j < ap.w; ++j) mask |= 1u << ap.q[j];
  for (int j = 0; j < pr.w; ++j) mask |= 1u << pr.q[j];
  int lb = amp == 16 ? 3 : 4;
  if (lb > ap.D) lb = ap.D;
  auto count = [&](int lbits) {
    uint32_t m = mask | ((1u << lbits) - 1u);
    return __builtin_popcount(m);
  };
  while (count(lb) < 12 && lb < ap.D) ++lb;
  const uint32_t tmask = mask | ((1u << lb) - 1u);
  f.lb = lb;
  int nh = 0, no = 0;
  for (int q = lb; q < ap.D; ++q) {
    if (tmask & (1u << q)) f.hbits[nh++] = q;
  }
  for (int q = 0; q < ap.D; ++q) {
    if (!(tmask & (1u << q))) f.obits[no++] = q;
  }
  f.nt = lb + nh;
  f.nout = no;
  for (int j = 0; j < 4; ++j) {
    f.qa[j] = j < ap.w ? tile_pos(ap.q[j], lb, f.hbits, nh) : 0;
    f.qp[j] = j < pr.w ? tile_pos(pr.q[j], lb, f.hbits, nh) : 0;
  }
  // the tensor-core pass for pairs with a weight-4 block (a weight-2 block of the pair as K (x) I over
  // two spectator bits); two weight-2 blocks are faster on the CUDA cores
  if (precision == QEC_C64_TC && (ap.w == 4 || pr.w == 4) && f.nt == 12) {
    oz_block_bits(ap.w, f.qa, f.qa_s, f.nt);
    oz_block_bits(pr.w, f.qp, f.qp_s, f.nt);
    const size_t tsmem = kTcSmem;
    // sized for two resident CTAs per SM (113 KiB each; the occupancy query under-reports this
    // shape), capped by the tile count
    int64_t g = 2ll * num_sms;
    if (g > (1ll << f.nout)) g = 1ll << f.nout;
    f.grid = (int)(g < MAX_PASS_GRID ? g : MAX_PASS_GRID);
    k_fused_tc<<<f.grid, 256, tsmem, s>>>(f);
    return cudaGetLastError();
  }
  const size_t smem = 2 * amp * ((size_t)1 << f.nt) + sizeof(uint32_t) * ((size_t)1 << nh);
  if (smem > (size_t)kFusedSmemMax) return cudaErrorInvalidValue;
  const int key = (ap.w == 4 ? 2 : 0) + (pr.w == 4 ? 1 : 0);
  if (is_f64(precision)) {
    switch (key) {
      case 0: return fused_t<double, 2, 2>(f, smem, num_sms, s);
      case 1: return fused_t<double, 2, 4>(f, smem, num_sms, s);
      case 2: return fused_t<double, 4, 2>(f, smem, num_sms, s);
      default: return fused_t<double, 4, 4>(f, smem, num_sms, s);
    }
  }
  switch (key) {
    case 0: return fused_t<float, 2, 2>(f, smem, num_sms, s);
    case 1: return fused_t<float, 2, 4>(f, smem, num_sms, s);
    case 2: return fused_t<float, 4, 2>(f, smem, num_sms, s);
    default: return fused_t<float, 4, 4>(f, smem, num_sms, s);
  }
}

// Tile of one block's qubits plus low bits, >= 2^12 amplitudes (shared with the fused launchers).
static void block_tile(const PassArgs& ap, const PassArgs& pr, int lb0, int bits, FusedArgs& f) {
  uint32_t mask = 0;
  for (int j = 0; j < ap.w; ++j) mask |= 1u << ap.q[j];
  for (int j = 0; j < pr.w; ++j) mask |= 1u << pr.q[j];
  int lb = lb0 > ap.D ? ap.D : lb0;
  while (__builtin_popcount(mask | ((1u << lb) - 1u)) < bits && lb < ap.D) ++lb;
  const uint32_t tmask = mask | ((1u << lb) - 1u);
  f.lb = lb;
  int nh = 0, no = 0;
  for (int q = lb; q < ap.D; ++q)
    if (tmask & (1u << q)) f.hbits[nh++] = q;
  for (int q = 0; q < ap.D; ++q)
    if (!(tmask & (1u << q))) f.obits[no++] = q;
  f.nt = lb + nh;
  f.nout = no;
  for (int j = 0; j < 4; ++j) {
    f.qa[j] = j < ap.w ? tile_pos(ap.q[j], lb, f.hbits, nh) : 0;
    f.qp[j] = j < pr.w ? tile_pos(pr.q[j], lb, f.hbits, nh) : 0;
  }
}

bool apply_oz_applies(const PassArgs& ap) {
  if (ap.w != 2 && ap.w != 4) return false;
  FusedArgs f;
  block_tile(ap, ap, 3, kOzTileBits, f);
  return f.nt == kOzTileBits;
}

static cudaError_t launch_oz(int mode, bool skip_unless_uncertain, const PassArgs& ap, int num_sms, cudaStream_t s) {
  FusedArgs f;
  f.ap = ap;
  f.pr = ap;
  f.skip_unless_uncertain = skip_unless_uncertain ? 1 : 0;
  block_tile(ap, ap, 3, kOzTileBits, f);
  if ((ap.w != 2 && ap.w != 4) || f.nt != kOzTileBits) return cudaErrorInvalidValue;
  if (ap.w == 2) {   // spectators: the two lowest tile bits outside the block
    int k = 2;
    for (int b = 0; b < f.nt && k < 4; ++b)
      if (b != f.qa[0] && b != f.qa[1]) f.qa[k++] = b;
  }
  for (int j = 0; j < 4; ++j) f.qp[j] = f.qa[j];
  std::sort(f.qp, f.qp + 4);
  int64_t g = 2ll * num_sms;   // two CTAs per SM: 103 KiB of shared memory and 256 TMEM columns each
  if (g > (1ll << f.nout)) g = 1ll << f.nout;
  if (g > MAX_PASS_GRID) g = MAX_PASS_GRID;
  if (mode == OZ_PROB_BOUND && 3 * g > 2 * MAX_PASS_GRID) g = 2 * MAX_PASS_GRID / 3;   // 3 partial sums per CTA
  f.grid = (int)g;
  if (mode == OZ_APPLY) k_oz<OZ_APPLY><<<f.grid, 256, kOzSmem, s>>>(f);
  else if (mode == OZ_PROB) k_oz<OZ_PROB><<<f.grid, 256, kOzSmem, s>>>(f);
  else k_oz<OZ_PROB_BOUND><<<f.grid, 256, kOzSmem, s>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_apply_oz(const PassArgs& ap, int num_sms, cudaStream_t s) {
  return launch_oz(OZ_APPLY, false, ap, num_sms, s);
}
// The probability pass: the bounded 3-slice pass, then the exact pass, which returns at once
// unless the bounded pass left the outcome undecided.
cudaError_t launch_prob_oz(const PassArgs& ap, int num_sms, cudaStream_t s) {
  cudaError_t e = launch_oz(OZ_PROB_BOUND, false, ap, num_sms, s);
  return e != cudaSuccess ? e : launch_oz(OZ_PROB, true, ap, num_sms, s);
}

bool fused_oz_applies(const PassArgs& ap, const PassArgs& pr) {
  if ((ap.w != 2 && ap.w != 4) || (pr.w != 2 && pr.w != 4)) return false;
  FusedArgs f;
  block_tile(ap, pr, 3, kOzTileBits, f);
  return f.nt == kOzTileBits;
}

// A weight-2 block's spectators: the two lowest tile bits outside it; q[0..3] then holds its two
// qubits and the spectators, qs the same bits sorted.
static void oz_block_bits(int w, int* q, int* qs, int nt) {
  if (w == 2) {
    int k = 2;
    for (int b = 0; b < nt && k < 4; ++b)
      if (b != q[0] && b != q[1]) q[k++] = b;
  }
  for (int j = 0; j < 4; ++j) qs[j] = q[j];
  std::sort(qs, qs + 4);
}

cudaError_t launch_fused_oz(const PassArgs& ap, const PassArgs& pr, int num_sms, cudaStream_t s) {
  FusedArgs f;
  f.ap = ap;
  f.pr = pr;
  f.skip_unless_uncertain = 0;
  block_tile(ap, pr, 3, kOzTileBits, f);
  if ((ap.w != 2 && ap.w != 4) || (pr.w != 2 && pr.w != 4) || f.nt != kOzTileBits) return cudaErrorInvalidValue;
  oz_block_bits(ap.w, f.qa, f.qa_s, f.nt);
  oz_block_bits(pr.w, f.qp, f.qp_s, f.nt);
  int64_t g = 2ll * num_sms;   // two CTAs per SM: 109 KiB of shared memory and 256 TMEM columns each
  if (g > (1ll << f.nout)) g = 1ll << f.nout;
  if (3 * g > 2 * MAX_PASS_GRID) g = 2 * MAX_PASS_GRID / 3;   // 3 partial sums per CTA
  f.grid = (int)g;
  k_ozf<<<f.grid, 256, kOzfSmem, s>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_prob_oz_check(const PassArgs& pr, int num_sms, cudaStream_t s) {
  PassArgs a = pr;
  a.store_n = 0;   // the fused pass's norm estimate stays
  return launch_oz(OZ_PROB, true, a, num_sms, s);
}

// The speculative pass's tile and grid: block ap's qubits (a weight-2 block with two spectators, as K
// (x) I) plus low bits in a 2^11-amplitude tile, two CTAs per SM, 4 partial sums per CTA.
static bool spec_args(const PassArgs& ap, double* n_next, bool unit_in, int num_sms, FusedArgs& f) {
  f.ap = ap;
  f.pr = ap;
  f.skip_unless_uncertain = 0;
  block_tile(ap, ap, 3, kOzTileBits, f);
  if ((ap.w != 2 && ap.w != 4) || f.nt != kOzTileBits || ap.src == ap.dst) return false;
  oz_block_bits(ap.w, f.qa, f.qa_s, f.nt);
  f.n_next = n_next;
  f.spec_unit = unit_in ? 1 : 0;
  int64_t g = 2ll * num_sms;
  if (g > (1ll << f.nout)) g = 1ll << f.nout;
  if (g > MAX_PASS_GRID / 2) g = MAX_PASS_GRID / 2;
  f.grid = (int)g;
  return true;
}

// The FP64 CUDA-core speculative pass: grid-stride over groups, one wave of resident CTAs, 4 partial
// sums per CTA.
static bool spec_fp64_args(const PassArgs& ap, double* n_next, bool unit_in, int num_sms, FusedArgs& f) {
  if ((ap.w != 2 && ap.w != 4) || ap.src == ap.dst) return false;
  f.ap = ap;
  f.pr = ap;
  f.n_next = n_next;
  f.spec_unit = unit_in ? 1 : 0;
  const void* fn = ap.w == 4 ? (const void*)k_apply_spec<4, false> : (const void*)k_apply_spec<2, false>;
  f.grid = wave_grid(fn, 0, num_sms, ((1ll << (ap.D - ap.w)) + 255) / 256);
  if (f.grid > MAX_PASS_GRID / 2) f.grid = MAX_PASS_GRID / 2;
  return true;
}

// The complex64 speculative pass: k_fused's tile rule for block ap alone (low bits for 128-byte runs,
// raised to at least 2^12 amplitudes), one wave of resident CTAs, 4 partial sums per CTA.
static bool spec_c64_args(const PassArgs& ap, double* n_next, bool unit_in, int num_sms, FusedArgs& f,
                          size_t& smem) {
  if ((ap.w != 2 && ap.w != 4) || ap.src == ap.dst) return false;
  f.ap = ap;
  f.pr = ap;
  f.n_next = n_next;
  f.spec_unit = unit_in ? 1 : 0;
  block_tile(ap, ap, 4, 12, f);
  smem = 2 * 8 * ((size_t)1 << f.nt) + sizeof(uint32_t) * ((size_t)1 << (f.nt - f.lb));
  if (smem > (size_t)kFusedSmemMax) return false;
  const void* fn = ap.w == 4 ? (const void*)k_fused_spec<4, false> : (const void*)k_fused_spec<2, false>;
  f.grid = wave_grid(fn, smem, num_sms, 1ll << f.nout);
  if (f.grid > MAX_PASS_GRID / 2) f.grid = MAX_PASS_GRID / 2;
  return true;
}

// QEC_C64_TC: weight-4 blocks whose tile has 2^12 amplitudes on the tensor cores (k_fused_tc_spec, two
// CTAs per SM), the rest as QEC_C64.
template <bool FIX>
static cudaError_t launch_spec_c64(int precision, const PassArgs& ap, double* n_next, bool unit_in, int num_sms,
                                   cudaStream_t s) {
  FusedArgs f;
  size_t smem = 0;
  if (!spec_c64_args(ap, n_next, unit_in, num_sms, f, smem)) return cudaErrorInvalidValue;
  if (precision == QEC_C64_TC && ap.w == 4 && f.nt == 12) {
    oz_block_bits(ap.w, f.qa, f.qa_s, f.nt);
    int64_t g = 2ll * num_sms;
    if (g > (1ll << f.nout)) g = 1ll << f.nout;
    if (g > MAX_PASS_GRID / 2) g = MAX_PASS_GRID / 2;
    f.grid = (int)g;
    k_fused_tc_spec<FIX><<<f.grid, 256, kTcSmem, s>>>(f);
    return cudaGetLastError();
  }
  if (ap.w == 4) k_fused_spec<4, FIX><<<f.grid, 256, smem, s>>>(f);
  else k_fused_spec<2, FIX><<<f.grid, 256, smem, s>>>(f);
  return cudaGetLastError();
}

static bool spec_on_tensor_cores(int precision, const PassArgs& ap) {
  return precision == QEC_C128_TC && apply_oz_applies(ap);
}

cudaError_t launch_spec(int precision, const PassArgs& ap, double* n_next, bool unit_in, int num_sms, cudaStream_t s) {
  if (!is_f64(precision)) return launch_spec_c64<false>(precision, ap, n_next, unit_in, num_sms, s);
  FusedArgs f;
  if (spec_on_tensor_cores(precision, ap)) {
    if (!spec_args(ap, n_next, unit_in, num_sms, f)) return cudaErrorInvalidValue;
    k_ozs<false><<<f.grid, 256, kOzsSmem, s>>>(f);
    return cudaGetLastError();
  }
  if (!is_f64(precision) || !spec_fp64_args(ap, n_next, unit_in, num_sms, f)) return cudaErrorInvalidValue;
  if (ap.w == 4) k_apply_spec<4, false><<<f.grid, 256, 0, s>>>(f);
  else k_apply_spec<2, false><<<f.grid, 256, 0, s>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_spec_fix(int precision, const PassArgs& ap, double* n_next, bool unit_in, int num_sms,
                            cudaStream_t s) {
  if (!is_f64(precision)) return launch_spec_c64<true>(precision, ap, n_next, unit_in, num_sms, s);
  FusedArgs f;
  if (spec_on_tensor_cores(precision, ap)) {
    if (!spec_args(ap, n_next, unit_in, num_sms, f)) return cudaErrorInvalidValue;
    PassArgs a = ap;
    a.store_n = 0;   // *N keeps the scale both applies of this block use
    cudaError_t e = launch_oz(OZ_PROB, true, a, num_sms, s);
    if (e != cudaSuccess) return e;
    k_ozs<true><<<f.grid, 256, kOzsSmem, s>>>(f);
    return cudaGetLastError();
  }
  if (!is_f64(precision) || !spec_fp64_args(ap, n_next, unit_in, num_sms, f)) return cudaErrorInvalidValue;
  if (ap.w == 4) k_apply_spec<4, true><<<f.grid, 256, 0, s>>>(f);
  else k_apply_spec<2, true><<<f.grid, 256, 0, s>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(unsigned int* status, long limit, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(status, limit);
  return cudaGetLastError();
}

cudaError_t launch_set_basis0(int precision, void* psi, int D, cudaStream_t s) {
  const int64_t n = 1ll << D;
  int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (is_f64(precision)) k_set_basis0<double><<<grid, 256, 0, s>>>(psi, n);
  else k_set_basis0<float><<<grid, 256, 0, s>>>(psi, n);
  return cudaGetLastError();
}

// Function attributes are per process, not per simulator: always set the ceiling for the
// largest supported register (d = 5), so simulators of different sizes can coexist.
cudaError_t setup_kernels(int precision, int D) {
  (void)D;
  const int smem = (int)sample_smem(25);
  if (is_f64(precision)) {
    cudaError_t e = cudaFuncSetAttribute(k_sample<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = fused_attrs<double>();
    auto oz_attrs = [&](const void* fn) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    };
    oz_attrs((const void*)k_oz<OZ_APPLY>);
    oz_attrs((const void*)k_oz<OZ_PROB>);
    oz_attrs((const void*)k_oz<OZ_PROB_BOUND>);
    if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_ozf, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzfSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_ozf, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    for (const void* fn : {(const void*)k_ozs<false>, (const void*)k_ozs<true>}) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzsSmem);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    return e;
  }
  cudaError_t e = cudaFuncSetAttribute(k_sample<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = fused_attrs<float>();
  for (const void* fn : {(const void*)k_fused_spec<2, false>, (const void*)k_fused_spec<2, true>,
                         (const void*)k_fused_spec<4, false>, (const void*)k_fused_spec<4, true>}) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmemMax);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
  for (const void* fn : {(const void*)k_fused_tc, (const void*)k_fused_tc_spec<false>, (const void*)k_fused_tc_spec<true>}) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmemMax);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
  return e;
}

// ---- host instantiation (test hook; same op arithmetic as inst_block) -------------------
void instantiate_block_host(const InstArgs& a, int blk, uint64_t seed, uint64_t traj,
                            double2* k0, double2* k1, double* u) {
  const int k = blk % a.nstab;
  const int rnd = a.round_base + blk / a.nstab;
  const BlockInfo bi = a.blocks[k];
  const int w = bi.w, C = 1 << w;
  const double (*sm)[16][2] = reinterpret_cast<const double (*)[16][2]>(a.mats);
  double2 U[32 * 16];
  for (int i = 0; i < 32 * 16; ++i) {
    int r = i / 16, c = i % 16;
    U[i] = make_double2((r < C && r == c) ? 1.0 : 0.0, 0.0);
  }
  for (int oi = bi.op_begin; oi < bi.op_end; ++oi) {
    const ProgOp op = a.ops[oi];
    if (op.kind == OP_T1 || op.kind == OP_T2) {
      if (!twirl_fires(op, a.prob[op.pidx], seed, traj, rnd)) continue;
      if (op.kind == OP_T1) {
        for (int it = 0; it < items_1q(w); ++it) apply1_item(U, w, op.q0, sm[op.mat], it);
      } else {
        for (int it = 0; it < items_2q(w); ++it) apply2_item(U, w, op.q0, op.q1, sm[op.mat], it);
      }
      continue;
    }
    if (op.kind == OP_N1 || op.kind == OP_N2) {
      const int code = noise_code(op, a.prob[op.pidx], seed, traj, rnd);
      if (!code) continue;
      if (op.kind == OP_N1) {
        for (int it = 0; it < items_1q(w); ++it) apply1_item(U, w, op.q0, sm[code], it);
      } else {
        const int pa = code >> 2, pd = code & 3;
        if (pa) for (int it = 0; it < items_1q(w); ++it) apply1_item(U, w, op.q0, sm[pa], it);
        if (pd) for (int it = 0; it < items_1q(w); ++it) apply1_item(U, w, op.q1, sm[pd], it);
      }
    } else if (op.kind == OP_U1) {
      for (int it = 0; it < items_1q(w); ++it) apply1_item(U, w, op.q0, sm[op.mat], it);
    } else {
      for (int it = 0; it < items_2q(w); ++it) apply2_item(U, w, op.q0, op.q1, sm[op.mat], it);
    }
  }
  for (int i = 0; i < 256; ++i) {
    const int r = i / 16, c = i % 16;
    k0[i] = (r < C && c < C) ? U[r * 16 + c] : make_double2(0, 0);
    k1[i] = (r < C && c < C) ? U[(C + r) * 16 + c] : make_double2(0, 0);
  }
  *u = uniform53(draw(seed, traj, (uint64_t)rnd, 0u, (uint32_t)(a.nd + k), TAG_MEASURE).v[0]);
}

}  // namespace qec
