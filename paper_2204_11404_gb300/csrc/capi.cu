// C-ABI of the simulator: handle lifetime, device buffers, the noise-free init
// round, the per-trajectory CUDA graph, and the host-side test hooks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/qecsv.h"
#include "common.cuh"
#include "kernels.hpp"
#include "ozaki.cuh"
#include "program.hpp"

using namespace qec;

namespace {

thread_local std::string g_err;

qec_status fail(qec_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define QEC_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? QEC_ENOMEM : QEC_ECUDA,              \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    }                                                                                    \
  } while (0)

constexpr uint32_t kBatchCap = 1024;
constexpr int kCtlRing = 8;          // pinned control headers in flight per simulator
constexpr int kMaxRounds = 64;       // per-block buffers are sized for this many rounds

}  // namespace

namespace qec {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace qec

struct qec_sim {
  qec_params p{};
  int device = 0, num_sms = 0;
  cudaStream_t work = nullptr;          // owned; all kernels and the graph run here
  cudaStream_t user = nullptr;          // caller's stream (ordering only)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaEvent_t kev[3] = {nullptr, nullptr, nullptr};   // event-record nodes around the instrumented block
  int timed_block = -1;
  Program init_prog, prog;
  int D = 0, nstab = 0, R = 0, S = 0;
  size_t amp = 16;
  void* psi = nullptr;
  void* psi0 = nullptr;
  void* psi2 = nullptr;                        // second working state of the speculative passes
  bool spec = false;                           // QEC_C128_TC with every block on the speculative pass
  ProgOp* d_ops[2] = {nullptr, nullptr};       // [0] init, [1] noisy
  BlockInfo* d_blocks[2] = {nullptr, nullptr};
  double* d_mats[2] = {nullptr, nullptr};
  void* d_kraus = nullptr;                     // S (>= nstab) blocks
  double* d_u = nullptr;
  double* d_A = nullptr;
  double* d_N = nullptr;
  int* d_m = nullptr;
  double* d_partials = nullptr;
  Ctl* d_ctl = nullptr;
  Ctl* h_ctl = nullptr;                        // pinned ring of kCtlRing headers
  cudaEvent_t ctl_ev[kCtlRing] = {};           // recorded after each header's H2D copy
  int ctl_next = 0;
  size_t ops_cap = 0;                          // ProgOp entries d_ops[1] holds
  double* d_hist_part = nullptr;
  double* d_hist = nullptr;
  uint8_t* d_syn = nullptr;
  uint8_t* d_bits = nullptr;
  uint8_t* d_log = nullptr;
  int32_t* d_events = nullptr;
  uint32_t ev_cap = 0;
  // One trajectory is one graph; event-record nodes bracket the instrumented block's passes.
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool ran = false;
  int blk_cap = 0;      // blocks the Kraus/measurement buffers hold
  int syn_cap = 0;      // bytes per trajectory the syndrome buffer holds

  int syn_stride() const { return (R + 1) * nstab; }
};

namespace {

template <typename T>
qec_status dmalloc(T** p, size_t bytes) {
  QEC_CUDA(cudaMalloc((void**)p, bytes));
  return QEC_OK;
}

qec_status upload_program(qec_sim* s, int which, const Program& P) {
  qec_status st;
  size_t cap = P.ops.size() + 1;
  if (which == 1) {   // room for every noise site and coherent op, so qec_reconfigure never reallocates
    qec_params full = s->p;
    full.noise = qec_noise{1, 1, 1, 1, 1, 1, 1, 1, 1, 0};
    Program F;
    std::string err;
    if (build_program(full, true, F, err, true) && F.ops.size() + 1 > cap) cap = F.ops.size() + 1;
    s->ops_cap = cap;
  }
  if ((st = dmalloc(&s->d_ops[which], sizeof(ProgOp) * cap)) != QEC_OK) return st;
  if ((st = dmalloc(&s->d_blocks[which], sizeof(BlockInfo) * P.blocks.size())) != QEC_OK) return st;
  if ((st = dmalloc(&s->d_mats[which], sizeof(P.mats))) != QEC_OK) return st;
  if (!P.ops.empty())
    QEC_CUDA(cudaMemcpy(s->d_ops[which], P.ops.data(), sizeof(ProgOp) * P.ops.size(), cudaMemcpyHostToDevice));
  QEC_CUDA(cudaMemcpy(s->d_blocks[which], P.blocks.data(), sizeof(BlockInfo) * P.blocks.size(), cudaMemcpyHostToDevice));
  QEC_CUDA(cudaMemcpy(s->d_mats[which], P.mats, sizeof(P.mats), cudaMemcpyHostToDevice));
  return QEC_OK;
}

InstArgs inst_args(const qec_sim* s, int which, int round_base, int nblk, bool with_ctl) {
  const Program& P = which ? s->prog : s->init_prog;
  InstArgs a;
  a.ops = s->d_ops[which];
  a.blocks = s->d_blocks[which];
  a.mats = s->d_mats[which];
  for (int i = 0; i < PR_COUNT; ++i) a.prob[i] = P.prob[i];
  a.nstab = s->nstab;
  a.nd = s->D;
  a.round_base = round_base;
  a.nblk = nblk;
  a.kraus = s->d_kraus;
  a.u = s->d_u;
  a.ctl = with_ctl ? s->d_ctl : nullptr;
  a.events = (with_ctl && s->ev_cap) ? s->d_events : nullptr;
  return a;
}

PassArgs pass_args(const qec_sim* s, const Program& P, int blk, const void* src, void* dst, bool forced,
                   uint8_t* syn, int syn_idx) {
  const BlockInfo& bi = P.blocks[blk % s->nstab];
  PassArgs a;
  a.src = src;
  a.dst = dst;
  a.D = s->D;
  a.w = bi.w;
  for (int j = 0; j < 4; ++j) a.q[j] = bi.q[j] < 0 ? 0 : bi.q[j];
  a.kraus = static_cast<const char*>(s->d_kraus) + (size_t)blk * KRAUS_STRIDE * s->amp;
  a.u = s->d_u + blk;
  a.forced = forced ? bi.offset : -1;
  a.A = s->d_A + blk;
  a.N = s->d_N + blk;
  a.m = s->d_m + blk;
  a.ctl = s->d_ctl;
  a.partials = s->d_partials;
  a.syn = syn;
  a.syn_stride = s->syn_stride();
  a.syn_idx = syn_idx;
  a.offset = bi.offset;
  return a;
}

// Noise-free init round with outcomes forced to the zero syndrome (Sec. III.B); result in psi0.
qec_status run_init_round(qec_sim* s) {
  QEC_CUDA(launch_set_basis0(s->p.precision, s->psi0, s->D, s->work));
  QEC_CUDA(launch_instantiate(s->p.precision, inst_args(s, 0, 0, s->nstab, false), s->work));
  for (int k = 0; k < s->nstab; ++k) {
    PassArgs a = pass_args(s, s->init_prog, k, s->psi0, s->psi0, true, nullptr, 0);
    QEC_CUDA(launch_prob(s->p.precision, a, pass_grid_for(s->p.precision, true, s->D, a.w, s->num_sms), s->work));
    QEC_CUDA(launch_apply(s->p.precision, a, pass_grid_for(s->p.precision, false, s->D, a.w, s->num_sms), s->work));
  }
  return QEC_OK;   // no host wait: every later call is ordered after it on the same stream
}

// The instrumented block: the first weight-4 block of the middle noisy round, or its first block
// when the code has none (the repetition code).
int pick_timed_block(const qec_sim* s) {
  const int rnd = (s->R + 1) / 2;
  for (int k = 0; k < s->nstab; ++k)
    if (s->prog.blocks[k].w == 4) return (rnd - 1) * s->nstab + k;
  return (rnd - 1) * s->nstab;
}

PassArgs traj_pass(const qec_sim* s, int b) {
  const void* src = b == 0 ? s->psi0 : s->psi;
  const int rnd = 1 + b / s->nstab, k = b % s->nstab;
  return pass_args(s, s->prog, b, src, s->psi, false, s->d_syn, rnd * s->nstab + k);
}

// Speculative passes (every form): block b reads the state block b-1 wrote (block 0 the init state)
// and writes the other working buffer, so that a wrong guess is corrected from its untouched input.
void* spec_out(const qec_sim* s, int b) { return (b & 1) ? s->psi2 : s->psi; }

PassArgs spec_pass(const qec_sim* s, int b) {
  PassArgs a = traj_pass(s, b);
  a.src = b == 0 ? s->psi0 : spec_out(s, b - 1);
  a.dst = spec_out(s, b);
  a.spec_prev = b >= s->nstab ? a.syn_idx - s->nstab : -1;
  return a;
}

bool spec_applies(const qec_sim*) { return true; }

// The state the last block wrote (the init state when there are no noisy rounds).
const void* final_state(const qec_sim* s) {
  if (s->S == 0) return s->psi0;
  return s->spec ? spec_out(s, s->S - 1) : s->psi;
}

// Block b's apply pass is fused with block b+1's probability pass (one HBM read + write per
// stabilizer) in the complex64 forms (k_fused, k_fused_tc) and in the tensor-core complex128 form
// (k_ozf) wherever both blocks fit one tile; the FP64 CUDA-core form keeps them separate (both of its
// passes are bound by the FP64 pipe, so one pass saves no time there).  The complex128 forms take
// this path only with their speculative passes switched off (qec_debug_speculation).
bool fused_step(const qec_sim* s, int b) {
  if (b < 0 || b + 1 >= s->S) return false;
  if (!is_f64(s->p.precision)) return true;
  if (s->p.precision != QEC_C128_TC) return false;
  return fused_oz_applies(traj_pass(s, b), traj_pass(s, b + 1));
}

// One probability / apply pass of a block outside the fused steps: on the tensor cores for
// QEC_C128_TC blocks whose tile fits, else the CUDA-core pass of the precision.
cudaError_t prob_pass(qec_sim* s, const PassArgs& a) {
  if (s->p.precision == QEC_C128_TC && apply_oz_applies(a)) return launch_prob_oz(a, s->num_sms, s->work);
  return launch_prob(s->p.precision, a, pass_grid_for(s->p.precision, true, s->D, a.w, s->num_sms), s->work);
}

cudaError_t apply_pass(qec_sim* s, const PassArgs& a) {
  if (s->p.precision == QEC_C128_TC && apply_oz_applies(a)) return launch_apply_oz(a, s->num_sms, s->work);
  return launch_apply(s->p.precision, a, pass_grid_for(s->p.precision, false, s->D, a.w, s->num_sms), s->work);
}

qec_status record(qec_sim* s, int i) {
  QEC_CUDA(cudaEventRecordWithFlags(s->kev[i], s->work, cudaEventRecordExternal));
  return QEC_OK;
}

qec_status enqueue_readout(qec_sim* s) {
  ReadArgs r;
  r.src = final_state(s);
  r.D = s->D;
  r.k1 = hist_k1(s->D);
  r.d = s->p.d;
  r.rounds = s->R;
  r.grid_hist = hist_grid(s->D, s->num_sms);
  r.hist_part = s->d_hist_part;
  r.hist = s->d_hist;
  r.ctl = s->d_ctl;
  r.bits = s->d_bits;
  r.logical = s->d_log;
  r.syn = s->d_syn;
  r.syn_stride = s->syn_stride();
  r.nstab = s->nstab;
  QEC_CUDA(launch_readout(s->p.precision, r, s->work));
  return QEC_OK;
}

// The whole trajectory: instantiate, then per block b its probability pass (unless block b-1's
// fused pass computed it) and its apply pass (fused with block b+1's probability pass where
// fused_step), or with the speculative passes its speculative pass and that pass's completion;
// then the readout.  The instrumented block's passes are bracketed by event-record nodes:
// kev[0]..kev[1] its separate probability pass (empty when fused into the previous block's pass, and
// with the speculative passes), kev[1]..kev[2] its apply, fused or speculative pass (without the
// exact-probability and corrective launches that follow the tensor-core passes).
qec_status enqueue_trajectory(qec_sim* s) {
  const int tb = s->timed_block;
  qec_status st = QEC_OK;
  if (s->S > 0) QEC_CUDA(launch_instantiate(s->p.precision, inst_args(s, 1, 1, s->S, true), s->work));
  if (s->spec) {   // per block: the speculative pass (kev[1]..kev[2]), then its completion
    for (int b = 0; b < s->S && st == QEC_OK; ++b) {
      const bool timed = b == tb;
      const PassArgs a = spec_pass(s, b);
      double* n_next = b + 1 < s->S ? s->d_N + b + 1 : nullptr;
      if (timed && ((st = record(s, 0)) || (st = record(s, 1)))) return st;
      QEC_CUDA(launch_spec(s->p.precision, a, n_next, b == 0, s->num_sms, s->work));
      if (timed && (st = record(s, 2))) return st;
      QEC_CUDA(launch_spec_fix(s->p.precision, a, n_next, b == 0, s->num_sms, s->work));
    }
    return st == QEC_OK ? enqueue_readout(s) : st;
  }
  for (int b = 0; b < s->S && st == QEC_OK; ++b) {
    const bool timed = b == tb, fused = fused_step(s, b);
    if (timed && (st = record(s, 0))) return st;
    if (b == 0 || !fused_step(s, b - 1)) QEC_CUDA(prob_pass(s, traj_pass(s, b)));
    if (timed && (st = record(s, 1))) return st;
    const PassArgs a = traj_pass(s, b);
    if (fused) {
      PassArgs n = traj_pass(s, b + 1);
      n.src = s->psi;
      if (s->p.precision == QEC_C128_TC) {
        QEC_CUDA(launch_fused_oz(a, n, s->num_sms, s->work));
        if (timed && (st = record(s, 2))) return st;
        QEC_CUDA(launch_prob_oz_check(n, s->num_sms, s->work));
        continue;
      }
      QEC_CUDA(launch_fused(s->p.precision, a, n, s->num_sms, s->work));
    } else {
      QEC_CUDA(apply_pass(s, a));
    }
    if (timed) st = record(s, 2);
  }
  if (st == QEC_OK) st = enqueue_readout(s);
  return st;
}

qec_status capture(qec_sim* s) {
  QEC_CUDA(cudaStreamBeginCapture(s->work, cudaStreamCaptureModeThreadLocal));
  qec_status st = enqueue_trajectory(s);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s->work, &g);
  if (st != QEC_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(QEC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  s->graph = g;
  QEC_CUDA(cudaGraphInstantiate(&s->gexec, g, 0));
  return QEC_OK;
}

qec_status ensure_graph(qec_sim* s) {
  if (s->gexec) return QEC_OK;
  return capture(s);
}

qec_status launch_trajectory(qec_sim* s) {
  QEC_CUDA(cudaGraphLaunch(s->gexec, s->work));
  return QEC_OK;
}

void drop_graph(qec_sim* s) {
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->graph) cudaGraphDestroy(s->graph);
  s->gexec = nullptr;
  s->graph = nullptr;
}

void free_all(qec_sim* s) {
  drop_graph(s);
  void* ptrs[] = {s->psi, s->psi0, s->psi2, s->d_kraus, s->d_u, s->d_A, s->d_N, s->d_m, s->d_partials, s->d_ctl,
                  s->d_hist_part, s->d_hist, s->d_syn, s->d_bits, s->d_log, s->d_events,
                  s->d_ops[0], s->d_ops[1], s->d_blocks[0], s->d_blocks[1], s->d_mats[0], s->d_mats[1]};
  for (void* p : ptrs) if (p) cudaFree(p);
  if (s->h_ctl) cudaFreeHost(s->h_ctl);
  for (cudaEvent_t ev : s->kev) if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : s->ctl_ev) if (ev) cudaEventDestroy(ev);
  if (s->ev_in) cudaEventDestroy(s->ev_in);
  if (s->ev_out) cudaEventDestroy(s->ev_out);
  if (s->work) cudaStreamDestroy(s->work);
}

qec_status create_impl(const qec_params* params, void* stream, qec_sim** out) {
  if (!params || !out) return fail(QEC_EINVAL, "null argument");
  *out = nullptr;
  std::string err;
  if (!validate_params(*params, err)) return fail(QEC_EINVAL, err);
  if (params->layout != QEC_LAYOUT_REDUCED)
    return fail(QEC_EUNSUPPORTED, "only the reduced (d^2+1 qubit) register runs on the GPU");
  qec_sim* s = new (std::nothrow) qec_sim();
  if (!s) return fail(QEC_ENOMEM, "host allocation failed");
  qec_status st = QEC_OK;
  auto bail = [&](qec_status x) { free_all(s); delete s; return x; };
  s->p = *params;
  s->user = static_cast<cudaStream_t>(stream);
  if (!build_program(s->p, false, s->init_prog, err) || !build_program(s->p, true, s->prog, err))
    return bail(fail(QEC_EINVAL, err));
  s->D = s->prog.nd;
  s->nstab = s->prog.nstab;
  s->R = s->p.rounds;
  s->S = s->nstab * s->R;
  s->amp = is_f64(s->p.precision) ? 16 : 8;
  if (s->R > 0) s->timed_block = pick_timed_block(s);
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
  int prio = 0;   // the work stream inherits the caller's stream priority
  if (e == cudaSuccess && s->user) e = cudaStreamGetPriority(s->user, &prio);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->work, cudaStreamNonBlocking, prio);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreate(&s->kev[i]);
  for (int i = 0; i < kCtlRing && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&s->ctl_ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = setup_kernels(s->p.precision, s->D);
  if (e != cudaSuccess) return bail(fail(QEC_ECUDA, std::string("CUDA setup: ") + cudaGetErrorString(e)));
  const size_t state_bytes = ((size_t)1 << s->D) * s->amp;
  const int nblk = s->nstab * kMaxRounds;   // room for any round count (qec_reconfigure)
  const int k1 = hist_k1(s->D);
  s->spec = spec_applies(s);
  if (s->spec && (st = dmalloc(&s->psi2, state_bytes))) return bail(st);
  if ((st = dmalloc(&s->psi, state_bytes)) || (st = dmalloc(&s->psi0, state_bytes)) ||
      (st = dmalloc(&s->d_kraus, (size_t)nblk * KRAUS_STRIDE * s->amp)) ||
      (st = dmalloc(&s->d_u, sizeof(double) * nblk)) || (st = dmalloc(&s->d_A, sizeof(double) * nblk)) ||
      (st = dmalloc(&s->d_N, sizeof(double) * nblk)) || (st = dmalloc(&s->d_m, sizeof(int) * nblk)) ||
      (st = dmalloc(&s->d_partials, sizeof(double) * 2 * MAX_PASS_GRID)) ||
      (st = dmalloc(&s->d_ctl, sizeof(Ctl))) ||
      (st = dmalloc(&s->d_hist_part, sizeof(double) * ((size_t)hist_grid(s->D, s->num_sms) << k1))) ||
      (st = dmalloc(&s->d_hist, sizeof(double) << k1)) ||
      (st = dmalloc(&s->d_syn, (size_t)kBatchCap * (kMaxRounds + 1) * s->nstab)) ||
      (st = dmalloc(&s->d_bits, (size_t)kBatchCap * s->D)) || (st = dmalloc(&s->d_log, kBatchCap)))
    return bail(st);
  s->blk_cap = nblk;
  s->syn_cap = (kMaxRounds + 1) * s->nstab;
  e = cudaMallocHost((void**)&s->h_ctl, sizeof(Ctl) * kCtlRing);
  if (e != cudaSuccess) return bail(fail(QEC_ENOMEM, "pinned allocation failed"));
  std::memset(s->h_ctl, 0, sizeof(Ctl) * kCtlRing);
  e = cudaMemcpy(s->d_ctl, s->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(fail(QEC_ECUDA, cudaGetErrorString(e)));
  if ((st = upload_program(s, 0, s->init_prog)) || (st = upload_program(s, 1, s->prog))) return bail(st);
  if ((st = run_init_round(s))) return bail(st);
  *out = s;
  return QEC_OK;
}

qec_status run_impl(qec_sim* s, uint64_t seed, uint64_t first, uint32_t n, uint8_t* syn, uint8_t* bits,
                    uint8_t* logical, bool host_out) {
  if (!s) return fail(QEC_EINVAL, "null handle");
  qec_status st = ensure_graph(s);
  if (st) return st;
  if (s->user) {
    QEC_CUDA(cudaEventRecord(s->ev_in, s->user));
    QEC_CUDA(cudaStreamWaitEvent(s->work, s->ev_in, 0));
  }
  const cudaMemcpyKind kind = host_out ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const size_t ss = (size_t)s->syn_stride(), bs = (size_t)s->D;
  for (uint32_t done = 0; done < n;) {
    const uint32_t chunk = (n - done) < kBatchCap ? (n - done) : kBatchCap;
    if (done > 0) QEC_CUDA(cudaStreamSynchronize(s->work));   // the device output batch is reused
    const int slot = s->ctl_next;
    s->ctl_next = (s->ctl_next + 1) % kCtlRing;
    QEC_CUDA(cudaEventSynchronize(s->ctl_ev[slot]));          // this header's previous copy is done
    Ctl* h = s->h_ctl + slot;
    h->seed = seed;
    h->first = first + done;
    h->traj = first + done;
    h->ticket = 0;
    h->ev_cap = s->ev_cap;
    const size_t head = done == 0 ? offsetof(Ctl, prob_uncertain) : offsetof(Ctl, ticket);   // events reset per call
    if (done == 0) h->n_events = 0;
    QEC_CUDA(cudaMemcpyAsync(s->d_ctl, h, head, cudaMemcpyHostToDevice, s->work));
    QEC_CUDA(cudaEventRecord(s->ctl_ev[slot], s->work));
    for (uint32_t t = 0; t < chunk; ++t) {
      st = launch_trajectory(s);
      if (st) return st;
    }
    if (syn) QEC_CUDA(cudaMemcpyAsync(syn + done * ss, s->d_syn, chunk * ss, kind, s->work));
    if (bits) QEC_CUDA(cudaMemcpyAsync(bits + done * bs, s->d_bits, chunk * bs, kind, s->work));
    if (logical) QEC_CUDA(cudaMemcpyAsync(logical + done, s->d_log, chunk, kind, s->work));
    done += chunk;
  }
  if (s->user) {
    QEC_CUDA(cudaEventRecord(s->ev_out, s->work));
    QEC_CUDA(cudaStreamWaitEvent(s->user, s->ev_out, 0));
  }
  if (host_out) {
    QEC_CUDA(cudaStreamSynchronize(s->work));
    unsigned int status = 0;
    QEC_CUDA(cudaMemcpy(&status, &s->d_ctl->status, sizeof(status), cudaMemcpyDeviceToHost));
    if (status) return fail(QEC_ETIMEOUT, "a bounded device wait gave up; results are invalid");
  }
  QEC_CUDA(cudaGetLastError());
  if (n) s->ran = true;
  return QEC_OK;
}

}  // namespace

extern "C" {

qec_status qec_create(const qec_params* params, void* cuda_stream, qec_sim** out) {
  try {
    return create_impl(params, cuda_stream, out);
  } catch (...) {
    return fail(QEC_ENOMEM, "exception in qec_create");
  }
}

qec_status qec_run_trajectories(qec_sim* sim, uint64_t seed, uint64_t first_traj, uint32_t n,
                                uint8_t* syndromes, uint8_t* data_bits, uint8_t* raw_logical) {
  try {
    return run_impl(sim, seed, first_traj, n, syndromes, data_bits, raw_logical, true);
  } catch (...) {
    return fail(QEC_ENOMEM, "exception in qec_run_trajectories");
  }
}

qec_status qec_run_trajectories_device(qec_sim* sim, uint64_t seed, uint64_t first_traj, uint32_t n,
                                       uint8_t* d_syndromes, uint8_t* d_data_bits, uint8_t* d_raw_logical) {
  try {
    return run_impl(sim, seed, first_traj, n, d_syndromes, d_data_bits, d_raw_logical, false);
  } catch (...) {
    return fail(QEC_ENOMEM, "exception in qec_run_trajectories_device");
  }
}

uint64_t qec_state_len(const qec_sim* sim) { return sim ? (1ull << sim->D) : 0ull; }

qec_status qec_get_state(qec_sim* s, void* host_buf, size_t bytes) {
  if (!s || !host_buf) return fail(QEC_EINVAL, "null argument");
  const size_t n = (size_t)1 << s->D;
  if (bytes < 16 * n) return fail(QEC_EINVAL, "host buffer too small");
  if (!s->ran) return fail(QEC_EINVAL, "no trajectory has run yet");
  QEC_CUDA(cudaStreamSynchronize(s->work));
  Ctl c;
  QEC_CUDA(cudaMemcpy(&c, s->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  const void* src = final_state(s);
  double* out = static_cast<double*>(host_buf);
  const double scale = 1.0 / std::sqrt(c.final_norm);
  if (is_f64(s->p.precision)) {
    QEC_CUDA(cudaMemcpy(out, src, 16 * n, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < 2 * n; ++i) out[i] *= scale;
  } else {
    std::vector<float> tmp(2 * n);
    QEC_CUDA(cudaMemcpy(tmp.data(), src, 8 * n, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < 2 * n; ++i) out[i] = (double)tmp[i] * scale;
  }
  return QEC_OK;
}

qec_status qec_record_events(qec_sim* s, uint32_t max_events) {
  if (!s) return fail(QEC_EINVAL, "null handle");
  QEC_CUDA(cudaStreamSynchronize(s->work));
  if (s->d_events) {
    QEC_CUDA(cudaFree(s->d_events));
    s->d_events = nullptr;
  }
  s->ev_cap = 0;
  if (max_events) {
    qec_status st = dmalloc(&s->d_events, (size_t)max_events * 5 * sizeof(int32_t));
    if (st) return st;
    s->ev_cap = max_events;
  }
  drop_graph(s);   // the instantiate node holds the events pointer
  return QEC_OK;
}

qec_status qec_get_events(qec_sim* s, int32_t* host_events, uint32_t max_events, uint32_t* count) {
  if (!s || !count) return fail(QEC_EINVAL, "null argument");
  QEC_CUDA(cudaStreamSynchronize(s->work));
  Ctl c;
  QEC_CUDA(cudaMemcpy(&c, s->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  uint32_t n = c.n_events < s->ev_cap ? c.n_events : s->ev_cap;
  if (n > max_events) n = max_events;
  *count = n;
  if (n && host_events) QEC_CUDA(cudaMemcpy(host_events, s->d_events, (size_t)n * 5 * sizeof(int32_t), cudaMemcpyDeviceToHost));
  return QEC_OK;
}

qec_status qec_reconfigure(qec_sim* s, const qec_params* params) {
  if (!s || !params) return fail(QEC_EINVAL, "null argument");
  std::string err;
  if (!validate_params(*params, err)) return fail(QEC_EINVAL, err);
  if (params->d != s->p.d || params->gates != s->p.gates || params->precision != s->p.precision ||
      params->layout != s->p.layout || params->code != s->p.code)
    return fail(QEC_EINVAL, "qec_reconfigure keeps d, gate set, precision, layout and code");
  Program P;
  if (!build_program(*params, true, P, err)) return fail(QEC_EINVAL, err);
  if (params->rounds > kMaxRounds) return fail(QEC_EINVAL, "rounds exceed the simulator's capacity");
  if (P.ops.size() + 1 > s->ops_cap) return fail(QEC_EINVAL, "program larger than the simulator's capacity");
  QEC_CUDA(cudaStreamSynchronize(s->work));   // in-flight work still reads the old program
  drop_graph(s);
  const int S = s->nstab * params->rounds;
  s->prog = P;
  if (!P.ops.empty())
    QEC_CUDA(cudaMemcpyAsync(s->d_ops[1], s->prog.ops.data(), sizeof(ProgOp) * P.ops.size(), cudaMemcpyHostToDevice,
                             s->work));
  QEC_CUDA(cudaMemcpyAsync(s->d_blocks[1], s->prog.blocks.data(), sizeof(BlockInfo) * P.blocks.size(),
                           cudaMemcpyHostToDevice, s->work));
  QEC_CUDA(cudaMemcpyAsync(s->d_mats[1], s->prog.mats, sizeof(P.mats), cudaMemcpyHostToDevice, s->work));
  QEC_CUDA(cudaStreamSynchronize(s->work));   // the host copies in s->prog must outlive the uploads
  s->p = *params;
  s->R = params->rounds;
  s->S = S;
  s->timed_block = s->R > 0 ? pick_timed_block(s) : -1;
  s->ran = false;
  return QEC_OK;
}

qec_status qec_selftest_wait(qec_sim* s, uint32_t polls) {
  if (!s) return fail(QEC_EINVAL, "null handle");
  if (polls == 0 || polls > 10000000) return fail(QEC_EINVAL, "polls must be in [1, 1e7]");
  QEC_CUDA(cudaStreamSynchronize(s->work));
  QEC_CUDA(cudaMemsetAsync(&s->d_ctl->status, 0, sizeof(unsigned int), s->work));
  QEC_CUDA(launch_wait_selftest(&s->d_ctl->status, (long)polls, s->work));
  QEC_CUDA(cudaStreamSynchronize(s->work));
  unsigned int status = 0;
  QEC_CUDA(cudaMemcpy(&status, &s->d_ctl->status, sizeof(status), cudaMemcpyDeviceToHost));
  QEC_CUDA(cudaMemsetAsync(&s->d_ctl->status, 0, sizeof(unsigned int), s->work));   // leave the sim usable
  QEC_CUDA(cudaStreamSynchronize(s->work));
  if (status) return fail(QEC_ETIMEOUT, "bounded device wait gave up (self-test)");
  return QEC_OK;
}

qec_status qec_kernel_times(qec_sim* s, float* ms, int32_t* block) {
  if (!s || !ms || !block) return fail(QEC_EINVAL, "null argument");
  if (!s->ran || s->timed_block < 0) return fail(QEC_EINVAL, "no instrumented trajectory has run");
  QEC_CUDA(cudaStreamSynchronize(s->work));
  QEC_CUDA(cudaEventElapsedTime(&ms[0], s->kev[0], s->kev[1]));
  QEC_CUDA(cudaEventElapsedTime(&ms[1], s->kev[1], s->kev[2]));
  *block = s->timed_block;
  return QEC_OK;
}

qec_status qec_select_timed_block(qec_sim* s, int32_t w_apply, int32_t w_next, int32_t* block) {
  if (!s || !block) return fail(QEC_EINVAL, "null argument");
  if (s->R <= 0) return fail(QEC_EINVAL, "the sim has no noisy round");
  const int rnd = (s->R + 1) / 2;
  for (int k = 0; k < s->nstab; ++k) {
    const int b = (rnd - 1) * s->nstab + k;
    if (b + 1 >= s->S) break;
    if (s->prog.blocks[k].w == w_apply && s->prog.blocks[(k + 1) % s->nstab].w == w_next) {
      drop_graph(s);   // the next trajectory records the events around block b
      s->timed_block = b;
      *block = b;
      return QEC_OK;
    }
  }
  return fail(QEC_EINVAL, "no block of the middle noisy round with those weights");
}

qec_status qec_destroy(qec_sim* s) {
  if (!s) return QEC_OK;
  if (s->work) cudaStreamSynchronize(s->work);
  free_all(s);
  delete s;
  return QEC_OK;
}

const char* qec_last_error(void) { return g_err.c_str(); }

qec_status qec_debug_program(const qec_params* params, int32_t* ops, uint32_t cap, uint32_t* n_ops,
                             int32_t* block_info, uint32_t block_cap, uint32_t* n_blocks) {
  if (!params || !n_ops || !n_blocks) return fail(QEC_EINVAL, "null argument");
  std::string err;
  Program P;
  if (!build_program(*params, true, P, err)) return fail(QEC_EINVAL, err);
  *n_ops = (uint32_t)P.ops.size();
  *n_blocks = (uint32_t)P.blocks.size();
  for (size_t b = 0; b < P.blocks.size(); ++b) {
    const BlockInfo& bi = P.blocks[b];
    if (block_info && b < block_cap) {
      int32_t* o = block_info + 6 * b;
      o[0] = bi.w; o[1] = bi.q[0]; o[2] = bi.q[1]; o[3] = bi.q[2]; o[4] = bi.q[3]; o[5] = bi.offset;
    }
    for (int i = bi.op_begin; i < bi.op_end; ++i) {
      if (ops && (uint32_t)i < cap) {
        const ProgOp& op = P.ops[i];
        int32_t* o = ops + 6 * i;
        o[0] = (int32_t)b; o[1] = op.kind; o[2] = op.q0; o[3] = op.q1; o[4] = op.step; o[5] = (int32_t)op.site;
      }
    }
  }
  return QEC_OK;
}

// Variant 4: the fused pass's probability arithmetic on the CPU, A as one tile (one exponent for all
// of A, one for all of B), as the fused kernel's threads hold it: 16 inputs and 16 outputs each.
static void ozaki_fused_prob(const double* A, const double* B, int m, double* out) {
  int Et = 0, EP = 0;
  for (int i = 0; i < m * 32; ++i) Et = std::max(Et, oz::bexp(A[i]));
  for (int i = 0; i < 32 * 32; ++i) EP = std::max(EP, oz::bexp(B[i]));
  Et = std::max(Et, 24);
  std::vector<int> da((size_t)m * 32 * 3), db(32 * 32 * 3);
  std::vector<uint32_t> a24((size_t)m * 32);
  for (int i = 0; i < m * 32; ++i) {
    const uint32_t a = oz::top24(oz::d2u(A[i]), Et);
    a24[i] = a;
    const int neg = (int)(oz::d2u(A[i]) >> 63);
    for (int p = 0; p < 3; ++p) da[(size_t)i * 3 + p] = (neg ? -1 : 1) * (int)((a >> (16 - 8 * p)) & 0xFF);
  }
  for (int i = 0; i < 32 * 32; ++i) {   // B: the top 3 bytes of its 56-bit magnitude under EP
    const uint64_t X = EP ? oz::mag56(B[i], EP) : 0ull;
    const int neg = (int)(oz::d2u(B[i]) >> 63);
    for (int p = 0; p < 3; ++p) db[(size_t)i * 3 + p] = (neg ? -1 : 1) * (int)((X >> (48 - 8 * p)) & 0xFF);
  }
  for (int r = 0; r < m; ++r) {
    oz::FusedSums sums;   // the row's two threads' sums, as the kernel's threads accumulate them
    for (int h = 0; h < 2; ++h) {   // a thread's 16 outputs n = 16h..16h+15 and 16 inputs k = 16h..16h+15
      uint64_t aacc = 0, nacc = 0;
      for (int n = 16 * h; n < 16 * h + 16; ++n) {
        float D[3];
        for (int t = 0; t < 3; ++t) {
          float acc = 0.f;   // exact: integers below 2^23
          for (int p = 0; p <= t; ++p)
            for (int k = 0; k < 32; ++k)
              acc += (float)(da[((size_t)r * 32 + k) * 3 + p] * db[((size_t)n * 32 + k) * 3 + (t - p)]);
          D[t] = acc;
        }
        const int64_t z = oz::combine3(D);
        aacc += (uint64_t)(z * z);
        const uint64_t a = a24[(size_t)r * 32 + n];
        nacc += a * a;
      }
      sums.add_tile(nacc, aacc, Et, EP);
    }
    double sn, en, sa, ea;
    sums.finish(sn, en, sa, ea);
    out[r * 32] = sa;
    out[r * 32 + 1] = ea;
    out[r * 32 + 2] = sn;
    out[r * 32 + 3] = en;
  }
}

// Variant 5: the speculative pass's two sums of squares on the CPU, over the reals of A (m rows of
// 32, each row two threads' 16): out[r][0], out[r][1] = the input-side sum of row r (each real's top
// 24 bits under the row's largest exponent, as the slicing holds them) and its bound; out[r][2],
// out[r][3] = the output-side sum of the same reals (top 24 bits under the largest exponent of all of
// A, as one tile) and its bound.
static void ozaki_spec_sums(const double* A, int m, double* out) {
  int Et = 0;
  for (int i = 0; i < m * 32; ++i) Et = std::max(Et, oz::bexp(A[i]));
  Et = std::max(Et, 24);
  for (int r = 0; r < m; ++r) {
    int E = 0;
    for (int k = 0; k < 32; ++k) E = std::max(E, oz::bexp(A[r * 32 + k]));
    oz::SqSum24 in, o;
    for (int h = 0; h < 2; ++h) {
      uint64_t nin = 0, nout = 0;
      for (int k = 16 * h; k < 16 * h + 16; ++k) {
        const uint64_t a = (E ? oz::mag56(A[r * 32 + k], E) : 0ull) >> 32;
        const uint64_t b = oz::top24(oz::d2u(A[r * 32 + k]), Et);
        nin += a * a;
        nout += b * b;
      }
      in.add(nin, E);
      o.add(nout, Et);
    }
    in.finish(out[r * 32], out[r * 32 + 1]);
    o.finish(out[r * 32 + 2], out[r * 32 + 3]);
  }
}

qec_status qec_debug_ozaki_gemm(const double* A, const double* B, int32_t m, int32_t variant, double* out) {
  if (!A || !B || !out || m <= 0 || variant < 0 || variant > 5) return fail(QEC_EINVAL, "bad argument");
  if (variant == 4) {
    ozaki_fused_prob(A, B, m, out);
    return QEC_OK;
  }
  if (variant == 5) {
    ozaki_spec_sums(A, m, out);
    return QEC_OK;
  }
  std::vector<int> ea(m), eb(32);
  std::vector<int> da((size_t)m * 32 * oz::kSlices), db(32 * 32 * oz::kSlices);
  for (int r = 0; r < m; ++r) {
    int E = 0;
    for (int k = 0; k < 32; ++k) E = std::max(E, oz::bexp(A[r * 32 + k]));
    ea[r] = E;
    for (int k = 0; k < 32; ++k) oz::split7(A[r * 32 + k], E, &da[((size_t)r * 32 + k) * oz::kSlices]);
  }
  int EB = 0;   // variant 2 (probability pass): one exponent for all of B
  for (int i = 0; i < 32 * 32; ++i) EB = std::max(EB, oz::bexp(B[i]));
  for (int n = 0; n < 32; ++n) {
    int E = 0;
    for (int k = 0; k < 32; ++k) E = std::max(E, oz::bexp(B[n * 32 + k]));
    eb[n] = (variant == 2 || variant == 3) ? EB : E;
    for (int k = 0; k < 32; ++k) oz::split7(B[n * 32 + k], eb[n], &db[((size_t)n * 32 + k) * oz::kSlices]);
  }
  for (int r = 0; r < m; ++r) {
    oz::SqAcc sa, sn;   // variants 2, 3: parts of kPart reals of a row, as the pass's threads hold them
    oz::SqAccS ss;
    double A2 = 0.0, N2 = 0.0, E3 = 0.0;
    for (int n = 0; n < 32; ++n) {
      if (variant == 3) {   // the bounded pass: 3 slices each, every product, diagonals 0..4
        float D5[5];
        for (int t = 0; t < 5; ++t) {
          float acc = 0.f;
          for (int p = 0; p < 3; ++p) {
            const int q = t - p;
            if (q < 0 || q > 2) continue;
            for (int k = 0; k < 32; ++k)
              acc += (float)(da[((size_t)r * 32 + k) * oz::kSlices + p] * db[((size_t)n * 32 + k) * oz::kSlices + q]);
          }
          D5[t] = acc;
        }
        ss.add(oz::combine5(D5));
        if (n % oz::kPart == oz::kPart - 1) {
          const double ah = (ea[r] && EB) ? ss.take(2 * (ea[r] + EB - 2092)) : ss.take(-4000);
          A2 += ah;
          if (ea[r] && EB) E3 += oz::part_bound(ah, ea[r] + EB);
        }
        continue;
      }
      float D[oz::kSlices];
      for (int t = 0; t < oz::kSlices; ++t) {
        float acc = 0.f;   // exact: every partial sum is an integer below 2^24
        for (int p = 0; p <= t; ++p)
          for (int k = 0; k < 32; ++k)
            acc += (float)(da[((size_t)r * 32 + k) * oz::kSlices + p] * db[((size_t)n * 32 + k) * oz::kSlices + (t - p)]);
        D[t] = acc;
      }
      if (variant == 2) {
        const int64_t z = oz::combine7(D);
        sa.add((uint64_t)(z < 0 ? -z : z));
        sn.add(ea[r] ? oz::mag56(A[r * 32 + n], ea[r]) : 0ull);
        if (n % oz::kPart == oz::kPart - 1) {
          A2 += (ea[r] && EB) ? sa.take(2 * (ea[r] + EB - 2098)) : sa.take(-4000);
          N2 += sn.take(2 * (ea[r] - 1078));
        }
        continue;
      }
      if (variant == 1) {   // the apply pass's choice: checked only when the row may leave the range
        int cmin = 4095, cmax = 0;
        for (int j = 0; j < 32; ++j) {
          if (eb[j]) cmin = std::min(cmin, eb[j]);
          cmax = std::max(cmax, eb[j]);
        }
        const bool in_range = ea[r] == 0 || (ea[r] + cmin >= 1076 && ea[r] + cmax <= 2980);
        out[r * 32 + n] = in_range ? oz::assemble7_cvt_inrange(D, ea[r], eb[n]) : oz::assemble7_cvt(D, ea[r], eb[n]);
      } else {
        out[r * 32 + n] = oz::assemble7(D, ea[r], eb[n]);
      }
    }
    if (variant == 2) {
      out[r * 32] = A2;
      out[r * 32 + 1] = N2;
    }
    if (variant == 3) {
      out[r * 32] = A2;
      out[r * 32 + 1] = E3;
    }
  }
  return QEC_OK;
}

qec_status qec_debug_exact_probability(qec_sim* sim, int32_t force, uint64_t* fallbacks) {
  if (!sim || force < -1 || force > 1) return fail(QEC_EINVAL, "bad argument");
  QEC_CUDA(cudaStreamSynchronize(sim->work));
  if (force >= 0) {
    const unsigned int v = (unsigned int)force;
    QEC_CUDA(cudaMemcpy(reinterpret_cast<char*>(sim->d_ctl) + offsetof(Ctl, prob_force_exact), &v, sizeof(v),
                        cudaMemcpyHostToDevice));
  }
  if (fallbacks) {
    unsigned long long c = 0;
    QEC_CUDA(cudaMemcpy(&c, reinterpret_cast<char*>(sim->d_ctl) + offsetof(Ctl, prob_fallbacks), sizeof(c),
                        cudaMemcpyDeviceToHost));
    *fallbacks = c;
  }
  return QEC_OK;
}

qec_status qec_debug_speculation(qec_sim* sim, int32_t enable, uint64_t* misses) {
  if (!sim || enable < -1 || enable > 1) return fail(QEC_EINVAL, "bad argument");
  QEC_CUDA(cudaStreamSynchronize(sim->work));
  if (enable >= 0) {
    if (enable == 1 && !sim->psi2) return fail(QEC_EUNSUPPORTED, "no speculative pass for this simulator");
    if ((enable == 1) != sim->spec) {
      drop_graph(sim);
      sim->spec = enable == 1;
      sim->ran = false;   // the last trajectory's state may sit in the other buffer
    }
  }
  if (misses) {
    unsigned long long c = 0;
    QEC_CUDA(cudaMemcpy(&c, reinterpret_cast<char*>(sim->d_ctl) + offsetof(Ctl, spec_misses), sizeof(c),
                        cudaMemcpyDeviceToHost));
    *misses = c;
  }
  return QEC_OK;
}

qec_status qec_debug_blocks(const qec_params* params, uint64_t seed, uint64_t traj, int32_t round,
                            double* kraus, double* u) {
  if (!params || !kraus || !u) return fail(QEC_EINVAL, "null argument");
  std::string err;
  Program P;
  if (round < 0 || !build_program(*params, round > 0, P, err)) return fail(QEC_EINVAL, err.empty() ? "bad round" : err);
  InstArgs a;
  a.ops = P.ops.data();
  a.blocks = P.blocks.data();
  a.mats = &P.mats[0][0][0];
  for (int i = 0; i < PR_COUNT; ++i) a.prob[i] = P.prob[i];
  a.nstab = P.nstab;
  a.nd = P.nd;
  a.round_base = round;
  a.nblk = P.nstab;
  for (int k = 0; k < P.nstab; ++k) {
    double2* k0 = reinterpret_cast<double2*>(kraus) + (size_t)k * 512;
    instantiate_block_host(a, k, seed, traj, k0, k0 + 256, u + k);
  }
  return QEC_OK;
}

}  // extern "C"
