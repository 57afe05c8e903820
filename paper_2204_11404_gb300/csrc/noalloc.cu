// Trajectory entry point that makes no device allocation.
//
// For callers that cannot call cudaMalloc: code that runs while its framework
// owns every byte of device memory through its own pool or arena, code on a
// latency-critical path where cudaMalloc's implicit device synchronisation is
// not acceptable, or plug-ins that are handed a stream and output buffers but
// no allocator.  All device working memory of the call (circuit program,
// state vectors, Kraus blocks, reduction partials, readout histogram, control
// word) lives in one file-scope static device array below; the caller passes
// only the inputs (parameters, seed, trajectory range) and the device output
// buffers.  The array is sized for the d = 3 register (2^9 amplitudes) with at
// most kNoAllocMaxRounds noisy rounds, and every GPU that loads this library
// holds it until the process exits.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/qecsv.h"
#include "common.cuh"
#include "kernels.hpp"
#include "program.hpp"

using namespace qec;

namespace {

constexpr size_t kNoAllocBytes = (size_t)2 << 20;   // 2 MiB
constexpr int kNoAllocMaxD = 3;
constexpr int kNoAllocMaxRounds = 16;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device (host code must not use the symbol itself:
// in host code its name is only a host-side stand-in).
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

qec_status nfail(qec_status s, const std::string& m) {
  set_last_error(m);   // reported by qec_last_error()
  return s;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off = up256(off + bytes);
    return o;
  }
};

qec_status run_noalloc(const qec_params* params, uint64_t seed, uint64_t first_traj, uint32_t n,
                       uint8_t* d_syndromes, uint8_t* d_data_bits, uint8_t* d_raw_logical, void* cuda_stream) {
  if (!params) return nfail(QEC_EINVAL, "null params");
  std::string err;
  if (!validate_params(*params, err)) return nfail(QEC_EINVAL, err);
  if (params->layout != QEC_LAYOUT_REDUCED) return nfail(QEC_EUNSUPPORTED, "only the reduced register runs on the GPU");
  if (params->d > kNoAllocMaxD || params->rounds > kNoAllocMaxRounds)
    return nfail(QEC_EINVAL, "qec_run_trajectories_noalloc: its static device scratch (2 MiB) holds at most d = 3 "
                             "and 16 noisy rounds; use qec_create/qec_run_trajectories for larger runs");
  if (n == 0) return QEC_OK;
  if (!d_syndromes || !d_data_bits || !d_raw_logical) return nfail(QEC_EINVAL, "null output buffer");

  Program init_prog, prog;
  if (!build_program(*params, false, init_prog, err) || !build_program(*params, true, prog, err))
    return nfail(QEC_EINVAL, err);
  const int D = prog.nd, nstab = prog.nstab, R = params->rounds, S = nstab * R;
  const int prec = params->precision;
  const size_t amp = is_f64(prec) ? 16 : 8;

  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return nfail(QEC_ECUDA, std::string("device query: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return nfail(QEC_EUNSUPPORTED, "device index too large");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {   // once per device, with that device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return nfail(QEC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  }

  const int nblk = S > nstab ? S : nstab;
  const int k1 = hist_k1(D), hgrid = hist_grid(D, sms);
  int pgrid = pass_grid(D, 2, sms);
  const int pg4 = pass_grid(D, 4, sms);
  if (pg4 > pgrid) pgrid = pg4;
  Carve c;
  const size_t o_psi = c.take(((size_t)1 << D) * amp), o_psi0 = c.take(((size_t)1 << D) * amp);
  const size_t o_psi2 = c.take(((size_t)1 << D) * amp);   // second working state (speculative passes)
  const size_t o_ops0 = c.take(sizeof(ProgOp) * (init_prog.ops.size() + 1));
  const size_t o_ops1 = c.take(sizeof(ProgOp) * (prog.ops.size() + 1));
  const size_t o_blk0 = c.take(sizeof(BlockInfo) * nstab), o_blk1 = c.take(sizeof(BlockInfo) * nstab);
  const size_t o_mat0 = c.take(sizeof(prog.mats)), o_mat1 = c.take(sizeof(prog.mats));
  const size_t o_kraus = c.take((size_t)nblk * KRAUS_STRIDE * amp);
  const size_t o_u = c.take(sizeof(double) * nblk), o_A = c.take(sizeof(double) * nblk);
  const size_t o_N = c.take(sizeof(double) * nblk), o_m = c.take(sizeof(int) * nblk);
  const size_t o_part = c.take(sizeof(double) * 2 * (pgrid > MAX_PASS_GRID ? pgrid : MAX_PASS_GRID));
  const size_t o_ctl = c.take(sizeof(Ctl));
  const size_t o_hp = c.take(sizeof(double) * ((size_t)hgrid << k1)), o_h = c.take(sizeof(double) << k1);
  if (c.off > kNoAllocBytes) return nfail(QEC_EINVAL, "request does not fit the 2 MiB static scratch");

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void* psi = base + o_psi;
  void* psi0 = base + o_psi0;
  void* psi2 = base + o_psi2;
  ProgOp* ops[2] = {reinterpret_cast<ProgOp*>(base + o_ops0), reinterpret_cast<ProgOp*>(base + o_ops1)};
  BlockInfo* blks[2] = {reinterpret_cast<BlockInfo*>(base + o_blk0), reinterpret_cast<BlockInfo*>(base + o_blk1)};
  double* mats[2] = {reinterpret_cast<double*>(base + o_mat0), reinterpret_cast<double*>(base + o_mat1)};
  const Program* progs[2] = {&init_prog, &prog};
  for (int i = 0; i < 2; ++i) {
    const Program& P = *progs[i];
    if (!P.ops.empty() && e == cudaSuccess)
      e = cudaMemcpyAsync(ops[i], P.ops.data(), sizeof(ProgOp) * P.ops.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(blks[i], P.blocks.data(), sizeof(BlockInfo) * nstab, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mats[i], P.mats, sizeof(P.mats), cudaMemcpyHostToDevice, st);
  }
  // The control word is the only scratch that must start from known values (the reduction
  // ticket at 0); everything else is written before it is read.
  Ctl h_ctl;
  std::memset(&h_ctl, 0, sizeof(h_ctl));
  h_ctl.seed = seed;
  h_ctl.first = first_traj;
  h_ctl.traj = first_traj;
  Ctl* ctl = reinterpret_cast<Ctl*>(base + o_ctl);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctl, &h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return nfail(QEC_ECUDA, std::string("scratch upload: ") + cudaGetErrorString(e));

  auto inst = [&](int which, int round_base, int nb, bool with_ctl) {
    const Program& P = *progs[which];
    InstArgs a;
    a.ops = ops[which];
    a.blocks = blks[which];
    a.mats = mats[which];
    for (int i = 0; i < PR_COUNT; ++i) a.prob[i] = P.prob[i];
    a.nstab = nstab;
    a.nd = D;
    a.round_base = round_base;
    a.nblk = nb;
    a.kraus = base + o_kraus;
    a.u = reinterpret_cast<double*>(base + o_u);
    a.ctl = with_ctl ? ctl : nullptr;
    a.events = nullptr;
    return a;
  };
  auto pass = [&](const Program& P, int blk, const void* src, bool forced, uint8_t* syn, int syn_idx) {
    const BlockInfo& bi = P.blocks[blk % nstab];
    PassArgs a;
    a.src = src;
    a.dst = psi;
    a.D = D;
    a.w = bi.w;
    for (int j = 0; j < 4; ++j) a.q[j] = bi.q[j] < 0 ? 0 : bi.q[j];
    a.kraus = base + o_kraus + (size_t)blk * KRAUS_STRIDE * amp;
    a.u = reinterpret_cast<double*>(base + o_u) + blk;
    a.forced = forced ? bi.offset : -1;
    a.A = reinterpret_cast<double*>(base + o_A) + blk;
    a.N = reinterpret_cast<double*>(base + o_N) + blk;
    a.m = reinterpret_cast<int*>(base + o_m) + blk;
    a.ctl = ctl;
    a.partials = reinterpret_cast<double*>(base + o_part);
    a.syn = syn;
    a.syn_stride = (R + 1) * nstab;
    a.syn_idx = syn_idx;
    a.offset = bi.offset;
    return a;
  };

  // The same launches, grids and kernel sequence as qec_create / qec_run_trajectories, so that the
  // reductions add in the same order and the results are identical: per block the speculative pass
  // and its corrective launch, alternating between two working states.  (At d <= 3 the tensor-core
  // passes do not apply: their tiles are larger than the register.)
  auto prob = [&](const PassArgs& a) { return launch_prob(prec, a, pass_grid_for(prec, true, D, a.w, sms), st); };
  auto apply = [&](const PassArgs& a) { return launch_apply(prec, a, pass_grid_for(prec, false, D, a.w, sms), st); };
  auto spec_out = [&](int b) { return (b & 1) ? psi2 : psi; };
  // Noise-free init round with outcomes forced to the zero syndrome (Sec. III.B), in psi0.
  e = launch_set_basis0(prec, psi0, D, st);
  if (e == cudaSuccess) e = launch_instantiate(prec, inst(0, 0, nstab, false), st);
  for (int k = 0; k < nstab && e == cudaSuccess; ++k) {
    PassArgs a = pass(init_prog, k, psi0, true, nullptr, 0);
    a.dst = psi0;
    e = prob(a);
    if (e == cudaSuccess) e = apply(a);
  }
  auto traj_pass = [&](int b) {
    const int rnd = 1 + b / nstab, k = b % nstab;
    return pass(prog, b, b == 0 ? psi0 : spec_out(b - 1), false, d_syndromes, rnd * nstab + k);
  };
  for (uint32_t t = 0; t < n && e == cudaSuccess; ++t) {
    if (S > 0) e = launch_instantiate(prec, inst(1, 1, S, true), st);
    for (int b = 0; b < S && e == cudaSuccess; ++b) {
      PassArgs a = traj_pass(b);
      a.src = b == 0 ? psi0 : spec_out(b - 1);
      a.dst = spec_out(b);
      a.spec_prev = b >= nstab ? a.syn_idx - nstab : -1;
      double* n_next = b + 1 < S ? reinterpret_cast<double*>(base + o_N) + b + 1 : nullptr;
      e = launch_spec(prec, a, n_next, b == 0, sms, st);
      if (e == cudaSuccess) e = launch_spec_fix(prec, a, n_next, b == 0, sms, st);
    }
    if (e != cudaSuccess) break;
    ReadArgs r;
    r.src = S > 0 ? spec_out(S - 1) : psi0;
    r.D = D;
    r.k1 = k1;
    r.d = params->d;
    r.rounds = R;
    r.grid_hist = hgrid;
    r.hist_part = reinterpret_cast<double*>(base + o_hp);
    r.hist = reinterpret_cast<double*>(base + o_h);
    r.ctl = ctl;
    r.bits = d_data_bits;
    r.logical = d_raw_logical;
    r.syn = d_syndromes;
    r.syn_stride = (R + 1) * nstab;
    r.nstab = nstab;
    e = launch_readout(prec, r, st);
  }
  if (e != cudaSuccess) return nfail(QEC_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return QEC_OK;
}

}  // namespace

extern "C" qec_status qec_run_trajectories_noalloc(const qec_params* params, uint64_t seed, uint64_t first_traj,
                                                   uint32_t n, uint8_t* d_syndromes, uint8_t* d_data_bits,
                                                   uint8_t* d_raw_logical, void* cuda_stream) {
  try {
    return run_noalloc(params, seed, first_traj, n, d_syndromes, d_data_bits, d_raw_logical, cuda_stream);
  } catch (...) {   // a host allocation of the circuit program failed: nothing crosses the C ABI
    return nfail(QEC_ENOMEM, "exception in qec_run_trajectories_noalloc");
  }
}
