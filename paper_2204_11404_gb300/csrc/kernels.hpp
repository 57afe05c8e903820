// Launch interface of the trajectory kernels (kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "program.hpp"

namespace qec {

// Device control block of one simulator.
struct Ctl {
  unsigned long long seed;
  unsigned long long first;     // first trajectory index of the current call
  unsigned long long traj;      // trajectory being simulated (advanced by the readout)
  unsigned int ticket;          // last-CTA ticket of the reductions (always returned to 0)
  unsigned int n_events;
  unsigned int ev_cap;
  unsigned int prob_uncertain;  // the bounded probability pass left the outcome undecided
  double final_norm;            // sum |psi|^2 of the state the readout sampled
  unsigned int status;          // bit 0: a bounded device wait gave up (results invalid)
  unsigned int prob_force_exact;        // test hook: the bounded pass never decides
  unsigned long long prob_fallbacks;    // exact probability passes run after an undecided one
  unsigned int tile_next;       // tile counter of the tensor-core complex128 apply pass (returned to 0)
  unsigned int tile_done;       // CTAs of such a pass that have finished (returned to 0)
  unsigned long long spec_misses;       // corrective applies after a speculative pass guessed wrong
};

constexpr int KRAUS_STRIDE = 768;

// complex128 storage (QEC_C128, QEC_C128_TC) vs complex64.
inline bool is_f64(int precision) { return precision == QEC_C128 || precision == QEC_C128_TC; }   // per block: K0, K1, M = K1^dagger K1, 16x16 each
constexpr int MAX_PASS_GRID = 2048;

struct InstArgs {
  const ProgOp* ops;
  const BlockInfo* blocks;
  const double* mats;     // [M_COUNT][16][2]
  double prob[PR_COUNT];
  int nstab, nd;
  int round_base;         // round of block 0 of this launch
  int nblk;               // blocks in this launch (nstab x rounds)
  void* kraus;            // [nblk][KRAUS_STRIDE] complex (T2)
  double* u;              // [nblk] measurement uniforms
  Ctl* ctl;               // seed / trajectory source; nullptr = trajectory 0, seed 0 (init round)
  int32_t* events;        // [ev_cap][5] (traj, round, step, site, code) or nullptr
};

struct PassArgs {
  const void* src;
  void* dst;
  int D;                  // data-register qubits (2^D amplitudes)
  int w;                  // 2 or 4
  int q[4];               // data bits of the block, ascending
  const void* kraus;      // this block's KRAUS_STRIDE entries
  const double* u;        // this block's measurement uniform
  int forced;             // -1: sample; else forced raw outcome
  double* A;              // this block's <psi|K1^dag K1|psi>
  double* N;              // this block's <psi|psi>
  int* m;                 // this block's raw outcome
  Ctl* ctl;
  double* partials;       // [MAX_PASS_GRID][2]
  uint8_t* syn;           // syndrome output (nullptr = none)
  int syn_stride;         // bytes per trajectory
  int syn_idx;            // round * nstab + stab
  int offset;             // syndrome = raw ^ offset
  int store_n = 1;        // 0: the pass leaves *N as it is (the exact pass after a fused tensor-core
                          // complex128 pass, whose norm estimate renormalises the state)
  int spec_prev = -1;     // speculative pass: syndrome index of the same stabilizer one round
                          // earlier, whose raw outcome is the guess; -1: the init round's (offset)
};

// Fused pass: apply block s (ap) and accumulate the probability of block s+1 (pr) on tiles
// of amplitudes staged in shared memory, one HBM read + one write per stabilizer.
// Tile index bits: [0, lb) = register bits [0, lb); [lb, nt) = register bits hbits[0..nt-lb).
struct FusedArgs {
  PassArgs ap;
  PassArgs pr;
  int nt, lb;
  int hbits[16];
  int nout;
  int obits[32];          // register bits outside the tile, ascending
  int qa[4];              // apply block's qubits as tile-index bits (ascending; the tensor-core
                          // complex128 passes: a weight-2 block's two qubits, then two spectators)
  int qp[4];              // probability block's qubits as tile-index bits (ascending; the
                          // tensor-core complex128 passes: qa sorted)
  int qa_s[4], qp_s[4];   // fused tensor-core complex128 pass: qa and qp (each with its own
                          // spectators) sorted ascending, for the group base addresses
  int skip_unless_uncertain;   // exact tensor-core probability pass: run only if ctl->prob_uncertain
  int grid;
  double* n_next = nullptr;    // speculative pass: receives |output|^2, the next block's *N (or null)
  int spec_unit = 0;           // speculative pass: the input's scale is 1 (block 0, the init state)
};

struct ReadArgs {
  const void* src;
  int D, k1, d;
  int rounds;
  int grid_hist;
  double* hist_part;      // [grid_hist][2^k1]
  double* hist;           // [2^k1]
  Ctl* ctl;
  uint8_t* bits;          // [traj][D] (one bit per data qubit)
  uint8_t* logical;       // [traj]
  uint8_t* syn;           // [traj][syn_stride]; round-0 row zeroed here
  int syn_stride;
  int nstab;
};

cudaError_t launch_instantiate(int precision, const InstArgs& a, cudaStream_t s);
cudaError_t launch_prob(int precision, const PassArgs& a, int grid, cudaStream_t s);
cudaError_t launch_apply(int precision, const PassArgs& a, int grid, cudaStream_t s);
cudaError_t launch_readout(int precision, const ReadArgs& a, cudaStream_t s);
// Builds the tile for (apply block ap, probability block pr) and launches the fused pass.
cudaError_t launch_fused(int precision, const PassArgs& ap, const PassArgs& pr, int num_sms, cudaStream_t s);
cudaError_t launch_set_basis0(int precision, void* psi, int D, cudaStream_t s);
cudaError_t setup_kernels(int precision, int D);
cudaError_t launch_wait_selftest(unsigned int* status, long limit, cudaStream_t s);
// complex128 apply / probability passes on the tensor cores (weight-4 blocks, tiles of 2^11
// amplitudes: registers of at least 11 qubits).
bool apply_oz_applies(const PassArgs& ap);
cudaError_t launch_apply_oz(const PassArgs& ap, int num_sms, cudaStream_t s);
cudaError_t launch_prob_oz(const PassArgs& ap, int num_sms, cudaStream_t s);   // once per process/device, before any capture
// Fused tensor-core complex128 pass: apply block `ap`, then block `pr`'s bounded probability on the
// same tiles, then the exact probability launch that runs only if the bound left the outcome open.
// Both blocks' qubits must fit one 2^11-amplitude tile (fused_oz_applies).
bool fused_oz_applies(const PassArgs& ap, const PassArgs& pr);
cudaError_t launch_fused_oz(const PassArgs& ap, const PassArgs& pr, int num_sms, cudaStream_t s);
// The exact probability launch of block pr after a fused pass (returns at once unless needed).
cudaError_t launch_prob_oz_check(const PassArgs& pr, int num_sms, cudaStream_t s);
// Speculative complex128 pass of block ap (ap.src and ap.dst distinct buffers): applies K_g / sqrt(*ap.N)
// (scale 1 with unit_in) for the guessed outcome g, decides the outcome (on the tensor cores where
// its bound allows), and stores |output|^2 in *n_next (n_next may be null).  QEC_C128_TC blocks whose
// tile fits (apply_oz_applies) run on the tensor cores, every other complex128 block on the FP64
// CUDA cores; QEC_C64_TC weight-4 blocks whose tile has 2^12 amplitudes on the tensor cores (3xTF32),
// every other complex64 block on the FP32 CUDA cores (shared-memory tiles).
cudaError_t launch_spec(int precision, const PassArgs& ap, double* n_next, bool unit_in, int num_sms, cudaStream_t s);
// Its completion: on the tensor cores the exact probability launch (returns at once unless the bound
// left the outcome open); then the corrective apply (returns at once unless the outcome is not g).
cudaError_t launch_spec_fix(int precision, const PassArgs& ap, double* n_next, bool unit_in, int num_sms,
                            cudaStream_t s);
int pass_grid(int D, int w, int num_sms);
// One wave of resident CTAs for the probability (prob = true) or apply pass kernel.
int pass_grid_for(int precision, bool prob, int D, int w, int num_sms);
int hist_k1(int D);
int hist_grid(int D, int num_sms);

// Sets the thread-local message returned by qec_last_error().
void set_last_error(const std::string& msg);

// Host version of the per-block instantiation (same arithmetic as the device kernel).
void instantiate_block_host(const InstArgs& a, int blk, uint64_t seed, uint64_t traj,
                            double2* k0, double2* k1, double* u);

}  // namespace qec
