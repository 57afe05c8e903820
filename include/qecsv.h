/*
 * qecsv: GB300 state-vector trajectories of the rotated surface code under
 * Pauli + coherent noise (Katsuda, Mitarai, Fujii, arXiv:2204.11404).
 *
 * C ABI.  No C++ types cross it; nothing throws across it.  Every call returns
 * a qec_status; on a non-OK status, qec_last_error() gives a thread-local
 * message and the caller's output buffers hold unspecified contents.
 * A qec_sim handle is not thread-safe: use one handle per host thread.
 */
#ifndef QECSV_H
#define QECSV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QEC_OK = 0,
  QEC_EINVAL = -1,       /* bad argument: size, pointer, enum or parameter range */
  QEC_ENOMEM = -2,       /* device or host allocation failed */
  QEC_ECUDA = -3,        /* a CUDA runtime call failed (message has the CUDA error string) */
  QEC_ETIMEOUT = -4,     /* a bounded device wait gave up */
  QEC_EUNSUPPORTED = -6  /* valid request the library does not implement (e.g. unreduced layout in a qec_sim) */
} qec_status;

/* Register layout (Sec. II.B).  REDUCED: d^2 data qubits + one reused ancilla
 * (26 qubits at d=5); UNREDUCED: all 2d^2-1 qubits (only the oracle runs it). */
typedef enum { QEC_LAYOUT_REDUCED = 0, QEC_LAYOUT_UNREDUCED = 1 } qec_layout;
/* The code whose memory experiment runs.  SURFACE: the rotated surface code (Sec. II.A,
 * Table I), d^2 data qubits, d^2 - 1 stabilizers.  REPETITION: the one-dimensional bit-flip
 * repetition code of Sec. II.B, Fig. 2 (the paper's illustration of the delayed register), d
 * data qubits on a line, d - 1 stabilizers Z_k Z_{k+1} measured in the Z part of the round
 * (steps 7-11) with gate order q_{k+1}, q_k; the X part of its round is idle. */
typedef enum { QEC_CODE_SURFACE = 0, QEC_CODE_REPETITION = 1 } qec_code;

/* Gate set.  CNOT: H + CNOT stabilizer circuits (Fig. 1b/c).  CR: the
 * cross-resonance native set {Rx(pi/2), Rx^dagger(pi/2), Rzx(pi/2), Rz(pi/2)}
 * with data corrections after each part (Sec. III.A, Fig. 4). */
typedef enum { QEC_GATES_CNOT = 0, QEC_GATES_CR = 1 } qec_gateset;

/* Amplitude storage / arithmetic.  C128: complex128 state, FP64 arithmetic, one
 * speculative pass per block as described under C128_TC, with FP64 sums that
 * decide every outcome directly.
 * C64: complex64 state, FP32 gate arithmetic, FP64 probability reductions;
 * one speculative pass per block as described under C128_TC (FP32 sums per
 * tile, FP64 across tiles, deciding every outcome directly).
 * C64_TC: complex64 state; the speculative pass of every weight-4 block on the
 * tensor cores (3xTF32 split, FP32 accumulation; tiles of 2^12 amplitudes, so
 * d >= 5), of the weight-2 blocks as C64; FP64 reductions across tiles.  With
 * the speculative passes off, the fused apply + next-probability pass of every
 * pair of blocks with a weight-4 block on the tensor cores (a weight-2 block of
 * the pair as K (x) I over two spectator qubits), pairs of weight-2 blocks on
 * the CUDA cores.
 * C128_TC: complex128 state; the apply of every stabilizer block (tiles of
 * 2^11 amplitudes, so registers of at least 11 qubits: the d = 5 surface code
 * and the repetition code from d = 11; smaller registers as C128) as emulated
 * FP64 products on the FP16 tensor cores: each operand row split into 7
 * signed 8-bit slices under one exponent, slice products accumulated exactly,
 * recombined in integers and rounded once (Ozaki scheme).  One speculative
 * pass per block (qec_debug_speculation): it applies the Kraus operator of the
 * outcome the same stabilizer gave one round earlier (the init round's for the
 * first noisy round) into a second working state, and on the same tiles sums
 * |input|^2 and |output|^2 as 24-bit truncations with rigorous error bounds;
 * the outcome is decided from them where the bounds settle it, else by the
 * exact pass on the untouched input (qec_debug_exact_probability), and a wrong
 * guess is re-applied from that input.  Init and readout in FP64.  Same
 * outcomes and, to within a few FP64 roundings, the same amplitudes as C128. */
typedef enum { QEC_C128 = 0, QEC_C64 = 1, QEC_C64_TC = 2, QEC_C128_TC = 3 } qec_precision;

/* Noise (Sec. III.A).  Probabilities in [0, 1]; angles in radians, |angle| <= 4. */
typedef struct {
  double p1;        /* Eq. 1 after every one-qubit gate */
  double p2;        /* Eq. 2 (15 non-identity pairs, uniform) after every two-qubit gate */
  double p_idle;    /* Eq. 1 on a qubit that waits during a step */
  double theta_rx;  /* extra R_X(theta) = exp(-i theta X/2) after every Rx / Rx^dagger */
  double theta_rz;  /* extra R_Z(theta) after every Rz */
  double theta_rzx; /* extra exp(-i theta Z(x)X/2) after every Rzx */
  double phi_zz;    /* ZZ crosstalk exp(-i phi Z(x)Z) after every two-qubit gate */
  double round_rz;  /* R_Z(angle) on every data qubit at the start of each noisy round */
  double round_rx;  /* R_X(angle) on every data qubit at the start of each noisy round */
  double twirl;     /* 0: coherent terms as unitaries; 1: each replaced by its Pauli twirl, the
                       generator Pauli A with probability sin^2(theta/2) (ZZ: sin^2(phi)) (Sec. III.A) */
  double overrot_follows; /* 0: the extra rotation has the same sign after every gate (Sec. III.A
                       read literally); 1: after Rx^dagger(pi/2), the X-ancilla preparation and the
                       schedule's only negative-angle rotation, it is R_X(-theta_rx) (the angle's
                       magnitude grows).  Must be 0 or 1. */
} qec_noise;

typedef struct {
  int32_t d;          /* code distance: odd; surface code 3 <= d <= 5 (2^(d^2) amplitudes resident),
                         repetition code 9 <= d <= 25 (2^d) */
  int32_t rounds;     /* noisy syndrome rounds after the noise-free init round, 0..64 */
  int32_t layout;     /* qec_layout; only QEC_LAYOUT_REDUCED runs on the GPU */
  int32_t gates;      /* qec_gateset */
  int32_t precision;  /* qec_precision */
  int32_t code;       /* qec_code */
  qec_noise noise;
} qec_params;

typedef struct qec_sim qec_sim;

/*
 * Create a simulator (Sec. III.B protocol): allocates the state vectors on
 * the current CUDA device, builds the per-round circuit program, and runs the
 * noise-free init round whose outcomes are forced to the zero syndrome; the
 * resulting code state stays resident and seeds every trajectory.
 * cuda_stream: a cudaStream_t owned by the caller (e.g. torch's current
 * stream) that every run is ordered after and before (through events), or
 * NULL.  Kernels run on a stream owned by the sim, created with the caller
 * stream's priority.
 * *out receives the handle; the sim owns all device memory it allocates.
 */
qec_status qec_create(const qec_params* params, void* cuda_stream, qec_sim** out);

/*
 * Run trajectories first_traj .. first_traj+n-1 (Sec. III.B: init state, then
 * `rounds` noisy rounds of the X part and Z part, then a Z measurement of every
 * data qubit in index order).  Results are a pure function of (params, seed,
 * trajectory index): noise and measurement draws come from Philox4x64-10 with
 * key (seed, 0) and counter (trajectory, round, step<<32 | physical site, tag).
 * Outputs are caller-owned HOST buffers (may be NULL to skip):
 *   syndromes  [n][rounds+1][S]  uint8: row 0 is the forced init round (all 0);
 *              S = d*d-1 stabilizers in Table I order, X then Z (surface
 *              code), or S = d-1 in line order (repetition code)
 *   data_bits  [n][Q]            uint8: final Z outcome of each data qubit,
 *              Q = d*d (surface) or d (repetition)
 *   raw_logical[n]               uint8: parity of data_bits over data qubits
 *              0..d-1 (logical Z: the first row of the surface code, the whole
 *              line of the repetition code), before any decoding
 * Blocks until the results are on the host.
 */
qec_status qec_run_trajectories(qec_sim* sim, uint64_t seed, uint64_t first_traj, uint32_t n,
                                uint8_t* syndromes, uint8_t* data_bits, uint8_t* raw_logical);

/*
 * Same as qec_run_trajectories, but the outputs are DEVICE buffers of the
 * same shapes (on the sim's device), filled asynchronously on the sim's
 * stream; nothing is copied to the host and the call does not synchronize.
 */
qec_status qec_run_trajectories_device(qec_sim* sim, uint64_t seed, uint64_t first_traj, uint32_t n,
                                       uint8_t* d_syndromes, uint8_t* d_data_bits, uint8_t* d_raw_logical);

/*
 * Re-point an existing simulator at new noise parameters and round count,
 * keeping its device buffers and its resident init code state (which does not
 * depend on noise or rounds).  d, gate set, precision, layout and code must
 * match the handle's (QEC_EINVAL otherwise).  Waits for the handle's queued work.
 */
qec_status qec_reconfigure(qec_sim* sim, const qec_params* params);

/* Number of amplitudes of the resident data register (2^Q, Q data qubits); the
 * reused ancilla is |0> at every point a snapshot can be taken. */
uint64_t qec_state_len(const qec_sim* sim);

/*
 * Test hook: copy the normalised data-register state after the last noisy
 * round of the most recent trajectory (before the final readout, which does
 * not modify it) into host_buf as complex128 (re, im) pairs, whatever the
 * precision.  bytes must be >= 16 * qec_state_len(sim).
 */
qec_status qec_get_state(qec_sim* sim, void* host_buf, size_t bytes);

/*
 * Test hook: enable (max_events > 0) or disable recording of the Pauli errors
 * sampled on the device (Eqs. 1-2).  qec_get_events copies the events of the
 * most recent trajectory as int32 quadruples (round, step, physical site,
 * code) in unspecified order; code = Pauli 1..3 (X, Y, Z) for Eq. 1 sites and
 * 4*ancilla_pauli + data_pauli for Eq. 2 sites.  *count gets the number
 * recorded (capped at max_events).
 */
qec_status qec_record_events(qec_sim* sim, uint32_t max_events);
qec_status qec_get_events(qec_sim* sim, int32_t* host_events, uint32_t max_events, uint32_t* count);

/*
 * Measurement hook: device time in milliseconds of the probability pass
 * (ms[0]) and of the collapse/apply pass (ms[1]) of one weight-4 stabilizer
 * block of the middle noisy round, in the most recent trajectory (CUDA events
 * recorded inside the trajectory's graph).  With the fused passes ms[0] is
 * empty for a block whose probability the previous pass computed; with the
 * speculative passes (the complex128 forms) ms[0] is empty and ms[1] is the
 * block's speculative pass, without the launches that complete it.  *block gets that block's index
 * (round-major, d^2-1 per round).  QEC_EINVAL if no trajectory ran yet or the
 * sim has no noisy round.
 */
qec_status qec_kernel_times(qec_sim* sim, float* ms, int32_t* block);

/*
 * Measurement hook: instrument, from the next trajectory on, the first block
 * of the middle noisy round whose weight is w_apply and whose successor's
 * weight is w_next (2 or 4; ms[1] of qec_kernel_times is then that block's
 * speculative pass, or with the fused passes the pass that applies that block
 * and computes its successor's probability).  *block gets its index.  QEC_EINVAL if the sim has no noisy
 * round or no such pair of blocks.  The trajectory graph is rebuilt at the
 * next run; results do not change.
 */
qec_status qec_select_timed_block(qec_sim* sim, int32_t w_apply, int32_t w_next, int32_t* block);

/*
 * Self-test of failure detection: runs, on the sim's stream, the bounded
 * mbarrier wait used by the tensor-core pass on a barrier that nothing ever
 * arrives on, giving up after `polls` polls (1..1e7).  Returns QEC_ETIMEOUT
 * when the wait ran out and was reported through the device status word
 * (the expected result); the sim stays usable afterwards.
 */
qec_status qec_selftest_wait(qec_sim* sim, uint32_t polls);

/*
 * Trajectories without any device allocation (the paper has no counterpart;
 * this is a deployment variant of qec_run_trajectories_device).
 * For callers that cannot call cudaMalloc: code whose framework owns all
 * device memory through its own pool or arena, code on a latency-critical
 * path where cudaMalloc's implicit device synchronisation is not acceptable,
 * or plug-ins handed only a stream and output buffers.  The caller passes the
 * parameters, the trajectory range and DEVICE output buffers with the shapes
 * of qec_run_trajectories (all three required when n > 0); results are
 * identical to qec_run_trajectories for the same parameters, seed and
 * trajectory indices: it launches the same kernels with the same grids in the
 * same order (per block the speculative pass and its corrective launch, over
 * two working states), so every reduction adds in the same order.  Work
 * is enqueued asynchronously on cuda_stream (NULL = the legacy default
 * stream); no sim handle is involved.  At the sizes it accepts none of its
 * kernels waits on a barrier or flag, so it has no bounded-wait timeout to
 * report.
 * All device working memory (program, state vectors, Kraus blocks, reduction
 * and readout scratch) is one static 2 MiB device array inside the library,
 * which every GPU that loads the library holds until the process exits.  It
 * fits d = 3 with at most 16 noisy rounds; larger requests return QEC_EINVAL.
 * The first call on a device looks up that array's device address (once per
 * device, with the device current).  Every call reuses the same array and
 * resets what must start from zero, so calls that overlap on the GPU
 * (different streams, or concurrent host threads) race and corrupt each
 * other: serialise them.
 */
qec_status qec_run_trajectories_noalloc(const qec_params* params, uint64_t seed, uint64_t first_traj, uint32_t n,
                                        uint8_t* d_syndromes, uint8_t* d_data_bits, uint8_t* d_raw_logical,
                                        void* cuda_stream);

/* ---- Batched form: many small-register trajectories in one persistent launch ----------- */
typedef struct qec_batch qec_batch;

/*
 * Batched simulator for the d = 3 delayed-measurement register (9 data qubits
 * + reused ancilla, Sec. II.B), `rounds` noisy rounds, gate set `gates`.
 * One warp runs one trajectory in shared memory; a single graph-captured
 * persistent kernel processes a whole batch, taking trajectories from a
 * device work counter.  max_traj bounds n of every run.  Only d = 3 is
 * accepted (QEC_EUNSUPPORTED otherwise).  cuda_stream as in qec_create.
 */
qec_status qec_batch_create(int32_t d, int32_t rounds, int32_t gates, uint32_t max_traj, void* cuda_stream,
                            qec_batch** out);

/*
 * Run n trajectories (Sec. III.B protocol, as qec_run_trajectories), each with
 * its own trajectory index traj[i], kind[i] = precision (QEC_C128 or QEC_C64)
 * + 2 * layout, and noise parameters noise[i] (Sec. III.A).  Layout
 * QEC_LAYOUT_REDUCED runs the 10-qubit delayed register (one warp, Sec. II.B);
 * QEC_LAYOUT_UNREDUCED runs all 17 qubits time-ordered, every ancilla of a part
 * active at once (one CTA; the other part's ancillas are |0>, so a
 * 2^13-amplitude slab holds the exact state).  Inputs and outputs are HOST
 * arrays: syndromes [n][rounds+1][8], data_bits [n][9], raw_logical [n] (any
 * output may be NULL).  Trajectory i equals qec_run_trajectories for
 * (noise[i], kind[i], seed, traj[i]).  Blocks until the outputs are on the host.
 */
qec_status qec_batch_run(qec_batch* b, uint64_t seed, uint32_t n, const uint64_t* traj, const int32_t* kind,
                         const qec_noise* noise, uint8_t* syndromes, uint8_t* data_bits, uint8_t* raw_logical);

/*
 * Autotuner: times qec_batch_run on the given sample and keeps the fastest
 * configuration of each engine, each timed on the sample's trajectories of its
 * register: the reduced-register engine's CTA shape (warps per CTA, one
 * resident wave per SM), then the unreduced engine's fusion width k (2..6 slab
 * bits per pass: consecutive gate units on disjoint bits, which commute, are
 * applied in one pass over the 2^13-amplitude slab) and threads per CTA (128,
 * 256).  *chosen_warps gets the reduced engine's warps per CTA, *best_ms the
 * device time of the whole sample with the chosen configuration;
 * qec_batch_config reports all three choices.
 */
qec_status qec_batch_autotune(qec_batch* b, uint64_t seed, uint32_t n, const uint64_t* traj, const int32_t* kind,
                              const qec_noise* noise, int32_t* chosen_warps, float* best_ms);

/* The current configuration: reduced engine warps per CTA, unreduced engine fusion width and
 * threads per CTA. */
qec_status qec_batch_config(const qec_batch* b, int32_t* warps_per_cta, int32_t* fusion_width, int32_t* u_threads);

/* Sets the configuration by hand (QEC_EINVAL outside warps 2..10 that fit, fusion width 2..6,
 * threads 128/256; QEC_EUNSUPPORTED when a shape does not fit an SM).  Results do not depend on it. */
qec_status qec_batch_set_config(qec_batch* b, int32_t warps_per_cta, int32_t fusion_width, int32_t u_threads);

/*
 * Test hook: choose one trajectory of the next qec_batch_run (item = its index i in that call's
 * arrays, 0 <= i < n; -1 = none) whose data-register state after its last noisy round is
 * recorded on the device, so that its amplitudes can be compared with another simulation of
 * the same trajectory (Sec. II.B: the reduced and the unreduced register hold the same data
 * state).  QEC_EINVAL on a null handle or item < -1.
 */
qec_status qec_batch_snapshot(qec_batch* b, int64_t item);

/*
 * Copy the state recorded by the last qec_batch_run that had a snapshot item: the 2^9
 * amplitudes of the nine data qubits (every ancilla is |0> after the round), normalised, as
 * complex128 (re, im) pairs whatever the trajectory's precision.  bytes must be >= 16 * 512.
 * QEC_EINVAL if no such run has completed, or the item was not below that run's n.
 */
qec_status qec_batch_get_state(qec_batch* b, void* host_buf, size_t bytes);

/* Device time (ms, CUDA events around the persistent launch) of the last qec_batch_run. */
qec_status qec_batch_last_ms(const qec_batch* b, float* ms);
qec_status qec_batch_destroy(qec_batch* b);

qec_status qec_destroy(qec_sim* sim);
const char* qec_last_error(void);

/*
 * Host-only test hook (no GPU needed): the static per-round circuit program
 * that the device instantiates, for checking the schedule on the CPU.
 * Writes up to `cap` int32 sextuples per op (block, kind, local q0, local q1,
 * step, site) in block order and returns the op count in *n_ops; block
 * metadata goes to block_info as int32 sextuples (w, q0, q1, q2, q3, offset).
 */
qec_status qec_debug_program(const qec_params* params, int32_t* ops, uint32_t cap, uint32_t* n_ops,
                             int32_t* block_info, uint32_t block_cap, uint32_t* n_blocks);

/*
 * Host-only test hook (no GPU needed): the batched form's plan for one round
 * of the unreduced 17-qubit register (d = 3, gate set `gates`, every noise
 * site present), at fusion width k.  items: int32 quadruples (kind 0 = unit /
 * 1 = measurement, qubits 1 or 2, slab bit qa, slab bit qb or -1) in
 * execution order, *n_items of them.  pass_units: the unit items the passes
 * apply, in order (*n_pass_units).  absorbs: int32 triples (one-qubit item,
 * two-qubit item it is folded into, mode: bit 0 = from the left (after),
 * bit 1 = on the unit's first qubit), *n_absorbs of them.  All arrays hold up
 * to `cap` entries; QEC_EINVAL if that is too small.
 */
qec_status qec_debug_unreduced_plan(int32_t gates, int32_t k, int32_t* items, uint32_t cap, uint32_t* n_items,
                                    int32_t* pass_units, uint32_t* n_pass_units, int32_t* absorbs,
                                    uint32_t* n_absorbs);

/*
 * Host-only test hook (no GPU needed): runs the same block-instantiation code
 * the device runs, on the CPU, for trajectory `traj` of round `round` (0 = the
 * forced init round).  For each of the d^2-1 blocks writes K0 and K1 (16x16
 * complex128, row-major, (re, im) pairs; rows/cols beyond 2^w are zero) to
 * kraus[block][2][16][16][2] and the measurement uniform to u[block].
 */
qec_status qec_debug_blocks(const qec_params* params, uint64_t seed, uint64_t traj, int32_t round,
                            double* kraus, double* u);

/*
 * Host-only test hook (no GPU needed): the FP64-exact emulated product that the tensor-core
 * complex128 pass computes, run on the CPU with the same slicing and recombination code.
 * out[m][32] = A[m][32] . B[32][32]^T (row-major FP64); each entry is the dot product of
 * the 56-bit truncated inputs (truncation relative to each row's largest exponent) with
 * slice products of weight below 2^-56 dropped, rounded once to FP64: absolute error at
 * most 2^-44 * max|A[r]| * max|B[n]| + 2^-53 * |exact|.  variant 0: recombination in
 * integers with rounding to nearest, ties away (the probability pass); 1: through one
 * int64 -> FP64 conversion, ties to even (the apply pass); 2: the probability pass's sums,
 * with one exponent for all of B: out[r][0] = sum_n (A[r] . B[n])^2, out[r][1] =
 * sum_k A[r][k]^2 (each half-row's squares summed in integers, converted once), the rest
 * untouched; 3: the bounded probability pass: out[r][0] = sum_n y^_n^2 from the top 3
 * slices of each operand, out[r][1] = its error bound (|sum_n (A[r] . B[n])^2 - out[r][0]|
 * <= out[r][1]); 4: the fused tensor-core pass's probability, A taken as one tile (one exponent for
 * all of A and one for all of B), 24-bit truncations, 3 slices each, diagonals 0..2:
 * out[r][0] = estimate of sum_n (A[r] . B[n])^2, out[r][1] its error bound, out[r][2] = estimate
 * of sum_k A[r][k]^2, out[r][3] its error bound; 5: the speculative pass's sums of squares of A's
 * reals (B unused): out[r][0] = estimate of sum_k A[r][k]^2 from each real's top 24 bits under
 * the row's largest exponent, out[r][1] its error bound, out[r][2] = the same sum from the top 24
 * bits under the largest exponent of all of A, out[r][3] its error bound.  Returns QEC_EINVAL for
 * any other variant.  The paper has no counterpart
 * (an arithmetic form of the gate application of Sec. III).  Returns QEC_EINVAL on null
 * pointers or m <= 0.
 */
qec_status qec_debug_ozaki_gemm(const double* A, const double* B, int32_t m, int32_t variant, double* out);

/*
 * Test hook for QEC_C128_TC (the paper has no counterpart: an evaluation order of Sec. II.B's
 * measurement probability).  Each outcome is first decided from estimates with a rigorous
 * error bound: A = |K_1 psi|^2 and N = |psi|^2 from the speculative pass's sums (see
 * qec_debug_speculation), or A from the top 3 of the 7 slices of each operand in the fused pass;
 * the device decides when |u N - A| exceeds twice the bound plus 1e-10 (A + N), where the exact
 * pass must decide the same way, and otherwise runs the exact pass.  force = 1: every outcome goes through the exact pass; 0: the default; -1: unchanged.
 * *fallbacks (may be NULL) receives the number of exact passes run on this handle so far.
 * Waits for the handle's queued work.  QEC_EINVAL on a null handle or force outside -1..1.
 */
qec_status qec_debug_exact_probability(qec_sim* sim, int32_t force, uint64_t* fallbacks);

/*
 * Test hook (the paper has no counterpart: an evaluation order of Sec. II.B's measurement and
 * collapse).  enable = 1: the speculative passes (the default); 0: the passes that compute each
 * probability before its apply (QEC_C128: a probability pass and an apply pass per block;
 * QEC_C128_TC: per block pair, the apply fused with the next block's 3-slice bounded
 * probability; the complex64 forms: the apply fused with the next block's probability);
 * -1: unchanged.  Both give the same outcomes (except within the rounding of a threshold) and
 * states within a few roundings of the form's arithmetic.  *misses (may be NULL) receives the
 * number of corrective applies run on this handle so far (outcomes that differed from the
 * guess).  Waits for the handle's queued work; switching rebuilds the trajectory graph and
 * requires a new run before qec_get_state.  QEC_EINVAL on a null handle or enable outside
 * -1..1.
 */
qec_status qec_debug_speculation(qec_sim* sim, int32_t enable, uint64_t* misses);

#ifdef __cplusplus
}
#endif
#endif
