// Static per-round circuit program of the delayed-measurement register.
//
// One round of syndrome extraction (X part, steps 1-6, then Z part, steps
// 7-11; Sec. II.A, Sec. III.A/D) becomes d^2-1 blocks, one per stabilizer in
// serial order (Table I order, X then Z; Sec. II.B).  A block holds every op
// on its ancilla and on its <= 4 data qubits that falls between those data
// qubits' neighbouring gates, so the delayed, one-ancilla order reproduces
// each qubit's own time order.  Noise sites are placeholders here; the device
// draws them per trajectory and fuses each block into two Kraus matrices.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qecsv.h"

namespace qec {

// OP_T1 / OP_T2: a twirled coherent term: the Pauli (product) `mat` with probability prob[pidx]
// (site field = factor << 24 | physical site, drawn with its own stream tag).
enum OpKind : uint8_t { OP_U1 = 0, OP_U2 = 1, OP_N1 = 2, OP_N2 = 3, OP_T1 = 4, OP_T2 = 5 };
enum ProbId : uint8_t {
  PR_P1 = 0, PR_P2 = 1, PR_IDLE = 2,
  PR_TW_RX = 3, PR_TW_RZ = 4, PR_TW_RZX = 5, PR_TW_ZZ = 6, PR_TW_ROUND_RZ = 7, PR_TW_ROUND_RX = 8,
  PR_COUNT = 9
};

// Local qubits of a block: data j = 0..w-1 (ascending global bit), ancilla = w.
struct ProgOp {
  uint8_t kind;   // OpKind
  uint8_t q0;     // U1/N1: qubit; U2: first-listed (control side); N2: ancilla
  uint8_t q1;     // U2: second-listed (target side); N2: data qubit
  uint8_t pidx;   // N1/N2: ProbId
  uint16_t mat;   // U1/U2: matrix id
  uint16_t step;  // N1/N2: circuit step 1..11 (0 = round start)
  uint32_t site;  // N1/N2: physical site (data 0..d^2-1, ancilla of stabilizer k: d^2+k)
};

struct BlockInfo {
  int32_t op_begin, op_end;
  int32_t w;        // number of data qubits (2 or 4)
  int32_t q[4];     // global data bits, ascending; unused entries -1
  int32_t offset;   // syndrome bit = raw ancilla bit ^ offset
  int32_t stab;     // stabilizer index in serial order
};

enum MatId : uint16_t {
  M_I = 0, M_X, M_Y, M_Z, M_H, M_RX90, M_RX90DG, M_RZ90, M_CNOT, M_RZX90,
  M_ROT_RX, M_ROT_RZ, M_ROT_RZX, M_ZZ, M_ROUND_RZ, M_ROUND_RX, M_PZX, M_PZZ, M_ROT_RXP, M_COUNT
};

struct Program {
  int d = 0, nd = 0, nstab = 0;
  std::vector<ProgOp> ops;
  std::vector<BlockInfo> blocks;    // nstab blocks, serial order
  double mats[M_COUNT][16][2];      // 4x4 complex row-major; one-qubit gates in the top-left 2x2
  double prob[PR_COUNT];            // p1, p2, p_idle, twirl probabilities (0 in the init program)
};

struct Stab {
  char kind;        // 'X' or 'Z'
  int slots[4];     // data qubit per gate slot in gate order, -1 = wait
  int w;
};

// Time-ordered program of the unreduced register (all 2d^2-1 qubits, Sec. II.B), on a slab of
// d^2 + (d^2-1)/2 qubits: data q -> bit q; the active part's ancilla j -> bit d^2 + j.  The four (at
// d=3) ancillas of the part not in progress are |0> (reset after their measurement, untouched
// until their part starts), so the slab holds the exact 2d^2-1 qubit state.  A round is a list of
// items in execution order: fused units (one qubit, or one two-qubit gate pair, at one step; their
// ops in order gate, coherent terms, Pauli) and ancilla measurements (after steps 6 and 11).
struct UItem {
  int32_t kind;           // 0: unit, 1: measurement
  int32_t op_begin, op_end;   // unit ops (ProgOp, q0/q1 = slab bits)
  int32_t nq;             // unit: 1 or 2 qubits
  int32_t qa, qb;         // unit: slab bits (qa = first-listed); measurement: qa = slab bit
  int32_t stab;           // measurement: stabilizer index (serial order)
  int32_t offset;         // measurement: syndrome = raw ^ offset
};

struct UProgram {
  int d = 0, nd = 0, nstab = 0, nbits = 0;
  std::vector<ProgOp> ops;
  std::vector<UItem> items;         // one round
  double mats[M_COUNT][16][2];
  double prob[PR_COUNT];
};

// all_slots: emit every noise site and both the unitary and the twirled form of every coherent
// term (probabilities and angles then decide per trajectory) -- the batched form's template.
bool build_unreduced_program(const qec_params& p, bool noisy, UProgram& out, std::string& err,
                             bool all_slots = false);

// Serial-order stabilizers of the code (qec_code): the rotated surface code (Table I order, X then
// Z) or the repetition code's Z_k Z_{k+1}.
std::vector<Stab> make_stabilizers(int d, int code);
bool validate_params(const qec_params& p, std::string& err);
// noisy = false: the noise-free init round (no noise sites, no coherent terms).
bool build_program(const qec_params& p, bool noisy, Program& out, std::string& err, bool all_slots = false);
// The twirl probabilities prob[PR_TW_*] of a noise setting (0 when twirl is off).
void twirl_probs(const qec_noise& nz, double* prob);

}  // namespace qec
