// Builds the static per-round block program (see program.hpp).
#include "program.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <tuple>

namespace qec {

namespace {

// Plaquette with top-left grid cell (r, c); X-type iff r + c odd (Table I, Fig. 1a).
struct Plaq { int r, c; char kind; };

int cell(int d, int r, int c) { return (r >= 0 && r < d && c >= 0 && c < d) ? r * d + c : -1; }

void set_mat(double m[16][2], int idx, double re, double im) { m[idx][0] = re; m[idx][1] = im; }

void mat1(double m[16][2], double a_re, double a_im, double b_re, double b_im,
          double c_re, double c_im, double d_re, double d_im) {
  for (int i = 0; i < 16; ++i) m[i][0] = m[i][1] = 0.0;
  set_mat(m, 0, a_re, a_im); set_mat(m, 1, b_re, b_im);
  set_mat(m, 4, c_re, c_im); set_mat(m, 5, d_re, d_im);
}

// exp(-i theta/2 P) for P in {X, Z} on one qubit
void rot1(double m[16][2], char P, double theta) {
  double c = std::cos(theta / 2), s = std::sin(theta / 2);
  if (P == 'X') mat1(m, c, 0, 0, -s, 0, -s, c, 0);
  else mat1(m, c, -s, 0, 0, 0, 0, c, s);
}

// exp(-i theta/2 Z(x)X), local index 2*a + b (a: Z side, b: X side)
void rot_zx(double m[16][2], double theta) {
  double c = std::cos(theta / 2), s = std::sin(theta / 2);
  for (int i = 0; i < 16; ++i) m[i][0] = m[i][1] = 0.0;
  for (int r = 0; r < 4; ++r) {
    set_mat(m, 5 * r, c, 0);
    int a = r >> 1, b = r & 1;
    int col = (a << 1) | (b ^ 1);             // X flips b
    double sign = a ? -1.0 : 1.0;             // Z phase on a
    m[4 * r + col][1] += -s * sign;
  }
}

void fill_mats(Program& P, const qec_noise& nz, bool noisy) {
  const double h = 1.0 / std::sqrt(2.0);
  mat1(P.mats[M_I], 1, 0, 0, 0, 0, 0, 1, 0);
  mat1(P.mats[M_X], 0, 0, 1, 0, 1, 0, 0, 0);
  mat1(P.mats[M_Y], 0, 0, 0, -1, 0, 1, 0, 0);
  mat1(P.mats[M_Z], 1, 0, 0, 0, 0, 0, -1, 0);
  mat1(P.mats[M_H], h, 0, h, 0, h, 0, -h, 0);
  rot1(P.mats[M_RX90], 'X', M_PI / 2);
  rot1(P.mats[M_RX90DG], 'X', -M_PI / 2);
  rot1(P.mats[M_RZ90], 'Z', M_PI / 2);
  for (int i = 0; i < 16; ++i) P.mats[M_CNOT][i][0] = P.mats[M_CNOT][i][1] = 0.0;
  P.mats[M_CNOT][0][0] = P.mats[M_CNOT][5][0] = P.mats[M_CNOT][11][0] = P.mats[M_CNOT][14][0] = 1.0;
  rot_zx(P.mats[M_RZX90], M_PI / 2);
  double g = noisy ? 1.0 : 0.0;
  rot1(P.mats[M_ROT_RX], 'X', g * nz.theta_rx);
  rot1(P.mats[M_ROT_RXP], 'X', (nz.overrot_follows != 0.0 ? -g : g) * nz.theta_rx);   // after the Rx^dagger prep
  rot1(P.mats[M_ROT_RZ], 'Z', g * nz.theta_rz);
  rot_zx(P.mats[M_ROT_RZX], g * nz.theta_rzx);
  for (int i = 0; i < 16; ++i) P.mats[M_ZZ][i][0] = P.mats[M_ZZ][i][1] = 0.0;
  for (int r = 0; r < 4; ++r) {               // exp(-i phi Z(x)Z): eigenvalue +1 on 00, 11
    double zz = ((r >> 1) ^ (r & 1)) ? -1.0 : 1.0;
    double ph = -g * nz.phi_zz * zz;
    set_mat(P.mats[M_ZZ], 5 * r, std::cos(ph), std::sin(ph));
  }
  rot1(P.mats[M_ROUND_RZ], 'Z', g * nz.round_rz);
  rot1(P.mats[M_ROUND_RX], 'X', g * nz.round_rx);
  // Pauli products Z(x)X and Z(x)Z (twirled Rzx and ZZ terms), local index 2*a + b
  for (int i = 0; i < 16; ++i) P.mats[M_PZX][i][0] = P.mats[M_PZX][i][1] = P.mats[M_PZZ][i][0] = P.mats[M_PZZ][i][1] = 0.0;
  for (int r = 0; r < 4; ++r) {
    const int a = r >> 1, b = r & 1;
    P.mats[M_PZX][4 * r + ((a << 1) | (b ^ 1))][0] = a ? -1.0 : 1.0;
    P.mats[M_PZZ][5 * r][0] = (a ^ b) ? -1.0 : 1.0;
  }
}

bool finite_in(double v, double lo, double hi) { return std::isfinite(v) && v >= lo && v <= hi; }

}  // namespace

std::vector<Stab> make_stabilizers(int d, int code) {
  if (code == QEC_CODE_REPETITION) {   // Z_k Z_{k+1} on a line; gate order q_{k+1}, q_k (Fig. 2(b))
    std::vector<Stab> out;
    for (int k = 0; k + 1 < d; ++k) {
      Stab s;
      s.kind = 'Z';
      s.w = 2;
      const int sl[4] = {k + 1, k, -1, -1};
      std::copy(sl, sl + 4, s.slots);
      out.push_back(s);
    }
    return out;
  }
  std::vector<std::tuple<int, int, Stab>> xs, zs;
  for (int r = -1; r < d; ++r) {
    for (int c = -1; c < d; ++c) {
      int tl = cell(d, r, c), tr = cell(d, r, c + 1), bl = cell(d, r + 1, c), br = cell(d, r + 1, c + 1);
      int w = (tl >= 0) + (tr >= 0) + (bl >= 0) + (br >= 0);
      char kind = ((r + c) & 1) ? 'X' : 'Z';
      bool top_bottom = (r == -1 || r == d - 1), left_right = (c == -1 || c == d - 1);
      bool keep = (w == 4) || (w == 2 && kind == 'X' && top_bottom && !left_right) ||
                  (w == 2 && kind == 'Z' && left_right && !top_bottom);
      if (!keep) continue;
      Stab s;
      s.kind = kind;
      s.w = w;
      if (kind == 'X') {  // clockwise from bottom-right
        int sl[4] = {br, bl, tl, tr};
        std::copy(sl, sl + 4, s.slots);
        xs.emplace_back(r, c, s);
      } else {            // clockwise from top-right
        int sl[4] = {tr, br, bl, tl};
        std::copy(sl, sl + 4, s.slots);
        zs.emplace_back(c, -r, s);
      }
    }
  }
  auto key_less = [](const std::tuple<int, int, Stab>& a, const std::tuple<int, int, Stab>& b) {
    return std::make_pair(std::get<0>(a), std::get<1>(a)) < std::make_pair(std::get<0>(b), std::get<1>(b));
  };
  std::sort(xs.begin(), xs.end(), key_less);
  std::sort(zs.begin(), zs.end(), key_less);
  std::vector<Stab> out;
  for (auto& t : xs) out.push_back(std::get<2>(t));
  for (auto& t : zs) out.push_back(std::get<2>(t));
  return out;
}

bool validate_params(const qec_params& p, std::string& err) {
  if (p.code != QEC_CODE_SURFACE && p.code != QEC_CODE_REPETITION) { err = "bad code"; return false; }
  if (p.code == QEC_CODE_SURFACE && (p.d < 3 || p.d > 5 || (p.d % 2) == 0)) { err = "d must be 3 or 5"; return false; }
  if (p.code == QEC_CODE_REPETITION && (p.d < 9 || p.d > 25 || (p.d % 2) == 0)) {
    err = "repetition code: d must be odd, 9..25";
    return false;
  }
  if (p.rounds < 0 || p.rounds > 64) { err = "rounds must be in [0, 64]"; return false; }
  if (p.layout != QEC_LAYOUT_REDUCED && p.layout != QEC_LAYOUT_UNREDUCED) { err = "bad layout"; return false; }
  if (p.gates != QEC_GATES_CNOT && p.gates != QEC_GATES_CR) { err = "bad gate set"; return false; }
  if (p.precision != QEC_C128 && p.precision != QEC_C64 && p.precision != QEC_C64_TC && p.precision != QEC_C128_TC) {
    err = "bad precision";
    return false;
  }
  const qec_noise& n = p.noise;
  if (!finite_in(n.p1, 0, 1) || !finite_in(n.p2, 0, 1) || !finite_in(n.p_idle, 0, 1)) {
    err = "noise probabilities must be in [0, 1]";
    return false;
  }
  const double a[6] = {n.theta_rx, n.theta_rz, n.theta_rzx, n.phi_zz, n.round_rz, n.round_rx};
  for (double v : a) {
    if (!finite_in(v, -4.0, 4.0)) { err = "angles must be finite with |angle| <= 4"; return false; }
  }
  if (n.twirl != 0.0 && n.twirl != 1.0) { err = "twirl must be 0 or 1"; return false; }
  if (n.overrot_follows != 0.0 && n.overrot_follows != 1.0) { err = "overrot_follows must be 0 or 1"; return false; }
  return true;
}

void twirl_probs(const qec_noise& nz, double* prob) {
  const bool on = nz.twirl != 0.0;
  auto half = [&](double th) { return on ? std::sin(th / 2) * std::sin(th / 2) : 0.0; };
  prob[PR_TW_RX] = half(nz.theta_rx);
  prob[PR_TW_RZ] = half(nz.theta_rz);
  prob[PR_TW_RZX] = half(nz.theta_rzx);
  prob[PR_TW_ZZ] = on ? std::sin(nz.phi_zz) * std::sin(nz.phi_zz) : 0.0;   // exp(-i phi ZZ) = R_ZZ(2 phi)
  prob[PR_TW_ROUND_RZ] = half(nz.round_rz);
  prob[PR_TW_ROUND_RX] = half(nz.round_rx);
}

bool build_program(const qec_params& p, bool noisy, Program& P, std::string& err, bool all_slots) {
  if (!validate_params(p, err)) return false;
  const int d = p.d, nd = p.code == QEC_CODE_REPETITION ? d : d * d;
  const bool cr = p.gates == QEC_GATES_CR;
  const qec_noise& nz = p.noise;
  std::vector<Stab> S = make_stabilizers(d, p.code);
  P = Program();
  P.d = d;
  P.nd = nd;
  P.nstab = (int)S.size();
  fill_mats(P, nz, noisy);
  P.prob[PR_P1] = noisy ? nz.p1 : 0.0;
  P.prob[PR_P2] = noisy ? nz.p2 : 0.0;
  P.prob[PR_IDLE] = noisy ? nz.p_idle : 0.0;
  twirl_probs(nz, P.prob);
  if (!noisy)
    for (int i = PR_TW_RX; i < PR_COUNT; ++i) P.prob[i] = 0.0;
  const bool twirl = noisy && nz.twirl != 0.0;

  // Gate steps of each data qubit, in serial (block) order.
  std::vector<int> nx(nd, 0), nzc(nd, 0);
  std::vector<std::vector<std::pair<int, int>>> gates_of(nd);   // (step, block)
  for (int k = 0; k < P.nstab; ++k) {
    for (int i = 0; i < 4; ++i) {
      int q = S[k].slots[i];
      if (q < 0) continue;
      (S[k].kind == 'X' ? nx : nzc)[q]++;
      gates_of[q].push_back({S[k].kind == 'X' ? 2 + i : 7 + i, k});
    }
  }
  for (int q = 0; q < nd; ++q) {
    for (size_t i = 1; i < gates_of[q].size(); ++i) {
      if (gates_of[q][i].first <= gates_of[q][i - 1].first) {
        err = "serial order does not respect a data qubit's gate order";
        return false;
      }
    }
  }
  // Single-qubit events of each data qubit: steps 0..11 without a gate on it.
  // Each goes to the block of the next gate on that qubit (pre) or, after the
  // last gate of the round, to the block of the last gate (post).
  std::vector<std::vector<std::pair<int, int>>> pre(P.nstab), post(P.nstab);   // (data qubit, step)
  for (int q = 0; q < nd; ++q) {
    const auto& g = gates_of[q];
    for (int t = 0; t <= 11; ++t) {
      bool busy = false;
      for (auto& e : g) busy |= (e.first == t);
      if (busy) continue;
      int blk = -1;
      for (auto& e : g) {
        if (e.first > t) { blk = e.second; break; }
      }
      if (blk >= 0) pre[blk].push_back({q, t});
      else post[g.back().second].push_back({q, t});
    }
  }

  for (int k = 0; k < P.nstab; ++k) {
    const Stab& s = S[k];
    BlockInfo bi;
    bi.op_begin = (int)P.ops.size();
    bi.w = s.w;
    std::vector<int> qs;
    for (int i = 0; i < 4; ++i) if (s.slots[i] >= 0) qs.push_back(s.slots[i]);
    std::sort(qs.begin(), qs.end());
    for (int i = 0; i < 4; ++i) bi.q[i] = i < (int)qs.size() ? qs[i] : -1;
    bi.offset = (cr && s.w == 2) ? 1 : 0;
    bi.stab = k;
    const uint8_t anc = (uint8_t)s.w;
    const uint32_t site_a = (uint32_t)(nd + k);
    auto local = [&](int q) { return (uint8_t)(std::find(qs.begin(), qs.end(), q) - qs.begin()); };
    auto u1 = [&](uint8_t q, uint16_t m) { P.ops.push_back({OP_U1, q, 0, 0, m, 0, 0}); };
    auto u2 = [&](uint8_t a, uint8_t b, uint16_t m) { P.ops.push_back({OP_U2, a, b, 0, m, 0, 0}); };
    auto n1 = [&](uint8_t q, int step, uint32_t site, uint8_t pid) {
      if (all_slots || P.prob[pid] > 0.0) P.ops.push_back({OP_N1, q, 0, pid, 0, (uint16_t)step, site});
    };
    auto n2 = [&](uint8_t a, uint8_t b, int step, uint32_t site) {
      if (all_slots || P.prob[PR_P2] > 0.0) P.ops.push_back({OP_N2, a, b, PR_P2, 0, (uint16_t)step, site});
    };
    // A coherent term: the unitary `um` (angle != 0), or twirled, the Pauli `tm` with
    // probability prob[pid], drawn at (step, factor << 24 | site).
    auto coh1 = [&](uint8_t q, int step, uint32_t site, int factor, uint16_t um, uint16_t tm, double angle, uint8_t pid) {
      if (!noisy) return;
      if (all_slots || (!twirl && angle != 0.0)) u1(q, um);
      if (all_slots || (twirl && P.prob[pid] > 0.0))
        P.ops.push_back({OP_T1, q, 0, pid, tm, (uint16_t)step, ((uint32_t)factor << 24) | site});
    };
    auto coh2 = [&](uint8_t a, uint8_t b, int step, uint32_t site, int factor, uint16_t um, uint16_t tm, double angle,
                    uint8_t pid) {
      if (!noisy) return;
      if (all_slots || (!twirl && angle != 0.0)) u2(a, b, um);
      if (all_slots || (twirl && P.prob[pid] > 0.0))
        P.ops.push_back({OP_T2, a, b, pid, tm, (uint16_t)step, ((uint32_t)factor << 24) | site});
    };
    auto data_event = [&](int q, int t) {
      uint8_t lq = local(q);
      if (t == 0) {
        coh1(lq, t, (uint32_t)q, 6, M_ROUND_RZ, M_Z, nz.round_rz, PR_TW_ROUND_RZ);
        coh1(lq, t, (uint32_t)q, 7, M_ROUND_RX, M_X, nz.round_rx, PR_TW_ROUND_RX);
      } else if (cr && (t == 6 || t == 11)) {
        int nfac = t == 6 ? nx[q] : nzc[q];
        for (int f = 0; f < nfac; ++f) {
          u1(lq, t == 6 ? M_RX90 : M_RZ90);
          if (t == 6) coh1(lq, t, (uint32_t)q, f, M_ROT_RX, M_X, nz.theta_rx, PR_TW_RX);
          else coh1(lq, t, (uint32_t)q, f, M_ROT_RZ, M_Z, nz.theta_rz, PR_TW_RZ);
        }
        n1(lq, t, (uint32_t)q, nfac ? PR_P1 : PR_IDLE);   // no correction gate: the qubit idles
      } else {
        n1(lq, t, (uint32_t)q, PR_IDLE);
      }
    };
    for (auto& e : pre[k]) data_event(e.first, e.second);
    const int t0 = s.kind == 'X' ? 1 : 7, t1 = s.kind == 'X' ? 6 : 11;
    for (int t = t0; t <= t1; ++t) {
      if (s.kind == 'X' && (t == 1 || t == 6)) {
        if (!cr) {
          u1(anc, M_H);
        } else {
          u1(anc, t == 1 ? M_RX90DG : M_RX90);
          coh1(anc, t, site_a, 0, t == 1 ? M_ROT_RXP : M_ROT_RX, M_X, nz.theta_rx, PR_TW_RX);
        }
        n1(anc, t, site_a, PR_P1);
        continue;
      }
      if (s.kind == 'Z' && t == 11) {
        n1(anc, t, site_a, PR_IDLE);
        continue;
      }
      int q = s.slots[s.kind == 'X' ? t - 2 : t - 7];
      if (q < 0) {
        n1(anc, t, site_a, PR_IDLE);
        continue;
      }
      uint8_t lq = local(q);
      uint8_t first = s.kind == 'X' ? anc : lq, second = s.kind == 'X' ? lq : anc;
      if (!cr) {
        u2(first, second, M_CNOT);
      } else {
        u2(first, second, M_RZX90);
        coh2(first, second, t, (uint32_t)q, 4, M_ROT_RZX, M_PZX, nz.theta_rzx, PR_TW_RZX);
      }
      coh2(first, second, t, (uint32_t)q, 5, M_ZZ, M_PZZ, nz.phi_zz, PR_TW_ZZ);
      n2(anc, lq, t, (uint32_t)q);
    }
    for (auto& e : post[k]) data_event(e.first, e.second);
    bi.op_end = (int)P.ops.size();
    P.blocks.push_back(bi);
  }
  return true;
}

bool build_unreduced_program(const qec_params& p, bool noisy, UProgram& U, std::string& err, bool all_slots) {
  if (!validate_params(p, err)) return false;
  if (p.code != QEC_CODE_SURFACE) { err = "the unreduced register is built for the surface code"; return false; }
  const int d = p.d, nd = d * d;
  const bool cr = p.gates == QEC_GATES_CR;
  const qec_noise& nz = p.noise;
  std::vector<Stab> S = make_stabilizers(d, p.code);
  const int nst = (int)S.size(), half = nst / 2;
  U = UProgram();
  U.d = d;
  U.nd = nd;
  U.nstab = nst;
  U.nbits = nd + half;
  {
    Program tmp;
    tmp.d = d;
    fill_mats(tmp, nz, noisy);
    std::memcpy(U.mats, tmp.mats, sizeof(U.mats));
  }
  U.prob[PR_P1] = noisy ? nz.p1 : 0.0;
  U.prob[PR_P2] = noisy ? nz.p2 : 0.0;
  U.prob[PR_IDLE] = noisy ? nz.p_idle : 0.0;
  twirl_probs(nz, U.prob);
  if (!noisy)
    for (int i = PR_TW_RX; i < PR_COUNT; ++i) U.prob[i] = 0.0;
  const bool twirl = noisy && nz.twirl != 0.0;
  std::vector<int> nx(nd, 0), nzc(nd, 0);
  for (const Stab& s : S)
    for (int i = 0; i < 4; ++i)
      if (s.slots[i] >= 0) (s.kind == 'X' ? nx : nzc)[s.slots[i]]++;
  auto u1 = [&](int q, uint16_t m) { U.ops.push_back({OP_U1, (uint8_t)q, 0, 0, m, 0, 0}); };
  auto u2 = [&](int a, int b, uint16_t m) { U.ops.push_back({OP_U2, (uint8_t)a, (uint8_t)b, 0, m, 0, 0}); };
  auto n1 = [&](int q, int step, uint32_t site, uint8_t pid) {
    if (all_slots || U.prob[pid] > 0.0) U.ops.push_back({OP_N1, (uint8_t)q, 0, pid, 0, (uint16_t)step, site});
  };
  auto n2 = [&](int a, int b, int step, uint32_t site) {
    if (all_slots || U.prob[PR_P2] > 0.0)
      U.ops.push_back({OP_N2, (uint8_t)a, (uint8_t)b, PR_P2, 0, (uint16_t)step, site});
  };
  auto coh1 = [&](int q, int step, uint32_t site, int factor, uint16_t um, uint16_t tm, double angle, uint8_t pid) {
    if (!noisy) return;
    if (all_slots || (!twirl && angle != 0.0)) u1(q, um);
    if (all_slots || (twirl && U.prob[pid] > 0.0))
      U.ops.push_back({OP_T1, (uint8_t)q, 0, pid, tm, (uint16_t)step, ((uint32_t)factor << 24) | site});
  };
  auto coh2 = [&](int a, int b, int step, uint32_t site, int factor, uint16_t um, uint16_t tm, double angle,
                  uint8_t pid) {
    if (!noisy) return;
    if (all_slots || (!twirl && angle != 0.0)) u2(a, b, um);
    if (all_slots || (twirl && U.prob[pid] > 0.0))
      U.ops.push_back({OP_T2, (uint8_t)a, (uint8_t)b, pid, tm, (uint16_t)step, ((uint32_t)factor << 24) | site});
  };
  auto unit = [&](int nq, int qa, int qb, int begin) {
    if ((int)U.ops.size() > begin) U.items.push_back({0, begin, (int32_t)U.ops.size(), nq, qa, qb, -1, 0});
  };
  for (int part = 0; part < 2; ++part) {
    const char kind = part == 0 ? 'X' : 'Z';
    const int k0 = part == 0 ? 0 : half;
    const int t0 = part == 0 ? 1 : 7, t1 = part == 0 ? 6 : 11;
    for (int t = (part == 0 ? 0 : t0); t <= t1; ++t) {
      std::vector<int> busy(nd, 0);
      for (int j = 0; j < half; ++j) {   // ancilla units of this step
        const Stab& s = S[k0 + j];
        const int a = nd + j;
        const uint32_t site_a = (uint32_t)(nd + k0 + j);
        if (t == 0) continue;
        const int begin = (int)U.ops.size();
        if (kind == 'X' && (t == 1 || t == 6)) {
          if (!cr) {
            u1(a, M_H);
          } else {
            u1(a, t == 1 ? M_RX90DG : M_RX90);
            coh1(a, t, site_a, 0, t == 1 ? M_ROT_RXP : M_ROT_RX, M_X, nz.theta_rx, PR_TW_RX);
          }
          n1(a, t, site_a, PR_P1);
          unit(1, a, 0, begin);
          continue;
        }
        if (kind == 'Z' && t == 11) {
          n1(a, t, site_a, PR_IDLE);
          unit(1, a, 0, begin);
          continue;
        }
        const int q = s.slots[kind == 'X' ? t - 2 : t - 7];
        if (q < 0) {
          n1(a, t, site_a, PR_IDLE);
          unit(1, a, 0, begin);
          continue;
        }
        busy[q] = 1;
        const int first = kind == 'X' ? a : q, second = kind == 'X' ? q : a;
        if (!cr) {
          u2(first, second, M_CNOT);
        } else {
          u2(first, second, M_RZX90);
          coh2(first, second, t, (uint32_t)q, 4, M_ROT_RZX, M_PZX, nz.theta_rzx, PR_TW_RZX);
        }
        coh2(first, second, t, (uint32_t)q, 5, M_ZZ, M_PZZ, nz.phi_zz, PR_TW_ZZ);
        n2(a, q, t, (uint32_t)q);
        unit(2, first, second, begin);
      }
      for (int q = 0; q < nd; ++q) {     // data qubits not in a two-qubit gate
        if (busy[q]) continue;
        const int begin = (int)U.ops.size();
        if (t == 0) {
          coh1(q, t, (uint32_t)q, 6, M_ROUND_RZ, M_Z, nz.round_rz, PR_TW_ROUND_RZ);
          coh1(q, t, (uint32_t)q, 7, M_ROUND_RX, M_X, nz.round_rx, PR_TW_ROUND_RX);
        } else if (cr && (t == 6 || t == 11)) {
          const int nfac = t == 6 ? nx[q] : nzc[q];
          for (int f = 0; f < nfac; ++f) {
            u1(q, t == 6 ? M_RX90 : M_RZ90);
            if (t == 6) coh1(q, t, (uint32_t)q, f, M_ROT_RX, M_X, nz.theta_rx, PR_TW_RX);
            else coh1(q, t, (uint32_t)q, f, M_ROT_RZ, M_Z, nz.theta_rz, PR_TW_RZ);
          }
          n1(q, t, (uint32_t)q, PR_P1);
        } else {
          n1(q, t, (uint32_t)q, PR_IDLE);
        }
        unit(1, q, 0, begin);
      }
    }
    for (int j = 0; j < half; ++j) {     // measurements of this part's ancillas, serial order
      const Stab& s = S[k0 + j];
      U.items.push_back({1, 0, 0, 1, nd + j, 0, k0 + j, (cr && s.w == 2) ? 1 : 0});
    }
  }
  return true;
}

}  // namespace qec
