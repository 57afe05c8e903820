"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (CPU only).

Each test checks the oracle against something other than itself: the paper's
printed table and examples, an independent Philox implementation (numpy's),
scipy's matrix exponential, brute-force dense operators, a stabilizer-tableau
simulator, closed forms, and the register-reduction equivalence of Sec. II.B.
"""
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import run_trajectory
from oracle import gates as G
from oracle import tableau as TB
from oracle.circuit import Trajectory
from oracle.lattice import logical_z_support, stabilizers
from oracle.philox import philox4x64_10, uniform53
from oracle.runner import run_ops

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- Philox ------------------------------------------------------------------------------
@pytest.mark.parametrize("ctr,key", [((1, 0, 0, 0), (0, 0)), ((5, 7, 11, 13), (123, 456)),
                                     ((2**64 - 2, 3, 2**63, 9), (2**64 - 1, 77)),
                                     ((999, 5, (6 << 32) | 17, 0), (2000, 0))])
def test_philox_matches_numpy(ctr, key):
    # numpy's Philox BitGenerator is Philox4x64-10; it increments its counter before generating.
    c = list(ctr)
    c[0] -= 1
    bg = np.random.Philox(counter=np.array(c, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    assert philox4x64_10(ctr, key) == tuple(int(x) for x in bg.random_raw(4))


def test_uniform53_range():
    assert uniform53(0) == 0.0
    assert uniform53(2**64 - 1) == 1.0 - 2.0**-53


# ---- lattice -----------------------------------------------------------------------------
def _read_table1():
    xs, zs = [], []
    with open(os.path.join(GOLDEN, "table1_d5.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            _, xsup, zsup = line.split()
            xs.append(sorted(int(v) - 1 for v in xsup.split(",")))
            zs.append(sorted(int(v) - 1 for v in zsup.split(",")))
    return xs, zs


def test_table1_d5():
    xs, zs = _read_table1()
    S = stabilizers(5)
    assert [s["support"] for s in S if s["kind"] == "X"] == xs
    assert [s["support"] for s in S if s["kind"] == "Z"] == zs


def test_gate_order_examples():
    S = stabilizers(5)
    with open(os.path.join(GOLDEN, "gate_order_examples.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for kind, sup, order in rows:
        support = sorted(int(v) - 1 for v in sup.split(","))
        (s,) = [s for s in S if s["kind"] == kind and s["support"] == support]
        got = ["w" if q is None else str(q + 1) for q in s["slots"]]
        assert got == order.split(",")


@pytest.mark.parametrize("d", [3, 5, 7])
def test_code_structure(d):
    S = stabilizers(d)
    xs = [set(s["support"]) for s in S if s["kind"] == "X"]
    zs = [set(s["support"]) for s in S if s["kind"] == "Z"]
    assert len(xs) == len(zs) == (d * d - 1) // 2
    for a in xs:
        for b in zs:
            assert len(a & b) % 2 == 0            # X and Z stabilizers commute
    zl = set(logical_z_support(d))
    xl = {r * d for r in range(d)}                # X on the first column
    assert all(len(zl & a) % 2 == 0 for a in xs)
    assert all(len(xl & b) % 2 == 0 for b in zs)
    assert len(zl & xl) % 2 == 1
    # X/Z stabilizers are independent: GF(2) rank equals their count
    for grp in (xs, zs):
        M = np.array([[1 if q in s else 0 for q in range(d * d)] for s in grp], dtype=np.uint8)
        assert _gf2_rank(M) == len(grp)


def _gf2_rank(M):
    M = M.copy()
    r = 0
    for c in range(M.shape[1]):
        piv = [i for i in range(r, M.shape[0]) if M[i, c]]
        if not piv:
            continue
        M[[r, piv[0]]] = M[[piv[0], r]]
        for i in range(M.shape[0]):
            if i != r and M[i, c]:
                M[i] ^= M[r]
        r += 1
    return r


def test_printed_logical_z_is_not_a_logical():
    # Sec. III.B prints Z1 Z7 Z13 Z19 Z25; it overlaps X1X2 on one qubit, so it cannot be used.
    diag = {0, 6, 12, 18, 24}
    xs = [set(s["support"]) for s in stabilizers(5) if s["kind"] == "X"]
    assert any(len(diag & a) % 2 for a in xs)


def test_register_sizes():
    for d, red, unred in ((3, 10, 17), (5, 26, 49)):
        assert Trajectory(d, 1, "cr", "reduced", {}, 0, 0).n == red
        assert 2 * d * d - 1 == unred
    assert Trajectory(3, 1, "cr", "unreduced", {}, 0, 0).n == 17


def test_step_count_per_cycle():
    # Sec. III.D counts 11 steps per syndrome cycle: 6 for the X part, 5 for the Z part.
    T = Trajectory(3, 1, "cr", "unreduced", dict(p_idle=1.0, p1=1.0, p2=1.0), 0, 0).build()
    assert sorted({t for (r, t, s, c) in T.events if r == 1}) == list(range(1, 12))


# ---- gates -------------------------------------------------------------------------------
def test_gate_matrices_vs_expm():
    assert np.allclose(G.RX90, scipy.linalg.expm(-1j * np.pi / 4 * G.PX), atol=1e-14)
    assert np.allclose(G.RX90DG, scipy.linalg.expm(1j * np.pi / 4 * G.PX), atol=1e-14)
    assert np.allclose(G.RZ90, scipy.linalg.expm(-1j * np.pi / 4 * G.PZ), atol=1e-14)
    assert np.allclose(G.RZX90, scipy.linalg.expm(-1j * np.pi / 4 * np.kron(G.PZ, G.PX)), atol=1e-14)
    for th in (0.013, 0.7, -2.1):
        assert np.allclose(G.rot(G.PX, th), scipy.linalg.expm(-0.5j * th * G.PX), atol=1e-14)
        assert np.allclose(G.zz_crosstalk(th), scipy.linalg.expm(-1j * th * np.kron(G.PZ, G.PZ)), atol=1e-14)


def test_clifford_forms_used_by_tableau():
    S = np.diag([1, 1j])
    Hm = G.H
    assert TB._close_up_to_phase(G.RZ90, S)
    assert TB._close_up_to_phase(G.RX90, Hm @ S @ Hm)
    assert TB._close_up_to_phase(G.RX90DG, Hm @ S @ S @ S @ Hm)
    I2 = np.eye(2)
    Hb = np.kron(I2, Hm)
    Sb = np.kron(I2, S)
    assert TB._close_up_to_phase(G.RZX90, Hb @ G.CNOT @ Sb @ G.CNOT @ Hb)


def test_single_qubit_flip_closed_form():
    # Sec. III.A: <0| R_x(theta)^dagger P_1 R_x(theta) |0> = sin^2(theta/2)
    for th in (0.02, 0.3, 1.1):
        v = G.rot(G.PX, th) @ np.array([1, 0], dtype=complex)
        assert abs(abs(v[1]) ** 2 - np.sin(th / 2) ** 2) < 1e-16


# ---- C core vs brute force ---------------------------------------------------------------
def _full_1q(n, q, m):
    out = np.array([[1.0]], dtype=complex)
    for b in reversed(range(n)):
        out = np.kron(out, m if b == q else np.eye(2))
    return out


def _full_2q(n, qa, qb, m):
    dim = 1 << n
    U = np.zeros((dim, dim), dtype=complex)
    for i in range(dim):
        ca = 2 * ((i >> qa) & 1) + ((i >> qb) & 1)
        for l in range(4):
            j = i & ~(1 << qa) & ~(1 << qb) | ((l >> 1) << qa) | ((l & 1) << qb)
            U[j, i] += m[l, ca]
    return U


def _haar(k, rng):
    z = (rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("n", [3, 5])
def test_core_gates_vs_dense(n):
    rng = np.random.default_rng(n)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    ref = psi.copy()
    ops = []
    for _ in range(12):
        if rng.random() < 0.5:
            q = int(rng.integers(n))
            m = _haar(2, rng)
            ops.append(("U1", q, m))
            ref = _full_1q(n, q, m) @ ref
        else:
            qa, qb = (int(v) for v in rng.choice(n, 2, replace=False))
            m = _haar(4, rng)
            ops.append(("U2", qa, qb, m))
            ref = _full_2q(n, qa, qb, m) @ ref
    run_ops(psi, n, ops)
    assert np.abs(psi - ref).max() < 1e-14


@pytest.mark.parametrize("reset", [0, 1])
def test_core_measure_vs_projector(reset):
    n = 4
    rng = np.random.default_rng(3)
    for q in range(n):
        for u in (0.1, 0.9):
            psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
            psi /= np.linalg.norm(psi)
            P1 = np.diag([float((i >> q) & 1) for i in range(1 << n)])
            p1 = float(np.real(psi.conj() @ P1 @ psi))
            out = 1 if u < p1 else 0
            proj = P1 if out else np.eye(1 << n) - P1
            ref = proj @ psi / np.sqrt(np.real(psi.conj() @ proj @ psi))
            if reset and out:
                ref = _full_1q(n, q, G.PX) @ ref
            got = psi.copy()
            outs, p1s = run_ops(got, n, [("M", q, u, -1, reset)])
            assert outs[0] == out and abs(p1s[0] - p1) < 1e-15
            assert np.abs(got - ref).max() < 1e-15


# ---- circuit-level pins ------------------------------------------------------------------
@pytest.mark.parametrize("gates", ["cnot", "cr"])
@pytest.mark.parametrize("layout", ["reduced", "unreduced"])
def test_noiseless_rounds_have_zero_syndrome(gates, layout):
    r = run_trajectory(3, 3, gates, layout, {}, seed=0, traj=0, want_state=True)
    assert not r["syndromes"].any()
    assert r["raw_logical"] == 0
    assert abs(np.linalg.norm(r["state"]) - 1) < 1e-14


@pytest.mark.parametrize("gates", ["cnot", "cr"])
def test_noiseless_d5_zero_syndrome_tableau(gates):
    T = Trajectory(5, 2, gates, "reduced", {}, 0, 0).build()
    outs, _ = TB.run_ops(TB.Tableau(T.n), T.ops)
    nm = sum(1 for m in T.meas if m[0] == "anc")
    syn = [o ^ m[3] for o, m in zip(outs[:nm], T.meas[:nm])]
    assert not any(syn)


def test_init_state_closed_form_cnot():
    # With H/CNOT circuits, projecting |0..0> onto the +1 eigenspace of every stabilizer gives
    # equal amplitude 2^{-(d^2-1)/4} on the 2^{(d^2-1)/2} states of the X-stabilizer orbit of |0..0>.
    d = 3
    r = run_trajectory(d, 0, "cnot", "reduced", {}, 0, 0, want_state=True)
    psi = r["state"]
    orbit = {0}
    for s in stabilizers(d):
        if s["kind"] == "X":
            mask = sum(1 << q for q in s["support"])
            orbit |= {v ^ mask for v in orbit}
    assert len(orbit) == 2 ** ((d * d - 1) // 2)
    ref = np.zeros_like(psi)
    ref[sorted(orbit)] = 2.0 ** (-(d * d - 1) / 4)
    assert np.abs(psi - ref).max() < 1e-15


def _apply_pauli_string(psi, n, xs, zs):
    idx = np.arange(1 << n)
    xm = sum(1 << q for q in xs)
    out = psi[idx ^ xm].copy()
    for q in zs:
        out *= np.where(((idx >> q) & 1) == 1, -1.0, 1.0)
    return out


def test_init_state_is_code_state_cr():
    d = 3
    r = run_trajectory(d, 0, "cr", "reduced", {}, 0, 0, want_state=True)
    psi = r["state"]
    n = r["n_qubits"]
    for s in stabilizers(d):
        if s["kind"] == "X":
            got = _apply_pauli_string(psi, n, s["support"], [])
        else:
            got = _apply_pauli_string(psi, n, [], s["support"])
        assert np.abs(got - psi).max() < 1e-14
    assert np.abs(_apply_pauli_string(psi, n, [], logical_z_support(d)) - psi).max() < 1e-14


NOISY = dict(p1=0.03, p2=0.03, p_idle=0.02, theta_rx=0.1, theta_rz=0.07, theta_rzx=0.05,
             phi_zz=0.08, round_rz=0.1, round_rx=0.05)


@pytest.mark.parametrize("gates", ["cnot", "cr"])
def test_reduced_register_equals_unreduced(gates):
    # Sec. II.B: delaying the stabilizer circuits onto one reused ancilla does not change the system.
    for traj in range(12):
        a = run_trajectory(3, 3, gates, "reduced", NOISY, seed=7, traj=traj, want_state=True)
        b = run_trajectory(3, 3, gates, "unreduced", NOISY, seed=7, traj=traj, want_state=True)
        assert (a["syndromes"] == b["syndromes"]).all()
        assert (a["data_bits"] == b["data_bits"]).all()
        assert sorted(a["events"]) == sorted(b["events"])
        sa = a["state"].reshape(2, 512)
        sb = b["state"].reshape(256, 512)
        assert np.abs(sa[0] - sb[0]).max() < 1e-13
        assert np.abs(sa[1]).max() == 0 and np.abs(sb[1:]).max() == 0


@pytest.mark.parametrize("gates", ["cnot", "cr"])
@pytest.mark.parametrize("layout", ["reduced", "unreduced"])
def test_pauli_noise_matches_tableau(gates, layout):
    nz = dict(p1=0.05, p2=0.05, p_idle=0.04)
    for traj in range(8):
        T = Trajectory(3, 3, gates, layout, nz, 11, traj).build()
        outs, _ = TB.run_ops(TB.Tableau(T.n), T.ops)
        sv = run_trajectory(3, 3, gates, layout, nz, seed=11, traj=traj)
        sv_outs = [rec[4] for rec in sv["anc_records"]] + [rec[3] for rec in sv["readout_records"]]
        assert outs == sv_outs


@pytest.mark.parametrize("gates", ["cnot", "cr"])
@pytest.mark.parametrize("code", [1, 2, 3])
def test_single_pauli_flips_predicted_stabilizers(gates, code):
    d = 3
    S = stabilizers(d)
    for q in range(d * d):
        r = run_trajectory(d, 2, gates, "reduced", {}, 0, 0, inject=[(1, 0, q, G.PAULI[code])])
        pred = [int(q in s["support"] and ((s["kind"] == "Z" and code in (1, 2)) or
                                           (s["kind"] == "X" and code in (2, 3)))) for s in S]
        assert r["syndromes"][1].tolist() == pred
        assert r["syndromes"][2].tolist() == pred


@pytest.mark.parametrize("gates", ["cnot", "cr"])
def test_over_rotation_flip_probability(gates):
    # Sec. III.A: one R_X(theta) on a data qubit of the code state flips its Z-stabilizers
    # with probability sin^2(theta/2).
    d = 3
    S = stabilizers(d)
    th = 0.37
    q = 4
    r = run_trajectory(d, 1, gates, "reduced", {}, 0, 0, inject=[(1, 0, q, G.rot(G.PX, th))])
    first_z = [k for k, s in enumerate(S) if s["kind"] == "Z" and q in s["support"]][0]
    (rec,) = [x for x in r["anc_records"] if x[0] == 1 and x[1] == first_z]
    offset = 1 if (gates == "cr" and S[first_z]["weight"] == 2) else 0
    p_flip = rec[3] if offset == 0 else 1 - rec[3]
    assert abs(p_flip - np.sin(th / 2) ** 2) < 1e-14
    for k, s in enumerate(S):
        if s["kind"] == "X":
            (x,) = [x for x in r["anc_records"] if x[0] == 1 and x[1] == k]
            assert min(x[3], 1 - x[3]) < 1e-14


@pytest.mark.parametrize("d", [3, 5])
def test_over_rotation_sign_closed_form(d):
    """X-stabilizer readout of the code state under theta_rx alone (Sec. III.A, CR compile of Sec. II.C).

    The ancilla sees Rx(pi/2 + theta) U Rx(-pi/2 + s theta)|0>, s = +1 with the same-sign reading and
    -1 with the sign-follows variant.  On the +1 eigenspace of a weight-4 X stabilizer the four Rzx
    gates multiply to a phase, so P(1) = sin^2((1 + s) theta / 2); for weight 2 they multiply to
    -+i Z_anc, so P(1) = cos^2((1 - s) theta / 2).  Data over-rotations commute with X stabilizers."""
    S = stabilizers(d)
    th = 0.31
    for fol, s in ((0, 1.0), (1, -1.0)):
        r = run_trajectory(d, 1, "cr", "reduced", {"theta_rx": th, "overrot_follows": fol}, 0, 0)
        for k, st in enumerate(S):
            if st["kind"] != "X":
                continue
            (x,) = [x for x in r["anc_records"] if x[0] == 1 and x[1] == k]
            want = np.sin((1 + s) * th / 2) ** 2 if st["weight"] == 4 else np.cos((1 - s) * th / 2) ** 2
            assert abs(x[3] - want) < 1e-13, (fol, k, x[3], want)   # FP64 sums over 2^26 amplitudes


def _n_sites(d, rounds):
    # per round: every data qubit at each of the 11 steps, plus each ancilla's own steps
    # (X: 6 - weight, Z: 5 - weight; its gate steps share the data qubit's site)
    S = stabilizers(d)
    anc = sum((6 if s["kind"] == "X" else 5) - s["weight"] for s in S)
    return rounds * (d * d * 11 + anc)


def test_noise_occurrence_rate():
    p, rounds = 0.2, 40
    T = Trajectory(3, rounds, "cr", "reduced", dict(p1=p, p2=p, p_idle=p), 5, 0).build()
    n = _n_sites(3, rounds)
    assert abs(len(T.events) / n - p) < 4 * np.sqrt(p * (1 - p) / n)


def _chi2_ok(counts, k):
    counts = np.asarray(counts, dtype=float)
    e = counts.sum() / k
    chi2 = ((counts - e) ** 2 / e).sum()
    return chi2 < k - 1 + 5 * np.sqrt(2 * (k - 1))


def test_one_qubit_pauli_types_uniform():
    # Eq. 1: X, Y, Z with p/3 each.  Only one-qubit sites are noisy here.
    T = Trajectory(3, 60, "cr", "reduced", dict(p1=0.5, p_idle=0.5), 9, 0).build()
    codes = [c for (_, _, _, c) in T.events]
    assert set(codes) <= {1, 2, 3}
    assert _chi2_ok([codes.count(c) for c in (1, 2, 3)], 3)


def test_two_qubit_pauli_pairs_uniform():
    # Eq. 2 read with normalised weights: one of the 15 non-identity pairs, uniformly.
    T = Trajectory(3, 150, "cnot", "reduced", dict(p2=0.5), 9, 0).build()
    codes = [c for (_, _, _, c) in T.events]
    assert set(codes) <= set(range(1, 16))
    assert _chi2_ok([codes.count(c) for c in range(1, 16)], 15)


def test_norm_conserved_with_coherent_noise():
    r = run_trajectory(3, 4, "cr", "reduced", NOISY, seed=3, traj=5, want_state=True)
    assert abs(np.linalg.norm(r["state"]) - 1) < 1e-13


# ---- twirled variant (Sec. III.A: decohered coherent terms act as Pauli errors) -------------
TWIRLED = dict(NOISY, twirl=1, theta_rx=0.4, theta_rz=0.3, theta_rzx=0.3, phi_zz=0.2, round_rz=0.3, round_rx=0.25)


@pytest.mark.parametrize("gates", ["cnot", "cr"])
@pytest.mark.parametrize("layout", ["reduced", "unreduced"])
def test_twirled_noise_is_clifford_and_matches_tableau(gates, layout):
    for traj in range(6):
        T = Trajectory(3, 3, gates, layout, TWIRLED, 13, traj).build()
        assert T.twirls                      # the twirled terms do fire at these angles
        outs, _ = TB.run_ops(TB.Tableau(T.n), T.ops)
        sv = run_trajectory(3, 3, gates, layout, TWIRLED, seed=13, traj=traj)
        sv_outs = [rec[4] for rec in sv["anc_records"]] + [rec[3] for rec in sv["readout_records"]]
        assert outs == sv_outs


@pytest.mark.parametrize("gates", ["cnot", "cr"])
def test_twirled_reduced_register_equals_unreduced(gates):
    for traj in range(8):
        a = Trajectory(3, 3, gates, "reduced", TWIRLED, 5, traj).build()
        b = Trajectory(3, 3, gates, "unreduced", TWIRLED, 5, traj).build()
        assert sorted(a.twirls) == sorted(b.twirls) and sorted(a.events) == sorted(b.events)


def test_twirl_probability_is_sin2_half_angle():
    # round_rx alone, twirled: every data qubit gets X with probability sin^2(theta/2) per round
    th = 0.5
    fired = trials = 0
    for traj in range(40):
        T = Trajectory(3, 10, "cr", "reduced", dict(round_rx=th, twirl=1), 3, traj).build()
        fired += sum(1 for (r, t, s, f) in T.twirls if f == 7)
        trials += 10 * 9
    p = np.sin(th / 2) ** 2
    assert abs(fired / trials - p) < 4 * np.sqrt(p * (1 - p) / trials)
