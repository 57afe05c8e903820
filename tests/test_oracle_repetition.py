"""Pins of the oracle's one-dimensional repetition code (Sec. II.B, Fig. 2) against facts fixed by
the code itself: its stabilizers, a stabilizer-tableau simulator, single-error syndromes, and the
paper's claim that delaying the syndrome circuits onto one reused ancilla leaves the simulated
system unchanged."""
import numpy as np
import pytest

from oracle import run_trajectory
from oracle import gates as G
from oracle import tableau as TB
from oracle.circuit import Trajectory
from oracle.lattice import code_stabilizers, logical_z_support

D = 9
NOISY = dict(p1=0.03, p2=0.03, p_idle=0.02, theta_rx=0.1, theta_rz=0.07, theta_rzx=0.05,
             phi_zz=0.08, round_rz=0.1, round_rx=0.05)


def test_structure_and_time_order():
    S = code_stabilizers(D, "repetition")
    assert len(S) == D - 1
    for k, s in enumerate(S):
        assert s["kind"] == "Z" and s["support"] == [k, k + 1] and s["weight"] == 2
    # serial order k = 0, 1, ...: each qubit's gate steps increase along it (Fig. 2(b))
    seen = {}
    for s in S:
        for step, q in enumerate(s["slots"]):
            if q is not None:
                assert seen.get(q, -1) < step
                seen[q] = step
    # Z on every qubit of the line is Z_0 times stabilizers when d is odd
    assert logical_z_support(D, "repetition") == list(range(D))


@pytest.mark.parametrize("gates", ["cnot", "cr"])
@pytest.mark.parametrize("layout", ["reduced", "unreduced"])
def test_noiseless_rounds_zero_syndrome(gates, layout):
    r = run_trajectory(D, 3, gates, layout, {}, 0, 0, code="repetition")
    assert not r["syndromes"].any() and not r["data_bits"].any() and r["raw_logical"] == 0


@pytest.mark.parametrize("gates", ["cnot", "cr"])
@pytest.mark.parametrize("pauli", [1, 2, 3])
def test_single_pauli_flips_predicted_stabilizers(gates, pauli):
    S = code_stabilizers(D, "repetition")
    for q in range(D):
        r = run_trajectory(D, 2, gates, "reduced", {}, 0, 0, inject=[(1, 0, q, G.PAULI[pauli])], code="repetition")
        pred = [int(q in s["support"] and pauli in (1, 2)) for s in S]    # X and Y flip Z-stabilizers
        assert r["syndromes"][1].tolist() == pred and r["syndromes"][2].tolist() == pred
        assert r["raw_logical"] == (1 if pauli in (1, 2) else 0)          # the flip reaches the readout


@pytest.mark.parametrize("gates", ["cnot", "cr"])
@pytest.mark.parametrize("layout", ["reduced", "unreduced"])
def test_pauli_noise_matches_tableau(gates, layout):
    nz = dict(p1=0.05, p2=0.05, p_idle=0.04)
    for traj in range(6):
        T = Trajectory(D, 3, gates, layout, nz, 13, traj, code="repetition").build()
        outs, _ = TB.run_ops(TB.Tableau(T.n), T.ops)
        sv = run_trajectory(D, 3, gates, layout, nz, seed=13, traj=traj, code="repetition")
        assert outs == [rec[4] for rec in sv["anc_records"]] + [rec[3] for rec in sv["readout_records"]]


@pytest.mark.parametrize("gates", ["cnot", "cr"])
def test_delayed_register_equals_parallel(gates):
    """Fig. 2: one reused ancilla (d + 1 qubits) against d - 1 ancillas measured in parallel
    (2d - 1 qubits), every noise term on: same syndromes, readout, sampled Paulis, amplitudes."""
    n = D + D - 1
    for traj in range(8):
        a = run_trajectory(D, 3, gates, "reduced", NOISY, seed=5, traj=traj, want_state=True, code="repetition")
        b = run_trajectory(D, 3, gates, "unreduced", NOISY, seed=5, traj=traj, want_state=True, code="repetition")
        assert (a["syndromes"] == b["syndromes"]).all()
        assert (a["data_bits"] == b["data_bits"]).all()
        assert sorted(a["events"]) == sorted(b["events"])
        sa = a["state"].reshape(2, 1 << D)
        sb = b["state"].reshape(1 << (n - D), 1 << D)
        assert np.abs(sa[0] - sb[0]).max() < 1e-13
        assert np.abs(sa[1]).max() == 0 and np.abs(sb[1:]).max() == 0
