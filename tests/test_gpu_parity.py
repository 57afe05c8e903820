"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Sampled Pauli errors, syndromes and final data bits are compared bit for bit
(subject to the near-threshold rule in parity_util); amplitudes after the last
round within 1e-12 (complex128) and 2e-5 (complex64) max-abs.
"""
import numpy as np
import pytest

import workloads as W
from oracle import run_trajectory
from parity_util import AMP_TOL, TAU, compare_trajectory, min_margin, unambiguous

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2204_11404_gb300.simulator import Simulator  # noqa: E402


def oracle_traj(d, rounds, gates, noise, seed, traj, want_state=False):
    return run_trajectory(d, rounds, gates, "reduced", noise, seed=seed, traj=traj, want_state=want_state)


def check_batch(sim, d, rounds, gates, noise, seed, first, n, prec, oracle_idx=None):
    syn, bits, log = sim.run(seed, first, n)
    idx = range(n) if oracle_idx is None else oracle_idx
    kinds = []
    for i in idx:
        o = oracle_traj(d, rounds, gates, noise, seed, first + i)
        kinds.append(compare_trajectory(syn[i], bits[i], o, TAU[prec]))
        if kinds[-1] == "exact":
            assert log[i] == o["raw_logical"]
    return kinds


def test_d3_cnot_workload_matches_oracle():
    w = W.D3_CNOT
    with Simulator(w["d"], w["rounds"], w["gates"], "c128", **w["noise"]) as sim:
        kinds = check_batch(sim, w["d"], w["rounds"], w["gates"], w["noise"], w["seed"], 0, 200, "c128")
    assert kinds.count("exact") == len(kinds)


@pytest.mark.parametrize("gates", ["cnot", "cr"])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_d3_stress_matches_oracle(gates, prec):
    nz = W.STRESS
    with Simulator(3, 3, gates, prec, **nz) as sim:
        kinds = check_batch(sim, 3, 3, gates, nz, 31, 0, 60, prec)
        assert kinds.count("ambiguous") <= (0 if prec == "c128" else 2)
        sim.record_events(4096)
        # three trajectories whose oracle run has no near-threshold draw: every form must then
        # match outcomes exactly and amplitudes within its bar (no comparison is skipped)
        picked = unambiguous(lambda t: oracle_traj(3, 3, gates, nz, 31, t, want_state=True), range(3, 40), TAU[prec], 3)
        for traj, o in picked:
            syn, bits, log = sim.run(31, traj, 1)
            assert compare_trajectory(syn[0], bits[0], o, TAU[prec]) == "exact"
            ref = o["state"][: 1 << 9]
            assert np.abs(sim.state() - ref).max() < AMP_TOL[prec]
            ev = sorted(tuple(int(x) for x in e[1:]) for e in sim.events())
            assert all(int(e[0]) == traj for e in sim.events())
            assert ev == sorted(o["events"])



@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_d3_certain_noise_matches_oracle(prec):
    """Degenerate noise rates: p = 1 at every site (a Pauli at every step of every qubit) beside
    p = 0 for the idle steps, with the coherent terms on.  The occurrence test compares a 53-bit
    uniform with p, so p = 1 always fires and p = 0 never does; draws, syndromes, bits and the state
    must still match the oracle."""
    nz = dict(p1=1.0, p2=1.0, p_idle=0.0, theta_rx=0.1, phi_zz=0.05)
    with Simulator(3, 2, "cr", prec, **nz) as sim:
        kinds = check_batch(sim, 3, 2, "cr", nz, 37, 0, 24, prec)
        assert kinds.count("ambiguous") <= (0 if prec == "c128" else 2)
        sim.record_events(4096)
        [(traj, o)] = unambiguous(lambda t: oracle_traj(3, 2, "cr", nz, 37, t, want_state=True), range(24, 60), TAU[prec])
        syn, bits, log = sim.run(37, traj, 1)
        assert compare_trajectory(syn[0], bits[0], o, TAU[prec]) == "exact"
        assert np.abs(sim.state() - o["state"][: 1 << 9]).max() < AMP_TOL[prec]
        ev = sorted(tuple(int(x) for x in e[1:]) for e in sim.events())
        assert ev == sorted(o["events"]) and len(ev) > 0

def test_offsets_chunking_and_device_outputs():
    nz = W.STRESS
    n = 1100   # more than one internal batch
    with Simulator(3, 2, "cr", "c128", **nz) as sim:
        syn, bits, log = sim.run(5, 0, n)
        syn_a, bits_a, log_a = sim.run(5, 0, 600)
        syn_b, bits_b, log_b = sim.run(5, 600, n - 600)
        assert (np.concatenate([syn_a, syn_b]) == syn).all()
        assert (np.concatenate([bits_a, bits_b]) == bits).all()
        assert (np.concatenate([log_a, log_b]) == log).all()
        d_syn = torch.zeros((n, 3, 8), dtype=torch.uint8, device="cuda")
        d_bits = torch.zeros((n, 9), dtype=torch.uint8, device="cuda")
        d_log = torch.zeros((n,), dtype=torch.uint8, device="cuda")
        sim.run_device(5, 0, n, d_syn.data_ptr(), d_bits.data_ptr(), d_log.data_ptr())
        torch.cuda.synchronize()
        assert (d_syn.cpu().numpy() == syn).all()
        assert (d_bits.cpu().numpy() == bits).all()
        assert (d_log.cpu().numpy() == log).all()
        for i in (0, 599, 600, 1023, 1024, 1099):
            o = oracle_traj(3, 2, "cr", nz, 5, i)
            assert compare_trajectory(syn[i], bits[i], o, TAU["c128"]) == "exact"
        syn0, _, _ = sim.run(5, 0, 0)
        assert syn0.shape == (0, 3, 8)


@pytest.mark.parametrize("gates", ["cnot", "cr"])
def test_zero_rounds_samples_init_state(gates):
    with Simulator(3, 0, gates, "c128", **W.STRESS) as sim:
        syn, bits, log = sim.run(2, 0, 40)
        assert not syn.any()
        for i in range(40):
            o = oracle_traj(3, 0, gates, W.STRESS, 2, i)
            assert (bits[i] == o["data_bits"]).all() and log[i] == o["raw_logical"] == 0


def test_d5_noiseless_properties():
    with Simulator(5, 2, "cr", "c128") as sim:
        syn, bits, log = sim.run(0, 0, 2)
        assert not syn.any() and not log.any()
        psi = sim.state()
        assert abs(np.vdot(psi, psi).real - 1) < 1e-12
        # the code state has 2^12 equal-magnitude amplitudes (X-stabilizer orbit of a basis state)
        mags = np.abs(psi[np.abs(psi) > 1e-9])
        assert mags.size == 4096 and np.allclose(mags, 1 / 64, atol=1e-12)


_D5 = {}


def _d5_oracle():
    if "o" not in _D5:
        pt = W.D5_CR["points"][-1]          # p = 5e-3, theta_rx = 0.05, phi_zz = 0.02
        seed = W.D5_CR["seed_base"] + len(W.D5_CR["points"]) - 1
        _D5["o"] = (pt, seed, oracle_traj(5, 5, "cr", pt, seed, 0, want_state=True))
    return _D5["o"]


@pytest.mark.parametrize("prec", ["c128", "c64", "c64tc", "c128tc"])
def test_d5_full_size_trajectory_matches_oracle(prec):
    pt, seed, o = _d5_oracle()
    # this trajectory has no draw within 1e-4 of its probability (checked here), so every form,
    # complex64 included, must reproduce its outcomes exactly and its amplitudes within the bar
    assert min_margin(o) >= TAU[prec]
    with Simulator(5, 5, "cr", prec, **pt) as sim:
        sim.record_events(1 << 16)
        syn, bits, log = sim.run(seed, 0, 1)
        assert compare_trajectory(syn[0], bits[0], o, TAU[prec]) == "exact"
        ref = o["state"][: 1 << 25]
        _D5["err_" + prec] = float(np.abs(sim.state() - ref).max())
        assert np.abs(o["state"][1 << 25:]).max() == 0
        assert np.abs(sim.state() - ref).max() < AMP_TOL[prec]
        ev = sorted(tuple(int(x) for x in e[1:]) for e in sim.events())
        assert ev == sorted(o["events"])
        ms_prob, ms_apply, blk = sim_kernel_times(sim)
        assert ms_prob > 0 and ms_apply > 0 and blk >= 0


def sim_kernel_times(sim):
    from paper_2204_11404_gb300 import capi
    return capi.qec_kernel_times(sim.h)


TWIRLED = dict(W.STRESS, twirl=1, theta_rx=0.4, theta_rz=0.3, theta_rzx=0.3, phi_zz=0.2, round_rz=0.3, round_rx=0.25)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_d3_twirled_matches_oracle(prec):
    with Simulator(3, 3, "cr", prec, **TWIRLED) as sim:
        kinds = check_batch(sim, 3, 3, "cr", TWIRLED, 47, 0, 40, prec)
        assert kinds.count("ambiguous") <= (0 if prec == "c128" else 2)
        [(traj, o)] = unambiguous(lambda t: oracle_traj(3, 3, "cr", TWIRLED, 47, t, want_state=True), range(5, 40),
                                  TAU[prec])
        syn, bits, log = sim.run(47, traj, 1)
        assert compare_trajectory(syn[0], bits[0], o, TAU[prec]) == "exact"
        assert np.abs(sim.state() - o["state"][: 1 << 9]).max() < AMP_TOL[prec]


SIGN_FOLLOWS = dict(W.STRESS, theta_rx=0.35, overrot_follows=1)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_d3_sign_follows_variant_matches_oracle(prec):
    """Over-rotation R_X(-theta) after the Rx^dagger preparation (the flagged sign variant)."""
    with Simulator(3, 3, "cr", prec, **SIGN_FOLLOWS) as sim:
        kinds = check_batch(sim, 3, 3, "cr", SIGN_FOLLOWS, 53, 0, 40, prec)
        assert kinds.count("ambiguous") <= (0 if prec == "c128" else 2)


@pytest.mark.parametrize("prec,d,rounds,n,bar", [("c128", 3, 4, 16, 1e-13), ("c128", 5, 2, 1, 1e-13),
                                                 ("c64", 3, 4, 16, 4e-5)])
def test_speculative_pass_matches_probability_passes_and_oracle(prec, d, rounds, n, bar):
    """The FP64 and complex64 CUDA-core forms apply each block's guessed outcome (the same
    stabilizer's previous outcome) and re-apply from the untouched input where the drawn outcome
    differs.  On the stress noise (every trajectory's draws at least 2e-4 from their probabilities):
    against the FP64 oracle (outcomes identical, amplitudes within the form's bar), against the
    same form with each probability computed before its apply (identical outcomes, states within a
    few roundings), and one corrective apply per outcome change."""
    from paper_2204_11404_gb300 import capi
    pt = dict(W.STRESS)
    with Simulator(d, rounds, "cr", prec, **pt) as a:
        m0 = capi.qec_debug_speculation(a.h, 1)
        ra = a.run(77, 0, n)
        sa = a.state()
        m1 = capi.qec_debug_speculation(a.h, 0)
        rb = a.run(77, 0, n)
        sb = a.state()
    for x, y in zip(ra, rb):
        assert (x == y).all()
    assert np.abs(sa - sb).max() < bar
    changes = int(np.sum(np.diff(ra[0].astype(np.int8), axis=1) != 0))
    assert m1 - m0 == changes and changes > 0
    o = oracle_traj(d, rounds, "cr", pt, 77, n - 1, want_state=True)
    assert compare_trajectory(ra[0][n - 1], ra[1][n - 1], o, TAU[prec]) == "exact"
    assert np.abs(sa - o["state"][: 1 << (d * d)]).max() < AMP_TOL[prec]
