"""Batched form (many d=3 trajectories in one persistent launch) against the oracle and the
single-trajectory path: per-trajectory precision and noise, bit-exact outcomes (near-threshold
rule for complex64)."""
import numpy as np
import pytest

import workloads as W
from oracle import run_trajectory
from parity_util import AMP_TOL, TAU, compare_trajectory, unambiguous

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2204_11404_gb300.simulator import BatchSimulator, Simulator  # noqa: E402


@pytest.mark.parametrize("gates", ["cr", "cnot"])
def test_batched_mix_matches_oracle(gates):
    n = 96
    traj = [1000 + 7 * i for i in range(n)]
    kinds = ["c128" if i % 3 else "c64" for i in range(n)]
    rng = np.random.default_rng(3)
    noise = []
    for i in range(n):
        if i % 4 == 0:
            noise.append(dict(W.STRESS))
        else:
            p = float(rng.uniform(1e-4, 3e-2))
            noise.append(dict(p1=p, p2=p, p_idle=p, theta_rx=float(rng.uniform(0, 0.1)), phi_zz=0.02))
    with BatchSimulator(3, gates, max_traj=256) as b:
        syn, bits, log = b.run(77, traj, kinds, noise)
    amb = 0
    for i in range(n):
        o = run_trajectory(3, 3, gates, "reduced", noise[i], seed=77, traj=traj[i])
        kind = compare_trajectory(syn[i], bits[i], o, TAU[kinds[i]])
        if kinds[i] == "c128":
            assert kind == "exact"
        amb += kind == "ambiguous"
        if kind == "exact":
            assert log[i] == o["raw_logical"]
    assert amb <= 2


def test_batched_equals_single_trajectory_path_and_autotune():
    traj, kinds, noise, rounds, seed = W.batched_mix(n=512, unreduced=False)
    with BatchSimulator(rounds, "cr", max_traj=512) as b:
        w, ms = b.autotune(seed, traj, kinds, noise)
        assert w > 0 and ms > 0
        syn, bits, log = b.run(seed, traj, kinds, noise)
        syn2, bits2, log2 = b.run(seed, traj, kinds, noise)
    assert (syn == syn2).all() and (bits == bits2).all() and (log == log2).all()
    for i in (0, 1, 2, 3, 200, 511):
        with Simulator(3, rounds, "cr", kinds[i], **noise[i]) as sim:
            s1, b1, l1 = sim.run(seed, traj[i], 1)
        if kinds[i] == "c128":
            assert (s1[0] == syn[i]).all() and (b1[0] == bits[i]).all() and l1[0] == log[i]


@pytest.mark.parametrize("gates", ["cr", "cnot"])
def test_batched_unreduced_register_matches_oracle_and_reduced(gates):
    # 17-qubit time-ordered register in the same launch as 10-qubit trajectories
    n = 40
    traj = [300 + i for i in range(n)]
    kinds = ["c128u", "c64u", "c128", "c64"] * (n // 4)
    noise = [dict(W.STRESS) if i % 2 else dict(p1=0.02, p2=0.02, p_idle=0.01, theta_rx=0.08, phi_zz=0.03)
             for i in range(n)]
    for i in range(0, n, 3):                 # a third of them with twirled coherent terms
        noise[i] = dict(noise[i], twirl=1, theta_rx=0.4, phi_zz=0.2, round_rz=0.3)
    with BatchSimulator(3, gates, max_traj=64) as b:
        syn, bits, log = b.run(91, traj, kinds, noise)
    amb = 0
    for i in range(n):
        layout = "unreduced" if kinds[i].endswith("u") else "reduced"
        prec = kinds[i].rstrip("u")
        o = run_trajectory(3, 3, gates, layout, noise[i], seed=91, traj=traj[i])
        kind = compare_trajectory(syn[i], bits[i], o, TAU[prec])
        if prec == "c128":
            assert kind == "exact", (i, kinds[i])
        amb += kind == "ambiguous"
    assert amb <= 2


def test_batched_sign_follows_variant_matches_oracle():
    """Per-trajectory over-rotation sign variant, all four kinds in one launch."""
    n = 32
    traj = [500 + i for i in range(n)]
    kinds = ["c128u", "c64u", "c128", "c64"] * (n // 4)
    noise = [dict(p1=0.01, p2=0.01, p_idle=0.01, theta_rx=0.3, overrot_follows=i % 2) for i in range(n)]
    with BatchSimulator(3, "cr", max_traj=64) as b:
        syn, bits, log = b.run(93, traj, kinds, noise)
    amb = 0
    for i in range(n):
        layout = "unreduced" if kinds[i].endswith("u") else "reduced"
        prec = kinds[i].rstrip("u")
        o = run_trajectory(3, 3, "cr", layout, noise[i], seed=93, traj=traj[i])
        kind = compare_trajectory(syn[i], bits[i], o, TAU[prec])
        if prec == "c128":
            assert kind == "exact", (i, kinds[i])
        amb += kind == "ambiguous"
    assert amb <= 2


@pytest.mark.parametrize("gates", ["cr", "cnot"])
def test_batched_amplitudes_match_oracle(gates):
    """The state of one trajectory of each kind (10 and 17 qubits x complex128 and complex64),
    recorded inside a mixed batch, against the oracle's state of the same trajectory: within
    1e-12 (complex128) and 2e-5 (complex64) max-abs.  The unreduced register's data state (every
    ancilla |0> after the round) is compared with the oracle's unreduced run."""
    n = 48
    kinds = ["c128", "c64", "c128u", "c64u"] * (n // 4)
    noise = [dict(W.STRESS) if i % 2 else dict(p1=0.01, p2=0.01, p_idle=0.01, theta_rx=0.08, phi_zz=0.03)
             for i in range(n)]
    traj = [700 + i for i in range(n)]
    with BatchSimulator(3, gates, max_traj=64) as b:
        for k, kind in enumerate(("c128", "c64", "c128u", "c64u")):
            layout = "unreduced" if kind.endswith("u") else "reduced"
            prec = kind.rstrip("u")
            cand = [i for i in range(n) if kinds[i] == kind]
            [(item, o)] = unambiguous(
                lambda i: run_trajectory(3, 3, gates, layout, noise[i], seed=95, traj=traj[i], want_state=True),
                cand, TAU[prec])
            b.snapshot(item)
            syn, bits, log = b.run(95, traj, kinds, noise)
            assert compare_trajectory(syn[item], bits[item], o, TAU[prec]) == "exact"
            ref = o["state"][: 1 << 9]
            assert np.abs(o["state"][1 << 9:]).max() < 1e-15     # every ancilla |0> after the round
            err = np.abs(b.state() - ref).max()
            assert err < AMP_TOL[prec], (kind, err)
        b.snapshot(-1)


def test_unreduced_engine_fusion_widths_are_bit_identical_and_autotuned():
    """The 17-qubit engine applies consecutive gate units on disjoint slab bits in one pass of up to
    k bits; inside a pass every amplitude still sees the units in program order, so every fusion
    width and CTA size gives the same outcomes and the same state bits.  The autotuner then picks a
    configuration among them and reports it."""
    n = 24
    traj = [900 + i for i in range(n)]
    kinds = ["c128u", "c64u"] * (n // 2)
    noise = [dict(W.STRESS) if i % 3 else dict(W.STRESS, twirl=1, theta_rx=0.4, phi_zz=0.2) for i in range(n)]
    ref = None
    with BatchSimulator(3, "cr", max_traj=128) as b:
        for k in (2, 3, 4, 5, 6):
            for thr in (128, 256):
                b.set_config(8, k, thr)
                assert b.config() == (8, k, thr)
                b.snapshot(5)
                out = b.run(97, traj, kinds, noise)
                st = b.state()
                if ref is None:
                    ref = (out, st)
                    continue
                for x, y in zip(out, ref[0]):
                    assert (x == y).all(), (k, thr)
                assert np.array_equal(st.view(np.uint64), ref[1].view(np.uint64)), (k, thr)
        w, ms = b.autotune(97, traj * 4, kinds * 4, noise * 4)
        warps, k, thr = b.config()
        assert w == warps and 2 <= k <= 6 and thr in (128, 256) and ms > 0
    o = run_trajectory(3, 3, "cr", "unreduced", noise[5], seed=97, traj=traj[5], want_state=True)
    assert compare_trajectory(ref[0][0][5], ref[0][1][5], o, TAU["c64"]) in ("exact", "ambiguous")
