"""Tensor-core forms on d=5 trajectories (the tensor-core passes need 4096-amplitude tiles):
complex64 with weight-4 contractions in 3xTF32, and complex128 with weight-4 applications as
FP64-exact 8-bit-slice products on the FP16 tensor cores.  Checked against the FP64 oracle and
against the CUDA-core forms of the same storage."""
import numpy as np
import pytest

import workloads as W
from oracle import run_trajectory
from parity_util import AMP_TOL, TAU, compare_trajectory, min_margin

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2204_11404_gb300.simulator import Simulator  # noqa: E402


def test_tensor_core_form_matches_oracle_two_rounds():
    pt = dict(W.STRESS)
    o = run_trajectory(5, 2, "cr", "reduced", pt, seed=42, traj=3, want_state=True)
    # no draw of this trajectory lies within 1e-4 of its probability (margin 0.031), so the
    # complex64 form must match its outcomes exactly and its amplitudes within 2e-5
    assert min_margin(o) >= TAU["c64tc"]
    with Simulator(5, 2, "cr", "c64tc", **pt) as sim:
        syn, bits, log = sim.run(42, 3, 1)
        assert compare_trajectory(syn[0], bits[0], o, TAU["c64tc"]) == "exact"
        err = np.abs(sim.state() - o["state"][: 1 << 25]).max()
        assert err < AMP_TOL["c64tc"], err


def test_tensor_core_form_agrees_with_cuda_core_form():
    pts = W.D5_CR["points"]
    agree = 0
    for i in (2, 5, 8):
        with Simulator(5, 5, "cr", "c64tc", **pts[i]) as a, Simulator(5, 5, "cr", "c64", **pts[i]) as b:
            ra = a.run(2000 + i, 0, 2)
            rb = b.run(2000 + i, 0, 2)
            agree += int(all((x == y).all() for x, y in zip(ra, rb)))
            sa, sb = a.state(), b.state()
            assert np.abs(sa - sb).max() < 2 * AMP_TOL["c64"]
    assert agree >= 2


def test_emulated_fp64_form_matches_oracle_two_rounds():
    pt = dict(W.STRESS)
    o = run_trajectory(5, 2, "cr", "reduced", pt, seed=42, traj=3, want_state=True)
    with Simulator(5, 2, "cr", "c128tc", **pt) as sim:
        syn, bits, log = sim.run(42, 3, 1)
        assert compare_trajectory(syn[0], bits[0], o, TAU["c128tc"]) == "exact"
        err = np.abs(sim.state() - o["state"][: 1 << 25]).max()
        assert err < AMP_TOL["c128tc"], err


def test_emulated_fp64_form_agrees_with_fp64_form():
    """Same outcomes bit for bit, and states within a few FP64 roundings of each other."""
    pts = W.D5_CR["points"]
    for i in (0, 4, 8):
        with Simulator(5, 3, "cr", "c128tc", **pts[i]) as a, Simulator(5, 3, "cr", "c128", **pts[i]) as b:
            ra = a.run(2000 + i, 0, 2)
            rb = b.run(2000 + i, 0, 2)
            for x, y in zip(ra, rb):
                assert (x == y).all()
            assert np.abs(a.state() - b.state()).max() < 1e-13


def test_emulated_fp64_form_on_d3_uses_fp64_passes():
    """d=3 tiles are below 2^12 amplitudes: the form falls back to the FP64 passes, bit-identical."""
    pt = dict(W.STRESS)
    with Simulator(3, 3, "cr", "c128tc", **pt) as a, Simulator(3, 3, "cr", "c128", **pt) as b:
        ra = a.run(7, 0, 20)
        rb = b.run(7, 0, 20)
        for x, y in zip(ra, rb):
            assert (x == y).all()
        assert np.array_equal(a.state(), b.state())


def test_bounded_probability_pass_decides_like_the_exact_pass():
    """c128tc decides most outcomes from a 24-bit probability with a rigorous error bound (in the
    pass fused with the previous block's apply, and in the first block's own bounded pass).
    Sending every outcome through the exact pass instead changes no outcome and no amplitude bit
    (the exact pass decides the outcome but leaves the norm that renormalises the next apply), and
    the exact pass runs only when forced or when the bound leaves the outcome open (rare)."""
    from paper_2204_11404_gb300 import capi
    pts = W.D5_CR["points"]
    for i in (2, 8):
        with Simulator(5, 3, "cr", "c128tc", **pts[i]) as a:
            f0 = capi.qec_debug_exact_probability(a.h, 0)
            ra = a.run(3000 + i, 0, 2)
            sa = a.state()
            f1 = capi.qec_debug_exact_probability(a.h, 1)
            rb = a.run(3000 + i, 0, 2)
            sb = a.state()
            f2 = capi.qec_debug_exact_probability(a.h, 0)
        for x, y in zip(ra, rb):
            assert (x == y).all()
        assert np.array_equal(sa, sb)
        assert f2 - f1 == 2 * 3 * 24          # every noisy-round measurement, forced
        assert f1 - f0 <= 2                   # unforced: the bound decided (almost) every outcome


def test_emulated_fp64_form_is_bit_reproducible():
    """A rerun of the same trajectory, in the same simulator and in a new one, must give the same
    bits and the same amplitudes bit for bit: the passes' sums are reduced in a fixed order, and a
    tile skipped or done twice, or a mix-up of the two working states, would change the state."""
    pt = W.D5_CR["points"][7]
    with Simulator(5, 2, "cr", "c128tc", **pt) as a:
        r1 = a.run(91, 4, 1)
        s1 = a.state().copy()
        r2 = a.run(91, 4, 1)
        s2 = a.state().copy()
    with Simulator(5, 2, "cr", "c128tc", **pt) as b:
        r3 = b.run(91, 4, 1)
        s3 = b.state()
    for x, y, z in zip(r1, r2, r3):
        assert (x == y).all() and (x == z).all()
    assert np.array_equal(s1.view(np.uint64), s2.view(np.uint64))
    assert np.array_equal(s1.view(np.uint64), s3.view(np.uint64))


def test_fused_pass_matches_separate_passes_and_oracle_on_stress_noise():
    """The fused tensor-core pass (block s's apply and block s+1's probability on the same tiles)
    against the FP64 oracle on the stress noise at d=5, where every noise channel and coherent term
    is on: outcomes identical, amplitudes within 1e-12; and against the FP64 CUDA-core form on the
    same trajectories: identical outcomes, states within 1e-13."""
    pt = dict(W.STRESS)
    o = run_trajectory(5, 2, "cr", "reduced", pt, seed=42, traj=3, want_state=True)
    with Simulator(5, 2, "cr", "c128tc", **pt) as a, Simulator(5, 2, "cr", "c128", **pt) as b:
        ra = a.run(42, 3, 1)
        assert compare_trajectory(ra[0][0], ra[1][0], o, TAU["c128tc"]) == "exact"
        assert np.abs(a.state() - o["state"][: 1 << 25]).max() < AMP_TOL["c128tc"]
        ra = a.run(42, 10, 3)
        rb = b.run(42, 10, 3)
        for x, y in zip(ra, rb):
            assert (x == y).all()
        assert np.abs(a.state() - b.state()).max() < 1e-13


def test_fused_pass_on_repetition_code():
    """Weight-2 blocks in the fused pass (K (x) I over spectator qubits of the union tile): the
    d=25 repetition code against the FP64 CUDA-core form."""
    pt = dict(p1=0.01, p2=0.01, p_idle=0.01, theta_rx=0.05, phi_zz=0.02)
    with Simulator(25, 2, "cr", "c128tc", code="repetition", **pt) as a, \
            Simulator(25, 2, "cr", "c128", code="repetition", **pt) as b:
        ra = a.run(8, 0, 2)
        rb = b.run(8, 0, 2)
        for x, y in zip(ra, rb):
            assert (x == y).all()
        assert np.abs(a.state() - b.state()).max() < 1e-13


def _detections(syn):
    """Outcome changes of each stabilizer from one round to the next (the init round's row is 0)."""
    return int(np.sum(np.diff(syn.astype(np.int8), axis=1) != 0))


def test_speculative_pass_matches_oracle_with_corrections():
    """The speculative pass guesses each outcome from the same stabilizer's previous outcome; a
    wrong guess is re-applied from the untouched input.  On the stress noise (many detection events)
    the trajectory must still match the FP64 oracle: outcomes identical, amplitudes within 1e-12;
    and the corrective applies run exactly once per outcome change."""
    from paper_2204_11404_gb300 import capi
    pt = dict(W.STRESS)
    o = run_trajectory(5, 2, "cr", "reduced", pt, seed=42, traj=3, want_state=True)
    with Simulator(5, 2, "cr", "c128tc", **pt) as sim:
        m0 = capi.qec_debug_speculation(sim.h, 1)
        syn, bits, log = sim.run(42, 3, 1)
        misses = capi.qec_debug_speculation(sim.h, -1) - m0
        assert compare_trajectory(syn[0], bits[0], o, TAU["c128tc"]) == "exact"
        assert np.abs(sim.state() - o["state"][: 1 << 25]).max() < AMP_TOL["c128tc"]
    assert misses == _detections(syn) and misses > 0


@pytest.mark.parametrize("prec,bar", [("c128tc", 1e-13), ("c64tc", 4e-5)])
def test_speculative_pass_agrees_with_fused_pass(prec, bar):
    """The same trajectories with the speculative passes and with the fused apply +
    next-probability passes (bounded, for c128tc): identical outcomes, states within a few
    roundings, and one corrective apply per outcome change."""
    from paper_2204_11404_gb300 import capi
    pts = W.D5_CR["points"]
    for i in (1, 8):
        with Simulator(5, 3, "cr", prec, **pts[i]) as a:
            m0 = capi.qec_debug_speculation(a.h, 1)
            ra = a.run(5000 + i, 0, 2)
            sa = a.state()
            m1 = capi.qec_debug_speculation(a.h, 0)
            rb = a.run(5000 + i, 0, 2)
            sb = a.state()
            m2 = capi.qec_debug_speculation(a.h, 1)
        for x, y in zip(ra, rb):
            assert (x == y).all()
        assert np.abs(sa - sb).max() < bar
        assert m1 - m0 == _detections(ra[0])
        assert m2 == m1                       # the fused passes never correct


def test_speculation_hook_rejects_bad_mode():
    from paper_2204_11404_gb300 import capi
    with Simulator(3, 1, "cr", "c64tc", **W.STRESS) as a:
        for bad in (2, -2):
            with pytest.raises(capi.QecError):
                capi.qec_debug_speculation(a.h, bad)
        assert capi.qec_debug_speculation(a.h, 0) == 0
