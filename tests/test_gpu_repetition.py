"""The one-dimensional repetition code of Fig. 2 on the GPU (the paper's illustration of the
delayed register), against the FP64 oracle: d = 9 and 15 on every form, and d = 25, whose
25-qubit register is the d=5 surface code's size, on the tensor-core complex128 form."""
import numpy as np
import pytest

import workloads as W
from oracle import run_trajectory
from parity_util import AMP_TOL, TAU, compare_trajectory

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2204_11404_gb300.simulator import Simulator  # noqa: E402


def _oracle(d, rounds, gates, noise, seed, traj, want_state=False):
    return run_trajectory(d, rounds, gates, "reduced", noise, seed=seed, traj=traj, want_state=want_state,
                          code="repetition")


@pytest.mark.parametrize("gates", ["cr", "cnot"])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_d9_matches_oracle(gates, prec):
    nz = W.STRESS
    with Simulator(9, 3, gates, prec, code="repetition", **nz) as sim:
        syn, bits, log = sim.run(61, 0, 24)
        assert syn.shape == (24, 4, 8) and bits.shape == (24, 9)
        kinds = []
        for i in range(24):
            o = _oracle(9, 3, gates, nz, 61, i, want_state=(i == 23))
            kinds.append(compare_trajectory(syn[i], bits[i], o, TAU[prec]))
            if kinds[-1] == "exact":
                assert log[i] == o["raw_logical"]
        assert kinds.count("ambiguous") <= (0 if prec == "c128" else 2)
        if kinds[-1] == "exact":
            assert np.abs(sim.state() - o["state"][: 1 << 9]).max() < AMP_TOL[prec]


def test_d15_c64_matches_oracle():
    nz = dict(W.STRESS, overrot_follows=1)
    with Simulator(15, 2, "cr", "c64", code="repetition", **nz) as sim:
        syn, bits, log = sim.run(67, 0, 6)
        kinds = [compare_trajectory(syn[i], bits[i], _oracle(15, 2, "cr", nz, 67, i), TAU["c64"]) for i in range(6)]
        assert kinds.count("ambiguous") <= 1


def test_d25_tensor_core_form_matches_oracle():
    """25 data qubits: every Z_k Z_{k+1} block runs as K (x) I on the tensor cores."""
    pt = W.D5_CR["points"][-1]
    with Simulator(25, 1, "cr", "c128tc", code="repetition", **pt) as sim:
        syn, bits, log = sim.run(71, 0, 1)
        o = _oracle(25, 1, "cr", pt, 71, 0, want_state=True)
        assert compare_trajectory(syn[0], bits[0], o, TAU["c128tc"]) == "exact"
        assert log[0] == o["raw_logical"]
        assert np.abs(sim.state() - o["state"][: 1 << 25]).max() < AMP_TOL["c128tc"]


def test_d25_tensor_core_form_agrees_with_fp64_form():
    pt = W.D5_CR["points"][4]
    with Simulator(25, 3, "cr", "c128tc", code="repetition", **pt) as a, \
            Simulator(25, 3, "cr", "c128", code="repetition", **pt) as b:
        ra, rb = a.run(73, 0, 2), b.run(73, 0, 2)
        for x, y in zip(ra, rb):
            assert (x == y).all()
        assert np.abs(a.state() - b.state()).max() < 1e-13


@pytest.mark.parametrize("d", [11, 13])
def test_smallest_tensor_core_registers_agree_with_fp64_form(d):
    """d = 11: the whole register is one 2^11-amplitude tile (a single CTA runs each pass, and the
    bounded probability pass reduces one partial); d = 13: four tiles."""
    pt = dict(W.STRESS)
    with Simulator(d, 3, "cr", "c128tc", code="repetition", **pt) as a, \
            Simulator(d, 3, "cr", "c128", code="repetition", **pt) as b:
        ra, rb = a.run(79, 0, 6), b.run(79, 0, 6)
        for x, y in zip(ra, rb):
            assert (x == y).all()
        assert np.abs(a.state() - b.state()).max() < 1e-13
    o = _oracle(d, 3, "cr", pt, 79, 5)
    assert compare_trajectory(ra[0][5], ra[1][5], o, TAU["c128tc"]) == "exact"
