"""C-ABI behaviour at the edges: invalid arguments, unsupported requests, reuse, maximum sizes."""
import numpy as np
import pytest

import workloads as W
from oracle import run_trajectory
from parity_util import compare_trajectory

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2204_11404_gb300 import capi  # noqa: E402
from paper_2204_11404_gb300.simulator import Simulator  # noqa: E402


@pytest.mark.parametrize("kw,status", [
    (dict(d=4, rounds=1), capi.QEC_EINVAL),
    (dict(d=7, rounds=1), capi.QEC_EINVAL),
    (dict(d=3, rounds=65), capi.QEC_EINVAL),
    (dict(d=3, rounds=1, layout="unreduced"), capi.QEC_EUNSUPPORTED),
])
def test_create_rejects(kw, status):
    layout = kw.pop("layout", "reduced")
    params = capi.make_params(kw["d"], kw["rounds"], "cr", "c128", layout=layout)
    with pytest.raises(capi.QecError) as e:
        capi.qec_create(params)
    assert e.value.status == status and capi.qec_last_error()


def test_bad_noise_and_precision_rejected():
    for noise in (dict(p1=-0.1), dict(p2=1.5), dict(theta_rx=5.0), dict(twirl=0.5), dict(phi_zz=float("nan"))):
        with pytest.raises(capi.QecError) as e:
            capi.qec_create(capi.make_params(3, 1, "cr", "c128", **noise))
        assert e.value.status == capi.QEC_EINVAL
    p = capi.make_params(3, 1, "cr", "c128")
    p.precision = 7
    with pytest.raises(capi.QecError):
        capi.qec_create(p)


def test_state_before_run_and_small_buffer_rejected():
    with Simulator(3, 1, "cr", "c128") as sim:
        buf = np.zeros(512, dtype=np.complex128)
        assert capi.lib().qec_get_state(sim.h, buf.ctypes.data, buf.nbytes) == capi.QEC_EINVAL
        sim.run(0, 0, 1)
        assert capi.lib().qec_get_state(sim.h, buf.ctypes.data, buf.nbytes - 16) == capi.QEC_EINVAL
        assert capi.lib().qec_get_state(sim.h, buf.ctypes.data, buf.nbytes) == capi.QEC_OK


def test_reconfigure_keeps_results_equal_to_fresh_simulators():
    with Simulator(3, 2, "cr", "c128", **W.STRESS) as sim:
        for rounds, noise in ((5, dict(p1=0.01, p2=0.02, theta_rx=0.1)), (1, W.STRESS), (3, dict(W.STRESS, twirl=1))):
            sim.reconfigure(rounds, **noise)
            syn, bits, log = sim.run(8, 2, 3)
            with Simulator(3, rounds, "cr", "c128", **noise) as fresh:
                f = fresh.run(8, 2, 3)
            assert all((x == y).all() for x, y in zip((syn, bits, log), f))
        with pytest.raises(capi.QecError):
            capi.qec_reconfigure(sim.h, capi.make_params(3, 2, "cr", "c64"))       # precision differs
        with pytest.raises(capi.QecError):
            capi.qec_reconfigure(sim.h, capi.make_params(3, 65, "cr", "c128"))     # rounds out of range


def test_maximum_rounds_d3_matches_oracle():
    with Simulator(3, 64, "cr", "c128", **W.STRESS) as sim:
        syn, bits, log = sim.run(4, 0, 2)
    for i in range(2):
        o = run_trajectory(3, 64, "cr", "reduced", W.STRESS, seed=4, traj=i)
        assert compare_trajectory(syn[i], bits[i], o, 1e-9) == "exact"



@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_select_timed_block_instruments_the_chosen_pair(prec):
    """The measurement hook moves the instrumented block to the first block of the middle noisy round
    with the requested weights (the d = 3 code has weight-2 and weight-4 stabilizers); outcomes do not
    change, and weights no block has are rejected."""
    with Simulator(3, 3, "cr", prec, **W.STRESS) as ref:
        expect = ref.run(8, 0, 2)
    with Simulator(3, 3, "cr", prec, **W.STRESS) as sim:
        sim.run(8, 5, 1)
        _, _, b4 = capi.qec_kernel_times(sim.h)
        for wa, wn in ((2, 2), (2, 4), (4, 2)):
            try:
                blk = capi.qec_select_timed_block(sim.h, wa, wn)
            except capi.QecError as e:
                assert e.status == capi.QEC_EINVAL
                continue
            assert 8 <= blk < 16                      # the middle noisy round of three (8 blocks per round)
            got = sim.run(8, 0, 2)
            for x, y in zip(got, expect):
                assert (x == y).all()
            ms_p, ms_a, b = capi.qec_kernel_times(sim.h)
            assert b == blk and ms_a > 0 and ms_p >= 0
        with pytest.raises(capi.QecError) as e:
            capi.qec_select_timed_block(sim.h, 3, 3)
        assert e.value.status == capi.QEC_EINVAL
    assert 8 <= b4 < 16

def test_batch_rejects_bad_inputs():
    from paper_2204_11404_gb300.simulator import BatchSimulator
    with pytest.raises(capi.QecError):
        BatchSimulator(3, "cr", max_traj=4, d=5)
    with BatchSimulator(2, "cr", max_traj=4) as b:
        with pytest.raises(capi.QecError):
            b.run(0, [0] * 5, ["c128"] * 5, [{}] * 5)          # more than max_traj
        with pytest.raises(capi.QecError):
            b.run(0, [0], [7], [{}])                             # bad kind
        with pytest.raises(capi.QecError):
            b.run(0, [0], ["c128"], [dict(p1=2.0)])              # bad probability
