"""Failure detection without a GPU fault: a bounded device wait that runs out (a barrier that
nothing arrives on) reports QEC_ETIMEOUT through the status word, and the context stays usable."""
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


def test_bounded_wait_times_out_and_context_survives():
    with Simulator(3, 2, "cr", "c128", **W.STRESS) as sim:
        assert capi.qec_selftest_wait(sim.h, 20000) == capi.QEC_ETIMEOUT
        assert "gave up" in capi.qec_last_error()
        syn, bits, log = sim.run(3, 0, 4)        # the simulator and the context still work
        for i in range(4):
            o = run_trajectory(3, 2, "cr", "reduced", W.STRESS, seed=3, traj=i)
            assert compare_trajectory(syn[i], bits[i], o, 1e-9) == "exact"
        assert capi.qec_selftest_wait(sim.h, 0) == capi.QEC_EINVAL
