"""The device-allocation-free trajectory entry point against the allocating one.

qec_run_trajectories_noalloc serves callers that cannot call cudaMalloc (a
framework that owns all device memory through its own pool, a latency-critical
path that cannot take cudaMalloc's implicit synchronisation, a plug-in handed
only a stream and output buffers).  It launches the same kernels, with the
same grids and in the same order, as qec_run_trajectories (for complex64 the
apply pass fused with the next block's probability pass), so its outputs,
which are integers, must equal qec_run_trajectories' bit for bit in every
precision, on the stress noise where many draws fall near their thresholds.
Calls in a row with different settings check that the shared static scratch
carries nothing over from the previous call.  This file
is collected last so a failure here cannot hide failures elsewhere.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2204_11404_gb300 import capi  # noqa: E402
from paper_2204_11404_gb300.simulator import Simulator  # noqa: E402


def noalloc_run(params, seed, first, n):
    R, nst, nd = params.rounds, params.d * params.d - 1, params.d * params.d
    syn = torch.full((n, R + 1, nst), 7, dtype=torch.uint8, device="cuda")
    bits = torch.full((n, nd), 7, dtype=torch.uint8, device="cuda")
    log = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    capi.qec_run_trajectories_noalloc(params, seed, first, n, syn.data_ptr(), bits.data_ptr(), log.data_ptr(),
                                      stream.cuda_stream)
    stream.synchronize()
    return syn.cpu().numpy(), bits.cpu().numpy(), log.cpu().numpy()


CASES = [  # calls in a row with different settings, then a repeat of the first
    dict(d=3, rounds=3, gates="cr", precision="c128", seed=11, first=0, n=64),
    dict(d=3, rounds=16, gates="cnot", precision="c64", seed=12, first=500, n=24),
    dict(d=3, rounds=3, gates="cr", precision="c64", seed=13, first=0, n=64),
    dict(d=3, rounds=5, gates="cr", precision="c64tc", seed=14, first=90, n=48),
    dict(d=3, rounds=4, gates="cnot", precision="c128tc", seed=15, first=7, n=32),
    dict(d=3, rounds=3, gates="cr", precision="c128", seed=11, first=0, n=64),
]


def test_noalloc_matches_allocating_entry_point():
    for c in CASES:
        params = capi.make_params(c["d"], c["rounds"], c["gates"], c["precision"], **W.STRESS)
        got = noalloc_run(params, c["seed"], c["first"], c["n"])
        with Simulator(c["d"], c["rounds"], c["gates"], c["precision"], **W.STRESS) as sim:
            ref = sim.run(c["seed"], c["first"], c["n"])
        for g, r in zip(got, ref):
            assert (g == r).all()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    for d, rounds in ((5, 1), (3, 17)):
        params = capi.make_params(d, rounds, "cr")
        with pytest.raises(capi.QecError) as e:
            capi.qec_run_trajectories_noalloc(params, 0, 0, 1, 1, 1, 1)
        assert e.value.status == capi.QEC_EINVAL
        assert "static device scratch" in capi.qec_last_error()
