"""Serving: jobs admitted as memory frees up, overlapping on the device; every result equals
the same job run alone (and, for d=3, the oracle)."""
import numpy as np
import pytest

import workloads as W
from oracle import run_trajectory
from parity_util import TAU, compare_trajectory

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2204_11404_gb300.serve import Job, Server, latency_summary, state_bytes  # noqa: E402
from paper_2204_11404_gb300.simulator import Simulator  # noqa: E402


@pytest.mark.parametrize("policy", ["fifo", "sjf"])
def test_continuous_batching_results_equal_solo_runs(policy):
    trace = W.serving_trace(n_req=14, rate=200.0, seed=11, max_traj=3, precisions=("c64", "c64", "c128"))
    for j in trace:                          # keep d=5 complex128 jobs short
        if j["d"] == 5 and j["precision"] == "c128":
            j["rounds"] = 1
            j["n_traj"] = 1
    jobs = [Job(**j) for j in trace]
    budget = 2 * state_bytes(5, "c64") + state_bytes(5, "c128") // 2 + 64 * 2**20   # forces waiting
    srv = Server(budget, policy=policy)
    # complex128 at d=5 is served by the tensor-core complex128 engine; its solo runs below use the
    # FP64 CUDA-core engine, so the equality checks cover the two FP64-accurate engines against each
    # other.  complex64 at d=5 is served by the tensor-core complex64 engine, and its solo runs use the
    # same engine (the two complex64 engines agree only within FP32 roundings).
    assert [srv.engine(j) for j in jobs if j.d == 5 and j.precision == "c128"] == \
        ["c128tc"] * sum(j.d == 5 and j.precision == "c128" for j in jobs)
    assert [srv.engine(j) for j in jobs if j.d == 5 and j.precision == "c64"] == \
        ["c64tc"] * sum(j.d == 5 and j.precision == "c64" for j in jobs)
    try:
        srv.run(jobs)
    finally:
        srv.close()
    assert all(j.t_done is not None for j in jobs)
    admits = [t for (t, ev, _) in srv.log if ev == "admit"]
    dones = [t for (t, ev, _) in srv.log if ev == "done"]
    assert admits and dones and min(dones) < max(admits)   # later jobs admitted while others ran
    for j in jobs:
        solo = srv.engine(j) if j.precision == "c64" else j.precision
        with Simulator(j.d, j.rounds, j.gates, solo, **j.noise) as sim:
            syn, bits, log = sim.run(j.seed, j.first_traj, j.n_traj)
        assert (syn == j.syndromes).all() and (bits == j.data_bits).all() and (log == j.raw_logical).all()
        if j.d == 3:
            for t in range(j.n_traj):
                o = run_trajectory(3, j.rounds, j.gates, "reduced", j.noise, seed=j.seed, traj=j.first_traj + t)
                assert compare_trajectory(syn[t], bits[t], o, TAU[j.precision]) in ("exact", "ambiguous")
    s = latency_summary(jobs)
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_job_larger_than_budget_rejected():
    srv = Server(1 << 20)
    try:
        with pytest.raises(ValueError):
            srv.run([Job(jid=0, d=5, rounds=1, n_traj=1, precision="c64", noise={}, seed=0)], realtime=False)
    finally:
        srv.close()
