"""Serving loop with continuous batching of trajectory jobs.

Jobs of different distance, rounds, noise and precision arrive over time.
The server keeps a pool of resident simulator slots, one per (d, gate set,
precision) state layout, each on its own CUDA stream.  A slot holds the
working state vector and the resident init code state: 2 x 2^(d^2)
amplitudes, which is 1 GiB for d=5 complex128 and 0.5 GiB for d=5 complex64.

Admission:
- a job is admitted as soon as a free slot of its layout exists, or the memory
  budget has room for a new slot;
- an idle slot of another layout may be freed to make room;
- waiting jobs are scanned in arrival order, so a small job is not blocked
  behind a large one that does not fit yet.

Scheduling:
- light jobs (d = 3, kilobyte registers) run on high-priority streams and are
  admitted at once;
- heavy jobs (d = 5) are capped at `max_heavy` running at a time.  One d = 5
  pass already fills the GPU, so running more of them concurrently only
  time-slices the same throughput and delays every one of them.

Admitted jobs run concurrently on their slots' streams, so their kernels
overlap on the GPU.  A slot is re-pointed at a new job's noise and round count
without recomputing its code state (qec_reconfigure).  Results do not depend
on what else is running: every draw is keyed by (seed, trajectory index).
"""
import time
from dataclasses import dataclass, field

import numpy as np

from .simulator import Simulator


@dataclass
class Job:
    jid: int
    d: int
    rounds: int
    n_traj: int
    precision: str
    noise: dict
    seed: int
    first_traj: int = 0
    gates: str = "cr"
    arrival: float = 0.0          # seconds after the trace starts
    t_admit: float = None
    t_done: float = None
    syndromes: np.ndarray = None
    data_bits: np.ndarray = None
    raw_logical: np.ndarray = None

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.arrival


def state_bytes(d, precision):
    """Device bytes of one slot: two working states (the speculative passes) + the resident init
    state."""
    return 3 * (1 << (d * d)) * (16 if precision.startswith("c128") else 8)


@dataclass
class Slot:
    key: tuple
    sim: Simulator
    stream: object
    nbytes: int
    job: Job = None
    outs: tuple = None
    event: object = None
    last_used: float = field(default_factory=time.perf_counter)


class Server:
    """fp64_on_tensor_cores: complex128 jobs with d >= 5 run on the tensor-core complex128 engine
    ("c128tc": the same outcomes, amplitudes within a few FP64 roundings, about 10x faster); False
    keeps them on the FP64 CUDA-core engine.  fp32_on_tensor_cores: complex64 jobs with d >= 5 run on
    the tensor-core complex64 engine ("c64tc": 3xTF32 products with FP32 accumulation, within the
    complex64 tolerance of the oracle, about 1.2x faster); False keeps them on the FP32 CUDA cores.
    policy: the order in which waiting jobs are admitted as slots and memory free up: "sjf" (shortest
    estimated work first, `work`, aged: a job's work counts divided by 1 + its wait / sjf_aging_s, so
    that long jobs are not held back indefinitely by a stream of short ones) or "fifo" (arrival
    order)."""

    # relative device time of one trajectory-round per engine at d = 5 (measured rounds/s: c128tc 102,
    # c64tc 346, c64 261, c128 13.8); d = 3 jobs are far cheaper and run beside the heavy ones
    COST_D5 = {"c128tc": 1.0 / 102, "c64tc": 1.0 / 346, "c64": 1.0 / 261, "c128": 1.0 / 13.8}

    def __init__(self, mem_budget_bytes, device=0, max_heavy=2, heavy_d=5, fp64_on_tensor_cores=True,
                 fp32_on_tensor_cores=True, policy="sjf", sjf_aging_s=30.0):
        import torch

        self.torch = torch
        self.device = device
        self.budget = int(mem_budget_bytes)
        self.max_heavy = int(max_heavy)
        self.heavy_d = int(heavy_d)
        self.fp64_on_tensor_cores = bool(fp64_on_tensor_cores)
        self.fp32_on_tensor_cores = bool(fp32_on_tensor_cores)
        if policy not in ("fifo", "sjf"):
            raise ValueError("policy must be 'fifo' or 'sjf'")
        self.policy = policy
        self.sjf_aging_s = float(sjf_aging_s)
        lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
        self.prio_light = min(lo, hi)      # numerically lower = higher priority
        self.prio_heavy = max(lo, hi)
        self.slots = []
        self.used = 0
        self.log = []       # (time, event, job id)

    # ---- slots ----------------------------------------------------------------------------
    def _free_slot(self, slot):
        slot.sim.close()
        self.slots.remove(slot)
        self.used -= slot.nbytes

    def engine(self, job):
        """The simulator precision that serves a job's requested precision."""
        if job.precision == "c128" and job.d >= 5 and self.fp64_on_tensor_cores:
            return "c128tc"
        if job.precision == "c64" and job.d >= 5 and self.fp32_on_tensor_cores:
            return "c64tc"
        return job.precision

    def work(self, job):
        """Estimated device seconds of a job on its engine (trajectories x rounds x cost per
        trajectory-round; d < 5 counted as 1/1000 of d = 5)."""
        per = self.COST_D5.get(self.engine(job), 0.1) * (1.0 if job.d >= 5 else 1e-3)
        return job.n_traj * (job.rounds + 1) * per

    def _acquire(self, job):
        eng = self.engine(job)
        key = (job.d, job.gates, eng)
        for s in self.slots:
            if s.key == key and s.job is None:
                return s
        need = state_bytes(job.d, eng)
        if need > self.budget:
            raise ValueError("job %d needs %d bytes, more than the whole budget" % (job.jid, need))
        if self.used + need > self.budget:
            idle = sorted((s for s in self.slots if s.job is None), key=lambda s: s.last_used)
            freed = 0
            victims = []
            for s in idle:
                if self.used - freed + need <= self.budget:
                    break
                victims.append(s)
                freed += s.nbytes
            if self.used - freed + need > self.budget:
                return None
            for s in victims:
                self._free_slot(s)
        light = job.d < self.heavy_d
        stream = self.torch.cuda.Stream(device=self.device, priority=self.prio_light if light else self.prio_heavy)
        sim = Simulator(job.d, job.rounds, job.gates, eng, stream=stream.cuda_stream, **job.noise)
        slot = Slot(key, sim, stream, need)
        self.slots.append(slot)
        self.used += need
        return slot

    def _launch(self, job, slot, now):
        torch = self.torch
        sim = slot.sim
        sim.reconfigure(job.rounds, **job.noise)
        n, nst, nd = job.n_traj, job.d * job.d - 1, job.d * job.d
        with torch.cuda.stream(slot.stream):
            syn = torch.empty((n, job.rounds + 1, nst), dtype=torch.uint8, device="cuda")
            bits = torch.empty((n, nd), dtype=torch.uint8, device="cuda")
            log = torch.empty((n,), dtype=torch.uint8, device="cuda")
            sim.run_device(job.seed, job.first_traj, n, syn.data_ptr(), bits.data_ptr(), log.data_ptr())
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        slot.job, slot.outs, slot.event = job, (syn, bits, log), ev
        job.t_admit = now
        self.log.append((now, "admit", job.jid))

    def _poll(self, now):
        changed = False
        for slot in self.slots:
            if slot.job is not None and slot.event.query():
                job = slot.job
                job.syndromes, job.data_bits, job.raw_logical = (t.cpu().numpy() for t in slot.outs)
                job.t_done = now
                self.log.append((now, "done", job.jid))
                slot.job, slot.outs, slot.event = None, None, None
                slot.last_used = time.perf_counter()
                changed = True
        return changed

    # ---- trace ----------------------------------------------------------------------------
    def run(self, jobs, realtime=True):
        """Serve jobs (arrival times in seconds from now).  Returns the jobs with results and
        admission/completion times filled in."""
        pending = sorted(jobs, key=lambda j: j.arrival)
        waiting = []
        t0 = time.perf_counter()
        done = 0
        i = 0
        while done < len(jobs):
            now = time.perf_counter() - t0
            while i < len(pending) and (pending[i].arrival <= now or not realtime):
                waiting.append(pending[i])
                i += 1
            progressed = self._poll(time.perf_counter() - t0)
            still = []
            heavy_running = sum(1 for s in self.slots if s.job is not None and s.job.d >= self.heavy_d)
            if self.policy == "sjf":   # shortest aged estimated work first (ties: arrival order)
                waiting.sort(key=lambda j: (self.work(j) / (1.0 + max(0.0, now - j.arrival) / self.sjf_aging_s),
                                            j.arrival))
            for job in waiting:
                if job.d >= self.heavy_d and heavy_running >= self.max_heavy:
                    still.append(job)
                    continue
                slot = self._acquire(job)
                if slot is None:
                    still.append(job)
                    continue
                self._launch(job, slot, time.perf_counter() - t0)
                heavy_running += job.d >= self.heavy_d
                progressed = True
            waiting = still
            done = sum(1 for j in jobs if j.t_done is not None)
            if not progressed:
                time.sleep(0.0002)
        return jobs

    def close(self):
        for s in list(self.slots):
            self._free_slot(s)


def latency_summary(jobs):
    lat = np.array([j.latency for j in jobs])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
