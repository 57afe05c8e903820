"""Benchmark: d=5 rotated-surface-code noisy QEC rounds per second on GB300.

Workload (one "step" = one trajectory of the whole hot path): d=5 reduced
register (25 data qubits resident + the ancilla, 2^26 amplitudes of the
d^2+1 register), cross-resonance gate set, 5 noisy rounds after the noise-free
init round, final Z readout; the 9 noise points p in {1e-3, 3e-3, 5e-3} x
theta_rx in {0, 0.01, 0.05}, ZZ crosstalk 0.02, taken in turn by successive
steps.  value = noisy rounds / s over the timed steps (inputs resident in HBM,
outputs left in device memory); e2e = the same through the host-output call.

Multi-GPU (torchrun): trajectories are independent; each rank runs its own
trajectory indices with no data-path collective (weak scaling).

--impl reference times the FP64 CPU oracle on the host cores, on bounded
samples of the same workload (one stabilizer circuit of a d=5 round per step).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "d=5 QEC rounds/s (26-qubit SV), HBM GB/s vs peak; serve p50/p99 latency"
UNIT = "rounds/s"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2070 MHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=9)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="c128tc", choices=["c128", "c64", "c64tc", "c128tc"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--code", default="surface", choices=["surface", "repetition"],
                    help="repetition: the d=25 line code of Fig. 2 (same 25-qubit register, 24 stabilizers); "
                         "no CPU baseline")
    ap.add_argument("--points", type=int, default=9, help="noise points used (1..9); fewer = smaller device footprint")
    ap.add_argument("--workload", default="d5", choices=["d5", "batched", "serve", "precision", "sweep"],
                    help="d5: the d=5 26-qubit trajectories (default); batched: 8192 d=3 trajectories per "
                         "launch; serve: Poisson trace of mixed jobs through the continuous-batching server")
    ap.add_argument("--requests", type=int, default=32, help="serve: requests in the trace")
    ap.add_argument("--rate", type=float, default=50.0, help="serve: mean arrival rate (requests/s)")
    ap.add_argument("--max-traj", type=int, default=64, help="serve: trajectories per request drawn from 1..max")
    ap.add_argument("--sustainable-requests", type=int, default=20,
                    help="serve: requests in the second trace, at 0.7 of the capacity the first one measured")
    ap.add_argument("--no-serve", action="store_true", help="d5: skip the serving trace added to the line")
    ap.add_argument("--mem-gib", type=float, default=32.0, help="serve: device memory budget for state vectors")
    ap.add_argument("--policy", default="sjf", choices=["fifo", "sjf"],
                    help="serve: admission order of waiting jobs (shortest aged estimated work first, or arrival order)")
    ap.add_argument("--kinds", default="c128,c64,c128u,c64u",
                    help="batched: the kinds kept from the 8192-trajectory mix (comma-separated; a subset runs "
                         "fewer trajectories)")
    ap.add_argument("--config", default=None,
                    help="batched: W,K,T = reduced-engine warps per CTA, unreduced fusion width, unreduced threads "
                         "per CTA, instead of the autotuner's choice")
    ap.add_argument("--noise", default="full", choices=["full", "idle", "twirl", "follows"],
                    help="sweep: full = p on every step (Eqs. 1-2); idle = p on waiting qubits only; "
                         "twirl = full with the coherent terms replaced by their Pauli twirl")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---- clocks ---------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---- oracle (CPU baseline / reference arm) -----------------------------------------------------
class OracleSampler:
    """The FP64 oracle on bounded samples of the d=5 workload: stabilizer circuits of a noisy round
    (the ops between two ancilla measurements, measurement included) on a resident 26-qubit state
    that starts from the code state (the oracle's own noise-free init round)."""

    def __init__(self, point_index=8):
        import numpy as np

        from oracle.circuit import Trajectory
        from oracle.runner import build_core, get_threads, run_ops

        build_core()
        self.run_ops, self.threads = run_ops, get_threads()
        pt = W.D5_CR["points"][point_index]
        T = Trajectory(5, 1, "cr", "reduced", pt, W.D5_CR["seed_base"] + point_index, 0).build()
        self.n, self.nstab = T.n, 24
        groups, cur = [], []
        for op in T.ops:
            cur.append(op)
            if op[0] == "M" and op[4] == 1:
                groups.append(cur)
                cur = []
        self.init_ops = [op for g in groups[: self.nstab] for op in g]
        self.blocks = groups[self.nstab: 2 * self.nstab]
        self.psi = np.zeros(1 << self.n, dtype=np.complex128)
        self.psi[0] = 1.0
        self.run_ops(self.psi, self.n, self.init_ops)
        self.next = 0

    def run(self, n_samples):
        t0 = time.perf_counter()
        for _ in range(n_samples):
            self.run_ops(self.psi, self.n, self.blocks[self.next % self.nstab])
            self.next += 1
        return time.perf_counter() - t0


def reference_arm(args, rank, world):
    if rank != 0:
        return
    smp = OracleSampler()
    smp.run(args.warmup)
    secs = smp.run(args.steps)
    nst, threads = args.steps, smp.threads
    rounds = nst / 24.0
    value = rounds / secs
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%d stabilizer circuits (with measurement) of a d=5 cr noisy round, "
                                   "p=5e-3 theta_rx=0.05 phi_zz=0.02, on a resident 2^26 FP64 state; "
                                   "rounds = circuits / 24" % nst},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def workload_config(args, world):
    if args.code == "repetition":
        return {"workload": "d=25 one-dimensional repetition code (Fig. 2), reduced 26-qubit register (25 data "
                            "resident + ancilla), cr gate set, 5 noisy rounds + init + Z readout, 9 noise points "
                            "(p x theta_rx) with ZZ 0.02",
                "d": 25, "code": "repetition", "rounds": 5, "precision": args.precision,
                "trajectories_per_rank": args.steps, "parallelism": "trajectory-sharded x%d" % world,
                "l2": "state 512 MiB (c128) / 256 MiB (c64) per pass > 129 MB L2, no flush needed"}
    return {"workload": "d=5 rotated surface code, reduced 26-qubit register (25 data resident + ancilla), "
                        "cr gate set, 5 noisy rounds + init + Z readout, 9 noise points "
                        "(p x theta_rx) with ZZ 0.02",
            "d": 5, "rounds": 5, "precision": args.precision, "trajectories_per_rank": args.steps,
            "parallelism": "trajectory-sharded x%d" % world,
            "l2": "state 512 MiB (c128) / 256 MiB (c64) per pass > 129 MB L2, no flush needed"}


# ---- native arm ------------------------------------------------------------------------------
def traffic_record(precision):
    """dram bytes per launch of the apply pass from the committed ncu summary, if it was taken
    on the current kernel source (sha256 of kernels.cu and ozaki.cuh); else None."""
    path = os.path.join(ROOT, "profiles", "apply_pass_traffic.json")
    try:
        rec = json.load(open(path)).get(precision, {})
    except (OSError, ValueError):
        return None
    if rec.get("source_sha256") != kernel_source_sha():
        return None
    return rec.get("dram_bytes_per_launch")


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("kernels.cu", "ozaki.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2204_11404_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def native_arm(args, rank, world, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2204_11404_gb300 import capi
    from paper_2204_11404_gb300.shard import interleaved_index
    from paper_2204_11404_gb300.simulator import Simulator

    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    pts = W.D5_CR["points"][: max(1, min(args.points, len(W.D5_CR["points"])))]
    R = W.D5_CR["rounds"]
    dd = 25 if args.code == "repetition" else 5   # 25 data qubits and 24 stabilizers either way
    # every run is ordered after and before this stream (through the handle's events), so the CUDA
    # events of the timed region, recorded on it, bracket all of the simulators' work (torch's
    # default stream is the legacy stream, handle 0, which the C ABI reads as "no stream")
    bstream = torch.cuda.Stream()
    sims = [Simulator(dd, R, "cr", args.precision, stream=bstream.cuda_stream, code=args.code, **pt) for pt in pts]
    seeds = [W.D5_CR["seed_base"] + i for i in range(len(pts))]
    nst = 24
    syn = torch.empty((1, R + 1, nst), dtype=torch.uint8, device="cuda")
    bits = torch.empty((1, 25), dtype=torch.uint8, device="cuda")
    log = torch.empty((1,), dtype=torch.uint8, device="cuda")

    def traj_index(i):
        return interleaved_index(i, len(pts), rank, world)

    def step(i):
        j = i % len(pts)
        sims[j].run_device(seeds[j], traj_index(i), 1, syn.data_ptr(), bits.data_ptr(), log.data_ptr())

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    stream = bstream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fb0 = [capi.qec_debug_exact_probability(s.h, -1) for s in sims] if args.precision == "c128tc" else None
    sm0 = [capi.qec_debug_speculation(s.h, -1) for s in sims]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(args.steps):
            step(args.warmup + i)
        e1.record(stream)
        torch.cuda.synchronize()
    # the instrumented block's device times, from event-record nodes inside each simulator's
    # trajectory graph (its most recent trajectory), read after the timed region
    used = sorted({(args.warmup + i) % len(pts) for i in range(args.steps)})
    kt = [capi.qec_kernel_times(sims[j].h) for j in used]
    fallbacks = (sum(capi.qec_debug_exact_probability(s.h, -1) for s in sims) - sum(fb0)) if fb0 else None
    misses = sum(capi.qec_debug_speculation(s.h, -1) for s in sims) - sum(sm0)
    if world > 1:
        dist.barrier()
    secs = e0.elapsed_time(e1) / 1e3
    if world > 1:
        t = torch.tensor([secs], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        secs = float(t.item())
    rounds = world * args.steps * R
    value = rounds / secs

    # e2e through the host-output call (inputs: seed + trajectory index; outputs copied to host),
    # over as many trajectories as the timed steps
    n_e2e = args.steps
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    for i in range(n_e2e):
        j = i % len(pts)
        sims[j].run(seeds[j], 10_000 + traj_index(i), 1)
    e2e_secs = time.perf_counter() - h0
    if world > 1:
        t = torch.tensor([e2e_secs], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_secs = float(t.item())
    e2e = {"value": world * n_e2e * R / e2e_secs, "unit": UNIT,
           "h2d_bytes_per_step": 32, "d2h_bytes_per_step": (R + 1) * nst + 25 + 1}

    # roofline of the dominant kernel: the pass that applies a weight-4 block (psi <- K_m psi / sqrt(N));
    # in the complex64 forms it also computes the next block's probability (fused: one read + one
    # write of the register per stabilizer); in the complex128 forms it applies the guessed outcome's
    # operator and sums |in|^2 and |out|^2 for the decision (one read + one write)
    ms_prob = float(np.mean([k[0] for k in kt]))
    ms_apply = float(np.mean([k[1] for k in kt]))
    amps = 1 << 25
    # 16x16 complex mat-vec per 16 amplitudes: 16 cmacs/amp; the FP64 speculative pass adds |in|^2 and
    # |out|^2 (2 FMA each per amplitude)
    flops_apply = amps * (16 * 8 + (8 if args.precision == "c128" else 0))
    bytes_apply = amps * (32 if args.precision in ("c128", "c128tc") else 16)
    if args.precision == "c128":
        roof = {"bound": "alu", "achieved": flops_apply / (ms_apply * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s"}
    else:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        roof = {"bound": "hbm", "achieved": bytes_apply / (ms_apply * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # the fused pass of a pair of two weight-2 blocks (a quarter of the stabilizer pairs at d = 5),
    # instrumented on three more trajectories after the timed region
    if args.code == "surface" and args.precision != "c128":
        blk = capi.qec_select_timed_block(sims[0].h, 2, 2)
        ms22 = []
        for t in range(3):
            sims[0].run_device(seeds[0], 20_000 + t, 1, syn.data_ptr(), bits.data_ptr(), log.data_ptr())
            ms22.append(capi.qec_kernel_times(sims[0].h)[1])
        ms22 = float(np.median(ms22))
        roof["weight2_pair"] = {
            "kernel": {"c64": "k_fused_spec<2,false> (weight-2 block)", "c64tc": "k_fused_spec<2,false> (CUDA cores)",
                       "c128tc": "k_ozs<false> (weight-2 block as K (x) I)"}[args.precision],
            "block": blk, "ms": ms22, "achieved": bytes_apply / (ms22 * 1e-3) / 1e9,
            "frac": bytes_apply / (ms22 * 1e-3) / 1e9 / roof["peak"], "unit": "GB/s"}
    roof["traffic"] = traffic_record(args.precision)
    roof["kernel"] = {"c128": "k_apply_spec<4,false> (FP64: speculative apply of a weight-4 block, the outcome "
                              "guessed from the previous round, + FP64 |in|^2 and |out|^2 sums, 2^25 amplitudes)",
                      "c64": "k_fused_spec<4,false> (FP32: speculative apply of a weight-4 block, the outcome guessed "
                             "from the previous round, + |in|^2 and |out|^2 sums, 2^25 amplitudes)",
                      "c64tc": "k_fused_tc_spec<false> (tcgen05 3xTF32: speculative apply of a weight-4 block, the "
                               "outcome guessed from the previous round, + |in|^2 and |out|^2 sums, 2^25 amplitudes)",
                      "c128tc": "k_ozs<false> (tcgen05: speculative apply of a weight-4 block, the outcome guessed "
                                "from the previous round, as FP64-exact 8-bit-slice products + bounded |in|^2 and "
                                "|out|^2 sums on the same tiles, 2^25 amplitudes)",
                      }[args.precision]
    if args.code == "repetition":
        roof["kernel"] = roof["kernel"].replace("weight-4 block", "weight-2 block Z_k Z_(k+1)")
    roof["ms_apply"] = ms_apply
    roof["ms_prob"] = ms_prob
    roof["apply_hbm_gbs"] = bytes_apply / (ms_apply * 1e-3) / 1e9
    roof["timed_blocks"] = len(kt)

    # launches per trajectory: instantiate; the complex64 forms: the first block's probability pass,
    # per later block one fused pass, the last block's apply; the complex128 forms: per block the
    # speculative pass and the corrective launch (returns at once unless the guess was wrong), with
    # the exact-probability launch between them on the tensor cores (returns at once unless the
    # bound left the outcome open); the readout (3)
    S = nst * R
    launches_per_traj = {"c128": 1 + 2 * S + 3, "c128tc": 1 + 3 * S + 3,
                         "c64": 1 + 2 * S + 3, "c64tc": 1 + 2 * S + 3}[args.precision]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"c128": "f64", "c64": "f32", "c64tc": "tf32x3",
                                                                 "c128tc": "f64 (fp16 slices)"}[args.precision],
        "data": "synthetic", "config": workload_config(args, world), "clocks": clk.summary(),
        "e2e": e2e, "gpu_launches": launches_per_traj * args.steps, "roofline": roof,
    }
    if fallbacks is not None:   # measurements the bound left open (exact pass run), of S per trajectory
        out["exact_probability_passes"] = {"count": fallbacks, "measurements": S * args.steps}
    # outcomes that differed from the guess (corrective apply run)
    out["speculation"] = {"corrective_applies": misses, "measurements": S * args.steps}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.code == "surface":
        from oracle.runner import set_threads

        smp = OracleSampler()
        secs_o = smp.run(24)
        set_threads(1)   # the same oracle on one core: 2 of the round's 24 circuits, scaled to a round
        secs_1 = smp.run(2) * 12
        set_threads(smp.threads)
        out["cpu_baseline"] = {"value": 1.0 / secs_o, "unit": UNIT, "cores": smp.threads, "kind": "oracle",
                               "sample": "one d=5 cr noisy round (24 stabilizer circuits with measurement), "
                                         "p=5e-3 theta_rx=0.05 phi_zz=0.02, on a resident 2^26 FP64 state",
                               "value_1_core": 1.0 / secs_1,
                               "sample_1_core": "2 of the same round's stabilizer circuits on one thread, x 12"}
    for s in sims:
        s.close()
    if not args.no_serve and args.code == "surface":   # serve p50/p99 (the metric's third part)
        rep = serve_measure(args, rank, world, local)
        rep.pop("out_bytes", None)
        out["serve"] = rep
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def batched_arm(args, rank, world, local):
    """8192 d=3 reduced-register trajectories (half complex128, half complex64, per-trajectory p and
    theta) per step, one persistent launch; the CTA shape is autotuned on a 1024-trajectory sample."""
    import torch

    from paper_2204_11404_gb300.simulator import BatchSimulator

    torch.cuda.set_device(local)
    traj, kinds, noise, rounds, seed = W.batched_mix(n=8192)
    traj = [t + rank * 8192 for t in traj]
    keep = set(args.kinds.split(","))
    sel = [i for i in range(len(traj)) if kinds[i] in keep]
    traj, kinds, noise = [traj[i] for i in sel], [kinds[i] for i in sel], [noise[i] for i in sel]
    with BatchSimulator(rounds, "cr", max_traj=8192) as b:
        if args.config:
            b.set_config(*(int(x) for x in args.config.split(",")))
        else:
            b.autotune(seed, traj[:1024], kinds[:1024], noise[:1024])
        warps, fusion_k, u_threads = b.config()
        for _ in range(args.warmup):
            b.run(seed, traj, kinds, noise)
        dev_ms = []
        with ClockSampler(local) as clk:
            h0 = time.perf_counter()
            for _ in range(args.steps):
                b.run(seed, traj, kinds, noise)
                dev_ms.append(b.last_ms())
            wall = time.perf_counter() - h0
    dev = sum(dev_ms) / 1e3
    n = len(traj)
    out = {
        "metric": "batched d=3 trajectories/s (one persistent launch: 10q/17q x c128/c64 mix)",
        "value": world * n * args.steps / dev,
        "unit": "trajectories/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dev / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": "8192 d=3 trajectories per step in equal quarters: reduced 10-qubit and "
                               "unreduced 17-qubit registers x complex128/complex64; 3 rounds, cr gates, "
                               "p~U[1e-4,1e-2], theta_rx~U[0,0.1]",
                   ("configured" if args.config else "autotuned"): {
                       "reduced_warps_per_cta": warps, "unreduced_fusion_width": fusion_k,
                       "unreduced_threads_per_cta": u_threads,
                       "sample": "--config" if args.config else
                                 "the first 1024 trajectories, each engine on its own register's"},
                   "kinds": args.kinds,
                   "rounds_per_s": world * n * rounds * args.steps / dev},
        "clocks": clk.summary(),
        "e2e": {"value": world * n * args.steps / wall, "unit": "trajectories/s",
                "h2d_bytes_per_step": n * (8 + 4 + 72) + 16, "d2h_bytes_per_step": n * ((rounds + 1) * 8 + 9 + 1)},
        "gpu_launches": 2 * args.steps,   # per step: the 10-qubit and the 17-qubit persistent kernels
    }
    if rank == 0:
        print(json.dumps(out))


def serve_measure(args, rank, world, local):
    """A Poisson trace of mixed jobs (the serving configuration: d in {3, 5}, rounds U{1..10},
    trajectories U{1..max_traj}, complex64 or complex128, per-job noise) through the continuous-batching
    server, then a second trace at 0.7 of the capacity the first one measured.  Returns the report."""
    import torch

    from paper_2204_11404_gb300.serve import Job, Server, latency_summary

    torch.cuda.set_device(local)
    warm = [Job(**j) for j in W.serving_trace(n_req=4, rate=1e6, seed=1, max_traj=1)]
    trace = W.serving_trace(n_req=args.requests, rate=args.rate, seed=5000 + rank, max_traj=args.max_traj)
    jobs = [Job(**j) for j in trace]
    srv = Server(int(args.mem_gib * 2**30), policy=args.policy)
    try:
        srv.run(warm)
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            srv.run(jobs)
            makespan = time.perf_counter() - t0
    finally:
        srv.close()
    traj = sum(j.n_traj for j in jobs)
    tr_rounds = sum(j.n_traj * j.rounds for j in jobs)
    span = max(j.arrival for j in jobs)
    out_bytes = sum(j.n_traj * ((j.rounds + 1) * (j.d * j.d - 1) + j.d * j.d + 1) for j in jobs)
    offered = tr_rounds / span if span > 0 else None
    rep = {"trace": "Poisson arrivals, d in {3,5}, rounds U{1..10}, trajectories U{1..%d}, c64/c128 "
                    "(d=5 on the tensor-core engines), p~U[1e-4,1e-2], theta_rx~U[0,0.1]"
                    % args.max_traj,
           "requests": len(jobs), "rate_per_s": args.rate, "trajectories": traj,
           "trajectories_per_s": world * traj / makespan, "makespan_s": makespan,
           "latency_ms": latency_summary(jobs),
           "offered_trajectory_rounds_per_s": offered, "achieved_trajectory_rounds_per_s": tr_rounds / makespan,
           "mem_budget_gib": args.mem_gib, "policy": args.policy, "clocks": clk.summary(), "out_bytes": out_bytes}
    # second trace at a sustainable rate: utilisation about 0.7 of the capacity the first one measured
    if offered and args.sustainable_requests > 0:
        rate2 = 0.7 * args.rate * (tr_rounds / makespan) / offered
        jobs2 = [Job(**j) for j in W.serving_trace(n_req=args.sustainable_requests, rate=rate2, seed=6000 + rank,
                                                    max_traj=args.max_traj)]
        srv = Server(int(args.mem_gib * 2**30), policy=args.policy)
        try:
            t1 = time.perf_counter()
            srv.run(jobs2)
            span2 = time.perf_counter() - t1
        finally:
            srv.close()
        tr2 = sum(j.n_traj * j.rounds for j in jobs2)
        rep["sustainable_trace"] = {"rate_per_s": rate2, "utilisation_target": 0.7, "requests": len(jobs2),
                                    "offered_trajectory_rounds_per_s": tr2 / max(j.arrival for j in jobs2),
                                    "achieved_trajectory_rounds_per_s": tr2 / span2,
                                    "latency_ms": latency_summary(jobs2)}
    return rep


def serve_arm(args, rank, world, local):
    rep = serve_measure(args, rank, world, local)
    out = {
        "metric": "serving: trajectories/s with p50/p99 job latency (continuous batching)",
        "value": rep["trajectories_per_s"], "unit": "trajectories/s", "n_gpus": world, "steps": rep["requests"],
        "warmup": 4, "ms_per_step": 1e3 * rep["makespan_s"] / rep["requests"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": rep["trace"], "requests": rep["requests"], "rate_per_s": args.rate,
                   "mem_budget_gib": args.mem_gib, "policy": args.policy,
                   "offered_trajectory_rounds_per_s": rep["offered_trajectory_rounds_per_s"],
                   "achieved_trajectory_rounds_per_s": rep["achieved_trajectory_rounds_per_s"]},
        "latency_ms": rep["latency_ms"], "clocks": rep["clocks"],
        "e2e": {"value": rep["trajectories_per_s"], "unit": "trajectories/s",
                "h2d_bytes_per_step": 32, "d2h_bytes_per_step": rep["out_bytes"] / rep["requests"]},
        "sustainable_trace": rep.get("sustainable_trace"),
    }
    if rank == 0:
        print(json.dumps(out))


def _oracle_state_file(point_index, rounds, path):
    """Worker (spawned process): trajectory 0 of a d=5 noise point on the FP64 oracle; saves the
    state after the last round and the smallest |u - P(1)| of the trajectory; returns the path."""
    import numpy as np

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle import run_trajectory
    from parity_util import min_margin

    pt = W.D5_CR["points"][point_index]
    o = run_trajectory(5, rounds, "cr", "reduced", pt, seed=W.D5_CR["seed_base"] + point_index, traj=0,
                       want_state=True)
    np.save(path, o["state"][: 1 << 25])
    return path, min_margin(o), o["syndromes"].tolist(), o["data_bits"].tolist()


def precision_arm(args, rank, world, local):
    """Error of every form against the FP64 oracle, per noise point of the d=5 workload: trajectory 0
    of each point on the oracle (a spawned worker on the host cores, overlapping the GPU work) against
    the same trajectory in complex128, complex128 on the tensor cores, complex64 and complex64 on the
    tensor cores (max |psi - psi_oracle| after the last round, and whether the outcomes match); then
    --steps trajectories per point in the three fast forms: how many have outcomes identical to the
    tensor-core complex128 form (itself bit-identical to the oracle), and the decoded logical error
    rates."""
    import multiprocessing
    import tempfile

    ctx = multiprocessing.get_context("spawn")   # started before the first GPU call
    pool = ctx.Pool(1)
    tmp = tempfile.mkdtemp(prefix="qec_prec_")
    R = W.D5_CR["rounds"]
    npts = max(1, min(args.points, len(W.D5_CR["points"])))
    futs = [pool.apply_async(_oracle_state_file, (i, R, os.path.join(tmp, "o%d.npy" % i))) for i in range(npts)]
    pool.close()
    import numpy as np
    import torch

    from paper_2204_11404_gb300.decoder import Decoder
    from paper_2204_11404_gb300.simulator import Simulator

    torch.cuda.set_device(local)
    n = max(1, args.steps)
    dec = Decoder(5)
    rows = []
    t0 = time.perf_counter()
    for i in range(npts):
        pt = W.D5_CR["points"][i]
        seed = W.D5_CR["seed_base"] + i
        row = {"p": pt["p1"], "theta_rx": pt["theta_rx"], "phi_zz": pt["phi_zz"]}
        # (1) the same trajectories in the fast forms, outcomes against the tensor-core complex128 form
        res = {}
        for prec in ("c128tc", "c64", "c64tc"):
            with Simulator(5, R, "cr", prec, **pt) as sim:
                res[prec] = sim.run(seed, 0, n)
        ref = res["c128tc"]
        row["trajectories"] = n
        row["pL"] = {prec: dec.logical_error_rate(*res[prec]) for prec in res}
        row["identical_outcomes_to_c128tc"] = {
            prec: int(sum(bool((res[prec][0][t] == ref[0][t]).all() and (res[prec][1][t] == ref[1][t]).all())
                          for t in range(n))) for prec in ("c64", "c64tc")}
        # (2) trajectory 0 of every form against the oracle
        path, margin, o_syn, o_bits = futs[i].get()
        psi_o = np.load(path)
        os.remove(path)
        row["oracle_min_margin"] = margin
        row["amp_maxabs_vs_oracle"] = {}
        row["outcomes_equal_oracle"] = {}
        for prec in ("c128", "c128tc", "c64", "c64tc"):
            with Simulator(5, R, "cr", prec, **pt) as sim:
                syn, bits, _ = sim.run(seed, 0, 1)
                same = bool((syn[0] == np.array(o_syn)).all() and (bits[0] == np.array(o_bits)).all())
                row["outcomes_equal_oracle"][prec] = same
                row["amp_maxabs_vs_oracle"][prec] = float(np.abs(sim.state() - psi_o).max()) if same else None
        del psi_o
        rows.append(row)
        print("point %d done after %.0f s" % (i, time.perf_counter() - t0), file=sys.stderr, flush=True)
    pool.join()
    if rank == 0:
        print(json.dumps({"metric": "error of each form against the FP64 oracle per noise point (d=5, %d rounds)" % R,
                          "unit": "per-point report", "data": "synthetic", "points": rows,
                          "bars": {"c128": 1e-12, "c128tc": 1e-12, "c64": 2e-5, "c64tc": 2e-5},
                          "decoder_fallbacks": dec.fallbacks}))


def sweep_arm(args, rank, world, local):
    """Logical error rate p_L over (p, c) at d=5, 5 rounds (Sec. III.B-C) and the effective-model fit
    p_eff = (1 + alpha c^2) p.  Over-rotation theta = 2 c sqrt(p) after every rotation gate (Rx, Rx^dagger,
    Rz and the two-qubit Rzx, each about its own generator), p on every step, decoded by the host
    matcher; complex64 tensor-core form.  --steps trajectories at p = 3e-3, scaled by 3e-3 / p below
    it so that each point sees a similar number of failures."""
    import numpy as np
    import torch

    from paper_2204_11404_gb300.decoder import Decoder, count_failures
    from paper_2204_11404_gb300.effective import bootstrap_alpha, fit_effective_model
    from paper_2204_11404_gb300.simulator import Simulator

    torch.cuda.set_device(local)
    n0 = max(1, args.steps)
    dec = Decoder(5)
    rows = []
    cs = (0.0,) if args.noise == "idle" else (0.0, 0.25, 0.5, 0.75, 1.0)
    for c in cs:
        for p in (1e-3, 2e-3, 3e-3, 5e-3):
            n = n0 * max(1, int(round(3e-3 / p)))
            th = 2 * c * np.sqrt(p)
            g = 0.0 if args.noise == "idle" else p
            nz = dict(p1=g, p2=g, p_idle=p, theta_rx=th, theta_rz=th, theta_rzx=th,
                      twirl=1.0 if args.noise == "twirl" else 0.0,
                      overrot_follows=1.0 if args.noise == "follows" else 0.0)
            with Simulator(5, 5, "cr", "c64tc", **nz) as sim:
                syn, bits, log = sim.run(7000, rank * n, n)
            # unit weights, and log-likelihood weights estimated from this point's detection events
            k, kw = count_failures(dec, syn, bits, log)
            if world > 1:
                import torch.distributed as dist
                t = torch.tensor([k, kw], dtype=torch.int64, device="cuda")
                dist.all_reduce(t)
                k, kw = (int(v) for v in t.tolist())
            nt = n * world
            rows.append({"c": c, "p": p, "trajectories": nt, "failures": k, "pL": k / nt,
                         "pL_err": float(np.sqrt(max(k, 1) * (1 - k / nt)) / nt),
                         "failures_weighted": kw, "pL_weighted": kw / nt,
                         "paper_fit_c0": 6.5e5 * p ** 2.92 if c == 0 else None})
    out = {"metric": "logical error rate p_L(p, c), d=5, 5 rounds, noise=" + args.noise, "unit": "per-point report",
           "data": "synthetic", "points": rows, "decoder_fallbacks": dec.fallbacks}
    if len(cs) > 1:
        try:
            fit = fit_effective_model(rows)
            sd, (lo, hi) = bootstrap_alpha(rows)
            out["effective_model"] = {"fit_range_p": [1e-3, 3e-3], "A": fit.A, "xi": fit.xi,
                                      "B": {str(c): b for c, b in fit.B.items()}, "alpha": fit.alpha,
                                      "alpha_spread": sd, "alpha_16_84": [lo, hi],
                                      "paper": {"A": 6.5e5, "xi": 2.92, "alpha": 0.872}}
        except ValueError as e:
            out["effective_model"] = {"error": str(e)}
        try:   # the same fit on the log-likelihood-weighted failure counts
            rows_w = [dict(r, failures=r["failures_weighted"]) for r in rows]
            fit_w = fit_effective_model(rows_w)
            out["effective_model_weighted_decoder"] = {"A": fit_w.A, "xi": fit_w.xi, "alpha": fit_w.alpha,
                                                       "alpha_16_84": list(bootstrap_alpha(rows_w)[1])}
        except ValueError as e:
            out["effective_model_weighted_decoder"] = {"error": str(e)}
    if rank == 0:
        print(json.dumps(out))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
    elif args.workload == "batched":
        batched_arm(args, rank, world, local)
    elif args.workload == "serve":
        serve_arm(args, rank, world, local)
    elif args.workload == "precision":
        precision_arm(args, rank, world, local)
    elif args.workload == "sweep":
        sweep_arm(args, rank, world, local)
    else:
        native_arm(args, rank, world, local)


if __name__ == "__main__":
    main()
