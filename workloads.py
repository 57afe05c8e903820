"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle's callers.

Holds only inputs (code distance, rounds, gate set, noise parameters, seeds,
trajectory ranges); none of the method's arithmetic.
"""

# d=3, reduced 10-qubit register, CNOT gate set, 3 rounds, depolarizing p = 1e-3 after every
# gate, coherent RZ over-rotation 0.02 rad on every data qubit once per round; 1000 trajectories.
D3_CNOT = dict(d=3, rounds=3, gates="cnot", noise=dict(p1=1e-3, p2=1e-3, round_rz=0.02), seed=0, n_traj=1000)

# d=5, reduced 26-qubit register (2^26 amplitudes with the ancilla), cross-resonance gate set,
# 5 rounds; p in {1e-3, 3e-3, 5e-3} applied to every step (Eqs. 1-2), RX over-rotation theta in
# {0, 0.01, 0.05} rad, ZZ crosstalk exp(-i 0.02 ZZ) on every two-qubit gate; 100 trajectories
# per point, seed 2000 + point index.
D5_P = (1e-3, 3e-3, 5e-3)
D5_THETA = (0.0, 0.01, 0.05)


def d5_points():
    pts = []
    for p in D5_P:
        for th in D5_THETA:
            pts.append(dict(p1=p, p2=p, p_idle=p, theta_rx=th, phi_zz=0.02))
    return pts


D5_CR = dict(d=5, rounds=5, gates="cr", points=d5_points(), seed_base=2000, n_traj_per_point=100)

# Stress noise for parity tests: every noise channel and coherent term on, at rates that make
# most trajectories carry several errors.
STRESS = dict(p1=0.03, p2=0.03, p_idle=0.02, theta_rx=0.1, theta_rz=0.07, theta_rzx=0.05,
              phi_zz=0.08, round_rz=0.1, round_rx=0.05)


def batched_mix(n=8192, seed=4000, rounds=3, unreduced=True):
    """Config of the batched form: n trajectories of the d=3 register in equal quarters of
    reduced 10-qubit complex128, reduced complex64, unreduced 17-qubit complex128 and unreduced
    complex64 (interleaved), each with its own noise: p ~ U[1e-4, 1e-2] on every step (Eqs. 1-2)
    and an Rx over-rotation theta ~ U[0, 0.1] rad, drawn with numpy's seeded generator.
    unreduced=False keeps only the reduced register.  Returns (traj indices, kinds, noise dicts,
    rounds, seed)."""
    import numpy as np

    rng = np.random.default_rng(seed)
    p = rng.uniform(1e-4, 1e-2, n)
    th = rng.uniform(0.0, 0.1, n)
    cycle = ["c128", "c64", "c128u", "c64u"] if unreduced else ["c128", "c64"]
    kinds = [cycle[i % len(cycle)] for i in range(n)]
    noise = [dict(p1=float(p[i]), p2=float(p[i]), p_idle=float(p[i]), theta_rx=float(th[i])) for i in range(n)]
    return list(range(n)), kinds, noise, rounds, seed


def serving_trace(n_req=64, rate=50.0, seed=5000, max_traj=8, d_choices=(3, 5), precisions=("c64", "c128")):
    """Poisson arrivals (mean `rate` per second) of jobs: d from d_choices, rounds U{1..10},
    trajectories U{1..max_traj}, precision from `precisions`, noise p ~ U[1e-4, 1e-2] on every
    step and theta_rx ~ U[0, 0.1] rad, cross-resonance gate set.  Returns a list of dicts."""
    import numpy as np

    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_req))
    jobs = []
    for i in range(n_req):
        p = float(rng.uniform(1e-4, 1e-2))
        jobs.append(dict(jid=i, d=int(rng.choice(d_choices)), rounds=int(rng.integers(1, 11)),
                         n_traj=int(rng.integers(1, max_traj + 1)), precision=str(rng.choice(precisions)),
                         noise=dict(p1=p, p2=p, p_idle=p, theta_rx=float(rng.uniform(0, 0.1))),
                         seed=seed + i, first_traj=0, arrival=float(t[i])))
    return jobs
