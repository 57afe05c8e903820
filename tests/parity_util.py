"""Comparison helpers for GPU-vs-oracle parity (shared by the GPU tests and the smoke check)."""
import numpy as np

# Near-threshold rule: a measurement whose oracle probability is within TAU of its uniform may
# legitimately come out differently under another summation order; such a trajectory is
# compared only up to that measurement.
TAU = {"c128": 1e-9, "c64": 1e-4, "c64tc": 1e-4, "c128tc": 1e-9}
AMP_TOL = {"c128": 1e-12, "c64": 2e-5, "c64tc": 2e-5, "c128tc": 1e-12}


def measurement_sequence(o):
    """(outcome-as-reported, u, P(1)) for every measurement of an oracle trajectory, in time order."""
    seq = []
    offs = {}
    for (rnd, k, u, p1, out) in o["anc_records"]:
        seq.append((("syn", rnd, k), out, u, p1))
    for (j, u, p1, out) in o["readout_records"]:
        seq.append((("bit", j), out, u, p1))
    return seq


def compare_trajectory(gpu_syn, gpu_bits, o, tau):
    """Returns 'exact' or 'ambiguous'; raises AssertionError on a real mismatch."""
    syn_o, bits_o = o["syndromes"], o["data_bits"]
    if (gpu_syn == syn_o).all() and (gpu_bits == bits_o).all():
        return "exact"
    for key, out, u, p1 in measurement_sequence(o):
        if key[0] == "syn":
            same = gpu_syn[key[1], key[2]] == syn_o[key[1], key[2]]
        else:
            same = gpu_bits[key[1]] == bits_o[key[1]]
        if not same:
            assert abs(u - p1) < tau, "mismatch at %s: u=%.17g P(1)=%.17g" % (key, u, p1)
            return "ambiguous"
    raise AssertionError("outputs differ but no measurement differs")


def min_margin(o):
    """Smallest |u - P(1)| over every measurement of an oracle trajectory (ancillas and readout).
    A trajectory whose margin is at least TAU[form] has no draw that another summation order may
    legitimately decide differently, so its outcomes and amplitudes must match outright."""
    m = [abs(u - p1) for (rnd, _, u, p1, _) in o["anc_records"] if rnd > 0]   # round 0: outcomes forced
    m += [abs(u - p1) for (_, u, p1, _) in o["readout_records"]]
    return min(m) if m else float("inf")


def unambiguous(oracle_fn, candidates, tau, count=1):
    """The first `count` trajectory indices among `candidates` whose oracle run (oracle_fn(traj),
    computed with want_state=True) has no near-threshold draw; returns [(traj, oracle result)]."""
    out = []
    for t in candidates:
        o = oracle_fn(t)
        if min_margin(o) >= tau:
            out.append((t, o))
            if len(out) == count:
                return out
    raise AssertionError("no trajectory without a near-threshold draw among %r" % (list(candidates),))
