"""ctypes wrapper of the C state-vector core; runs one trajectory end to end.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import ctypes
import os
import subprocess

import numpy as np

from .circuit import Trajectory, logical_parity

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libsvoracle.so")
_lib = None

OP_DTYPE = np.dtype([("type", "<i4"), ("q0", "<i4"), ("q1", "<i4"), ("flag", "<i4"),
                     ("u", "<f8"), ("m", "<f8", (32,))])


def build_core(force=False):
    """Compile sv_core.c with gcc (OpenMP) into oracle/_build/libsvoracle.so."""
    src = os.path.join(_HERE, "sv_core.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_core())
        _lib.sv_run.restype = ctypes.c_int64
        _lib.sv_run.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_void_p, ctypes.c_void_p]
        _lib.sv_set_threads.argtypes = [ctypes.c_int]
        _lib.sv_get_threads.restype = ctypes.c_int
    return _lib


def set_threads(t):
    lib().sv_set_threads(int(t))


def get_threads():
    return int(lib().sv_get_threads())


def encode_ops(ops):
    arr = np.zeros(len(ops), dtype=OP_DTYPE)
    for i, op in enumerate(ops):
        if op[0] == "U1":
            arr[i]["type"], arr[i]["q0"] = 1, op[1]
            m = op[2].reshape(-1)
            arr[i]["m"][0:8:2], arr[i]["m"][1:8:2] = m.real, m.imag
        elif op[0] == "U2":
            arr[i]["type"], arr[i]["q0"], arr[i]["q1"] = 2, op[1], op[2]
            m = op[3].reshape(-1)
            arr[i]["m"][0:32:2], arr[i]["m"][1:32:2] = m.real, m.imag
        else:  # ("M", qubit, u, forced, reset)
            arr[i]["type"], arr[i]["q0"], arr[i]["q1"], arr[i]["flag"] = 3, op[1], op[4], op[3]
            arr[i]["u"] = op[2]
    return arr


def run_ops(psi, n, ops):
    """Apply encoded ops to psi (complex128, length 2^n) in place; return (outcomes, p1s)."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == (1 << n)
    arr = encode_ops(ops)
    nm = sum(1 for o in ops if o[0] == "M")
    outs = np.zeros(max(nm, 1), dtype=np.int32)
    p1s = np.zeros(max(nm, 1), dtype=np.float64)
    r = lib().sv_run(psi.ctypes.data, n, arr.ctypes.data, len(arr), outs.ctypes.data, p1s.ctypes.data)
    if r < 0:
        raise RuntimeError("measurement with zero-weight kept branch at op %d" % (-r - 1))
    return outs[:nm], p1s[:nm]


def run_trajectory(d, rounds, gates="cr", layout="reduced", noise=None, seed=0, traj=0,
                   inject=None, want_state=False, code="surface"):
    """Simulate one trajectory.  Returns a dict with syndromes [rounds+1][d^2-1] (row 0 is the
    forced init round), data_bits [d^2], raw_logical, events (sampled Paulis), the per-measurement
    records (u, P(1), outcome) and, if want_state, the state after the last round (before readout)."""
    T = Trajectory(d, rounds, gates, layout, noise, seed, traj, inject, code).build()
    if T.n > 30:
        raise ValueError("register too large for the oracle")
    psi = np.zeros(1 << T.n, dtype=np.complex128)
    psi[0] = 1.0
    cut = T.readout_start()
    outs, p1s = run_ops(psi, T.n, T.ops[:cut])
    state = psi.copy() if want_state else None
    ro_outs, ro_p1 = run_ops(psi, T.n, T.ops[cut:])
    nst = T.nstab
    syn = np.zeros((rounds + 1, nst), dtype=np.uint8)
    recs = []
    for (kind, rnd, k, offset, u), o, p in zip(T.meas[:len(outs)], outs, p1s):
        syn[rnd, k] = int(o) ^ offset
        recs.append((rnd, k, u, float(p), int(o)))
    data_bits = np.asarray(ro_outs, dtype=np.uint8)
    ro_recs = [(j, m[4], float(p), int(o)) for j, (m, o, p) in enumerate(zip(T.meas[len(outs):], ro_outs, ro_p1))]
    return {
        "syndromes": syn,
        "data_bits": data_bits,
        "raw_logical": logical_parity(d, data_bits, code),
        "events": list(T.events),
        "anc_records": recs,
        "readout_records": ro_recs,
        "state": state,
        "n_qubits": T.n,
    }
