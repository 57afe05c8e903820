"""ctypes binding of include/qecsv.h: same names, argument marshalling only.

Every step of the simulation runs in libqecsv.so (CUDA kernels for sm_103a);
this module only converts arguments.  If the library is missing or fails to
load, importing a function raises: there is no CPU fallback.
"""
import ctypes
import os

from .build import LIB, build

QEC_OK, QEC_EINVAL, QEC_ENOMEM, QEC_ECUDA, QEC_ETIMEOUT, QEC_EUNSUPPORTED = 0, -1, -2, -3, -4, -6
QEC_LAYOUT_REDUCED, QEC_LAYOUT_UNREDUCED = 0, 1
QEC_GATES_CNOT, QEC_GATES_CR = 0, 1
QEC_CODE_SURFACE, QEC_CODE_REPETITION = 0, 1
QEC_C128, QEC_C64, QEC_C64_TC, QEC_C128_TC = 0, 1, 2, 3

NOISE_FIELDS = ("p1", "p2", "p_idle", "theta_rx", "theta_rz", "theta_rzx", "phi_zz", "round_rz", "round_rx", "twirl",
                "overrot_follows")


class qec_noise(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in NOISE_FIELDS]


class qec_params(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("rounds", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("gates", ctypes.c_int32), ("precision", ctypes.c_int32), ("code", ctypes.c_int32),
                ("noise", qec_noise)]


class QecError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("qecsv status %d: %s" % (status, msg))
        self.status = status


_lib = None
_P = ctypes.c_void_p
_U8P = ctypes.POINTER(ctypes.c_uint8)

SIGNATURES = {
    "qec_create": ([ctypes.POINTER(qec_params), _P, ctypes.POINTER(_P)], ctypes.c_int),
    "qec_run_trajectories": ([_P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _P, _P, _P], ctypes.c_int),
    "qec_run_trajectories_device": ([_P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _P, _P, _P], ctypes.c_int),
    "qec_state_len": ([_P], ctypes.c_uint64),
    "qec_reconfigure": ([_P, ctypes.POINTER(qec_params)], ctypes.c_int),
    "qec_get_state": ([_P, _P, ctypes.c_size_t], ctypes.c_int),
    "qec_record_events": ([_P, ctypes.c_uint32], ctypes.c_int),
    "qec_get_events": ([_P, _P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "qec_kernel_times": ([_P, _P, _P], ctypes.c_int),
    "qec_select_timed_block": ([_P, ctypes.c_int32, ctypes.c_int32, _P], ctypes.c_int),
    "qec_debug_unreduced_plan": ([ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_uint32, _P, _P, _P, _P, _P],
                                 ctypes.c_int),
    "qec_selftest_wait": ([_P, ctypes.c_uint32], ctypes.c_int),
    "qec_run_trajectories_noalloc": ([ctypes.POINTER(qec_params), ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                      _P, _P, _P, _P], ctypes.c_int),
    "qec_destroy": ([_P], ctypes.c_int),
    "qec_batch_create": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, _P, ctypes.POINTER(_P)],
                         ctypes.c_int),
    "qec_batch_run": ([_P, ctypes.c_uint64, ctypes.c_uint32, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "qec_batch_autotune": ([_P, ctypes.c_uint64, ctypes.c_uint32, _P, _P, _P, _P, _P], ctypes.c_int),
    "qec_batch_config": ([_P, _P, _P, _P], ctypes.c_int),
    "qec_batch_set_config": ([_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "qec_batch_snapshot": ([_P, ctypes.c_int64], ctypes.c_int),
    "qec_batch_get_state": ([_P, _P, ctypes.c_size_t], ctypes.c_int),
    "qec_batch_last_ms": ([_P, _P], ctypes.c_int),
    "qec_batch_destroy": ([_P], ctypes.c_int),
    "qec_last_error": ([], ctypes.c_char_p),
    "qec_debug_program": ([ctypes.POINTER(qec_params), _P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32),
                           _P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "qec_debug_blocks": ([ctypes.POINTER(qec_params), ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, _P, _P],
                         ctypes.c_int),
    "qec_debug_ozaki_gemm": ([_P, _P, ctypes.c_int32, ctypes.c_int32, _P], ctypes.c_int),
    "qec_debug_exact_probability": ([_P, ctypes.c_int32, _P], ctypes.c_int),
    "qec_debug_speculation": ([_P, ctypes.c_int32, _P], ctypes.c_int),
}


def lib(path=None):
    """Load libqecsv.so (building it in-tree if absent or stale)."""
    global _lib
    if _lib is None:
        p = path or os.environ.get("QECSV_LIB") or build()
        L = ctypes.CDLL(p)
        for name, (argtypes, restype) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = argtypes
            fn.restype = restype
        _lib = L
    return _lib


def check(status):
    if status != QEC_OK:
        raise QecError(status, lib().qec_last_error().decode(errors="replace"))
    return status


def make_params(d, rounds, gates="cr", precision="c128", layout="reduced", code="surface", **noise):
    p = qec_params()
    p.d, p.rounds = int(d), int(rounds)
    p.layout = {"reduced": QEC_LAYOUT_REDUCED, "unreduced": QEC_LAYOUT_UNREDUCED}[layout]
    p.gates = {"cnot": QEC_GATES_CNOT, "cr": QEC_GATES_CR}[gates]
    p.precision = {"c128": QEC_C128, "c64": QEC_C64, "c64tc": QEC_C64_TC, "c128tc": QEC_C128_TC}[precision]
    p.code = {"surface": QEC_CODE_SURFACE, "repetition": QEC_CODE_REPETITION}[code]
    for k, v in noise.items():
        if k not in NOISE_FIELDS:
            raise KeyError(k)
        setattr(p.noise, k, float(v))
    return p


def qec_create(params, cuda_stream=None):
    h = _P()
    check(lib().qec_create(ctypes.byref(params), cuda_stream, ctypes.byref(h)))
    return h


def qec_run_trajectories(sim, seed, first_traj, n, syndromes_ptr, data_bits_ptr, raw_logical_ptr):
    return check(lib().qec_run_trajectories(sim, seed, first_traj, n, syndromes_ptr, data_bits_ptr, raw_logical_ptr))


def qec_run_trajectories_device(sim, seed, first_traj, n, d_syn_ptr, d_bits_ptr, d_log_ptr):
    return check(lib().qec_run_trajectories_device(sim, seed, first_traj, n, d_syn_ptr, d_bits_ptr, d_log_ptr))


def qec_reconfigure(sim, params):
    return check(lib().qec_reconfigure(sim, ctypes.byref(params)))


def qec_state_len(sim):
    return int(lib().qec_state_len(sim))


def qec_get_state(sim, host_ptr, nbytes):
    return check(lib().qec_get_state(sim, host_ptr, nbytes))


def qec_record_events(sim, max_events):
    return check(lib().qec_record_events(sim, max_events))


def qec_get_events(sim, host_ptr, max_events):
    c = ctypes.c_uint32(0)
    check(lib().qec_get_events(sim, host_ptr, max_events, ctypes.byref(c)))
    return int(c.value)


def qec_kernel_times(sim):
    """(probability-pass ms, apply-pass ms, block index) of the instrumented block."""
    ms = (ctypes.c_float * 2)()
    blk = ctypes.c_int32(0)
    check(lib().qec_kernel_times(sim, ctypes.cast(ms, _P), ctypes.cast(ctypes.pointer(blk), _P)))
    return float(ms[0]), float(ms[1]), int(blk.value)


def qec_select_timed_block(sim, w_apply, w_next):
    """Instrument the first block of the middle noisy round with weight w_apply followed by one of
    weight w_next; returns its index."""
    blk = ctypes.c_int32(0)
    check(lib().qec_select_timed_block(sim, w_apply, w_next, ctypes.cast(ctypes.pointer(blk), _P)))
    return int(blk.value)


def qec_run_trajectories_noalloc(params, seed, first_traj, n, d_syn_ptr, d_bits_ptr, d_log_ptr, cuda_stream=None):
    """Device-allocation-free variant of qec_run_trajectories_device (d = 3, <= 16 rounds)."""
    return check(lib().qec_run_trajectories_noalloc(ctypes.byref(params), seed, first_traj, n, d_syn_ptr, d_bits_ptr,
                                                    d_log_ptr, cuda_stream))


def qec_batch_create(d, rounds, gates, max_traj, cuda_stream=None):
    h = _P()
    check(lib().qec_batch_create(d, rounds, gates, max_traj, cuda_stream, ctypes.byref(h)))
    return h


def qec_batch_run(b, seed, n, traj_ptr, kind_ptr, noise_ptr, syn_ptr, bits_ptr, log_ptr):
    return check(lib().qec_batch_run(b, seed, n, traj_ptr, kind_ptr, noise_ptr, syn_ptr, bits_ptr, log_ptr))


def qec_batch_autotune(b, seed, n, traj_ptr, kind_ptr, noise_ptr):
    w = ctypes.c_int32(0)
    ms = ctypes.c_float(0)
    check(lib().qec_batch_autotune(b, seed, n, traj_ptr, kind_ptr, noise_ptr, ctypes.cast(ctypes.pointer(w), _P),
                                   ctypes.cast(ctypes.pointer(ms), _P)))
    return int(w.value), float(ms.value)


def qec_batch_config(b):
    """(reduced-engine warps per CTA, unreduced-engine fusion width, unreduced-engine threads per CTA)."""
    v = [ctypes.c_int32(0) for _ in range(3)]
    check(lib().qec_batch_config(b, *[ctypes.cast(ctypes.pointer(x), _P) for x in v]))
    return tuple(int(x.value) for x in v)


def qec_batch_set_config(b, warps_per_cta, fusion_width, u_threads):
    return check(lib().qec_batch_set_config(b, warps_per_cta, fusion_width, u_threads))


def qec_batch_snapshot(b, item):
    return check(lib().qec_batch_snapshot(b, item))


def qec_batch_get_state(b, host_ptr, nbytes):
    return check(lib().qec_batch_get_state(b, host_ptr, nbytes))


def qec_batch_last_ms(b):
    ms = ctypes.c_float(0)
    check(lib().qec_batch_last_ms(b, ctypes.cast(ctypes.pointer(ms), _P)))
    return float(ms.value)


def qec_batch_destroy(b):
    return check(lib().qec_batch_destroy(b))


def qec_selftest_wait(sim, polls):
    """Returns the raw status (QEC_ETIMEOUT expected) without raising."""
    return int(lib().qec_selftest_wait(sim, polls))


def qec_destroy(sim):
    return check(lib().qec_destroy(sim))


def qec_last_error():
    return lib().qec_last_error().decode(errors="replace")


def qec_debug_program(params, ops_ptr, cap, block_ptr, block_cap):
    n_ops, n_blk = ctypes.c_uint32(0), ctypes.c_uint32(0)
    check(lib().qec_debug_program(ctypes.byref(params), ops_ptr, cap, ctypes.byref(n_ops), block_ptr, block_cap,
                                  ctypes.byref(n_blk)))
    return int(n_ops.value), int(n_blk.value)


def qec_debug_unreduced_plan(gates, k, cap=512):
    """(items [n][4], pass unit items [m], absorptions [a][3]) of the batched form's unreduced round plan."""
    import numpy as np

    items = np.zeros((cap, 4), np.int32)
    pu = np.zeros(cap, np.int32)
    ab = np.zeros((cap, 3), np.int32)
    ni, npu, na = ctypes.c_uint32(0), ctypes.c_uint32(0), ctypes.c_uint32(0)
    check(lib().qec_debug_unreduced_plan(gates, k, items.ctypes.data, cap, ctypes.byref(ni), pu.ctypes.data,
                                         ctypes.byref(npu), ab.ctypes.data, ctypes.byref(na)))
    return items[: ni.value].copy(), pu[: npu.value].copy(), ab[: na.value].copy()


def qec_debug_blocks(params, seed, traj, rnd, kraus_ptr, u_ptr):
    return check(lib().qec_debug_blocks(ctypes.byref(params), seed, traj, rnd, kraus_ptr, u_ptr))


def qec_debug_exact_probability(sim, force):
    """Set the exact-probability mode (1, 0, or -1 = unchanged); returns the exact passes run so far."""
    c = ctypes.c_uint64(0)
    check(lib().qec_debug_exact_probability(sim, force, ctypes.byref(c)))
    return int(c.value)


def qec_debug_speculation(sim, enable):
    """Set the speculative-pass mode (1, 0, or -1 = unchanged); returns the corrective applies run so far."""
    c = ctypes.c_uint64(0)
    check(lib().qec_debug_speculation(sim, enable, ctypes.byref(c)))
    return int(c.value)


def qec_debug_ozaki_gemm(A_ptr, B_ptr, m, variant, out_ptr):
    return check(lib().qec_debug_ozaki_gemm(A_ptr, B_ptr, m, variant, out_ptr))
