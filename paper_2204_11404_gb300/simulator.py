"""Convenience wrapper over the C ABI (argument marshalling only)."""
import ctypes

import numpy as np

from . import capi


class Simulator:
    """One qec_sim handle: d, rounds, gate set, precision, code and noise are fixed at creation.

    ``stream``: an integer cudaStream_t (e.g. ``torch.cuda.current_stream().cuda_stream``)
    that the simulator's work is ordered after/before, or None.
    ``code``: "surface" (rotated surface code, d^2 data qubits) or "repetition" (Fig. 2's
    one-dimensional code, d data qubits).
    """

    def __init__(self, d, rounds, gates="cr", precision="c128", stream=None, code="surface", **noise):
        self.d, self.rounds, self.code = int(d), int(rounds), code
        self.nd = self.d if code == "repetition" else self.d * self.d
        self.nstab = self.nd - 1
        self.params = capi.make_params(d, rounds, gates, precision, code=code, **noise)
        self.h = capi.qec_create(self.params, ctypes.c_void_p(stream) if stream else None)

    def reconfigure(self, rounds, **noise):
        """New noise parameters and round count; d, gate set and precision stay."""
        g = {capi.QEC_GATES_CNOT: "cnot", capi.QEC_GATES_CR: "cr"}[self.params.gates]
        pr = {capi.QEC_C128: "c128", capi.QEC_C64: "c64", capi.QEC_C64_TC: "c64tc",
              capi.QEC_C128_TC: "c128tc"}[self.params.precision]
        params = capi.make_params(self.d, rounds, g, pr, code=self.code, **noise)
        capi.qec_reconfigure(self.h, params)
        self.params, self.rounds = params, int(rounds)

    def run(self, seed, first_traj, n):
        """Host outputs: syndromes [n][rounds+1][stabilizers], data_bits [n][data qubits], raw_logical [n]
        (uint8)."""
        syn = np.zeros((n, self.rounds + 1, self.nstab), dtype=np.uint8)
        bits = np.zeros((n, self.nd), dtype=np.uint8)
        log = np.zeros(n, dtype=np.uint8)
        capi.qec_run_trajectories(self.h, seed, first_traj, n, syn.ctypes.data, bits.ctypes.data, log.ctypes.data)
        return syn, bits, log

    def run_device(self, seed, first_traj, n, syn_ptr, bits_ptr, log_ptr):
        """Device outputs (raw device pointers of the same shapes); asynchronous."""
        capi.qec_run_trajectories_device(self.h, seed, first_traj, n, syn_ptr, bits_ptr, log_ptr)

    def state(self):
        n = capi.qec_state_len(self.h)
        out = np.zeros(n, dtype=np.complex128)
        capi.qec_get_state(self.h, out.ctypes.data, out.nbytes)
        return out

    def record_events(self, max_events):
        capi.qec_record_events(self.h, max_events)
        self._ev_cap = max_events

    def events(self):
        cap = getattr(self, "_ev_cap", 0)
        buf = np.zeros((max(cap, 1), 5), dtype=np.int32)
        n = capi.qec_get_events(self.h, buf.ctypes.data, cap)
        return buf[:n]

    def close(self):
        if getattr(self, "h", None):
            capi.qec_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSimulator:
    """qec_batch handle: d = 3 trajectories with per-trajectory register (reduced 10-qubit or
    unreduced 17-qubit), precision and noise in one launch.  kind strings: "c128", "c64" (reduced),
    "c128u", "c64u" (unreduced)."""

    def __init__(self, rounds, gates="cr", max_traj=8192, stream=None, d=3):
        self.d, self.rounds, self.nstab = d, rounds, d * d - 1
        self.h = capi.qec_batch_create(d, rounds, {"cnot": capi.QEC_GATES_CNOT, "cr": capi.QEC_GATES_CR}[gates],
                                       max_traj, ctypes.c_void_p(stream) if stream else None)

    @staticmethod
    def _inputs(traj, kind, noise):
        n = len(traj)
        t = np.ascontiguousarray(traj, dtype=np.uint64)
        # kind: precision, plus 2 for the unreduced (2d^2-1 qubit, time-ordered) register
        codes = {"c128": 0, "c64": 1, "c128u": 2, "c64u": 3}
        k = np.ascontiguousarray([codes.get(x, x) for x in kind], dtype=np.int32)
        nz = (capi.qec_noise * max(n, 1))()
        for i, d in enumerate(noise):
            for f in capi.NOISE_FIELDS:
                setattr(nz[i], f, float(d.get(f, 0.0)))
        return n, t, k, nz

    def run(self, seed, traj, kind, noise):
        n, t, k, nz = self._inputs(traj, kind, noise)
        syn = np.zeros((n, self.rounds + 1, self.nstab), dtype=np.uint8)
        bits = np.zeros((n, self.d * self.d), dtype=np.uint8)
        log = np.zeros(n, dtype=np.uint8)
        capi.qec_batch_run(self.h, seed, n, t.ctypes.data, k.ctypes.data, ctypes.addressof(nz), syn.ctypes.data,
                           bits.ctypes.data, log.ctypes.data)
        return syn, bits, log

    def autotune(self, seed, traj, kind, noise):
        n, t, k, nz = self._inputs(traj, kind, noise)
        return capi.qec_batch_autotune(self.h, seed, n, t.ctypes.data, k.ctypes.data, ctypes.addressof(nz))

    def config(self):
        """(warps per CTA of the reduced engine, fusion width and threads per CTA of the unreduced one)."""
        return capi.qec_batch_config(self.h)

    def set_config(self, warps_per_cta, fusion_width, u_threads):
        capi.qec_batch_set_config(self.h, warps_per_cta, fusion_width, u_threads)

    def snapshot(self, item):
        """Record the final data-register state of trajectory `item` (index into the next run's
        arrays; -1 = none) during the next run."""
        capi.qec_batch_snapshot(self.h, int(item))

    def state(self):
        """The normalised 2^9-amplitude data-register state recorded by the last run with a
        snapshot item (complex128)."""
        out = np.zeros(1 << 9, dtype=np.complex128)
        capi.qec_batch_get_state(self.h, out.ctypes.data, out.nbytes)
        return out

    def last_ms(self):
        return capi.qec_batch_last_ms(self.h)

    def close(self):
        if getattr(self, "h", None):
            capi.qec_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
