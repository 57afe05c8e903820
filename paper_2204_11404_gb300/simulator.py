"""Convenience wrapper over the C ABI (argument marshalling only)."""
import ctypes

import numpy as np

from . import capi


class Simulator:
    """One qec_sim handle: d, rounds, gate set, precision and noise are fixed at creation.

    ``stream``: an integer cudaStream_t (e.g. ``torch.cuda.current_stream().cuda_stream``)
    that the simulator's work is ordered after/before, or None.
    """

    def __init__(self, d, rounds, gates="cr", precision="c128", stream=None, **noise):
        self.d, self.rounds = int(d), int(rounds)
        self.nstab = self.d * self.d - 1
        self.params = capi.make_params(d, rounds, gates, precision, **noise)
        self.h = capi.qec_create(self.params, ctypes.c_void_p(stream) if stream else None)

    def run(self, seed, first_traj, n):
        """Host outputs: syndromes [n][rounds+1][d^2-1], data_bits [n][d^2], raw_logical [n] (uint8)."""
        syn = np.zeros((n, self.rounds + 1, self.nstab), dtype=np.uint8)
        bits = np.zeros((n, self.d * self.d), dtype=np.uint8)
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
