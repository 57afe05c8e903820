"""Numpy application of the library's host-instantiated Kraus blocks (CPU check of the compile path).

Takes the blocks produced by qec_debug_blocks (the same fusion arithmetic the
device kernel runs) and applies them with plain numpy to a dense data
register, so the schedule, op assignment and fusion can be compared with the
oracle on the CPU.  It does not exercise the GPU kernels.
"""
import ctypes

import numpy as np

from paper_2204_11404_gb300 import capi


def ndata(params):
    """Data qubits of the code: d^2 (surface) or d (repetition)."""
    return params.d if params.code == capi.QEC_CODE_REPETITION else params.d * params.d


def blocks(params, seed, traj, rnd):
    nst = ndata(params) - 1
    kr = np.zeros((nst, 2, 16, 16), dtype=np.complex128)
    u = np.zeros(nst, dtype=np.float64)
    capi.qec_debug_blocks(params, seed, traj, rnd, kr.ctypes.data, u.ctypes.data)
    return kr, u


def block_meta(params):
    nst = ndata(params) - 1
    ops = np.zeros((4096, 6), dtype=np.int32)
    info = np.zeros((nst, 6), dtype=np.int32)
    capi.qec_debug_program(params, ops.ctypes.data, 4096, info.ctypes.data, nst)
    return info


def apply_block(psi, D, qs, K):
    w = len(qs)
    t = psi.reshape([2] * D)
    axes = [D - 1 - q for q in reversed(qs)]
    t = np.moveaxis(t, axes, list(range(D - w, D)))
    shp = t.shape
    g = t.reshape(-1, 1 << w) @ K.T
    t = np.moveaxis(g.reshape(shp), list(range(D - w, D)), axes)
    return np.ascontiguousarray(t).reshape(-1)


def run(params, seed, traj, speculative=False):
    """One trajectory with numpy.  Each noisy measurement draws m with P(1) = |K_1 psi|^2 / |psi|^2
    and continues with K_m psi / |psi|.  speculative: the order of the speculative passes instead,
    K_g applied first for the guess g (the same stabilizer's previous raw outcome), P(1) taken from
    |K_g psi|^2 (as 1 - P(0) for g = 0), K_m re-applied from the input where m != g; returns the
    number of such corrections as a third value."""
    R = params.rounds
    D = ndata(params)
    nst = D - 1
    info = block_meta(params)
    psi = np.zeros(1 << D, dtype=np.complex128)
    psi[0] = 1.0
    syn = np.zeros((R + 1, nst), dtype=np.uint8)
    raw = np.zeros(nst, dtype=np.int64)
    fixes = 0
    for rnd in range(R + 1):
        kr, u = blocks(params, seed, traj, rnd)
        for k in range(nst):
            w, offset = info[k, 0], info[k, 5]
            qs = [int(x) for x in info[k, 1:1 + w]]
            C = 1 << w
            K = (kr[k, 0, :C, :C], kr[k, 1, :C, :C])
            N = np.vdot(psi, psi).real
            if rnd == 0:
                m = offset
                out = apply_block(psi, D, qs, K[m])
            elif speculative:
                g = int(raw[k])
                out = apply_block(psi, D, qs, K[g])
                pg = np.vdot(out, out).real / N
                m = int(u[k] < (pg if g else 1.0 - pg))
                if m != g:
                    fixes += 1
                    out = apply_block(psi, D, qs, K[m])
            else:
                y1 = apply_block(psi, D, qs, K[1])
                m = int(u[k] < np.vdot(y1, y1).real / N)
                out = y1 if m else apply_block(psi, D, qs, K[0])
            psi = out / np.sqrt(N)
            raw[k] = m
            syn[rnd, k] = m ^ offset
    psi = psi / np.linalg.norm(psi)
    return (syn, psi, fixes) if speculative else (syn, psi)
