"""CPU checks of the library's host side: exported symbols, the static program, and the
host-instantiated Kraus blocks against the oracle (no GPU needed)."""
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import run_trajectory
from paper_2204_11404_gb300 import capi
from kraus_ref import run as kraus_run

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "qecsv.h")).read()
    declared = set(re.findall(r"^\s*(?:qec_status|uint64_t|const char\*)\s+(qec_\w+)\s*\(", hdr, re.M))
    assert len(declared) >= 10
    out = subprocess.check_output(["nm", "-D", "--defined-only", capi.lib()._name]).decode()
    exported = set(re.findall(r" T (qec_\w+)", out))
    assert declared <= exported, declared - exported
    for name in declared:
        getattr(capi.lib(), name)


NOISY = dict(p1=0.03, p2=0.03, p_idle=0.02, theta_rx=0.1, theta_rz=0.07, theta_rzx=0.05,
             phi_zz=0.08, round_rz=0.1, round_rx=0.05)


@pytest.mark.parametrize("gates", ["cnot", "cr"])
def test_host_blocks_match_oracle_d3(gates):
    params = capi.make_params(3, 3, gates, **NOISY)
    for traj in range(6):
        syn, psi = kraus_run(params, 17, traj)
        o = run_trajectory(3, 3, gates, "reduced", NOISY, seed=17, traj=traj, want_state=True)
        assert (syn == o["syndromes"]).all()
        ref = o["state"][: 1 << 9]
        assert np.abs(o["state"][1 << 9:]).max() == 0
        assert np.abs(psi - ref).max() < 1e-13


def test_invalid_params_rejected():
    bad = capi.make_params(4, 3)
    n = np.zeros(8, dtype=np.int32)
    with pytest.raises(capi.QecError) as e:
        capi.qec_debug_program(bad, n.ctypes.data, 0, n.ctypes.data, 0)
    assert e.value.status == capi.QEC_EINVAL
    p = capi.make_params(3, 3, p1=1.5)
    with pytest.raises(capi.QecError):
        capi.qec_debug_program(p, n.ctypes.data, 0, n.ctypes.data, 0)


TWIRLED = dict(NOISY, twirl=1, theta_rx=0.4, theta_rz=0.3, theta_rzx=0.3, phi_zz=0.2, round_rz=0.3, round_rx=0.25)


@pytest.mark.parametrize("gates", ["cnot", "cr"])
def test_host_blocks_match_oracle_twirled(gates):
    params = capi.make_params(3, 3, gates, **TWIRLED)
    for traj in range(6):
        syn, psi = kraus_run(params, 23, traj)
        o = run_trajectory(3, 3, gates, "reduced", TWIRLED, seed=23, traj=traj, want_state=True)
        assert (syn == o["syndromes"]).all()
        assert np.abs(psi - o["state"][: 1 << 9]).max() < 1e-13


SIGN_FOLLOWS = dict(NOISY, theta_rx=0.35, overrot_follows=1)


@pytest.mark.parametrize("noise", [SIGN_FOLLOWS, dict(SIGN_FOLLOWS, twirl=1)])
def test_host_blocks_match_oracle_sign_follows(noise):
    """The sign-follows over-rotation variant (R_X(-theta) after the Rx^dagger preparation)."""
    params = capi.make_params(3, 3, "cr", **noise)
    for traj in range(6):
        syn, psi = kraus_run(params, 29, traj)
        o = run_trajectory(3, 3, "cr", "reduced", noise, seed=29, traj=traj, want_state=True)
        assert (syn == o["syndromes"]).all()
        assert np.abs(psi - o["state"][: 1 << 9]).max() < 1e-13


def test_sign_follows_changes_the_blocks():
    base = capi.make_params(3, 3, "cr", theta_rx=0.35)
    var = capi.make_params(3, 3, "cr", theta_rx=0.35, overrot_follows=1)
    (s0, p0), (s1, p1) = kraus_run(base, 3, 0), kraus_run(var, 3, 0)
    assert np.abs(p0 - p1).max() > 1e-3
    with pytest.raises(capi.QecError):
        capi.qec_debug_program(capi.make_params(3, 3, "cr", overrot_follows=0.5),
                               np.zeros(8, dtype=np.int32).ctypes.data, 0, np.zeros(8, dtype=np.int32).ctypes.data, 0)


@pytest.mark.parametrize("gates", ["cnot", "cr"])
def test_host_blocks_match_oracle_repetition_code(gates):
    """The one-dimensional repetition code of Fig. 2 (d = 9, Z_k Z_{k+1}), every noise term on."""
    params = capi.make_params(9, 3, gates, code="repetition", **NOISY)
    for traj in range(6):
        syn, psi = kraus_run(params, 31, traj)
        o = run_trajectory(9, 3, gates, "reduced", NOISY, seed=31, traj=traj, want_state=True, code="repetition")
        assert (syn == o["syndromes"]).all()
        assert np.abs(psi - o["state"][: 1 << 9]).max() < 1e-13


def test_repetition_code_params_validated():
    n = np.zeros(8, dtype=np.int32)
    for d in (7, 10, 27):
        with pytest.raises(capi.QecError):
            capi.qec_debug_program(capi.make_params(d, 2, code="repetition"), n.ctypes.data, 0, n.ctypes.data, 0)
    p = capi.make_params(9, 2)
    p.code = 2
    with pytest.raises(capi.QecError):
        capi.qec_debug_program(p, n.ctypes.data, 0, n.ctypes.data, 0)


@pytest.mark.parametrize("d,gates", [(3, "cr"), (3, "cnot"), (5, "cr")])
def test_kraus_pairs_are_complete(d, gates):
    """The speculative passes take P(1) = 1 - |K_0 psi|^2 / |psi|^2 when they apply K_0 (Sec. II.B with
    K_0^dagger K_0 + K_1^dagger K_1 = I: the ancilla's two outcomes exhaust its measurement).  The
    pairs the device builds (the host copy runs the same arithmetic) must be complete far inside the
    1e-10 margin of the decision, on every block of noisy rounds with every noise term on."""
    from kraus_ref import blocks, block_meta
    params = capi.make_params(d, 2, gates, **NOISY)
    info = block_meta(params)
    worst = 0.0
    for traj in range(3):
        for rnd in (1, 2):
            kr, _ = blocks(params, 29, traj, rnd)
            for k in range(kr.shape[0]):
                c = 1 << int(info[k, 0])
                k0, k1 = kr[k, 0, :c, :c], kr[k, 1, :c, :c]
                gram = k0.conj().T @ k0 + k1.conj().T @ k1
                worst = max(worst, float(np.abs(gram - np.eye(c)).max()))
    assert worst < 1e-13, worst


@pytest.mark.parametrize("gates", ["cnot", "cr"])
def test_speculative_order_matches_oracle_d3(gates):
    """Reading R19 on the CPU: the speculative order of evaluation (apply the previous outcome's
    Kraus operator, take P(1) from its output, re-apply from the input on a change) reproduces the
    FP64 oracle's syndromes and states on the stress noise, and corrects exactly the outcome
    changes between rounds."""
    params = capi.make_params(3, 3, gates, **NOISY)
    total = 0
    for traj in range(6):
        syn, psi, fixes = kraus_run(params, 23, traj, speculative=True)
        o = run_trajectory(3, 3, gates, "reduced", NOISY, seed=23, traj=traj, want_state=True)
        assert (syn == o["syndromes"]).all()
        assert np.abs(psi - o["state"][: 1 << 9]).max() < 1e-13
        assert fixes == int(np.sum(np.diff(syn.astype(np.int8), axis=0) != 0))
        total += fixes
    assert total > 0
