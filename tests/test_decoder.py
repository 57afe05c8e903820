"""Host decoder on oracle trajectories (CPU): detection events, single-error correction, and the
code-distance scaling of the logical error rate."""
import numpy as np
import pytest

from oracle import run_trajectory
from oracle import gates as G
from oracle.lattice import stabilizers
from paper_2204_11404_gb300.decoder import Decoder


def test_z_stabilizers_match_table1_order():
    zs = [s["support"] for s in stabilizers(5) if s["kind"] == "Z"]
    assert Decoder(5).zs == zs


@pytest.mark.parametrize("gates", ["cnot", "cr"])
def test_noiseless_has_no_events_and_no_failure(gates):
    dec = Decoder(3)
    r = run_trajectory(3, 3, gates, "reduced", {}, seed=0, traj=0)
    assert dec.detection_events(r["syndromes"], r["data_bits"]) == []
    assert dec.logical_failure(r["syndromes"], r["data_bits"], r["raw_logical"]) == 0


@pytest.mark.parametrize("gates", ["cnot", "cr"])
@pytest.mark.parametrize("rnd", [1, 2])
def test_any_single_x_error_is_corrected_d3(gates, rnd):
    dec = Decoder(3)
    for q in range(9):
        r = run_trajectory(3, 2, gates, "reduced", {}, seed=0, traj=q, inject=[(rnd, 0, q, G.PX)])
        ev = dec.detection_events(r["syndromes"], r["data_bits"])
        assert 1 <= len(ev) <= 2
        assert dec.logical_failure(r["syndromes"], r["data_bits"], r["raw_logical"]) == 0


def test_single_x_error_before_readout_is_corrected_d5():
    # an X on a data qubit right before readout shows only in the final (data-derived) events;
    # d=5 state vectors are large for the CPU suite, so the record is built directly
    dec = Decoder(5)
    syn = np.zeros((3, 24), dtype=np.uint8)
    for q in range(25):
        bits = np.zeros(25, dtype=np.uint8)
        bits[q] = 1
        raw = int(bits[:5].sum() % 2)
        ev = dec.detection_events(syn, bits)
        assert all(r == 2 for r, _ in ev) and 1 <= len(ev) <= 2
        assert dec.logical_failure(syn, bits, raw) == 0


def test_measurement_error_pairs_in_time():
    dec = Decoder(3)
    syn = np.zeros((4, 8), dtype=np.uint8)
    syn[2, 5] = 1                                   # one Z-stabilizer misread in round 2 only
    bits = np.zeros(9, dtype=np.uint8)
    assert dec.detection_events(syn, bits) == [(1, 1), (2, 1)]
    assert dec.logical_failure(syn, bits, 0) == 0


def test_distance_three_corrects_one_error_but_not_two_on_a_column():
    # X on two of the three qubits of the first column: the minimal completion is the third qubit,
    # which makes logical X (a column), so the decoder fails; one error is corrected
    dec = Decoder(3)
    syn = np.zeros((2, 8), dtype=np.uint8)
    one = np.array([1, 0, 0, 0, 0, 0, 0, 0, 0], dtype=np.uint8)
    two = np.array([1, 0, 0, 1, 0, 0, 0, 0, 0], dtype=np.uint8)
    assert dec.logical_failure(syn, one, int(one[:3].sum() % 2)) == 0
    assert dec.logical_failure(syn, two, int(two[:3].sum() % 2)) == 1
    # X on two qubits of the top row is the X-stabilizer X1X2 of Table I's rule: no failure
    stab = np.array([1, 1, 0, 0, 0, 0, 0, 0, 0], dtype=np.uint8)
    assert dec.detection_events(syn, stab) == []
    assert dec.logical_failure(syn, stab, int(stab[:3].sum() % 2)) == 0


def test_logical_error_rate_grows_with_p_d3():
    dec = Decoder(3)
    rates = []
    for p in (0.004, 0.03):
        nz = dict(p1=p, p2=p, p_idle=p)
        f = []
        for t in range(60):
            r = run_trajectory(3, 2, "cr", "reduced", nz, seed=21, traj=t)
            f.append(dec.logical_failure(r["syndromes"], r["data_bits"], r["raw_logical"]))
        rates.append(np.mean(f))
    assert rates[0] < rates[1]


@pytest.mark.parametrize("gates", ["cnot", "cr"])
def test_error_between_two_z_gates_is_one_diagonal_edge(gates):
    # data qubit 4 (centre, d=3) is BR of Z{0,1,3,4} (gate at step 8) and TL of Z{4,5,7,8}
    # (gate at step 10); an X error at step 9 is seen by the later-gated stabilizer in round 1
    # and by the earlier-gated one only in round 2
    dec = Decoder(3)
    r = run_trajectory(3, 2, gates, "reduced", {}, seed=0, traj=0, inject=[(1, 9, 4, G.PX)])
    ev = dec.detection_events(r["syndromes"], r["data_bits"])
    zs = dec.zs
    k_early, k_late = zs.index([0, 1, 3, 4]), zs.index([4, 5, 7, 8])
    assert sorted(ev) == sorted([(0, k_late), (1, k_early)])
    adj, B = dec._graph(len(r["syndromes"]))
    dist, _ = dec._bfs(adj, B, 0 * dec.nz + k_late)
    assert dist[1 * dec.nz + k_early] == 1
    assert dec.logical_failure(r["syndromes"], r["data_bits"], r["raw_logical"]) == 0


def test_repetition_code_corrects_up_to_four_flips_d9():
    """Fig. 2's repetition code at d = 9: any (d-1)/2 = 4 X errors in one round are corrected; the
    stabilizer list matches the oracle's line order."""
    from oracle.lattice import code_stabilizers
    d = 9
    dec = Decoder(d, "repetition")
    assert dec.zs == [s["support"] for s in code_stabilizers(d, "repetition")]
    rng = np.random.default_rng(3)
    for trial in range(6):
        qs = sorted(rng.choice(d, size=1 + trial % 4, replace=False).tolist())
        inject = [(1, 0, q, G.PX) for q in qs]
        r = run_trajectory(d, 2, "cr", "reduced", {}, seed=0, traj=trial, inject=inject, code="repetition")
        assert r["raw_logical"] == len(qs) % 2
        assert dec.logical_failure(r["syndromes"], r["data_bits"], r["raw_logical"]) == 0
    # five flips on a distance-9 line are a logical error after decoding
    r = run_trajectory(d, 2, "cr", "reduced", {}, seed=0, traj=9, inject=[(1, 0, q, G.PX) for q in range(5)],
                       code="repetition")
    assert dec.logical_failure(r["syndromes"], r["data_bits"], r["raw_logical"]) == 1


def test_repetition_code_measurement_error_is_a_time_pair():
    d = 9
    dec = Decoder(d, "repetition")
    syn = np.zeros((4, d - 1), dtype=np.uint8)
    syn[2, 3] = 1                      # one wrong outcome in round 2: events in layers 2 and 3
    assert dec.logical_failure(syn, np.zeros(d, dtype=np.uint8), 0) == 0
    assert len(dec.detection_events(syn, np.zeros(d, dtype=np.uint8))) == 2


def _sample_edges(dec, layers, p, n, rng):
    """Independent edge mechanisms with probabilities p: detection events [n][nodes] and the true
    logical flip of each sample (parity of the flipped edges across the logical support)."""
    E = dec.edges(layers)
    inc = np.zeros((len(E), layers * dec.nz), dtype=np.int64)
    par = np.zeros(len(E), dtype=np.int64)
    for i, (u, v, pr, kind) in enumerate(E):
        inc[i, u] ^= 1
        if kind != "boundary":
            inc[i, v] ^= 1
        par[i] = pr
    flips = (rng.random((n, len(E))) < p).astype(np.int64)
    return ((flips @ inc) % 2).astype(np.uint8), (flips @ par) % 2


def _boundary_groups(E):
    groups = {}
    for i, (u, _, _, kind) in enumerate(E):
        if kind == "boundary":
            groups.setdefault(u, []).append(i)
    return groups


def test_edge_probabilities_are_recovered_from_detection_events():
    """The two-point estimator recovers independent edge probabilities (d=3, 4 layers); a node's
    boundary edges are recovered as their combined probability."""
    rng = np.random.default_rng(11)
    dec, layers = Decoder(3), 4
    E = dec.edges(layers)
    p = rng.uniform(0.002, 0.03, len(E))
    X, _ = _sample_edges(dec, layers, p, 400_000, rng)
    est = dec.estimate_edge_probabilities(X)
    for i, (_, _, _, kind) in enumerate(E):
        if kind != "boundary":
            assert abs(est[i] - p[i]) < 1.5e-3, (i, kind, est[i], p[i])
    for u, idx in _boundary_groups(E).items():
        both = lambda q: 0.5 * (1.0 - np.prod(1.0 - 2.0 * q[idx]))
        assert abs(both(est) - both(p)) < 2e-3, (u, both(est), both(p))


def test_log_likelihood_weights_beat_unit_weights_when_measurement_errors_dominate():
    """Time edges (measurement errors) 15 times likelier than the rest: matching with weights from
    the true probabilities, or from probabilities estimated on the same events, fails less often
    than unit-weight matching."""
    rng = np.random.default_rng(5)
    dec, layers = Decoder(3), 4
    E = dec.edges(layers)
    p = np.array([0.06 if kind == "time" else 0.004 for _, _, _, kind in E])
    X, truth = _sample_edges(dec, layers, p, 4000, rng)

    def failures():
        fails = 0
        for x, t in zip(X, truth):
            defects = [divmod(int(v), dec.nz) for v in np.nonzero(x)[0]]
            fails += int(dec.correction_parity(defects, layers) != t)
        return fails

    unit = failures()
    dec.set_edge_probabilities(layers, p)
    true_w = failures()
    dec.set_edge_probabilities(layers, dec.estimate_edge_probabilities(X))
    est_w = failures()
    dec.clear_weights()
    assert true_w < 0.8 * unit and est_w < 0.8 * unit, (unit, true_w, est_w)


def test_count_failures_reports_both_weightings_and_restores_the_decoder():
    """Oracle trajectories at d=3: the unit-weight count equals logical_failure summed, the
    log-likelihood count is a count over the same trajectories, and no weights stay set."""
    from paper_2204_11404_gb300.decoder import count_failures
    dec = Decoder(3)
    noise = dict(p1=8e-3, p2=8e-3, p_idle=8e-3)
    trajs = [run_trajectory(3, 3, "cr", "reduced", noise, seed=23, traj=i) for i in range(40)]
    syn = [t["syndromes"] for t in trajs]
    bits = [t["data_bits"] for t in trajs]
    log = [t["raw_logical"] for t in trajs]
    unit, weighted = count_failures(dec, syn, bits, log)
    assert unit == sum(dec.logical_failure(s, b, l) for s, b, l in zip(syn, bits, log))
    assert 0 <= weighted <= len(trajs)
    assert not dec._w
