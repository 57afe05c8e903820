"""Host logic of the batched form's 17-qubit engine: which one-qubit units are folded into which
two-qubit unit, and which units the passes still apply, checked against the round's item order
(host-only hook; no GPU)."""
import numpy as np
import pytest

from paper_2204_11404_gb300 import capi

GATES = {"cr": capi.QEC_GATES_CR, "cnot": capi.QEC_GATES_CNOT}


def plan(gates, k):
    items, pu, ab = capi.qec_debug_unreduced_plan(GATES[gates], k)
    return items, [int(x) for x in pu], {int(a): (int(t), int(m)) for a, t, m in ab}


def is1(items, i):
    return items[i][0] == 0 and items[i][1] == 1


def is2(items, i):
    return items[i][0] == 0 and items[i][1] == 2


def touches(items, i, b):
    kind, nq, qa, qb = (int(x) for x in items[i])
    return qa == b or (kind == 0 and nq == 2 and qb == b)


def run_around(items, b, a):
    """The run of consecutive one-qubit units on bit b that contains item a, and the items on b
    directly before and after it (None at the round's ends)."""
    seq = [i for i in range(len(items)) if touches(items, i, b)]
    p = seq.index(a)
    lo, hi = p, p
    while lo > 0 and is1(items, seq[lo - 1]):
        lo -= 1
    while hi + 1 < len(seq) and is1(items, seq[hi + 1]):
        hi += 1
    prev = seq[lo - 1] if lo > 0 else None
    nxt = seq[hi + 1] if hi + 1 < len(seq) else None
    return seq[lo:hi + 1], prev, nxt


@pytest.mark.parametrize("gates", ["cr", "cnot"])
@pytest.mark.parametrize("k", [2, 4, 6])
def test_units_are_applied_or_folded_once(gates, k):
    items, pu, ab = plan(gates, k)
    units = [i for i in range(len(items)) if items[i][0] == 0]
    assert sorted(pu + list(ab)) == units            # every unit exactly once
    assert pu == sorted(pu)                          # the passes keep program order
    assert all(is2(items, t) for t, _ in ab.values())
    assert all(is1(items, a) for a in ab)


@pytest.mark.parametrize("gates", ["cr", "cnot"])
def test_folds_are_whole_runs_next_to_their_unit(gates):
    items, _, ab = plan(gates, 4)
    for a, (t, mode) in ab.items():
        b = int(items[a][2])
        assert touches(items, t, b)
        assert bool(mode & 1) == (a > t)             # folded from the left when it follows the unit
        assert bool(mode & 2) == (int(items[t][2]) == b)
        run, prev, nxt = run_around(items, b, a)
        assert t in (prev, nxt)                      # the unit is adjacent to the run on bit b
        assert all(ab.get(i, (None,))[0] == t for i in run)   # the whole run goes to the same unit
        if prev is not None and nxt is not None and is2(items, prev) and is2(items, nxt):
            # between two two-qubit units, the one whose second qubit is b takes the run
            want = nxt if (int(items[nxt][3]) == b or int(items[prev][3]) != b) else prev
            assert t == want
        elif nxt is not None and is2(items, nxt):
            assert t == nxt
        else:
            assert t == prev


@pytest.mark.parametrize("gates", ["cr", "cnot"])
def test_unfolded_one_qubit_units_have_no_two_qubit_neighbour(gates):
    items, pu, ab = plan(gates, 4)
    for i in pu:
        if not is1(items, i):
            continue
        _, prev, nxt = run_around(items, int(items[i][2]), i)
        assert not (prev is not None and is2(items, prev)) and not (nxt is not None and is2(items, nxt))


def test_folding_does_not_depend_on_the_fusion_width():
    ref = plan("cr", 2)[2]
    for k in (3, 4, 5, 6):
        assert plan("cr", k)[2] == ref


def test_plan_rejects_bad_width():
    with pytest.raises(capi.QecError):
        capi.qec_debug_unreduced_plan(capi.QEC_GATES_CR, 7)
    items = plan("cr", 5)[0]
    assert int(np.sum(items[:, 0] == 1)) == 8        # the round's 4 X and 4 Z ancilla measurements
