"""Fit of the effective model of coherent error (Sec. III.C), on counts synthesised from the model."""
import numpy as np
import pytest

from paper_2204_11404_gb300.effective import (bootstrap_alpha, fit_alpha, fit_effective_model, fit_power_law,
                                              fit_scale)

# the paper's fitted values (Sec. III.C): A = 6.5e5, xi = 2.92, alpha = 0.872
A0, XI0, ALPHA0 = 6.5e5, 2.92, 0.872
PS = (1.0e-3, 1.5e-3, 2.0e-3, 3.0e-3)
CS = (0.0, 0.25, 0.5, 0.75, 1.0)


def _rows(n=10**9, alpha=ALPHA0, extra_p=()):
    rows = []
    for c in CS:
        for p in PS + tuple(extra_p):
            pl = A0 * ((1 + alpha * c * c) * p) ** XI0
            rows.append({"c": c, "p": p, "trajectories": n, "failures": round(pl * n)})
    return rows


def test_exact_counts_recover_the_papers_parameters():
    f = fit_effective_model(_rows())
    assert f.A == pytest.approx(A0, rel=1e-4)
    assert f.xi == pytest.approx(XI0, rel=1e-5)
    for c, b in f.B.items():
        assert b == pytest.approx(1 + ALPHA0 * c * c, rel=1e-5)
    assert f.alpha == pytest.approx(ALPHA0, rel=1e-4)


def test_points_outside_the_fit_range_are_ignored():
    rows = _rows(extra_p=(5e-3,))
    for r in rows:
        if r["p"] == 5e-3:
            r["failures"] = r["trajectories"] // 2      # far off the model: must not enter the fit
    assert fit_effective_model(rows).alpha == pytest.approx(ALPHA0, rel=1e-4)


def test_twirl_limit_alpha_one_and_no_coherence():
    """A fully decohered over-rotation adds c^2 p per term: alpha = 1 (Sec. III.A); no c-dependence: 0."""
    assert fit_effective_model(_rows(alpha=1.0)).alpha == pytest.approx(1.0, rel=1e-4)
    assert abs(fit_effective_model(_rows(alpha=0.0)).alpha) < 1e-4


def test_power_law_slope_and_zero_count_points():
    p = np.array([1e-3, 2e-3, 4e-3, 8e-3])
    n = np.full(4, 10**8)
    k = np.round(3.0 * p ** 2 * n)
    A, xi = fit_power_law(np.append(p, 1e-6), np.append(k, 0), np.append(n, 100))   # k = 0: no weight
    assert xi == pytest.approx(2.0, rel=1e-5) and A == pytest.approx(3.0, rel=1e-4)
    assert fit_scale(3.0, 2.0, p, np.round(3.0 * (1.5 * p) ** 2 * n), n) == pytest.approx(1.5, rel=1e-5)
    assert fit_alpha([0.5, 1.0], [1.25, 2.0]) == pytest.approx(1.0)
    with pytest.raises(ValueError):
        fit_power_law([1e-3], [5], [100])


def test_bootstrap_spread_shrinks_with_statistics():
    """The spread of alpha from redrawn binomial counts falls like 1/sqrt(trajectories)."""
    small, _ = bootstrap_alpha(_rows(n=2000), n=200, seed=1)
    large, (lo, hi) = bootstrap_alpha(_rows(n=200000), n=200, seed=1)
    assert 0 < large < small
    assert 5 < small / large < 20                 # sqrt(100) = 10
    assert lo < ALPHA0 < hi
