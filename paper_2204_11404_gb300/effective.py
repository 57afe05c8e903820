"""Effective stochastic model of coherent error (Sec. III.C).

The logical error rate under over-rotations theta = 2 c sqrt(p) is modelled as the c = 0 rate at an
effective physical rate p_eff = (1 + alpha c^2) p (Eq. 9), with the c = 0 rate a power law
p_L = A p^xi (Eq. 8, fitted over p = 1e-3 .. 3e-3).  The fit follows the three steps of Sec. III.C:

1. (A, xi) from the c = 0 points;
2. for each c > 0, B from p_L = A (B p)^xi with A and xi held fixed;
3. alpha from B(c) = 1 + alpha c^2.

The paper does not say how the fits are weighted.  Here steps 1 and 2 are least squares on log p_L
weighted by the failure count k of each point (the variance of log p_L is about 1/k for binomial
counts with small p_L); points with k = 0 carry no weight.  Step 3 is unweighted least squares of
B - 1 against c^2 through the origin.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class EffectiveFit:
    A: float
    xi: float
    B: dict          # c -> B(c)
    alpha: float


def fit_power_law(p, k, n):
    """(A, xi) of p_L = A p^xi from failure counts k out of n trajectories at rates p."""
    p, k, n = (np.asarray(v, dtype=float) for v in (p, k, n))
    m = k > 0
    if m.sum() < 2:
        raise ValueError("need at least two points with failures")
    x, y, w = np.log(p[m]), np.log(k[m] / n[m]), k[m]
    X = np.stack([np.ones_like(x), x], axis=1)
    W = np.diag(w)
    la, xi = np.linalg.solve(X.T @ W @ X, X.T @ W @ y)
    return float(np.exp(la)), float(xi)


def fit_scale(A, xi, p, k, n):
    """B of p_L = A (B p)^xi with A and xi fixed: weighted mean of log(p_L / A) / xi - log p."""
    p, k, n = (np.asarray(v, dtype=float) for v in (p, k, n))
    m = k > 0
    if not m.any():
        raise ValueError("no point with failures")
    lb = (np.log(k[m] / n[m]) - np.log(A)) / xi - np.log(p[m])
    with np.errstate(over="ignore"):
        return float(np.exp(np.sum(k[m] * lb) / np.sum(k[m])))


def fit_alpha(c, B):
    """alpha of B = 1 + alpha c^2 (least squares through B = 1 at c = 0)."""
    c2 = np.asarray(c, dtype=float) ** 2
    b = np.asarray(B, dtype=float) - 1.0
    if not np.any(c2 > 0):
        raise ValueError("need a point with c > 0")
    return float(np.sum(c2 * b) / np.sum(c2 * c2))


def fit_effective_model(rows, p_range=(1.0e-3, 3.0e-3)):
    """rows: dicts with keys c, p, failures, trajectories.  Only points with p in p_range enter."""
    sel = [r for r in rows if p_range[0] * (1 - 1e-9) <= r["p"] <= p_range[1] * (1 + 1e-9)]
    c0 = [r for r in sel if r["c"] == 0]
    A, xi = fit_power_law([r["p"] for r in c0], [r["failures"] for r in c0], [r["trajectories"] for r in c0])
    B = {}
    for c in sorted({r["c"] for r in sel if r["c"] > 0}):
        pts = [r for r in sel if r["c"] == c]
        B[c] = fit_scale(A, xi, [r["p"] for r in pts], [r["failures"] for r in pts], [r["trajectories"] for r in pts])
    alpha = fit_alpha(list(B.keys()), list(B.values())) if B else float("nan")
    return EffectiveFit(A, xi, B, alpha)


def bootstrap_alpha(rows, n=400, seed=0, p_range=(1.0e-3, 3.0e-3)):
    """Statistical spread of alpha: the failure counts redrawn as binomial(trajectories, p_L) at the
    measured rates, the whole fit repeated; returns (half the 16-84 percentile width, (16th, 84th
    percentiles)).  Percentiles, not a standard deviation: with few failures at the lowest p some
    resamples make the c = 0 power law nearly flat and B(c) huge.  Resamples where a fit is
    undefined are skipped."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        rs = [dict(r, failures=int(rng.binomial(r["trajectories"], r["failures"] / r["trajectories"])))
              for r in rows]
        try:
            a = fit_effective_model(rs, p_range).alpha
        except (ValueError, np.linalg.LinAlgError):
            continue
        if np.isfinite(a):
            out.append(a)
    if len(out) < 2:
        return float("nan"), (float("nan"), float("nan"))
    lo, hi = float(np.percentile(out, 16)), float(np.percentile(out, 84))
    return 0.5 * (hi - lo), (lo, hi)
