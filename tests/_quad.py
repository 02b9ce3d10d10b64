"""Quadrature CDFs of unnormalised 1-D log densities, for Kolmogorov-Smirnov pins.

The log densities handed in are built by the tests from scipy.stats densities
of the model's own terms (Section 4.1, Figure 3), not from the oracle.
"""
import numpy as np
from scipy import integrate, stats


class GridDist:
    """Normalised density on a grid from an unnormalised log density."""

    def __init__(self, logf, lo, hi, n=200001):
        x = np.linspace(lo, hi, n)
        lf = np.array([logf(v) for v in x]) if not getattr(logf, "vectorized", False) else logf(x)
        lf = np.where(np.isfinite(lf), lf, -np.inf)
        p = np.exp(lf - np.max(lf))
        cdf = integrate.cumulative_trapezoid(p, x, initial=0.0)
        self.mass_edge = max(p[0], p[-1])
        self.x, self.cdf_vals = x, cdf / cdf[-1]

    def cdf(self, v):
        return np.interp(v, self.x, self.cdf_vals, left=0.0, right=1.0)

    def ppf(self, q):
        return np.interp(q, self.cdf_vals, self.x)

    def sample(self, n, rng):
        return self.ppf(rng.uniform(size=n))

    def mean(self):
        dens = np.gradient(self.cdf_vals, self.x)
        return float(integrate.trapezoid(self.x * dens, self.x))


def vectorized(f):
    f.vectorized = True
    return f


def ks_pvalue(draws, dist):
    return stats.kstest(np.asarray(draws), dist.cdf).pvalue


def bracket(logf, center, scale, lo_bound=-np.inf, hi_bound=np.inf, drop=60.0):
    """Grid end points where logf has fallen `drop` below its peak near center."""
    xs = center + scale * np.linspace(-60, 60, 24001)
    xs = xs[(xs > lo_bound) & (xs < hi_bound)]
    lf = logf(xs) if getattr(logf, "vectorized", False) else np.array([logf(v) for v in xs])
    keep = np.isfinite(lf) & (lf > np.nanmax(lf[np.isfinite(lf)]) - drop)
    idx = np.nonzero(keep)[0]
    lo, hi = xs[max(idx[0] - 1, 0)], xs[min(idx[-1] + 1, xs.size - 1)]
    return max(lo, lo_bound), min(hi, hi_bound)
