"""Distributional checks used as pins: moments with their standard errors and
the Kolmogorov-Smirnov distance to a continuous CDF (plain numpy/scipy)."""
import math

import numpy as np


def normal_cdf(x):
    from scipy.special import ndtr
    return ndtr(x)


def ks_distance(sample, cdf) -> float:
    """sup |F_n - F| for a continuous F, from the sorted sample."""
    x = np.sort(np.asarray(sample, dtype=np.float64))
    n = x.size
    f = cdf(x)
    i = np.arange(1, n + 1, dtype=np.float64)
    return float(max(np.max(i / n - f), np.max(f - (i - 1) / n)))


def ks_critical(n: int, alpha: float = 1e-3) -> float:
    """Asymptotic one-sample KS critical value sqrt(-ln(alpha/2)/2)/sqrt(n)."""
    return math.sqrt(-math.log(alpha / 2.0) / 2.0) / math.sqrt(n)


def check_standard_normal_moments(z, nsig: float = 5.0):
    """Mean 0, variance 1, skewness 0, excess kurtosis 0 within nsig standard
    errors (1/sqrt(n), sqrt(2/n), sqrt(6/n), sqrt(24/n))."""
    z = np.asarray(z, dtype=np.float64)
    n = z.size
    m1 = z.mean()
    d = z - m1
    m2 = np.mean(d * d)
    skew = np.mean(d ** 3) / m2 ** 1.5
    kurt = np.mean(d ** 4) / m2 ** 2 - 3.0
    assert abs(m1) < nsig / math.sqrt(n), ("mean", m1)
    assert abs(m2 - 1.0) < nsig * math.sqrt(2.0 / n), ("variance", m2)
    assert abs(skew) < nsig * math.sqrt(6.0 / n), ("skewness", skew)
    assert abs(kurt) < nsig * math.sqrt(24.0 / n), ("excess kurtosis", kurt)
    return m1, m2, skew, kurt
