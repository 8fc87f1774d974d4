"""Per-bin two-sample Poisson test of two count sinograms.

If A and B are independent Poisson counts with equal means in every bin,
then given n = A + B > 0 a bin's A is Binomial(n, 1/2), and the per-bin
chi-square term (A - B)^2 / n has conditional mean exactly 1 and variance
2 - 2/n (the fourth moment of a sum of n random signs is 3 n^2 - 2 n).  Over
the K bins with n > 0:
  * the classical statistic T = sum (A - B)^2 / (A + B) against chi2(K), which
    is conservative where counts are low (a bin with n = 1 always adds 1);
  * the exact-moment z = (T - K) / sqrt(sum (2 - 2/n)), asymptotically
    normal, two-sided, which also fails sinograms that agree too well (the
    same stream twice).
"""
import math

import numpy as np
from scipy import stats


def per_bin_poisson(A, B):
    A = np.asarray(A, dtype=np.float64).ravel()
    B = np.asarray(B, dtype=np.float64).ravel()
    n = A + B
    keep = n > 0
    A, B, n = A[keep], B[keep], n[keep]
    T = float(((A - B) ** 2 / n).sum())
    K = int(keep.sum())
    var = float((2.0 - 2.0 / n).sum())
    z = (T - K) / math.sqrt(var) if var > 0 else 0.0
    return {"bins": K, "chi2": T, "p_chi2": float(stats.chi2.sf(T, K)), "z": z,
            "p_z": float(2.0 * stats.norm.sf(abs(z))), "mean_count": float(n.mean()) / 2.0}


def assert_same_poisson_means(A, B, p_min=0.01):
    r = per_bin_poisson(A, B)
    assert r["p_chi2"] > p_min and r["p_z"] > p_min, r
    return r
