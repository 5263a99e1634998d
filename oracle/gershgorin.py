"""Gershgorin spectral bounds (oracle; test infrastructure only).

Sec. II B: the initial normalisation layer needs approximate lower and upper
bounds of the spectrum of H, "for example, by Gershgorin circles"; Alg. 1
takes them as the inputs eps_1 and eps_N.

Gershgorin's theorem: every eigenvalue of H lies in a disc centred at some
H_ii with radius R_i = sum_{j != i} |H_ij|.  For symmetric H the eigenvalues
are real, so they lie in [min_i(H_ii - R_i), max_i(H_ii + R_i)].

Pinned by: a hand-computed 3x3 fixture (tests/golden/gershgorin_3x3.json)
and the containment of the exact spectrum on random matrices.
"""

import numpy as np


def gershgorin_bounds(H):
    """Return (eps_1, eps_N) = (min_i H_ii - R_i, max_i H_ii + R_i) in float64."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    lo = np.inf
    hi = -np.inf
    for i in range(n):
        radius = np.sum(np.abs(H[i, :])) - abs(H[i, i])
        lo = min(lo, H[i, i] - radius)
        hi = max(hi, H[i, i] + radius)
    return float(lo), float(hi)
