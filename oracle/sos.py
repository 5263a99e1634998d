"""Density matrix and first-order response by their definitions (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``density_matrix``: the matrix step function P = theta(mu I - H) of
  Eq. (eq:theta) (Sec. II B; zero temperature, orthogonal basis, Z = I):
  the spectral projector onto the n_occ lowest eigenvectors of H.
* ``response_sos``: the first-order response P1 = d/dlambda
  theta(mu I - H - lambda H1) at lambda = 0 (Eq. (eq:D_k) with k = 1, and
  the Gateaux-derivative definition of D^(1) in Sec. IV A).  By the
  Daleckii-Krein theorem quoted in Sec. IV A, the derivative of a matrix
  function f at H = V diag(eps) V^T in the direction H1 is
  V (F o (V^T H1 V)) V^T with F_ij the divided difference f[eps_i, eps_j].
  For the step function with occupations f_i (1 for the n_occ lowest
  levels, else 0): F_ij = (f_i - f_j) / (eps_i - eps_j) when f_i != f_j and
  0 when f_i == f_j (both derivatives of the step vanish away from mu).
  The method reaches exactly this limit (Sec. IV A).

Sec. III A restricts the theory to non-degenerate systems: a gap between
level n_occ and n_occ + 1 is required, and these functions raise if it is
missing.

``response2_from_eigs`` / ``response2_sos`` give the second-order response
D2 = (1/2) d^2P/dlambda^2 (Eq. (eq:D_k), k = 2) by the second-order
Daleckii-Krein formula.

``density_from_eigs`` and ``response_columns`` evaluate the same
definitions from a known eigendecomposition (the synthetic inputs are built
as H = Q diag(eps) Q^T), the latter from the occupied-virtual block of F
only, which makes the whole P1 at n = 8192 affordable on the host.

Pinned by: the 2x2 closed form differentiated symbolically
(tests/golden/two_level.json and the sympy test), the invariants P^2 = P,
Tr P = n_occ, [H, P] = 0, Tr P1 = 0, P P1 + P1 P = P1,
[H, P1] + [H1, P] = 0, central finite differences of ``density_matrix``
(Eq. (FnD_2) and (FnD_4)), and agreement with ``sp2.sp2_pt``.
"""

import numpy as np


def _occupations(n, n_occ):
    f = np.zeros(n)
    f[:n_occ] = 1.0
    return f


def _check_gap(eps, n_occ):
    n = eps.shape[0]
    if 0 < n_occ < n and not eps[n_occ - 1] < eps[n_occ]:
        raise ValueError("degenerate HOMO/LUMO: the response is undefined (Sec. III A)")


def density_from_eigs(eps, V, n_occ):
    """P = V diag(f) V^T from a known eigendecomposition (``eps`` ascending):
    the projector on the first n_occ columns of V, formed as Vo Vo^T."""
    eps = np.asarray(eps, dtype=np.float64)
    _check_gap(eps, n_occ)
    Vo = np.asarray(V, dtype=np.float64)[:, :n_occ]
    return Vo @ Vo.T


def density_matrix(H, n_occ):
    """P = theta(mu I - H): projector on the n_occ lowest eigenvectors."""
    H = np.asarray(H, dtype=np.float64)
    eps, V = np.linalg.eigh(H)
    _check_gap(eps, n_occ)
    Vo = V[:, :n_occ]
    return Vo @ Vo.T


def response_from_eigs(eps, V, H1, n_occ):
    """(P, P1) from a known eigendecomposition H = V diag(eps) V^T.

    ``eps`` ascending; ``H1`` one (n, n) perturbation.  Plain definition:
    P = V diag(f) V^T, P1 = V (F o (V^T H1 V)) V^T.
    """
    eps = np.asarray(eps, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    H1 = np.asarray(H1, dtype=np.float64)
    n = eps.shape[0]
    _check_gap(eps, n_occ)
    f = _occupations(n, n_occ)
    df = f[:, None] - f[None, :]
    de = eps[:, None] - eps[None, :]
    F = np.zeros((n, n))
    mask = df != 0.0
    F[mask] = df[mask] / de[mask]
    Y = V.T @ H1 @ V
    P = (V * f[None, :]) @ V.T
    P1 = V @ (F * Y) @ V.T
    return P, P1


def response_sos(H, H1, n_occ):
    """(P, P1) for one perturbation H1, or (P, [P1_k]) for a stack of them."""
    H = np.asarray(H, dtype=np.float64)
    eps, V = np.linalg.eigh(H)
    H1 = np.asarray(H1, dtype=np.float64)
    if H1.ndim == 2:
        return response_from_eigs(eps, V, H1, n_occ)
    P = None
    P1s = []
    for h1 in H1:
        P, p1 = response_from_eigs(eps, V, h1, n_occ)
        P1s.append(p1)
    return P, np.stack(P1s)


def response_columns(eps, V, H1, n_occ, cols):
    """Selected columns P1[:, cols] from a known eigendecomposition.

    Uses only the occupied-virtual block of F (the other blocks of F are
    zero by the definition above), so it costs O(n^2 n_occ) instead of the
    full transform.  Same definition as ``response_from_eigs``.
    """
    eps = np.asarray(eps, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    _check_gap(eps, n_occ)
    Vo, Vv = V[:, :n_occ], V[:, n_occ:]
    Fov = 1.0 / (eps[:n_occ, None] - eps[None, n_occ:])
    Yov = Vo.T @ (np.asarray(H1, dtype=np.float64) @ Vv)
    M = Fov * Yov                                   # (n_occ, n - n_occ)
    cols = np.asarray(cols)
    # P1 = Vo M Vv^T + Vv M^T Vo^T, column j: Vo (M Vv[j]) + Vv (M^T Vo[j])
    return Vo @ (M @ Vv[cols, :].T) + Vv @ (M.T @ Vo[cols, :].T)


def _second_divided_differences(eps, f, m):
    """F2[i, j] = f[eps_i, eps_m, eps_j] for the step occupations f (0/1).

    First divided differences f[x, y] = (f(x) - f(y)) / (x - y), and
    f'(x) = 0 away from mu; second ones f[a, b, c] = (f[a, b] - f[b, c]) /
    (a - c), and at a = c the derivative of f[a, b] in a, which is
    -(f(a) - f(b)) / (a - b)^2 (0 when b = a as well).
    """
    n = eps.shape[0]
    d1 = np.zeros(n)                      # f[eps_i, eps_m]
    mask = np.arange(n) != m
    d1[mask] = (f[mask] - f[m]) / (eps[mask] - eps[m])
    num = d1[:, None] - d1[None, :]       # f[i, m] - f[m, j]
    den = eps[:, None] - eps[None, :]
    F2 = np.zeros((n, n))
    off = ~np.eye(n, dtype=bool)
    F2[off] = num[off] / den[off]
    diag = np.zeros(n)
    diag[mask] = -(f[mask] - f[m]) / (eps[mask] - eps[m]) ** 2
    F2[np.arange(n), np.arange(n)] = diag
    return F2


def response2_from_eigs(eps, V, H1, n_occ):
    """Second-order response D2 = (1/2) d^2 P(H + lambda H1)/dlambda^2 at 0.

    Eq. (eq:D_k) with k = 2 (a linear perturbation, H2 = 0).  The second
    Daleckii-Krein formula for a spectral function f:
        D2 = V [ sum_m f[eps_i, eps_m, eps_j] Y_im Y_mj ]_ij V^T,  Y = V^T H1 V,
    with the second divided differences of the step occupations (all
    eigenvalues away from mu).  O(n^3) time, O(n^2) memory.
    """
    eps = np.asarray(eps, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    n = eps.shape[0]
    _check_gap(eps, n_occ)
    f = _occupations(n, n_occ)
    Y = V.T @ np.asarray(H1, dtype=np.float64) @ V
    M = np.zeros((n, n))
    for m in range(n):
        M += _second_divided_differences(eps, f, m) * np.outer(Y[:, m], Y[m, :])
    return V @ M @ V.T


def response2_sos(H, H1, n_occ):
    """D2 for one perturbation via eigh (see response2_from_eigs)."""
    eps, V = np.linalg.eigh(np.asarray(H, dtype=np.float64))
    return response2_from_eigs(eps, V, H1, n_occ)
