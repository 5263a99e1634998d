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
