"""Self-consistent first-order response (oracle; test infrastructure only).

The response of a self-consistent-charge model (Sec. III A: the response
equations "have to be solved self-consistently"; Sec. IV B, SCC-DFTB, where
the paper itself skips this step) with an orthogonal basis (O = I): the
perturbation felt by the electrons is the external one plus the potential
of the induced charges q1 = diag(P1), coupled through an SPD kernel gamma:

    H1_eff = H1_ext + diag(gamma q1),    P1 = R(H1_eff),    q1 = diag(P1),

where R is the first-order density-matrix response of ``sos`` (a linear map).
The self-consistent P1 is the fixed point; it is computed here by linear
mixing of the charges, q_in <- (1 - alpha) q_in + alpha diag(R(H1_ext +
diag(gamma q_in))), until the relative change of q is below ``tol``.

Pinned by: the fixed-point residual of the result (a second, independent
evaluation of R), and, on a small system, the closed form
q1 = (I - chi gamma)^-1 chi v for a diagonal external potential v, with the
charge susceptibility chi assembled column by column from R.
"""

import numpy as np

from .sos import response_from_eigs


def scc_response(H, H1_ext, gamma, n_occ, tol=1e-12, mixing=0.8, max_iter=1000):
    """Return (P1, q1, iterations) of the self-consistent response."""
    H = np.asarray(H, dtype=np.float64)
    H1_ext = np.asarray(H1_ext, dtype=np.float64)
    gamma = np.asarray(gamma, dtype=np.float64)
    eps, V = np.linalg.eigh(H)
    n = H.shape[0]
    q = np.zeros(n)
    for it in range(1, max_iter + 1):
        _, P1 = response_from_eigs(eps, V, H1_ext + np.diag(gamma @ q), n_occ)
        q_out = np.diag(P1).copy()
        res = np.linalg.norm(q_out - q) / max(np.linalg.norm(q_out), 1e-300)
        q = (1.0 - mixing) * q + mixing * q_out
        if res < tol:
            break
    _, P1 = response_from_eigs(eps, V, H1_ext + np.diag(gamma @ q), n_occ)
    return P1, np.diag(P1).copy(), it
