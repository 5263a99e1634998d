"""Seeded synthetic inputs for the SP2 density-matrix response path.

This module only builds inputs.  It holds none of the method's arithmetic
(no spectral bounds, no SP2 layers, no response formulas), so both the
CUDA path and the FP64 oracle can draw their inputs from it.

The paper's own workloads (DFTB water boxes, Sec. IV B; Hartree-Fock water
clusters, Sec. IV C) are not available, so these generators stand in for
them.  Every Hamiltonian is built from a known eigendecomposition:

* ``H = Q diag(eps) Q^T`` with ``Q`` the orthogonal factor of a QR
  decomposition of a seeded standard-Gaussian matrix (column signs fixed by
  ``sign(diag R)``), and ``eps`` drawn uniformly from a gapped interval pair:
  ``n_occ`` occupied levels below the gap and ``n - n_occ`` virtual levels
  above it.  ``eps`` is returned sorted ascending and ``Q``'s columns match.
* A "symmetric Gaussian" perturbation is ``s * (G + G^T) / 2`` with ``G``
  iid N(0, 1).
* A dipole-like perturbation is ``diag(x_k) + 0.001 * sym-Gauss`` with
  orbital coordinates ``x ~ U[0, 20]^3``: the overlap-free (O = I) case of
  the field coupling ``H1 = (O R + R O)/2`` of Sec. IV B.

Seeds: the Hamiltonian (spectrum, then Q) of workload ``cfg`` draws from
``1000 * cfg``; the Gaussian part of perturbation ``k`` from
``1000 * cfg + 1 + k``; the orbital coordinates from ``1000 * cfg + 99``;
instance ``i`` of the uneven batch from ``1000 * 5 + 10 * i``.

Large sizes (QR of an 8192 x 8192 matrix) are slow in numpy, so a
``backend="torch"`` path builds the same recipe with torch (on a CUDA device
when one is given).  The two backends use different random streams: the
same seed gives the same distribution, not the same matrix.  Inside one
process both sides of a comparison always receive the very same arrays.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Instance",
    "WORKLOADS",
    "make_workload",
    "make_instance",
    "sym_gauss",
    "uneven_batch",
    "scc_gamma",
]


@dataclass
class Instance:
    """One synthetic problem: H, its perturbations and how it was made."""

    name: str
    n: int
    n_occ: int
    H: "np.ndarray"                  # (n, n) float64, symmetric
    H1: "np.ndarray"                 # (k, n, n) float64, each symmetric
    eps: "np.ndarray"                # (n,) ascending eigenvalues of H
    Q: "np.ndarray"                  # (n, n) eigenvectors of H (columns)
    extra: dict = field(default_factory=dict)

    @property
    def k(self) -> int:
        return int(self.H1.shape[0])


# Each workload: n, n_occ rule, occupied / virtual eigenvalue intervals,
# perturbation kind and count.  (Sizes and spectra follow the five
# synthetic stand-ins for the paper's systems.)
WORKLOADS = {
    1: dict(name="plain-n128", n=128, occ=(-2.0, -0.5), virt=(0.5, 2.0),
            h1="gauss", k=1, scale=0.01),
    2: dict(name="precision-n4096", n=4096, occ=(-2.0, -0.1), virt=(0.1, 2.0),
            h1="gauss", k=1, scale=0.01),
    3: dict(name="dipole3-n8192", n=8192, occ=(-2.0, -0.1), virt=(0.1, 2.0),
            h1="dipole", k=3, scale=0.001),
    4: dict(name="adjoint-n4096", n=4096, occ=(-2.0, -0.1), virt=(0.1, 2.0),
            h1="gauss", k=1, scale=1.0),
}


def _np_sym_gauss(rng: np.random.Generator, n: int, scale: float) -> np.ndarray:
    g = rng.standard_normal((n, n))
    return scale * (g + g.T) * 0.5


def sym_gauss(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """``scale * (G + G^T)/2`` with G iid N(0,1) from ``default_rng(seed)``."""
    return _np_sym_gauss(np.random.default_rng(seed), n, scale)


def _np_hamiltonian(rng, n, n_occ, occ, virt):
    eps = np.concatenate([rng.uniform(occ[0], occ[1], n_occ),
                          rng.uniform(virt[0], virt[1], n - n_occ)])
    eps.sort()
    a = rng.standard_normal((n, n))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    h = (q * eps[None, :]) @ q.T
    h = 0.5 * (h + h.T)
    return h, eps, q


def _torch_hamiltonian(seed, n, n_occ, occ, virt, device):
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    eps = torch.cat([torch.rand(n_occ, generator=g, dtype=torch.float64) * (occ[1] - occ[0]) + occ[0],
                     torch.rand(n - n_occ, generator=g, dtype=torch.float64) * (virt[1] - virt[0]) + virt[0]])
    eps, _ = torch.sort(eps)
    a = torch.randn(n, n, generator=g, dtype=torch.float64).to(device)
    q, r = torch.linalg.qr(a)
    q = q * torch.sign(torch.diagonal(r))[None, :]
    eps_d = eps.to(device)
    h = (q * eps_d[None, :]) @ q.T
    h = 0.5 * (h + h.T)
    return h, eps_d, q


def _perturbations(kind, n, k, scale, seed0, backend, device):
    """k perturbations; perturbation j draws from seed ``seed0 + 1 + j``."""
    out = []
    if backend == "numpy":
        for j in range(k):
            rng = np.random.default_rng(seed0 + 1 + j)
            if kind == "gauss":
                out.append(_np_sym_gauss(rng, n, scale))
            else:
                # one coordinate triple per orbital; direction j uses coordinate j
                xyz = np.random.default_rng(seed0 + 99).uniform(0.0, 20.0, (n, 3))
                out.append(np.diag(xyz[:, j % 3]) + _np_sym_gauss(rng, n, scale))
        return np.stack(out)
    import torch
    for j in range(k):
        g = torch.Generator(device="cpu").manual_seed(seed0 + 1 + j)
        m = torch.randn(n, n, generator=g, dtype=torch.float64).to(device)
        m = scale * 0.5 * (m + m.T)
        if kind == "dipole":
            gx = torch.Generator(device="cpu").manual_seed(seed0 + 99)
            xyz = torch.rand(n, 3, generator=gx, dtype=torch.float64) * 20.0
            m = m + torch.diag(xyz[:, j % 3].to(device))
        out.append(m)
    return torch.stack(out)


def make_instance(name, n, n_occ, occ, virt, h1="gauss", k=1, scale=0.01,
                  seed=0, backend="numpy", device="cpu") -> Instance:
    """Build one instance of the recipe above (see the module docstring)."""
    if not (0 <= n_occ <= n):
        raise ValueError("n_occ out of range")
    if backend == "numpy":
        rng = np.random.default_rng(seed)
        h, eps, q = _np_hamiltonian(rng, n, n_occ, occ, virt)
    elif backend == "torch":
        h, eps, q = _torch_hamiltonian(seed, n, n_occ, occ, virt, device)
    else:
        raise ValueError(backend)
    h1s = _perturbations(h1, n, k, scale, seed, backend, device)
    return Instance(name=name, n=n, n_occ=n_occ, H=h, H1=h1s, eps=eps, Q=q,
                    extra=dict(seed=seed, occ=occ, virt=virt, h1=h1, scale=scale,
                               backend=backend))


def make_workload(cfg: int, n: Optional[int] = None, k: Optional[int] = None,
                  backend: str = "numpy", device: str = "cpu") -> Instance:
    """Workload ``cfg`` (1-4) of the synthetic suite, optionally at another n.

    ``n`` overrides the size (keeping n_occ = n/2 and the spectrum), so the
    same recipe can be exercised at sizes the oracle finishes in seconds.
    """
    w = WORKLOADS[cfg]
    n = int(w["n"] if n is None else n)
    k = int(w["k"] if k is None else k)
    name = w["name"] if n == w["n"] else f'{w["name"].rsplit("-", 1)[0]}-n{n}'
    return make_instance(name, n, n // 2, w["occ"], w["virt"], w["h1"], k,
                         w["scale"], seed=1000 * cfg, backend=backend, device=device)


def uneven_batch(count: int = 64, n_min: int = 256, n_max: int = 2048,
                 backend: str = "numpy", device: str = "cpu") -> List[Instance]:
    """The uneven batch: ``count`` instances, n log-uniform in [n_min, n_max].

    Instance i: n_occ = n // 2, gap ~ U[0.1, 0.5] centred at 0, spectrum
    within [-2, 2], one symmetric-Gaussian perturbation scaled by 0.01.
    """
    out = []
    for i in range(count):
        seed = 1000 * 5 + 10 * i
        rng = np.random.default_rng(seed)
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        gap = rng.uniform(0.1, 0.5)
        out.append(make_instance(f"uneven-{i}-n{n}", n, n // 2, (-2.0, -gap / 2),
                                 (gap / 2, 2.0), "gauss", 1, 0.01, seed=seed + 1,
                                 backend=backend, device=device))
    return out


def scc_gamma(n: int, seed: int = 1000 * 3 + 99, scale: float = 40.0,
              backend: str = "numpy", device: str = "cpu"):
    """SPD charge-coupling kernel for the self-consistent response.

    gamma_ij = (scale / n) / sqrt(|x_i - x_j|^2 + 1) with orbital coordinates
    x ~ U[0, 20]^3 from ``default_rng(seed)`` (by default the coordinates of
    the dipole perturbations).  The inverse-multiquadric kernel
    1/sqrt(r^2 + c^2) is strictly positive definite for distinct points, so
    gamma is SPD; it decays like 1/r.  The 1/n factor keeps the coupling of
    the induced charges of comparable strength across sizes.
    """
    xyz = np.random.default_rng(seed).uniform(0.0, 20.0, (n, 3))
    d2 = ((xyz[:, None, :] - xyz[None, :, :]) ** 2).sum(-1)
    g = (scale / n) / np.sqrt(d2 + 1.0)
    if backend == "torch":
        import torch
        return torch.from_numpy(g).to(device)
    return g
