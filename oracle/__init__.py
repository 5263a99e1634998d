"""FP64 CPU oracle for the SP2 density-matrix response path.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import or run anything in this package.  The
product path (the CUDA library and its Python binding) never calls it and
shares no code with it.

Contents (all float64 numpy, plain and slow on purpose):

* ``gershgorin``: spectral bounds by Gershgorin discs (Sec. II B; Alg. 1
  input "spectral bound estimates").
* ``sos``: the plain definitions the method converges to -- the density
  matrix ``P = theta(mu I - H)`` (Eq. (eq:theta)) and its first-order
  response ``P1 = dP(H + lambda H1)/dlambda`` (Eq. (eq:D_k), k = 1) written
  as a sum over states with the Daleckii-Krein divided differences
  (Sec. IV A).
* ``sp2``: the paper's DNN-SP2-PT recursion in FP64, step by step in the
  order of Algorithms 1-3, and the hand-derived adjoint of that recursion.
* ``scc``: the self-consistent-charge response (fixed point of
  H1 = H1_ext + diag(gamma diag(P1))) by linear mixing.

Parity status of each function is stated in its own docstring; every
function here is pinned by a ``-m "not gpu"`` test that does not reuse the
function's own formula.
"""

from .gershgorin import gershgorin_bounds
from .sos import density_matrix, density_from_eigs, response_sos, response_from_eigs
from .sp2 import sp2_pt, SP2Result, sp2_adjoint
from .scc import scc_response

__all__ = [
    "gershgorin_bounds",
    "density_matrix",
    "density_from_eigs",
    "response_sos",
    "response_from_eigs",
    "sp2_pt",
    "SP2Result",
    "sp2_adjoint",
    "scc_response",
]
