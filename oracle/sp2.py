"""DNN-SP2-PT in plain FP64 numpy, in the order of Algorithms 1-3 (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The recursion (Sec. II B, Eq. (LinTransf), Eq. (eq:Sn); Sec. III A,
Eq. (initialization), Eq. (S_n detailed), Eq. (dB)):

    S_0   = (eps_N I - H) / (eps_N - eps_1)          initial normalisation
    S1_0  = -H1 / (eps_N - eps_1)                     (Sec. III A, S_0(lambda))
    X_n   = S_{n-1}^2                                 activation f^(0)
    X1_n  = S_{n-1} S1_{n-1} + S1_{n-1} S_{n-1}       activation f^(1)
    S_n   = sigma_n X_n  + (1 - sigma_n) S_{n-1}
    S1_n  = sigma_n X1_n + (1 - sigma_n) S1_{n-1}

with sigma_n chosen by Algorithm 1 and the layers stopped by the
parameter-free criteria of Algorithm 2 (D^(0)) and Algorithm 3 (D^(1),
Eq. (ConvCrit) with C_pt = 9).

Readings taken where the text is silent or inconsistent:

* The bias is (1 - sigma_n) S_{n-1} (Alg. 2 and Sec. II B's prose); the
  S_n in the bias definition after Eq. (LinTransf) is read as S_{n-1}.
* sign(0) in the branch rule of Alg. 1 gives sigma = -1 (2S - S^2).
* At the layer n_c where D^(0) is declared converged, Alg. 2 leaves W_n
  unset; the sigma_{n_c} computed by Alg. 1 at that layer is used for the
  S1 update, and the flips sigma_n = -sigma_{n-1} follow from n_c + 1.
* FroErr^(1)_{n-2} of Alg. 3 is undefined in the first two layers of the
  D^(1) phase (n < n_c + 2); it is taken as +inf, so the test cannot fire
  before one full sigma-flip pair has been applied.
* Alg. 3 compares with a strict ">", which never fires when both sides are
  exactly zero (an exactly idempotent S_0 and an exact S1, e.g. the 2x2
  pin); ">=" is used.  A layer cap (max_layers) ends a run that does not
  converge.
* With several perturbations sharing one S_0 recursion, each direction k
  runs its own Alg. 3 test and is frozen once it converges; the loop ends
  when D^(0) and every direction have converged.
* n_occ = 0 or n_occ = n are the trivial projectors 0 and I with zero
  response; no layer runs.

Everything else (N_X = Tr X_n, the N_S bookkeeping of Alg. 2, FroErr^(0)
from the X_n of the converging layer) follows the algorithms as printed.

Higher orders (order = m >= 2): S^(o) for o = 2..m follow Eq. (S_n
detailed) with S^(o)_0 = 0 (a linear perturbation), each stopped by the
Alg. 3 test applied to its own idempotency error (the paper states the
criteria for orders 0 and 1 only; this is the reading taken for o >= 2).

Pinned by: agreement with ``sos.response_sos`` (a different route to the
same limit), the 2x2 closed form, the invariants, and an independent plain
SP2 run on the 2n x 2n block upper-triangular matrix [[H, H1], [0, H]]
(Sec. III B) whose upper-right block must equal S1 layer by layer.  Orders
o >= 2 are pinned by the (m+1)n block matrix with H1 on the block
superdiagonal, sympy derivatives of the 2x2 projector, finite differences
of the second-order sum over states, and the identities of each order.
The stopping rules (Alg. 2 with both clauses, Alg. 3 with C_pt, FroErr^(0)
and the n - 2 index) are pinned by a hand-worked diagonal case whose values
are exact dyadic rationals (tests/golden/stopping_rules_dyadic.json): the
branch sequence, every IdErr_n, the layer where the second clause of Alg. 2
fires, FroErr^(0), the FroErr^(1) history and the layer where Alg. 3 fires,
for three settings of the two constants.
"""

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .gershgorin import gershgorin_bounds


@dataclass
class SP2Result:
    P: np.ndarray                       # S_0 at exit  (D^(0), orthogonal basis)
    P1: np.ndarray                      # (k, n, n) S1 at exit (D^(1))
    layers: int                         # number of layers run (last n)
    d0_layer: int                       # n_c: layer at which D^(0) converged
    converged: bool
    sigma: List[int] = field(default_factory=list)        # sigma_1..sigma_layers
    iderr: List[float] = field(default_factory=list)      # IdErr_n of the D^(0) phase
    froerr0: float = 0.0
    froerr1: List[List[float]] = field(default_factory=list)  # per k, indexed by n-1 (nan if unset)
    d1_layer: List[int] = field(default_factory=list)    # per k: layer whose test fired
    bounds: tuple = (0.0, 0.0)
    checkpoints: dict = field(default_factory=dict)       # n -> S_n (if requested)
    d2_layer: List[int] = field(default_factory=list)    # order 2: layer whose test fired
    P2: Optional[np.ndarray] = None     # (k, n, n) S2 at exit (D^(2)), order >= 2
    Pk: List[np.ndarray] = field(default_factory=list)   # [S^(o) at exit, (k, n, n)] for o = 1..order
    dk_layer: List[List[int]] = field(default_factory=list)  # per order o = 1..order, per direction


def _sign_tie_minus(x):
    return 1 if x > 0 else -1


def sp2_pt(H, H1, n_occ, c_pt=9.0, c_d0=4.5, max_layers=100, bounds=None,
           keep_states=False, order=1):
    """Algorithms 1-3 in FP64.  H1: one (n, n) matrix or a (k, n, n) stack.

    order = m >= 2 also propagates the higher-order terms of
    Eq. (S_n detailed) (a linear perturbation: H^(o) = 0 for o >= 2, so
    S^(o)_0 = 0):
        S^(o)_n = sigma_n sum_{a=0..o} S^(a)_{n-1} S^(o-a)_{n-1}
                  + (1 - sigma_n) S^(o)_{n-1},
    every activation formed from the states at the start of the layer.  The
    paper gives stopping criteria for orders 0 and 1 only; the reading taken
    here applies the test of Alg. 3 to each order's idempotency error
    FroErr^(o)_n = ||S^(o) - sum_a S^(a) S^(o-a)||_F with the same C_pt and
    FroErr^(0) (Eq. (ConvCrit) in the same form), each direction's S^(o)
    freezing when it fires; higher orders keep using the (possibly frozen)
    lower ones.
    """
    H = np.asarray(H, dtype=np.float64)
    H1 = np.asarray(H1, dtype=np.float64)
    if H1.ndim == 2:
        H1 = H1[None]
    n = H.shape[0]
    k = H1.shape[0]
    if order < 1:
        raise ValueError("order >= 1")
    if not (0 <= n_occ <= n):
        raise ValueError("n_occ out of range")
    if n_occ == 0 or n_occ == n:
        P = np.zeros((n, n)) if n_occ == 0 else np.eye(n)
        zeros = [np.zeros((k, n, n)) for _ in range(order)]
        return SP2Result(P=P, P1=zeros[0], layers=0, d0_layer=0,
                         converged=True, froerr1=[[] for _ in range(k)],
                         d1_layer=[0] * k, P2=zeros[1] if order >= 2 else None,
                         d2_layer=[0] * k, Pk=zeros, dk_layer=[[0] * k for _ in range(order)])

    # Alg. 1 inputs: spectral bound estimates of H^(0)
    eps1, epsN = gershgorin_bounds(H) if bounds is None else bounds
    # initial transform (Alg. 1): W_0 = -(eps_N - eps_1)^-1, B_0 = eps_N (eps_N - eps_1)^-1 I
    W0 = -1.0 / (epsN - eps1)
    S0 = W0 * H + (epsN / (epsN - eps1)) * np.eye(n)
    NS = np.trace(S0)
    # S[o][j]: order o = 1..order of direction j; B_0^(1) = 0, S^(o)_0 = 0 for o >= 2
    S = {1: [W0 * H1[j] for j in range(k)]}
    for o in range(2, order + 1):
        S[o] = [np.zeros((n, n)) for _ in range(k)]
    conv = {o: [False] * k for o in range(1, order + 1)}
    froerr = {o: [dict() for _ in range(k)] for o in range(1, order + 1)}
    dlayer = {o: [0] * k for o in range(1, order + 1)}

    n_layer = 1
    d0_conv = False
    sigma = {}
    iderr = {}
    froerr0 = None
    d0_layer = 0
    ckpt = {0: S0.copy()} if keep_states else {}
    converged = True

    def all_conv():
        return all(all(conv[o]) for o in conv)

    while not (d0_conv and all_conv()):
        if n_layer > max_layers:
            converged = False
            n_layer -= 1
            break
        # activations f^(o) of every direction still running, from the layer-start states
        X = {o: [None] * k for o in range(1, order + 1)}
        for o in range(1, order + 1):
            for j in range(k):
                if conv[o][j]:
                    continue
                acc = S0 @ S[o][j] + S[o][j] @ S0
                for a in range(1, o):
                    acc = acc + S[a][j] @ S[o - a][j]
                X[o][j] = acc
        if not d0_conv:
            X0 = S0 @ S0                                  # activation f^(0)
            NX = np.trace(X0)
            iderr[n_layer] = NS - NX
            sigma[n_layer] = _sign_tie_minus(abs(2.0 * NS - NX - n_occ) - abs(NX - n_occ))
            # ---- Alg. 2
            stop = False
            if iderr[n_layer] <= 0.0:
                stop = True
            elif (n_layer > 2 and sigma[n_layer - 1] != sigma[n_layer - 2]
                  and iderr[n_layer] > c_d0 * iderr[n_layer - 2] ** 2):
                stop = True
            if stop:
                d0_conv = True
                d0_layer = n_layer
                froerr0 = np.linalg.norm(S0 - X0, "fro")
            else:
                s = sigma[n_layer]
                S0 = s * X0 + (1 - s) * S0
                NS = s * NX + (1 - s) * NS
                if keep_states:
                    ckpt[n_layer] = S0.copy()
        else:
            sigma[n_layer] = -sigma[n_layer - 1]           # the sigma flip
        # ---- Alg. 3 (and its reading for o >= 2), per order and direction
        s = sigma[n_layer]
        for o in range(1, order + 1):
            for j in range(k):
                if conv[o][j]:
                    continue
                if d0_conv:
                    fe = np.linalg.norm(S[o][j] - X[o][j], "fro")
                    froerr[o][j][n_layer] = fe
                    prev = froerr[o][j].get(n_layer - 2)
                    if n_layer - 2 >= d0_layer and prev is not None and fe >= c_pt * froerr0 * prev:
                        conv[o][j] = True
                        dlayer[o][j] = n_layer
                if not conv[o][j]:
                    S[o][j] = s * X[o][j] + (1 - s) * S[o][j]
        n_layer += 1
    else:
        n_layer -= 1

    layers = n_layer
    fe_lists = []
    for j in range(k):
        fe_lists.append([froerr[1][j].get(m, float("nan")) for m in range(1, layers + 1)])
    Pk = [np.stack(S[o]) for o in range(1, order + 1)]
    return SP2Result(P=S0, P1=Pk[0], layers=layers, d0_layer=d0_layer,
                     converged=converged, P2=Pk[1] if order >= 2 else None,
                     d2_layer=dlayer[2] if order >= 2 else [0] * k,
                     sigma=[sigma[m] for m in range(1, layers + 1)],
                     iderr=[iderr[m] for m in sorted(iderr)],
                     froerr0=float(froerr0) if froerr0 is not None else float("nan"),
                     froerr1=fe_lists, d1_layer=dlayer[1], bounds=(eps1, epsN),
                     checkpoints=ckpt, Pk=Pk, dk_layer=[dlayer[o] for o in range(1, order + 1)])


def sp2_adjoint(H, G, n_occ, sigma_d0, bounds):
    """dL/dH of L = Tr[G S_final] through the S_0 recursion with fixed branches.

    The branch choices sigma_1..sigma_m of the layers that updated S_0 and
    the spectral bounds are held constant (they are piecewise constant in H).
    Reverse mode of S_n = sigma_n S_{n-1}^2 + (1 - sigma_n) S_{n-1} with a
    symmetric cotangent Gbar_n = dL/dS_n gives
        Gbar_{n-1} = sigma_n (S_{n-1} Gbar_n + Gbar_n S_{n-1}) + (1 - sigma_n) Gbar_n,
    and S_0 = (eps_N I - H)/(eps_N - eps_1) gives dL/dH = -Gbar_0/(eps_N - eps_1).
    Not in the paper; at convergence it equals the response P1 with H1 := G
    (the Daleckii-Krein derivative is self-adjoint), which pins it.
    """
    H = np.asarray(H, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    n = H.shape[0]
    eps1, epsN = bounds
    S = ((epsN * np.eye(n)) - H) / (epsN - eps1)
    states = [S]
    for s in sigma_d0:
        S = s * (S @ S) + (1 - s) * S
        states.append(S)
    Gbar = 0.5 * (G + G.T)
    for idx in range(len(sigma_d0) - 1, -1, -1):
        s = sigma_d0[idx]
        Sp = states[idx]
        Gbar = s * (Sp @ Gbar + Gbar @ Sp) + (1 - s) * Gbar
    return -Gbar / (epsN - eps1)
