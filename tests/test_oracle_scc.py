"""Pins for the self-consistent response oracle (oracle/scc.py)."""

import numpy as np
import pytest

import oracle
from oracle.sos import response_from_eigs
from paper_2203_09621_gb300.workloads import make_workload, scc_gamma


def test_gamma_is_spd_and_decays():
    g = scc_gamma(64)
    assert np.array_equal(g, g.T)
    assert np.linalg.eigvalsh(g).min() > 0
    xyz = np.random.default_rng(1000 * 3 + 99).uniform(0.0, 20.0, (64, 3))
    r = np.sqrt(((xyz[:, None] - xyz[None]) ** 2).sum(-1))
    far, near = r > 15, (r > 0) & (r < 3)
    assert g[far].max() < g[near].min()


@pytest.mark.parametrize("n", [32, 96])
def test_fixed_point_residual(n):
    inst = make_workload(3, n=n, k=1)
    g = scc_gamma(n)
    P1, q, it = oracle.scc_response(inst.H, inst.H1[0], g, inst.n_occ)
    # an independent evaluation of the response at the returned charges
    _, P1b = oracle.response_sos(inst.H, inst.H1[0] + np.diag(g @ np.diag(P1)), inst.n_occ)
    assert np.linalg.norm(P1 - P1b) / np.linalg.norm(P1) < 1e-10
    _, P1_0 = oracle.response_sos(inst.H, inst.H1[0], inst.n_occ)
    assert np.linalg.norm(P1 - P1_0) / np.linalg.norm(P1_0) > 0.05   # the coupling matters


def test_closed_form_small_system():
    n = 32
    inst = make_workload(3, n=n, k=1)
    g = scc_gamma(n)
    eps, V = np.linalg.eigh(inst.H)
    # charge susceptibility, column c: diag of the response to e_c e_c^T
    chi = np.stack([np.diag(response_from_eigs(eps, V, np.diag(np.eye(n)[c]), inst.n_occ)[1])
                    for c in range(n)], axis=1)
    q0 = np.diag(response_from_eigs(eps, V, inst.H1[0], inst.n_occ)[1])
    q_closed = np.linalg.solve(np.eye(n) - chi @ g, q0)
    _, q, _ = oracle.scc_response(inst.H, inst.H1[0], g, inst.n_occ)
    assert np.linalg.norm(q - q_closed) / np.linalg.norm(q_closed) < 1e-10
    # screening: chi is symmetric negative semidefinite
    assert np.allclose(chi, chi.T, atol=1e-12)
    assert np.linalg.eigvalsh(0.5 * (chi + chi.T)).max() < 1e-12
