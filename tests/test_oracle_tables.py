"""Pins of the oracle's velocity space against the paper's printed values.

Tab. velocity_set_Q=4, Eq. (Q4_kernels), App. A.3 kernel identities and the
exact recovery of equilibrium moments up to third order (App. A.4).
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from analytic import load_golden
from conftest import GOLDEN


@pytest.fixture(scope="module")
def golden():
    return load_golden(os.path.join(GOLDEN, "q4_quadrature_and_kernels.txt"))


def test_velocities_are_printed_roots(golden):
    v, w = oracle.quadrature()
    for a in range(4):
        assert v[a] == pytest.approx(golden[f"v{a}"], rel=1e-15, abs=0)
    # roots of H_4 = x^4 - 6x^2 + 3 (Fig. stencils caption)
    assert np.abs(v**4 - 6 * v**2 + 3).max() < 1e-13


def test_2d_weights_match_table(golden):
    v, w = oracle.quadrature()
    W = np.outer(w, w)
    small = [1, 2]
    for a, b in itertools.product(range(4), range(4)):
        key = ("small" if a in small else "big") + "_" + ("small" if b in small else "big")
        key = {"small_small": "w2d_small_small", "big_big": "w2d_big_big"}.get(key, "w2d_small_big")
        assert W[a, b] == pytest.approx(golden[key], rel=2e-15)
    assert W.sum() == pytest.approx(1.0, rel=1e-15)


def test_kernels_match_printed_matrices(golden):
    K, Kt = oracle.kernels()
    for a, b in itertools.product(range(4), range(4)):
        assert K[a, b] == pytest.approx(golden[f"K{a}{b}"], rel=1e-14, abs=1e-15)
        assert Kt[a, b] == pytest.approx(golden[f"Kt{a}{b}"], rel=1e-14, abs=1e-15)


def test_kernel_identities_app_A3():
    v, _ = oracle.quadrature()
    K, Kt = oracle.kernels()
    # sum_k K_{k,k'} = sum_k Kt_{k,k'} = 0
    assert np.abs(K.sum(axis=0)).max() < 1e-14
    assert np.abs(Kt.sum(axis=0)).max() < 1e-14
    # sum_k K_{k,k'} v_k = -1 ; sum_k Kt_{k,k'} v_k = -v_{k'}
    assert np.abs((K * v[:, None]).sum(axis=0) + 1.0).max() < 1e-14
    assert np.abs((Kt * v[:, None]).sum(axis=0) + v).max() < 1e-14
    # Ktilde is the derivative of (f v): Kt = K diag(v)
    assert np.abs(Kt - K * v[None, :]).max() < 1e-14


def _moments(f, v):
    va = np.repeat(v, 4)   # k = 4a + b -> v_theta = v[a]
    vb = np.tile(v, 4)     # v_phi = v[b]
    V = np.stack([va, vb])
    m0 = f.sum()
    m1 = V @ f
    m2 = np.einsum("ak,bk,k->ab", V, V, f)
    m3 = np.einsum("ak,bk,ck,k->abc", V, V, V, f)
    return m0, m1, m2, m3


@pytest.mark.parametrize("n,ut,up,T", [(1.0, 0.0, 0.0, 1.0), (1.3, 0.05, -0.02, 1.0),
                                       (0.7, -0.2, 0.3, 1.0), (4.0, 0.0, 0.0, 1.5),
                                       (2.0, 0.1, -0.3, 0.8)])
def test_equilibrium_moments_exact_to_third_order(n, ut, up, T):
    """Q = 4 recovers moments up to order 3 of the Maxwellian exactly (App. A.4)."""
    v, _ = oracle.quadrature()
    f = oracle.equilibrium(n, ut, up, T)
    m0, m1, m2, m3 = _moments(f, v)
    u = np.array([ut, up])
    d = np.eye(2)
    assert m0 == pytest.approx(n, rel=1e-14)
    assert np.allclose(m1, n * u, rtol=0, atol=1e-14 * n)
    assert np.allclose(m2, n * (np.outer(u, u) + T * d), rtol=0, atol=1e-14 * n)
    sym = (np.einsum("a,bc->abc", u, d) + np.einsum("b,ca->abc", u, d) + np.einsum("c,ab->abc", u, d))
    assert np.allclose(m3, n * (np.einsum("a,b,c->abc", u, u, u) + T * sym), rtol=0, atol=1e-13 * n)


def test_equilibrium_is_projection_of_maxwellian():
    """f^eq_k / w_k equals the Hermite series of Eq. (feq_series) truncated at l = 3."""
    v, w = oracle.quadrature()
    n, ut, up = 1.1, 0.07, -0.04
    f = oracle.equilibrium(n, ut, up, 1.0)
    for a, b in itertools.product(range(4), range(4)):
        vv = np.array([v[a], v[b]])
        u = np.array([ut, up])
        H1 = vv
        H2 = np.outer(vv, vv) - np.eye(2)
        H3 = (np.einsum("a,b,c->abc", vv, vv, vv) - np.einsum("ab,c->abc", np.eye(2), vv)
              - np.einsum("bc,a->abc", np.eye(2), vv) - np.einsum("ca,b->abc", np.eye(2), vv))
        series = 1 + u @ H1 + 0.5 * np.einsum("a,b,ab", u, u, H2) + np.einsum("a,b,c,abc", u, u, u, H3) / 6
        assert f[4 * a + b] == pytest.approx(n * w[a] * w[b] * series, rel=1e-13)
