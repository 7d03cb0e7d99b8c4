"""Pins of the oracle's symmetric contraction (MACE's product basis of
correlation order 2; the MACE table of the paper: correlation 2).

For one node with aggregated features A [(L+1)^2, C] and species weights
w1 [L+1, C], w2 [Q, C] the contraction is
    B[l3 m3] = w1[l3] A[l3 m3] + sum_q w2[q] sum C^q[m3][m1][m2] A[l1 m1] A[l2 m2]
over the couplings q = (l1 <= l2, l3).  Nothing numeric is printed for it, so
it is pinned by what the definition fixes: the coupling list, closed forms of
single couplings (identity, scalar times feature, squared norm, the norm of
the quadrupole of a vector), homogeneity, equivariance under Wigner-D
matrices of proper and improper rotations, and its adjoint against central
differences.  The whole-model pins (invariances, forces = dual numbers =
finite differences, stress = strain derivative) run on models with the
contraction in test_oracle_model.py.
"""
import math

import numpy as np
import pytest

import oracle


def _dirs(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _wigner_D(l, R):
    X = _dirs(64, 200 + l)
    A = np.array([oracle.real_sh(l, x)[l * l:] for x in X])
    B = np.array([oracle.real_sh(l, R @ x)[l * l:] for x in X])
    D = np.linalg.lstsq(A, B, rcond=None)[0].T
    assert np.abs(A @ D.T - B).max() < 1e-12
    return D


def _rot(seed, proper=True):
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.normal(size=(3, 3)))
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q if proper else -Q


def _one_path(L, q, C, val=1.0):
    Q = len(oracle.sc_paths(L))
    w2 = np.zeros((Q, C))
    w2[q] = val
    return np.zeros((L + 1, C)), w2


def test_coupling_list():
    """(l1 <= l2 <= L, l3 <= L), triangle rule, l1 + l2 + l3 even, lexicographic."""
    assert oracle.sc_paths(2) == [(0, 0, 0), (0, 1, 1), (0, 2, 2), (1, 1, 0), (1, 1, 2), (1, 2, 1),
                                  (2, 2, 0), (2, 2, 2)]
    p3 = oracle.sc_paths(3)
    assert p3 == [(0, 0, 0), (0, 1, 1), (0, 2, 2), (0, 3, 3), (1, 1, 0), (1, 1, 2), (1, 2, 1), (1, 2, 3),
                  (1, 3, 2), (2, 2, 0), (2, 2, 2), (2, 3, 1), (2, 3, 3), (3, 3, 0), (3, 3, 2)]


@pytest.mark.parametrize("L", [2, 3])
def test_linear_term_alone_is_a_channel_scaling(L):
    rng = np.random.default_rng(1)
    D, C = (L + 1) ** 2, 5
    A = rng.normal(size=(D, C))
    w1 = rng.normal(size=(L + 1, C))
    w2 = np.zeros((len(oracle.sc_paths(L)), C))
    B = oracle.sym_contract(L, A, w1, w2)
    for l in range(L + 1):
        np.testing.assert_allclose(B[l * l:(l + 1) ** 2], w1[l] * A[l * l:(l + 1) ** 2], rtol=0, atol=1e-15)


@pytest.mark.parametrize("L", [2, 3])
def test_scalar_times_feature_couplings(L):
    """(0, l, l): B_l = w A_0 A_l (the l1 = 0 coupling is the identity)."""
    rng = np.random.default_rng(2)
    D, C = (L + 1) ** 2, 4
    A = rng.normal(size=(D, C))
    for q, (l1, l2, l3) in enumerate(oracle.sc_paths(L)):
        if l1 != 0:
            continue
        w1, w2 = _one_path(L, q, C, 0.7)
        B = oracle.sym_contract(L, A, w1, w2)
        want = np.zeros_like(A)
        want[l3 * l3:(l3 + 1) ** 2] = 0.7 * A[0] * A[l2 * l2:(l2 + 1) ** 2]
        np.testing.assert_allclose(B, want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("L", [2, 3])
def test_scalar_couplings_are_squared_norms(L):
    """(l, l, 0): B_0 = w |A_l|^2 / sqrt(2l + 1) (positive first entry)."""
    rng = np.random.default_rng(3)
    D, C = (L + 1) ** 2, 3
    A = rng.normal(size=(D, C))
    for q, (l1, l2, l3) in enumerate(oracle.sc_paths(L)):
        if l3 != 0:
            continue
        w1, w2 = _one_path(L, q, C, -1.3)
        B = oracle.sym_contract(L, A, w1, w2)
        blk = A[l1 * l1:(l1 + 1) ** 2]
        np.testing.assert_allclose(B[0], -1.3 * (blk ** 2).sum(0) / math.sqrt(2 * l1 + 1), rtol=1e-14)
        assert np.abs(B[1:]).max() == 0.0


def test_quadrupole_of_a_vector():
    """(1, 1, 2) of an l = 1 feature a: an isometry onto the symmetric
    traceless part of a a^T, so |B_2|^2 = w^2 |a a^T - |a|^2 I / 3|_F^2
    = w^2 (2/3) |a|^4, and B_2 is parallel to Y_2(a / |a|)."""
    L, C = 2, 1
    q = oracle.sc_paths(L).index((1, 1, 2))
    w1, w2 = _one_path(L, q, C, 0.9)
    for a in _dirs(5, 4) * np.array([[0.5], [1.0], [2.0], [3.0], [0.1]]):
        A = np.zeros((9, C))
        A[1:4, 0] = [a[1], a[2], a[0]]  # real l = 1 components in (y, z, x) order
        B = oracle.sym_contract(L, A, w1, w2)[:, 0]
        n2 = np.dot(a, a)
        assert abs((B[4:9] ** 2).sum() - 0.81 * 2.0 / 3.0 * n2 * n2) < 1e-13 * n2 * n2
        y2 = oracle.real_sh(2, a)[4:9]
        cosang = np.dot(B[4:9], y2) / (np.linalg.norm(B[4:9]) * np.linalg.norm(y2))
        assert abs(abs(cosang) - 1.0) < 1e-13
        assert np.abs(B[:4]).max() == 0.0


@pytest.mark.parametrize("L", [2, 3])
def test_homogeneous_quadratic(L):
    rng = np.random.default_rng(5)
    D, C = (L + 1) ** 2, 6
    A = rng.normal(size=(D, C))
    w2 = rng.normal(size=(len(oracle.sc_paths(L)), C))
    w1 = np.zeros((L + 1, C))
    B1 = oracle.sym_contract(L, A, w1, w2)
    B2 = oracle.sym_contract(L, -2.5 * A, w1, w2)
    np.testing.assert_allclose(B2, 6.25 * B1, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("L", [2, 3])
@pytest.mark.parametrize("proper", [True, False])
def test_equivariance(L, proper):
    """B(D A) = D B(A) with block-diagonal Wigner-D of a rotation (or a
    rotation-reflection: natural parity keeps improper rotations too)."""
    rng = np.random.default_rng(6)
    D_, C = (L + 1) ** 2, 4
    A = rng.normal(size=(D_, C))
    w1 = rng.normal(size=(L + 1, C))
    w2 = rng.normal(size=(len(oracle.sc_paths(L)), C))
    R = _rot(7, proper)
    Dm = np.zeros((D_, D_))
    for l in range(L + 1):
        Dm[l * l:(l + 1) ** 2, l * l:(l + 1) ** 2] = _wigner_D(l, R)
    lhs = oracle.sym_contract(L, Dm @ A, w1, w2)
    rhs = Dm @ oracle.sym_contract(L, A, w1, w2)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12 * np.abs(rhs).max())


@pytest.mark.parametrize("L", [2, 3])
def test_adjoint_matches_central_differences(L):
    rng = np.random.default_rng(8)
    D, C = (L + 1) ** 2, 3
    A = rng.normal(size=(D, C))
    w1 = rng.normal(size=(L + 1, C))
    w2 = rng.normal(size=(len(oracle.sc_paths(L)), C))
    GB = rng.normal(size=(D, C))
    GA = oracle.sym_contract_adjoint(L, A, w1, w2, GB)
    for k in range(4):
        V = rng.normal(size=(D, C))
        h = 1e-5
        fd = (np.sum(GB * oracle.sym_contract(L, A + h * V, w1, w2)) -
              np.sum(GB * oracle.sym_contract(L, A - h * V, w1, w2))) / (2 * h)
        # B is quadratic in A: the central difference is exact up to rounding
        assert abs(fd - np.sum(GA * V)) < 1e-8 * max(1.0, abs(fd))
