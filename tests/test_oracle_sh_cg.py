"""Pins of the oracle's harmonics, Clebsch-Gordan tables, paths and radial basis.

Each check is against something other than the oracle's own formula: closed
forms, textbook tables, orthonormality by quadrature, representation theory
(Wigner-D intertwining estimated from the harmonics themselves) and the Gaunt
integrals computed by quadrature.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_dirs(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _quadrature(n_theta=12, n_phi=24):
    """Gauss-Legendre in cos(theta) x uniform phi: exact for the products of
    harmonics used here (degree <= 2 * n_theta - 1 in z, < n_phi in phi)."""
    z, wz = np.polynomial.legendre.leggauss(n_theta)
    phi = np.arange(n_phi) * 2 * np.pi / n_phi
    Z, PHI = np.meshgrid(z, phi, indexing="ij")
    s = np.sqrt(1 - Z ** 2)
    pts = np.stack([s * np.cos(PHI), s * np.sin(PHI), Z], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).reshape(-1)
    return pts, w


# ------------------------------------------------------------ harmonics
def test_sh_closed_forms():
    """Standard real-harmonic polynomials (no Condon-Shortley phase)."""
    for x, y, z in _rand_dirs(20, 1):
        Y = oracle.real_sh(3, [x, y, z])
        pi = math.pi
        ref = {
            (0, 0): 0.5 / math.sqrt(pi),
            (1, -1): math.sqrt(3 / (4 * pi)) * y,
            (1, 0): math.sqrt(3 / (4 * pi)) * z,
            (1, 1): math.sqrt(3 / (4 * pi)) * x,
            (2, -2): 0.5 * math.sqrt(15 / pi) * x * y,
            (2, -1): 0.5 * math.sqrt(15 / pi) * y * z,
            (2, 0): 0.25 * math.sqrt(5 / pi) * (3 * z * z - 1),
            (2, 1): 0.5 * math.sqrt(15 / pi) * x * z,
            (2, 2): 0.25 * math.sqrt(15 / pi) * (x * x - y * y),
            (3, -3): 0.25 * math.sqrt(35 / (2 * pi)) * y * (3 * x * x - y * y),
            (3, -2): 0.5 * math.sqrt(105 / pi) * x * y * z,
            (3, -1): 0.25 * math.sqrt(21 / (2 * pi)) * y * (5 * z * z - 1),
            (3, 0): 0.25 * math.sqrt(7 / pi) * z * (5 * z * z - 3),
            (3, 1): 0.25 * math.sqrt(21 / (2 * pi)) * x * (5 * z * z - 1),
            (3, 2): 0.25 * math.sqrt(105 / pi) * z * (x * x - y * y),
            (3, 3): 0.25 * math.sqrt(35 / (2 * pi)) * x * (x * x - 3 * y * y),
        }
        for (l, m), v in ref.items():
            assert abs(Y[l * l + m + l] - v) < 1e-14, (l, m)


def test_sh_direction_only():
    v = np.array([0.3, -1.2, 0.7])
    np.testing.assert_allclose(oracle.real_sh(3, v), oracle.real_sh(3, 7.5 * v), atol=1e-15)


def test_sh_addition_theorem():
    for v in _rand_dirs(10, 2):
        Y = oracle.real_sh(6, v)
        for l in range(7):
            s = np.sum(Y[l * l:(l + 1) ** 2] ** 2)
            assert abs(s - (2 * l + 1) / (4 * math.pi)) < 1e-13


def test_sh_orthonormal_by_quadrature():
    pts, w = _quadrature()
    Y = np.array([oracle.real_sh(4, p) for p in pts])
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(25), atol=1e-12)


def test_sh_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    for _ in range(5):
        v = rng.normal(size=3) * 2
        J = oracle.real_sh_grad(3, v)
        h = 1e-6
        for a in range(3):
            e = np.zeros(3); e[a] = h
            fd = (oracle.real_sh(3, v + e) - oracle.real_sh(3, v - e)) / (2 * h)
            np.testing.assert_allclose(J[:, a], fd, atol=1e-8)


def test_real_complex_basis_change():
    """U_l Y^complex = Y^real at random points, and U_l is unitary."""
    for l in range(4):
        U = oracle.real_basis_U(l)
        np.testing.assert_allclose(U @ U.conj().T, np.eye(2 * l + 1), atol=1e-14)
        for v in _rand_dirs(5, 10 + l):
            yc = oracle.complex_sh(l, v)
            yr = oracle.real_sh(l, v)[l * l:(l + 1) ** 2]
            np.testing.assert_allclose(U @ yc, yr, atol=1e-14)


def test_complex_sh_orthonormal_and_condon_shortley():
    pts, w = _quadrature()
    for l in range(4):
        Y = np.array([oracle.complex_sh(l, p) for p in pts])
        G = (Y.conj() * w[:, None]).T @ Y
        np.testing.assert_allclose(G, np.eye(2 * l + 1), atol=1e-12)
    # Y_1^1 = -sqrt(3/8pi) (x + i y): the Condon-Shortley sign
    v = np.array([0.6, 0.0, 0.8])
    y = oracle.complex_sh(1, v)
    assert abs(y[2] - (-math.sqrt(3 / (8 * math.pi)) * 0.6)) < 1e-14


# ----------------------------------------------------------------- CG
def _golden_cg():
    rows = []
    with open(os.path.join(GOLDEN, "cg_complex_1x1.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            l1, m1, l2, m2, l3, m3, sg, num, den = line.split()
            v = math.sqrt(int(num) / int(den)) * (1 if sg == "+" else -1)
            rows.append(((int(l1), int(m1), int(l2), int(m2), int(l3), int(m3)), v))
    return rows


def test_cg_textbook_table():
    for args, v in _golden_cg():
        assert abs(oracle.cg_complex(*args) - v) < 1e-14, args


def test_cg_trivial_coupling():
    for l in range(5):
        for m in range(-l, l + 1):
            assert abs(oracle.cg_complex(l, m, 0, 0, l, m) - 1) < 1e-14
            assert abs(oracle.cg_complex(0, 0, l, m, l, m) - 1) < 1e-14


def test_cg_orthogonality():
    for l1 in range(4):
        for l2 in range(4):
            rows, labels = [], []
            for l3 in range(abs(l1 - l2), l1 + l2 + 1):
                for m3 in range(-l3, l3 + 1):
                    rows.append([oracle.cg_complex(l1, m1, l2, m2, l3, m3)
                                 for m1 in range(-l1, l1 + 1) for m2 in range(-l2, l2 + 1)])
            A = np.array(rows)
            # complete and orthonormal: A is square orthogonal
            assert A.shape[0] == A.shape[1]
            np.testing.assert_allclose(A @ A.T, np.eye(A.shape[0]), atol=1e-13)


def _wigner_D(l, R, seed=0):
    """D^l(R) fitted from Y(R x_k) = D Y(x_k) on 64 random points."""
    X = _rand_dirs(64, 100 + seed)
    A = np.array([oracle.real_sh(l, x)[l * l:] for x in X])
    B = np.array([oracle.real_sh(l, R @ x)[l * l:] for x in X])
    D, res, *_ = np.linalg.lstsq(A, B, rcond=None)
    D = D.T
    assert np.abs(A @ D.T - B).max() < 1e-12
    return D


def _rand_rotation(seed, proper=True):
    rng = np.random.default_rng(seed)
    Q, Rm = np.linalg.qr(rng.normal(size=(3, 3)))
    Q = Q * np.sign(np.diag(Rm))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    if not proper:
        Q = -Q
    return Q


@pytest.mark.parametrize("L", [2, 3])
def test_real_cg_intertwines_rotations(L):
    """D^{l3} C = C (D^{l1} x D^{l2}) for every path, proper and improper R."""
    for proper in (True, False):
        R = _rand_rotation(5, proper)
        D = [_wigner_D(l, R) for l in range(4)]
        for (l1, l2, l3) in oracle.paths(L):
            C = oracle.real_cg(l1, l2, l3)
            lhs = np.einsum("ab,bij->aij", D[l3], C)
            rhs = np.einsum("aij,ip,jq->apq", C, D[l1], D[l2])
            np.testing.assert_allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("L", [2, 3])
def test_real_cg_is_normalised_gaunt(L):
    """Real CG = +-Gaunt integral normalised per row; sign rule: first entry
    (lexicographic in m3, m1, m2) with |c| > 1e-8 is positive."""
    pts, w = _quadrature(12, 24)
    Y = np.array([oracle.real_sh(3, p) for p in pts])
    for (l1, l2, l3) in oracle.paths(L):
        Y1, Y2, Y3 = (Y[:, l * l:(l + 1) ** 2] for l in (l1, l2, l3))
        G = np.einsum("k,ka,kb,kc->abc", w, Y3, Y1, Y2)
        norms = np.sqrt((G ** 2).sum(axis=(1, 2)))
        np.testing.assert_allclose(norms, norms[0], rtol=1e-10)
        G = G / norms[0]
        flat = G.reshape(-1)
        first = flat[np.argmax(np.abs(flat) > 1e-8)]
        G = G * np.sign(first)
        C = oracle.real_cg(l1, l2, l3)
        np.testing.assert_allclose(C, G, atol=1e-12)


def test_real_cg_rows_orthonormal_and_real():
    for (l1, l2, l3) in oracle.paths(3):
        C = oracle.real_cg(l1, l2, l3).reshape(2 * l3 + 1, -1)
        np.testing.assert_allclose(C @ C.T, np.eye(2 * l3 + 1), atol=1e-13)


def test_paths_match_enumeration():
    with open(os.path.join(GOLDEN, "paths.txt")) as f:
        lines = [l for l in f if l.startswith("L=")]
    ref = {int(l[2]): [tuple(int(c) for c in tok) for tok in l.split(":")[1].split()] for l in lines}
    assert oracle.paths(2) == ref[2]
    assert oracle.paths(3) == ref[3]
    assert len(ref[2]) == 13 and len(ref[3]) == 23


# -------------------------------------------------------------- radial
def test_bessel_orthonormal_with_r2_weight():
    """int_0^rc B_n B_m r^2 dr = delta_nm (Gauss-Legendre, 64 points)."""
    rc = 5.0
    x, wx = np.polynomial.legendre.leggauss(64)
    r = 0.5 * rc * (x + 1); wr = 0.5 * rc * wx
    B = np.array([[oracle.bessel(n, ri, rc) for ri in r] for n in range(1, 9)])
    G = (B * r ** 2 * wr) @ B.T
    np.testing.assert_allclose(G, np.eye(8), atol=1e-12)


def test_bessel_small_r_limit():
    rc = 5.0
    for n in range(1, 9):
        lim = math.sqrt(2 / rc) * n * math.pi / rc
        assert abs(oracle.bessel(n, 1e-7, rc) - lim) < 1e-9


def test_envelope_boundary_conditions():
    p = 6
    assert oracle.envelope(0.0, p) == 1.0
    for x in (1.0, 1.2, 3.0):
        assert oracle.envelope(x, p) == 0.0
    u = lambda x: oracle.envelope(x, p)
    # triple zero at x = 1 (value, first and second derivative vanish, third
    # does not): u(1 - e) ~ k e^3, so u(1 - e) / u(1 - 2e) -> 1/8
    for e in (1e-2, 1e-3):
        ratio = u(1 - e) / u(1 - 2 * e)
        assert abs(ratio - 0.125) < 0.02
    assert abs(u(1 - 1e-4)) < 1e-9
    assert 0.0 < u(0.5) < 1.0
    xs = np.linspace(0, 1, 201)
    assert np.all(np.diff([u(x) for x in xs]) <= 1e-15)   # decreasing on [0, 1]
