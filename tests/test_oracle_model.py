"""Whole-model pins of the FP64 oracle.

The potential has no published values to compare with (random weights), so the
oracle is pinned by what the mathematics fixes: invariances of E, covariance of
F, extensivity over a supercell, momentum conservation, forces equal to
forward-mode dual derivatives and to finite differences, stress equal to the
strain derivative, a dimer reduced by hand, and equivariance of the
feature-level tensor product under Wigner-D matrices.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def tiny_spec(L=2, T=2, C=8, H=16, avg_nb=10.0, correlation=0, gate=0):
    return synth.ModelSpec(S=4, T=T, C=C, L=L, H=H, avg_nb=avg_nb, correlation=correlation, gate=gate)


def _rot(seed, proper=True):
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.normal(size=(3, 3)))
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q if proper else -Q


def small_water(n_mol=8, seed=11):
    return synth.water_box(n_mol, synth.water_side_for(n_mol) * 1.0, seed=seed, d_oo=2.5)


@pytest.fixture(scope="module", params=[(0, 0), (2, 0), (0, 1)], ids=["plain", "symcontract2", "gated"])
def models(request):
    """Models of both node orders: the plain layer, with the symmetric
    contraction of correlation order 2 after every scatter-sum, and with the
    species self-connection and gated update."""
    out = {}
    for L in (2, 3):
        spec = tiny_spec(L=L, correlation=request.param[0], gate=request.param[1])
        out[L] = (spec, oracle.Model(spec, synth.make_weights(spec, 100 + L)))
    return out


def test_dimer_closed_form():
    """T = 1 and scalar initial features: only the (0,0,0) path reaches the
    energy, E = sum_i W_out[z_i] . (h0_i + silu(s w000(r) h0_j Y00 W_mix0)) + E0."""
    spec = synth.model_spec("small")
    w = synth.make_weights(spec, 5)
    P = synth.split_weights(spec, w)
    # give E0 nonzero values to pin that term as well
    w = w.copy()
    w[-4:] = np.array([0.1, -0.2, 0.3, -0.4], np.float32)
    P = synth.split_weights(spec, w)
    m = oracle.Model(spec, w)
    z = np.array([1, 3], np.int32)
    rc, s = spec.rc, 1.0 / spec.avg_nb

    def closed(r):
        n = np.arange(1, 9)
        x = r / rc
        u = 1 - 28 * x ** 6 + 48 * x ** 7 - 21 * x ** 8 if x < 1 else 0.0
        b = math.sqrt(2 / rc) * np.sin(n * math.pi * r / rc) / r * u
        silu = lambda a: a / (1 + np.exp(-a))
        z2 = silu(silu(b @ P["W1.0"].astype(np.float64)) @ P["W2.0"].astype(np.float64))
        w000 = z2 @ P["W3.0"][:, 0, :].astype(np.float64)
        h0 = P["W_emb"].astype(np.float64)[z]
        Y00 = 0.5 / math.sqrt(math.pi)
        E = 0.0
        for i, j in ((0, 1), (1, 0)):
            mi = s * w000 * h0[j] * Y00
            h1 = h0[i] + silu(mi @ P["Wmix.0"][0].astype(np.float64))
            E += P["W_out"].astype(np.float64)[z[i]] @ h1 + float(P["E0"][z[i]])
        return E

    for r in (0.8, 1.7, 3.3, 4.9, 5.5):
        pos = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3]]) + np.array([[0, 0, 0], [r / math.sqrt(3)] * 3])
        out = m.energy_forces(pos, z, np.eye(3) * 20, np.zeros(3, np.uint8))
        assert abs(out["energy"] - closed(r)) < 1e-12 * max(1, abs(closed(r)))
        h = 1e-5
        dEdr = (closed(r + h) - closed(r - h)) / (2 * h)
        u = (pos[1] - pos[0]) / r
        # F_1 = -dE/dr * u ; F_0 = +dE/dr * u
        np.testing.assert_allclose(out["forces"][1], -dEdr * u, atol=1e-8)
        np.testing.assert_allclose(out["forces"][0], dEdr * u, atol=1e-8)


@pytest.mark.parametrize("L", [2, 3])
def test_rotation_reflection_invariance(models, L):
    spec, m = models[L]
    s = synth.cluster(20, seed=3, side=6.0)
    ref = m.energy_forces(s.pos, s.species, s.cell, s.pbc)
    for k, proper in enumerate((True, False, True)):
        R = _rot(10 + k, proper)
        pos = s.pos @ R.T + np.array([1.5, -2.0, 0.7])
        out = m.energy_forces(pos, s.species, s.cell, s.pbc)
        assert abs(out["energy"] - ref["energy"]) < 1e-12 * abs(ref["energy"])
        np.testing.assert_allclose(out["forces"], ref["forces"] @ R.T, atol=1e-12 * np.abs(ref["forces"]).max() * 10)


@pytest.mark.parametrize("L", [2, 3])
def test_periodic_invariances(models, L):
    spec, m = models[L]
    s = small_water()
    ref = m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True)
    E0 = ref["energy"]
    tol = 1e-11 * abs(E0)
    # translation
    out = m.energy_forces(s.pos + np.array([0.37, -1.1, 2.9]), s.species, s.cell, s.pbc)
    assert abs(out["energy"] - E0) < tol
    # permutation (with species)
    perm = np.random.default_rng(4).permutation(s.n)
    out = m.energy_forces(s.pos[perm], s.species[perm], s.cell, s.pbc)
    assert abs(out["energy"] - E0) < tol
    np.testing.assert_allclose(out["forces"], ref["forces"][perm], atol=1e-13)
    # lattice-vector shifts of single atoms
    pos = s.pos.copy()
    pos[0] += s.cell[0] * 2 - s.cell[2]
    pos[5] -= s.cell[1]
    out = m.energy_forces(pos, s.species, s.cell, s.pbc)
    assert abs(out["energy"] - E0) < tol
    np.testing.assert_allclose(out["forces"], ref["forces"], atol=1e-12)
    # rotating the whole periodic system (cell and positions)
    R = _rot(21)
    out = m.energy_forces(s.pos @ R.T, s.species, s.cell @ R.T, s.pbc, stress=True)
    assert abs(out["energy"] - E0) < tol
    np.testing.assert_allclose(out["stress"], R @ ref["stress"] @ R.T, atol=1e-12)


def test_supercell_extensive(models):
    spec, m = models[2]
    s = small_water(n_mol=6, seed=12)
    ref = m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True)
    reps = [np.array([a, b, c]) for a in range(2) for b in range(2) for c in range(2)]
    pos = np.concatenate([s.pos + r @ s.cell for r in reps])
    sp = np.tile(s.species, 8)
    out = m.energy_forces(pos, sp, s.cell * 2, s.pbc, stress=True)
    assert abs(out["energy"] - 8 * ref["energy"]) < 1e-11 * abs(8 * ref["energy"])
    np.testing.assert_allclose(out["forces"], np.tile(ref["forces"], (8, 1)), atol=1e-12)
    np.testing.assert_allclose(out["stress"], ref["stress"], atol=1e-13)


@pytest.mark.parametrize("L", [2, 3])
def test_forces_match_dual_numbers(models, L):
    spec, m = models[L]
    s = small_water(n_mol=5, seed=13)
    ref = m.energy_forces(s.pos, s.species, s.cell, s.pbc)
    F = ref["forces"]
    assert np.abs(F.sum(0)).max() < 1e-13 * max(1.0, np.abs(F).max() * s.n)
    for a in range(s.n):
        for ax in range(3):
            E, dE = m.energy_dual(s.pos, s.species, s.cell, s.pbc, a, ax)
            assert abs(E - ref["energy"]) < 1e-13 * abs(E)
            assert abs(-dE - F[a, ax]) < 1e-12 * np.abs(F).max()


def test_forces_match_finite_differences(models):
    spec, m = models[3]
    s = synth.cluster(16, seed=7, side=5.0)
    ref = m.energy_forces(s.pos, s.species, s.cell, s.pbc)
    h = 1e-4
    scale = np.abs(ref["forces"]).max()
    for a in (0, 5, 11):
        for ax in range(3):
            p1 = s.pos.copy(); p1[a, ax] += h
            p2 = s.pos.copy(); p2[a, ax] -= h
            fd = -(m.energy(p1, s.species, s.cell, s.pbc) - m.energy(p2, s.species, s.cell, s.pbc)) / (2 * h)
            assert abs(fd - ref["forces"][a, ax]) < 1e-6 * scale


@pytest.mark.parametrize("L", [2, 3])
def test_stress_matches_strain_derivative(models, L):
    spec, m = models[L]
    s = small_water(n_mol=6, seed=14)
    # a triclinic cell exercises the off-diagonal terms
    cell = s.cell + np.array([[0, 0.4, -0.3], [0.2, 0, 0.5], [-0.1, 0.3, 0]])
    ref = m.energy_forces(s.pos, s.species, cell, s.pbc, stress=True)
    V = abs(np.linalg.det(cell))
    S = ref["stress"]
    np.testing.assert_allclose(S, S.T, atol=1e-13)
    h = 1e-5
    for a in range(3):
        for b in range(3):
            eps = np.zeros((3, 3)); eps[a, b] += 0.5 * h; eps[b, a] += 0.5 * h
            Ep = m.energy(s.pos @ (np.eye(3) + eps).T, s.species, cell @ (np.eye(3) + eps).T, s.pbc)
            Em = m.energy(s.pos @ (np.eye(3) - eps).T, s.species, cell @ (np.eye(3) - eps).T, s.pbc)
            fd = (Ep - Em) / (2 * h) / V
            assert abs(fd - S[a, b]) < 1e-7 * np.abs(S).max() + 1e-12


def test_thin_triclinic_cell_images(models):
    """A cell thinner than the cutoff: many self-images; invariances still hold."""
    spec, m = models[2]
    cell = np.array([[3.1, 0.0, 0.0], [1.2, 3.4, 0.0], [0.5, -0.7, 9.0]])
    rng = np.random.default_rng(8)
    pos = rng.uniform(size=(4, 3)) @ cell
    sp = np.array([0, 1, 2, 3], np.int32)
    pbc = np.ones(3, np.uint8)
    ref = m.energy_forces(pos, sp, cell, pbc, stress=True)
    assert np.abs(ref["forces"].sum(0)).max() < 1e-12
    # 2x1x1 supercell is extensive
    pos2 = np.concatenate([pos, pos + cell[0]])
    out = m.energy_forces(pos2, np.tile(sp, 2), cell * np.array([[2], [1], [1]]), pbc)
    assert abs(out["energy"] - 2 * ref["energy"]) < 1e-11 * abs(ref["energy"])


@pytest.mark.parametrize("L", [2, 3])
def test_tensor_product_equivariance(L):
    """TP(D h, R v) = D TP(h, v) for features of every l, random weights."""
    from test_oracle_sh_cg import _wigner_D  # noqa
    rng = np.random.default_rng(9)
    C = 5
    D_L = (L + 1) ** 2
    P = len(oracle.paths(L))
    h = rng.normal(size=(D_L, C))
    w = rng.normal(size=(P, C))
    v = rng.normal(size=3)
    for proper in (True, False):
        R = _rot(30, proper)
        Ds = [_wigner_D(l, R) for l in range(L + 1)]
        Dbig = np.zeros((D_L, D_L))
        for l in range(L + 1):
            Dbig[l * l:(l + 1) ** 2, l * l:(l + 1) ** 2] = Ds[l]
        t = oracle.tp(L, 3, h, v, w)
        t_rot = oracle.tp(L, 3, Dbig @ h, R @ v, w)
        np.testing.assert_allclose(t_rot, Dbig @ t, atol=1e-12)
        # every path contributes: zeroing one path's weight changes the output
    for p in range(P):
        w2 = w.copy(); w2[p] = 0
        assert np.abs(oracle.tp(L, 3, h, v, w2) - oracle.tp(L, 3, h, v, w)).max() > 1e-6


def test_cutoff_and_isolated_atoms():
    """Atoms farther apart than rc interact not at all: E = sum of readouts of
    the embeddings (with T layers of zero messages)."""
    spec = tiny_spec(L=2)
    w = synth.make_weights(spec, 77)
    P = synth.split_weights(spec, w)
    m = oracle.Model(spec, w)
    pos = np.array([[0, 0, 0], [5.0001, 0, 0], [0, 0, 10.5]])
    sp = np.array([0, 2, 3], np.int32)
    out = m.energy_forces(pos, sp, np.eye(3), np.zeros(3, np.uint8))
    silu0 = 0.0  # silu(0) = 0, so zero messages leave h unchanged
    Eref = sum(float(P["W_out"][z].astype(np.float64) @ P["W_emb"][z].astype(np.float64)) for z in sp) + silu0
    assert abs(out["energy"] - Eref) < 1e-12
    assert np.abs(out["forces"]).max() == 0.0
