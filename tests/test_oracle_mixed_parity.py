"""Pins of the oracle's mixed-parity option (parity = 1): the irreps of the
paper's NequIP table (Table tbl:nequip_params, 0e + 0o + 1o + 1e + 2e + 2o),
here with C/2 channels of each order and parity; channel c < C/2 is the even
block.  Paths: every triangle-valid (l1, l2, l3), odd l1 + l2 + l3 included
(pseudotensor couplings); an odd-l2 path couples a channel to its partner in
the other block; the odd scalars take tanh (an odd function) in the update.

Pinned against: a hand list of the 18 paths for l_max 2; the (1, 1, 1)
coupling equal to the cross product in the (y, z, x) component order of the
harmonics; CG orthogonality; Wigner-D intertwining of every odd path, with the
extra sign -1 under improper rotations (pseudotensors); node features of
every layer transforming by their parity labels under proper and improper
rotations; energy invariance under rotations and reflections; forces equal to
central differences; the weights outside the parity blocks having no effect."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth

PATHS_L2 = [(0, 0, 0), (0, 1, 1), (0, 2, 2),
            (1, 0, 1), (1, 1, 0), (1, 1, 1), (1, 1, 2), (1, 2, 1), (1, 2, 2), (1, 3, 2),
            (2, 0, 2), (2, 1, 1), (2, 1, 2), (2, 2, 0), (2, 2, 1), (2, 2, 2), (2, 3, 1), (2, 3, 2)]


def _rand_dirs(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _wigner_D(l, R):
    X = _rand_dirs(64, 7)
    A = np.array([oracle.real_sh(l, x)[l * l:] for x in X])
    B = np.array([oracle.real_sh(l, R @ x)[l * l:] for x in X])
    D = np.linalg.lstsq(A, B, rcond=None)[0].T
    assert np.abs(A @ D.T - B).max() < 1e-12
    return D


def _rotation(seed, proper):
    Q, Rm = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    Q = Q * np.sign(np.diag(Rm))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q if proper else -Q


def test_paths_l2_hand_list():
    assert oracle.paths(2, 3, all_parities=True) == PATHS_L2
    assert len(oracle.paths(3, 3, all_parities=True)) == 34
    natural = oracle.paths(3, 3)
    assert [p for p in oracle.paths(3, 3, all_parities=True) if sum(p) % 2 == 0] == natural


def test_111_is_the_cross_product():
    """(a x b) in the harmonics' (y, z, x) order: C[k][i][j] = eps(c_k, c_i, c_j) / sqrt 2
    with c = (y, z, x) -> Cartesian (1, 2, 0); the sign rule makes C[0][1][2] positive."""
    cart = [1, 2, 0]
    eps = np.zeros((3, 3, 3))
    for (a, b, c), v in {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1, (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}.items():
        eps[a, b, c] = v
    want = np.array([[[eps[cart[k], cart[i], cart[j]] for j in range(3)] for i in range(3)] for k in range(3)])
    np.testing.assert_allclose(oracle.real_cg(1, 1, 1), want / np.sqrt(2.0), atol=1e-14)


@pytest.mark.parametrize("L", [2, 3])
def test_odd_paths_orthonormal_and_pseudotensor_intertwiners(L):
    Dp = [_wigner_D(l, _rotation(3, True)) for l in range(4)]
    Di = [_wigner_D(l, _rotation(4, False)) for l in range(4)]
    for (l1, l2, l3) in oracle.paths(L, 3, all_parities=True):
        if (l1 + l2 + l3) % 2 == 0:
            continue
        C = oracle.real_cg(l1, l2, l3)
        G = np.einsum("aij,bij->ab", C, C)
        np.testing.assert_allclose(G, np.eye(2 * l3 + 1), atol=1e-12)
        for D, sign in ((Dp, 1.0), (Di, -1.0)):  # improper rotations: the pseudotensor's extra -1
            lhs = np.einsum("ab,bij->aij", D[l3], C)
            rhs = np.einsum("aij,ip,jq->apq", C, D[l1], D[l2])
            np.testing.assert_allclose(lhs, sign * rhs, atol=1e-12)


def _model(T=3, C=8, L=2, seed=5):
    # a small message scale 1/avg_nb = 4 makes the odd scalars of the third layer
    # large enough (~3e-3 of max |h|) that an activation without odd symmetry
    # there would break the feature pin well above its tolerance
    spec = synth.ModelSpec(S=4, T=T, C=C, L=L, H=16, avg_nb=0.25, parity=1)
    return spec, oracle.Model(spec, synth.make_weights(spec, seed))


def _cluster():
    return synth.cluster(10, seed=3, side=4.0)


@pytest.mark.parametrize("proper", [True, False])
def test_features_transform_by_their_parity(proper):
    """h_t(R x) = f D^l(R) h_t(x) per order l and block: f = 1 for proper R and
    p (-1)^l for improper R (p = +1 even block, -1 odd block), at every layer
    of a three-layer model (the odd scalars appear at the third)."""
    spec, m = _model(T=3)
    s = _cluster()
    R = _rotation(11, proper)
    Ch = spec.C // 2
    D = [_wigner_D(l, R) for l in range(spec.L + 1)]
    seen_odd_scalar = False
    for t in range(1, spec.T + 1):
        h = m.node_features(s.pos, s.species, s.cell, s.pbc, t)
        hr = m.node_features(s.pos @ R.T, s.species, s.cell, s.pbc, t)
        scale = np.abs(h).max()
        for l in range(spec.L + 1):
            blk = slice(l * l, (l + 1) ** 2)
            for b, p in ((slice(0, Ch), 1.0), (slice(Ch, spec.C), -1.0)):
                f = 1.0 if proper else p * (-1.0) ** l
                want = f * np.einsum("ab,nbc->nac", D[l], h[:, blk, b])
                np.testing.assert_allclose(hr[:, blk, b], want, atol=1e-11 * scale)
        seen_odd_scalar |= np.abs(h[:, 0, Ch:]).max() > 1e-3 * scale
    assert seen_odd_scalar  # the odd scalars (and their tanh) take part


def test_energy_invariant_under_rotations_and_reflections():
    spec, m = _model(T=3)
    s = _cluster()
    E0 = m.energy_forces(s.pos, s.species, s.cell, s.pbc)["energy"]
    for seed, proper in ((1, True), (2, False), (3, False)):
        R = _rotation(seed, proper)
        E = m.energy_forces(s.pos @ R.T + np.array([0.3, -1.1, 2.0]), s.species, s.cell, s.pbc)["energy"]
        assert abs(E - E0) <= 1e-12 * max(1.0, abs(E0))


def test_forces_equal_central_differences():
    spec, m = _model(T=2)
    s = _cluster()
    F = m.energy_forces(s.pos, s.species, s.cell, s.pbc)["forces"]
    h = 1e-5
    for i, a in ((0, 0), (4, 1), (9, 2)):
        p1, p2 = s.pos.copy(), s.pos.copy()
        p1[i, a] += h
        p2[i, a] -= h
        fd = -(m.energy_forces(p1, s.species, s.cell, s.pbc)["energy"] -
               m.energy_forces(p2, s.species, s.cell, s.pbc)["energy"]) / (2 * h)
        assert abs(F[i, a] - fd) <= 1e-6 * np.abs(F).max()
    assert np.abs(F.sum(axis=0)).max() <= 1e-12 * np.abs(F).max() * s.n


def test_weights_outside_the_parity_blocks_have_no_effect():
    spec, m = _model(T=2)
    w = synth.make_weights(spec, 5)
    parts = synth.split_weights(spec, w.copy())
    Ch = spec.C // 2
    parts["W_emb"][:, Ch:] += 1.0
    parts["W_out"][:, Ch:] -= 2.0
    for t in range(spec.T):
        parts[f"Wmix.{t}"][:, :Ch, Ch:] += 0.5
        parts[f"Wmix.{t}"][:, Ch:, :Ch] -= 0.5
    w2 = np.concatenate([parts[name].reshape(-1) for name, _, _ in spec.weight_shapes()]).astype(np.float32)
    s = _cluster()
    a = m.energy_forces(s.pos, s.species, s.cell, s.pbc)
    b = oracle.Model(spec, w2).energy_forces(s.pos, s.species, s.cell, s.pbc)
    assert a["energy"] == b["energy"] and np.array_equal(a["forces"], b["forces"])


def test_mixed_parity_excludes_the_other_options():
    spec = dataclasses.replace(_model()[0], gate=1)
    with pytest.raises(ValueError):
        oracle.Model(spec, synth.make_weights(spec, 1))
