"""Pins of the oracle's Hessian rows (Eq. full_hessian; the subsampled rows of
Eq. sampled_hessian2), computed by hyper-dual numbers through the templated
energy: every row equals the central differences of the oracle's own forces
(H = -dF/dr), the Hessian is symmetric, translation invariance makes every
row sum to zero over the atoms, the 3x3 blocks rotate as R H R^T, and a row
of a batch of non-interacting graphs is the concatenation of each graph's
row (zero on the other graphs' atoms).  On every model variant."""
import numpy as np
import pytest

import oracle
import synth

VARIANTS = {
    "plain": {},
    "symcontract2": {"correlation": 2},
    "gated": {"gate": 1},
    "charged": {"charges": 1, "coulomb_r0": 2.5},
}


@pytest.fixture(scope="module", params=list(VARIANTS))
def model(request):
    spec = synth.ModelSpec(S=4, T=2, C=8, L=2, H=16, avg_nb=10.0, **VARIANTS[request.param])
    m = oracle.Model(spec, synth.make_weights(spec, 41))
    if spec.charges:
        m.set_total_charge(1.0)
    return spec, m


def _cluster():
    return synth.cluster(12, seed=5, side=4.5)


def test_rows_equal_differences_of_the_forces(model):
    spec, m = model
    s = _cluster()
    h = 1e-4
    for atom, axis in ((0, 0), (3, 1), (9, 2)):
        H = m.hessian_row(s.pos, s.species, s.cell, s.pbc, atom, axis)
        p1 = s.pos.copy(); p1[atom, axis] += h
        p2 = s.pos.copy(); p2[atom, axis] -= h
        fd = -(m.energy_forces(p1, s.species, s.cell, s.pbc)["forces"] -
               m.energy_forces(p2, s.species, s.cell, s.pbc)["forces"]) / (2 * h)
        assert np.abs(H - fd).max() < 1e-6 * np.abs(H).max()


def test_symmetric_and_translation_invariant(model):
    spec, m = model
    s = _cluster()
    rows = {(i, a): m.hessian_row(s.pos, s.species, s.cell, s.pbc, i, a) for i in (1, 6) for a in range(3)}
    scale = max(np.abs(r).max() for r in rows.values())
    for (i, a), r in rows.items():
        assert np.abs(r.sum(axis=0)).max() < 1e-12 * scale * s.n
        for (j, b), q in rows.items():
            assert abs(r[j, b] - q[i, a]) < 1e-12 * scale


def test_blocks_rotate(model):
    spec, m = model
    s = _cluster()
    rng = np.random.default_rng(3)
    Q, Rr = np.linalg.qr(rng.normal(size=(3, 3)))
    R = Q * np.sign(np.diag(Rr))
    i = 4
    H = np.stack([m.hessian_row(s.pos, s.species, s.cell, s.pbc, i, a) for a in range(3)])  # [a][j][b]
    Hr = np.stack([m.hessian_row(s.pos @ R.T, s.species, s.cell, s.pbc, i, a) for a in range(3)])
    want = np.einsum("ap,pjq,bq->ajb", R, H, R)
    np.testing.assert_allclose(Hr, want, atol=1e-11 * np.abs(H).max())


def test_row_of_a_batch_of_graphs_concatenates_the_graphs_rows():
    """Eq. sampled_hessian2: distinct graphs do not interact, so the row of
    atom i of graph g in the batch is graph g's own row, zero elsewhere."""
    spec = synth.ModelSpec(S=4, T=2, C=8, L=2, H=16, avg_nb=10.0)
    m = oracle.Model(spec, synth.make_weights(spec, 41))
    a, b = synth.cluster(7, seed=1, side=4.0), synth.cluster(6, seed=2, side=4.0)
    shift = np.array([40.0, 0.0, 0.0])  # far beyond T rc: separate graphs
    pos = np.concatenate([a.pos, b.pos + shift])
    sp = np.concatenate([a.species, b.species]).astype(np.int32)
    cell, pbc = np.eye(3), np.zeros(3, np.uint8)
    for atom, axis, own, off, other in ((2, 1, a, 0, slice(7, 13)), (9, 0, b, 7, slice(0, 7))):
        row = m.hessian_row(pos, sp, cell, pbc, atom, axis)
        alone = m.hessian_row(own.pos, own.species, cell, pbc, atom - off, axis)
        np.testing.assert_allclose(row[off:off + own.n], alone, rtol=0, atol=1e-13 * np.abs(alone).max())
        assert np.abs(row[other]).max() == 0.0
