"""Pins of the oracle's neighbour list and velocity-Verlet integrator.

The neighbour list is compared with a naive enumeration written here in numpy
over a generous fixed range of images (independent of the oracle's reach
computation), with the same inclusion arithmetic: no fused multiply-add, the
shift summed as (S0 h0 + S1 h1) + S2 h2 and d2 as (dx^2 + dy^2) + dz^2.
"""
import numpy as np
import pytest

import oracle
import synth


def naive_pairs(pos, cell, pbc, rc, reach=6):
    rng = [range(-reach, reach + 1) if p else range(0, 1) for p in pbc]
    out = set()
    n = len(pos)
    for S0 in rng[0]:
        for S1 in rng[1]:
            for S2 in rng[2]:
                sv = (S0 * cell[0] + S1 * cell[1]) + S2 * cell[2] if any(pbc) else np.zeros(3)
                d = (pos[None, :, :] - pos[:, None, :]) + sv          # [i, j]
                d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
                ii, jj = np.nonzero(d2 < rc * rc)
                for i, j in zip(ii, jj):
                    if i == j and S0 == 0 and S1 == 0 and S2 == 0:
                        continue
                    out.add((int(i), int(j), S0, S1, S2))
    return out


CASES = [
    ("open", lambda r: (r.uniform(size=(24, 3)) * 8, np.eye(3) * 8, np.zeros(3, np.uint8))),
    ("cubic", lambda r: (r.uniform(size=(20, 3)) * 7, np.eye(3) * 7, np.ones(3, np.uint8))),
    ("thin-triclinic", lambda r: (r.uniform(size=(6, 3)) @ np.array([[2.1, 0, 0], [0.9, 2.4, 0], [0.4, -0.6, 11.0]]),
                                  np.array([[2.1, 0, 0], [0.9, 2.4, 0], [0.4, -0.6, 11.0]]), np.ones(3, np.uint8))),
    ("slab", lambda r: (r.uniform(size=(15, 3)) * np.array([4.0, 5.0, 12.0]), np.diag([4.0, 5.0, 30.0]),
                        np.array([1, 1, 0], np.uint8))),
    ("unwrapped", lambda r: (r.uniform(size=(12, 3)) * 30 - 10, np.array([[6.0, 0, 0], [1.0, 6.5, 0], [0, 0.5, 5.5]]),
                             np.ones(3, np.uint8))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_neighbors_match_naive_enumeration(name, make):
    rng = np.random.default_rng(sum(ord(ch) for ch in name))
    pos, cell, pbc = make(rng)
    recv, send, shift = oracle.neighbors(pos, cell, pbc, 5.0)
    got = [(int(a), int(b), *map(int, s)) for a, b, s in zip(recv, send, shift)]
    assert got == sorted(got)                          # canonical order
    assert len(set(got)) == len(got)
    assert set(got) == naive_pairs(pos, cell, pbc, 5.0)


def test_neighbors_symmetric_and_reverse_edges():
    s = synth.water_box(10, synth.water_side_for(10), seed=5)
    recv, send, shift = oracle.neighbors(s.pos, s.cell, s.pbc, 5.0)
    edges = set((int(a), int(b), *map(int, sh)) for a, b, sh in zip(recv, send, shift))
    for (i, j, a, b, c) in edges:
        assert (j, i, -a, -b, -c) in edges


def test_vv_time_reversible_and_conserving():
    spec = synth.ModelSpec(S=4, T=2, C=8, L=2, H=16, avg_nb=10.0)
    m = oracle.Model(spec, synth.make_weights(spec, 3))
    s = synth.water_box(6, synth.water_side_for(6), seed=9)
    masses = np.asarray(spec.masses)[s.species]
    v0 = synth.maxwell_boltzmann(masses, 300.0, seed=2)
    p1, v1, pe, ke = m.vv_nve(s.pos, v0, s.species, np.asarray(spec.masses), s.cell, s.pbc, 0.5, 20)
    p2, v2, _, _ = m.vv_nve(p1, -v1, s.species, np.asarray(spec.masses), s.cell, s.pbc, 0.5, 20)
    np.testing.assert_allclose(p2, s.pos, atol=1e-10)
    np.testing.assert_allclose(-v2, v0, atol=1e-12)
    etot = pe + ke
    assert np.abs(etot - etot[0]).max() < 1e-3 * max(1e-3, ke.mean())


def test_maxwell_boltzmann_statistics():
    masses = np.full(20000, 15.999)
    v = synth.maxwell_boltzmann(masses, 300.0, seed=1)
    kB, kappa = 8.617333262e-5, 9.648533212e-3
    ke = 0.5 * (masses[:, None] * v ** 2).sum() / kappa
    T = 2 * ke / (3 * masses.size * kB)
    assert abs(T - 300.0) < 6.0
    np.testing.assert_allclose((masses[:, None] * v).sum(0), 0, atol=1e-9)
