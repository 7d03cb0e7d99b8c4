"""Pins of the oracle's charge head, charge correction (Eq. charge_correction)
and soft-core Coulomb term (Eq. long_range_interaction, PhysNet's surrogate
distance chi).

Fixed by physics and by the definition: Coulomb's law for point charges
beyond the soft-core radius (energy, forces, each pair counted once,
superposition), the surrogate's limits (exactly 1/r beyond r0, value 1 at
r -> 0, value and slope continuous at r0), forces and charge derivatives
against central differences inside the soft core, and for whole models with
the charge head: corrected charges summing to the total charge, forces equal
to forward-mode dual numbers and to differences, invariances, momentum
conservation, and a dimer reduced by hand.
"""
import math

import numpy as np
import pytest

import oracle
import synth

KE = 14.3996454784  # e^2 / (4 pi eps0), eV A


def test_coulombs_law_for_two_charges():
    r0 = 2.5
    for r, q1, q2 in ((3.0, 0.4, -0.7), (5.5, 1.0, 1.0), (12.0, -0.3, 0.9)):
        u = np.array([0.36, -0.48, 0.8])
        pos = np.array([[0.1, 0.2, -0.3], [0.1, 0.2, -0.3]]) + np.outer([0.0, r], u)
        E, g, F = oracle.coulomb(pos, [q1, q2], r0)
        assert abs(E - KE * q1 * q2 / r) < 1e-13 * abs(E)
        np.testing.assert_allclose(g, [KE * q2 / r, KE * q1 / r], rtol=1e-13)
        # like charges repel: the force on atom 1 points away from atom 0
        np.testing.assert_allclose(F[1], KE * q1 * q2 / r ** 2 * u, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(F[0], -F[1], rtol=1e-13, atol=1e-15)


def test_superposition_each_pair_once():
    rng = np.random.default_rng(1)
    pos = rng.uniform(0, 20, size=(6, 3))
    pos[:, 0] += 7.0 * np.arange(6)  # every pair beyond the soft core
    q = rng.normal(size=6)
    E, _, _ = oracle.coulomb(pos, q, 2.5)
    want = sum(KE * q[i] * q[j] / np.linalg.norm(pos[i] - pos[j]) for i in range(6) for j in range(i + 1, 6))
    assert abs(E - want) < 1e-12 * abs(want)


def test_surrogate_distance_limits():
    r0 = 2.5
    for r in (2.5, 2.6, 4.0, 9.0):
        assert oracle.inv_chi(r, r0) == pytest.approx(1.0 / r, rel=1e-15)
    assert abs(oracle.inv_chi(1e-7, r0) - 1.0) < 1e-6
    # value and slope continuous at r0
    h = 1e-6
    assert abs(oracle.inv_chi(r0 - h, r0) - 1.0 / r0) < 2 * h / r0 ** 2
    slope_in = (oracle.inv_chi(r0 - h, r0) - oracle.inv_chi(r0 - 2 * h, r0)) / h
    assert abs(slope_in + 1.0 / r0 ** 2) < 1e-5


def test_soft_core_forces_and_charge_derivatives_match_differences():
    rng = np.random.default_rng(2)
    pos = rng.uniform(0, 3.0, size=(5, 3))  # most pairs inside the soft core
    q = rng.normal(size=5)
    r0 = 2.5
    E, g, F = oracle.coulomb(pos, q, r0)
    h = 1e-6
    for a in range(5):
        for ax in range(3):
            p1 = pos.copy(); p1[a, ax] += h
            p2 = pos.copy(); p2[a, ax] -= h
            fd = -(oracle.coulomb(p1, q, r0)[0] - oracle.coulomb(p2, q, r0)[0]) / (2 * h)
            assert abs(fd - F[a, ax]) < 1e-7 * max(1.0, np.abs(F).max())
        q1 = q.copy(); q1[a] += h
        q2 = q.copy(); q2[a] -= h
        fd = (oracle.coulomb(pos, q1, r0)[0] - oracle.coulomb(pos, q2, r0)[0]) / (2 * h)
        assert abs(fd - g[a]) < 1e-7 * max(1.0, np.abs(g).max())


@pytest.fixture(scope="module")
def charged():
    spec = synth.ModelSpec(S=4, T=2, C=8, L=2, H=16, avg_nb=10.0, charges=1, coulomb_r0=2.5)
    return spec, oracle.Model(spec, synth.make_weights(spec, 33))


@pytest.mark.parametrize("Q", [0.0, -1.0, 2.0])
def test_corrected_charges_sum_to_the_total(charged, Q):
    spec, m = charged
    s = synth.cluster(30, seed=4, side=7.0)
    m.set_total_charge(Q)
    q = m.charges(s.pos, s.species)
    assert abs(q.sum() - Q) < 1e-12 * max(1.0, np.abs(q).sum())
    m.set_total_charge(0.0)


@pytest.mark.parametrize("Q", [0.0, 1.0])
def test_forces_match_dual_numbers_and_differences(charged, Q):
    spec, m = charged
    m.set_total_charge(Q)
    s = synth.cluster(14, seed=6, side=5.0)
    ref = m.energy_forces(s.pos, s.species, s.cell, s.pbc)
    F = ref["forces"]
    assert np.abs(F.sum(0)).max() < 1e-12 * max(1.0, np.abs(F).max() * s.n)
    for a in range(s.n):
        for ax in range(3):
            E, dE = m.energy_dual(s.pos, s.species, s.cell, s.pbc, a, ax)
            assert abs(-dE - F[a, ax]) < 1e-12 * np.abs(F).max()
    h = 1e-4
    for a in (0, 7):
        for ax in range(3):
            p1 = s.pos.copy(); p1[a, ax] += h
            p2 = s.pos.copy(); p2[a, ax] -= h
            fd = -(m.energy(p1, s.species, s.cell, s.pbc) - m.energy(p2, s.species, s.cell, s.pbc)) / (2 * h)
            assert abs(fd - F[a, ax]) < 1e-6 * np.abs(F).max()
    m.set_total_charge(0.0)


def test_invariances(charged):
    spec, m = charged
    m.set_total_charge(-1.0)
    s = synth.cluster(20, seed=3, side=6.0)
    ref = m.energy_forces(s.pos, s.species, s.cell, s.pbc)
    rng = np.random.default_rng(9)
    Qm, Rm = np.linalg.qr(rng.normal(size=(3, 3)))
    Rot = Qm * np.sign(np.diag(Rm))
    for R in (Rot, -Rot):  # proper and improper
        out = m.energy_forces(s.pos @ R.T + np.array([2.0, -1.0, 0.5]), s.species, s.cell, s.pbc)
        assert abs(out["energy"] - ref["energy"]) < 1e-12 * abs(ref["energy"])
        np.testing.assert_allclose(out["forces"], ref["forces"] @ R.T, atol=1e-12 * np.abs(ref["forces"]).max() * 10)
    perm = rng.permutation(s.n)
    out = m.energy_forces(s.pos[perm], s.species[perm], s.cell, s.pbc)
    assert abs(out["energy"] - ref["energy"]) < 1e-12 * abs(ref["energy"])
    np.testing.assert_allclose(out["forces"], ref["forces"][perm], atol=1e-13 * np.abs(ref["forces"]).max() * 10)
    m.set_total_charge(0.0)


def test_periodic_systems_are_rejected(charged):
    spec, m = charged
    s = synth.water_box(8, synth.water_side_for(8), seed=1, d_oo=2.5)
    with pytest.raises(ValueError):
        m.energy_forces(s.pos, s.species, s.cell, s.pbc)


def test_dimer_closed_form_with_charges():
    """T = 1, scalar features: h_i = h0_i + silu(s w000(r) h0_j Y00 W_mix0);
    q_i = W_q[z_i] . h_i + q0[z_i], corrected to Q over the two atoms, and
    E = sum_i (W_out[z_i] . h_i + E0[z_i]) + k qt_0 qt_1 / r beyond r0."""
    spec = synth.dataclasses.replace(synth.model_spec("small"), charges=1, coulomb_r0=2.5)
    w = synth.make_weights(spec, 5).copy()
    w[-4:] = np.array([0.05, -0.1, 0.2, -0.15], np.float32)  # q0
    P = synth.split_weights(spec, w)
    m = oracle.Model(spec, w)
    z = np.array([1, 3], np.int32)
    rc, s = spec.rc, 1.0 / spec.avg_nb
    silu = lambda a: a / (1 + np.exp(-a))
    f64 = lambda k: P[k].astype(np.float64)

    def closed(r, Q):
        n = np.arange(1, 9)
        x = r / rc
        u = 1 - 28 * x ** 6 + 48 * x ** 7 - 21 * x ** 8 if x < 1 else 0.0
        b = math.sqrt(2 / rc) * np.sin(n * math.pi * r / rc) / r * u
        w000 = silu(silu(b @ f64("W1.0")) @ f64("W2.0")) @ f64("W3.0")[:, 0, :]
        h0 = f64("W_emb")[z]
        Y00 = 0.5 / math.sqrt(math.pi)
        h1 = [h0[i] + silu((s * w000 * h0[j] * Y00) @ f64("Wmix.0")[0]) for i, j in ((0, 1), (1, 0))]
        E = sum(f64("W_out")[z[i]] @ h1[i] + float(P["E0"][z[i]]) for i in range(2))
        q = np.array([f64("W_q")[z[i]] @ h1[i] + float(P["q0"][z[i]]) for i in range(2)])
        q -= (q.sum() - Q) / 2
        return E + KE * q[0] * q[1] / r

    for Q in (0.0, 1.0):
        m.set_total_charge(Q)
        for r in (2.7, 3.3, 4.9, 5.5):
            pos = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3]]) + np.array([[0, 0, 0], [r / math.sqrt(3)] * 3])
            out = m.energy_forces(pos, z, np.eye(3) * 20, np.zeros(3, np.uint8))
            assert abs(out["energy"] - closed(r, Q)) < 1e-12 * max(1, abs(closed(r, Q)))
            h = 1e-5
            dEdr = (closed(r + h, Q) - closed(r - h, Q)) / (2 * h)
            u = (pos[1] - pos[0]) / r
            np.testing.assert_allclose(out["forces"][1], -dEdr * u, atol=1e-8)
    m.set_total_charge(0.0)
