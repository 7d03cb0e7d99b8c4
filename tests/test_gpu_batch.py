"""GPU checks of batched evaluation: several independent systems evaluated as
one graph (the disjoint union of their neighbour graphs).

A system's results must not depend on the rest of its batch: every per-system
sum runs over chunks counted from the system's own first atom, per-receiver
sums run in the receiver's own edge order, and the FP16 operand scale of the
adjoint is chosen per system.  So the batch results are compared with the
single-system call bit for bit, and one batch is checked against the oracle.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    torch.cuda.init()
    from paper_2605_22698_gb300 import build
    build.build()
    from paper_2605_22698_gb300 import binding
    binding.lib()
    return binding


def _systems():
    """Open clusters of assorted sizes and two periodic water boxes."""
    out = []
    for n, seed in [(64, 1), (300, 7), (9, 3), (1500, 11)]:
        s = synth.cluster(n, seed=seed)
        out.append((s.pos, s.species, s.cell, s.pbc))
    for nmol, seed in [(100, 2), (400, 5)]:
        s = synth.water_box(nmol, synth.water_side_for(nmol), seed=seed)
        out.append((s.pos, s.species, s.cell, s.pbc))
    return out


PRECS = ["fp32", "f16", "bf16"]


def _model(B, prec):
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    p = {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16, "bf16": B.MLIP_PREC_BF16}[prec]
    return B.Model(spec, w, p), spec, w


@pytest.mark.parametrize("prec", PRECS)
def test_batch_equals_single_calls(B, prec):
    m, _, _ = _model(B, prec)
    systems = _systems()
    single = [m.energy_forces(p, z, c, b) for p, z, c, b in systems]
    for order in (list(range(len(systems))), [5, 2, 0, 4, 1, 3]):
        batch = [systems[k] for k in order]
        E, F, _ = m.energy_forces_batch(batch)
        for j, k in enumerate(order):
            assert E[j] == single[k]["energy"][0], (prec, k, E[j], single[k]["energy"][0])
            assert np.array_equal(F[j], single[k]["forces"]), (prec, k, np.abs(F[j] - single[k]["forces"]).max())


@pytest.mark.parametrize("prec", ["fp32", "f16"])
def test_batch_stress_equals_single_calls(B, prec):
    m, _, _ = _model(B, prec)
    systems = [sy for sy in _systems() if sy[3].all()]
    E, F, S = m.energy_forces_batch(systems, stress=True)
    for j, (p, z, c, b) in enumerate(systems):
        one = m.energy_forces(p, z, c, b, stress=True)
        assert E[j] == one["energy"][0]
        assert np.array_equal(F[j], one["forces"])
        assert np.array_equal(S[j], one["stress"])


def test_batch_fp32_against_oracle(B):
    m, spec, w = _model(B, "fp32")
    systems = _systems()[:3] + _systems()[4:5]
    E, F, _ = m.energy_forces_batch(systems)
    om = oracle.Model(spec, w)
    for j, (p, z, c, b) in enumerate(systems):
        ref = om.energy_forces(p, z, c, b, atom_energies=True)
        scale = max(abs(ref["energy"]), float(np.abs(ref["atom_energies"]).sum()))
        assert abs(E[j] - ref["energy"]) <= 1e-6 * scale, (j, E[j], ref["energy"])
        fmax = np.abs(ref["forces"]).max()
        assert np.abs(F[j] - ref["forces"]).max() <= 1e-5 * fmax


def test_batch_errors(B):
    m, _, _ = _model(B, "fp32")
    systems = _systems()[:2]
    with pytest.raises(B.MlipError) as e:  # stress of an open system
        m.energy_forces_batch(systems, stress=True)
    assert e.value.code == B.MLIP_ERR_CELL
    bad = [(systems[0][0], np.full(64, 9, np.int32), systems[0][2], systems[0][3])]
    with pytest.raises(B.MlipError) as e:
        m.energy_forces_batch(bad)
    assert e.value.code == B.MLIP_ERR_INVALID_ARG
    # the model stays usable after the errors
    E, F, _ = m.energy_forces_batch(systems)
    assert np.isfinite(E).all()


@pytest.mark.parametrize("prec", ["fp32", "f16"])
def test_batched_md_equals_single_trajectories(B, prec):
    """Replicas advanced together (mlip_md_nve_batch) follow the trajectories
    each one follows alone (mlip_md_nve), bit for bit."""
    m, spec, _ = _model(B, prec)
    masses = np.asarray(spec.masses)
    reps = [synth.water_box(60, synth.water_side_for(60), seed=30 + k) for k in range(3)]
    vels = [synth.maxwell_boltzmann(masses[r.species], 300.0, seed=40 + k) for k, r in enumerate(reps)]
    off = np.cumsum([0] + [r.n for r in reps])
    pos = np.concatenate([r.pos for r in reps])
    vel = np.concatenate(vels)
    sp = np.concatenate([r.species for r in reps])
    cells = np.stack([r.cell for r in reps])
    pbc = np.stack([r.pbc for r in reps])
    P, V, PE, KE = m.md_nve_batch(off, pos, vel, sp, cells, pbc, 0.5, 8)
    for k, r in enumerate(reps):
        p1, v1, pe1, ke1 = m.md_nve(r.pos, vels[k], r.species, r.cell, r.pbc, 0.5, 8)
        assert np.array_equal(P[off[k]:off[k + 1]], p1) and np.array_equal(V[off[k]:off[k + 1]], v1)
        assert np.array_equal(PE[:, k], pe1) and np.array_equal(KE[:, k], ke1)
