"""GPU parity of models with the charge head, the charge correction and the
soft-core Coulomb term against the FP64 oracle: energy, forces and corrected
charges for open systems of several total charges, in the plain FP32 form
(1e-6 energy, 1e-5 forces and charges) and the fused F16 form (2e-3); batch
invariance, graph replays, and the error paths."""
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


def _ref(spec, w, s, Q):
    om = oracle.Model(spec, w)
    om.set_total_charge(Q)
    r = om.energy_forces(s.pos, s.species, s.cell, s.pbc, atom_energies=True)
    r["charges"] = om.charges(s.pos, s.species)
    return r


def _check(out, ref, tol, etol):
    scale = max(abs(ref["energy"]), float(np.abs(ref["atom_energies"]).sum()))
    E = float(np.asarray(out["energy"]).reshape(-1)[0])
    assert abs(E - ref["energy"]) <= etol * scale, (E, ref["energy"], scale)
    fmax = np.abs(ref["forces"]).max()
    err = np.abs(np.asarray(out["forces"]) - ref["forces"]).max()
    assert err <= tol * fmax, (err, fmax)
    q = np.asarray(out["charges"])
    assert np.abs(q - ref["charges"]).max() <= tol * np.abs(ref["charges"]).max()
    return err / fmax


@pytest.mark.parametrize("Q", [0.0, 1.0, -2.0])
def test_small_model_fp32(B, Q):
    spec = synth.model_spec("small_charged")
    w = synth.make_weights(spec, 9)
    s = synth.cluster64(3)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    out = m.energy_forces_charged(s.pos, s.species, Q)
    assert abs(float(out["charges"].sum()) - Q) < 1e-9
    rel = _check(out, _ref(spec, w, s, Q), 1e-5, 1e-6)
    print(f"small_charged Q={Q} fp32: {rel:.2e}")


@pytest.mark.parametrize("name", ["water_charged", "water_mace_charged"])
@pytest.mark.parametrize("prec,tol,etol", [("fp32", 1e-5, 1e-6), ("f16", 2e-3, 2e-3)])
def test_cluster(B, name, prec, tol, etol):
    spec = synth.model_spec(name)
    w = synth.make_weights(spec, 21)
    s = synth.cluster(400, seed=12)
    m = B.Model(spec, w, {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16}[prec])
    rel = _check(m.energy_forces_charged(s.pos, s.species, 1.0), _ref(spec, w, s, 1.0), tol, etol)
    print(f"{name} cluster400 {prec}: {rel:.2e}")


def test_large_cluster_fp32(B):
    """1500 atoms: every atom's pair loop runs many lane iterations."""
    spec = synth.model_spec("small_charged")
    w = synth.make_weights(spec, 9)
    s = synth.cluster(1500, seed=5)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    rel = _check(m.energy_forces_charged(s.pos, s.species, -1.0), _ref(spec, w, s, -1.0), 1e-5, 1e-6)
    print(f"small_charged cluster1500 fp32: {rel:.2e}")


def test_batch_graph_and_entry_points_agree(B):
    spec = synth.model_spec("water_charged")
    w = synth.make_weights(spec, 21)
    systems = [synth.cluster(k, seed=60 + k) for k in (90, 150, 120)]
    m = B.Model(spec, w, B.MLIP_PREC_F16)
    singles = [m.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True) for s in systems]
    energy, forces, _ = m.energy_forces_batch([(s.pos, s.species, s.cell, s.pbc) for s in systems], forces=True)
    for k, one in enumerate(singles):
        assert energy[k] == one["energy"][0]
        assert np.array_equal(forces[k], one["forces"])
        c = m.energy_forces_charged(systems[k].pos, systems[k].species, 0.0)
        assert c["energy"][0] == one["energy"][0] and np.array_equal(c["forces"], one["forces"])
    s = systems[1]
    first = m.energy_forces_charged(s.pos, s.species, 0.5)
    for _ in range(5):  # exact, eager, capture, replays
        r = m.energy_forces_charged(s.pos, s.species, 0.5)
        assert all(np.array_equal(r[k], first[k]) for k in first)


def test_errors(B):
    spec = synth.model_spec("small_charged")
    m = B.Model(spec, synth.make_weights(spec, 9), B.MLIP_PREC_FP32)
    wb = synth.water_box(8, synth.water_side_for(8), seed=1, d_oo=2.5)
    with pytest.raises(B.MlipError) as e:
        m.energy_forces(wb.pos, wb.species, wb.cell, wb.pbc)
    assert e.value.code == B.MLIP_ERR_CELL
    plain = B.Model(synth.model_spec("small"), synth.make_weights(synth.model_spec("small"), 9), B.MLIP_PREC_FP32)
    s = synth.cluster64(2)
    with pytest.raises(B.MlipError) as e:
        plain.energy_forces_charged(s.pos, s.species, 0.0)
    assert e.value.code == B.MLIP_ERR_INVALID_ARG
