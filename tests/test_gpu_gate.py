"""GPU parity of models with the gated update and the species self-connection
(NequIP's gate nonlinearity and self-connection on the uniform irreps)
against the FP64 oracle: plain FP32 form (1e-6 energy, 1e-5 forces and
stress) and fused F16 form (2e-3), node orders 2 and 3, together with the
symmetric contraction; batch invariance, graph replays, parameter file."""
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


_REF = {}


def _ref(key, spec, w, s, stress):
    if key not in _REF:
        _REF[key] = oracle.Model(spec, w).energy_forces(s.pos, s.species, s.cell, s.pbc, stress=stress,
                                                       atom_energies=True)
    return _REF[key]


def _check(out, ref, tol, etol, cell=None, n_edges=0):
    scale = max(abs(ref["energy"]), float(np.abs(ref["atom_energies"]).sum()))
    E = float(np.asarray(out["energy"]).reshape(-1)[0])
    assert abs(E - ref["energy"]) <= etol * scale, (E, ref["energy"])
    fmax = np.abs(ref["forces"]).max()
    err = np.abs(np.asarray(out["forces"]) - ref["forces"]).max()
    assert err <= tol * fmax, (err, fmax)
    if "stress" in ref:
        sref = ref["stress"]
        serr = np.abs(np.asarray(out["stress"]) - sref).max()
        print(f" stress: max|ds|/max|s_ref| = {serr / np.abs(sref).max():.2e} (bar {tol:g})", end="")
        assert serr <= tol * np.abs(sref).max()
    return err / fmax


PRECS = [("fp32", 1e-5, 1e-6), ("f16", 2e-3, 2e-3)]


@pytest.mark.parametrize("prec,tol,etol", PRECS)
def test_water_periodic(B, prec, tol, etol):
    spec = synth.model_spec("water_gated")
    w = synth.make_weights(spec, 21)
    s = synth.water_box(100, synth.water_side_for(100), seed=2)
    ref = _ref("water300", spec, w, s, True)
    m = B.Model(spec, w, {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16}[prec])
    ne = len(oracle.neighbors(s.pos, s.cell, s.pbc, 5.0)[0])
    rel = _check(m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True), ref, tol, etol, s.cell, ne)
    print(f"water_gated 300 {prec}: {rel:.2e}")


@pytest.mark.parametrize("prec,tol,etol", PRECS)
def test_fcc_l3(B, prec, tol, etol):
    spec = synth.model_spec("fcc_gated")
    w = synth.make_weights(spec, 31)
    s = synth.fcc((3, 4, 5), seed=3)
    ref = _ref("fcc240", spec, w, s, True)
    m = B.Model(spec, w, {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16}[prec])
    ne = len(oracle.neighbors(s.pos, s.cell, s.pbc, 5.0)[0])
    rel = _check(m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True), ref, tol, etol, s.cell, ne)
    print(f"fcc_gated 240 {prec}: {rel:.2e}")


@pytest.mark.parametrize("prec,tol,etol", PRECS)
def test_with_the_contraction_open_cluster(B, prec, tol, etol):
    spec = synth.model_spec("water_mace_gated")
    w = synth.make_weights(spec, 4)
    s = synth.cluster(300, seed=12)
    ref = _ref("cluster300", spec, w, s, False)
    m = B.Model(spec, w, {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16}[prec])
    rel = _check(m.energy_forces(s.pos, s.species, s.cell, s.pbc), ref, tol, etol)
    print(f"water_mace_gated cluster300 {prec}: {rel:.2e}")


def test_batch_graph_and_params_file(B, tmp_path):
    spec = synth.model_spec("water_gated")
    w = synth.make_weights(spec, 21)
    systems = [synth.water_box(k, synth.water_side_for(k), seed=40 + k) for k in (40, 70, 55)]
    m = B.Model(spec, w, B.MLIP_PREC_F16)
    singles = [m.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True) for s in systems]
    energy, forces, _ = m.energy_forces_batch([(s.pos, s.species, s.cell, s.pbc) for s in systems], forces=True)
    for k, one in enumerate(singles):
        assert energy[k] == one["energy"][0]
        assert np.array_equal(forces[k], one["forces"])
    s = systems[1]
    fresh = B.Model(spec, w, B.MLIP_PREC_F16)
    first = fresh.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True)
    for _ in range(5):  # exact, eager, capture, replays
        r = fresh.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True)
        assert all(np.array_equal(r[k], first[k]) for k in first)
    p = tmp_path / "gated.bin"
    synth.write_params(str(p), spec, w)
    h = B.mlip_model_load(str(p), B.MLIP_PREC_F16)
    try:
        b = B.mlip_energy_forces(h, s.pos, s.species, s.cell, s.pbc, True, False, None, None)
    finally:
        B.mlip_model_free(h)
    assert b["energy"][0] == first["energy"][0] and np.array_equal(b["forces"], first["forces"])
