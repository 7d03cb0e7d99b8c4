"""GPU parity of models with the symmetric contraction of correlation order 2
(MACE's product basis after every scatter-sum) against the FP64 oracle, in
the plain FP32 form (tolerances 1e-6 energy, 1e-5 forces and stress) and the
fused F16 form (2e-3); batch invariance and graph replays bit for bit."""
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


_REF = {}


def _ref(key, spec, w, s, stress):
    if key not in _REF:
        _REF[key] = oracle.Model(spec, w).energy_forces(s.pos, s.species, s.cell, s.pbc, stress=stress,
                                                       atom_energies=True)
    return _REF[key]


def test_small_model_fp32_cluster(B):
    spec = synth.model_spec("small_mace")
    w = synth.make_weights(spec, 9)
    s = synth.cluster64(3)
    ref = _ref("small64", spec, w, s, False)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    rel = _check(m.energy_forces(s.pos, s.species, s.cell, s.pbc), ref, 1e-5, 1e-6)
    print(f"small_mace cluster64 fp32: {rel:.2e}")


@pytest.mark.parametrize("prec,tol,etol", [("fp32", 1e-5, 1e-6), ("f16", 2e-3, 2e-3)])
def test_water_periodic(B, prec, tol, etol):
    spec = synth.model_spec("water_mace")
    w = synth.make_weights(spec, 21)
    s = synth.water_box(100, synth.water_side_for(100), seed=2)
    ref = _ref("water300", spec, w, s, True)
    m = B.Model(spec, w, {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16}[prec])
    ne = len(oracle.neighbors(s.pos, s.cell, s.pbc, 5.0)[0])
    rel = _check(m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True), ref, tol, etol, s.cell, ne)
    print(f"water_mace 300 {prec}: {rel:.2e}")


@pytest.mark.parametrize("prec,tol,etol", [("fp32", 1e-5, 1e-6), ("f16", 2e-3, 2e-3)])
def test_fcc_l3(B, prec, tol, etol):
    spec = synth.model_spec("fcc_mace")
    w = synth.make_weights(spec, 31)
    s = synth.fcc((3, 4, 5), seed=3)
    ref = _ref("fcc240", spec, w, s, True)
    m = B.Model(spec, w, {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16}[prec])
    ne = len(oracle.neighbors(s.pos, s.cell, s.pbc, 5.0)[0])
    rel = _check(m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True), ref, tol, etol, s.cell, ne)
    print(f"fcc_mace 240 {prec}: {rel:.2e}")


def test_open_cluster_f16(B):
    spec = synth.model_spec("water_mace")
    w = synth.make_weights(spec, 4)
    s = synth.cluster(300, seed=12)
    ref = _ref("cluster300", spec, w, s, False)
    m = B.Model(spec, w, B.MLIP_PREC_F16)
    rel = _check(m.energy_forces(s.pos, s.species, s.cell, s.pbc), ref, 2e-3, 2e-3)
    print(f"water_mace cluster300 f16: {rel:.2e}")


def test_batch_and_graph_replays_bit_identical(B):
    """A system's results with the contraction do not depend on its batch,
    and graph replays equal the first (synchronising) evaluation."""
    spec = synth.model_spec("water_mace")
    w = synth.make_weights(spec, 21)
    systems = [synth.water_box(k, synth.water_side_for(k), seed=40 + k) for k in (40, 70, 55)]
    m = B.Model(spec, w, B.MLIP_PREC_F16)
    singles = [m.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True) for s in systems]
    energy, forces, _ = m.energy_forces_batch([(s.pos, s.species, s.cell, s.pbc) for s in systems], forces=True)
    for k, one in enumerate(singles):
        assert energy[k] == one["energy"][0]
        assert np.array_equal(forces[k], one["forces"])
    fresh = B.Model(spec, w, B.MLIP_PREC_F16)
    s = systems[1]
    first = fresh.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True)
    for _ in range(5):  # exact, eager, capture, replays
        r = fresh.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True)
        assert all(np.array_equal(r[k], first[k]) for k in first)


def test_params_file_with_the_contraction(B, tmp_path):
    spec = synth.model_spec("small_mace")
    w = synth.make_weights(spec, 9)
    p = tmp_path / "mace.bin"
    synth.write_params(str(p), spec, w)
    s = synth.cluster64(5)
    a = B.Model(spec, w, B.MLIP_PREC_FP32).energy_forces(s.pos, s.species, s.cell, s.pbc)
    h = B.mlip_model_load(str(p), B.MLIP_PREC_FP32)
    try:
        b = B.mlip_energy_forces(h, s.pos, s.species, s.cell, s.pbc, True, False, None, None)
    finally:
        B.mlip_model_free(h)
    assert a["energy"][0] == b["energy"][0] and np.array_equal(a["forces"], b["forces"])
