"""GPU parity of mixed-parity models (parity = 1: the irreps of the paper's
NequIP table with C/2 channels of each order and parity, pseudotensor paths
included) in the plain FP32 form against the FP64 oracle: energy within 1e-6
of max(|E|, sum |E_i|), forces and stress within 1e-5 of their maxima.
Periodic water box (l <= 2, 128 channels), periodic FCC cell (l <= 3), and a
three-layer 32-channel model with a large message scale on an open cluster, so
that the odd scalars (and their tanh update) reach the energy path; energy
invariant under a reflection; the parameter file (version 3) round trip; the
16-bit forms refuse the option."""
import dataclasses
import os
import tempfile

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


def _check(out, ref, stress=False, label=""):
    scale = max(abs(ref["energy"]), float(np.abs(ref["atom_energies"]).sum()))
    E = float(np.asarray(out["energy"]).reshape(-1)[0])
    assert abs(E - ref["energy"]) <= 1e-6 * scale, (E, ref["energy"])
    fmax = np.abs(ref["forces"]).max()
    err = np.abs(np.asarray(out["forces"]) - ref["forces"]).max()
    print(f" {label}: max|dF|/max|F| = {err / fmax:.2e} (bar 1e-05)", end="")
    assert err <= 1e-5 * fmax
    if stress:
        smax = np.abs(ref["stress"]).max()
        assert np.abs(np.asarray(out["stress"]) - ref["stress"]).max() <= 1e-5 * smax


def test_water_box_l2(B):
    spec = synth.model_spec("water_parity")
    w = synth.make_weights(spec, 21)
    s = synth.water_box(100, synth.water_side_for(100), seed=2)
    ref = oracle.Model(spec, w).energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True, atom_energies=True)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    _check(m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True), ref, True, "water300 parity")
    m.close()


def test_fcc_cell_l3(B):
    spec = synth.model_spec("fcc_parity")
    w = synth.make_weights(spec, 31)
    s = synth.fcc((3, 4, 5), seed=3)
    ref = oracle.Model(spec, w).energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True, atom_energies=True)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    _check(m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True), ref, True, "fcc240 parity")
    m.close()


def test_odd_scalars_three_layers_and_reflection(B):
    spec = synth.ModelSpec(S=4, T=3, C=32, L=2, H=32, avg_nb=0.5, parity=1)
    w = synth.make_weights(spec, 9)
    s = synth.cluster(60, seed=4, side=7.0)
    om = oracle.Model(spec, w)
    h = om.node_features(s.pos, s.species, s.cell, s.pbc, 2)
    assert np.abs(h[:, 0, 16:]).max() == 0.0  # no odd scalar before the third layer
    ref = om.energy_forces(s.pos, s.species, s.cell, s.pbc, atom_energies=True)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    out = m.energy_forces(s.pos, s.species, s.cell, s.pbc)
    _check(out, ref, False, "cluster60 T3 C32 parity")
    R = np.diag([-1.0, 1.0, 1.0])  # the mirror x -> -x
    mir = m.energy_forces(s.pos @ R.T, s.species, s.cell, s.pbc)
    scale = max(abs(ref["energy"]), float(np.abs(ref["atom_energies"]).sum()))
    assert abs(mir["energy"][0] - out["energy"][0]) <= 1e-6 * scale
    m.close()


def test_parameter_file_round_trip_and_16bit_refused(B):
    spec = synth.model_spec("water_parity")
    w = synth.make_weights(spec, 21)
    s = synth.cluster(50, seed=8)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "p.bin")
        synth.write_params(path, spec, w)
        a = B.Model(spec, w, B.MLIP_PREC_FP32).energy_forces(s.pos, s.species, s.cell, s.pbc)
        h = B.mlip_model_load(path, B.MLIP_PREC_FP32)
        b = B.mlip_energy_forces(h, s.pos, s.species, s.cell, s.pbc)
        B.mlip_model_free(h)
    assert a["energy"][0] == b["energy"][0] and np.array_equal(a["forces"], b["forces"])
    with pytest.raises(B.MlipError) as e:
        B.Model(spec, w, B.MLIP_PREC_F16)
    assert e.value.code == B.MLIP_ERR_INVALID_ARG
    with pytest.raises(B.MlipError):
        B.Model(dataclasses.replace(spec, gate=1), synth.make_weights(dataclasses.replace(spec, gate=1), 1),
                B.MLIP_PREC_FP32)
