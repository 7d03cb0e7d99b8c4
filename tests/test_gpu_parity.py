"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances (FP32 form): energy |E - E_ref| <= 1e-6 max(|E_ref|, sum_i |E_i,ref|);
forces max |F - F_ref| <= 1e-5 max |F_ref|; stress max |s - s_ref| <= 1e-5 max |s_ref|.
Neighbour lists must be identical (bit-exact, canonical order).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

E_TOL, F_TOL, S_TOL = 1e-6, 1e-5, 1e-5


@pytest.fixture(scope="module")
def B():
    import torch
    torch.cuda.init()
    from paper_2605_22698_gb300 import build
    build.build()
    from paper_2605_22698_gb300 import binding
    binding.lib()
    return binding


def _cases():
    r = np.random.default_rng(5)
    out = []
    out.append(("open24", r.uniform(size=(24, 3)) * 8, np.eye(3) * 8, np.zeros(3, np.uint8)))
    out.append(("cubic20", r.uniform(size=(20, 3)) * 7, np.eye(3) * 7, np.ones(3, np.uint8)))
    h = np.array([[2.1, 0, 0], [0.9, 2.4, 0], [0.4, -0.6, 11.0]])
    out.append(("thin-triclinic", r.uniform(size=(6, 3)) @ h, h, np.ones(3, np.uint8)))
    out.append(("slab", r.uniform(size=(15, 3)) * np.array([4.0, 5.0, 12.0]), np.diag([4.0, 5.0, 30.0]),
                np.array([1, 1, 0], np.uint8)))
    h = np.array([[6.0, 0, 0], [1.0, 6.5, 0], [0, 0.5, 5.5]])
    out.append(("unwrapped", r.uniform(size=(12, 3)) * 30 - 10, h, np.ones(3, np.uint8)))
    s = synth.water_box(1000, 31.0, seed=2)
    out.append(("water3000", s.pos, s.cell, s.pbc))
    s = synth.fcc((5, 10, 10), seed=3)
    out.append(("fcc2000", s.pos, s.cell, s.pbc))
    s = synth.cluster(700, seed=9)
    out.append(("cluster700", s.pos, s.cell, s.pbc))
    out.append(("single", np.array([[1.0, 2.0, 3.0]]), np.eye(3), np.zeros(3, np.uint8)))
    out.append(("planar", np.c_[r.uniform(size=(30, 2)) * 9, np.zeros(30)], np.eye(3), np.zeros(3, np.uint8)))
    out.append(("linear", np.c_[np.arange(12) * 1.3, np.zeros(12), np.zeros(12)], np.eye(3), np.zeros(3, np.uint8)))
    out.append(("coincident-images", np.array([[0.0, 0, 0], [0.0, 0, 0.0]]) + 0.5, np.eye(3) * 3.0,
                np.ones(3, np.uint8)))
    out.append(("single-periodic", np.array([[1.0, 2.0, 3.0]]), np.eye(3) * 4.0, np.ones(3, np.uint8)))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_neighbors_bit_exact(B, case):
    _, pos, cell, pbc = case
    r0, s0, sh0 = oracle.neighbors(pos, cell, pbc, 5.0)
    r1, s1, sh1 = B.mlip_neighbors(np.ascontiguousarray(pos), cell, pbc, 5.0)
    assert len(r1) == len(r0)
    np.testing.assert_array_equal(r1, r0)
    np.testing.assert_array_equal(s1, s0)
    np.testing.assert_array_equal(sh1.astype(np.int32), sh0)


def test_neighbors_device_input_and_capacity(B):
    import torch
    s = synth.water_box(200, synth.water_side_for(200), seed=4)
    r0, s0, sh0 = oracle.neighbors(s.pos, s.cell, s.pbc, 5.0)
    pos = torch.tensor(s.pos, device="cuda")
    r1, s1, sh1 = B.mlip_neighbors(pos, s.cell, s.pbc, 5.0)
    np.testing.assert_array_equal(r1.cpu().numpy(), r0)
    np.testing.assert_array_equal(s1.cpu().numpy(), s0)
    np.testing.assert_array_equal(sh1.cpu().numpy().astype(np.int32), sh0)
    with pytest.raises(B.MlipError) as e:
        B.mlip_neighbors(s.pos, s.cell, s.pbc, 5.0, capacity=len(r0) - 1)
    assert e.value.code == B.MLIP_ERR_CAPACITY


def _compare(out, ref, stress=False, etol=E_TOL, ftol=F_TOL, stol=S_TOL):
    scale = max(abs(ref["energy"]), float(np.abs(ref["atom_energies"]).sum()))
    E = float(np.asarray(out["energy"]).reshape(-1)[0])
    assert abs(E - ref["energy"]) <= etol * scale, (E, ref["energy"], scale)
    F = np.asarray(out["forces"])
    fmax = np.abs(ref["forces"]).max()
    err = np.abs(F - ref["forces"]).max()
    assert err <= ftol * fmax, (err, fmax)
    if stress:
        S = np.asarray(out["stress"])
        smax = np.abs(ref["stress"]).max()
        assert np.abs(S - ref["stress"]).max() <= stol * smax, (S, ref["stress"])
    return err / fmax


def _ref(spec, w, s, stress=False):
    return oracle.Model(spec, w).energy_forces(s.pos, s.species, s.cell, s.pbc, stress=stress, atom_energies=True)


def test_cluster64_fp32(B):
    spec = synth.model_spec("small")
    w = synth.make_weights(spec, 7)
    s = synth.cluster64(1)
    ref = _ref(spec, w, s)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    _compare(m.energy_forces(s.pos, s.species, s.cell, s.pbc), ref)


def test_small_model_two_layers_l3_fp32(B):
    """C = 16, T = 2, L = 3 on a periodic triclinic box (all paths active)."""
    spec = synth.ModelSpec(S=4, T=2, C=16, L=3, H=32, avg_nb=20.0)
    w = synth.make_weights(spec, 11)
    s = synth.water_box(40, synth.water_side_for(40), seed=6)
    s.cell = s.cell + np.array([[0, 0.5, -0.3], [0.2, 0, 0.4], [-0.1, 0.3, 0]])
    ref = _ref(spec, w, s, stress=True)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    _compare(m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True), ref, stress=True)


def test_water3000_fp32_energy_forces_stress(B):
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    s = synth.water_box(1000, 31.0, seed=2)
    ref = _ref(spec, w, s, stress=True)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    _compare(m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True), ref, stress=True)


def test_fcc_subcell_l3_fp32(B):
    spec = synth.model_spec("fcc")
    w = synth.make_weights(spec, 31)
    s = synth.fcc((5, 10, 10), seed=3)
    ref = _ref(spec, w, s, stress=True)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    _compare(m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True), ref, stress=True)


def test_edge_cases(B):
    spec = synth.ModelSpec(S=4, T=2, C=16, L=2, H=32, avg_nb=20.0)
    w = synth.make_weights(spec, 3)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    om = oracle.Model(spec, w)
    systems = [
        (np.array([[0.0, 0.0, 0.0]]), np.array([2], np.int32)),                          # one atom, no edges
        (np.array([[0.0, 0, 0], [6.0, 0, 0]]), np.array([0, 1], np.int32)),              # beyond the cutoff
        (np.array([[0.0, 0, 0], [20.0, 0, 0], [1.5, 0, 0], [21.0, 0.5, 0]]), np.array([0, 1, 2, 3], np.int32)),
        (np.array([[0.0, 0, 0], [4.999, 0, 0]]), np.array([3, 3], np.int32)),             # just inside
    ]
    for pos, z in systems:
        cell, pbc = np.eye(3), np.zeros(3, np.uint8)
        ref = om.energy_forces(pos, z, cell, pbc, atom_energies=True)
        out = m.energy_forces(pos, z, cell, pbc)
        E = float(out["energy"][0])
        scale = max(abs(ref["energy"]), float(np.abs(ref["atom_energies"]).sum()))
        assert abs(E - ref["energy"]) <= E_TOL * scale
        fmax = np.abs(ref["forces"]).max()
        assert np.abs(out["forces"] - ref["forces"]).max() <= max(F_TOL * fmax, 1e-12)


def test_errors(B):
    spec = synth.model_spec("small")
    m = B.Model(spec, synth.make_weights(spec, 1), B.MLIP_PREC_FP32)
    s = synth.cluster64(1)
    bad = s.species.copy(); bad[3] = 9
    with pytest.raises(B.MlipError) as e:
        m.energy_forces(s.pos, bad, s.cell, s.pbc)
    assert e.value.code == B.MLIP_ERR_INVALID_ARG
    with pytest.raises(B.MlipError) as e:
        m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True)
    assert e.value.code == B.MLIP_ERR_CELL
    with pytest.raises(B.MlipError) as e:
        m.energy_forces(s.pos, s.species, np.zeros((3, 3)), np.ones(3, np.uint8))
    assert e.value.code == B.MLIP_ERR_CELL


def test_device_path_matches_host_path_and_is_deterministic(B):
    import torch
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    s = synth.water_box(300, synth.water_side_for(300), seed=8)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    host = m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True)
    pos = torch.tensor(s.pos, device="cuda")
    sp = torch.tensor(s.species, device="cuda")
    d1 = m.energy_forces(pos, sp, s.cell, s.pbc, stress=True)
    d2 = m.energy_forces(pos, sp, s.cell, s.pbc, stress=True)
    torch.cuda.synchronize()
    assert float(d1["energy"].item()) == float(host["energy"][0])
    np.testing.assert_array_equal(d1["forces"].cpu().numpy(), host["forces"])
    np.testing.assert_array_equal(d1["forces"].cpu().numpy(), d2["forces"].cpu().numpy())
    np.testing.assert_array_equal(d1["stress"].cpu().numpy(), d2["stress"].cpu().numpy())


def test_rotation_invariance_on_gpu(B):
    spec = synth.ModelSpec(S=4, T=2, C=16, L=3, H=32, avg_nb=20.0)
    w = synth.make_weights(spec, 12)
    s = synth.cluster(60, seed=2, side=8.0)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    a = m.energy_forces(s.pos, s.species, s.cell, s.pbc)
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    b = m.energy_forces(s.pos @ Q.T + 3.0, s.species, s.cell, s.pbc)
    assert abs(a["energy"][0] - b["energy"][0]) <= 1e-5 * abs(a["energy"][0])
    fmax = np.abs(a["forces"]).max()
    assert np.abs(b["forces"] - a["forces"] @ Q.T).max() <= 1e-4 * fmax
