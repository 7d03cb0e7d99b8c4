"""GPU velocity-Verlet NVE against the FP64 oracle's trajectory (first 20 steps), and the separate
forward and backward entry points behind the torch.autograd.Function."""
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


def _traj(B, prec, steps=20):
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    s = synth.water_box(60, synth.water_side_for(60), seed=13)
    masses = np.asarray(spec.masses)
    v0 = synth.maxwell_boltzmann(masses[s.species], 300.0, seed=5)
    ref = oracle.Model(spec, w).vv_nve(s.pos, v0, s.species, masses, s.cell, s.pbc, 0.5, steps)
    m = B.Model(spec, w, prec)
    got = m.md_nve(s.pos, v0, s.species, s.cell, s.pbc, 0.5, steps)
    return ref, got


def test_vv_fp32_matches_oracle_trajectory(B):
    (rp, rv, rpe, rke), (gp, gv, gpe, gke) = _traj(B, B.MLIP_PREC_FP32)
    assert np.abs(gp - rp).max() < 1e-9
    assert np.abs(gv - rv).max() < 1e-10
    scale = np.abs(rpe).max() + np.abs(rke).max()
    assert np.abs(gpe - rpe).max() < 1e-6 * scale
    assert np.abs(gke - rke).max() < 1e-9 * scale


def test_vv_f16_matches_oracle_trajectory(B):
    (rp, rv, rpe, rke), (gp, gv, gpe, gke) = _traj(B, B.MLIP_PREC_F16)
    assert np.abs(gp - rp).max() < 1e-6
    scale = np.abs(rpe).max() + np.abs(rke).max()
    assert np.abs(gpe - rpe).max() < 2e-3 * scale


def test_vv_device_inplace_and_reversible(B):
    import torch
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 3)
    s = synth.water_box(40, synth.water_side_for(40), seed=4)
    masses = np.asarray(spec.masses)
    v0 = synth.maxwell_boltzmann(masses[s.species], 300.0, seed=6)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    pos = torch.tensor(s.pos, device="cuda"); vel = torch.tensor(v0, device="cuda")
    sp = torch.tensor(s.species, device="cuda")
    m.md_nve(pos, vel, sp, s.cell, s.pbc, 0.5, 10)
    vel.neg_()
    m.md_nve(pos, vel, sp, s.cell, s.pbc, 0.5, 10)
    torch.cuda.synchronize()
    assert np.abs(pos.cpu().numpy() - s.pos).max() < 1e-8
    assert np.abs(-vel.cpu().numpy() - v0).max() < 1e-9


ADJOINT_KERNELS = {"grad_init", "mix_bwd", "mix_tc_bwd", "tp_bwd", "tp_fused_bwd", "radial_bwd", "radial_bwd_tc",
                   "sym_contract_bwd", "gate_bwd", "charge_grad", "dw_scales", "edge_grad", "forces_virial",
                   "coulomb_add_forces", "grad_from_forces"}


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("f16", 2e-3)])
def test_autograd_forward_then_backward(B, prec, tol):
    """torch.autograd through the separate forward and backward entry points:
    the forward launches no adjoint kernel (per-kernel records of the
    library's tracing); the backward recomputes the harmonics and radial
    weights (edge_sh and radial_tc run again in the fused form) and its
    gradient equals -g F of the FP64 oracle element by element, within the
    form's force tolerance; a second backward of the same forward gives the
    same gradient; another evaluation in between makes the backward fail."""
    import torch
    from paper_2605_22698_gb300 import autograd as AG
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    p = {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16}[prec]
    m = B.Model(spec, w, p)
    s = synth.water_box(100, synth.water_side_for(100), seed=5)
    ref = oracle.Model(spec, w).energy_forces(s.pos, s.species, s.cell, s.pbc, atom_energies=True)
    pos = torch.tensor(s.pos, device="cuda", requires_grad=True)
    sp = torch.tensor(s.species, device="cuda")
    B.mlip_profile_select(None)
    B.mlip_profile_enable(True)
    E = AG.energy(m, pos, sp, s.cell, s.pbc)
    torch.cuda.synchronize()
    fwd = set(B.mlip_profile_report()["kernels"])
    B.mlip_profile_enable(True)  # clears the records
    (g,) = torch.autograd.grad(2.5 * E, pos, retain_graph=True)
    torch.cuda.synchronize()
    bwd = set(B.mlip_profile_report()["kernels"])
    B.mlip_profile_enable(False)
    assert not (fwd & ADJOINT_KERNELS), fwd & ADJOINT_KERNELS
    assert {"grad_init", "forces_virial", "grad_from_forces"} <= bwd
    if prec == "f16":
        assert {"edge_sh", "radial_tc", "tp_fused_bwd", "radial_bwd_tc"} <= bwd  # recomputed, then the adjoint
    scale = max(abs(ref["energy"]), float(np.abs(ref["atom_energies"]).sum()))
    assert abs(float(E.item()) - ref["energy"]) <= (1e-6 if prec == "fp32" else tol) * scale
    want = -2.5 * ref["forces"]
    err = np.abs(g.cpu().numpy() - want).max()
    print(f" autograd {prec}: max|dg|/max|g| = {err / np.abs(want).max():.2e} (bar {tol:g})", end="")
    assert err <= tol * np.abs(want).max()
    (g2,) = torch.autograd.grad(2.5 * E, pos)  # a second backward of the same forward
    assert torch.equal(g, g2)
    E3 = AG.energy(m, pos, sp, s.cell, s.pbc)
    m.energy_forces(s.pos, s.species, s.cell, s.pbc)  # overwrites what the forward kept
    with pytest.raises(B.MlipError):
        torch.autograd.grad(E3, pos)
    m.close()


def test_backward_entry_point_host_arrays_and_stress(B):
    """The C ABI pair with host arrays: g dE/dr and g sigma equal -g F and g
    sigma of the one-call entry point (the same kernels, bit for bit in FP32;
    FP16 form to its tolerance)."""
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    s = synth.water_box(100, synth.water_side_for(100), seed=6)
    for p in (B.MLIP_PREC_FP32, B.MLIP_PREC_F16):
        m = B.Model(spec, w, p)
        one = m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True)
        e = m.energy_forward(s.pos, s.species, s.cell, s.pbc)
        gpos, gs = m.energy_backward(s.n, -0.5, stress=True)
        assert e == one["energy"][0]
        np.testing.assert_array_equal(gpos, 0.5 * one["forces"])
        np.testing.assert_array_equal(gs, -0.5 * one["stress"])
        m.close()
