"""GPU velocity-Verlet NVE against the FP64 oracle's trajectory (first 20 steps)."""
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


@pytest.mark.parametrize("prec", ["fp32", "f16"])
def test_autograd_function_gradient(B, prec):
    """torch.autograd through the library's adjoint: dE/dr = -F, and it matches
    central finite differences of the library's own energy (FP64 positions)."""
    import torch
    from paper_2605_22698_gb300 import autograd as AG
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    p = {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16}[prec]
    m = B.Model(spec, w, p)
    s = synth.water_box(60, synth.water_side_for(60), seed=5)
    pos = torch.tensor(s.pos, device="cuda", requires_grad=True)
    sp = torch.tensor(s.species, device="cuda")
    E = AG.energy(m, pos, sp, s.cell, s.pbc)
    (g,) = torch.autograd.grad(2.0 * E, pos)
    F = m.energy_forces(s.pos, s.species, s.cell, s.pbc)["forces"]
    assert np.allclose(g.cpu().numpy(), -2.0 * F, rtol=0, atol=1e-12 * np.abs(F).max())
    # directional central difference of the FP64 oracle energy
    om = oracle.Model(spec, w)
    rng = np.random.default_rng(3)
    d = rng.standard_normal(s.pos.shape)
    d /= np.linalg.norm(d)
    h = 1e-4
    ep = om.energy(s.pos + h * d, s.species, s.cell, s.pbc)
    em = om.energy(s.pos - h * d, s.species, s.cell, s.pbc)
    ep = ep[0] if isinstance(ep, tuple) else ep
    em = em[0] if isinstance(em, tuple) else em
    fd = (ep - em) / (2 * h)
    an = float((g.cpu().numpy() / 2.0 * d).sum())
    # |sum_i dF_i . d_i| <= max|dF| * ||d||_1 <= tol max|F| sqrt(3n)
    tol = (2e-3 if prec == "f16" else 1e-5) * np.abs(F).max() * np.sqrt(3 * s.n)
    assert abs(fd - an) <= tol, (fd, an, tol)
