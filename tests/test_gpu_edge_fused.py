"""Degenerate inputs through the fused 16-bit form and the model options:
one atom, pairs beyond the cutoff (no edges), a handful of edges (one partial
tile), pairs just inside the cutoff; repeated calls through the replayed
graph; the Coulomb term acting beyond the cutoff with no edges at all.

Bar of the F16 form: 2e-3 of max|F_ref| (energy: of max(|E|, sum|E_i|)), the
same as on the large systems.  On two isolated pairs the forces are far below
the size of the per-edge terms (cancelling paths and layers), so W3's own FP16
rounding moves the oracle's forces by 1.6e-3 of max|F| there (3.9e-4 on the
300-atom water box); the form's other products carry no 16-bit rounding, and
each check prints the measured error.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SYSTEMS = [
    ("one atom", np.array([[0.0, 0.0, 0.0]]), np.array([2], np.int32)),
    ("beyond the cutoff", np.array([[0.0, 0, 0], [6.0, 0, 0]]), np.array([0, 1], np.int32)),
    ("two far pairs", np.array([[0.0, 0, 0], [20.0, 0, 0], [1.5, 0, 0], [21.0, 0.5, 0]]), np.array([0, 1, 2, 3], np.int32)),
    ("just inside", np.array([[0.0, 0, 0], [4.999, 0, 0]]), np.array([3, 3], np.int32)),
    ("partial tile", np.array([[0.0, 0, 0], [1.0, 0.2, 0], [0.3, 1.1, 0.4], [2.0, 2.0, 0.1], [-1.2, 0.4, 0.9]]),
     np.array([0, 1, 2, 3, 1], np.int32)),
]


@pytest.fixture(scope="module")
def B():
    import torch
    torch.cuda.init()
    from paper_2605_22698_gb300 import build
    build.build()
    from paper_2605_22698_gb300 import binding
    binding.lib()
    return binding


def _assert_close(out, ref, tol, label=""):
    scale = max(abs(ref["energy"]), float(np.abs(ref["atom_energies"]).sum()))
    ebar, fbar = tol * scale, tol * np.abs(ref["forces"]).max()
    assert abs(float(np.asarray(out["energy"]).reshape(-1)[0]) - ref["energy"]) <= max(ebar, 1e-12)
    err = np.abs(np.asarray(out["forces"]) - ref["forces"]).max()
    if fbar >= 1e-12:
        print(f" {label}: max|dF|/max|F| = {err / np.abs(ref['forces']).max():.2e} (bar {tol:g})", end="")
    else:  # forces at the round-off level (a pair at the cutoff, where the envelope vanishes)
        print(f" {label}: max|dF| = {err:.1e} with max|F| = {np.abs(ref['forces']).max():.1e} (bar 1e-12 absolute)",
              end="")
    assert err <= max(fbar, 1e-12), (err, fbar)


@pytest.mark.parametrize("name", ["water", "water_mace"])
def test_fused_degenerate_systems(B, name):
    spec = synth.model_spec(name)
    w = synth.make_weights(spec, 21)
    om = oracle.Model(spec, w)
    cell, pbc = np.eye(3), np.zeros(3, np.uint8)
    for label, pos, z in SYSTEMS:
        ref = om.energy_forces(pos, z, cell, pbc, atom_energies=True)
        m = B.Model(spec, w, B.MLIP_PREC_F16)
        first = m.energy_forces(pos, z, cell, pbc)
        _assert_close(first, ref, 2e-3, label)
        for _ in range(4):  # eager, capture, replays: the same numbers
            r = m.energy_forces(pos, z, cell, pbc)
            assert all(np.array_equal(r[k], first[k]) for k in first), label
        m.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("f16", 2e-3)])
def test_charged_degenerate_systems(B, prec, tol):
    """With charges the Coulomb term acts between every pair of the system,
    edges or not: two atoms beyond the cutoff still attract or repel."""
    spec = synth.model_spec("water_charged")
    w = synth.make_weights(spec, 21)
    om = oracle.Model(spec, w)
    p = {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16}[prec]
    for Q in (0.0, 1.0):
        om.set_total_charge(Q)
        for label, pos, z in SYSTEMS:
            ref = om.energy_forces(pos, z, np.eye(3), np.zeros(3, np.uint8), atom_energies=True)
            m = B.Model(spec, w, p)
            out = m.energy_forces_charged(pos, z, Q)
            _assert_close(out, ref, tol, label)
            np.testing.assert_allclose(out["charges"], om.charges(pos, z), rtol=0,
                                       atol=tol * max(1.0, np.abs(om.charges(pos, z)).max()))
            if label == "beyond the cutoff" and Q == 0.0:
                assert np.abs(out["forces"]).max() > 0.0  # the long-range term alone
            m.close()
