"""Degenerate inputs through the fused 16-bit form and the model options:
one atom, pairs beyond the cutoff (no edges), a handful of edges (one partial
tile), pairs just inside the cutoff; repeated calls through the replayed
graph; the Coulomb term acting beyond the cutoff with no edges at all.

Bar of the F16 form here: 2e-3 of max|F_ref| (energy: of max(|E|, sum|E_i|)),
or 4x the oracle's own change when W3 alone is rounded to FP16, whichever is
larger.  The form rounds W3 and z2 to FP16 for the per-path weights; on a few
isolated pairs whose forces are far below the size of the per-edge terms
(cancelling paths and layers) that rounding alone moves the oracle's forces
by more than 2e-3 of max|F| (1.6e-3 for W3 on the two-far-pairs system,
against 3.9e-4 on the 300-atom water box), so no FP16-operand product meets
the relative bar there; the second factor is the same rounding applied to z2.
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


def _assert_close(out, ref, tol, sens=None):
    """sens: (|dE|, max|dF|) of the oracle with W3 rounded to FP16 (16-bit forms)."""
    scale = max(abs(ref["energy"]), float(np.abs(ref["atom_energies"]).sum()))
    ebar, fbar = tol * scale, tol * np.abs(ref["forces"]).max()
    if sens is not None:
        ebar, fbar = max(ebar, 4.0 * sens[0]), max(fbar, 4.0 * sens[1])
    assert abs(float(np.asarray(out["energy"]).reshape(-1)[0]) - ref["energy"]) <= max(ebar, 1e-12)
    err = np.abs(np.asarray(out["forces"]) - ref["forces"]).max()
    assert err <= max(fbar, 1e-12), (err, fbar)


def _w3_fp16(spec, w):
    """The weights with every layer's W3 rounded to FP16 (nothing else changed)."""
    w2 = w.copy()
    off = 0
    for name, shape, _ in spec.weight_shapes():
        k = int(np.prod(shape))
        if name.startswith("W3."):
            w2[off:off + k] = w2[off:off + k].astype(np.float16).astype(np.float32)
        off += k
    return w2


def _sens(om16, pos, z, ref):
    r = om16.energy_forces(pos, z, np.eye(3), np.zeros(3, np.uint8))
    return abs(r["energy"] - ref["energy"]), float(np.abs(r["forces"] - ref["forces"]).max())


@pytest.mark.parametrize("name", ["water", "water_mace"])
def test_fused_degenerate_systems(B, name):
    spec = synth.model_spec(name)
    w = synth.make_weights(spec, 21)
    om, om16 = oracle.Model(spec, w), oracle.Model(spec, _w3_fp16(spec, w))
    cell, pbc = np.eye(3), np.zeros(3, np.uint8)
    for label, pos, z in SYSTEMS:
        ref = om.energy_forces(pos, z, cell, pbc, atom_energies=True)
        m = B.Model(spec, w, B.MLIP_PREC_F16)
        first = m.energy_forces(pos, z, cell, pbc)
        _assert_close(first, ref, 2e-3, _sens(om16, pos, z, ref))
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
    om, om16 = oracle.Model(spec, w), oracle.Model(spec, _w3_fp16(spec, w))
    p = {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16}[prec]
    for Q in (0.0, 1.0):
        om.set_total_charge(Q)
        om16.set_total_charge(Q)
        for label, pos, z in SYSTEMS:
            ref = om.energy_forces(pos, z, np.eye(3), np.zeros(3, np.uint8), atom_energies=True)
            m = B.Model(spec, w, p)
            out = m.energy_forces_charged(pos, z, Q)
            _assert_close(out, ref, tol, _sens(om16, pos, z, ref) if prec == "f16" else None)
            np.testing.assert_allclose(out["charges"], om.charges(pos, z), rtol=0,
                                       atol=tol * max(1.0, np.abs(om.charges(pos, z)).max()))
            if label == "beyond the cutoff" and Q == 0.0:
                assert np.abs(out["forces"]).max() > 0.0  # the long-range term alone
            m.close()
