"""GPU checks of the graph-replayed evaluation (evaluate_fused_graph).

Repeated calls with the same layout run the first evaluation with a
synchronising neighbour build, the second with the same launches as the
graph, the third captures a CUDA graph and later ones replay it; capacity
overflows are detected after the replay and the call is redone.  Every one
of these routes must give the same numbers, bit for bit, as a fresh model's
first (synchronising) call.
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


def _model(B, prec="f16"):
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    p = {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16, "bf16": B.MLIP_PREC_BF16}[prec]
    return B.Model(spec, w, p), spec, w


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in a)


def _fresh(B, s, stress):
    m, _, _ = _model(B)
    return m.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True, stress=stress)


@pytest.mark.parametrize("stress", [False, True])
def test_repeated_calls_equal_a_fresh_call(B, stress):
    s = synth.water_box(200, synth.water_side_for(200), seed=3)
    ref = _fresh(B, s, stress)
    m, _, _ = _model(B)
    for _ in range(6):  # exact, eager, capture, replays
        r = m.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True, stress=stress)
        assert _same(r, ref)


def test_device_arrays_and_changing_positions(B):
    import torch
    s = synth.water_box(150, synth.water_side_for(150), seed=8)
    rng = np.random.default_rng(5)
    pos_b = s.pos + rng.normal(0.0, 0.05, s.pos.shape)
    ref_a = _fresh(B, s, False)
    sb = synth.System(pos_b, s.species, s.cell, s.pbc)
    ref_b = _fresh(B, sb, False)
    m, _, _ = _model(B)
    tsp = torch.tensor(s.species, device="cuda")
    for k in range(8):
        p = s.pos if k % 2 == 0 else pos_b
        r = m.energy_forces(torch.tensor(p, device="cuda"), tsp, s.cell, s.pbc, forces=True)
        r = {key: v.cpu().numpy() for key, v in r.items()}
        assert _same(r, ref_a if k % 2 == 0 else ref_b), k


def test_edge_capacity_overflow_is_redone(B):
    """After the graph exists, a denser configuration with the same atoms has
    more edges than the graph's capacity (and receivers above its degree
    capacity): the call is redone exactly."""
    s = synth.water_box(100, synth.water_side_for(100), seed=4)
    m, _, _ = _model(B)
    for _ in range(4):
        m.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True)
    for scale in (0.75, 0.55):  # 2.4x and 6x the density
        dense = synth.System(s.pos * scale, s.species, s.cell * scale, s.pbc)
        r = m.energy_forces(dense.pos, dense.species, dense.cell, dense.pbc, forces=True)
        assert _same(r, _fresh(B, dense, False))
        # and the layout keeps working afterwards
        r2 = m.energy_forces(dense.pos, dense.species, dense.cell, dense.pbc, forces=True)
        assert _same(r2, r)


def test_graph_results_against_the_oracle(B):
    s = synth.water_box(100, synth.water_side_for(100), seed=9)
    m, spec, w = _model(B)
    for _ in range(4):
        r = m.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True, stress=True)
    ref = oracle.Model(spec, w).energy_forces(s.pos, s.species, s.cell, s.pbc, stress=True)
    fmax = np.abs(ref["forces"]).max()
    assert np.abs(r["forces"] - ref["forces"]).max() <= 2e-3 * fmax


def test_timing_and_launch_count_through_replays(B):
    s = synth.water_box(100, synth.water_side_for(100), seed=4)
    m, _, _ = _model(B)
    B.mlip_profile_enable(True)
    try:
        for _ in range(3):
            m.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True)
        B.mlip_profile_enable(True)  # clears the records: what follows are replays
        l0 = B.mlip_launch_count()
        for _ in range(4):
            m.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True)
        launches = B.mlip_launch_count() - l0
        rep = B.mlip_profile_report()["kernels"]
    finally:
        B.mlip_profile_enable(False)
    # 4 replays x 4 adjoint path-group launches (2 layers, L = 2), each timed by the graph's event nodes
    assert rep["tp_fused_bwd"][0] == 16 and rep["tp_fused_bwd"][1] > 0.0
    assert launches == sum(v[0] for v in rep.values())
