"""GPU checks of the skin-list MD driver (mlip_md_nve_skin).

The candidate list (pairs within rc + skin) is built before every block of
steps and compacted at every step to the pairs within rc, in the canonical
order; while no atom has moved more than skin/2 since the build this is the
list a fresh build finds, so the trajectories must equal mlip_md_nve_batch's
(a fresh list at every force evaluation) bit for bit, with and without CUDA
graphs, and also when an atom leaves its skin and the block is run again.
"""
import numpy as np
import pytest

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
    return B.Model(spec, w, p), spec


def _replicas(spec, nrep=3, nmol=60, cluster=True):
    """Periodic water replicas (and one open cluster): concatenated arrays."""
    masses = np.asarray(spec.masses)
    systems = [synth.water_box(nmol, synth.water_side_for(nmol), seed=30 + k) for k in range(nrep)]
    if cluster:
        c = synth.cluster(120, seed=5)
        c.species[:] = c.species % len(masses)
        systems.append(c)
    vels = [synth.maxwell_boltzmann(masses[s.species], 300.0, seed=40 + k) for k, s in enumerate(systems)]
    off = np.cumsum([0] + [s.n for s in systems])
    return (off, np.concatenate([s.pos for s in systems]), np.concatenate(vels),
            np.concatenate([s.species for s in systems]).astype(np.int32), np.stack([s.cell for s in systems]),
            np.stack([s.pbc for s in systems]))


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_skin_md_equals_fresh_lists(B, prec):
    m, spec = _model(B, prec)
    off, pos, vel, sp, cells, pbc = _replicas(spec)
    ref = m.md_nve_batch(off, pos, vel, sp, cells, pbc, 0.5, 35)
    P, V, PE, KE, rep = m.md_nve_skin(off, pos, vel, sp, cells, pbc, 0.5, 35, skin=2.0, rebuild_every=10)
    assert _same((P, V, PE, KE), ref)
    # builds at steps 0, 10, 20, 30; the first full block runs eagerly (a
    # graph is captured only once the workspace has its sizes), later full
    # blocks run as a graph, the partial last block eagerly
    assert rep["builds"] == 4 and rep["redone_blocks"] == 0
    assert rep["graph_captures"] >= 1 and rep["graph_launches"] >= 1
    assert 0.0 < rep["max_displacement"] < 1.0
    assert rep["max_candidates"] > 0


def test_skin_md_without_graphs_is_the_same(B):
    m, spec = _model(B)
    off, pos, vel, sp, cells, pbc = _replicas(spec)
    a = m.md_nve_skin(off, pos, vel, sp, cells, pbc, 0.5, 25, skin=2.0, rebuild_every=10, use_graph=True)
    b = m.md_nve_skin(off, pos, vel, sp, cells, pbc, 0.5, 25, skin=2.0, rebuild_every=10, use_graph=False)
    assert _same(a[:4], b[:4])
    assert b[4]["graph_captures"] == 0 and b[4]["graph_launches"] == 0


def test_skin_md_block_rerun_when_an_atom_leaves_its_skin(B):
    """A skin of 0.02 A is left within a few steps: the block is run again
    with a fresh list at every step, and the trajectory is still exact."""
    m, spec = _model(B)
    off, pos, vel, sp, cells, pbc = _replicas(spec, nrep=2, cluster=False)
    ref = m.md_nve_batch(off, pos, vel, sp, cells, pbc, 0.5, 20)
    P, V, PE, KE, rep = m.md_nve_skin(off, pos, vel, sp, cells, pbc, 0.5, 20, skin=0.02, rebuild_every=10)
    assert rep["redone_blocks"] >= 1
    assert rep["max_displacement"] > 0.01
    assert _same((P, V, PE, KE), ref)


def test_skin_md_single_step_blocks(B):
    """rebuild_every = 1: a build before every step (the start's build serves
    the first); graphs replayed per step."""
    m, spec = _model(B)
    off, pos, vel, sp, cells, pbc = _replicas(spec, nrep=1, cluster=True)
    ref = m.md_nve_batch(off, pos, vel, sp, cells, pbc, 0.5, 6)
    P, V, PE, KE, rep = m.md_nve_skin(off, pos, vel, sp, cells, pbc, 0.5, 6, skin=1.0, rebuild_every=1)
    assert _same((P, V, PE, KE), ref)
    assert rep["builds"] == 6 and rep["graph_launches"] >= 1


def test_skin_md_device_arrays(B):
    """torch CUDA tensors are integrated in place, same results."""
    import torch
    m, spec = _model(B)
    off, pos, vel, sp, cells, pbc = _replicas(spec, nrep=2, cluster=False)
    ref = m.md_nve_skin(off, pos, vel, sp, cells, pbc, 0.5, 12, skin=2.0, rebuild_every=5)
    tp = torch.tensor(pos, device="cuda")
    tv = torch.tensor(vel, device="cuda")
    ts = torch.tensor(sp, device="cuda")
    P, V, PE, KE, _ = m.md_nve_skin(off, tp, tv, ts, cells, pbc, 0.5, 12, skin=2.0, rebuild_every=5)
    assert np.array_equal(tp.cpu().numpy(), ref[0]) and np.array_equal(tv.cpu().numpy(), ref[1])
    assert np.array_equal(PE.cpu().numpy(), ref[2]) and np.array_equal(KE.cpu().numpy(), ref[3])


def test_skin_md_errors(B):
    m32, spec = _model(B, "fp32")
    off, pos, vel, sp, cells, pbc = _replicas(spec, nrep=1, cluster=False)
    with pytest.raises(B.MlipError) as e:
        m32.md_nve_skin(off, pos, vel, sp, cells, pbc, 0.5, 4)
    assert e.value.code == B.MLIP_ERR_INVALID_ARG
    m, _ = _model(B)
    for kw in [dict(skin=0.0), dict(skin=-1.0), dict(rebuild_every=0)]:
        with pytest.raises(B.MlipError) as e:
            m.md_nve_skin(off, pos, vel, sp, cells, pbc, 0.5, 4, **kw)
        assert e.value.code == B.MLIP_ERR_INVALID_ARG
    # no steps: the start only
    P, V, PE, KE, rep = m.md_nve_skin(off, pos, vel, sp, cells, pbc, 0.5, 0)
    ref = m.md_nve_batch(off, pos, vel, sp, cells, pbc, 0.5, 0)
    assert _same((P, V, PE, KE), ref) and rep["builds"] == 1
