"""Parity at the full sizes of the benchmark workloads.

The oracle cannot evaluate 108,000 atoms in a test, but the force on one atom
depends only on atoms within 2 T r_c of it (the energy of atom k depends on
atoms within T r_c of k through T message-passing layers, and only atoms k
within T r_c of atom i have energies that move with r_i).  So the force on a
sampled atom of the full periodic system equals the force on the same atom
in the open cluster of every atom within 2 T r_c (+ margin) of it, which the
oracle evaluates.  The batched MD workload is checked by its own property
(every replica's result equals the replica evaluated alone, bit for bit) and
one replica against the oracle.
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


def _min_image(s, centre):
    inv = np.linalg.inv(s.cell)
    f = (s.pos - centre) @ inv
    f -= np.round(f)
    return f @ s.cell


def _region_clusters(s, radius, n_regions=4, per_region=8, seed=11):
    """Sampled atoms in n_regions spots of the periodic system: the per_region
    atoms nearest to each of n_regions random centres, with the open cluster
    of every atom within `radius` of any of them (minimum images; the cell is
    wider than twice the cluster).  Yields (sampled atom indices, cluster
    positions, cluster species, rows of the sampled atoms in the cluster)."""
    rng = np.random.default_rng(seed)
    for c in rng.choice(s.n, size=n_regions, replace=False):
        d = _min_image(s, s.pos[c])
        r2 = np.einsum("ij,ij->i", d, d)
        sampled = np.argsort(r2, kind="stable")[:per_region]
        reach = np.sqrt(r2[sampled].max()) + radius
        sel = np.flatnonzero(r2 < reach * reach)
        rows = np.searchsorted(sel, sampled)
        assert np.array_equal(sel[rows], sampled)
        yield sampled, s.pos[c] + d[sel], s.species[sel].astype(np.int32), rows


@pytest.fixture(scope="module")
def fcc108k():
    spec = synth.model_spec("fcc")
    return spec, synth.make_weights(spec, 31), synth.fcc((30, 30, 30), seed=3)


@pytest.fixture(scope="module")
def fcc108k_oracle_forces(fcc108k):
    """Oracle forces of 32 sampled atoms (4 spots x 8 atoms), each from the
    open cluster of every atom within 2 T r_c + 0.5 A of the spot's atoms."""
    spec, w, s = fcc108k
    radius = 2 * spec.T * spec.rc + 0.5
    om = oracle.Model(spec, w)
    idx, ref = [], []
    for sampled, cp, csp, rows in _region_clusters(s, radius):
        r = om.energy_forces(cp, csp, np.eye(3) * 1000.0, np.zeros(3, np.uint8))
        idx.append(sampled)
        ref.append(r["forces"][rows])
    idx = np.concatenate(idx)
    assert len(set(s.species[idx].tolist())) == 2  # both species sampled
    return idx, np.concatenate(ref)


@pytest.mark.parametrize("prec,tol", [("f16", 2e-3), ("fp32", 1e-5)])
def test_fcc108k_sampled_forces_against_the_oracle(B, fcc108k, fcc108k_oracle_forces, prec, tol):
    spec, w, s = fcc108k
    assert s.n == 108000
    p = {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16}[prec]
    m = B.Model(spec, w, p)
    r = m.energy_forces(s.pos, s.species, s.cell, s.pbc, forces=True, stress=True)
    m.close()
    F = r["forces"]
    fmax = np.abs(F).max()
    # forces sum to zero over the whole periodic system
    assert np.abs(F.sum(axis=0)).max() <= 1e-6 * fmax * np.sqrt(s.n)
    idx, ref = fcc108k_oracle_forces
    err = np.abs(F[idx] - ref).max()
    print(f"fcc108k {prec}: max |dF| over {len(idx)} sampled atoms = {err / fmax:.3e} of max|F| (bar {tol})")
    assert err <= tol * fmax, (prec, err, fmax)


def test_md64_batch_equals_replicas_and_oracle(B):
    """The batched-MD workload's evaluation (64 replicas of 5001 atoms as one
    graph): every replica's energy and forces equal the replica alone bit for
    bit; one replica against the oracle."""
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    m = B.Model(spec, w, B.MLIP_PREC_F16)
    import multiprocessing as mp
    import os
    with mp.get_context("spawn").Pool(min(64, os.cpu_count() or 1)) as pool:  # spawn: CUDA is initialised
        reps = pool.starmap(synth.water_box, [(1667, 36.76, 500 + k) for k in range(64)])
    energy, forces, _ = m.energy_forces_batch([(r.pos, r.species, r.cell, r.pbc) for r in reps], forces=True)
    assert sum(r.n for r in reps) == 320064
    for k in (0, 17, 63):
        one = m.energy_forces(reps[k].pos, reps[k].species, reps[k].cell, reps[k].pbc, forces=True)
        assert energy[k] == one["energy"][0]
        assert np.array_equal(forces[k], one["forces"])
    ref = oracle.Model(spec, w).energy_forces(reps[5].pos, reps[5].species, reps[5].cell, reps[5].pbc)
    assert np.abs(forces[5] - ref["forces"]).max() <= 2e-3 * np.abs(ref["forces"]).max()
