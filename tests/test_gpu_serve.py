"""GPU checks of the serving engine (continuous batching).

Every request's result must equal the single-system call on its own (alone vs
in a mix), bit for bit: the batch evaluation is independent of the other
systems in it, and the velocity-Verlet updates are per atom.  NVE batches that
keep their members step on a skin neighbour list kept on the device (equal to
fresh lists bit for bit, rebuilt when an atom leaves its skin), and served
results of both kinds agree with the FP64 oracle within the form's tolerance.
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


def _model(B, prec):
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    p = {"fp32": B.MLIP_PREC_FP32, "f16": B.MLIP_PREC_F16}[prec]
    return B.Model(spec, w, p), spec


def _mix():
    """Open clusters of the serving size mix plus one periodic box."""
    out = []
    for n, seed in [(40, 1), (230, 2), (8, 3), (900, 4), (120, 5), (2000, 6)]:
        s = synth.cluster(n, seed=seed)
        out.append(s)
    out.append(synth.water_box(100, synth.water_side_for(100), seed=2))
    return out


@pytest.mark.parametrize("prec", ["fp32", "f16"])
def test_energy_forces_requests_match_single_calls(B, prec):
    m, _ = _model(B, prec)
    ref_model, _ = _model(B, prec)
    systems = _mix()
    srv = B.Server(m, max_slots=64)
    ids = []
    for k, s in enumerate(systems):
        ids.append(srv.submit(B.MLIP_REQ_ENERGY_FORCES, s.pos, s.species, cell=s.cell, pbc=s.pbc,
                              want_stress=bool(s.pbc.all())))
    res = [srv.wait(i, 60000) for i in ids]
    st = srv.stats()
    srv.close()
    for s, r in zip(systems, res):
        assert r["status"] == 0
        one = ref_model.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=bool(s.pbc.all()))
        assert r["energy"] == one["energy"][0]
        assert np.array_equal(r["forces"], one["forces"])
        if s.pbc.all():
            assert np.array_equal(r["stress"], one["stress"])
        assert r["t_arrive"] <= r["t_admit"] <= r["t_done"]
    assert st["completed"] == len(systems) and st["failed"] == 0
    assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]


@pytest.mark.parametrize("prec", ["fp32", "f16"])
def test_nve_requests_match_single_trajectories(B, prec):
    """NVE requests of different lengths and time steps, mixed with energy+forces
    requests that come and go: each trajectory equals mlip_md_nve alone."""
    m, spec = _model(B, prec)
    ref_model, _ = _model(B, prec)
    systems = _mix()[:5]
    masses = np.asarray(spec.masses)
    srv = B.Server(m, max_slots=16)
    nve = []
    for k, s in enumerate(systems[:3]):
        v = synth.maxwell_boltzmann(masses[s.species], 300.0, seed=10 + k)
        steps, dt = [6, 3, 9][k], [0.5, 0.25, 0.5][k]
        nve.append((s, v, steps, dt, srv.submit(B.MLIP_REQ_NVE, s.pos, s.species, cell=s.cell, pbc=s.pbc,
                                                 vel=v, n_steps=steps, dt_fs=dt)))
    ef = [srv.submit(B.MLIP_REQ_ENERGY_FORCES, s.pos, s.species, cell=s.cell, pbc=s.pbc) for s in systems[3:]]
    for s, v, steps, dt, rid in nve:
        r = srv.wait(rid, 120000)
        assert r["status"] == 0
        pos, vel, pe, ke = ref_model.md_nve(s.pos, v, s.species, s.cell, s.pbc, dt, steps)
        assert np.array_equal(r["pe"], pe) and np.array_equal(r["ke"], ke)
        assert np.array_equal(r["pos"], pos) and np.array_equal(r["vel"], vel)
    for rid in ef:
        assert srv.wait(rid, 60000)["status"] == 0
    st = srv.stats()
    srv.close()
    assert st["iterations"] >= 10  # the longest run takes n_steps + 1 = 10 evaluations
    assert st["mean_batch_requests"] > 1.0


def test_maxwell_boltzmann_velocities(B):
    """vel = NULL: velocities from SplitMix64 normals by Box-Muller with the
    centre-of-mass velocity removed (the same recipe as synth.maxwell_boltzmann)."""
    m, spec = _model(B, "fp32")
    s = synth.cluster(50, seed=8)
    srv = B.Server(m)
    rid = srv.submit(B.MLIP_REQ_NVE, s.pos, s.species, temperature_K=450.0, seed=77, n_steps=0, dt_fs=0.5)
    r = srv.wait(rid, 60000)
    srv.close()
    ref = synth.maxwell_boltzmann(np.asarray(spec.masses)[s.species], 450.0, seed=77)
    assert np.abs(r["vel"] - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.array_equal(r["pos"], s.pos)
    assert len(r["pe"]) == 1


def test_budget_slots_and_lifecycle(B):
    m, _ = _model(B, "f16")
    systems = _mix()[:4]
    # a budget of 200 MB holds under 2000 atoms of this model: 4000 are rejected
    srv = B.Server(m, hbm_budget_bytes=200 << 20, max_slots=2, bucket_edges=(100, 1000))
    big = synth.cluster(4000, seed=9)
    with pytest.raises(B.MlipError) as e:
        srv.submit(B.MLIP_REQ_ENERGY_FORCES, big.pos, big.species)
    assert e.value.code == B.MLIP_ERR_BUDGET
    ids = [srv.submit(B.MLIP_REQ_ENERGY_FORCES, s.pos, s.species) for s in systems]
    long_id = srv.submit(B.MLIP_REQ_NVE, systems[1].pos, systems[1].species, n_steps=1000, dt_fs=0.5, seed=3)
    for i in ids:
        assert srv.wait(i, 60000)["status"] == 0
    with pytest.raises(B.MlipError) as e:  # still running
        srv.wait(long_id, 0)
    assert e.value.code == B.MLIP_ERR_TIMEOUT
    assert srv.release(long_id) == B.MLIP_PENDING
    r = srv.wait(long_id, 300000)
    assert r["status"] == 0 and len(r["pe"]) == 1001
    assert srv.release(long_id) == 0
    with pytest.raises(B.MlipError) as e:
        srv.poll(long_id)
    assert e.value.code == B.MLIP_ERR_NOT_FOUND
    st = srv.stats()
    srv.close()
    assert st["rejected"] == 1 and st["completed"] == 5
    assert st["mean_batch_requests"] <= 2.0
    assert sum(st["bucket_count"]) == 5 and len(st["bucket_count"]) == 3


def test_invalid_requests(B):
    m, _ = _model(B, "fp32")
    s = synth.cluster(30, seed=1)
    srv = B.Server(m)
    bad = s.species.copy()
    bad[3] = 7
    for kw, code in [(dict(species=bad), B.MLIP_ERR_INVALID_ARG),
                     (dict(want_stress=True), B.MLIP_ERR_CELL)]:
        args = dict(pos=s.pos, species=s.species)
        args.update(kw)
        with pytest.raises(B.MlipError) as e:
            srv.submit(B.MLIP_REQ_ENERGY_FORCES, args.pop("pos"), args.pop("species"), **args)
        assert e.value.code == code
    p = s.pos.copy()
    p[0, 0] = np.nan
    with pytest.raises(B.MlipError) as e:
        srv.submit(B.MLIP_REQ_ENERGY_FORCES, p, s.species)
    assert e.value.code == B.MLIP_ERR_INVALID_ARG
    with pytest.raises(B.MlipError) as e:
        srv.submit(B.MLIP_REQ_NVE, s.pos, s.species, n_steps=5, dt_fs=-1.0)
    assert e.value.code == B.MLIP_ERR_INVALID_ARG
    rid = srv.submit(B.MLIP_REQ_ENERGY_FORCES, s.pos, s.species)
    assert srv.wait(rid, 60000)["status"] == 0
    srv.close()


def test_host_wait_limit_stops_the_server(B):
    """device_poll_limit_us bounds the host's wait for an iteration; a limit of
    1 us runs out (a host-side timeout, the GPU work itself completes): the
    requests fail with MLIP_ERR_DEVICE_TIMEOUT and the server admits nothing."""
    m, _ = _model(B, "fp32")
    s = synth.cluster(1500, seed=4)
    srv = B.Server(m, device_poll_limit_us=1)
    rid = srv.submit(B.MLIP_REQ_NVE, s.pos, s.species, n_steps=50, dt_fs=0.5, seed=1)
    r = srv.wait(rid, 120000)
    assert r["status"] == B.MLIP_ERR_DEVICE_TIMEOUT
    with pytest.raises(B.MlipError) as e:
        srv.submit(B.MLIP_REQ_ENERGY_FORCES, s.pos, s.species)
    assert e.value.code == B.MLIP_ERR_DEVICE_TIMEOUT
    st = srv.stats()
    srv.close()
    assert st["failed"] == 1
    # the model is usable again once the server is gone
    out = m.energy_forces(s.pos, s.species, s.cell, s.pbc)
    assert np.isfinite(out["energy"][0])


def test_nve_batch_on_the_resident_skin_list(B):
    """Two NVE requests admitted together and nothing else: after the first
    iteration the batch keeps its members, so its steps run on the resident
    skin list (skin_steps counts them).  One request drifts as a whole at
    0.05 A/fs, so it moves more than skin/2 = 1 A within 40 steps and the list
    is rebuilt mid-run.  Both trajectories equal mlip_md_nve's (a fresh list
    at every step) bit for bit."""
    m, spec = _model(B, "f16")
    ref_model, _ = _model(B, "f16")
    masses = np.asarray(spec.masses)
    a, b = synth.cluster(300, seed=21), synth.cluster(120, seed=22)
    va = synth.maxwell_boltzmann(masses[a.species], 300.0, seed=31)
    vb = synth.maxwell_boltzmann(masses[b.species], 300.0, seed=32) + np.array([0.05, 0.0, 0.0])
    srv = B.Server(m, max_slots=8)
    ids = [srv.submit(B.MLIP_REQ_NVE, a.pos, a.species, vel=va, n_steps=60, dt_fs=0.5),
           srv.submit(B.MLIP_REQ_NVE, b.pos, b.species, vel=vb, n_steps=60, dt_fs=0.5)]
    res = [srv.wait(i, 120000) for i in ids]
    st = srv.stats()
    srv.close()
    for (s, v), r in zip(((a, va), (b, vb)), res):
        assert r["status"] == 0
        pos, vel, pe, ke = ref_model.md_nve(s.pos, v, s.species, s.cell, s.pbc, 0.5, 60)
        assert np.array_equal(r["pos"], pos) and np.array_equal(r["vel"], vel)
        assert np.array_equal(r["pe"], pe) and np.array_equal(r["ke"], ke)
    assert st["skin_steps"] >= 50, st["skin_steps"]  # steps 1..60, all but the first iteration or two
    assert st["skin_builds"] >= 2  # the first build, and at least one after the drift


def test_resident_list_threshold(B):
    """resident_after < 0: no resident list at all (every step a fresh list,
    the same trajectory bit for bit); resident_after = 1: the list from the
    first unchanged iteration on.  The statistics count the iterations whose
    membership changed (here only the first)."""
    spec_m, spec = _model(B, "f16")
    masses = np.asarray(spec.masses)
    a = synth.cluster(200, seed=23)
    va = synth.maxwell_boltzmann(masses[a.species], 300.0, seed=33)
    out = {}
    for ra in (-1, 1):
        srv = B.Server(spec_m, resident_after=ra)
        r = srv.wait(srv.submit(B.MLIP_REQ_NVE, a.pos, a.species, vel=va, n_steps=20, dt_fs=0.5), 120000)
        st = srv.stats()
        srv.close()
        assert r["status"] == 0
        out[ra] = (r, st)
    (r0, s0), (r1, s1) = out[-1], out[1]
    assert s0["skin_steps"] == 0 and s0["skin_builds"] == 0
    assert s1["skin_steps"] >= 15 and s1["skin_builds"] >= 1
    assert np.array_equal(r0["pos"], r1["pos"]) and np.array_equal(r0["pe"], r1["pe"])
    for st in (s0, s1):
        assert st["iterations"] == 21 and st["changed_iterations"] == 1
        assert 0.0 < st["changed_busy_s"] <= st["busy_s"]


def test_served_results_against_the_oracle(B):
    """One served energy+forces request and one served 10-step NVE request
    against the FP64 oracle: forces within 2e-3 of max|F| (FP16 form), the NVE
    trajectory's positions within 1e-6 A and its energies within 2e-3 of
    their scale (the bars of the single-call tests)."""
    m, spec = _model(B, "f16")
    w = synth.make_weights(spec, 21)
    om = oracle.Model(spec, w)
    masses = np.asarray(spec.masses)
    s1, s2 = synth.cluster(200, seed=41), synth.cluster(150, seed=42)
    v2 = synth.maxwell_boltzmann(masses[s2.species], 300.0, seed=43)
    srv = B.Server(m, max_slots=8)
    i1 = srv.submit(B.MLIP_REQ_ENERGY_FORCES, s1.pos, s1.species)
    i2 = srv.submit(B.MLIP_REQ_NVE, s2.pos, s2.species, vel=v2, n_steps=10, dt_fs=0.5)
    r1, r2 = srv.wait(i1, 60000), srv.wait(i2, 60000)
    srv.close()
    ref = om.energy_forces(s1.pos, s1.species, s1.cell, s1.pbc, atom_energies=True)
    scale = max(abs(ref["energy"]), float(np.abs(ref["atom_energies"]).sum()))
    assert abs(r1["energy"] - ref["energy"]) <= 2e-3 * scale
    err = np.abs(r1["forces"] - ref["forces"]).max() / np.abs(ref["forces"]).max()
    print(f" served E+F: max|dF|/max|F| = {err:.2e} (bar 0.002)", end="")
    assert err <= 2e-3
    rp, rv, rpe, rke = om.vv_nve(s2.pos, v2, s2.species, masses, s2.cell, s2.pbc, 0.5, 10)
    assert np.abs(r2["pos"] - rp).max() < 1e-6
    esc = np.abs(rpe).max() + np.abs(rke).max()
    assert np.abs(r2["pe"] - rpe).max() < 2e-3 * esc
    assert np.abs(r2["ke"] - rke).max() < 2e-3 * esc
