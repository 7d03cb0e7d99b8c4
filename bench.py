#!/usr/bin/env python
"""Benchmark: energy+force atom-steps/s of the equivariant interaction layer.

Default workload (the metric's configuration): a periodic FCC cell of
30 x 30 x 30 conventional cells (108,000 atoms, a = 3.6 A, Gaussian
displacements of 0.1 A, two species 50/50), the two-layer, 128-channel,
l <= 3 model with l <= 3 edge harmonics and a 64-wide radial MLP (random
weights), in the FP16-operand tensor-core form, with the plain FP32 GPU form
timed beside it.  One step = one full evaluation through the library's C ABI
with the positions resident on the GPU: neighbour list (cell list), edge
geometry, harmonics, radial basis and MLP, tensor product and segmented sum,
channel mixes, readout and FP64 energy, then the adjoint: forces and virial
stress.  The same line carries the 3000-atom water box (1000 H2O in a 31.0 A
cube) and a bounded serving phase (requests of 8-5000 atoms, 70 % energy+forces
and 30 % 100-step NVE, Poisson arrivals; p50/p99 latency) as sub-objects.
The synthetic systems stand in for the paper's MD benchmark systems (Table
tbl:performance), which are not available here.

Between timed steps L2 is flushed by writing a 512 MB buffer (outside the
per-step CUDA-event pairs).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload on the host cores.  --gpus N runs N
independent replicas, one process per GPU (launched through
torch.distributed.run when the environment holds no rank).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "energy+force atom-steps/s"
UNIT = "atom-steps/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}


# DRAM bytes (read + write) per launch of a kernel from one ncu capture, keyed by
# (workload, precision, kernel), with the SHA-256 prefix of the source file the
# kernel was built from at capture time.  When the file has changed since, the
# counters no longer describe the running kernel and the roofline reports no
# traffic.
# fcc108k: captured on the 20^3-cell FCC (32,000 atoms, 1,439,826 edges; the full cell is
# too large for a capture), mean of the five adjoint launches of one evaluation, scaled by
# the edge count (the sender gathers are per edge)
NCU_TRAFFIC = {("water3000", "f16", "tp_fused_bwd"): (129.7e6, "fused_bf16.cu", None),
               ("fcc108k", "f16", "tp_fused_bwd"): (26.035007e9 / 5 * 4860690 / 1439826, "fused_bf16.cu",
                                                    "ce5b70cb78f48cf8")}
# DRAM bytes per launch of the symmetric contraction's kernels at fcc108k: captured on the
# 20^3-cell FCC (32,000 atoms; the full workload is too large for a capture) and scaled by the
# atom count (traffic grows in proportion: per-node tensors)
NCU_TRAFFIC_SC = {("fcc108k_mace", "f16", "sym_contract"): (991.3e6 * 108000 / 32000, "sym_contract.cu", None),
                  ("fcc108k_mace", "f16", "sym_contract_bwd"): (741.2e6 * 108000 / 32000, "sym_contract.cu", None)}


def _src_digest(fname: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, "paper_2605_22698_gb300", "csrc", fname), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_of(table, key):
    """Captured DRAM bytes per launch, or None when unknown or when the kernel's
    source changed since the capture (digest None: captured before digests were
    recorded, so it cannot be shown to describe the running kernel)."""
    ent = table.get(key)
    if not ent:
        return None
    nbytes, fname, digest = ent
    if digest is None or _src_digest(fname) != digest:
        return None
    return nbytes


# FP32 ALU peak from unit counts and the maximum SM clock: 152 SMs x 128 FP32
# lanes x 2 flop (FMA) x 2.07 GHz.
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0])); mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def barrier(world: int) -> None:
    """Barrier over the ranks (no-op on one rank), with the device idle on both sides."""
    if world <= 1:
        return
    import torch
    import torch.distributed as dist
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def max_over_ranks(t: float, world: int) -> float:
    """The largest of the ranks' times (the job's time); t itself on one rank."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    tt = torch.tensor([t], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def _with_option(spec_w_s, name):
    """The same workload on the model with the symmetric contraction of
    correlation order 2 after every scatter-sum (suffix _mace) or with the
    gated update and species self-connection (suffix _gated)."""
    import dataclasses
    base, opt = name.rsplit("_", 1)
    spec, _, *rest = spec_w_s
    spec = dataclasses.replace(spec, **({"correlation": 2} if opt == "mace" else {"gate": 1}))
    seed = {"water3000": 21, "fcc108k": 31}[base]
    return (spec, synth.make_weights(spec, seed), *rest)


def workload(name: str, rank: int = 0, fcc_cells: int = 30):
    if name.endswith(("_mace", "_gated")):
        return _with_option(workload(name.rsplit("_", 1)[0], rank, fcc_cells), name)
    if name == "water3000":
        spec = synth.model_spec("water")
        sysm = synth.water_box(1000, 31.0, seed=2 + 1000 * rank)
        return spec, synth.make_weights(spec, 21), sysm
    if name == "fcc108k":
        spec = synth.model_spec("fcc")
        nc = (fcc_cells,) * 3  # 30^3 cells = 108,000 atoms; fewer only for small profiling captures
        return spec, synth.make_weights(spec, 31), synth.fcc(nc, seed=3 + 1000 * rank)
    if name == "cluster64":
        spec = synth.model_spec("small")
        return spec, synth.make_weights(spec, 7), synth.cluster64(1 + rank)
    if name == "cluster5000_charged":  # the largest serving request, model with charges and the Coulomb term
        spec = synth.model_spec("water_charged")
        return spec, synth.make_weights(spec, 21), synth.cluster(5000, seed=7 + 1000 * rank)
    raise ValueError(name)


def sample_workload(name: str):
    """Bounded CPU sample of the same workload for the oracle baseline."""
    if name.endswith(("_mace", "_gated")):
        return _with_option(sample_workload(name.rsplit("_", 1)[0]), name)
    if name == "water3000":
        spec = synth.model_spec("water")
        return spec, synth.make_weights(spec, 21), synth.water_box(100, synth.water_side_for(100), seed=2), \
            "100 H2O (300 atoms) periodic box at the same density, same model"
    if name == "fcc108k":
        spec = synth.model_spec("fcc")
        return spec, synth.make_weights(spec, 31), synth.fcc((3, 3, 4), seed=3), \
            "FCC 3x3x4 cells (144 atoms), same model"
    if name == "md64":
        spec = synth.model_spec("water")
        return spec, synth.make_weights(spec, 21), synth.water_box(100, synth.water_side_for(100), seed=500), \
            "one 100 H2O (300 atoms) periodic box at the replicas' density, same model"
    if name == "cluster5000_charged":
        spec = synth.model_spec("water_charged")
        return spec, synth.make_weights(spec, 21), synth.cluster(200, seed=7), \
            "one 200-atom open cluster, same model with charges"
    if name == "serve":
        spec = synth.model_spec("water")
        return spec, synth.make_weights(spec, 21), synth.cluster(200, seed=4), \
            "one 200-atom open cluster (the median request size) energy+forces, same model"
    spec = synth.model_spec("small")
    return spec, synth.make_weights(spec, 7), synth.cluster64(1), "the full 64-atom cluster"


def time_oracle(name: str, min_seconds: float, max_evals: int = 1000):
    import oracle
    spec, w, s, desc = sample_workload(name)
    m = oracle.Model(spec, w)
    stress = bool(s.pbc.all())
    m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=stress)  # warm-up
    t0 = time.perf_counter()
    k = 0
    while True:
        m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=stress)
        k += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds or k >= max_evals:
            break
    return {"value": s.n * k / dt, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{desc}; {k} energy+force(+stress) evaluations in {dt:.1f} s"}


# Nonzero real Clebsch-Gordan entries of each coupling path (l1, l2, l3),
# natural parity, l2 <= 3: a property of the paths (counted once from the
# coupling tables), used for the algorithmic flop counts below.
CG_NNZ = {
    (0, 0, 0): 1, (0, 1, 1): 3, (0, 2, 2): 5, (0, 3, 3): 7, (1, 0, 1): 3, (1, 1, 0): 3, (1, 1, 2): 11,
    (1, 2, 1): 11, (1, 2, 3): 21, (1, 3, 2): 21, (2, 0, 2): 5, (2, 1, 1): 11, (2, 1, 3): 21, (2, 2, 0): 5,
    (2, 2, 2): 25, (2, 3, 1): 21, (2, 3, 3): 41, (3, 0, 3): 7, (3, 1, 2): 21, (3, 2, 1): 21, (3, 2, 3): 41,
    (3, 3, 0): 7, (3, 3, 2): 41,
}


def model_paths(spec):
    out = []
    for l1 in range(spec.L + 1):
        for l2 in range(spec.Lsh + 1):
            for l3 in range(spec.L + 1):
                if abs(l1 - l2) <= l3 <= l1 + l2 and (l1 + l2 + l3) % 2 == 0:
                    out.append((l1, l2, l3))
    return out


def tp_flops_per_edge_channel(spec, first: bool, backward: bool) -> int:
    """FP32 flops of the tensor product per edge and channel.
    forward:  per path (2 l1 + 1) products w h, then 2 flops per CG entry;
    backward: dE/dh (not first layer): 2 (2 l3 + 1) products s w Gm + 2 per entry;
              T_p: 3 per entry (h Gt product, FMA with the coefficient);
              dE/dw and dE/dY: 2 (2 l2 + 1) each."""
    tot = 0
    for (l1, l2, l3) in model_paths(spec):
        if first and l1 != 0:
            continue
        nz = CG_NNZ[(l1, l2, l3)]
        if not backward:
            tot += (2 * l1 + 1) + 2 * nz
        else:
            if not first:
                tot += 2 * (2 * l3 + 1) + 2 * nz
            tot += 3 * nz + 4 * (2 * l2 + 1)
    return tot


def algorithmic_flops(spec, E: int, n: int):
    """Algorithmic flops per step per kernel name (edge counts x per-edge work)."""
    P0 = spec.L + 1
    P = len(model_paths(spec))
    C, H, T = spec.C, spec.H, spec.T
    pw = [P0] + [P] * (T - 1)
    fwd_tp = sum(tp_flops_per_edge_channel(spec, t == 0, False) for t in range(T)) * E * C
    bwd_tp = sum(tp_flops_per_edge_channel(spec, t == 0, True) for t in range(T)) * E * C
    mlp_out = sum(2 * E * H * C * p for p in pw)          # w = z2 W3 (one product)
    return {
        "sgemm": 2 * mlp_out,                              # forward w and backward dz2 (plain form)
        "tp_fwd": fwd_tp, "tp_bwd": bwd_tp,
        "tp_fused": fwd_tp, "tp_fused_bwd": bwd_tp,        # FP32 ALU work; the MMAs run on the tensor pipe
        "tensor_fused": mlp_out, "tensor_fused_bwd": 2 * mlp_out,
    }


def measure_fp32_peak():
    """FP32 FMA rate measured on this GPU by the library's microbenchmark, with
    the SM clock sampled while it runs; the derived figure if it fails."""
    import torch
    from paper_2605_22698_gb300 import binding as B
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    try:
        B.mlip_fp32_fma_rate(2000)  # warm-up
        runs = [B.mlip_fp32_fma_rate(20000) for _ in range(5)]
    except Exception as e:  # noqa: BLE001
        sampler.stop()
        return {"tflops": FP32_ALU_TFLOPS, "src": f"derived (measurement failed: {e})"}
    clocks = sampler.stop()
    best = max(runs, key=lambda r: r["tflops"])
    return {"tflops": round(best["tflops"], 2), "sms": best["sms"], "ms": round(best["ms"], 3),
            "src": (f"measured: FP32 FMA microbenchmark (independent FMA chains filling all {best['sms']} SMs), "
                    "best of 5 launches, CUDA events"),
            "clocks": clocks, "derived_at_max_clock": round(FP32_ALU_TFLOPS, 1)}


def measure(args, rank, world, name, steps, warmup, fp32_peak, plain=True, cpu=True, fcc_cells=30):
    """One workload through mlip_energy_forces: the timed device steps, the
    end-to-end steps with host arrays, the dominant kernel's roofline, the
    kernel shares and (optionally) the plain FP32 form and the oracle."""
    import torch
    from paper_2605_22698_gb300 import binding as B
    dev = torch.device("cuda", torch.cuda.current_device())
    spec, w, s = workload(name, rank, fcc_cells)
    precision = args.precision
    if spec.C != 128 or spec.H != 64:
        precision = "fp32"  # the fused 16-bit form serves 128-channel, hidden-64 models only
    prec = {"fp32": B.MLIP_PREC_FP32, "bf16": B.MLIP_PREC_BF16, "f16": B.MLIP_PREC_F16}[precision]
    model = B.Model(spec, w, prec)
    pos = torch.tensor(s.pos, device=dev)
    sp = torch.tensor(s.species, device=dev)
    stress = bool(s.pbc.all())
    out = {"energy": torch.zeros(1, dtype=torch.float64, device=dev),
           "forces": torch.zeros((s.n, 3), dtype=torch.float64, device=dev)}
    if stress:
        out["stress"] = torch.zeros((3, 3), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        model.energy_forces(pos, sp, s.cell, s.pbc, forces=True, stress=stress, stream=stream, out=out)

    for _ in range(warmup):
        step()
    # kernel shares: every kernel timed, on steps outside the timed region (the
    # evaluation is a replayed CUDA graph after three calls with one layout and
    # one timing configuration; the shares come from replays)
    B.mlip_profile_select(None)
    B.mlip_profile_enable(True)
    for _ in range(3):
        step()
    B.mlip_profile_enable(True)  # clears the records
    n_share = 4
    for _ in range(n_share):
        step()
    share_rep = B.mlip_profile_report().get("kernels", {})
    B.mlip_profile_enable(False)
    top_name = max(share_rep.items(), key=lambda kv: kv[1][1])[0] if share_rep else None
    # the timed region times the dominant kernel only (events around its launches)
    B.mlip_profile_select([top_name] if top_name else None)
    B.mlip_profile_enable(True)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    barrier(world)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    B.mlip_profile_enable(True)  # clears the records
    launches0 = B.mlip_launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t_wall0 = time.perf_counter()
    for k in range(steps):
        flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    t_wall = time.perf_counter() - t_wall0
    launches = B.mlip_launch_count() - launches0
    prof = B.mlip_profile_report()
    B.mlip_profile_enable(False)
    B.mlip_profile_select(None)
    clocks = sampler.stop() if sampler else None
    ms = [a.elapsed_time(b) for a, b in evs]
    t_dev = max_over_ranks(sum(ms) / 1e3, world)
    value = world * s.n * steps / t_dev
    # edge count of this structure (for the algorithmic counts)
    r, _, _ = B.mlip_neighbors(np.ascontiguousarray(s.pos), s.cell, s.pbc, spec.rc)
    E_edges = len(r)
    del r

    # end-to-end: host arrays in pinned memory, copies inside the timed region
    pin_pos = torch.empty((s.n, 3), dtype=torch.float64, pin_memory=True).numpy()
    pin_pos[:] = s.pos
    pin_sp = torch.empty(s.n, dtype=torch.int32, pin_memory=True).numpy()
    pin_sp[:] = s.species
    for _ in range(4):  # past the graph capture
        model.energy_forces(pin_pos, pin_sp, s.cell, s.pbc, forces=True, stress=stress)
    k_e2e = max(3, steps // 2)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        res = model.energy_forces(pin_pos, pin_sp, s.cell, s.pbc, forces=True, stress=stress)
        _ = float(res["energy"][0])
    t_e2e = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": round(world * s.n * k_e2e / t_e2e, 1), "unit": UNIT,
           "h2d_bytes_per_step": int(pin_pos.nbytes + pin_sp.nbytes),
           "d2h_bytes_per_step": int(8 + s.n * 3 * 8 + (72 if stress else 0)), "steps": k_e2e}

    # roofline of the dominant kernel
    peak = fp32_peak["tflops"]
    kern = prof.get("kernels", {})
    roof = None
    if kern:
        top = max(kern.items(), key=lambda kv: kv[1][1])
        kname, (nl, tot_ms) = top
        flops = algorithmic_flops(spec, E_edges, s.n)
        roof = {"kernel": kname, "bound": "alu", "achieved": None, "peak": peak, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "launches": nl, "avg_launch_ms": round(tot_ms / nl, 5),
                "peak_src": fp32_peak["src"] + " (of measured)"}
        if kname in flops:
            per_step = flops[kname]
            achieved = per_step * steps / (tot_ms / 1e3) / 1e12
            nl_step = max(1, round(nl / steps))
            roof.update({"achieved": round(achieved, 3), "frac": round(achieved / peak, 4),
                         "flops_per_launch": round(per_step / nl_step),
                         "traffic": traffic_of(NCU_TRAFFIC, (name, precision, kname))
                         if (name != "fcc108k" or fcc_cells == 30) else None})
            if kname in ("tp_fused", "tp_fused_bwd"):
                tk = "tensor_" + kname[3:]
                tens = flops[tk] * steps / (tot_ms / 1e3) / 1e12
                roof["tensor_pipe"] = {"achieved": round(tens, 2), "peak": peaks()["bf16_tflops"],
                                       "frac": round(tens / peaks()["bf16_tflops"], 4), "unit": "TFLOP/s"}
    # the symmetric contraction's kernels (node-wise, bound by memory): algorithmic bytes per launch
    # over their mean launch time in the shares pass
    sc_roof = None
    if "sym_contract" in share_rep:
        nodes = s.n * (spec.L + 1) ** 2 * spec.C * 4
        n_in = 2 if precision != "fp32" else 1  # the fused form's two partial message buffers
        sc_roof = {}
        for kname, nbytes in (("sym_contract", (n_in + 2) * nodes), ("sym_contract_bwd", 3 * nodes)):
            nl_, tot_ = share_rep.get(kname, (0, 0.0))
            if nl_:
                gbs = nbytes / (tot_ / nl_ / 1e3) / 1e9
                sc_roof[kname] = {"bound": "hbm", "bytes_per_launch": int(nbytes), "avg_launch_ms": round(tot_ / nl_, 5),
                                  "achieved": round(gbs, 1), "peak": peaks()["hbm_gbs"], "unit": "GB/s",
                                  "frac": round(gbs / peaks()["hbm_gbs"], 4),
                                  "traffic": traffic_of(NCU_TRAFFIC_SC, (name, precision, kname))
                                  if fcc_cells == 30 else None}
    # the gated update's kernels, per step over all layers, each direction: 4 C^2 (D + L) algorithmic
    # flops per node and layer; algorithmic bytes per node and layer (FP32): forward reads the two
    # message buffers and h, writes pre and h' (D rows each) and the gates (L rows), the adjoint reads
    # and writes dE/dh' (two buffers), reads pre and the gates, writes dE/dpre, dE/dg, dE/dm and dE/dh.
    # The fused form runs them on the tensor cores (split FP16, three products per term; latency-bound
    # at these sizes, so the HBM figure is reported beside the flop rate); the plain form on the ALUs.
    gate_roof = None
    if "gate_fwd" in share_rep:
        D_ = (spec.L + 1) ** 2
        flop = 4.0 * spec.C * spec.C * (D_ + spec.L) * s.n * spec.T
        nbytes = {"fwd": (5 * D_ + spec.L) * spec.C * 4.0 * s.n * spec.T,
                  "bwd": (10 * D_ + 3 * spec.L) * spec.C * 4.0 * s.n * spec.T}
        tensor = precision != "fp32"
        tpk = peaks()["bf16_tflops"] if tensor else peak
        gate_roof = {}
        for key, names in (("fwd", ("gate_fwd",)), ("bwd", ("gate_prep", "gate_bwd"))):
            ms = sum(share_rep.get(k_, (0, 0.0))[1] for k_ in names) / n_share
            if ms <= 0:
                continue
            tf = flop / (ms / 1e3) / 1e12
            gbs = nbytes[key] / (ms / 1e3) / 1e9
            gate_roof[key] = {"kernels": list(names), "ms_per_step": round(ms, 4), "flops_per_step": flop,
                              "bound": "tensor" if tensor else "alu", "achieved": round(tf, 2), "peak": tpk,
                              "unit": "TFLOP/s", "frac": round(tf / tpk, 4),
                              "hbm": {"bytes_per_step": nbytes[key], "achieved": round(gbs, 1),
                                      "peak": peaks()["hbm_gbs"], "unit": "GB/s",
                                      "frac": round(gbs / peaks()["hbm_gbs"], 4)}}
    # the Coulomb term (models with charges): pair evaluations per second of its all-pairs kernel
    coul = None
    if "coulomb_pairs" in share_rep:
        nl_, tot_ = share_rep["coulomb_pairs"]
        pairs = s.n * (s.n - 1)  # ordered pairs: every atom's sum runs over all others
        gps = pairs / (tot_ / nl_ / 1e3) / 1e9
        coul = {"kernel": "coulomb_pairs", "pairs_per_launch": int(pairs), "avg_launch_ms": round(tot_ / nl_, 5),
                "gpairs_per_s": round(gps, 2)}
    share = {}
    tot_all = sum(v[1] for v in share_rep.values()) or 1.0
    for k_, v in sorted(share_rep.items(), key=lambda kv: -kv[1][1])[:8]:
        share[k_] = round(v[1] / tot_all, 4)
    model.close()
    del model

    # the plain FP32 form on the same workload, reported beside the headline form
    plain_line = None
    if plain and precision != "fp32":
        pm = B.Model(spec, w, B.MLIP_PREC_FP32)

        def pstep():
            pm.energy_forces(pos, sp, s.cell, s.pbc, forces=True, stress=stress, stream=stream, out=out)
        for _ in range(3):
            pstep()
        kp = max(5, steps // 4)
        pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(kp)]
        barrier(world)
        for k in range(kp):
            flush.zero_()
            pev[k][0].record(stream)
            pstep()
            pev[k][1].record(stream)
        torch.cuda.synchronize()
        tp = max_over_ranks(sum(a.elapsed_time(b) for a, b in pev) / 1e3, world)
        plain_line = {"precision": "fp32", "value": round(world * s.n * kp / tp, 1), "unit": UNIT, "steps": kp,
                      "ms_per_step": round(1e3 * tp / kp, 4), "speedup_of_headline_form": round(value / (world * s.n * kp / tp), 3)}
        pm.close()
        del pm
    del flush
    torch.cuda.empty_cache()

    cpu_line = None
    if cpu and rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_line = time_oracle(name, args.cpu_seconds)

    return {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": round(1e3 * t_dev / steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16 tensor-core MLP + f32", "f16": "f16 tensor-core MLP + f32"}[precision],
        "data": "synthetic", "impl": "ours",
        "config": {"workload": name, "atoms": s.n, "edges": E_edges,
                   "model": f"T{spec.T} C{spec.C} L{spec.L} H{spec.H}" + (" SC2" if spec.correlation else "")
                   + (" gated" if spec.gate else ""),
                   "precision": precision, "parallelism": f"replicas x{world}" if world > 1 else "single",
                   "l2": "flushed between steps (512 MB write)", "stress": stress},
        "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "kernel_share": share,
        "kernel_ms_per_step": round(tot_all / n_share, 4),
        "sym_contract_roofline": sc_roof,
        "coulomb": coul,
        "gate_roofline": gate_roof,
        "timing": "timed steps: CUDA events around the dominant kernel's launches only (graph event nodes); "
                  "kernel_share from 4 steps with every kernel timed, outside the timed region",
        "plain_fp32": plain_line,
        "cpu_baseline": cpu_line, "clocks": clocks, "wall_s": round(t_wall, 3),
    }


def hessian_phase(n_graphs: int = 128, atoms: int = 24, R: int = 8, reps: int = 3):
    """Subsampled Hessian rows (Eq. sampled_hessian2) of a batch of small open
    clusters (the paper's Hessian-labelled molecules have at most 31 atoms and
    8 rows are sampled per graph): host arrays in, rows out, timed on the host
    around mlip_hessian_rows (it synchronises)."""
    from paper_2605_22698_gb300 import binding as B
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    m = B.Model(spec, w, B.MLIP_PREC_F16)
    systems = []
    for g in range(n_graphs):
        c = synth.cluster(atoms, seed=7000 + g, side=6.0)
        systems.append((c.pos, c.species, c.cell, c.pbc))
    rng = np.random.default_rng(5)
    rows = np.stack([rng.choice(atoms, size=R, replace=False) for _ in range(n_graphs)]).astype(np.int32)
    m.hessian_rows(systems, rows)  # warm-up (workspace)
    t0 = time.perf_counter()
    for _ in range(reps):
        out = m.hessian_rows(systems, rows)
    dt = (time.perf_counter() - t0) / reps
    m.close()
    n_rows = n_graphs * R * 3
    return {"graphs": n_graphs, "atoms_per_graph": atoms, "rows_per_graph": R * 3, "model": "T2 C128 L2 H64",
            "rows_per_s": round(n_rows / dt, 1), "ms_per_batch": round(1e3 * dt, 3),
            "row_length": int(out.shape[2] * 3),
            "note": "rows of length 3n (n = all atoms of the batch: each graph's part of its rows, zero elsewhere); "
                    "host arrays in and out, timed on the host"}


def run_ours(args, rank, world):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    fp32_peak = measure_fp32_peak()
    line = measure(args, rank, world, args.workload, args.steps, args.warmup, fp32_peak,
                   plain=not args.no_plain, cpu=True, fcc_cells=args.fcc_cells)
    if args.workload == "fcc108k" and args.fcc_cells == 30 and not args.no_extras:
        # the smaller periodic box of the same metric (water, l <= 2) and a bounded serving phase
        wl = measure(args, rank, world, "water3000", 20, 3, fp32_peak, plain=not args.no_plain, cpu=False)
        line["water3000"] = {k: wl[k] for k in ("value", "unit", "ms_per_step", "steps", "config", "e2e", "roofline",
                                                "kernel_share", "plain_fp32", "clocks")}
        line["serving"] = serve_phase(args, rank, world, args.serve_requests, sweep=[], alone=False,
                                      fixed_rate=args.serve_fixed_rate)
        line["hessian_rows"] = hessian_phase()
    line["fp32_peak"] = fp32_peak
    line["peaks"] = peaks()
    if rank == 0:
        print(json.dumps(line), flush=True)


def serve_requests(n_requests: int, seed: int, rate: float):
    """The serving mix: Poisson arrivals, N = floor(exp U(ln 8, ln 5000)) atoms
    in an open cube at 0.1 atoms/A^3 (d_min 0.9 A, 4 species), 70 % energy+forces,
    30 % 100-step NVE at dt 0.5 fs from Maxwell-Boltzmann velocities at 300 K."""
    import multiprocessing as mp
    reqs = synth.serving_stream(n_requests, rate_per_s=rate, seed=seed)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        systems = pool.starmap(synth.cluster, [(r.n, r.seed) for r in reqs])
    return reqs, systems


def serve_phase(args, rank, world, R, sweep, alone, fixed_rate=None):
    """The serving workload: a warm-up, every request queued at once
    (saturated throughput), then Poisson arrivals at 0.7x the saturated request
    rate (the headline p50/p99), optionally further arrival rates and single
    requests on an idle server.  Returns the measurements as a dict."""
    import torch
    from paper_2605_22698_gb300 import binding as B
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    prec = {"fp32": B.MLIP_PREC_FP32, "bf16": B.MLIP_PREC_BF16, "f16": B.MLIP_PREC_F16}[args.precision]
    model = B.Model(spec, w, prec)
    edges = (100, 1000)

    def submit(srv, r, sy):
        if r.kind == 1:
            return srv.submit(B.MLIP_REQ_NVE, sy.pos, sy.species, n_steps=r.n_steps, dt_fs=r.dt_fs,
                              temperature_K=r.temperature_K, seed=r.seed)
        return srv.submit(B.MLIP_REQ_ENERGY_FORCES, sy.pos, sy.species)

    def atom_evals(reqs):
        return sum(r.n * (r.n_steps + 1 if r.kind == 1 else 1) for r in reqs)

    # warm-up: a few requests through a throw-away server (workspace growth)
    reqs, systems = serve_requests(min(R, 16), 100 + rank, 1.0)
    srv = B.Server(model, bucket_edges=edges, resident_after=args.serve_resident_after)
    for i in [submit(srv, r, sy) for r, sy in zip(reqs, systems)]:
        srv.wait(i)
    srv.close()

    # phase 1: saturated (every request queued at once)
    reqs, systems = serve_requests(R, 4 + rank, 1.0)
    srv = B.Server(model, bucket_edges=edges, resident_after=args.serve_resident_after)
    barrier(world)
    l0 = B.mlip_launch_count()
    t0 = time.perf_counter()
    ids = [submit(srv, r, sy) for r, sy in zip(reqs, systems)]
    for i in ids:
        assert srv.wait(i)["status"] == 0
    t_sat = time.perf_counter() - t0
    barrier(world)
    t_sat = max_over_ranks(t_sat, world)
    launches = B.mlip_launch_count() - l0
    st_sat = srv.stats()
    srv.close()
    ae = atom_evals(reqs)
    sat_rps = R / t_sat

    def iter_ms(st):
        """Mean worker time per iteration, split by whether the membership changed."""
        it, ci = st["iterations"], st["changed_iterations"]
        same = (st["busy_s"] - st["changed_busy_s"]) / (it - ci) * 1e3 if it > ci else None
        chg = st["changed_busy_s"] / ci * 1e3 if ci else None
        return {"iterations": int(it), "changed": int(ci), "ms_changed": round(chg, 3) if chg else None,
                "ms_same": round(same, 3) if same else None}

    def open_loop(factor, seed, sampler=None, rate=None):
        """Poisson arrivals at factor x the saturated request rate (or at a fixed
        rate per second), submitted at their arrival times; the server's
        statistics and the served atom-steps/s."""
        lam = rate if rate else factor * sat_rps
        rq, sy_list = serve_requests(R, seed, lam)
        srv = B.Server(model, bucket_edges=edges, resident_after=args.serve_resident_after)
        if sampler:
            sampler.start()
        ids = []
        t0 = time.perf_counter()
        for r, sy in zip(rq, sy_list):
            dt = r.t_arrive - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids.append(submit(srv, r, sy))
        res = [srv.wait(i) for i in ids]
        t_run = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        clk = sampler.stop() if sampler else None
        assert all(r["status"] == 0 for r in res)
        return lam, st, atom_evals(rq) / t_run, clk

    # phase 2: open loop at 0.7x the saturated request rate (the headline latency)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    lam, st, thr2, clocks = open_loop(0.7, 5 + rank, sampler)
    # phase 3: the other arrival rates of the sweep
    sw = []
    for k, f in enumerate(sweep):
        lam_f, st_f, thr_f, _ = open_loop(f, 6 + k + rank)
        sw.append({"factor": f, "rate_per_s": round(lam_f, 2), "p50_ms": round(st_f["p50_ms"], 2),
                   "p99_ms": round(st_f["p99_ms"], 2), "throughput_atom_steps_per_s": round(thr_f, 1),
                   "mean_batch_requests": round(st_f["mean_batch_requests"], 2)})
    # phase 3b: a fixed arrival rate, independent of the saturated rate (which
    # moves with every change of the kernels), so that builds compare at the same load
    fixed = None
    if fixed_rate:
        lam_x, st_x, thr_x, _ = open_loop(0.0, 5 + rank, rate=fixed_rate)  # the headline phase's stream
        fixed = {"rate_per_s": round(lam_x, 2), "p50_ms": round(st_x["p50_ms"], 2), "p99_ms": round(st_x["p99_ms"], 2),
                 "mean_ms": round(st_x["mean_ms"], 2), "throughput_atom_steps_per_s": round(thr_x, 1),
                 "mean_batch_requests": round(st_x["mean_batch_requests"], 2),
                 "bucket_p99_ms": [round(x, 2) for x in st_x["bucket_p99_ms"]], "iterations": iter_ms(st_x)}
    # phase 4: single requests on an idle server (latency alone, against the mix's buckets)
    alone_ms = []
    if alone:
        srv = B.Server(model, bucket_edges=edges, resident_after=args.serve_resident_after)
        for n_at, kind in ((50, 0), (200, 0), (2000, 0), (200, 1)):
            sy = synth.cluster(n_at, 77 + n_at)
            r = synth.RequestSpec(0.0, n_at, kind, 77 + n_at, 100 if kind else 0)
            lat = []
            for _ in range(4):
                t0 = time.perf_counter()
                assert srv.wait(submit(srv, r, sy))["status"] == 0
                lat.append(1e3 * (time.perf_counter() - t0))
            alone_ms.append({"atoms": n_at, "kind": "nve100" if kind else "energy_forces",
                             "ms": round(float(np.median(lat[1:])), 2)})
        srv.close()
    model.close()
    return {
        "requests": R, "model": f"T{spec.T} C{spec.C} L{spec.L} H{spec.H}", "precision": args.precision,
        "mix": "70% E+F, 30% 100-step NVE at 0.5 fs; N = exp U(ln 8, ln 5000) atoms, open clusters at 0.1 /A^3",
        "saturated_atom_steps_per_s": round(world * ae / t_sat, 1), "saturated_ms_per_request": round(1e3 * t_sat / R, 4),
        # the headline p50 / p99: the fixed arrival rate (the same load whatever the kernels' speed;
        # 0.7x the saturated rate grows with every speed-up, and the saturated rate comes from batches
        # far larger than the open loop's, so that phase runs near or above capacity)
        "p50_ms": fixed["p50_ms"] if fixed else round(st["p50_ms"], 2),
        "p99_ms": fixed["p99_ms"] if fixed else round(st["p99_ms"], 2),
        "headline_phase": "fixed_rate" if fixed else "latency",
        "latency": {"rate_per_s": round(lam, 2), "load": "0.7x the saturated request rate", "p50_ms": round(st["p50_ms"], 2), "p99_ms": round(st["p99_ms"], 2),
                    "mean_ms": round(st["mean_ms"], 2), "max_ms": round(st["max_ms"], 2),
                    "throughput_atom_steps_per_s": round(thr2, 1),
                    "buckets_atoms": ["<=100", "101-1000", ">1000"],
                    "bucket_p50_ms": [round(x, 2) for x in st["bucket_p50_ms"]],
                    "bucket_p99_ms": [round(x, 2) for x in st["bucket_p99_ms"]],
                    "mean_batch_atoms": round(st["mean_batch_atoms"], 1),
                    "mean_batch_requests": round(st["mean_batch_requests"], 2),
                    "skin_steps": int(st["skin_steps"]), "skin_builds": int(st["skin_builds"]),
                    "iterations": iter_ms(st)},
        "rate_sweep": sw,
        "fixed_rate": fixed,
        "alone_ms": alone_ms,
        "saturated": {"requests_per_s": round(sat_rps, 2), "p50_ms": round(st_sat["p50_ms"], 2),
                      "p99_ms": round(st_sat["p99_ms"], 2), "busy_atom_steps_per_s": round(st_sat["atom_steps_per_s"], 1),
                      "iterations": st_sat["iterations"], "mean_batch_atoms": round(st_sat["mean_batch_atoms"], 1)},
        "e2e": {"value": round(world * ae / t_sat, 1), "unit": UNIT,
                "h2d_bytes_per_step": int(sum(sy.n * 28 for sy in systems) / R),
                "d2h_bytes_per_step": int(sum(sy.n * 24 * (3 if r.kind == 1 else 1) + 16 * (r.n_steps + 1)
                                              for r, sy in zip(reqs, systems)) / R)},
        "gpu_launches": int(launches), "clocks": clocks,
    }


def run_serve(args, rank, world):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    R = args.requests
    sv = serve_phase(args, rank, world, R, args.rate_sweep, alone=True, fixed_rate=args.serve_fixed_rate)
    line = {
        "metric": METRIC, "value": sv["saturated_atom_steps_per_s"], "unit": UNIT, "n_gpus": world, "steps": R,
        "warmup": 16, "ms_per_step": sv["saturated_ms_per_request"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16 tensor-core MLP + f32",
                                       "f16": "f16 tensor-core MLP + f32"}[args.precision],
        "data": "synthetic", "impl": "ours",
        "config": {"workload": "serve", "requests": R, "model": sv["model"],
                   "precision": args.precision, "mix": sv["mix"],
                   "step": "one request (value: atom-evaluations/s with every request queued at once)",
                   "l2": "inputs change every iteration (no flush)"},
        "p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"], "headline_phase": sv["headline_phase"],
        "latency": sv["latency"], "rate_sweep": sv["rate_sweep"], "fixed_rate": sv["fixed_rate"],
        "alone_ms": sv["alone_ms"],
        "saturated": sv["saturated"], "e2e": sv["e2e"], "gpu_launches": sv["gpu_launches"], "clocks": sv["clocks"],
        "cpu_baseline": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def _oracle_vv(spec_name, w, pos, vel, species, cell, pbc, dt, steps, threads):
    """The FP64 oracle's velocity-Verlet trajectory (pe, ke per step) of one
    replica, on `threads` host threads (0: all)."""
    import oracle
    if threads > 0:
        oracle.set_threads(threads)
    spec = synth.model_spec(spec_name)
    t0 = time.perf_counter()
    _, _, pe, ke = oracle.Model(spec, w).vv_nve(pos, vel, species, np.asarray(spec.masses), cell, pbc, dt, steps)
    return pe, ke, time.perf_counter() - t0, oracle.max_threads()


def run_md64(args, rank, world):
    """Batched MD: 64 replicas of 1667 H2O (5001 atoms) in 36.76 A periodic
    cells, different seeds, velocity Verlet at dt 0.5 fs from Maxwell-Boltzmann
    velocities at 300 K; every step evaluates all replicas as one graph.  One
    step = one MD step of all replicas (320,064 atoms).  The node tensors
    (1.5 GB per layer tensor) exceed L2, so no flush is needed.

    The timed run starts from the initial state (the warm-up run is undone).
    After the GPU work the FP64 oracle integrates replica 0 from the same
    state for the first --md-oracle-steps steps; the line reports both
    total-energy trajectories' drift and their largest gap."""
    R, nmol, side, dt = 64, 1667, 36.76, 0.5
    steps = args.steps
    # the replicas are generated by a spawned process pool before any CUDA call
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(R, os.cpu_count() or 1)) as pool:
        reps = pool.starmap(synth.water_box, [(nmol, side, 500 + 64 * rank + k) for k in range(R)])
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    masses = np.asarray(spec.masses)
    vels = [synth.maxwell_boltzmann(masses[r.species], 300.0, seed=900 + 64 * rank + k) for k, r in enumerate(reps)]
    k_or = min(args.md_oracle_steps, steps) if rank == 0 else 0
    import torch
    from paper_2605_22698_gb300 import binding as B
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda", torch.cuda.current_device())
    prec = {"fp32": B.MLIP_PREC_FP32, "bf16": B.MLIP_PREC_BF16, "f16": B.MLIP_PREC_F16}[args.precision]
    model = B.Model(spec, w, prec)
    off = np.cumsum([0] + [r.n for r in reps]).astype(np.int64)
    pos0 = np.concatenate([r.pos for r in reps])
    vel0 = np.concatenate(vels)
    sp0 = np.concatenate([r.species for r in reps])
    pos = torch.tensor(pos0, device=dev)
    vel = torch.tensor(vel0, device=dev)
    sp = torch.tensor(sp0, device=dev)
    cells = np.stack([r.cell for r in reps])
    pbc = np.stack([r.pbc for r in reps])
    n = int(off[-1])
    stream = torch.cuda.current_stream()
    skin = args.md_list == "skin"

    def run(k, p=pos, v=vel):
        if skin:  # candidates within rc + 2 A, rebuilt before every 10-step block, blocks replayed as CUDA graphs
            return model.md_nve_skin(off, p, v, sp if isinstance(p, torch.Tensor) else sp0, cells, pbc, dt, k,
                                     skin=2.0, rebuild_every=10, use_graph=True, stream=stream)
        return model.md_nve_batch(off, p, v, sp if isinstance(p, torch.Tensor) else sp0, cells, pbc, dt, k,
                                  stream=stream) + ({},)

    def reset():
        pos.copy_(torch.from_numpy(pos0))
        vel.copy_(torch.from_numpy(vel0))

    # kernel shares and the dominant kernel's launch time: a profiled run outside
    # the timed region (the MD driver runs eagerly while kernels are timed)
    run(args.warmup)
    reset()
    B.mlip_profile_select(None)
    B.mlip_profile_enable(True)
    k_prof = min(20, steps)
    run(k_prof)
    torch.cuda.synchronize()
    share_rep = B.mlip_profile_report().get("kernels", {})
    B.mlip_profile_enable(False)
    reset()
    run(args.warmup)  # graphs again, past their capture
    reset()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    barrier(world)
    l0 = B.mlip_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, _, pe, ke, rep = run(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = B.mlip_launch_count() - l0
    clocks = sampler.stop() if sampler else None
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3, world)
    etot = (pe + ke).cpu().numpy()  # [steps + 1, R]
    nat = np.diff(off).astype(np.float64)
    drift = (etot[-1] - etot[0]) / nat / (steps * dt * 1e-3)  # eV / atom / ps per replica
    # edge count at the initial state (for the algorithmic flop count)
    E_edges = 0
    for r in reps:
        rr, _, _ = B.mlip_neighbors(np.ascontiguousarray(r.pos), r.cell, r.pbc, spec.rc)
        E_edges += len(rr)
    roof = None
    share = {}
    if share_rep:
        tot_all = sum(v[1] for v in share_rep.values()) or 1.0
        for k_, v in sorted(share_rep.items(), key=lambda kv: -kv[1][1])[:8]:
            share[k_] = round(v[1] / tot_all, 4)
        kname, (nl, tot_ms) = max(share_rep.items(), key=lambda kv: kv[1][1])
        flops = algorithmic_flops(spec, E_edges, n)
        fp32_peak = measure_fp32_peak()
        peak = fp32_peak["tflops"]
        roof = {"kernel": kname, "bound": "alu", "achieved": None, "peak": peak, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "launches": nl, "avg_launch_ms": round(tot_ms / nl, 5),
                "peak_src": fp32_peak["src"] + " (of measured)",
                "timing": f"CUDA events around every launch of {k_prof} MD steps outside the timed region "
                          "(the MD driver runs without graphs while kernels are timed)"}
        if kname in flops:
            nl_step = max(1, round(nl / k_prof))
            achieved = flops[kname] / nl_step / (tot_ms / nl / 1e3) / 1e12
            roof.update({"achieved": round(achieved, 3), "frac": round(achieved / peak, 4),
                         "flops_per_launch": round(flops[kname] / nl_step)})
    # end to end: host arrays through the public call (copies of positions,
    # velocities and species in, positions, velocities and energies out)
    k_e2e = max(10, steps // 10)
    barrier(world)
    t0 = time.perf_counter()
    p_h, v_h, pe_h, _, _ = run(k_e2e, pos0, vel0)
    t_e2e = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": round(world * n * k_e2e / t_e2e, 1), "unit": UNIT,
           "h2d_bytes_per_step": int((pos0.nbytes + vel0.nbytes + sp0.nbytes) / k_e2e),
           "d2h_bytes_per_step": int((pos0.nbytes + vel0.nbytes + 2 * 8 * R * (k_e2e + 1)) / k_e2e),
           "steps": k_e2e, "note": "one call of k steps with host arrays; bytes per step = the call's copies / k"}
    model.close()
    oracle_cmp = None
    if k_or > 0:  # the oracle's replica-0 trajectory from the same state, after the GPU work
        ope, oke, o_s, o_threads = _oracle_vv("water", w, reps[0].pos, vels[0], reps[0].species, reps[0].cell,
                                              reps[0].pbc, dt, k_or, 0)
        eo = ope + oke
        eg = etot[: k_or + 1, 0]
        oracle_cmp = {
            "replica": 0, "atoms": int(nat[0]), "steps": k_or,
            "drift_eV_per_atom_ps": {"gpu": float((eg[-1] - eg[0]) / nat[0] / (k_or * dt * 1e-3)),
                                     "oracle": float((eo[-1] - eo[0]) / nat[0] / (k_or * dt * 1e-3))},
            "max_abs_dE_total_eV_per_atom": float(np.abs(eg - eo).max() / nat[0]),
            "max_abs_dE_potential_eV_per_atom": float(np.abs(pe.cpu().numpy()[: k_or + 1, 0] - ope).max() / nat[0]),
            "oracle_seconds": round(o_s, 1), "oracle_threads": o_threads}
    cpu_line = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_line = time_oracle("md64", args.cpu_seconds)
    line = {
        "metric": METRIC, "value": round(world * n * steps / t, 1), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t / steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16 tensor-core MLP + f32", "f16": "f16 tensor-core MLP + f32"}[args.precision],
        "data": "synthetic", "impl": "ours",
        "config": {"workload": "md64", "replicas": R, "atoms": n, "edges_at_start": E_edges,
                   "model": f"T{spec.T} C{spec.C} L{spec.L} H{spec.H}",
                   "precision": args.precision, "dt_fs": dt,
                   "neighbour_list": ("skin 2 A, rebuilt every 10 steps, compacted every step; 10-step blocks "
                                      "replayed as CUDA graphs" if skin else "rebuilt at every force evaluation"),
                   "l2": "working set (1.5 GB per node tensor) exceeds L2; no flush"},
        "drift_eV_per_atom_ps": {"median": float(np.median(drift)), "max_abs": float(np.abs(drift).max()),
                                 "over_steps": steps},
        "energy_fluctuation_eV_per_atom": float(np.median(etot.std(axis=0) / nat)),
        "oracle_first_steps": oracle_cmp,
        "skin_report": rep or None, "e2e": e2e, "roofline": roof, "kernel_share": share,
        "gpu_launches": int(launches), "clocks": clocks, "cpu_baseline": cpu_line,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    res = None
    t0 = time.perf_counter()
    import oracle
    spec, w, s, desc = sample_workload(args.workload)
    m = oracle.Model(spec, w)
    stress = bool(s.pbc.all())
    for _ in range(args.warmup):
        m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=stress)
    t1 = time.perf_counter()
    for _ in range(args.steps):
        m.energy_forces(s.pos, s.species, s.cell, s.pbc, stress=stress)
    dt = time.perf_counter() - t1
    value = s.n * args.steps / dt
    cpu = {"value": round(value, 2), "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
           "sample": f"{desc}; one step = one energy+force(+stress) evaluation"}
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "sample_atoms": s.n},
            "cpu_baseline": cpu,
            "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(time.perf_counter() - t0, 2)}
    print(json.dumps(line), flush=True)


def _relaunch(args_gpus: int) -> int:
    """Run this script under torch.distributed.run with one process per GPU."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args_gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 20; md64: 1000)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fcc108k", choices=["water3000", "fcc108k", "cluster64", "serve", "md64",
                                                               "water3000_mace", "fcc108k_mace",
                                                               "cluster5000_charged", "water3000_gated", "fcc108k_gated"])
    ap.add_argument("--precision", default="f16", choices=["fp32", "bf16", "f16"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 form beside the headline")
    ap.add_argument("--no-extras", action="store_true",
                    help="fcc108k: skip the water3000 and serving sub-objects of the default line")
    ap.add_argument("--requests", type=int, default=300, help="serve: requests per phase")
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="requests per phase of the serving sub-object of the default line")
    ap.add_argument("--serve-resident-after", type=int, default=0,
                    help="serving: iterations of unchanged NVE-only membership before a resident neighbour list "
                         "(0: the server's default; negative: never)")
    ap.add_argument("--serve-fixed-rate", type=float, default=41.7,
                    help="serving: one more open-loop phase at this absolute arrival rate (requests/s; 0: none)")
    ap.add_argument("--rate-sweep", type=lambda v: [float(x) for x in v.split(",") if x], default=[0.5, 0.9, 1.1],
                    help="serve: further open-loop arrival rates, as factors of the saturated rate")
    ap.add_argument("--fcc-cells", type=int, default=30,
                    help="FCC workloads: conventional cells per edge (30 = 108,000 atoms; smaller for ncu captures)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--md-oracle-steps", type=int, default=20,
                    help="md64: steps of replica 0 integrated by the FP64 oracle beside the GPU run (0: none)")
    ap.add_argument("--md-list", default="skin", choices=["skin", "fresh"],
                    help="md64: skin list rebuilt every 10 steps with graph replay, or a fresh list every step")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 1000 if (args.workload == "md64" and args.impl == "ours") else 20
    if args.gpus < 1:
        print("bench.py: --gpus must be at least 1", file=sys.stderr)
        sys.exit(2)
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        sys.exit(_relaunch(args.gpus))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world != args.gpus:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world}", file=sys.stderr)
        sys.exit(2)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.workload == "serve":
        run_serve(args, rank, world)
    elif args.workload == "md64":
        run_md64(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
