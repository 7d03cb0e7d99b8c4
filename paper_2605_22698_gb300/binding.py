"""Thin ctypes binding of libmlip.so: argument marshalling only.

Every function here forwards to the C ABI of include/mlip.h with the same
name.  Host arrays are numpy; device arrays are torch CUDA tensors (their
data pointers are passed with on_device = 1).  No step of the computation runs
in Python, and nothing falls back to another implementation: if the library is
missing the import fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmlip.so")

MLIP_OK = 0
MLIP_PENDING = 1
MLIP_ERR_INVALID_ARG = -1
MLIP_ERR_CUDA = -2
MLIP_ERR_OOM = -3
MLIP_ERR_BUDGET = -4
MLIP_ERR_CAPACITY = -5
MLIP_ERR_CELL = -6
MLIP_ERR_DEGENERATE = -7
MLIP_ERR_TIMEOUT = -8
MLIP_ERR_DEVICE_TIMEOUT = -9
MLIP_ERR_NOT_FOUND = -10
MLIP_PREC_FP32 = 0
MLIP_PREC_BF16 = 1
MLIP_PREC_F16 = 2


class MlipError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mlip error {code}: {msg}")
        self.code = code


class mlip_model_desc(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int32), ("n_layers", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("l_max", ctypes.c_int32), ("sh_l_max", ctypes.c_int32), ("n_basis", ctypes.c_int32),
                ("hidden", ctypes.c_int32), ("envelope_p", ctypes.c_int32), ("cutoff", ctypes.c_double),
                ("avg_num_neighbors", ctypes.c_double), ("masses", ctypes.POINTER(ctypes.c_double)),
                ("correlation", ctypes.c_int32), ("charges", ctypes.c_int32), ("coulomb_r0", ctypes.c_double),
                ("gate", ctypes.c_int32), ("parity", ctypes.c_int32)]


class mlip_md_options(ctypes.Structure):
    _fields_ = [("skin", ctypes.c_double), ("rebuild_every", ctypes.c_int32), ("use_graph", ctypes.c_int32)]


class mlip_md_report(ctypes.Structure):
    _fields_ = [("builds", ctypes.c_int64), ("redone_blocks", ctypes.c_int64), ("graph_captures", ctypes.c_int64),
                ("graph_launches", ctypes.c_int64), ("max_candidates", ctypes.c_int64),
                ("max_displacement", ctypes.c_double)]


_lib = None


def lib():
    """Load libmlip.so (built by paper_2605_22698_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2605_22698_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.mlip_last_error.restype = ctypes.c_char_p
        L.mlip_model_num_weights.argtypes = [ctypes.POINTER(mlip_model_desc), ctypes.POINTER(ctypes.c_int64)]
        L.mlip_model_create.argtypes = [ctypes.POINTER(mlip_model_desc), P, i64, i32, ctypes.POINTER(P)]
        L.mlip_model_load.argtypes = [ctypes.c_char_p, i32, ctypes.POINTER(P)]
        L.mlip_model_free.argtypes = [P]
        L.mlip_neighbors.argtypes = [P, i64, P, P, f64, P, P, P, i64, ctypes.POINTER(ctypes.c_int64), i32, P]
        L.mlip_energy_forces.argtypes = [P, P, P, i64, P, P, P, P, P, i32, P]
        L.mlip_energy_forces_charged.argtypes = [P, P, P, i64, ctypes.c_double, P, P, P, i32, P]
        L.mlip_energy_forward.argtypes = [P, P, P, i64, P, P, P, i32, P]
        L.mlip_hessian_rows.argtypes = [P, i32, P, P, P, P, P, i32, P, P, i32, P]
        L.mlip_energy_backward.argtypes = [P, P, P, P, i32, P]
        L.mlip_energy_forces_batch.argtypes = [P, i32, P, P, P, P, P, P, P, P, i32, P]
        L.mlip_neighbors_noalloc.argtypes = [P, i64, P, P, f64, P, P, P, i64, ctypes.POINTER(ctypes.c_int64), P]
        L.mlip_md_nve.argtypes = [P, P, P, P, i64, P, P, f64, i64, P, P, i32, P]
        L.mlip_md_nve_batch.argtypes = [P, i32, P, P, P, P, P, P, f64, i64, P, P, i32, P]
        L.mlip_md_nve_skin.argtypes = [P, i32, P, P, P, P, P, P, f64, i64, ctypes.POINTER(mlip_md_options), P, P,
                                       ctypes.POINTER(mlip_md_report), i32, P]
        L.mlip_selftest.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
        L.mlip_profile_enable.argtypes = [i32]
        L.mlip_profile_select.argtypes = [ctypes.c_char_p]
        L.mlip_launch_count.restype = ctypes.c_longlong
        L.mlip_profile_report.argtypes = [ctypes.c_char_p, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
        L.mlip_fp32_fma_rate.argtypes = [i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int)]
        _lib = L
    return _lib


def exported_symbols():
    """Names of the mlip_* functions declared in include/mlip.h."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "mlip.h")
    with open(hdr) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(mlip_[a-z0-9_]+)\s*\(", text)))


def _check(rc: int):
    if rc < 0:
        raise MlipError(rc, lib().mlip_last_error().decode())
    return rc


def _ptr(a):
    """Data pointer and on-device flag of a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p), 0
    return ctypes.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0)


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def make_desc(spec, masses=None):
    m = np.ascontiguousarray(masses if masses is not None else spec.masses, dtype=np.float64)
    d = mlip_model_desc(spec.S, spec.T, spec.C, spec.L, spec.Lsh, spec.NB, spec.H, spec.p, spec.rc, spec.avg_nb,
                        m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), getattr(spec, "correlation", 0),
                        getattr(spec, "charges", 0), getattr(spec, "coulomb_r0", 0.0), getattr(spec, "gate", 0),
                        getattr(spec, "parity", 0))
    d._keep = m
    return d


def mlip_model_num_weights(desc) -> int:
    n = ctypes.c_int64(0)
    _check(lib().mlip_model_num_weights(ctypes.byref(desc), ctypes.byref(n)))
    return int(n.value)


def mlip_model_create(desc, weights: np.ndarray, precision: int = MLIP_PREC_FP32):
    w = np.ascontiguousarray(weights, dtype=np.float32)
    h = ctypes.c_void_p()
    _check(lib().mlip_model_create(ctypes.byref(desc), w.ctypes.data_as(ctypes.c_void_p), w.size, precision,
                                   ctypes.byref(h)))
    return h


def mlip_model_load(path: str, precision: int = MLIP_PREC_FP32):
    h = ctypes.c_void_p()
    _check(lib().mlip_model_load(path.encode(), precision, ctypes.byref(h)))
    return h


def mlip_model_free(h) -> None:
    if h:
        lib().mlip_model_free(h)


def mlip_neighbors(pos, cell, pbc, cutoff: float, capacity: int = 0, stream=None, out=None):
    """Host (numpy) or device (torch) positions.  Returns (recv, send, shift)
    as numpy arrays for host input, torch tensors for device input."""
    cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(3)
    n = int(pos.shape[0])
    pp, dev = _ptr(pos)
    ne = ctypes.c_int64(0)
    st = _stream_ptr(stream)
    if capacity <= 0:
        rc = lib().mlip_neighbors(pp, n, cell.ctypes.data_as(ctypes.c_void_p), pbc.ctypes.data_as(ctypes.c_void_p),
                                  cutoff, None, None, None, 0, ctypes.byref(ne), dev, st)
        if rc not in (MLIP_OK, MLIP_ERR_CAPACITY):
            _check(rc)
        capacity = int(ne.value)
    if dev:
        import torch
        recv = torch.empty(max(capacity, 1), dtype=torch.int32, device=pos.device)
        send = torch.empty_like(recv)
        shift = torch.empty((max(capacity, 1), 3), dtype=torch.int8, device=pos.device)
    else:
        recv = np.empty(max(capacity, 1), np.int32); send = np.empty_like(recv)
        shift = np.empty((max(capacity, 1), 3), np.int8)
    _check(lib().mlip_neighbors(pp, n, cell.ctypes.data_as(ctypes.c_void_p), pbc.ctypes.data_as(ctypes.c_void_p),
                                cutoff, _ptr(recv)[0], _ptr(send)[0], _ptr(shift)[0], capacity, ctypes.byref(ne),
                                dev, st))
    E = int(ne.value)
    return recv[:E], send[:E], shift[:E]


def mlip_neighbors_noalloc(pos, cell, pbc, cutoff: float, recv, send, shift, stream=None) -> int:
    """Allocation-free neighbour list into caller-provided device tensors
    (recv/send int32 [cap], shift int8 [cap, 3]); returns the edge count."""
    cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(3)
    ne = ctypes.c_int64(0)
    _check(lib().mlip_neighbors_noalloc(_ptr(pos)[0], int(pos.shape[0]), cell.ctypes.data_as(ctypes.c_void_p),
                                        pbc.ctypes.data_as(ctypes.c_void_p), cutoff, _ptr(recv)[0], _ptr(send)[0],
                                        _ptr(shift)[0], int(recv.shape[0]), ctypes.byref(ne), _stream_ptr(stream)))
    return int(ne.value)


def mlip_energy_forces(h, pos, species, cell, pbc, forces: bool = True, stress: bool = False, stream=None,
                       out=None):
    """Host call (numpy in, numpy out) or device call (torch CUDA tensors in;
    outputs are torch CUDA tensors, or the tensors given in `out`)."""
    cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(3)
    n = int(pos.shape[0])
    pp, dev = _ptr(pos)
    sp, dev2 = _ptr(species)
    if dev != dev2:
        raise ValueError("positions and species must both be host or both be device arrays")
    if dev:
        import torch
        if out is None:
            out = {"energy": torch.zeros(1, dtype=torch.float64, device=pos.device)}
            if forces:
                out["forces"] = torch.zeros((n, 3), dtype=torch.float64, device=pos.device)
            if stress:
                out["stress"] = torch.zeros((3, 3), dtype=torch.float64, device=pos.device)
    else:
        out = {"energy": np.zeros(1)}
        if forces:
            out["forces"] = np.zeros((n, 3))
        if stress:
            out["stress"] = np.zeros((3, 3))
    _check(lib().mlip_energy_forces(h, pp, sp, n, cell.ctypes.data_as(ctypes.c_void_p),
                                    pbc.ctypes.data_as(ctypes.c_void_p), _ptr(out["energy"])[0],
                                    _ptr(out["forces"])[0] if forces else None,
                                    _ptr(out["stress"])[0] if stress else None, dev, _stream_ptr(stream)))
    return out


def mlip_energy_forward(h, pos, species, cell, pbc, stream=None):
    """Energy of one system with no adjoint (host arrays in: a float; CUDA
    tensors in: a one-element float64 CUDA tensor); the model keeps what
    mlip_energy_backward needs."""
    cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(3)
    pp, dev = _ptr(pos)
    sp, dev2 = _ptr(species)
    if dev != dev2:
        raise ValueError("positions and species must both be host or both be device arrays")
    if dev:
        import torch
        e = torch.zeros(1, dtype=torch.float64, device=pos.device)
    else:
        e = np.zeros(1)
    _check(lib().mlip_energy_forward(h, pp, sp, int(pos.shape[0]), cell.ctypes.data_as(ctypes.c_void_p),
                                     pbc.ctypes.data_as(ctypes.c_void_p), _ptr(e)[0], dev, _stream_ptr(stream)))
    return e if dev else float(e[0])


def mlip_energy_backward(h, n: int, grad_energy, stress: bool = False, stream=None):
    """Gradient of g E with respect to the positions of the last forward
    (g = grad_energy: a float for host output, a one-element float64 CUDA
    tensor for device output); with stress also g times the stress."""
    if isinstance(grad_energy, (float, int)):
        g = np.array([float(grad_energy)])
        out, so = np.zeros((n, 3)), (np.zeros((3, 3)) if stress else None)
        dev = 0
    else:
        import torch
        g = grad_energy.reshape(1).to(torch.float64).contiguous()
        out = torch.zeros((n, 3), dtype=torch.float64, device=g.device)
        so = torch.zeros((3, 3), dtype=torch.float64, device=g.device) if stress else None
        dev = 1
    _check(lib().mlip_energy_backward(h, _ptr(g)[0], _ptr(out)[0], _ptr(so)[0] if stress else None, dev,
                                      _stream_ptr(stream)))
    return (out, so) if stress else out


def mlip_hessian_rows(h, systems, row_atoms, stream=None):
    """Subsampled Hessian rows of a batch: systems = [(pos, species, cell, pbc)]
    (numpy host arrays), row_atoms int [n_systems][R] (indices within each
    system).  Returns float64 [R][3][n][3], n the total atom count:
    rows[rho][a][j][b] = -dF_rho,a/dr_jb with F_rho the sum over systems of the
    force on each system's row atom rho."""
    ns = len(systems)
    off = np.zeros(ns + 1, np.int64)
    for k, (p, _, _, _) in enumerate(systems):
        off[k + 1] = off[k] + len(p)
    n = int(off[-1])
    pos = np.ascontiguousarray(np.concatenate([np.asarray(p, np.float64).reshape(-1, 3) for p, _, _, _ in systems]))
    sp = np.ascontiguousarray(np.concatenate([np.asarray(z, np.int32) for _, z, _, _ in systems]))
    cells = np.ascontiguousarray(np.stack([np.asarray(c, np.float64).reshape(9) for _, _, c, _ in systems]))
    pbc = np.ascontiguousarray(np.stack([np.asarray(b, np.uint8).reshape(3) for _, _, _, b in systems]))
    ra = np.ascontiguousarray(np.asarray(row_atoms, np.int32).reshape(ns, -1))
    R = int(ra.shape[1])
    out = np.zeros((R, 3, n, 3))
    _check(lib().mlip_hessian_rows(h, ns, off.ctypes.data_as(ctypes.c_void_p), pos.ctypes.data_as(ctypes.c_void_p),
                                   sp.ctypes.data_as(ctypes.c_void_p), cells.ctypes.data_as(ctypes.c_void_p),
                                   pbc.ctypes.data_as(ctypes.c_void_p), R, ra.ctypes.data_as(ctypes.c_void_p),
                                   out.ctypes.data_as(ctypes.c_void_p), 0, _stream_ptr(stream)))
    return out


def mlip_energy_forces_charged(h, pos, species, total_charge: float = 0.0, forces: bool = True, stream=None):
    """One open system of the given total charge with a model with charges:
    energy, forces and the corrected charges (host or device arrays, as
    mlip_energy_forces)."""
    n = int(pos.shape[0])
    pp, dev = _ptr(pos)
    sp, dev2 = _ptr(species)
    if dev != dev2:
        raise ValueError("positions and species must both be host or both be device arrays")
    if dev:
        import torch
        out = {"energy": torch.zeros(1, dtype=torch.float64, device=pos.device),
               "charges": torch.zeros(n, dtype=torch.float64, device=pos.device)}
        if forces:
            out["forces"] = torch.zeros((n, 3), dtype=torch.float64, device=pos.device)
    else:
        out = {"energy": np.zeros(1), "charges": np.zeros(n)}
        if forces:
            out["forces"] = np.zeros((n, 3))
    _check(lib().mlip_energy_forces_charged(h, pp, sp, n, float(total_charge), _ptr(out["energy"])[0],
                                            _ptr(out["forces"])[0] if forces else None, _ptr(out["charges"])[0],
                                            dev, _stream_ptr(stream)))
    return out


def mlip_energy_forces_batch(h, systems, forces: bool = True, stress: bool = False, stream=None):
    """Batch of host systems [(pos [n,3], species [n], cell [3,3], pbc [3]), ...]
    evaluated in one call.  Returns (energy [n_sys], forces list, stress [n_sys,3,3])."""
    ns = len(systems)
    off = np.zeros(ns + 1, dtype=np.int64)
    for k, (p, _, _, _) in enumerate(systems):
        off[k + 1] = off[k] + int(np.asarray(p).shape[0])
    pos = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1, 3) for p, _, _, _ in systems]))
    sp = np.ascontiguousarray(np.concatenate([np.asarray(z, dtype=np.int32).reshape(-1) for _, z, _, _ in systems]))
    cells = np.ascontiguousarray(np.stack([np.asarray(c, dtype=np.float64).reshape(9) for _, _, c, _ in systems]))
    pbcs = np.ascontiguousarray(np.stack([np.asarray(b, dtype=np.uint8).reshape(3) for _, _, _, b in systems]))
    energy = np.zeros(ns)
    F = np.zeros((int(off[-1]), 3)) if forces else None
    S = np.zeros((ns, 3, 3)) if stress else None
    _check(lib().mlip_energy_forces_batch(h, ns, off.ctypes.data_as(ctypes.c_void_p), _ptr(pos)[0], _ptr(sp)[0],
                                          cells.ctypes.data_as(ctypes.c_void_p),
                                          pbcs.ctypes.data_as(ctypes.c_void_p), _ptr(energy)[0],
                                          _ptr(F)[0] if forces else None, _ptr(S)[0] if stress else None, 0,
                                          _stream_ptr(stream)))
    Fl = [F[off[k]:off[k + 1]] for k in range(ns)] if forces else None
    return energy, Fl, S


def mlip_md_nve(h, pos, vel, species, cell, pbc, dt_fs: float, n_steps: int, stream=None):
    """Velocity-Verlet NVE.  numpy inputs: copies are integrated and returned
    with the energy traces; torch CUDA tensors: integrated in place."""
    cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(3)
    if isinstance(pos, np.ndarray):
        pos = np.array(pos, dtype=np.float64, copy=True)
        vel = np.array(vel, dtype=np.float64, copy=True)
        species = np.ascontiguousarray(species, dtype=np.int32)
        pe = np.zeros(n_steps + 1); ke = np.zeros(n_steps + 1)
    else:
        import torch
        pe = torch.zeros(n_steps + 1, dtype=torch.float64, device=pos.device)
        ke = torch.zeros_like(pe)
    pp, dev = _ptr(pos)
    _check(lib().mlip_md_nve(h, pp, _ptr(vel)[0], _ptr(species)[0], int(pos.shape[0]),
                             cell.ctypes.data_as(ctypes.c_void_p), pbc.ctypes.data_as(ctypes.c_void_p), dt_fs,
                             n_steps, _ptr(pe)[0], _ptr(ke)[0], dev, _stream_ptr(stream)))
    return pos, vel, pe, ke


def mlip_md_nve_batch(h, atom_off, pos, vel, species, cells, pbc, dt_fs: float, n_steps: int, stream=None):
    """Velocity-Verlet NVE of a batch of systems (atoms of system s are
    atom_off[s]:atom_off[s+1] of the concatenated arrays).  numpy inputs: copies
    are integrated and returned; torch CUDA tensors: integrated in place.
    Returns (pos, vel, pe [n_steps+1, n_sys], ke [n_steps+1, n_sys])."""
    off = np.ascontiguousarray(atom_off, dtype=np.int64)
    ns = len(off) - 1
    cells = np.ascontiguousarray(cells, dtype=np.float64).reshape(ns, 9)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(ns, 3)
    if isinstance(pos, np.ndarray):
        pos = np.array(pos, dtype=np.float64, copy=True)
        vel = np.array(vel, dtype=np.float64, copy=True)
        species = np.ascontiguousarray(species, dtype=np.int32)
        pe = np.zeros((n_steps + 1, ns)); ke = np.zeros((n_steps + 1, ns))
    else:
        import torch
        pe = torch.zeros((n_steps + 1, ns), dtype=torch.float64, device=pos.device)
        ke = torch.zeros_like(pe)
    pp, dev = _ptr(pos)
    _check(lib().mlip_md_nve_batch(h, ns, off.ctypes.data_as(ctypes.c_void_p), pp, _ptr(vel)[0], _ptr(species)[0],
                                   cells.ctypes.data_as(ctypes.c_void_p), pbc.ctypes.data_as(ctypes.c_void_p),
                                   dt_fs, n_steps, _ptr(pe)[0], _ptr(ke)[0], dev, _stream_ptr(stream)))
    return pos, vel, pe, ke


def mlip_md_nve_skin(h, atom_off, pos, vel, species, cells, pbc, dt_fs: float, n_steps: int, skin: float = 2.0,
                     rebuild_every: int = 10, use_graph: bool = True, stream=None):
    """mlip_md_nve_batch with a skin neighbour list rebuilt before every block
    of rebuild_every steps and compacted at every step (blocks replayed as CUDA
    graphs when use_graph).  Returns (pos, vel, pe, ke, report dict)."""
    off = np.ascontiguousarray(atom_off, dtype=np.int64)
    ns = len(off) - 1
    cells = np.ascontiguousarray(cells, dtype=np.float64).reshape(ns, 9)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(ns, 3)
    if isinstance(pos, np.ndarray):
        pos = np.array(pos, dtype=np.float64, copy=True)
        vel = np.array(vel, dtype=np.float64, copy=True)
        species = np.ascontiguousarray(species, dtype=np.int32)
        pe = np.zeros((n_steps + 1, ns)); ke = np.zeros((n_steps + 1, ns))
    else:
        import torch
        pe = torch.zeros((n_steps + 1, ns), dtype=torch.float64, device=pos.device)
        ke = torch.zeros_like(pe)
    opt = mlip_md_options(float(skin), int(rebuild_every), 1 if use_graph else 0)
    rep = mlip_md_report()
    pp, dev = _ptr(pos)
    _check(lib().mlip_md_nve_skin(h, ns, off.ctypes.data_as(ctypes.c_void_p), pp, _ptr(vel)[0], _ptr(species)[0],
                                  cells.ctypes.data_as(ctypes.c_void_p), pbc.ctypes.data_as(ctypes.c_void_p),
                                  dt_fs, n_steps, ctypes.byref(opt), _ptr(pe)[0], _ptr(ke)[0], ctypes.byref(rep),
                                  dev, _stream_ptr(stream)))
    report = {k: getattr(rep, k) for k, _ in mlip_md_report._fields_}
    return pos, vel, pe, ke, report


def mlip_selftest(which: int) -> float:
    r = ctypes.c_double(0.0)
    _check(lib().mlip_selftest(which, ctypes.byref(r)))
    return float(r.value)


def mlip_fp32_fma_rate(iters: int = 20000) -> dict:
    """Measured FP32 FMA throughput of the current device: TFLOP/s, the timed
    milliseconds and the SM count."""
    tf, ms, sms = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_int(0)
    _check(lib().mlip_fp32_fma_rate(int(iters), ctypes.byref(tf), ctypes.byref(ms), ctypes.byref(sms)))
    return {"tflops": float(tf.value), "ms": float(ms.value), "sms": int(sms.value)}


def mlip_profile_enable(on: bool) -> None:
    _check(lib().mlip_profile_enable(1 if on else 0))


def mlip_profile_select(names) -> None:
    """Time only the named kernels (an iterable of names; None: all)."""
    _check(lib().mlip_profile_select(",".join(names).encode() if names else None))


def mlip_launch_count() -> int:
    return int(lib().mlip_launch_count())


def mlip_profile_report() -> dict:
    import json
    need = ctypes.c_longlong(0)
    _check(lib().mlip_profile_report(None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(int(need.value) + 16)
    _check(lib().mlip_profile_report(buf, len(buf), ctypes.byref(need)))
    return json.loads(buf.value.decode())


class Model:
    """Owning wrapper of a model handle."""

    def __init__(self, spec, weights: np.ndarray, precision: int = MLIP_PREC_FP32):
        self.spec = spec
        self.desc = make_desc(spec)
        self.h = mlip_model_create(self.desc, weights, precision)
        self.precision = precision

    def energy_forces(self, pos, species, cell, pbc, forces=True, stress=False, stream=None, out=None):
        return mlip_energy_forces(self.h, pos, species, cell, pbc, forces, stress, stream, out)

    def energy_forward(self, pos, species, cell, pbc, stream=None):
        return mlip_energy_forward(self.h, pos, species, cell, pbc, stream)

    def energy_backward(self, n, grad_energy, stress=False, stream=None):
        return mlip_energy_backward(self.h, n, grad_energy, stress, stream)

    def hessian_rows(self, systems, row_atoms, stream=None):
        return mlip_hessian_rows(self.h, systems, row_atoms, stream)

    def energy_forces_charged(self, pos, species, total_charge=0.0, forces=True, stream=None):
        return mlip_energy_forces_charged(self.h, pos, species, total_charge, forces, stream)

    def energy_forces_batch(self, systems, forces=True, stress=False, stream=None):
        return mlip_energy_forces_batch(self.h, systems, forces, stress, stream)

    def md_nve(self, pos, vel, species, cell, pbc, dt_fs, n_steps, stream=None):
        return mlip_md_nve(self.h, pos, vel, species, cell, pbc, dt_fs, n_steps, stream)

    def md_nve_batch(self, atom_off, pos, vel, species, cells, pbc, dt_fs, n_steps, stream=None):
        return mlip_md_nve_batch(self.h, atom_off, pos, vel, species, cells, pbc, dt_fs, n_steps, stream)

    def md_nve_skin(self, atom_off, pos, vel, species, cells, pbc, dt_fs, n_steps, skin=2.0, rebuild_every=10,
                    use_graph=True, stream=None):
        return mlip_md_nve_skin(self.h, atom_off, pos, vel, species, cells, pbc, dt_fs, n_steps, skin,
                                rebuild_every, use_graph, stream)

    def close(self):
        if getattr(self, "h", None):
            mlip_model_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving
MLIP_REQ_ENERGY_FORCES = 0
MLIP_REQ_NVE = 1


class mlip_serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32), ("n_buckets", ctypes.c_int32),
                ("bucket_edges", ctypes.c_int64 * 8), ("device_poll_limit_us", ctypes.c_int64),
                ("resident_after", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class mlip_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("want_stress", ctypes.c_int32), ("n", ctypes.c_int64),
                ("pos", ctypes.c_void_p), ("species", ctypes.c_void_p), ("cell", ctypes.c_double * 9),
                ("pbc", ctypes.c_uint8 * 3), ("vel", ctypes.c_void_p), ("temperature_K", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("n_steps", ctypes.c_int64), ("dt_fs", ctypes.c_double)]


class mlip_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32), ("n", ctypes.c_int64),
                ("n_steps", ctypes.c_int64), ("energy", ctypes.c_double), ("stress", ctypes.c_double * 9),
                ("forces", ctypes.POINTER(ctypes.c_double)), ("pos", ctypes.POINTER(ctypes.c_double)),
                ("vel", ctypes.POINTER(ctypes.c_double)), ("pe", ctypes.POINTER(ctypes.c_double)),
                ("ke", ctypes.POINTER(ctypes.c_double)), ("t_arrive", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class mlip_serve_statistics(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("iterations", ctypes.c_int64), ("atom_evals", ctypes.c_int64), ("elapsed_s", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("atom_steps_per_s", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("mean_batch_atoms", ctypes.c_double), ("mean_batch_requests", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("n_buckets", ctypes.c_int32),
                ("bucket_count", ctypes.c_int64 * 9), ("bucket_p50_ms", ctypes.c_double * 9),
                ("bucket_p99_ms", ctypes.c_double * 9), ("skin_steps", ctypes.c_int64),
                ("skin_builds", ctypes.c_int64), ("changed_iterations", ctypes.c_int64),
                ("changed_busy_s", ctypes.c_double)]


def _serve_lib():
    L = lib()
    if not getattr(L, "_serve_types", False):
        P = ctypes.c_void_p
        L.mlip_serve_create.argtypes = [P, ctypes.POINTER(mlip_serve_config), ctypes.POINTER(P)]
        L.mlip_serve_submit.argtypes = [P, ctypes.POINTER(mlip_request), ctypes.POINTER(ctypes.c_uint64)]
        L.mlip_serve_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(mlip_result)]
        L.mlip_serve_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(mlip_result)]
        L.mlip_serve_release.argtypes = [P, ctypes.c_uint64]
        L.mlip_serve_stats.argtypes = [P, ctypes.POINTER(mlip_serve_statistics)]
        L.mlip_serve_destroy.argtypes = [P]
        L._serve_types = True
    return L


def mlip_serve_create(h, hbm_budget_bytes: int = 0, max_slots: int = 0, bucket_edges=(),
                      device_poll_limit_us: int = 0, resident_after: int = 0):
    c = mlip_serve_config()
    c.resident_after = int(resident_after)
    c.hbm_budget_bytes = int(hbm_budget_bytes)
    c.max_slots = int(max_slots)
    c.n_buckets = len(bucket_edges)
    for k, e in enumerate(bucket_edges):
        c.bucket_edges[k] = int(e)
    c.device_poll_limit_us = int(device_poll_limit_us)
    out = ctypes.c_void_p()
    _check(_serve_lib().mlip_serve_create(h, ctypes.byref(c), ctypes.byref(out)))
    return out


def mlip_serve_submit(srv, kind, pos, species, cell=None, pbc=(0, 0, 0), want_stress=False, vel=None,
                      temperature_K=300.0, seed=0, n_steps=0, dt_fs=0.5) -> int:
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    species = np.ascontiguousarray(species, dtype=np.int32).reshape(-1)
    q = mlip_request()
    q.kind = int(kind)
    q.want_stress = 1 if want_stress else 0
    q.n = int(pos.shape[0])
    q.pos = pos.ctypes.data
    q.species = species.ctypes.data
    cell = np.eye(3) if cell is None else np.asarray(cell, dtype=np.float64)
    for k, v in enumerate(cell.reshape(9)):
        q.cell[k] = float(v)
    for k, v in enumerate(np.asarray(pbc).reshape(3)):
        q.pbc[k] = int(v)
    if vel is not None:
        vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
        q.vel = vel.ctypes.data
    q.temperature_K = float(temperature_K)
    q.seed = int(seed)
    q.n_steps = int(n_steps)
    q.dt_fs = float(dt_fs)
    rid = ctypes.c_uint64(0)
    _check(_serve_lib().mlip_serve_submit(srv, ctypes.byref(q), ctypes.byref(rid)))
    return int(rid.value)


def _result_dict(r: mlip_result) -> dict:
    n, ns = int(r.n), int(r.n_steps)
    d = {"status": int(r.status), "kind": int(r.kind), "n": n, "n_steps": ns, "energy": float(r.energy),
         "stress": np.array(r.stress[:]).reshape(3, 3), "t_arrive": r.t_arrive, "t_admit": r.t_admit,
         "t_done": r.t_done}

    def arr(p, count, shape):
        return np.ctypeslib.as_array(p, shape=(count,)).copy().reshape(shape) if p else None
    d["forces"] = arr(r.forces, 3 * n, (n, 3))
    d["pos"] = arr(r.pos, 3 * n, (n, 3))
    d["vel"] = arr(r.vel, 3 * n, (n, 3))
    d["pe"] = arr(r.pe, ns + 1, (ns + 1,))
    d["ke"] = arr(r.ke, ns + 1, (ns + 1,))
    return d


def mlip_serve_poll(srv, rid: int):
    r = mlip_result()
    rc = _check(_serve_lib().mlip_serve_poll(srv, rid, ctypes.byref(r)))
    return None if rc == MLIP_PENDING else _result_dict(r)


def mlip_serve_wait(srv, rid: int, timeout_ms: int = -1):
    r = mlip_result()
    _check(_serve_lib().mlip_serve_wait(srv, rid, int(timeout_ms), ctypes.byref(r)))
    return _result_dict(r)


def mlip_serve_release(srv, rid: int) -> int:
    return _check(_serve_lib().mlip_serve_release(srv, rid))


def mlip_serve_stats(srv) -> dict:
    s = mlip_serve_statistics()
    _check(_serve_lib().mlip_serve_stats(srv, ctypes.byref(s)))
    d = {k: getattr(s, k) for k, _ in mlip_serve_statistics._fields_ if not k.startswith("bucket_")}
    nb = int(s.n_buckets) + 1
    d["bucket_count"] = list(s.bucket_count[:nb])
    d["bucket_p50_ms"] = list(s.bucket_p50_ms[:nb])
    d["bucket_p99_ms"] = list(s.bucket_p99_ms[:nb])
    return d


def mlip_serve_destroy(srv) -> None:
    _check(_serve_lib().mlip_serve_destroy(srv))


class Server:
    """Owning wrapper of a server handle (the model must outlive it)."""

    def __init__(self, model: "Model", **cfg):
        self.model = model
        self.h = mlip_serve_create(model.h, **cfg)

    def submit(self, kind, pos, species, **kw) -> int:
        return mlip_serve_submit(self.h, kind, pos, species, **kw)

    def poll(self, rid):
        return mlip_serve_poll(self.h, rid)

    def wait(self, rid, timeout_ms=-1):
        return mlip_serve_wait(self.h, rid, timeout_ms)

    def release(self, rid):
        return mlip_serve_release(self.h, rid)

    def stats(self):
        return mlip_serve_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            mlip_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
