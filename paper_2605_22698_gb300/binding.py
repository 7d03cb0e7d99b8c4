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
                ("avg_num_neighbors", ctypes.c_double), ("masses", ctypes.POINTER(ctypes.c_double))]


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
        L.mlip_neighbors_noalloc.argtypes = [P, i64, P, P, f64, P, P, P, i64, ctypes.POINTER(ctypes.c_int64), P]
        L.mlip_md_nve.argtypes = [P, P, P, P, i64, P, P, f64, i64, P, P, i32, P]
        L.mlip_selftest.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
        L.mlip_profile_enable.argtypes = [i32]
        L.mlip_launch_count.restype = ctypes.c_longlong
        L.mlip_profile_report.argtypes = [ctypes.c_char_p, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
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
                        m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
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


def mlip_selftest(which: int) -> float:
    r = ctypes.c_double(0.0)
    _check(lib().mlip_selftest(which, ctypes.byref(r)))
    return float(r.value)


def mlip_profile_enable(on: bool) -> None:
    _check(lib().mlip_profile_enable(1 if on else 0))


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

    def md_nve(self, pos, vel, species, cell, pbc, dt_fs, n_steps, stream=None):
        return mlip_md_nve(self.h, pos, vel, species, cell, pbc, dt_fs, n_steps, stream)

    def close(self):
        if getattr(self, "h", None):
            mlip_model_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
