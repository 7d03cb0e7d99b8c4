"""Python access to the FP64 CPU oracle (test infrastructure only).

The oracle is a plain double-precision C++ evaluation of the equivariant
interaction potential (see mlip_oracle.cpp for the definitions it writes out).
Only the tests, the smoke check and the CPU-baseline leg of the benchmark use
it; the library never imports, links or runs anything here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlip_oracle.cpp")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (OpenMP, no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
               "-o", tmp, _SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.oracle_real_sh.argtypes = [i32, P, P]
        L.oracle_real_sh_grad.argtypes = [i32, P, P]
        L.oracle_complex_sh.argtypes = [i32, P, P, P]
        L.oracle_cg_complex.argtypes = [i32] * 6
        L.oracle_cg_complex.restype = f64
        L.oracle_real_basis_U.argtypes = [i32, P, P]
        L.oracle_real_cg.argtypes = [i32, i32, i32, P]
        L.oracle_paths.argtypes = [i32, i32, P]
        L.oracle_paths_all.argtypes = [i32, i32, P]
        L.oracle_node_features.argtypes = [P, P, P, i64, P, P, i32, P]
        L.oracle_bessel.argtypes = [i32, f64, f64]
        L.oracle_bessel.restype = f64
        L.oracle_envelope.argtypes = [f64, i32]
        L.oracle_envelope.restype = f64
        L.oracle_num_weights.argtypes = [P]
        L.oracle_num_weights.restype = i64
        L.oracle_model_create.argtypes = [P, P, P]
        L.oracle_model_create.restype = P
        L.oracle_model_free.argtypes = [P]
        L.oracle_neighbors.argtypes = [P, i64, P, P, f64, P, P, P, i64]
        L.oracle_neighbors.restype = i64
        L.oracle_energy_forces.argtypes = [P, P, P, i64, P, P, P, P, P, P]
        L.oracle_energy.argtypes = [P, P, P, i64, P, P, P, P]
        L.oracle_energy_dual.argtypes = [P, P, P, i64, P, P, i64, i32, P, P]
        L.oracle_tp.argtypes = [i32, i32, i32, P, P, P, P]
        L.oracle_sc_paths.argtypes = [i32, P]
        L.oracle_model_set_total_charge.argtypes = [P, f64]
        L.oracle_charges.argtypes = [P, P, P, i64, P]
        L.oracle_coulomb.argtypes = [P, P, i64, f64, P, P, P]
        L.oracle_inv_chi.argtypes = [f64, f64]
        L.oracle_hessian_row.argtypes = [P, P, P, i64, P, P, i64, i32, P]
        L.oracle_inv_chi.restype = f64
        L.oracle_sym_contract.argtypes = [i32, i32, P, P, P, P]
        L.oracle_sym_contract_adjoint.argtypes = [i32, i32, P, P, P, P, P]
        L.oracle_vv_nve.argtypes = [P, P, P, P, P, i64, P, P, f64, i64, P, P]
        L.oracle_set_threads.argtypes = [i32]
        L.oracle_max_threads.restype = i32
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def real_sh(lmax: int, v) -> np.ndarray:
    v = _c(v, np.float64)
    out = np.zeros((lmax + 1) ** 2)
    assert lib().oracle_real_sh(lmax, _p(v), _p(out)) == 0
    return out


def real_sh_grad(lmax: int, v) -> np.ndarray:
    v = _c(v, np.float64)
    out = np.zeros(((lmax + 1) ** 2, 3))
    assert lib().oracle_real_sh_grad(lmax, _p(v), _p(out)) == 0
    return out


def complex_sh(l: int, v) -> np.ndarray:
    v = _c(v, np.float64)
    re = np.zeros(2 * l + 1); im = np.zeros(2 * l + 1)
    lib().oracle_complex_sh(l, _p(v), _p(re), _p(im))
    return re + 1j * im


def cg_complex(l1, m1, l2, m2, l3, m3) -> float:
    return float(lib().oracle_cg_complex(l1, m1, l2, m2, l3, m3))


def real_basis_U(l: int) -> np.ndarray:
    n = 2 * l + 1
    re = np.zeros(n * n); im = np.zeros(n * n)
    lib().oracle_real_basis_U(l, _p(re), _p(im))
    return (re + 1j * im).reshape(n, n)


def real_cg(l1: int, l2: int, l3: int) -> np.ndarray:
    out = np.zeros((2 * l3 + 1) * (2 * l1 + 1) * (2 * l2 + 1))
    assert lib().oracle_real_cg(l1, l2, l3, _p(out)) == 0
    return out.reshape(2 * l3 + 1, 2 * l1 + 1, 2 * l2 + 1)


def paths(L: int, Lsh: int = 3, all_parities: bool = False) -> list:
    """Coupling paths (l1, l2, l3): natural parity, or every triangle-valid
    triple (the mixed-parity model's paths)."""
    f = lib().oracle_paths_all if all_parities else lib().oracle_paths
    n = f(L, Lsh, None)
    out = np.zeros(3 * n, dtype=np.int32)
    f(L, Lsh, _p(out))
    return [tuple(int(x) for x in out[3 * k:3 * k + 3]) for k in range(n)]


def bessel(n: int, r: float, rc: float) -> float:
    return float(lib().oracle_bessel(n, r, rc))


def envelope(x: float, p: int = 6) -> float:
    return float(lib().oracle_envelope(x, p))


def tp(L: int, Lsh: int, h: np.ndarray, v, w: np.ndarray) -> np.ndarray:
    """Feature-level tensor product for one edge; h [(L+1)^2, C], w [P, C]."""
    h = _c(h, np.float64); w = _c(w, np.float64); v = _c(v, np.float64)
    C = h.shape[1]
    out = np.zeros_like(h)
    lib().oracle_tp(L, Lsh, C, _p(h), _p(v), _p(w), _p(out))
    return out


def sc_paths(L: int) -> list:
    """Couplings (l1 <= l2, l3) of the symmetric contraction of order 2."""
    n = lib().oracle_sc_paths(L, None)
    out = np.zeros(3 * n, dtype=np.int32)
    lib().oracle_sc_paths(L, _p(out))
    return [tuple(int(x) for x in out[3 * k:3 * k + 3]) for k in range(n)]


def sym_contract(L: int, A: np.ndarray, w1: np.ndarray, w2: np.ndarray) -> np.ndarray:
    """Symmetric contraction of one node; A [(L+1)^2, C], w1 [L+1, C], w2 [Q, C]."""
    A = _c(A, np.float64); w1 = _c(w1, np.float64); w2 = _c(w2, np.float64)
    out = np.zeros_like(A)
    lib().oracle_sym_contract(L, A.shape[1], _p(A), _p(w1), _p(w2), _p(out))
    return out


def sym_contract_adjoint(L: int, A, w1, w2, GB) -> np.ndarray:
    A = _c(A, np.float64); w1 = _c(w1, np.float64); w2 = _c(w2, np.float64); GB = _c(GB, np.float64)
    out = np.zeros_like(A)
    lib().oracle_sym_contract_adjoint(L, A.shape[1], _p(A), _p(w1), _p(w2), _p(GB), _p(out))
    return out


def inv_chi(r: float, r0: float) -> float:
    """Soft-core pair function 1/chi(r) of the Coulomb term."""
    return float(lib().oracle_inv_chi(r, r0))


def coulomb(pos, qt, r0: float):
    """The Coulomb term alone: (E, dE/dqt [n], forces [n, 3]) for corrected charges qt."""
    pos = _c(pos, np.float64); qt = _c(qt, np.float64)
    n = pos.shape[0]
    E = np.zeros(1); g = np.zeros(n); F = np.zeros((n, 3))
    lib().oracle_coulomb(_p(pos), _p(qt), n, r0, _p(E), _p(g), _p(F))
    return float(E[0]), g, F


def neighbors(pos, cell, pbc, rc: float):
    """Brute-force neighbour list sorted by (recv, send, shift)."""
    pos = _c(pos, np.float64); cell = _c(cell, np.float64); pbc = _c(pbc, np.uint8)
    n = pos.shape[0]
    cap = 0
    e = lib().oracle_neighbors(_p(pos), n, _p(cell), _p(pbc), rc, None, None, None, 0)
    if e < 0:
        raise ValueError("singular cell")
    recv = np.zeros(max(e, 1), np.int32); send = np.zeros(max(e, 1), np.int32)
    shift = np.zeros((max(e, 1), 3), np.int32)
    cap = e
    e2 = lib().oracle_neighbors(_p(pos), n, _p(cell), _p(pbc), rc, _p(recv), _p(send), _p(shift), cap)
    assert e2 == e
    return recv[:e], send[:e], shift[:e]


class Model:
    """Oracle model built from the flat float32 weights of synth.make_weights."""

    def __init__(self, spec, weights: np.ndarray):
        self.spec = spec
        self._hyper = _c(np.append(spec.hyper, [getattr(spec, "correlation", 0), getattr(spec, "charges", 0),
                                                getattr(spec, "gate", 0), getattr(spec, "parity", 0)]), np.int32)
        self._dhyper = _c(np.append(spec.dhyper, getattr(spec, "coulomb_r0", 0.0)), np.float64)
        nw = lib().oracle_num_weights(_p(self._hyper))
        w = _c(weights, np.float32)
        if w.size != nw:
            raise ValueError(f"expected {nw} weights, got {w.size}")
        self._w = w
        self._h = lib().oracle_model_create(_p(self._hyper), _p(self._dhyper), _p(w))
        if not self._h:
            raise ValueError("unsupported model options")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_model_free(h)
            self._h = None

    def set_total_charge(self, Q: float) -> None:
        """Total charge of the systems evaluated next (models with the charge head)."""
        lib().oracle_model_set_total_charge(self._h, float(Q))

    def charges(self, pos, species) -> np.ndarray:
        """Corrected charges of an open system."""
        pos = _c(pos, np.float64); species = _c(species, np.int32)
        q = np.zeros(pos.shape[0])
        if lib().oracle_charges(self._h, _p(pos), _p(species), pos.shape[0], _p(q)) != 0:
            raise ValueError("oracle_charges failed")
        return q

    def energy_forces(self, pos, species, cell, pbc, stress: bool = False, atom_energies: bool = False):
        pos = _c(pos, np.float64); species = _c(species, np.int32)
        cell = _c(cell, np.float64); pbc = _c(pbc, np.uint8)
        n = pos.shape[0]
        E = np.zeros(1); F = np.zeros((n, 3))
        S = np.zeros((3, 3)) if stress else None
        A = np.zeros(n) if atom_energies else None
        rc = lib().oracle_energy_forces(self._h, _p(pos), _p(species), n, _p(cell), _p(pbc), _p(E), _p(F),
                                        _p(S) if stress else None, _p(A) if atom_energies else None)
        if rc != 0:
            raise ValueError(f"oracle_energy_forces failed: {rc}")
        out = {"energy": float(E[0]), "forces": F}
        if stress:
            out["stress"] = S
        if atom_energies:
            out["atom_energies"] = A
        return out

    def energy(self, pos, species, cell, pbc, atom_energies: bool = False):
        pos = _c(pos, np.float64); species = _c(species, np.int32)
        cell = _c(cell, np.float64); pbc = _c(pbc, np.uint8)
        n = pos.shape[0]
        E = np.zeros(1)
        A = np.zeros(n) if atom_energies else None
        rc = lib().oracle_energy(self._h, _p(pos), _p(species), n, _p(cell), _p(pbc), _p(E),
                                 _p(A) if atom_energies else None)
        if rc != 0:
            raise ValueError(f"oracle_energy failed: {rc}")
        return (float(E[0]), A) if atom_energies else float(E[0])

    def energy_dual(self, pos, species, cell, pbc, atom: int, axis: int):
        pos = _c(pos, np.float64); species = _c(species, np.int32)
        cell = _c(cell, np.float64); pbc = _c(pbc, np.uint8)
        E = np.zeros(1); dE = np.zeros(1)
        rc = lib().oracle_energy_dual(self._h, _p(pos), _p(species), pos.shape[0], _p(cell), _p(pbc),
                                      atom, axis, _p(E), _p(dE))
        if rc != 0:
            raise ValueError("oracle_energy_dual failed")
        return float(E[0]), float(dE[0])

    def node_features(self, pos, species, cell, pbc, layer: int) -> np.ndarray:
        """Node features after `layer` interaction layers, [n][(L+1)^2][C]."""
        pos = _c(pos, np.float64)
        n = pos.shape[0]
        D = (self.spec.L + 1) ** 2
        out = np.zeros((n, D, self.spec.C))
        rc = lib().oracle_node_features(self._h, _p(pos), _p(_c(species, np.int32)), n, _p(_c(cell, np.float64)),
                                        _p(_c(pbc, np.uint8)), int(layer), _p(out))
        if rc != 0:
            raise ValueError("oracle_node_features failed")
        return out

    def hessian_row(self, pos, species, cell, pbc, atom: int, axis: int) -> np.ndarray:
        """d2E / dr_{atom,axis} dr_{j,b} for every atom j and axis b: [n, 3]."""
        pos = _c(pos, np.float64); species = _c(species, np.int32)
        cell = _c(cell, np.float64); pbc = _c(pbc, np.uint8)
        out = np.zeros((pos.shape[0], 3))
        rc = lib().oracle_hessian_row(self._h, _p(pos), _p(species), pos.shape[0], _p(cell), _p(pbc), atom, axis,
                                      _p(out))
        if rc != 0:
            raise ValueError("oracle_hessian_row failed")
        return out

    def vv_nve(self, pos, vel, species, masses, cell, pbc, dt: float, n_steps: int):
        pos = np.array(pos, dtype=np.float64, copy=True); vel = np.array(vel, dtype=np.float64, copy=True)
        species = _c(species, np.int32); masses = _c(masses, np.float64)
        cell = _c(cell, np.float64); pbc = _c(pbc, np.uint8)
        pe = np.zeros(n_steps + 1); ke = np.zeros(n_steps + 1)
        rc = lib().oracle_vv_nve(self._h, _p(pos), _p(vel), _p(species), _p(masses), pos.shape[0], _p(cell),
                                 _p(pbc), dt, n_steps, _p(pe), _p(ke))
        if rc != 0:
            raise ValueError("oracle_vv_nve failed")
        return pos, vel, pe, ke
