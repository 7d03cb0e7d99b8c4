"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only draws random numbers and lays out structures and weight
arrays.  It holds none of the potential's arithmetic (no harmonics, no
Clebsch-Gordan coefficients, no radial functions), so both the FP64 oracle and
the CUDA library can be fed from it without sharing any of the method.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014): state_k =
seed + k * 0x9E3779B97F4A7C15, output = mix(state_k).  Uniform doubles take
the top 53 bits; normals use Box-Muller.

Workloads (stand-ins for the paper's molecular datasets, which are not
available here; Sec. 5 "Dataset and pre-trained models" and Table
tbl:performance use SPICE2/OMOL25 and the PDB systems 1UAO/1ABT):
  cluster64   64 atoms, 4 species, uniform in a 10 A cube, d_min 0.9 A, open
  water       n H2O in a periodic cube, O-O >= 2.5 A by random sequential
              addition, O-H 0.96 A, H-O-H 104.5 deg, uniform random rotations
  fcc         FCC lattice (a = 3.6 A) with Gaussian displacements, 2 species
  cluster     N atoms at 0.1 atoms/A^3 in an open cube, d_min 0.9 A
"""
from __future__ import annotations

import math
import struct
import dataclasses
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64 stream (vectorised)."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            k = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + k * _GAMMA
            self.state = self.state + np.uint64(n) * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1)."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller (one normal per pair of uniforms)."""
        u = self.uniform(2 * n).reshape(n, 2)
        return np.sqrt(-2.0 * np.log1p(-u[:, 0])) * np.cos(2.0 * math.pi * u[:, 1])

    def integers(self, n: int, hi: int) -> np.ndarray:
        """Integers uniform in [0, hi)."""
        return np.minimum((self.uniform(n) * hi).astype(np.int64), hi - 1)


# --------------------------------------------------------------------- models
# hyper = (S species, T layers, C channels, L node l_max, Lsh edge l_max,
#          NB Bessel functions, H radial hidden width, p envelope exponent)
# dhyper = (cutoff rc in A, average neighbour count used as message scale 1/n)

@dataclass
class ModelSpec:
    S: int
    T: int
    C: int
    L: int
    H: int
    rc: float = 5.0
    avg_nb: float = 52.0
    Lsh: int = 3
    NB: int = 8
    p: int = 6
    masses: tuple = (1.008, 12.011, 14.007, 15.999)
    correlation: int = 0  # 0: no symmetric contraction; 2: MACE's of correlation order 2
    charges: int = 0      # 1: charge head + charge correction + Coulomb term (open systems)
    coulomb_r0: float = 0.0  # soft-core radius of the Coulomb term, A (charges = 1)
    gate: int = 0         # 1: species self-connection and gated update of the l > 0 features
    parity: int = 0       # 1: mixed-parity features (even and odd channel blocks, pseudotensor paths)

    @property
    def hyper(self) -> np.ndarray:
        return np.array([self.S, self.T, self.C, self.L, self.Lsh, self.NB, self.H, self.p], dtype=np.int32)

    @property
    def dhyper(self) -> np.ndarray:
        return np.array([self.rc, self.avg_nb], dtype=np.float64)

    @property
    def n_paths(self) -> int:
        """Number of (l1, l2, l3) triples with l1, l3 <= L, l2 <= Lsh, triangle
        rule and even l1 + l2 + l3 (any parity for mixed-parity models; a count,
        not part of the method's arithmetic)."""
        n = 0
        for l1 in range(self.L + 1):
            for l2 in range(self.Lsh + 1):
                for l3 in range(self.L + 1):
                    if abs(l1 - l2) <= l3 <= l1 + l2 and (self.parity or (l1 + l2 + l3) % 2 == 0):
                        n += 1
        return n

    @property
    def n_sc_paths(self) -> int:
        """Number of (l1 <= l2, l3) triples with l1, l2, l3 <= L, triangle rule
        and even l1 + l2 + l3 (a count, not part of the method's arithmetic)."""
        n = 0
        for l1 in range(self.L + 1):
            for l2 in range(l1, self.L + 1):
                for l3 in range(self.L + 1):
                    if abs(l1 - l2) <= l3 <= l1 + l2 and (l1 + l2 + l3) % 2 == 0:
                        n += 1
        return n

    def weight_shapes(self):
        """(name, shape, fan_in) in the flat parameter order."""
        P = self.n_paths
        out = [("W_emb", (self.S, self.C), self.S)]
        for t in range(self.T):
            out += [
                (f"W1.{t}", (self.NB, self.H), self.NB),
                (f"W2.{t}", (self.H, self.H), self.H),
                (f"W3.{t}", (self.H, P, self.C), self.H),
                (f"Wmix.{t}", (self.L + 1, self.C, self.C), self.C),
            ]
            if self.correlation == 2:
                Q = self.n_sc_paths
                out += [(f"Wsc1.{t}", (self.S, self.L + 1, self.C), 1),
                        (f"Wsc2.{t}", (self.S, Q, self.C), Q)]
            if self.gate:
                LC = self.L * self.C
                out += [(f"Wself.{t}", (self.S, self.L + 1, self.C, self.C), self.C),
                        (f"Wgate.{t}", (self.C, LC), self.C),
                        (f"Wselfgate.{t}", (self.S, self.C, LC), self.C)]
        out += [("W_out", (self.S, self.C), self.C), ("E0", (self.S,), 0)]
        if self.charges:
            out += [("W_q", (self.S, self.C), self.C), ("q0", (self.S,), 0)]
        return out

    def n_weights(self) -> int:
        return int(sum(int(np.prod(s)) for _, s, _ in self.weight_shapes()))


def model_spec(name: str) -> ModelSpec:
    """Model configurations of the workloads.

    small   1 layer, 16 channels, l <= 2 features, MLP 8 -> 32 -> 32 -> paths*C
    water   2 layers, 128 channels, l <= 2, hidden 64 (Table tbl:nequip_params)
    fcc     2 layers, 128 channels, l <= 3, hidden 64, 2 species
    <name>_mace  the same with the symmetric contraction of correlation order 2
                 after every scatter-sum (Table tbl:mace_params: correlation 2)
    <name>_gated  the same with the gated update and the species self-connection
    <name>_charged  the same with a charge head, the charge correction and the
                 soft-core Coulomb term (Eqs. charge_correction, long_range_interaction)
    <name>_parity  the same with mixed-parity features, the irreps of Table
                 tbl:nequip_params (0e + 0o + 1o + 1e + 2e + 2o) with C/2 channels each
    """
    if name == "small":
        return ModelSpec(S=4, T=1, C=16, L=2, H=32, avg_nb=20.0)
    if name == "water":
        return ModelSpec(S=4, T=2, C=128, L=2, H=64, avg_nb=52.0)
    if name == "fcc":
        return ModelSpec(S=2, T=2, C=128, L=3, H=64, avg_nb=42.0, masses=(63.546, 58.693))
    if name.endswith("_mace"):  # the same model with the symmetric contraction of correlation order 2
        return dataclasses.replace(model_spec(name[:-5]), correlation=2)
    if name.endswith("_gated"):  # the same model with the gated update and the species self-connection
        return dataclasses.replace(model_spec(name[:-6]), gate=1)
    if name.endswith("_parity"):  # the same model with mixed-parity features (C/2 channels of each parity)
        return dataclasses.replace(model_spec(name[:-7]), parity=1)
    if name.endswith("_charged"):  # the same model with the charge head and the Coulomb term (r0 = rc / 2)
        base = model_spec(name[:-8])
        return dataclasses.replace(base, charges=1, coulomb_r0=0.5 * base.rc)
    raise ValueError(name)


def make_weights(spec: ModelSpec, seed: int) -> np.ndarray:
    """Flat float32 parameters, each block N(0, 1/fan_in); E0 = 0."""
    rng = SplitMix64(seed)
    parts = []
    for _, shape, fan_in in spec.weight_shapes():
        n = int(np.prod(shape))
        if fan_in == 0:
            parts.append(np.zeros(n))
        else:
            parts.append(rng.normal(n) / math.sqrt(fan_in))
    return np.concatenate(parts).astype(np.float32)


def split_weights(spec: ModelSpec, w: np.ndarray) -> dict:
    out, off = {}, 0
    for name, shape, _ in spec.weight_shapes():
        n = int(np.prod(shape))
        out[name] = w[off:off + n].reshape(shape)
        off += n
    return out


PARAMS_MAGIC = b"MLIPPRM1"


def write_params(path: str, spec: ModelSpec, w: np.ndarray) -> None:
    """Parameter file: magic, u32 version, 8 x i32 hyper, (versions 2 and 3:
    i32 correlation, i32 charges, f64 coulomb_r0, i32 gate; version 3: i32
    parity), 2 x f64 (rc, avg_nb), S x f64 masses, i64 count, count x f32
    weights; little-endian.  Version 1 for models with none of the options,
    3 for mixed-parity models, else 2."""
    w = np.ascontiguousarray(w, dtype=np.float32)
    assert w.size == spec.n_weights()
    parity = getattr(spec, "parity", 0)
    v2 = bool(spec.correlation or spec.charges or spec.gate or parity)
    with open(path, "wb") as f:
        f.write(PARAMS_MAGIC)
        f.write(struct.pack("<I", 3 if parity else (2 if v2 else 1)))
        f.write(spec.hyper.astype("<i4").tobytes())
        if v2:
            f.write(struct.pack("<iidi", spec.correlation, spec.charges, spec.coulomb_r0, spec.gate))
        if parity:
            f.write(struct.pack("<i", parity))
        f.write(spec.dhyper.astype("<f8").tobytes())
        f.write(np.asarray(spec.masses, dtype="<f8").tobytes())
        f.write(struct.pack("<q", w.size))
        f.write(w.astype("<f4").tobytes())


# ----------------------------------------------------------------- structures

@dataclass
class System:
    pos: np.ndarray          # (N, 3) float64, A
    species: np.ndarray      # (N,) int32
    cell: np.ndarray         # (3, 3) float64, rows are lattice vectors
    pbc: np.ndarray          # (3,) uint8
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _rsa(rng: SplitMix64, n: int, lo: np.ndarray, span: np.ndarray, dmin: float,
         periodic: bool, max_tries: int = 2000000) -> np.ndarray:
    """Random sequential addition of n points in a box with min separation dmin
    (minimum-image distance when periodic), on a grid of bins for speed."""
    nb = np.maximum(1, np.floor(span / dmin).astype(np.int64))
    bw = span / nb
    grid: dict = {}
    pts = np.zeros((n, 3))
    k, tries = 0, 0
    batch = 256
    while k < n:
        cand = lo + rng.uniform(3 * batch).reshape(batch, 3) * span
        for c in cand:
            tries += 1
            if tries > max_tries:
                raise RuntimeError("random sequential addition did not converge")
            b = np.floor((c - lo) / bw).astype(np.int64)
            b = np.minimum(b, nb - 1)
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        q = b + (dx, dy, dz)
                        if periodic:
                            q = q % nb
                        elif np.any(q < 0) or np.any(q >= nb):
                            continue
                        for idx in grid.get(tuple(q), ()):
                            d = c - pts[idx]
                            if periodic:
                                d -= span * np.round(d / span)
                            if d @ d < dmin * dmin:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                pts[k] = c
                grid.setdefault(tuple(b), []).append(k)
                k += 1
                if k == n:
                    break
    return pts


def cluster(n: int, seed: int, density: float = 0.1, dmin: float = 0.9, n_species: int = 4,
            side: float | None = None) -> System:
    """Open cluster: n atoms uniform in a cube of side (n/density)^(1/3) (or
    `side`), rejection at dmin, species uniform in [0, n_species)."""
    rng = SplitMix64(seed)
    L = side if side is not None else (n / density) ** (1.0 / 3.0)
    pos = _rsa(rng, n, np.zeros(3), np.full(3, L), dmin, periodic=False)
    species = rng.integers(n, n_species).astype(np.int32)
    return System(pos, species, np.eye(3) * L, np.zeros(3, np.uint8), name=f"cluster{n}")


def cluster64(seed: int = 1) -> System:
    """64 atoms, 4 species, uniform in a non-periodic 10 A cube, d_min 0.9 A."""
    s = cluster(64, seed, dmin=0.9, side=10.0)
    s.name = "cluster64"
    return s


def _random_rotations(rng: SplitMix64, n: int) -> np.ndarray:
    """Uniform random rotation matrices from uniform unit quaternions (Shoemake)."""
    u = rng.uniform(3 * n).reshape(n, 3)
    a = np.sqrt(1 - u[:, 0]); b = np.sqrt(u[:, 0])
    q = np.stack([a * np.sin(2 * np.pi * u[:, 1]), a * np.cos(2 * np.pi * u[:, 1]),
                  b * np.sin(2 * np.pi * u[:, 2]), b * np.cos(2 * np.pi * u[:, 2])], axis=1)
    w, x, y, z = q[:, 3], q[:, 0], q[:, 1], q[:, 2]
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - z * w); R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w); R[:, 2, 1] = 2 * (y * z + x * w); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


H_SPECIES, O_SPECIES = 0, 3


def water_box(n_mol: int = 1000, side: float = 31.0, seed: int = 2, d_oo: float = 2.5) -> System:
    """n_mol H2O in a periodic cube: O by random sequential addition at
    O-O >= d_oo, O-H 0.96 A, H-O-H 104.5 deg, uniform random orientation.
    Atom order: O, H, H per molecule.  Species: H = 0, O = 3."""
    rng = SplitMix64(seed)
    O = _rsa(rng, n_mol, np.zeros(3), np.full(3, side), d_oo, periodic=True)
    R = _random_rotations(rng, n_mol)
    half = math.radians(104.5) / 2
    local = np.array([[0.96 * math.sin(half), 0.0, 0.96 * math.cos(half)],
                      [-0.96 * math.sin(half), 0.0, 0.96 * math.cos(half)]])
    Hs = O[:, None, :] + np.einsum("nij,kj->nki", R, local)
    pos = np.concatenate([O[:, None, :], Hs], axis=1).reshape(-1, 3)
    species = np.tile(np.array([O_SPECIES, H_SPECIES, H_SPECIES], np.int32), n_mol)
    return System(pos, species, np.eye(3) * side, np.ones(3, np.uint8), name=f"water{3 * n_mol}")


def water_side_for(n_mol: int) -> float:
    """Cube side keeping 1000 molecules per 31.0^3 A^3."""
    return 31.0 * (n_mol / 1000.0) ** (1.0 / 3.0)


def fcc(nc=(30, 30, 30), a: float = 3.6, sigma: float = 0.1, seed: int = 3) -> System:
    """FCC lattice of nc[0] x nc[1] x nc[2] conventional cells, Gaussian
    displacements of std sigma, species Bernoulli(1/2) in {0, 1}, periodic."""
    rng = SplitMix64(seed)
    nc = tuple(int(v) for v in nc)
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    g = np.stack(np.meshgrid(np.arange(nc[0]), np.arange(nc[1]), np.arange(nc[2]), indexing="ij"), -1).reshape(-1, 3)
    pos = ((g[:, None, :] + basis[None]) * a).reshape(-1, 3)
    pos = pos + sigma * rng.normal(pos.size).reshape(pos.shape)
    species = (rng.uniform(pos.shape[0]) < 0.5).astype(np.int32)
    cell = np.diag(np.array(nc, dtype=np.float64) * a)
    return System(pos, species, cell, np.ones(3, np.uint8), name=f"fcc{pos.shape[0]}")


def maxwell_boltzmann(masses: np.ndarray, temperature_K: float, seed: int) -> np.ndarray:
    """Velocities (A/fs), each component N(0, kB T kappa / m), centre-of-mass
    velocity removed.  kB = 8.617333262e-5 eV/K, kappa = 9.648533212e-3."""
    kB, kappa = 8.617333262e-5, 9.648533212e-3
    rng = SplitMix64(seed)
    m = np.asarray(masses, dtype=np.float64)
    v = rng.normal(3 * m.size).reshape(-1, 3) * np.sqrt(kB * temperature_K * kappa / m)[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    return v


# ------------------------------------------------------------ serving stream

@dataclass
class RequestSpec:
    t_arrive: float       # seconds from the start of the stream
    n: int
    kind: int             # 0 = energy+forces, 1 = NVE
    seed: int
    n_steps: int = 0
    dt_fs: float = 0.5
    temperature_K: float = 300.0


def serving_stream(n_requests: int = 2000, rate_per_s: float = 100.0, seed: int = 4,
                   n_min: int = 8, n_max: int = 5000, frac_md: float = 0.3, md_steps: int = 100):
    """Poisson arrivals; N = floor(exp(U(ln n_min, ln n_max))); 30 % NVE runs."""
    rng = SplitMix64(seed)
    gaps = -np.log1p(-rng.uniform(n_requests)) / rate_per_s
    t = np.cumsum(gaps)
    ns = np.floor(np.exp(math.log(n_min) + rng.uniform(n_requests) * (math.log(n_max) - math.log(n_min))))
    kinds = (rng.uniform(n_requests) < frac_md).astype(int)
    seeds = rng.next_u64(n_requests)
    return [RequestSpec(float(t[k]), int(ns[k]), int(kinds[k]), int(seeds[k] % (2 ** 31)),
                        md_steps if kinds[k] else 0) for k in range(n_requests)]
