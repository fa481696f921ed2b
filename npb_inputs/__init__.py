"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws numbers and places atoms; it holds none of the
solver's arithmetic (no dielectric maps, no charge spreading, no boundary
potentials, no time stepping).  Both sides of every parity test receive the
same arrays from here.

Inputs stand in for the paper's PDB proteins and MSMS surfaces (Sec. 5.1,
Tables 10-16), which are not available: molecules are confined self-avoiding
random walks with 3.8 A steps and a 3.0 A minimum separation, radii drawn
from U[1.5, 2.0] A and partial charges from U[-0.8, 0.8] e_c shifted so that
the net charge is an integer.  The size range (hundreds to twenty thousand
atoms) and the grid spacing h = 0.5 A follow Sec. 5.1 and Tables 15-16.

Random numbers come from xoshiro256** seeded through splitmix64, both written
out below from their published definitions (Blackman & Vigna), so that the
same seed gives the same molecule on every machine and numpy version.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_WALK_SRC = os.path.join(_HERE, "walk.c")
_WALK_LIB = os.path.join(_HERE, "_build", "libwalk.so")
_walk = None


def build_walk() -> str:
    """Compile walk.c (the random-walk placement) with gcc into npb_inputs/_build."""
    os.makedirs(os.path.dirname(_WALK_LIB), exist_ok=True)
    if os.path.exists(_WALK_LIB) and os.path.getmtime(_WALK_LIB) >= os.path.getmtime(_WALK_SRC):
        return _WALK_LIB
    tmp = _WALK_LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp,
                           _WALK_SRC, "-lm"])
    os.replace(tmp, _WALK_LIB)
    return _WALK_LIB


def _walk_lib():
    global _walk
    if _walk is None:
        lib = ctypes.CDLL(build_walk())
        lib.rw_place.restype = ctypes.c_int
        lib.rw_place.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.POINTER(ctypes.c_uint64), ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_long, ctypes.POINTER(ctypes.c_double)]
        _walk = lib
    return _walk

_MASK64 = (1 << 64) - 1

# Physical constants used to state the problem (not the method):
# Coulomb's constant in kcal*A/(mol*e^2) and kT at 298 K in kcal/mol (Sec. 2.1).
COULOMB_KCAL_A = 332.0637
KT_KCAL = 0.592183


def _splitmix64(state: int) -> tuple[int, int]:
    state = (state + 0x9E3779B97F4A7C15) & _MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return state, z ^ (z >> 31)


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & _MASK64


class Xoshiro256ss:
    """xoshiro256** generator; `uniform()` returns doubles in [0, 1)."""

    def __init__(self, seed: int):
        st = seed & _MASK64
        s = []
        for _ in range(4):
            st, z = _splitmix64(st)
            s.append(z)
        self.s = s

    def next_u64(self) -> int:
        s = self.s
        result = (_rotl((s[1] * 5) & _MASK64, 7) * 9) & _MASK64
        t = (s[1] << 17) & _MASK64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def below(self, n: int) -> int:
        return int(self.uniform() * n) % n


@dataclass
class Problem:
    """One molecule on one cubic grid, in the paper's problem statement (Sec. 2.1).

    xyz: (n_atoms, 3) positions in A; q: charges in e_c; radius: A.
    Node (i, j, k) sits at origin + h*(i, j, k); n = (nx, ny, nz).
    kappa2 is the modified Debye-Hueckel parameter squared in A^-2 (Eq. DebyeHuckel).
    """

    xyz: np.ndarray
    q: np.ndarray
    radius: np.ndarray
    eps_in: float
    eps_out: float
    kappa2: float
    h: float
    n: tuple[int, int, int]
    origin: tuple[float, float, float]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.xyz.shape[0])

    def interior_points(self) -> int:
        nx, ny, nz = self.n
        return (nx - 2) * (ny - 2) * (nz - 2)


def born_sphere(kappa2: float = 0.0, n: int = 33, h: float = 0.5, radius: float = 2.0,
                charge: float = 1.0, eps_in: float = 1.0, eps_out: float = 80.0) -> Problem:
    """A single charge at the centre node of a dielectric sphere (the Born ion).

    The box is centred on the charge, so the charge sits exactly on node
    ((n-1)/2, (n-1)/2, (n-1)/2).  Defaults: R = 2 A, q = +1, eps 1/80, 33^3 at h = 0.5.
    """
    if n % 2 != 1:
        raise ValueError("n must be odd so that the charge sits on a node")
    half = 0.5 * (n - 1) * h
    return Problem(
        xyz=np.zeros((1, 3)), q=np.array([charge], dtype=np.float64),
        radius=np.array([radius], dtype=np.float64), eps_in=eps_in, eps_out=eps_out,
        kappa2=kappa2, h=h, n=(n, n, n), origin=(-half, -half, -half),
        name=f"born_n{n}_h{h}_k{kappa2}")


def random_walk_positions(n_atoms: int, lo: float, hi: float, rng: Xoshiro256ss,
                          step: float = 3.8, min_sep: float = 3.0,
                          max_reject: int = 100) -> np.ndarray:
    """Confined self-avoiding random walk with branching restarts (walk.c).

    Each new atom is one `step` from the current atom in a direction uniform on
    the sphere; it is rejected if it leaves the cube [lo, hi]^3 or comes closer
    than `min_sep` to any placed atom.  After `max_reject` consecutive
    rejections the walk restarts from a uniformly chosen placed atom.  The
    generator `rng` advances exactly as many draws as the walk consumed.
    """
    pos = np.zeros((n_atoms, 3))
    state = (ctypes.c_uint64 * 4)(*rng.s)
    budget = 400 * n_atoms + 10000  # total rejections allowed before giving up
    placed = _walk_lib().rw_place(n_atoms, lo, hi, state, step, min_sep, max_reject, budget,
                                  pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    rng.s = [int(x) for x in state]
    if placed < n_atoms:
        raise RuntimeError(f"random walk jammed after {placed} of {n_atoms} atoms")
    return pos


def integer_net_charges(n_atoms: int, rng: Xoshiro256ss, qmax: float = 0.8) -> np.ndarray:
    """Charges from U[-qmax, qmax], shifted uniformly so that their sum is an integer."""
    q = np.array([rng.uniform(-qmax, qmax) for _ in range(n_atoms)])
    total = q.sum()
    q -= (total - round(total)) / n_atoms
    return q


def grid_size_for(n_atoms: int, h: float, n_min: int, n_max: int,
                  vol_per_atom: float = 64.0, margin: float = 6.0) -> int:
    """Smallest N = 32k + 1 in [n_min, n_max] whose confinement cube holds the molecule.

    The confinement cube is the grid box shrunk by `margin` A per face; it must
    offer at least `vol_per_atom` A^3 per atom (a 3 A self-avoiding walk cannot
    pack much denser).  Capped at n_max.
    """
    n = n_min
    while n <= n_max:
        side = (n - 1) * h - 2.0 * margin
        if side > 0 and side ** 3 >= vol_per_atom * n_atoms:
            return n
        n += 32
    return n_max


def random_walk_molecule(n_atoms: int, n: int, h: float = 0.5, seed: int = 0,
                         eps_in: float = 1.0, eps_out: float = 80.0, kappa2: float = 0.84,
                         margin: float = 6.0) -> Problem:
    """A seeded random-walk molecule inside an n^3 grid with spacing h (origin at 0).

    Atoms are confined to the box shrunk by `margin` A per face, so every atom,
    its radius and its 8-node charge stencil stay well inside the interior.
    """
    rng = Xoshiro256ss(seed)
    side = (n - 1) * h
    lo, hi = margin, side - margin
    if hi <= lo:
        raise ValueError("grid too small for the confinement margin")
    xyz = random_walk_positions(n_atoms, lo, hi, rng)
    radius = np.array([rng.uniform(1.5, 2.0) for _ in range(n_atoms)])
    q = integer_net_charges(n_atoms, rng)
    return Problem(xyz=xyz, q=q, radius=radius, eps_in=eps_in, eps_out=eps_out,
                   kappa2=kappa2, h=h, n=(n, n, n), origin=(0.0, 0.0, 0.0),
                   name=f"rw{n_atoms}_n{n}_s{seed:#x}", meta={"seed": seed})


# Seeds: workload c uses base 0x4E50420000 + c; molecule m of a batch uses base + m.
SEED_BASE = 0x4E50420000


def log_uniform_int(rng: Xoshiro256ss, lo: int, hi: int) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def protein_1k() -> Problem:
    """1,000-atom random-walk molecule on 129^3 at h = 0.5 A, kappa2 = 0.84 A^-2."""
    return random_walk_molecule(1000, 129, 0.5, seed=SEED_BASE + 2)


def large_20k() -> Problem:
    """20,000-atom random-walk molecule on 257^3 at h = 0.5 A."""
    return random_walk_molecule(20000, 257, 0.5, seed=SEED_BASE + 4)


def batch_molecules(count: int = 64, lo_atoms: int = 200, hi_atoms: int = 5000,
                    n_min: int = 65, n_max: int = 161, h: float = 0.5) -> list[Problem]:
    """Seeded batch: atom counts log-uniform on [lo, hi]; each grid by grid_size_for."""
    base = SEED_BASE + 3
    sizes = Xoshiro256ss(base + 10**6)
    out = []
    for m in range(count):
        na = log_uniform_int(sizes, lo_atoms, hi_atoms)
        n = grid_size_for(na, h, n_min, n_max)
        out.append(random_walk_molecule(na, n, h, seed=base + m))
    return out


def serving_stream(count: int, rate_hz: float = 50.0, lo_atoms: int = 100,
                   hi_atoms: int = 20000, seed: int = SEED_BASE + 5):
    """Poisson arrivals: yields (arrival_time_s, Problem).

    h is 0.25 or 0.5 A with equal odds; the grid is the smallest 32k+1 in
    [33, 257] holding 40 A^3 per atom, falling back to h = 0.5 A when h = 0.25 A
    cannot hold the molecule within 257^3.
    """
    rng = Xoshiro256ss(seed + 10**6)
    t = 0.0
    for m in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate_hz
        na = log_uniform_int(rng, lo_atoms, hi_atoms)
        h = 0.25 if rng.uniform() < 0.5 else 0.5
        n = grid_size_for(na, h, 33, 257)
        side = (n - 1) * h - 12.0
        if h == 0.25 and (side <= 0 or side ** 3 < 64.0 * na):
            h = 0.5
            n = grid_size_for(na, h, 33, 257)
        yield t, random_walk_molecule(na, n, h, seed=seed + m)
