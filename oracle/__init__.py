"""CPU oracle for the LODIE2 pseudo-transient NPB solver (arXiv 1410.2788).

TEST INFRASTRUCTURE ONLY: the slow, obviously correct FP64 reference that the
CUDA path is checked against.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline / reference leg of `bench.py` may import this package; the CUDA
library never calls it and shares no code with it.

The arithmetic lives in `npb_oracle.c` (plain C, FP64, Thomas per line); this
module builds it with gcc, holds the problem set-up glue in numpy, and combines
legs into the solvation energy:

  * `setup`     - node eps and kbar^2 maps, trilinear charges Q, Dirichlet data
                  (Sec. 2.1, Eqs. RhoEq / DebyeHuckel / BoundaryCond, Sec. 3.1)
  * `lod_leg`   - one pseudo-time integration from u = 0 (Sec. 2.2, LODIE2 of Sec. 3.1)
  * `energy`    - Eq. (deltaG3) with Richardson extrapolation Eq. (rich) (Sec. 5.3)
  * `vacuum_fft` - phi_0^FFT of Eq. (deltaG2): the vacuum Poisson problem solved directly with
                  the sine transform (Sec. 5.1); `energy_fft` - Eq. (deltaG2)

Readings where the paper is silent:
  * C = e_c^2/(k_B T) = 332.0637 / 0.592183 A (Coulomb constant over kT at 298 K);
  * the discrete source is Q_p = 4 pi C qtilde_p / h^3 (Eq. RhoEq with a trilinear delta);
  * vacuum legs use eps = eps_in everywhere, kbar = 0 and Coulomb boundary data;
  * the initial interior potential is zero (the trivial solution of Sec. 2.2).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sysconfig
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "npb_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

COULOMB_KCAL_A = 332.0637
KT_KCAL = 0.592183
C_BJERRUM = COULOMB_KCAL_A / KT_KCAL  # e_c^2/(k_B T) in A at 298 K

SOLVENT, VACUUM = 0, 1
LODIE1, LODIE2, LODCN1, LODCN2 = 1, 2, 3, 4
AOSIE1, AOSIE2, AOSCN1, AOSCN2, MAOSIE, MAOSCN = 5, 6, 7, 8, 9, 10


def build(force: bool = False) -> str:
    """Compile npb_oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.POINTER
    dp = P(ctypes.c_double)
    i = ctypes.c_int
    d = ctypes.c_double
    u8 = P(ctypes.c_uint8)
    lib.or_mask_vdw.argtypes = [i, i, i, d, dp, i, dp, dp, u8]
    lib.or_charge_spread.argtypes = [i, i, i, d, dp, i, dp, dp, dp]
    lib.or_charge_spread.restype = i
    lib.or_boundary.argtypes = [i, i, i, d, dp, i, dp, dp, d, d, d, dp]
    lib.or_eps_half_harmonic.argtypes = [i, i, i, dp, dp, dp, dp]
    lib.or_sweep.argtypes = [i, i, i, dp, dp, i, d]
    lib.or_sweep_cn.argtypes = [i, i, i, dp, dp, i, d]
    lib.or_ana3.argtypes = [d, d]
    lib.or_ana3.restype = d
    lib.or_nonlinear.argtypes = [i, i, i, dp, dp, d]
    lib.or_source.argtypes = [i, i, i, dp, dp, d]
    lib.or_lod_run.argtypes = [i, i, i, dp, dp, dp, dp, dp, dp, d, d, i, i]
    lib.or_euler_run.argtypes = [i, i, i, dp, dp, dp, dp, dp, dp, dp, d, d, i]
    lib.or_additive_run.argtypes = [i, i, i, dp, dp, dp, dp, dp, dp, dp, d, d, i, i]
    lib.or_set_threads.argtypes = [i]
    lib.or_get_threads.restype = i
    _lib = lib
    return lib


def _p(a: np.ndarray, ctype=ctypes.c_double):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def get_threads() -> int:
    return int(_load().or_get_threads())


def grid_shape(problem) -> tuple[int, int, int]:
    """numpy shape (nz, ny, nx) of a node array; index [k, j, i]."""
    nx, ny, nz = problem.n
    return (nz, ny, nx)


# ---------------------------------------------------------------- set-up (Sec. 2.1, 3.1)
def mask_vdw(problem) -> np.ndarray:
    """uint8 node map: 1 on/inside the union of atomic balls (Omega_m), else 0."""
    nx, ny, nz = problem.n
    out = np.zeros(grid_shape(problem), dtype=np.uint8)
    xyz = np.ascontiguousarray(problem.xyz, dtype=np.float64)
    rad = np.ascontiguousarray(problem.radius, dtype=np.float64)
    org = np.ascontiguousarray(problem.origin, dtype=np.float64)
    _load().or_mask_vdw(nx, ny, nz, problem.h, _p(org), problem.n_atoms, _p(xyz), _p(rad),
                        _p(out, ctypes.c_uint8))
    return out


def charge_spread(problem) -> np.ndarray:
    """Trilinear node charges qtilde (e_c), shape (nz, ny, nx)."""
    nx, ny, nz = problem.n
    out = np.zeros(grid_shape(problem))
    xyz = np.ascontiguousarray(problem.xyz, dtype=np.float64)
    q = np.ascontiguousarray(problem.q, dtype=np.float64)
    org = np.ascontiguousarray(problem.origin, dtype=np.float64)
    rc = _load().or_charge_spread(nx, ny, nz, problem.h, _p(org), problem.n_atoms, _p(xyz),
                                  _p(q), _p(out))
    if rc != 0:
        raise ValueError("an atom's charge stencil touches the boundary")
    return out


def boundary(problem, medium: int, u: np.ndarray) -> None:
    """Write Eq. (BoundaryCond) face values into u (in place)."""
    nx, ny, nz = problem.n
    if medium == SOLVENT:
        eps, kbar = problem.eps_out, math.sqrt(problem.kappa2)
    else:
        eps, kbar = problem.eps_in, 0.0
    xyz = np.ascontiguousarray(problem.xyz, dtype=np.float64)
    q = np.ascontiguousarray(problem.q, dtype=np.float64)
    org = np.ascontiguousarray(problem.origin, dtype=np.float64)
    _load().or_boundary(nx, ny, nz, problem.h, _p(org), problem.n_atoms, _p(xyz), _p(q),
                        eps, kbar, C_BJERRUM, _p(u))


def eps_half_harmonic(eps_node: np.ndarray):
    nz, ny, nx = eps_node.shape
    ex, ey, ez = (np.zeros_like(eps_node) for _ in range(3))
    _load().or_eps_half_harmonic(nx, ny, nz, _p(eps_node), _p(ex), _p(ey), _p(ez))
    return ex, ey, ez


def eps_half_midpoint(problem, medium: int):
    """eps at each half point by the location of the half point itself (Sec. 3.1 reading)."""
    nx, ny, nz = problem.n
    h = problem.h
    org = np.asarray(problem.origin)
    out = []
    for d in range(3):
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        pts = np.stack([org[0] + i * h, org[1] + j * h, org[2] + k * h], axis=-1)
        pts[..., d] += 0.5 * h
        inside = np.zeros(grid_shape(problem), dtype=bool)
        for a in range(problem.n_atoms):
            dd = ((pts - problem.xyz[a]) ** 2).sum(-1)
            inside |= dd <= problem.radius[a] ** 2
        if medium == VACUUM:
            e = np.full(grid_shape(problem), problem.eps_in)
        else:
            e = np.where(inside, problem.eps_in, problem.eps_out)
        last = [slice(None)] * 3
        last[2 - d] = -1
        e[tuple(last)] = 0.0
        out.append(np.ascontiguousarray(e))
    return tuple(out)


@dataclass
class Setup:
    in_mol: np.ndarray      # uint8 node map of Omega_m
    qt: np.ndarray          # trilinear node charges (e_c)
    rho: np.ndarray         # discrete source 4 pi C qt / h^3 (Eq. RhoEq)
    eps_node: np.ndarray
    kappa2_node: np.ndarray
    e_half: tuple           # (ex, ey, ez)
    u0: np.ndarray          # zero interior, Dirichlet faces


def setup(problem, medium: int, eps_mode: str = "harmonic") -> Setup:
    in_mol = mask_vdw(problem)
    qt = charge_spread(problem)
    rho = 4.0 * math.pi * C_BJERRUM * qt / problem.h ** 3
    if medium == SOLVENT:
        eps_node = np.where(in_mol == 1, problem.eps_in, problem.eps_out).astype(np.float64)
        kappa2_node = np.where(in_mol == 1, 0.0, problem.kappa2).astype(np.float64)
    else:
        eps_node = np.full(grid_shape(problem), float(problem.eps_in))
        kappa2_node = np.zeros(grid_shape(problem))
    if eps_mode == "harmonic":
        e_half = eps_half_harmonic(eps_node)
    elif eps_mode == "midpoint":
        e_half = eps_half_midpoint(problem, medium)
    else:
        raise ValueError(eps_mode)
    u0 = np.zeros(grid_shape(problem))
    boundary(problem, medium, u0)
    return Setup(in_mol, qt, rho, eps_node, kappa2_node, e_half, u0)


# ---------------------------------------------------------------- stages and steps
def sweep(u: np.ndarray, e_half: np.ndarray, direction: int, tau: float, h: float) -> None:
    nz, ny, nx = u.shape
    _load().or_sweep(nx, ny, nz, _p(u), _p(e_half), direction, tau / (h * h))


def sweep_cn(u: np.ndarray, e_half: np.ndarray, direction: int, tau: float, h: float) -> None:
    """Eqs. (LODCN1_2)-(LODCN1_4): the Crank-Nicolson sweep along `direction`."""
    nz, ny, nx = u.shape
    _load().or_sweep_cn(nx, ny, nz, _p(u), _p(e_half), direction, tau / (h * h))


def nonlinear(u: np.ndarray, kappa2_node: np.ndarray, tau: float) -> None:
    nz, ny, nx = u.shape
    _load().or_nonlinear(nx, ny, nz, _p(u), _p(kappa2_node), tau)


def ana3(w: float, a: float) -> float:
    return float(_load().or_ana3(w, a))


def source(u: np.ndarray, rho: np.ndarray, tau: float) -> None:
    nz, ny, nx = u.shape
    _load().or_source(nx, ny, nz, _p(u), _p(rho), tau)


def lod_run(u: np.ndarray, st: Setup, tau: float, h: float, n_steps: int,
            scheme: int = LODIE2) -> None:
    """n_steps of `scheme`: the LOD schemes of Sec. 3.1 (1-4) or the additive ones of
    Sec. 3.2 / 3.3 (AOSIE1 ... MAOSCN, 5-10)."""
    nz, ny, nx = u.shape
    ex, ey, ez = st.e_half
    if scheme >= AOSIE1:
        work = np.empty((4,) + u.shape)
        _load().or_additive_run(nx, ny, nz, _p(u), _p(work), _p(st.rho), _p(st.kappa2_node), _p(ex),
                                _p(ey), _p(ez), tau, h, n_steps, scheme)
        return
    _load().or_lod_run(nx, ny, nz, _p(u), _p(st.rho), _p(st.kappa2_node), _p(ex), _p(ey),
                       _p(ez), tau, h, n_steps, scheme)


def euler_run(u: np.ndarray, st: Setup, tau: float, h: float, n_steps: int) -> None:
    nz, ny, nx = u.shape
    work = np.empty_like(u)
    ex, ey, ez = st.e_half
    _load().or_euler_run(nx, ny, nz, _p(u), _p(work), _p(st.rho), _p(st.kappa2_node), _p(ex),
                         _p(ey), _p(ez), tau, h, n_steps)


def lod_leg(problem, medium: int, tau: float, n_steps: int, scheme: int = LODIE2,
            eps_mode: str = "harmonic", st: Setup | None = None) -> np.ndarray:
    """One pseudo-time leg from the trivial initial solution (Sec. 2.2)."""
    st = st or setup(problem, medium, eps_mode)
    u = st.u0.copy()
    lod_run(u, st, tau, problem.h, n_steps, scheme)
    return u


# ---------------------------------------------------------------- energy (Sec. 5.1, 5.3)
def delta_g(qt: np.ndarray, u_solvent: np.ndarray, u_vacuum: np.ndarray) -> float:
    """Eq. (deltaG3): 1/2 sum Q (phi_m - phi_0), phi = 0.592183 u (kcal/mol)."""
    return 0.5 * KT_KCAL * float(np.sum(qt * (u_solvent - u_vacuum)))


def energy(problem, tau: float, n_steps: int, richardson: bool = True, scheme: int = LODIE2,
           eps_mode: str = "harmonic", return_legs: bool = False):
    """LODIE2 RE+V solvation energy (kcal/mol), Eqs. (rich) and (deltaG3).

    Legs: solvent and vacuum, each at tau with n steps and (with Richardson) at
    tau/2 with 2n steps; the Richardson potential is 2 u^{tau/2} - u^{tau}.
    """
    st_s = setup(problem, SOLVENT, eps_mode)
    st_v = setup(problem, VACUUM, eps_mode)
    legs = {}
    legs["solvent_tau"] = lod_leg(problem, SOLVENT, tau, n_steps, scheme, st=st_s)
    legs["vacuum_tau"] = lod_leg(problem, VACUUM, tau, n_steps, scheme, st=st_v)
    if richardson:
        legs["solvent_half"] = lod_leg(problem, SOLVENT, 0.5 * tau, 2 * n_steps, scheme, st=st_s)
        legs["vacuum_half"] = lod_leg(problem, VACUUM, 0.5 * tau, 2 * n_steps, scheme, st=st_v)
        us = 2.0 * legs["solvent_half"] - legs["solvent_tau"]
        uv = 2.0 * legs["vacuum_half"] - legs["vacuum_tau"]
    else:
        us, uv = legs["solvent_tau"], legs["vacuum_tau"]
    dg = delta_g(st_s.qt, us, uv)
    if return_legs:
        return dg, legs, st_s
    return dg


# ---------------------------------------------------------------- FFT vacuum potential (Sec. 5.1, 5.3)
def poisson_dst(f: np.ndarray, h: float) -> np.ndarray:
    """Solve -Delta_h v = f on the interior nodes of a box with zero Dirichlet faces, Delta_h the
    central 7-point difference: the sine vectors sin(pi k i / (N+1)) diagonalise it with eigenvalue
    sum_d (2 - 2 cos(pi k_d / (N_d + 1))) / h^2, so v = DST-I^-1 (DST-I(f) / lambda) (the fast
    Poisson solver the paper names for phi_0; scipy's type-1 DST is the library step)."""
    from scipy.fft import dstn, idstn

    lam = np.zeros(f.shape)
    for axis, n in enumerate(f.shape):
        k = np.arange(1, n + 1, dtype=np.float64)
        shape = [1, 1, 1]
        shape[axis] = n
        lam = lam + ((2.0 - 2.0 * np.cos(math.pi * k / (n + 1))) / (h * h)).reshape(shape)
    return idstn(dstn(f, type=1) / lam, type=1)


def vacuum_fft(problem) -> np.ndarray:
    """phi_0^FFT of Eq. (deltaG2) as u (dimensionless): the direct solution of the vacuum Poisson
    problem eps_in Delta_h u + rho = 0 with the vacuum Dirichlet faces.  The face values move to the
    right-hand side (each interior node adds its face neighbours / h^2), leaving zero faces."""
    st = setup(problem, VACUUM)
    u = st.u0.copy()
    h = problem.h
    nb = (u[2:, 1:-1, 1:-1] + u[:-2, 1:-1, 1:-1] + u[1:-1, 2:, 1:-1] + u[1:-1, :-2, 1:-1] +
          u[1:-1, 1:-1, 2:] + u[1:-1, 1:-1, :-2])  # zero at interior neighbours of u0
    f = st.rho[1:-1, 1:-1, 1:-1] / problem.eps_in + nb / (h * h)
    u[1:-1, 1:-1, 1:-1] = poisson_dst(f, h)
    return u


def energy_fft(problem, tau: float, n_steps: int, richardson: bool = True, scheme: int = LODIE2,
               eps_mode: str = "harmonic") -> float:
    """Eq. (deltaG2): the LOD solvent potential (Richardson-combined) against phi_0^FFT."""
    st_s = setup(problem, SOLVENT, eps_mode)
    us = lod_leg(problem, SOLVENT, tau, n_steps, scheme, st=st_s)
    if richardson:
        us = 2.0 * lod_leg(problem, SOLVENT, 0.5 * tau, 2 * n_steps, scheme, st=st_s) - us
    return delta_g(st_s.qt, us, vacuum_fft(problem))


def born_closed_form(q: float, radius: float, eps_in: float, eps_out: float) -> float:
    """Born solvation energy (kcal/mol) of an ion in a dielectric sphere, kappa = 0."""
    return -0.5 * COULOMB_KCAL_A * q * q / radius * (1.0 / eps_in - 1.0 / eps_out)
