"""GB300-native LOD solver for the nonlinear Poisson-Boltzmann equation (arXiv 1410.2788).

A thin ctypes binding over the C ABI of ``include/npb.h`` (``libnpb.so``, built
in-tree by ``paper_1410_2788_gb300.build``).  Every function here only
marshals arguments; every stage of the solve runs in the library's CUDA
kernels.  There is no CPU fallback: importing works without a GPU, but the
first call raises if the library is missing or no CUDA device is present.

Problems are passed as any object with the attributes of the paper's problem
statement (Sec. 2.1): ``xyz`` (n, 3) in A, ``q`` (e_c), ``radius`` (A),
``eps_in``, ``eps_out``, ``kappa2`` (kbar^2, A^-2), ``h`` (A), ``n`` = (nx, ny,
nz) and ``origin`` (A).
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnpb.so")

NPB_OK, NPB_PENDING = 0, 1
NPB_EINVAL, NPB_ENOMEM, NPB_ECUDA, NPB_ETIMEOUT, NPB_ENOTFOUND, NPB_ESHUTDOWN = -1, -2, -3, -4, -5, -6
NPB_SOLVENT, NPB_VACUUM = 0, 1
NPB_LODIE1, NPB_LODIE2, NPB_LODCN1, NPB_LODCN2 = 1, 2, 3, 4
NPB_AOSIE1, NPB_AOSIE2, NPB_AOSCN1, NPB_AOSCN2, NPB_MAOSIE, NPB_MAOSCN = 5, 6, 7, 8, 9, 10
NPB_FP64, NPB_FP32_SWEEP = 0, 1
NPB_EPS_HARMONIC, NPB_EPS_MIDPOINT = 0, 1
NPB_LEG_SOLVENT_TAU, NPB_LEG_SOLVENT_HALF, NPB_LEG_VACUUM_TAU, NPB_LEG_VACUUM_HALF = 0, 1, 2, 3
NPB_LEG_VACUUM_FFT, NPB_LEG_RECOVERED = 4, 5  # npb_potential only
NPB_OP_SOURCE, NPB_OP_SWEEP_X, NPB_OP_SWEEP_Y, NPB_OP_SWEEP_Z, NPB_OP_NONLINEAR, NPB_OP_STEP = range(6)
NPB_EXPORT_MASK, NPB_EXPORT_QTILDE, NPB_EXPORT_U0_SOLVENT, NPB_EXPORT_U0_VACUUM = range(4)

_dp = ctypes.POINTER(ctypes.c_double)


class NpbError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"npb error {code}: {message}")
        self.code = code


class npb_problem(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("xyz", _dp), ("q", _dp), ("radius", _dp),
                ("eps_in", ctypes.c_double), ("eps_out", ctypes.c_double),
                ("kappa2", ctypes.c_double), ("h", ctypes.c_double),
                ("n", ctypes.c_int32 * 3), ("origin", ctypes.c_double * 3)]


class npb_opts(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("alpha", ctypes.c_double), ("n_steps", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("richardson", ctypes.c_int32),
                ("vacuum_recovery", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("eps_mode", ctypes.c_int32)]


class npb_result(ctypes.Structure):
    _fields_ = [("dG_kcal_mol", ctypes.c_double), ("wall_ms", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("point_steps", ctypes.c_int64),
                ("status", ctypes.c_int32), ("n", ctypes.c_int32 * 3)]


# Every symbol include/npb.h declares, with (restype, argtypes).
_V = ctypes.c_void_p
_I = ctypes.c_int
_I32 = ctypes.c_int32
_SZ = ctypes.c_size_t
SIGNATURES = {
    "npb_ctx_create": (_I, [_I, _SZ, ctypes.POINTER(_V)]),
    "npb_ctx_destroy": (None, [_V]),
    "npb_ctx_set_stream": (_I, [_V, _V]),
    "npb_ctx_profile": (_I, [_V, _I32]),
    "npb_ctx_kernel_stats": (_I, [_V, _I32, ctypes.POINTER(ctypes.c_char_p),
                                  ctypes.POINTER(ctypes.c_int64), _dp]),
    "npb_ctx_memory": (_I, [_V, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "npb_ctx_probe_wait_expiry": (_I, [_V, ctypes.c_int64]),
    "npb_grid_create": (_I, [_V, ctypes.POINTER(npb_problem), ctypes.POINTER(_V)]),
    "npb_grid_destroy": (None, [_V]),
    "npb_grid_refresh": (_I, [_V]),
    "npb_grid_footprint": (_SZ, [ctypes.POINTER(npb_problem), _I32]),
    "npb_lod_solve": (_I, [_V, ctypes.POINTER(npb_opts), _I32, ctypes.c_double]),
    "npb_energy": (_I, [_V, ctypes.POINTER(npb_opts), _dp]),
    "npb_energy_batch": (_I, [ctypes.POINTER(_V), _I32, ctypes.POINTER(npb_opts), ctypes.POINTER(ctypes.c_double)]),
    "npb_lod_run": (_I, [_V, ctypes.POINTER(npb_opts), _I32, _I32, _dp, _dp, _SZ]),
    "npb_euler_run": (_I, [_V, ctypes.POINTER(npb_opts), _I32, _I32, _dp, _SZ]),
    "npb_potential": (_I, [_V, _I32, _dp, _SZ]),
    "npb_apply": (_I, [_V, ctypes.POINTER(npb_opts), _I32, _I32, _dp, _SZ]),
    "npb_grid_export": (_I, [_V, _I32, _V, _SZ]),
    "npb_submit": (_I, [_V, ctypes.POINTER(npb_problem), ctypes.POINTER(npb_opts),
                        ctypes.POINTER(ctypes.c_uint64)]),
    "npb_poll": (_I, [_V, ctypes.c_uint64, _I32, ctypes.POINTER(npb_result)]),
    "npb_autotune": (_I, [_V, ctypes.POINTER(npb_opts), _I32, ctypes.c_char_p, _SZ]),
    "npb_sweep_time": (_I, [_V, ctypes.POINTER(npb_opts), _I32, _I32, _I32, _I32, _dp]),
    "npb_measure_fp64": (_I, [_V, _dp, _dp]),
    "npb_tune_save": (_I, [_V, ctypes.c_char_p]),
    "npb_tune_load": (_I, [_V, ctypes.c_char_p, ctypes.POINTER(_I32)]),
    "npb_tune_set": (_I, [_V, _I32, _I32, _I32, _I32, _I32, _I32, _I32]),
    "npb_tune_get": (_I, [_V, _I32, _I32, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                          ctypes.POINTER(_I32)]),
    "npb_charge_list_static": (_I, [_dp, _dp, _I32, ctypes.POINTER(_I32), ctypes.c_double, _dp, _V, _V, _V, _V,
                                    _V, _V, _V]),
    "npb_last_error": (ctypes.c_char_p, []),
    "npb_version": (ctypes.c_char_p, []),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libnpb.so (raises if it has not been built) and declare every ABI symbol."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1410_2788_gb300.build`"
                          " (the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int) -> int:
    if rc < 0:
        msg = load_library().npb_last_error()
        raise NpbError(rc, msg.decode() if msg else "")
    return rc


class _Arrays:
    """Keeps the contiguous arrays of one problem alive while a call reads them."""

    def __init__(self, p):
        self.xyz = np.ascontiguousarray(p.xyz, dtype=np.float64).reshape(-1)
        self.q = np.ascontiguousarray(p.q, dtype=np.float64)
        self.radius = np.ascontiguousarray(p.radius, dtype=np.float64)
        s = npb_problem()
        s.n_atoms = int(self.q.shape[0])
        s.xyz = self.xyz.ctypes.data_as(_dp)
        s.q = self.q.ctypes.data_as(_dp)
        s.radius = self.radius.ctypes.data_as(_dp)
        s.eps_in, s.eps_out, s.kappa2, s.h = float(p.eps_in), float(p.eps_out), float(p.kappa2), float(p.h)
        for d in range(3):
            s.n[d] = int(p.n[d])
            s.origin[d] = float(p.origin[d])
        self.struct = s


def make_opts(dt: float, alpha: float, n_steps: int, scheme: int = NPB_LODIE2, richardson: bool = True,
              vacuum_recovery: bool = True, precision: int = NPB_FP64,
              eps_mode: int = NPB_EPS_HARMONIC) -> npb_opts:
    o = npb_opts()
    o.dt, o.alpha, o.n_steps = float(dt), float(alpha), int(n_steps)
    o.scheme, o.richardson, o.vacuum_recovery = int(scheme), int(bool(richardson)), int(bool(vacuum_recovery))
    o.precision, o.eps_mode = int(precision), int(eps_mode)
    return o


# ----------------------------------------------------------------------------- the C calls
def npb_ctx_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    h = _V()
    _check(load_library().npb_ctx_create(device, hbm_budget_bytes, ctypes.byref(h)))
    return h.value


def npb_ctx_destroy(ctx: int) -> None:
    load_library().npb_ctx_destroy(ctx)


def npb_ctx_set_stream(ctx: int, stream: int | None) -> None:
    _check(load_library().npb_ctx_set_stream(ctx, stream or None))


def npb_ctx_profile(ctx: int, enable: bool) -> None:
    _check(load_library().npb_ctx_profile(ctx, int(enable)))


def npb_ctx_kernel_stats(ctx: int) -> dict:
    n = 32
    names = (ctypes.c_char_p * n)()
    launches = (ctypes.c_int64 * n)()
    ms = (ctypes.c_double * n)()
    k = _check(load_library().npb_ctx_kernel_stats(ctx, n, names, launches, ms))
    return {names[i].decode(): {"launches": int(launches[i]), "ms": float(ms[i])} for i in range(k)}


def npb_ctx_probe_wait_expiry(ctx: int, cycles: int) -> None:
    """cycles > 0: a bounded-wait probe that expires after `cycles` SM cycles runs before every TMA
    sweep launch (testing the NPB_ETIMEOUT path); 0: off."""
    _check(load_library().npb_ctx_probe_wait_expiry(ctx, int(cycles)))


def npb_ctx_memory(ctx: int) -> tuple[int, int]:
    a, b = _SZ(), _SZ()
    _check(load_library().npb_ctx_memory(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def npb_grid_create(ctx: int, problem) -> int:
    arr = _Arrays(problem)
    h = _V()
    _check(load_library().npb_grid_create(ctx, ctypes.byref(arr.struct), ctypes.byref(h)))
    return h.value


def npb_grid_destroy(grid: int) -> None:
    load_library().npb_grid_destroy(grid)


def npb_grid_refresh(grid: int) -> None:
    _check(load_library().npb_grid_refresh(grid))


def npb_grid_footprint(problem, precision: int) -> int:
    arr = _Arrays(problem)
    return int(load_library().npb_grid_footprint(ctypes.byref(arr.struct), precision))


def npb_lod_solve(grid: int, opts: npb_opts, medium: int, dt_scale: float = 1.0) -> None:
    _check(load_library().npb_lod_solve(grid, ctypes.byref(opts), medium, dt_scale))


def npb_energy(grid: int, opts: npb_opts) -> float:
    out = ctypes.c_double()
    _check(load_library().npb_energy(grid, ctypes.byref(opts), ctypes.byref(out)))
    return out.value


def npb_energy_batch(grids, opts: npb_opts) -> list:
    """RE+V energies (kcal/mol) of several grids in one batched, graph-captured solve."""
    n = len(grids)
    arr = (_V * n)(*grids)
    out = (ctypes.c_double * n)()
    _check(load_library().npb_energy_batch(arr, n, ctypes.byref(opts), out))
    return list(out)


def npb_lod_run(grid: int, opts: npb_opts, leg: int, n_steps: int, u: np.ndarray, source=None) -> np.ndarray:
    """n LOD steps of one leg from the dense FP64 state u (faces = Dirichlet data); with `source`
    (dense FP64 rho) stage S adds tau*rho instead of the molecule's charges.  Returns the new state."""
    out = np.ascontiguousarray(u, dtype=np.float64).copy()
    src = None if source is None else np.ascontiguousarray(source, dtype=np.float64)
    _check(load_library().npb_lod_run(grid, ctypes.byref(opts), leg, n_steps, out.ctypes.data_as(_dp),
                                      None if src is None else src.ctypes.data_as(_dp), out.size))
    return out


def npb_euler_run(grid: int, opts: npb_opts, leg: int, n_steps: int, u: np.ndarray) -> np.ndarray:
    """n explicit Euler steps of one leg from the dense FP64 state u (faces = Dirichlet data)."""
    out = np.ascontiguousarray(u, dtype=np.float64).copy()
    _check(load_library().npb_euler_run(grid, ctypes.byref(opts), leg, n_steps, out.ctypes.data_as(_dp), out.size))
    return out


def npb_potential(grid: int, leg: int, shape) -> np.ndarray:
    out = np.empty(tuple(shape), dtype=np.float64)
    _check(load_library().npb_potential(grid, leg, out.ctypes.data_as(_dp), out.size))
    return out


def npb_apply(grid: int, opts: npb_opts, leg: int, op: int, u: np.ndarray) -> np.ndarray:
    buf = np.ascontiguousarray(u, dtype=np.float64).copy()
    _check(load_library().npb_apply(grid, ctypes.byref(opts), leg, op, buf.ctypes.data_as(_dp), buf.size))
    return buf


def npb_grid_export(grid: int, what: int, shape) -> np.ndarray:
    dtype = np.uint8 if what == NPB_EXPORT_MASK else np.float64
    out = np.empty(tuple(shape), dtype=dtype)
    _check(load_library().npb_grid_export(grid, what, out.ctypes.data_as(_V), out.size))
    return out


def npb_submit(ctx: int, problem, opts: npb_opts) -> int:
    arr = _Arrays(problem)
    t = ctypes.c_uint64()
    _check(load_library().npb_submit(ctx, ctypes.byref(arr.struct), ctypes.byref(opts), ctypes.byref(t)))
    return t.value


def npb_poll(ctx: int, ticket: int, timeout_ms: int = -1):
    """Returns an npb_result when done, None while pending."""
    r = npb_result()
    rc = _check(load_library().npb_poll(ctx, ticket, timeout_ms, ctypes.byref(r)))
    return None if rc == NPB_PENDING else r


def npb_autotune(grid: int, opts: npb_opts, reps: int = 5) -> list:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load_library().npb_autotune(grid, ctypes.byref(opts), reps, buf, len(buf)))
    return json.loads(buf.value.decode() or "[]")


KIND_TILE, KIND_TMA, KIND_TMA_INNER, KIND_LINE = 0, 1, 2, 3


def npb_tune_save(ctx: int, path: str) -> None:
    """Write the context's pinned line-solver shapes to a JSON file."""
    _check(load_library().npb_tune_save(ctx, os.fsencode(path)))


def npb_tune_load(ctx: int, path: str) -> int:
    """Pin the shapes a JSON tuning file lists; returns how many were pinned."""
    n = _I32()
    _check(load_library().npb_tune_load(ctx, os.fsencode(path), ctypes.byref(n)))
    return n.value


def npb_measure_fp64(ctx: int) -> tuple[float, float]:
    """(FP64 fused multiply-adds per second, FP64 divisions per second) of the context's device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load_library().npb_measure_fp64(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def npb_sweep_time(grid: int, opts: npb_opts, direction: int, n_legs: int = 4, reps: int = 8,
                   rounds: int = 5) -> float:
    """Average device ms of one sweep launch along `direction` over n_legs legs, as a solve issues
    it (graph-captured back-to-back launches, CUDA events on the context stream)."""
    out = ctypes.c_double()
    _check(load_library().npb_sweep_time(grid, ctypes.byref(opts), direction, n_legs, reps, rounds,
                                         ctypes.byref(out)))
    return out.value


def npb_tune_set(ctx: int, precision: int, direction: int, n: int, kind: int, tx: int, seg: int,
                 length: int) -> None:
    """Pin the line-solver shape (kind, lines per block, segments, rows per segment) for lines of
    n nodes along `direction`."""
    _check(load_library().npb_tune_set(ctx, precision, direction, n, kind, tx, seg, length))


def npb_tune_get(ctx: int, precision: int, direction: int, n: int) -> tuple[int, int, int, int]:
    """(kind, tx, seg, len) used for lines of n nodes along `direction`."""
    k, a, b, c = _I32(), _I32(), _I32(), _I32()
    _check(load_library().npb_tune_get(ctx, precision, direction, n, ctypes.byref(k), ctypes.byref(a),
                                       ctypes.byref(b), ctypes.byref(c)))
    return k.value, a.value, b.value, c.value


NPB_STATIC_MAX_ATOMS = 20000
NPB_STATIC_MAX_LINES = 288 * 288


def npb_charge_list_static(problem, d_line_begin: int, d_line_count: int, d_ent_x: int, d_ent_qt: int,
                           d_ent_off: int, d_n_entries: int, stream: int | None = None) -> None:
    """Charge list into caller-owned device buffers (raw device pointers), with no allocation."""
    arr = _Arrays(problem)
    n = (_I32 * 3)(*[int(v) for v in problem.n])
    org = (ctypes.c_double * 3)(*[float(v) for v in problem.origin])
    _check(load_library().npb_charge_list_static(
        arr.xyz.ctypes.data_as(_dp), arr.q.ctypes.data_as(_dp), arr.struct.n_atoms, n, float(problem.h), org,
        d_line_begin, d_line_count, d_ent_x, d_ent_qt, d_ent_off, d_n_entries, stream or None))


def npb_last_error() -> str:
    return load_library().npb_last_error().decode()


def npb_version() -> str:
    return load_library().npb_version().decode()


def grid_shape(problem) -> tuple[int, int, int]:
    nx, ny, nz = problem.n
    return (nz, ny, nx)


def interior_point_steps(problem, n_steps: int, richardson: bool = True) -> int:
    """Interior nodes x steps summed over the legs of one RE+V solve."""
    nx, ny, nz = problem.n
    legs = 6 if richardson else 2  # n + 2n steps per medium with Richardson
    return (nx - 2) * (ny - 2) * (nz - 2) * n_steps * legs
