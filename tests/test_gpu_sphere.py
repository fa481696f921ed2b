"""The paper's manufactured-solution sphere benchmark (Sec. 4.1) on the GPU path.

npb_lod_run takes the benchmark's initial data (Eq. InitSolutions), its Dirichlet faces (the
exact solution) and its dense source (4 pi eps_m / h^3 at the centre, kbar^2 sinh(1/(eps r))
outside) and runs the LOD steps on the device.  The results are compared with the oracle on the
same inputs and with the LODIE rows of Table 2 and the LOD row of Table 1.
"""
import os

import numpy as np
import pytest

import npb_inputs as I

from . import sphere_case

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def npb():
    import paper_1410_2788_gb300 as m
    from paper_1410_2788_gb300 import build

    build.build()
    return m


@pytest.fixture(scope="module")
def O(oracle_lib):
    oracle_lib.set_threads(os.cpu_count() or 8)
    return oracle_lib


def _table2():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "paper_table2_lodie.txt")):
        f = line.split()
        if f and not line.startswith("#"):
            rows[float(f[0])] = (float(f[1]), float(f[2]))
    return rows


def gpu_sphere(npb, h, precision=0, scheme=2, eps_mode="midpoint", dt=None, n_steps=None, H=1.0, T=10.0):
    """The benchmark on the GPU: one ball of radius R = 1 at the centre of [-3, 3]^3 gives the
    mask (eps_m inside, eps_s and kbar = 1 outside); the charge is carried by the dense source."""
    st, exact, keep = sphere_case.build(h, H, eps_mode)
    dt = dt if dt is not None else h * h / 20.0
    n = n_steps if n_steps is not None else int(round(T / dt))
    c = npb.npb_ctx_create(0, 0)
    try:
        g = npb.npb_grid_create(c, I.born_sphere(kappa2=sphere_case.KBAR2, n=int(round(6.0 / h)) + 1, h=h,
                                                 radius=sphere_case.R, charge=0.0, eps_in=sphere_case.EPS_M,
                                                 eps_out=sphere_case.EPS_S))
        try:
            mode = npb.NPB_EPS_MIDPOINT if eps_mode == "midpoint" else npb.NPB_EPS_HARMONIC
            o = npb.make_opts(dt, 1.0, n, scheme=scheme, precision=precision, eps_mode=mode)
            u = npb.npb_lod_run(g, o, npb.NPB_LEG_SOLVENT_TAU, n, st.u0, st.rho)
        finally:
            npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(c)
    return sphere_case.errors(u, exact, keep), u


def linf_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("h", [0.5, 0.25])
@pytest.mark.parametrize("scheme", [2, 1])
def test_sphere_fp64_matches_oracle(npb, O, h, scheme):
    """FP64 GPU path = the oracle on the benchmark's inputs (midpoint eps, LODIE2 and LODIE1)."""
    _, u = gpu_sphere(npb, h, scheme=scheme)
    _, ref = sphere_case.run(h, scheme=scheme)
    assert linf_rel(u, ref) <= 1e-10


@pytest.mark.parametrize("h", [0.5, 0.25, 0.125, 0.0625])
def test_sphere_reproduces_table2(npb, h):
    """Table 2, LODIE rows: the printed relative L2 and Linf errors, to the printed three digits,
    down to h = 0.0625 (a 97^3 grid, 51,200 steps), which the CPU oracle cannot reach in a test."""
    (l2, linf), _ = gpu_sphere(npb, h)
    ref_l2, ref_linf = _table2()[h]
    assert abs(l2 - ref_l2) <= 0.006 * ref_l2, (h, l2, ref_l2)
    assert abs(linf - ref_linf) <= 0.006 * ref_linf, (h, linf, ref_linf)


@pytest.mark.parametrize("eps_mode", ["midpoint", "harmonic"])
def test_sphere_fp32_matches_oracle(npb, O, eps_mode):
    """FP32 sweeps (the one-tile-per-block kernel for midpoint eps, the interior-row TMA kernel
    for harmonic eps) against the FP64 oracle at h = 0.25, 1e-4 relative."""
    _, u = gpu_sphere(npb, 0.25, precision=1, eps_mode=eps_mode)
    st, exact, keep = sphere_case.build(0.25, 1.0, eps_mode)
    ref = st.u0.copy()
    O.lod_run(ref, st, 0.25 * 0.25 / 20.0, 0.25, int(round(10.0 / (0.25 * 0.25 / 20.0))), 2)
    assert linf_rel(u, ref) <= 1e-4


@pytest.mark.parametrize("H", [1.0, 20.0])
@pytest.mark.parametrize("h", [0.5, 0.25])
@pytest.mark.parametrize("precision", [0, 1])
def test_sphere_table1_stable_at_dt5(npb, H, h, precision):
    """Table 1, LOD row: finite up to dt = 5 with T = 1e4 dt, H = 1 and 20, h = 0.5 and 0.25."""
    (l2, linf), u = gpu_sphere(npb, h, precision=precision, dt=5.0, n_steps=10000, H=H)
    assert np.all(np.isfinite(u)) and np.isfinite(l2) and l2 < 10.0


def _table2_lodcn():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "paper_table2_lodcn.txt")):
        f = line.split()
        if f and not line.startswith("#"):
            rows[float(f[0])] = (float(f[1]), float(f[2]))
    return rows


@pytest.mark.parametrize("scheme", [4, 3])
def test_sphere_lodcn_fp64_matches_oracle(npb, O, scheme):
    """Crank-Nicolson LOD (LODCN2, LODCN1) on the GPU = the oracle, 1e-10 (h = 0.5)."""
    _, u = gpu_sphere(npb, 0.5, scheme=scheme)
    _, ref = sphere_case.run(0.5, scheme=scheme)
    assert linf_rel(u, ref) <= 1e-10


@pytest.mark.parametrize("h", [0.5, 0.25, 0.125, 0.0625])
def test_sphere_reproduces_table2_lodcn(npb, h):
    """Table 2, LODCN rows, to the printed three digits, down to h = 0.0625."""
    (l2, linf), _ = gpu_sphere(npb, h, scheme=4)
    ref_l2, ref_linf = _table2_lodcn()[h]
    assert abs(l2 - ref_l2) <= 0.006 * ref_l2, (h, l2, ref_l2)
    assert abs(linf - ref_linf) <= 0.006 * ref_linf, (h, linf, ref_linf)


# --------------------------------------------------------------------------- AOS / MAOS (Sec. 3.2, 3.3)
def _golden_cols(name):
    rows = {}
    for line in open(os.path.join(HERE, "golden", name)):
        f = line.split()
        if f and not line.startswith("#"):
            rows[float(f[0])] = [float(v) for v in f[1:]]
    return rows


# scheme -> (golden table, column pair)
ADDITIVE_ROWS = {5: ("paper_table3_aosie.txt", 0), 6: ("paper_table3_aosie.txt", 1),
                 7: ("paper_table4_aoscn.txt", 0), 8: ("paper_table4_aoscn.txt", 1),
                 9: ("paper_table5_maos.txt", 0), 10: ("paper_table5_maos.txt", 1)}


@pytest.mark.parametrize("scheme", [5, 6, 7, 8, 9, 10])
def test_sphere_additive_fp64_matches_oracle(npb, O, scheme):
    """AOSIE1/2, AOSCN1/2, MAOSIE, MAOSCN on the GPU = the oracle, 1e-10 (h = 0.5, FP64)."""
    _, u = gpu_sphere(npb, 0.5, scheme=scheme)
    _, ref = sphere_case.run(0.5, scheme=scheme)
    assert linf_rel(u, ref) <= 1e-10


@pytest.mark.parametrize("eps_mode", ["midpoint", "harmonic"])
@pytest.mark.parametrize("scheme", [5, 8, 10])
def test_sphere_additive_fp32_matches_oracle(npb, O, scheme, eps_mode):
    """FP32 additive steps (one-tile-per-block sweeps for midpoint eps, interior-row TMA sweeps on
    the extra states for harmonic eps) against the FP64 oracle at h = 0.25, 1e-4 relative."""
    _, u = gpu_sphere(npb, 0.25, precision=1, scheme=scheme, eps_mode=eps_mode)
    st, exact, keep = sphere_case.build(0.25, 1.0, eps_mode)
    ref = st.u0.copy()
    dt = 0.25 * 0.25 / 20.0
    O.lod_run(ref, st, dt, 0.25, int(round(10.0 / dt)), scheme)
    assert linf_rel(u, ref) <= 1e-4


@pytest.mark.parametrize("H", [1.0, 20.0])
@pytest.mark.parametrize("scheme", [5, 8, 9, 10])
def test_sphere_additive_table1_stable_at_dt5(npb, H, scheme):
    """Table 1, rows AOS and MAOS: finite after 1e4 steps of dt = 5 (h = 0.25, FP32)."""
    (l2, _), u = gpu_sphere(npb, 0.25, precision=1, scheme=scheme, dt=5.0, n_steps=10000, H=H)
    assert np.all(np.isfinite(u)) and np.isfinite(l2) and l2 < 10.0


@pytest.mark.parametrize("h", [0.125, 0.0625])
@pytest.mark.parametrize("scheme", [5, 6, 7, 8, 9, 10])
def test_sphere_reproduces_additive_tables(npb, h, scheme):
    """Tables 3-5 at h = 0.125 and 0.0625 (49^3 and 97^3 grids, 12,800 and 51,200 steps), FP32
    sweeps: the Crank-Nicolson columns (AOSCN1/2, MAOSCN1) to the printed three digits; the
    implicit-Euler columns (AOSIE1/2, MAOSIE1) to the printed Linf digits and within 4% in L2."""
    name, col = ADDITIVE_ROWS[scheme]
    ref_l2, ref_linf = _golden_cols(name)[h][2 * col:2 * col + 2]
    (l2, linf), _ = gpu_sphere(npb, h, precision=1, scheme=scheme)
    tol_l2 = 0.006 if scheme in (7, 8, 10) else 0.04
    assert abs(l2 - ref_l2) <= tol_l2 * ref_l2, (h, scheme, l2, ref_l2)
    assert abs(linf - ref_linf) <= 0.006 * ref_linf, (h, scheme, linf, ref_linf)
