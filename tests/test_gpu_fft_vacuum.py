"""phi_0^FFT (Eq. deltaG2), the vacuum_recovery = 0 energy and the recovered potential of
Sec. 5.3 on the GPU, against the oracle."""
import os

import numpy as np
import pytest

import npb_inputs as I

from .test_gpu_parity import small_molecule

pytestmark = pytest.mark.gpu


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


def linf_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


MOLS = [small_molecule, lambda: I.random_walk_molecule(150, 65, 0.5, seed=I.SEED_BASE + 90)]


@pytest.mark.parametrize("make", MOLS)
@pytest.mark.parametrize("richardson", [True, False])
def test_energy_fft_vacuum_fp64(npb, O, make, richardson):
    """vacuum_recovery = 0: the solvent legs against phi_0^FFT, 1e-10 relative to the oracle; the
    FFT vacuum potential itself matches the oracle's sine-transform solve to 1e-10."""
    p = make()
    c = npb.npb_ctx_create(0, 0)
    try:
        g = npb.npb_grid_create(c, p)
        try:
            o = npb.make_opts(0.4, 0.04, 6, richardson=richardson, vacuum_recovery=False)
            dg = npb.npb_energy(g, o)
            vac = npb.npb_potential(g, npb.NPB_LEG_VACUUM_FFT, npb.grid_shape(p))
        finally:
            npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(c)
    ref = O.energy_fft(p, 10.0, 6, richardson=richardson)
    assert abs(dg - ref) <= 1e-10 * abs(ref), (dg, ref)
    assert linf_rel(vac, O.vacuum_fft(p)) <= 1e-10


def test_energy_fft_vacuum_fp32(npb, O):
    p = MOLS[1]()
    c = npb.npb_ctx_create(0, 0)
    try:
        g = npb.npb_grid_create(c, p)
        try:
            dg = npb.npb_energy(g, npb.make_opts(0.4, 0.04, 6, vacuum_recovery=False, precision=1))
        finally:
            npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(c)
    ref = O.energy_fft(p, 10.0, 6)
    assert abs(dg - ref) <= 1e-4 * abs(ref), (dg, ref)


def test_recovered_potential(npb, O):
    """phi_m^LOD + phi_0^LOD - phi_0^FFT after an RE+V solve (FP64), against the oracle's legs."""
    p = small_molecule()
    c = npb.npb_ctx_create(0, 0)
    try:
        g = npb.npb_grid_create(c, p)
        try:
            npb.npb_energy(g, npb.make_opts(0.4, 0.04, 6))
            rec = npb.npb_potential(g, npb.NPB_LEG_RECOVERED, npb.grid_shape(p))
            npb.npb_energy(g, npb.make_opts(0.4, 0.04, 6, vacuum_recovery=False))
            with pytest.raises(npb.NpbError):  # needs the LOD vacuum legs
                npb.npb_potential(g, npb.NPB_LEG_RECOVERED, npb.grid_shape(p))
        finally:
            npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(c)
    _, legs, _ = O.energy(p, 10.0, 6, return_legs=True)
    us = 2 * legs["solvent_half"] - legs["solvent_tau"]
    uv = 2 * legs["vacuum_half"] - legs["vacuum_tau"]
    assert linf_rel(rec, us + uv - O.vacuum_fft(p)) <= 1e-10
