"""npb_energy_batch: many molecules of uneven grid sizes in shared persistent launches."""
import numpy as np
import pytest

import npb_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def npb():
    import paper_1410_2788_gb300 as m
    from paper_1410_2788_gb300 import build

    build.build()
    return m


@pytest.fixture(scope="module")
def O(oracle_lib):
    import os

    oracle_lib.set_threads(os.cpu_count() or 8)
    return oracle_lib


def _mols():
    # grids 65^3 (three molecules), 97^3 (two) and 57^3 (one): three groups of uneven size
    spec = [(40, 65), (100, 65), (300, 97), (110, 65), (450, 97), (30, 57)]
    return [I.random_walk_molecule(na, n, 0.5, seed=I.SEED_BASE + 300 + i) for i, (na, n) in enumerate(spec)]


@pytest.mark.parametrize("precision,scheme", [(1, 2), (1, 1), (0, 2)])
def test_batch_equals_single_solves_bitwise(npb, precision, scheme):
    """Each batched energy is the single-grid npb_energy value bit for bit (same kernels, same
    shapes; legs of equal-size grids share launches), and a second call replays the graph."""
    c = npb.npb_ctx_create(0, 0)
    try:
        grids = [npb.npb_grid_create(c, p) for p in _mols()]
        try:
            o = npb.make_opts(0.4, 0.04, 6, scheme=scheme, precision=precision)
            single = [npb.npb_energy(g, o) for g in grids]
            batch = npb.npb_energy_batch(grids, o)
            again = npb.npb_energy_batch(grids, o)
            assert batch == single
            assert again == single
            sub = npb.npb_energy_batch(grids[1:4], o)  # a different composition, its own plan
            assert sub == single[1:4]
        finally:
            for g in grids:
                npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(c)


def test_batch_matches_oracle(npb, O):
    """FP32 batch against the FP64 oracle, molecule by molecule (1e-4 relative dG)."""
    mols = _mols()[:3]
    c = npb.npb_ctx_create(0, 0)
    try:
        grids = [npb.npb_grid_create(c, p) for p in mols]
        try:
            dg = npb.npb_energy_batch(grids, npb.make_opts(0.4, 0.04, 6, precision=1))
        finally:
            for g in grids:
                npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(c)
    for p, v in zip(mols, dg):
        ref = O.energy(p, 10.0, 6)
        assert abs(v - ref) <= 1e-4 * abs(ref), (v, ref)


def test_batch_after_destroy_and_invalid(npb):
    c = npb.npb_ctx_create(0, 0)
    try:
        mols = _mols()
        grids = [npb.npb_grid_create(c, p) for p in mols]
        o = npb.make_opts(0.4, 0.04, 4, precision=1)
        ref = npb.npb_energy_batch(grids, o)
        npb.npb_grid_destroy(grids[0])  # drops the cached plan that names it
        rest = grids[1:]
        assert npb.npb_energy_batch(rest, o) == ref[1:]
        g_new = npb.npb_grid_create(c, mols[0])  # may reuse the freed address
        assert npb.npb_energy_batch([g_new] + rest, o) == ref
        with pytest.raises(npb.NpbError):
            npb.npb_energy_batch([rest[0], rest[0]], o)
        with pytest.raises(npb.NpbError):
            npb.npb_energy_batch([], o)
        for g in [g_new] + rest:
            npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(c)


def test_batch_with_tuned_shapes_and_tuning_cache(npb, O, tmp_path):
    """The autotuner picks the line solver per (direction, grid size) -- the candidates span the
    paper's Thomas per line (kind 3) and the segmented Thomas/PCR hybrids -- the picks survive a save/load round trip through the tuning cache, and the batched energies
    with those shapes still equal the single solves bit for bit and the oracle to 1e-4."""
    mols = _mols()
    c = npb.npb_ctx_create(0, 0)
    try:
        grids = [npb.npb_grid_create(c, p) for p in mols]
        try:
            o = npb.make_opts(0.4, 0.04, 6, precision=1)
            seen = set()
            for p, g in zip(mols, grids):
                if p.n[0] not in seen:
                    seen.add(p.n[0])
                    rep = npb.npb_autotune(g, o, reps=2)
                    kinds = {r["kind"] for r in rep}
                    assert {2, 3} <= kinds, kinds  # hybrids and the line-per-thread-pair Thomas
            shapes = {(d, n): npb.npb_tune_get(c, 1, d, n) for n in seen for d in range(3)}
            path = str(tmp_path / "tune.json")
            npb.npb_tune_save(c, path)
            single = [npb.npb_energy(g, o) for g in grids]
            batch = npb.npb_energy_batch(grids, o)
            assert batch == single
        finally:
            for g in grids:
                npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(c)
    c2 = npb.npb_ctx_create(0, 0)
    try:
        assert npb.npb_tune_load(c2, path) == len(shapes)
        assert {k: npb.npb_tune_get(c2, 1, k[0], k[1]) for k in shapes} == shapes
    finally:
        npb.npb_ctx_destroy(c2)
    for p, v in zip(mols[:2], batch[:2]):
        ref = O.energy(p, 10.0, 6)
        assert abs(v - ref) <= 1e-4 * abs(ref), (v, ref)


def test_shape_pinned_after_a_captured_solve_takes_effect(npb):
    """A solve that came back (and so replays a captured CUDA graph) runs the line-solver shape
    pinned since: its energy equals bit for bit that of a fresh context with the new shape pinned
    from the start, for each of several x shapes in turn."""
    p = _mols()[0]
    nx = p.n[0]
    o = npb.make_opts(0.4, 0.04, 6, precision=1)
    seq = [(2, 8, 24, 11), (2, 8, 16, 17), (2, 8, 8, 9), (2, 8, 20, 13)]
    fresh = []
    for sh in seq:
        c = npb.npb_ctx_create(0, 0)
        try:
            npb.npb_tune_set(c, 1, 0, nx, *sh)
            g = npb.npb_grid_create(c, p)
            try:
                fresh.append(npb.npb_energy(g, o))
            finally:
                npb.npb_grid_destroy(g)
        finally:
            npb.npb_ctx_destroy(c)
    c = npb.npb_ctx_create(0, 0)
    try:
        g = npb.npb_grid_create(c, p)
        try:
            for sh, want in zip(seq, fresh):
                npb.npb_tune_set(c, 1, 0, nx, *sh)
                got = [npb.npb_energy(g, o) for _ in range(3)]  # direct, captured, replayed
                assert got == [want] * 3, (sh, got, want)
        finally:
            npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(c)


def test_source_launch_of_its_own_equals_fused(npb, O):
    """Large charge lists (8,300 atoms: 66,400 entry slots) take LODIE2's S as a launch of its own
    over the charge entries before the x sweep; the batched path keeps it fused into the x sweep's
    load.  Both add the same FP32 product to the same node value, so the energies agree bit for
    bit, and with the oracle to 1e-4."""
    p = I.random_walk_molecule(8300, 177, 0.5, seed=I.SEED_BASE + 310)
    assert 8 * p.n_atoms >= 65536
    o = npb.make_opts(0.4, 0.04, 6, precision=1)
    c = npb.npb_ctx_create(0, 0)
    try:
        g = npb.npb_grid_create(c, p)
        try:
            single = npb.npb_energy(g, o)
            assert npb.npb_energy_batch([g], o) == [single]
        finally:
            npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(c)
    ref = O.energy(p, 10.0, 6)
    assert abs(single - ref) <= 1e-4 * abs(ref), (single, ref)
