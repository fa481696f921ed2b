"""Continuous batching through npb_submit / npb_poll.

Requests of different grid sizes and precisions are submitted together and while others
run; every result must equal (bit for bit) the same problem solved alone with npb_energy,
admission must respect the HBM budget, and invalid requests fail without disturbing others.
"""
import time

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


def _alone(npb, p, opts):
    c = npb.npb_ctx_create(0, 0)
    try:
        g = npb.npb_grid_create(c, p)
        try:
            return npb.npb_energy(g, opts)
        finally:
            npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(c)


def _cases(npb):
    mols = [I.random_walk_molecule(150, 65, 0.5, seed=I.SEED_BASE + 200 + k) for k in range(3)]
    mols += [I.random_walk_molecule(400, 97, 0.5, seed=I.SEED_BASE + 210), I.born_sphere(0.84)]
    cases = []
    for k, p in enumerate(mols):
        prec = npb.NPB_FP32_SWEEP if k % 2 == 0 else npb.NPB_FP64
        n = 8 + 3 * k
        cases.append((p, npb.make_opts(0.4, 0.04, n, precision=prec)))
    return cases


def test_results_identical_alone_and_in_the_mix(npb):
    cases = _cases(npb)
    alone = [_alone(npb, p, o) for p, o in cases]
    ctx = npb.npb_ctx_create(0, 0)
    try:
        # half submitted up front, the rest while the first ones run
        tickets = [npb.npb_submit(ctx, p, o) for p, o in cases[:3]]
        time.sleep(0.002)
        tickets += [npb.npb_submit(ctx, p, o) for p, o in cases[3:]]
        res = [npb.npb_poll(ctx, t, 60000) for t in tickets]
    finally:
        npb.npb_ctx_destroy(ctx)
    for r, ref, (p, o) in zip(res, alone, cases):
        assert r is not None and r.status == npb.NPB_OK
        assert r.dG_kcal_mol == ref, (r.dG_kcal_mol, ref)
        assert tuple(r.n) == tuple(p.n)
        assert r.wall_ms >= r.queue_ms >= 0.0
        assert r.point_steps == npb.interior_point_steps(p, o.n_steps)


def test_admission_waits_for_memory(npb):
    """With a budget that holds one grid at a time, every request still completes."""
    p = I.random_walk_molecule(150, 65, 0.5, seed=I.SEED_BASE + 220)
    o = npb.make_opts(0.4, 0.04, 6, precision=npb.NPB_FP32_SWEEP)
    ref = _alone(npb, p, o)
    fp = npb.npb_grid_footprint(p, npb.NPB_FP32_SWEEP)
    ctx = npb.npb_ctx_create(0, int(1.5 * fp) + (64 << 20))
    try:
        tickets = [npb.npb_submit(ctx, p, o) for _ in range(4)]
        res = [npb.npb_poll(ctx, t, 60000) for t in tickets]
        used, budget = npb.npb_ctx_memory(ctx)
    finally:
        npb.npb_ctx_destroy(ctx)
    assert all(r.status == npb.NPB_OK and r.dG_kcal_mol == ref for r in res)
    assert used <= budget


def test_failures_are_isolated(npb):
    good = I.random_walk_molecule(150, 65, 0.5, seed=I.SEED_BASE + 230)
    bad = I.Problem(xyz=np.array([[0.1, 0.1, 0.1]]), q=np.array([1.0]), radius=np.array([1.0]), eps_in=1.0,
                    eps_out=80.0, kappa2=0.84, h=0.5, n=(33, 33, 33), origin=(0.0, 0.0, 0.0))
    o = npb.make_opts(0.4, 0.04, 5, precision=npb.NPB_FP32_SWEEP)
    ref = _alone(npb, good, o)
    ctx = npb.npb_ctx_create(0, 0)
    try:
        t1 = npb.npb_submit(ctx, bad, o)
        t2 = npb.npb_submit(ctx, good, o)
        r1 = npb.npb_poll(ctx, t1, 60000)
        r2 = npb.npb_poll(ctx, t2, 60000)
        with pytest.raises(npb.NpbError) as e:  # a final poll consumes the ticket
            npb.npb_poll(ctx, t2, 0)
        assert e.value.code == npb.NPB_ENOTFOUND
    finally:
        npb.npb_ctx_destroy(ctx)
    assert r1.status == npb.NPB_EINVAL
    assert r2.status == npb.NPB_OK and r2.dG_kcal_mol == ref


def test_poll_timeout_and_unknown_ticket(npb):
    ctx = npb.npb_ctx_create(0, 0)
    try:
        p = I.random_walk_molecule(150, 65, 0.5, seed=I.SEED_BASE + 240)
        t = npb.npb_submit(ctx, p, npb.make_opts(0.4, 0.04, 200, precision=npb.NPB_FP64))
        assert npb.npb_poll(ctx, t, 0) is None  # still running
        with pytest.raises(npb.NpbError) as e:
            npb.npb_poll(ctx, t + 1000, 0)
        assert e.value.code == npb.NPB_ENOTFOUND
        assert npb.npb_poll(ctx, t, 120000).status == npb.NPB_OK
    finally:
        npb.npb_ctx_destroy(ctx)


def test_large_molecules_sharing_launches(npb):
    """Two 8,300-atom molecules on 177^3 grids share their step launches in the serving loop; with
    charge lists of 66,400 entry slots their source stage is a launch of its own over both grids'
    legs (read from the leg table), where a molecule solved alone runs the by-value kernel of one
    grid.  Both add the same FP32 product, so the energies equal the lone solves bit for bit."""
    cases = [(I.random_walk_molecule(8300, 177, 0.5, seed=I.SEED_BASE + s),
              npb.make_opts(0.4, 0.04, 6, precision=npb.NPB_FP32_SWEEP)) for s in (311, 312)]
    assert all(8 * p.n_atoms >= 65536 for p, _ in cases)
    alone = [_alone(npb, p, o) for p, o in cases]
    ctx = npb.npb_ctx_create(0, 0)
    try:
        tickets = [npb.npb_submit(ctx, p, o) for p, o in cases]
        res = [npb.npb_poll(ctx, t, 120000) for t in tickets]
    finally:
        npb.npb_ctx_destroy(ctx)
    for r, ref in zip(res, alone):
        assert r is not None and r.status == npb.NPB_OK
        assert r.dG_kcal_mol == ref, (r.dG_kcal_mol, ref)
