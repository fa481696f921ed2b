"""Failure detection on the device without a GPU fault: a bounded wait that expires.

The TMA-pipelined sweeps bound every wait on their tile copies.  The probe runs, before every sweep
launch, blocks that wait with the same bounded-wait helper on a barrier that nothing arrives at (no
copy in flight); with a short bound (about a millisecond) the wait expires and sets the grid's error
flag as an expired sweep wait does, and the call reports NPB_ETIMEOUT.  The same context then solves
normally and bit for bit like a fresh one.
"""
import pytest

import npb_inputs as I

pytestmark = pytest.mark.gpu


def test_expired_device_wait_returns_timeout_and_context_recovers():
    import paper_1410_2788_gb300 as npb
    from paper_1410_2788_gb300 import build

    build.build()
    p = I.random_walk_molecule(120, 65, 0.5, seed=I.SEED_BASE + 73)
    o = npb.make_opts(0.4, 0.04, 3, precision=npb.NPB_FP32_SWEEP)
    ref_ctx = npb.npb_ctx_create(0, 0)
    try:
        g = npb.npb_grid_create(ref_ctx, p)
        ref = npb.npb_energy(g, o)
        npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(ref_ctx)
    ctx = npb.npb_ctx_create(0, 0)
    try:
        g = npb.npb_grid_create(ctx, p)
        try:
            npb.npb_ctx_probe_wait_expiry(ctx, 2_000_000)  # ~1 ms at 2 GHz
            with pytest.raises(npb.NpbError) as e:
                npb.npb_energy(g, o)
            assert e.value.code == npb.NPB_ETIMEOUT, e.value
            with pytest.raises(npb.NpbError) as e:  # the single-stage path reports it too
                npb.npb_lod_solve(g, o, npb.NPB_SOLVENT, 1.0)
            assert e.value.code == npb.NPB_ETIMEOUT
            npb.npb_ctx_probe_wait_expiry(ctx, 0)
            assert npb.npb_energy(g, o) == ref  # the flag was cleared and the context still works
            assert npb.npb_energy(g, o) == ref
        finally:
            npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(ctx)


def test_probe_rejects_negative_bounds():
    import paper_1410_2788_gb300 as npb

    ctx = npb.npb_ctx_create(0, 0)
    try:
        with pytest.raises(npb.NpbError) as e:
            npb.npb_ctx_probe_wait_expiry(ctx, -1)
        assert e.value.code == npb.NPB_EINVAL
    finally:
        npb.npb_ctx_destroy(ctx)
