"""The charge-list entry point that allocates nothing, against the allocating one.

Some callers cannot allocate device memory when they need a charge list (an application
whose own pool owns the device, or a latency-critical path that cannot take the implicit
synchronisation of cudaMalloc/cudaFree).
npb_charge_list_static serves them from a fixed array inside the library.  This file is
collected last on purpose, so that a run stopping at its first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import npb_inputs as I

pytestmark = pytest.mark.gpu


def _dense_from_list(p, begin, count, ent_x, ent_qt, ent_off, n_ent):
    nx, ny, nz = p.n
    pitch = (nx + 31) // 32 * 32
    out = np.zeros((nz, ny, nx))
    assert int(count.sum()) == n_ent
    for ln in np.nonzero(count)[0]:
        z, y = divmod(int(ln), ny)
        b, c = int(begin[ln]), int(count[ln])
        xs = ent_x[b:b + c]
        assert np.all(np.diff(xs) > 0)  # each node once, ascending x within the line
        assert np.array_equal(ent_off[b:b + c], (z * ny + y) * pitch + xs)
        out[z, y, xs] = ent_qt[b:b + c]
    return out


def test_static_charge_list_matches_allocating_entry_point():
    import torch

    import paper_1410_2788_gb300 as npb
    from paper_1410_2788_gb300 import build

    build.build()
    ctx = npb.npb_ctx_create(0, 0)
    try:
        cases = [I.protein_1k(), I.protein_1k(), I.born_sphere(0.84)]  # two calls in a row, then another
        for p in cases:
            nx, ny, nz = p.n
            g = npb.npb_grid_create(ctx, p)
            try:
                ref = npb.npb_grid_export(g, npb.NPB_EXPORT_QTILDE, npb.grid_shape(p))
            finally:
                npb.npb_grid_destroy(g)
            cap = 8 * p.n_atoms
            dev = torch.device("cuda", 0)
            # poison the outputs so that stale or unwritten entries cannot pass
            begin = torch.full((ny * nz,), -7, dtype=torch.int32, device=dev)
            count = torch.full((ny * nz,), -7, dtype=torch.int32, device=dev)
            ex = torch.full((cap,), -7, dtype=torch.int32, device=dev)
            eq = torch.full((cap,), float("nan"), dtype=torch.float64, device=dev)
            eo = torch.full((cap,), -7, dtype=torch.int64, device=dev)
            ne = torch.full((1,), -7, dtype=torch.int32, device=dev)
            stream = torch.cuda.current_stream(dev)
            npb.npb_charge_list_static(p, begin.data_ptr(), count.data_ptr(), ex.data_ptr(), eq.data_ptr(),
                                       eo.data_ptr(), ne.data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize()
            n_ent = int(ne.item())
            assert 0 < n_ent <= cap
            got = _dense_from_list(p, begin.cpu().numpy(), count.cpu().numpy(), ex.cpu().numpy(),
                                   eq.cpu().numpy(), eo.cpu().numpy(), n_ent)
            assert np.array_equal(got, ref)  # the set-up tests hold charges bit-exact too
    finally:
        npb.npb_ctx_destroy(ctx)


def test_static_charge_list_rejects_oversized_inputs():
    import paper_1410_2788_gb300 as npb

    p = I.born_sphere(0.0)
    big = I.Problem(xyz=np.zeros((npb.NPB_STATIC_MAX_ATOMS + 1, 3)), q=np.zeros(npb.NPB_STATIC_MAX_ATOMS + 1),
                    radius=np.ones(npb.NPB_STATIC_MAX_ATOMS + 1), eps_in=1.0, eps_out=80.0, kappa2=0.0, h=0.5,
                    n=p.n, origin=p.origin)
    with pytest.raises(npb.NpbError) as e:
        npb.npb_charge_list_static(big, 1, 1, 1, 1, 1, 1)
    assert e.value.code == npb.NPB_EINVAL and "static scratch limit" in str(e.value)
