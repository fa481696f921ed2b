"""One RE+V solve of a benchmark molecule, for profiling the kernels under ncu.

    python -m paper_1410_2788_gb300.profile_solve WORKLOAD N_STEPS [x-shape y-shape z-shape]

WORKLOAD is protein_1k (129^3, 1,000 atoms) or large_20k (257^3, 20,000 atoms); each optional shape
is kind,tx,seg,len for one sweep direction (or "default").  FP32 sweeps, dt = 0.4, alpha = 0.04.
"""
import sys

import npb_inputs as I

import paper_1410_2788_gb300 as npb


def main(argv):
    w, n = argv[1], int(argv[2])
    p = I.protein_1k() if w == "protein_1k" else I.large_20k()
    ctx = npb.npb_ctx_create(0, 0)
    dims = npb.grid_shape(p)[::-1]
    for d, spec in enumerate(argv[3:6]):
        if spec != "default":
            k, tx, seg, ln = map(int, spec.split(","))
            npb.npb_tune_set(ctx, npb.NPB_FP32_SWEEP, d, dims[d], k, tx, seg, ln)
    g = npb.npb_grid_create(ctx, p)
    print("dG", npb.npb_energy(g, npb.make_opts(0.4, 0.04, n, precision=npb.NPB_FP32_SWEEP)))
    npb.npb_grid_destroy(g)
    npb.npb_ctx_destroy(ctx)


if __name__ == "__main__":
    main(sys.argv)
