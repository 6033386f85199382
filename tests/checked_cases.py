"""Cases run twice by test_gpu_checked.py: once through the normal library and once, in a
child process (PFGPU_CHECKED=1), through the checked variant, whose kernels fill their shared
memory with NaN before staging. A kernel that reads a shared-memory slot that staging or an
earlier sub-step did not write gives NaN, or other bits, in the checked run.

Each case returns the final fields as float32 arrays. The set covers every kernel family
that stages through shared memory:

* the 2D tile body for every model, tile and depth on ragged grids;
* the other 2D stencils;
* the cluster and band kernels;
* the general, TMA, depth-2 and box 3D kernels;
* the batch;
* the adjoints.

Run as a script: ``python checked_cases.py OUT.npz`` writes the results."""
import ctypes
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import synthetic  # noqa: E402

COEFFS = {"ac": (1.0, 1.0), "ch": (1.0, 1.0, 1.0), "gs": (0.2, 0.1, 0.04, 0.06),
          "c": (1.0, 1.0, 1.0, 1.0, 1.0)}
DT = {"ac": 0.05, "ch": 0.01, "gs": 0.5, "c": 0.005}
KS = {"ac": (1, 2, 4), "gs": (1, 2, 4), "ch": (1, 2), "c": (1, 2)}


def fields(model, shape, seed):
    if model == "ac":
        return (synthetic.allen_cahn_init(shape, seed=100 + seed, lo=-0.5, hi=0.5),)
    if model == "ch":
        return (synthetic.cahn_hilliard_init(shape, seed=200 + seed, amp=0.3),)
    if model == "c":
        return (synthetic.allen_cahn_init(shape, seed=400 + seed, lo=-0.5, hi=0.5),
                synthetic.cahn_hilliard_init(shape, seed=450 + seed, amp=0.4))
    n_seeds = max(2, int(np.prod(shape)) // 2000)
    return synthetic.gray_scott_init(shape, seed=300 + seed, n_seeds=n_seeds, side=4,
                                     noise=0.05)


def run_grid(pf, model, shape, n, tuning=None, stencil=None, seed=0):
    x0 = fields(model, shape, seed)
    g = pf.Grid(shape, n_fields=len(x0)).set_model(model, COEFFS[model], DT[model], force=True)
    if stencil:
        g.set_stencil(stencil)
    if tuning:
        g.set_tuning(*tuning)
    g.write_fields(x0)
    g.step(n)
    out = g.read_fields()
    g.close()
    return list(out)


def run_cases(pf):
    res = {}
    # 2D tile body: every model, tile and depth, a ragged grid (nx % 4 != 0) and a regular one
    for model in ("ac", "ch", "gs", "c"):
        for tx, ty in ((64, 16), (128, 16), (32, 32), (128, 32)):
            for k in KS[model]:
                for shape in ((33, 70), (64, 96)):
                    res[f"tile_{model}_{tx}x{ty}_k{k}_{shape[0]}x{shape[1]}"] = run_grid(
                        pf, model, shape, 9, (tx, ty, k))
    # the other 2D stencils
    for model in ("ac", "gs"):
        for st in ("iso", "4th"):
            for tx, ty in ((64, 16), (128, 32)):
                res[f"stencil_{model}_{st}_{tx}x{ty}"] = run_grid(pf, model, (33, 70), 7,
                                                                  (tx, ty, 2), stencil=st)
    # the cluster kernel (full rows, ny / CS rows per CTA)
    for model, k in (("ac", 4), ("gs", 4), ("ch", 2), ("c", 2)):
        for cs in (16, 8):
            try:
                res[f"cluster_{model}_k{k}"] = run_grid(pf, model, (128, 128), 13,
                                                        (128, 128 // cs, k))
                break
            except pf.PfError:
                continue
    # the band kernel
    for model, shape in (("ch", (256, 512)), ("ac", (77, 388)), ("ch", (333, 388))):
        res[f"bands_{model}_{shape[0]}x{shape[1]}"] = run_grid(
            pf, model, shape, 11, (shape[1], pf.PF_TILE_BANDS, 1))
    # 3D: the general kernel (all models), the TMA kernels and the depth-2 kernel
    for model in ("ac", "ch", "gs", "c"):
        for tile in ((32, 16), (64, 8)):
            res[f"3d_general_{model}_{tile[0]}x{tile[1]}"] = run_grid(pf, model, (10, 20, 36), 5,
                                                                     (tile[0], tile[1], 1))
    for model in ("ac", "gs"):
        res[f"3d_tma_{model}"] = run_grid(pf, model, (12, 32, 128), 5, (64, 16, 1))
        res[f"3d_depth2_{model}"] = run_grid(pf, model, (12, 16, 128), 6, (128, 8, 2))
    for model in ("ch", "c"):  # the radius-2 TMA kernel
        for tile in ((64, 16), (128, 8)):
            res[f"3d_tma_r2_{model}_{tile[0]}x{tile[1]}"] = run_grid(
                pf, model, (9, 32, 128), 5, (tile[0], tile[1], 1))
    for model in ("ch", "c"):  # the box kernel, both depths, boxes past every edge
        for k in (1, 2):
            res[f"3d_box_{model}_k{k}"] = run_grid(pf, model, (11, 13, 36), 5, (32, 8, k))
    # N coupled species (3 and 4 fields): the 2D tile and the 3D plane ring, ragged shapes,
    # z-chunks of one plane and of several
    rd3 = pf.rd_coeffs((0.2, 0.05, 0.12),
                       [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 2, 0], [2, 0, 1], [0, 0, 3]],
                       [[0.03, -0.03, 0.0, 0.1, -1.0, 0.0, 0.0],
                        [0.0, 0.0, -0.09, 0.0, 1.0, -0.4, 0.0],
                        [0.0, 0.05, 0.0, -0.2, 0.0, 0.4, -0.3]])
    rd4 = pf.rd_coeffs((0.1, 0.15, 0.05, 0.02),
                       [[1, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 0, 0, 0]],
                       [[-1.2, 0.5, 0.3, -0.05, 0.0], [-1.2, 0.5, 0.0, 0.0, 0.05],
                        [1.2, -0.7, 0.0, 0.0, 0.0], [0.0, 0.2, -0.3, 0.0, 0.0]])
    for nf, c in ((3, rd3), (4, rd4)):
        for shape in ((33, 70), (10, 20, 36), (3, 17, 33), (40, 16, 64)):
            n = int(np.prod(shape))
            x0 = tuple(synthetic.uniform(90 + nf, 60 + i, n, 0.05, 0.9).reshape(shape)
                       .astype(np.float32) for i in range(nf))
            g = pf.Grid(shape, nf).set_model("rd", c, 0.2)
            g.write_fields(x0)
            g.step(7)
            res[f"rd{nf}_{'x'.join(map(str, shape))}"] = list(g.read_fields())
            g.close()
    # the batch
    shapes = [(64, 64), (97, 130), (5, 7), (33, 300)]
    specs = [dict(ny=s[0], nx=s[1], Du=0.2, Dv=0.1, F=0.03 + 0.005 * i, k=0.05 + 0.003 * i)
             for i, s in enumerate(shapes)]
    b = pf.Batch(specs, 0.5)
    for i, s in enumerate(shapes):
        u, v = fields("gs", s, 60 + i)
        b.write(i, 0, u).write(i, 1, v)
    b.run(9)
    out = []
    for i in range(len(shapes)):
        out += [b.read(i, 0), b.read(i, 1)]
    b.close()
    res["batch"] = out
    # the adjoints (Gray-Scott; Models A and B)
    from paper_2109_02598_gb300 import _lib
    for model, shape, coeffs, dt in (("gs", (40, 48), COEFFS["gs"], 0.5),
                                     ("ac", (33, 70), (0.9, 1.1), 0.02),
                                     ("ch", (33, 70), (0.8, 1.1, 0.7), 0.004)):
        x0 = fields(model, shape, 70)
        g = pf.Grid(shape, len(x0)).set_model(model, coeffs, dt)
        g.write_fields(x0)
        _lib.check(g._lib.pf_adj_forward(g.handle, 12, 4))
        xN = g.read_fields()
        d = [np.ascontiguousarray(0.5 * x, dtype=np.float32) for x in xN]
        g0 = [np.empty_like(x) for x in xN]
        dth = (ctypes.c_double * 4)()
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        _lib.check(g._lib.pf_adj_backward(
            g.handle, vp(d[0]), vp(d[1]) if len(d) > 1 else None, 0, vp(g0[0]),
            vp(g0[1]) if len(g0) > 1 else None, dth))
        g.close()
        res[f"adjoint_{model}"] = g0 + [np.array(list(dth), dtype=np.float64)]
    return res


if __name__ == "__main__":
    import paper_2109_02598_gb300 as pf
    out = run_cases(pf)
    flat = {f"{k}__{i}": a for k, v in out.items() for i, a in enumerate(v)}
    np.savez(sys.argv[1], **flat)
    print(f"{len(out)} cases")
