"""Batched 2D Gray-Scott through the C ABI: every instance against the FP64 oracle, and
bitwise against the same grid stepped alone (the batch runs the same tile body)."""
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

DT, DU, DV = 0.5, 0.2, 0.1


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02598_gb300.build import build
    build()
    import paper_2109_02598_gb300 as pf
    return pf


def make_specs(shapes, seed=7):
    F = synthetic.uniform(seed, 20, len(shapes), 0.02, 0.06)
    k = synthetic.uniform(seed, 21, len(shapes), 0.045, 0.07)
    return [dict(ny=s[0], nx=s[1], Du=DU, Dv=DV, F=float(f), k=float(kk))
            for s, f, kk in zip(shapes, F, k)]


SHAPES = [(64, 64), (97, 130), (5, 7), (200, 33), (1, 9), (128, 256), (70, 70), (33, 300)]


def init(shape, i):
    return synthetic.gray_scott_init(shape, seed=500 + i, n_seeds=max(1, shape[0] * shape[1] // 1500),
                                     side=4, noise=0.05)


def test_batch_matches_oracle_and_single_grids(pf):
    specs = make_specs(SHAPES)
    b = pf.Batch(specs, DT)
    x0 = [init(s, i) for i, s in enumerate(SHAPES)]
    for i, (u, v) in enumerate(x0):
        b.write(i, 0, u).write(i, 1, v)
    n = 13
    b.run(n)
    for i, (s, sp) in enumerate(zip(SHAPES, specs)):
        coeffs = (DU, DV, sp["F"], sp["k"])
        got = (b.read(i, 0), b.read(i, 1))
        ref = oracle.run("gs", x0[i], coeffs, DT, n)
        err = max(np.abs(g.astype(np.float64) - r).max() for g, r in zip(got, ref))
        assert err <= 2e-5 * max(np.abs(r).max() for r in ref), (i, s)
        g = pf.Grid(s, 2).set_model("gs", coeffs, DT)
        g.write_fields(x0[i]).step(n)
        alone = g.read_fields()
        g.close()
        assert np.array_equal(got[0], alone[0]) and np.array_equal(got[1], alone[1]), (i, s)
    b.close()


def test_batch_tunings_replays_and_autotune_agree_bitwise(pf):
    specs = make_specs(SHAPES, seed=8)
    x0 = [init(s, i) for i, s in enumerate(SHAPES)]

    def run(tuning, chunks):
        b = pf.Batch(specs, DT)
        for i, (u, v) in enumerate(x0):
            b.write(i, 0, u).write(i, 1, v)
        if tuning == "auto":
            b.autotune(2)
        else:
            b.set_tuning(*tuning)
        for c in chunks:
            b.run(c)
        out = [(b.read(i, 0), b.read(i, 1)) for i in range(len(SHAPES))]
        b.close()
        return out

    base = run((64, 16, 1), [12])
    S = pf.PF_TILE_STRIPS
    for tuning, chunks in [((128, 16, 2), [12]), ((32, 32, 4), [5, 7]), ((128, 32, 4), [6, 6]),
                           ((64, 16, 2), [3, 3, 3, 3]), ((128, S, 4), [5, 7]),
                           ((128, S, 2), [12]), ((128, S, 1), [4, 8]), ((64, S, 4), [12]),
                           ((64, S, 2), [5, 7]), ((64, S, 1), [12]), ("auto", [12])]:
        got = run(tuning, chunks)
        for (a0, a1), (b0, b1) in zip(base, got):
            assert np.array_equal(a0, b0) and np.array_equal(a1, b1), tuning


def test_batch_workload_recipe_runs(pf):
    specs = synthetic.batch_instances(n=64, seed=4)
    full = [dict(n=s["n"], Du=DU, Dv=DV, F=s["F"], k=s["k"]) for s in specs]
    b = pf.Batch(full, DT)
    for i, s in enumerate(specs):
        u, v = synthetic.batch_instance_init(s["n"], i)
        b.write(i, 0, u).write(i, 1, v)
    b.run(200)
    for i in (0, 17, 63):
        u, v = b.read(i, 0), b.read(i, 1)
        assert np.isfinite(u).all() and np.isfinite(v).all()
        assert u.min() >= -0.01 and u.max() <= 1.01
    assert b.sites == sum(s["n"] ** 2 for s in specs)
    b.close()


def test_batch_rejects_unstable_dt(pf):
    from paper_2109_02598_gb300 import PfError
    with pytest.raises(PfError, match="stability"):
        pf.Batch(make_specs([(16, 16)]), 5.0)


def test_full_batch_configuration(pf):
    # the batched configuration itself: 512 instances, sides log-uniform in [64, 512], seeded
    # F and k. After 1000 steps, four instances (the smallest, the largest and two more) are
    # within the 1000-step tolerance of the oracle; after 2000 every instance is finite and
    # within [-0.01, 1.01]
    specs = synthetic.batch_instances(512, seed=4)
    b = pf.Batch([dict(n=q["n"], Du=0.2, Dv=0.1, F=q["F"], k=q["k"]) for q in specs], 0.5)
    x0 = [synthetic.batch_instance_init(q["n"], i) for i, q in enumerate(specs)]
    for i, (u, v) in enumerate(x0):
        b.write(i, 0, u).write(i, 1, v)
    b.autotune(3)
    b.run(1000)
    sides = [q["n"] for q in specs]
    picks = {int(np.argmin(sides)), int(np.argmax(sides)), 100, 300}
    for i in picks:
        coeffs = (0.2, 0.1, specs[i]["F"], specs[i]["k"])
        ref = oracle.run("gs", x0[i], coeffs, 0.5, 1000)
        got = (b.read(i, 0), b.read(i, 1))
        num = np.sqrt(sum(((g.astype(np.float64) - r) ** 2).sum() for g, r in zip(got, ref)))
        den = np.sqrt(sum((r ** 2).sum() for r in ref))
        assert num / den <= 1e-3, (i, sides[i], num / den)
    b.run(1000)
    for i in range(len(specs)):
        u, v = b.read(i, 0), b.read(i, 1)
        assert np.isfinite(u).all() and np.isfinite(v).all(), i
        assert u.min() >= -0.01 and u.max() <= 1.01 and v.min() >= -0.01 and v.max() <= 1.01, i
    b.close()


def _rel(got, ref, norm):
    if norm == "inf":
        num = max(np.abs(g.astype(np.float64) - r).max() for g, r in zip(got, ref))
        return num / max(np.abs(r).max() for r in ref)
    num = np.sqrt(sum(((g.astype(np.float64) - r) ** 2).sum() for g, r in zip(got, ref)))
    return num / np.sqrt(sum((r ** 2).sum() for r in ref))


def test_full_batch_every_instance_against_the_oracle(pf):
    # the 512-instance configuration with the autotuner's tuning (the one the bench times):
    # every instance within the single-step bar after one step and after one launch of the
    # tuned depth k; 16 instances spread over the sizes within the 1000-step bar. The oracle
    # runs in worker processes (spawned: this process already holds a CUDA context).
    specs = synthetic.batch_instances(512, seed=4)
    coeffs = [(0.2, 0.1, q["F"], q["k"]) for q in specs]
    x0 = [synthetic.batch_instance_init(q["n"], i) for i, q in enumerate(specs)]

    def batch_after(steps, tuning):
        b = pf.Batch([dict(n=q["n"], Du=0.2, Dv=0.1, F=q["F"], k=q["k"]) for q in specs], 0.5)
        for i, (u, v) in enumerate(x0):
            b.write(i, 0, u).write(i, 1, v)
        if tuning is None:
            b.autotune(3)
        else:
            b.set_tuning(*tuning)
        t = b.tuning
        b.run(steps)
        out = [(b.read(i, 0), b.read(i, 1)) for i in range(len(specs))]
        b.close()
        return out, tuple(t)

    sides = np.array([q["n"] for q in specs])
    order = np.argsort(sides, kind="stable")
    picks = [int(order[j]) for j in np.linspace(0, len(specs) - 1, 16).round().astype(int)]
    workers = min(16, os.cpu_count() or 1)
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        long_ref = {i: ex.submit(oracle.run, "gs", x0[i], coeffs[i], 0.5, 1000) for i in picks}
        one, tuning = batch_after(1, None)
        k = tuning[2]
        ref1 = list(ex.map(oracle.run, ["gs"] * len(specs), x0, coeffs, [0.5] * len(specs),
                           [1] * len(specs), chunksize=8))
        for i, (got, ref) in enumerate(zip(one, ref1)):
            assert _rel(got, ref, "inf") <= 1e-6, (i, sides[i])
        if k > 1:
            refk = list(ex.map(oracle.run, ["gs"] * len(specs), x0, coeffs,
                               [0.5] * len(specs), [k] * len(specs), chunksize=8))
            launch, _ = batch_after(k, tuning)
            for i, (got, ref) in enumerate(zip(launch, refk)):
                assert _rel(got, ref, "inf") <= 1e-6, (i, sides[i], k)
        thousand, _ = batch_after(1000, tuning)
        for i in picks:
            err = _rel(thousand[i], long_ref[i].result(), "l2")
            assert err <= 1e-3, (i, sides[i], err)


def test_full_batch_strip_kernel_is_bitwise_the_tiled_batch(pf):
    # the 512-instance configuration: the strip kernel (every instance's width split evenly
    # over strips of 128 or 64 columns) gives every instance the bits of the tiled batch, at
    # every depth
    specs = synthetic.batch_instances(512, seed=4)
    x0 = [synthetic.batch_instance_init(q["n"], i) for i, q in enumerate(specs)]

    def run(tuning, steps):
        b = pf.Batch([dict(n=q["n"], Du=0.2, Dv=0.1, F=q["F"], k=q["k"]) for q in specs], 0.5)
        for i, (u, v) in enumerate(x0):
            b.write(i, 0, u).write(i, 1, v)
        b.set_tuning(*tuning)
        b.run(steps)
        out = [(b.read(i, 0), b.read(i, 1)) for i in range(len(specs))]
        b.close()
        return out

    ref = run((32, 32, 4), 12)
    for width, k in ((128, 4), (128, 2), (128, 1), (64, 4), (64, 2), (64, 1)):
        got = run((width, pf.PF_TILE_STRIPS, k), 12)
        for i, ((a0, a1), (b0, b1)) in enumerate(zip(ref, got)):
            assert np.array_equal(a0, b0) and np.array_equal(a1, b1), (i, specs[i]["n"], width, k)
    with pytest.raises(pf.PfError, match="strip kernel"):
        pf.Batch(make_specs([(16, 16)]), DT).set_tuning(96, pf.PF_TILE_STRIPS, 1)
