"""A grid split into slabs over ranks (paper_2109_02598_gb300.slab), on the CPU with gloo.

The bookkeeping is checked directly; the exchange with world sizes 2 and 3 runs each rank's
local grid with the FP64 oracle, storing the state in float32 after every step (as the GPU
grids do), against the undivided grid stepped the same way: the gathered result must be the
same bits."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synthetic
from paper_2109_02598_gb300.slab import SlabGrid, SlabLayout, slab_range


@pytest.mark.parametrize("n,world,radius,k", [(64, 2, 1, 4), (37, 3, 2, 2), (10, 1, 2, 3),
                                              (256, 8, 1, 2)])
def test_layout_covers_the_grid_and_pairs_the_exchanges(n, world, radius, k):
    lays = [SlabLayout(n, world, r, radius, k) for r in range(world)]
    owned = np.concatenate([np.arange(L.lo, L.hi) for L in lays])
    assert np.array_equal(owned, np.arange(n))
    for L in lays:
        gp = L.global_planes()
        assert L.local == L.n_local + 2 * L.g and len(gp) == L.local
        assert gp[L.g:L.g + L.n_local] == list(range(L.lo, L.hi))
        nxt, prv = lays[L.next], lays[L.prev]
        # what this rank sends up is what the next rank's bottom ghosts hold, and down likewise
        sh, rl = L.send_hi, nxt.recv_lo
        assert gp[sh[0]:sh[0] + sh[1]] == nxt.global_planes()[rl[0]:rl[0] + rl[1]]
        sl, rh = L.send_lo, prv.recv_hi
        assert gp[sl[0]:sl[0] + sl[1]] == prv.global_planes()[rh[0]:rh[0] + rh[1]]
    with pytest.raises(ValueError, match="thinner"):
        SlabLayout(8, 4, 0, 2, 2)  # 2 planes per rank, 4 ghost planes


def test_slab_range_is_balanced():
    sizes = [slab_range(100, r, 7)[1] - slab_range(100, r, 7)[0] for r in range(7)]
    assert sum(sizes) == 100 and max(sizes) - min(sizes) <= 1


class OracleGrid:
    """A local grid stepped by the oracle, its state stored in float32 after every step."""

    def __init__(self, model, coeffs, dt, h):
        self.model, self.coeffs, self.dt, self.h = model, coeffs, dt, h
        self.x = None

    def write_fields(self, fields):
        self.x = [np.asarray(f, dtype=np.float32).copy() for f in fields]
        return self

    def read_fields(self):
        return tuple(a.copy() for a in self.x)

    def step(self, n):
        for _ in range(n):
            y = oracle.euler_step(self.model, self.x, self.coeffs, self.dt, self.h)
            self.x = [a.astype(np.float32) for a in y]

    def copy_planes(self, f, first, count, buf, to_buf):
        if to_buf:
            buf.copy_(torch.from_numpy(self.x[f][first:first + count].copy()))
        else:
            self.x[f][first:first + count] = buf.numpy()

    def mass_planes(self, f, first, count):
        return float(self.h ** self.x[f].ndim * self.x[f][first:first + count].astype(np.float64).sum())


CASES = {
    "gs2d": dict(model="gs", coeffs=(0.2, 0.1, 0.04, 0.06), dt=0.5, h=1.0, shape=(40, 24), k=3,
                 steps=17),
    "ch3d": dict(model="ch", coeffs=(1.0, 1.0, 1.0), dt=0.01, h=1.0, shape=(24, 8, 10), k=2,
                 steps=9),
    "rd3": dict(model="rd", coeffs=oracle.rd_pack((0.2, 0.1, 0.05), [[1, 1, 0], [0, 0, 1]],
                                                  [[-1.0, 0.4], [-1.0, 0.4], [1.0, -0.4]]),
                dt=0.2, h=0.9, shape=(30, 12), k=4, steps=13),
}


def _fields(name):
    c = CASES[name]
    nf = {"gs": 2, "ch": 1, "rd": 3}[c["model"]]
    return tuple(synthetic.allen_cahn_init(c["shape"], seed=70 + i, lo=0.05, hi=0.9)
                 for i in range(nf))


def _worker(rank, world, port, name, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = CASES[name]
        x0 = _fields(name)
        sg = SlabGrid(c["shape"], len(x0), c["model"], c["coeffs"], c["dt"], c["h"], k=c["k"],
                      backend=OracleGrid(c["model"], c["coeffs"], c["dt"], c["h"]))
        sg.write_global(x0)
        sg.step(c["steps"])
        full = sg.gather(0)
        mass = sg.mass(0)
        if rank == 0:
            np.savez(out_path, *full, mass=np.array([mass]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("name,world", [("gs2d", 2), ("ch3d", 3), ("rd3", 2), ("gs2d", 1)])
def test_slabs_give_the_undivided_grid_bit_for_bit(tmp_path, name, world):
    out = str(tmp_path / "out.npz")
    mp.start_processes(_worker, args=(world, _free_port(), name, out), nprocs=world,
                       start_method="spawn")
    c = CASES[name]
    ref = OracleGrid(c["model"], c["coeffs"], c["dt"], c["h"]).write_fields(_fields(name))
    ref.step(c["steps"])
    got = np.load(out)
    for f, r in enumerate(ref.read_fields()):
        assert np.array_equal(got[f"arr_{f}"], r), (name, world, f)
    assert abs(float(got["mass"][0]) - ref.mass_planes(0, 0, c["shape"][0])) <= \
        1e-12 * abs(ref.mass_planes(0, 0, c["shape"][0]))
