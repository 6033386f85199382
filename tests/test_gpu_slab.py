"""A grid split into slabs over two ranks, each rank a process with its own grid on the same
GPU, the boundary planes exchanged through host memory with gloo (kernels never wait on one
another: every exchange is a host-side send and receive between launches). The gathered
result must be the bits of the undivided grid stepped alone."""
import os
import socket

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

CASES = {
    "gs3d": dict(model="gs", coeffs=(0.2, 0.1, 0.04, 0.06), dt=0.5, shape=(48, 32, 128), k=4,
                 steps=50),
    "c3d": dict(model="c", coeffs=(1.0,) * 5, dt=0.005, shape=(24, 16, 64), k=2, steps=21),
    "ch2d": dict(model="ch", coeffs=(1.0, 1.0, 1.0), dt=0.01, shape=(96, 80), k=3, steps=40),
    "rd2d": dict(model="rd", coeffs=oracle.rd_pack((0.2, 0.1, 0.05), [[1, 1, 0], [0, 0, 1]],
                                                   [[-1.0, 0.4], [-1.0, 0.4], [1.0, -0.4]]),
                 dt=0.2, shape=(64, 40), k=4, steps=30),
}


def _fields(name):
    c = CASES[name]
    if c["model"] == "gs":
        return synthetic.gray_scott_init(c["shape"], seed=31, n_seeds=6, side=4, noise=0.05)
    nf = {"c": 2, "ch": 1, "rd": 3}[c["model"]]
    lo, hi = (0.05, 0.9) if c["model"] == "rd" else (-0.5, 0.5)  # concentrations are >= 0
    return tuple(synthetic.allen_cahn_init(c["shape"], seed=80 + i, lo=lo, hi=hi)
                 for i in range(nf))


def _worker(rank, world, port, name, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2109_02598_gb300 as pf
        c = CASES[name]
        x0 = _fields(name)
        sg = pf.SlabGrid(c["shape"], len(x0), c["model"], c["coeffs"], c["dt"], k=c["k"])
        sg.write_global(x0)
        sg.step(c["steps"])
        full = sg.gather(0)
        mass = sg.mass(0)
        sg.close()
        if rank == 0:
            np.savez(out_path, *full, mass=np.array([mass]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("name", list(CASES))
def test_two_slabs_on_one_gpu_give_the_undivided_grid(tmp_path, name):
    import torch
    import torch.multiprocessing as mp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02598_gb300.build import build
    build()
    import paper_2109_02598_gb300 as pf
    out = str(tmp_path / "out.npz")
    mp.start_processes(_worker, args=(2, _free_port(), name, out), nprocs=2,
                       start_method="spawn")
    c = CASES[name]
    x0 = _fields(name)
    g = pf.Grid(c["shape"], len(x0)).set_model(c["model"], c["coeffs"], c["dt"]).write_fields(x0)
    g.step(c["steps"])
    ref = g.read_fields()
    m_ref = g.mass(0)
    g.close()
    got = np.load(out)
    for f, r in enumerate(ref):
        assert np.array_equal(got[f"arr_{f}"], r), (name, f)
    assert abs(float(got["mass"][0]) - m_ref) <= 1e-9 * max(1.0, abs(m_ref))
