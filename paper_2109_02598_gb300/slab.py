"""One periodic grid split into slabs along its slowest axis (z in 3D, y in 2D) over the ranks
of a process group: the multi-GPU form of a single forward-Euler run (Sec. 2.4.1).

Each rank holds its slab of n_local planes plus g = k R ghost planes on either side (R the
model's stencil radius per step: 1 for Models A and Gray-Scott and the N-species model, 2 for
Models B and C) as an ordinary periodic grid of n_local + 2 g planes. Before every k steps the
ranks exchange boundary planes: a rank sends its first g interior planes to the previous rank
and its last g to the next, and receives theirs into its ghost planes. Its local grid then runs
k steps with any kernel. The wrap of the local grid puts wrong values into the ghost planes,
but they travel at most R planes per step, so after k steps they have reached only the ghost
planes; every interior site has computed exactly what the undivided grid computes there, with
the same per-site arithmetic, so the interior is the undivided grid's bit for bit. The cost is
the redundant work on 2 g planes per rank and one exchange of 2 g planes per field per k steps.

The exchange uses point-to-point sends and receives of the process group (NCCL for device
buffers, gloo for host buffers); mass sums are all-reduced. This module only schedules: the
stepping runs in the library's kernels, and the plane copies in and out of a grid go through the
C ABI (pf_copy_planes).
"""
from __future__ import annotations

import numpy as np

from .grid import Grid

MODEL_RADIUS = {"ac": 1, "gs": 1, "rd": 1, "ch": 2, "c": 2}


def slab_range(n: int, rank: int, world: int):
    """Planes [lo, hi) of ``n`` that rank ``rank`` of ``world`` owns (balanced, contiguous)."""
    return n * rank // world, n * (rank + 1) // world


class SlabLayout:
    """Bookkeeping of one rank's slab: interior range, ghost width, local extent, neighbours,
    and the local plane ranges that are sent and received (no GPU needed)."""

    def __init__(self, n: int, world: int, rank: int, radius: int, k: int):
        if world < 1 or not 0 <= rank < world:
            raise ValueError("bad rank / world")
        if k < 1 or radius < 1:
            raise ValueError("k and radius must be >= 1")
        self.n, self.world, self.rank = int(n), int(world), int(rank)
        self.k, self.radius = int(k), int(radius)
        self.lo, self.hi = slab_range(self.n, self.rank, self.world)
        self.n_local = self.hi - self.lo
        self.g = self.radius * self.k  # ghost planes per side
        if self.n_local < self.g:
            raise ValueError(f"slab of {self.n_local} planes is thinner than its ghost width "
                             f"{self.g} (k {self.k} x radius {self.radius}): fewer ranks or a "
                             "smaller k")
        self.local = self.n_local + 2 * self.g
        self.prev = (self.rank - 1) % self.world
        self.next = (self.rank + 1) % self.world
        g, nl = self.g, self.n_local
        self.send_lo = (g, g)        # first g interior planes -> previous rank's top ghosts
        self.send_hi = (nl, g)       # last g interior planes -> next rank's bottom ghosts
        self.recv_lo = (0, g)        # bottom ghosts <- previous rank's last g interior planes
        self.recv_hi = (g + nl, g)   # top ghosts <- next rank's first g interior planes

    def global_planes(self):
        """Global index of every local plane (periodic)."""
        return [(self.lo - self.g + i) % self.n for i in range(self.local)]


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


class SlabGrid:
    """This rank's slab of a ``global_shape`` grid (axis 0 is the split axis: z of a 3D
    (nz, ny, nx) array, y of a 2D (ny, nx) one). ``k`` steps run between exchanges.
    ``backend``: a grid-like object of the local shape (``step``, ``copy_planes``,
    ``mass_planes``, ``write_fields``, ``read_fields``) in place of a GPU ``Grid``; the
    exchange buffers live on the host unless the group's backend is NCCL."""

    def __init__(self, global_shape, n_fields: int, model: str, coeffs, dt: float,
                 h: float = 1.0, k: int = 4, group=None, backend=None, stream=None):
        self.global_shape = tuple(int(s) for s in global_shape)
        self.n_fields = int(n_fields)
        self.group = group
        dist = _dist()
        world = dist.get_world_size(group) if dist else 1
        rank = dist.get_rank(group) if dist else 0
        self.layout = SlabLayout(self.global_shape[0], world, rank, MODEL_RADIUS[model], k)
        self.local_shape = (self.layout.local,) + self.global_shape[1:]
        if backend is None:
            backend = Grid(self.local_shape, self.n_fields, h, stream=stream).set_model(
                model, coeffs, dt)
        self.grid = backend
        self.steps_done = 0
        on_device = bool(dist) and dist.get_backend(group) == "nccl"
        import torch
        shape = (self.layout.g,) + self.global_shape[1:]
        dev = torch.device("cuda", torch.cuda.current_device()) if on_device else None
        mk = (lambda: torch.empty(shape, dtype=torch.float32, device=dev)) if on_device else \
            (lambda: torch.from_numpy(np.empty(shape, dtype=np.float32)))
        self._buf = [{key: mk() for key in ("send_lo", "send_hi", "recv_lo", "recv_hi")}
                     for _ in range(self.n_fields)]

    # ----------------------------------------------------------------- state in and out
    def write_global(self, fields):
        """Take this rank's slab, ghosts included, from full arrays of the global shape."""
        idx = self.layout.global_planes()
        self.grid.write_fields(tuple(np.ascontiguousarray(np.take(np.asarray(f), idx, axis=0))
                                     for f in fields))
        return self

    def read_interior(self):
        """This rank's interior planes (the slab it owns), one array per field."""
        g, nl = self.layout.g, self.layout.n_local
        return tuple(np.asarray(f)[g:g + nl] for f in self.grid.read_fields())

    def gather(self, dst: int = 0):
        """The whole grid on rank ``dst`` (None on the others), from every rank's interior."""
        dist = _dist()
        mine = self.read_interior()
        if dist is None:
            return mine
        parts = [None] * self.layout.world if self.layout.rank == dst else None
        dist.gather_object(mine, parts, dst=dst, group=self.group)
        if self.layout.rank != dst:
            return None
        return tuple(np.concatenate([p[f] for p in parts], axis=0) for f in range(self.n_fields))

    # ----------------------------------------------------------------- stepping
    def exchange(self):
        """Refresh the ghost planes from the neighbouring slabs."""
        L = self.layout
        for f in range(self.n_fields):
            b = self._buf[f]
            self.grid.copy_planes(f, L.send_lo[0], L.send_lo[1], b["send_lo"], True)
            self.grid.copy_planes(f, L.send_hi[0], L.send_hi[1], b["send_hi"], True)
        dist = _dist()
        if dist is None or L.world == 1:
            for f in range(self.n_fields):
                b = self._buf[f]
                b["recv_lo"].copy_(b["send_hi"])
                b["recv_hi"].copy_(b["send_lo"])
        else:
            # sends in the order (hi -> next, lo -> prev) and receives (lo <- prev, hi <- next),
            # with tags, so that two ranks (prev == next) still pair them correctly where the
            # backend matches by order
            ops = []
            for f in range(self.n_fields):
                b = self._buf[f]
                ops.append(dist.P2POp(dist.isend, b["send_hi"], L.next, self.group, 2 * f + 1))
                ops.append(dist.P2POp(dist.isend, b["send_lo"], L.prev, self.group, 2 * f))
                ops.append(dist.P2POp(dist.irecv, b["recv_lo"], L.prev, self.group, 2 * f + 1))
                ops.append(dist.P2POp(dist.irecv, b["recv_hi"], L.next, self.group, 2 * f))
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for f in range(self.n_fields):
            b = self._buf[f]
            self.grid.copy_planes(f, L.recv_lo[0], L.recv_lo[1], b["recv_lo"], False)
            self.grid.copy_planes(f, L.recv_hi[0], L.recv_hi[1], b["recv_hi"], False)

    def step(self, n_steps: int):
        """``n_steps`` forward-Euler steps of the whole grid: an exchange before every k."""
        left = int(n_steps)
        while left > 0:
            s = min(self.layout.k, left)
            self.exchange()
            self.grid.step(s)
            left -= s
            self.steps_done += s
        return self

    def mass(self, field: int = 0) -> float:
        """h^d sum of a field over the whole grid: each rank's interior by the library's
        reduction, all-reduced over the ranks."""
        local = self.grid.mass_planes(field, self.layout.g, self.layout.n_local)
        dist = _dist()
        if dist is None:
            return local
        import torch
        t = torch.tensor([local], dtype=torch.float64,
                         device="cuda" if dist.get_backend(self.group) == "nccl" else "cpu")
        dist.all_reduce(t, group=self.group)
        return float(t.item())

    def close(self):
        if hasattr(self.grid, "close"):
            self.grid.close()
