"""Domain decomposition of the periodic element block into z-slabs (one per GPU).

A periodic nx x ny x NZ block of elements is cut along z into ``ws`` slabs of
nz = NZ / ws element layers.  Each rank holds its slab plus one ghost element
layer below and one above, whose control points are the neighbours' (taken from
the global mesh, wrapping periodically), so the kernels' neighbour indexing
inside the extended nx x ny x (nz + 2) block is already right for every
interior element.  The state of an element layer is a contiguous
[nx*ny][5][n^3] slice, so before every RK stage a rank sends its first and last
interior layers to the ranks below and above, which store them in their ghost
layers: the one exchange of the method (the face states of the partition
faces follow from the ghost states).  Ghost elements get face states but no
volume pass and no stage update (their outer neighbours are not theirs); the
next exchange refills them.  The time step is the CFL step of the largest wave
speed over all ranks.

Two exchangers move the layers: ``DistExchanger`` (torch.distributed point-to-
point operations, NCCL between GPUs or gloo, with a timeout that turns a
missing or late message into ``HaloTimeout``) and ``LocalSlabs`` (several slabs
in one process, exchanged by copies; used to check the decomposition against
the undecomposed solver on one GPU).
"""
from __future__ import annotations

import datetime

import numpy as np

from .nsfr import Solver


class HaloTimeout(RuntimeError):
    """A halo message did not arrive within the exchanger's timeout."""


def slab_range(nz_global, ws, rank):
    """(z0, nz): the first global element layer and the number of layers of ``rank``."""
    if nz_global % ws:
        raise ValueError(f"{nz_global} element layers do not split into {ws} slabs")
    nz = nz_global // ws
    return rank * nz, nz


def extended_layers(a, shape, z0, nz):
    """The element layers z0-1 .. z0+nz (periodic in the global index) of a global
    per-element array ``a`` [N_e][...] with element e = ex + nx (ey + ny ez): control
    points [N_e][q^3][3] or a state [N_e][5][n^3]."""
    nx, ny, NZ = shape
    L = nx * ny
    layers = [(z0 - 1 + k) % NZ for k in range(nz + 2)]
    return np.ascontiguousarray(np.concatenate([a[z * L:(z + 1) * L] for z in layers]))


def halo_views(t, layer):
    """(send_down, send_up, recv_from_above, recv_from_below) views of an extended state
    [(nz+2) layers][...]: the first and last interior layers, the top and bottom ghosts."""
    L = layer
    return t[L:2 * L], t[-2 * L:-L], t[-L:], t[:L]


class DistExchanger:
    """Halo exchange with torch.distributed (ranks ordered along z, periodic)."""

    def __init__(self, dist, rank, ws, timeout_s=60.0, group=None):
        self.dist, self.rank, self.ws, self.group = dist, rank, ws, group
        self.timeout = datetime.timedelta(seconds=timeout_s)

    def exchange(self, t, layer):
        send_down, send_up, recv_top, recv_bottom = halo_views(t, layer)
        if self.ws == 1:  # the neighbour is the slab itself
            recv_top.copy_(send_down)
            recv_bottom.copy_(send_up)
            return
        d = self.dist
        # gloo moves host memory only: device layers go through host copies
        staged = t.is_cuda and d.get_backend(self.group) == "gloo"
        if staged:
            bufs = [send_down.cpu(), send_up.cpu(), recv_top.cpu(), recv_bottom.cpu()]
        else:
            bufs = [send_down, send_up, recv_top, recv_bottom]
        below, above = (self.rank - 1) % self.ws, (self.rank + 1) % self.ws
        # the same order on every rank: sends (down, up), receives (from above, from
        # below), so that pairs of ranks (ws = 2: below == above) match in posting order
        ops = [d.P2POp(d.isend, bufs[0], below, self.group, 1),
               d.P2POp(d.isend, bufs[1], above, self.group, 0),
               d.P2POp(d.irecv, bufs[2], above, self.group, 1),
               d.P2POp(d.irecv, bufs[3], below, self.group, 0)]
        works = d.batch_isend_irecv(ops)
        for w in works:
            try:
                ok = w.wait(self.timeout)
            except Exception as exc:  # the backend reports the timeout as an error
                raise HaloTimeout(f"rank {self.rank}: halo exchange failed or timed out: {exc}") from exc
            if ok is False:
                raise HaloTimeout(f"rank {self.rank}: halo exchange timed out")
        if staged:
            recv_top.copy_(bufs[2])
            recv_bottom.copy_(bufs[3])

    def global_max(self, x):
        if self.ws == 1:
            return x
        import torch
        dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"  # gloo: host
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return float(t.item())


class Slab:
    """One rank's slab of the global mesh, with its ghost layers and RK arrays."""

    def __init__(self, ctrl, shape, p, rank, ws, exchanger=None, copies=1, **solver_kw):
        """``ctrl`` [nx*ny*NZ][q^3][3] and ``shape`` (nx, ny, NZ) describe the periodic mesh;
        with ``copies`` > 1 the decomposed mesh is that many copies of it stacked along z
        (nx x ny x copies*NZ elements, a weak-scaling workload that needs one copy in memory)."""
        import torch
        nx, ny, NZ = shape
        self.shape, self.p, self.rank, self.ws = tuple(shape), p, rank, ws
        self.z0, self.nz = slab_range(NZ * copies, ws, rank)
        self.layer = nx * ny
        self.ctrl = extended_layers(ctrl, shape, self.z0, self.nz)  # layer indices wrap mod NZ
        self.solver = Solver(self.ctrl, (nx, ny, self.nz + 2), p, **solver_kw)
        self.exchanger = exchanger
        n = self.solver.n
        self.state_shape = (self.layer * (self.nz + 2), 5, n ** 3)
        self.ustage = torch.empty(self.state_shape, dtype=torch.float64, device="cuda")
        self.acc = torch.empty_like(self.ustage)
        # CFL spacing of the global mesh (the extended block's extent wraps around)
        lo = ctrl.reshape(-1, 3).min(axis=0)
        hi = ctrl.reshape(-1, 3).max(axis=0)
        self.dx = float(min((hi[d] - lo[d]) / (shape[d] * (p + 1)) for d in range(3)))

    def interior(self, t):
        return t[self.layer:-self.layer]

    def extend(self, u_global):
        """This rank's extended state (device) cut from a global host state (one copy of
        the mesh's state with ``copies`` > 1)."""
        import torch
        return torch.from_numpy(extended_layers(u_global, self.shape, self.z0, self.nz)).cuda()

    def node_coords(self):
        return self.solver.node_coords()

    def stage(self, u, st, dt):
        # the interior elements only: the ghost layers are refilled by the next exchange
        self.solver.rk_stage(u, self.ustage, self.acc, st, dt,
                             elements=(self.layer, self.layer * (self.nz + 1)))

    def step(self, u, cfl=0.1, dt=None):
        """One RK4 step of the decomposed problem (every rank calls it); returns dt."""
        ex = self.exchanger
        ex.exchange(u, self.layer)
        if dt is None:
            lam = ex.global_max(self.solver.max_wavespeed(u))
            dt = cfl * self.dx / lam
        for st in range(4):
            if st > 0:
                ex.exchange(self.ustage, self.layer)
            self.stage(u, st, dt)
        return dt


class LocalSlabs:
    """All ``ws`` slabs of a mesh in one process, exchanged by copies (lockstep)."""

    def __init__(self, ctrl, shape, p, ws, **solver_kw):
        self.slabs = [Slab(ctrl, shape, p, r, ws, None, **solver_kw) for r in range(ws)]
        self.ws = ws

    def _exchange(self, tensors):
        L = self.slabs[0].layer
        views = [halo_views(t, L) for t in tensors]
        for r in range(self.ws):
            below, above = (r - 1) % self.ws, (r + 1) % self.ws
            views[r][2].copy_(views[above][0])  # top ghost <- first interior layer of the rank above
            views[r][3].copy_(views[below][1])  # bottom ghost <- last interior layer of the rank below

    def step(self, us, cfl=0.1, dt=None):
        self._exchange(us)
        if dt is None:
            lam = max(s.solver.max_wavespeed(u) for s, u in zip(self.slabs, us))
            dt = cfl * self.slabs[0].dx / lam
        for st in range(4):
            if st > 0:
                self._exchange([s.ustage for s in self.slabs])
            for s, u in zip(self.slabs, us):
                s.stage(u, st, dt)
        return dt
