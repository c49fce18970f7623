"""Slab decomposition of one grid along y: the multi-GPU layout of the step.

The update (Sec. III.A.1, Eq. finalDiscretePDE) reads a cross-shaped stencil
two cells wide along each axis (Sec. III.A.2), so a band of rows needs, per
step, the two boundary rows of each neighbouring band at the same time level.
Each band is a libdvbm context whose inner y sides are ``EXTERNAL``;
``dvbm_halo_pack`` / ``dvbm_halo_unpack`` move the rows between the context's
padded buffer and contiguous [npop, 2, Nx] halo buffers, and this module only
moves those buffers between bands: device-to-device copies between contexts
of one process (``LocalSlabs``), or point-to-point send/recv between ranks
(``exchange``, ``RankSlab``; NCCL on GPUs, gloo on CPU).  Every step and every
halo copy in and out of a band runs in libdvbm; this module does no
arithmetic of the method.

Exchange pattern per step (after every band stepped): a band sends its two
highest rows up and its two lowest rows down, and receives its lower ghost
rows from the band below and its upper ghost rows from the band above.  The
time step is the smallest of the bands' CFL steps (``dvbm_set_dt``), domain
totals are sums over bands.

The adjoint of a y-periodic grid runs band by band with the stepwise backward
pass (``dvbm_adjoint_begin`` / ``_advance`` / ``_finish``): every action of
the pass (lambda^N, a restored checkpoint, a recomputed segment state, an
adjoint step) is followed by the same two-row exchange of the buffer it
produced (``dvbm_adjoint_halo_pack`` / ``_unpack``), all bands take the same
actions in the same order, and dL/d(mu, Pr, gamma) is the sum of the bands'
shares.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

from . import dvbm as D

# tags of the two message kinds (gloo matches on them; NCCL matches two
# messages between the same pair of ranks in the order they are posted, and
# every rank posts them in the same order)
TAG_HI_ROWS, TAG_LO_ROWS = 0, 1


def neighbours(rank: int, world: int, periodic: bool):
    """(lower, upper) band indices of band ``rank`` of ``world`` bands; None
    at a non-periodic domain edge."""
    lower = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    upper = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return lower, upper


def split_rows(Ny: int, parts: int, align: int = 8) -> List[int]:
    """Band heights summing to Ny: multiples of ``align`` where possible (the
    step kernel's tile height, so that bands tile the grid exactly as the
    undecomposed run does), the remainder on the last band; every band keeps
    at least 4 rows."""
    if parts < 1 or Ny < 4 * parts:
        raise ValueError(f"cannot split {Ny} rows into {parts} bands of >= 4 rows")
    base = max(align * (Ny // (parts * align)), 4) if align > 0 else Ny // parts
    if base * parts > Ny:
        base = Ny // parts
    heights = [base] * (parts - 1)
    heights.append(Ny - base * (parts - 1))
    return heights


def exchange(dist, rank: int, world: int, periodic: bool, send_lo, send_hi, recv_lo, recv_hi):
    """Point-to-point halo exchange of one band with its neighbours through
    ``torch.distributed`` (any backend).  send_lo / send_hi: this band's two
    lowest / highest rows; recv_lo / recv_hi: buffers for the ghost rows below
    / above it.  Buffers of a missing neighbour may be None.  Blocks until
    the received rows have landed."""
    lower, upper = neighbours(rank, world, periodic)
    if world == 1:
        if periodic:  # the band is its own neighbour on both sides
            recv_lo.copy_(send_hi)
            recv_hi.copy_(send_lo)
        return
    ops = []
    if upper is not None:
        ops.append(dist.P2POp(dist.isend, send_hi, upper, tag=TAG_HI_ROWS))
    if lower is not None:
        ops.append(dist.P2POp(dist.isend, send_lo, lower, tag=TAG_LO_ROWS))
    if lower is not None:
        ops.append(dist.P2POp(dist.irecv, recv_lo, lower, tag=TAG_HI_ROWS))
    if upper is not None:
        ops.append(dist.P2POp(dist.irecv, recv_hi, upper, tag=TAG_LO_ROWS))
    for w in dist.batch_isend_irecv(ops):
        w.wait()


def band_bcs(bcs: Optional[Sequence], k: int, parts: int):
    """Boundary entries of band k (as ``dvbm.make_bcs`` takes them): the
    grid's x sides; EXTERNAL on inner y sides and on both y sides of every
    band of a y-periodic grid; the grid's own y side at a non-periodic domain
    edge.  Also returns whether the grid is periodic in y."""
    g = [D.PERIODIC] * 4 if bcs is None else list(bcs)
    kind = lambda b: int(b[0]) if isinstance(b, (tuple, list)) else int(b)
    periodic_y = kind(g[D.YLO]) == D.PERIODIC
    lo = D.EXTERNAL if (periodic_y or k > 0) else g[D.YLO]
    hi = D.EXTERNAL if (periodic_y or k < parts - 1) else g[D.YHI]
    return [g[D.XLO], g[D.XHI], lo, hi], periodic_y


class LocalSlabs:
    """A grid split into bands along y, one libdvbm context per band on the
    current device, halos exchanged by device-to-device copies on the
    contexts' (shared) stream.  Same interface as ``dvbm.Simulation`` for
    init / step / moments / totals / populations."""

    def __init__(self, Nx: int, Ny: int, parts: int, Pr: float, gamma: float, mu: float, bcs=None,
                 storage: int = D.FP64, lattice: int = D.D2Q25_SPLIT_II, heights=None, **opts):
        self.Nx, self.Ny = int(Nx), int(Ny)
        self.heights = list(heights) if heights else split_rows(self.Ny, parts)
        if sum(self.heights) != self.Ny:
            raise ValueError("band heights must sum to Ny")
        Lx = float(opts.pop("Lx", 1.0))
        Ly = float(opts.pop("Ly", 0.0)) or Lx * self.Ny / self.Nx
        dy = Ly / self.Ny
        self.fixed_dt = float(opts.get("dt", 0.0)) > 0
        self.sims = []
        for k, h in enumerate(self.heights):
            bk, self.periodic = band_bcs(bcs, k, len(self.heights))
            self.sims.append(D.Simulation(self.Nx, h, Pr, gamma, mu, bcs=bk, storage=storage, lattice=lattice,
                                          Lx=Lx, Ly=dy * h, **opts))
        n = len(self.sims)
        self.nb = [neighbours(k, n, self.periodic) for k in range(n)]
        self.out_lo = [s.halo_buffer() for s in self.sims]
        self.out_hi = [s.halo_buffer() for s in self.sims]

    def _rows(self, a):
        out, y = [], 0
        for h in self.heights:
            out.append(a[y:y + h])
            y += h
        return out

    def exchange(self):
        for k, s in enumerate(self.sims):
            lower, upper = self.nb[k]
            s.halo_pack(self.out_lo[k] if lower is not None else None,
                        self.out_hi[k] if upper is not None else None)
        for k, s in enumerate(self.sims):
            lower, upper = self.nb[k]
            s.halo_unpack(self.out_hi[lower] if lower is not None else None,
                          self.out_lo[upper] if upper is not None else None)

    def init(self, rho, ux, uy, T):
        parts = [self._rows(a) for a in (rho, ux, uy, T)]
        for k, s in enumerate(self.sims):
            s.init(*(p[k] for p in parts))
        if not self.fixed_dt:  # every band steps with the smallest CFL step
            dt = min(s.dt for s in self.sims)
            for s in self.sims:
                s.set_dt(dt)
        self.exchange()
        return self

    def step(self, n: int = 1):
        for _ in range(int(n)):
            for s in self.sims:
                s.step(1)
            self.exchange()
        return self

    @property
    def dt(self) -> float:
        return self.sims[0].dt

    def moments(self):
        import torch
        ms = [s.moments() for s in self.sims]
        return {k: torch.cat([m[k] for m in ms], dim=0) for k in ("rho", "ux", "uy", "T")}

    def populations(self):
        import torch
        return torch.cat([s.populations() for s in self.sims], dim=1)

    def totals(self):
        t = [s.totals() for s in self.sims]
        return tuple(sum(v[i] for v in t) for i in range(4))

    # -- adjoint (FP64, D2Q25 / split II, y-periodic grid)
    def record(self, every: int):
        for s in self.sims:
            s.record(every)
        return self

    def _adjoint_exchange(self):
        for k, s in enumerate(self.sims):
            lower, upper = self.nb[k]
            s.adjoint_halo_pack(self.out_lo[k] if lower is not None else None,
                                self.out_hi[k] if upper is not None else None)
        for k, s in enumerate(self.sims):
            lower, upper = self.nb[k]
            s.adjoint_halo_unpack(self.out_hi[lower] if lower is not None else None,
                                  self.out_lo[upper] if upper is not None else None)

    def adjoint(self, dL_drho=None, dL_dT=None):
        """Gradients of a loss of the final (rho, T) fields, as
        ``dvbm.Simulation.adjoint``: every band runs the stepwise backward pass,
        with the halo rows of the buffer each action produced exchanged after
        it; the bands' parameter gradients add up."""
        import torch
        n = len(self.sims)
        parts = [self._rows(a) if a is not None else [None] * n for a in (dL_drho, dL_dT)]
        for k, s in enumerate(self.sims):
            s.adjoint_begin(parts[0][k], parts[1][k])
        self._adjoint_exchange()
        while True:
            acts = {s.adjoint_advance() for s in self.sims}
            if len(acts) != 1:
                raise RuntimeError(f"bands out of step in the backward pass: {sorted(acts)}")
            if acts == {0}:
                break
            self._adjoint_exchange()
        res = [s.adjoint_finish() for s in self.sims]
        out = {k: torch.cat([r[k] for r in res], dim=0) for k in ("rho0", "ux0", "uy0", "T0")}
        for k in ("mu", "Pr", "gamma"):
            out[k] = sum(r[k] for r in res)
        return out

    def close(self):
        for s in self.sims:
            s.close()


class RankSlab:
    """Band ``rank`` of a grid split over ``world`` processes (one GPU each),
    halos exchanged with ``exchange`` (NCCL), dt and totals reduced over the
    process group."""

    def __init__(self, dist, Nx: int, Ny_band: int, Pr: float, gamma: float, mu: float, bcs=None,
                 storage: int = D.FP64, lattice: int = D.D2Q25_SPLIT_II, **opts):
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        kinds, self.periodic = band_bcs(bcs, self.rank, self.world)
        self.fixed_dt = float(opts.get("dt", 0.0)) > 0
        self.sim = D.Simulation(Nx, Ny_band, Pr, gamma, mu, bcs=kinds, storage=storage, lattice=lattice, **opts)
        lower, upper = neighbours(self.rank, self.world, self.periodic)
        s = self.sim
        self.send_lo = s.halo_buffer() if lower is not None else None
        self.send_hi = s.halo_buffer() if upper is not None else None
        self.recv_lo = s.halo_buffer() if lower is not None else None
        self.recv_hi = s.halo_buffer() if upper is not None else None

    def exchange(self):
        self.sim.halo_pack(self.send_lo, self.send_hi)
        exchange(self.dist, self.rank, self.world, self.periodic, self.send_lo, self.send_hi, self.recv_lo,
                 self.recv_hi)
        self.sim.halo_unpack(self.recv_lo, self.recv_hi)

    def init(self, rho, ux, uy, T):
        import torch
        self.sim.init(rho, ux, uy, T)
        if not self.fixed_dt:
            t = torch.tensor([self.sim.dt], dtype=torch.float64, device=self.sim.device)
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN)
            self.sim.set_dt(float(t.item()))
        self.exchange()
        return self

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.sim.step(1)
            self.exchange()
        return self

    def totals(self):
        import torch
        t = torch.tensor(self.sim.totals(), dtype=torch.float64, device=self.sim.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return tuple(float(v) for v in t.cpu())

    # -- adjoint (FP64, D2Q25 / split II, y-periodic grid)
    def record(self, every: int):
        self.sim.record(every)
        return self

    def _adjoint_exchange(self):
        self.sim.adjoint_halo_pack(self.send_lo, self.send_hi)
        exchange(self.dist, self.rank, self.world, self.periodic, self.send_lo, self.send_hi, self.recv_lo,
                 self.recv_hi)
        self.sim.adjoint_halo_unpack(self.recv_lo, self.recv_hi)

    def adjoint(self, dL_drho=None, dL_dT=None):
        """This band's share of the grid's backward pass (the gradients of its
        own initial fields) and dL/d(mu, Pr, gamma) of the whole grid (an
        all-reduce SUM over the bands).  Every rank takes the same actions in
        the same order, so the point-to-point exchanges pair up as in the
        forward steps."""
        import torch
        self.sim.adjoint_begin(dL_drho, dL_dT)
        self._adjoint_exchange()
        while self.sim.adjoint_advance():
            self._adjoint_exchange()
        out = self.sim.adjoint_finish()
        p = torch.tensor([out["mu"], out["Pr"], out["gamma"]], dtype=torch.float64, device=self.sim.device)
        self.dist.all_reduce(p, op=self.dist.ReduceOp.SUM)
        out["mu"], out["Pr"], out["gamma"] = (float(v) for v in p.cpu())
        return out

    def close(self):
        self.sim.close()
