"""Several GPUs: (event, plane) units spread over devices, no collective.

The planes of a detector are simulated independently of one another and so
are events (Sec. 2.1 treats each plane on its own; Sec. 3.3 and Fig. 4 fill
several GPUs with independent processes).  The units (event e, plane p) of a
list of events therefore shard with no exchange on the data path: each
device gets a contiguous range of events (every plane of them), its own
planes (response spectra, workspace), batch workspace, stream and outputs,
and runs one ``ws_simulate_batch`` over its range.  Results do not depend on
the split: a unit's random numbers are keyed by its global event id
(``params.event_id + e``) and its plane, never by the device.

Ranges are contiguous so that a device's events keep consecutive event ids
(``ws_simulate_batch`` numbers the events of a call from
``params.event_id``), and they are balanced by a cost model of a unit: the
FFT convolution, proportional to the plane's grid cells, plus the raster,
proportional to its depos.  The split minimises the largest range cost
(exact for contiguous ranges: bisection on the bound with greedy packing).

Two forms:

* ``MultiBatch``: one process driving several devices (each shard's launches
  go to its own device and stream, so the devices run concurrently);
* ``rank_range`` / ``gather_units``: one process per GPU (torchrun); each rank
  takes its range and, only if the caller wants the waveforms in one place,
  ``gather_units`` sends them point to point to one rank.

A plane too large for one GPU's time budget splits by depos instead
(``depo_slices`` / ``simulate_depo_split``): each rank simulates a
contiguous slice of the plane's depos, with the slice's offset in the list
(``Params.depo_offset``) so that its random draws are the whole list's,
and the waveforms are summed across ranks (an all-reduce, or a
reduce-scatter that leaves each rank a band of wire rows).  Eq. 1 is
linear in S and S is the sum of the slices' grids, so the sum is the whole
plane's waveform (bin for bin in S when fluctuating; the transforms'
rounding in M).  This is the one path with a collective on the data.
"""
from __future__ import annotations

import dataclasses

# Device time of a unit, for balancing only (measured on the three-plane
# detector, 6000 ticks): the three transform stages take ~5.1 ns per grid
# cell, the raster with binomial fluctuation ~0.27 us per thousand depos.
CELL_COST = 5.1e-9
DEPO_COST = 2.7e-7


def unit_cost(nwires: int, nticks: int, ndepos: int, cell_cost: float = CELL_COST,
              depo_cost: float = DEPO_COST) -> float:
    """Estimated device seconds of one (event, plane) unit."""
    return cell_cost * nwires * nticks + depo_cost * ndepos


def event_costs(plane_shapes, events, cell_cost: float = CELL_COST, depo_cost: float = DEPO_COST):
    """Cost of each event: the sum over its planes.  plane_shapes: (nwires,
    nticks) per plane; events[e][p]: anything with ``.n`` (depos of event e
    on plane p)."""
    out = []
    for ev in events:
        if len(ev) != len(plane_shapes):
            raise ValueError(f"an event has {len(ev)} planes, the detector {len(plane_shapes)}")
        out.append(sum(unit_cost(nw, nt, d.n, cell_cost, depo_cost) for (nw, nt), d in zip(plane_shapes, ev)))
    return out


def _greedy_ranges(costs, bound: float):
    """Contiguous ranges, each as long as it stays within bound."""
    ranges, start, acc = [], 0, 0.0
    for i, c in enumerate(costs):
        if i > start and acc + c > bound:
            ranges.append((start, i))
            start, acc = i, 0.0
        acc += c
    ranges.append((start, len(costs)))
    return ranges


def partition_contiguous(costs, nparts: int):
    """Split items 0 .. n-1 into nparts contiguous ranges [e0, e1) that
    minimise the largest range cost.  Ranges are in order and cover every
    item; when there are fewer items than parts the last ranges are empty."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    costs = [float(c) for c in costs]
    if any(c < 0 for c in costs):
        raise ValueError("costs must be non-negative")
    n = len(costs)
    if n == 0:
        return [(0, 0)] * nparts
    # hi: the total with headroom for the greedy's own rounding (so it is
    # always feasible)
    lo, hi = max(costs), sum(costs) * (1.0 + 1e-9) + 1e-300
    if len(_greedy_ranges(costs, lo)) > nparts:
        # the smallest feasible bound lies in (lo, hi]: bisect on it
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if len(_greedy_ranges(costs, mid)) <= nparts:
                hi = mid
            else:
                lo = mid
            if hi - lo <= 1e-12 * max(hi, 1e-300):
                break
        bound = hi
    else:
        bound = lo
    ranges = _greedy_ranges(costs, bound)
    # use every part while items remain: split the costliest multi-item range
    while len(ranges) < nparts and any(e1 - e0 > 1 for e0, e1 in ranges):
        j = max((r for r in range(len(ranges)) if ranges[r][1] - ranges[r][0] > 1),
                key=lambda r: sum(costs[ranges[r][0]:ranges[r][1]]))
        e0, e1 = ranges[j]
        # the split point that best halves the range's cost
        tot, acc, best, best_gap = sum(costs[e0:e1]), 0.0, e0 + 1, float("inf")
        for i in range(e0, e1 - 1):
            acc += costs[i]
            gap = abs(tot - 2.0 * acc)
            if gap < best_gap:
                best, best_gap = i + 1, gap
        ranges[j:j + 1] = [(e0, best), (best, e1)]
    ranges += [(n, n)] * (nparts - len(ranges))
    return ranges


def rank_range(costs, world: int, rank: int):
    """Events [e0, e1) of rank ``rank`` out of ``world`` (one process per GPU)."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside 0 .. {world - 1}")
    return partition_contiguous(costs, world)[rank]


def units_of(ranges, nplanes: int):
    """Owner rank of every unit u = e * nplanes + p, in unit order."""
    owner = []
    for r, (e0, e1) in enumerate(ranges):
        owner += [r] * ((e1 - e0) * nplanes)
    return owner


def gather_units(dist, local_outs, ranges, nplanes: int, shapes, dst: int = 0, make=None):
    """Collect every unit's waveform on rank ``dst`` in unit order (point to
    point sends from the rank that owns it; the ranks' own work needs none
    of this).  local_outs: this rank's outputs, in unit order of its range;
    shapes[p]: (nwires, nticks) of plane p; make(shape, like): a receive
    buffer (default: ``torch.empty`` beside the local outputs).  Returns the
    list of all units' tensors on dst, None elsewhere."""
    import torch
    rank = dist.get_rank()
    e0, e1 = ranges[rank]
    if len(local_outs) != (e1 - e0) * nplanes:
        raise ValueError(f"rank {rank}: {len(local_outs)} outputs for {e1 - e0} events x {nplanes} planes")
    owner = units_of(ranges, nplanes)
    if rank != dst:
        for o in local_outs:
            dist.send(o.contiguous(), dst)
        return None
    like = local_outs[0] if local_outs else None
    if make is None:
        def make(shape, like):
            dev = like.device if like is not None else "cpu"
            return torch.empty(shape, dtype=torch.float32, device=dev)
    out, mine = [], iter(local_outs)
    for u, r in enumerate(owner):
        if r == dst:
            out.append(next(mine))
            continue
        t = make(tuple(shapes[u % nplanes]), like)
        dist.recv(t, r)
        out.append(t)
    return out


@dataclasses.dataclass
class Shard:
    device: object
    e0: int
    e1: int
    planes: list
    events: list
    batch: object
    stream: object


class MultiBatch:
    """The units of ``events`` over several devices from one process.

    devices: torch devices (a device may repeat: its shards then run side by
    side on separate streams); planes: specs with ``nwires``, ``nticks``,
    ``response`` (K_w x K_t) and ``plane_id`` (``inputs.PlaneSpec``);
    events[e][p]: host depos of event e on plane p (``.q``, ``.x_mm``,
    ``.t_us`` arrays); params: ``wiresim.Params`` (its ``event_id`` is the
    first event's).  Each device gets its own copies of the planes and of
    its events' depos, a batch workspace, a stream and the outputs.
    ``run()`` enqueues every shard without waiting; ``outputs()`` lists the
    units' waveforms (on their devices) in unit order e * nplanes + p."""

    def __init__(self, devices, planes, events, params, units_per_wave: int = 0, costs=None):
        import torch

        from . import wiresim
        self.devices = [torch.device(d) for d in devices]
        if not self.devices:
            raise ValueError("no devices")
        self.plane_specs = list(planes)
        self.nplanes = len(self.plane_specs)
        self.nevents = len(events)
        shapes = [(sp.nwires, sp.nticks) for sp in self.plane_specs]
        if costs is None:
            costs = event_costs(shapes, events)
        self.ranges = partition_contiguous(costs, len(self.devices))
        self.shards = []
        for dev, (e0, e1) in zip(self.devices, self.ranges):
            if e1 <= e0:
                continue
            pls = [wiresim.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id, device=dev)
                   for sp in self.plane_specs]
            evs = [[wiresim.DeviceDepos(d.q, d.x_mm, d.t_us, device=dev) for d in ev] for ev in events[e0:e1]]
            pe = wiresim.Params(**{**params.__dict__, "event_id": params.event_id + e0})
            b = wiresim.Batch(pls, evs, pe, units_per_wave=units_per_wave, device=dev)
            self.shards.append(Shard(dev, e0, e1, pls, evs, b, torch.cuda.Stream(dev)))

    def autotune(self):
        """Each shard's wave size by the library's autotuner, on its own inputs."""
        import torch
        for s in self.shards:
            with torch.cuda.device(s.device):
                s.batch.autotune(s.stream)

    def run(self):
        """Enqueue every shard on its device's stream (returns at once)."""
        import torch
        for s in self.shards:
            with torch.cuda.device(s.device):
                s.stream.wait_stream(torch.cuda.current_stream(s.device))
                s.batch.run(s.stream)
        return self

    def synchronize(self):
        for s in self.shards:
            s.stream.synchronize()

    def outputs(self):
        """Every unit's waveform tensor (on its shard's device) in unit order;
        valid once the shards' streams have finished (``synchronize``)."""
        out = []
        for s in self.shards:
            out += s.batch.outs
        return out

    def gather(self):
        """Every unit's waveform as a host numpy array, in unit order."""
        self.synchronize()
        return [o.cpu().numpy() for o in self.outputs()]

    def close(self):
        for s in self.shards:
            for pl in s.planes:
                pl.close()
        self.shards = []


def depo_slices(n: int, nparts: int):
    """Contiguous slices [lo, hi) of n depos over nparts ranks, sizes
    differing by at most one (the raster's cost is per depo; the
    convolution is the whole plane's on every rank)."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    q, r = divmod(n, nparts)
    out, lo = [], 0
    for k in range(nparts):
        hi = lo + q + (1 if k < r else 0)
        out.append((lo, hi))
        lo = hi
    return out


def wire_bands(nwires: int, nparts: int):
    """Wire-row bands [w0, w1) of a reduce-scatter of M over nparts ranks."""
    return depo_slices(nwires, nparts)


def simulate_depo_split(dist, plane, depos, params, out=None, scatter: bool = False, simulate=None):
    """One plane's event split by depos over the ranks of ``dist``: this rank
    simulates depos [lo, hi) of its slice (``depo_slices``) with
    ``depo_offset = lo``, then the ranks' waveforms are summed: all-reduced
    (every rank returns the whole M), or with ``scatter`` reduce-scattered
    by wire rows (each rank returns its band of ``wire_bands`` and the band;
    the plane's wires must split evenly).  ``depos``: the plane's whole
    depo list as host arrays (``inputs.PlaneDepos``); ``simulate(plane,
    q, x, t, params)`` runs one slice (default: ``plane.simulate`` on
    device copies).  The plane's noise term, if any, must be set on one
    rank only (each rank's waveform is added once)."""
    import torch
    world, rank = dist.get_world_size(), dist.get_rank()
    lo, hi = depo_slices(len(depos.q), world)[rank]
    p = dataclasses.replace(params, depo_offset=params.depo_offset + lo)
    if simulate is None:
        from . import wiresim

        def simulate(plane, q, x, t, p):
            dd = wiresim.DeviceDepos(q, x, t, device=plane.device)
            return plane.simulate(dd, p, out=out)
    M = simulate(plane, depos.q[lo:hi], depos.x_mm[lo:hi], depos.t_us[lo:hi], p)
    if not scatter:
        dist.all_reduce(M)
        return M
    nw = M.shape[0]
    if nw % world:
        raise ValueError(f"{nw} wires do not split evenly over {world} ranks")
    w0, w1 = wire_bands(nw, world)[rank]
    band = torch.empty((w1 - w0,) + tuple(M.shape[1:]), dtype=M.dtype, device=M.device)
    dist.reduce_scatter_tensor(band, M.contiguous())
    return band, (w0, w1)
