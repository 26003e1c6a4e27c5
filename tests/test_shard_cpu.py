"""Host logic of the multi-GPU split (Sec. 3.3): contiguous event ranges
balanced by cost, and the point-to-point gather of the units' waveforms.

The partition is checked against brute force over every contiguous split of
small cost lists; the gather runs as two gloo ranks on 127.0.0.1, each rank
simulating its own range of events with the FP64 oracle (binomial mode, so a
unit's result depends on its global event id) and rank 0 comparing the
gathered units with the whole list simulated in one process."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2203_02479_gb300 import inputs, shard  # noqa: E402


def _brute_best(costs, nparts):
    n = len(costs)
    best = float("inf")
    for k in range(1, min(n, nparts) + 1):
        for cuts in itertools.combinations(range(1, n), k - 1):
            b = (0,) + cuts + (n,)
            best = min(best, max(sum(costs[b[i]:b[i + 1]]) for i in range(k)))
    return best


def _check_ranges(ranges, n, nparts):
    assert len(ranges) == nparts
    pos = 0
    for e0, e1 in ranges:
        assert e0 == pos and e1 >= e0
        pos = e1
    assert pos == n


@pytest.mark.parametrize("seed", range(12))
def test_partition_is_optimal_and_covers_in_order(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 9))
    nparts = int(rng.integers(1, 5))
    costs = list(np.exp(rng.uniform(0, 4, n)))
    ranges = shard.partition_contiguous(costs, nparts)
    _check_ranges(ranges, n, nparts)
    worst = max(sum(costs[e0:e1]) for e0, e1 in ranges)
    assert worst <= _brute_best(costs, nparts) * (1 + 1e-9)
    # every part used while there are items for it
    assert sum(1 for e0, e1 in ranges if e1 > e0) == min(n, nparts)


def test_partition_edge_cases():
    assert shard.partition_contiguous([], 3) == [(0, 0)] * 3
    assert shard.partition_contiguous([5.0], 2) == [(0, 1), (1, 1)]
    assert shard.partition_contiguous([1.0, 1.0, 1.0, 1.0], 2) == [(0, 2), (2, 4)]
    # one dominant item stands alone
    assert shard.partition_contiguous([1.0, 100.0, 1.0], 3) == [(0, 1), (1, 2), (2, 3)]
    # zero costs still spread over the parts
    r = shard.partition_contiguous([0.0] * 5, 2)
    _check_ranges(r, 5, 2)
    assert all(e1 > e0 for e0, e1 in r)
    with pytest.raises(ValueError):
        shard.partition_contiguous([1.0], 0)
    with pytest.raises(ValueError):
        shard.partition_contiguous([-1.0], 1)
    with pytest.raises(ValueError):
        shard.rank_range([1.0, 2.0], 2, 2)


def test_costs_follow_the_model_and_balance_the_batched_workload():
    w = inputs.batched_events(16, seed=1002)
    shapes = [(sp.nwires, sp.nticks) for sp in w.planes]
    costs = shard.event_costs(shapes, w.events)
    e = w.events[3]
    want = sum(shard.CELL_COST * nw * nt + shard.DEPO_COST * d.n for (nw, nt), d in zip(shapes, e))
    assert costs[3] == pytest.approx(want, rel=1e-12)
    for nparts in (2, 4, 8):
        ranges = shard.partition_contiguous(costs, nparts)
        parts = [sum(costs[a:b]) for a, b in ranges]
        # no range above the optimum's bound: the largest single event or an
        # even share plus one event
        assert max(parts) <= max(max(costs), sum(costs) / nparts + max(costs)) * (1 + 1e-12)
    assert shard.units_of([(0, 2), (2, 3)], 3) == [0] * 6 + [1] * 3
    with pytest.raises(ValueError):
        shard.event_costs(shapes[:2], w.events)


# ------------------------------------------------------- two gloo ranks
NW, NT = 24, 400
NPL = 2
NEV = 5


def _events():
    evs = []
    for e in range(NEV):
        n = 20 + 35 * e
        evs.append([inputs.uniform_depos(n, NW, seed=300 + 10 * e + p, nticks=NT) for p in range(NPL)])
    return evs


def _unit(oracle, ev, e, p, R):
    d = ev[p]
    return oracle.simulate(d.q, d.x_mm, d.t_us, NW, NT, R, 10, fluctuate=True, p=0.7, seed=77,
                           event_id=e, plane_id=p)


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2203_02479_gb300 import inputs as inp, shard as sh
    dist.init_process_group("gloo", rank=rank, world_size=world)
    evs = _events()
    R = inp.response("bipolar")
    shapes = [(NW, NT)] * NPL
    costs = sh.event_costs(shapes, evs)
    ranges = sh.partition_contiguous(costs, world)
    e0, e1 = sh.rank_range(costs, world, rank)
    assert (e0, e1) == ranges[rank]
    # this rank's units, each keyed by its global event id
    mine = [torch.from_numpy(_unit(oracle, evs[e], e, p, R).astype(np.float32))
            for e in range(e0, e1) for p in range(NPL)]
    got = sh.gather_units(dist, mine, ranges, NPL, shapes, dst=0)
    if rank == 0:
        want = [_unit(oracle, evs[e], e, p, R).astype(np.float32) for e in range(NEV) for p in range(NPL)]
        ok = len(got) == len(want) and all(np.array_equal(g.numpy(), w) for g, w in zip(got, want))
        q.put((rank, ranges, ok, len(got)))
    else:
        q.put((rank, ranges, got is None, len(mine)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_and_gather():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ranges0, ok0, n0), (r1, ranges1, ok1, n1) = res
    assert ranges0 == ranges1
    _check_ranges(ranges0, NEV, 2)
    assert all(e1 > e0 for e0, e1 in ranges0)
    assert ok0 and n0 == NEV * NPL          # rank 0 holds every unit, in order
    assert ok1 and n1 == (ranges0[1][1] - ranges0[1][0]) * NPL


def test_depo_and_wire_slices():
    from paper_2203_02479_gb300 import shard as sh
    for n, k in ((0, 1), (1, 3), (10, 3), (1000, 7), (7, 7)):
        s = sh.depo_slices(n, k)
        assert len(s) == k and s[0][0] == 0 and s[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(s, s[1:]))
        sizes = [b - a for a, b in s]
        assert max(sizes) - min(sizes) <= 1
    assert sh.wire_bands(800, 4) == [(0, 200), (200, 400), (400, 600), (600, 800)]
    with pytest.raises(ValueError):
        sh.depo_slices(5, 0)


SPLIT_NW, SPLIT_NT = 24, 600


def _split_main(rank, world, port, q, mode):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2203_02479_gb300 import inputs as inp, shard as sh, wiresim
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = inp.uniform_depos(500, SPLIT_NW, seed=61, nticks=SPLIT_NT)
    R = inp.response("unipolar")
    params = wiresim.Params(fluctuate=1, p_survive=0.7, seed=5, event_id=9)
    kw = dict(fluctuate=1, p=0.7, seed=5, event_id=9, plane_id=2)

    def sim(plane, qq, xx, tt, p):   # one slice by the oracle, keyed by the slice's offset
        return torch.from_numpy(oracle.simulate(qq, xx, tt, SPLIT_NW, SPLIT_NT, R, 10, depo_offset=p.depo_offset,
                                                **kw))
    whole = oracle.simulate(d.q, d.x_mm, d.t_us, SPLIT_NW, SPLIT_NT, R, 10, **kw)
    if mode == "all":
        M = sh.simulate_depo_split(dist, None, d, params, simulate=sim).numpy()
        ok = np.allclose(M, whole, rtol=0, atol=1e-9 * np.abs(whole).max())
    else:
        band, (w0, w1) = sh.simulate_depo_split(dist, None, d, params, scatter=True, simulate=sim)
        ok = (w0, w1) == sh.wire_bands(SPLIT_NW, world)[rank] and \
            np.allclose(band.numpy(), whole[w0:w1], rtol=0, atol=1e-9 * np.abs(whole).max())
    q.put((rank, bool(ok)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["all", "scatter"])
def test_two_gloo_ranks_split_one_plane_by_depos(mode):
    """A plane's depos over two ranks: each simulates its slice (the oracle,
    random draws keyed by the depos' indices in the whole list), the
    waveforms are summed across ranks, and the sum is the whole list's
    waveform (all-reduce: on every rank; reduce-scatter: a band of wire
    rows each)."""
    import torch.distributed as dist
    if mode == "scatter" and not dist.is_available():
        pytest.skip("torch.distributed unavailable")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_main, args=(r, 2, port, q, mode)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, True), (1, True)]
