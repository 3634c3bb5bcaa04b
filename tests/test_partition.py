"""The multi-GPU partition on the CPU: the library's row-strip plan and LPT
field split (host arithmetic of the C ABI), and world-size-2 gloo runs in which
each rank evaluates its share with the oracle and the gathered result equals
the single-process one bit for bit.  The partition needs no data exchange, so
the only collectives are the gathers that check it."""

import itertools
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as O
from paper_2510_01190_gb300 import synth


@pytest.fixture(scope="module")
def binding():
    from paper_2510_01190_gb300 import _binding

    try:
        _binding.load()  # build once here, before any child process loads it
    except RuntimeError as e:
        pytest.skip(f"library not buildable here: {e}")
    return _binding


@pytest.mark.parametrize("h", [2, 3, 10, 97, 721])
@pytest.mark.parametrize("n", [1, 2, 3, 8, 16, 800])
def test_strips_cover_every_cell_row_once_with_their_halos(binding, h, n):
    covered = []
    for r in range(n):
        vb, ve, cb, ce = binding.lcp_strip_plan(h, n, r)
        assert 0 <= cb <= ce <= h - 1
        covered.extend(range(cb, ce))
        if cb == ce:
            assert vb == ve
            continue
        assert vb == max(cb - 1, 0) and ve == min(ce + 2, h)
        assert ve - vb >= 2  # a grid of its own
    assert covered == list(range(h - 1))
    sizes = [binding.lcp_strip_plan(h, n, r)[3] - binding.lcp_strip_plan(h, n, r)[2] for r in range(n)]
    assert max(sizes) - min(sizes) <= 1


def test_strip_plan_rejects_bad_arguments(binding):
    with pytest.raises(RuntimeError):
        binding.lcp_strip_plan(1, 2, 0)
    with pytest.raises(RuntimeError):
        binding.lcp_strip_plan(10, 2, 2)
    with pytest.raises(RuntimeError):
        binding.lcp_strip_plan(10, 0, 0)


def _strip_lcp(u, v, iso, n, r, strip):
    """The oracle on one rank's strip, cut to its kept cell rows."""
    vb, ve, cb, ce = strip
    k = len(iso)
    if cb == ce:
        return np.zeros((k, 0, u.shape[2] - 1)), np.zeros((k, 0, u.shape[2] - 1), bool)
    ref = O.lcp_closed_form(u[:, vb:ve], v[:, vb:ve], 1.0, 0.5, iso)
    keep = slice(cb - vb, ce - vb)
    return ref["lcp"][:, keep], ref["mask"][:, keep]


@pytest.mark.parametrize("n", [2, 3, 5])
def test_strips_of_the_oracle_reassemble_the_whole_grid(binding, n):
    """Single process, several strips: the halo makes every kept row exact."""
    d = synth.fourier_ensemble(5, h=23, w=31, m=6, k=3)
    u, v, iso = d["u"], d["v"], d["isovalues"]
    whole = O.lcp_closed_form(u, v, 1.0, 0.5, iso)
    parts = [_strip_lcp(u, v, iso, n, r, binding.lcp_strip_plan(23, n, r)) for r in range(n)]
    assert np.array_equal(np.concatenate([p[0] for p in parts], axis=1), whole["lcp"])
    assert np.array_equal(np.concatenate([p[1] for p in parts], axis=1), whole["mask"])


def test_a_strip_without_its_halo_is_wrong(binding):
    """Positive control: evaluating only the strip's own vertex rows puts a
    one-sided difference where the grid has a central one."""
    d = synth.fourier_ensemble(5, h=23, w=31, m=6, k=3)
    u, v, iso = d["u"], d["v"], d["isovalues"]
    whole = O.lcp_closed_form(u, v, 1.0, 0.5, iso)
    vb, ve, cb, ce = binding.lcp_strip_plan(23, 3, 1)
    bad = O.lcp_closed_form(u[:, cb:ce + 1], v[:, cb:ce + 1], 1.0, 0.5, iso)["lcp"]
    assert not np.array_equal(bad, whole["lcp"][:, cb:ce])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _strip_worker(rank, world, port, ret):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2510_01190_gb300 import _binding

    d = synth.fourier_ensemble(8, h=41, w=37, m=5, k=2)  # every rank builds the same seeded field
    strip = _binding.lcp_strip_plan(41, world, rank)
    lcp, mask = _strip_lcp(d["u"], d["v"], d["isovalues"], world, rank, strip)
    rows = torch.tensor([lcp.shape[1]])
    all_rows = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_rows, rows)
    width = max(int(r) for r in all_rows)
    pad = np.zeros((lcp.shape[0], width, lcp.shape[2]))
    pad[:, :lcp.shape[1]] = lcp
    got = [torch.zeros(pad.shape, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(got, torch.from_numpy(pad))
    padm = np.zeros(pad.shape, np.uint8)
    padm[:, :mask.shape[1]] = mask
    gotm = [torch.zeros(padm.shape, dtype=torch.uint8) for _ in range(world)]
    dist.all_gather(gotm, torch.from_numpy(padm))
    if rank == 0:
        parts = [g.numpy()[:, :int(n)] for g, n in zip(got, all_rows)]
        partm = [g.numpy()[:, :int(n)].astype(bool) for g, n in zip(gotm, all_rows)]
        whole = O.lcp_closed_form(d["u"], d["v"], 1.0, 0.5, d["isovalues"])
        ret["lcp"] = bool(np.array_equal(np.concatenate(parts, axis=1), whole["lcp"]))
        ret["mask"] = bool(np.array_equal(np.concatenate(partm, axis=1), whole["mask"]))
    dist.barrier()
    dist.destroy_process_group()


def _lpt_worker(rank, world, port, ret):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2510_01190_gb300 import _binding

    g = np.random.Generator(np.random.PCG64(4))
    shapes = [(int(g.integers(4, 16)), int(g.integers(3, 14)), int(g.integers(3, 14))) for _ in range(7)]
    costs = [2 * m * h * w * 4 for (m, h, w) in shapes]
    owner, load = _binding.lcp_lpt_assign(costs, world)
    mine = [i for i in range(len(shapes)) if owner[i] == rank]
    # the plan is the same on every rank
    all_owner = [torch.zeros(len(shapes), dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_owner, torch.tensor(owner))
    sums = []
    for i in mine:
        m, h, w = shapes[i]
        d = synth.fourier_ensemble(20 + i, h=h, w=w, m=m, k=2)
        sums.append((i, float(O.lcp_closed_form(d["u"], d["v"], 1.0, 1.0, d["isovalues"])["lcp"].sum())))
    out = [None] * world
    dist.all_gather_object(out, sums)
    if rank == 0:
        ret["same_plan"] = all(torch.equal(a, all_owner[0]) for a in all_owner)
        got = dict(x for part in out for x in part)
        ref = {}
        for i, (m, h, w) in enumerate(shapes):
            d = synth.fourier_ensemble(20 + i, h=h, w=w, m=m, k=2)
            ref[i] = float(O.lcp_closed_form(d["u"], d["v"], 1.0, 1.0, d["isovalues"])["lcp"].sum())
        ret["fields"] = got == ref
        ret["load"] = load
        ret["costs"] = costs
    dist.barrier()
    dist.destroy_process_group()


def _spawn(target):
    ctx = mp.get_context("spawn")
    ret = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, 2, port, ret)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    return ret


def test_two_ranks_strips_gathered_equal_the_whole_grid(binding):
    ret = _spawn(_strip_worker)
    assert ret["lcp"] and ret["mask"]


def test_two_ranks_lpt_fields_gathered_equal_the_single_process_results(binding):
    ret = _spawn(_lpt_worker)
    assert ret["same_plan"] and ret["fields"]
    assert sum(ret["load"]) == sum(ret["costs"])


def _best_makespan(costs, m):
    best = None
    for assign in itertools.product(range(m), repeat=len(costs)):
        loads = [0] * m
        for c, a in zip(costs, assign):
            loads[a] += c
        best = max(loads) if best is None else min(best, max(loads))
    return best


@pytest.mark.parametrize("m", [2, 3])
def test_lpt_within_grahams_bound_of_the_best_split(binding, m):
    g = np.random.Generator(np.random.PCG64(m))
    for _ in range(25):
        costs = [int(x) for x in g.integers(1, 1000, size=int(g.integers(1, 8)))]
        owner, load = binding.lcp_lpt_assign(costs, m)
        assert sum(load) == sum(costs)
        assert all(load[owner[i]] >= costs[i] for i in range(len(costs)))
        opt = _best_makespan(costs, m)
        assert max(load) <= (4.0 / 3.0 - 1.0 / (3 * m)) * opt + 1e-9


def test_lpt_list_scheduling_bound_and_determinism(binding):
    """Any list schedule ends within total/m + (1 - 1/m) max cost; the plan is
    a function of the costs alone."""
    g = np.random.Generator(np.random.PCG64(9))
    costs = [int(x) for x in g.integers(1, 10 ** 9, size=256)]
    for m in (1, 2, 4, 8):
        owner, load = binding.lcp_lpt_assign(costs, m)
        assert max(load) <= sum(costs) / m + (1 - 1 / m) * max(costs)
        assert binding.lcp_lpt_assign(costs, m) == (owner, load)
    owner, load = binding.lcp_lpt_assign([], 3)
    assert owner == [] and load == [0, 0, 0]
    with pytest.raises(RuntimeError):
        binding.lcp_lpt_assign([5, -1], 2)
