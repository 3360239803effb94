"""Host logic of the multi-rank path, on the CPU with two gloo ranks: the
assignment of independent lattices to ranks, the max-over-ranks timing and
summed counters, and that sharded results equal single-process results."""
import json
import socket

import numpy as np
import pytest

from paper_2512_01032_gb300 import shard
from tests import _gloo_worker as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_assign_partitions_and_balances():
    rng = np.random.Generator(np.random.PCG64(7))
    cells = [int(v) for v in rng.integers(1, 1000, size=37)]
    for world in (1, 2, 3, 8):
        parts = shard.assign(cells, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(cells)))
        loads = [sum(cells[i] for i in p) for p in parts]
        # largest-first greedy: no rank exceeds the mean by more than the largest item
        assert max(loads) <= sum(cells) / world + max(cells)
        assert parts == shard.assign(cells, world)  # deterministic
    assert shard.assign([5, 5], 4)[2:] == [[], []]
    assert shard.assign([], 3) == [[], [], []]
    # equal sizes: lowest index to the least-loaded rank, ties to the lowest rank
    assert shard.assign([4, 4, 4], 2) == [[0, 2], [1]]
    assert shard.my_items([4, 4, 4], 1, 2) == [1]
    with pytest.raises(ValueError):
        shard.my_items([4], 2, 2)
    with pytest.raises(ValueError):
        shard.assign(cells, 0)


def test_reductions_without_process_group_are_identity():
    assert shard.reduce_max([1.5, 2.0]) == [1.5, 2.0]
    assert shard.reduce_sum([3.0]) == [3.0]
    assert shard.gather({"a": 1}) == [{"a": 1}]


def test_two_gloo_ranks_match_one_process(tmp_path):
    import torch.multiprocessing as mp
    out = tmp_path / "rank0.json"
    mp.spawn(W.rank_main, args=(2, _free_port(), str(out)), nprocs=2, join=True)
    got = json.loads(out.read_text())
    specs = W.lattice_specs()
    cells = [a * b * c for a, b, c, _ in specs]
    assert got["n_sum"] == len(specs) and got["cells_sum"] == sum(cells)
    assert got["probe_max"] == 2.0
    assert got["t_max"] >= got["t_rank0"]
    assert got["owned"] == shard.assign(cells, 2)
    for i, spec in enumerate(specs):
        want = W.run_item(spec)
        assert got["results"][str(i)] == want  # same oracle, one thread: bitwise
    lat_all = sorted(0.5 + 0.37 * k for k in range(23))
    assert got["merged"] == lat_all
    assert got["p50"] == shard.nearest_rank(lat_all, 0.5) == lat_all[11]
    assert got["p99"] == shard.nearest_rank(lat_all, 0.99) == lat_all[22]


def test_nearest_rank_percentiles():
    v = [1.0, 2.0, 3.0, 4.0]
    assert shard.nearest_rank(v, 0.5) == 2.0
    assert shard.nearest_rank(v, 0.99) == 4.0
    assert shard.nearest_rank(v, 0.01) == 1.0
    assert shard.nearest_rank([], 0.5) == 0.0
    assert shard.merged_sorted([3, 1, 2]) == [1.0, 2.0, 3.0]  # no process group: local
