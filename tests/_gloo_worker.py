"""Rank body of the two-process sharding test (spawned, gloo on CPU): each
rank advances its own share of small independent lattices with the oracle
and the ranks combine timings and results only on the host."""
import json
import os
import time


def lattice_specs():
    """Small uneven periodic droplet lattices (nx, ny, nz, R)."""
    return [(12, 10, 8, 3.0), (16, 12, 10, 4.0), (8, 8, 8, 2.5), (14, 14, 6, 2.0),
            (10, 16, 12, 3.5), (9, 11, 13, 3.0), (20, 8, 8, 2.5)]


def run_item(spec, steps=6):
    import oracle as O
    import synth
    nx, ny, nz, R = spec
    p = synth.static_droplet_params()
    op = {k: v for k, v in p.items() if k in ("sigma", "W", "M", "rho_H", "rho_L", "nu_H", "nu_L")}
    L = O.OracleLattice(nx, ny, nz, nthreads=1, **op)
    c = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    L.init_phi(O.tanh_phi(0, (nx, ny, nz), c, R, p["W"]))
    L.step(steps)
    m = L.macros()
    return {"mass": float(m["phi"].sum()), "p_max": float(m["P"].max())}


def rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    from paper_2512_01032_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        specs = lattice_specs()
        cells = [a * b * c for a, b, c, _ in specs]
        mine = shard.my_items(cells, rank, world)
        t0 = time.perf_counter()
        res = {i: run_item(specs[i]) for i in mine}
        dt = time.perf_counter() - t0
        t_max, = shard.reduce_max([dt])
        n_sum, cells_sum = shard.reduce_sum([len(mine), sum(cells[i] for i in mine)])
        probe_max, = shard.reduce_max([rank + 1.0])
        allres = shard.gather(res)
        # serving statistics over ranks: each rank holds its requests' latencies
        lat_all = [0.5 + 0.37 * k for k in range(23)]
        mine_lat = [v for k, v in enumerate(lat_all) if k % world == rank]
        lat_merged = shard.merged_sorted(mine_lat)
        p50, p99 = shard.nearest_rank(lat_merged, 0.5), shard.nearest_rank(lat_merged, 0.99)
        if rank == 0:
            merged = {}
            for r in allres:
                for k, v in r.items():
                    assert k not in merged, "item computed twice"
                    merged[k] = v
            with open(out_path, "w") as f:
                json.dump({"results": {str(k): v for k, v in merged.items()},
                           "t_max": t_max, "t_rank0": dt, "n_sum": n_sum,
                           "cells_sum": cells_sum, "probe_max": probe_max,
                           "owned": [shard.my_items(cells, r, world) for r in range(world)],
                           "merged": lat_merged, "p50": p50, "p99": p99},
                          f)
        dist.barrier()
    finally:
        dist.destroy_process_group()
