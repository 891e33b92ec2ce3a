"""The multi-rank path on CPU: world_size 2 with the gloo backend.

Each rank owns a contiguous range of trajectory indices (no data exchange);
the ranks' statistics are merged with all_gather_object and Chan's formula.
The per-trajectory results come from the oracle here (no GPU in this test);
the merge must equal the statistics of the whole index range at once."""
import os
import socket

import numpy as np
import pytest

from paper_2212_02197_gb300 import shards, workloads as W

T_PER_RANK = 6
EDGES = (0.0, 20.0, 16)


def local_stats(r):
    phi = r["phi"]
    fin = phi[np.isfinite(phi)]
    h, _ = np.histogram(np.clip(fin, EDGES[0], np.nextafter(EDGES[1], 0)), bins=EDGES[2],
                        range=EDGES[:2])
    return {"n_traj": len(phi), "phi_mean": float(fin.mean()),
            "phi_var": float(fin.var(ddof=1)) if len(fin) > 1 else 0.0,
            "phi_min": float(fin.min()), "phi_max": float(fin.max()),
            "n_nonfinite": int((~np.isfinite(phi)).sum()),
            "n_ocp_failed": int(r["n_ocp_failed"].sum()), "sqp_iters": int(r["sqp_iters"].sum()),
            "ls_trials": int(r["ls_trials"].sum()), "n_ocp": int(r["n_ocp"].sum()),
            "hist": h, "bin_lo": EDGES[0], "bin_hi": EDGES[1]}


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=24)
    j0, j1 = shards.shard_range(rank, T_PER_RANK)
    r = oracle.run(m, w["nmpc"], w["seed"], j0, j1, threads=1)
    merged = shards.allgather_stats(local_stats(r), dist)
    if rank == 0:
        q.put({k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in merged.items()})
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_merge_equals_whole_range():
    import torch.multiprocessing as mp

    import oracle

    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    merged = q.get()
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=24)
    whole = local_stats(oracle.run(m, w["nmpc"], w["seed"], 0, 2 * T_PER_RANK, threads=2))
    assert merged["n_traj"] == whole["n_traj"] == 2 * T_PER_RANK
    assert merged["phi_mean"] == pytest.approx(whole["phi_mean"], rel=1e-12)
    assert merged["phi_var"] == pytest.approx(whole["phi_var"], rel=1e-10)
    assert merged["phi_min"] == whole["phi_min"] and merged["phi_max"] == whole["phi_max"]
    assert np.array_equal(merged["hist"], whole["hist"])
    for k in ("n_ocp_failed", "sqp_iters", "ls_trials", "n_ocp"):
        assert merged[k] == whole[k]


def test_ranges_partition_the_indices():
    for n in (0, 1, 7, 30000):
        for world in (1, 2, 3, 8):
            got = [shards.split_range(n, world, r) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            for a, b in zip(got, got[1:]):
                assert a[1] == b[0]
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1
    assert shards.shard_range(3, 100) == (300, 400)


def test_merge_rejects_mismatched_histograms():
    a = {"n_traj": 2, "phi_mean": 1.0, "phi_var": 0.5, "phi_min": 0.5, "phi_max": 1.5,
         "hist": np.array([1, 1]), "bin_lo": 0.0, "bin_hi": 2.0}
    b = dict(a, bin_hi=3.0)
    with pytest.raises(ValueError):
        shards.merge_stats([a, b])
