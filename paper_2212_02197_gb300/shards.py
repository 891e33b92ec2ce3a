"""Trajectory sharding across ranks and the host-side merge of the statistics.

Trajectories are independent and their noise is counter-based, so a study of
T trajectories per rank is split into contiguous index ranges with no data
exchange; only the reduced statistics (count, mean, M2, min, max, counter sums,
histogram) travel, merged by Chan et al.'s pairwise formula.
"""
from __future__ import annotations

import numpy as np

STAT_KEYS = ("n_ocp_failed", "n_ls_fail", "n_hess_reset", "n_nonfinite", "sqp_iters",
             "ls_trials", "qp_iters", "qp_fail", "n_ocp")


def shard_range(rank: int, per_rank: int) -> tuple[int, int]:
    """Weak scaling: rank r owns trajectories r*T .. (r+1)*T - 1."""
    return rank * per_rank, (rank + 1) * per_rank


def split_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Strong scaling: n trajectories in `world` nearly equal contiguous parts."""
    base, extra = divmod(n, world)
    j0 = rank * base + min(rank, extra)
    return j0, j0 + base + (1 if rank < extra else 0)


def merge_stats(parts: list[dict]) -> dict:
    """Merge per-rank statistics dicts (as returned by MonteCarlo.stats()).

    Histograms are added bin by bin and must share their bin edges."""
    out = {"n_traj": 0, "phi_mean": 0.0, "phi_var": 0.0, "phi_min": float("inf"),
           "phi_max": float("-inf")}
    for k in STAT_KEYS:
        out[k] = 0
    n, mean, m2 = 0.0, 0.0, 0.0
    hist, edges = None, None
    for p in parts:
        nf = p["n_traj"] - p.get("n_nonfinite", 0)
        if nf > 0:
            pm2 = p["phi_var"] * (nf - 1) if nf > 1 else 0.0
            if n == 0:
                n, mean, m2 = float(nf), p["phi_mean"], pm2
            else:
                nt = n + nf
                d = p["phi_mean"] - mean
                mean = mean + d * nf / nt
                m2 = m2 + pm2 + d * d * n * nf / nt
                n = nt
            out["phi_min"] = min(out["phi_min"], p["phi_min"])
            out["phi_max"] = max(out["phi_max"], p["phi_max"])
        out["n_traj"] += p["n_traj"]
        for k in STAT_KEYS:
            out[k] += p.get(k, 0)
        if "hist" in p:
            e = (p["bin_lo"], p["bin_hi"], len(p["hist"]))
            if hist is None:
                hist, edges = np.array(p["hist"], dtype=np.int64), e
            else:
                if e != edges:
                    raise ValueError("histograms with different bins cannot be merged")
                hist = hist + np.asarray(p["hist"], dtype=np.int64)
    out["phi_mean"] = mean
    out["phi_var"] = m2 / (n - 1) if n > 1 else 0.0
    if hist is not None:
        out["hist"], out["bin_lo"], out["bin_hi"] = hist, edges[0], edges[1]
    return out


def allgather_stats(local: dict, dist=None) -> dict:
    """Merge the statistics of all ranks of the default process group."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return merge_stats([local])
    parts = [None] * dist.get_world_size()
    payload = {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in local.items()}
    dist.all_gather_object(parts, payload)
    return merge_stats(parts)
