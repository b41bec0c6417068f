"""Exact merge of sampling runs across ranks.

Samples are keyed by id, so ranks that draw disjoint id ranges of one seed
produce partial integer sums whose total is the single-run result.  The only
exchange is an all-reduce of those integers; values up to 128 bits are split
into 32-bit limbs so that int64 tensor sums stay exact for any world size
below 2^31.  The estimate of the merged sums is formed by the library
(tc_estimate_from_sums), the same arithmetic as a single run's.
"""
import torch
import torch.distributed as dist

from . import tc

_LIMBS = 4


def allreduce_exact(values, group=None, device="cpu"):
    """Sum non-negative Python ints (< 2^128) over all ranks, exactly."""
    limbs = []
    for v in values:
        v = int(v)
        if v < 0 or v >> (32 * _LIMBS):
            raise ValueError("value out of range")
        limbs += [(v >> (32 * i)) & 0xFFFFFFFF for i in range(_LIMBS)]
    t = torch.tensor(limbs, dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    t = t.cpu().tolist()
    return [sum(int(t[_LIMBS * j + i]) << (32 * i) for i in range(_LIMBS)) for j in range(len(values))]


def merge_runs(local, W, group=None, device="cpu"):
    """Merge this rank's run {sum_x, sum_x2, hits, k} into the global
    estimate of Alg. 5 (C_hat = sum_x * W / k) and its standard error."""
    sx, sx2, hits, k = allreduce_exact([local["sum_x"], local["sum_x2"], local["hits"], local["k"]], group, device)
    est, se = tc.tc_estimate_from_sums(sx, sx2, k, W)
    return {"sum_x": sx, "sum_x2": sx2, "hits": hits, "k": k, "W": int(W), "estimate": est, "std_err": se}


def merge_batch(local, group=None, device="cpu"):
    """Merge this rank's per-query runs (a list of {sum_x, sum_x2, hits, k,
    W}, as tc_batch_run returns) into per-query global estimates with one
    all-reduce; every rank must hold the same queries (W is per query and
    the same on every rank)."""
    vals = []
    for r in local:
        vals += [r["sum_x"], r["sum_x2"], r["hits"], r["k"]]
    tot = allreduce_exact(vals, group, device) if vals else []
    out = []
    for j, r in enumerate(local):
        sx, sx2, hits, k = tot[4 * j:4 * j + 4]
        est, se = tc.tc_estimate_from_sums(sx, sx2, k, r["W"])
        out.append({"sum_x": sx, "sum_x2": sx2, "hits": hits, "k": k, "W": int(r["W"]), "estimate": est,
                    "std_err": se})
    return out


def rank_range(k_total, rank, world):
    """Sample-id range [offset, offset + count) of a rank."""
    base, extra = divmod(int(k_total), int(world))
    offset = rank * base + min(rank, extra)
    return offset, base + (1 if rank < extra else 0)
