"""Event sharding across GPUs and the exact merge of the per-shard results.

Events are independent and the smearing is keyed by the global event id
(Philox counter = (block, variation, event id)), so a chunk split into
contiguous event ranges, one per rank, gives per-event results that do not
depend on the split.  The only exchange is at the end: integer sums of the
cut flows, histograms and recheck counts, and the concatenation of the
per-event outputs (mask, surviving variations, reconstructed quantities, the
chosen variation of best-of-variations) in rank order.  Uses torch.distributed with whatever backend the process group has
(NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np


def shard_range(n_events: int, rank: int, world: int):
    """Contiguous [lo, hi) of rank `rank` out of `world` (sizes differ by at most one)."""
    base, rem = divmod(int(n_events), int(world))
    lo = rank * base + min(rank, rem)
    hi = lo + base + (1 if rank < rem else 0)
    return lo, hi


def merge_results(res: dict, group=None, device="cpu") -> dict:
    """Merges one rank's results (numpy arrays as returned by Engine.fetch or
    DeviceResults.numpy) with every other rank's.  Returns the merged dict on
    every rank: cutflow, hist and recheck_count summed exactly (int64), mask,
    n_surv, reco and (best-of-variations) best_v concatenated in rank order."""
    import torch
    import torch.distributed as dist
    out = {}
    for k in ("cutflow", "hist"):
        if k in res:
            t = torch.from_numpy(np.asarray(res[k]).astype(np.int64)).to(device)
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            out[k] = t.cpu().numpy().astype(np.uint64)
    if "recheck_count" in res:
        t = torch.tensor([int(np.asarray(res["recheck_count"]).sum())], dtype=torch.int64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        out["recheck_count"] = int(t.item())
    world = dist.get_world_size(group)
    n_local = len(res["mask"]) if "mask" in res else 0
    sizes = torch.tensor([n_local], dtype=torch.int64, device=device)
    all_sizes = [torch.zeros_like(sizes) for _ in range(world)]
    dist.all_gather(all_sizes, sizes, group=group)
    all_sizes = [int(x.item()) for x in all_sizes]
    nmax = max(all_sizes) if all_sizes else 0
    for k, dtype, width in (("mask", np.uint8, 1), ("n_surv", np.uint16, 1), ("reco", np.float32, 4),
                            ("best_v", np.uint16, 1)):
        if k not in res:
            continue
        a = np.asarray(res[k], dtype=dtype).reshape(n_local, width)
        # gather as int32 / float32 (gloo lacks some small integer types), padded to the largest shard
        td = torch.float32 if dtype == np.float32 else torch.int32
        pad = torch.zeros((nmax, width), dtype=td, device=device)
        pad[:n_local] = torch.from_numpy(a.astype(np.float32 if td == torch.float32 else np.int32)).to(device)
        parts = [torch.zeros_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        cat = np.concatenate([p.cpu().numpy()[:n] for p, n in zip(parts, all_sizes)])
        cat = cat.astype(dtype)
        out[k] = cat if width > 1 else cat.reshape(-1)
    return out
