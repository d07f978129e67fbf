"""The FP64 oracle over a whole chunk in spawned host processes (test helper).

The chunk is cut into contiguous slices, each run by oracle.run with its
global event ids (so its smearing is the whole chunk's), and the results are
merged exactly: integer sums of the cut flow and histogram, concatenation of
the per-event outputs.  Processes are spawned, never forked, so that a test
process that already holds a CUDA context can use it."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _run_slice(args):
    an, cols, seed, V, first = args
    import oracle
    return oracle.run(an, cols, seed=seed, V=V, first_event_id=first)


def run(an, cols, *, seed=0, V=1, first_event_id=0, procs=None, pieces=None):
    """Same result as oracle.run(an, cols, ...) (see there)."""
    N = cols.n_events
    procs = procs or os.cpu_count() or 1
    pieces = max(1, min(N, pieces or 4 * procs))
    bounds = np.linspace(0, N, pieces + 1).astype(np.int64)
    jobs = [(an, cols.slice(int(lo), int(hi)), seed, V, first_event_id + int(lo))
            for lo, hi in zip(bounds[:-1], bounds[1:]) if hi > lo]
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(_run_slice, jobs, chunksize=1)
    out = dict(cutflow=sum(p["cutflow"] for p in parts), hist=sum(p["hist"] for p in parts))
    for k in ("mask", "n_surv", "reco", "reco_abs"):
        out[k] = np.concatenate([p[k] for p in parts])
    return out
