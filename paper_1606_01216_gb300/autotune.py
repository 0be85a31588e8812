"""Schedule autotuner for batched solves (airga_batch_*).

The batched launch needs two choices the library cannot know in advance:
the rows each CTA of a system's group owns (small groups mean fewer barrier
participants and more systems side by side; large groups finish one system
sooner) and the cost of each system (rows x CG iterations decides the list
schedule).  The tuner measures instead of guessing:

  1. plan with cost = rows and the default rows per CTA, solve once, read the
     CG iterations of every system;
  2. for each candidate rows-per-CTA, plan with cost = rows x iterations and
     time the solve on the device (CUDA events, best of `reps`);
  3. keep the fastest plan.

All timing goes through the C ABI; the tuner holds no compute of its own.
"""
from __future__ import annotations

import torch

from . import airga as G

DEFAULT_CANDIDATES = (512, 1024, 2048, 4096, 8192)


def _time_solve(batch, stream, reps):
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.solve(stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(systems, opts=None, candidates=DEFAULT_CANDIDATES, reps=2, stream=None):
    """Return (best Batch, report).  systems: list of (A, P, f, x)."""
    stream = stream or torch.cuda.current_stream()
    first = G.Batch(systems, opts=opts, stream=stream)
    first.solve(stream=stream)
    torch.cuda.synchronize()
    iters = first.iters.cpu().tolist()
    cost = [float(s[0].n) * max(1, it) for s, it in zip(systems, iters)]
    del first
    report = []
    best, best_ms = None, float("inf")
    for rows in candidates:
        b = G.Batch(systems, opts=opts, cost=cost, rows_per_cta=rows, stream=stream)
        ms = _time_solve(b, stream, reps)
        info = b.info()
        report.append(dict(rows_per_cta=rows, ms=round(ms, 4), rows_max=info["rows_max"],
                           est_makespan=info["makespan"]))
        if ms < best_ms:
            best, best_ms = b, ms
        else:
            del b
    return best, dict(candidates=report, best_rows_per_cta=best.info()["rows_target"],
                      best_ms=round(best_ms, 4))
