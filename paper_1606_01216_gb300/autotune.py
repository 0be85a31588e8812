"""Schedule autotuner for batched solves (airga_batch_*).

The batched launch needs choices the library cannot know in advance:
  * rows per CTA of a system's group, i.e. how many CTAs a system gets
    (small groups mean fewer barrier participants and more systems side by
    side; large groups finish one system sooner).  The target is capped by
    shared memory: every target at or above the cap (`rows_max` of the
    largest candidate) gives the same plan, which is where the sweep ends;
  * right-hand-side grouping: the systems that share one (A, P) — the
    right-hand sides of one shift — either scheduled one by one wherever CTAs
    free up, or as one job back to back on one CTA group, so that they reuse
    the bands while these sit in L2;
  * CTAs per SM: one CTA slot per SM (sm_share 1), or two with half an SM
    each (sm_share 2), whose systems fill each other's barrier gaps;
  * the cost of each system (rows x CG iterations decides the list schedule).
The tuner measures instead of guessing:

  1. plan with cost = rows and the default rows per CTA, solve once, read the
     CG iterations of every system;
  2. for each (CTAs per SM, rows per CTA, grouping) candidate, plan with cost = rows x
     iterations and time the solve on the device (CUDA events, best of
     `reps`);
  3. keep the fastest plan.

All timing goes through the C ABI; the tuner holds no compute of its own.
"""
from __future__ import annotations

import torch

from . import airga as G

DEFAULT_CANDIDATES = (512, 1024, 2048, 4096, 5120, 6144, 8192)
GROUPING = (False, True)
SHARES = (1, 2)


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


def rhs_groups(systems):
    """Group id per system: systems with the same matrix and preconditioner
    handles (the right-hand sides of one shift) share an id."""
    ids, out = {}, []
    for s in systems:
        key = (s[0].h.value, s[1].h.value if s[1] is not None else 0)
        out.append(ids.setdefault(key, len(ids)))
    return out


def _with_share(opts, share):
    o = G.options()
    if opts is not None:
        for name, _ in G.Options._fields_:
            setattr(o, name, getattr(opts, name))
    o.sm_share = share
    return o


def tune(systems, opts=None, candidates=DEFAULT_CANDIDATES, grouping=GROUPING, reps=2,
         stream=None, shares=SHARES):
    """Return (best Batch, report).  systems: list of (A, P, f, x)."""
    stream = stream or torch.cuda.current_stream()
    first = G.Batch(systems, opts=opts, stream=stream)
    first.solve(stream=stream)
    torch.cuda.synchronize()
    iters = first.iters.cpu().tolist()
    cost = [float(s[0].n) * max(1, it) for s, it in zip(systems, iters)]
    del first
    groups = rhs_groups(systems)
    report = []
    best, best_ms, best_key = None, float("inf"), None
    caps = {}
    for share in shares:
        o = _with_share(opts, share)
        for grouped in grouping:
            prev = None
            for rows in candidates:
                b = G.Batch(systems, opts=o, cost=cost, rows_per_cta=rows, stream=stream,
                            group=groups if grouped else None)
                info = b.info()
                if info["rows_target"] == prev:
                    del b          # past the shared-memory cap: the same plan as the cap
                    continue
                prev = info["rows_target"]
                caps[share] = max(caps.get(share, 0), info["rows_target"])
                ms = _time_solve(b, stream, reps)
                report.append(dict(sm_share=share, rows_per_cta=rows, rhs_grouped=grouped,
                                   ms=round(ms, 4), rows_max=info["rows_max"],
                                   grid=info["grid"], est_makespan=info["makespan"]))
                if ms < best_ms:
                    best, best_ms, best_key = b, ms, (rows, grouped, share)
                else:
                    del b
    return best, dict(candidates=report, best_rows_per_cta=best.info()["rows_target"],
                      best_rhs_grouped=best_key[1], best_sm_share=best_key[2],
                      best_ms=round(best_ms, 4), rows_cap=caps, rhs_groups=max(groups) + 1,
                      note="targets above the shared-memory cap give the cap's plan and are "
                           "not timed again")
