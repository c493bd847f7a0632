"""Autotuner of the batched solver: tile shapes, then the FP32 inner floor.

The batched solver (`msrcg_batch_solve`, one CTA per problem) smooths the
levels it keeps in global memory in one pass over column strips (see
`fused_smooth` in csrc/msrcg_solve.cu).  Its tile shape is the strip width
(output columns per strip) and the smallest level that takes the single pass;
the plain per-half-sweep passes are the alternative.  Which is fastest depends
on the problem sizes, the batch and the GPU, so `tune` times the candidates on
the actual workload and `best` returns the winner recorded for this GPU.

A second stage tunes the floor of the FP32 inner levels (`inner_floor`: an
inner PCG also stops once ||r_k|| < floor ||b_k||) on the winning tile shape:
a candidate qualifies only if every solve converges without the FP64 rerun,
meets the tolerance in its true residual and needs no more outer (level-0)
iterations than the library's 1e-6; the fastest qualifying one wins.  The
FP64 outer PCG keeps the result at the requested tolerance either way.

Records live in `tuned.json` beside this module, keyed by GPU name and a
workload key chosen by the caller; `python -m paper_math_9809043_gb300.tune
--out FILE` tunes the 1024^2 batch, the uneven batch and the 128^3 batch (its
inner floor only: the single pass is 2D) and writes them.
"""
from __future__ import annotations

import json
import os
import statistics
from typing import Dict, List, Optional

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")

# candidate settings (fields of msrcg_opts); the first is the library default
CANDIDATES: List[Dict[str, int]] = [
    {},
    {"plain_sweeps": 1},
    {"fuse_width": 96},
    {"fuse_width": 64},
    {"fuse_min_cells": 262144},
]


# candidate floors of the FP32 inner levels (the first is the library's)
FLOORS: List[float] = [1e-6, 1e-5, 1e-4, 1e-3, 3e-3, 1e-2, 3e-2, 1e-1]


def key_of(cand: Dict[str, int]) -> str:
    return ",".join(f"{k}={v}" for k, v in sorted(cand.items())) or "default"


def load_table(path: str = TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def record(table: dict, gpu: str, workload: str, best: Dict[str, float], times: Dict[str, Optional[float]]) -> dict:
    table.setdefault(gpu, {})[workload] = {"best": best, "ms": times}
    return table


def best(gpu: str, workload: str, path: str = TABLE) -> Optional[Dict[str, int]]:
    """The recorded fastest settings for (gpu, workload), or None."""
    ent = load_table(path).get(gpu, {}).get(workload)
    return dict(ent["best"]) if ent else None


def _time(problems, opts_kw, precision, tol, steps, dev):
    """Mean ms of one batched solve (after a warm-up) and the last stats."""
    import torch

    from . import msrcg as M

    opts = M.default_opts(precision=precision, **opts_kw)
    hs = [M.Hierarchy.from_problem(p, opts, device=dev) for p in problems]
    bs = [h.rhs_for(p) for h, p in zip(hs, problems)]
    M.batch_solve(hs, bs, tol, check=False)
    torch.cuda.synchronize(dev)
    per, sts = [], None
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, sts = M.batch_solve(hs, bs, tol, check=False)
        e1.record()
        torch.cuda.synchronize(dev)
        per.append(e0.elapsed_time(e1))
    del hs, bs
    torch.cuda.empty_cache()
    return statistics.mean(per), sts


def tune(problems, precision: int = 1, tol: float = 1e-8, steps: int = 2,
         candidates: List[Dict[str, int]] = CANDIDATES, floors: List[float] = FLOORS, device=None):
    """Time one batched solve of `problems` per tile-shape candidate, then per
    inner floor on the fastest shape (precision 1); return (fastest settings,
    {candidate key: mean ms})."""
    import torch

    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    base_floor = {"inner_floor": floors[0]} if precision else {}
    times: Dict[str, float] = {}
    for cand in candidates:
        ms, sts = _time(problems, {**base_floor, **cand}, precision, tol, steps, dev)
        if any(s["status"] != 0 for s in sts):
            raise RuntimeError(f"candidate {key_of(cand)} did not converge")
        times[key_of(cand)] = ms
    fastest = dict(min(candidates, key=lambda c: times[key_of(c)]))
    if not precision:
        return fastest, times
    ref_ms, ref = times[key_of(fastest)], None
    _, ref = _time(problems, {**base_floor, **fastest}, precision, tol, 1, dev)
    outer = max(s["iters"][0] for s in ref)
    best_ms, best_floor = ref_ms, floors[0]
    for fl in floors[1:]:
        ms, sts = _time(problems, {**fastest, "inner_floor": fl}, precision, tol, steps, dev)
        ok = all(s["status"] == 0 and s["escalated"] == 0 and s["relres_true"] < tol and s["iters"][0] <= outer
                 for s in sts)
        times[key_of({**fastest, "inner_floor": fl})] = ms if ok else None  # None: did not qualify
        if ok and ms < best_ms:
            best_ms, best_floor = ms, fl
    if best_floor != floors[0]:
        fastest["inner_floor"] = best_floor
    return fastest, times


def _grf_batch(n_problems: int, side: int):
    import numpy as np

    from . import problems as P

    base = P.config_problem(1, scale=side)
    out = []
    for j in range(n_problems):
        rng = np.random.default_rng(1001 * 1000 + j)
        out.append(P.Problem(dim=2, n=base.n, h=base.h, K=base.K, bc=base.bc, gD=base.gD,
                             f=rng.standard_normal(base.N), pbf=base.pbf))
    return out


def _grf3d_batch(n_problems: int, side: int):
    import numpy as np

    from . import problems as P

    base = P.grf3d_problem(side)
    out = []
    for j in range(n_problems):
        rng = np.random.default_rng(1002 * 1000 + j)
        out.append(P.Problem(dim=3, n=base.n, h=base.h, K=base.K, bc=base.bc, gD=base.gD,
                             f=rng.standard_normal(base.N), pbf=base.pbf))
    return out


def main(argv=None) -> int:
    import argparse

    import torch

    from . import problems as P

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--workloads", default="grf1024,uneven256,grf3d128",
                    help="comma-separated subset of grf1024, uneven256, grf3d128")
    args = ap.parse_args(argv)
    gpu = torch.cuda.get_device_name()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    table = load_table(args.out)
    # the single pass is 2D only: the 3D batch tunes the inner floor alone
    work = {"grf1024": lambda: (f"grf1024x{sms}", _grf_batch(sms, 1024), CANDIDATES),
            "uneven256": lambda: ("uneven256", P.batch_problems(256), CANDIDATES),
            "grf3d128": lambda: (f"grf3d128x{sms}", _grf3d_batch(sms, 128), [{}])}
    for name in args.workloads.split(","):
        workload, probs, cands = work[name]()
        fastest, times = tune(probs, candidates=cands)
        record(table, gpu, workload, fastest, times)
        print(workload, key_of(fastest), {k: (round(v, 2) if v is not None else None) for k, v in times.items()},
              flush=True)
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
