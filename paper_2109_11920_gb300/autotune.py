"""Autotuner for the launch shape of the fused MLEM kernel, per size class.

For every size class of a ragged batch it times each launch configuration
(CTAs of 2n / 4n / 8n threads, four or two views per sample grid) on that
class's own candidates with a few MLEM iterations, and keeps the fastest.
Results are memoised per (GPU, image side, views, candidate count) for the
life of the process, and can be saved to / loaded from a JSON file.
"""
from __future__ import annotations

import json
import os

import torch

from . import api
from ._lib import BoacError

_CACHE: dict[tuple, int] = {}


def _key(g, count, device) -> tuple:
    return (torch.cuda.get_device_name(device), int(g.n), int(g.n_views), int(count))


def _time_config(sub: "api.RaggedBatch", cfg: int, repeats: int) -> float:
    try:
        sub.prepare([cfg])
        sub.run()  # warm-up
    except (BoacError, ValueError):
        return float("inf")
    st = torch.cuda.current_stream(sub.device)
    best = float("inf")
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        sub.run()
        b.record(st)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_ragged(batch: "api.RaggedBatch", probe_iters: int = 3, repeats: int = 2,
                verbose: bool = False) -> list[int]:
    """Fastest configuration id per size class of ``batch`` (see RaggedBatch)."""
    configs = []
    cls_of = [batch.cands[b].cls for b in range(batch.B)]
    for c, g in enumerate(batch.classes):
        members = [b for b in range(batch.B) if cls_of[b] == c]
        if not members:  # unused class: any valid id will do
            configs.append(0 if g.n_views % 4 == 0 else 1)
            continue
        key = _key(g, len(members), batch.device)
        if key in _CACHE:
            configs.append(_CACHE[key])
            continue
        mus, Ss = [], []
        for b in members:
            d = batch.cands[b]
            mus.append(batch.mu_pool[d.mu_off:d.mu_off + g.n * g.n].view(g.n, g.n))
            Ss.append(batch.S_pool[d.S_off:d.S_off + g.n_views * g.n_bins].view(g.n_views, g.n_bins))
        sub = api.RaggedBatch([g], [0] * len(members), [probe_iters] * len(members), mus, Ss,
                              device=batch.device)
        times = {cfg: _time_config(sub, cfg, repeats) for cfg in range(api.N_CONFIGS)
                 if api.config_valid(g, cfg)}
        best = min(times, key=times.get)
        if times[best] == float("inf"):
            raise RuntimeError(f"no launch configuration runs for class {g}")
        if verbose:
            print(f"class {g}: " + ", ".join(f"{k}:{v:.3f}ms" for k, v in sorted(times.items())))
        _CACHE[key] = best
        configs.append(best)
    return configs


def save(path: str) -> None:
    with open(path, "w") as fh:
        json.dump([list(k) + [v] for k, v in _CACHE.items()], fh, indent=1)


def load(path: str) -> None:
    if not os.path.exists(path):
        return
    with open(path) as fh:
        for row in json.load(fh):
            _CACHE[tuple(row[:-1])] = int(row[-1])
