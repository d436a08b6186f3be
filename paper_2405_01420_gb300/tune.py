"""Autotuner for the launch shapes and list schedules of the nonbonded path.

What it tunes, by timing the caller's own workload on the GPU:

* the force kernel's launch shape (threads per CTA, list entries staged per
  warp, CTAs per SM; ``nb_set_force_shape``);
* after a prune, the tile form: gathered 4 x 8 tiles computed 32 j atoms at a
  time, or 8 x 8 cluster-pair tiles (``nb_set_flags``);
* for one-shot batches (search + forces), whether to prune the outer list to
  the cutoff before the force call;
* for trajectories, the prune interval and the inner-list margin
  r_inner - rc of the rolling prune (§III-A: the buffered list and the
  "Prune-only kernel"), subject to the displacement checks staying clean.

The cluster size (8) and one warp per i-cluster are fixed by the kernels; the
tunables above are what the kernels expose. Results can be cached in a JSON
file (``NB_TUNE_CACHE`` or an explicit path) keyed by device name and a
workload signature. The selection and caching logic (``select_best``,
``TuneCache``) is plain Python and runs without a GPU.
"""
from __future__ import annotations

import json
import os
import statistics
from typing import Callable, Iterable

FORCE_SHAPES = [(256, 16, 0), (256, 8, 0), (128, 16, 0), (128, 8, 0), (256, 16, 3), (128, 16, 6)]


def select_best(candidates: Iterable, measure: Callable[[object], float | None]) -> tuple[object, dict]:
    """Measure every candidate (lower is better; None = invalid) and return (best, {repr: time})."""
    times = {}
    best, best_t = None, None
    for c in candidates:
        t = measure(c)
        times[repr(c)] = t
        if t is not None and (best_t is None or t < best_t):
            best, best_t = c, t
    if best is None:
        raise RuntimeError("autotuner: no valid candidate")
    return best, times


class TuneCache:
    """JSON file of tuned choices keyed by (device, workload signature)."""

    def __init__(self, path: str | None = None):
        self.path = path if path is not None else os.environ.get("NB_TUNE_CACHE")
        self.data = {}
        if self.path and os.path.exists(self.path):
            with open(self.path) as fh:
                self.data = json.load(fh)

    @staticmethod
    def key(device: str, signature: str) -> str:
        return f"{device}|{signature}"

    def get(self, device: str, signature: str):
        return self.data.get(self.key(device, signature))

    def put(self, device: str, signature: str, value) -> None:
        self.data[self.key(device, signature)] = value
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(self.data, fh, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def _median_ms(fn: Callable[[], None], reps: int) -> float:
    import torch
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def tune_force_shape(pairlist, call: Callable[[], None], reps: int = 7, shapes=FORCE_SHAPES,
                     signature: str | None = None, cache: TuneCache | None = None):
    """Pick the fastest force-kernel launch shape for ``call`` (one nb_forces on ``pairlist``).

    Leaves the pair list set to the chosen shape and returns (shape, times).
    """
    from . import nb
    if cache is not None and signature is not None:
        hit = cache.get(_device_name(), "force_shape|" + signature)
        if hit is not None:
            nb.nb_set_force_shape(pairlist.handle, *hit["shape"])
            return tuple(hit["shape"]), hit["times"]

    def measure(shape):
        nb.nb_set_force_shape(pairlist.handle, *shape)
        call()
        return _median_ms(call, reps)

    best, times = select_best(shapes, measure)
    nb.nb_set_force_shape(pairlist.handle, *best)
    if cache is not None and signature is not None:
        cache.put(_device_name(), "force_shape|" + signature, {"shape": list(best), "times": times})
    return best, times


def tune_tile_form(pairlist, call: Callable[[], None], reps: int = 7, count_pairs: bool = False,
                   sort_lists: bool = True):
    """After a prune: the gathered 4 x 8 tiles or the 8 x 8 cluster-pair tiles,
    whichever makes ``call`` (an nb_forces on ``pairlist``) faster. Leaves the
    pair list set to it and returns ("gathered" | "cluster", times)."""
    def measure(form):
        pairlist.set_flags(count_pairs=count_pairs, sort_lists=sort_lists, cluster_tiles=(form == "cluster"))
        call()
        return _median_ms(call, reps)

    best, times = select_best(["gathered", "cluster"], measure)
    pairlist.set_flags(count_pairs=count_pairs, sort_lists=sort_lists, cluster_tiles=(best == "cluster"))
    return best, times


def tune_batch_prune(search: Callable[[], None], prune: Callable[[], None], forces: Callable[[], None],
                     reps: int = 5):
    """One-shot batches: search + forces, or search + prune + forces. Returns (use_prune, times)."""
    def measure(use_prune):
        def run():
            search()
            if use_prune:
                prune()
            forces()
        run()
        return _median_ms(run, reps)

    return select_best([False, True], measure)


def tune_trajectory(make_engine: Callable[[float, int], object], run_frames: Callable[[object], None],
                    rc: float, intervals=(5, 10, 20), margins=(0.02, 0.04, 0.06), reps: int = 2):
    """Rolling-prune schedule: (prune interval, r_inner - rc) with the lowest time per trajectory.

    ``make_engine(r_inner, interval)`` builds an engine; ``run_frames(engine)``
    runs the trajectory through it. Candidates whose lists went stale (device
    error word set) are rejected.
    """
    def measure(cand):
        interval, margin = cand
        eng = make_engine(rc + margin, interval)
        run_frames(eng)
        if eng.check() != 0:
            eng.close()
            return None
        t = _median_ms(lambda: run_frames(eng), reps)
        ok = eng.check() == 0
        eng.close()
        return t if ok else None

    return select_best([(i, m) for i in intervals for m in margins], measure)
