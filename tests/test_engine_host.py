"""Host logic of the search / rolling-prune schedule (engine.py) on a fake
pair list, no GPU.

The fake moves every atom by a * sqrt(frames since the search) (a random
walk's growth), sets the device's stale-list error bits when the kernels
would (a prune on a frame displaced more than (rlist - r_inner)/2 since the
search, a force call displaced more than (r_inner - rc)/2 since the prune),
and answers both the synchronising tracker read and the queued copy.
"""
import math

import numpy as np
import pytest
import torch

from paper_2405_01420_gb300 import nb
from paper_2405_01420_gb300.engine import NonbondedEngine

RC, R_INNER, RLIST = 1.0, 1.04, 1.1


class FakePairlist:
    def __init__(self, a_search: float, a_prune: float | None = None, fail_at: int | None = None):
        self.a_s = a_search
        self.a_p = a_search if a_prune is None else a_prune
        self.fail_at = fail_at
        self.frame = 0  # frames evaluated so far; the coming coordinates are frame `frame`
        self.f_search = None
        self.f_prune = None
        self.err = 0
        self.last = (0.0, 0.0)
        self.log = []
        self.sync_reads = 0

    def disp_search(self, f):
        return self.a_s * math.sqrt(f - self.f_search)

    def disp_prune(self, f):
        return self.a_p * math.sqrt(f - self.f_prune)

    def search(self, coords, box, rlist, eo, ei, stream):
        self.f_search = self.frame
        self.f_prune = self.frame
        self.log.append(("search", self.frame))

    def prune(self, coords, r_inner, stream):
        if self.disp_search(self.frame) > 0.5 * (RLIST - R_INNER):
            self.err |= nb.NB_DEV_STALE_SEARCH
        self.f_prune = self.frame
        self.log.append(("prune", self.frame))

    def forces(self, coords, q, t, lj, rc, beta, F, E, want_energy, stream):
        if self.disp_prune(self.frame) > 0.5 * (R_INNER - RC):
            self.err |= nb.NB_DEV_STALE_PRUNE
        if self.fail_at is not None and self.frame == self.fail_at:
            self.err |= nb.NB_DEV_NONFINITE
        self.last = (self.disp_search(self.frame), self.disp_prune(self.frame))
        self.frame += 1
        return None, None

    def stats(self, stream=None):
        self.sync_reads += 1
        return {"error_word": self.err, "max_disp_search": self.last[0], "max_disp_prune": self.last[1]}

    def tracker_enqueue(self, words, stream=None):
        d2 = np.array([self.last[0] ** 2, self.last[1] ** 2], np.float32)
        words[0] = int(np.int32(np.uint32(self.err)))
        words[1:3] = torch.from_numpy(d2.view(np.int32))

    def status(self, clear=False, stream=None):
        return self.err

    def close(self):
        pass


def run(fake, evals, lag, interval=10):
    eng = NonbondedEngine(100, [3.0, 3.0, 3.0], RC, 3.0, RLIST, R_INNER, interval, lag=lag, pairlist=fake)
    for _ in range(evals):
        eng.compute(None, None, None, None)
    return eng


@pytest.mark.parametrize("a", [0.001, 0.003, 0.005])
def test_queued_reads_keep_every_list_complete(a):
    fake = FakePairlist(a)
    eng = run(fake, 300, lag=2)
    assert fake.err == 0
    assert eng.check() == 0
    assert eng.n_sync_reads == 0 and fake.sync_reads == 0, "a prune point drained the stream"


@pytest.mark.parametrize("a", [0.003, 0.005])
def test_queued_reads_search_about_as_often_as_synchronous_ones(a):
    sync = run(FakePairlist(a), 300, lag=0)
    late = run(FakePairlist(a), 300, lag=2)
    assert sync.n_sync_reads > 0
    assert abs(late.n_search - sync.n_search) <= 1
    assert late.n_prune >= sync.n_prune - 1


def test_tracker_words_decode():
    w = torch.zeros(3, dtype=torch.int32)
    FakePairlist(0.0).tracker_enqueue(w)
    d = nb.decode_tracker(w.numpy())
    assert d == {"error_word": 0, "max_disp_search": 0.0, "max_disp_prune": 0.0}
    f = FakePairlist(0.004)
    f.search(None, None, None, None, None, None)
    for _ in range(9):
        f.forces(None, None, None, None, None, None, None, None, True, None)
    f.err = 0x80000001
    f.tracker_enqueue(w)
    d = nb.decode_tracker(w.numpy())
    assert d["error_word"] == 0x80000001
    assert d["max_disp_search"] == pytest.approx(0.004 * math.sqrt(8), rel=1e-6)


def test_an_error_bit_raises_at_a_later_prune_point():
    fake = FakePairlist(0.001, fail_at=23)
    with pytest.raises(nb.NBError, match="error word"):
        run(fake, 60, lag=2)
    # seen at the first prune point whose queued copy follows frame 23: the copy after frame 27
    assert fake.frame <= 31


def test_fast_prune_displacement_shortens_the_interval():
    # the search budget holds for long, but atoms leave the prune buffer quickly
    fake = FakePairlist(0.0005, a_prune=0.0065)
    eng = run(fake, 100, lag=2)
    assert eng.interval < 10
    assert fake.err & nb.NB_DEV_STALE_PRUNE == 0


def test_short_intervals_fall_back_to_synchronous_reads():
    fake = FakePairlist(0.001)
    eng = run(fake, 30, lag=2, interval=2)
    assert eng.n_sync_reads > 0 and fake.err == 0


def test_the_probe_shortens_the_first_interval_for_fast_dynamics():
    # atoms leave the prune buffer (0.02 nm) after 7 frames: interval 10 would go stale at once
    fake = FakePairlist(0.0075)
    eng = run(fake, 200, lag=2)
    assert fake.err == 0, hex(fake.err)
    assert eng.interval <= 6


def test_slow_dynamics_keep_the_interval():
    fake = FakePairlist(0.001)
    eng = run(fake, 200, lag=2)
    assert eng.interval == 10 and fake.err == 0


class NoisyFake(FakePairlist):
    """The largest displacement over many atoms fluctuates from frame to frame."""

    def __init__(self, a, seed=0):
        super().__init__(a)
        self.rng = np.random.default_rng(seed)

    def forces(self, *args):
        out = super().forces(*args)
        k = 1.0 + 0.15 * self.rng.random()
        self.last = (self.last[0] * k, self.last[1] * k)
        return out


@pytest.mark.parametrize("seed", range(5))
def test_noisy_maxima_keep_the_interval_and_the_queued_reads(seed):
    fake = NoisyFake(0.0088, seed)
    eng = run(fake, 200, lag=2)
    assert fake.err == 0
    assert 3 <= eng.interval <= 5
    assert eng.n_sync_reads <= eng.n_search
