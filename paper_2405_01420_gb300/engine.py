"""Search / rolling-prune / force schedule around one pair list.

The paper's MD step re-runs the pair search every few steps and, between
searches, a prune-only kernel that shrinks the buffered list ("pair list
buffer", "Prune-only kernel", §III-A). This driver applies that schedule to a
stream of frames:

* search at the first frame (outer list at ``rlist``) and prune right away
  (inner list at ``r_inner``);
* prune again every ``prune_interval`` frames;
* re-search instead of pruning when the displacement tracker predicts that
  atoms will have moved more than (rlist - r_inner)/2 since the search by the
  time of the prune.

Correctness does not rest on the prediction: the kernels record the largest
displacement since the search and since the prune on every call and set a
sticky device error bit if a list could have missed a pair. The driver
reads that word at every prune point and raises if it is set.

Reading the tracker does not drain the stream: ``lag`` calls before each
prune point the driver enqueues a copy of the tracker into page-locked host
memory (nb_tracker_enqueue) and records an event; at the prune point it
waits for that event, while the last ``lag`` evaluations are still queued
on the GPU, and scales the maxima to the present by the square root of the
elapsed frames (random-walk growth). An error bit set in those last
``lag`` evaluations is seen at the next prune point or by check().

Frames are counted from the list's own frame: after n evaluations since a
search, the last one ran on the frame n - 1 frames after the search frame,
and a prune now would run on the frame n frames after it.

The prune interval adapts to the dynamics, up to ``prune_interval``. A
probe copy queued 3 evaluations after each search (read ``lag`` evaluations
later) and every prune point give the growth of the squared displacement
per frame (the maximum since the search, and since the prune once that
spans 3 frames or more: a maximum over one or two frames is too noisy to
extrapolate); the interval is set so that the displacement predicted for
the last frame before the next prune stays within 0.9 of the prune budget
(r_inner - rc)/2.
"""
from __future__ import annotations

import math

import torch

from . import nb


class _TrackerReader:
    """A tracker copy in page-locked memory and the event that marks it."""

    def __init__(self, pl, stream):
        cuda = torch.cuda.is_available()
        self.pl = pl
        self.stream = stream
        self.words = torch.zeros(3, dtype=torch.int32, pin_memory=cuda)
        self.event = torch.cuda.Event() if cuda else None

    def enqueue(self):
        self.pl.tracker_enqueue(self.words, self.stream)
        if self.event is not None:
            self.event.record(self.stream if self.stream is not None else torch.cuda.current_stream())

    def read(self) -> dict:
        if self.event is not None:
            self.event.synchronize()
        return nb.decode_tracker(self.words.numpy())


class NonbondedEngine:
    def __init__(self, n_atoms: int, box, rc: float, beta: float, rlist: float,
                 r_inner: float | None = None, prune_interval: int = 10, excl_off=None, excl_idx=None,
                 capacity_entries: int = 0, stream=None, count_pairs: bool = False, lag: int = 2,
                 pairlist=None):
        self.n_atoms = int(n_atoms)
        self.box = [float(v) for v in box]
        self.rc = float(rc)
        self.beta = float(beta)
        self.rlist = float(rlist)
        self.r_inner = None if r_inner is None else float(r_inner)
        if self.r_inner is not None and not (self.rc <= self.r_inner <= self.rlist):
            raise ValueError("need rc <= r_inner <= rlist")
        self.prune_interval = max(1, int(prune_interval))
        self.lag = max(0, int(lag))
        self.excl_off = excl_off
        self.excl_idx = excl_idx
        self.stream = stream
        self.pl = pairlist if pairlist is not None else nb.Pairlist(self.n_atoms, capacity_entries, count_pairs)
        self.reader = _TrackerReader(self.pl, stream)
        self.snapshot = None  # (search number, evals since search, evals since prune) of the queued copy
        self.probe_reader = _TrackerReader(self.pl, stream)
        self.probe = None     # (search number, evals since search) of the queued probe copy
        self.evals = 0
        self.evals_since_search = None
        self.evals_since_prune = 0
        self.interval = self.prune_interval
        self.n_search = 0
        self.n_prune = 0
        self.n_sync_reads = 0

    # budgets on the largest atom displacement (nm), as the kernels check them
    def _budget_search(self) -> float:
        r = self.r_inner if self.r_inner is not None else self.rc
        return 0.5 * (self.rlist - r) - 1e-5

    def _budget_prune(self) -> float:
        return 0.5 * (self.r_inner - self.rc) - 1e-5

    PROBE_AT = 3  # evaluations after a search at which the probe copy is queued

    def _fit_interval(self, rate: float):
        """Set the prune interval so that a random walk whose squared
        displacement grows by `rate` per frame stays within 0.9 of the
        prune budget on the last frame before the next prune."""
        if self.r_inner is None or not rate > 0.0:
            return
        m_max = int((0.9 * self._budget_prune()) ** 2 / (1.1 * rate)) + 1
        self.interval = max(1, min(self.prune_interval, m_max))

    def _search(self, coords):
        self.pl.search(coords, self.box, self.rlist, self.excl_off, self.excl_idx, self.stream)
        self.n_search += 1
        self.evals_since_search = 0
        self.snapshot = None
        self.probe = None
        if self.r_inner is not None:
            self._prune(coords)

    def _prune(self, coords):
        self.pl.prune(coords, self.r_inner, self.stream)
        self.n_prune += 1
        self.evals_since_prune = 0

    def _tracker(self):
        """Tracker values and the evaluation counts (since the search, since
        the prune) they were taken at: the queued copy if it belongs to the
        current search, else a synchronising read of the present."""
        snap = self.snapshot
        self.snapshot = None
        if snap is not None and snap[0] == self.n_search and snap[1] >= 1 and snap[2] >= 1:
            return self.reader.read(), snap[1], snap[2]
        self.n_sync_reads += 1
        st = self.pl.stats(self.stream)
        return st, self.evals_since_search, self.evals_since_prune

    def _checkpoint(self) -> bool:
        """Check the tracker; return True if a search is due."""
        st, n_then, m_then = self._tracker()
        bad = st["error_word"]
        if bad:
            raise nb.NBError(nb.NB_ERR_STATE, f"device error word 0x{bad:x} during the last interval")
        # frames since the search / the prune of the values read, and of the coming prune's frame
        fs_then, fp_then = max(1, n_then - 1), m_then - 1
        fs_next = max(1, self.evals_since_search)
        pred = st["max_disp_search"] * math.sqrt(fs_next / fs_then) * 1.05
        rate = st["max_disp_search"] ** 2 / fs_then
        if fp_then >= 3:
            rate = max(rate, st["max_disp_prune"] ** 2 / fp_then)
        self._fit_interval(rate)
        return pred > self._budget_search()

    def compute(self, coords, q, type_, ljparams, forces=None, energies=None, want_energy=True):
        """Forces (and energies) of one frame; searches / prunes as scheduled."""
        if self.evals_since_search is None:
            self._search(coords)
        elif self.evals_since_prune >= self.interval:
            if self._checkpoint():
                self._search(coords)
            elif self.r_inner is not None:
                self._prune(coords)
            else:
                self.evals_since_prune = 0
        out = self.pl.forces(coords, q, type_, ljparams, self.rc, self.beta, forces, energies, want_energy,
                             self.stream)
        self.evals += 1
        self.evals_since_search += 1
        self.evals_since_prune += 1
        if self.lag > 0 and self.evals_since_prune == self.interval - self.lag:
            self.reader.enqueue()
            self.snapshot = (self.n_search, self.evals_since_search, self.evals_since_prune)
        if self.r_inner is not None:
            if self.evals_since_search == self.PROBE_AT:
                self.probe_reader.enqueue()
                self.probe = (self.n_search, self.evals_since_search)
            elif self.probe is not None and self.evals_since_search == self.PROBE_AT + max(1, self.lag):
                if self.probe[0] == self.n_search:
                    self._fit_interval(self.probe_reader.read()["max_disp_search"] ** 2 / (self.probe[1] - 1))
                self.probe = None
        return out

    def check(self) -> int:
        """Synchronise and return the device error word (0 = every list was complete)."""
        return self.pl.status(False, self.stream)

    def close(self):
        self.pl.close()
