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
reads that word at every prune point (one stream synchronisation per prune
interval) and raises if it is set.
"""
from __future__ import annotations

import math

import torch

from . import nb


class NonbondedEngine:
    def __init__(self, n_atoms: int, box, rc: float, beta: float, rlist: float,
                 r_inner: float | None = None, prune_interval: int = 10, excl_off=None, excl_idx=None,
                 capacity_entries: int = 0, stream=None, count_pairs: bool = False):
        self.n_atoms = int(n_atoms)
        self.box = [float(v) for v in box]
        self.rc = float(rc)
        self.beta = float(beta)
        self.rlist = float(rlist)
        self.r_inner = None if r_inner is None else float(r_inner)
        if self.r_inner is not None and not (self.rc <= self.r_inner <= self.rlist):
            raise ValueError("need rc <= r_inner <= rlist")
        self.prune_interval = max(1, int(prune_interval))
        self.excl_off = excl_off
        self.excl_idx = excl_idx
        self.stream = stream
        self.pl = nb.Pairlist(self.n_atoms, capacity_entries, count_pairs)
        self.evals = 0
        self.evals_since_search = None
        self.evals_since_prune = 0
        self.interval = self.prune_interval
        self.n_search = 0
        self.n_prune = 0

    # budgets on the largest atom displacement (nm), as the kernels check them
    def _budget_search(self) -> float:
        r = self.r_inner if self.r_inner is not None else self.rc
        return 0.5 * (self.rlist - r) - 1e-5

    def _budget_prune(self) -> float:
        return 0.5 * (self.r_inner - self.rc) - 1e-5

    def _search(self, coords):
        self.pl.search(coords, self.box, self.rlist, self.excl_off, self.excl_idx, self.stream)
        self.n_search += 1
        self.evals_since_search = 0
        if self.r_inner is not None:
            self._prune(coords)

    def _prune(self, coords):
        self.pl.prune(coords, self.r_inner, self.stream)
        self.n_prune += 1
        self.evals_since_prune = 0

    def _checkpoint(self) -> bool:
        """Read the tracker (synchronises); return True if a search is due."""
        st = self.pl.stats(self.stream)
        bad = st["error_word"]
        if bad:
            raise nb.NBError(nb.NB_ERR_STATE, f"device error word 0x{bad:x} during the last interval")
        n = max(1, self.evals_since_search)
        # random-walk growth: displacement ~ sqrt(frames since the search)
        pred = st["max_disp_search"] * math.sqrt((n + 1) / n) * 1.05
        dp = st["max_disp_prune"]
        if self.r_inner is not None and dp > 0.9 * self._budget_prune() and self.interval > 1:
            self.interval = max(1, self.interval // 2)
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
        return out

    def check(self) -> int:
        """Synchronise and return the device error word (0 = every list was complete)."""
        return self.pl.status(False, self.stream)

    def close(self):
        self.pl.close()
