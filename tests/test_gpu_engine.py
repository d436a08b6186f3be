"""The search / rolling-prune schedule (engine.py) on the GPU: a trajectory
fast enough to force several searches, forces and energies of frames along
it against the oracle, no stale-list error, and the tracker read from the
queued copies (no drained stream) at the prune points.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import E_TOL, compare_forces, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    from paper_2405_01420_gb300 import nb as nbmod
    nbmod.load_library()
    return nbmod


def test_trajectory_matches_the_oracle(nb):
    from paper_2405_01420_gb300.engine import NonbondedEngine
    b = synth.water_box(4000, 21)  # 12,000 atoms
    # sigma 0.002 nm per frame: the search budget (0.03 nm) runs out after about 12 frames and the
    # prune budget (0.02 nm) after about 6, so the engine has to shorten its prune interval of 10
    frames = synth.random_walk_frames(b, 40, 0.002, seed=21)
    rc, rlist, r_inner = 1.0, 1.1, 1.04
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    eng = NonbondedEngine(b.n_atoms, b.box, rc, beta, rlist, r_inner, 10, d["excl_off"], d["excl_idx"])
    fd = torch.from_numpy(frames).cuda()
    F = torch.empty((b.n_atoms, 3), dtype=torch.float32, device="cuda")
    E = torch.zeros((40, 2), dtype=torch.float64, device="cuda")
    keep = {}
    for i in range(40):
        eng.compute(fd[i], d["q"], d["type"], d["lj"], F, E[i])
        if i in (0, 17, 39):
            keep[i] = F.cpu().numpy()
    assert eng.check() == 0, "a list went stale"
    assert eng.n_search >= 2
    assert eng.interval < 10, "the probe did not shorten the prune interval"
    # at most the first prune point after a search reads synchronously
    assert eng.n_sync_reads <= eng.n_search
    E = E.cpu().numpy()
    for i, Fi in keep.items():
        Fo, elj, ec, _ = oracle.energy_forces(frames[i], b.q, b.type, b.ljparams, b.box, rc, beta, b.excl_off,
                                              b.excl_idx)
        compare_forces(Fi, Fo)
        assert rel(E[i, 0], elj) <= E_TOL and rel(E[i, 1], ec) <= E_TOL
    eng.close()


def test_tracker_copy_matches_stats(nb):
    b = synth.water_box(512, 3)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms)
    pl.search(d["coords"], b.box, 1.0, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 0.95)
    x = d["coords"] + 0.003 * torch.randn_like(d["coords"])
    pl.forces(x, d["q"], d["type"], d["lj"], 0.9, synth.ewald_beta(0.9))
    words = torch.zeros(3, dtype=torch.int32).pin_memory()
    pl.tracker_enqueue(words)
    torch.cuda.synchronize()
    t = nb.decode_tracker(words.numpy())
    st = pl.stats()
    assert t["error_word"] == st["error_word"] == 0
    assert t["max_disp_search"] == pytest.approx(st["max_disp_search"], rel=1e-6)
    assert t["max_disp_prune"] == pytest.approx(st["max_disp_prune"], rel=1e-6)
    assert 0.003 < t["max_disp_search"] < 0.05
    pl.close()


def test_every_evaluation_covers_the_pairs_within_rc(nb):
    """Along a trajectory that forces searches and prunes, every evaluation
    counts exactly the oracle's FP32 pairs within rc (images relative to the
    frame of the last search), and its forces and energies match."""
    from paper_2405_01420_gb300.engine import NonbondedEngine
    b = synth.water_box(2000, 23)  # 6,000 atoms
    n_frames = 30
    frames = synth.random_walk_frames(b, n_frames, 0.002, seed=23)
    rc, rlist, r_inner = 1.0, 1.1, 1.04
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    eng = NonbondedEngine(b.n_atoms, b.box, rc, beta, rlist, r_inner, 10, d["excl_off"], d["excl_idx"],
                          count_pairs=True)
    fd = torch.from_numpy(frames).cuda()
    F = torch.empty((b.n_atoms, 3), dtype=torch.float32, device="cuda")
    E = torch.zeros(2, dtype=torch.float64, device="cuda")
    searched_at = []
    for i in range(n_frames):
        eng.compute(fd[i], d["q"], d["type"], d["lj"], F, E)
        s = i + 1 - eng.evals_since_search  # frame of the search the list was built on
        if not searched_at or searched_at[-1] != s:
            searched_at.append(s)
        st = eng.pl.stats()
        assert st["error_word"] == 0, (i, st["error_word"])
        ref = oracle.pairs_f32(frames[s], frames[i], b.box, rc, b.excl_off, b.excl_idx, count_only=True)
        assert st["pairs_last"] == ref, (i, st["pairs_last"], ref)
        Fo, elj, ec, _ = oracle.energy_forces(frames[i], b.q, b.type, b.ljparams, b.box, rc, beta, b.excl_off,
                                              b.excl_idx)
        compare_forces(F.cpu().numpy(), Fo)
        e = E.cpu().numpy()
        assert rel(e[0], elj) <= E_TOL and rel(e[1], ec) <= E_TOL, i
    assert len(searched_at) >= 2 and eng.n_prune > eng.n_search, (searched_at, eng.n_prune)
    eng.close()
