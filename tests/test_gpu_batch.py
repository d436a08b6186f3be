"""Batched form: many independent boxes in one pair list, one set of launches.

Each system's forces and energies from the batch must equal the oracle's
for that system alone (standard tolerances) and the plain single-system
path's; the batch must replay correctly from a captured CUDA graph.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import E_TOL, compare_forces, rel, tiled_along_z

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    from paper_2405_01420_gb300 import nb as nbmod
    nbmod.load_library()
    return nbmod


def concat(boxes):
    off = np.zeros(len(boxes) + 1, np.int32)
    for k, b in enumerate(boxes):
        off[k + 1] = off[k] + b.n_atoms
    x = np.concatenate([b.coords for b in boxes])
    q = np.concatenate([b.q for b in boxes])
    t = np.concatenate([b.type for b in boxes])
    eo = [np.zeros(1, np.int32)]
    ei = []
    base = 0
    for k, b in enumerate(boxes):
        eo.append(b.excl_off[1:] + base)
        ei.append(b.excl_idx + off[k])
        base += b.excl_off[-1]
    return off, x, q, t, np.concatenate(eo), np.concatenate(ei), np.stack([b.box for b in boxes])


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def batch():
    sizes = [1536, 3000, 903, 6003, 2400]  # atoms, rounded down to whole waters (every box edge > 2 rlist)
    return [synth.water_box_for_atoms(n, 100 + k) for k, n in enumerate(sizes)]


def test_batch_matches_oracle_and_plain(nb, batch):
    rc, rlist = 0.9, 1.0
    beta = synth.ewald_beta(rc)
    off, x, q, t, eo, ei, boxes = concat(batch)
    lj = dev(batch[0].ljparams)
    pl = nb.Pairlist.batch(off, boxes, count_pairs=True)
    pl.search(dev(x), None, rlist, dev(eo), dev(ei))
    F, E = pl.forces(dev(x), dev(q), dev(t), lj, rc, beta)
    assert pl.status() == 0
    F = F.cpu().numpy()
    E = E.cpu().numpy().reshape(-1, 2)
    total_pairs = 0
    for k, b in enumerate(batch):
        Fo, elj, ec, n = oracle.energy_forces(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, b.excl_off,
                                              b.excl_idx)
        compare_forces(F[off[k]:off[k + 1]], Fo)
        assert rel(E[k, 0], elj) <= E_TOL and rel(E[k, 1], ec) <= E_TOL, k
        total_pairs += oracle.pairs_f32(b.coords, b.coords, b.box, rc, b.excl_off, b.excl_idx, count_only=True)
        # the plain path on this system alone
        p1 = nb.Pairlist(b.n_atoms)
        p1.search(dev(b.coords), b.box, rlist, dev(b.excl_off), dev(b.excl_idx))
        F1, E1 = p1.forces(dev(b.coords), dev(b.q), dev(b.type), lj, rc, beta)
        np.testing.assert_allclose(F[off[k]:off[k + 1]], F1.cpu().numpy(), rtol=0,
                                   atol=1e-5 * np.abs(Fo).max())
        # A small system alone splits its i-clusters' lists over more warps than the batch does,
        # so the two sum their FP32 pair energies in different orders: both meet the oracle's bar.
        assert rel(E1[0].item(), elj) <= E_TOL and rel(E1[1].item(), ec) <= E_TOL, k
        assert rel(E[k, 0], E1[0].item()) <= E_TOL and rel(E[k, 1], E1[1].item()) <= E_TOL
        p1.close()
    assert pl.stats()["pairs_last"] == total_pairs
    # prune on top of the batch list
    pl.prune(dev(x), rc + 0.02)
    F2, E2 = pl.forces(dev(x), dev(q), dev(t), lj, rc, beta)
    assert pl.status() == 0
    np.testing.assert_allclose(F2.cpu().numpy(), F, rtol=0, atol=1e-5 * np.abs(F).max())
    pl.close()


def test_batch_graph_replay(nb, batch):
    """search + forces of the whole batch captured in one CUDA graph and replayed."""
    rc, rlist = 0.9, 1.0
    beta = synth.ewald_beta(rc)
    off, x, q, t, eo, ei, boxes = concat(batch)
    xd, qd, td, eod, eid = dev(x), dev(q), dev(t), dev(eo), dev(ei)
    lj = dev(batch[0].ljparams)
    pl = nb.Pairlist.batch(off, boxes)
    F = torch.empty((pl.n_atoms, 3), dtype=torch.float32, device="cuda")
    E = torch.empty(2 * pl.n_systems, dtype=torch.float64, device="cuda")
    # eager once (also runs every one-time set-up outside the capture)
    pl.search(xd, None, rlist, eod, eid)
    pl.forces(xd, qd, td, lj, rc, beta, F, E)
    torch.cuda.synchronize()
    F_eager, E_eager = F.clone(), E.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            pl.search(xd, None, rlist, eod, eid, stream=s)
            pl.forces(xd, qd, td, lj, rc, beta, F, E, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        F.zero_()
        E.zero_()
        g.replay()
        torch.cuda.synchronize()
        torch.testing.assert_close(F, F_eager, rtol=0, atol=1e-5 * F_eager.abs().max().item())
        torch.testing.assert_close(E, E_eager, rtol=1e-9, atol=0)
    assert pl.status() == 0
    pl.close()


def test_batch_with_long_and_short_columns(nb):
    """Six 1,536-atom boxes (columns of about 61 atoms) and one 2.48 x 2.48 x 19.9 nm box (columns of
    about 490 atoms): the columns average below 128 atoms, so the grid sort takes eight columns per
    CTA, sorts the short ones in warp registers and the long ones with the whole CTA in shared
    memory. Pair counts, forces and energies of every system against the oracle: at 1,536 atoms the
    FP32 rounding of the displacements alone moves E_C by up to about 1e-6 of it, so the energies are
    held to 1e-6 of the oracle's energies at the FP32 contract's distances, and to that bar plus the
    contract's own offset against the FP64 oracle."""
    rc, rlist = 0.9, 1.0
    beta = synth.ewald_beta(rc)
    boxes = [synth.water_box(512, 300 + k) for k in range(6)] + [tiled_along_z(synth.water_box(512, 1), 8)]
    off, x, q, t, eo, ei, bx = concat(boxes)
    lj = dev(boxes[0].ljparams)
    pl = nb.Pairlist.batch(off, bx, count_pairs=True)
    pl.search(dev(x), None, rlist, dev(eo), dev(ei))
    st = pl.stats()
    assert pl.n_atoms <= 128 * st["n_columns"]  # short columns on average
    F, E = pl.forces(dev(x), dev(q), dev(t), lj, rc, beta)
    assert pl.status() == 0
    F = F.cpu().numpy()
    E = E.cpu().numpy().reshape(-1, 2)
    total_pairs = 0
    for k, b in enumerate(boxes):
        Fo, elj, ec, _ = oracle.energy_forces(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, b.excl_off,
                                              b.excl_idx)
        compare_forces(F[off[k]:off[k + 1]], Fo)
        e32_lj, e32_c, n32 = oracle.energy_f32(b.coords, b.coords, b.q, b.type, b.ljparams, b.box, rc, beta,
                                               b.excl_off, b.excl_idx)
        assert rel(E[k, 0], e32_lj) <= E_TOL and rel(E[k, 1], e32_c) <= E_TOL, k
        assert abs(E[k, 0] - elj) <= E_TOL * abs(elj) + abs(e32_lj - elj), k
        assert abs(E[k, 1] - ec) <= E_TOL * abs(ec) + abs(e32_c - ec), k
        total_pairs += n32
    assert pl.stats()["pairs_last"] == total_pairs
    pl.close()


def test_full_size_batch_of_256_boxes(nb):
    """The batched benchmark's workload at full size: 256 boxes of 1,536..24,000 atoms (3.27M atoms),
    searched at rlist 1.0, pruned to rc 0.9 and computed on gathered tiles, as the benchmark times it.
    Every box's pair count is the oracle's FP32 set's; its E_C is within 1e-6 of the oracle's energy at
    the contract's distances (R28), its E_LJ within 1e-6 of max(|E_LJ|, sum |e_LJ|) of it (R18: in some
    boxes attraction and repulsion nearly balance, E_LJ ~ 1/400 of sum |e_LJ|, and FP32 rounding of 1/r
    at close contacts alone moves it by ~2e-6 of itself); forces of four boxes (the smallest, the
    largest and two others) against the FP64 oracle, and their energies against it at the same bars
    plus the contract's offset."""
    rc, rlist = 0.9, 1.0
    beta = synth.ewald_beta(rc)
    boxes = synth.batch_boxes(256, 1536, 24000, seed=5)
    off, x, q, t, eo, ei, bx = concat(boxes)
    xd = dev(x)
    pl = nb.Pairlist.batch(off, bx, count_pairs=True)
    pl.search(xd, None, rlist, dev(eo), dev(ei))
    pl.prune(xd, rc)
    F, E = pl.forces(xd, dev(q), dev(t), dev(boxes[0].ljparams), rc, beta)
    assert pl.status() == 0
    total = pl.stats()["pairs_last"]
    pl.close()
    F = F.cpu().numpy()
    E = E.cpu().numpy().reshape(-1, 2)

    def reference(b):  # the C oracle runs without the GIL: the boxes go to threads
        return oracle.energy_f32(b.coords, b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, b.excl_off,
                                 b.excl_idx, abs_sums=True)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        refs = list(ex.map(reference, boxes))
    assert total == sum(r[2] for r in refs)
    for k, (e32_lj, e32_c, _, (a_lj, _)) in enumerate(refs):
        assert abs(E[k, 0] - e32_lj) <= E_TOL * max(abs(e32_lj), a_lj), k
        assert rel(E[k, 1], e32_c) <= E_TOL, k
    sizes = np.array([b.n_atoms for b in boxes])
    for k in sorted({int(sizes.argmin()), int(sizes.argmax()), 7, 200}):
        b = boxes[k]
        Fo, elj, ec, _ = oracle.energy_forces(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, b.excl_off,
                                              b.excl_idx)
        compare_forces(F[off[k]:off[k + 1]], Fo)
        assert abs(E[k, 0] - elj) <= E_TOL * max(abs(elj), refs[k][3][0]) + abs(refs[k][0] - elj), k
        assert abs(E[k, 1] - ec) <= E_TOL * abs(ec) + abs(refs[k][1] - ec), k
