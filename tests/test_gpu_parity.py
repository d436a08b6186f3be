"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Pair coverage is compared bit for bit with the oracle's FP32 pair set;
forces per atom within 1e-4 rms(F) and energies within 1e-6 relative of the
FP64 oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import (E_TOL, assert_same_pairs, compare_forces, expand_counted_pairs, expand_tile_pairs, oracle_ref,
                        pair_set, rel, tiled_along_z, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    from paper_2405_01420_gb300 import nb as nbmod
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    nbmod.load_library()
    return nbmod


def check_energies(E, elj, ec):
    e = E.cpu().numpy()
    assert rel(e[0], elj) <= E_TOL, (e[0], elj)
    assert rel(e[1], ec) <= E_TOL, (e[1], ec)
    assert rel(e[0] + e[1], elj + ec) <= E_TOL


# ------------------------------------------------------------ plain method

def test_small_box_search_and_forces(nb):
    """1,536 atoms, rc = rlist = 0.9 nm: one search, one force evaluation."""
    b = synth.water_box(512, 1)
    rc = 0.9
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.search(d["coords"], b.box, rc, d["excl_off"], d["excl_idx"])
    F, E = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta)
    torch.cuda.synchronize()
    assert pl.status() == 0
    exp = pl.export(nb.NB_LIST_OUTER)
    y = oracle.image_f32(b.coords, b.coords, b.box)
    counted = expand_counted_pairs(exp, y, b.box, rc)
    ref = oracle.pairs_f32(b.coords, b.coords, b.box, rc, b.excl_off, b.excl_idx)
    assert len(pair_set(counted)) == len(counted), "an atom pair is listed twice"
    assert pair_set(counted) == pair_set(ref)
    assert pl.stats()["pairs_last"] == len(ref)
    Fo, elj, ec, _ = oracle_ref(b, rc, beta)
    compare_forces(F.cpu().numpy(), Fo)
    check_energies(E, elj, ec)
    pl.close()


@pytest.mark.parametrize("nw, seed", [(4000, 7), (1111, 8)])
def test_grid_sort_is_a_bijection_into_compact_clusters(nb, nw, seed):
    """The grid sort: every atom has exactly one cluster slot, padding slots
    close a cluster, the atoms of a cluster share one xy grid column, and a
    column's clusters hold its atoms in z order."""
    b = synth.water_box(nw, seed)
    n = b.n_atoms
    d = to_dev(b)
    pl = nb.Pairlist(n)
    pl.search(d["coords"], b.box, 1.0, d["excl_off"], d["excl_idx"])
    assert pl.status() == 0
    perm = pl.export(nb.NB_LIST_OUTER)["perm"].reshape(-1, 8)
    st = pl.stats()
    pl.close()
    assert perm.shape[0] == st["n_clusters"]
    real = perm >= 0
    assert np.array_equal(np.sort(perm[real]), np.arange(n)), "not a permutation of the atoms"
    # padding only after the real atoms of a cluster, and no cluster without atoms
    assert (np.diff(real.astype(np.int8), axis=1) <= 0).all()
    assert real[:, 0].all()
    # one xy column per cluster (a cubic box: ncx = ncy)
    ncx = int(round(np.sqrt(st["n_columns"])))
    assert ncx * ncx == st["n_columns"]
    w = b.box[:2].astype(np.float64) / ncx
    y = oracle.image_f32(b.coords, b.coords, b.box).astype(np.float64)
    cols = []
    for c in range(perm.shape[0]):
        a = perm[c][real[c]]
        xy = y[a, :2]
        assert (xy.max(axis=0) - xy.min(axis=0) <= w + 1e-5).all(), f"cluster {c} spans columns"
        z = y[a, 2]
        assert (np.diff(z) >= -1e-6).all(), f"cluster {c} not z-sorted"
        cols.append(tuple(np.floor(xy.mean(axis=0) / w).astype(int)))
    # clusters of one column, in slot order, cover disjoint rising z ranges
    last_top = {}
    for c, col in enumerate(cols):
        a = perm[c][real[c]]
        z = y[a, 2]
        if col in last_top:
            assert z.min() >= last_top[col] - 1e-6, f"column {col}: cluster {c} out of z order"
        last_top[col] = z.max()


def test_list_covers_rlist(nb):
    """Every pair within rlist (FP32 contract) has its mask bit in the outer list."""
    b = synth.water_box(4000, 7)
    rlist = 1.1
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.search(d["coords"], b.box, rlist, d["excl_off"], d["excl_idx"])
    exp = pl.export(nb.NB_LIST_OUTER)
    assert pl.status() == 0
    y = oracle.image_f32(b.coords, b.coords, b.box)
    counted = expand_counted_pairs(exp, y, b.box, rlist)
    ref = oracle.pairs_f32(b.coords, b.coords, b.box, rlist, b.excl_off, b.excl_idx)
    assert len(pair_set(counted)) == len(counted)
    assert pair_set(counted) == pair_set(ref)
    # the list is ordered: every entry has ci <= cj, and no (ci, cj, shift) twice
    assert (exp["ci"] <= exp["cj"]).all()
    keys = exp["ci"].astype(np.int64) * 10 ** 9 + exp["cj"].astype(np.int64) * 32 + exp["shift"]
    assert np.unique(keys).size == keys.size
    pl.close()


def test_prune_and_displaced_frames(nb):
    """12k atoms, rc 1.0 / rlist 1.1 / r_inner 1.04; prune and forces on a random walk."""
    b = synth.water_box(4000, 3)
    rc, rlist, r_in = 1.0, 1.1, 1.04
    beta = synth.ewald_beta(rc)
    frames = synth.random_walk_frames(b, 14, 0.001, seed=31)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    x0 = frames[0]
    pl.search(torch.from_numpy(x0).cuda(), b.box, rlist, d["excl_off"], d["excl_idx"])
    for f in range(14):
        xf = torch.from_numpy(frames[f]).cuda()
        if f % 10 == 0:
            pl.prune(xf, r_in)
        F, E = pl.forces(xf, d["q"], d["type"], d["lj"], rc, beta)
        if f in (0, 5, 13):
            torch.cuda.synchronize()
            assert pl.status() == 0
            exp = pl.export(nb.NB_LIST_INNER)
            y = oracle.image_f32(x0, frames[f], b.box)
            counted = expand_counted_pairs(exp, y, b.box, rc)
            ref = oracle.pairs_f32(x0, frames[f], b.box, rc, b.excl_off, b.excl_idx)
            assert len(pair_set(counted)) == len(counted)
            assert pair_set(counted) == pair_set(ref), f
            assert pl.stats()["pairs_last"] == len(ref)
            Fo, elj, ec, _ = oracle_ref(b, rc, beta, frames[f])
            compare_forces(F.cpu().numpy(), Fo)
            check_energies(E, elj, ec)
    pl.close()


@pytest.mark.parametrize("nw,seed", [(4000, 3), (391, 8)])
def test_gathered_tiles_cover_r_inner(nb, nw, seed):
    """The gathered 4 x 8 tiles of a prune hold every pair within r_inner once
    (bit for bit against the FP32 pair set), and no mask bit on a pad slot."""
    b = synth.water_box(nw, seed)
    rlist, r_in = 1.1, 1.04
    frames = synth.random_walk_frames(b, 2, 0.002, seed=seed + 40)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.search(torch.from_numpy(frames[0]).cuda(), b.box, rlist, d["excl_off"], d["excl_idx"])
    pl.prune(torch.from_numpy(frames[1]).cuda(), r_in)
    torch.cuda.synchronize()
    assert pl.status() == 0
    tiles = pl.export_tiles()
    exp = pl.export(nb.NB_LIST_INNER)
    y = oracle.image_f32(frames[0], frames[1], b.box)
    got = expand_tile_pairs(tiles, exp["perm"], y, b.box, r_in)
    ref = oracle.pairs_f32(frames[0], frames[1], b.box, r_in, b.excl_off, b.excl_idx)
    assert len(pair_set(got)) == len(got), "an atom pair is in two tiles"
    assert pair_set(got) == pair_set(ref)
    # every set bit is within r_inner (nothing beyond the prune radius kept)
    assert len(expand_tile_pairs(tiles, exp["perm"], y, b.box, 1e3)) == len(got)
    # each half's tiles are dense: all but its last tile have 8 occupied columns
    hid = tiles["half_id"]
    last = np.r_[hid[1:] != hid[:-1], True]
    cols = np.zeros(hid.size, np.int64)
    for p_ in range(8):
        cols += ((tiles["masks"] >> np.uint32(p_)) & np.uint32(0x01010101)) != 0
    assert (cols[~last] == 8).all()
    # the prune's own count of the tiles it wrote (nb_pairlist_stats)
    assert pl.stats()["gathered_tiles"] == hid.size
    pl.close()


@pytest.mark.parametrize("want_energy", [True, False])
def test_cluster_tiles_and_gathered_tiles_agree(nb, want_energy):
    """After a prune both force kernels (8 x 8 cluster tiles / gathered 4 x 8
    tiles) meet the oracle bar and count the same pairs."""
    b = synth.water_box(3000, 12)
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    out = []
    for cluster_tiles in (False, True):
        pl = nb.Pairlist(b.n_atoms, count_pairs=True, cluster_tiles=cluster_tiles)
        pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
        pl.prune(d["coords"], 1.04)
        F, E = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta, want_energy=want_energy)
        torch.cuda.synchronize()
        assert pl.status() == 0
        out.append((F.cpu().numpy(), None if E is None else E.cpu().numpy(), pl.stats()["pairs_last"]))
        pl.close()
    Fo, elj, ec, _ = oracle_ref(b, rc, beta)
    n32 = oracle.pairs_f32(b.coords, b.coords, b.box, rc, b.excl_off, b.excl_idx, count_only=True)
    for F, E, np_ in out:
        compare_forces(F, Fo)
        assert np_ == n32
        if want_energy:
            assert rel(E[0], elj) <= E_TOL and rel(E[1], ec) <= E_TOL


def test_force_only_path_matches(nb):
    b = synth.water_box(2000, 9)
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms)  # no pair counting: the kernels without the counter
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    F1, _ = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta, want_energy=False)
    assert pl.stats()["pairs_last"] == -1
    F2, E2 = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta)
    Fo, elj, ec, _ = oracle_ref(b, rc, beta)
    compare_forces(F1.cpu().numpy(), Fo)
    compare_forces(F2.cpu().numpy(), Fo)
    check_energies(E2, elj, ec)
    assert pl.status() == 0
    pl.close()


def test_four_types_random_charges(nb):
    """24,000 atoms with per-atom charges N(0, 0.4) and 4 LJ types (geometric rule)."""
    b = synth.water_box(8000, 4)
    p = synth.diff_params(b, seed=4)
    lj = synth.combine_geometric(p["c6"], p["c12"]).astype(np.float32)
    q = p["q"].astype(np.float32)
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    F, E = pl.forces(d["coords"], torch.from_numpy(q).cuda(), torch.from_numpy(p["type"]).cuda(),
                     torch.from_numpy(lj).cuda(), rc, beta)
    Fo, elj, ec, _ = oracle.energy_forces(b.coords, q, p["type"], lj, b.box, rc, beta, b.excl_off, b.excl_idx)
    compare_forces(F.cpu().numpy(), Fo)
    check_energies(E, elj, ec)
    assert pl.status() == 0
    pl.close()


def test_repeated_search_is_deterministic(nb):
    b = synth.water_box(1000, 12)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.search(d["coords"], b.box, 1.0, d["excl_off"], d["excl_idx"])
    e1 = pl.export(nb.NB_LIST_OUTER)
    pl.search(d["coords"], b.box, 1.0, d["excl_off"], d["excl_idx"])
    e2 = pl.export(nb.NB_LIST_OUTER)
    for k in ("ci", "cj", "shift", "mask", "perm"):
        np.testing.assert_array_equal(e1[k], e2[k])
    pl.close()


# ------------------------------------------------------------ full sizes

def test_production_box_96k(nb):
    """96,000 atoms (32,000 waters), rc 1.0 / rlist 1.1, as the benchmark launches it."""
    b = synth.water_box(32000, 2)
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    F, E = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta)
    torch.cuda.synchronize()
    assert pl.status() == 0
    Fo, elj, ec, n64 = oracle_ref(b, rc, beta)
    compare_forces(F.cpu().numpy(), Fo)
    check_energies(E, elj, ec)
    ref = oracle.pairs_f32(b.coords, b.coords, b.box, rc, b.excl_off, b.excl_idx)
    assert pl.stats()["pairs_last"] == len(ref)
    assert abs(len(ref) - n64) <= 5
    # the pair sets themselves, bit for bit: the 8 x 8 inner list and the gathered tiles the
    # force kernel reads, each expanded under the FP32 contract at rc
    y = oracle.image_f32(b.coords, b.coords, b.box)
    inner = pl.export(nb.NB_LIST_INNER)
    assert_same_pairs(expand_counted_pairs(inner, y, b.box, rc), ref, b.n_atoms)
    tiles = pl.export_tiles()
    assert_same_pairs(expand_tile_pairs(tiles, inner["perm"], y, b.box, rc), ref, b.n_atoms)
    pl.close()


def test_million_atom_box_sampled(nb):
    """~1,000,000 atoms (333,334 waters): energies in full, forces on 3,000 sampled atoms."""
    b = synth.water_box(333334, 3)
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    F, E = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta)
    torch.cuda.synchronize()
    assert pl.status() == 0
    _, elj, ec, n64 = oracle_ref(b, rc, beta)
    check_energies(E, elj, ec)
    rng = np.random.default_rng(5)
    atoms = np.sort(rng.choice(b.n_atoms, 3000, replace=False))
    Fs = oracle.forces_subset(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, atoms, b.excl_off, b.excl_idx)
    Fg = F.cpu().numpy()[atoms].astype(np.float64)
    rms = np.sqrt((Fs ** 2).sum(1).mean())
    assert np.sqrt(((Fg - Fs) ** 2).sum(1)).max() <= 1e-4 * rms
    n32 = oracle.pairs_f32(b.coords, b.coords, b.box, rc, b.excl_off, b.excl_idx, count_only=True)
    assert pl.stats()["pairs_last"] == n32
    assert abs(n32 - n64) <= 20
    pl.close()


# ------------------------------------------------------------ edge cases

def test_single_water(nb):
    b = synth.water_box(1, 1)
    box = np.array([3.0, 3.0, 3.0], np.float32)
    d = to_dev(b)
    pl = nb.Pairlist(3, count_pairs=True)
    pl.search(d["coords"], box, 0.9, d["excl_off"], d["excl_idx"])
    F, E = pl.forces(d["coords"], d["q"], d["type"], d["lj"], 0.9, synth.ewald_beta(0.9))
    assert pl.status() == 0
    assert torch.count_nonzero(F).item() == 0
    assert E.cpu().numpy().tolist() == [0.0, 0.0]
    assert pl.stats()["pairs_last"] == 0
    pl.close()


@pytest.mark.parametrize("nw", [2, 7, 27, 64])
def test_ragged_small_systems(nb, nw):
    """Atom counts that leave partly filled clusters; O(N^2) oracle."""
    b = synth.water_box(nw, 20 + nw)
    L = max(2.0, float(b.box[0]))
    box = np.array([L, L, L], np.float32)
    coords = b.coords.copy()
    rc = 0.9
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.search(d["coords"], box, rc, d["excl_off"], d["excl_idx"])
    F, E = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta)
    assert pl.status() == 0
    Fo, elj, ec, n, (alj, ac) = oracle.energy_forces(coords, b.q, b.type, b.ljparams, box, rc, beta, b.excl_off,
                                                     b.excl_idx, abs_sums=True)
    if n:
        compare_forces(F.cpu().numpy(), Fo)
        # A handful of pairs cannot average FP32 rounding: the bound here is
        # 1e-6 of the larger of |E| and the sum of |pair energies|.
        e = E.cpu().numpy()
        assert abs(e[0] - elj) <= 1e-6 * max(abs(elj), alj)
        assert abs(e[1] - ec) <= 1e-6 * max(abs(ec), ac)
    assert pl.stats()["pairs_last"] == oracle.pairs_f32(coords, coords, box, rc, b.excl_off, b.excl_idx,
                                                       count_only=True)
    pl.close()


def test_unwrapped_and_edge_coordinates(nb):
    """Inputs outside [0, L), and atoms exactly at 0 and at L, give the wrapped result."""
    b = synth.water_box(512, 1)
    rc = 0.9
    beta = synth.ewald_beta(rc)
    L = b.box.astype(np.float64)
    rng = np.random.default_rng(2)
    shift = rng.integers(-2, 3, size=b.coords.shape) * L
    x_unwrapped = (b.coords.astype(np.float64) + shift).astype(np.float32)
    x_edge = b.coords.copy()
    x_edge[0, 0] = 0.0
    x_edge[3, 1] = np.float32(L[1])  # x = L wraps to 0
    d = to_dev(b)
    for x in (x_unwrapped, x_edge):
        xd = torch.from_numpy(x).cuda()
        pl = nb.Pairlist(b.n_atoms, count_pairs=True)
        pl.search(xd, b.box, rc, d["excl_off"], d["excl_idx"])
        F, E = pl.forces(xd, d["q"], d["type"], d["lj"], rc, beta)
        assert pl.status() == 0
        xw = oracle.image_f32(x, x, b.box)  # contract positions (wrapped, to within an ulp)
        Fo, elj, ec, _ = oracle_ref(b, rc, beta, xw)
        compare_forces(F.cpu().numpy(), Fo)
        check_energies(E, elj, ec)
        pl.close()


@pytest.mark.parametrize("prune", [False, True])
def test_cutoff_just_below_half_the_box(nb, prune):
    """rc = rlist one float below L/2 (the largest the search accepts): every
    pair has exactly one image within rc, and cluster pairs may be listed
    with several shifts; coverage, forces and energies still match."""
    b = synth.water_box(512, 3)
    rc = float(np.nextafter(np.float32(b.box.min()) / np.float32(2), np.float32(0)))
    assert 2.0 * rc < float(b.box.min())
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.search(d["coords"], b.box, rc, d["excl_off"], d["excl_idx"])
    if prune:
        pl.prune(d["coords"], rc)
    F, E = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta)
    torch.cuda.synchronize()
    assert pl.status() == 0
    y = oracle.image_f32(b.coords, b.coords, b.box)
    ref = oracle.pairs_f32(b.coords, b.coords, b.box, rc, b.excl_off, b.excl_idx)
    counted = expand_counted_pairs(pl.export(nb.NB_LIST_OUTER), y, b.box, rc)
    assert len(pair_set(counted)) == len(counted), "an atom pair is listed twice"
    assert pair_set(counted) == pair_set(ref)
    assert pl.stats()["pairs_last"] == len(ref)
    Fo, elj, ec, _ = oracle_ref(b, rc, beta)
    compare_forces(F.cpu().numpy(), Fo)
    check_energies(E, elj, ec)
    pl.close()


def test_zero_charges(nb):
    b = synth.water_box(512, 1)
    rc = 0.9
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    q0 = torch.zeros_like(d["q"])
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.search(d["coords"], b.box, rc, d["excl_off"], d["excl_idx"])
    F, E = pl.forces(d["coords"], q0, d["type"], d["lj"], rc, beta)
    Fo, elj, ec, _ = oracle.energy_forces(b.coords, np.zeros(b.n_atoms), b.type, b.ljparams, b.box, rc, beta,
                                          b.excl_off, b.excl_idx)
    assert ec == 0.0 and E[1].item() == 0.0
    compare_forces(F.cpu().numpy(), Fo)
    assert rel(E[0].item(), elj) <= E_TOL
    pl.close()


# ------------------------------------------------------------ errors without faults

def test_host_argument_errors(nb):
    b = synth.water_box(64, 1)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    F = torch.empty((b.n_atoms, 3), device="cuda")
    with pytest.raises(nb.NBError) as e:
        pl.forces(d["coords"], d["q"], d["type"], d["lj"], 0.5, 3.0, F)
    assert e.value.code == nb.NB_ERR_STATE
    with pytest.raises(nb.NBError) as e:
        pl.search(d["coords"], b.box, float(b.box[0]), d["excl_off"], d["excl_idx"])  # box < 2 rlist
    assert e.value.code == nb.NB_ERR_ARG
    pl.search(d["coords"], b.box, 0.5, d["excl_off"], d["excl_idx"])
    with pytest.raises(nb.NBError) as e:
        pl.forces(d["coords"], d["q"], d["type"], d["lj"], 0.6, 3.0, F)  # rc > rlist
    assert e.value.code == nb.NB_ERR_ARG
    with pytest.raises(nb.NBError) as e:
        pl.prune(d["coords"], 0.7)  # r_inner > rlist
    assert e.value.code == nb.NB_ERR_ARG
    assert pl.status() == 0
    pl.close()


def test_device_error_bits(nb):
    """Overflow, bad types, non-finite input and stale lists set status bits; the context survives."""
    b = synth.water_box(512, 1)
    rc = 0.9
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    small = nb.Pairlist(b.n_atoms, capacity_entries=100)
    small.search(d["coords"], b.box, rc, d["excl_off"], d["excl_idx"])
    small.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta)
    assert small.status() & nb.NB_DEV_LIST_OVERFLOW
    small.close()

    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    bad_t = d["type"].clone()
    bad_t[5] = 7
    pl.search(d["coords"], b.box, rc, d["excl_off"], d["excl_idx"])
    pl.forces(d["coords"], d["q"], bad_t, d["lj"], rc, beta)
    assert pl.status(clear=True) & nb.NB_DEV_BAD_TYPE

    x_nan = d["coords"].clone()
    x_nan[10, 1] = float("nan")
    pl.search(x_nan, b.box, rc, d["excl_off"], d["excl_idx"])
    assert pl.status(clear=True) & nb.NB_DEV_NONFINITE

    # stale: move one atom 0.06 nm after a search at rlist 1.1 - rc 1.0 allows 0.05
    b2 = synth.water_box(4000, 3)
    d2 = to_dev(b2)
    pl2 = nb.Pairlist(b2.n_atoms)
    pl2.search(d2["coords"], b2.box, 1.1, d2["excl_off"], d2["excl_idx"])
    moved = d2["coords"].clone()
    moved[100, 0] += 0.06
    pl2.forces(moved, d2["q"], d2["type"], d2["lj"], 1.0, synth.ewald_beta(1.0))
    assert pl2.status(clear=True) & nb.NB_DEV_STALE_SEARCH
    pl2.prune(d2["coords"], 1.04)
    moved = d2["coords"].clone()
    moved[7, 2] += 0.025  # (1.04 - 1.0)/2 = 0.02 allowed after the prune
    pl2.forces(moved, d2["q"], d2["type"], d2["lj"], 1.0, synth.ewald_beta(1.0))
    assert pl2.status(clear=True) & nb.NB_DEV_STALE_PRUNE
    # the context still works
    F, E = pl2.forces(d2["coords"], d2["q"], d2["type"], d2["lj"], 1.0, synth.ewald_beta(1.0))
    assert pl2.status() == 0
    pl2.close()
    pl.close()


def test_list_sorting_does_not_change_results(nb):
    """Post-prune sorting by list length only reorders work: same forces and energies."""
    b = synth.water_box(4000, 13)
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    out = []
    for sort in (True, False):
        pl = nb.Pairlist(b.n_atoms, count_pairs=True, sort_lists=sort)
        pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
        pl.prune(d["coords"], 1.04)
        F, E = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta)
        assert pl.status() == 0
        out.append((F.cpu().numpy(), E.cpu().numpy(), pl.stats()["pairs_last"]))
        pl.close()
    (F1, E1, n1), (F2, E2, n2) = out
    assert n1 == n2
    np.testing.assert_allclose(F1, F2, rtol=0, atol=1e-5 * np.abs(F2).max())
    assert rel(E1[0], E2[0]) <= 1e-7 and rel(E1[1], E2[1]) <= 1e-7


def test_elongated_orthorhombic_box(nb):
    """2.48 x 2.48 x 19.9 nm (512 waters tiled 8 times along z): grid columns of about 490 atoms
    (the column sort's larger sorting network), long z ranges in the search, per-axis minimum
    images; pair coverage, forces and energies against the oracle."""
    b = tiled_along_z(synth.water_box(512, 1), 8)
    rc, rlist, r_in = 0.9, 1.0, 0.95
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.search(d["coords"], b.box, rlist, d["excl_off"], d["excl_idx"])
    st = pl.stats()
    assert st["n_clusters"] * 8 >= b.n_atoms and b.n_atoms / st["n_columns"] > 256
    pairs = oracle.pairs_f32(b.coords, b.coords, b.box, rc, b.excl_off, b.excl_idx)
    for prune in (False, True):
        if prune:
            pl.prune(d["coords"], r_in)
        F, E = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta)
        torch.cuda.synchronize()
        assert pl.status() == 0
        assert pl.stats()["pairs_last"] == len(pairs)
        Fo, elj, ec, _ = oracle.energy_forces(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, b.excl_off,
                                              b.excl_idx)
        compare_forces(F.cpu().numpy(), Fo)
        check_energies(E, elj, ec)
    pl.close()


@pytest.mark.parametrize("cluster_tiles", [False, True])
def test_thirty_two_lj_types(nb, cluster_tiles):
    """The largest LJ table the API takes (32 types, geometric rule, random charges), on both tile
    forms after a prune."""
    b = synth.water_box(1000, 9)
    p = synth.diff_params(b, seed=9, ntype=32)
    lj = synth.combine_geometric(p["c6"], p["c12"]).astype(np.float32)
    q = p["q"].astype(np.float32)
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True, cluster_tiles=cluster_tiles)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    F, E = pl.forces(d["coords"], torch.from_numpy(q).cuda(), torch.from_numpy(p["type"]).cuda(),
                     torch.from_numpy(lj).cuda(), rc, beta)
    torch.cuda.synchronize()
    assert pl.status() == 0
    assert int(p["type"].max()) == 31
    Fo, elj, ec, _ = oracle.energy_forces(b.coords, q, p["type"], lj, b.box, rc, beta, b.excl_off, b.excl_idx)
    compare_forces(F.cpu().numpy(), Fo)
    check_energies(E, elj, ec)
    pl.close()
