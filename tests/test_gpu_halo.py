"""Local / non-local split (nb_set_home, nb_forces_part) on one GPU with a
synthetic halo: the waters whose oxygen sits in the left half of the box are
home atoms (numbered first), the rest are halo atoms.

The local part computes the pairs of two home atoms without reading the halo
atoms' inputs (the test leaves NaN there until the non-local part); the two
parts together equal the oracle; each part's energies and pair count equal
the oracle over that part's pairs (in/out decided under the FP32 contract on
both sides).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import E_TOL, compare_forces, expand_tile_pairs, pair_set, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    from paper_2405_01420_gb300 import nb as nbmod
    nbmod.load_library()
    return nbmod


class Box:
    pass


@pytest.fixture(scope="module")
def halo_box():
    """12,000-atom water box, molecules reordered: home (O at x < L/2) first."""
    b = synth.water_box(4000, 17)
    nw = b.n_atoms // 3
    o_x = b.coords[0::3, 0]
    home = np.flatnonzero(o_x < b.box[0] / 2)
    halo = np.flatnonzero(o_x >= b.box[0] / 2)
    order = np.concatenate([home, halo])
    atoms = (3 * order[:, None] + np.arange(3)[None, :]).reshape(-1)
    r = Box()
    r.coords = np.ascontiguousarray(b.coords[atoms])
    r.q = np.ascontiguousarray(b.q[atoms])
    r.type = np.ascontiguousarray(b.type[atoms])
    r.ljparams = b.ljparams
    r.box = b.box
    r.n_atoms = b.n_atoms
    r.n_home = 3 * len(home)
    # intramolecular exclusions in the new numbering (each molecule's 3 atoms are consecutive)
    r.excl_off = (2 * np.arange(b.n_atoms + 1)).astype(np.int32)
    idx = np.empty(2 * b.n_atoms, np.int32)
    base = 3 * (np.arange(b.n_atoms) // 3)
    k = np.arange(b.n_atoms) % 3
    idx[0::2] = base + (k + 1) % 3
    idx[1::2] = base + (k + 2) % 3
    r.excl_idx = idx
    assert 0 < r.n_home < b.n_atoms and nw == len(order)
    return r


def part_pairs(b, rc):
    pairs = oracle.pairs_f32(b.coords, b.coords, b.box, rc, b.excl_off, b.excl_idx)
    local = (pairs[:, 0] < b.n_home) & (pairs[:, 1] < b.n_home)
    return pairs, pairs[local], pairs[~local]


@pytest.mark.parametrize("prune", [True, False])
def test_parts_sum_to_the_oracle_and_local_reads_no_halo(nb, halo_box, prune):
    b = halo_box
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.set_home(b.n_home)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    if prune:
        pl.prune(d["coords"], 1.04)
    pairs, lp, nlp = part_pairs(b, rc)
    # local part with NaN in every halo coordinate: it must not read them
    x = d["coords"].clone()
    x[b.n_home:] = float("nan")
    E = torch.empty(2, dtype=torch.float64, device="cuda")
    pl.forces_part(nb.NB_PART_LOCAL, x, d["q"], d["type"], d["lj"], rc, beta, None, E)
    torch.cuda.synchronize()
    assert pl.status() == 0, "the local part read a halo coordinate"
    assert pl.stats()["pairs_last"] == len(lp)
    _, elj_l, ec_l = oracle.energy_forces_coul_pairs(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, lp)
    e = E.cpu().numpy().copy()
    assert rel(e[0], elj_l) <= E_TOL and rel(e[1], ec_l) <= E_TOL
    # the halo coordinates arrive; the non-local part completes the evaluation
    x[b.n_home:] = d["coords"][b.n_home:]
    F, _ = pl.forces_part(nb.NB_PART_NONLOCAL, x, d["q"], d["type"], d["lj"], rc, beta, None, E)
    torch.cuda.synchronize()
    assert pl.status() == 0
    assert pl.stats()["pairs_last"] == len(nlp)
    Fo, elj, ec = oracle.energy_forces_coul_pairs(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, pairs)
    compare_forces(F.cpu().numpy(), Fo)
    e = E.cpu().numpy()
    assert rel(e[0], elj) <= E_TOL and rel(e[1], ec) <= E_TOL
    # the whole evaluation in one call gives the same
    F2, E2 = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta)
    torch.cuda.synchronize()
    assert pl.stats()["pairs_last"] == len(pairs)
    compare_forces(F2.cpu().numpy(), Fo)
    assert rel(E2.cpu().numpy()[1], ec) <= E_TOL
    pl.close()


def test_gathered_tiles_of_both_parts_cover_r_inner(nb, halo_box):
    b = halo_box
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms)
    pl.set_home(b.n_home)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    torch.cuda.synchronize()
    assert pl.status() == 0
    tiles = pl.export_tiles()
    exp = pl.export(nb.NB_LIST_INNER)
    y = oracle.image_f32(b.coords, b.coords, b.box)
    got = expand_tile_pairs(tiles, exp["perm"], y, b.box, 1.04)
    ref = oracle.pairs_f32(b.coords, b.coords, b.box, 1.04, b.excl_off, b.excl_idx)
    assert len(pair_set(got)) == len(got), "a pair is in two tiles (or both parts)"
    assert pair_set(got) == pair_set(ref)
    pl.close()


def test_adjoint_with_a_halo(nb, halo_box):
    b = halo_box
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    g = np.random.default_rng(6).normal(size=(b.n_atoms, 3)).astype(np.float32)
    pl = nb.Pairlist(b.n_atoms)
    pl.set_home(b.n_home)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    gx, gq, glj = pl.backward(d["coords"], d["q"], d["type"], d["lj"], rc, beta, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert pl.status() == 0
    ox, oq, olj = oracle.force_vjp(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, g, b.excl_off, b.excl_idx)
    err = np.sqrt(((gx.cpu().numpy() - ox) ** 2).sum(1)).max() / np.sqrt((ox ** 2).sum(1).mean())
    assert err <= 1e-3
    pl.close()


def test_without_a_halo_the_parts_still_compose(nb):
    b = synth.water_box(2000, 5)
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms)
    pl.set_home(b.n_atoms)  # no halo
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    E = torch.empty(2, dtype=torch.float64, device="cuda")
    pl.forces_part(nb.NB_PART_LOCAL, d["coords"], d["q"], d["type"], d["lj"], rc, beta, None, E)
    F, _ = pl.forces_part(nb.NB_PART_NONLOCAL, d["coords"], d["q"], d["type"], d["lj"], rc, beta, None, E)
    torch.cuda.synchronize()
    assert pl.status() == 0
    Fo, elj, ec, _ = oracle.energy_forces(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, b.excl_off, b.excl_idx)
    compare_forces(F.cpu().numpy(), Fo)
    e = E.cpu().numpy()
    assert rel(e[0], elj) <= E_TOL and rel(e[1], ec) <= E_TOL
    pl.close()


def test_split_argument_errors(nb):
    b = synth.water_box(512, 1)
    pl = nb.Pairlist(b.n_atoms)
    for bad in (0, b.n_atoms + 1):
        with pytest.raises(nb.NBError):
            pl.set_home(bad)
    d = to_dev(b)
    pl.search(d["coords"], b.box, 0.9, d["excl_off"], d["excl_idx"])
    with pytest.raises(nb.NBError):
        nb.nb_forces_part(pl.handle, 7, d["coords"], d["q"], d["type"], d["lj"], 0.9, 3.0,
                          torch.empty((b.n_atoms, 3), device="cuda"), None)
    off = np.array([0, 768, 1536], np.int32)
    bt = nb.Pairlist.batch(off, np.stack([b.box, b.box]).astype(np.float32))
    with pytest.raises(nb.NBError):
        bt.set_home(100)
    bt.close()
    pl.close()
