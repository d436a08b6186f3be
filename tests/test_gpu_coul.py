"""GPU parity of the Coulomb options (reaction field, Ewald shift,
excluded-pair correction) with the oracle's energy_forces_coul /
force_vjp_coul, through the C ABI: forces per atom within 1e-4 rms(F),
energies within 1e-6 relative, on the 8 x 8 path (search only) and the
gathered-tile path (after a prune); the adjoint within the tolerances of
test_gpu_adjoint.py; a batch of ragged systems per system.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import E_TOL, compare_forces, rel, to_dev

pytestmark = pytest.mark.gpu

GX_TOL, GQ_TOL = 1e-3, 1e-4


@pytest.fixture(scope="module")
def nb():
    from paper_2405_01420_gb300 import nb as nbmod
    nbmod.load_library()
    return nbmod


OPTIONS = [
    dict(kind="rf", eps_rf=0.0),
    dict(kind="rf", eps_rf=78.5),
    dict(kind="rf", eps_rf=0.0, excl_corr=True),
    dict(kind="ewald", shift=True),
    dict(kind="ewald", excl_corr=True),
    dict(kind="ewald", shift=True, excl_corr=True),
]


def ids(o):
    return "-".join(f"{k}={v}" for k, v in o.items())


@pytest.mark.parametrize("opts", OPTIONS, ids=ids)
@pytest.mark.parametrize("prune", [False, True])
def test_forces_and_energies(nb, opts, prune):
    b = synth.water_box(4000, 13)  # 12,000 atoms
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms, count_pairs=True)
    pl.set_coulomb(**opts)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    if prune:
        pl.prune(d["coords"], 1.04)
    F, E = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta)
    torch.cuda.synchronize()
    assert pl.status() == 0
    # which pairs are in range is decided, on both sides, under the FP32
    # contract (for a finite eps_rf the reaction-field force does not vanish
    # at rc, so the FP64 and FP32 decisions on pairs within 1e-5 nm of rc
    # would differ by a visible force); the pair terms are FP64 in the oracle
    pairs = oracle.pairs_f32(b.coords, b.coords, b.box, rc, b.excl_off, b.excl_idx)
    assert pl.stats()["pairs_last"] == len(pairs)
    Fo, elj, ec = oracle.energy_forces_coul_pairs(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, pairs,
                                                  b.excl_off, b.excl_idx, **opts)
    compare_forces(F.cpu().numpy(), Fo)
    e = E.cpu().numpy()
    assert rel(e[0], elj) <= E_TOL, (e[0], elj)
    assert rel(e[1], ec) <= E_TOL, (e[1], ec)
    pl.close()


@pytest.mark.parametrize("opts", [dict(kind="rf", eps_rf=0.0), dict(kind="rf", eps_rf=78.5, excl_corr=True),
                                  dict(kind="ewald", excl_corr=True)], ids=ids)
@pytest.mark.parametrize("cluster_tiles", [False, True])
def test_adjoint(nb, opts, cluster_tiles):
    b = synth.water_box(512, 1)  # 1,536 atoms
    p = synth.diff_params(b, seed=5, ntype=2)
    lj = synth.combine_geometric(p["c6"], p["c12"]).astype(np.float32)
    q = p["q"].astype(np.float32)
    rc = 0.9
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    g = np.random.default_rng(4).normal(size=(b.n_atoms, 3)).astype(np.float32)
    pl = nb.Pairlist(b.n_atoms, cluster_tiles=cluster_tiles)
    pl.set_coulomb(**opts)
    pl.search(d["coords"], b.box, 1.0, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 0.94)
    gx, gq, glj = pl.backward(d["coords"], torch.from_numpy(q).cuda(), torch.from_numpy(p["type"]).cuda(),
                              torch.from_numpy(lj).cuda(), rc, beta, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert pl.status() == 0
    ox, oq, olj = oracle.force_vjp_coul(b.coords, q, p["type"], lj, b.box, rc, beta, g, b.excl_off, b.excl_idx,
                                        kind=opts["kind"], eps_rf=opts.get("eps_rf", 0.0),
                                        excl_corr=opts.get("excl_corr", False))

    def err(a, o):
        a = np.asarray(a, np.float64).reshape(len(o), -1)
        o = np.asarray(o, np.float64).reshape(len(o), -1)
        return float(np.sqrt(((a - o) ** 2).sum(1)).max() / np.sqrt((o ** 2).sum(1).mean()))

    assert err(gx.cpu().numpy(), ox) <= GX_TOL
    assert err(gq.cpu().numpy(), oq) <= GQ_TOL
    np.testing.assert_allclose(glj.cpu().numpy(), olj, rtol=1e-4, atol=1e-6 * np.abs(olj).max())
    pl.close()


def test_batch_with_reaction_field_and_correction(nb):
    sizes = [1536, 903, 3000]
    boxes = [synth.water_box_for_atoms(n, 30 + k) for k, n in enumerate(sizes)]
    x = np.concatenate([bx.coords for bx in boxes])
    q = np.concatenate([bx.q for bx in boxes])
    t = np.concatenate([bx.type for bx in boxes])
    off = np.cumsum([0] + [bx.n_atoms for bx in boxes]).astype(np.int32)
    eo = [np.zeros(1, np.int32)]
    ei = []
    for k, bx in enumerate(boxes):
        eo.append(bx.excl_off[1:] + eo[-1][-1])
        ei.append(bx.excl_idx + off[k])
    eo = np.concatenate(eo).astype(np.int32)
    ei = np.concatenate(ei).astype(np.int32)
    L = np.stack([bx.box for bx in boxes]).astype(np.float32)
    rc = 0.9
    pl = nb.Pairlist.batch(off, L)
    pl.set_coulomb(kind="rf", eps_rf=0.0, excl_corr=True)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    pl.search(dev(x), None, 1.0, dev(eo), dev(ei))
    pl.prune(dev(x), 0.94)
    F, E = pl.forces(dev(x), dev(q), dev(t), dev(boxes[0].ljparams), rc, 0.0)
    torch.cuda.synchronize()
    assert pl.status() == 0
    F = F.cpu().numpy()
    E = E.cpu().numpy()
    for k, bx in enumerate(boxes):
        pairs = oracle.pairs_f32(bx.coords, bx.coords, bx.box, rc, bx.excl_off, bx.excl_idx)
        Fo, elj, ec = oracle.energy_forces_coul_pairs(bx.coords, bx.q, bx.type, bx.ljparams, bx.box, rc, 0.0, pairs,
                                                      bx.excl_off, bx.excl_idx, kind="rf", eps_rf=0.0, excl_corr=True)
        compare_forces(F[off[k]:off[k + 1]], Fo)
        assert rel(E[2 * k], elj) <= E_TOL
        assert rel(E[2 * k + 1], ec) <= E_TOL
    pl.close()


def test_coulomb_argument_errors(nb):
    b = synth.water_box(512, 1)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms)
    for bad in [dict(kind=5), dict(kind=nb.NB_COUL_RF, flags=nb.NB_COUL_SHIFT), dict(kind=nb.NB_COUL_RF, eps_rf=0.5),
                dict(kind=nb.NB_COUL_EWALD, flags=0x10)]:
        with pytest.raises(nb.NBError) as e:
            nb.nb_set_coulomb(pl.handle, bad.get("kind", 0), bad.get("eps_rf", 0.0), bad.get("flags", 0))
        assert e.value.code == nb.NB_ERR_ARG
    # the correction needs the exclusion lists of the search
    pl.set_coulomb(kind="ewald", excl_corr=True)
    pl.search(d["coords"], b.box, 0.9)
    with pytest.raises(nb.NBError) as e:
        pl.forces(d["coords"], d["q"], d["type"], d["lj"], 0.9, synth.ewald_beta(0.9))
    assert e.value.code == nb.NB_ERR_STATE
    # ... given to a search made while the correction was set: turned on after the search, it is refused
    pl.set_coulomb(kind="ewald")
    pl.search(d["coords"], b.box, 0.9, d["excl_off"], d["excl_idx"])
    pl.set_coulomb(kind="ewald", excl_corr=True)
    with pytest.raises(nb.NBError) as e:
        pl.forces(d["coords"], d["q"], d["type"], d["lj"], 0.9, synth.ewald_beta(0.9))
    assert e.value.code == nb.NB_ERR_STATE
    with pytest.raises(nb.NBError) as e:
        pl.backward(d["coords"], d["q"], d["type"], d["lj"], 0.9, synth.ewald_beta(0.9),
                    torch.zeros((b.n_atoms, 3), device="cuda"))
    assert e.value.code == nb.NB_ERR_STATE
    pl.close()
