"""Every force-kernel launch shape gives the same (oracle-parity) results; the
autotuner runs on the GPU and leaves a valid shape selected."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import E_TOL, compare_forces, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2405_01420_gb300 import nb
    nb.load_library()
    b = synth.water_box(4000, 21)
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    pl = nb.Pairlist(b.n_atoms)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    Fo, elj, ec, _ = oracle.energy_forces(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, b.excl_off,
                                          b.excl_idx)
    yield nb, b, d, pl, rc, beta, Fo, elj, ec
    pl.close()


@pytest.mark.parametrize("shape", [(256, 16, 0), (256, 8, 0), (128, 16, 0), (128, 8, 0), (256, 16, 1), (128, 8, 3)])
def test_force_shapes_agree_with_oracle(setup, shape):
    nb, b, d, pl, rc, beta, Fo, elj, ec = setup
    nb.nb_set_force_shape(pl.handle, *shape)
    F, E = pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta)
    assert pl.status() == 0
    compare_forces(F.cpu().numpy(), Fo)
    e = E.cpu().numpy()
    assert rel(e[0], elj) <= E_TOL and rel(e[1], ec) <= E_TOL
    nb.nb_set_force_shape(pl.handle, 0, 0, 0)


def test_bad_shape_rejected(setup):
    nb, b, d, pl, rc, beta, *_ = setup
    with pytest.raises(nb.NBError):
        nb.nb_set_force_shape(pl.handle, 96, 16, 0)


def test_autotuner_selects_a_shape(setup):
    from paper_2405_01420_gb300.tune import tune_force_shape
    nb, b, d, pl, rc, beta, Fo, elj, ec = setup
    F = torch.empty((b.n_atoms, 3), dtype=torch.float32, device="cuda")
    E = torch.empty(2, dtype=torch.float64, device="cuda")
    best, times = tune_force_shape(pl, lambda: pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta, F, E),
                                   reps=3)
    assert best in [tuple(s) for s in [(256, 16, 0), (256, 8, 0), (128, 16, 0), (128, 8, 0), (256, 16, 3),
                                       (128, 16, 6)]]
    assert all(t is not None and t > 0 for t in times.values())
    pl.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta, F, E)
    compare_forces(F.cpu().numpy(), Fo)
    nb.nb_set_force_shape(pl.handle, 0, 0, 0)


def test_tile_form_tuner_after_prune(setup):
    """Both tile forms meet the oracle bar; the tuner leaves the pair list on one of them."""
    from paper_2405_01420_gb300.tune import tune_tile_form
    nb, b, d, pl, rc, beta, Fo, elj, ec = setup
    q = nb.Pairlist(b.n_atoms)
    q.search(d["coords"], b.box, rc + 0.1, d["excl_off"], d["excl_idx"])
    q.prune(d["coords"], rc + 0.04)
    F = torch.empty((b.n_atoms, 3), dtype=torch.float32, device="cuda")
    E = torch.empty(2, dtype=torch.float64, device="cuda")
    call = lambda: q.forces(d["coords"], d["q"], d["type"], d["lj"], rc, beta, F, E)
    for form in ("gathered", "cluster"):
        q.set_flags(cluster_tiles=(form == "cluster"))
        call()
        torch.cuda.synchronize()
        compare_forces(F.cpu().numpy(), Fo)
    best, times = tune_tile_form(q, call, reps=3)
    assert best in ("gathered", "cluster") and all(t > 0 for t in times.values())
    call()
    compare_forces(F.cpu().numpy(), Fo)
    with pytest.raises(nb.NBError):
        nb.nb_set_flags(q.handle, 0x80)
    q.close()
