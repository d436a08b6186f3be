"""The allocation-free entry point against the regular one.

nb_forces_noalloc serves callers that cannot allocate device memory (a
plug-in whose host program owns every device allocation, or a real-time
loop that must not enter the allocator): it keeps all scratch memory in a
static device array. Here it must give the same forces and energies as
nb_search + nb_forces on a pair list created the usual way, within the
tolerances of the other parity tests, on two calls in a row (the second
one reuses the array the first one left behind, with new coordinates).
This file is collected last so that a failure here stops a run only after
every other test has run.
"""
import numpy as np
import pytest
import torch

import synth
from gpu_common import E_TOL, rel, to_dev

pytestmark = pytest.mark.gpu


def regular(nb, b, d, x, rc, beta):
    pl = nb.Pairlist(b.n_atoms)
    pl.search(x, b.box, rc, d["excl_off"], d["excl_idx"])
    F, E = pl.forces(x, d["q"], d["type"], d["lj"], rc, beta)
    assert pl.status() == 0
    pl.close()
    return F.cpu().numpy().astype(np.float64), E.cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice():
    from paper_2405_01420_gb300 import nb
    nb.load_library()
    b = synth.water_box(512, 1)  # 1,536 atoms
    rc = 0.9
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    frames = synth.random_walk_frames(b, 2, 0.002, seed=77)
    for call in range(2):
        x = torch.from_numpy(frames[call]).cuda()
        F = torch.full((b.n_atoms, 3), float("nan"), dtype=torch.float32, device="cuda")
        E = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        word = nb.nb_forces_noalloc(x, b.box, d["q"], d["type"], d["lj"], rc, beta, F, E, d["excl_off"],
                                    d["excl_idx"])
        assert word == 0, f"call {call}: device error word 0x{word:x}"
        F_ref, E_ref = regular(nb, b, d, x, rc, beta)
        Fn = F.cpu().numpy().astype(np.float64)
        rms = np.sqrt((F_ref ** 2).sum(1).mean())
        assert np.isfinite(Fn).all()
        assert np.sqrt(((Fn - F_ref) ** 2).sum(1)).max() <= 1e-4 * rms, call
        e = E.cpu().numpy()
        assert rel(e[0], E_ref[0]) <= E_TOL and rel(e[1], E_ref[1]) <= E_TOL, (call, e, E_ref)


def test_noalloc_rejects_too_many_atoms():
    from paper_2405_01420_gb300 import nb
    n = nb.NB_NOALLOC_MAX_ATOMS + 1
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    q = torch.zeros(n, dtype=torch.float32, device="cuda")
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    lj = torch.zeros((1, 1, 2), dtype=torch.float32, device="cuda")
    F = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(nb.NBError) as e:
        nb.nb_forces_noalloc(x, [10.0, 10.0, 10.0], q, t, lj, 0.9, 3.0, F)
    assert e.value.code == nb.NB_ERR_CAPACITY
    assert "NB_NOALLOC_MAX_ATOMS" in str(e.value)
