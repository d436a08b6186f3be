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


def _system_of(n_atoms, seed):
    """A water box of n_atoms; a count that is not a multiple of 3 gets one
    or two extra uncharged atoms of the LJ-free type at random positions."""
    b = synth.water_box(max(1, n_atoms // 3), seed)
    extra = n_atoms - b.n_atoms
    if extra == 0:
        return b
    rng = np.random.default_rng(seed)
    L = b.box.astype(np.float64)
    b.coords = np.concatenate([b.coords, (rng.uniform(0, 1, (extra, 3)) * L).astype(np.float32)])
    b.q = np.concatenate([b.q, np.zeros(extra, np.float32)])
    b.type = np.concatenate([b.type, np.full(extra, b.ljparams.shape[0] - 1, np.int32)])
    b.excl_off = np.concatenate([b.excl_off, np.full(extra, b.excl_off[-1], b.excl_off.dtype)])
    return b


def _noalloc(nb, b, d, x, box, rc, beta):
    F = torch.full((b.n_atoms, 3), float("nan"), dtype=torch.float32, device="cuda")
    E = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    word = nb.nb_forces_noalloc(x, box, d["q"], d["type"], d["lj"], rc, beta, F, E, d["excl_off"], d["excl_idx"])
    assert word == 0, f"device error word 0x{word:x}"
    return F, E


def _regular_box(nb, b, d, x, box, rc, beta):
    pl = nb.Pairlist(b.n_atoms)
    pl.search(x, box, rc, d["excl_off"], d["excl_idx"])
    F, E = pl.forces(x, d["q"], d["type"], d["lj"], rc, beta)
    assert pl.status() == 0
    pl.close()
    return F.cpu().numpy().astype(np.float64), E.cpu().numpy()


def _agree(F, E, F_ref, E_ref, what):
    Fn = F.cpu().numpy().astype(np.float64)
    assert np.isfinite(Fn).all(), what
    rms = np.sqrt((F_ref ** 2).sum(1).mean())
    if rms > 0:
        assert np.sqrt(((Fn - F_ref) ** 2).sum(1)).max() <= 1e-4 * rms, what
    else:
        assert not Fn.any(), what
    e = E.cpu().numpy()
    for k in range(2):
        if E_ref[k] == 0.0:
            assert e[k] == 0.0, (what, e, E_ref)
        else:
            assert rel(e[k], E_ref[k]) <= E_TOL, (what, e, E_ref)


def test_noalloc_at_its_atom_limit_with_the_largest_cutoff():
    """4,096 atoms (the limit) with rc one float below half the box edge:
    the densest pair list the call can be asked for fits its scratch list."""
    from paper_2405_01420_gb300 import nb
    nb.load_library()
    b = _system_of(nb.NB_NOALLOC_MAX_ATOMS, 41)
    assert b.n_atoms == nb.NB_NOALLOC_MAX_ATOMS
    rc = float(np.nextafter(np.float32(0.5) * b.box.astype(np.float32).min(), np.float32(0)))
    assert np.all(b.box.astype(np.float32) > np.float32(2) * np.float32(rc))
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    x = d["coords"]
    F, E = _noalloc(nb, b, d, x, b.box, rc, beta)
    _agree(F, E, *_regular_box(nb, b, d, x, b.box, rc, beta), "4096 atoms, rc just below L/2")


def test_noalloc_large_then_small_allocates_nothing():
    """A call at the limit, then a single water (one cluster, one grid column),
    then a 6-atom system, then the limit again: each against the regular
    entry point. The later calls reuse scratch that an earlier, larger call
    filled, past the smaller system's clusters. Around the calls the free
    device memory and torch's allocated bytes must not move."""
    from paper_2405_01420_gb300 import nb
    nb.load_library()
    cases = []
    for n, seed, box in ((4096, 42, None), (3, 1, [3.0, 3.0, 3.0]), (6, 5, [2.0, 2.0, 2.0]), (4095, 43, None)):
        b = _system_of(n, seed)
        box = b.box if box is None else np.asarray(box, np.float32)
        d = to_dev(b)
        F = torch.full((b.n_atoms, 3), float("nan"), dtype=torch.float32, device="cuda")
        E = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        cases.append((b, box, d, F, E))
    rc = 0.9
    beta = synth.ewald_beta(rc)

    def run_all():
        for b, box, d, F, E in cases:
            word = nb.nb_forces_noalloc(d["coords"], box, d["q"], d["type"], d["lj"], rc, beta, F, E,
                                        d["excl_off"], d["excl_idx"])
            assert word == 0, f"{b.n_atoms} atoms: device error word 0x{word:x}"

    run_all()  # loads every kernel the calls use (a first launch may map code into device memory)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    run_all()
    run_all()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "free device memory changed across the calls"
    assert torch.cuda.memory_allocated() == alloc0
    for b, box, d, F, E in cases:
        _agree(F, E, *_regular_box(nb, b, d, d["coords"], box, rc, beta), f"{b.n_atoms} atoms")


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
