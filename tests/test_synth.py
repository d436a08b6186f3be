"""The seeded input generator against the workload recipe it states: water
geometry, density, charges, LJ table, exclusions, close contacts, the Ewald
splitting parameter, the random walk and the force-matching parameters."""
import math

import numpy as np
import pytest

import synth


def molecules(b):
    """Atom positions [M, 3 (O, H, H), 3], each molecule made whole by minimum image from its O."""
    x = b.coords.astype(np.float64).reshape(-1, 3, 3)
    L = b.box.astype(np.float64)
    d = x - x[:, :1, :]
    return x[:, :1, :] + d - L * np.rint(d / L)


@pytest.mark.parametrize("nw, seed", [(512, 1), (1000, 7), (37, 3)])
def test_rigid_water_geometry_and_box(nw, seed):
    b = synth.water_box(nw, seed)
    assert b.n_atoms == 3 * nw and b.coords.dtype == np.float32
    L = float(b.box[0])
    assert np.allclose(b.box, L)
    assert nw / L ** 3 == pytest.approx(33.4, rel=1e-5)
    assert (b.coords >= 0).all() and (b.coords < b.box).all()
    m = molecules(b)
    oh1 = np.linalg.norm(m[:, 1] - m[:, 0], axis=1)
    oh2 = np.linalg.norm(m[:, 2] - m[:, 0], axis=1)
    assert np.allclose(oh1, 0.1, atol=2e-6) and np.allclose(oh2, 0.1, atol=2e-6)
    cosang = ((m[:, 1] - m[:, 0]) * (m[:, 2] - m[:, 0])).sum(1) / (oh1 * oh2)
    assert np.allclose(np.degrees(np.arccos(cosang)), 109.47, atol=2e-3)


def test_documented_box_edges():
    assert synth.box_edge(512) == pytest.approx(2.4841, abs=1e-4)
    assert synth.box_edge(8000) == pytest.approx(6.2103, abs=1e-4)
    assert synth.box_edge(32000) == pytest.approx(9.8583, abs=1e-4)
    assert synth.box_edge(333334) == pytest.approx(21.530, abs=1e-3)


def test_charges_types_lj_and_exclusions():
    b = synth.water_box(64, 5)
    assert np.array_equal(b.q[:3], np.array([-0.8476, 0.4238, 0.4238], np.float32))
    assert abs(float(b.q.astype(np.float64).sum())) < 1e-5
    assert np.array_equal(b.type[:3], [0, 1, 1]) and b.ntype == 2
    sigma, eps = 0.3166, 0.650
    assert b.ljparams[0, 0, 0] == pytest.approx(4 * eps * sigma ** 6, rel=1e-6)
    assert b.ljparams[0, 0, 1] == pytest.approx(4 * eps * sigma ** 12, rel=1e-6)
    assert (b.ljparams[0, 1] == 0).all() and (b.ljparams[1, 0] == 0).all() and (b.ljparams[1, 1] == 0).all()
    # each atom excludes exactly the other two atoms of its molecule, symmetrically
    N = b.n_atoms
    assert np.array_equal(b.excl_off, 2 * np.arange(N + 1))
    pairs = set()
    for i in range(N):
        js = b.excl_idx[b.excl_off[i]:b.excl_off[i + 1]]
        assert sorted(js) == sorted(set(range(3 * (i // 3), 3 * (i // 3) + 3)) - {i})
        pairs.update((i, int(j)) for j in js)
    assert all((j, i) in pairs for i, j in pairs)


def test_no_close_contacts_between_molecules():
    b = synth.water_box(216, 11)
    x = b.coords.astype(np.float64)
    L = b.box.astype(np.float64)
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    mol = np.arange(b.n_atoms) // 3
    other = mol[:, None] != mol[None, :]
    assert r[other].min() >= 0.15 - 1e-6


def test_generator_is_seeded():
    a, b, c = synth.water_box(100, 4), synth.water_box(100, 4), synth.water_box(100, 5)
    assert np.array_equal(a.coords, b.coords)
    assert not np.array_equal(a.coords, c.coords)


@pytest.mark.parametrize("rc", [0.9, 1.0, 1.2])
def test_ewald_beta_meets_its_tolerance(rc):
    beta = synth.ewald_beta(rc)
    assert math.erfc(beta * rc) == pytest.approx(1e-5, rel=1e-6)
    assert beta * rc == pytest.approx(3.1234132743, rel=1e-8)


def test_random_walk():
    b = synth.water_box(500, 2)
    sigma = 0.001
    f = synth.random_walk_frames(b, 6, sigma, seed=9)
    assert f.shape == (6, b.n_atoms, 3) and f.dtype == np.float32
    assert (f >= 0).all() and (f < b.box).all()
    L = b.box.astype(np.float64)
    prev = b.coords.astype(np.float64)
    for k in range(6):
        step = f[k].astype(np.float64) - prev
        step -= L * np.rint(step / L)
        assert step.std() == pytest.approx(sigma, rel=0.05)  # 4,500 samples per frame
        assert abs(step.mean()) < 5 * sigma / math.sqrt(step.size)
        prev = f[k].astype(np.float64)
    assert np.array_equal(f, synth.random_walk_frames(b, 6, sigma, seed=9))


def test_force_matching_parameters():
    b = synth.water_box(8000, 4)
    p = synth.diff_params(b, seed=4)
    q = p["q"]
    assert abs(q.sum()) < 1e-9 * b.n_atoms
    assert q.std() == pytest.approx(0.4, rel=0.02)
    assert set(np.unique(p["type"])) == {0, 1, 2, 3}
    assert ((p["c6"] >= 1e-3) & (p["c6"] <= 3e-3)).all()
    assert ((p["c12"] >= 1e-6) & (p["c12"] <= 3e-6)).all()
    lj = synth.combine_geometric(p["c6"], p["c12"])
    assert lj.shape == (4, 4, 2)
    assert np.allclose(lj, lj.transpose(1, 0, 2))
    assert np.allclose(lj[np.arange(4), np.arange(4), 0], p["c6"])
    assert lj[0, 1, 1] == pytest.approx(math.sqrt(p["c12"][0] * p["c12"][1]))


def test_batch_boxes():
    boxes = synth.batch_boxes(n_boxes=6, lo=1536, hi=3000, seed=5)
    assert len(boxes) == 6
    for b in boxes:
        assert 1536 - 2 <= b.n_atoms <= 3000 and b.n_atoms % 3 == 0
        assert b.n_waters / float(b.box[0]) ** 3 == pytest.approx(33.4, rel=1e-5)
    assert len({b.n_atoms for b in boxes}) > 1  # uneven sizes
    again = synth.batch_boxes(n_boxes=6, lo=1536, hi=3000, seed=5)
    assert all(np.array_equal(a.coords, b.coords) for a, b in zip(boxes, again))
