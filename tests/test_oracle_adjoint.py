"""Pins for the oracle's force adjoint (vector-Jacobian product).

The adjoint is checked against central finite differences of phi = g . F,
computed through the independent force code path, and against two
invariants: translation invariance (sum of dphi/dx_k = 0) and the symmetry
of the Hessian (v . J(w) = w . J(v), since J = dF/dx = -H is symmetric).
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def system():
    b = synth.water_box(216, 8)  # 648 atoms, L = 1.86 nm
    p = synth.diff_params(b, seed=8)
    lj = synth.combine_geometric(p["c6"], p["c12"])
    rc = 0.9
    beta = synth.ewald_beta(rc)
    rng = np.random.default_rng(1)
    g = rng.normal(size=(b.n_atoms, 3))
    return b, p["q"], p["type"], lj, rc, beta, g


def phi(b, x, q, t, lj, rc, beta, g):
    F, _, _, n = oracle.energy_forces(x, q, t, lj, b.box, rc, beta, b.excl_off, b.excl_idx, "n2")
    return float((g * F).sum()), n


def vjp(b, x, q, t, lj, rc, beta, g):
    return oracle.force_vjp(x, q, t, lj, b.box, rc, beta, g, b.excl_off, b.excl_idx)


def test_vjp_positions_match_finite_differences(system):
    b, q, t, lj, rc, beta, g = system
    x = b.coords.astype(np.float64)
    gx, _, _ = vjp(b, x, q, t, lj, rc, beta, g)
    _, n0 = phi(b, x, q, t, lj, rc, beta, g)
    h = 1e-5
    rng = np.random.default_rng(2)
    checked = 0
    for atom in rng.choice(b.n_atoms, 10, replace=False):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[atom, k] += h
            xm[atom, k] -= h
            fp, np_ = phi(b, xp, q, t, lj, rc, beta, g)
            fm, nm = phi(b, xm, q, t, lj, rc, beta, g)
            if np_ != n0 or nm != n0:
                continue  # a pair crossed rc: the force is discontinuous there
            fd = (fp - fm) / (2 * h)
            assert fd == pytest.approx(gx[atom, k], rel=1e-5, abs=1e-3), (atom, k)
            checked += 1
    assert checked >= 24


def test_vjp_charges_match_finite_differences(system):
    b, q, t, lj, rc, beta, g = system
    x = b.coords.astype(np.float64)
    _, gq, _ = vjp(b, x, q, t, lj, rc, beta, g)
    for atom in (0, 1, 5, 100, 647):
        h = 1e-3
        qp, qm = q.copy(), q.copy()
        qp[atom] += h
        qm[atom] -= h
        fd = (phi(b, x, qp, t, lj, rc, beta, g)[0] - phi(b, x, qm, t, lj, rc, beta, g)[0]) / (2 * h)
        assert fd == pytest.approx(gq[atom], rel=1e-7, abs=1e-9)


def test_vjp_lj_matches_finite_differences(system):
    b, q, t, lj, rc, beta, g = system
    x = b.coords.astype(np.float64)
    _, _, glj = vjp(b, x, q, t, lj, rc, beta, g)
    np.testing.assert_allclose(glj, glj.transpose(1, 0, 2), rtol=1e-12, atol=0)
    for (a, c) in [(0, 0), (0, 1), (2, 3), (3, 3)]:
        for comp in (0, 1):
            h = 1e-3 * lj[a, c, comp]
            lp, lm = lj.copy(), lj.copy()
            lp[a, c, comp] += h
            lm[a, c, comp] -= h
            if a != c:
                lp[c, a, comp] += h
                lm[c, a, comp] -= h
            fd = (phi(b, x, q, t, lp, rc, beta, g)[0] - phi(b, x, q, t, lm, rc, beta, g)[0]) / (2 * h)
            want = glj[a, c, comp] + (glj[c, a, comp] if a != c else 0.0)
            assert fd == pytest.approx(want, rel=1e-6), (a, c, comp)


def test_vjp_translation_invariance_and_hessian_symmetry(system):
    b, q, t, lj, rc, beta, g = system
    x = b.coords.astype(np.float64)
    gx, _, _ = vjp(b, x, q, t, lj, rc, beta, g)
    assert np.abs(gx.sum(0)).max() <= 1e-10 * np.abs(gx).max() * b.n_atoms
    rng = np.random.default_rng(4)
    v = rng.normal(size=g.shape)
    w = rng.normal(size=g.shape)
    jv, _, _ = vjp(b, x, q, t, lj, rc, beta, v)
    jw, _, _ = vjp(b, x, q, t, lj, rc, beta, w)
    assert float((v * jw).sum()) == pytest.approx(float((w * jv).sum()), rel=1e-10)


def test_force_matching_loss_gradient(system):
    """dL/dx of L = (1/3N) sum |F - T|^2 by finite differences of L itself."""
    b, q, t, lj, rc, beta, _ = system
    x = b.coords.astype(np.float64)
    rng = np.random.default_rng(6)
    T = rng.normal(scale=100.0, size=(b.n_atoms, 3))
    L, gx, gq, glj, F = oracle.force_matching(x, q, t, lj, b.box, rc, beta, T, b.excl_off, b.excl_idx)
    assert L == pytest.approx(((F - T) ** 2).sum() / (3 * b.n_atoms), rel=1e-14)
    h = 1e-5
    atom, k = 17, 1
    xp, xm = x.copy(), x.copy()
    xp[atom, k] += h
    xm[atom, k] -= h
    Lp = oracle.force_matching(xp, q, t, lj, b.box, rc, beta, T, b.excl_off, b.excl_idx)[0]
    Lm = oracle.force_matching(xm, q, t, lj, b.box, rc, beta, T, b.excl_off, b.excl_idx)[0]
    assert (Lp - Lm) / (2 * h) == pytest.approx(gx[atom, k], rel=1e-4)
