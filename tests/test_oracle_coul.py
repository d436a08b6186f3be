"""Pins for the oracle's Coulomb options: reaction field, Ewald potential
shift, excluded-pair correction (oracle_energy_forces_coul /
oracle_force_vjp_coul).

None of these re-types the options' formulas. Each checks a consequence
against something fixed independently: the already-pinned Ewald path (the
default options, and reaction field at eps_rf = 1, which is bare Coulomb
shifted to 0 at rc), the vanishing of the reaction-field energy and, for
eps_rf = infinity, force at rc, the exact identity erf = 1 - erfc applied to
whole systems (a run with exclusions and the correction equals a run without
exclusion lists minus the excluded pairs' bare Coulomb terms), F = -dE/dx by
central differences, and the adjoint against finite differences of g.F.
"""
import numpy as np
import pytest

import oracle
import synth

F_COUL = 138.935458


@pytest.fixture(scope="module")
def box():
    b = synth.water_box(200, 1)  # 600 atoms, L = 1.815 nm
    return b


def run(b, x=None, **kw):
    x = b.coords if x is None else x
    return oracle.energy_forces_coul(x, b.q, b.type, b.ljparams, b.box, kw.pop("rc", 0.9), kw.pop("beta", 3.47),
                                     b.excl_off, b.excl_idx, **kw)


def two_atoms(r, q1=0.7, q2=-0.4, L=10.0):
    u = np.array([1.0, 2.0, -0.5])
    u /= np.linalg.norm(u)
    c = np.full(3, L / 2)
    x = np.stack([c + 0.5 * r * u, c - 0.5 * r * u])
    return x, np.array([q1, q2]), np.zeros(2, np.int32), np.zeros((1, 1, 2)), np.array([L, L, L]), u


def excluded_pairs(b):
    """(i, j) with i < j from the exclusion lists."""
    out = []
    for i in range(b.n_atoms):
        for k in range(b.excl_off[i], b.excl_off[i + 1]):
            j = int(b.excl_idx[k])
            if j > i:
                out.append((i, j))
    return out


def bare_coulomb_of(b, pairs, x=None):
    """Energy and forces of plain Coulomb f q_i q_j / r over the given pairs (minimum image)."""
    x = b.coords.astype(np.float64) if x is None else x
    E = 0.0
    F = np.zeros((b.n_atoms, 3))
    for i, j in pairs:
        d = x[i] - x[j]
        d -= b.box * np.rint(d / b.box)
        r = np.linalg.norm(d)
        K = F_COUL * float(b.q[i]) * float(b.q[j])
        E += K / r
        F[i] += K / r ** 3 * d
        F[j] -= K / r ** 3 * d
    return E, F


# ---------------------------------------------------------------- consistency

def test_default_options_equal_the_plain_oracle(box):
    b = box
    F0, el0, ec0, n0 = oracle.energy_forces(b.coords, b.q, b.type, b.ljparams, b.box, 0.9, 3.47, b.excl_off,
                                            b.excl_idx)
    F1, el1, ec1, n1 = run(b)
    assert n0 == n1
    assert el1 == pytest.approx(el0, rel=1e-12)
    assert ec1 == pytest.approx(ec0, rel=1e-12)
    assert np.abs(F1 - F0).max() <= 1e-9 * np.abs(F0).max()


def test_rf_at_eps_one_is_shifted_bare_coulomb(box):
    """eps_rf = 1: k_rf = 0, c_rf = 1/rc, i.e. f q q (1/r - 1/rc): the Ewald
    path at beta = 0 (erfc = 1, pinned to Coulomb's law) with the shift."""
    b = box
    Fr, elr, ecr, nr = run(b, kind="rf", eps_rf=1.0)
    Fe, ele, ece, ne = run(b, kind="ewald", beta=0.0, shift=True)
    assert nr == ne
    assert ecr == pytest.approx(ece, rel=1e-11)
    assert elr == pytest.approx(ele, rel=1e-12)
    assert np.abs(Fr - Fe).max() <= 1e-9 * np.abs(Fe).max()


@pytest.mark.parametrize("opts", [dict(kind="rf", eps_rf=78.5, excl_corr=True), dict(kind="ewald", shift=True),
                                  dict(kind="ewald", excl_corr=True)])
def test_explicit_pair_set_equals_the_cutoff_form(box, opts):
    """Given the FP64 brute-force pair set, the explicit-set form equals the cutoff form."""
    b = box
    pairs = oracle.pairs_f64(b.coords, b.box, 0.9, b.excl_off, b.excl_idx)
    F1, el1, ec1, n1 = run(b, **dict(opts))
    F2, el2, ec2 = oracle.energy_forces_coul_pairs(b.coords, b.q, b.type, b.ljparams, b.box, 0.9, 3.47, pairs,
                                                   b.excl_off, b.excl_idx, **opts)
    assert len(pairs) == n1
    assert el2 == pytest.approx(el1, rel=1e-12)
    assert ec2 == pytest.approx(ec1, rel=1e-11)
    assert np.abs(F2 - F1).max() <= 1e-9 * np.abs(F1).max()


# ---------------------------------------------------------------- reaction field at the cutoff

@pytest.mark.parametrize("eps_rf", [0.0, 78.5, 4.0])
def test_rf_pair_energy_vanishes_at_cutoff(eps_rf):
    rc = 0.9
    x, q, t, lj, L, _ = two_atoms(rc * (1 - 1e-9))
    _, _, ec, n = oracle.energy_forces_coul(x, q, t, lj, L, rc, 0.0, kind="rf", eps_rf=eps_rf)
    assert n == 1
    x2, *_ = two_atoms(0.3)
    _, _, ec_in, _ = oracle.energy_forces_coul(x2, q, t, lj, L, rc, 0.0, kind="rf", eps_rf=eps_rf)
    assert abs(ec) <= 1e-7 * abs(ec_in)


def test_rf_force_vanishes_at_cutoff_for_conducting_boundary():
    """eps_rf = infinity (conducting boundary): the force goes to 0 at rc too;
    for a finite eps_rf it does not."""
    rc = 0.9
    x, q, t, lj, L, u = two_atoms(rc * (1 - 1e-9))
    F, _, _, _ = oracle.energy_forces_coul(x, q, t, lj, L, rc, 0.0, kind="rf", eps_rf=0.0)
    x2, *_ = two_atoms(0.3)
    F2, _, _, _ = oracle.energy_forces_coul(x2, q, t, lj, L, rc, 0.0, kind="rf", eps_rf=0.0)
    assert np.abs(F).max() <= 1e-6 * np.abs(F2).max()
    F3, _, _, _ = oracle.energy_forces_coul(x, q, t, lj, L, rc, 0.0, kind="rf", eps_rf=4.0)
    assert np.abs(F3).max() >= 1e-3 * np.abs(F2).max()
    # a huge finite eps_rf approaches the conducting boundary
    F4, _, e4, _ = oracle.energy_forces_coul(x2, q, t, lj, L, rc, 0.0, kind="rf", eps_rf=1e12)
    F5, _, e5, _ = oracle.energy_forces_coul(x2, q, t, lj, L, rc, 0.0, kind="rf", eps_rf=0.0)
    assert e4 == pytest.approx(e5, rel=1e-9)


def test_ewald_shift_vanishes_at_cutoff_and_keeps_forces(box):
    rc, beta = 0.9, 3.47
    x, q, t, lj, L, _ = two_atoms(rc * (1 - 1e-9))
    _, _, ec, n = oracle.energy_forces_coul(x, q, t, lj, L, rc, beta, shift=True)
    _, _, ec_u, _ = oracle.energy_forces_coul(x, q, t, lj, L, rc, beta, shift=False)
    assert n == 1 and abs(ec_u) > 1e-5
    assert abs(ec) <= 1e-9 * abs(ec_u) / 1e-5
    Fs, _, ecs, _ = run(box, shift=True)
    Fu, _, ecu, _ = run(box, shift=False)
    assert np.array_equal(Fs, Fu)
    assert ecs != ecu


# ---------------------------------------------------------------- exclusion correction

@pytest.mark.parametrize("kind,eps_rf", [("ewald", 0.0), ("rf", 0.0), ("rf", 78.5)])
def test_exclusion_correction_identity(box, kind, eps_rf):
    """With exclusions and the correction, excluded pairs carry (erfc - 1)/r
    (Ewald) or k r^2 - c (RF): exactly the run without exclusion lists minus
    the excluded pairs' bare Coulomb f q q / r, in energy and forces. (The
    no-exclusion run also counts LJ on excluded pairs; H has no LJ and O-O
    pairs are never excluded in water, so LJ agrees.)"""
    b = box
    Fc, elc, ecc, _ = run(b, kind=kind, eps_rf=eps_rf, excl_corr=True)
    Fn, eln, ecn, _ = oracle.energy_forces_coul(b.coords, b.q, b.type, b.ljparams, b.box, 0.9, 3.47, None, None,
                                                kind=kind, eps_rf=eps_rf)
    Eb, Fb = bare_coulomb_of(b, excluded_pairs(b))
    assert elc == pytest.approx(eln, rel=1e-12)
    assert ecc == pytest.approx(ecn - Eb, rel=1e-10, abs=1e-9 * abs(Eb))
    assert np.abs(Fc - (Fn - Fb)).max() <= 1e-8 * np.abs(Fn).max()
    # and the correction changes the result
    Fx, _, ecx, _ = run(b, kind=kind, eps_rf=eps_rf, excl_corr=False)
    assert abs(ecx - ecc) > 1e-3 * abs(ecc)


# ---------------------------------------------------------------- F = -dE/dx

@pytest.mark.parametrize("opts", [dict(kind="rf", eps_rf=0.0), dict(kind="rf", eps_rf=78.5, excl_corr=True),
                                  dict(kind="ewald", excl_corr=True), dict(kind="ewald", shift=True)])
def test_forces_are_minus_energy_gradient(box, opts):
    b = box
    x = b.coords.astype(np.float64)
    F, _, _, n = run(b, x=x, **dict(opts))
    rng = np.random.default_rng(5)
    h = 1e-6
    checked = 0
    for atom in rng.choice(b.n_atoms, 10, replace=False):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[atom, k] += h
            xm[atom, k] -= h
            _, elp, ecp, np_ = run(b, x=xp, **dict(opts))
            _, elm, ecm, nm = run(b, x=xm, **dict(opts))
            if np_ != n or nm != n:
                continue
            fd = -((elp + ecp) - (elm + ecm)) / (2 * h)
            assert fd == pytest.approx(F[atom, k], rel=1e-6, abs=1e-4), (atom, k)
            checked += 1
    assert checked >= 25


# ---------------------------------------------------------------- adjoint

@pytest.fixture(scope="module")
def small():
    b = synth.water_box(64, 9)  # 192 atoms, L = 1.24 nm
    p = synth.diff_params(b, seed=9, ntype=2)
    lj = synth.combine_geometric(p["c6"], p["c12"])
    rng = np.random.default_rng(2)
    return b, p["q"], p["type"], lj, rng.normal(size=(b.n_atoms, 3))


def test_vjp_default_options_equal_the_plain_adjoint(small):
    b, q, t, lj, g = small
    rc, beta = 0.6, synth.ewald_beta(0.6)
    a = oracle.force_vjp_coul(b.coords, q, t, lj, b.box, rc, beta, g, b.excl_off, b.excl_idx)
    c = oracle.force_vjp(b.coords, q, t, lj, b.box, rc, beta, g, b.excl_off, b.excl_idx)
    for u, v in zip(a, c):
        assert np.abs(u - v).max() <= 1e-9 * max(np.abs(v).max(), 1e-30)


@pytest.mark.parametrize("opts", [dict(kind="rf", eps_rf=0.0), dict(kind="rf", eps_rf=78.5, excl_corr=True),
                                  dict(kind="ewald", excl_corr=True)])
def test_vjp_matches_finite_differences(small, opts):
    """d(g.F)/dx, d(g.F)/dq, d(g.F)/dC from the adjoint against central differences."""
    b, q, t, lj, g = small
    rc = 0.6
    beta = synth.ewald_beta(rc)

    def phi(x=b.coords, qq=q, ljp=lj):
        F, _, _, n = oracle.energy_forces_coul(x, qq, t, ljp, b.box, rc, beta, b.excl_off, b.excl_idx, **opts)
        return float((g * F).sum()), n

    gx, gq, glj = oracle.force_vjp_coul(b.coords, q, t, lj, b.box, rc, beta, g, b.excl_off, b.excl_idx,
                                        kind=opts["kind"], eps_rf=opts.get("eps_rf", 0.0),
                                        excl_corr=opts.get("excl_corr", False))
    x = b.coords.astype(np.float64)
    _, n0 = phi(x)
    rng = np.random.default_rng(7)
    h = 1e-6
    checked = 0
    for atom in rng.choice(b.n_atoms, 8, replace=False):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[atom, k] += h
            xm[atom, k] -= h
            (pp, n1), (pm, n2) = phi(xp), phi(xm)
            if n1 != n0 or n2 != n0:
                continue
            assert (pp - pm) / (2 * h) == pytest.approx(gx[atom, k], rel=1e-5, abs=1e-3)
            checked += 1
    assert checked >= 18
    for atom in rng.choice(b.n_atoms, 6, replace=False):
        hq = 1e-6
        qp, qm = q.copy(), q.copy()
        qp[atom] += hq
        qm[atom] -= hq
        fd = (phi(qq=qp)[0] - phi(qq=qm)[0]) / (2 * hq)
        assert fd == pytest.approx(gq[atom], rel=1e-5, abs=1e-3)
    for a in range(2):
        for c in range(2):
            for w in range(2):
                hc = 1e-6 * max(abs(lj[a, c, w]), 1e-8)
                lp, lm = lj.copy(), lj.copy()
                lp[a, c, w] += hc
                lm[a, c, w] -= hc
                if a != c:  # keep the matrix symmetric: perturb both entries, half each
                    lp[c, a, w] += hc
                    lm[c, a, w] -= hc
                fd = (phi(ljp=lp)[0] - phi(ljp=lm)[0]) / (2 * hc)
                want = glj[a, c, w] + (glj[c, a, w] if a != c else 0.0)
                assert fd == pytest.approx(want, rel=1e-5, abs=1e-6 * abs(fd) + 1e-8)
