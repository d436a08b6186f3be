"""Parity of the hand-written adjoint (nb_backward) with the oracle's.

The oracle's adjoint is itself pinned by finite differences (see
test_oracle_adjoint.py); here the GPU gradients are compared with it on the
same inputs, checked directly against FP64 finite differences of the oracle
on the 1,536-atom box, and run end to end through torch.autograd for a
force-matching loss.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import to_dev

pytestmark = pytest.mark.gpu

GX_TOL = 1e-3   # per-atom |d grad_x| <= GX_TOL * rms(grad_x)
GQ_TOL = 1e-4   # per-atom |d grad_q| <= GQ_TOL * rms(grad_q)
GLJ_TOL = 1e-4  # relative, per LJ matrix entry


@pytest.fixture(scope="module")
def nb():
    from paper_2405_01420_gb300 import nb as nbmod
    nbmod.load_library()
    return nbmod


def per_atom_err(a, b):
    a = np.asarray(a, np.float64).reshape(len(b), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    rms = np.sqrt((b ** 2).sum(1).mean())
    return float(np.sqrt(((a - b) ** 2).sum(1)).max() / rms)


@pytest.fixture(scope="module")
def diffbox():
    """24,000 atoms: charges N(0, 0.4) neutralised, 4 LJ types, geometric rule."""
    b = synth.water_box(8000, 4)
    p = synth.diff_params(b, seed=4)
    lj = synth.combine_geometric(p["c6"], p["c12"]).astype(np.float32)
    return b, p, lj


@pytest.mark.parametrize("cluster_tiles", [False, True])
def test_backward_matches_oracle_adjoint(nb, diffbox, cluster_tiles):
    """After a prune: the gathered-tile adjoint (default) and the 8 x 8 cluster-tile one."""
    b, p, lj = diffbox
    rc = 1.0
    beta = synth.ewald_beta(rc)
    q = p["q"].astype(np.float32)
    d = to_dev(b)
    rng = np.random.default_rng(3)
    g = rng.normal(size=(b.n_atoms, 3)).astype(np.float32)
    pl = nb.Pairlist(b.n_atoms, cluster_tiles=cluster_tiles)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    gx, gq, glj = pl.backward(d["coords"], torch.from_numpy(q).cuda(), torch.from_numpy(p["type"]).cuda(),
                              torch.from_numpy(lj).cuda(), rc, beta, torch.from_numpy(g).cuda())
    assert pl.status() == 0
    ox, oq, olj = oracle.force_vjp(b.coords, q, p["type"], lj, b.box, rc, beta, g, b.excl_off, b.excl_idx)
    assert per_atom_err(gx.cpu().numpy(), ox) <= GX_TOL
    assert per_atom_err(gq.cpu().numpy(), oq) <= GQ_TOL
    np.testing.assert_allclose(glj.cpu().numpy(), olj, rtol=GLJ_TOL)
    # translation invariance of g.F
    s = gx.double().sum(0).abs().max().item()
    assert s <= 1e-5 * gx.abs().max().item() * np.sqrt(b.n_atoms)
    pl.close()


@pytest.mark.parametrize("ntype", [1, 2])
def test_backward_water_types(nb, ntype):
    """Water with 2 types (LJ on O only) and with 1 type (every atom O-like):
    the gathered-tile adjoint's one- and two-type forms against the oracle."""
    b = synth.water_box(3000, 21)
    rc = 1.0
    beta = synth.ewald_beta(rc)
    if ntype == 2:
        typ, lj = b.type, b.ljparams
    else:
        typ = np.zeros(b.n_atoms, np.int32)
        lj = b.ljparams.reshape(-1, 2)[:1].reshape(1, 1, 2).astype(np.float32)
    d = to_dev(b)
    rng = np.random.default_rng(ntype)
    g = rng.normal(size=(b.n_atoms, 3)).astype(np.float32)
    pl = nb.Pairlist(b.n_atoms)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    gx, gq, glj = pl.backward(d["coords"], d["q"], torch.from_numpy(typ).cuda(), torch.from_numpy(lj).cuda(), rc,
                              beta, torch.from_numpy(g).cuda())
    assert pl.status() == 0
    ox, oq, olj = oracle.force_vjp(b.coords, b.q, typ, lj, b.box, rc, beta, g, b.excl_off, b.excl_idx)
    assert per_atom_err(gx.cpu().numpy(), ox) <= GX_TOL
    assert per_atom_err(gq.cpu().numpy(), oq) <= GQ_TOL
    nz = np.abs(olj) > 0
    np.testing.assert_allclose(glj.cpu().numpy()[nz], olj[nz], rtol=GLJ_TOL)
    pl.close()


def test_backward_water_against_finite_differences(nb):
    """1,536-atom box: GPU dL/dx and dL/dq against FP64 central differences of g.F."""
    b = synth.water_box(512, 1)
    rc = 0.9
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    rng = np.random.default_rng(8)
    g = rng.normal(size=(b.n_atoms, 3))
    pl = nb.Pairlist(b.n_atoms)
    pl.search(d["coords"], b.box, rc, d["excl_off"], d["excl_idx"])
    gx, gq, glj = pl.backward(d["coords"], d["q"], d["type"], d["lj"], rc, beta,
                              torch.from_numpy(g.astype(np.float32)).cuda())
    assert pl.status() == 0
    gx = gx.cpu().numpy().astype(np.float64)
    gq = gq.cpu().numpy().astype(np.float64)
    x = b.coords.astype(np.float64)
    q = b.q.astype(np.float64)
    g32 = g.astype(np.float32).astype(np.float64)

    def phi(xx, qq):
        F, _, _, n = oracle.energy_forces(xx, qq, b.type, b.ljparams, b.box, rc, beta, b.excl_off, b.excl_idx, "n2")
        return float((g32 * F).sum()), n

    _, n0 = phi(x, q)
    scale_x = np.sqrt((gx ** 2).sum(1).mean())
    checked = 0
    for atom in rng.choice(b.n_atoms, 8, replace=False):
        for k in range(3):
            h = 1e-5
            xp, xm = x.copy(), x.copy()
            xp[atom, k] += h
            xm[atom, k] -= h
            fp, n1 = phi(xp, q)
            fm, n2 = phi(xm, q)
            if n1 != n0 or n2 != n0:
                continue
            assert abs((fp - fm) / (2 * h) - gx[atom, k]) <= 1e-3 * scale_x, (atom, k)
            checked += 1
        h = 1e-3
        qp, qm = q.copy(), q.copy()
        qp[atom] += h
        qm[atom] -= h
        fd = (phi(x, qp)[0] - phi(x, qm)[0]) / (2 * h)
        assert abs(fd - gq[atom]) <= 1e-4 * np.sqrt((gq ** 2).mean()), atom
    assert checked >= 18
    pl.close()


def test_hessian_symmetry_on_gpu(nb, diffbox):
    """v . J(w) = w . J(v) for J = dF/dx (symmetric), within FP32 accuracy."""
    b, p, lj = diffbox
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    qd = torch.from_numpy(p["q"].astype(np.float32)).cuda()
    td = torch.from_numpy(p["type"]).cuda()
    ljd = torch.from_numpy(lj).cuda()
    pl = nb.Pairlist(b.n_atoms)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    gen = torch.Generator(device="cuda").manual_seed(5)
    v = torch.randn((b.n_atoms, 3), device="cuda", generator=gen)
    w = torch.randn((b.n_atoms, 3), device="cuda", generator=gen)
    jv, _, _ = pl.backward(d["coords"], qd, td, ljd, rc, beta, v)
    jw, _, _ = pl.backward(d["coords"], qd, td, ljd, rc, beta, w)
    a = float((v.double() * jw.double()).sum())
    c = float((w.double() * jv.double()).sum())
    assert abs(a - c) <= 1e-5 * max(abs(a), abs(c))
    pl.close()


def test_autograd_force_matching(nb, diffbox):
    """loss.backward() through NonbondedForces equals the oracle's force-matching gradients."""
    from paper_2405_01420_gb300.autograd import force_matching_loss, lj_matrix, nonbonded_forces
    b, p, _ = diffbox
    rc = 1.0
    beta = synth.ewald_beta(rc)
    d = to_dev(b)
    # targets: forces with parameters perturbed by 5% (from the oracle, FP64)
    lj_t = synth.combine_geometric(p["c6_target"], p["c12_target"])
    T, _, _, _ = oracle.energy_forces(b.coords, p["q_target"], p["type"], lj_t, b.box, rc, beta, b.excl_off,
                                      b.excl_idx)
    x = d["coords"].clone().requires_grad_(True)
    q = torch.from_numpy(p["q"].astype(np.float32)).cuda().requires_grad_(True)
    c6 = torch.from_numpy(p["c6"]).cuda().requires_grad_(True)
    c12 = torch.from_numpy(p["c12"]).cuda().requires_grad_(True)
    td = torch.from_numpy(p["type"]).cuda()
    pl = nb.Pairlist(b.n_atoms)
    pl.search(d["coords"], b.box, 1.1, d["excl_off"], d["excl_idx"])
    pl.prune(d["coords"], 1.04)
    F, _ = nonbonded_forces(x, q, lj_matrix(c6, c12), pl, td, rc, beta)
    loss = force_matching_loss(F, torch.from_numpy(T).cuda())
    loss.backward()
    assert pl.status() == 0
    lj = synth.combine_geometric(p["c6"], p["c12"]).astype(np.float32)
    L, _, _, _, _ = oracle.force_matching(b.coords, p["q"].astype(np.float32), p["type"], lj, b.box, rc, beta, T,
                                          b.excl_off, b.excl_idx)
    # F - T is ~5% of F, so the 1e-5 rms force error is amplified ~20x in L
    assert loss.item() == pytest.approx(L, rel=1e-3)
    # the adjoint itself: the oracle's VJP at the same dL/dF the GPU used
    g = 2.0 * (F.detach().double().cpu().numpy() - T) / (3 * b.n_atoms)
    ox, oq, olj = oracle.force_vjp(b.coords, p["q"].astype(np.float32), p["type"], lj, b.box, rc, beta, g,
                                   b.excl_off, b.excl_idx)
    assert per_atom_err(x.grad.cpu().numpy(), ox) <= GX_TOL
    assert per_atom_err(q.grad.cpu().numpy(), oq) <= GQ_TOL
    # chain rule through C_ab = sqrt(c_a c_b), written out in numpy for the oracle
    for comp, (par, grad) in enumerate([(p["c6"], c6.grad), (p["c12"], c12.grad)]):
        nt = len(par)
        want = np.zeros(nt)
        for a in range(nt):
            for c in range(nt):
                dCa = 1.0 if a == c else 0.5 * np.sqrt(par[c] / par[a])
                want[a] += olj[a, c, comp] * dCa + (olj[c, a, comp] * dCa if a != c else 0.0)
        np.testing.assert_allclose(grad.cpu().numpy(), want, rtol=GLJ_TOL)
    pl.close()
