"""Pins for the differentiation oracle: element jets against independent derivative routes,
the assembled potential against finite differences, and the implicit adjoint of a step against
finite differences of the oracle's own Newton step."""
import numpy as np
import pytest

import synth
from oracle import diff as D
from oracle import geometry as G
from oracle import newton as N
from oracle import stencil as S
from oracle import tet as TT

MU, LAM = TT.snh_params(1e5, 0.4)


def _well_conditioned(d, lo=0.05, hi=0.9, min_sin2=1e-10):
    """Indices of stencils whose g lies in [lo, hi] and, for the edge-edge-derived types, whose
    edges are at least ~1e-5 rad from parallel: float64 derivatives through the line-line normal
    equations lose about 1 / sin(angle) to cancellation, so the float routes (these jets, the GPU's
    hyper-duals) are only checked where that loss stays below 1e-6."""
    keep = []
    for i in range(d["stencils"].shape[1]):
        typ, verts = G.decode(d["stencils"][:, i])
        P = [d["x"][:, v] for v in verts]
        geo = G.exact_geometry(typ, P, d["dhat"])
        if not lo <= float(geo["g"]) <= hi:
            continue
        if typ in (G.EE, G.EE_PAR) or G.PARALLEL[typ]:
            a, b = P[1] - P[0], P[3] - P[2]
            s2 = float(np.sum(np.cross(a, b) ** 2)) / (float(a @ a) * float(b @ b))
            if s2 < min_sin2:
                continue
        keep.append(i)
    return keep


def test_stencil_jet_matches_the_exact_rational_gradient():
    """Jets over float coordinates vs the oracle's stencil path (exact rational geometry): the same
    energy and gradient by an independent route, on every type."""
    d = synth.unit_stencils(k=160, seed=21)
    eps = S.compute_eps_x(d["x"], d["stencils"])
    seen = set()
    for i in _well_conditioned(d):
        typ, verts = G.decode(d["stencils"][:, i])
        P = [d["x"][:, v] for v in verts]
        J = D.stencil_energy_jet(typ, P, float(eps[i]), d["dhat"], 1e3)
        ref = S.eval_stencil(typ, P, float(eps[i]), d["dhat"], 1e3)
        assert J.v == pytest.approx(ref["energy"], rel=1e-7)
        g = np.array(J.g)
        assert np.abs(g - ref["grad"][:len(g)]).max() <= 1e-6 * np.abs(ref["grad"]).max()
        seen.add(typ)
    assert len(seen) >= 5


def test_stencil_jet_hessian_is_the_derivative_of_its_gradient():
    d = synth.unit_stencils(k=120, seed=22)
    eps = S.compute_eps_x(d["x"], d["stencils"])
    for i in _well_conditioned(d)[:25]:
        typ, verts = G.decode(d["stencils"][:, i])
        P = [d["x"][:, v].copy() for v in verts]
        J = D.stencil_energy_jet(typ, P, float(eps[i]), d["dhat"], 1e3)
        H = np.array(J.h)
        assert np.allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())
        h = 1e-3 * d["dhat"]
        for k in range(len(J.g)):
            Pp = [p.copy() for p in P]
            Pm = [p.copy() for p in P]
            Pp[k // 3][k % 3] += h
            Pm[k // 3][k % 3] -= h
            fd = (np.array(D.stencil_energy_jet(typ, Pp, float(eps[i]), d["dhat"], 1e3).g) -
                  np.array(D.stencil_energy_jet(typ, Pm, float(eps[i]), d["dhat"], 1e3).g)) / (2 * h)
            assert np.abs(fd - H[k]).max() <= 2e-3 * np.abs(H).max()


def test_tet_jet_hessian_is_the_unprojected_chain_rule():
    """d2E/dx2 from jets over x equals scale vol dF/dx^T (d2 Psi / dF2) dF/dx from jets over F."""
    rng = np.random.default_rng(5)
    rest = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.1
    inv, vol = TT.rest_shape(rest)
    Dx = TT.dF_dx(inv)
    for _ in range(5):
        pts = rest + rng.normal(scale=0.03, size=(4, 3))
        J = D.tet_energy_jet(pts, inv.reshape(-1), vol, MU, LAM, 1e-4)
        Ds = (pts[1:] - pts[0]).T
        F = Ds @ inv
        _, gF, HF = TT.psi_derivs(F, MU, LAM)
        ref_g = 1e-4 * vol * Dx.T @ gF
        ref_H = 1e-4 * vol * Dx.T @ HF @ Dx
        assert np.abs(np.array(J.g) - ref_g).max() <= 1e-9 * np.abs(ref_g).max()
        assert np.abs(np.array(J.h) - ref_H).max() <= 1e-9 * np.abs(ref_H).max()


def _scene(m=3, gap_frac=0.5, v=-0.05):
    sc0 = synth.two_cubes(gap=0.0, velocity=v, m=m)
    x = sc0["x"].copy()
    n0 = m ** 3
    rng = np.random.default_rng(3)
    x[:, n0:] += np.array([0.031, 0.017, 0.0])[:, None]
    x += 1e-4 * rng.normal(size=x.shape)
    dh = 1e-3 * sc0["l"]
    x[2, n0:] += gap_frac * dh
    prm = dict(dhat=dh, kappa=1e3, dt=0.01, mu=MU, lam=LAM, gravity=(0.0, 0.0, -9.81), eps_d=1e-9,
               pcg_tol=1e-14, max_pcg=2000, max_newton=60, max_ls=40)
    sc = N.build_scene(dict(sc0, x=x), prm, 1000.0)
    return sc0, sc, x, prm


def test_potential_gradient_and_hessian_against_finite_differences():
    from oracle import contact as C
    sc0, sc, x, prm = _scene()
    st, eps = C.find_contacts(x, sc["rest_x"], sc["tris"], sc["edges"], sc["verts"], prm["dhat"])
    assert st.shape[1] > 0
    rng = np.random.default_rng(2)
    xt = x + 1e-4 * rng.normal(size=x.shape)
    args = (sc["mass"], sc["tets"], sc["Dm_inv"], sc["vol"], MU, LAM, prm["dt"] ** 2, st, eps, prm["dhat"], 1e3)
    E, g, H = D.potential(x, xt, *args)
    u = rng.normal(size=x.shape)
    h = 1e-7
    Ep = D.potential(x + h * u, xt, *args, hessian=False)[0]
    Em = D.potential(x - h * u, xt, *args, hessian=False)[0]
    assert (Ep - Em) / (2 * h) == pytest.approx(float(np.sum(g * u)), rel=1e-5)
    gp = D.potential(x + h * u, xt, *args, hessian=False)[1]
    gm = D.potential(x - h * u, xt, *args, hessian=False)[1]
    Hu = (H @ u.T.reshape(-1)).reshape(-1, 3).T
    assert np.abs((gp - gm) / (2 * h) - Hu).max() <= 1e-4 * np.abs(Hu).max()
    assert abs(H - H.T).max() <= 1e-10 * abs(H).max()


@pytest.mark.slow
def test_adjoint_step_matches_finite_differences_of_the_newton_step():
    """L = w . x_1 after one tightly converged step: the adjoint's dL/dv0 (along a direction) and
    E dL/dE against central differences of the oracle's Newton step."""
    sc0, sc, x0, prm = _scene()
    v0 = sc0["v"].copy()
    rng = np.random.default_rng(7)
    w = rng.normal(size=x0.shape)
    x1, v1, st = N.newton_step(sc, x0, v0, prm)
    assert st["contacts"][-1] > 0
    ax, av, logE = D.adjoint_step(x1, sc, prm, w, np.zeros_like(w))
    dirv = rng.normal(size=v0.shape)
    dirv[:, np.asarray(sc["fixed"], bool)] = 0.0
    h = 1e-5
    Lp = np.sum(w * N.newton_step(sc, x0, v0 + h * dirv, prm)[0])
    Lm = np.sum(w * N.newton_step(sc, x0, v0 - h * dirv, prm)[0])
    fd = (Lp - Lm) / (2 * h)
    assert float(np.sum(av * dirv)) == pytest.approx(fd, rel=1e-4)
    # Young's modulus: E dL/dE = dL/d(log E)
    r = 1e-3
    outs = []
    for s_ in (1 + r, 1 - r):
        mu, lam = TT.snh_params(1e5 * s_, 0.4)
        prm2 = dict(prm, mu=mu, lam=lam)
        outs.append(np.sum(w * N.newton_step(sc, x0, v0, prm2)[0]))
    fdE = (outs[0] - outs[1]) / (np.log(1 + r) - np.log(1 - r))
    assert logE == pytest.approx(fdE, rel=1e-3)
