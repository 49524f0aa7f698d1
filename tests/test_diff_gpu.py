"""GPU differentiation path against the differentiation oracle and finite differences.

* gipc_potential_derivs (energy, exact gradient, exact Hessian-vector product by hyper-dual
  kernels) against oracle.diff.potential (second-order jets) at a contact configuration;
* the autograd binding: backward is the gradient kernel, double backward the Hessian-vector kernel;
* gipc_potential_hessian (assembled exact Hessian) against the oracle's sparse Hessian;
* gipc_adjoint_step against oracle.diff.adjoint_step at the same converged step;
* the adjoint through two GPU steps against central differences of the GPU forward (dL/dv0 along
  a direction and E dL/dE).
Float routes on both sides: agreement to ~1e-9 relative where the contact geometry is well
conditioned (the scene keeps its edges >= 1e-4 rad from parallel)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import contact as C  # noqa: E402
from oracle import diff as D  # noqa: E402
from oracle import newton as N  # noqa: E402
from oracle import tet as TT  # noqa: E402

MU, LAM = TT.snh_params(1e5, 0.4)


@pytest.fixture(scope="module")
def gipc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_09400_gb300 as g
    return g


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _scene(m=3, v=-0.05):
    sc0 = synth.two_cubes(gap=0.0, velocity=v, m=m)
    x = sc0["x"].copy()
    n0 = m ** 3
    rng = np.random.default_rng(3)
    x[:, n0:] += np.array([0.031, 0.017, 0.0])[:, None]
    x += 1e-4 * rng.normal(size=x.shape)
    dh = 1e-3 * sc0["l"]
    x[2, n0:] += 0.5 * dh
    prm = dict(dhat=dh, kappa=1e3, dt=0.01, mu=MU, lam=LAM, gravity=(0.0, 0.0, -9.81), eps_d=1e-9,
               pcg_tol=1e-14, max_pcg=2000, max_newton=60, max_ls=40)
    sc = N.build_scene(dict(sc0, x=x), prm, 1000.0)
    return sc0, sc, x, prm


def _gpu_scene(g, sc0, x, sc):
    srf = g.Surface(_dev(sc0["tris"]), _dev(sc0["edges"]), _dev(sc0["verts"]))
    return g.Scene(_dev(x), _dev(sc0["tets"]), srf, 1000.0, fixed=_dev(sc0["fixed"]), l=sc["l"])


def _gkw(prm):
    return dict(dt=prm["dt"], mu=prm["mu"], lam=prm["lam"], dhat=prm["dhat"], kappa=prm["kappa"],
                eps_d=prm["eps_d"], pcg_tol=prm["pcg_tol"], max_pcg=prm["max_pcg"], max_newton=prm["max_newton"],
                max_ls=prm["max_ls"])


def _state(g):
    sc0, sc, x, prm = _scene()
    scene = _gpu_scene(g, sc0, x, sc)
    rng = np.random.default_rng(9)
    xq = x + 2e-4 * rng.normal(size=x.shape)      # a configuration inside the contact zone
    xq[:, np.asarray(sc["fixed"], bool)] = x[:, np.asarray(sc["fixed"], bool)]
    st, eps = g.find_contacts(_dev(xq), scene.rest_x, scene.surface, prm["dhat"])
    return sc0, sc, x, prm, scene, xq, st, eps, rng


def test_derivatives_match_the_oracle(gipc):
    sc0, sc, x, prm, scene, xq, st, eps, rng = _state(gipc)
    assert st.shape[1] > 0
    xt = xq + 1e-4 * rng.normal(size=xq.shape)
    u = rng.normal(size=xq.shape)
    dt2 = prm["dt"] ** 2
    out = gipc.potential_derivs(scene, _dev(xq), st, eps, prm["dhat"], prm["kappa"], MU, LAM, dt2, xt=_dev(xt),
                                u=_dev(u), want=("energy", "grad"))
    E, g, H = D.potential(xq, xt, sc["mass"], sc["tets"], sc["Dm_inv"], sc["vol"], MU, LAM, dt2,
                          st.cpu().numpy(), eps.cpu().numpy(), prm["dhat"], prm["kappa"])
    assert out["energy"] == pytest.approx(E, rel=1e-10)
    gg = out["grad"].cpu().numpy()
    assert np.abs(gg - g).max() <= 1e-9 * np.abs(g).max()
    Hu = (H @ u.T.reshape(-1)).reshape(-1, 3).T
    assert np.abs(out["Hu"].cpu().numpy() - Hu).max() <= 1e-9 * np.abs(Hu).max()


def test_autograd_backward_and_double_backward(gipc):
    sc0, sc, x, prm, scene, xq, st, eps, rng = _state(gipc)
    dt2 = prm["dt"] ** 2
    xt = _dev(xq + 1e-4 * rng.normal(size=xq.shape))
    X = _dev(xq).requires_grad_(True)
    I = gipc.incremental_potential(X, scene, xt, st, eps, prm["dhat"], prm["kappa"], MU, LAM, dt2)
    (gX,) = torch.autograd.grad(I, X, create_graph=True)
    ref = gipc.potential_derivs(scene, _dev(xq), st, eps, prm["dhat"], prm["kappa"], MU, LAM, dt2, xt=xt,
                                want=("grad",))["grad"]
    assert torch.equal(gX.detach(), ref)
    u = _dev(rng.normal(size=xq.shape))
    (Hu,) = torch.autograd.grad((gX * u).sum(), X)
    ref_hu = gipc.potential_derivs(scene, _dev(xq), st, eps, prm["dhat"], prm["kappa"], MU, LAM, dt2, xt=xt, u=u,
                                   want=())["Hu"]
    assert torch.equal(Hu, ref_hu)


def test_exact_hessian_matches_the_oracle(gipc):
    sc0, sc, x, prm, scene, xq, st, eps, rng = _state(gipc)
    dt2 = prm["dt"] ** 2
    Hb = gipc.potential_hessian(scene, _dev(xq), st, eps, prm["dhat"], prm["kappa"], MU, LAM, dt2)
    n = xq.shape[1]
    Hd = np.zeros((3 * n, 3 * n))
    rp, ci, vals = Hb["rowptr"].cpu().numpy(), Hb["colidx"].cpu().numpy(), Hb["vals"].cpu().numpy()
    for r in range(n):
        for p in range(rp[r], rp[r + 1]):
            c = ci[p]
            Hd[3 * r:3 * r + 3, 3 * c:3 * c + 3] = vals[p]
    _, _, H = D.potential(xq, None, sc["mass"], sc["tets"], sc["Dm_inv"], sc["vol"], MU, LAM, dt2,
                          st.cpu().numpy(), eps.cpu().numpy(), prm["dhat"], prm["kappa"])
    Ho = H.toarray()
    assert np.abs(Hd - Ho).max() <= 1e-9 * np.abs(Ho).max()
    assert np.abs(Hd - Hd.T).max() <= 1e-12 * np.abs(Hd).max()


def test_adjoint_step_matches_the_oracle(gipc):
    sc0, sc, x, prm = _scene()
    scene = _gpu_scene(gipc, sc0, x, sc)
    x1, v1 = _dev(x), _dev(sc0["v"])
    stt = gipc.newton_step(scene, x1, v1, **_gkw(prm))
    assert stt["converged"] == 1 and stt["contacts"] > 0
    rng = np.random.default_rng(4)
    w = rng.normal(size=x.shape)
    wv = rng.normal(size=x.shape)
    ax, av, logE, its = gipc.adjoint_step(scene, x1, _dev(x), _dev(sc0["v"]), _dev(w), _dev(wv), prm["dt"], MU, LAM,
                                          prm["dhat"], prm["kappa"], pcg_tol=1e-26, max_pcg=20000)
    oax, oav, ologE = D.adjoint_step(x1.cpu().numpy(), sc, prm, w, wv)
    assert np.abs(av.cpu().numpy() - oav).max() <= 1e-7 * np.abs(oav).max()
    assert np.abs(ax.cpu().numpy() - oax).max() <= 1e-7 * np.abs(oax).max()
    assert logE == pytest.approx(ologE, rel=1e-7)


def test_polish_reaches_the_minimiser(gipc):
    """A loosely converged projected-Newton step refined by exact Newton: a few iterations, the
    gradient of I vanishes to rounding, and the result agrees with a tightly converged step."""
    sc0, sc, x, prm = _scene()
    scene = _gpu_scene(gipc, sc0, x, sc)
    x0, v0 = _dev(x), _dev(sc0["v"])
    xa, va = x0.clone(), v0.clone()
    gipc.newton_step(scene, xa, va, **dict(_gkw(prm), eps_d=1e-4))
    its, step = gipc.newton_polish(scene, xa, va, x0, v0, prm["dt"], MU, LAM, prm["dhat"], prm["kappa"],
                                   eps_polish=1e-13)
    assert 1 <= its <= 6 and step <= 1e-13
    xb, vb = x0.clone(), v0.clone()
    gipc.newton_step(scene, xb, vb, **_gkw(prm))                     # eps_d 1e-9
    span = np.abs(xb.cpu().numpy() - x).max()
    assert np.abs(xa.cpu().numpy() - xb.cpu().numpy()).max() <= 1e-7 * span
    assert np.array_equal(va.cpu().numpy(), (xa.cpu().numpy() - x0.cpu().numpy()) / prm["dt"])
    st, eps = gipc.find_contacts(xa, scene.rest_x, scene.surface, prm["dhat"])
    xt = x0 + prm["dt"] * v0
    xt[2] += prm["dt"] ** 2 * -9.81
    fixed = torch.tensor(sc["fixed"], device="cuda").bool()
    xt[:, fixed] = x0[:, fixed]
    g = gipc.potential_derivs(scene, xa, st, eps, prm["dhat"], prm["kappa"], MU, LAM, prm["dt"] ** 2, xt=xt,
                              want=("grad",))["grad"]
    inertia = (scene.mass * (xa - xt)).abs().max().item()
    assert g[:, ~fixed].abs().max().item() <= 1e-9 * inertia


def test_adjoint_through_two_steps_matches_finite_differences(gipc):
    """Steps refined to eps 1e-13 by newton_polish; central differences with h = 1e-6 in v0 and
    1e-4 in log E."""
    sc0, sc, x, prm = _scene()
    scene = _gpu_scene(gipc, sc0, x, sc)
    kw = dict(_gkw(prm), eps_d=1e-6)
    pol = dict(eps_polish=1e-13)
    rng = np.random.default_rng(6)
    w = _dev(rng.normal(size=x.shape))
    xT, vT, cps = gipc.simulate(scene, _dev(x), _dev(sc0["v"]), 2, polish=pol, **kw)
    ax0, av0, logE, its = gipc.adjoint(scene, cps, w, torch.zeros_like(w), prm["dt"], MU, LAM, prm["dhat"],
                                       prm["kappa"], pcg_tol=1e-26, max_pcg=20000)
    dirv = rng.normal(size=x.shape)
    dirv[:, np.asarray(sc["fixed"], bool)] = 0.0
    dv = _dev(dirv)
    h = 1e-6

    def L(v0, mu=MU, lam=LAM):
        k2 = dict(kw, mu=mu, lam=lam)
        xx, _, _ = gipc.simulate(scene, _dev(x), v0, 2, polish=pol, **k2)
        return float((w * xx).sum())

    v0 = _dev(sc0["v"])
    fd = (L(v0 + h * dv) - L(v0 - h * dv)) / (2 * h)
    assert float((av0 * dv).sum()) == pytest.approx(fd, rel=1e-6)
    r = 1e-4
    mp, lp = TT.snh_params(1e5 * (1 + r), 0.4)
    mm, lm = TT.snh_params(1e5 * (1 - r), 0.4)
    fdE = (L(v0, mp, lp) - L(v0, mm, lm)) / (np.log(1 + r) - np.log(1 - r))
    assert logE == pytest.approx(fdE, rel=1e-5)
