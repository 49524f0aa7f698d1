"""GPU parity of gipc_find_contacts, gipc_ccd_max_step and gipc_newton_step against the oracle.

Contact lists (stencil tuples and eps_x) are compared bit for bit: both sides take every decision
(box test, distance below dhat, closest feature, parallel test) with the same float64 operations.
The CCD step is compared exactly as well (same per-pair arithmetic, order-independent minimum).
The Newton step is compared on its iteration path (iterations, contacts) and its positions, which
differ only by the rounding of the PCG's reductions.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import contact as C  # noqa: E402
from oracle import geometry as G  # noqa: E402
from oracle import newton as N  # noqa: E402
from oracle import tet as TT  # noqa: E402


@pytest.fixture(scope="module")
def gipc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_09400_gb300 as g
    return g


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _rotz(x, idx, th, c):
    X = x[:, idx] - np.asarray(c, float)[:, None]
    R = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    x[:, idx] = R @ X + np.asarray(c, float)[:, None]


def _variant(kind):
    """Two unit cubes with the top one placed 0.5 dhat above the bottom one."""
    sc = synth.two_cubes(gap=0.0)
    x = sc["x"].copy()
    dh = 1e-3 * sc["l"]
    top = np.arange(125, 250)
    if kind == "generic":            # shifted and jittered: interior point-triangle / edge-edge
        rng = np.random.default_rng(3)
        x[:, 125:] += np.array([0.031, 0.017, 0.0])[:, None]
        x += 1e-4 * rng.normal(size=x.shape)
    elif kind == "shifted":          # half a cell over and turned by 2e-3 rad: nearly parallel edges
        x[0, 125:] += 0.125
        _rotz(x, top, 2e-3, (0.625, 0.5, 0.0))
    elif kind == "rot45":            # turned by 45 degrees: crossing edges, corners over faces
        _rotz(x, top, np.pi / 4, (0.5, 0.5, 0.0))
    x[2, 125:] += 0.5 * dh           # "aligned": only this offset
    return sc, x, dh


def _surface(g, sc):
    return g.Surface(_dev(sc["tris"]), _dev(sc["edges"]), _dev(sc["verts"]))


KINDS = ("generic", "aligned", "shifted", "rot45")


def test_variants_cover_every_stencil_type():
    seen = set()
    for kind in KINDS:
        sc, x, dh = _variant(kind)
        st, _ = C.find_contacts(x, sc["x"], sc["tris"], sc["edges"], sc["verts"], dh)
        seen |= {G.decode(st[:, i])[0] for i in range(st.shape[1])}
    assert seen == set(range(7))


@pytest.mark.parametrize("kind", KINDS)
def test_find_contacts_bit_exact(gipc, kind):
    sc, x, dh = _variant(kind)
    ref_st, ref_eps = C.find_contacts(x, sc["x"], sc["tris"], sc["edges"], sc["verts"], dh)
    st, eps = gipc.find_contacts(_dev(x), _dev(sc["x"]), _surface(gipc, sc), dh)
    assert st.shape == ref_st.shape
    assert np.array_equal(st.cpu().numpy(), ref_st)
    assert np.array_equal(eps.cpu().numpy(), ref_eps)


def test_find_contacts_ball_grid_and_capacity(gipc):
    """Thousands of surface primitives (several tiles, ragged tails) and the capacity protocol."""
    sc = synth.sphere_grid(2, 2, radius=0.05, cells=8, gap=1e-3, floor_cells=6)
    x = sc["x"].copy()
    rng = np.random.default_rng(11)
    x += 2e-4 * rng.normal(size=x.shape)
    dh = 2e-3
    ref_st, ref_eps = C.find_contacts(x, sc["x"], sc["tris"], sc["edges"], sc["verts"], dh)
    assert ref_st.shape[1] > 100
    srf = _surface(gipc, sc)
    st, eps = gipc.find_contacts(_dev(x), _dev(sc["x"]), srf, dh, capacity=None)
    assert np.array_equal(st.cpu().numpy(), ref_st)
    assert np.array_equal(eps.cpu().numpy(), ref_eps)
    with pytest.raises(gipc.GipcError, match="CAPACITY"):
        gipc.find_contacts(_dev(x), _dev(sc["x"]), srf, dh, capacity=ref_st.shape[1] - 1)
    st2, _ = gipc.find_contacts(_dev(x), _dev(sc["x"]), srf, dh, capacity=ref_st.shape[1])
    assert np.array_equal(st2.cpu().numpy(), ref_st)


def test_find_contacts_empty_inputs(gipc):
    sc, x, dh = _variant("aligned")
    empty3 = torch.zeros((3, 0), dtype=torch.int32, device="cuda")
    empty2 = torch.zeros((2, 0), dtype=torch.int32, device="cuda")
    empty1 = torch.zeros(0, dtype=torch.int32, device="cuda")
    st, eps = gipc.find_contacts(_dev(x), _dev(sc["x"]), gipc.Surface(empty3, empty2, empty1), dh)
    assert st.shape == (4, 0) and eps.shape == (0,)
    # far apart: no contacts
    x[2, 125:] += 1.0
    st, _ = gipc.find_contacts(_dev(x), _dev(sc["x"]), _surface(gipc, sc), dh)
    assert st.shape[1] == 0


@pytest.mark.parametrize("kind", KINDS)
def test_ccd_step_exact(gipc, kind):
    sc, x, dh = _variant(kind)
    rng = np.random.default_rng(5)
    d = np.zeros_like(x)
    d[2, 125:] = -4 * dh                         # would pass through the bottom cube's top face
    d[:, 125:] += 0.5 * dh * rng.normal(size=(3, 125))
    ref = C.max_step(x, d, sc["tris"], sc["edges"], sc["verts"])
    got = gipc.ccd_max_step(_dev(x), _dev(d), _surface(gipc, sc))
    assert 0.0 < ref < 1.0
    assert got == ref
    # moving apart: the full step is feasible
    d2 = np.zeros_like(x)
    d2[2, 125:] = 3 * dh
    assert gipc.ccd_max_step(_dev(x), _dev(d2), _surface(gipc, sc)) == 1.0 == \
        C.max_step(x, d2, sc["tris"], sc["edges"], sc["verts"])


def _newton_case():
    sc0, x0, dh = _variant("generic")
    mu, lam = TT.snh_params(1e5, 0.4)
    prm = dict(dhat=dh, kappa=1e3, dt=0.01, mu=mu, lam=lam, gravity=(0.0, 0.0, -9.81), eps_d=1e-2,
               pcg_tol=1e-4, max_pcg=500, max_newton=8, max_ls=30)
    return sc0, x0, prm


def test_newton_step_matches_oracle(gipc):
    sc0, x0, prm = _newton_case()
    osc = N.build_scene(dict(sc0, x=x0), prm, 1000.0)
    xo, vo, so = N.newton_step(osc, x0, sc0["v"], prm)
    scene = gipc.Scene(_dev(x0), _dev(sc0["tets"]), _surface(gipc, sc0), 1000.0,
                       fixed=_dev(sc0["fixed"]), l=osc["l"])
    x, v = _dev(x0), _dev(sc0["v"])
    st = gipc.newton_step(scene, x, v, dt=prm["dt"], mu=prm["mu"], lam=prm["lam"], dhat=prm["dhat"],
                          kappa=prm["kappa"], gravity=prm["gravity"], eps_d=prm["eps_d"], pcg_tol=prm["pcg_tol"],
                          max_pcg=prm["max_pcg"], max_newton=prm["max_newton"], max_ls=prm["max_ls"])
    xg, vg = x.cpu().numpy(), v.cpu().numpy()
    assert st["newton_iters"] == so["newton"]
    assert st["contacts"] == so["contacts"][-1]
    assert st["last_alpha"] == pytest.approx(so["alpha"][-1], rel=1e-8)
    assert abs(st["pcg_iters"] - sum(so["pcg"])) <= 2
    # measured ~1e-12 of the step (the same iteration counts; only the reductions' summation order
    # differs); the bound keeps a factor 1000 of margin
    scale = np.abs(xo - x0).max()
    err = np.abs(xg - xo).max() / scale
    assert err <= 1e-9, f"position error {err:.3e} of the step"
    assert np.abs(vg - vo).max() <= 1e-9 * np.abs(vo).max()
    assert st["energy"] == pytest.approx(so["energy"], rel=1e-9)
    assert C.count_intersections(xg, sc0["tris"], sc0["edges"]) == 0


def test_literal_two_cube_step_has_no_contact_and_matches_oracle(gipc):
    """The two-cube scene as configured: the top cube 0.5 above the bottom one (gap 0.5, far beyond
    dhat = 1e-3 l) falling at 2 m/s.  One step of dt = 0.01 moves it 0.02, so no contact arises and
    the step is elasticity, inertia and gravity alone; it must match the oracle's step."""
    sc0 = synth.two_cubes()
    x0 = sc0["x"].copy()
    assert x0[2, 125:].min() - x0[2, :125].max() == pytest.approx(0.5)
    mu, lam = TT.snh_params(1e5, 0.4)
    dh = 1e-3 * sc0["l"]
    prm = dict(dhat=dh, kappa=1e3, dt=0.01, mu=mu, lam=lam, gravity=(0.0, 0.0, -9.81), eps_d=1e-2,
               pcg_tol=1e-4, max_pcg=500, max_newton=8, max_ls=30)
    osc = N.build_scene(dict(sc0, x=x0), prm, 1000.0)
    xo, vo, so = N.newton_step(osc, x0, sc0["v"], prm)
    assert max(so["contacts"]) == 0
    scene = gipc.Scene(_dev(x0), _dev(sc0["tets"]), _surface(gipc, sc0), 1000.0, fixed=_dev(sc0["fixed"]),
                       l=osc["l"])
    x, v = _dev(x0), _dev(sc0["v"])
    st = gipc.newton_step(scene, x, v, dt=prm["dt"], mu=mu, lam=lam, dhat=dh, kappa=prm["kappa"],
                          gravity=prm["gravity"], eps_d=prm["eps_d"], pcg_tol=prm["pcg_tol"], max_pcg=prm["max_pcg"],
                          max_newton=prm["max_newton"], max_ls=prm["max_ls"])
    assert st["contacts"] == 0 and st["newton_iters"] == so["newton"]
    xg = x.cpu().numpy()
    scale = np.abs(xo - x0).max()
    assert np.abs(xg - xo).max() <= 1e-9 * scale
    assert np.abs(v.cpu().numpy() - vo).max() <= 1e-9 * np.abs(vo).max()


def test_newton_step_mixed_and_rank1_converge_to_the_same_positions(gipc):
    """float32 Hessian storage / SpMV and the rank-1 stencil form change the search directions,
    not the minimiser (the gradient stays float64): run to a tight Newton tolerance, both land
    within 1e-6 l (l the bounding-box diagonal) of each other."""
    sc0, x0, prm = _newton_case()
    scene = gipc.Scene(_dev(x0), _dev(sc0["tets"]), _surface(gipc, sc0), 1000.0, fixed=_dev(sc0["fixed"]))
    out = {}
    for prec, hm in (("fp64", "dense"), ("mixed", "rank1")):
        x, v = _dev(x0), _dev(sc0["v"])
        st = gipc.newton_step(scene, x, v, dt=prm["dt"], mu=prm["mu"], lam=prm["lam"], dhat=prm["dhat"],
                              kappa=prm["kappa"], eps_d=1e-7, pcg_tol=1e-8, max_pcg=2000, max_newton=200,
                              precision=prec, hess_mode=hm)
        assert st["converged"] == 1, (prec, st)
        out[prec] = x.cpu().numpy()
        assert C.count_intersections(out[prec], sc0["tris"], sc0["edges"]) == 0
    err = np.abs(out["mixed"] - out["fp64"]).max()
    assert err <= 1e-6 * scene.l, f"converged-position difference {err:.3e}"


def test_newton_steps_on_a_ball_grid_keep_the_exact_contact_set(gipc):
    """Several time steps of balls settling on a floor.  Within a step the time-step driver reuses
    its broad-phase candidates while the surface stays within their margin.  After every step its
    contact count must equal a fresh detection at the result, and the result must be free of
    intersections."""
    sc = synth.sphere_grid(2, 2, radius=0.05, cells=8, gap=1e-3, floor_cells=6)
    srf = _surface(gipc, sc)
    scene = gipc.Scene(_dev(sc["x"]), _dev(sc["tets"]), srf, 1000.0, fixed=_dev(sc["fixed"]), l=sc["l"])
    mu, lam = gipc.snh_params(1e5, 0.4)
    dh = 1e-3 * sc["l"]
    x, v = _dev(sc["x"]), _dev(sc["v"])
    total_iters = 0
    for _ in range(4):
        st = gipc.newton_step(scene, x, v, dt=0.01, mu=mu, lam=lam, dhat=dh, kappa=1e3, eps_d=1e-4, pcg_tol=1e-6,
                              max_pcg=1000, max_newton=50)
        total_iters += st["newton_iters"]
        fresh, _ = gipc.find_contacts(x, scene.rest_x, srf, dh, capacity=None)
        assert st["contacts"] == fresh.shape[1]
        xs = x.cpu().numpy()
        assert C.count_intersections(xs, sc["tris"], sc["edges"]) == 0
    assert total_iters > 4 and st["contacts"] > 0


def _soup(seed, cells=(6, 6, 8), pitch=0.01, dh=2e-3):
    """One independent, nearly flat triangle per cell of a lattice, against the ceiling of its cell
    in even layers and the floor in odd ones, kept a random 0.2-1.5 dhat inside the cell, so that
    the pairs of layers face each other 0.4-3 dhat apart and nothing intersects.  Generic
    triangles (heights jittered by 0.3 dhat), slivers (third corner within 1e-4 of the size off
    the line of the other two), needles (one edge 1e-6 of the size) and flat triangles dhat
    (1 + 1e-7 j) / 2 from the wall (nearly parallel edges, distances within rounding of dhat)."""
    rng = np.random.default_rng(seed)
    corners = []
    k = 0
    for ix in range(cells[0]):
        for iy in range(cells[1]):
            for iz in range(cells[2]):
                lo = np.array([ix, iy, iz], float) * pitch
                g = rng.uniform(0.2, 1.5, size=(2, 3)) * dh
                a, b = lo + g[0], lo + pitch - g[1]
                up = iz % 2 == 0   # against the ceiling (facing the next layer up)

                def u():
                    q = a + (b - a) * rng.uniform(0.0, 1.0, 3)
                    q[2] = b[2] - rng.uniform(0.0, 0.3) * dh if up else a[2] + rng.uniform(0.0, 0.3) * dh
                    return q
                kind = k % 4
                if kind == 0:
                    t = np.array([u(), u(), u()])
                elif kind == 1:
                    p0, p1 = u(), u()
                    t = np.clip(np.array([p0, p1, p0 + rng.uniform(0.2, 0.8) * (p1 - p0) +
                                          1e-4 * pitch * rng.normal(size=3)]), a, b)
                elif kind == 2:
                    p0 = u()
                    t = np.clip(np.array([p0, p0 + 1e-6 * pitch * rng.normal(size=3), u()]), a, b)
                else:
                    t = np.array([u(), u(), u()])
                    half = 0.5 * dh * (1.0 + 1e-7 * rng.integers(-3, 4))
                    t[:, 2] = lo[2] + pitch - half if up else lo[2] + half
                corners.append(t)
                k += 1
    x = np.ascontiguousarray(np.concatenate(corners).T)
    m = x.shape[1]
    tris = np.arange(m, dtype=np.int32).reshape(-1, 3).T.copy()
    edges = np.concatenate([tris[[0, 1]], tris[[1, 2]], tris[[2, 0]]], axis=1).astype(np.int32)
    return x, tris, np.ascontiguousarray(edges), np.arange(m, dtype=np.int32)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_soup_contacts_and_ccd_bit_exact(gipc, seed):
    """Degenerate and borderline shapes against the oracle: most candidate pairs are dropped by the
    float32 prefilter before the float64 classification and CCD, which must change no result."""
    dh = 2e-3
    x, tris, edges, verts = _soup(seed, dh=dh)
    ref_st, ref_eps = C.find_contacts(x, x, tris, edges, verts, dh)
    srf = gipc.Surface(_dev(tris), _dev(edges), _dev(verts))
    st, eps = gipc.find_contacts(_dev(x), _dev(x), srf, dh, capacity=None)
    assert ref_st.shape[1] > 20
    assert np.array_equal(st.cpu().numpy(), ref_st)
    assert np.array_equal(eps.cpu().numpy(), ref_eps)
    rng = np.random.default_rng(100 + seed)
    for scale in (0.05 * dh, 0.5 * dh, 3 * dh):
        d = scale * rng.normal(size=x.shape)
        ref = C.max_step(x, d, tris, edges, verts)
        got = gipc.ccd_max_step(_dev(x), _dev(d), srf)
        assert got == ref, (scale, got, ref)
        assert 0.0 < ref <= 1.0
