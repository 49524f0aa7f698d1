"""Pins for the contact oracle: closest-feature classification against brute-force minima,
contact-set completeness, conservative CCD, exact intersection checks, and the Newton step's
energy decrease and non-intersection."""
import math

import numpy as np
import pytest

import synth
from oracle import contact as C
from oracle import newton as N
from oracle import tet as TT


def _tri_min(p, T, k=241):
    u = np.linspace(0, 1, k)
    A, B = np.meshgrid(u, u, indexing="ij")
    m = A + B <= 1
    Q = T[0] + A[m][:, None] * (T[1] - T[0]) + B[m][:, None] * (T[2] - T[0])
    return ((Q - p) ** 2).sum(1).min()


def _seg_seg_min(a0, a1, b0, b1, k=801):
    u = np.linspace(0, 1, k)
    P = a0 + u[:, None] * (a1 - a0)
    Q = b0 + u[:, None] * (b1 - b0)
    return ((P[:, None, :] - Q[None, :, :]) ** 2).sum(-1).min()


def test_point_triangle_distance_and_type():
    rng = np.random.default_rng(1)
    seen = set()
    for _ in range(120):
        T = rng.uniform(0, 1, (3, 3))
        p = rng.uniform(-0.3, 1.3, 3)
        res = C.classify_pt(tuple(p), *map(tuple, T))
        seen.add(res[0])
        bf = _tri_min(p, T)
        assert res[1] <= bf * (1 + 1e-12) + 1e-15
        assert bf <= res[1] + 2e-2 * math.sqrt(res[1]) * 0.01 + 1e-5
        if res[0] == "PP":
            assert res[1] == pytest.approx(((p - T[res[2]]) ** 2).sum(), rel=1e-12)
    assert seen == {"PT", "PE", "PP"}


def test_edge_edge_distance_and_type():
    rng = np.random.default_rng(2)
    seen = set()
    for _ in range(120):
        a0, a1, b0, b1 = rng.uniform(0, 1, (4, 3))
        res = C.classify_ee(*map(tuple, (a0, a1, b0, b1)))
        seen.add(res[0])
        bf = _seg_seg_min(a0, a1, b0, b1)
        assert res[1] <= bf * (1 + 1e-12) + 1e-15
        assert bf <= res[1] + 1e-5
    assert {"EE", "PE", "PP"} <= seen
    # exactly parallel edges fall back to endpoint features
    res = C.classify_ee((0, 0, 0), (1, 0, 0), (0.2, 0.1, 0), (1.5, 0.1, 0))
    assert res[0] == "PE" and res[1] == pytest.approx(0.01, rel=1e-12)


def _scene():
    sc = synth.two_cubes(gap=0.0)
    x = sc["x"].copy()
    rng = np.random.default_rng(3)
    x[:, 125:] += np.array([0.031, 0.017, 0.0])[:, None]          # break the alignment
    x += 1e-4 * rng.normal(size=x.shape)
    return sc, x


def test_contact_set_is_complete_and_filtered():
    sc, x = _scene()
    dhat = 2e-3
    x[2, 125:] += 1.0e-3                                       # put the faces within dhat
    st, eps = C.find_contacts(x, x, sc["tris"], sc["edges"], sc["verts"], dhat)
    assert st.shape[1] > 50
    # brute force: every point-triangle pair under dhat appears (as some stencil on that point)
    pts_in = {(-int(st[0, i]) - 1) for i in range(st.shape[1]) if st[0, i] < 0}
    for p in sc["verts"][::7]:
        for t in range(sc["tris"].shape[1]):
            tri = sc["tris"][:, t]
            if p in tri:
                continue
            if _tri_min(x[:, p], x[:, tri].T, 61) < dhat * dhat * 0.5:
                assert int(p) in pts_in
    # all listed contacts are closer than dhat
    from oracle import geometry as G
    for i in range(st.shape[1]):
        typ, verts = G.decode(st[:, i])
        g = G.exact_geometry(typ, [x[:, v] for v in verts], dhat)["g"]
        assert g < 1


def test_accd_is_conservative():
    rng = np.random.default_rng(4)
    for kind in ("PT", "EE"):
        for _ in range(25):
            X = [tuple(v) for v in rng.uniform(0, 1, (4, 3))]
            P = [tuple(v) for v in rng.normal(scale=0.6, size=(4, 3))]
            t = C.accd(X, P, kind)
            assert 0.0 <= t <= 1.0
            f = C.classify_pt if kind == "PT" else C.classify_ee
            for s in np.linspace(0, t, 200):
                Xs = [tuple(np.add(X[i], np.multiply(s, P[i]))) for i in range(4)]
                assert f(*Xs)[1] > 0.0
    # a point falling onto a triangle stops short of it
    X = [(0.1, 0.1, 0.01), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    P = [(0, 0, -0.02), (0, 0, 0), (0, 0, 0), (0, 0, 0)]
    assert 0.3 < C.accd(X, P, "PT") < 0.5
    assert C.accd(X, [(0, 0, 0.02)] + P[1:], "PT") == 1.0


# ---- ACCD against the time of impact of linear motions --------------------------------------
# For two primitives translating toward each other along the common normal, the distance falls
# linearly, d(t) = h - v t, and the relative speed bound l_p of additive CCD equals v.  Its first
# advance (1 - s) d0 / l_p then lands exactly at distance s d0, and the next advance would go
# below s d0, so the returned step is (1 - s) TOI with TOI = h / v (capped at 1).  For an oblique
# translation (speed |P| > normal speed a) the distance is still h - a t and the steps follow the
# advance law t += 0.9 d / l_p until the next one would end below s d0.

def _accd_expected(h, a, L, s=0.1, tmax=1.0):
    """The ACCD step for the exact distance d(t) = h - a t and speed bound L."""
    t = 0.0
    tl = (1.0 - s) * h / L
    while True:
        d_next = h - a * (t + tl)
        if t > 0.0 and d_next < s * h:
            return t
        t = t + tl
        if t > tmax:
            return tmax
        tl = 0.9 * d_next / L


def _head_on_cases():
    tri = [(-1.0, -1.0, 0.0), (2.0, -1.0, 0.0), (-1.0, 2.0, 0.0)]
    for h, vp, vt in ((0.01, 0.02, 0.0), (0.003, 0.01, 0.004), (0.2, 0.05, 0.0), (1e-4, 3e-3, 1e-3)):
        X = [(0.2, 0.3, h)] + tri
        P = [(0.0, 0.0, -vp)] + [(0.0, 0.0, vt)] * 3
        yield "PT", X, P, h / (vp + vt)
    for h, u, v in ((0.01, 0.01, 0.01), (0.004, 0.0, 0.02), (0.3, 0.1, 0.05)):
        X = [(-1.0, 0.1, 0.0), (1.0, 0.1, 0.0), (0.2, -1.0, h), (0.2, 1.0, h)]
        P = [(0.0, 0.0, u)] * 2 + [(0.0, 0.0, -v)] * 2
        yield "EE", X, P, h / (u + v)


def _check_head_on(accd):
    worst = 0.0
    for kind, X, P, toi in _head_on_cases():
        want = min(1.0, 0.9 * toi)
        worst = max(worst, abs(accd(X, P, kind) - want) / want)
    return worst


def _check_oblique(accd):
    worst = 0.0
    tri = [(-1.0, -1.0, 0.0), (2.0, -1.0, 0.0), (-1.0, 2.0, 0.0)]
    for h, a, tang in ((0.01, 0.02, 0.03), (0.002, 0.001, 0.004), (0.05, 0.01, 0.002)):
        X = [(0.1, 0.2, h)] + tri
        P = [(tang, 0.0, -a)] + [(0.0, 0.0, 0.0)] * 3
        want = _accd_expected(h, a, math.hypot(tang, a))
        worst = max(worst, abs(accd(X, P, "PT") - want) / want)
    return worst


def test_accd_step_is_the_time_of_impact_law():
    assert _check_head_on(C.accd) < 1e-12
    assert _check_oblique(C.accd) < 1e-12


def test_accd_pins_catch_planted_mistakes():
    import inspect
    src = inspect.getsource(C.accd)

    def mutant(old, new):
        assert src.count(old) == 1, old
        ns = dict(vars(C))
        exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
        return ns["accd"]

    halved = mutant("    return t\n", "    return 0.5 * t\n")
    timid_first = mutant("tl = (1.0 - s) * d / lp", "tl = 0.5 * (1.0 - s) * d / lp")
    timid_later = mutant("tl = 0.9 * d / lp", "tl = 0.5 * d / lp")
    for m in (halved, timid_first, timid_later):
        assert max(_check_head_on(m), _check_oblique(m)) > 1e-3


def test_intersection_check():
    sc = synth.two_cubes()
    x = sc["x"].copy()
    x[0, 125:] += 0.1
    x[1, 125:] += 0.07
    assert C.count_intersections(x, sc["tris"], sc["edges"]) == 0
    x[2, 125:] -= 0.6
    assert C.count_intersections(x, sc["tris"], sc["edges"]) > 0


@pytest.mark.slow
def test_newton_step_decreases_energy_and_stays_intersection_free():
    sc0, x0 = _scene()
    dh = 1e-3 * sc0["l"]
    x0[2, 125:] += 0.5 * dh
    mu, lam = TT.snh_params(1e5, 0.4)
    prm = dict(dhat=dh, kappa=1e3, dt=0.01, mu=mu, lam=lam, gravity=(0, 0, -9.81), eps_d=1e-2,
               pcg_tol=1e-4, max_pcg=500, max_newton=8, max_ls=30)
    sc = N.build_scene(dict(sc0, x=x0), prm, 1000.0)
    v0 = sc0["v"]
    xt = x0.copy()
    free = ~sc["fixed"].astype(bool)
    xt[:, free] += 0.01 * v0[:, free] + 1e-4 * np.array([0, 0, -9.81])[:, None]
    I0, _, _ = N.potential(x0, xt, sc, prm)
    hist = []
    x, v, st = N.newton_step(sc, x0, v0, prm, history=hist)
    assert st["energy"] <= I0
    assert st["contacts"][0] > 0
    for h in hist:
        assert C.count_intersections(h, sc["tris"], sc["edges"]) == 0
