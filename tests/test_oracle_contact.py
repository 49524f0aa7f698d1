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
