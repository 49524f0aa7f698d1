"""Pins for the oracle: each checks it against something other than itself.

Sources of truth: closed forms the paper prints (supplement Sec. S3, Appendix A/B,
Sec. 6.2 p/k1/k2), the mathematics (finite differences, brute-force minima,
textbook Gauss-Newton for point-point, independent distance formulas,
eigendecompositions of directly differentiated J-space Hessians), and special
cases.  None of these needs a GPU.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import barrier as B
from oracle import geometry as geo
from oracle import stencil as S
from oracle.jet import Dual, Jet, jlog, jsqrt

DHAT = synth.UNIT_DHAT
KAPPA = 1e3


# ----------------------------------------------------------------------------- jets
def test_dual_exact_rational_derivatives():
    z = Fraction(0)
    x = Dual.variable(Fraction(3, 7), 0, 2, z)
    y = Dual.variable(Fraction(-5, 11), 1, 2, z)
    f = x * y + x / y - (x - y) * (x - y)
    xv, yv = Fraction(3, 7), Fraction(-5, 11)
    assert f.v == xv * yv + xv / yv - (xv - yv) ** 2
    assert f.d[0] == yv + 1 / yv - 2 * (xv - yv)
    assert f.d[1] == xv - xv / yv ** 2 + 2 * (xv - yv)


def test_jet_second_order_matches_closed_form_and_fd():
    def fn(a, b):
        return jlog(a * b) + jsqrt(a) / b

    a0, b0 = 0.7, 1.9
    j = fn(Jet.variable(a0, 0, 2), Jet.variable(b0, 1, 2))
    # closed form
    ga = 1 / a0 + 0.5 / (math.sqrt(a0) * b0)
    gb = 1 / b0 - math.sqrt(a0) / b0 ** 2
    haa = -1 / a0 ** 2 - 0.25 / (a0 ** 1.5 * b0)
    hab = -0.5 / (math.sqrt(a0) * b0 ** 2)
    hbb = -1 / b0 ** 2 + 2 * math.sqrt(a0) / b0 ** 3
    np.testing.assert_allclose(j.g, [ga, gb], rtol=1e-14)
    np.testing.assert_allclose(j.h, [[haa, hab], [hab, hbb]], rtol=1e-13)
    h = 1e-5
    f = lambda a, b: math.log(a * b) + math.sqrt(a) / b
    fd_aa = (f(a0 + h, b0) - 2 * f(a0, b0) + f(a0 - h, b0)) / h ** 2
    assert abs(fd_aa - haa) < 1e-5 * abs(haa)


# ----------------------------------------------------------------------------- decoding
def test_decode_all_types_including_vertex_zero():
    N = geo.NULL
    cases = {
        (0, 1, 2, 3): (geo.EE, (0, 1, 2, 3)),
        (-1, 1, 2, 3): (geo.PT, (0, 1, 2, 3)),
        (-1, 5, 6, N): (geo.PE, (0, 5, 6)),
        (-8, 0, N, N): (geo.PP, (7, 0)),
        (4, -1, 2, 3): (geo.EE_PAR, (4, 0, 2, 3)),
        (-1, -2, 3, -5): (geo.PE_PAR, (0, 1, 3, 4)),
        (-1, -2, -3, -4): (geo.PP_PAR, (0, 1, 2, 3)),
    }
    for t, want in cases.items():
        assert geo.decode(t) == want
    # the generator's encoding decodes back to the same ids
    for kind in synth.TYPE_IDS:
        ids = [10, 11, 12, 13][: geo.N_VERTS[synth.TYPE_IDS[kind]]]
        assert geo.decode(synth.encode(kind, ids)) == (synth.TYPE_IDS[kind], tuple(ids))
    for bad in [(-1, 1, N, 3), (0, 1, -3, 3), (-1, -2, 3, 4), (-1, -2, -3, 4), (N, 1, 2, 3)]:
        with pytest.raises(ValueError):
            geo.decode(bad)


# ----------------------------------------------------------------------------- geometry
def _F(p):
    return [Fraction(float(v)) for v in p]


def test_distance_special_cases():
    # point above the z=0 triangle: d = height
    p = _F([0.2, 0.3, 0.125])
    assert geo.sqdist_point_plane(p, _F([0, 0, 0]), _F([1, 0, 0]), _F([0, 1, 0])) == Fraction(1, 64)
    # x-axis line vs y-direction line at height 0.25
    assert geo.sqdist_line_line(_F([0, 0, 0]), _F([1, 0, 0]), _F([0.5, -1, 0.25]),
                                _F([0.5, 1, 0.25])) == Fraction(1, 16)
    # point vs x-axis
    assert geo.sqdist_point_line(_F([0.3, 0.5, 0.0]), _F([0, 0, 0]), _F([2, 0, 0])) == Fraction(1, 4)
    assert geo.sqdist_point_point(_F([1, 2, 3]), _F([1, 2, 3.5])) == Fraction(1, 4)
    # parallel measure of orthogonal unit edges is 1, of parallel edges 0
    assert geo.parallel_measure(_F([0, 0, 0]), _F([1, 0, 0]), _F([0, 0, 1]), _F([0, 1, 1])) == 1
    assert geo.parallel_measure(_F([0, 0, 0]), _F([1, 0, 0]), _F([0, 0, 1]), _F([3, 0, 1])) == 0


def test_distances_match_cross_product_forms_exactly():
    """Normal-equation minima equal the independent cross-product expressions exactly."""
    rng = np.random.default_rng(5)
    for _ in range(40):
        P = [_F(v) for v in rng.uniform(0, 1, (4, 3))]
        sub = lambda a, b: [a[i] - b[i] for i in range(3)]
        dot = lambda a, b: sum(a[i] * b[i] for i in range(3))
        cross = lambda a, b: [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2],
                              a[0] * b[1] - a[1] * b[0]]
        n = cross(sub(P[2], P[1]), sub(P[3], P[1]))
        assert geo.sqdist_point_plane(P[0], P[1], P[2], P[3]) == dot(sub(P[0], P[1]), n) ** 2 / dot(n, n)
        n = cross(sub(P[1], P[0]), sub(P[3], P[2]))
        assert geo.sqdist_line_line(P[0], P[1], P[2], P[3]) == dot(sub(P[2], P[0]), n) ** 2 / dot(n, n)
        e = sub(P[2], P[1])
        w = cross(sub(P[0], P[1]), e)
        assert geo.sqdist_point_line(P[0], P[1], P[2]) == dot(w, w) / dot(e, e)


def test_distance_is_minimum_brute_force():
    """The PT / EE value is the minimum over a dense parameter grid (up to grid resolution)."""
    rng = np.random.default_rng(11)
    for kind in ("PT", "EE"):
        P = synth.make_stencil(kind, rng, 0.05)
        d2 = float(geo.exact_geometry(synth.TYPE_IDS[kind], P, 1.0)["g"])
        u = np.linspace(-0.5, 1.5, 801)
        A, Bm = np.meshgrid(u, u, indexing="ij")
        if kind == "PT":
            Q = P[1] + A[..., None] * (P[2] - P[1]) + Bm[..., None] * (P[3] - P[1])
            dist2 = ((Q - P[0]) ** 2).sum(-1)
        else:
            Q1 = P[0] + A[..., None] * (P[1] - P[0])
            Q2 = P[2] + Bm[..., None] * (P[3] - P[2])
            dist2 = ((Q1 - Q2) ** 2).sum(-1)
        assert dist2.min() >= d2 * (1 - 1e-12)
        assert dist2.min() <= d2 + 1e-4 * math.sqrt(d2) + 1e-6


@pytest.mark.parametrize("kind", list(synth.TYPE_IDS))
def test_exact_gradients_match_finite_differences(kind):
    """Exact Dual gradients vs central differences taken in exact rationals (step 2^-70)."""
    rng = np.random.default_rng(17 + synth.TYPE_IDS[kind])
    typ = synth.TYPE_IDS[kind]
    h = Fraction(1, 2 ** 70)
    for _ in range(3):
        P = synth.make_stencil(kind, rng, DHAT)
        G = geo.exact_geometry(typ, P, DHAT)
        dh2 = Fraction(float(DHAT)) ** 2
        fns = [("dg", lambda Q: geo._squared_distance(typ, Q) / dh2)]
        if geo.PARALLEL[typ]:
            fns.append(("dc", lambda Q: geo.parallel_measure(Q[0], Q[1], Q[2], Q[3])))
        for grad, fn in fns:
            for idx in range(3 * len(P)):
                Qp = [_F(v) for v in P]
                Qm = [_F(v) for v in P]
                Qp[idx // 3][idx % 3] += h
                Qm[idx // 3][idx % 3] -= h
                fd = (fn(Qp) - fn(Qm)) / (2 * h)
                scale = max(abs(G[grad][i]) for i in range(3 * len(P)))
                assert abs(fd - G[grad][idx]) <= Fraction(1, 10 ** 12) * scale


# ----------------------------------------------------------------------------- barrier
GS = np.unique(np.concatenate([10.0 ** np.linspace(-9, -0.01, 60), 1 - 10.0 ** np.linspace(-1, -6, 12)]))


def test_stiff_barrier_values():
    for dh in (1.0, 0.37):
        g = 0.25
        assert B.b_stiff(g, dh) == pytest.approx(dh ** 4 * 0.75 ** 2 * math.log(0.25) ** 2, rel=1e-15)
        assert B.b_stiff(1.0, dh) == 0.0


@pytest.mark.parametrize("dh", [1.0, 0.37, DHAT])
def test_supplement_expanded_eigenvalues_for_eq12(dh):
    """Sec. S3 prints lambda_1 and d lambda_1/dg for the Eq. 12 barrier."""
    for g in GS:
        lg = math.log(g)
        lam1 = 2 * dh ** 4 * (6 * g + 2 * g * lg - 7 * g ** 2 - 6 * g ** 2 * lg + 1) / g
        assert B.lambda1(g, dh, B.b_log) == pytest.approx(lam1, rel=1e-9, abs=1e-14 * dh ** 4)
        dlam = -2 * dh ** 4 * (13 * g ** 2 - 2 * g + 6 * g ** 2 * lg + 1) / g ** 2
        h = 1e-6 * g
        fd = (B.lambda1(g + h, dh, B.b_log) - B.lambda1(g - h, dh, B.b_log)) / (2 * h)
        assert fd == pytest.approx(dlam, rel=1e-5)
        # lambda_{2,3}: the supplement prints a 1/g^2 denominator; differentiating Eq. 12 gives 1/g
        lam23 = -2 * dh ** 4 * (g - 1) * (g + 2 * g * lg - 1) / g
        assert B.lambda23(g, dh, B.b_log) == pytest.approx(lam23, rel=1e-9, abs=1e-14 * dh ** 4)


@pytest.mark.parametrize("barrier", [B.b_log, B.b_stiff])
def test_eigenvalue_signs_on_unit_interval(barrier):
    """lambda_1 > 0 and decreasing, lambda_2,3 <= 0 on g in (0,1) (Sec. S3; Eq. 24 keeps it, Sec. 5.4)."""
    lam1 = np.array([B.lambda1(g, 1.0, barrier) for g in GS])
    lam23 = np.array([B.lambda23(g, 1.0, barrier) for g in GS])
    assert (lam1 > 0).all()
    assert (np.diff(lam1) < 0).all()
    assert (lam23 <= 0).all()


def test_lambda1_is_second_derivative_in_f():
    """With g = f^2, Eq. 18 equals d^2 b / d f^2 (finite differences in f)."""
    for g in GS[5:-3]:
        f = math.sqrt(g)
        h = 1e-3 * min(f, 1 - f)
        bf = lambda ff: B.b_stiff(ff * ff, 1.0)
        fd2 = lambda hh: (bf(f + hh) - 2 * bf(f) + bf(f - hh)) / hh ** 2
        fd = (4 * fd2(h / 2) - fd2(h)) / 3          # Richardson: O(h^4) truncation
        assert B.lambda1(g, 1.0) == pytest.approx(fd, rel=2e-6)


def _fd12(fn, x, h):
    """Richardson-extrapolated central differences (first, second derivative)."""
    d1 = lambda hh: (fn(x + hh) - fn(x - hh)) / (2 * hh)
    d2 = lambda hh: (fn(x + hh) - 2 * fn(x) + fn(x - hh)) / hh ** 2
    return (4 * d1(h / 2) - d1(h)) / 3, (4 * d2(h / 2) - d2(h)) / 3


def test_appendix_a_point_point_scalar():
    """App. A: with f = sqrt(d) (so g = d) the GN scalar is lambda_1/(4d) = b_dd + b_d/(2d)."""
    for d in (1e-4, 3e-3, 0.05, 0.4, 0.9):
        lam = B.lambda1(d, 1.0, lambda g, dh: B.b_ipc(g, dh))
        fd_bd, fd_bdd = _fd12(lambda dd: B.b_ipc(dd, 1.0), d, 1e-3 * min(d, 1 - d))
        assert lam / (4 * d) == pytest.approx(fd_bdd + fd_bd / (2 * d), rel=1e-6)


def test_filter_eq23():
    eg = B.eps_g_of(0.1)
    assert eg == pytest.approx(0.01, rel=1e-15)
    thr = B.lambda1(eg, DHAT)
    for g in GS:
        lf = B.lambda1_filtered(g, DHAT)
        assert lf == (thr if g < eg else B.lambda1(g, DHAT))
        assert lf == pytest.approx(min(B.lambda1(g, DHAT), thr), rel=1e-15)
    # continuous at eps_g
    assert B.lambda1_filtered(eg * (1 + 1e-12), DHAT) == pytest.approx(thr, rel=1e-9)


def test_mollifier_eq25():
    ex = 2.5e-4
    assert B.mollifier(ex, ex, ex) == 1.0
    e1 = B.mollifier(ex * (1 - 1e-9), ex * (1 - 1e-9), ex)
    assert e1 == pytest.approx(1.0, abs=1e-15)
    _, de, _ = B.derivs1(lambda gm, _: B.mollifier(gm, gm.v, ex), ex * (1 - 1e-12), None)
    assert abs(de) < 1e-8 / ex
    assert B.mollifier(0.0, 0.0, ex) == 0.0


# ----------------------------------------------------------------------------- stencils
def _energy_fn(typ, eps_x):
    return lambda P: S.eval_stencil(typ, P, eps_x, DHAT, KAPPA)["energy"]


def _stencil(kind, seed, filtered=None):
    """An active stencil of the kind; ``filtered`` True/False forces which side of eps_g."""
    rng = np.random.default_rng(seed)
    typ = synth.TYPE_IDS[kind]
    while True:
        P = synth.make_stencil(kind, rng, DHAT)
        eps_x = geo.eps_x_rest(typ, P)
        r = S.eval_stencil(typ, P, eps_x, DHAT, KAPPA)
        if not r["flags"] & S.FLAG_ACTIVE:
            continue
        if filtered is None or bool(r["flags"] & S.FLAG_FILTERED) == filtered:
            return typ, P, eps_x, r


@pytest.mark.parametrize("kind", list(synth.TYPE_IDS))
def test_gradient_matches_fd_of_energy(kind):
    for seed in range(4):
        typ, P, eps_x, r = _stencil(kind, 100 + seed, filtered=seed % 2 == 0)
        d = math.sqrt(r["aux"]["g"]) * DHAT
        E = _energy_fn(typ, eps_x)
        fd = np.zeros(3 * len(P))
        # the step must be small against every length the energy varies on: d, and for the
        # mollified family the lateral offset |e| sin(theta) ~ sqrt(c) of the nearly parallel edges
        h = 1e-4 * min(d, math.sqrt(r["aux"]["c"])) if geo.PARALLEL[typ] else 1e-4 * d
        for idx in range(3 * len(P)):
            Pp, Pm = P.copy(), P.copy()
            Pp[idx // 3, idx % 3] += h
            Pm[idx // 3, idx % 3] -= h
            hh = (Pp[idx // 3, idx % 3] - Pm[idx // 3, idx % 3])
            fd[idx] = (E(Pp) - E(Pm)) / hh
        assert np.linalg.norm(fd - r["grad"]) <= 1e-5 * np.linalg.norm(r["grad"])


@pytest.mark.parametrize("kind", list(synth.TYPE_IDS))
def test_hessian_symmetric_psd_rank_one(kind):
    for seed in range(4):
        _, P, _, r = _stencil(kind, 200 + seed)
        H = r["hess"]
        assert np.array_equal(H, H.T) or np.abs(H - H.T).max() <= 1e-15 * np.abs(H).max()
        ev = np.linalg.eigvalsh(0.5 * (H + H.T))
        assert ev.min() >= -1e-12 * ev.max()
        sv = np.linalg.svd(H, compute_uv=False)
        assert sv[1] <= 1e-12 * sv[0]
        np.testing.assert_allclose(H, r["lam"] * np.outer(r["w"], r["w"]), rtol=1e-12,
                                   atol=1e-14 * np.abs(H).max())


def test_inactive_beyond_dhat():
    for kind, P in [("PP", np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3 + 1.0001 * DHAT]])),
                    ("PT", np.array([[0.2, 0.3, 1.5 * DHAT], [0, 0, 0], [1, 0, 0], [0, 1, 0]]))]:
        r = S.eval_stencil(synth.TYPE_IDS[kind], P, 0.0, DHAT, KAPPA)
        assert r["flags"] == 0 and r["energy"] == 0 and not r["grad"].any() and not r["hess"].any()


def test_point_point_is_textbook_gauss_newton():
    """PP: kappa * B''(d) grad d grad d^T with B(d) = b((d/dhat)^2), grad d = (u, -u) (unfiltered range)."""
    for ratio in (0.11, 0.3, 0.75, 0.97):
        u = np.array([0.48, -0.6, 0.64])
        P = np.array([[0.3, 0.4, 0.5], [0.3, 0.4, 0.5]]) + np.array([[0, 0, 0], -ratio * DHAT * u])
        r = S.eval_stencil(geo.PP, P, 0.0, DHAT, KAPPA)
        d = math.sqrt(r["aux"]["g"]) * DHAT
        Bd = lambda dd: B.b_stiff((dd / DHAT) ** 2, DHAT)
        h = 1e-4 * d
        Bdd = (Bd(d + h) - 2 * Bd(d) + Bd(d - h)) / h ** 2
        nd = (P[0] - P[1]) / np.linalg.norm(P[0] - P[1])
        gd = np.concatenate([nd, -nd])
        np.testing.assert_allclose(r["hess"], KAPPA * Bdd * np.outer(gd, gd), rtol=1e-4,
                                   atol=1e-6 * np.abs(r["hess"]).max())


@pytest.mark.parametrize("kind", ["PT", "EE", "PE", "PP"])
def test_appendix_b_norms(kind):
    """App. B: ||db/dx|| = -2 sqrt(g) b_g ||grad f|| and ||H||_F = lambda_1 ||grad f||^2."""
    for seed in range(4):
        typ, P, eps_x, r = _stencil(kind, 300 + seed, filtered=seed % 2 == 0)
        a = r["aux"]
        gf = r["w"]
        assert np.linalg.norm(r["grad"]) == pytest.approx(
            -2 * math.sqrt(a["g"]) * a["b_g"] * np.linalg.norm(gf) * KAPPA, rel=1e-12)
        assert np.linalg.norm(r["hess"]) == pytest.approx(a["lambda1_hat"] * gf @ gf * KAPPA, rel=1e-12)


def _jspace_hessian(typ, aux, eps_x, m):
    """Direct 2nd derivatives of b (or btilde) w.r.t. all m*m entries of J at the evaluation point."""
    n = m * m
    J0 = np.eye(m)
    if geo.PARALLEL[typ]:
        J0[1, 1] = math.sqrt(aux["c"])
    J0[m - 1, m - 1] = aux["f"]
    Jv = [[Jet.variable(J0[i, j], i + m * j, n) for j in range(m)] for i in range(m)]
    col = lambda j: sum((Jv[i][j] * Jv[i][j] for i in range(m)), Jet.const(0.0, n))
    g = col(m - 1)                                  # ||J n_g||^2
    b = B.b_stiff(g, DHAT)
    if geo.PARALLEL[typ]:
        gam = col(1)                                # ||J n_gamma||^2
        b = B.mollifier(gam, aux["c"], eps_x) * b
    return np.array(b.h)


@pytest.mark.parametrize("kind", ["PT", "EE", "PE", "PP"])
def test_plain_jspace_eigensystem(kind):
    """Eq. 18-21: eigenvalues {lambda_1, 2 b_g (m-1 times), 0...}; Q_1 = e_m e_m^T."""
    typ = synth.TYPE_IDS[kind]
    m = S.M_DIM[typ]
    for seed in range(4):
        _, P, eps_x, r = _stencil(kind, 400 + seed, filtered=seed % 2 == 0)
        a = r["aux"]
        H = _jspace_hessian(typ, a, eps_x, m)
        want = sorted([a["lambda1"]] + [a["lambda23"]] * (m - 1) + [0.0] * (m * m - m))
        np.testing.assert_allclose(np.linalg.eigvalsh(H), want, rtol=1e-9,
                                   atol=1e-12 * abs(a["lambda1"]))
        q1 = np.zeros(m * m)
        q1[(m - 1) + m * (m - 1)] = 1.0
        np.testing.assert_allclose(H @ q1, a["lambda1"] * q1, rtol=1e-9, atol=1e-12 * abs(a["lambda1"]))
        np.testing.assert_allclose(a["Q1"].reshape(-1, order="F"), q1)


@pytest.mark.parametrize("kind", ["EE_PAR", "PE_PAR", "PP_PAR"])
def test_mollified_jspace_eigensystem(kind):
    """Sec. 6.2 / S4: direct 9x9 J-space Hessian has the structure and eigenvalues of Eq. 32-35."""
    typ = synth.TYPE_IDS[kind]
    n7p_pos = 0
    for seed in range(8):
        _, P, eps_x, r = _stencil(kind, 500 + seed, filtered=seed % 2 == 0)
        a = r["aux"]
        H = _jspace_hessian(typ, a, eps_x, 3)
        lam_g1_raw = 2 * (a["bt_g"] + 2 * a["g"] * a["bt_gg"])
        # structure: diag entries and the single cross term 4t at (5,9)/(9,5) (supplement, aux matrix)
        sc = 1e-9 * max(abs(H).max(), 1e-300)
        assert H[4, 4] == pytest.approx(a["lam_gam1"], rel=1e-9, abs=sc)
        assert H[8, 8] == pytest.approx(lam_g1_raw, rel=1e-9, abs=sc)
        assert H[4, 8] == pytest.approx(4 * a["t"], rel=1e-9, abs=sc)
        for i in (3, 5):
            assert H[i, i] == pytest.approx(a["lam_gam23"], rel=1e-9, abs=sc)
        for i in (6, 7):
            assert H[i, i] == pytest.approx(a["lam_g23"], rel=1e-9, abs=sc)
        off = H.copy()
        for i, j in [(3, 3), (5, 5), (6, 6), (7, 7), (4, 4), (8, 8), (4, 8), (8, 4)]:
            off[i, j] = 0
        assert np.abs(off).max() <= sc
        # closed forms of the 2x2 eigenproblem (Eq. 34-35): p, k1, k2
        lg1 = a["lam_g1"]
        lgam1, t = a["lam_gam1"], a["t"]
        p = 0.5 * math.sqrt(lgam1 ** 2 - 2 * lgam1 * lg1 + lg1 ** 2 + 64 * t * t)
        assert a["lam8p"] == pytest.approx(0.5 * (lgam1 + lg1) + p, rel=1e-10, abs=1e-14 * p)
        assert a["lam7p"] == pytest.approx(0.5 * (lgam1 + lg1) - p, rel=1e-8, abs=1e-12 * p)
        if t != 0:
            k2 = (lgam1 - lg1 + 2 * p) / (8 * t)
            q = a["q8p"]
            np.testing.assert_allclose(q, np.array([k2, 1.0]) / math.sqrt(1 + k2 * k2), rtol=1e-8,
                                       atol=1e-12)
        # sign claims of Sec. 6.2
        assert a["lam_gam23"] >= 0 and lg1 >= 0 and a["lam_g23"] <= 0
        gam, ex = a["c"], eps_x
        if gam < ex / 3 * (1 - 1e-9):
            assert lgam1 > 0
        elif gam > ex / 3 * (1 + 1e-9):
            assert lgam1 <= 0
        n7p_pos += a["lam7p"] > 0
        # unfiltered eigenvalues of the full 9x9: {gam2, gam3, g2, g3, lam7, lam8, 0, 0, 0}
        if not r["flags"] & S.FLAG_FILTERED:
            want = sorted([a["lam_gam23"]] * 2 + [a["lam_g23"]] * 2 + [a["lam7p"], a["lam8p"]] + [0.0] * 3)
            np.testing.assert_allclose(np.linalg.eigvalsh(H), want, rtol=1e-8, atol=1e-10 * abs(H).max())
    assert n7p_pos == 0


@pytest.mark.parametrize("kind", ["EE_PAR", "PE_PAR", "PP_PAR"])
def test_mollified_x_space_chain(kind):
    """The x-space block equals the GN Hessian of x -> btilde(J linearised at x0) minus the
    dropped lambda_7' eigenpair: checks dJ/dx (grad sqrt(c), grad f) and Eq. 36 together."""
    typ = synth.TYPE_IDS[kind]
    for seed in range(3):
        _, P, eps_x, r = _stencil(kind, 600 + seed, filtered=False)
        a = r["aux"]
        G = geo.exact_geometry(typ, P, DHAT)
        gs = np.array([float(v) for v in G["dc"]]) / (2 * math.sqrt(a["c"]))
        gf = np.array([float(v) for v in G["dg"]]) / (2 * a["f"])
        s0, f0 = math.sqrt(a["c"]), a["f"]

        def phi(dx):
            s = s0 + gs @ dx
            f = f0 + gf @ dx
            return B.mollifier(s * s, a["c"], eps_x) * B.b_stiff(f * f, DHAT)

        n = 3 * len(P)
        Hfd = np.zeros((n, n))
        h = 1e-3 * min(s0 / np.linalg.norm(gs), f0 / np.linalg.norm(gf))
        E = np.eye(n) * h
        for i in range(n):
            for j in range(n):
                Hfd[i, j] = (phi(E[i] + E[j]) - phi(E[i] - E[j]) - phi(-E[i] + E[j]) + phi(-E[i] - E[j])) / (4 * h * h)
        q7 = np.array([-a["q8p"][1], a["q8p"][0]])
        w7 = q7[0] * gs + q7[1] * gf
        full = r["hess"] / KAPPA + a["lam7p"] * np.outer(w7, w7)
        np.testing.assert_allclose(full, Hfd, rtol=1e-4, atol=1e-5 * np.abs(Hfd).max())


def test_mollifier_inactive_equals_plain_edge_edge():
    """EE-par with c >= eps_x is the plain EE barrier (e = 1, Eq. 25)."""
    rng = np.random.default_rng(77)
    for _ in range(5):
        P = synth.make_stencil("EE", rng, DHAT)
        ex = geo.eps_x_rest(geo.EE, P)
        r1 = S.eval_stencil(geo.EE, P, ex, DHAT, KAPPA)
        r2 = S.eval_stencil(geo.EE_PAR, P, ex, DHAT, KAPPA)
        assert r2["flags"] & S.FLAG_MOLLIFIED == 0
        assert r2["energy"] == pytest.approx(r1["energy"], rel=1e-14)
        np.testing.assert_allclose(r2["grad"], r1["grad"], rtol=1e-12, atol=1e-14 * np.abs(r1["grad"]).max())
        np.testing.assert_allclose(r2["hess"], r1["hess"], rtol=1e-10, atol=1e-12 * np.abs(r1["hess"]).max())


def test_mollified_energy_continuous_at_eps_x():
    rng = np.random.default_rng(78)
    P = synth.make_stencil("EE", rng, DHAT)
    G = geo.exact_geometry(geo.EE_PAR, P, DHAT)
    c = float(G["c"])
    lo = S.eval_stencil(geo.EE_PAR, P, c * (1 + 1e-10), DHAT, KAPPA)
    hi = S.eval_stencil(geo.EE_PAR, P, c * (1 - 1e-10), DHAT, KAPPA)
    assert lo["flags"] & S.FLAG_MOLLIFIED and not hi["flags"] & S.FLAG_MOLLIFIED
    assert lo["energy"] == pytest.approx(hi["energy"], rel=1e-9)
    np.testing.assert_allclose(lo["grad"], hi["grad"], rtol=1e-6, atol=1e-9 * np.abs(hi["grad"]).max())
