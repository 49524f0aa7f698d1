"""Contact set, classification and continuous collision step (oracle; test infrastructure only).

* Contact set (Eq. 3): every point-triangle pair (a surface vertex and a surface triangle not
  containing it) and every edge-edge pair (two surface edges without a shared vertex) whose
  distance is below dhat.  The distance of a pair is the constrained minimum of Eq. 4 / Eq. 5;
  the active constraints at the minimiser give its stencil type (Sec. 3.1 and Sec. 7.2): an
  interior point-triangle or edge-edge minimum, a point-edge minimum or a point-point minimum.
  Edge-edge pairs with parallel measure c < eps_x (Sec. 6.1) use the nearly-parallel types,
  which keep all four edge vertices.  Each pair contributes one stencil; the list is ordered by
  (surface vertex, triangle) and then by (edge i, edge j), i < j.
* Classification arithmetic is plain float64 with every operation written out in a fixed order,
  so the same decisions are reproduced by any IEEE implementation of the same formulas.
* Step filter (Alg. 1, "maxFeasibleStepSize"): additive CCD -- conservative advancement of
  every pair whose swept bounding boxes overlap, the common displacement removed, steps of
  (1 - s) d / l_p then 0.9 d / l_p until the distance falls below s times the initial
  distance -- with slackness s = 0.1 (reading), capped at 1.
"""
import math

import numpy as np

NULL = -2147483648


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def point_segment(p, a, b):
    """(kind, d2, t): kind 0 = interior (point-edge), 1 = end a, 2 = end b."""
    ab = _sub(b, a)
    ap = _sub(p, a)
    L = _dot(ab, ab)
    t = _dot(ap, ab) / L
    if t <= 0.0:
        return 1, _dot(ap, ap)
    if t >= 1.0:
        bp = _sub(p, b)
        return 2, _dot(bp, bp)
    c = _cross(ap, ab)
    return 0, _dot(c, c) / L


def classify_pt(p, t0, t1, t2):
    """Closest feature of triangle (t0,t1,t2) to p: ('PT', d2) or ('PE', d2, i, j) or ('PP', d2, i)
    with i, j local triangle corner indices."""
    e0 = _sub(t1, t0)
    e1 = _sub(t2, t0)
    v = _sub(p, t0)
    a = _dot(e0, e0)
    b = _dot(e0, e1)
    c = _dot(e1, e1)
    d = _dot(e0, v)
    e = _dot(e1, v)
    det = a * c - b * b
    if det > 0.0:
        s1 = (c * d - b * e) / det
        s2 = (a * e - b * d) / det
        if s1 >= 0.0 and s2 >= 0.0 and s1 + s2 <= 1.0:
            n = _cross(e0, e1)
            vn = _dot(v, n)
            return ("PT", vn * vn / _dot(n, n))
    T = (t0, t1, t2)
    best = None
    for i, j in ((0, 1), (1, 2), (2, 0)):
        kind, d2 = point_segment(p, T[i], T[j])
        cand = ("PE", d2, i, j) if kind == 0 else ("PP", d2, i if kind == 1 else j)
        if best is None or d2 < best[1]:
            best = cand
    return best


def classify_ee(a0, a1, b0, b1):
    """('EE', d2) for an interior minimum, or ('PE', d2, P, E) / ('PP', d2, P, Q) with P a local
    endpoint index (0,1 on edge a; 2,3 on edge b) and E the opposite edge (0 = a, 1 = b), Q the
    other endpoint."""
    e1 = _sub(a1, a0)
    e2 = _sub(b1, b0)
    w = _sub(a0, b0)
    a = _dot(e1, e1)
    b = _dot(e1, e2)
    c = _dot(e2, e2)
    d = _dot(e1, w)
    e = _dot(e2, w)
    det = a * c - b * b
    if det > 1e-14 * a * c:
        s = (b * e - c * d) / det
        t = (a * e - b * d) / det
        if 0.0 < s < 1.0 and 0.0 < t < 1.0:
            n = _cross(e1, e2)
            wn = _dot(w, n)
            return ("EE", wn * wn / _dot(n, n))
    X = (a0, a1, b0, b1)
    best = None
    for P, (sa, sb), E in ((0, (2, 3), 1), (1, (2, 3), 1), (2, (0, 1), 0), (3, (0, 1), 0)):
        kind, d2 = point_segment(X[P], X[sa], X[sb])
        cand = ("PE", d2, P, E) if kind == 0 else ("PP", d2, P, sa if kind == 1 else sb)
        if best is None or d2 < best[1]:
            best = cand
    return best


def parallel_measure(a0, a1, b0, b1):
    n = _cross(_sub(a1, a0), _sub(b1, b0))
    return _dot(n, n)


def eps_x_of(ra0, ra1, rb0, rb1):
    """Same expression (and evaluation order) as the per-stencil eps_x: 1e-3 |a|^2 |b|^2."""
    ea = _sub(ra1, ra0)
    eb = _sub(rb1, rb0)
    return 1e-3 * _dot(ea, ea) * _dot(eb, eb)


def _neg(i):
    return -(int(i) + 1)


def _pt_stencil(pi, tri, res):
    if res[0] == "PT":
        return (_neg(pi), int(tri[0]), int(tri[1]), int(tri[2]))
    if res[0] == "PE":
        return (_neg(pi), int(tri[res[2]]), int(tri[res[3]]), NULL)
    return (_neg(pi), int(tri[res[2]]), NULL, NULL)


def _ee_stencil(ea, eb, res, parallel):
    V = (int(ea[0]), int(ea[1]), int(eb[0]), int(eb[1]))
    mate = {0: 1, 1: 0, 2: 3, 3: 2}
    if res[0] == "EE":
        return (V[0], _neg(V[1]), V[2], V[3]) if parallel else V
    P = res[2]
    if res[0] == "PE":
        E = res[3]
        e0, e1 = (V[0], V[1]) if E == 0 else (V[2], V[3])
        if parallel:
            return (_neg(V[P]), _neg(V[mate[P]]), e0, _neg(e1))
        return (_neg(V[P]), e0, e1, NULL)
    Q = res[3]
    if parallel:
        return (_neg(V[P]), _neg(V[mate[P]]), _neg(V[Q]), _neg(V[mate[Q]]))
    return (_neg(V[P]), V[Q], NULL, NULL)


def _pt(x, i):
    return (float(x[0, i]), float(x[1, i]), float(x[2, i]))


def _aabb(x, ids, pad):
    P = x[:, ids]
    return P.min(axis=-1) - pad, P.max(axis=-1) + pad


def find_contacts(x, rest_x, tris, edges, verts, dhat):
    """Stencil tuples (4, k) int32 and eps_x (k) for all pairs closer than dhat."""
    x = np.asarray(x, dtype=float)
    dh2 = dhat * dhat
    pad = dhat * (1.0 + 1e-9)
    out, eps = [], []
    # point-triangle: conservative AABB prefilter, exact classification decides
    tlo = np.minimum(np.minimum(x[:, tris[0]], x[:, tris[1]]), x[:, tris[2]]) - pad
    thi = np.maximum(np.maximum(x[:, tris[0]], x[:, tris[1]]), x[:, tris[2]]) + pad
    for p in verts:
        xp = x[:, p][:, None]
        cand = np.nonzero(((xp >= tlo) & (xp <= thi)).all(axis=0))[0]
        for t in cand:
            tri = tris[:, t]
            if p in (tri[0], tri[1], tri[2]):
                continue
            res = classify_pt(_pt(x, p), _pt(x, tri[0]), _pt(x, tri[1]), _pt(x, tri[2]))
            if res[1] < dh2:
                out.append(_pt_stencil(p, tri, res))
                eps.append(0.0)
    elo = np.minimum(x[:, edges[0]], x[:, edges[1]]) - pad
    ehi = np.maximum(x[:, edges[0]], x[:, edges[1]]) + pad
    for i in range(edges.shape[1]):
        cand = np.nonzero(((elo[:, i:i + 1] <= ehi) & (ehi[:, i:i + 1] >= elo)).all(axis=0))[0]
        for j in cand:
            if j <= i:
                continue
            ea, eb = edges[:, i], edges[:, j]
            if len({int(ea[0]), int(ea[1]), int(eb[0]), int(eb[1])}) < 4:
                continue
            A0, A1, B0, B1 = _pt(x, ea[0]), _pt(x, ea[1]), _pt(x, eb[0]), _pt(x, eb[1])
            res = classify_ee(A0, A1, B0, B1)
            if res[1] < dh2:
                ex = eps_x_of(_pt(rest_x, ea[0]), _pt(rest_x, ea[1]), _pt(rest_x, eb[0]), _pt(rest_x, eb[1]))
                par = parallel_measure(A0, A1, B0, B1) < ex
                out.append(_ee_stencil(ea, eb, res, par))
                eps.append(ex)
    st = np.array(out, dtype=np.int64).T.astype(np.int32) if out else np.zeros((4, 0), np.int32)
    return np.ascontiguousarray(st), np.array(eps, dtype=float)


# ----------------------------------------------------------------------------- CCD
def _pair_d(X, kind):
    res = classify_pt(*X) if kind == "PT" else classify_ee(*X)
    return math.sqrt(res[1])


def accd(X, P, kind, s=0.1, tmax=1.0, max_iter=100000):
    """Additive CCD of one pair: largest conservative step in [0, tmax] along P."""
    pb = tuple(0.25 * (((P[0][c] + P[1][c]) + P[2][c]) + P[3][c]) for c in range(3))
    Pc = [_sub(P[i], pb) for i in range(4)]
    nrm = [math.sqrt(_dot(q, q)) for q in Pc]
    if kind == "PT":
        lp = nrm[0] + max(nrm[1], nrm[2], nrm[3])
    else:
        lp = max(nrm[0], nrm[1]) + max(nrm[2], nrm[3])
    if lp == 0.0:
        return tmax
    Xc = [tuple(q) for q in X]
    d = _pair_d(Xc, kind)
    if not d > 0.0:
        return 0.0
    g = s * d
    t = 0.0
    tl = (1.0 - s) * d / lp
    for _ in range(max_iter):
        Xc = [(Xc[i][0] + tl * Pc[i][0], Xc[i][1] + tl * Pc[i][1], Xc[i][2] + tl * Pc[i][2]) for i in range(4)]
        d = _pair_d(Xc, kind)
        if t > 0.0 and d < g:
            break
        t = t + tl
        if t > tmax:
            return tmax
        tl = 0.9 * d / lp
    return t


def max_step(x, d, tris, edges, verts, s=0.1):
    """min(1, min over candidate pairs of accd) for the motion x -> x + d."""
    x = np.asarray(x, dtype=float)
    y = x + np.asarray(d, dtype=float)
    lo, hi = np.minimum(x, y), np.maximum(x, y)
    tlo = np.minimum(np.minimum(lo[:, tris[0]], lo[:, tris[1]]), lo[:, tris[2]])
    thi = np.maximum(np.maximum(hi[:, tris[0]], hi[:, tris[1]]), hi[:, tris[2]])
    alpha = 1.0
    for p in verts:
        cand = np.nonzero(((lo[:, p:p + 1] <= thi) & (hi[:, p:p + 1] >= tlo)).all(axis=0))[0]
        for t in cand:
            tri = tris[:, t]
            if p in (tri[0], tri[1], tri[2]):
                continue
            ids = (p, tri[0], tri[1], tri[2])
            X = [_pt(x, i) for i in ids]
            P = [(float(d[0, i]), float(d[1, i]), float(d[2, i])) for i in ids]
            alpha = min(alpha, accd(X, P, "PT", s, 1.0))
    elo = np.minimum(lo[:, edges[0]], lo[:, edges[1]])
    ehi = np.maximum(hi[:, edges[0]], hi[:, edges[1]])
    for i in range(edges.shape[1]):
        cand = np.nonzero(((elo[:, i:i + 1] <= ehi) & (ehi[:, i:i + 1] >= elo)).all(axis=0))[0]
        for j in cand:
            if j <= i:
                continue
            ea, eb = edges[:, i], edges[:, j]
            ids = (ea[0], ea[1], eb[0], eb[1])
            if len(set(int(q) for q in ids)) < 4:
                continue
            X = [_pt(x, q) for q in ids]
            P = [(float(d[0, q]), float(d[1, q]), float(d[2, q])) for q in ids]
            alpha = min(alpha, accd(X, P, "EE", s, 1.0))
    return alpha


# ----------------------------------------------------------------------------- intersection check
def _orient(a, b, c, d):
    """Sign of det[b-a, c-a, d-a] in exact rational arithmetic."""
    from fractions import Fraction as Fr
    A = [Fr(float(v)) for v in a]
    u = [Fr(float(b[i])) - A[i] for i in range(3)]
    v = [Fr(float(c[i])) - A[i] for i in range(3)]
    w = [Fr(float(d[i])) - A[i] for i in range(3)]
    det = (u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0])
           + u[2] * (v[0] * w[1] - v[1] * w[0]))
    return (det > 0) - (det < 0)


def count_intersections(x, tris, edges):
    """Number of (surface edge, surface triangle) pairs without a shared vertex whose segment
    properly crosses the triangle (exact orientation predicates); 0 for an intersection-free
    surface."""
    x = np.asarray(x, dtype=float)
    tlo = np.minimum(np.minimum(x[:, tris[0]], x[:, tris[1]]), x[:, tris[2]])
    thi = np.maximum(np.maximum(x[:, tris[0]], x[:, tris[1]]), x[:, tris[2]])
    hits = 0
    for i in range(edges.shape[1]):
        a, b = int(edges[0, i]), int(edges[1, i])
        lo = np.minimum(x[:, a], x[:, b])[:, None]
        hi = np.maximum(x[:, a], x[:, b])[:, None]
        for t in np.nonzero(((lo <= thi) & (hi >= tlo)).all(axis=0))[0]:
            t0, t1, t2 = (int(q) for q in tris[:, t])
            if len({a, b, t0, t1, t2}) < 5:
                continue
            P = [x[:, q] for q in (a, b, t0, t1, t2)]
            s1, s2 = _orient(P[2], P[3], P[4], P[0]), _orient(P[2], P[3], P[4], P[1])
            if s1 * s2 >= 0:
                continue
            o1 = _orient(P[0], P[1], P[2], P[3])
            o2 = _orient(P[0], P[1], P[3], P[4])
            o3 = _orient(P[0], P[1], P[4], P[2])
            if (o1 > 0 and o2 > 0 and o3 > 0) or (o1 < 0 and o2 < 0 and o3 < 0):
                hits += 1
    return hits
