"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only builds input arrays (vertex positions, sign-encoded stencil
tuples, index spaces).  It holds none of the method's arithmetic: no gap
function, barrier, derivative or eigensystem is computed here.

Stencil tuples use the sign encoding of the paper's Sec. 7.2 with -(i+1) for a
negative slot and INT32_MIN for the '#' placeholder.
"""
import math

import numpy as np

NULL = -2147483648
TYPE_IDS = {"PT": 0, "EE": 1, "PE": 2, "PP": 3, "EE_PAR": 4, "PE_PAR": 5, "PP_PAR": 6}

# Unit-set mix: 40% PT, 40% EE of which a quarter nearly parallel (those split 60/20/20
# into EE-par, PE-par and PP-par by where their closest points fall), 10% PE, 10% PP.
DEFAULT_MIX = (("PT", 0.40), ("EE", 0.30), ("PE", 0.10), ("PP", 0.10),
               ("EE_PAR", 0.06), ("PE_PAR", 0.02), ("PP_PAR", 0.02))

UNIT_DHAT = math.sqrt(3.0) * 1e-3     # 1e-3 x bbox diagonal of [0,1]^3


def _unit(rng):
    while True:
        v = rng.normal(size=3)
        n = np.linalg.norm(v)
        if n > 1e-3:
            return v / n


def _perp(rng, u):
    while True:
        v = np.cross(u, _unit(rng))
        n = np.linalg.norm(v)
        if n > 1e-2:
            return v / n


def _distance(rng, dhat):
    """d = dhat * 10^U(-4, 0), kept away from the filter threshold 0.1 dhat and from dhat."""
    while True:
        r = 10.0 ** rng.uniform(-4.0, 0.0)
        if abs(r - 0.1) > 1e-9 and r < 1.0 - 1e-9:
            return dhat * r


def _segment(rng, min_len=0.1):
    while True:
        a, b = rng.uniform(0.0, 1.0, 3), rng.uniform(0.0, 1.0, 3)
        if np.linalg.norm(b - a) >= min_len:
            return a, b


def _triangle(rng):
    """Triangle with all angles >= 10 degrees and area >= 1e-3 in the unit cube."""
    while True:
        P = rng.uniform(0.0, 1.0, (3, 3))
        area = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
        if area < 1e-3:
            continue
        ok = True
        for i in range(3):
            u, v = P[(i + 1) % 3] - P[i], P[(i + 2) % 3] - P[i]
            cosang = np.dot(u, v) / (np.linalg.norm(u) * np.linalg.norm(v))
            if cosang > math.cos(math.radians(10.0)):
                ok = False
        if ok:
            return P


def _parallel_angle(rng):
    return 10.0 ** rng.uniform(-7.0, -2.0)


def make_stencil(kind, rng, dhat):
    """Vertices (s x 3, slot order) of one stencil of the given kind with a target distance."""
    d = _distance(rng, dhat)
    if kind == "PT":
        T = _triangle(rng)
        while True:
            beta = rng.dirichlet((1.0, 1.0, 1.0))
            if beta.min() >= 0.05:
                break
        foot = beta @ T
        n = np.cross(T[1] - T[0], T[2] - T[0])
        n /= np.linalg.norm(n)
        p = foot + rng.choice((-1.0, 1.0)) * d * n
        return np.stack([p, T[0], T[1], T[2]])
    if kind in ("EE", "EE_PAR"):
        a0, a1 = _segment(rng)
        e1 = (a1 - a0) / np.linalg.norm(a1 - a0)
        p1 = a0 + rng.uniform(0.1, 0.9) * (a1 - a0)
        nrm = _perp(rng, e1)
        m = np.cross(e1, nrm)
        th = _parallel_angle(rng) if kind == "EE_PAR" else rng.uniform(0.05, math.pi / 2)
        e2 = math.cos(th) * e1 + math.sin(th) * m
        p2 = p1 + rng.choice((-1.0, 1.0)) * d * nrm
        L2 = rng.uniform(0.1, 0.8)
        g2 = rng.uniform(0.1, 0.9)
        b0 = p2 - g2 * L2 * e2
        return np.stack([a0, a1, b0, b0 + L2 * e2])
    if kind in ("PE", "PE_PAR"):
        e0, e1p = _segment(rng)
        ed = (e1p - e0) / np.linalg.norm(e1p - e0)
        foot = e0 + rng.uniform(0.1, 0.9) * (e1p - e0)
        nrm = _perp(rng, ed)
        p = foot + d * nrm
        if kind == "PE":
            return np.stack([p, e0, e1p])
        th = _parallel_angle(rng)
        L1 = rng.uniform(0.1, 0.8)
        direction = math.cos(th) * rng.choice((-1.0, 1.0)) * ed + math.sin(th) * nrm
        return np.stack([p, p + L1 * direction, e0, e1p])
    if kind in ("PP", "PP_PAR"):
        p = rng.uniform(0.0, 1.0, 3)
        a = _unit(rng)
        q = p + d * a
        if kind == "PP":
            return np.stack([p, q])
        th = _parallel_angle(rng)
        m = _perp(rng, a)
        L1, L2 = rng.uniform(0.1, 0.8), rng.uniform(0.1, 0.8)
        return np.stack([p, p - L1 * a, q, q + L2 * (math.cos(th) * a + math.sin(th) * m)])
    raise ValueError(kind)


def encode(kind, ids):
    """Sign-encoded tuple for vertex ids in slot order (Sec. 7.2)."""
    neg = lambda i: -(int(i) + 1)
    if kind == "PT":
        return (neg(ids[0]), ids[1], ids[2], ids[3])
    if kind == "EE":
        return (ids[0], ids[1], ids[2], ids[3])
    if kind == "PE":
        return (neg(ids[0]), ids[1], ids[2], NULL)
    if kind == "PP":
        return (neg(ids[0]), ids[1], NULL, NULL)
    if kind == "EE_PAR":
        return (ids[0], neg(ids[1]), ids[2], ids[3])
    if kind == "PE_PAR":
        return (neg(ids[0]), neg(ids[1]), ids[2], neg(ids[3]))
    if kind == "PP_PAR":
        return (neg(ids[0]), neg(ids[1]), neg(ids[2]), neg(ids[3]))
    raise ValueError(kind)


def type_counts(k, mix=DEFAULT_MIX):
    counts = [int(round(k * f)) for _, f in mix]
    counts[0] += k - sum(counts)
    return [(kind, c) for (kind, _), c in zip(mix, counts)]


def unit_stencils(k=10000, seed=20230809, mix=DEFAULT_MIX, dhat=UNIT_DHAT, shuffle=False):
    """Random stencil set in which every stencil owns its vertices.

    Returns dict(x=(3, n) float64 SoA positions, stencils=(4, k) int32, dhat, kinds=list).
    Stencils come grouped by kind in the order of ``mix`` unless ``shuffle``.
    """
    rng = np.random.default_rng(seed)
    verts, tuples, kinds = [], [], []
    nv = 0
    for kind, cnt in type_counts(k, mix):
        for _ in range(cnt):
            P = make_stencil(kind, rng, dhat)
            ids = list(range(nv, nv + len(P)))
            nv += len(P)
            verts.append(P)
            tuples.append(encode(kind, ids))
            kinds.append(kind)
    x = np.ascontiguousarray(np.concatenate(verts).T)
    st = np.array(tuples, dtype=np.int64).T.astype(np.int32)
    if shuffle:
        perm = rng.permutation(k)
        st = np.ascontiguousarray(st[:, perm])
        kinds = [kinds[i] for i in perm]
    return {"x": x, "stencils": np.ascontiguousarray(st), "dhat": dhat, "kinds": kinds}


# ----------------------------------------------------------------------------- vectorised batch
def _v_unit(rng, m):
    v = rng.normal(size=(m, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _v_perp(rng, u):
    w = np.cross(u, _v_unit(rng, len(u)))
    return w / np.linalg.norm(w, axis=1, keepdims=True)


def _v_distance(rng, m, dhat):
    r = 10.0 ** rng.uniform(-4.0, 0.0, m)
    bad = (np.abs(r - 0.1) <= 1e-9) | (r >= 1.0 - 1e-9)
    r[bad] = 0.5
    return dhat * r


def _v_segments(rng, m, min_len=0.1):
    a, b = rng.uniform(0, 1, (m, 3)), rng.uniform(0, 1, (m, 3))
    short = np.linalg.norm(b - a, axis=1) < min_len
    while short.any():
        a[short], b[short] = rng.uniform(0, 1, (short.sum(), 3)), rng.uniform(0, 1, (short.sum(), 3))
        short = np.linalg.norm(b - a, axis=1) < min_len
    return a, b


def _v_triangles(rng, m):
    out = np.empty((m, 3, 3))
    filled = 0
    cmin = math.cos(math.radians(10.0))
    while filled < m:
        P = rng.uniform(0, 1, (2 * (m - filled) + 16, 3, 3))
        area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
        ok = area >= 1e-3
        for i in range(3):
            u, v = P[:, (i + 1) % 3] - P[:, i], P[:, (i + 2) % 3] - P[:, i]
            cosang = (u * v).sum(1) / (np.linalg.norm(u, axis=1) * np.linalg.norm(v, axis=1))
            ok &= cosang <= cmin
        P = P[ok][: m - filled]
        out[filled:filled + len(P)] = P
        filled += len(P)
    return out


def _v_bary(rng, m):
    out = np.empty((m, 3))
    filled = 0
    while filled < m:
        b = rng.dirichlet((1.0, 1.0, 1.0), 2 * (m - filled) + 16)
        b = b[b.min(1) >= 0.05][: m - filled]
        out[filled:filled + len(b)] = b
        filled += len(b)
    return out


def _v_make(kind, rng, m, dhat):
    """Vertices (m, s, 3) of m stencils of one kind (same recipe as ``make_stencil``)."""
    d = _v_distance(rng, m, dhat)[:, None]
    sign = rng.choice((-1.0, 1.0), (m, 1))
    if kind == "PT":
        T = _v_triangles(rng, m)
        foot = np.einsum("mi,mij->mj", _v_bary(rng, m), T)
        n = np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0])
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        return np.stack([foot + sign * d * n, T[:, 0], T[:, 1], T[:, 2]], 1)
    if kind in ("EE", "EE_PAR"):
        a0, a1 = _v_segments(rng, m)
        e1 = (a1 - a0) / np.linalg.norm(a1 - a0, axis=1, keepdims=True)
        p1 = a0 + rng.uniform(0.1, 0.9, (m, 1)) * (a1 - a0)
        nrm = _v_perp(rng, e1)
        mm = np.cross(e1, nrm)
        th = (10.0 ** rng.uniform(-7, -2, (m, 1))) if kind == "EE_PAR" else rng.uniform(0.05, math.pi / 2, (m, 1))
        e2 = np.cos(th) * e1 + np.sin(th) * mm
        p2 = p1 + sign * d * nrm
        L2 = rng.uniform(0.1, 0.8, (m, 1))
        b0 = p2 - rng.uniform(0.1, 0.9, (m, 1)) * L2 * e2
        return np.stack([a0, a1, b0, b0 + L2 * e2], 1)
    if kind in ("PE", "PE_PAR"):
        e0, e1 = _v_segments(rng, m)
        ed = (e1 - e0) / np.linalg.norm(e1 - e0, axis=1, keepdims=True)
        nrm = _v_perp(rng, ed)
        p = e0 + rng.uniform(0.1, 0.9, (m, 1)) * (e1 - e0) + d * nrm
        if kind == "PE":
            return np.stack([p, e0, e1], 1)
        th = 10.0 ** rng.uniform(-7, -2, (m, 1))
        L1 = rng.uniform(0.1, 0.8, (m, 1))
        direction = np.cos(th) * sign * ed + np.sin(th) * nrm
        return np.stack([p, p + L1 * direction, e0, e1], 1)
    if kind in ("PP", "PP_PAR"):
        p = rng.uniform(0, 1, (m, 3))
        a = _v_unit(rng, m)
        q = p + d * a
        if kind == "PP":
            return np.stack([p, q], 1)
        th = 10.0 ** rng.uniform(-7, -2, (m, 1))
        mm = _v_perp(rng, a)
        L1, L2 = rng.uniform(0.1, 0.8, (m, 1)), rng.uniform(0.1, 0.8, (m, 1))
        return np.stack([p, p - L1 * a, q, q + L2 * (np.cos(th) * a + np.sin(th) * mm)], 1)
    raise ValueError(kind)


def _v_encode(kind, ids):
    """Sign-encoded tuples (4, m) for vertex ids (m, s) in slot order."""
    m = ids.shape[0]
    t = np.full((4, m), NULL, dtype=np.int64)
    neg = lambda a: -(a + 1)
    if kind == "PT":
        t[0], t[1], t[2], t[3] = neg(ids[:, 0]), ids[:, 1], ids[:, 2], ids[:, 3]
    elif kind == "EE":
        t[:] = ids.T
    elif kind == "PE":
        t[0], t[1], t[2] = neg(ids[:, 0]), ids[:, 1], ids[:, 2]
    elif kind == "PP":
        t[0], t[1] = neg(ids[:, 0]), ids[:, 1]
    elif kind == "EE_PAR":
        t[0], t[1], t[2], t[3] = ids[:, 0], neg(ids[:, 1]), ids[:, 2], ids[:, 3]
    elif kind == "PE_PAR":
        t[0], t[1], t[2], t[3] = neg(ids[:, 0]), neg(ids[:, 1]), ids[:, 2], neg(ids[:, 3])
    elif kind == "PP_PAR":
        t[:] = neg(ids.T)
    return t


def batch_stencils(k, seed=20230810, mix=DEFAULT_MIX, dhat=UNIT_DHAT):
    """Vectorised generator of the same recipe as ``unit_stencils`` for large k (own vertices)."""
    rng = np.random.default_rng(seed)
    xs, ts, kinds = [], [], []
    nv = 0
    for kind, cnt in type_counts(k, mix):
        if cnt == 0:
            continue
        P = _v_make(kind, rng, cnt, dhat)
        s = P.shape[1]
        ids = nv + np.arange(cnt * s, dtype=np.int64).reshape(cnt, s)
        nv += cnt * s
        xs.append(P.reshape(-1, 3))
        ts.append(_v_encode(kind, ids))
        kinds.append((kind, cnt))
    x = np.ascontiguousarray(np.concatenate(xs).T)
    st = np.ascontiguousarray(np.concatenate(ts, axis=1).astype(np.int32))
    return {"x": x, "stencils": st, "dhat": dhat, "kind_counts": kinds}


# ----------------------------------------------------------------------------- two-sheet index space
def sheet_index_space(k, seed=20230811, side=388, radius=0, mix=DEFAULT_MIX, ordered=True, return_ids=False):
    """Stencil tuples over two triangulated side x side vertex grids (ids [0, 2 side^2)).

    Each stencil couples a primitive of one sheet with a primitive of the other
    within ``radius`` cells of the same grid cell (a point, a grid edge or a grid
    triangle as its type needs), so the index pattern is that of two sheets in
    contact.  Used for assembly and SpMV workloads; the block values come from
    the own-vertex geometry of ``batch_stencils`` with the same type counts.
    With ``ordered`` the stencils of each type follow their cells in row-major
    order, the order in which a broad phase that walks the primitives emits them;
    otherwise they are in random order.
    Returns (4, k) int32 tuples (same type order as ``type_counts``) and n; with ``return_ids``
    also the plain vertex ids of every stencil in slot order, a list of (count, s) int64 arrays
    in the same order (the tuples before sign encoding).
    """
    rng = np.random.default_rng(seed)
    N = side
    n = 2 * N * N

    def vid(sheet, i, j):
        return sheet * N * N + i * N + j

    def cells(m):
        return rng.integers(0, N - 1, m), rng.integers(0, N - 1, m)

    def partner(i, j):
        pi = np.clip(i + rng.integers(-radius, radius + 1, len(i)), 0, N - 2)
        pj = np.clip(j + rng.integers(-radius, radius + 1, len(j)), 0, N - 2)
        return pi, pj

    def point(sheet, i, j):
        di, dj = rng.integers(0, 2, len(i)), rng.integers(0, 2, len(i))
        return vid(sheet, i + di, j + dj)[:, None]

    def edge(sheet, i, j):
        kind = rng.integers(0, 3, len(i))
        a = vid(sheet, i, j)
        b = np.where(kind == 0, vid(sheet, i + 1, j), np.where(kind == 1, vid(sheet, i, j + 1),
                                                                 vid(sheet, i + 1, j + 1)))
        return np.stack([a, b], 1)

    def tri(sheet, i, j):
        up = rng.integers(0, 2, len(i)).astype(bool)
        a = vid(sheet, i, j)
        b = np.where(up, vid(sheet, i + 1, j), vid(sheet, i + 1, j + 1))
        c = np.where(up, vid(sheet, i + 1, j + 1), vid(sheet, i, j + 1))
        return np.stack([a, b, c], 1)

    ts, raw = [], []
    for kind, cnt in type_counts(k, mix):
        if cnt == 0:
            continue
        i, j = cells(cnt)
        if ordered:
            o = np.lexsort((j, i))
            i, j = i[o], j[o]
        pi, pj = partner(i, j)
        sa = rng.integers(0, 2, cnt)
        sb = 1 - sa
        if kind == "PT":
            ids = np.concatenate([point(sa, i, j), tri(sb, pi, pj)], 1)
        elif kind == "PE":
            ids = np.concatenate([point(sa, i, j), edge(sb, pi, pj)], 1)
        elif kind == "PP":
            ids = np.concatenate([point(sa, i, j), point(sb, pi, pj)], 1)
        else:  # EE-derived: two edges
            ids = np.concatenate([edge(sa, i, j), edge(sb, pi, pj)], 1)
        ts.append(_v_encode(kind, ids.astype(np.int64)))
        raw.append(ids.astype(np.int64))
    st = np.ascontiguousarray(np.concatenate(ts, axis=1).astype(np.int32))
    return (st, n, raw) if return_ids else (st, n)


def sheet_mass(side=388, density=1000.0):
    """Lumped vertex masses of the two sheets: density x (spacing^3) per vertex (unit-square sheets
    of thickness one grid spacing)."""
    h = 1.0 / (side - 1)
    return np.full(2 * side * side, density * h ** 3)


# ----------------------------------------------------------------------------- assembly inputs
def random_elements(n, k, T, seed=7, mix=DEFAULT_MIX, hub=None, hub_count=0):
    """Random element lists over vertex ids [0, n) with random local blocks (assembly tests).

    Stencils follow ``mix`` with distinct vertices per stencil; tetrahedra are 4 distinct
    ids.  ``hub``: optionally force ``hub_count`` PT stencils to use vertex ``hub`` as their
    point (long rows).  Returns dict of numpy arrays: stencils (4,k) i32, tets (4,T) i32,
    dense stencil blocks hess (144,k), rank-one lam (k), w (12,k), grad (12,k), tet_hess
    (144,T), tet_grad (12,T), mass (n), grad_base (3,n).
    """
    rng = np.random.default_rng(seed)
    ts = []
    for kind, cnt in type_counts(k, mix):
        if cnt == 0:
            continue
        s = {"PT": 4, "EE": 4, "PE": 3, "PP": 2}.get(kind, 4)
        ids = np.argsort(rng.random((cnt, n)), axis=1)[:, :s] if n <= 64 else \
            np.stack([rng.choice(n, s, replace=False) for _ in range(cnt)])
        if kind == "PT" and hub is not None:
            m = min(hub_count, cnt)
            for r in range(m):
                row = [v for v in ids[r] if v != hub][:3]
                while len(row) < 3:
                    c = int(rng.integers(0, n))
                    if c != hub and c not in row:
                        row.append(c)
                ids[r] = [hub] + row
        ts.append(_v_encode(kind, ids.astype(np.int64)))
    st = np.ascontiguousarray(np.concatenate(ts, axis=1).astype(np.int32)) if ts else np.zeros((4, 0), np.int32)
    tets = np.stack([rng.choice(n, 4, replace=False) for _ in range(T)], 1).astype(np.int32) if T else \
        np.zeros((4, 0), np.int32)
    return {
        "stencils": st, "tets": np.ascontiguousarray(tets),
        "hess": rng.normal(size=(144, k)), "lam": rng.uniform(0.1, 2.0, k), "w": rng.normal(size=(12, k)),
        "grad": rng.normal(size=(12, k)), "tet_hess": rng.normal(size=(144, T)),
        "tet_grad": rng.normal(size=(12, T)), "mass": rng.uniform(0.5, 1.5, n),
        "grad_base": rng.normal(size=(3, n)),
    }


# ----------------------------------------------------------------------------- tetrahedral meshes
_KUHN = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def tet_box(nx, ny, nz, spacing=1.0, origin=(0.0, 0.0, 0.0)):
    """Vertex grid nx x ny x nz split into 6 tetrahedra per cell (Freudenthal/Kuhn split along
    the cell diagonal), every tetrahedron positively oriented.

    Returns (x (3, n) float64, tets (4, T) int32); vertex (i, j, k) has id (i*ny + j)*nz + k."""
    I, Jg, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    x = np.stack([I.ravel() * spacing + origin[0], Jg.ravel() * spacing + origin[1],
                  K.ravel() * spacing + origin[2]]).astype(np.float64)
    vid = lambda i, j, k: (i * ny + j) * nz + k
    ci, cj, ck = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), np.arange(nz - 1), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    tets = []
    for perm in _KUHN:
        p = [np.array([ci, cj, ck])]
        cur = p[0].copy()
        for ax in perm:
            cur = cur.copy()
            cur[ax] += 1
            p.append(cur)
        v = [vid(q[0], q[1], q[2]) for q in p]
        odd = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b]) % 2
        if odd:
            v[1], v[2] = v[2], v[1]
        tets.append(np.stack(v))
    T = np.concatenate(tets, axis=1).astype(np.int32)
    # make every element positively oriented
    P = [x[:, T[a]] for a in range(4)]
    det = np.einsum("ij,ij->j", P[1] - P[0], np.cross((P[2] - P[0]).T, (P[3] - P[0]).T).T)
    flip = det < 0
    T[1, flip], T[2, flip] = T[2, flip].copy(), T[1, flip].copy()
    return x, np.ascontiguousarray(T)


def deform(x, seed, amplitude=0.05, jitter=0.01):
    """Smooth random deformation plus jitter (for elasticity tests); same shape as x."""
    rng = np.random.default_rng(seed)
    A = np.eye(3) + amplitude * rng.normal(size=(3, 3))
    k = rng.normal(size=(3, 3)) * 2.0
    y = A @ x + amplitude * np.sin(k @ x) + jitter * rng.normal(size=x.shape) * (np.ptp(x) / 50 + 1e-12)
    return np.ascontiguousarray(y)


# ----------------------------------------------------------------------------- scenes
def surface_lists(x, tets):
    """Boundary of a tetrahedral mesh: triangles (3, m) oriented outward, edges (2, e) with a < b,
    and boundary vertices (v,); all int32, sorted canonically (triangles by their sorted vertex
    triple, edges lexicographically, vertices ascending)."""
    T = tets.shape[1]
    tt = tets.T.astype(np.int64)
    opp_idx = [(1, 2, 3, 0), (0, 2, 3, 1), (0, 1, 3, 2), (0, 1, 2, 3)]   # face vertices + opposite
    F = np.concatenate([tt[:, list(o[:3])] for o in opp_idx])             # (4T, 3)
    O = np.concatenate([tt[:, o[3]] for o in opp_idx])                    # opposite vertex
    key = np.sort(F, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    b = cnt[inv.ravel()] == 1
    F, O, key = F[b], O[b], key[b]
    nrm = np.cross(x[:, F[:, 1]].T - x[:, F[:, 0]].T, x[:, F[:, 2]].T - x[:, F[:, 0]].T)
    inward = np.einsum("ij,ij->i", nrm, x[:, O].T - x[:, F[:, 0]].T) > 0
    F[inward, 1], F[inward, 2] = F[inward, 2].copy(), F[inward, 1].copy()
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0]))
    tris = F[order].T
    E = np.concatenate([tris[[0, 1]], tris[[1, 2]], tris[[2, 0]]], axis=1)
    E = np.unique(np.sort(E, axis=0), axis=1)
    verts = np.unique(tris.ravel())
    return (np.ascontiguousarray(tris.astype(np.int32)), np.ascontiguousarray(E.astype(np.int32)),
            np.ascontiguousarray(verts.astype(np.int32)))


def _merge(parts):
    xs, ts, off = [], [], 0
    for x, t in parts:
        xs.append(x)
        ts.append(t + off)
        off += x.shape[1]
    return np.ascontiguousarray(np.concatenate(xs, axis=1)), np.ascontiguousarray(np.concatenate(ts, axis=1).astype(np.int32))


def two_cubes(gap=0.5, velocity=-2.0, m=5):
    """Two unit cubes of m x m x m vertices each (m = 5: 125 verts, 384 tets); the top one `gap`
    above the bottom one moving at `velocity` in z; the bottom face z = 0 is fixed.
    Returns dict(x, v, tets, fixed, tris, edges, verts, l)."""
    xa, ta = tet_box(m, m, m, spacing=1.0 / (m - 1))
    xb, tb = tet_box(m, m, m, spacing=1.0 / (m - 1), origin=(0.0, 0.0, 1.0 + gap))
    x, tets = _merge([(xa, ta), (xb, tb)])
    n = x.shape[1]
    na = xa.shape[1]
    v = np.zeros((3, n))
    v[2, na:] = velocity
    fixed = np.zeros(n, np.uint8)
    fixed[:na][xa[2] == 0.0] = 1
    tris, edges, verts = surface_lists(x, tets)
    l = float(np.linalg.norm(x.max(axis=1) - x.min(axis=1)))
    return {"x": x, "v": v, "tets": tets, "fixed": fixed, "tris": tris, "edges": edges, "verts": verts, "l": l}


def ball(radius=0.1, cells=14, center=(0.0, 0.0, 0.0)):
    """Voxel ball: the Freudenthal grid of the bounding cube with `cells` cells per side, keeping
    the tetrahedra whose centroid lies inside the sphere; unused vertices dropped."""
    h = 2.0 * radius / cells
    x, t = tet_box(cells + 1, cells + 1, cells + 1, spacing=h, origin=tuple(c - radius for c in center))
    cen = (x[:, t[0]] + x[:, t[1]] + x[:, t[2]] + x[:, t[3]]) / 4.0
    keep = np.linalg.norm(cen - np.asarray(center)[:, None], axis=0) <= radius
    t = t[:, keep]
    used = np.unique(t)
    remap = -np.ones(x.shape[1], np.int64)
    remap[used] = np.arange(len(used))
    return np.ascontiguousarray(x[:, used]), np.ascontiguousarray(remap[t].astype(np.int32))


def sphere_grid(nx=8, ny=8, radius=0.1, cells=14, gap=1e-3, floor_cells=64, jitter=0.25, seed=20230812):
    """nx x ny balls of `radius` on a floor (top face z = 0), neighbours and floor `gap` apart.
    Each ball centre is moved by a seeded offset uniform in [-jitter*gap/2, jitter*gap/2]^3 (z only
    upward), so the lattice has no exact symmetry.  The floor is a fixed thin tetrahedral slab of
    floor_cells x floor_cells x 1 grid cells, so every primitive comes from a tetrahedral mesh and
    no floor vertex is shared by a large share of the contacts.  Returns the same dict as
    two_cubes."""
    parts = []
    pitch = 2 * radius + gap
    rng = np.random.default_rng(seed)
    for i in range(nx):
        for j in range(ny):
            o = 0.5 * jitter * gap * rng.uniform(-1.0, 1.0, 3)
            o[2] = abs(o[2])
            parts.append(ball(radius, cells, center=(i * pitch + o[0], j * pitch + o[1], radius + gap + o[2])))
    lo, hi = -radius - 0.05, (max(nx, ny) - 1) * pitch + radius + 0.05
    slab_x, slab_t = tet_box(floor_cells + 1, floor_cells + 1, 2, spacing=1.0)
    slab_x = slab_x.copy()
    slab_x[0] = lo + slab_x[0] / floor_cells * (hi - lo)
    slab_x[1] = lo + slab_x[1] / floor_cells * (hi - lo)
    slab_x[2] = -0.05 + slab_x[2] * 0.05
    parts.append((slab_x, slab_t))
    x, tets = _merge(parts)
    n = x.shape[1]
    fixed = np.zeros(n, np.uint8)
    fixed[n - slab_x.shape[1]:] = 1
    tris, edges, verts = surface_lists(x, tets)
    l = float(np.linalg.norm(x.max(axis=1) - x.min(axis=1)))
    return {"x": x, "v": np.zeros((3, n)), "tets": tets, "fixed": fixed, "tris": tris, "edges": edges,
            "verts": verts, "l": l}


def beam_on_plate(beam=(41, 11, 11), plate=(65, 65, 4), beam_cell=0.025, plate_side=2.0, turn=0.3,
                  gap_frac=0.5, velocity=(0.05, 0.0, -0.1), dhat_rel=1e-3):
    """A tet-meshed beam (vertex grid `beam`, cell `beam_cell`: 41 x 11 x 11 is 1.0 x 0.25 x 0.25)
    turned by `turn` rad about z and lying `gap_frac` dhat above a tet-meshed plate (vertex grid
    `plate` over a square of side `plate_side`, same cell height as width) whose bottom layer is
    fixed; dhat = dhat_rel l (l the bounding-box diagonal).  The turn keeps the two grids out of
    alignment.  The beam moves at `velocity`.  Returns the same dict as two_cubes plus "dhat"."""
    px, pt = tet_box(*plate, spacing=1.0)
    px = px.copy()
    hp = plate_side / (plate[0] - 1)
    px[0] = -plate_side / 2 + px[0] * hp
    px[1] = -plate_side / 2 + px[1] * (plate_side / (plate[1] - 1))
    px[2] = -(plate[2] - 1) * hp + px[2] * hp
    bx, bt = tet_box(*beam, spacing=beam_cell)
    bx = bx.copy()
    bx -= ((np.array(beam) - 1) * beam_cell / 2.0)[:, None]
    c, s_ = np.cos(turn), np.sin(turn)
    bx[0], bx[1] = c * bx[0] - s_ * bx[1], s_ * bx[0] + c * bx[1]
    bx[2] -= bx[2].min()
    lo = np.minimum(px.min(axis=1), bx.min(axis=1))
    hi = np.maximum(px.max(axis=1), bx.max(axis=1))
    dhat = dhat_rel * float(np.linalg.norm(hi - lo))
    bx[2] += gap_frac * dhat
    x, tets = _merge([(bx, bt), (px, pt)])
    n, nb = x.shape[1], bx.shape[1]
    v = np.zeros((3, n))
    v[:, :nb] = np.asarray(velocity, float)[:, None]
    fixed = np.zeros(n, np.uint8)
    fixed[nb:][px[2] <= px[2].min() + 1e-12] = 1
    tris, edges, verts = surface_lists(x, tets)
    l = float(np.linalg.norm(x.max(axis=1) - x.min(axis=1)))
    return {"x": x, "v": v, "tets": tets, "fixed": fixed, "tris": tris, "edges": edges, "verts": verts, "l": l,
            "dhat": dhat_rel * l}


def stack_scene(rng, n_bodies, target_verts, dhat, size=0.2):
    """One scene of `n_bodies` tet-meshed cubes or balls (about target_verts vertices in all)
    stacked along z, each gap uniform in [0, 2 dhat] (below dhat the bodies start in contact),
    with small seeded lateral offsets and turns; the lowest layer of the bottom body is fixed."""
    per = max(target_verts / n_bodies, 27.0)
    parts, z = [], 0.0
    for b in range(n_bodies):
        if rng.random() < 0.5:
            m = max(3, int(round(per ** (1.0 / 3.0))))
            xb, tb = tet_box(m, m, m, spacing=size / (m - 1))
        else:
            cells = max(4, int(round((per / 0.52) ** (1.0 / 3.0))) - 1)
            xb, tb = ball(size / 2, cells, center=(size / 2, size / 2, size / 2))
        xb = xb.copy()
        th = rng.uniform(-0.3, 0.3)
        c, s_ = np.cos(th), np.sin(th)
        cx = xb[0] - size / 2
        cy = xb[1] - size / 2
        xb[0] = c * cx - s_ * cy + size / 2 + rng.uniform(-0.2, 0.2) * size
        xb[1] = s_ * cx + c * cy + size / 2 + rng.uniform(-0.2, 0.2) * size
        xb[2] = xb[2] - xb[2].min() + z
        parts.append((xb, tb))
        z = xb[2].max() + rng.uniform(0.0, 2.0) * dhat
    x, tets = _merge(parts)
    n = x.shape[1]
    fixed = np.zeros(n, np.uint8)
    n0 = parts[0][0].shape[1]
    fixed[:n0][parts[0][0][2] <= parts[0][0][2].min() + 1e-12] = 1
    tris, edges, verts = surface_lists(x, tets)
    l = float(np.linalg.norm(x.max(axis=1) - x.min(axis=1)))
    return {"x": x, "v": np.zeros((3, n)), "tets": tets, "fixed": fixed, "tris": tris, "edges": edges,
            "verts": verts, "l": l}


def batch_scenes(n_scenes=256, seed=20230813, vmin=200, vmax=5000, dhat=5e-4):
    """Independent scenes of 2 to 6 stacked cubes / balls each, vertex counts log-uniform in
    [vmin, vmax] per scene; one dhat for the batch.  Returns (list of scene dicts, dhat)."""
    rng = np.random.default_rng(seed)
    scenes = []
    for _ in range(n_scenes):
        nb = int(rng.integers(2, 7))
        tv = float(np.exp(rng.uniform(np.log(vmin), np.log(vmax))))
        scenes.append(stack_scene(rng, nb, tv, dhat))
    return scenes, dhat
