"""Global Hessian and gradient assembly into 3x3-block BSR (oracle; test infrastructure only).

The Newton system of Alg. 1 uses H = M + sum_e P_e^T H_e P_e, the mass matrix
plus every element's projected local Hessian scattered by its local-to-global
vertex map (supplement Sec. S6, the decomposition of the system matrix into
local matrices), and g = g_0 + sum_e P_e^T g_e.  This module builds that sum
plainly:

* pattern: every ordered vertex pair (v_a, v_b) of every element, plus the
  diagonal (i, i) of every vertex with mass, as a set; rows sorted, columns
  sorted within a row;
* values: for each 3x3 block, start from zero, add the mass m_i I_3 on the
  diagonal first, then the (a, b) sub-blocks of the contributing elements in
  ascending global element id (tetrahedra first, then stencils);
* gradient: g_0 (if given) plus each element's slot-a gradient, again in
  ascending element id.

Element local blocks use the library's entry-major layout: entry (p, q) of the
3s x 3s block of element e at hess[p*3s + q, e]; rank-one stencil blocks are
lam[e] * w[:, e] w[:, e]^T.
"""
import numpy as np

from . import geometry as geo


def element_vertices(stencils=None, tets=None):
    """List of (global element id, vertex ids in slot order); tets first, then stencils."""
    out = []
    if tets is not None:
        for e in range(tets.shape[1]):
            out.append(tuple(int(v) for v in tets[:, e]))
    if stencils is not None:
        for e in range(stencils.shape[1]):
            out.append(geo.decode(stencils[:, e])[1])
    return out


def _local_block(kind, data, e_local, s, a, b):
    n3 = 3 * s
    if kind == "dense":
        H = data["hess"]
        return np.array([[H[(3 * a + i) * n3 + 3 * b + j, e_local] for j in range(3)] for i in range(3)],
                        dtype=np.float64)
    lam, w = data["lam"], data["w"]
    wa = w[3 * a:3 * a + 3, e_local].astype(np.float64)
    wb = w[3 * b:3 * b + 3, e_local].astype(np.float64)
    return float(lam[e_local]) * np.outer(wa, wb)


def assemble(n, stencils=None, stencil_data=None, tets=None, tet_data=None, mass=None, grad_base=None,
             rows=None):
    """Plain assembly.

    ``stencil_data`` / ``tet_data``: dict(kind='dense'|'rank1', hess=..., lam=..., w=..., grad=...).
    ``rows``: optional iterable of block rows to assemble (others are skipped) for sampled checks.
    Returns dict(rowptr, colidx, vals (nnzb, 3, 3), grad (3, n)) -- over the requested rows only
    when ``rows`` is given (rowptr then indexes those rows in the given order).
    """
    T = 0 if tets is None else tets.shape[1]
    elems = element_vertices(stencils, tets)
    want = None if rows is None else set(int(r) for r in rows)
    blocks = {}   # (r, c) -> list of (order key, contribution 3x3)
    gparts = {}   # r -> list of (order key, 3-vector)

    def add(r, c, key, val):
        blocks.setdefault((r, c), []).append((key, val))

    if mass is not None:
        for i in range(n):
            if want is None or i in want:
                add(i, i, -1, float(mass[i]) * np.eye(3))
    for eid, verts in enumerate(elems):
        if eid < T:
            data, el = tet_data, eid
        else:
            data, el = stencil_data, eid - T
        s = len(verts)
        for a in range(s):
            r = verts[a]
            if want is not None and r not in want:
                continue
            if data.get("grad") is not None:
                gparts.setdefault(r, []).append((eid, np.array(data["grad"][3 * a:3 * a + 3, el], dtype=np.float64)))
            for b in range(s):
                add(r, verts[b], eid, _local_block(data["kind"], data, el, s, a, b))

    row_list = sorted(want) if want is not None else range(n)
    by_row = {}
    for (r, c) in blocks:
        by_row.setdefault(r, []).append(c)
    rowptr = [0]
    colidx, vals = [], []
    for r in row_list:
        for c in sorted(by_row.get(r, [])):
            acc = np.zeros((3, 3))
            for _, v in sorted(blocks[(r, c)], key=lambda t: t[0]):
                acc = acc + v
            colidx.append(c)
            vals.append(acc)
        rowptr.append(len(colidx))
    grad = np.zeros((3, n))
    for r in row_list:
        acc = np.zeros(3) if grad_base is None else np.array(grad_base[:, r], dtype=np.float64)
        for _, v in sorted(gparts.get(r, []), key=lambda t: t[0]):
            acc = acc + v
        grad[:, r] = acc
    return {"rowptr": np.array(rowptr, dtype=np.int64), "colidx": np.array(colidx, dtype=np.int64),
            "vals": np.array(vals, dtype=np.float64).reshape(-1, 3, 3), "grad": grad,
            "rows": np.array(list(row_list), dtype=np.int64)}


def to_dense(n, A):
    """Dense 3n x 3n matrix of a full BSR assembly (for brute-force checks on tiny n)."""
    H = np.zeros((3 * n, 3 * n))
    for r in range(n):
        for p in range(A["rowptr"][r], A["rowptr"][r + 1]):
            c = A["colidx"][p]
            H[3 * r:3 * r + 3, 3 * c:3 * c + 3] = A["vals"][p]
    return H


def bsr_matvec(A, p):
    """y = H p for a full BSR (p, y as (3, n))."""
    n = len(A["rowptr"]) - 1
    y = np.zeros((3, n))
    for r in range(n):
        acc = np.zeros(3)
        for q in range(A["rowptr"][r], A["rowptr"][r + 1]):
            acc = acc + A["vals"][q] @ p[:, A["colidx"][q]]
        y[:, r] = acc
    return y
