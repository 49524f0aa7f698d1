"""Per-stencil barrier energy, gradient and PSD-projected Hessian (oracle; test infrastructure only).

The steps follow the paper in its own order and notation (Alg. 2 per pair):

1. Gather the stencil's vertices (``getLocalContactVertices``) and measure the
   gap function g = f^2, f = d/dhat (Eq. 7-11) exactly (``oracle.geometry``).
2. Build the diagonal constraint Jacobian J (Eq. 10; Eq. 28 for the
   nearly-parallel edge-edge family) and the selecting normals.
3. Non-mollified types (PT, EE, PE, PP):
   * barrier b(g) of Eq. 24, gradient dB/dx = dJ/dx : (b_g dg/dJ), dg/dJ = 2JN  (Eq. 13-14);
   * eigenpair lambda_1 = 4 g b_gg + 2 b_g, Q_1 = J N / sqrt(g)                (Eq. 18, 21);
   * filter: lambda_1 -> lambda_1(eps_g) when g < eps_g                        (Eq. 23);
   * d2b/dJ2 ~= lambda_1 Q_1 (x) Q_1, mapped by dJ/dx, second term of Eq. 15 dropped.
4. Mollified types (EE, PE, PP nearly parallel), btilde = e(gamma) b(g) (Eq. 25-29):
   * lambda_(*)1 = 2(btilde_* + 2 (*) btilde_**), lambda_(*)2,3 = 2 btilde_*     (Sec. 6.2);
   * t = btilde_gamma,g sqrt(c) f                                               (Eq. 33);
   * the auxiliary 2x2 eigenproblem on [[lambda_gamma1, 4t], [4t, lambda_g1]]
     (supplement Sec. S4, aux matrix M) gives lambda_7' <= lambda_8' and Q_8';
   * d2btilde/dJ2 ~= lambda_g2 Q_g2 (x) Q_g2 + lambda_g3 Q_g3 (x) Q_g3 + lambda_8' Q_8' (x) Q_8' (Eq. 36).
   Reading: the filter of Eq. 23 is applied to lambda_g1 (its lambda_1(g) factor) before M is formed.
5. Energy kappa*b, gradient kappa*db/dx, Hessian kappa*(dJ/dx)^T (d2b/dJ2) (dJ/dx).

Every Hessian here has rank one in x-space, H = lam * w w^T; ``lam``/``w`` are
returned too, with the sign of w fixed so that the coefficient of the g-normal
(the (3,3) entry of the kept eigenmatrix; (m,m) for the plain types) is >= 0.
"""
import math

import numpy as np

from . import geometry as geo
from .barrier import b_stiff, derivs1, lambda1, eps_g_of, mollifier
from .jet import Jet

M_DIM = {geo.PT: 3, geo.EE: 3, geo.PE: 2, geo.PP: 1}

FLAG_ACTIVE, FLAG_FILTERED, FLAG_MOLLIFIED = 1, 2, 4


def _vec(A):
    """Column-stacking vectorisation vec(A) (Sec. 5.1, notation)."""
    return np.asarray(A, dtype=float).reshape(-1, order="F")


def _project(dJdx, dbdJ, HJ):
    """Map J-space derivatives to x-space through the change-of-basis tensor dJ/dx (Eq. 13, Eq. 15)."""
    m = dbdJ.shape[0]
    D = dJdx.reshape(m * m, -1, order="F")         # rows indexed like vec(J)
    grad = D.T @ _vec(dbdJ)
    hess = D.T @ HJ @ D
    return grad, hess, D


def eval_stencil(typ, pts, eps_x, dhat, kappa, d_thr_ratio=0.1):
    """Evaluate one stencil; ``pts`` is s x 3 (slot order of ``geometry.decode``)."""
    s = geo.N_VERTS[typ]
    n = 3 * s
    out = {"energy": 0.0, "grad": np.zeros(n), "hess": np.zeros((n, n)), "lam": 0.0,
           "w": np.zeros(n), "flags": 0, "aux": {}}
    G = geo.exact_geometry(typ, pts, dhat)
    if G["g"] >= 1:                     # d >= dhat: the clamped barrier is zero (Eq. 6)
        return out
    out["flags"] |= FLAG_ACTIVE
    g = float(G["g"])
    dg = np.array([float(v) for v in G["dg"]])
    f = math.sqrt(g)
    grad_f = dg / (2.0 * f)            # df/dx with f = sqrt(g)
    eps_g = eps_g_of(d_thr_ratio)
    filtered = g < eps_g
    if filtered:
        out["flags"] |= FLAG_FILTERED
    lam1_thr = lambda1(eps_g, dhat)
    aux = out["aux"]
    aux.update(g=g, f=f, eps_g=eps_g)

    if not geo.PARALLEL[typ]:
        m = M_DIM[typ]
        J = np.eye(m)
        J[m - 1, m - 1] = f                                 # Eq. 10
        nvec = np.zeros(m)
        nvec[m - 1] = 1.0                                   # n = e_m (Eq. 11)
        N = np.outer(nvec, nvec)
        b, b_g, b_gg = derivs1(b_stiff, g, dhat)            # Eq. 24
        lam1 = 4.0 * g * b_gg + 2.0 * b_g                   # Eq. 18
        lam1_hat = lam1_thr if filtered else lam1           # Eq. 23
        Q1 = J @ N / math.sqrt(g)                           # Eq. 21
        HJ = lam1_hat * np.outer(_vec(Q1), _vec(Q1))        # Eq. 20 / 23
        dbdJ = b_g * 2.0 * J @ N                            # Eq. 13-14
        dJdx = np.zeros((m, m, n))
        dJdx[m - 1, m - 1, :] = grad_f
        grad, hess, D = _project(dJdx, dbdJ, HJ)
        lam, w = lam1_hat, D.T @ _vec(Q1)
        aux.update(b=b, b_g=b_g, b_gg=b_gg, lambda1=lam1, lambda1_hat=lam1_hat,
                   lambda23=2.0 * b_g, HJ=HJ, Q1=Q1)
        energy = b
    else:
        c = float(G["c"])
        dc = np.array([float(v) for v in G["dc"]])
        sc = math.sqrt(c)
        mollified = c < eps_x
        if mollified:
            out["flags"] |= FLAG_MOLLIFIED
        J = np.diag([1.0, sc, f])                           # Eq. 28
        n_gam = np.array([0.0, 1.0, 0.0])
        n_g = np.array([0.0, 0.0, 1.0])
        N_gam, N_g = np.outer(n_gam, n_gam), np.outer(n_g, n_g)
        gam = float(np.dot(J @ n_gam, J @ n_gam))           # Eq. 26 (= c)
        # btilde(gamma, g) = e(gamma) b(g) (Eq. 27, 29) with a two-variable jet
        Jg = Jet.variable(gam, 0, 2)
        Jb = Jet.variable(g, 1, 2)
        bt = mollifier(Jg, c, eps_x) * b_stiff(Jb, dhat)
        bt_gam, bt_g = bt.g
        bt_gg_gam, bt_gg_g, bt_cross = bt.h[0][0], bt.h[1][1], bt.h[0][1]
        e_val = mollifier(gam, c, eps_x)
        lam_gam1 = 2.0 * (bt_gam + 2.0 * gam * bt_gg_gam)       # Sec. 6.2, first term
        lam_gam23 = 2.0 * bt_gam
        lam_g1 = 2.0 * (bt_g + 2.0 * g * bt_gg_g)               # Sec. 6.2, second term
        lam_g23 = 2.0 * bt_g
        if filtered:
            lam_g1 = e_val * lam1_thr                          # reading: Eq. 23 on lambda_g1
        t = bt_cross * sc * f                                  # Eq. 33
        Mx = np.array([[lam_gam1, 4.0 * t], [4.0 * t, lam_g1]])  # supplement, aux matrix M
        evals, evecs = np.linalg.eigh(Mx)
        lam7p, lam8p = float(evals[0]), float(evals[1])
        q = evecs[:, 1].copy()
        if q[1] < 0 or (q[1] == 0 and q[0] < 0):
            q = -q
        Q8p = np.diag([0.0, q[0], q[1]])                       # Eq. 35 (normalised)
        Tx = np.array([[0, 0, 0], [0, 0, 1], [0, -1, 0]], float)
        Tz = np.array([[0, 1, 0], [-1, 0, 0], [0, 0, 0]], float)
        Qg2, Qg3 = Tx @ N_gam, Tz @ N_gam                       # Eq. 32
        HJ = (lam_gam23 * np.outer(_vec(Qg2), _vec(Qg2))
              + lam_gam23 * np.outer(_vec(Qg3), _vec(Qg3))
              + lam8p * np.outer(_vec(Q8p), _vec(Q8p)))         # Eq. 36
        dbdJ = bt_gam * 2.0 * J @ N_gam + bt_g * 2.0 * J @ N_g  # Eq. 30 with Eq. 14
        dJdx = np.zeros((3, 3, n))
        # d sqrt(c)/dx; at exactly parallel edges (c = 0) sqrt(c) is not differentiable and the
        # mollified energy, its gradient and Hessian all vanish (e(0) = 0): take it as 0 (reading)
        dJdx[1, 1, :] = dc / (2.0 * sc) if sc > 0.0 else 0.0
        dJdx[2, 2, :] = grad_f
        grad, hess, D = _project(dJdx, dbdJ, HJ)
        lam, w = lam8p, D.T @ _vec(Q8p)
        aux.update(c=c, e=e_val, b=bt.v, lam_gam1=lam_gam1, lam_gam23=lam_gam23, lam_g1=lam_g1,
                   lam_g23=lam_g23, t=t, lam7p=lam7p, lam8p=lam8p, q8p=q, HJ=HJ,
                   bt_gam=bt_gam, bt_g=bt_g, bt_gamgam=bt_gg_gam, bt_gg=bt_gg_g, bt_cross=bt_cross)
        energy = bt.v

    out["energy"] = kappa * energy
    out["grad"] = kappa * grad
    out["hess"] = kappa * hess
    out["lam"] = kappa * lam
    out["w"] = w
    return out


def gather(x, verts):
    """Vertex coordinates from a (3, n) SoA position array, in slot order."""
    return [[float(x[0, v]), float(x[1, v]), float(x[2, v])] for v in verts]


def _eval_chunk(args):
    x, stencils, eps_x, dhat, kappa, d_thr_ratio, lo, hi = args
    k = hi - lo
    energy = np.zeros(k)
    grad = np.zeros((12, k))
    hess = np.zeros((144, k))
    lam = np.zeros(k)
    w = np.zeros((12, k))
    flags = np.zeros(k, dtype=np.uint8)
    for i in range(lo, hi):
        typ, verts = geo.decode(stencils[:, i])
        r = eval_stencil(typ, gather(x, verts), float(eps_x[i]), dhat, kappa, d_thr_ratio)
        n = 3 * geo.N_VERTS[typ]
        j = i - lo
        energy[j] = r["energy"]
        grad[:n, j] = r["grad"]
        hess[:n * n, j] = r["hess"].reshape(-1)
        lam[j] = r["lam"]
        w[:n, j] = r["w"]
        flags[j] = r["flags"]
    return energy, grad, hess, lam, w, flags


def eval_stencils(x, stencils, eps_x, dhat, kappa, d_thr_ratio=0.1, processes=1):
    """Evaluate a whole stencil list.

    Layout of the results (entry-major, stride k): energy[k]; grad[j, i] for
    j < 3s; hess[a*3s + b, i] for the 3s x 3s block (row-major); lam[k], w[j, i];
    flags[k].  Unused rows of a stencil with s < 4 stay zero.
    ``processes`` > 1 uses a spawn-started process pool.
    """
    x = np.asarray(x, dtype=float)
    stencils = np.asarray(stencils)
    eps_x = np.asarray(eps_x, dtype=float)
    k = stencils.shape[1]
    if processes <= 1 or k < 256:
        parts = [_eval_chunk((x, stencils, eps_x, dhat, kappa, d_thr_ratio, 0, k))]
    else:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        step = (k + 4 * processes - 1) // (4 * processes)
        jobs = [(x, stencils, eps_x, dhat, kappa, d_thr_ratio, lo, min(k, lo + step))
                for lo in range(0, k, step)]
        with ProcessPoolExecutor(processes, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_eval_chunk, jobs))
    energy = np.concatenate([p[0] for p in parts])
    grad = np.concatenate([p[1] for p in parts], axis=1)
    hess = np.concatenate([p[2] for p in parts], axis=1)
    lam = np.concatenate([p[3] for p in parts])
    w = np.concatenate([p[4] for p in parts], axis=1)
    flags = np.concatenate([p[5] for p in parts])
    return {"energy": energy, "grad": grad, "hess": hess, "lam": lam, "w": w, "flags": flags}


def compute_eps_x(rest_x, stencils):
    """eps_x per stencil from rest positions (Sec. 6.1); 0 for PT/PE/PP."""
    k = stencils.shape[1]
    out = np.zeros(k)
    for i in range(k):
        typ, verts = geo.decode(stencils[:, i])
        if geo.PARALLEL[typ] or typ == geo.EE:
            out[i] = geo.eps_x_rest(typ, gather(rest_x, verts))
    return out
