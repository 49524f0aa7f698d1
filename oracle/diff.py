"""Exact derivatives of the incremental potential and the implicit adjoint of one implicit step
(oracle; test infrastructure only).

The paper differentiates nothing with respect to the simulation inputs; this module is the
plain definition the differentiation extension is checked against.

* Element energies are those of the oracle's own modules -- the barrier of Eq. 24 with the
  mollifier of Eq. 25 on the squared distance of the stencil's type (``oracle.geometry``,
  ``oracle.barrier``) and the Stable neo-Hookean energy (``oracle.tet``) -- evaluated on
  second-order jets over the element's coordinates, so value, gradient and Hessian are exact
  derivatives of the energy (no projection).
* ``potential`` assembles I(x) = 1/2 (x - xt)^T M (x - xt) + scale sum vol Psi + sum kappa btilde,
  its gradient and its Hessian (a scipy sparse matrix, coordinate 3 v + c).
* ``adjoint_step`` differentiates a converged step x_new = argmin I through grad I(x_new) = 0:
  with a = dL/dx_new + dL/dv_new / dt on free vertices, H lambda = a (free rows / columns, sparse
  direct solve), then dL/dv_old = dt M lambda, dL/dx_old = M lambda - dL/dv_new / dt (free) or
  dL/dx_new - (H lambda) (fixed), and E dL/dE = -lambda . grad I_elastic.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import barrier as B
from . import contact as C
from . import geometry as G
from . import tet as TT
from .jet import Jet


def _jet_points(pts):
    s = len(pts)
    n = 3 * s
    return [[Jet.variable(float(pts[a][c]), 3 * a + c, n) for c in range(3)] for a in range(s)]


def stencil_energy_jet(typ, pts, eps_x, dhat, kappa):
    """kappa * e(c) * b(g) of one stencil with its exact gradient and Hessian (slot-major)."""
    P = _jet_points(pts)
    g = G._squared_distance(typ, P) / (dhat * dhat)
    if not (0.0 < g.v < 1.0):
        return Jet.const(0.0, 3 * len(pts))
    e = B.b_stiff(g, dhat)
    if G.PARALLEL[typ]:
        c = G.parallel_measure(P[0], P[1], P[2], P[3])
        e = B.mollifier(c, c.v, eps_x) * e
    return kappa * e


def tet_energy_jet(pts, Dm_inv_rowmajor, vol, mu, lam, scale):
    """scale * vol * Psi(Ds Dm^-1) of one tetrahedron with its exact gradient and Hessian."""
    P = _jet_points(pts)
    Dmi = np.asarray(Dm_inv_rowmajor, dtype=float).reshape(3, 3)
    Ds = [[P[k + 1][i] - P[0][i] for k in range(3)] for i in range(3)]
    F = [[Ds[i][0] * Dmi[0][j] + Ds[i][1] * Dmi[1][j] + Ds[i][2] * Dmi[2][j] for j in range(3)] for i in range(3)]
    Fv = [F[i][j] for j in range(3) for i in range(3)]      # column-major, as oracle.tet.psi takes it
    return (scale * vol) * TT.psi(Fv, mu, lam)


def potential(x, xt, mass, tets, Dm_inv, vol, mu, lam, scale, stencils, eps_x, dhat, kappa, hessian=True,
              tets_only=False):
    """(I, grad [3, n], H sparse [3n, 3n] or None) at x for the given contact list; xt may be
    None (no inertia term in I and grad; H still holds M)."""
    x = np.asarray(x, dtype=float)
    n = x.shape[1]
    grad = np.zeros((3, n))
    rows, cols, vals = [], [], []
    energy = 0.0
    if not tets_only:
        if xt is not None:
            d = x - xt
            energy = 0.5 * float(np.sum(mass * np.sum(d * d, axis=0)))
            grad += mass[None, :] * d
        if hessian:
            for c in range(3):
                rows.extend(3 * np.arange(n) + c)
                cols.extend(3 * np.arange(n) + c)
                vals.extend(mass)

    def add(verts, jet):
        nonlocal energy
        energy += jet.v
        s = len(verts)
        for a in range(s):
            for c in range(3):
                grad[c, verts[a]] += jet.g[3 * a + c]
        if hessian:
            for a in range(s):
                for c in range(3):
                    for b in range(s):
                        for d in range(3):
                            rows.append(3 * verts[a] + c)
                            cols.append(3 * verts[b] + d)
                            vals.append(jet.h[3 * a + c][3 * b + d])

    for t in range(tets.shape[1]):
        v = [int(i) for i in tets[:, t]]
        add(v, tet_energy_jet(x[:, v].T, Dm_inv[:, t], vol[t], mu, lam, scale))
    if not tets_only and stencils is not None:
        for i in range(stencils.shape[1]):
            typ, verts = G.decode(stencils[:, i])
            add(verts, stencil_energy_jet(typ, [x[:, v] for v in verts], float(eps_x[i]), dhat, kappa))
    H = sp.csr_matrix((vals, (rows, cols)), shape=(3 * n, 3 * n)) if hessian else None
    return energy, grad, H


def adjoint_step(x_new, sc, prm, adj_x_new, adj_v_new):
    """One step's adjoint at a converged x_new (``sc`` as oracle.newton.build_scene, ``prm`` as
    oracle.newton.newton_step).  Returns (dL/dx_old, dL/dv_old, E dL/dE of this step)."""
    dt = prm["dt"]
    n = x_new.shape[1]
    stencils, eps = C.find_contacts(x_new, sc["rest_x"], sc["tris"], sc["edges"], sc["verts"], prm["dhat"])
    _, _, H = potential(x_new, None, sc["mass"], sc["tets"], sc["Dm_inv"], sc["vol"], prm["mu"], prm["lam"], dt * dt,
                        stencils if stencils.shape[1] else None, eps, prm["dhat"], prm["kappa"])
    fixed = np.asarray(sc["fixed"], bool)
    free3 = np.repeat(~fixed, 3)                       # coordinate 3 v + c
    a = (adj_x_new + adj_v_new / dt).T.reshape(-1) * free3
    lam = np.zeros(3 * n)
    idx = np.nonzero(free3)[0]
    lam[idx] = spla.spsolve(H[idx][:, idx].tocsc(), a[idx])
    Hl = H @ lam
    m3 = np.repeat(sc["mass"], 3)
    ml = m3 * lam
    ax = np.where(free3, ml - (adj_v_new / dt).T.reshape(-1), adj_x_new.T.reshape(-1) - Hl)
    av = np.where(free3, dt * ml, 0.0)
    _, gel, _ = potential(x_new, None, sc["mass"], sc["tets"], sc["Dm_inv"], sc["vol"], prm["mu"], prm["lam"], dt * dt,
                          None, None, prm["dhat"], prm["kappa"], hessian=False, tets_only=True)
    logE = -float(lam @ gel.T.reshape(-1))
    return ax.reshape(n, 3).T.copy(), av.reshape(n, 3).T.copy(), logE
