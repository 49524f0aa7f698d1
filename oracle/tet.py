"""Per-tetrahedron elastic energy, gradient and PSD-projected Hessian (oracle; test infrastructure only).

The paper's deformable bodies use the Stable neo-Hookean energy of Smith et al. (its
Sec. 8, first paragraph; the analytic eigensystems of isotropic energies are the cited
Smith et al. 2019, Sec. 2 "Eigen Analysis").  The energy is not restated in the paper;
this module writes it from the Stable neo-Hookean paper (Smith, de Goes and Kim, ACM TOG
2018): its energy with the rest-stable offset alpha and its match of (mu, lam) to the Lame
parameters of linear elasticity:

    Psi(F) = mu/2 (I_C - 3) + lam/2 (J - alpha)^2 - mu/2 log(I_C + 1),
    I_C = ||F||_F^2,  J = det F,  alpha = 1 + mu/lam - mu/(4 lam)   (rest-stable: dPsi/dF(I) = 0)

with mu = 4/3 mu_L and lam = lam_L + 5/6 mu_L from the Lame parameters of (E, nu), so the
small-strain limit is linear elasticity with (mu_L, lam_L).

Per element with rest shape matrix Dm (columns xbar_i - xbar_0) and rest volume V:
    F = Ds Dm^-1,  energy = scale * V * Psi(F),
    gradient = scale * V * dF/dx^T vec(dPsi/dF),
    Hessian  = scale * V * dF/dx^T [d2Psi/dF2]_+ dF/dx,
where [.]_+ is the projection onto the positive semi-definite cone (eigenvalues clamped at
0), computed here by a numerical eigendecomposition -- the plain definition -- whereas the
CUDA path uses the analytic eigensystem.  Derivatives of Psi come from second-order jets over
the nine entries of F.
"""
import math

import numpy as np

from .jet import Jet, jlog


def lame(E, nu):
    mu_l = E / (2.0 * (1.0 + nu))
    lam_l = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu_l, lam_l


def snh_params(E, nu):
    """(mu, lam) of the Stable neo-Hookean energy matched to linear elasticity."""
    mu_l, lam_l = lame(E, nu)
    return 4.0 / 3.0 * mu_l, lam_l + 5.0 / 6.0 * mu_l


def psi(Fv, mu, lam):
    """Stable neo-Hookean energy of F given as 9 entries, column-major (jets or floats)."""
    F = [[Fv[i + 3 * j] for j in range(3)] for i in range(3)]
    Ic = sum(F[i][j] * F[i][j] for i in range(3) for j in range(3))
    J = (F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1])
         - F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0])
         + F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]))
    alpha = 1.0 + mu / lam - mu / (4.0 * lam)
    return 0.5 * mu * (Ic - 3.0) + 0.5 * lam * (J - alpha) * (J - alpha) - 0.5 * mu * jlog(Ic + 1.0)


def psi_derivs(F, mu, lam):
    """(Psi, dPsi/dvecF (9), d2Psi/dvecF2 (9x9)) at a 3x3 F (vec = column-major)."""
    fv = np.asarray(F, dtype=float).reshape(-1, order="F")
    jets = [Jet.variable(float(fv[k]), k, 9) for k in range(9)]
    j = psi(jets, mu, lam)
    return j.v, np.array(j.g), np.array(j.h)


def rest_shape(rest_pts):
    """Dm^-1 and rest volume from the four rest vertices (4 x 3)."""
    P = np.asarray(rest_pts, dtype=float)
    Dm = np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], axis=1)
    return np.linalg.inv(Dm), abs(np.linalg.det(Dm)) / 6.0


def dF_dx(Dm_inv):
    """Constant 9 x 12 matrix with vec(F) = dF_dx @ x (x = 4 vertices stacked, vec column-major)."""
    D = np.zeros((9, 12))
    for a in range(4):                 # vertex a, coordinate r
        for r in range(3):
            # d Ds / d x_{a,r}: Ds = [x1-x0, x2-x0, x3-x0]
            dDs = np.zeros((3, 3))
            if a == 0:
                dDs[r, :] = -1.0
            else:
                dDs[r, a - 1] = 1.0
            dF = dDs @ Dm_inv
            D[:, 3 * a + r] = dF.reshape(-1, order="F")
    return D


def project_psd(H):
    w, V = np.linalg.eigh(0.5 * (H + H.T))
    return (V * np.maximum(w, 0.0)) @ V.T


def eval_tet(pts, Dm_inv, vol, mu, lam, scale):
    """energy, grad (12), projected Hessian (12 x 12) of one tetrahedron (pts: 4 x 3)."""
    P = np.asarray(pts, dtype=float)
    Ds = np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], axis=1)
    F = Ds @ Dm_inv
    e, g9, H9 = psi_derivs(F, mu, lam)
    D = dF_dx(Dm_inv)
    k = scale * vol
    return {"energy": k * e, "grad": k * (D.T @ g9), "hess": k * (D.T @ project_psd(H9) @ D), "F": F}


def eval_tets(x, tets, Dm_inv, vol, mu, lam, scale):
    """Whole list; Dm_inv (9, T) row-major 3x3 per element.  Entry-major outputs."""
    x = np.asarray(x, dtype=float)
    T = tets.shape[1]
    energy = np.zeros(T)
    grad = np.zeros((12, T))
    hess = np.zeros((144, T))
    for t in range(T):
        pts = x[:, tets[:, t]].T
        r = eval_tet(pts, np.asarray(Dm_inv[:, t]).reshape(3, 3), float(vol[t]), mu, lam, scale)
        energy[t] = r["energy"]
        grad[:, t] = r["grad"]
        hess[:, t] = r["hess"].reshape(-1)
    return {"energy": energy, "grad": grad, "hess": hess}


def rest_state(rest_x, tets, density):
    """Dm^-1 (9, T) row-major, volumes (T), lumped masses (n): m_i = density * sum vol / 4,
    summed over the incident tetrahedra in ascending index."""
    T = tets.shape[1]
    n = rest_x.shape[1]
    Dmi = np.zeros((9, T))
    vol = np.zeros(T)
    mass = np.zeros(n)
    for t in range(T):
        inv, v = rest_shape(rest_x[:, tets[:, t]].T)
        Dmi[:, t] = inv.reshape(-1)
        vol[t] = v
    for t in range(T):
        for a in range(4):
            mass[tets[a, t]] += density * vol[t] / 4.0
    return Dmi, vol, mass
