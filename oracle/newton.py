"""One implicit time step by projected Newton with line search (oracle; test infrastructure only).

Alg. 1 of the paper, with the incremental potential of Sec. 3.1 (Eq. 1-2):

    I(x) = 1/2 (x - xtilde)^T M (x - xtilde) + dt^2 sum_T vol Psi(F) + kappa sum_k btilde_k(x),
    xtilde = x^t + dt v^t + dt^2 g   (fixed vertices: xtilde = x^t),

per Newton iteration: contacts at x, gradient and H = M + PSD-projected Hessians, the
modified-PCG solve H d = -g (fixed vertices filtered), alpha = min(1, CCD step), backtracking
alpha /= 2 until I(x_prev + alpha d) <= I_prev (contacts re-detected at every trial), and the
stop test ||d||_inf / (l dt) <= eps_d (l = bbox diagonal; the supplement's Sec. S9 form).
Velocities are (x^{t+1} - x^t) / dt.
"""
import numpy as np

from . import assembly as A
from . import contact as C
from . import pcg as P
from . import stencil as S
from . import tet as TT


def inertia(x, xt, mass):
    diff = x - xt
    return 0.5 * float(np.sum(mass * np.sum(diff * diff, axis=0)))


def potential(x, xt, sc, prm):
    """I(x) and the contact list at x."""
    st, eps = C.find_contacts(x, sc["rest_x"], sc["tris"], sc["edges"], sc["verts"], prm["dhat"])
    e = inertia(x, xt, sc["mass"])
    te = TT.eval_tets(x, sc["tets"], sc["Dm_inv"], sc["vol"], prm["mu"], prm["lam"], prm["dt"] ** 2)
    e += float(np.sum(te["energy"]))
    if st.shape[1]:
        r = S.eval_stencils(x, st, eps, prm["dhat"], prm["kappa"])
        e += float(np.sum(r["energy"]))
    return e, st, eps


def newton_step(sc, x0, v0, prm, history=None):
    """Returns (x, v, stats).  ``sc``: rest_x, tets, Dm_inv, vol, mass, tris, edges, verts, fixed, l.
    ``prm``: dhat, kappa, dt, mu, lam, gravity (3,), eps_d, pcg_tol, max_pcg, max_newton, max_ls."""
    x0 = np.asarray(x0, dtype=float)
    n = x0.shape[1]
    fixed = np.asarray(sc["fixed"], bool)
    free = ~fixed
    dt = prm["dt"]
    xt = x0.copy()
    g = np.asarray(prm["gravity"], dtype=float)[:, None]
    xt[:, free] = x0[:, free] + dt * v0[:, free] + dt * dt * g
    x = x0.copy()
    I_prev, st, eps = potential(x, xt, sc, prm)
    stats = {"newton": 0, "pcg": [], "alpha": [], "contacts": []}
    for it in range(prm["max_newton"]):
        te = TT.eval_tets(x, sc["tets"], sc["Dm_inv"], sc["vol"], prm["mu"], prm["lam"], dt * dt)
        sd = None
        if st.shape[1]:
            r = S.eval_stencils(x, st, eps, prm["dhat"], prm["kappa"])
            sd = {"kind": "dense", "hess": r["hess"], "grad": r["grad"]}
        gbase = sc["mass"][None, :] * (x - xt)
        H = A.assemble(n, st if st.shape[1] else None, sd, sc["tets"],
                       {"kind": "dense", "hess": te["hess"], "grad": te["grad"]}, sc["mass"], gbase)
        sol = P.pcg(H, n, -H["grad"], fixed=fixed, tol=prm["pcg_tol"], max_iter=prm["max_pcg"])
        d = sol["x"]
        alpha = C.max_step(x, d, sc["tris"], sc["edges"], sc["verts"])
        x_prev = x
        for _ in range(prm["max_ls"]):
            x = x_prev + alpha * d
            I_new, st_new, eps_new = potential(x, xt, sc, prm)
            if I_new <= I_prev:
                break
            alpha *= 0.5
        st, eps, I_prev = st_new, eps_new, I_new
        stats["newton"] += 1
        stats["pcg"].append(sol["iters"])
        stats["alpha"].append(alpha)
        stats["contacts"].append(st.shape[1])
        if history is not None:
            history.append(x.copy())
        if np.abs(d).max() / (sc["l"] * dt) <= prm["eps_d"]:
            break
    v = (x - x0) / dt
    stats["energy"] = I_prev
    return x, v, stats


def build_scene(scene, prm, density):
    """Rest state and masses for a scene dict of ``synth`` (rest = initial positions)."""
    Dmi, vol, mass = TT.rest_state(scene["x"], scene["tets"], density)
    return {"rest_x": scene["x"].copy(), "tets": scene["tets"], "Dm_inv": Dmi, "vol": vol, "mass": mass,
            "tris": scene["tris"], "edges": scene["edges"], "verts": scene["verts"], "fixed": scene["fixed"],
            "l": scene["l"]}
