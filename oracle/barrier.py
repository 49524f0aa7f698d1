"""Barrier functions, their g-derivatives and the eigenvalue formulas (oracle; test infrastructure only).

* ``b_stiff``  -- the quadratically stiffened barrier used throughout the paper,
  b(g) = (dhat^2 - dhat^2 g)^2 ln^2(g)                                  (Eq. 24)
* ``b_log``    -- the first form, b(g) = -(dhat^2 - dhat^2 g)^2 ln(g)    (Eq. 12),
  kept only so tests can compare with the expanded eigenvalues printed for it
  in the supplement (Sec. S3).
* ``b_ipc``    -- the original IPC barrier b(d) = -(dhat - d)^2 ln(d/dhat) (Eq. 6),
  kept for the Gauss-Newton comparison of Appendix A.
* ``mollifier`` -- e(gamma) = -gamma^2/eps_x^2 + 2 gamma/eps_x if c < eps_x, else 1 (Eq. 25).

Derivatives are taken with forward-mode jets (``oracle.jet``), never by hand.
``lambda1`` is Eq. 18 and ``lambda23`` Eq. 19; ``lambda1_filtered`` applies the
proximal filter of Eq. 23 with eps_g = (d_thr/dhat)^2 and d_thr = 0.1 dhat.
"""
from .jet import Jet, jlog


def b_stiff(g, dhat):
    """Eq. 24."""
    d2 = dhat * dhat
    lg = jlog(g)
    u = d2 - d2 * g
    return u * u * lg * lg


def b_log(g, dhat):
    """Eq. 12."""
    d2 = dhat * dhat
    u = d2 - d2 * g
    return -(u * u) * jlog(g)


def b_ipc(d, dhat):
    """Eq. 6 (for 0 < d < dhat)."""
    u = dhat - d
    return -(u * u) * jlog(d / dhat)


def derivs1(fn, x, *args):
    """(f, f', f'') of a scalar function at x by a one-variable jet."""
    j = fn(Jet.variable(float(x), 0, 1), *args)
    return j.v, j.g[0], j.h[0][0]


def lambda1(g, dhat, barrier=b_stiff):
    """Eq. 18: lambda_1 = 4 g b_gg + 2 b_g."""
    _, bg, bgg = derivs1(barrier, g, dhat)
    return 4.0 * g * bgg + 2.0 * bg


def lambda23(g, dhat, barrier=b_stiff):
    """Eq. 19: lambda_2 = lambda_3 = 2 b_g."""
    _, bg, _ = derivs1(barrier, g, dhat)
    return 2.0 * bg


def eps_g_of(d_thr_ratio):
    """eps_g = (d_thr/dhat)^2 with d_thr = ratio * dhat (Eq. 23)."""
    return d_thr_ratio * d_thr_ratio


def lambda1_filtered(g, dhat, d_thr_ratio=0.1):
    """Eq. 23: lambda_1 for g >= eps_g, else lambda_1 evaluated at d = d_thr (g = eps_g)."""
    eg = eps_g_of(d_thr_ratio)
    return lambda1(g if g >= eg else eg, dhat)


def mollifier(gamma, c, eps_x):
    """Eq. 25, as a function of gamma (a Jet or float); the branch is taken on c."""
    if c < eps_x:
        return -(gamma * gamma) / (eps_x * eps_x) + 2.0 * gamma / eps_x
    return gamma * 0.0 + 1.0
