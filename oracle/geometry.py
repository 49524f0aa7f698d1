"""Contact-stencil decoding and exact stencil geometry (oracle; test infrastructure only).

Follows the paper's problem statement:

* Stencil tuples (i0, i1, i2, i3) carry the contact type in the signs of the
  indices (Sec. 7.2, "Data structures"): EE [+,+,+,+], PT [-,+,+,+],
  PE [-,+,+,#], PP [-,+,#,#]; nearly-parallel EE [+,-,+,+], PE [-,-,+,-],
  PP [-,-,-,-].  Reading: a negative slot stores -(i+1) (= ~i), so vertex 0
  can be negative; the placeholder '#' is INT32_MIN.  Nearly-parallel PE/PP
  keep all four vertices of the two edges, so the parallelness measure c of
  Sec. 6.1 can be computed: PE-par = (point, other end of the point's edge,
  edge end 0, edge end 1); PP-par = (point a, other end of a's edge, point b,
  other end of b's edge).
* The distance d is the constrained minimum of Eq. 4 (point-triangle) or
  Eq. 5 (edge-edge) with the active set fixed by the stencil type (Sec. 3.1:
  the active constraints decide which distance measure applies).  With the
  active set fixed, each case is an unconstrained least-squares problem over
  the affine hull of the active primitives; this module solves its normal
  equations in exact rational arithmetic (``fractions.Fraction``) and carries
  first derivatives along with ``Dual`` numbers, so d^2, g = d^2/dhat^2 (Eq. 9,
  Eq. 11) and their gradients are exact before the final rounding to float.
* The parallelness measure c = ||(x12 - x11) x (x22 - x21)||^2 of Sec. 6.1 and
  its gradient, also exact.
"""
from fractions import Fraction

from .jet import Dual

PT, EE, PE, PP, EE_PAR, PE_PAR, PP_PAR = range(7)
TYPE_NAMES = ("PT", "EE", "PE", "PP", "EE_PAR", "PE_PAR", "PP_PAR")
NULL = -2147483648                     # the '#' placeholder
N_VERTS = (4, 4, 3, 2, 4, 4, 4)        # vertices per stencil type
PARALLEL = (False, False, False, False, True, True, True)


def decode(t):
    """Return (type, vertex ids in slot order) for a sign-encoded tuple (Sec. 7.2)."""
    i0, i1, i2, i3 = (int(v) for v in t)
    if i0 >= 0 and i1 >= 0:
        if min(i2, i3) < 0:
            raise ValueError(f"malformed EE tuple {t}")
        return EE, (i0, i1, i2, i3)
    if i0 >= 0 and i1 < 0:
        if i1 == NULL or min(i2, i3) < 0:
            raise ValueError(f"malformed EE-parallel tuple {t}")
        return EE_PAR, (i0, ~i1, i2, i3)
    if i0 == NULL:
        raise ValueError(f"malformed tuple {t}")
    if i1 >= 0:
        if i2 == NULL:
            if i3 != NULL:
                raise ValueError(f"malformed PP tuple {t}")
            return PP, (~i0, i1)
        if i2 < 0:
            raise ValueError(f"malformed tuple {t}")
        if i3 == NULL:
            return PE, (~i0, i1, i2)
        if i3 < 0:
            raise ValueError(f"malformed PT tuple {t}")
        return PT, (~i0, i1, i2, i3)
    if NULL in (i1, i2, i3):
        raise ValueError(f"malformed parallel tuple {t}")
    if i2 >= 0:
        if i3 >= 0:
            raise ValueError(f"malformed PE-parallel tuple {t}")
        return PE_PAR, (~i0, ~i1, i2, ~i3)
    if i3 >= 0:
        raise ValueError(f"malformed PP-parallel tuple {t}")
    return PP_PAR, (~i0, ~i1, ~i2, ~i3)


# ----------------------------------------------------------------------------- exact vectors
def _sub(a, b):
    return [a[i] - b[i] for i in range(3)]


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def _axpy(a, x, y):
    return [a * x[i] + y[i] for i in range(3)]


def _solve2(A, rhs):
    """Cramer's rule for a 2x2 system (exact over rationals)."""
    det = A[0][0] * A[1][1] - A[0][1] * A[1][0]
    return ((rhs[0] * A[1][1] - A[0][1] * rhs[1]) / det,
            (A[0][0] * rhs[1] - rhs[0] * A[1][0]) / det)


def sqdist_point_plane(p, a, b, c):
    """min over (beta1, beta2) of |p - a - beta1 (b-a) - beta2 (c-a)|^2 (Eq. 4, interior active set)."""
    e1, e2, w = _sub(b, a), _sub(c, a), _sub(p, a)
    G = [[_dot(e1, e1), _dot(e1, e2)], [_dot(e2, e1), _dot(e2, e2)]]
    beta1, beta2 = _solve2(G, [_dot(e1, w), _dot(e2, w)])
    r = _sub(w, _axpy(beta1, e1, [beta2 * e2[i] for i in range(3)]))
    return _dot(r, r)


def sqdist_line_line(a0, a1, b0, b1):
    """min over (gamma1, gamma2) of |a0 + gamma1 (a1-a0) - b0 - gamma2 (b1-b0)|^2 (Eq. 5, interior)."""
    a, b, w = _sub(a1, a0), _sub(b1, b0), _sub(a0, b0)
    # r = w + gamma1 a - gamma2 b ; normal equations a.r = 0 and b.r = 0
    A = [[_dot(a, a), -_dot(a, b)], [_dot(a, b), -_dot(b, b)]]
    g1, g2 = _solve2(A, [-_dot(a, w), -_dot(b, w)])
    r = [w[i] + g1 * a[i] - g2 * b[i] for i in range(3)]
    return _dot(r, r)


def sqdist_point_line(p, e0, e1):
    """min over t of |p - e0 - t (e1-e0)|^2 (point-edge, interior of the edge active)."""
    e, w = _sub(e1, e0), _sub(p, e0)
    t = _dot(w, e) / _dot(e, e)
    r = [w[i] - t * e[i] for i in range(3)]
    return _dot(r, r)


def sqdist_point_point(p, q):
    r = _sub(p, q)
    return _dot(r, r)


def parallel_measure(a0, a1, b0, b1):
    """c = ||(a1 - a0) x (b1 - b0)||^2 (Sec. 6.1)."""
    w = _cross(_sub(a1, a0), _sub(b1, b0))
    return _dot(w, w)


def _squared_distance(typ, P):
    if typ == PT:
        return sqdist_point_plane(P[0], P[1], P[2], P[3])
    if typ in (EE, EE_PAR):
        return sqdist_line_line(P[0], P[1], P[2], P[3])
    if typ == PE:
        return sqdist_point_line(P[0], P[1], P[2])
    if typ == PE_PAR:
        return sqdist_point_line(P[0], P[2], P[3])
    if typ == PP:
        return sqdist_point_point(P[0], P[1])
    if typ == PP_PAR:
        return sqdist_point_point(P[0], P[2])
    raise ValueError(typ)


def _dual_points(pts):
    """Stencil vertex coordinates as exact Dual variables, slot-major (x of slot j -> index 3j)."""
    s = len(pts)
    n = 3 * s
    zero = Fraction(0)
    return [[Dual.variable(Fraction(float(pts[j][k])), 3 * j + k, n, zero) for k in range(3)]
            for j in range(s)]


def exact_geometry(typ, pts, dhat):
    """Exact g = d^2/dhat^2 with its gradient and, for the nearly-parallel types, c with its gradient.

    ``pts`` are the stencil's vertices in slot order (s x 3 floats).  Returns a dict of
    Fractions: g, dg (list of 3s), and for parallel types c, dc.
    """
    P = _dual_points(pts)
    d2 = _squared_distance(typ, P)
    dh2 = Fraction(float(dhat)) ** 2
    out = {"g": d2.v / dh2, "dg": [a / dh2 for a in d2.d]}
    if PARALLEL[typ]:
        c = parallel_measure(P[0], P[1], P[2], P[3])
        out["c"] = c.v
        out["dc"] = list(c.d)
    return out


def eps_x_rest(typ, rest_pts):
    """Mollifier tolerance eps_x = 1e-3 ||xbar12 - xbar11||^2 ||xbar22 - xbar21||^2 (Sec. 6.1).

    Taken from the rest positions of the two edges of an EE-derived stencil
    (slots (0,1) and (2,3)); 0 for the other types.  Evaluated in float64.
    """
    if not PARALLEL[typ] and typ != EE:
        return 0.0
    a = [float(rest_pts[1][i]) - float(rest_pts[0][i]) for i in range(3)]
    b = [float(rest_pts[3][i]) - float(rest_pts[2][i]) for i in range(3)]
    return 1e-3 * (a[0] * a[0] + a[1] * a[1] + a[2] * a[2]) * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2])
