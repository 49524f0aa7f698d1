"""Modified preconditioned conjugate gradients (oracle; test infrastructure only).

The Newton system H d = -g of Alg. 1 is solved with modified-PCG (the paper
cites Baraff and Witkin's "large steps" variant, Sec. 7.2 "Parallel solver
optimizations") with a 3x3 block-diagonal preconditioner (Sec. 7.2,
"Preconditioning of the CG solver") and the termination rule
delta_new < 1e-4 delta_0 (Sec. 8, first paragraph).  The "modified" part is the
filter S that zeroes the components of constrained (fixed) vertices so the
search stays in the free subspace.

Iteration (x_0 given, default 0):
    r = S(b - A x);  z = P^-1 r;  c = S(z);  delta_new = r . z;  delta_0 = delta_new
    while k < max_iter and delta_new > 0 and delta_new >= tol * delta_0:
        q = S(A c);  alpha = delta_new / (c . q)
        x += alpha c;  r -= alpha q
        s = P^-1 r;  delta_old = delta_new;  delta_new = r . s
        c = S(s + (delta_new / delta_old) c);  k += 1
Vectors are (3, n) like positions; A is a BSR dict of ``oracle.assembly``.
The sparse product uses scipy's BSR matvec as a library step.
"""
import numpy as np
import scipy.sparse as sp


def bsr_to_scipy(A, n):
    vals = np.asarray(A["vals"], dtype=np.float64).reshape(-1, 3, 3)
    return sp.bsr_matrix((vals, np.asarray(A["colidx"]), np.asarray(A["rowptr"])), shape=(3 * n, 3 * n))


def block_jacobi_inverse(A, n):
    """Inverses of the 3x3 diagonal blocks H_ii (identity where a row has no diagonal block)."""
    inv = np.tile(np.eye(3), (n, 1, 1))
    vals = np.asarray(A["vals"], dtype=np.float64).reshape(-1, 3, 3)
    for r in range(n):
        for p in range(A["rowptr"][r], A["rowptr"][r + 1]):
            if A["colidx"][p] == r:
                inv[r] = np.linalg.inv(vals[p])
    return inv


def pcg(A, n, b, fixed=None, tol=1e-4, max_iter=1000, x0=None, history=False, trace=False):
    """Returns dict(x (3,n), iters, rel (delta_new/delta_0), delta_0, [deltas]).

    trace=True also returns the iterates, residuals and search directions of every iteration
    ("xs", "rs", "cs": lists of (n, 3) vertex-major arrays, index k after k iterations; "cs"[k]
    is the direction used by iteration k + 1) for checks of the iteration itself."""
    M = bsr_to_scipy(A, n)
    Pinv = block_jacobi_inverse(A, n)
    free = np.ones((n, 3)) if fixed is None else np.repeat((~np.asarray(fixed, bool))[:, None], 3, 1).astype(float)
    S = lambda v: v * free
    precond = lambda v: np.einsum("nij,nj->ni", Pinv, v)
    matvec = lambda v: (M @ v.reshape(-1)).reshape(n, 3)
    bb = np.asarray(b, dtype=np.float64).T.copy()            # (n, 3) vertex-major
    x = np.zeros((n, 3)) if x0 is None else S(np.asarray(x0, dtype=np.float64).T.copy())
    r = S(bb - matvec(x))
    z = precond(r)
    c = S(z)
    delta_new = float(np.sum(r * z))
    delta_0 = delta_new
    deltas = [delta_new]
    xs, rs, cs = [x], [r], [c]
    k = 0
    while k < max_iter and delta_new > 0 and delta_new >= tol * delta_0:
        q = S(matvec(c))
        alpha = delta_new / float(np.sum(c * q))
        x = x + alpha * c
        r = r - alpha * q
        s = precond(r)
        delta_old = delta_new
        delta_new = float(np.sum(r * s))
        c = S(s + (delta_new / delta_old) * c)
        k += 1
        deltas.append(delta_new)
        if trace:
            xs.append(x)
            rs.append(r)
            cs.append(c)
    out = {"x": x.T.copy(), "iters": k, "rel": delta_new / delta_0 if delta_0 > 0 else 0.0, "delta_0": delta_0}
    if history:
        out["deltas"] = deltas
    if trace:
        out.update(xs=xs, rs=rs, cs=cs)
    return out
