"""Pins for the oracle's modified PCG: dense direct solves, the filter, the stop rule."""
import numpy as np

import synth
from oracle import assembly as A
from oracle import pcg as P


def spd_system(n, k, T, seed):
    """A = M + sum of PSD element blocks (rank-one stencils, Gram tet blocks), b random."""
    d = synth.random_elements(n, k, T, seed=seed)
    rng = np.random.default_rng(seed + 1)
    th = np.stack([(B @ B.T).reshape(-1) for B in rng.normal(size=(T, 12, 4)) * 0.3], 1) if T else np.zeros((144, 0))
    sd = {"kind": "rank1", "lam": d["lam"], "w": d["w"], "grad": None}
    td = {"kind": "dense", "hess": th, "grad": None}
    R = A.assemble(n, d["stencils"], sd, d["tets"], td, d["mass"])
    return R, d["grad_base"], th, d


def test_converges_to_dense_solution():
    n = 40
    R, b, _, _ = spd_system(n, 90, 20, seed=30)
    H = A.to_dense(n, R)
    out = P.pcg(R, n, b, tol=1e-26, max_iter=10 * 3 * n)
    xd = np.linalg.solve(H, b.T.reshape(-1)).reshape(n, 3).T
    np.testing.assert_allclose(out["x"], xd, rtol=0, atol=1e-9 * np.abs(xd).max())


def test_filter_keeps_fixed_vertices_and_solves_free_subsystem():
    n = 36
    R, b, _, _ = spd_system(n, 80, 10, seed=31)
    fixed = np.zeros(n, bool)
    fixed[[0, 5, 6, 20]] = True
    H = A.to_dense(n, R)
    free = np.repeat(~fixed, 3)
    out = P.pcg(R, n, b, fixed=fixed, tol=1e-26, max_iter=10 * 3 * n)
    x = out["x"].T.reshape(-1)
    assert (x[~free] == 0).all()
    xf = np.linalg.solve(H[np.ix_(free, free)], b.T.reshape(-1)[free])
    np.testing.assert_allclose(x[free], xf, atol=1e-9 * np.abs(xf).max())


def test_block_diagonal_matrix_is_solved_in_one_iteration():
    n = 25
    rng = np.random.default_rng(32)
    blocks = [B @ B.T + np.eye(3) for B in rng.normal(size=(n, 3, 3))]
    R = {"rowptr": np.arange(n + 1), "colidx": np.arange(n), "vals": np.array(blocks)}
    b = rng.normal(size=(3, n))
    out = P.pcg(R, n, b, tol=1e-30, max_iter=50)
    assert out["iters"] == 1
    xd = np.stack([np.linalg.solve(blocks[i], b[:, i]) for i in range(n)], 1)
    np.testing.assert_allclose(out["x"], xd, rtol=1e-12)


def test_stop_rule_delta_new_below_tol_delta0():
    n = 60
    R, b, _, _ = spd_system(n, 150, 30, seed=33)
    out = P.pcg(R, n, b, tol=1e-4, max_iter=500, history=True)
    d = out["deltas"]
    assert d[-1] < 1e-4 * d[0]
    assert all(v >= 1e-4 * d[0] for v in d[:-1])
    assert out["iters"] == len(d) - 1


def test_block_jacobi_inverse():
    n = 30
    R, _, _, _ = spd_system(n, 60, 10, seed=34)
    inv = P.block_jacobi_inverse(R, n)
    for r in range(n):
        for p in range(R["rowptr"][r], R["rowptr"][r + 1]):
            if R["colidx"][p] == r:
                np.testing.assert_allclose(inv[r] @ R["vals"][p], np.eye(3), atol=1e-12)


# ---- the iteration itself (not only its limit) -----------------------------------------------
# Preconditioned CG on the free subsystem has three properties that fix every iterate, not just
# the converged solution: the residuals are orthogonal in the P^-1 inner product, the search
# directions are conjugate with respect to H, and x_k minimises the quadratic
# 1/2 x^T H x - b^T x over x_0 + K_k(P^-1 H, P^-1 r_0).  A wrong beta, a misplaced filter S or a
# wrong preconditioner application breaks at least one of them.

def _free_system(n=40, seed=35):
    R, b, _, _ = spd_system(n, 100, 24, seed=seed)
    fixed = np.zeros(n, bool)
    fixed[[1, 7, 22]] = True
    rng = np.random.default_rng(seed + 7)
    x0 = rng.normal(size=(3, n))
    return R, b, fixed, x0


def _pin_errors(pcg_fn, R, n, b, fixed, x0, k=8):
    """(max P^-1-orthogonality, max H-conjugacy, max Krylov-minimiser deviation, max |x| on fixed)."""
    H = A.to_dense(n, R)
    free = np.repeat(~fixed, 3)
    Hf = H[np.ix_(free, free)]
    Pinv = P.block_jacobi_inverse(R, n)
    Pd = np.zeros((3 * n, 3 * n))
    for i in range(n):
        Pd[3 * i:3 * i + 3, 3 * i:3 * i + 3] = Pinv[i]
    Pf = Pd[np.ix_(free, free)]
    out = pcg_fn(R, n, b, fixed=fixed, tol=0.0, max_iter=k, x0=x0, trace=True)
    flat = lambda v: np.asarray(v).reshape(-1)           # (n, 3) vertex-major -> 3n
    rs = [flat(r)[free] for r in out["rs"]]
    cs = [flat(c)[free] for c in out["cs"]]
    orth = conj = 0.0
    for i in range(len(rs)):
        for j in range(i):
            orth = max(orth, abs(rs[i] @ Pf @ rs[j]) / np.sqrt((rs[i] @ Pf @ rs[i]) * (rs[j] @ Pf @ rs[j])))
            conj = max(conj, abs(cs[i] @ Hf @ cs[j]) / np.sqrt((cs[i] @ Hf @ cs[i]) * (cs[j] @ Hf @ cs[j])))
    # x_0 as the solver uses it (filtered), r_0 of the free subsystem, Krylov basis by Gram-Schmidt
    x0f = x0.T.reshape(-1).copy()
    x0f[~free] = 0.0
    bf = b.T.reshape(-1)
    r0 = (bf - H @ x0f)[free]
    krylov = 0.0
    V = []
    v = Pf @ r0
    for kk in range(1, len(out["xs"])):
        for u in V:
            v = v - (u @ v) * u
        for u in V:                                       # second pass keeps the basis orthonormal
            v = v - (u @ v) * u
        V.append(v / np.linalg.norm(v))
        Vm = np.stack(V, 1)
        y = np.linalg.solve(Vm.T @ Hf @ Vm, Vm.T @ r0)
        xk = x0f[free] + Vm @ y
        got = flat(out["xs"][kk])[free]
        krylov = max(krylov, np.abs(got - xk).max() / np.abs(xk).max())
        v = Pf @ (Hf @ V[-1])
    fixed_mag = max(np.abs(flat(xx)[~free]).max() for xx in out["xs"])
    return orth, conj, krylov, fixed_mag


def test_residuals_orthogonal_directions_conjugate_iterates_minimise_over_krylov_space():
    n = 40
    R, b, fixed, x0 = _free_system(n)
    orth, conj, krylov, fixed_mag = _pin_errors(P.pcg, R, n, b, fixed, x0)
    assert orth < 1e-9 and conj < 1e-9
    assert krylov < 1e-9
    assert fixed_mag == 0.0


def _mutant(replacements):
    """The oracle's pcg with a planted mistake (source text replaced), for checking that the pins
    above would catch it."""
    import inspect
    src = inspect.getsource(P.pcg)
    for old, new in replacements:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    ns = dict(vars(P))
    exec(compile(src, "<mutant>", "exec"), ns)
    return ns["pcg"]


def test_pins_catch_planted_mistakes():
    n = 40
    R, b, fixed, x0 = _free_system(n)
    mutants = {
        # beta = (r.r)_new / (r.r)_old instead of (r.z)_new / (r.z)_old
        "beta_from_rr": [("        r = r - alpha * q\n", "        r_prev = r\n        r = r - alpha * q\n"),
                         ("c = S(s + (delta_new / delta_old) * c)",
                          "c = S(s + (float(np.sum(r * r)) / float(np.sum(r_prev * r_prev))) * c)")],
        # the filter left out of the product
        "S_dropped_on_q": [("q = S(matvec(c))", "q = matvec(c)")],
        # the filter left out of the initial residual (applied to the direction only)
        "S_dropped_on_r0": [("r = S(bb - matvec(x))", "r = bb - matvec(x)")],
    }
    for name, rep in mutants.items():
        orth, conj, krylov, fixed_mag = _pin_errors(_mutant(rep), R, n, b, fixed, x0)
        caught = orth > 1e-6 or conj > 1e-6 or krylov > 1e-6 or fixed_mag > 0.0
        assert caught, (name, orth, conj, krylov, fixed_mag)
