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
