"""Pins for the oracle's assembly: brute-force dense scatter, pattern as a set, gradient scatter."""
import numpy as np

import synth
from oracle import assembly as A
from oracle import geometry as geo


def _dense_reference(n, d, mode):
    """Independent dense scatter H[3va:3va+3, 3vb:3vb+3] += block (numpy add.at order irrelevant)."""
    H = np.zeros((3 * n, 3 * n))
    g = d["grad_base"].T.reshape(-1).copy()
    for i in range(n):
        H[3 * i:3 * i + 3, 3 * i:3 * i + 3] += d["mass"][i] * np.eye(3)
    for e in range(d["tets"].shape[1]):
        v = d["tets"][:, e]
        blk = d["tet_hess"][:, e].reshape(12, 12)
        for a in range(4):
            g[3 * v[a]:3 * v[a] + 3] += d["tet_grad"][3 * a:3 * a + 3, e]
            for b in range(4):
                H[3 * v[a]:3 * v[a] + 3, 3 * v[b]:3 * v[b] + 3] += blk[3 * a:3 * a + 3, 3 * b:3 * b + 3]
    for e in range(d["stencils"].shape[1]):
        _, v = geo.decode(d["stencils"][:, e])
        s = len(v)
        if mode == "dense":
            blk = d["hess"][: 9 * s * s, e].reshape(3 * s, 3 * s)
        else:
            w = d["w"][: 3 * s, e]
            blk = d["lam"][e] * np.outer(w, w)
        for a in range(s):
            g[3 * v[a]:3 * v[a] + 3] += d["grad"][3 * a:3 * a + 3, e]
            for b in range(s):
                H[3 * v[a]:3 * v[a] + 3, 3 * v[b]:3 * v[b] + 3] += blk[3 * a:3 * a + 3, 3 * b:3 * b + 3]
    return H, g.reshape(n, 3).T


def _assemble(n, d, mode, rows=None):
    sd = {"kind": mode, "hess": d["hess"], "lam": d["lam"], "w": d["w"], "grad": d["grad"]}
    td = {"kind": "dense", "hess": d["tet_hess"], "grad": d["tet_grad"]}
    return A.assemble(n, d["stencils"], sd, d["tets"], td, d["mass"], d["grad_base"], rows=rows)


def test_assembly_matches_dense_scatter():
    n = 24
    for mode in ("dense", "rank1"):
        d = synth.random_elements(n, 60, 15, seed=3)
        R = _assemble(n, d, mode)
        H, g = _dense_reference(n, d, mode)
        np.testing.assert_allclose(A.to_dense(n, R), H, rtol=0, atol=1e-12 * np.abs(H).max())
        np.testing.assert_allclose(R["grad"], g, rtol=0, atol=1e-12 * np.abs(g).max())
        # matvec of the BSR equals the dense product
        p = np.random.default_rng(0).normal(size=(3, n))
        np.testing.assert_allclose(A.bsr_matvec(R, p).T.reshape(-1), H @ p.T.reshape(-1), atol=1e-10)


def test_pattern_is_the_set_of_vertex_pairs():
    n = 40
    d = synth.random_elements(n, 80, 20, seed=4)
    R = _assemble(n, d, "dense")
    pairs = {(i, i) for i in range(n)}
    for e in range(d["tets"].shape[1]):
        v = d["tets"][:, e]
        pairs |= {(int(a), int(b)) for a in v for b in v}
    for e in range(d["stencils"].shape[1]):
        _, v = geo.decode(d["stencils"][:, e])
        pairs |= {(a, b) for a in v for b in v}
    got = {(r, int(c)) for r in range(n) for c in R["colidx"][R["rowptr"][r]:R["rowptr"][r + 1]]}
    assert got == pairs
    for r in range(n):
        cols = R["colidx"][R["rowptr"][r]:R["rowptr"][r + 1]]
        assert (np.diff(cols) > 0).all()


def test_row_sampling_matches_full_assembly():
    n = 50
    d = synth.random_elements(n, 120, 30, seed=5)
    full = _assemble(n, d, "rank1")
    rows = [3, 17, 18, 42]
    part = _assemble(n, d, "rank1", rows=rows)
    for q, r in enumerate(rows):
        a0, a1 = full["rowptr"][r], full["rowptr"][r + 1]
        b0, b1 = part["rowptr"][q], part["rowptr"][q + 1]
        np.testing.assert_array_equal(full["colidx"][a0:a1], part["colidx"][b0:b1])
        np.testing.assert_array_equal(full["vals"][a0:a1], part["vals"][b0:b1])
        np.testing.assert_array_equal(full["grad"][:, r], part["grad"][:, r])


def test_symmetric_local_blocks_give_a_symmetric_matrix():
    n = 30
    d = synth.random_elements(n, 70, 10, seed=6)
    d["hess"] = np.stack([((h := d["hess"][:, e].reshape(12, 12)) + h.T).reshape(-1) for e in range(70)], 1)
    d["tet_hess"] = np.stack([((h := d["tet_hess"][:, e].reshape(12, 12)) + h.T).reshape(-1)
                              for e in range(10)], 1)
    # compact blocks for s < 4 use the top-left (3s)^2 entries row-major; rebuild them symmetric too
    for e in range(70):
        _, v = geo.decode(d["stencils"][:, e])
        s3 = 3 * len(v)
        h = d["hess"][: s3 * s3, e].reshape(s3, s3)
        d["hess"][: s3 * s3, e] = (h + h.T).reshape(-1)
    H = A.to_dense(n, _assemble(n, d, "dense"))
    np.testing.assert_allclose(H, H.T, atol=1e-12 * np.abs(H).max())
