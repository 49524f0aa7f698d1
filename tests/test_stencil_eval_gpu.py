"""GPU parity of gipc_eval_stencils / gipc_compute_eps_x against the CPU oracle.

Tolerance (FP64 path): 1e-10 relative, per stencil -- every entry of a stencil's
gradient and Hessian block within 1e-10 of that stencil's largest entry, the
energy within 1e-10 of itself, lambda within 1e-10.  Flags and eps_x bit-exact.
Mixed path: per-block relative Frobenius error <= 1e-4.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import stencil as S  # noqa: E402

DHAT = synth.UNIT_DHAT
KAPPA = 1e3
RTOL = 1e-10
NPROC = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def gipc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_09400_gb300 as g
    return g


@pytest.fixture(scope="module")
def unit():
    d = synth.unit_stencils(k=10000, seed=20230809)
    eps = S.compute_eps_x(d["x"], d["stencils"])
    ref = S.eval_stencils(d["x"], d["stencils"], eps, DHAT, KAPPA, processes=NPROC)
    return d, eps, ref


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _n3(stencils):
    from oracle import geometry as geo
    return np.array([3 * geo.N_VERTS[geo.decode(stencils[:, i])[0]] for i in range(stencils.shape[1])])


def assert_parity(got, ref, stencils, rtol=RTOL, what=("energy", "grad", "hess")):
    n3 = _n3(stencils)
    assert np.array_equal(got["flags"], ref["flags"])
    if "energy" in what:
        e, er = got["energy"], ref["energy"]
        bad = np.abs(e - er) > rtol * np.abs(er)
        assert not bad.any(), f"energy mismatch at {np.nonzero(bad)[0][:10]}"
    for key in [w for w in ("grad", "hess") if w in what]:
        G, R = got[key], ref[key]
        for s in np.unique(n3):
            cols = np.nonzero(n3 == s)[0]
            rows = s if key == "grad" else s * s
            g, r = G[:rows, cols], R[:rows, cols]
            scale = np.abs(r).max(axis=0)
            err = np.abs(g - r).max(axis=0)
            bad = err > rtol * scale
            assert not bad.any(), f"{key} mismatch (3s={s}) at {cols[np.nonzero(bad)[0][:10]]}, " \
                                  f"worst rel {np.max(err / np.maximum(scale, 1e-300)):.3e}"


def _run(gipc, d, eps, **kw):
    x, st = _dev(d["x"]), _dev(d["stencils"])
    r = gipc.eval_stencils(x, st, _dev(eps), d["dhat"], KAPPA, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def test_eps_x_bit_exact(gipc, unit):
    d, eps, _ = unit
    got = gipc.compute_eps_x(_dev(d["x"]), _dev(d["stencils"])).cpu().numpy()
    assert np.array_equal(got, eps)


def test_fp64_dense_parity_unit_set(gipc, unit):
    d, eps, ref = unit
    got = _run(gipc, d, eps)
    assert (ref["flags"] & 1).sum() > 0.9 * len(eps)
    assert_parity(got, ref, d["stencils"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_blocks_layout_is_the_dense_layout_rearranged(gipc, unit, precision):
    """GIPC_HESS_BLOCKS holds the dense values bit for bit, each 3x3 sub-block contiguous."""
    d, eps, _ = unit
    dense = _run(gipc, d, eps, precision=precision, mode="dense", want=("hess",))["hess"]   # [144, k]
    blk = _run(gipc, d, eps, precision=precision, mode="blocks", want=("hess",))["hess"]    # [k, 144]
    n3 = _n3(d["stencils"])
    for s3 in (6, 9, 12):
        idx = np.nonzero(n3 == s3)[0]
        assert len(idx) > 0
        for a in range(s3):
            for b in range(s3):
                at = ((a // 3) * 4 + b // 3) * 9 + (a % 3) * 3 + b % 3
                assert np.array_equal(blk[idx, at], dense[a * s3 + b, idx])


def test_fp64_rank1_parity_unit_set(gipc, unit):
    d, eps, ref = unit
    got = _run(gipc, d, eps, mode="rank1", want=("energy", "grad", "hess", "lam", "flags"))
    np.testing.assert_array_equal(got["flags"], ref["flags"])
    lam_bad = np.abs(got["lam"] - ref["lam"]) > RTOL * np.abs(ref["lam"])
    assert not lam_bad.any()
    n3 = _n3(d["stencils"])
    for s in np.unique(n3):
        cols = np.nonzero(n3 == s)[0]
        w, wr = got["hess"][:s, cols], ref["w"][:s, cols]
        assert (np.abs(w - wr).max(0) <= RTOL * np.abs(wr).max(0)).all()


def test_mixed_precision_block_error(gipc, unit):
    d, eps, ref = unit
    got = _run(gipc, d, eps, precision="mixed")
    np.testing.assert_array_equal(got["flags"], ref["flags"])
    assert got["hess"].dtype == np.float32
    n3 = _n3(d["stencils"])
    worst = 0.0
    for s in np.unique(n3):
        cols = np.nonzero(n3 == s)[0]
        g = got["hess"][: s * s, cols].astype(np.float64)
        r = ref["hess"][: s * s, cols]
        nr = np.linalg.norm(r, axis=0)
        act = nr > 0
        rel = np.linalg.norm(g - r, axis=0)[act] / nr[act]
        worst = max(worst, rel.max())
    assert worst <= 1e-4, worst
    print(f"mixed: worst per-block relative Frobenius error {worst:.3e}")
    # energy and gradient stay float64; plain float64 geometry (no double-double outside
    # nearly-parallel edge-edge) loses up to ~1e-8 on edge-edge stencils at 1e-7 dhat
    assert_parity(got, ref, d["stencils"], rtol=1e-6, what=("energy", "grad"))


@pytest.mark.parametrize("k", [1, 31, 127, 129, 1003])
def test_ragged_sizes_and_shuffled_types(gipc, k):
    d = synth.unit_stencils(k=k, seed=1000 + k, shuffle=True)
    eps = S.compute_eps_x(d["x"], d["stencils"])
    ref = S.eval_stencils(d["x"], d["stencils"], eps, DHAT, KAPPA, processes=NPROC if k > 500 else 1)
    assert_parity(_run(gipc, d, eps), ref, d["stencils"])


def test_empty_list(gipc):
    x = torch.zeros((3, 4), dtype=torch.float64, device="cuda")
    st = torch.zeros((4, 0), dtype=torch.int32, device="cuda")
    r = gipc.eval_stencils(x, st, None, DHAT, KAPPA)
    assert r["energy"].numel() == 0


def test_invalid_and_inactive_stencils(gipc):
    N = synth.NULL
    x = np.array([[0.1, 0.1, 0.5, 0.9], [0.2, 0.2, 0.5, 0.1], [0.3, 0.3 + 2 * DHAT, 0.5, 0.2]])
    tuples = np.array([
        [-1, 1, N, N],        # PP at distance 2 dhat: inactive
        [-1, 7, N, N],        # index out of range
        [-1, 1, N, 3],        # malformed placeholder pattern
        [0, 1, -3, 3],        # EE with a negative third slot: malformed
        [N, 1, 2, 3],         # placeholder in slot 0
        [-1, -2, 2, 3],       # parallel PE needs a negative fourth slot
    ], dtype=np.int32).T
    got = _run(gipc, {"x": x, "stencils": tuples, "dhat": DHAT}, np.zeros(tuples.shape[1]))
    assert got["flags"][0] == 0 and got["energy"][0] == 0 and not got["hess"][:36, 0].any()
    assert (got["flags"][1:] == gipc.FLAG_INVALID).all()
    assert (got["energy"][1:] == 0).all()


def test_full_size_batch_sampled(gipc):
    """1M stencils in the launch configurations the benchmark times; 2000 sampled outputs vs the
    oracle: FP64 with entry-major and with 3x3 sub-block output (parity bar 1e-10), and the mixed
    rank-one output (lambda, w in float32; per-block relative Frobenius error of lambda w w^T
    <= 1e-4, energy and gradient 1e-6)."""
    d = synth.batch_stencils(1_000_000, seed=20230810)
    x, st = _dev(d["x"]), _dev(d["stencils"])
    eps = gipc.compute_eps_x(x, st)
    r = gipc.eval_stencils(x, st, eps, d["dhat"], KAPPA)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(3).choice(st.shape[1], 2000, replace=False))
    sub = np.ascontiguousarray(d["stencils"][:, idx])
    eps_ref = S.compute_eps_x(d["x"], sub)
    assert np.array_equal(eps.cpu().numpy()[idx], eps_ref)
    ref = S.eval_stencils(d["x"], sub, eps_ref, d["dhat"], KAPPA, processes=NPROC)
    got = {k: (v.cpu().numpy()[..., idx]) for k, v in r.items()}
    assert_parity(got, ref, sub)
    n3 = _n3(sub)
    # FP64, 3x3 sub-blocks per stencil (the FP64 step's layout): the same values as the oracle's
    ti = torch.tensor(idx, device=x.device)
    blk = gipc.eval_stencils(x, st, eps, d["dhat"], KAPPA, mode="blocks")
    hb = blk["hess"].index_select(0, ti).cpu().numpy()                   # [2000, 144]
    dense = np.zeros((144, len(idx)))
    for j, s3 in enumerate(n3):
        for a in range(s3):
            for b in range(s3):
                dense[a * s3 + b, j] = hb[j, ((a // 3) * 4 + b // 3) * 9 + (a % 3) * 3 + b % 3]
    got_b = {k: v.index_select(-1, ti).cpu().numpy() for k, v in blk.items() if k != "hess"}
    got_b["hess"] = dense
    assert_parity(got_b, ref, sub)
    # mixed, rank-one output (the mixed step's configuration)
    m = gipc.eval_stencils(x, st, eps, d["dhat"], KAPPA, precision="mixed", mode="rank1",
                           want=("energy", "grad", "hess", "lam", "flags"))
    mw = m["hess"].index_select(1, ti).cpu().numpy().astype(np.float64)   # w [12, 2000], float32
    ml = m["lam"].index_select(0, ti).cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(m["flags"].index_select(0, ti).cpu().numpy(), ref["flags"])
    worst = 0.0
    for j, s3 in enumerate(n3):
        hr = ref["hess"][: s3 * s3, j].reshape(s3, s3)
        nr = np.linalg.norm(hr)
        if nr > 0:
            hg = ml[j] * np.outer(mw[:s3, j], mw[:s3, j])
            worst = max(worst, np.linalg.norm(hg - hr) / nr)
    assert worst <= 1e-4, worst
    got_m = {k: m[k].index_select(-1, ti).cpu().numpy() for k in ("energy", "grad", "flags")}
    assert_parity(got_m, ref, sub, rtol=1e-6, what=("energy", "grad"))
