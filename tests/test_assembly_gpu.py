"""GPU parity of gipc_assemble_bsr against the oracle's plain assembly.

Pattern (rowptr, colidx) must match bit for bit.  FP64 values and the gradient
are summed in the same fixed order as the oracle (mass, tetrahedra by index,
stencils by index) with non-contracted IEEE operations, so they must match bit
for bit too.  Mixed (float32) values: within 1e-5 of each block's largest entry.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import assembly as A  # noqa: E402


@pytest.fixture(scope="module")
def gipc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_09400_gb300 as g
    return g


def _dev(a, dt=None):
    t = torch.tensor(np.ascontiguousarray(a), device="cuda")
    return t.to(dt) if dt is not None else t


def _gpu_assemble(gipc, n, d, mode="dense", precision="fp64", with_tets=True, with_mass=True, **kw):
    hdt = torch.float64 if precision == "fp64" else torch.float32
    st = _dev(d["stencils"])
    blocks = _dev(d["hess"] if mode == "dense" else d["w"], hdt)
    r = gipc.assemble_bsr(n, stencils=st, stencil_hess=blocks, stencil_mode=mode,
                          stencil_lam=_dev(d["lam"]), stencil_grad=_dev(d["grad"]),
                          tets=_dev(d["tets"]) if with_tets else None,
                          tet_hess=_dev(d["tet_hess"], hdt) if with_tets else None,
                          tet_grad=_dev(d["tet_grad"]) if with_tets else None,
                          mass=_dev(d["mass"]) if with_mass else None, grad_base=_dev(d["grad_base"]),
                          precision=precision, **kw)
    torch.cuda.synchronize()
    return {"rowptr": r["rowptr"].cpu().numpy(), "colidx": r["colidx"].cpu().numpy(),
            "vals": r["vals"].cpu().numpy().reshape(-1, 3, 3), "grad": r["grad"].cpu().numpy(), "nnzb": r["nnzb"]}


def _oracle(n, d, mode="dense", with_tets=True, with_mass=True, rows=None, f32=False):
    cast = (lambda a: a.astype(np.float32).astype(np.float64)) if f32 else (lambda a: a)
    sd = {"kind": mode, "hess": cast(d["hess"]), "lam": d["lam"], "w": cast(d["w"]), "grad": d["grad"]}
    td = {"kind": "dense", "hess": cast(d["tet_hess"]), "grad": d["tet_grad"]}
    return A.assemble(n, d["stencils"], sd, d["tets"] if with_tets else None, td if with_tets else None,
                      d["mass"] if with_mass else None, d["grad_base"], rows=rows)


@pytest.mark.parametrize("mode", ["dense", "rank1"])
def test_fp64_bit_exact(gipc, mode):
    n = 700
    d = synth.random_elements(n, 3000, 800, seed=11)
    got = _gpu_assemble(gipc, n, d, mode)
    ref = _oracle(n, d, mode)
    np.testing.assert_array_equal(got["rowptr"], ref["rowptr"])
    np.testing.assert_array_equal(got["colidx"], ref["colidx"])
    assert np.array_equal(got["vals"], ref["vals"])
    assert np.array_equal(got["grad"], ref["grad"])


def _to_blocks(h, n3):
    """[144, count] entry-major dense blocks (entry a * n3 + b) -> [count, 144] element-major 3x3
    sub-blocks (GIPC_HESS_BLOCKS)."""
    out = np.zeros((h.shape[1], 144))
    for s3 in np.unique(n3):
        idx = np.nonzero(n3 == s3)[0]
        for a in range(s3):
            for b in range(s3):
                out[idx, ((a // 3) * 4 + b // 3) * 9 + (a % 3) * 3 + b % 3] = h[a * s3 + b, idx]
    return out


def test_blocks_layout_assembles_bit_identically(gipc):
    """The same element values in the element-major 3x3 layout give the same BSR bit for bit (the
    sums run over the same contributions in the same order)."""
    from oracle import geometry as geo
    n = 700
    d = synth.random_elements(n, 3000, 800, seed=11)
    n3 = np.array([3 * geo.N_VERTS[geo.decode(d["stencils"][:, i])[0]] for i in range(d["stencils"].shape[1])])
    r = gipc.assemble_bsr(n, stencils=_dev(d["stencils"]), stencil_hess=_dev(_to_blocks(d["hess"], n3)),
                          stencil_mode="blocks", stencil_grad=_dev(d["grad"]), tets=_dev(d["tets"]),
                          tet_hess=_dev(_to_blocks(d["tet_hess"], np.full(d["tets"].shape[1], 12))),
                          tet_mode="blocks", tet_grad=_dev(d["tet_grad"]), mass=_dev(d["mass"]),
                          grad_base=_dev(d["grad_base"]))
    ref = _oracle(n, d, "dense")
    np.testing.assert_array_equal(r["rowptr"].cpu().numpy(), ref["rowptr"])
    np.testing.assert_array_equal(r["colidx"].cpu().numpy(), ref["colidx"])
    assert np.array_equal(r["vals"].cpu().numpy().reshape(-1, 3, 3), ref["vals"])
    assert np.array_equal(r["grad"].cpu().numpy(), ref["grad"])


def test_deterministic_across_runs(gipc):
    n = 500
    d = synth.random_elements(n, 4000, 300, seed=12)
    a = _gpu_assemble(gipc, n, d, "rank1")
    b = _gpu_assemble(gipc, n, d, "rank1")
    assert all(np.array_equal(a[k], b[k]) for k in ("rowptr", "colidx", "vals", "grad"))


def test_mixed_precision_values(gipc):
    n = 600
    d = synth.random_elements(n, 2500, 500, seed=13)
    got = _gpu_assemble(gipc, n, d, "rank1", precision="mixed")
    ref = _oracle(n, d, "rank1", f32=True)
    np.testing.assert_array_equal(got["colidx"], ref["colidx"])
    scale = np.abs(ref["vals"]).max(axis=(1, 2))
    err = np.abs(got["vals"] - ref["vals"]).max(axis=(1, 2))
    assert (err <= 1e-5 * scale).all()
    assert np.array_equal(got["grad"], ref["grad"])     # gradient stays float64


def test_no_mass_no_tets_and_ragged(gipc):
    for n, k in [(5, 1), (33, 7), (257, 129)]:
        d = synth.random_elements(n, k, 0, seed=n)
        got = _gpu_assemble(gipc, n, d, "dense", with_tets=False, with_mass=False)
        ref = _oracle(n, d, "dense", with_tets=False, with_mass=False)
        np.testing.assert_array_equal(got["rowptr"], ref["rowptr"])
        np.testing.assert_array_equal(got["colidx"], ref["colidx"])
        assert np.array_equal(got["vals"], ref["vals"])
        assert np.array_equal(got["grad"], ref["grad"])


def test_long_rows_use_the_block_sort(gipc):
    """A hub vertex in 700 point-triangle stencils gets 2800 contributions (> 512 per warp)."""
    n = 3000
    d = synth.random_elements(n, 1500, 0, seed=14, hub=7, hub_count=700)
    got = _gpu_assemble(gipc, n, d, "rank1", with_tets=False)
    rows = [7, 8, 100]
    ref = _oracle(n, d, "rank1", with_tets=False, rows=rows)
    for q, r in enumerate(rows):
        a0, a1 = got["rowptr"][r], got["rowptr"][r + 1]
        b0, b1 = ref["rowptr"][q], ref["rowptr"][q + 1]
        np.testing.assert_array_equal(got["colidx"][a0:a1], ref["colidx"][b0:b1])
        assert np.array_equal(got["vals"][a0:a1], ref["vals"][b0:b1])
    assert got["rowptr"][8] - got["rowptr"][7] > 512


def test_rows_beyond_the_block_sort_use_the_global_sort(gipc):
    """A hub vertex in 2100 point-triangle stencils gets 8401 contributions (> 8192 per block)."""
    n = 12000
    d = synth.random_elements(n, 2500, 0, seed=15, mix=(("PT", 1.0),), hub=3, hub_count=2100)
    got = _gpu_assemble(gipc, n, d, "rank1", with_tets=False)
    rows = [3, 4, 500]
    ref = _oracle(n, d, "rank1", with_tets=False, rows=rows)
    for q, r in enumerate(rows):
        a0, a1 = got["rowptr"][r], got["rowptr"][r + 1]
        b0, b1 = ref["rowptr"][q], ref["rowptr"][q + 1]
        np.testing.assert_array_equal(got["colidx"][a0:a1], ref["colidx"][b0:b1])
        assert np.array_equal(got["vals"][a0:a1], ref["vals"][b0:b1])
    assert np.array_equal(got["grad"][:, rows], ref["grad"][:, rows])
    assert got["rowptr"][4] - got["rowptr"][3] > 2000


def test_capacity_retry(gipc):
    n = 300
    d = synth.random_elements(n, 1000, 100, seed=16)
    got = _gpu_assemble(gipc, n, d, "dense", capacity=10)
    ref = _oracle(n, d, "dense")
    np.testing.assert_array_equal(got["colidx"], ref["colidx"])
    assert np.array_equal(got["vals"], ref["vals"])


def test_invalid_elements_are_skipped(gipc):
    n = 50
    d = synth.random_elements(n, 40, 5, seed=17)
    bad = d["stencils"].copy()
    bad[:, 0] = [-1, 99, 3, 4]          # vertex 99 >= n
    bad[:, 1] = [-1, 2, synth.NULL, 5]  # malformed
    d2 = dict(d, stencils=bad)
    got = _gpu_assemble(gipc, n, d2, "dense")
    keep = np.ones(40, bool)
    keep[:2] = False
    d3 = dict(d, stencils=bad[:, keep], hess=d["hess"][:, keep], grad=d["grad"][:, keep],
              w=d["w"][:, keep], lam=d["lam"][keep])
    ref = _oracle(n, d3, "dense")
    np.testing.assert_array_equal(got["colidx"], ref["colidx"])
    # summation order differs only by the skipped ids, which contribute nothing
    np.testing.assert_allclose(got["vals"], ref["vals"], rtol=0, atol=1e-12)


def test_full_size_sheet_space_sampled(gipc):
    """1M stencils over the 301,088-vertex two-sheet index space: ~4.1M blocks; 64 sampled rows."""
    st, n = synth.sheet_index_space(1_000_000)
    rng = np.random.default_rng(21)
    k = st.shape[1]
    d = {"stencils": st, "tets": np.zeros((4, 0), np.int32), "hess": np.zeros((1, k)),
         "lam": rng.uniform(0.1, 2.0, k), "w": rng.normal(size=(12, k)), "grad": rng.normal(size=(12, k)),
         "tet_hess": np.zeros((144, 0)), "tet_grad": np.zeros((12, 0)), "mass": synth.sheet_mass(),
         "grad_base": rng.normal(size=(3, n))}
    got = _gpu_assemble(gipc, n, d, "rank1", with_tets=False)
    assert 3.5e6 < got["nnzb"] < 5e6
    rows = sorted(rng.choice(n, 64, replace=False).tolist())
    ref = _oracle(n, d, "rank1", with_tets=False, rows=rows)
    for q, r in enumerate(rows):
        a0, a1 = got["rowptr"][r], got["rowptr"][r + 1]
        b0, b1 = ref["rowptr"][q], ref["rowptr"][q + 1]
        np.testing.assert_array_equal(got["colidx"][a0:a1], ref["colidx"][b0:b1])
        assert np.array_equal(got["vals"][a0:a1], ref["vals"][b0:b1])
        assert np.array_equal(got["grad"][:, r], ref["grad"][:, r])
