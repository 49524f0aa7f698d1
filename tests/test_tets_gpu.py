"""GPU parity of gipc_tet_rest / gipc_eval_tets against the tetrahedron oracle.

The kernel projects the Hessian with the closed-form eigensystem (rotation-variant SVD,
twist / flip / scaling modes); the oracle with a numerical eigendecomposition of the
directly differentiated 9x9 Hessian.  Per element, energy within 1e-10 relative, gradient
and Hessian entries within 1e-10 of the element's largest entry (FP64).  The mixed form keeps
energy and gradient in FP64 (same bound) and projects the Hessian in float32 arithmetic: per
block relative Frobenius error <= 1e-4 (the mixed form's block bound), symmetric, positive
semidefinite to float32 rounding.  Rest state within 1e-12, masses within 1e-13 relative.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import tet as O  # noqa: E402

E, NU, RHO, DT = 1e5, 0.4, 1000.0, 0.01


@pytest.fixture(scope="module")
def gipc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_09400_gb300 as g
    return g


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _mesh(seed, nx=6, ny=5, nz=4, amp=0.08, invert=0):
    rest, tets = synth.tet_box(nx, ny, nz, spacing=0.05, origin=(0.2, 0.1, 0.3))
    x = synth.deform(rest, seed, amplitude=amp)
    if invert:
        rng = np.random.default_rng(seed)
        for t in rng.choice(tets.shape[1], invert, replace=False):
            v = tets[:, t]
            x[:, v[3]] = x[:, v[0]] - 0.6 * (x[:, v[3]] - x[:, v[0]])
    return rest, x, tets


def _compare(got, ref, rtol):
    e, er = got["energy"], ref["energy"]
    assert (np.abs(e - er) <= rtol * np.abs(er) + 1e-300).all()
    for key in ("grad", "hess"):
        g, r = got[key].astype(np.float64), ref[key]
        scale = np.abs(r).max(axis=0)
        assert (np.abs(g - r).max(axis=0) <= rtol * scale).all(), \
            f"{key}: worst {np.max(np.abs(g - r).max(axis=0) / scale):.3e}"


def test_snh_parameters(gipc):
    mu, lam = gipc.snh_params(E, NU)
    assert (mu, lam) == pytest.approx(O.snh_params(E, NU), rel=1e-15)


@pytest.mark.parametrize("seed,invert", [(1, 0), (2, 3), (3, 10)])
def test_eval_tets_fp64_parity(gipc, seed, invert):
    rest, x, tets = _mesh(seed, invert=invert)
    mu, lam = O.snh_params(E, NU)
    Dmi, vol, mass = O.rest_state(rest, tets, RHO)
    ref = O.eval_tets(x, tets, Dmi, vol, mu, lam, DT * DT)
    g = gipc.eval_tets(_dev(x), _dev(tets), _dev(Dmi), _dev(vol), mu, lam, DT * DT)
    torch.cuda.synchronize()
    _compare({k: v.cpu().numpy() for k, v in g.items()}, ref, 1e-10)


def _scaling_block_definite(x, tets, Dmi, mu, lam):
    """Per element: is the 3x3 Hessian of the energy in the signed singular values positive
    definite?  (Where it is, the kernel takes the projection of those modes from a triangular
    factorisation, elsewhere from the eigenpairs.)"""
    alpha = 1.0 + mu / lam - mu / (4.0 * lam)
    out = []
    for t in range(tets.shape[1]):
        v = tets[:, t]
        Ds = np.stack([x[:, v[a]] - x[:, v[0]] for a in (1, 2, 3)], axis=1)
        F = Ds @ Dmi[:, t].reshape(3, 3)
        s = np.linalg.svd(F, compute_uv=False)
        if np.linalg.det(F) < 0:
            s[2] = -s[2]
        I2, J = (s * s).sum(), s.prod()
        A = np.empty((3, 3))
        for i in range(3):
            j, l = (i + 1) % 3, (i + 2) % 3
            A[i, i] = mu * (1 - 1 / (I2 + 1)) + 2 * mu * s[i] ** 2 / (I2 + 1) ** 2 + lam * (s[j] * s[l]) ** 2
            A[i, j] = A[j, i] = 2 * mu * s[i] * s[j] / (I2 + 1) ** 2 + lam * s[l] * (2 * J - alpha)
        out.append(np.linalg.eigvalsh(A).min() > 0)
    return np.array(out)


def test_eval_tets_fp64_parity_both_scaling_projections(gipc):
    # a large smooth deformation: about half the elements have a definite scaling block
    rest, x, tets = _mesh(4, amp=0.3)
    mu, lam = O.snh_params(E, NU)
    Dmi, vol, mass = O.rest_state(rest, tets, RHO)
    pd = _scaling_block_definite(x, tets, Dmi, mu, lam)
    assert pd.sum() >= 50 and (~pd).sum() >= 50
    ref = O.eval_tets(x, tets, Dmi, vol, mu, lam, DT * DT)
    g = gipc.eval_tets(_dev(x), _dev(tets), _dev(Dmi), _dev(vol), mu, lam, DT * DT)
    torch.cuda.synchronize()
    _compare({k: v.cpu().numpy() for k, v in g.items()}, ref, 1e-10)


def test_eval_tets_equal_stretches_and_tiny_coupling(gipc):
    # F^T F with two equal diagonal entries and an off-diagonal entry of 1e-25 (its square
    # underflows in float32), a pure rotation, the identity and a uniform scaling: near-repeated
    # singular values, where a rotation angle comes out as 0 / 0 unless guarded
    rest = np.array([[0.0, 1.0, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0], [0.0, 0.0, 0.0, 1.0]])
    c, s = np.cos(0.3), np.sin(0.3)
    Fs = [np.array([[1.0, 0.0, 0.1], [0.0, 1.0, 0.1], [1e-13, 1e-12, 1.4]]),
          np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]]),
          np.eye(3), 0.9 * np.eye(3),
          np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [1e-13, 1e-12, 1.0]])]
    xs, tets = [], []
    for e, F in enumerate(Fs):
        xs.append(F @ rest + 2.0 * e)
        tets.append(np.arange(4) + 4 * e)
    x = np.concatenate(xs, axis=1)
    rest_all = np.concatenate([rest + 2.0 * e for e in range(len(Fs))], axis=1)
    tets = np.stack(tets, axis=1).astype(np.int32)
    mu, lam = O.snh_params(E, NU)
    Dmi, vol, _ = O.rest_state(rest_all, tets, RHO)
    ref = O.eval_tets(x, tets, Dmi, vol, mu, lam, DT * DT)
    for prec in ("fp64", "mixed"):
        g = gipc.eval_tets(_dev(x), _dev(tets), _dev(Dmi), _dev(vol), mu, lam, DT * DT, precision=prec)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in g.items()}
        assert np.isfinite(got["hess"]).all()
        if prec == "fp64":
            assert (np.abs(got["energy"] - ref["energy"]) <= 1e-10 * np.abs(ref["energy"])).all()
            # the identity and the rotation are stress-free (zero gradient up to rounding): with
            # unit edge lengths the gradient is held to the element's Hessian scale
            hs = np.abs(ref["hess"]).max(axis=0)
            assert (np.abs(got["hess"] - ref["hess"]).max(axis=0) <= 1e-10 * hs).all()
            gs = np.maximum(np.abs(ref["grad"]).max(axis=0), hs)
            assert (np.abs(got["grad"] - ref["grad"]).max(axis=0) <= 1e-10 * gs).all()


def test_rest_state_and_mass(gipc):
    rest, _, tets = _mesh(4)
    Dmi, vol, mass = O.rest_state(rest, tets, RHO)
    gD, gv, gm = gipc.tet_rest(_dev(rest), _dev(tets), density=RHO)
    torch.cuda.synchronize()
    np.testing.assert_allclose(gD.cpu().numpy(), Dmi, rtol=1e-12, atol=1e-12 * np.abs(Dmi).max())
    np.testing.assert_allclose(gv.cpu().numpy(), vol, rtol=1e-12)
    np.testing.assert_allclose(gm.cpu().numpy(), mass, rtol=1e-13)
    gm2 = gipc.tet_rest(_dev(rest), _dev(tets), density=RHO)[2]
    assert torch.equal(gm, gm2)          # reproducible bit for bit


def test_rest_state_rejects_degenerate_elements(gipc):
    rest, _, tets = _mesh(5)
    tets = tets.copy()
    tets[3, 0] = tets[2, 0]               # repeated vertex: zero volume
    with pytest.raises(gipc.GipcError, match="degenerate"):
        gipc.tet_rest(_dev(rest), _dev(tets), density=RHO)


def test_eval_tets_mixed_precision(gipc):
    rest, x, tets = _mesh(6, invert=2)
    mu, lam = O.snh_params(E, NU)
    Dmi, vol, _ = O.rest_state(rest, tets, RHO)
    ref = O.eval_tets(x, tets, Dmi, vol, mu, lam, DT * DT)
    g = gipc.eval_tets(_dev(x), _dev(tets), _dev(Dmi), _dev(vol), mu, lam, DT * DT, precision="mixed")
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in g.items()}
    assert got["hess"].dtype == np.float32
    _compare({"energy": got["energy"], "grad": got["grad"], "hess": ref["hess"]}, ref, 1e-10)
    H = got["hess"].astype(np.float64).T.reshape(-1, 12, 12)
    Hr = ref["hess"].T.reshape(-1, 12, 12)
    err = np.linalg.norm(H - Hr, axis=(1, 2)) / np.linalg.norm(Hr, axis=(1, 2))
    assert err.max() <= 1e-4, err.max()
    assert np.array_equal(H, np.transpose(H, (0, 2, 1)))
    lo = np.linalg.eigvalsh(H).min(axis=1)
    assert (lo >= -1e-5 * np.abs(H).max(axis=(1, 2))).all()


def test_rest_configuration_is_stress_free(gipc):
    rest, _, tets = _mesh(7)
    mu, lam = O.snh_params(E, NU)
    gD, gv, _ = gipc.tet_rest(_dev(rest), _dev(tets))
    g = gipc.eval_tets(_dev(rest), _dev(tets), gD, gv, mu, lam, 1.0)
    torch.cuda.synchronize()
    assert g["grad"].abs().max().item() <= 1e-9 * mu * gv.max().item()


def test_invalid_tetrahedra_give_zero_energy(gipc):
    rest, x, tets = _mesh(8)
    tets = tets.copy()
    tets[0, 5] = rest.shape[1] + 3
    mu, lam = O.snh_params(E, NU)
    Dmi, vol, _ = O.rest_state(rest, np.where(tets >= rest.shape[1], 0, tets), RHO)
    g = gipc.eval_tets(_dev(x), _dev(tets), _dev(Dmi), _dev(vol), mu, lam, 1.0)
    assert g["energy"][5].item() == 0.0


def test_full_size_sampled(gipc):
    """~576k tetrahedra (a 41 x 41 x 61 vertex block, 6 per cell), 1500 sampled elements vs the oracle."""
    rest, tets = synth.tet_box(41, 41, 61, spacing=0.01)
    x = synth.deform(rest, 9, amplitude=0.05)
    mu, lam = O.snh_params(E, NU)
    gD, gv, gm = gipc.tet_rest(_dev(rest), _dev(tets), density=RHO)
    g = gipc.eval_tets(_dev(x), _dev(tets), gD, gv, mu, lam, DT * DT)
    torch.cuda.synchronize()
    assert tets.shape[1] == 576000
    idx = np.sort(np.random.default_rng(10).choice(tets.shape[1], 1500, replace=False))
    sub = np.ascontiguousarray(tets[:, idx])
    Dmi, vol, _ = O.rest_state(rest, sub, RHO)
    np.testing.assert_allclose(gD.cpu().numpy()[:, idx], Dmi, rtol=1e-12, atol=1e-9)
    ref = O.eval_tets(x, sub, Dmi, vol, mu, lam, DT * DT)
    got = {k: v.cpu().numpy()[..., idx] for k, v in g.items()}
    _compare(got, ref, 1e-10)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_blocks_layout_is_the_dense_layout_rearranged(gipc, precision):
    rest, x, tets = _mesh(7, invert=2)
    mu, lam = O.snh_params(E, NU)
    Dmi, vol, _ = O.rest_state(rest, tets, RHO)
    args = (_dev(x), _dev(tets), _dev(Dmi), _dev(vol), mu, lam, DT * DT)
    a = gipc.eval_tets(*args, precision=precision, want=("hess",))["hess"].cpu().numpy()                  # [144, T]
    b = gipc.eval_tets(*args, precision=precision, want=("hess",), layout="blocks")["hess"].cpu().numpy()  # [T, 144]
    at = [((r // 3) * 4 + c // 3) * 9 + (r % 3) * 3 + c % 3 for r in range(12) for c in range(12)]
    assert np.array_equal(b[:, at], a.T)
