"""Batched time step (gipc_newton_step_batch) against the oracle's Newton step run on every
scene alone, and against gipc_newton_step on every scene alone.

The scenes are independent: each keeps its own PCG scalars, CCD step, line search and stopping
test.  Per scene the batched FP64 step must reproduce the oracle's Newton iteration count,
contact count and final step length, and its positions to within the rounding of the solver's
reductions; the mixed form must land within the converged-position bar of the FP64 oracle.
Against the single-scene GPU step the batched step must agree to the rounding of the reductions
(the batched PCG sums each scene with one CTA, the single one over the whole grid)."""
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import contact as C  # noqa: E402

DT, E, NU, RHO, KAPPA = 0.01, 1e5, 0.4, 1000.0, 1e3


@pytest.fixture(scope="module")
def gipc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_09400_gb300 as g
    return g


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _single(g, sc, dhat, **kw):
    srf = g.Surface(_dev(sc["tris"]), _dev(sc["edges"]), _dev(sc["verts"]))
    scene = g.Scene(_dev(sc["x"]), _dev(sc["tets"]), srf, RHO, fixed=_dev(sc["fixed"]), l=sc["l"])
    mu, lam = g.snh_params(E, NU)
    x, v = _dev(sc["x"]), _dev(sc["v"])
    st = g.newton_step(scene, x, v, dt=DT, mu=mu, lam=lam, dhat=dhat, kappa=KAPPA, **kw)
    return x.cpu().numpy(), v.cpu().numpy(), st


def _batch(g, scenes, dhat, **kw):
    b = g.SceneBatch(scenes, RHO)
    mu, lam = g.snh_params(E, NU)
    x = b.scene.rest_x.clone()
    v = _dev(np.concatenate([s["v"] for s in scenes], axis=1))
    stats = g.newton_step_batch(b, x, v, dt=DT, mu=mu, lam=lam, dhat=dhat, kappa=KAPPA, **kw)
    return b, x.cpu().numpy(), v.cpu().numpy(), stats


def _scenes(n=5, seed=7, vmax=900):
    scenes, dhat = synth.batch_scenes(n, seed=seed, vmin=150, vmax=vmax, dhat=5e-4)
    for s in scenes:   # move them so every scene starts with some motion
        s["v"][2] = -0.5
    return scenes, dhat


ORACLE_SCENES = dict(n=4, seed=7, vmax=300)
MAX_NEWTON = 12


def _oracle_scene(k):
    """The oracle's time step of scene k of the oracle batch (run in a spawned worker)."""
    from oracle import newton as N
    from oracle import tet as TT
    scenes, dhat = _scenes(**ORACLE_SCENES)
    sc = scenes[k]
    mu, lam = TT.snh_params(E, NU)
    prm = dict(dhat=dhat, kappa=KAPPA, dt=DT, mu=mu, lam=lam, gravity=(0.0, 0.0, -9.81), eps_d=1e-2,
               pcg_tol=1e-4, max_pcg=1000, max_newton=MAX_NEWTON, max_ls=30)
    x, v, st = N.newton_step(N.build_scene(sc, prm, RHO), sc["x"], sc["v"], prm)
    return x, v, st


@pytest.fixture(scope="module")
def oracle_batch():
    """Oracle steps of every scene of a small batch (4 scenes of 150-300 vertices), one spawned
    process per scene (the pool starts without CUDA state of its own)."""
    scenes, dhat = _scenes(**ORACLE_SCENES)
    with ProcessPoolExecutor(len(scenes), mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_scene, range(len(scenes))))
    return scenes, dhat, res


@pytest.mark.parametrize("precision,hess_mode", [("fp64", "dense"), ("mixed", "rank1")])
def test_batch_matches_the_oracle_scene_by_scene(gipc, oracle_batch, precision, hess_mode):
    scenes, dhat, ref = oracle_batch
    b, xb, vb, stats = _batch(gipc, scenes, dhat, precision=precision, hess_mode=hess_mode, max_newton=MAX_NEWTON,
                              max_pcg=1000)
    assert sum(s["contacts"] for s in stats) > 0
    for k, sc in enumerate(scenes):
        xo, vo, so = ref[k]
        lo, hi = b.vert_off[k], b.vert_off[k + 1]
        step = np.abs(xo - sc["x"]).max()
        err = np.abs(xb[:, lo:hi] - xo).max()
        if precision == "fp64":
            assert stats[k]["newton_iters"] == so["newton"], (k, stats[k], so["newton"])
            assert stats[k]["contacts"] == so["contacts"][-1], (k, stats[k], so["contacts"])
            assert stats[k]["last_alpha"] == pytest.approx(so["alpha"][-1], rel=1e-8)
            assert stats[k]["energy"] == pytest.approx(so["energy"], rel=1e-9)
            # the single-scene step meets the oracle at ~1e-12 of the step; the batched solver's
            # per-scene reductions add rounding of the same order
            assert err <= 1e-9 * step, f"scene {k}: {err:.3e} of a {step:.3e} step"
        else:
            # float32 blocks, product and direction: the same minimiser within the converged-
            # position bar (1e-6 of the bounding-box diagonal l)
            assert err <= 1e-6 * sc["l"], f"scene {k}: {err:.3e} (l = {sc['l']:.3e})"
        assert C.count_intersections(xb[:, lo:hi], sc["tris"], sc["edges"]) == 0


@pytest.mark.parametrize("precision,hess_mode", [("fp64", "dense"), ("mixed", "rank1")])
def test_batch_matches_each_scene_alone(gipc, precision, hess_mode):
    scenes, dhat = _scenes()
    kw = dict(precision=precision, hess_mode=hess_mode, max_newton=12)
    b, xb, vb, stats = _batch(gipc, scenes, dhat, **kw)
    assert len(stats) == len(scenes)
    assert sum(s["contacts"] for s in stats) > 0
    for k, sc in enumerate(scenes):
        xs, vs, st = _single(gipc, sc, dhat, **kw)
        lo, hi = b.vert_off[k], b.vert_off[k + 1]
        assert stats[k]["newton_iters"] == st["newton_iters"], (k, stats[k], st)
        assert stats[k]["contacts"] == st["contacts"], (k, stats[k], st)
        assert stats[k]["converged"] == st["converged"]
        step = np.abs(xs - sc["x"]).max()
        err = np.abs(xb[:, lo:hi] - xs).max()
        # FP64: the reductions' order alone; mixed: the float32 copy of the direction rounds the
        # last-bit differences of alpha and beta up to float32 precision
        rtol = 1e-7 if precision == "fp64" else 1e-5
        assert err <= rtol * step + 1e-15, f"scene {k}: {err:.3e} of a {step:.3e} step"
        assert stats[k]["energy"] == pytest.approx(st["energy"], rel=1e-9)
        assert C.count_intersections(xb[:, lo:hi], sc["tris"], sc["edges"]) == 0


def test_scenes_never_touch_each_other(gipc):
    """Two copies of a stack at the same place in space: run together they must behave exactly
    like each alone (no contact across scenes)."""
    scenes, dhat = _scenes(n=1, seed=11)
    twin = [scenes[0], {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scenes[0].items()}]
    b, xb, _, stats = _batch(gipc, twin, dhat, max_newton=8)
    xs, _, st = _single(gipc, scenes[0], dhat, max_newton=8)
    n = scenes[0]["x"].shape[1]
    for k in range(2):
        assert stats[k]["contacts"] == st["contacts"]
        assert stats[k]["newton_iters"] == st["newton_iters"]
        step = np.abs(xs - scenes[0]["x"]).max()
        assert np.abs(xb[:, k * n:(k + 1) * n] - xs).max() <= 1e-7 * step + 1e-15
    # the two copies are bit-identical to each other (same arithmetic, scene by scene)
    assert np.array_equal(xb[:, :n], xb[:, n:])


def test_unordered_lists_are_rejected(gipc):
    scenes, dhat = _scenes(n=3, seed=5)
    b = gipc.SceneBatch(scenes, RHO)
    perm = torch.randperm(b.scene.tets.shape[1], device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    b.scene.tets = b.scene.tets[:, perm].contiguous()
    b.scene.Dm_inv = b.scene.Dm_inv[:, perm].contiguous()
    b.scene.vol = b.scene.vol[perm].contiguous()
    mu, lam = gipc.snh_params(E, NU)
    x = b.scene.rest_x.clone()
    v = torch.zeros_like(x)
    with pytest.raises(gipc.GipcError, match="ordered by scene"):
        gipc.newton_step_batch(b, x, v, dt=DT, mu=mu, lam=lam, dhat=dhat, kappa=KAPPA)


@pytest.mark.parametrize("precision,hess_mode", [("fp64", "dense"), ("mixed", "rank1")])
def test_product_variant_choice_changes_no_result(gipc, precision, hess_mode):
    """The batched product's staging variant is chosen at run time from measured times; the
    variants form every row in the same order and the scenes' dots are summed per scene, so the
    choice changes time only: a batch stepped with the tuner on (every variant timed, the fastest
    kept) and off (variant 0) gives bit-identical positions, velocities and statistics."""
    scenes, dhat = _scenes(n=8, seed=3)
    # a tight solver tolerance, so the solves run whole chunks of iterations to time
    kw = dict(precision=precision, hess_mode=hess_mode, max_newton=12, pcg_tol=1e-10, max_pcg=400)
    on, off = gipc.Context(), gipc.Context()
    for ctx in (on, off):   # the product kernel per iteration (the persistent batch solver has no variants)
        ctx.batch_persistent(False)
    on.spmv_autotune(True)
    off.spmv_autotune(False)
    _, x1, v1, s1 = _batch(gipc, scenes, dhat, ctx=on, **kw)
    _, x2, v2, s2 = _batch(gipc, scenes, dhat, ctx=off, **kw)
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)
    assert s1 == s2
    tunings = on.spmv_tunings()
    assert tunings and all(t["precision"] == precision for t in tunings)
    timed = [v["samples"] for t in tunings for v in t["variants"]]
    assert all(s >= 0 for s in timed)
    # several variants ran and were timed
    assert max(sum(v["samples"] > 0 for v in t["variants"]) for t in tunings) >= 2
    for t in tunings:
        if t["chosen"] >= 0:   # a choice is made only once every variant has its samples
            assert all(v["samples"] >= 32 for v in t["variants"])
            fastest = min(v["mean_us"] for v in t["variants"])
            assert t["variants"][t["chosen"]]["mean_us"] <= fastest * (1 + 1e-12)
    assert off.spmv_tunings() == []


@pytest.mark.parametrize("precision,hess_mode", [("fp64", "dense"), ("mixed", "rank1")])
def test_persistent_batch_solver_matches_the_per_iteration_kernels(gipc, precision, hess_mode):
    """The batched solve as one persistent launch (rows spread over the CTAs by vertex, scenes cut
    across CTAs, segmented dots) against the product + per-scene update kernels per iteration:
    the same Newton and PCG iteration counts per scene and positions within the rounding of the
    dots' summation order."""
    scenes, dhat = _scenes(n=12, seed=9, vmax=2500)
    kw = dict(precision=precision, hess_mode=hess_mode, max_newton=12)
    per, loop = gipc.Context(), gipc.Context()
    per.batch_persistent(False)
    b, x1, v1, s1 = _batch(gipc, scenes, dhat, ctx=loop, **kw)
    _, x2, v2, s2 = _batch(gipc, scenes, dhat, ctx=per, **kw)
    for k, sc in enumerate(scenes):
        assert s1[k]["newton_iters"] == s2[k]["newton_iters"], (k, s1[k], s2[k])
        assert s1[k]["contacts"] == s2[k]["contacts"]
        lo, hi = b.vert_off[k], b.vert_off[k + 1]
        step = np.abs(x2[:, lo:hi] - sc["x"]).max()
        rtol = 1e-7 if precision == "fp64" else 1e-5
        assert np.abs(x1[:, lo:hi] - x2[:, lo:hi]).max() <= rtol * step + 1e-15, k
