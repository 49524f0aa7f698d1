"""GB300-native Gauss-Newton IPC hot path (GIPC barrier, assembly, PCG).

Thin torch-facing binding over the C ABI of ``include/gipc.h``.  Tensors are
used for device memory and the current CUDA stream only; every step runs in the
library's own kernels.  Functions carry the names of the C entry points without
the ``gipc_`` prefix.
"""
import ctypes

import torch

from . import _abi
from ._abi import (FLAG_ACTIVE, FLAG_FILTERED, FLAG_INVALID, FLAG_MOLLIFIED, GipcError)

TYPE_IDS = {"PT": 0, "EE": 1, "PE": 2, "PP": 3, "EE_PAR": 4, "PE_PAR": 5, "PP_PAR": 6}
NULL_INDEX = -2147483648

__all__ = ["compute_eps_x", "eval_stencils", "assemble_bsr", "pcg", "pcg_noalloc", "snh_params", "tet_rest", "eval_tets",
           "Surface", "find_contacts", "ccd_max_step", "Scene", "newton_step", "SceneBatch", "newton_step_batch",
           "scatter_elements", "potential_derivs", "potential_hessian", "adjoint_step", "newton_polish",
           "incremental_potential",
           "IncrementalPotential", "simulate", "adjoint", "Context", "default_context", "GipcError", "FLAG_ACTIVE", "FLAG_FILTERED",
           "FLAG_MOLLIFIED", "FLAG_INVALID", "TYPE_IDS", "NULL_INDEX"]


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(t, name, dtype, shape0=None):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape0 is not None and (t.dim() < 1 or t.shape[0] != shape0):
        raise ValueError(f"{name} must have leading dimension {shape0}")


def compute_eps_x(rest_x, stencils, out=None, stream=None):
    """eps_x per stencil from rest positions (gipc_compute_eps_x)."""
    _check(rest_x, "rest_x", torch.float64, 3)
    _check(stencils, "stencils", torch.int32, 4)
    n, k = rest_x.shape[1], stencils.shape[1]
    if out is None:
        out = torch.empty(k, dtype=torch.float64, device=stencils.device)
    _abi.call("gipc_compute_eps_x", _ptr(rest_x), n, _ptr(stencils), k, _ptr(out), _stream(stream))
    return out


def eval_stencils(x, stencils, eps_x, dhat, kappa, d_thr_ratio=0.1, precision="fp64", mode="dense",
                  want=("energy", "grad", "hess", "flags"), out=None, stream=None):
    """Barrier energy / gradient / projected Hessian per stencil (gipc_eval_stencils).

    Returns a dict with the requested entries: energy [k] f64, grad [12, k] f64,
    hess [144, k] (dense), [k, 144] (blocks: each stencil's 3x3 sub-blocks contiguous) or [12, k]
    (rank1: w), lam [k] (rank1), flags [k] u8.
    Hessian tensors are float64 for precision='fp64' and float32 for 'mixed'.
    ``out`` may supply preallocated tensors under the same keys.
    """
    _check(x, "x", torch.float64, 3)
    _check(stencils, "stencils", torch.int32, 4)
    n, k = x.shape[1], stencils.shape[1]
    if eps_x is not None:
        _check(eps_x, "eps_x", torch.float64)
    prec = {"fp64": _abi.GIPC_FP64, "mixed": _abi.GIPC_MIXED}[precision]
    md = {"dense": _abi.GIPC_HESS_DENSE, "rank1": _abi.GIPC_HESS_RANK1, "blocks": _abi.GIPC_HESS_BLOCKS}[mode]
    hdt = torch.float64 if prec == _abi.GIPC_FP64 else torch.float32
    dev = x.device
    out = dict(out or {})
    want = set(want) | set(out)
    if md == _abi.GIPC_HESS_RANK1 and "hess" in want:
        want.add("lam")
    shapes = {"energy": ((k,), torch.float64), "grad": ((12, k), torch.float64),
              "hess": ({_abi.GIPC_HESS_DENSE: (144, k), _abi.GIPC_HESS_BLOCKS: (k, 144), _abi.GIPC_HESS_RANK1: (12, k)}[md],
                       hdt),
              "lam": ((k,), torch.float64), "flags": ((k,), torch.uint8)}
    for key in want:
        if key not in out:
            shp, dt = shapes[key]
            out[key] = torch.zeros(shp, dtype=dt, device=dev)
        else:
            _check(out[key], key, shapes[key][1])
    prm = _abi.BarrierParams(float(dhat), float(kappa), float(d_thr_ratio))
    _abi.call("gipc_eval_stencils", _ptr(x), n, _ptr(stencils), k, _ptr(eps_x), ctypes.byref(prm),
              prec, md, _ptr(out.get("energy")), _ptr(out.get("grad")), _ptr(out.get("hess")),
              _ptr(out.get("lam")), _ptr(out.get("flags")), _stream(stream))
    return out


class Context:
    """Owns a gipc_ctx (device scratch for assembly and the solver)."""

    def __init__(self):
        self._h = ctypes.c_void_p()
        _abi.call("gipc_create", ctypes.byref(self._h))

    @property
    def handle(self):
        return self._h

    def profile_begin(self):
        """Start timing this context's kernels with CUDA events on their launch stream."""
        _abi.call("gipc_profile_begin", self._h)

    def profile_read(self):
        """{kind: (launches, total_ms)} for every profiled kernel kind (synchronises on the events)."""
        out = {}
        for name, kid in _abi.PROF_KINDS.items():
            t = _abi.KernelTime()
            _abi.call("gipc_profile_read", self._h, kid, ctypes.byref(t))
            out[name] = (int(t.launches), float(t.total_ms))
        return out

    def profile_stop(self):
        _abi.call("gipc_profile_stop", self._h)

    def profile_sampling(self, kind, every):
        """Record one launch in `every` of the named kind (gipc_profile_sampling)."""
        _abi.call("gipc_profile_sampling", self._h, _abi.PROF_KINDS[kind], int(every))

    def solver_trace(self, enable=True):
        """Record the phase stamps of this context's persistent solves (gipc_profile_solver_trace)."""
        _abi.call("gipc_profile_solver_trace", self._h, 1 if enable else 0)

    def solver_phases(self):
        """{phase: median microseconds} of the last traced persistent solve, and the iterations
        used (gipc_profile_solver_phases)."""
        out = (ctypes.c_double * len(_abi.SOLVER_PHASES))()
        it = ctypes.c_int(0)
        _abi.call("gipc_profile_solver_phases", self._h, out, ctypes.byref(it))
        return dict(zip(_abi.SOLVER_PHASES, list(out))), it.value

    def batch_persistent(self, enable=True):
        """Run batched solves as one persistent launch (gipc_pcg_batch_persistent)."""
        _abi.call("gipc_pcg_batch_persistent", self._h, 1 if enable else 0)

    def spmv_autotune(self, enable=True):
        """Choose the batched product's staging variant at run time (gipc_spmv_autotune)."""
        _abi.call("gipc_spmv_autotune", self._h, 1 if enable else 0)

    def spmv_tunings(self):
        """The batched product's staging choices so far, one dict per precision and size class
        (gipc_spmv_tunings)."""
        cnt = ctypes.c_int(0)
        _abi.call("gipc_spmv_tunings", self._h, None, 0, ctypes.byref(cnt))
        arr = (_abi.SpmvTuning * max(1, cnt.value))()
        _abi.call("gipc_spmv_tunings", self._h, arr, cnt.value, ctypes.byref(cnt))
        out = []
        for t in arr[:cnt.value]:
            out.append({"precision": "fp64" if t.precision == _abi.GIPC_FP64 else "mixed", "size_class": t.size_class,
                        "chosen": t.chosen,
                        "variants": [{"U": t.U[i], "W": t.W[i], "NS": t.NS[i], "samples": t.samples[i],
                                      "mean_us": t.mean_us[i]} for i in range(_abi.SPMV_VARIANTS)]})
        return out

    def close(self):
        if self._h:
            _abi.lib().gipc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_contexts = {}


def default_context(device=None):
    dev = torch.cuda.current_device() if device is None else torch.device(device).index
    if dev not in _contexts:
        with torch.cuda.device(dev):
            _contexts[dev] = Context()
    return _contexts[dev]


def _elements(idx, blocks, mode, lam, grad):
    if idx is None:
        return None
    _check(idx, "element indices", torch.int32, 4)
    return _abi.Elements(idx.data_ptr(), idx.shape[1], {"dense": 0, "rank1": 1, "blocks": 2}[mode],
                         blocks.data_ptr() if blocks is not None else 0,
                         lam.data_ptr() if lam is not None else 0,
                         grad.data_ptr() if grad is not None else 0)


def assemble_bsr(n, stencils=None, stencil_hess=None, stencil_mode="dense", stencil_lam=None,
                 stencil_grad=None, tets=None, tet_hess=None, tet_grad=None, mass=None, grad_base=None,
                 precision="fp64", want_grad=True, capacity=None, ctx=None, stream=None, out=None, tet_mode="dense"):
    """Assemble the BSR Hessian and the gradient (gipc_assemble_bsr).

    Returns dict(rowptr [n+1] i32, colidx [nnzb] i32, vals [nnzb, 9] f64/f32, grad [3, n] f64, nnzb).
    ``out`` may hold preallocated colidx/vals (capacity = their length) and rowptr/grad.
    ``stencil_mode`` / ``tet_mode`` name the layout the blocks come in ("dense", "blocks", and for
    stencils "rank1").
    """
    ctx = ctx or default_context()
    dev = torch.device("cuda", torch.cuda.current_device())
    prec = {"fp64": _abi.GIPC_FP64, "mixed": _abi.GIPC_MIXED}[precision]
    vdt = torch.float64 if prec == _abi.GIPC_FP64 else torch.float32
    se = _elements(stencils, stencil_hess, stencil_mode, stencil_lam, stencil_grad)
    te = _elements(tets, tet_hess, tet_mode, None, tet_grad)
    ne = (0 if stencils is None else stencils.shape[1]) + (0 if tets is None else tets.shape[1])
    out = dict(out or {})
    rowptr = out.get("rowptr")
    if rowptr is None:
        rowptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
    grad = out.get("grad") if want_grad else None
    if want_grad and grad is None:
        grad = torch.empty((3, n), dtype=torch.float64, device=dev)
    colidx, vals = out.get("colidx"), out.get("vals")
    if colidx is None:
        cap = capacity if capacity is not None else max(1, min(16 * ne + n, 6 * ne + n))
        colidx = torch.empty(cap, dtype=torch.int32, device=dev)
        vals = torch.empty((cap, 9), dtype=vdt, device=dev)
    for attempt in range(2):
        bsr = _abi.Bsr(n, 0, colidx.shape[0], rowptr.data_ptr(), colidx.data_ptr(), vals.data_ptr(), prec)
        st = _abi.call_status("gipc_assemble_bsr", ctx.handle, n,
                              ctypes.byref(se) if se is not None else None,
                              ctypes.byref(te) if te is not None else None,
                              _ptr(mass), _ptr(grad_base), ctypes.byref(bsr), _ptr(grad), _stream(stream))
        if st == _abi.GIPC_ERR_CAPACITY and attempt == 0 and bsr.nnzb > colidx.shape[0]:
            colidx = torch.empty(int(bsr.nnzb), dtype=torch.int32, device=dev)
            vals = torch.empty((int(bsr.nnzb), 9), dtype=vdt, device=dev)
            continue
        if st != _abi.GIPC_OK:
            raise GipcError("gipc_assemble_bsr", st)
        break
    nnzb = int(bsr.nnzb)
    return {"rowptr": rowptr, "colidx": colidx[:nnzb], "vals": vals[:nnzb], "grad": grad, "nnzb": nnzb,
            "n": n, "precision": precision}


def _bsr_struct(A):
    prec = {"fp64": _abi.GIPC_FP64, "mixed": _abi.GIPC_MIXED}[A["precision"]]
    return _abi.Bsr(A["n"], A["nnzb"], A["colidx"].shape[0], A["rowptr"].data_ptr(), A["colidx"].data_ptr(),
                    A["vals"].data_ptr(), prec)


def pcg(A, rhs, x0=None, fixed=None, rel_tol=1e-4, max_iter=1000, check_every=0, raise_on_nonconvergence=False,
        product="native", stop_on_indefinite=False, ctx=None, stream=None):
    """Modified block-Jacobi PCG on an assembled BSR (gipc_pcg).

    ``A`` is the dict returned by ``assemble_bsr``; ``rhs`` float64 [3, n].  Returns
    (x [3, n], iterations, delta_new / delta_0).  A mixed-precision ``A`` (float32 blocks) is
    solved with a float32 product, float32 block-Jacobi factors, preconditioned residual and
    direction, and float64 x, r and dot products.  A capped solve with rel_tol > 0
    returns its last iterate unless ``raise_on_nonconvergence``.  ``product`` selects the
    arithmetic of H c for FP64 matrices: "native" or "float_pair" (gipc_product).  With
    ``stop_on_indefinite`` a direction with c.Hc <= 0 raises GipcError (GIPC_ERR_INDEFINITE).
    """
    ctx = ctx or default_context()
    n = A["n"]
    _check(rhs, "rhs", torch.float64, 3)
    x = torch.zeros_like(rhs) if x0 is None else x0.clone()
    if fixed is not None:
        _check(fixed, "fixed", torch.uint8)
    bsr = _bsr_struct(A)
    prm = _abi.PcgParams(float(rel_tol), int(max_iter), int(check_every),
                         {"native": _abi.GIPC_PRODUCT_NATIVE, "float_pair": _abi.GIPC_PRODUCT_FLOAT_PAIR}[product],
                         _abi.GIPC_PCG_STOP_ON_INDEFINITE if stop_on_indefinite else 0)
    iters = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = _abi.call_status("gipc_pcg", ctx.handle, ctypes.byref(bsr), _ptr(rhs), _ptr(x), _ptr(fixed),
                          ctypes.byref(prm), ctypes.byref(iters), ctypes.byref(rel), _stream(stream))
    if st != _abi.GIPC_OK and not (st == _abi.GIPC_ERR_NOT_CONVERGED and not raise_on_nonconvergence):
        raise GipcError("gipc_pcg", st)
    return x, iters.value, rel.value


PCG_NOALLOC_MAX_N = 32768


def pcg_noalloc(A, rhs, x0=None, fixed=None, rel_tol=1e-4, max_iter=1000, check_every=0,
                raise_on_nonconvergence=False, stream=None):
    """``pcg`` without a context or any device allocation by the library (gipc_pcg_noalloc).

    For callers that may not allocate device memory; the solver's working vectors live in a
    fixed array of the library (systems of at most PCG_NOALLOC_MAX_N block rows).  Calls that
    overlap on the GPU share that array and race: serialise them.
    """
    n = A["n"]
    _check(rhs, "rhs", torch.float64, 3)
    x = torch.zeros_like(rhs) if x0 is None else x0.clone()
    if fixed is not None:
        _check(fixed, "fixed", torch.uint8)
    bsr = _bsr_struct(A)
    prm = _abi.PcgParams(float(rel_tol), int(max_iter), int(check_every))
    iters = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = _abi.call_status("gipc_pcg_noalloc", ctypes.byref(bsr), _ptr(rhs), _ptr(x), _ptr(fixed),
                          ctypes.byref(prm), ctypes.byref(iters), ctypes.byref(rel), _stream(stream))
    if st != _abi.GIPC_OK and not (st == _abi.GIPC_ERR_NOT_CONVERGED and not raise_on_nonconvergence):
        raise GipcError("gipc_pcg_noalloc", st)
    return x, iters.value, rel.value


def snh_params(young, poisson):
    """(mu, lambda) of the Stable neo-Hookean energy for (E, nu) (gipc_snh_params)."""
    mu, lam = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _abi.call("gipc_snh_params", float(young), float(poisson), ctypes.byref(mu), ctypes.byref(lam))
    return mu.value, lam.value


def tet_rest(rest_x, tets, density=None, ctx=None, stream=None):
    """Dm^-1 [9, T], volumes [T] and (if density) lumped masses [n] (gipc_tet_rest)."""
    ctx = ctx or default_context()
    _check(rest_x, "rest_x", torch.float64, 3)
    _check(tets, "tets", torch.int32, 4)
    n, T = rest_x.shape[1], tets.shape[1]
    dev = rest_x.device
    Dmi = torch.empty((9, T), dtype=torch.float64, device=dev)
    vol = torch.empty(T, dtype=torch.float64, device=dev)
    mass = torch.empty(n, dtype=torch.float64, device=dev) if density is not None else None
    _abi.call("gipc_tet_rest", ctx.handle, _ptr(rest_x), n, _ptr(tets), T, float(density or 0.0), _ptr(Dmi),
              _ptr(vol), _ptr(mass), _stream(stream))
    return Dmi, vol, mass


def eval_tets(x, tets, Dm_inv, vol, mu, lam, scale, precision="fp64", want=("energy", "grad", "hess"),
              layout="dense", out=None, stream=None):
    """Stable neo-Hookean energy / gradient / projected Hessian per tetrahedron (gipc_eval_tets).

    ``layout`` "dense": hess [144, T] entry-major; "blocks": hess [T, 144] holding the 16 3x3
    sub-blocks of each element contiguously (GIPC_HESS_BLOCKS)."""
    _check(x, "x", torch.float64, 3)
    _check(tets, "tets", torch.int32, 4)
    n, T = x.shape[1], tets.shape[1]
    prec = {"fp64": _abi.GIPC_FP64, "mixed": _abi.GIPC_MIXED}[precision]
    hdt = torch.float64 if prec == _abi.GIPC_FP64 else torch.float32
    out = dict(out or {})
    hm = {"dense": _abi.GIPC_HESS_DENSE, "blocks": _abi.GIPC_HESS_BLOCKS}[layout]
    shapes = {"energy": ((T,), torch.float64), "grad": ((12, T), torch.float64),
              "hess": (((144, T) if hm == _abi.GIPC_HESS_DENSE else (T, 144)), hdt)}
    for key in set(want) | set(out):
        if key not in out:
            out[key] = torch.zeros(shapes[key][0], dtype=shapes[key][1], device=x.device)
    prm = _abi.ElasticParams(float(mu), float(lam), float(scale))
    _abi.call("gipc_eval_tets", _ptr(x), n, _ptr(tets), T, _ptr(Dm_inv), _ptr(vol), ctypes.byref(prm), prec, hm,
              _ptr(out.get("energy")), _ptr(out.get("grad")), _ptr(out.get("hess")), _stream(stream))
    return out


# ------------------------------------------------------------------------- contacts and time step
class Surface:
    """Collision surface: tris int32 [3, m], edges int32 [2, e], verts int32 [v] (CUDA tensors)."""

    def __init__(self, tris, edges, verts):
        _check(tris, "tris", torch.int32, 3)
        _check(edges, "edges", torch.int32, 2)
        _check(verts, "verts", torch.int32)
        self.tris, self.edges, self.verts = tris, edges, verts

    def struct(self):
        return _abi.Surface(self.tris.data_ptr(), self.tris.shape[1], self.edges.data_ptr(), self.edges.shape[1],
                            self.verts.data_ptr(), self.verts.shape[0])


def find_contacts(x, rest_x, surface, dhat, capacity=None, ctx=None, stream=None):
    """Contact stencils int32 [4, k] and eps_x [k] at positions x (gipc_find_contacts)."""
    ctx = ctx or default_context()
    _check(x, "x", torch.float64, 3)
    _check(rest_x, "rest_x", torch.float64, 3)
    n = x.shape[1]
    srf = surface.struct()
    cap = 4096 if capacity is None else int(capacity)
    for _ in range(2):
        st = torch.empty((4, max(cap, 1)), dtype=torch.int32, device=x.device)
        eps = torch.empty(max(cap, 1), dtype=torch.float64, device=x.device)
        cnt = ctypes.c_int64(0)
        s = _abi.call_status("gipc_find_contacts", ctx.handle, _ptr(x), _ptr(rest_x), n, ctypes.byref(srf),
                             float(dhat), _ptr(st), _ptr(eps), cap, ctypes.byref(cnt), _stream(stream))
        if s == _abi.GIPC_OK:
            k = cnt.value
            return st[:, :k].contiguous(), eps[:k].clone()
        if s != _abi.GIPC_ERR_CAPACITY or capacity is not None:
            raise GipcError("gipc_find_contacts", s)
        cap = cnt.value
    raise GipcError("gipc_find_contacts", s)


def ccd_max_step(x, d, surface, slack=0.1, ctx=None, stream=None):
    """Largest feasible step in [0, 1] along d by additive CCD (gipc_ccd_max_step)."""
    ctx = ctx or default_context()
    _check(x, "x", torch.float64, 3)
    _check(d, "d", torch.float64, 3)
    a = ctypes.c_double(0.0)
    srf = surface.struct()
    _abi.call("gipc_ccd_max_step", ctx.handle, _ptr(x), _ptr(d), x.shape[1], ctypes.byref(srf), float(slack),
              ctypes.byref(a), _stream(stream))
    return a.value


class Scene:
    """Device-resident scene of tetrahedral meshes for newton_step.

    ``x`` float64 [3, n] rest (= initial) positions, ``tets`` int32 [4, T], ``surface`` a Surface,
    ``fixed`` bool/uint8 [n] or None, ``l`` the bounding-box diagonal (computed if None)."""

    def __init__(self, rest_x, tets, surface, density, fixed=None, l=None, ctx=None):
        _check(rest_x, "rest_x", torch.float64, 3)
        self.rest_x = rest_x
        self.tets = tets
        self.surface = surface
        self.Dm_inv, self.vol, self.mass = tet_rest(rest_x, tets, density, ctx=ctx)
        n = rest_x.shape[1]
        self.fixed = (fixed.to(device=rest_x.device, dtype=torch.uint8).contiguous() if fixed is not None
                      else None)
        if l is None:
            ext = rest_x.max(dim=1).values - rest_x.min(dim=1).values
            l = float(torch.linalg.norm(ext))
        self.l = float(l)
        self.n = n

    def struct(self):
        return _abi.Scene(self.n, self.rest_x.data_ptr(), self.tets.data_ptr(), self.tets.shape[1],
                          self.Dm_inv.data_ptr(), self.vol.data_ptr(), self.mass.data_ptr(),
                          self.fixed.data_ptr() if self.fixed is not None else None, self.surface.struct(), self.l)


def newton_step(scene, x, v, dt, mu, lam, dhat, kappa, gravity=(0.0, 0.0, -9.81), d_thr_ratio=0.1, eps_d=1e-2,
                pcg_tol=1e-4, max_pcg=500, max_newton=50, max_ls=30, precision="fp64", hess_mode="dense",
                ctx=None, stream=None):
    """One implicit time step; updates x and v in place and returns a stats dict (gipc_newton_step)."""
    ctx = ctx or default_context()
    _check(x, "x", torch.float64, 3)
    _check(v, "v", torch.float64, 3)
    prm = _abi.StepParams()
    prm.dt = float(dt)
    prm.gravity[:] = [float(g) for g in gravity]
    prm.elastic = _abi.ElasticParams(float(mu), float(lam), 0.0)
    prm.barrier = _abi.BarrierParams(float(dhat), float(kappa), float(d_thr_ratio))
    prm.eps_d, prm.pcg_tol = float(eps_d), float(pcg_tol)
    prm.max_pcg, prm.max_newton, prm.max_ls = int(max_pcg), int(max_newton), int(max_ls)
    prm.prec = {"fp64": _abi.GIPC_FP64, "mixed": _abi.GIPC_MIXED}[precision]
    prm.hess_mode = {"dense": _abi.GIPC_HESS_DENSE, "rank1": _abi.GIPC_HESS_RANK1}[hess_mode]
    stats = _abi.StepStats()
    sc = scene.struct()
    _abi.call("gipc_newton_step", ctx.handle, ctypes.byref(sc), _ptr(x), _ptr(v), ctypes.byref(prm),
              ctypes.byref(stats), _stream(stream))
    return {f: getattr(stats, f) for f, _ in _abi.StepStats._fields_}


class SceneBatch:
    """Independent scenes concatenated for newton_step_batch.

    ``scenes``: list of dicts with numpy arrays x (3, n_k), tets (4, T_k), tris (3, m_k),
    edges (2, e_k), verts (v_k,) in the scene's own vertex ids, optional fixed (n_k,) and l
    (bounding-box diagonal; computed if absent).  Vertex ids are offset so scene k owns
    [vert_off[k], vert_off[k+1]); all lists stay ordered by scene."""

    def __init__(self, scenes, density, device="cuda", ctx=None):
        import numpy as np
        off = [0]
        for sc in scenes:
            off.append(off[-1] + sc["x"].shape[1])
        self.vert_off = np.array(off, dtype=np.int64)

        def cat(key, rows):
            parts = [np.asarray(sc[key], dtype=np.int64) + o for sc, o in zip(scenes, off)]
            a = np.concatenate(parts, axis=-1) if parts else np.zeros((rows, 0), np.int64)
            return torch.tensor(np.ascontiguousarray(a.astype(np.int32)), device=device)

        x = np.concatenate([np.asarray(sc["x"], dtype=np.float64) for sc in scenes], axis=1)
        fixed = np.concatenate([np.asarray(sc.get("fixed", np.zeros(sc["x"].shape[1])), dtype=np.uint8)
                                for sc in scenes])
        ls = []
        for sc in scenes:
            if sc.get("l") is not None:
                ls.append(float(sc["l"]))
            else:
                ext = sc["x"].max(axis=1) - sc["x"].min(axis=1)
                ls.append(float(np.linalg.norm(ext)))
        self.l = np.array(ls, dtype=np.float64)
        tets = cat("tets", 4)
        surface = Surface(cat("tris", 3), cat("edges", 2), cat("verts", 1).reshape(-1).contiguous())
        self.scene = Scene(torch.tensor(x, device=device), tets, surface, density,
                           fixed=torch.tensor(fixed, device=device), l=float(self.l.max()), ctx=ctx)
        self.nscenes = len(scenes)

    def split(self, a):
        """Per-scene views of a [3, n] array."""
        return [a[:, self.vert_off[k]:self.vert_off[k + 1]] for k in range(self.nscenes)]

    def struct(self):
        self._keep = (self.vert_off.copy(), self.l.copy())
        return _abi.SceneBatch(self.scene.struct(), self.nscenes, self._keep[0].ctypes.data, self._keep[1].ctypes.data)


def newton_step_batch(batch, x, v, dt, mu, lam, dhat, kappa, gravity=(0.0, 0.0, -9.81), d_thr_ratio=0.1, eps_d=1e-2,
                      pcg_tol=1e-4, max_pcg=500, max_newton=50, max_ls=30, precision="fp64", hess_mode="dense",
                      ctx=None, stream=None):
    """One implicit time step of every scene of a SceneBatch; updates x and v in place and returns a
    list of per-scene stats dicts (gipc_newton_step_batch)."""
    ctx = ctx or default_context()
    _check(x, "x", torch.float64, 3)
    _check(v, "v", torch.float64, 3)
    prm = _abi.StepParams()
    prm.dt = float(dt)
    prm.gravity[:] = [float(g) for g in gravity]
    prm.elastic = _abi.ElasticParams(float(mu), float(lam), 0.0)
    prm.barrier = _abi.BarrierParams(float(dhat), float(kappa), float(d_thr_ratio))
    prm.eps_d, prm.pcg_tol = float(eps_d), float(pcg_tol)
    prm.max_pcg, prm.max_newton, prm.max_ls = int(max_pcg), int(max_newton), int(max_ls)
    prm.prec = {"fp64": _abi.GIPC_FP64, "mixed": _abi.GIPC_MIXED}[precision]
    prm.hess_mode = {"dense": _abi.GIPC_HESS_DENSE, "rank1": _abi.GIPC_HESS_RANK1}[hess_mode]
    stats = (_abi.StepStats * batch.nscenes)()
    b = batch.struct()
    _abi.call("gipc_newton_step_batch", ctx.handle, ctypes.byref(b), _ptr(x), _ptr(v), ctypes.byref(prm), stats,
              _stream(stream))
    return [{f: getattr(s, f) for f, _ in _abi.StepStats._fields_} for s in stats]


# ------------------------------------------------------------------------- differentiation
def _step_params(dt, mu, lam, dhat, kappa, gravity=(0.0, 0.0, -9.81), d_thr_ratio=0.1, eps_d=1e-2, pcg_tol=1e-4,
                 max_pcg=500, max_newton=50, max_ls=30, precision="fp64", hess_mode="dense"):
    prm = _abi.StepParams()
    prm.dt = float(dt)
    prm.gravity[:] = [float(g) for g in gravity]
    prm.elastic = _abi.ElasticParams(float(mu), float(lam), 0.0)
    prm.barrier = _abi.BarrierParams(float(dhat), float(kappa), float(d_thr_ratio))
    prm.eps_d, prm.pcg_tol = float(eps_d), float(pcg_tol)
    prm.max_pcg, prm.max_newton, prm.max_ls = int(max_pcg), int(max_newton), int(max_ls)
    prm.prec = {"fp64": _abi.GIPC_FP64, "mixed": _abi.GIPC_MIXED}[precision]
    prm.hess_mode = {"dense": _abi.GIPC_HESS_DENSE, "rank1": _abi.GIPC_HESS_RANK1}[hess_mode]
    return prm


def scatter_elements(n, stencils=None, stencil_vec=None, tets=None, tet_vec=None, base=None, ctx=None, stream=None):
    """out [3, n] = base + per-vertex sums of element vectors [12, count] (gipc_scatter_elements)."""
    ctx = ctx or default_context()
    dev = (stencils if stencils is not None else tets).device
    out = torch.empty((3, n), dtype=torch.float64, device=dev)
    se = _abi.Elements(stencils.data_ptr(), stencils.shape[1], 0, None, None, stencil_vec.data_ptr()) \
        if stencils is not None else None
    te = _abi.Elements(tets.data_ptr(), tets.shape[1], 0, None, None, tet_vec.data_ptr()) if tets is not None else None
    _abi.call("gipc_scatter_elements", ctx.handle, n, ctypes.byref(se) if se else None,
              ctypes.byref(te) if te else None, _ptr(base), _ptr(out), _stream(stream))
    return out


def potential_derivs(scene, x, stencils, eps_x, dhat, kappa, mu, lam, scale, xt=None, u=None, want=("energy", "grad"),
                     ctx=None, stream=None):
    """Exact I(x), dI/dx and (d2I/dx2) u of the incremental potential for a contact list
    (gipc_potential_derivs).  Returns a dict with the requested keys (energy, grad, Hu)."""
    ctx = ctx or default_context()
    _check(x, "x", torch.float64, 3)
    n = x.shape[1]
    k = stencils.shape[1] if stencils is not None else 0
    bp = _abi.BarrierParams(float(dhat), float(kappa), 0.1)
    ep = _abi.ElasticParams(float(mu), float(lam), float(scale))
    e = ctypes.c_double(0.0)
    out = {}
    grad = torch.empty((3, n), dtype=torch.float64, device=x.device) if "grad" in want else None
    Hu = torch.empty((3, n), dtype=torch.float64, device=x.device) if u is not None else None
    sc = scene.struct()
    _abi.call("gipc_potential_derivs", ctx.handle, ctypes.byref(sc), _ptr(x), _ptr(xt),
              _ptr(stencils) if k else None, _ptr(eps_x) if k else None, k, ctypes.byref(bp), ctypes.byref(ep),
              _ptr(u), ctypes.byref(e) if "energy" in want else None, _ptr(grad), _ptr(Hu), _stream(stream))
    if "energy" in want:
        out["energy"] = e.value
    if grad is not None:
        out["grad"] = grad
    if Hu is not None:
        out["Hu"] = Hu
    return out


def potential_hessian(scene, x, stencils, eps_x, dhat, kappa, mu, lam, scale, ctx=None, stream=None):
    """The exact Hessian (mass + element Hessians) as a BSR dict (gipc_potential_hessian)."""
    ctx = ctx or default_context()
    n = x.shape[1]
    k = stencils.shape[1] if stencils is not None else 0
    bp = _abi.BarrierParams(float(dhat), float(kappa), 0.1)
    ep = _abi.ElasticParams(float(mu), float(lam), float(scale))
    rowptr = torch.empty(n + 1, dtype=torch.int32, device=x.device)
    cap = 64 * n + 1024
    sc = scene.struct()
    for _ in range(2):
        colidx = torch.empty(cap, dtype=torch.int32, device=x.device)
        vals = torch.empty(cap * 9, dtype=torch.float64, device=x.device)
        b = _abi.Bsr(n, 0, cap, rowptr.data_ptr(), colidx.data_ptr(), vals.data_ptr(), _abi.GIPC_FP64)
        s = _abi.call_status("gipc_potential_hessian", ctx.handle, ctypes.byref(sc), _ptr(x),
                             _ptr(stencils) if k else None, _ptr(eps_x) if k else None, k, ctypes.byref(bp),
                             ctypes.byref(ep), ctypes.byref(b), _stream(stream))
        if s == _abi.GIPC_OK:
            return {"n": n, "nnzb": b.nnzb, "rowptr": rowptr, "colidx": colidx[:b.nnzb],
                    "vals": vals[:9 * b.nnzb].reshape(-1, 3, 3), "prec": "fp64"}
        if s != _abi.GIPC_ERR_CAPACITY:
            raise GipcError("gipc_potential_hessian", s)
        cap = b.nnzb + 16
    raise GipcError("gipc_potential_hessian", s)


def adjoint_step(scene, x_new, x_old, v_old, adj_x_new, adj_v_new, dt, mu, lam, dhat, kappa, pcg_tol=1e-20,
                 max_pcg=20000, ctx=None, stream=None):
    """Adjoint of one converged implicit step (gipc_adjoint_step): returns
    (dL/dx_old, dL/dv_old, E dL/dE of this step, adjoint PCG iterations).  The adjoint solve stops
    once r.P^-1 r < pcg_tol times its start (squared norms: 1e-20 is a 1e-10 smaller residual) or
    after max_pcg iterations; GipcError if it does not reach pcg_tol."""
    ctx = ctx or default_context()
    prm = _step_params(dt, mu, lam, dhat, kappa, pcg_tol=pcg_tol, max_pcg=max_pcg)
    ax = torch.empty_like(x_new)
    av = torch.empty_like(x_new)
    le = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    sc = scene.struct()
    st = _abi.call_status("gipc_adjoint_step", ctx.handle, ctypes.byref(sc), _ptr(x_new), _ptr(x_old), _ptr(v_old),
                          ctypes.byref(prm), _ptr(adj_x_new), _ptr(adj_v_new), _ptr(ax), _ptr(av), ctypes.byref(le),
                          ctypes.byref(it), _stream(stream))
    if st != _abi.GIPC_OK:
        raise GipcError("gipc_adjoint_step", st)
    return ax, av, le.value, it.value


class _PotentialGrad(torch.autograd.Function):
    """x -> dI/dx; its backward is the exact Hessian-vector product (matrix free)."""

    @staticmethod
    def forward(ctx_, x, args):
        ctx_.save_for_backward(x)
        ctx_.args = args
        return potential_derivs(args["scene"], x.detach().contiguous(), args["stencils"], args["eps_x"], args["dhat"],
                                args["kappa"], args["mu"], args["lam"], args["scale"], xt=args["xt"],
                                want=("grad",))["grad"]

    @staticmethod
    def backward(ctx_, gout):
        (x,) = ctx_.saved_tensors
        a = ctx_.args
        Hu = potential_derivs(a["scene"], x.detach().contiguous(), a["stencils"], a["eps_x"], a["dhat"], a["kappa"],
                              a["mu"], a["lam"], a["scale"], xt=a["xt"], u=gout.contiguous(), want=())["Hu"]
        return Hu, None


class IncrementalPotential(torch.autograd.Function):
    """I(x) of one implicit step for a fixed contact list: backward is the exact gradient kernel,
    double backward the exact Hessian-vector kernel (use torch.autograd.grad(..., create_graph=True))."""

    @staticmethod
    def forward(ctx_, x, args):
        ctx_.save_for_backward(x)
        ctx_.args = args
        e = potential_derivs(args["scene"], x.detach().contiguous(), args["stencils"], args["eps_x"], args["dhat"],
                             args["kappa"], args["mu"], args["lam"], args["scale"], xt=args["xt"],
                             want=("energy",))["energy"]
        return torch.tensor(e, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx_, gout):
        (x,) = ctx_.saved_tensors
        g = _PotentialGrad.apply(x, ctx_.args)
        return gout * g, None


def incremental_potential(x, scene, xt, stencils, eps_x, dhat, kappa, mu, lam, scale):
    """Differentiable I(x) (see IncrementalPotential)."""
    args = dict(scene=scene, xt=xt, stencils=stencils, eps_x=eps_x, dhat=dhat, kappa=kappa, mu=mu, lam=lam,
                scale=scale)
    return IncrementalPotential.apply(x, args)


def newton_polish(scene, x, v, x_old, v_old, dt, mu, lam, dhat, kappa, eps_polish=1e-13, max_iters=8,
                  gravity=(0.0, 0.0, -9.81), d_thr_ratio=0.1, pcg_tol=1e-24, max_pcg=20000, ctx=None, stream=None):
    """Exact-Hessian Newton refinement of a step of newton_step (gipc_newton_polish): updates x and
    v in place; returns (iterations, last max|d| / (l dt)).  GipcError if eps_polish is not met."""
    ctx = ctx or default_context()
    for t, nm in ((x, "x"), (v, "v"), (x_old, "x_old"), (v_old, "v_old")):
        _check(t, nm, torch.float64, 3)
    prm = _step_params(dt, mu, lam, dhat, kappa, gravity=gravity, d_thr_ratio=d_thr_ratio, pcg_tol=pcg_tol,
                       max_pcg=max_pcg)
    it = ctypes.c_int(0)
    step = ctypes.c_double(0.0)
    sc = scene.struct()
    _abi.call("gipc_newton_polish", ctx.handle, ctypes.byref(sc), _ptr(x), _ptr(v), _ptr(x_old), _ptr(v_old),
              ctypes.byref(prm), float(eps_polish), int(max_iters), ctypes.byref(it), ctypes.byref(step),
              _stream(stream))
    return it.value, step.value


_POLISH_KEYS = ("gravity", "d_thr_ratio")


def simulate(scene, x0, v0, steps, dt, mu, lam, dhat, kappa, stats=None, polish=None, **kw):
    """Implicit steps with the state checkpointed before each step: returns (x, v, checkpoints),
    checkpoints = [(x_t, v_t)] for t = 0 .. steps (the last one is the result).  Each step's
    statistics are appended to `stats` when it is a list.  With `polish` (a dict of newton_polish
    keyword arguments) every step is refined by newton_polish after newton_step, so the adjoint's
    condition grad I(x_{t+1}) = 0 holds to that tolerance; the refinement's iteration count and
    final step are added to the step's statistics."""
    x, v = x0.clone(), v0.clone()
    cps = [(x.clone(), v.clone())]
    for _ in range(steps):
        st = newton_step(scene, x, v, dt=dt, mu=mu, lam=lam, dhat=dhat, kappa=kappa, **kw)
        if polish is not None:
            pk = {k: kw[k] for k in _POLISH_KEYS if k in kw}
            pk.update(polish)
            st["polish_iters"], st["polish_step"] = newton_polish(scene, x, v, cps[-1][0], cps[-1][1], dt, mu, lam, dhat,
                                                                  kappa, **pk)
        if stats is not None:
            stats.append(st)
        cps.append((x.clone(), v.clone()))
    return x, v, cps


def adjoint(scene, checkpoints, dL_dx_final, dL_dv_final, dt, mu, lam, dhat, kappa, **kw):
    """Implicit adjoint through the checkpointed steps (newest first): returns
    (dL/dx0, dL/dv0, dL/dE * E, adjoint PCG iterations per step)."""
    ax, av = dL_dx_final, dL_dv_final
    logE = 0.0
    its = []
    for t in range(len(checkpoints) - 1, 0, -1):
        x_new = checkpoints[t][0]
        x_old, v_old = checkpoints[t - 1]
        ax, av, le, it = adjoint_step(scene, x_new, x_old, v_old, ax, av, dt, mu, lam, dhat, kappa, **kw)
        logE += le
        its.append(it)
    return ax, av, logE, its
