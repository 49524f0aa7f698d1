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

__all__ = ["compute_eps_x", "eval_stencils", "GipcError", "FLAG_ACTIVE", "FLAG_FILTERED",
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
    hess [144, k] (dense) or [12, k] (rank1: w), lam [k] (rank1), flags [k] u8.
    Hessian tensors are float64 for precision='fp64' and float32 for 'mixed'.
    ``out`` may supply preallocated tensors under the same keys.
    """
    _check(x, "x", torch.float64, 3)
    _check(stencils, "stencils", torch.int32, 4)
    n, k = x.shape[1], stencils.shape[1]
    if eps_x is not None:
        _check(eps_x, "eps_x", torch.float64)
    prec = {"fp64": _abi.GIPC_FP64, "mixed": _abi.GIPC_MIXED}[precision]
    md = {"dense": _abi.GIPC_HESS_DENSE, "rank1": _abi.GIPC_HESS_RANK1}[mode]
    hdt = torch.float64 if prec == _abi.GIPC_FP64 else torch.float32
    dev = x.device
    out = dict(out or {})
    want = set(want) | set(out)
    if md == _abi.GIPC_HESS_RANK1 and "hess" in want:
        want.add("lam")
    shapes = {"energy": ((k,), torch.float64), "grad": ((12, k), torch.float64),
              "hess": (((144 if md == _abi.GIPC_HESS_DENSE else 12), k), hdt),
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
