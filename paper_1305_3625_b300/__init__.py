"""Python binding of the fftconv C ABI (include/fftconv.h).

Argument marshalling only: every step of the FFT convolution and of the CG
solve runs in the CUDA kernels of libfftconv.so.  Tensors are torch CUDA
tensors (torch provides device memory and streams); their data pointers and
the current stream are passed straight to the C entry points of the same
names.  If the shared library is missing this module raises at import: there
is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

FC_OK = 0
FC_EINVAL = -1
FC_ENOMEM = -2
FC_EBUDGET = -3
FC_ENOCONV = -4
FC_ENANINF = -5
FC_ETIMEOUT = -6
FC_ECUDA = -7
FC_ENOTFOUND = -8
FC_F32 = 1
FC_F64 = 2
FC_GREEN_POINT = 0
FC_GREEN_CELL = 1
FC_MODE_F64 = 0
FC_MODE_MIXED = 1
FC_REQ_BORROW = 1
FC_SHAPES_APPLY = 0
FC_SHAPES_SOLVE = 1
FC_SHAPES_BATCH = 2
FC_INJECT_ALLOC = 1
FC_INJECT_BARRIER = 2
FC_INJECT_TMA = 3

STATUS_NAMES = {0: "FC_OK", -1: "FC_EINVAL", -2: "FC_ENOMEM", -3: "FC_EBUDGET", -4: "FC_ENOCONV",
                -5: "FC_ENANINF", -6: "FC_ETIMEOUT", -7: "FC_ECUDA", -8: "FC_ENOTFOUND"}


class FcError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        msg = f"{what}: {STATUS_NAMES.get(code, code)}"
        err = _lib.fc_last_error().decode() if _lib is not None else ""
        if err:
            msg += f" ({err})"
        super().__init__(msg)


class cg_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mode", ctypes.c_int),
                ("refine_every", ctypes.c_int), ("max_refine", ctypes.c_int),
                ("inner_rtol", ctypes.c_double), ("x0_zero", ctypes.c_int), ("precond", ctypes.c_int),
                ("warm_resid", ctypes.c_int)]


class cg_tune(ctypes.Structure):
    _fields_ = [("shape_rfwd", ctypes.c_int), ("shape_col", ctypes.c_int), ("shape_rinv", ctypes.c_int),
                ("no_autotune", ctypes.c_int), ("shape_pers", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class cg_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("refinements", ctypes.c_int),
                ("resid_updated", ctypes.c_int), ("zero_start", ctypes.c_int), ("fp64_products", ctypes.c_int),
                ("true_rel_resid", ctypes.c_double),
                ("bnorm", ctypes.c_double), ("latency_s", ctypes.c_double), ("run_s", ctypes.c_double)]

    def as_dict(self):
        return {"status": self.status, "iters": self.iters, "refinements": self.refinements,
                "resid_updated": self.resid_updated, "zero_start": self.zero_start,
                "fp64_products": self.fp64_products,
                "true_rel_resid": self.true_rel_resid, "bnorm": self.bnorm,
                "latency_s": self.latency_s, "run_s": self.run_s}


class cg_batch_group(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("nb", ctypes.c_int), ("s", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("r", ctypes.c_void_p)]


class fc_run_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("steps_done", ctypes.c_int), ("iters", ctypes.c_longlong),
                ("fp64_products", ctypes.c_int), ("resid_updated", ctypes.c_int), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cg_request(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("mode", ctypes.c_int), ("rtol", ctypes.c_double),
                ("s", ctypes.c_void_p), ("b", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("tag", ctypes.c_uint64), ("precond", ctypes.c_int), ("flags", ctypes.c_int)]


LIB_PATH = _build.LIB


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_1305_3625_b300.build` "
                          "(or __graft_entry__.build()) first")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    lib.fc_version.restype = ctypes.c_char_p
    lib.fc_last_error.restype = ctypes.c_char_p
    lib.fftconv_plan_create.argtypes = [ctypes.POINTER(vp), i, i, ctypes.POINTER(cg_tune)]
    lib.fftconv_plan_create_green.argtypes = [ctypes.POINTER(vp), i, i, i, ctypes.POINTER(cg_tune)]
    ip3 = ctypes.c_int * 3
    lib.fftconv_plan_shapes.argtypes = [vp, i, ip3, ip3, ip3, ip3]
    ipt = ctypes.POINTER(ctypes.c_int)
    lib.fftconv_plan_solver.argtypes = [vp, i, ipt, ipt, ipt, ipt]
    lib.fftconv_plan_shape_set.argtypes = [vp, i, i, ip3, ip3, ip3, ipt]
    lib.fftconv_plan_destroy.argtypes = [vp]
    lib.fftconv_plan_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                      ctypes.POINTER(sz)]
    lib.fftconv_apply.argtypes = [vp, vp, vp, vp]
    lib.fftconv_apply_prec.argtypes = [vp, i, vp, vp, vp]
    lib.fftconv_cg_product.argtypes = [vp, i, vp, vp, vp, vp, ctypes.POINTER(d), vp]
    lib.cg_solve.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(cg_opts), ctypes.POINTER(cg_result), vp]
    lib.cg_solve_batch.argtypes = [vp, i, vp, vp, vp, vp, ctypes.POINTER(cg_opts), ctypes.POINTER(cg_result), vp]
    lib.cg_solve_groups.argtypes = [i, ctypes.POINTER(cg_batch_group), ctypes.POINTER(cg_opts), vp]
    lib.fc_masked_step.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.fc_front.argtypes = [vp, vp, vp, vp, vp]
    lib.fftconv_plan_sync_mode.argtypes = [vp, i]
    lib.fc_fracture_run.argtypes = [vp, vp, vp, vp, vp, vp, i, ctypes.POINTER(cg_opts), vp, vp,
                                    ctypes.POINTER(fc_run_result), vp]
    lib.fc_fracture_run_batch.argtypes = [vp, i, vp, vp, vp, vp, vp, i, ctypes.POINTER(cg_opts), vp, vp,
                                          ctypes.POINTER(fc_run_result), vp]
    lib.fc_masked_step_static.argtypes = [ctypes.c_int64, vp, vp, vp, vp, vp]
    lib.cg_server_create.argtypes = [ctypes.POINTER(vp), sz, i, vp]
    lib.cg_batch_submit.argtypes = [vp, ctypes.POINTER(cg_request), ctypes.POINTER(ctypes.c_uint64)]
    lib.cg_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(cg_result), ctypes.POINTER(i)]
    lib.cg_server_stats.argtypes = [vp, ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.cg_server_batches.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(i)]
    lib.cg_server_destroy.argtypes = [vp]
    lib.cg_server_reserve.argtypes = [vp, i, i]
    lib.fc_mem_stats.argtypes = [ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(ctypes.c_longlong), i]
    lib.fftconv_plan_check_guards.argtypes = [vp, ctypes.POINTER(i)]
    lib.fc_debug_inject.argtypes = [vp, i, ctypes.c_longlong]
    return lib


_lib = _load()


def fc_version() -> str:
    return _lib.fc_version().decode()


def fc_last_error() -> str:
    return _lib.fc_last_error().decode()


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, dtype, n, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Owning handle of an fftconv_plan (destroyed with the object)."""

    def __init__(self, handle, L, prec):
        self._h = handle
        self.L = L
        self.prec = prec
        Li, Mi, pi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nb = ctypes.c_size_t()
        _lib.fftconv_plan_info(self._h, ctypes.byref(Li), ctypes.byref(Mi), ctypes.byref(pi),
                               ctypes.byref(nb))
        self.M = Mi.value
        self.device_bytes = nb.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.fftconv_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fftconv_plan_create(L: int, prec: int = FC_F32 | FC_F64, shapes=None, no_autotune: bool = False,
                        persistent=None, green: int = None) -> Plan:
    """shapes: optional (pass A, pass B, pass C) compiled-shape indices (0-based)
    to force instead of the tuned choice; persistent: index of the persistent
    inner-CG kernel to force, or -1 for the per-pass graph loop; green:
    FC_GREEN_POINT (default) or FC_GREEN_CELL, the Green's function of Eq. 1c."""
    h = ctypes.c_void_p()
    tune = None
    if shapes is not None or no_autotune or persistent is not None:
        tune = cg_tune()
        if shapes is not None:
            tune.shape_rfwd, tune.shape_col, tune.shape_rinv = (int(k) + 1 for k in shapes)
        tune.no_autotune = int(bool(no_autotune))
        if persistent is not None:
            tune.shape_pers = -1 if persistent < 0 else int(persistent) + 1
    if green is None:
        rc = _lib.fftconv_plan_create(ctypes.byref(h), int(L), int(prec),
                                      ctypes.byref(tune) if tune is not None else None)
    else:
        rc = _lib.fftconv_plan_create_green(ctypes.byref(h), int(L), int(prec), int(green),
                                            ctypes.byref(tune) if tune is not None else None)
    if rc != FC_OK:
        raise FcError(rc, "fftconv_plan_create")
    return Plan(h, int(L), int(prec))


def fftconv_plan_create_green(L: int, prec: int = FC_F32 | FC_F64, green: int = FC_GREEN_POINT,
                              **kw) -> Plan:
    """fftconv_plan_create with the Green's function of Eq. 1c chosen."""
    return fftconv_plan_create(L, prec, green=green, **kw)


def fftconv_plan_destroy(plan: Plan) -> None:
    plan.close()


def fftconv_apply_prec(plan: Plan, prec: int, x, y, stream=None) -> None:
    dt = torch.float32 if prec == FC_F32 else torch.float64
    n = plan.L * plan.L
    rc = _lib.fftconv_apply_prec(plan.handle, int(prec), _ptr(x, dt, n, "x"), _ptr(y, dt, n, "y"),
                                 _stream(stream))
    if rc != FC_OK:
        raise FcError(rc, "fftconv_apply_prec")


def fftconv_apply(plan: Plan, x, y, stream=None) -> None:
    prec = FC_F32 if x.dtype == torch.float32 else FC_F64
    fftconv_apply_prec(plan, prec, x, y, stream)


def fftconv_cg_product(plan: Plan, prec: int, p, r, s, q, stream=None):
    """q = C p + s p as the CG passes form it; returns their (p.q, r.q, q.q)."""
    dt = torch.float32 if prec == FC_F32 else torch.float64
    n = plan.L * plan.L
    dots = (ctypes.c_double * 3)()
    rc = _lib.fftconv_cg_product(plan.handle, int(prec), _ptr(p, dt, n, "p"), _ptr(r, dt, n, "r"),
                                 _ptr(s, dt, n, "s"), _ptr(q, dt, n, "q"), dots, _stream(stream))
    if rc != FC_OK:
        raise FcError(rc, "fftconv_cg_product")
    return tuple(dots)


def _opts(rtol, mode, max_iter=0, refine_every=0, max_refine=0, inner_rtol=0.0, x0_zero=False, precond=False,
          warm_resid=True):
    return cg_opts(rtol=float(rtol), max_iter=int(max_iter), mode=int(mode),
                   refine_every=int(refine_every), max_refine=int(max_refine),
                   inner_rtol=float(inner_rtol), x0_zero=int(bool(x0_zero)), precond=int(bool(precond)),
                   warm_resid=0 if warm_resid else -1)


def cg_solve(plan: Plan, s, b, x, mask=None, rtol: float = 1e-10, mode: int = FC_MODE_F64,
             max_iter: int = 0, refine_every: int = 0, max_refine: int = 0,
             inner_rtol: float = 0.0, x0_zero: bool = False, precond: bool = False, stream=None,
             check: bool = False, warm_resid: bool = True) -> dict:
    """Solve P (C + S) P x = P b in place in x; returns the cg_result fields.
    warm_resid=False always recomputes the first true residual (no update from
    the plan's previous solve)."""
    n = plan.L * plan.L
    o = _opts(rtol, mode, max_iter, refine_every, max_refine, inner_rtol, x0_zero, precond, warm_resid)
    r = cg_result()
    rc = _lib.cg_solve(plan.handle, _ptr(s, torch.float64, n, "s"), _ptr(b, torch.float64, n, "b"),
                       _ptr(x, torch.float64, n, "x"), _ptr(mask, torch.uint8, n, "mask"),
                       ctypes.byref(o), ctypes.byref(r), _stream(stream))
    if rc in (FC_EINVAL, FC_ECUDA, FC_ENOMEM) or (check and rc != FC_OK):
        raise FcError(rc, "cg_solve")
    out = r.as_dict()
    out["rc"] = rc
    return out


def cg_solve_batch(plan: Plan, s, b, x, mask=None, rtol: float = 1e-10, mode: int = FC_MODE_F64,
                   max_iter: int = 0, refine_every: int = 0, max_refine: int = 0, inner_rtol: float = 0.0,
                   x0_zero: bool = False, precond: bool = False, stream=None, check: bool = False):
    """nb solves of the plan's size in one launch: s, b, x (float64) and mask
    (uint8, or None) hold nb*L*L elements, problem k at offset k*L*L (an
    (nb, L, L) or (nb, L*L) tensor).  Returns (rc, list of nb result dicts)."""
    n = plan.L * plan.L
    if not isinstance(x, torch.Tensor) or x.numel() % n or x.numel() == 0:
        raise ValueError(f"x must hold a positive multiple of {n} elements")
    nb = x.numel() // n
    o = _opts(rtol, mode, max_iter, refine_every, max_refine, inner_rtol, x0_zero, precond)
    rs = (cg_result * nb)()
    rc = _lib.cg_solve_batch(plan.handle, nb, _ptr(s, torch.float64, nb * n, "s"),
                             _ptr(b, torch.float64, nb * n, "b"), _ptr(x, torch.float64, nb * n, "x"),
                             _ptr(mask, torch.uint8, nb * n, "mask"), ctypes.byref(o), rs, _stream(stream))
    if rc in (FC_EINVAL, FC_ECUDA, FC_ENOMEM) or (check and rc != FC_OK):
        raise FcError(rc, "cg_solve_batch")
    return rc, [r.as_dict() for r in rs]


def cg_solve_groups(groups, rtol: float = 1e-10, mode: int = FC_MODE_F64, max_iter: int = 0,
                    refine_every: int = 0, max_refine: int = 0, inner_rtol: float = 0.0, x0_zero: bool = False,
                    precond: bool = False, stream=None, check: bool = False):
    """Batches of several sizes at once.  groups: list of (plan, s, b, x, mask)
    with the layout of cg_solve_batch, one distinct plan per group.  Returns
    (rc, list of per-group lists of result dicts)."""
    arr = (cg_batch_group * len(groups))()
    keep = []
    for k, (plan, s, b, x, mask) in enumerate(groups):
        n = plan.L * plan.L
        if not isinstance(x, torch.Tensor) or x.numel() % n or x.numel() == 0:
            raise ValueError(f"group {k}: x must hold a positive multiple of {n} elements")
        nb = x.numel() // n
        rs = (cg_result * nb)()
        keep.append(rs)
        g = arr[k]
        def val(ptr):
            return None if ptr is None else ptr.value
        g.plan = plan.handle.value
        g.nb = nb
        g.s = val(_ptr(s, torch.float64, nb * n, "s"))
        g.b = val(_ptr(b, torch.float64, nb * n, "b"))
        g.x = val(_ptr(x, torch.float64, nb * n, "x"))
        g.mask = val(_ptr(mask, torch.uint8, nb * n, "mask"))
        g.r = ctypes.cast(rs, ctypes.c_void_p).value
    o = _opts(rtol, mode, max_iter, refine_every, max_refine, inner_rtol, x0_zero, precond)
    rc = _lib.cg_solve_groups(len(groups), arr, ctypes.byref(o), _stream(stream))
    if rc in (FC_EINVAL, FC_ECUDA, FC_ENOMEM) or (check and rc != FC_OK):
        raise FcError(rc, "cg_solve_groups")
    return rc, [[r.as_dict() for r in rs] for rs in keep]


def fc_masked_step(plan: Plan, t, mask, x, removed, stream=None) -> None:
    n = plan.L * plan.L
    rc = _lib.fc_masked_step(plan.handle, _ptr(t, torch.float64, n, "t"),
                             _ptr(mask, torch.uint8, n, "mask"), _ptr(x, torch.float64, n, "x"),
                             _ptr(removed, torch.int64, 1, "removed"), _stream(stream))
    if rc != FC_OK:
        raise FcError(rc, "fc_masked_step")


def fftconv_plan_sync_mode(plan: Plan, blocking: bool) -> None:
    """Waits on this plan spin (False, default) or block the thread (True)."""
    rc = _lib.fftconv_plan_sync_mode(plan.handle, int(blocking))
    if rc != FC_OK:
        raise FcError(rc, "fftconv_plan_sync_mode")


def fc_front(plan: Plan, mask, first_intact, damage_end, stream=None) -> None:
    """Front readout per column (int32 tensors of L): first intact row and
    one past the last broken row."""
    L = plan.L
    rc = _lib.fc_front(plan.handle, _ptr(mask, torch.uint8, L * L, "mask"),
                       _ptr(first_intact, torch.int32, L, "first_intact"),
                       _ptr(damage_end, torch.int32, L, "damage_end"), _stream(stream))
    if rc != FC_OK:
        raise FcError(rc, "fc_front")


def fc_fracture_run(plan: Plan, s, b, t, mask, x, steps: int, removed, ratio=None, rtol: float = 1e-10,
                    mode: int = FC_MODE_F64, precond: bool = False, inner_rtol: float = 0.0,
                    max_iter: int = 0, warm_resid: bool = True, stream=None) -> dict:
    """`steps` breaking steps (solve, remove argmax |x|/t); removed (int64,
    steps) and ratio (float64, steps, optional) receive the per-step record."""
    n = plan.L * plan.L
    o = cg_opts(rtol=float(rtol), max_iter=int(max_iter), mode=int(mode), inner_rtol=float(inner_rtol),
                precond=int(bool(precond)), warm_resid=0 if warm_resid else -1)
    r = fc_run_result()
    rc = _lib.fc_fracture_run(plan.handle, _ptr(s, torch.float64, n, "s"), _ptr(b, torch.float64, n, "b"),
                              _ptr(t, torch.float64, n, "t"), _ptr(mask, torch.uint8, n, "mask"),
                              _ptr(x, torch.float64, n, "x"), int(steps), ctypes.byref(o),
                              _ptr(removed, torch.int64, int(steps), "removed"),
                              _ptr(ratio, torch.float64, int(steps), "ratio"), ctypes.byref(r), _stream(stream))
    if rc in (FC_EINVAL, FC_ECUDA, FC_ENOMEM):
        raise FcError(rc, "fc_fracture_run")
    return r.as_dict()


def fc_fracture_run_batch(plan: Plan, s, b, t, mask, x, steps: int, removed, ratio=None, rtol: float = 1e-10,
                          mode: int = FC_MODE_F64, precond: bool = False, inner_rtol: float = 0.0,
                          max_iter: int = 0, warm_resid: bool = True, stream=None):
    """nb breaking runs in lockstep: s, b, t, x (float64) and mask (uint8) hold
    nb*L*L elements (run k at offset k*L*L); removed (int64) and ratio
    (float64, optional) nb*steps (run k's step j at k*steps + j).  Returns
    (rc, list of nb run-result dicts)."""
    n = plan.L * plan.L
    if not isinstance(x, torch.Tensor) or x.numel() % n or x.numel() == 0:
        raise ValueError(f"x must hold a positive multiple of {n} elements")
    nb = x.numel() // n
    o = cg_opts(rtol=float(rtol), max_iter=int(max_iter), mode=int(mode), inner_rtol=float(inner_rtol),
                precond=int(bool(precond)), warm_resid=0 if warm_resid else -1)
    rs = (fc_run_result * nb)()
    rc = _lib.fc_fracture_run_batch(plan.handle, nb, _ptr(s, torch.float64, nb * n, "s"),
                                    _ptr(b, torch.float64, nb * n, "b"), _ptr(t, torch.float64, nb * n, "t"),
                                    _ptr(mask, torch.uint8, nb * n, "mask"), _ptr(x, torch.float64, nb * n, "x"),
                                    int(steps), ctypes.byref(o),
                                    _ptr(removed, torch.int64, nb * int(steps), "removed"),
                                    _ptr(ratio, torch.float64, nb * int(steps), "ratio"), rs, _stream(stream))
    if rc in (FC_EINVAL, FC_ECUDA, FC_ENOMEM):
        raise FcError(rc, "fc_fracture_run_batch")
    return rc, [r.as_dict() for r in rs]


def fftconv_plan_info(plan: Plan) -> dict:
    Li, Mi, pi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nb = ctypes.c_size_t()
    rc = _lib.fftconv_plan_info(plan.handle, ctypes.byref(Li), ctypes.byref(Mi), ctypes.byref(pi),
                                ctypes.byref(nb))
    if rc != FC_OK:
        raise FcError(rc, "fftconv_plan_info")
    return {"L": Li.value, "M": Mi.value, "prec": pi.value, "device_bytes": nb.value}


def fc_masked_step_static(t, mask, x, removed, stream=None) -> None:
    """Plan-free breaking step for callers that cannot allocate device memory
    at the call; its scratch is a fixed static device array (N <= 4096^2)."""
    n = t.numel()
    rc = _lib.fc_masked_step_static(int(n), _ptr(t, torch.float64, n, "t"),
                                    _ptr(mask, torch.uint8, n, "mask"), _ptr(x, torch.float64, n, "x"),
                                    _ptr(removed, torch.int64, 1, "removed"), _stream(stream))
    if rc != FC_OK:
        raise FcError(rc, "fc_masked_step_static")


def fftconv_plan_shapes(plan: Plan, prec: int) -> dict:
    """Compiled and chosen launch shapes of the three passes (A, B, C)."""
    ip3 = ctypes.c_int * 3
    n, ch, rad, per = ip3(), ip3(), ip3(), ip3()
    rc = _lib.fftconv_plan_shapes(plan.handle, int(prec), n, ch, rad, per)
    if rc != FC_OK:
        raise FcError(rc, "fftconv_plan_shapes")
    return {"n_shapes": list(n), "chosen": list(ch), "radix": list(rad), "per_block": list(per)}


def fftconv_plan_shape_set(plan: Plan, prec: int, which: int) -> dict:
    """Launch shapes of FC_SHAPES_APPLY, FC_SHAPES_SOLVE or FC_SHAPES_BATCH."""
    ip3 = ctypes.c_int * 3
    ch, rd, pb, tu = ip3(), ip3(), ip3(), ctypes.c_int()
    rc = _lib.fftconv_plan_shape_set(plan.handle, int(prec), int(which), ch, rd, pb, ctypes.byref(tu))
    if rc != FC_OK:
        raise FcError(rc, "fftconv_plan_shape_set")
    return {"chosen": list(ch), "radix": list(rd), "per_block": list(pb), "tuned": bool(tu.value)}


def fftconv_plan_batch_shapes(plan: Plan, prec: int) -> dict:
    return fftconv_plan_shape_set(plan, prec, FC_SHAPES_BATCH)


def fftconv_plan_solver(plan: Plan, prec: int) -> dict:
    """How the inner CG loop runs: persistent kernel index (-1: graph loop)."""
    n, ch, th, gr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = _lib.fftconv_plan_solver(plan.handle, int(prec), ctypes.byref(n), ctypes.byref(ch), ctypes.byref(th),
                                  ctypes.byref(gr))
    if rc != FC_OK:
        raise FcError(rc, "fftconv_plan_solver")
    return {"n": n.value, "chosen": ch.value, "threads": th.value, "grid": gr.value}



class Server:
    """Owning handle of a cg_server (continuous-batching solve server)."""

    def __init__(self, handle):
        self._h = handle
        self._keep = {}  # ticket -> host arrays that must outlive the request

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.cg_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cg_server_create(mem_budget_bytes: int, max_slots: int = 16) -> Server:
    h = ctypes.c_void_p()
    rc = _lib.cg_server_create(ctypes.byref(h), ctypes.c_size_t(int(mem_budget_bytes)), int(max_slots), None)
    if rc != FC_OK:
        raise FcError(rc, "cg_server_create")
    return Server(h)


def cg_server_reserve(sv: Server, L: int, nplans: int = 2) -> None:
    """Make up to nplans plans of size L before requests need them."""
    rc = _lib.cg_server_reserve(sv.handle, int(L), int(nplans))
    if rc != FC_OK:
        raise FcError(rc, "cg_server_reserve")


def cg_batch_submit(sv: Server, L: int, s, b, x_out=None, rtol: float = 1e-8, mode: int = FC_MODE_MIXED,
                    tag: int = 0, precond: bool = False, borrow: bool = False) -> int:
    """Queue one solve (host float64 arrays of L*L); x_out (float64, L*L,
    C-contiguous numpy array) receives the solution.  borrow: the server
    reads s and b when the request runs instead of copying them at submit
    (this wrapper keeps them alive until the request is polled done; the
    caller must not change them meanwhile).  Returns the ticket."""
    import numpy as np
    n = int(L) * int(L)
    s = np.ascontiguousarray(s, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if s.size != n or b.size != n:
        raise ValueError("s and b need L*L values")
    if x_out is not None and (x_out.dtype != np.float64 or not x_out.flags.c_contiguous or x_out.size != n):
        raise ValueError("x_out must be a contiguous float64 array of L*L values")
    rq = cg_request(L=int(L), mode=int(mode), rtol=float(rtol), s=s.ctypes.data, b=b.ctypes.data,
                    x=x_out.ctypes.data if x_out is not None else None, tag=int(tag),
                    precond=int(bool(precond)), flags=FC_REQ_BORROW if borrow else 0)
    t = ctypes.c_uint64()
    rc = _lib.cg_batch_submit(sv.handle, ctypes.byref(rq), ctypes.byref(t))
    if rc != FC_OK:
        raise FcError(rc, "cg_batch_submit")
    sv._keep[t.value] = (x_out, s, b) if borrow else x_out
    return t.value


def cg_poll(sv: Server, ticket: int):
    """Non-blocking: None while running, else the result dict."""
    r = cg_result()
    done = ctypes.c_int()
    rc = _lib.cg_poll(sv.handle, ctypes.c_uint64(ticket), ctypes.byref(r), ctypes.byref(done))
    if rc not in (FC_OK,) and not done.value:
        raise FcError(rc, "cg_poll")
    if not done.value:
        return None
    sv._keep.pop(ticket, None)
    out = r.as_dict()
    out["rc"] = rc
    return out


def cg_server_stats(sv: Server) -> dict:
    used, peak = ctypes.c_size_t(), ctypes.c_size_t()
    q, pl = ctypes.c_int(), ctypes.c_int()
    rc = _lib.cg_server_stats(sv.handle, ctypes.byref(used), ctypes.byref(peak), ctypes.byref(q), ctypes.byref(pl))
    if rc != FC_OK:
        raise FcError(rc, "cg_server_stats")
    return {"used": used.value, "peak": peak.value, "queued": q.value, "plans": pl.value}


def cg_server_batches(sv: Server) -> dict:
    """Batched solves the server ran, the requests they held, the largest batch."""
    nb, ns, mx = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
    rc = _lib.cg_server_batches(sv.handle, ctypes.byref(nb), ctypes.byref(ns), ctypes.byref(mx))
    if rc != FC_OK:
        raise FcError(rc, "cg_server_batches")
    return {"batches": nb.value, "solves": ns.value, "max_batch": mx.value}


def cg_server_destroy(sv: Server) -> None:
    sv.close()


def fc_mem_stats(reset_peak: bool = False) -> dict:
    """The library's own device memory: live and peak bytes, live allocations."""
    live, peak, n = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_longlong()
    rc = _lib.fc_mem_stats(ctypes.byref(live), ctypes.byref(peak), ctypes.byref(n), int(bool(reset_peak)))
    if rc != FC_OK:
        raise FcError(rc, "fc_mem_stats")
    return {"live_bytes": live.value, "peak_bytes": peak.value, "live_allocs": n.value}


def fftconv_plan_check_guards(plan: Plan) -> int:
    """Guard bands around the plan's buffers that were overwritten (0: none)."""
    d = ctypes.c_int()
    rc = _lib.fftconv_plan_check_guards(plan.handle, ctypes.byref(d))
    if rc != FC_OK:
        raise FcError(rc, "fftconv_plan_check_guards")
    return d.value


def fc_debug_inject(plan, kind: int, value: int) -> None:
    """Test hooks (FC_INJECT_ALLOC with plan None, FC_INJECT_BARRIER, FC_INJECT_TMA)."""
    rc = _lib.fc_debug_inject(plan.handle if plan is not None else None, int(kind), int(value))
    if rc != FC_OK:
        raise FcError(rc, "fc_debug_inject")
