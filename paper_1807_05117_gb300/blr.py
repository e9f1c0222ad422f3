"""Thin ctypes binding of libblr.so (include/blr.h).

Argument marshalling only: every function passes tensor data pointers and the
current CUDA stream to the C entry point of the same name and raises
``BlrError`` on a non-zero status.  There is no fallback: if the library is not
built, importing this module raises.

Coefficient tensors are torch.complex64 of shape (3, B1, B2, B3) (interleaved
complex, as the C-ABI expects); fields are torch.float32 of shape (N1, N2, N3)
or (3, N1, N2, N3); energies are torch.float64 of shape (3,) on the device.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from .build import LIB_PATH

BLR_OK = 0
BLR_EINVAL = -1
BLR_ENOMEM = -2
BLR_ECUDA = -3
BLR_ECFL = -4
BLR_ENAN = -5
BLR_ESTATE = -6
BLR_ECURV = -7
BLR_ETIMEOUT = -8

BLR_FP32 = 0
BLR_MIXED = 1
BLR_GAUSS_NEWTON = 0
BLR_NEWTON = 1
BLR_STATE_IMAGE = 0
BLR_STATE_DEFORMATION = 1


class blr_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("band", ctypes.c_int * 3), ("nt", ctypes.c_int),
                ("alpha", ctypes.c_double), ("gamma", ctypes.c_double), ("s", ctypes.c_double),
                ("sigma", ctypes.c_double), ("precision", ctypes.c_int),
                ("ckpt_every", ctypes.c_int), ("incompressible", ctypes.c_int),
                ("hessian", ctypes.c_int), ("nonstationary", ctypes.c_int),
                ("state_equation", ctypes.c_int)]


class blr_report(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("pcg_iters", ctypes.c_int),
                ("n_state", ctypes.c_int), ("n_hessvec", ctypes.c_int),
                ("n_halvings", ctypes.c_int), ("status", ctypes.c_int),
                ("energy0", ctypes.c_double), ("energy", ctypes.c_double),
                ("grad_inf_rel", ctypes.c_double)]


class BlrError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {blr_strerror(code)} (status {code})")


_P = ctypes.c_void_p
_SIGS = {
    "blr_plan_create": (ctypes.POINTER(blr_params), ctypes.POINTER(_P)),
    "blr_plan_destroy": (_P,),
    "blr_set_images": (_P, _P, _P, _P),
    "blr_expand": (_P, _P, _P, _P),
    "blr_project": (_P, _P, _P, _P),
    "blr_state": (_P, _P, _P, _P, _P),
    "blr_adjoint": (_P, _P, _P, _P),
    "blr_gradient": (_P, _P, _P, _P, _P),
    "blr_gradient_at_state": (_P, _P, _P),
    "blr_hessvec": (_P, _P, _P, _P),
    "blr_pcg": (_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                ctypes.POINTER(ctypes.c_double), _P),
    "blr_newton": (_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                   ctypes.POINTER(blr_report), _P),
    "blr_status": (_P, _P),
    "blr_test_expire_waits": (ctypes.c_int,),
    "blr_plan_tuning": (_P, ctypes.POINTER(ctypes.c_int), ctypes.c_int),
    "blr_plan_set_tuning": (_P, ctypes.POINTER(ctypes.c_int), ctypes.c_int),
    "blr_batch_create": (ctypes.POINTER(blr_params), ctypes.c_int, ctypes.POINTER(_P)),
    "blr_batch_destroy": (_P,),
    "blr_batch_tuning": (_P, ctypes.POINTER(ctypes.c_int), ctypes.c_int),
    "blr_batch_set_tuning": (_P, ctypes.POINTER(ctypes.c_int), ctypes.c_int),
    "blr_batch_set_images": (_P, ctypes.c_int, _P, _P, _P),
    "blr_batch_gradient": (_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _P),
    "blr_batch_hessvec": (_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _P),
    "blr_batch_newton": (_P, ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                         ctypes.c_double, ctypes.POINTER(blr_report), _P),
}

#: every symbol include/blr.h declares
EXPORTED = tuple(_SIGS) + ("blr_strerror", "blr_kernel_launches", "blr_expand_noalloc")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_1807_05117_gb300.build.build_library()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = list(args)
        fn.restype = ctypes.c_int
    lib.blr_strerror.argtypes = [ctypes.c_int]
    lib.blr_strerror.restype = ctypes.c_char_p
    lib.blr_kernel_launches.argtypes = []
    lib.blr_kernel_launches.restype = ctypes.c_ulonglong
    lib.blr_expand_noalloc.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       _P, _P, _P]
    lib.blr_expand_noalloc.restype = ctypes.c_int
    return lib


_lib = _load()


def blr_strerror(code: int) -> str:
    return _lib.blr_strerror(int(code)).decode()


def blr_kernel_launches() -> int:
    return int(_lib.blr_kernel_launches())


def _check(rc: int, where: str):
    if rc != BLR_OK:
        raise BlrError(rc, where)


def _stream(stream):
    if stream is None:
        import torch
        return _P(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _P(stream)
    return _P(stream.cuda_stream)


def _ptr(t, *, device_only=True, dtype=None, numel=None, optional=False, name="tensor",
         device=None):
    """Data pointer of `t` after checking what the C entry point cannot: element
    count (numel), dtype, contiguity, and for device pointers that the tensor is
    on the CUDA device `device` (an index; None skips the check)."""
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device_only and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if device is not None and t.is_cuda and t.device.index != device:
        raise ValueError(f"{name} is on {t.device}, the call runs on cuda:{device}")
    return _P(t.data_ptr())


@dataclass(frozen=True)
class _Shape:
    """Element counts of one plan's arrays (complex64 counts for coefficients)."""
    V: int          # voxels
    coef: int       # one velocity's coefficients: 3 B1 B2 B3
    nvel: int       # velocities in a parameter vector (nt when non-stationary)
    device: int     # CUDA device the plan was created on
    deformation: bool

    @property
    def param(self):
        return self.nvel * self.coef


_SHAPES: dict = {}


def _shape_of(params: blr_params, device: int) -> _Shape:
    n, b = list(params.n), list(params.band)
    return _Shape(V=n[0] * n[1] * n[2], coef=3 * b[0] * b[1] * b[2],
                  nvel=int(params.nt) if params.nonstationary else 1, device=int(device),
                  deformation=params.state_equation == BLR_STATE_DEFORMATION)


def _shape(plan) -> _Shape:
    try:
        return _SHAPES[int(plan)]
    except (KeyError, TypeError):
        raise ValueError("not a live plan handle of this binding") from None


def _current_device() -> int:
    import torch
    return torch.cuda.current_device()


def make_params(n, band, nt=10, alpha=3.0, gamma=1.0, s=2, sigma=1.0, precision=BLR_FP32,
                ckpt_every=0, incompressible=False, hessian=BLR_GAUSS_NEWTON,
                nonstationary=False, state_equation=BLR_STATE_IMAGE):
    p = blr_params()
    p.n[:] = [int(v) for v in n]
    p.band[:] = [int(v) for v in band]
    p.nt = int(nt)
    p.alpha, p.gamma, p.s, p.sigma = float(alpha), float(gamma), float(s), float(sigma)
    p.precision = int(precision)
    p.ckpt_every = int(ckpt_every)
    p.incompressible = 1 if incompressible else 0
    p.hessian = int(hessian)
    p.nonstationary = 1 if nonstationary else 0
    p.state_equation = int(state_equation)
    return p


# --- entry points (same names as the C-ABI) ---------------------------------


def blr_plan_create(params: blr_params) -> int:
    h = _P()
    _check(_lib.blr_plan_create(ctypes.byref(params), ctypes.byref(h)), "blr_plan_create")
    _SHAPES[h.value] = _shape_of(params, _current_device())
    return h.value


def blr_plan_destroy(plan: int):
    _SHAPES.pop(int(plan), None)
    _check(_lib.blr_plan_destroy(_P(plan)), "blr_plan_destroy")


def blr_set_images(plan, I0, I1, stream=None):
    import torch
    sh = _shape(plan)
    kw = dict(device_only=False, dtype=torch.float32, numel=sh.V, device=sh.device)
    _check(_lib.blr_set_images(_P(plan), _ptr(I0, name="I0", **kw), _ptr(I1, name="I1", **kw),
                               _stream(stream)), "blr_set_images")


def blr_expand(plan, vt, v, stream=None):
    import torch
    sh = _shape(plan)
    _check(_lib.blr_expand(_P(plan),
                           _ptr(vt, dtype=torch.complex64, numel=sh.coef, name="vt", device=sh.device),
                           _ptr(v, dtype=torch.float32, numel=3 * sh.V, name="v", device=sh.device),
                           _stream(stream)), "blr_expand")


def blr_expand_noalloc(n, band, vt, v, stream=None):
    """iota without a plan and without allocating (see include/blr.h): the
    library's fixed device scratch array holds the tables and intermediates.
    vt and v must be on the current device (the call runs there)."""
    import torch
    n, band = [int(x) for x in n], [int(x) for x in band]
    if len(n) != 3 or len(band) != 3:
        raise ValueError("n and band take three entries each")
    dev = _current_device()
    cn = (ctypes.c_int * 3)(*n)
    cb = (ctypes.c_int * 3)(*band)
    coef = 3 * band[0] * band[1] * band[2]
    V = n[0] * n[1] * n[2]
    _check(_lib.blr_expand_noalloc(cn, cb,
                                   _ptr(vt, dtype=torch.complex64, numel=coef, name="vt", device=dev),
                                   _ptr(v, dtype=torch.float32, numel=3 * V, name="v", device=dev),
                                   _stream(stream)), "blr_expand_noalloc")


def blr_project(plan, f, ft, stream=None):
    import torch
    sh = _shape(plan)
    _check(_lib.blr_project(_P(plan),
                            _ptr(f, dtype=torch.float32, numel=3 * sh.V, name="f", device=sh.device),
                            _ptr(ft, dtype=torch.complex64, numel=sh.coef, name="ft", device=sh.device),
                            _stream(stream)), "blr_project")


def blr_state(plan, vt, m1=None, energy=None, stream=None):
    import torch
    sh = _shape(plan)
    _check(_lib.blr_state(_P(plan),
                          _ptr(vt, dtype=torch.complex64, numel=sh.param, name="vt", device=sh.device),
                          _ptr(m1, dtype=torch.float32, numel=sh.V, optional=True, name="m1",
                               device=sh.device),
                          _ptr(energy, dtype=torch.float64, numel=3, optional=True, name="energy",
                               device=sh.device),
                          _stream(stream)), "blr_state")


def blr_adjoint(plan, b, lambda0=None, stream=None):
    import torch
    sh = _shape(plan)
    _check(_lib.blr_adjoint(_P(plan),
                            _ptr(b, dtype=torch.float32, numel=3 * sh.nvel * sh.V, name="b",
                                 device=sh.device),
                            _ptr(lambda0, dtype=torch.float32, numel=sh.V, optional=True,
                                 name="lambda0", device=sh.device),
                            _stream(stream)), "blr_adjoint")


def blr_gradient(plan, vt, g, energy=None, stream=None):
    import torch
    sh = _shape(plan)
    _check(_lib.blr_gradient(_P(plan),
                             _ptr(vt, dtype=torch.complex64, numel=sh.param, name="vt",
                                  device=sh.device),
                             _ptr(g, dtype=torch.complex64, numel=sh.param, name="g", device=sh.device),
                             _ptr(energy, dtype=torch.float64, numel=3, optional=True, name="energy",
                                  device=sh.device),
                             _stream(stream)), "blr_gradient")


def blr_gradient_at_state(plan, g, stream=None):
    import torch
    sh = _shape(plan)
    _check(_lib.blr_gradient_at_state(
        _P(plan), _ptr(g, dtype=torch.complex64, numel=sh.param, name="g", device=sh.device),
        _stream(stream)), "blr_gradient_at_state")


def blr_hessvec(plan, dvt, hdv, stream=None):
    import torch
    sh = _shape(plan)
    _check(_lib.blr_hessvec(_P(plan),
                            _ptr(dvt, dtype=torch.complex64, numel=sh.param, name="dvt",
                                 device=sh.device),
                            _ptr(hdv, dtype=torch.complex64, numel=sh.param, name="hdv",
                                 device=sh.device),
                            _stream(stream)), "blr_hessvec")


def blr_pcg(plan, rhs, x, maxit, eta, stream=None):
    import torch
    sh = _shape(plan)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    _check(_lib.blr_pcg(_P(plan),
                        _ptr(rhs, dtype=torch.complex64, numel=sh.param, name="rhs", device=sh.device),
                        _ptr(x, dtype=torch.complex64, numel=sh.param, name="x", device=sh.device),
                        int(maxit), float(eta), ctypes.byref(it), ctypes.byref(rel),
                        _stream(stream)), "blr_pcg")
    return it.value, rel.value


@dataclass
class Report:
    newton_iters: int
    pcg_iters: int
    n_state: int
    n_hessvec: int
    n_halvings: int
    status: int
    energy0: float
    energy: float
    grad_inf_rel: float


def blr_newton(plan, vt, max_newton, max_pcg, gtol, forcing=-1.0, stream=None,
               raise_on_error=True) -> Report:
    import torch
    sh = _shape(plan)
    rep = blr_report()
    rc = _lib.blr_newton(_P(plan), _ptr(vt, device_only=False, dtype=torch.complex64,
                                        numel=sh.param, name="vt", device=sh.device),
                         int(max_newton), int(max_pcg), float(gtol), float(forcing),
                         ctypes.byref(rep), _stream(stream))
    if raise_on_error:
        _check(rc, "blr_newton")
    return Report(*[getattr(rep, f) for f, _ in blr_report._fields_])


def blr_status(plan, stream=None) -> int:
    return int(_lib.blr_status(_P(plan), _stream(stream)))


def blr_test_expire_waits(on: bool):
    """Test hook: tensor-core DFT launches time out on purpose (include/blr.h)."""
    _check(_lib.blr_test_expire_waits(1 if on else 0), "blr_test_expire_waits")


class Plan:
    """Owning handle: ``with Plan(n, band, nt) as P: P.gradient(vt, g)``."""

    def __init__(self, n, band, nt=10, alpha=3.0, gamma=1.0, s=2, sigma=1.0,
                 precision=BLR_FP32, ckpt_every=0, incompressible=False,
                 hessian=BLR_GAUSS_NEWTON, nonstationary=False,
                 state_equation=BLR_STATE_IMAGE):
        self.params = make_params(n, band, nt, alpha, gamma, s, sigma, precision, ckpt_every,
                                  incompressible, hessian, nonstationary, state_equation)
        self.n = tuple(int(v) for v in n)
        self.band = tuple(int(v) for v in band)
        self.nt = int(nt)
        self.handle = blr_plan_create(self.params)
        self.point = 0          # bumped whenever the current point changes

    def close(self):
        if self.handle:
            blr_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_images(self, I0, I1, stream=None):
        blr_set_images(self.handle, I0, I1, stream)
        self.point += 1

    def expand(self, vt, v, stream=None):
        blr_expand(self.handle, vt, v, stream)

    def project(self, f, ft, stream=None):
        blr_project(self.handle, f, ft, stream)

    def state(self, vt, m1=None, energy=None, stream=None):
        blr_state(self.handle, vt, m1, energy, stream)
        self.point += 1

    def adjoint(self, b, lambda0=None, stream=None):
        blr_adjoint(self.handle, b, lambda0, stream)

    def gradient(self, vt, g, energy=None, stream=None):
        blr_gradient(self.handle, vt, g, energy, stream)
        self.point += 1

    def gradient_at_state(self, g, stream=None):
        blr_gradient_at_state(self.handle, g, stream)

    def hessvec(self, dvt, hdv, stream=None):
        blr_hessvec(self.handle, dvt, hdv, stream)

    def pcg(self, rhs, x, maxit, eta, stream=None):
        return blr_pcg(self.handle, rhs, x, maxit, eta, stream)

    def newton(self, vt, max_newton, max_pcg, gtol, forcing=-1.0, stream=None,
               raise_on_error=True):
        self.point += 1
        return blr_newton(self.handle, vt, max_newton, max_pcg, gtol, forcing, stream,
                          raise_on_error)

    def status(self, stream=None):
        return blr_status(self.handle, stream)

    TUNING_KEYS = ("wide_sweeps", "grad_kept", "adjoint_blocks_per_sm", "adjoint_reads_grad",
                   "incremental_form", "incremental_blocks_per_sm", "march_blocks_per_sm",
                   "march_chunk", "adjoint_march_chunk", "l2_persist_d4", "adjoint_two_step",
                   "adjoint_split", "gemm_tiles")

    def tuning(self) -> dict:
        """The sweep shapes the autotuner chose (blr_plan_tuning)."""
        vals = (ctypes.c_int * len(self.TUNING_KEYS))()
        _check(_lib.blr_plan_tuning(_P(self.handle), vals, len(vals)), "blr_plan_tuning")
        return dict(zip(self.TUNING_KEYS, [int(v) for v in vals]))

    def set_tuning(self, **changes):
        """Override sweep shapes (blr_plan_set_tuning): keys of tuning()."""
        cur = self.tuning()
        for k, v in changes.items():
            if k not in cur:
                raise ValueError(f"unknown tuning key {k}")
            cur[k] = int(v)
        vals = (ctypes.c_int * len(self.TUNING_KEYS))(*[cur[k] for k in self.TUNING_KEYS])
        _check(_lib.blr_plan_set_tuning(_P(self.handle), vals, len(vals)), "blr_plan_set_tuning")


def _ptr_array(tensors, shapes, numel, **kw):
    """Pointers of one tensor per pair, each checked against its pair's shape
    (numel(shape) elements, on the pair's device)."""
    if len(tensors) != len(shapes):
        raise ValueError(f"{len(tensors)} tensors for {len(shapes)} pairs")
    arr = (_P * len(tensors))()
    for i, (t, sh) in enumerate(zip(tensors, shapes)):
        arr[i] = _ptr(t, numel=numel(sh), device=sh.device, name=f"pair {i}", **kw)
    return arr


class Batch:
    """Many registration pairs advanced together (see blr_batch_* in include/blr.h).

    ``Batch([(n, band), ...], nt)`` or ``Batch([make_params(...), ...])``."""

    def __init__(self, shapes, nt=10, alpha=3.0, gamma=1.0, s=2, sigma=1.0):
        params = [sh if isinstance(sh, blr_params) else
                  make_params(sh[0], sh[1], nt, alpha, gamma, s, sigma) for sh in shapes]
        self.npairs = len(params)
        self._pair = [_shape_of(p, _current_device()) for p in params]
        self.shapes = [(tuple(p.n), tuple(p.band)) for p in params]
        arr = (blr_params * self.npairs)(*params)
        h = _P()
        _check(_lib.blr_batch_create(arr, self.npairs, ctypes.byref(h)), "blr_batch_create")
        self.handle = h.value

    def close(self):
        if self.handle:
            _check(_lib.blr_batch_destroy(_P(self.handle)), "blr_batch_destroy")
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    TUNING_KEYS = ("kept_gradients", "use_kept_gradients", "adjoint_chunk", "state_chunk",
                   "solo_min_voxels", "solo_pairs", "incremental_gather")

    def tuning(self) -> dict:
        """The batch's sweep choices (blr_batch_tuning)."""
        vals = (ctypes.c_int * len(self.TUNING_KEYS))()
        _check(_lib.blr_batch_tuning(_P(self.handle), vals, len(vals)), "blr_batch_tuning")
        return dict(zip(self.TUNING_KEYS, [int(v) for v in vals]))

    def set_tuning(self, **changes):
        """Override the sweep choices (blr_batch_set_tuning): keys of tuning() but
        the last (solo_pairs follows from solo_min_voxels)."""
        cur = self.tuning()
        for k, v in changes.items():
            if k not in cur or k == "solo_pairs":
                raise ValueError(f"unknown or read-only tuning key {k}")
            cur[k] = int(v)
        if not cur["use_kept_gradients"]:
            cur["incremental_gather"] = 0   # the gather form reads the kept gradients
        vals = (ctypes.c_int * len(self.TUNING_KEYS))(*[cur[k] for k in self.TUNING_KEYS])
        _check(_lib.blr_batch_set_tuning(_P(self.handle), vals, len(vals)), "blr_batch_set_tuning")

    def set_images(self, pair, I0, I1, stream=None):
        import torch
        if not 0 <= int(pair) < self.npairs:
            raise ValueError(f"pair {pair} out of range 0..{self.npairs - 1}")
        sh = self._pair[int(pair)]
        kw = dict(device_only=False, dtype=torch.float32, numel=sh.V, device=sh.device)
        _check(_lib.blr_batch_set_images(_P(self.handle), int(pair), _ptr(I0, name="I0", **kw),
                                         _ptr(I1, name="I1", **kw), _stream(stream)),
               "blr_batch_set_images")

    def gradient(self, vts, gs, stream=None):
        import torch
        coef = lambda sh: sh.coef  # noqa: E731
        _check(_lib.blr_batch_gradient(_P(self.handle),
                                       _ptr_array(vts, self._pair, coef, dtype=torch.complex64),
                                       _ptr_array(gs, self._pair, coef, dtype=torch.complex64),
                                       _stream(stream)), "blr_batch_gradient")

    def hessvec(self, dvts, hdvs, stream=None):
        import torch
        coef = lambda sh: sh.coef  # noqa: E731
        _check(_lib.blr_batch_hessvec(_P(self.handle),
                                      _ptr_array(dvts, self._pair, coef, dtype=torch.complex64),
                                      _ptr_array(hdvs, self._pair, coef, dtype=torch.complex64),
                                      _stream(stream)), "blr_batch_hessvec")

    def newton(self, vts, max_newton, max_pcg, gtol, forcing=-1.0, stream=None):
        import torch
        reps = (blr_report * self.npairs)()
        _check(_lib.blr_batch_newton(_P(self.handle),
                                     _ptr_array(vts, self._pair, lambda sh: sh.coef,
                                                device_only=False, dtype=torch.complex64),
                                     int(max_newton), int(max_pcg), float(gtol), float(forcing),
                                     reps, _stream(stream)), "blr_batch_newton")
        return [Report(*[getattr(r, f) for f, _ in blr_report._fields_]) for r in reps]
