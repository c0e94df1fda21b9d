"""Thin ctypes binding of the C ABI in ``include/sag.h`` (libsag.so).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels. Buffers may be torch CUDA tensors (device pointers, the
current torch stream is used unless one is given) or numpy arrays (host
pointers; the library copies them to and from the device inside the call).
If the library cannot be loaded the binding raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SAG_OK, SAG_EINVAL, SAG_ENOMEM, SAG_ECUDA, SAG_EUNSUPPORTED, SAG_ETIMEOUT, SAG_ENONFINITE = range(7)
SAG_CP, SAG_TT, SAG_CP_POWER = 0, 1, 2
SAG_FP64, SAG_FP32_SPLIT, SAG_FP32_SPLIT_EXACT = 0, 1, 2
SAG_HEUN, SAG_MIDPOINT = 0, 1

# Every function include/sag.h declares.
EXPORTS = [
    "sag_default_options", "sag_plan", "sag_plan_layout", "sag_plan_bytes", "sag_rhs",
    "sag_rhs_parts", "sag_rk2_step", "sag_integrate", "sag_sync_status", "sag_plan_destroy",
    "sag_last_error", "sag_version", "sag_profile_enable", "sag_profile_read", "sag_kernel_name",
    "sag_kernel_work", "sag_plan_describe", "sag_loss_noalloc", "sag_rhs_vjp", "sag_integrate_vjp",
    "sag_plan_update_factors", "sag_plan_factor_count", "sag_plan_set_wait_limit",
    "sag_kernel_method_work", "sag_rk2_stage", "sag_power_eval",
]
SAG_NUM_KERNELS = 13

_STATUS_NAMES = {0: "SAG_OK", 1: "SAG_EINVAL", 2: "SAG_ENOMEM", 3: "SAG_ECUDA",
                 4: "SAG_EUNSUPPORTED", 5: "SAG_ETIMEOUT", 6: "SAG_ENONFINITE"}


class SagError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _System(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("D", ctypes.c_int32), ("fmt", ctypes.c_int32),
                ("rank", ctypes.POINTER(ctypes.c_int32)), ("factors", ctypes.c_void_p),
                ("factors_on_device", ctypes.c_int32)]


class _Options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("rk", ctypes.c_int32),
                ("symmetrize_q", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("max_m2", ctypes.c_int32), ("m2", ctypes.POINTER(ctypes.c_int32)),
                ("n_m2", ctypes.c_int32), ("keep_repeats", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Opens libsag.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise OSError(f"libsag.so not found at {path}")
        lib = ctypes.CDLL(path)
        vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.sag_default_options.argtypes = [ctypes.POINTER(_Options)]
        lib.sag_default_options.restype = None
        lib.sag_plan.argtypes = [ctypes.POINTER(_System), i32, ctypes.POINTER(_Options),
                                 ctypes.POINTER(vp)]
        lib.sag_plan_layout.argtypes = [vp, ctypes.POINTER(i64)]
        lib.sag_plan_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        lib.sag_rhs.argtypes = [vp, vp, vp, vp]
        lib.sag_rhs_parts.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.sag_rk2_step.argtypes = [vp, vp, f64, vp]
        lib.sag_integrate.argtypes = [vp, vp, f64, i64, vp, vp]
        lib.sag_sync_status.argtypes = [vp, vp]
        lib.sag_plan_destroy.argtypes = [vp]
        lib.sag_plan_destroy.restype = None
        lib.sag_last_error.restype = ctypes.c_char_p
        lib.sag_version.restype = ctypes.c_char_p
        lib.sag_profile_enable.argtypes = [vp, i32]
        lib.sag_profile_read.argtypes = [vp, ctypes.POINTER(f64), ctypes.POINTER(i64), i32]
        lib.sag_kernel_name.argtypes = [i32]
        lib.sag_kernel_name.restype = ctypes.c_char_p
        lib.sag_kernel_work.argtypes = [vp, i32, ctypes.POINTER(f64), ctypes.POINTER(i32),
                                        ctypes.POINTER(f64)]
        lib.sag_kernel_method_work.argtypes = [vp, i32, ctypes.POINTER(f64), ctypes.POINTER(f64)]
        lib.sag_rk2_stage.argtypes = [vp, i32, vp, vp, vp, vp, f64, vp]
        lib.sag_power_eval.argtypes = [f64, f64, i32, vp, vp]
        lib.sag_plan_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
        lib.sag_loss_noalloc.argtypes = [ctypes.POINTER(_System), i32, vp, vp, vp]
        lib.sag_rhs_vjp.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.sag_integrate_vjp.argtypes = [vp, vp, f64, i64, i64, vp, vp, vp, vp]
        lib.sag_plan_update_factors.argtypes = [vp, vp, i32]
        lib.sag_plan_factor_count.argtypes = [vp, ctypes.POINTER(i64)]
        lib.sag_plan_set_wait_limit.argtypes = [vp, i64, i32]
        lib.sag_loss_noalloc.restype = ctypes.c_int
        for name in ("sag_plan", "sag_plan_layout", "sag_plan_bytes", "sag_rhs", "sag_rhs_parts",
                     "sag_rk2_step", "sag_integrate", "sag_sync_status", "sag_profile_enable",
                     "sag_profile_read", "sag_kernel_work", "sag_plan_describe", "sag_rhs_vjp",
                     "sag_integrate_vjp", "sag_plan_update_factors", "sag_plan_factor_count",
                     "sag_plan_set_wait_limit", "sag_kernel_method_work", "sag_rk2_stage",
                     "sag_power_eval"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(status: int):
    if status != SAG_OK:
        raise SagError(status, load().sag_last_error().decode())


def _ptr(x):
    """Device or host address of a torch tensor / numpy array (FP64, contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffers must be contiguous float64")
        return x.ctypes.data
    import torch
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("torch buffers must be contiguous float64")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream, *tensors):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    import torch
    if any(isinstance(t, torch.Tensor) and t.is_cuda for t in tensors):
        return torch.cuda.current_stream().cuda_stream
    return None


def loss_noalloc(N: int, D: int, ranks, factors, n, q, symmetrize_q: int = 1, stream=None):
    """sag_loss_noalloc: q = sum_d Q^(d)[n] for a CP system from device buffers
    (torch CUDA tensors), without any device allocation by the library."""
    lib = load()
    r = np.ascontiguousarray(np.asarray(ranks, dtype=np.int32))
    sysd = _System(int(N), int(D), SAG_CP, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                   _ptr(factors), 1)
    _check(lib.sag_loss_noalloc(ctypes.byref(sysd), int(symmetrize_q), _ptr(n), _ptr(q),
                                _stream(stream, n, q)))
    return q


def power_eval(u: float, a: float, N: int, out, stream=None):
    """sag_power_eval: out[i-1] = u i^a (i = 1..N) by the parametric factors'
    double-word generator, into a device FP64 tensor of N values."""
    _check(load().sag_power_eval(float(u), float(a), int(N), _ptr(out), _stream(stream, out)))
    return out


def default_options() -> dict:
    o = _Options()
    load().sag_default_options(ctypes.byref(o))
    return {"prec": o.prec, "rk": o.rk, "symmetrize_q": o.symmetrize_q, "autotune": o.autotune,
            "max_m2": o.max_m2, "m2": None if not o.m2 else list(o.m2[:o.n_m2]),
            "keep_repeats": o.keep_repeats}


class Plan:
    """A plan (sag_plan) for one system, or for several with ``Plan.batch``.
    ``factors`` is a flat float64 array in the layout of include/sag.h (numpy:
    host memory; torch CUDA tensor: device memory). State vectors of a batched
    plan are packed: system b occupies ``layout()[b]:layout()[b+1]``."""

    def __init__(self, N: int, D: int, ranks, factors, *, fmt: int = SAG_CP,
                 prec: int = SAG_FP32_SPLIT, rk: int = SAG_HEUN, symmetrize_q: int = 1,
                 autotune: int = 0, max_m2: int = 0, m2=None, keep_repeats: int = 0, _systems=None):
        lib = load()
        systems = _systems if _systems is not None else [(N, D, ranks, factors, fmt)]
        self.B = len(systems)
        self.N, self.D, self.fmt, self.prec = int(systems[0][0]), int(systems[0][1]), \
            int(systems[0][4]), int(prec)
        arr = (_System * self.B)()
        self._keep = []
        for b, (Nb, Db, rb, fb, fmtb) in enumerate(systems):
            r = np.ascontiguousarray(np.asarray(rb, dtype=np.int32))
            on_dev = 0
            try:
                import torch
                on_dev = int(isinstance(fb, torch.Tensor) and fb.is_cuda)
            except ImportError:
                pass
            if not on_dev:
                fb = np.ascontiguousarray(np.asarray(fb, dtype=np.float64))
            self._keep += [r, fb]
            arr[b] = _System(int(Nb), int(Db), int(fmtb),
                             r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _ptr(fb), on_dev)
        opt = _Options(int(prec), int(rk), int(symmetrize_q), int(autotune), int(max_m2))
        opt.keep_repeats = int(keep_repeats)
        if m2 is not None:  # M2 per order, e.g. [o["M2"] for o in plan.describe()["orders"]]
            m2a = np.ascontiguousarray(np.asarray(m2, dtype=np.int32))
            self._keep.append(m2a)
            opt.m2 = m2a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            opt.n_m2 = int(m2a.size)
        h = ctypes.c_void_p()
        _check(lib.sag_plan(arr, self.B, ctypes.byref(opt), ctypes.byref(h)))
        self._h = h
        self._lib = lib
        self._keep = None

    @classmethod
    def batch(cls, systems, *, prec: int = SAG_FP32_SPLIT, rk: int = SAG_HEUN,
              symmetrize_q: int = 1, autotune: int = 0, max_m2: int = 0, m2=None, keep_repeats: int = 0):
        """systems: list of (N, D, ranks, factors, fmt); one plan, one launch per kernel."""
        return cls(0, 0, None, None, prec=prec, rk=rk, symmetrize_q=symmetrize_q,
                   autotune=autotune, max_m2=max_m2, m2=m2, keep_repeats=keep_repeats,
                   _systems=list(systems))

    @property
    def handle(self):
        return self._h

    def layout(self):
        off = (ctypes.c_int64 * (self.B + 1))()
        _check(self._lib.sag_plan_layout(self._h, off))
        return [int(off[i]) for i in range(self.B + 1)]

    def device_bytes(self) -> int:
        b = ctypes.c_size_t()
        _check(self._lib.sag_plan_bytes(self._h, ctypes.byref(b)))
        return int(b.value)

    def rhs(self, n, dndt, stream=None):
        _check(self._lib.sag_rhs(self._h, _ptr(n), _ptr(dndt), _stream(stream, n, dndt)))
        return dndt

    def rhs_parts(self, n, p=None, q=None, outflow=None, stream=None):
        _check(self._lib.sag_rhs_parts(self._h, _ptr(n), _ptr(p), _ptr(q), _ptr(outflow),
                                       _stream(stream, n, p, q, outflow)))
        return p, q, outflow

    def rk2_step(self, n, dt: float, stream=None):
        _check(self._lib.sag_rk2_step(self._h, _ptr(n), float(dt), _stream(stream, n)))
        return n

    def rk2_stage(self, stage: int, n, nstar, k1, k, dt: float, stream=None):
        """sag_rk2_stage: one stage of the plan's RK2 rule from a given right-hand side k."""
        _check(self._lib.sag_rk2_stage(self._h, int(stage), _ptr(n), _ptr(nstar), _ptr(k1), _ptr(k),
                                       float(dt), _stream(stream, n, nstar, k1, k)))
        return n

    def integrate(self, n, dt: float, steps: int, diag=None, stream=None):
        _check(self._lib.sag_integrate(self._h, _ptr(n), float(dt), int(steps), _ptr(diag),
                                       _stream(stream, n, diag)))
        return n

    def sync_status(self, stream=None) -> int:
        """Returns the latched device status (SAG_OK, SAG_ENONFINITE, ...), clearing it."""
        st = self._lib.sag_sync_status(self._h, _stream(stream))
        return int(st)

    def set_wait_limit(self, cycles: int = 0, unmet: bool = False):
        """Clock-cycle limit of the device-side waits (0: the default); with
        unmet, every such wait targets a barrier nothing completes (a test of
        the timeout path; see include/sag.h)."""
        _check(self._lib.sag_plan_set_wait_limit(self._h, int(cycles), int(bool(unmet))))

    def profile(self, on: bool = True):
        """Turns per-kernel event timing on or off (non-graph launches only)."""
        _check(self._lib.sag_profile_enable(self._h, int(bool(on))))

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since the last read; waits for the work."""
        ms = (ctypes.c_double * SAG_NUM_KERNELS)()
        cnt = (ctypes.c_int64 * SAG_NUM_KERNELS)()
        _check(self._lib.sag_profile_read(self._h, ms, cnt, SAG_NUM_KERNELS))
        return {self._lib.sag_kernel_name(i).decode(): (ms[i], cnt[i])
                for i in range(SAG_NUM_KERNELS) if cnt[i]}

    def factor_count(self) -> int:
        c = ctypes.c_int64()
        _check(self._lib.sag_plan_factor_count(self._h, ctypes.byref(c)))
        return int(c.value)

    def rhs_vjp(self, n, g, gn=None, gU=None, stream=None):
        """gn = (dF/dn)^T g, gU = (dF/dU)^T g (vector layout)."""
        _check(self._lib.sag_rhs_vjp(self._h, _ptr(n), _ptr(g), _ptr(gn), _ptr(gU),
                                     _stream(stream, n, g, gn, gU)))
        return gn, gU

    def integrate_vjp(self, n0, dt: float, steps: int, g_final, g_n0=None, g_U=None, ckpt: int = 0,
                      stream=None):
        """Discrete adjoint of `steps` RK2 steps from n0 (checkpointed)."""
        _check(self._lib.sag_integrate_vjp(self._h, _ptr(n0), float(dt), int(steps), int(ckpt),
                                           _ptr(g_final), _ptr(g_n0), _ptr(g_U),
                                           _stream(stream, n0, g_final, g_n0, g_U)))
        return g_n0, g_U

    def update_factors(self, factors):
        """New factor values (same ranks), host numpy or device torch FP64."""
        on_dev = 0
        try:
            import torch
            on_dev = int(isinstance(factors, torch.Tensor) and factors.is_cuda)
        except ImportError:
            pass
        if not on_dev:
            factors = np.ascontiguousarray(np.asarray(factors, dtype=np.float64))
        _check(self._lib.sag_plan_update_factors(self._h, _ptr(factors), on_dev))

    def kernel_work(self, name_or_id) -> dict:
        """Algorithmic ops (FP32 or FP64 instructions) and HBM bytes of one launch."""
        kid = name_or_id
        if isinstance(name_or_id, str):
            names = [self._lib.sag_kernel_name(i).decode() for i in range(SAG_NUM_KERNELS)]
            kid = names.index(name_or_id)
        ops, f64, b = ctypes.c_double(), ctypes.c_int32(), ctypes.c_double()
        _check(self._lib.sag_kernel_work(self._h, int(kid), ctypes.byref(ops), ctypes.byref(f64),
                                         ctypes.byref(b)))
        return {"ops": ops.value, "ops_fp64": bool(f64.value), "bytes": b.value}

    def method_work(self, name_or_id) -> dict:
        """Nominal method flops and FFT-workspace bytes of one launch (sag_kernel_method_work)."""
        kid = name_or_id
        if isinstance(name_or_id, str):
            names = [self._lib.sag_kernel_name(i).decode() for i in range(SAG_NUM_KERNELS)]
            kid = names.index(name_or_id)
        fl, wb = ctypes.c_double(), ctypes.c_double()
        _check(self._lib.sag_kernel_method_work(self._h, int(kid), ctypes.byref(fl), ctypes.byref(wb)))
        return {"flops": fl.value, "workspace_bytes": wb.value}

    def describe(self) -> dict:
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        _check(self._lib.sag_plan_describe(self._h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.sag_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
