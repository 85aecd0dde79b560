"""ctypes binding of the tca C ABI (include/tca.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Importing this module loads ``libtca.so`` and raises ImportError when
it is missing - there is no CPU fallback.

Data arguments may be torch tensors (CUDA or CPU) or NumPy arrays; they are
passed to the library as raw pointers, so they must be C-contiguous and of the
plan's element type (float64 for a TCA_F64 plan, float32 otherwise).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtca.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"tca CUDA library not built ({LIB_PATH} missing); run "
        "`python -c 'import __graft_entry__ as g; g.build()'` first")

_lib = ctypes.CDLL(LIB_PATH)

# --- enums (tca.h) ---
OK = 0
ERR_INVALID_ARG = 1
ERR_SHAPE = 2
ERR_UNSUPPORTED = 3
ERR_ALLOC = 4
ERR_CUDA = 5
ERR_NOT_CONVERGED = 6
ERR_BREAKDOWN = 7
ERR_TIMEOUT = 8

F64, F32, BF16_IR, TF32_IR = 0, 1, 2, 3
FACTOR_DENSE, FACTOR_ELL4 = 0, 1
OP_FACTOR, OP_FACTOR_T, OP_GRAM = 0, 1, 2

PRECISIONS = {"f64": F64, "f32": F32, "bf16_ir": BF16_IR, "tf32_ir": TF32_IR}


class tca_factor(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("m", ctypes.c_int64),
                ("n", ctypes.c_int64), ("values", ctypes.c_void_p), ("col0", ctypes.c_void_p)]


class tca_reg(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_double), ("reg_mode_mask", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class tca_solve_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("x0_given", ctypes.c_int32),
                ("inner_rtol", ctypes.c_double), ("max_refine", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("precond", ctypes.c_int32), ("precond_shift", ctypes.c_double),
                ("tmg_coarse_rtol", ctypes.c_double), ("tmg_lambda_max", ctypes.c_double),
                ("tmg_nu", ctypes.c_int32), ("tmg_coarsen_mask", ctypes.c_int32)]


PRECOND_NONE, PRECOND_SEPARABLE, PRECOND_JACOBI, PRECOND_SEPARABLE_BANDED, PRECOND_TMG = 0, 1, 2, 3, 4


def _precond_code(precond) -> int:
    """None / "none" -> plain CG (Fig. 2); "separable" -> CG with the separable tensor-inverse
    preconditioner; "separable_banded" -> the same with 7-band truncated factors (one fused
    sweep per application); "jacobi" -> CG with the point-Jacobi preconditioner diag(K);
    "tmg" -> CG with one two-grid tensor multigrid cycle per iteration."""
    if precond in (None, "none", PRECOND_NONE):
        return PRECOND_NONE
    if precond in ("separable", PRECOND_SEPARABLE):
        return PRECOND_SEPARABLE
    if precond in ("jacobi", PRECOND_JACOBI):
        return PRECOND_JACOBI
    if precond in ("separable_banded", PRECOND_SEPARABLE_BANDED):
        return PRECOND_SEPARABLE_BANDED
    if precond in ("tmg", PRECOND_TMG):
        return PRECOND_TMG
    raise ValueError(f"unknown preconditioner {precond!r}")


class tca_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("refinements", ctypes.c_int32), ("rel_res_true", ctypes.c_double),
                ("rel_res_recursive", ctypes.c_double), ("seconds", ctypes.c_double),
                ("sweep_ms", ctypes.c_double), ("sweep_launches", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)
_lib.tca_plan.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _i64p, ctypes.POINTER(tca_factor),
                          ctypes.POINTER(tca_reg), ctypes.c_int, _vp]
_lib.tca_plan.restype = ctypes.c_int
for _name in ("tca_apply", "tca_apply_T", "tca_apply_normal"):
    getattr(_lib, _name).argtypes = [_vp, _vp, _vp, _vp]
    getattr(_lib, _name).restype = ctypes.c_int
_lib.tca_plan_scattered.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _i64p, ctypes.c_int64,
                                    ctypes.POINTER(tca_factor), ctypes.POINTER(tca_reg), ctypes.c_int, _vp]
_lib.tca_plan_scattered.restype = ctypes.c_int
_lib.tca_apply_mode.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _i64p, _vp, _vp, _vp]
_lib.tca_apply_mode.restype = ctypes.c_int
_lib.tca_solve.argtypes = [_vp, _vp, _vp, ctypes.POINTER(tca_solve_opts), ctypes.POINTER(tca_solve_info), _vp]
_lib.tca_solve.restype = ctypes.c_int
_lib.tca_solve_batched.argtypes = [ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                   ctypes.POINTER(tca_solve_opts), ctypes.POINTER(tca_solve_info), _vp]
_lib.tca_solve_batched.restype = ctypes.c_int
_lib.tca_autotune_batched.argtypes = [ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                      ctypes.POINTER(tca_solve_opts), ctypes.POINTER(ctypes.c_int), _vp]
_lib.tca_autotune_batched.restype = ctypes.c_int
_lib.tca_autotune.argtypes = [_vp, _vp]
_lib.tca_autotune.restype = ctypes.c_int
_lib.tca_autotuned_chunks.argtypes = [_vp]
_lib.tca_autotuned_chunks.restype = ctypes.c_int
_lib.tca_autotuned_rows.argtypes = [_vp]
_lib.tca_autotuned_rows.restype = ctypes.c_int
_lib.tca_precond_default_shift.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
_lib.tca_precond_default_shift.restype = ctypes.c_int
_lib.tca_apply_shear.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
_lib.tca_apply_shear.restype = ctypes.c_int
_lib.tca_apply_dft.argtypes = [ctypes.c_int, _i64p, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp,
                               _vp]
_lib.tca_apply_dft.restype = ctypes.c_int
_lib.tca_tmg_apply.argtypes = [_vp, _vp, _vp, ctypes.POINTER(tca_solve_opts), _vp]
_lib.tca_tmg_apply.restype = ctypes.c_int
_lib.tca_tmg_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), _i64p]
_lib.tca_tmg_info.restype = ctypes.c_int
_lib.tca_net_param_count.argtypes = []
_lib.tca_net_param_count.restype = ctypes.c_int64
_lib.tca_net_create.argtypes = [ctypes.POINTER(_vp), _vp, _vp]
_lib.tca_net_create.restype = ctypes.c_int
for _name in ("tca_net_set_params", "tca_net_get_params", "tca_net_get_grads"):
    getattr(_lib, _name).argtypes = [_vp, _vp, _vp]
    getattr(_lib, _name).restype = ctypes.c_int
_lib.tca_net_forward.argtypes = [_vp, _i64p, _vp, _vp, _vp]
_lib.tca_net_forward.restype = ctypes.c_int
_lib.tca_net_accumulate.argtypes = [_vp, _i64p, _vp, _vp, _vp]
_lib.tca_net_accumulate.restype = ctypes.c_int
_lib.tca_net_take_loss.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), _vp]
_lib.tca_net_take_loss.restype = ctypes.c_int
_lib.tca_net_adam.argtypes = [_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              _vp]
_lib.tca_net_adam.restype = ctypes.c_int
_lib.tca_solve_net.argtypes = [_vp, _vp, _vp, _vp, ctypes.POINTER(tca_solve_opts), ctypes.c_int,
                               ctypes.POINTER(tca_solve_info), _vp]
_lib.tca_solve_net.restype = ctypes.c_int
_lib.tca_net_use_tensor_cores.argtypes = [_vp, ctypes.c_int]
_lib.tca_net_use_tensor_cores.restype = ctypes.c_int
_lib.tca_net_destroy.argtypes = [_vp]
_lib.tca_net_destroy.restype = None
_lib.tca_rel_residual_noalloc.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp]
_lib.tca_rel_residual_noalloc.restype = ctypes.c_int
_lib.tca_vec_axpby.argtypes = [_vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int64, _vp]
_lib.tca_vec_axpby.restype = ctypes.c_int
_lib.tca_vec_dot.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp]
_lib.tca_vec_dot.restype = ctypes.c_int
_lib.tca_destroy.argtypes = [_vp]
_lib.tca_destroy.restype = None
_lib.tca_status_string.argtypes = [ctypes.c_int]
_lib.tca_status_string.restype = ctypes.c_char_p
_lib.tca_last_error_string.argtypes = []
_lib.tca_last_error_string.restype = ctypes.c_char_p
_lib.tca_kernel_launches.argtypes = [ctypes.c_int]
_lib.tca_kernel_launches.restype = ctypes.c_uint64
_lib.tca_version.argtypes = []
_lib.tca_version.restype = ctypes.c_int
_lib.tca_check_timeout.argtypes = [_vp]
_lib.tca_check_timeout.restype = ctypes.c_int
_lib.tca_wait_selftest.argtypes = [ctypes.c_int64, _vp]
_lib.tca_wait_selftest.restype = ctypes.c_int


class TcaError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = _lib.tca_status_string(status).decode()
        if status == ERR_CUDA:
            msg += f" ({_lib.tca_last_error_string().decode()})"
        super().__init__(f"{what}: {msg}")
        self.status = status


def _check(status: int, what: str, ok=(OK,)) -> int:
    if status not in ok:
        raise TcaError(status, what)
    return status


def _ptr(a) -> int:
    """Raw data pointer of a torch tensor or NumPy array (must be contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)!r}")


def _stream(stream) -> int:
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    try:
        import torch

        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover - torch missing
        pass
    return 0


def version() -> int:
    return _lib.tca_version()


def kernel_launches(reset: bool = False) -> int:
    return int(_lib.tca_kernel_launches(1 if reset else 0))


def check_timeout(stream=None) -> int:
    """Synchronise the stream; ERR_TIMEOUT (flag cleared) if a bounded device wait gave up, else OK."""
    return int(_lib.tca_check_timeout(_stream(stream)))


def wait_selftest(polls: int, stream=None) -> int:
    """Run a bounded wait that cannot succeed (at most `polls` polls); returns its status (ERR_TIMEOUT)."""
    return int(_lib.tca_wait_selftest(int(polls), _stream(stream)))


def _check_noalloc_args(rhs, kx, out) -> int:
    """Length n of the no-alloc residual's operands; ValueError unless rhs, kx and out
    are contiguous float64 CUDA tensors on one device with kx.numel() == n and out
    holding at least one value (the kernel reads n doubles of each and writes one)."""
    bufs = {"rhs": rhs, "kx": kx, "out": out}
    for name, t in bufs.items():
        if not (hasattr(t, "is_cuda") and hasattr(t, "dtype") and hasattr(t, "numel")):
            raise ValueError(f"{name} must be a torch CUDA tensor, got {type(t).__name__}")
        if not t.is_cuda:
            raise ValueError(f"{name} must live in device memory (got a host tensor)")
        if str(t.dtype) != "torch.float64":
            raise ValueError(f"{name} must be float64, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if len({t.device for t in bufs.values()}) != 1:
        raise ValueError("rhs, kx and out must be on the same device")
    n = int(rhs.numel())
    if int(kx.numel()) != n:
        raise ValueError(f"kx holds {kx.numel()} values, rhs {n}")
    if int(out.numel()) < 1:
        raise ValueError("out must hold at least one value")
    return n


def rel_residual_noalloc(rhs, kx, out, stream=None) -> int:
    """||rhs - kx|| / ||rhs|| of two FP64 device vectors into out (one FP64 device value).

    For callers that must not allocate device memory at this point: the library
    keeps the reduction scratch in a fixed device array of its own.  rhs, kx and
    out must be contiguous float64 torch CUDA tensors on one device (ValueError
    otherwise, before anything reaches the library).
    """
    n = _check_noalloc_args(rhs, kx, out)
    return _check(_lib.tca_rel_residual_noalloc(_ptr(rhs), _ptr(kx), n, _ptr(out), _stream(stream)),
                  "tca_rel_residual_noalloc")


def vec_axpby(y, x, a: float, b: float, stream=None):
    """y = a x + b y on float32 CUDA tensors of equal length (one library kernel)."""
    if y.numel() != x.numel():
        raise ValueError("x and y differ in length")
    _check(_lib.tca_vec_axpby(_ptr(y), _ptr(x), float(a), float(b), int(y.numel()), _stream(stream)), "tca_vec_axpby")
    return y


def vec_dot(a, b, out, stream=None):
    """out[0] = <a, b> (FP64 sum of FP32 products) for float32 CUDA tensors; out: a float64 CUDA tensor."""
    if a.numel() != b.numel() or out.numel() < 1:
        raise ValueError("a and b differ in length, or out is empty")
    _check(_lib.tca_vec_dot(_ptr(a), _ptr(b), int(a.numel()), _ptr(out), _stream(stream)), "tca_vec_dot")
    return out


SHEAR_KINDS = {"linear": 1, "cubic": 3}


def apply_shear(x, y, mode_a: int, mode_b: int, slope: float, center: float, kind="linear", stream=None):
    """y = the 1D shear transform of x along mode_a driven by mode_b (tca_apply_shear): every line
    along mode_a resampled at i_a - slope (i_b - center), linear or cubic-convolution kernel.
    x, y: contiguous CUDA tensors of one shape, both float32 or both float64."""
    if tuple(x.shape) != tuple(y.shape) or x.dtype != y.dtype:
        raise ValueError("x and y must have the same shape and dtype")
    if not (x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x and y must be contiguous")
    name = str(x.dtype)
    if name not in ("torch.float32", "torch.float64"):
        raise ValueError("float32 or float64 tensors")
    prec = F64 if name == "torch.float64" else F32
    dims = (ctypes.c_int64 * x.dim())(*[int(v) for v in x.shape])
    code = SHEAR_KINDS.get(kind, kind)
    _check(_lib.tca_apply_shear(x.dim(), dims, int(mode_a), int(mode_b), float(slope), float(center), int(code), prec,
                                _ptr(x), _ptr(y), _stream(stream)), "tca_apply_shear")
    return y


def apply_dft(re, im, re_out, im_out, modes, inverse: bool = False, stream=None):
    """(re_out, im_out) = the DFT of re + i im over ``modes`` (tca_apply_dft; im may be None for a
    real input): contiguous CUDA tensors of one shape, all float32 or all float64."""
    bufs = [t for t in (re, im, re_out, im_out) if t is not None]
    if any(tuple(t.shape) != tuple(re.shape) or t.dtype != re.dtype or not t.is_contiguous() for t in bufs):
        raise ValueError("re, im, re_out and im_out must be contiguous tensors of one shape and dtype")
    name = str(re.dtype)
    if name not in ("torch.float32", "torch.float64"):
        raise ValueError("float32 or float64 tensors")
    prec = F64 if name == "torch.float64" else F32
    mask = 0
    for k in modes:
        mask |= 1 << int(k)
    dims = (ctypes.c_int64 * re.dim())(*[int(v) for v in re.shape])
    _check(_lib.tca_apply_dft(re.dim(), dims, mask, 1 if inverse else 0, prec, _ptr(re),
                              None if im is None else _ptr(im), _ptr(re_out), _ptr(im_out), _stream(stream)),
           "tca_apply_dft")
    return re_out, im_out


def exported_symbols() -> list[str]:
    return ["tca_plan", "tca_plan_scattered", "tca_apply", "tca_apply_T", "tca_apply_normal", "tca_apply_mode", "tca_solve",
            "tca_solve_batched", "tca_autotune_batched", "tca_autotune", "tca_autotuned_chunks", "tca_autotuned_rows", "tca_precond_default_shift", "tca_tmg_apply", "tca_tmg_info", "tca_apply_shear", "tca_apply_dft", "tca_rel_residual_noalloc", "tca_destroy",
            "tca_net_param_count", "tca_net_create", "tca_net_set_params", "tca_net_get_params", "tca_net_get_grads",
            "tca_net_forward", "tca_net_accumulate", "tca_net_take_loss", "tca_net_adam", "tca_solve_net",
            "tca_net_use_tensor_cores", "tca_net_destroy", "tca_check_timeout", "tca_wait_selftest",
            "tca_status_string", "tca_last_error_string", "tca_kernel_launches", "tca_version", "tca_vec_axpby",
            "tca_vec_dot"]


class Factor:
    """Host copy of one mode's factor in the layout tca_factor describes."""

    def __init__(self, kind: int, m: int, n: int, values: np.ndarray, col0: np.ndarray | None = None):
        self.kind = kind
        self.m = int(m)
        self.n = int(n)
        self.values = np.ascontiguousarray(values, dtype=np.float64)
        self.col0 = None if col0 is None else np.ascontiguousarray(col0, dtype=np.int32)

    @classmethod
    def from_synth(cls, f) -> "Factor":
        if f.kind == "dense":
            return cls(FACTOR_DENSE, f.m, f.n, np.asarray(f.a))
        return cls(FACTOR_ELL4, f.m, f.n, np.asarray(f.w), np.asarray(f.col0))


class Plan:
    """A tca plan: ordered spaces, separable operator, regulariser and precision."""

    def __init__(self, shape, factors, lam: float = 0.0, reg_mask: int | None = None, precision="f32",
                 stream=None):
        self.shape = tuple(int(s) for s in shape)
        self.order = len(self.shape)
        self.factors = [f if isinstance(f, Factor) else Factor.from_synth(f) for f in factors]
        self.sample_shape = tuple(f.m for f in self.factors)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.dtype = np.float64 if self.precision == F64 else np.float32
        arr = (tca_factor * self.order)()
        for k, f in enumerate(self.factors):
            arr[k].kind = f.kind
            arr[k].reserved = 0
            arr[k].m = f.m
            arr[k].n = f.n
            arr[k].values = f.values.ctypes.data
            arr[k].col0 = f.col0.ctypes.data if f.col0 is not None else None
        n = (ctypes.c_int64 * self.order)(*self.shape)
        reg = tca_reg(float(lam), (1 << self.order) - 1 if reg_mask is None else int(reg_mask), 0)
        h = _vp()
        _check(_lib.tca_plan(ctypes.byref(h), self.order, n, arr, ctypes.byref(reg), self.precision,
                             _stream(stream)), "tca_plan")
        self._h = h
        self.lam = float(lam)

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.tca_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, x, y, stream=None):
        _check(_lib.tca_apply(self._h, _ptr(x), _ptr(y), _stream(stream)), "tca_apply")
        return y

    def apply_T(self, y, x, stream=None):
        _check(_lib.tca_apply_T(self._h, _ptr(y), _ptr(x), _stream(stream)), "tca_apply_T")
        return x

    def apply_normal(self, x, y, stream=None):
        _check(_lib.tca_apply_normal(self._h, _ptr(x), _ptr(y), _stream(stream)), "tca_apply_normal")
        return y

    def apply_mode(self, mode: int, op: int, dims, x, y, stream=None):
        d = (ctypes.c_int64 * self.order)(*[int(v) for v in dims])
        _check(_lib.tca_apply_mode(self._h, int(mode), int(op), d, _ptr(x), _ptr(y), _stream(stream)),
               "tca_apply_mode")
        return y

    def solve(self, b, x, rtol: float = 1e-6, max_iter: int = 10000, x0_given: bool = False,
              check_every: int = 0, inner_rtol: float = 0.0, max_refine: int = 0, stream=None,
              raise_on_error: bool = True, profile: bool = False, precond=None, precond_shift: float = 0.0,
              tmg_nu: int = 0, tmg_coarse_rtol: float = 0.0, tmg_lambda_max: float = 0.0,
              tmg_coarsen_mask: int = 0):
        """Solve (A^T A + lambda R) x = A^T b; returns (status, info dict).

        precond: None (the CG of Fig. 2), "jacobi", "separable" / "separable_banded" (the separable
        tensor-inverse preconditioner, shift ``precond_shift``, 0 for the plan's corner-model
        default) or "tmg" (a two-grid tensor multigrid cycle; the tmg_* arguments, 0 for each
        default)."""
        opts = tca_solve_opts(float(rtol), int(max_iter), 1 if x0_given else 0, float(inner_rtol),
                              int(max_refine), int(check_every), 1 if profile else 0, _precond_code(precond),
                              float(precond_shift), float(tmg_coarse_rtol), float(tmg_lambda_max), int(tmg_nu),
                              int(tmg_coarsen_mask))
        info = tca_solve_info()
        st = _lib.tca_solve(self._h, _ptr(b), _ptr(x), ctypes.byref(opts), ctypes.byref(info), _stream(stream))
        if raise_on_error:
            _check(st, "tca_solve", ok=(OK, ERR_NOT_CONVERGED))
        return st, _info_dict(info)

    def autotune(self, stream=None) -> int:
        """Time the CG sweep's tile extents (and, bfloat16 plans, worker layouts) on this GPU and
        keep the fastest; returns the chunk count chosen (0: none)."""
        _check(_lib.tca_autotune(self._h, _stream(stream)), "tca_autotune")
        return int(_lib.tca_autotuned_chunks(self._h))

    def autotuned_rows(self) -> int:
        """Core rows per worker thread the autotuner chose for a bfloat16 plan (0: not tuned)."""
        return int(_lib.tca_autotuned_rows(self._h))

    def precond_default_shift(self) -> float:
        """The shift the separable preconditioners take when none is given (the plan's corner model)."""
        v = ctypes.c_double(0.0)
        _check(_lib.tca_precond_default_shift(self._h, ctypes.byref(v)), "tca_precond_default_shift")
        return float(v.value)

    def tmg_apply(self, r, z, nu: int = 0, coarse_rtol: float = 0.0, lambda_max: float = 0.0,
                  coarsen_mask: int = 0, stream=None):
        """One tensor multigrid cycle z = V r (device buffers of the plan's element type)."""
        opts = tca_solve_opts(tmg_coarse_rtol=float(coarse_rtol), tmg_lambda_max=float(lambda_max),
                              tmg_nu=int(nu), tmg_coarsen_mask=int(coarsen_mask))
        _check(_lib.tca_tmg_apply(self._h, _ptr(r), _ptr(z), ctypes.byref(opts), _stream(stream)), "tca_tmg_apply")
        return z

    def tmg_info(self) -> dict:
        """lambda_max of D^-1 K the multigrid smoother uses and the coarse CG iterations since the
        last solve (or cycle) started."""
        lam = ctypes.c_double(0.0)
        its = ctypes.c_int64(0)
        _check(_lib.tca_tmg_info(self._h, ctypes.byref(lam), ctypes.byref(its)), "tca_tmg_info")
        return {"lambda_max": float(lam.value), "coarse_iters": int(its.value)}


class ScatteredPlan(Plan):
    """A plan for scattered samples: per mode k the m x n_k ELL-4 rows (col0s[k], ws[k]) of the
    samples' weights; the system tensor's rows are the Kronecker products of those rows."""

    def __init__(self, shape, col0s, ws, lam: float = 0.0, reg_mask: int | None = None, precision="f64",
                 stream=None):
        self.shape = tuple(int(v) for v in shape)
        self.order = len(self.shape)
        m = int(np.asarray(col0s[0]).shape[0])
        self.factors = []
        for c, w, n in zip(col0s, ws, self.shape):
            c = np.asarray(c, dtype=np.int32)
            w = np.asarray(w, dtype=np.float64)
            if w.shape != (c.shape[0], 4):
                raise ValueError(f"ELL-4 weights of shape {w.shape} for {c.shape[0]} rows")
            # each mode carries its own row count; the library checks they all equal m
            self.factors.append(Factor(FACTOR_ELL4, c.shape[0], n, w, c))
        self.sample_shape = (m,)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.dtype = np.float64 if self.precision == F64 else np.float32
        arr = (tca_factor * self.order)()
        for k, f in enumerate(self.factors):
            arr[k].kind, arr[k].reserved, arr[k].m, arr[k].n = f.kind, 0, f.m, f.n
            arr[k].values = f.values.ctypes.data
            arr[k].col0 = f.col0.ctypes.data
        n = (ctypes.c_int64 * self.order)(*self.shape)
        reg = tca_reg(float(lam), (1 << self.order) - 1 if reg_mask is None else int(reg_mask), 0)
        h = _vp()
        _check(_lib.tca_plan_scattered(ctypes.byref(h), self.order, n, m, arr, ctypes.byref(reg), self.precision,
                                       _stream(stream)), "tca_plan_scattered")
        self._h = h
        self.lam = float(lam)


def _info_dict(info) -> dict:
    return {"iters": info.iters, "refinements": info.refinements, "rel_res_true": info.rel_res_true,
            "rel_res_recursive": info.rel_res_recursive, "seconds": info.seconds,
            "sweep_ms": info.sweep_ms, "sweep_launches": info.sweep_launches}


def solve_batched(plans, bs, xs, rtol: float = 1e-6, max_iter: int = 10000, x0_given: bool = False,
                  check_every: int = 16, stream=None, raise_on_error: bool = True, precond=None,
                  precond_shift: float = 0.0):
    """Solve every plans[i] system for bs[i] into xs[i] in one graph launch; returns (status, [info dicts])."""
    count = len(plans)
    if not (len(bs) == count == len(xs)) or count == 0:
        raise ValueError("plans, bs and xs must be non-empty and of equal length")
    hp = (_vp * count)(*[p.handle for p in plans])
    bp = (_vp * count)(*[_ptr(b) for b in bs])
    xp = (_vp * count)(*[_ptr(x) for x in xs])
    opts = tca_solve_opts(float(rtol), int(max_iter), 1 if x0_given else 0, 0.0, 0, int(check_every), 0,
                          _precond_code(precond), float(precond_shift))
    infos = (tca_solve_info * count)()
    st = _lib.tca_solve_batched(count, hp, bp, xp, ctypes.byref(opts), infos, _stream(stream))
    if raise_on_error:
        _check(st, "tca_solve_batched", ok=(OK, ERR_NOT_CONVERGED))
    return st, [_info_dict(i) for i in infos]


def autotune_batched(plans, bs, xs, rtol: float = 1e-6, max_iter: int = 10000, x0_given: bool = False,
                     check_every: int = 16, stream=None, precond=None, precond_shift: float = 0.0) -> int:
    """Time the batch at each SM share and keep the fastest for these plans, buffers and options
    (later solve_batched calls with the same arguments use it); returns the share's denominator."""
    count = len(plans)
    if not (len(bs) == count == len(xs)) or count == 0:
        raise ValueError("plans, bs and xs must be non-empty and of equal length")
    hp = (_vp * count)(*[p.handle for p in plans])
    bp = (_vp * count)(*[_ptr(b) for b in bs])
    xp = (_vp * count)(*[_ptr(x) for x in xs])
    opts = tca_solve_opts(float(rtol), int(max_iter), 1 if x0_given else 0, 0.0, 0, int(check_every), 0,
                          _precond_code(precond), float(precond_shift))
    share = ctypes.c_int(0)
    _check(_lib.tca_autotune_batched(count, hp, bp, xp, ctypes.byref(opts), ctypes.byref(share), _stream(stream)),
           "tca_autotune_batched")
    return int(share.value)


def plan_from_instance(inst, precision="f32", reg_mask=None, stream=None) -> Plan:
    """Plan for a synthetic ``synth.Instance``."""
    return Plan(inst.shape, inst.factors, lam=inst.lam, reg_mask=reg_mask, precision=precision, stream=stream)


def _dims4(shape) -> ctypes.Array:
    shape = tuple(int(v) for v in shape)
    if len(shape) == 3:
        shape = shape + (1,)
    if len(shape) != 4:
        raise ValueError("network tensors are 3D or 4D")
    return (ctypes.c_int64 * 4)(*shape)


class Net:
    """The 4-layer 3x3x3 convolutional network that supplies the CG initial guess."""

    def __init__(self, params, stream=None):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.param_count():
            raise ValueError(f"expected {self.param_count()} parameters, got {p.size}")
        h = _vp()
        _check(_lib.tca_net_create(ctypes.byref(h), p.ctypes.data, _stream(stream)), "tca_net_create")
        self._h = h

    @staticmethod
    def param_count() -> int:
        return int(_lib.tca_net_param_count())

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.tca_net_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass

    def use_tensor_cores(self, enable: bool = True):
        _check(_lib.tca_net_use_tensor_cores(self._h, 1 if enable else 0), "tca_net_use_tensor_cores")

    def params(self, stream=None) -> np.ndarray:
        out = np.empty(self.param_count(), np.float32)
        _check(_lib.tca_net_get_params(self._h, out.ctypes.data, _stream(stream)), "tca_net_get_params")
        return out

    def set_params(self, params, stream=None):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(_lib.tca_net_set_params(self._h, p.ctypes.data, _stream(stream)), "tca_net_set_params")

    def grads(self, stream=None) -> np.ndarray:
        out = np.empty(self.param_count(), np.float32)
        _check(_lib.tca_net_get_grads(self._h, out.ctypes.data, _stream(stream)), "tca_net_get_grads")
        return out

    def forward(self, u, y, stream=None):
        _check(_lib.tca_net_forward(self._h, _dims4(u.shape), _ptr(u), _ptr(y), _stream(stream)), "tca_net_forward")
        return y

    def accumulate(self, u, t, stream=None):
        _check(_lib.tca_net_accumulate(self._h, _dims4(u.shape), _ptr(u), _ptr(t), _stream(stream)),
               "tca_net_accumulate")

    def take_loss(self, stream=None) -> float:
        v = ctypes.c_double()
        _check(_lib.tca_net_take_loss(self._h, ctypes.byref(v), _stream(stream)), "tca_net_take_loss")
        return float(v.value)

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, grad_scale: float = 1.0,
             stream=None):
        _check(_lib.tca_net_adam(self._h, lr, beta1, beta2, eps, grad_scale, _stream(stream)), "tca_net_adam")

    def solve(self, plan: "Plan", b, x, rtol: float = 1e-6, max_iter: int = 10000, check_every: int = 0,
              inner_rtol: float = 0.0, max_refine: int = 0, net_every: int = 0, stream=None,
              raise_on_error: bool = True, profile: bool = False, precond=None, precond_shift: float = 0.0):
        """tca_solve from x0 = s Net(A^T b / s), plus a network step every net_every iterations (0: none)."""
        opts = tca_solve_opts(float(rtol), int(max_iter), 1, float(inner_rtol), int(max_refine), int(check_every),
                              1 if profile else 0, _precond_code(precond), float(precond_shift))
        info = tca_solve_info()
        st = _lib.tca_solve_net(plan.handle, self._h, _ptr(b), _ptr(x), ctypes.byref(opts), int(net_every),
                                ctypes.byref(info), _stream(stream))
        if raise_on_error:
            _check(st, "tca_solve_net", ok=(OK, ERR_NOT_CONVERGED))
        return st, _info_dict(info)
