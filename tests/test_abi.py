"""The C-ABI library loads and exports every symbol include/*.h declares (no GPU needed).

Also exercises the argument checks that return before any device work.
"""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tca():
    from paper_1001_5460_gb300 import build

    build.build()
    from paper_1001_5460_gb300 import tca as t

    return t


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"^TCA_API\s+[\w\s\*]+?\b(tca_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("tca_plan", "tca_apply", "tca_apply_T", "tca_apply_normal", "tca_solve", "tca_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(tca):
    lib = ctypes.CDLL(tca.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def _header_struct_fields(name):
    text = open(os.path.join(ROOT, "include", "tca.h")).read()
    head = re.split(r"\}\s*" + name + ";", text)[0]
    body = head.rsplit("typedef struct {", 1)[1]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return re.findall(r"^\s*(double|int32_t|int64_t|float)\s+(\w+);", body, flags=re.M)


def test_binding_structs_match_the_header(tca):
    """The ctypes mirrors of tca_solve_opts / tca_solve_info list the header's fields in order,
    with the same C types (a mismatch would shift every later field across the ABI)."""
    ctype = {"double": ctypes.c_double, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64,
             "float": ctypes.c_float}
    for name, cls in (("tca_solve_opts", tca.tca_solve_opts), ("tca_solve_info", tca.tca_solve_info)):
        fields = _header_struct_fields(name)
        assert [(f, ctype[t]) for t, f in fields] == list(cls._fields_), name


def test_precond_names(tca):
    assert tca._precond_code(None) == tca.PRECOND_NONE
    assert tca._precond_code("separable") == tca.PRECOND_SEPARABLE
    assert tca._precond_code("jacobi") == tca.PRECOND_JACOBI
    assert tca._precond_code("tmg") == tca.PRECOND_TMG
    with pytest.raises(ValueError):
        tca._precond_code("multigrid-typo")


def test_status_strings_and_version(tca):
    assert tca._lib.tca_status_string(0) == b"ok"
    assert tca._lib.tca_status_string(tca.ERR_SHAPE) == b"shape mismatch"
    assert tca._lib.tca_status_string(99) == b"unknown status"
    assert tca.version() >> 16 == 1


def test_plan_rejects_bad_arguments_before_device_work(tca):
    fac = (tca.tca_factor * 3)()
    vals = np.ones((4, 3))
    for k in range(3):
        fac[k].kind = tca.FACTOR_DENSE
        fac[k].m, fac[k].n = 4, 3
        fac[k].values = vals.ctypes.data
    n = (ctypes.c_int64 * 3)(3, 3, 3)
    h = ctypes.c_void_p()
    reg = tca.tca_reg(0.1, 7, 0)
    # order must be 3 or 4
    assert tca._lib.tca_plan(ctypes.byref(h), 2, n, fac, ctypes.byref(reg), tca.F32, None) == tca.ERR_INVALID_ARG
    # factor n must match the space size
    n_bad = (ctypes.c_int64 * 3)(3, 5, 3)
    assert tca._lib.tca_plan(ctypes.byref(h), 3, n_bad, fac, ctypes.byref(reg), tca.F32, None) == tca.ERR_SHAPE
    # unknown precision, negative lambda, null pointers
    assert tca._lib.tca_plan(ctypes.byref(h), 3, n, fac, ctypes.byref(reg), 9, None) == tca.ERR_INVALID_ARG
    reg_neg = tca.tca_reg(-1.0, 7, 0)
    assert tca._lib.tca_plan(ctypes.byref(h), 3, n, fac, ctypes.byref(reg_neg), tca.F32, None) == tca.ERR_INVALID_ARG
    assert tca._lib.tca_plan(None, 3, n, fac, ctypes.byref(reg), tca.F32, None) == tca.ERR_INVALID_ARG
    fac[1].reserved = 1
    assert tca._lib.tca_plan(ctypes.byref(h), 3, n, fac, ctypes.byref(reg), tca.F32, None) == tca.ERR_INVALID_ARG
    # entry points reject a null plan
    assert tca._lib.tca_apply(None, None, None, None) == tca.ERR_INVALID_ARG
    assert tca._lib.tca_solve(None, None, None, None, None, None) == tca.ERR_INVALID_ARG
    shift = ctypes.c_double(0.0)
    assert tca._lib.tca_precond_default_shift(None, ctypes.byref(shift)) == tca.ERR_INVALID_ARG
    opts = tca.tca_solve_opts()
    assert tca._lib.tca_tmg_apply(None, None, None, ctypes.byref(opts), None) == tca.ERR_INVALID_ARG
    assert tca._lib.tca_tmg_info(None, ctypes.byref(shift), None) == tca.ERR_INVALID_ARG
    dims = (ctypes.c_int64 * 3)(4, 5, 6)
    bad = ctypes.c_void_p(16)
    other = ctypes.c_void_p(32)
    shear = tca._lib.tca_apply_shear
    assert shear(3, dims, 0, 1, 0.5, 2.0, 1, tca.F32, None, other, None) == tca.ERR_INVALID_ARG
    assert shear(3, dims, 0, 1, 0.5, 2.0, 1, tca.F32, bad, bad, None) == tca.ERR_INVALID_ARG    # aliased
    assert shear(1, dims, 0, 1, 0.5, 2.0, 1, tca.F32, bad, other, None) == tca.ERR_INVALID_ARG  # order
    assert shear(3, dims, 1, 1, 0.5, 2.0, 1, tca.F32, bad, other, None) == tca.ERR_INVALID_ARG  # same mode
    assert shear(3, dims, 0, 3, 0.5, 2.0, 1, tca.F32, bad, other, None) == tca.ERR_INVALID_ARG  # mode range
    assert shear(3, dims, 0, 1, 0.5, 2.0, 2, tca.F32, bad, other, None) == tca.ERR_INVALID_ARG  # kind
    assert shear(3, dims, 0, 1, float("nan"), 2.0, 1, tca.F32, bad, other, None) == tca.ERR_INVALID_ARG
    assert shear(3, dims, 0, 1, 0.5, 2.0, 1, tca.BF16_IR, bad, other, None) == tca.ERR_INVALID_ARG
    zero = (ctypes.c_int64 * 3)(4, 0, 6)
    assert shear(3, zero, 0, 1, 0.5, 2.0, 1, tca.F32, bad, other, None) == tca.ERR_SHAPE
    dft = tca._lib.tca_apply_dft
    third = ctypes.c_void_p(48)
    fourth = ctypes.c_void_p(64)
    assert dft(3, dims, 0b011, 0, tca.F32, None, None, other, third, None) == tca.ERR_INVALID_ARG
    assert dft(3, dims, 0, 0, tca.F32, bad, None, other, third, None) == tca.ERR_INVALID_ARG       # empty mask
    assert dft(3, dims, 0b1000, 0, tca.F32, bad, None, other, third, None) == tca.ERR_INVALID_ARG  # past order
    assert dft(3, dims, 0b001, 0, tca.F32, bad, other, other, third, None) == tca.ERR_INVALID_ARG  # aliasing
    assert dft(3, dims, 0b001, 0, tca.F32, bad, None, other, other, None) == tca.ERR_INVALID_ARG
    assert dft(3, dims, 0b001, 0, tca.TF32_IR, bad, fourth, other, third, None) == tca.ERR_INVALID_ARG
    assert dft(3, zero, 0b001, 0, tca.F32, bad, fourth, other, third, None) == tca.ERR_SHAPE
    # scattered plans: order, negative sample count, precision
    assert tca._lib.tca_plan_scattered(ctypes.byref(h), 2, n, 5, fac, ctypes.byref(reg), tca.F64,
                                       None) == tca.ERR_INVALID_ARG
    assert tca._lib.tca_plan_scattered(ctypes.byref(h), 3, n, -1, fac, ctypes.byref(reg), tca.F64,
                                       None) == tca.ERR_INVALID_ARG
    assert tca._lib.tca_plan_scattered(ctypes.byref(h), 3, n, 5, fac, ctypes.byref(reg), tca.BF16_IR,
                                       None) == tca.ERR_UNSUPPORTED
    tca._lib.tca_destroy(None)  # NULL is ignored


def test_product_path_has_no_cpu_fallback():
    """The binding imports nothing from the oracle and the library sources name no oracle."""
    pkg = os.path.join(ROOT, "paper_1001_5460_gb300")
    for path in glob.glob(os.path.join(pkg, "*.py")) + glob.glob(os.path.join(pkg, "csrc", "*")):
        text = open(path).read()
        assert "import oracle" not in text and "from oracle" not in text, path


def test_net_entry_points_check_arguments(tca):
    from oracle import net_oracle as NO

    assert tca.Net.param_count() == NO.n_params()
    h = ctypes.c_void_p()
    assert tca._lib.tca_net_create(ctypes.byref(h), None, None) == tca.ERR_INVALID_ARG
    assert tca._lib.tca_net_create(None, None, None) == tca.ERR_INVALID_ARG
    assert tca._lib.tca_net_forward(None, None, None, None, None) == tca.ERR_INVALID_ARG
    assert tca._lib.tca_net_accumulate(None, None, None, None, None) == tca.ERR_INVALID_ARG
    assert tca._lib.tca_net_adam(None, 1e-3, 0.9, 0.999, 1e-8, 1.0, None) == tca.ERR_INVALID_ARG
    assert tca._lib.tca_solve_net(None, None, None, None, None, 0, None, None) == tca.ERR_INVALID_ARG
    assert tca._lib.tca_solve_batched(0, None, None, None, None, None, None) == tca.ERR_INVALID_ARG
    assert tca._lib.tca_autotune(None, None) == tca.ERR_INVALID_ARG
    tca._lib.tca_net_destroy(None)


def test_net_init_params_layout():
    from oracle import net_oracle as NO
    from paper_1001_5460_gb300 import synth

    p = synth.net_init_params(3)
    assert p.dtype == np.float32 and p.size == NO.n_params()
    layers = NO.unpack_params(p.astype(np.float64))
    for li, ((w, b), (ci, co)) in enumerate(zip(layers, NO.LAYERS)):
        assert w.shape == (co, ci, 3, 3, 3) and not b.any()
        std = np.sqrt(2.0 / (27 * ci)) * (0.1 if li == 3 else 1.0)
        assert abs(w.std() / std - 1.0) < 0.25


def test_noalloc_binding_rejects_bad_buffers_before_the_call(tca):
    """rel_residual_noalloc hands raw pointers to a kernel that reads n doubles of rhs and kx
    and writes one to out: host arrays, host tensors, other dtypes, a shorter kx or an empty
    out are refused in Python, before anything reaches the library."""
    import torch

    class FakeDev:
        """Stands in for a CUDA tensor (none exists on this machine); never reaches the library."""

        def __init__(self, n, dtype=torch.float64, device="cuda:0", contiguous=True):
            self.is_cuda, self.dtype, self.device, self._n, self._c = True, dtype, device, n, contiguous

        def numel(self):
            return self._n

        def is_contiguous(self):
            return self._c

        def data_ptr(self):  # pragma: no cover - a call getting here is the failure
            raise AssertionError("validation let a bad buffer through")

    good = FakeDev(8)
    h = np.zeros(8)
    with pytest.raises(ValueError, match="torch CUDA tensor"):
        tca.rel_residual_noalloc(h, good, FakeDev(1))
    with pytest.raises(ValueError, match="device memory"):
        tca.rel_residual_noalloc(torch.zeros(8, dtype=torch.float64), good, FakeDev(1))
    with pytest.raises(ValueError, match="float64"):
        tca.rel_residual_noalloc(FakeDev(8, dtype=torch.float32), good, FakeDev(1))
    with pytest.raises(ValueError, match="kx holds"):
        tca.rel_residual_noalloc(good, FakeDev(7), FakeDev(1))
    with pytest.raises(ValueError, match="at least one"):
        tca.rel_residual_noalloc(good, FakeDev(8), FakeDev(0))
    with pytest.raises(ValueError, match="same device"):
        tca.rel_residual_noalloc(good, FakeDev(8, device="cuda:1"), FakeDev(1))
    with pytest.raises(ValueError, match="contiguous"):
        tca.rel_residual_noalloc(good, FakeDev(8, contiguous=False), FakeDev(1))


def test_shear_and_dft_bindings_check_buffers_in_python(tca):
    """apply_shear and apply_dft refuse mismatched shapes, dtypes and non-contiguous buffers in
    Python; host tensors that pass those checks are refused by the library (host memory) before
    any device work."""
    import torch

    x = torch.zeros((4, 6), dtype=torch.float32)
    with pytest.raises(ValueError):
        tca.apply_shear(x, torch.zeros((6, 4), dtype=torch.float32), 0, 1, 0.5, 2.0)
    with pytest.raises(ValueError):
        tca.apply_shear(x, torch.zeros((4, 6), dtype=torch.float64), 0, 1, 0.5, 2.0)
    with pytest.raises(ValueError):
        tca.apply_shear(x, torch.zeros((6, 4), dtype=torch.float32).t(), 0, 1, 0.5, 2.0)
    with pytest.raises(ValueError):
        tca.apply_shear(x.to(torch.int32), torch.zeros((4, 6), dtype=torch.int32), 0, 1, 0.5, 2.0)
    with pytest.raises(tca.TcaError) as e:
        tca.apply_shear(x, torch.zeros((4, 6), dtype=torch.float32), 0, 1, 0.5, 2.0)
    assert e.value.status == tca.ERR_INVALID_ARG
    y, z = torch.zeros((4, 6)), torch.zeros((4, 6))
    with pytest.raises(ValueError):
        tca.apply_dft(x, None, y, torch.zeros((4, 7)), (0,))
    with pytest.raises(ValueError):
        tca.apply_dft(x, torch.zeros((4, 6), dtype=torch.float64), y, z, (0,))
    with pytest.raises(tca.TcaError) as e:
        tca.apply_dft(x, None, y, z, (0, 1))
    assert e.value.status == tca.ERR_INVALID_ARG
