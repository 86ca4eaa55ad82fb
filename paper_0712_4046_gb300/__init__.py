"""Python binding of the GB300 multipoint Kronecker-substitution library.

Thin ctypes marshalling over the C ABI declared in ``include/ks.h``: every
step of the product runs in the library's CUDA kernels.  Polynomials are
torch tensors of shape ``(L, limbs)`` holding the uint64 limbs (dtype int64 or
uint64; the bits are what count).  There is no CPU fallback: if ``libks.so``
is missing the import fails.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libks.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError("paper_0712_4046_gb300: %s is not built; run "
                      "`python -c 'import __graft_entry__ as g; g.build()'` first" % _LIB_PATH)

lib = ctypes.CDLL(_LIB_PATH)

KS_AUTO, KS_1, KS_2, KS_3, KS_4 = 0, 1, 2, 3, 4
KS_C = 5  # complex evaluation points (Sec. 2.5), ks_mul_bivariate_mod only
ENGINE_AUTO, ENGINE_SCHOOLBOOK, ENGINE_NTT, ENGINE_TC = 0, 1, 2, 3
KS_OK, KS_EINVAL, KS_ERANGE, KS_ENOMEM, KS_ECUDA, KS_ETIMEOUT, KS_ENOTSUP = 0, -1, -2, -3, -4, -5, -6

_i64, _ci, _vp, _u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64


class KSProblem(ctypes.Structure):
    _fields_ = [("h", _vp), ("f", _vp), ("g", _vp), ("len_f", _i64), ("len_g", _i64),
                ("coeff_bits", ctypes.c_int32), ("is_signed", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("coeff_bits_g", ctypes.c_int32)]


def _sig(name, res, *args):
    fn = getattr(lib, name)
    fn.restype = res
    fn.argtypes = list(args)
    return fn


_sig("ks_out_limbs", _ci, _i64, _i64, _ci, _ci)
_sig("ks_out_limbs_bits", _ci, _i64, _i64, _ci, _ci, _ci)
_sig("ks_eval_bits", _ci, _i64, _i64, _ci, _ci)
_sig("ks_workspace_bytes", _i64, _i64, _i64, _ci, _ci, _ci, _ci)
_sig("ks_mul", _ci, _vp, _vp, _i64, _vp, _i64, _ci, _ci, _ci, _vp)
_sig("ks_mul_ex", _ci, _vp, _vp, _i64, _vp, _i64, _ci, _ci, _ci, _ci, _vp, _i64, _vp)
_sig("ks_mul_host", _ci, _vp, _vp, _i64, _vp, _i64, _ci, _ci, _ci, _ci, _vp)
_sig("ks_mul_mod", _ci, _vp, _vp, _i64, _vp, _i64, _u64, _ci, _vp)
_sig("ks_mul_bivariate_mod", _ci, _vp, _vp, _vp, _i64, _i64, _u64, _ci, _vp)
_sig("ks_mul_bits", _ci, _vp, _vp, _i64, _ci, _vp, _i64, _ci, _ci, _ci, _vp)
_sig("ks_mul_batch", _ci, ctypes.POINTER(KSProblem), _i64, _vp)
_sig("ks_plan_create", _ci, ctypes.POINTER(_vp), ctypes.POINTER(KSProblem), _i64, _ci)
_sig("ks_plan_execute", _ci, _vp, _vp)
_sig("ks_plan_capture", _ci, _vp, _vp)
_sig("ks_plan_launches", ctypes.c_longlong, _vp)
_sig("ks_plan_workspace_bytes", _i64, _vp)
_sig("ks_plan_choice", _ci, _vp, _i64, ctypes.POINTER(_ci), ctypes.POINTER(_ci))
_sig("ks_plan_destroy", None, _vp)
_sig("ks_plan_status", _ci, _vp)
_sig("ks_debug_fail_allocs", None, _ci)
_sig("ks_debug_tc_stall", None, _ci, _i64)
_sig("ks_debug_norm_form", None, _ci)
_sig("ks_debug_tc_split", _ci, _i64, _i64, _ci, _ci, _ci, _ci, ctypes.POINTER(_i64),
     ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_i64))
_sig("ks_set_pdl", None, _ci)

DISPATCH_AUTO, DISPATCH_KS1, DISPATCH_TABLE, DISPATCH_MLP = 0, 1, 2, 3

_fp = ctypes.POINTER(ctypes.c_float)
_sig("ks_tune_time", _ci, _i64, _i64, _ci, _ci, _ci, _ci, _ci, _ci, ctypes.POINTER(ctypes.c_double))
_sig("ks_dispatch_set_table", _ci, _i64, ctypes.POINTER(ctypes.c_int32))
_sig("ks_mlp_param_count", _i64)
_sig("ks_mlp_set_params", _ci, _fp)
_sig("ks_mlp_train", _ci, _fp, _fp, _fp, _fp, _i64, _ci, ctypes.c_float, _fp)
_sig("ks_mlp_grad", _ci, _fp, _fp, _fp, _fp, _i64, _fp, _fp)
_sig("ks_mlp_predict", _ci, _fp, _i64, _fp)
MLP_IN, MLP_HIDDEN, MLP_OUT = 5, 32, 12
_sig("ks_mul_static", _ci, _vp, _vp, _i64, _vp, _i64, _ci, _ci, _ci, _vp)

STATIC_SCRATCH_BYTES = 16 << 20
_sig("ks_status_sync", _ci, _vp)
_sig("ks_choose", _ci, _i64, _i64, _ci, _ci, ctypes.POINTER(_ci), ctypes.POINTER(_ci))
_sig("ks_strerror", ctypes.c_char_p, _ci)
_sig("ks_last_cuda_error", ctypes.c_char_p)
_sig("ks_version", _ci)
_sig("ks_release_cache", None)
_sig("ks_launch_count", ctypes.c_longlong)
_sig("ks_profile_enable", None, _ci)
_sig("ks_profile_collect", _ci, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
     _ci)
_sig("ks_phase_name", ctypes.c_char_p, _ci)
_sig("ks_plan_info", _ci, _i64, _i64, _ci, _ci, _ci, _ci, ctypes.POINTER(_i64), _ci)
_sig("ks_plan_info_bits", _ci, _i64, _i64, _ci, _ci, _ci, _ci, _ci, ctypes.POINTER(_i64), _ci)

PLAN_FIELDS = ("variant", "engine", "N", "d", "nprod", "nA", "nB", "ncols", "nwords", "nnorm",
               "M", "chain", "nseeds", "out_limbs", "in_limbs", "workspace_bytes", "ntt_log",
               "off_digits", "off_cols", "off_words", "off_seeds", "seed_words", "nchains0",
               "nchains1")

N_PHASES = 7


class KSError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = "%s failed: %s (%d)" % (what, lib.ks_strerror(status).decode(), status)
        if status == KS_ECUDA or status == KS_ENOMEM:
            msg += ": " + lib.ks_last_cuda_error().decode()
        super().__init__(msg)
        self.status = status


def _check(status: int, what: str) -> None:
    if status != KS_OK:
        raise KSError(status, what)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _limbs(bits: int) -> int:
    return (int(bits) + 63) // 64


def _check_poly(t, rows, limbs, name) -> None:
    """A polynomial tensor of the layout the C ABI reads: (rows, limbs), 8-byte
    elements, contiguous.  Checked before any device pointer is taken, so a
    wrongly shaped tensor never reaches the kernels."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError("%s: expected a torch tensor" % name)
    if t.dtype not in (torch.int64, torch.uint64):
        raise ValueError("%s: expected dtype int64 or uint64, got %s" % (name, t.dtype))
    if t.dim() != 2:
        raise ValueError("%s: expected a 2-d tensor (coefficients, limbs), got %d-d"
                         % (name, t.dim()))
    want_rows = t.shape[0] if rows is None else rows
    if tuple(t.shape) != (want_rows, limbs) or t.shape[0] < 1:
        raise ValueError("%s: expected shape (%s, %d), got %s"
                         % (name, want_rows if rows is not None else "L >= 1", limbs,
                            tuple(t.shape)))
    if not t.is_contiguous():
        raise ValueError("%s: expected a contiguous tensor" % name)


def _check_device(*ts) -> None:
    """All tensors on the current CUDA device (the C ABI works there, and its
    streams, caches and status word are per device)."""
    import torch
    for t in ts:
        if not t.is_cuda:
            raise ValueError("expected CUDA tensors")
    dev = torch.cuda.current_device()
    for t in ts:
        if t.device.index != dev:
            raise ValueError("tensor on cuda:%d, but the current device is cuda:%d; "
                             "call inside torch.cuda.device(...)" % (t.device.index, dev))


def _check_product(h, f, g, bits_f, bits_g, is_signed) -> None:
    if bits_f < 1 or bits_g < 1:
        raise ValueError("coefficient bits must be >= 1")
    _check_poly(f, None, _limbs(bits_f), "f")
    _check_poly(g, None, _limbs(bits_g), "g")
    ol = out_limbs_bits(f.shape[0], g.shape[0], bits_f, bits_g, is_signed)
    _check_poly(h, f.shape[0] + g.shape[0] - 1, ol, "h")
    _check_device(h, f, g)


def out_limbs(len_f: int, len_g: int, coeff_bits: int, is_signed: bool) -> int:
    r = lib.ks_out_limbs(len_f, len_g, coeff_bits, int(is_signed))
    if r < 0:
        raise KSError(r, "ks_out_limbs")
    return r


def out_limbs_bits(len_f: int, len_g: int, bits_f: int, bits_g: int, is_signed: bool) -> int:
    """Output limbs for bits_f-bit coefficients in f and bits_g-bit ones in g."""
    r = lib.ks_out_limbs_bits(len_f, len_g, bits_f, bits_g, int(is_signed))
    if r < 0:
        raise KSError(r, "ks_out_limbs_bits")
    return r


def eval_bits(len_f: int, len_g: int, coeff_bits: int, variant: int) -> int:
    r = lib.ks_eval_bits(len_f, len_g, coeff_bits, variant)
    if r < 0:
        raise KSError(r, "ks_eval_bits")
    return r


def workspace_bytes(len_f, len_g, coeff_bits, is_signed, variant=KS_AUTO, engine=ENGINE_AUTO):
    r = lib.ks_workspace_bytes(len_f, len_g, coeff_bits, int(is_signed), variant, engine)
    if r < 0:
        raise KSError(int(r), "ks_workspace_bytes")
    return r


def choose(len_f, len_g, coeff_bits, is_signed):
    v, e = _ci(0), _ci(0)
    _check(lib.ks_choose(len_f, len_g, coeff_bits, int(is_signed), ctypes.byref(v),
                         ctypes.byref(e)), "ks_choose")
    return v.value, e.value


def ks_mul(h, f, g, coeff_bits, is_signed, variant=KS_AUTO, stream=None):
    """h = f * g with device tensors (L, limbs); h preallocated (Lh, out_limbs)."""
    _check_product(h, f, g, coeff_bits, coeff_bits, is_signed)
    _check(lib.ks_mul(_dptr(h), _dptr(f), f.shape[0], _dptr(g), g.shape[0], coeff_bits,
                      int(is_signed), variant, _stream_ptr(stream)), "ks_mul")


def ks_mul_ex(h, f, g, coeff_bits, is_signed, variant, engine, workspace, stream=None):
    _check_product(h, f, g, coeff_bits, coeff_bits, is_signed)
    _check_device(workspace)
    _check(lib.ks_mul_ex(_dptr(h), _dptr(f), f.shape[0], _dptr(g), g.shape[0], coeff_bits,
                         int(is_signed), variant, engine, _dptr(workspace),
                         workspace.numel() * workspace.element_size(), _stream_ptr(stream)),
           "ks_mul_ex")


def ks_mul_host(h, f, g, coeff_bits, is_signed, variant=KS_AUTO, engine=ENGINE_AUTO,
                stream=None):
    """Host numpy uint64 arrays in and out (synchronous)."""
    import numpy as np
    for a in (h, f, g):
        if not (isinstance(a, np.ndarray) and a.dtype == np.uint64 and a.flags.c_contiguous):
            raise ValueError("expected C-contiguous uint64 numpy arrays")
    il = _limbs(coeff_bits)
    if f.ndim != 2 or g.ndim != 2 or f.shape[1] != il or g.shape[1] != il:
        raise ValueError("f and g must be (L, %d) arrays" % il)
    ol = out_limbs(f.shape[0], g.shape[0], coeff_bits, is_signed)
    if h.shape != (f.shape[0] + g.shape[0] - 1, ol):
        raise ValueError("h must be (%d, %d)" % (f.shape[0] + g.shape[0] - 1, ol))
    _check(lib.ks_mul_host(h.ctypes.data, f.ctypes.data, f.shape[0], g.ctypes.data, g.shape[0],
                           coeff_bits, int(is_signed), variant, engine, _stream_ptr(stream)),
           "ks_mul_host")


def ks_mul_static(h, f, g, coeff_bits, is_signed, variant=KS_AUTO, stream=None):
    """As ks_mul, but the library allocates nothing: its scratch is a fixed
    device array inside the library (STATIC_SCRATCH_BYTES), for callers that
    may not allocate device memory at call time.  Calls sharing the array must
    not overlap on the GPU; larger problems raise KSError (KS_ERANGE)."""
    _check_product(h, f, g, coeff_bits, coeff_bits, is_signed)
    _check(lib.ks_mul_static(_dptr(h), _dptr(f), f.shape[0], _dptr(g), g.shape[0], coeff_bits,
                             int(is_signed), variant, _stream_ptr(stream)), "ks_mul_static")


def ks_mul_mod(h, f, g, p, variant=KS_AUTO, stream=None):
    """(Z/pZ)[x] product: residues in [0, p), one limb each; h is (Lf + Lg - 1, 1)."""
    _check_poly(f, None, 1, "f")
    _check_poly(g, None, 1, "g")
    _check_poly(h, f.shape[0] + g.shape[0] - 1, 1, "h")
    _check_device(h, f, g)
    _check(lib.ks_mul_mod(_dptr(h), _dptr(f), f.shape[0], _dptr(g), g.shape[0], p, variant,
                          _stream_ptr(stream)), "ks_mul_mod")


def ks_mul_bits(h, f, bits_f, g, bits_g, is_signed, variant=KS_AUTO, stream=None):
    """h = f g with bits_f-bit coefficients in f and bits_g-bit ones in g (device
    tensors of shape (L, ceil(bits / 64))); h has out_limbs_bits(..) limbs (N from
    bits_f + bits_g)."""
    _check_product(h, f, g, bits_f, bits_g, is_signed)
    _check(lib.ks_mul_bits(_dptr(h), _dptr(f), f.shape[0], bits_f, _dptr(g), g.shape[0], bits_g,
                           int(is_signed), variant, _stream_ptr(stream)), "ks_mul_bits")


def ks_mul_bivariate_mod(h, f, g, p, variant=KS_AUTO, stream=None):
    """(Z/pZ)[x, y] product (Sec. 2): f, g are (ly, lx) device tensors of residues
    (row i, column j: the coefficient of x^j y^i); h is (2 ly - 1, 2 lx - 1)."""
    import torch
    if f.dim() != 2 or tuple(f.shape) != tuple(g.shape):
        raise ValueError("f and g must be (ly, lx) tensors of the same shape")
    ly, lx = f.shape
    if tuple(h.shape) != (2 * ly - 1, 2 * lx - 1):
        raise ValueError("h must be (2 ly - 1, 2 lx - 1)")
    for t, n in ((h, "h"), (f, "f"), (g, "g")):
        if t.dtype not in (torch.int64, torch.uint64) or not t.is_contiguous():
            raise ValueError("%s: expected a contiguous int64 or uint64 tensor" % n)
    _check_device(h, f, g)
    _check(lib.ks_mul_bivariate_mod(_dptr(h), _dptr(f), _dptr(g), lx, ly, p, variant,
                                    _stream_ptr(stream)), "ks_mul_bivariate_mod")


def _problems(problems):
    arr = (KSProblem * len(problems))()
    for i, q in enumerate(problems):
        bg = q.get("coeff_bits_g", 0)
        _check_product(q["h"], q["f"], q["g"], q["coeff_bits"], bg or q["coeff_bits"],
                       q["is_signed"])
        arr[i] = KSProblem(_dptr(q["h"]).value, _dptr(q["f"]).value, _dptr(q["g"]).value,
                           q["f"].shape[0], q["g"].shape[0], q["coeff_bits"],
                           int(q["is_signed"]), q.get("variant", KS_AUTO),
                           q.get("engine", ENGINE_AUTO), bg)
    return arr


def ks_mul_batch(problems, stream=None):
    """problems: list of dicts with h, f, g (tensors), coeff_bits, is_signed, variant, engine."""
    _check(lib.ks_mul_batch(_problems(problems), len(problems), _stream_ptr(stream)),
           "ks_mul_batch")


class Plan:
    """A batched plan (ks_plan_*): create once, execute many times."""

    def __init__(self, problems, dispatch=DISPATCH_AUTO):
        self._keep = problems  # the tensors must outlive the plan
        self.n = len(problems)
        self.ptr = ctypes.c_void_p()
        _check(lib.ks_plan_create(ctypes.byref(self.ptr), _problems(problems), self.n, dispatch),
               "ks_plan_create")

    def execute(self, stream=None):
        _check(lib.ks_plan_execute(self.ptr, _stream_ptr(stream)), "ks_plan_execute")

    def capture(self, stream):
        _check(lib.ks_plan_capture(self.ptr, _stream_ptr(stream)), "ks_plan_capture")

    def status(self) -> None:
        """Waits for the plan's last execute and raises KSError if its device
        status word records a failure (a bounded wait that gave up, a range check)."""
        _check(lib.ks_plan_status(self.ptr), "ks_plan_status")

    def launches(self) -> int:
        return int(lib.ks_plan_launches(self.ptr))

    def workspace_bytes(self) -> int:
        return int(lib.ks_plan_workspace_bytes(self.ptr))

    def choice(self, i):
        v, e = _ci(0), _ci(0)
        _check(lib.ks_plan_choice(self.ptr, i, ctypes.byref(v), ctypes.byref(e)), "ks_plan_choice")
        return v.value, e.value

    def close(self):
        if self.ptr:
            lib.ks_plan_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def status_sync(stream=None) -> None:
    _check(lib.ks_status_sync(_stream_ptr(stream)), "ks_status_sync")


def mul(f, g, coeff_bits, is_signed, variant=KS_AUTO, engine=ENGINE_AUTO, stream=None):
    """Allocating convenience wrapper: returns h = f * g as a new device tensor."""
    import torch
    _check_poly(f, None, _limbs(coeff_bits), "f")
    _check_poly(g, None, _limbs(coeff_bits), "g")
    ol = out_limbs(f.shape[0], g.shape[0], coeff_bits, is_signed)
    h = torch.empty((f.shape[0] + g.shape[0] - 1, ol), dtype=torch.int64, device=f.device)
    if engine == ENGINE_AUTO:
        ks_mul(h, f, g, coeff_bits, is_signed, variant, stream)
    else:
        ws = torch.empty(max(workspace_bytes(f.shape[0], g.shape[0], coeff_bits, is_signed,
                                             variant, engine), 8) // 8 + 32,
                         dtype=torch.int64, device=f.device)
        ks_mul_ex(h, f, g, coeff_bits, is_signed, variant, engine, ws, stream)
    return h


def set_pdl(enabled: bool) -> None:
    """Launch overlap: enabled, every kernel may be scheduled while the previous
    kernel of its stream runs and waits for it on the device (programmatic
    dependent launch); off (the default), kernels start after the previous one
    ends.  Results are identical either way."""
    lib.ks_set_pdl(1 if enabled else 0)


def debug_fail_allocs(n: int) -> None:
    """Host-side fault injection: the library's next n device allocations fail
    (the calls return KS_ENOMEM); 0 clears it."""
    lib.ks_debug_fail_allocs(int(n))


def debug_tc_stall(on: bool, wait_ns: int = 0) -> None:
    """Test hook: the tensor-core kernel gives up on a barrier nothing completes
    (every wait bounded by wait_ns), so the call reports KS_ETIMEOUT."""
    lib.ks_debug_tc_stall(int(on), int(wait_ns))


def launch_count() -> int:
    return int(lib.ks_launch_count())


def release_cache() -> None:
    """Frees the workspaces the library has cached for the current device."""
    lib.ks_release_cache()


def profile_enable(on: bool = True) -> None:
    lib.ks_profile_enable(int(on))


def profile_collect() -> dict:
    """{phase name: (total ms, records)} for the calls made since the last collect."""
    ms = (ctypes.c_double * N_PHASES)()
    cnt = (ctypes.c_longlong * N_PHASES)()
    _check(lib.ks_profile_collect(ms, cnt, N_PHASES), "ks_profile_collect")
    return {lib.ks_phase_name(i).decode(): (ms[i], cnt[i]) for i in range(N_PHASES)}


def tc_split(len_f, len_g, coeff_bits, is_signed, variant, grid) -> dict:
    """The tensor-core engine's split of one product's work over `grid` CTAs
    (host only): {"at": grid + 1 positions, "first_q", "first_tile", "total"}."""
    at = (_i64 * (grid + 1))()
    fq = (ctypes.c_int32 * grid)()
    ft = (ctypes.c_int32 * grid)()
    tot = _i64(0)
    _check(lib.ks_debug_tc_split(len_f, len_g, coeff_bits, int(is_signed), variant, grid, at, fq,
                                 ft, ctypes.byref(tot)), "ks_debug_tc_split")
    return {"at": list(at), "first_q": list(fq), "first_tile": list(ft), "total": tot.value}


def plan_info(len_f, len_g, coeff_bits, is_signed, variant=KS_AUTO, engine=ENGINE_AUTO,
              bits_g=None) -> dict:
    """The plan the library would run for this problem (sizes of every stage);
    bits_g: g's coefficient bits when they differ from f's (coeff_bits)."""
    arr = (_i64 * len(PLAN_FIELDS))()
    bg = coeff_bits if bits_g is None else bits_g
    _check(lib.ks_plan_info_bits(len_f, len_g, coeff_bits, bg, int(is_signed), variant, engine,
                                 arr, len(PLAN_FIELDS)), "ks_plan_info_bits")
    return dict(zip(PLAN_FIELDS, [int(x) for x in arr]))


# ------------------------------------------------------------------ dispatch
def _f32(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def tune_time(len_f, len_g, coeff_bits, is_signed, variant, engine, batch=1, reps=5) -> float:
    """Device milliseconds per product of one (variant, engine) configuration."""
    ms = ctypes.c_double(0.0)
    _check(lib.ks_tune_time(len_f, len_g, coeff_bits, int(is_signed), variant, engine, batch,
                            reps, ctypes.byref(ms)), "ks_tune_time")
    return ms.value


def dispatch_set_table(rows) -> None:
    """rows: iterable of (len_f, len_g, coeff_bits, is_signed, variant, engine)."""
    import numpy as np
    arr = np.ascontiguousarray(np.array(list(rows), dtype=np.int32).reshape(-1, 6))
    _check(lib.ks_dispatch_set_table(arr.shape[0],
                                     arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
           "ks_dispatch_set_table")


def mlp_param_count() -> int:
    return int(lib.ks_mlp_param_count())


def mlp_set_params(params) -> None:
    if params is None:
        _check(lib.ks_mlp_set_params(None), "ks_mlp_set_params")
        return
    p, pp = _f32(params)
    _check(lib.ks_mlp_set_params(pp), "ks_mlp_set_params")


def mlp_train(params, x, t, mask, steps, lr):
    """Returns (trained params, final loss); every step runs on the GPU."""
    import numpy as np
    p = np.array(params, dtype=np.float32, copy=True)
    pp = p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    xa, xp = _f32(x)
    ta, tp = _f32(t)
    ma, mp = _f32(mask)
    loss = ctypes.c_float(0.0)
    _check(lib.ks_mlp_train(pp, xp, tp, mp, xa.shape[0], steps, lr, ctypes.byref(loss)),
           "ks_mlp_train")
    return p, float(loss.value)


def mlp_grad(params, x, t, mask):
    """One forward + backward on the GPU: (gradient, loss)."""
    import numpy as np
    pa, pp = _f32(params)
    xa, xp = _f32(x)
    ta, tp = _f32(t)
    ma, mp = _f32(mask)
    g = np.zeros(mlp_param_count(), dtype=np.float32)
    loss = ctypes.c_float(0.0)
    _check(lib.ks_mlp_grad(pp, xp, tp, mp, xa.shape[0],
                           g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)),
           "ks_mlp_grad")
    return g, float(loss.value)


def mlp_predict(x):
    """Inference kernel over feature rows (installed parameters)."""
    import numpy as np
    xa, xp = _f32(x)
    y = np.zeros((xa.shape[0], MLP_OUT), dtype=np.float32)
    _check(lib.ks_mlp_predict(xp, xa.shape[0], y.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
           "ks_mlp_predict")
    return y


def _install_dispatch_state():
    """Installs the committed autotuned table and cost model when they were
    measured on this kind of device (name and SM count); silent otherwise."""
    try:
        import torch
        if not torch.cuda.is_available():
            return False
        from . import dispatch
        return dispatch.install()
    except Exception:
        return False


DISPATCH_STATE_INSTALLED = _install_dispatch_state()
