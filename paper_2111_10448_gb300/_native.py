"""ctypes binding of libttsketch.so: the C ABI of include/ttsketch.h, one
Python function per C entry point, same names, argument marshalling only.

Loading fails loudly when the library has not been built: there is no CPU
fallback anywhere in this package.
"""
import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libttsketch.so")

TT_MAXD = 16
TT_MAXL = 64

TT_OK, TT_ERR_INVALID_ARG, TT_ERR_UNSUPPORTED, TT_ERR_CUDA, TT_ERR_STATE, \
    TT_ERR_RANK_DEFICIENT, TT_ERR_TIMEOUT, TT_WARN_RANK_CAP, TT_ERR_NO_DEVICE, TT_ERR_NONFINITE = range(10)
TT_F32, TT_F64 = 0, 1
TT_PREC_FP64, TT_PREC_TF32, TT_PREC_BF16, TT_PREC_FP16 = 0, 1, 2, 3
TT_FLAG_DIFF = 1
TT_FLAG_ONESIDED = 2
TT_FLAG_KR = 4
TT_FLAG_SHORT_CHAINS = 8

STATUS_NAMES = {
    0: "TT_OK", 1: "TT_ERR_INVALID_ARG", 2: "TT_ERR_UNSUPPORTED", 3: "TT_ERR_CUDA",
    4: "TT_ERR_STATE", 5: "TT_ERR_RANK_DEFICIENT", 6: "TT_ERR_TIMEOUT", 7: "TT_WARN_RANK_CAP",
    8: "TT_ERR_NO_DEVICE", 9: "TT_ERR_NONFINITE",
}


class tt_problem(C.Structure):
    _fields_ = [
        ("d", C.c_int),
        ("n", C.c_int64 * TT_MAXD),
        ("eps", C.c_double),
        ("ranks", C.c_int * (TT_MAXD + 1)),
        ("rmax", C.c_int),
        ("p", C.c_int),
        ("seed", C.c_uint64),
        ("passes", C.c_int),
        ("x_dtype", C.c_int),
        ("prec", C.c_int),
        ("flags", C.c_int),
        ("x_scale_log2", C.c_int),
    ]


class TTError(RuntimeError):
    def __init__(self, status, where):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")
        self.status = status


_lib = None

_P = C.c_void_p
_SIGS = {
    "tt_sketch_plan": (C.c_int, [C.POINTER(tt_problem), C.POINTER(_P)]),
    "tt_sketch_plan_batched": (C.c_int, [C.POINTER(tt_problem), C.c_int, C.POINTER(_P)]),
    "tt_plan_destroy": (None, [_P]),
    "tt_workspace_release": (None, [_P]),
    "tt_plan_sizes": (C.c_int, [_P, C.POINTER(C.c_size_t), C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "tt_plan_core_layout": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "tt_plan_problem": (C.c_int, [_P, C.c_int, C.POINTER(tt_problem)]),
    "tt_plan_sketch_info": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "tt_sketch_kernel_kind": (C.c_int, [_P, C.c_int64]),
    "tt_pstt2": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "tt_pstt2_noalloc": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "tt_plan_batch_config": (C.c_int, [_P, C.c_int, C.c_int, C.c_int]),
    "tt_selftest_wait_timeout": (C.c_int, [C.c_int64, _P, _P]),
    "tt_plan_autotune": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "tt_pstt2_begin": (C.c_int, [_P, _P, _P]),
    "tt_pstt2_state_size": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
    "tt_pstt2_sync": (C.c_int, [_P, _P, _P]),
    "tt_pstt2_export_state": (C.c_int, [_P, _P, _P, C.c_size_t, _P]),
    "tt_pstt2_import_state": (C.c_int, [_P, _P, _P, C.c_size_t, _P]),
    "tt_pstt2_accumulate": (C.c_int, [_P, _P, C.c_int64, C.c_int64, _P, _P]),
    "tt_pstt2_finalize": (C.c_int, [_P, _P, _P, _P, _P]),
    "tt_pstt2_batched": (C.c_int, [_P, C.POINTER(_P), _P, _P, _P, _P]),
    "tt_pstt2_backward": (C.c_int, [_P, _P, _P, _P, _P]),
    "tt_reconstruct": (C.c_int, [_P, _P, _P, C.c_int, _P, _P]),
    "tt_reconstruct_error": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "tt_reconstruct_backward": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, _P]),
    "tt_query_status": (C.c_int, [_P, _P, _P, C.POINTER(C.c_int), C.POINTER(C.c_int), _P]),
    "tt_status_string": (C.c_char_p, [C.c_int]),
    "tt_x_scale_log2": (C.c_int, [_P, C.c_int, C.c_int64, C.POINTER(C.c_int), _P]),
    "tt_test_matrix": (C.c_int, [C.c_uint64, C.c_int, C.c_int64, C.c_int64, C.c_int, C.c_int, _P, _P]),
    "tt_philox4x32_10": (C.c_int, [_P, C.c_uint32, C.c_uint32, _P, C.c_int64, _P]),
    "tt_generate_hilbert_type": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.c_int64, C.c_int64, _P,
                                           C.c_int, _P]),
    "tt_generate_hilbert": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.c_int64, C.c_int64, _P, C.c_int, _P]),
    "tt_generate_gaussian_bumps": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.c_int, C.c_double, _P,
                                             C.c_int64, C.c_int64, _P, C.c_int, _P]),
    "tt_core_mode2": (C.c_int, [_P, C.c_int, C.c_int64, C.c_int, _P, C.c_int64, _P, _P]),
    "tt_swap12": (C.c_int, [_P, C.c_int64, C.c_int64, C.c_int64, _P, _P]),
    "tt_kernel_launches": (C.c_int64, []),
    "tt_version": (C.c_char_p, []),
}

# Every extern "C" symbol declared in include/ttsketch.h.
EXPORTED = tuple(_SIGS)


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
                " (the CUDA library is required; there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status, where):
    if status != TT_OK:
        raise TTError(status, where)
    return status


def make_problem(dims, *, ranks=None, eps=0.0, rmax=0, p=5, seed=1, passes=1,
                 x_dtype=TT_F32, prec=TT_PREC_FP64, flags=0, x_scale_log2=0):
    q = tt_problem()
    q.d = len(dims)
    if q.d > TT_MAXD:
        raise ValueError("d too large")
    for k, n in enumerate(dims):
        q.n[k] = int(n)
    q.eps = float(eps)
    if ranks is not None:
        for k, r in enumerate(ranks):
            q.ranks[k] = int(r)
    q.rmax = int(rmax)
    q.p = int(p)
    q.seed = int(seed)
    q.passes = int(passes)
    q.x_dtype = int(x_dtype)
    q.prec = int(prec)
    q.flags = int(flags)
    q.x_scale_log2 = int(x_scale_log2)
    return q
