"""ctypes binding of libtbk (include/tbk.h): argument marshalling only.

The shared library is built in-tree by ``paper_1812_05264_gb300.build``; loading fails loudly when
it is missing -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

TBK_OK = 0
TBK_ERR_ARG = -1
TBK_ERR_CUDA = -2
TBK_ERR_OOM = -3
TBK_ERR_SPECTRUM = -4
TBK_ERR_NOCONV = -5
TBK_ERR_TIMEOUT = -6

TBK_MIXED = 0
TBK_FP64 = 1
TBK_MOMENTS_DIRECT = 2
TBK_PLAIN_KERNEL = 4
TBK_NO_GRAPH = 8
TBK_TENSOR_CORES = 16
TBK_WINDOWED = 32
TBK_FUSED_ADJOINT = 64
TBK_TC_OUTER = 128
TBK_DAMP_NONE = 0
TBK_DAMP_JACKSON = 1
TBK_FN_FERMI = 0
TBK_FN_ENERGY = 1
TBK_FN_FREE = 2
TBK_MODEL_SK = 1
TBK_MODEL_TABLE = 2
TBK_KERNEL_NONE = 0
TBK_KERNEL_STEP = 1
TBK_KERNEL_BACKWARD = 2
TBK_KERNEL_WINDOW = 3

_NAMES = {TBK_ERR_ARG: "TBK_ERR_ARG", TBK_ERR_CUDA: "TBK_ERR_CUDA", TBK_ERR_OOM: "TBK_ERR_OOM",
          TBK_ERR_SPECTRUM: "TBK_ERR_SPECTRUM", TBK_ERR_NOCONV: "TBK_ERR_NOCONV",
          TBK_ERR_TIMEOUT: "TBK_ERR_TIMEOUT"}


class TbkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class tbk_model(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_orb", C.c_int32), ("sk_V", C.c_double * 10),
                ("sk_r0", C.c_double), ("sk_decay", C.c_double), ("onsite_spd", C.c_double * 3),
                ("n_disp", C.c_int32), ("disp", C.c_void_p), ("disp_blocks", C.c_void_p),
                ("disp_tol", C.c_double), ("onsite_site", C.c_void_p)]


class tbk_bsr(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("n_orb", C.c_int32), ("nnzb", C.c_int64),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


_P = C.c_void_p
_D = C.c_double
_I = C.c_int32
_L = C.c_int64
_U = C.c_uint64

# name -> argtypes (every entry point returns int except where noted)
SIGNATURES = {
    "tbk_create": [C.POINTER(_P), C.c_int, _P],
    "tbk_destroy": [_P],
    "tbk_test_stall_next_step": [_P],
    "tbk_test_stall_next_adjoint": [_P],
    "tbk_autotune": [_P, C.POINTER(tbk_bsr), _D, _D, _I, C.POINTER(_I)],
    "tbk_kernel_timer": [_P, _I],
    "tbk_kernel_timer_read": [_P, _I, C.POINTER(_D), C.POINTER(_L)],
    "tbk_build_neighbors": [_P, _P, _I, _P, _D, _P, _P, _L, C.POINTER(_L)],
    "tbk_batched_build_neighbors": [_P, _I, C.POINTER(_P), C.POINTER(_I), _D, C.POINTER(_P),
                                    C.POINTER(_P), C.POINTER(_L), C.POINTER(_L)],
    "tbk_welsh_powell": [_I, _P, _P, _P, C.POINTER(_I)],
    "tbk_assemble_H": [_P, C.POINTER(tbk_model), _P, _I, _P, _P, _P, _L, _P],
    "tbk_spectral_bounds": [_P, C.POINTER(tbk_bsr), _I, _D, _U, C.POINTER(_D), C.POINTER(_D)],
    "tbk_batched_spectral_bounds": [_P, _I, C.POINTER(tbk_bsr), _I, _D, _U, C.POINTER(_D), C.POINTER(_D)],
    "tbk_chebyshev_coefficients": [_P, _I, _I, _D, _D, _D, _D, _I, _P],
    "tbk_chebyshev_moments": [_P, C.POINTER(tbk_bsr), _D, _D, _U, _I, _I, _I, _P],
    "tbk_chebyshev_probe_moments": [_P, C.POINTER(tbk_bsr), _D, _D, _U, _I, _I, _I, _P, _P],
    "tbk_chebyshev_moments_noalloc": [_P, C.POINTER(tbk_bsr), _D, _D, _U, _I, _I, _I, _P],
    "tbk_energies_and_forces": [_P, C.POINTER(tbk_bsr), C.POINTER(tbk_model), _P, _P, _D, _D, _U,
                                _I, _I, _D, _D, _I, _I, _L, _P, C.POINTER(_D), _P, _P],
    "tbk_batched_moments": [_P, _I, C.POINTER(tbk_bsr), C.POINTER(_D), C.POINTER(_D), C.POINTER(_U),
                            _I, C.POINTER(_I), _I, _P],
    "tbk_batched_fermi_level": [_P, _I, _P, C.POINTER(_I), C.POINTER(_D), C.POINTER(_D),
                                C.POINTER(_D), C.POINTER(_D), _I, C.POINTER(_D)],
    "tbk_batched_density_and_forces": [_P, _I, C.POINTER(tbk_bsr), C.POINTER(tbk_model),
                                       C.POINTER(_P), C.POINTER(_D), C.POINTER(_D),
                                       C.POINTER(_U), _I, C.POINTER(_I), C.POINTER(_D),
                                       C.POINTER(_D), _I, _I, _L, C.POINTER(_P), C.POINTER(_P)],
    "tbk_batched_energies_and_forces": [_P, _I, C.POINTER(tbk_bsr), C.POINTER(tbk_model),
                                        C.POINTER(_P), C.POINTER(_D), C.POINTER(_D),
                                        C.POINTER(_U), _I, C.POINTER(_I), C.POINTER(_D),
                                        C.POINTER(_D), _I, _I, _L, _P, C.POINTER(_D),
                                        C.POINTER(_P), C.POINTER(_P)],
    "tbk_fermi_level": [_P, _P, _I, _D, _D, _D, _D, _D, _I, C.POINTER(_D)],
    "tbk_density_and_forces": [_P, C.POINTER(tbk_bsr), C.POINTER(tbk_model), _P, _P, _D, _D, _U,
                               _I, _I, _D, _D, _I, _I, _L, _P, _P],
    "tbk_direct_density": [_P, C.POINTER(tbk_bsr), C.POINTER(tbk_model), _P, _P, _D, _D, _U, _I, _I,
                           _D, _D, _I, _I, _P, _P, _P],
    "tbk_local_density": [_P, C.POINTER(tbk_bsr), _P, _P, _D, _D, _D, _I, _D, _D, _I, _I, _P, _P],
    "tbk_rational_density": [_P, C.POINTER(tbk_bsr), C.POINTER(tbk_model), _P, _P, _U, _I, _D, _D, _I, _D,
                             _I, _I, _P, _P, _P, C.POINTER(_D)],
    "tbk_colored_moments": [_P, C.POINTER(tbk_bsr), _D, _D, _U, _P, _I, _I, _I, _I, _I, _P],
    "tbk_colored_energies_and_forces": [_P, C.POINTER(tbk_bsr), C.POINTER(tbk_model), _P, _P, _D, _D,
                                        _U, _P, _I, _I, _I, _I, _D, _D, _I, _I, _L, _P,
                                        C.POINTER(_D), _P, _P],
}
OTHER = {"tbk_last_error": ([], C.c_char_p), "tbk_launch_count": ([_P], C.c_int64)}

_lib = None


def load(path: str = LIB):
    """Load libtbk.so (once) and declare its prototypes."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtbk.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, args in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    for name, (args, res) in OTHER.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def check(code: int):
    if code != TBK_OK:
        msg = load().tbk_last_error().decode(errors="replace")
        raise TbkError(code, msg)


def call(name: str, *args):
    check(getattr(load(), name)(*args))
