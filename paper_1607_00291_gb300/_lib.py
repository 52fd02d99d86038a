"""ctypes binding of libtc's C ABI (``include/tc.h``): argument marshalling only."""
import ctypes
import os
import threading

from . import build as _build

c_i32, c_i64, c_dbl, c_vp, c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
MAX_RANK = 16

TC_F64, TC_F32 = 0, 1
TC_MODE_F64, TC_MODE_BF16X3, TC_MODE_BF16X6 = 0, 1, 2
TC_ACCESS_BOX, TC_ACCESS_BLOCK, TC_ACCESS_SCATTER, TC_ACCESS_PACKED, TC_ACCESS_AUTO = 0, 1, 2, 3, 4
TC_REDUCE_COMPENSATED, TC_REDUCE_F64 = 0, 1
TC_OK = 0
STATUS = {0: "TC_OK", -1: "TC_ERR_ARG", -2: "TC_ERR_LABEL", -3: "TC_ERR_EXTENT", -4: "TC_ERR_OVERLAP",
          -5: "TC_ERR_WORKSPACE", -6: "TC_ERR_CUDA", -7: "TC_ERR_DEVICE_TIMEOUT",
          -8: "TC_ERR_UNSUPPORTED", -9: "TC_ERR_DEVICE_BOUNDS", -10: "TC_ERR_SCRATCH_LIMIT"}


class TcTensor(ctypes.Structure):
    _fields_ = [("rank", c_i32), ("len", ctypes.POINTER(c_i64)), ("stride", ctypes.POINTER(c_i64)),
                ("labels", ctypes.c_char_p), ("data", c_vp)]


class TcProblem(ctypes.Structure):
    _fields_ = [("alpha", c_dbl), ("beta", c_dbl), ("A", TcTensor), ("B", TcTensor), ("C", TcTensor)]


class TcPlanInfo(ctypes.Structure):
    _fields_ = [("swapped", c_i32), ("nI", c_i32), ("nJ", c_i32), ("nP", c_i32),
                ("m", c_i64), ("n", c_i64), ("k", c_i64),
                ("I_len", c_i64 * MAX_RANK), ("I_sA", c_i64 * MAX_RANK), ("I_sC", c_i64 * MAX_RANK),
                ("J_len", c_i64 * MAX_RANK), ("J_sB", c_i64 * MAX_RANK), ("J_sC", c_i64 * MAX_RANK),
                ("P_len", c_i64 * MAX_RANK), ("P_sA", c_i64 * MAX_RANK), ("P_sB", c_i64 * MAX_RANK),
                ("I_labels", (ctypes.c_char * (MAX_RANK + 1)) * MAX_RANK),
                ("J_labels", (ctypes.c_char * (MAX_RANK + 1)) * MAX_RANK),
                ("P_labels", (ctypes.c_char * (MAX_RANK + 1)) * MAX_RANK),
                ("a_k_contig", c_i32), ("b_k_contig", c_i32), ("c_m_contig", c_i32)]


# every entry point of include/tc.h with its ctypes signature
SIGNATURES = {
    "tc_plan_describe": (c_i32, [ctypes.POINTER(TcTensor)] * 3 + [ctypes.POINTER(TcPlanInfo)]),
    "tc_workspace_size": (c_i32, [c_i32, c_i32] + [ctypes.POINTER(TcTensor)] * 3 + [ctypes.POINTER(c_sz)]),
    "tc_contract": (c_i32, [c_i32, c_i32, c_dbl, ctypes.POINTER(TcTensor), ctypes.POINTER(TcTensor), c_dbl,
                            ctypes.POINTER(TcTensor), c_vp, c_sz, c_vp]),
    "tc_batched_workspace_size": (c_i32, [c_i32, c_i32, c_i32, ctypes.POINTER(TcProblem), ctypes.POINTER(c_sz)]),
    "tc_contract_batched": (c_i32, [c_i32, c_i32, c_i32, ctypes.POINTER(TcProblem), c_vp, c_sz, c_vp]),
    "tc_plan_create": (c_i32, [c_i32, c_i32, c_i32, ctypes.POINTER(TcProblem), ctypes.POINTER(c_vp)]),
    "tc_plan_workspace_size": (c_i32, [c_vp, ctypes.POINTER(c_sz)]),
    "tc_plan_config": (c_i32, [c_vp, c_i32, ctypes.POINTER(c_i32)]),
    "tc_plan_execute": (c_i32, [c_vp, c_vp, c_sz, c_vp]),
    "tc_plan_destroy": (None, [c_vp]),
    "tc_scatter_count": (c_i32, [ctypes.POINTER(TcTensor)] * 3 + [c_i32, ctypes.POINTER(c_i64)]),
    "tc_build_scatter": (c_i32, [ctypes.POINTER(TcTensor)] * 3 + [c_i32, c_vp, c_i64, c_vp]),
    "tc_get_device_error": (c_i32, [c_vp, ctypes.POINTER(c_i32)]),
    "tc_contract_noalloc": (c_i32, [c_i32, c_dbl, ctypes.POINTER(TcTensor), ctypes.POINTER(TcTensor), c_dbl,
                                    ctypes.POINTER(TcTensor), c_vp]),
    "tc_set_access": (c_i32, [c_i32]),
    "tc_set_split_reduction": (c_i32, [c_i32]),
    "tc_set_checks": (c_i32, [c_i32]),
    "tc_box_access": (c_i32, [c_i32, c_i32] + [ctypes.POINTER(TcTensor)] * 3 +
                      [ctypes.POINTER(c_i32), ctypes.POINTER(c_i32)]),
    "tc_plan_form": (c_i32, [c_vp, ctypes.POINTER(c_i32)]),
    "tc_operand_form": (c_i32, [c_i32, c_i32] + [ctypes.POINTER(TcTensor)] * 3 +
                        [ctypes.POINTER(c_i32)]),
    "tc_set_mainloop_events": (c_i32, [c_vp, c_vp]),
    "tc_launch_count": (ctypes.c_uint64, []),
    "tc_status_string": (ctypes.c_char_p, [c_i32]),
    "tc_version": (c_i32, []),
}

_lib = None
_lock = threading.Lock()


def lib():
    """Load libtc.so (building it first when the sources are newer).  Raises if
    the library cannot be built or loaded: there is no fallback path."""
    global _lib
    with _lock:
        if _lib is None:
            if not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libtc.so is missing; run __graft_entry__.build()")
            L = ctypes.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class TcError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        s = lib().tc_status_string(code).decode()
        super().__init__(f"{where}: {STATUS.get(code, code)} ({s})")


def check(code, where=""):
    if code != TC_OK:
        raise TcError(code, where)


def make_tensor(shape, strides, labels: str, data_ptr: int, keep: list) -> TcTensor:
    """Build a tc_tensor; arrays are appended to ``keep`` to outlive the call."""
    if len(shape) != len(strides) or len(labels) != len(shape):
        raise ValueError("shape, strides and labels must have one entry per dimension")
    r = len(shape)
    lens = (c_i64 * max(1, r))(*[int(v) for v in shape])
    strs = (c_i64 * max(1, r))(*[int(v) for v in strides])
    lab = labels.encode("latin-1")
    keep.extend([lens, strs, lab])
    return TcTensor(r, lens, strs, lab, c_vp(int(data_ptr)))
