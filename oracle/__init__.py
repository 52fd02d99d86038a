"""CPU oracle for the general tensor contraction (Section 4 of the paper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
product path (``paper_1607_00291_gb300``) never imports it, and it imports
nothing from the product path.

* ``contract``        -- C := alpha * sum_P A*B + beta * C, plain FP64 loops
                          (``tc_oracle.c``), with per-element magnitudes for
                          error normalisation.
* ``scatter``          -- the scatter vector of one index bundle (Section 6.1).
* ``block_scatter``    -- the block-scatter vector (Section 6.2).
* ``bundle``           -- label classification and the five-step dimension
                          heuristic (Section 7.3); see ``oracle/bundle.py``.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against values the paper prints, closed forms and library routines.
"""
import ctypes
import os

import numpy as np

from . import build as _build
from .bundle import classify, normalize  # noqa: F401

_lib = None

OR_OK, OR_ERR_ARG, OR_ERR_LABEL, OR_ERR_EXTENT = 0, -1, -2, -3


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_contract.restype = ctypes.c_int
        lib.oracle_contract.argtypes = [
            ctypes.c_double,
            ctypes.c_int, i64p, i64p, ctypes.c_char_p, ctypes.c_void_p,
            ctypes.c_int, i64p, i64p, ctypes.c_char_p, ctypes.c_void_p,
            ctypes.c_double,
            ctypes.c_int, i64p, i64p, ctypes.c_char_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
        ]
        lib.oracle_scatter.restype = None
        lib.oracle_scatter.argtypes = [ctypes.c_int, i64p, i64p, i64p]
        lib.oracle_block_scatter.restype = None
        lib.oracle_block_scatter.argtypes = [i64p, ctypes.c_int64, ctypes.c_int64, i64p]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def num_threads(requested: int = 0) -> int:
    return _load().oracle_num_threads(requested)


def _i64(seq):
    arr = (ctypes.c_int64 * max(1, len(seq)))()
    for i, v in enumerate(seq):
        arr[i] = int(v)
    return arr


def _desc(x: np.ndarray, labels: str):
    if x.dtype != np.float64:
        raise TypeError("the oracle works in float64; upcast first")
    if len(labels) != x.ndim:
        raise ValueError("one label per dimension")
    strides = [s // x.itemsize for s in x.strides]
    if any(s * x.itemsize != b for s, b in zip(strides, x.strides)):
        raise ValueError("strides must be whole elements")
    return (x.ndim, _i64(x.shape), _i64(strides), labels.encode(), ctypes.c_void_p(x.ctypes.data))


def contract_(alpha, A: np.ndarray, labA: str, B: np.ndarray, labB: str, beta, C: np.ndarray,
              labC: str, *, mag: bool = True, begin: int = 0, end: int = -1, threads: int = 0):
    """Contract in place into ``C`` (any strides).  Returns the magnitude array
    (colexicographic order over C's dimensions, i.e. Fortran order of C's shape)
    or None.  Raises ValueError on an invalid contraction."""
    lib = _load()
    numel = int(np.prod(C.shape, dtype=np.int64)) if C.ndim else 1
    m = np.zeros(numel, dtype=np.float64) if mag else None
    rc = lib.oracle_contract(
        float(alpha), *_desc(A, labA), *_desc(B, labB), float(beta), *_desc(C, labC),
        ctypes.c_void_p(m.ctypes.data) if m is not None else None,
        int(begin), int(end), int(threads))
    if rc != OR_OK:
        raise ValueError(f"oracle rejected the contraction (code {rc})")
    if m is None:
        return None
    return m.reshape(C.shape, order="F") if C.ndim else m.reshape(())


def contract(alpha, A, labA, B, labB, beta, C, labC, **kw):
    """Functional form: returns (C_new, mag) with C_new a fresh array of C's shape."""
    Cn = np.array(C, dtype=np.float64, copy=True)
    m = contract_(alpha, np.asarray(A, dtype=np.float64), labA, np.asarray(B, dtype=np.float64),
                  labB, beta, Cn, labC, **kw)
    return Cn, m


def scatter(lens, strides) -> np.ndarray:
    """scat[x] = sum_k u_k(x) * s_k over the bundle dims ``lens`` (first fastest)."""
    lib = _load()
    n = int(np.prod(lens, dtype=np.int64)) if len(lens) else 1
    out = np.zeros(max(n, 1), dtype=np.int64)
    lib.oracle_scatter(len(lens), _i64(lens), _i64(strides),
                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return out[:n]


def block_scatter(scat, b: int) -> np.ndarray:
    """Block-scatter vector of ``scat`` with blocking parameter ``b`` (Section 6.2)."""
    lib = _load()
    scat = np.ascontiguousarray(scat, dtype=np.int64)
    nb = (len(scat) + b - 1) // b
    out = np.zeros(max(nb, 1), dtype=np.int64)
    lib.oracle_block_scatter(scat.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(scat), b,
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return out[:nb]
