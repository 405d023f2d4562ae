"""CPU oracle for the Mojette erasure code over GF(2).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers. The product path (the CUDA library and
its Python binding) never imports this package, and this package imports
nothing from the product.

The arithmetic lives in ``mojette_oracle.c`` (plain C, built here with gcc);
this module only marshals numpy arrays. Functions follow the paper:

* ``bin_count``   -- Eq. 2 with q = 1.
* ``bin_min``     -- smallest bin position b = l p - x, by enumeration (Eq. 1).
* ``katz``        -- the reconstruction criterion, Eq. 3.
* ``encode``      -- forward Mojette transform, Eq. 1 (XOR addition, Sec. 3).
* ``decode``      -- inverse Mojette transform by peeling, Sec. 2.2.
* ``sys_decode``  -- the systematic form (data lines are packets, parity
  packets are projections; mentioned in Sec. 2.3 and Sec. 4, not defined
  there): surviving lines copied and removed from the parity bins, the lost
  lines peeled as in Sec. 2.2.

Layout: images are ``uint64[S, Q, P]`` (row l = data line, x = column);
projections are ``uint64[S, sum_i B_i]`` with projection i at offset
``off_i = sum_{i' < i} B_i'`` and bin b stored at ``j = b - b_min_i``.

parity unpinned: nothing. Every function here is pinned in
``tests/test_oracle_pins.py`` against something other than itself.
"""
from __future__ import annotations

import ctypes
import errno
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mojette_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_I64 = ctypes.c_int64
_INT = ctypes.c_int
_PTR = ctypes.c_void_p


class OracleError(RuntimeError):
    """A negative errno returned by the oracle."""

    def __init__(self, code: int, what: str):
        self.code = code
        name = errno.errorcode.get(-code, str(code))
        super().__init__(f"{what}: {name} ({code})")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no architecture flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L",
                    "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC],
                   check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_bin_count.restype = _I64
            lib.oracle_bin_count.argtypes = [_INT, _INT, _INT]
            lib.oracle_bin_min.restype = _I64
            lib.oracle_bin_min.argtypes = [_INT, _INT, _INT]
            lib.oracle_total_bins.restype = _I64
            lib.oracle_total_bins.argtypes = [_INT, _INT, _PTR, _INT]
            lib.oracle_katz.restype = _INT
            lib.oracle_katz.argtypes = [_INT, _INT, _PTR, _INT, ctypes.c_uint32]
            lib.oracle_encode.restype = _INT
            lib.oracle_encode.argtypes = [_INT, _INT, _PTR, _INT, _PTR, _PTR,
                                          _I64, _INT]
            lib.oracle_decode.restype = _INT
            lib.oracle_decode.argtypes = [_INT, _INT, _PTR, _INT, _PTR, _PTR,
                                          _I64, _PTR, _I64, _INT]
            lib.oracle_sys_decode.restype = _INT
            lib.oracle_sys_decode.argtypes = [_INT, _INT, _PTR, _INT, _PTR, _PTR,
                                              _PTR, _I64, _PTR, _I64, _INT]
            _lib = lib
    return _lib


def _dirs(p):
    arr = np.ascontiguousarray(np.asarray(list(p), dtype=np.int32))
    return arr, arr.ctypes.data_as(_PTR)


def bin_count(p: int, P: int, Q: int) -> int:
    """Eq. 2 with q = 1."""
    return int(_load().oracle_bin_count(int(p), int(P), int(Q)))


def bin_min(p: int, P: int, Q: int) -> int:
    """Smallest b = l p - x over the P x Q lattice."""
    return int(_load().oracle_bin_min(int(p), int(P), int(Q)))


def offsets(p, P: int, Q: int):
    """Per-projection (offset, bin count, b_min) and the stripe's total bins."""
    off, bins, bmins, t = [], [], [], 0
    for pi in p:
        off.append(t)
        b = bin_count(pi, P, Q)
        bins.append(b)
        bmins.append(bin_min(pi, P, Q))
        t += b
    return off, bins, bmins, t


def total_bins(p, P: int, Q: int) -> int:
    arr, ptr = _dirs(p)
    r = int(_load().oracle_total_bins(int(P), int(Q), ptr, len(arr)))
    if r < 0:
        raise OracleError(r, "total_bins")
    return r


def katz(p, P: int, Q: int, mask: int) -> bool:
    """Eq. 3 over the projections whose bit is clear in ``mask``."""
    arr, ptr = _dirs(p)
    return bool(_load().oracle_katz(int(P), int(Q), ptr, len(arr),
                                    ctypes.c_uint32(int(mask) & 0xFFFFFFFF)))


def encode(img: np.ndarray, p, threads: int = 1) -> np.ndarray:
    """Forward transform of ``img`` (uint64[S, Q, P]) -> uint64[S, total]."""
    img = np.ascontiguousarray(img, dtype=np.uint64)
    if img.ndim == 2:
        img = img[None]
    S, Q, P = img.shape
    arr, ptr = _dirs(p)
    out = np.empty((S, total_bins(p, P, Q)), dtype=np.uint64)
    r = _load().oracle_encode(P, Q, ptr, len(arr), img.ctypes.data_as(_PTR),
                              out.ctypes.data_as(_PTR), S, int(threads))
    if r < 0:
        raise OracleError(r, "encode")
    return out


def decode(proj: np.ndarray, p, P: int, Q: int, masks, threads: int = 1) -> np.ndarray:
    """Inverse transform -> uint64[S, Q, P].

    ``masks`` is one erasure mask (bit i set: projection i lost) or one per
    stripe. Raises OracleError(-ENOTRECOVERABLE) when Eq. 3 fails or peeling
    stalls.
    """
    proj = np.ascontiguousarray(proj, dtype=np.uint64)
    if proj.ndim == 1:
        proj = proj[None]
    S = proj.shape[0]
    arr, ptr = _dirs(p)
    if proj.shape[1] != total_bins(p, P, Q):
        raise ValueError("projection buffer does not match the geometry")
    m = np.ascontiguousarray(np.atleast_1d(np.asarray(masks, dtype=np.uint64))
                             .astype(np.uint32))
    out = np.empty((S, Q, P), dtype=np.uint64)
    r = _load().oracle_decode(int(P), int(Q), ptr, len(arr),
                              proj.ctypes.data_as(_PTR), out.ctypes.data_as(_PTR),
                              S, m.ctypes.data_as(_PTR), len(m), int(threads))
    if r < 0:
        raise OracleError(r, "decode")
    return out


def sys_decode(data: np.ndarray, parity: np.ndarray, p, P: int, Q: int, masks,
               threads: int = 1) -> np.ndarray:
    """Systematic decode -> uint64[S, Q, P].

    ``data`` (uint64[S, Q, P]) holds the data lines as received (lost lines
    are never read); ``parity`` (uint64[S, total]) the projections along
    ``p``. Mask bit l < Q: data line l lost; bit Q + i: projection i lost.
    Raises OracleError(-ENOTRECOVERABLE) when the peeling stalls.
    """
    data = np.ascontiguousarray(data, dtype=np.uint64)
    parity = np.ascontiguousarray(parity, dtype=np.uint64)
    if data.ndim == 2:
        data = data[None]
    if parity.ndim == 1:
        parity = parity[None]
    S = data.shape[0]
    if data.shape != (S, Q, P) or parity.shape != (S, total_bins(p, P, Q)):
        raise ValueError("buffers do not match the geometry")
    arr, ptr = _dirs(p)
    m = np.ascontiguousarray(np.atleast_1d(np.asarray(masks, dtype=np.uint64))
                             .astype(np.uint32))
    out = np.empty((S, Q, P), dtype=np.uint64)
    r = _load().oracle_sys_decode(int(P), int(Q), ptr, len(arr),
                                  data.ctypes.data_as(_PTR), parity.ctypes.data_as(_PTR),
                                  out.ctypes.data_as(_PTR), S, m.ctypes.data_as(_PTR),
                                  len(m), int(threads))
    if r < 0:
        raise OracleError(r, "sys_decode")
    return out
