"""Thin ctypes binding over libmojette.so (C ABI: include/mojette.h).

Argument marshalling only: every step of encode and decode runs in the CUDA
library. Functions keep the C names. Device buffers may be given as torch
tensors (8-byte elements, on the current CUDA device; ``data_ptr()`` is
passed) or as raw integer device addresses. ``stream`` defaults to torch's
current stream on the current device.

Loading builds the library in-tree with nvcc when it is missing or stale and
raises if that fails: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import errno
import os
import re
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

_I64 = ctypes.c_int64
_INT = ctypes.c_int
_U32 = ctypes.c_uint32
_PTR = ctypes.c_void_p

HEADER = os.path.join(_build.ROOT, "include", "mojette.h")


class MojetteError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str):
        self.code = code
        name = errno.errorcode.get(-code, str(code))
        super().__init__(f"{what}: {msg} ({name})")


def lib():
    """The loaded library (built on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            L.mojette_plan.argtypes = [_INT, _INT, _PTR, _INT, ctypes.POINTER(_PTR)]
            L.mojette_plan_destroy.argtypes = [_PTR]
            L.mojette_plan_ex.argtypes = [_INT, _INT, _PTR, _INT, _U32, ctypes.POINTER(_PTR)]
            L.mojette_plan_bins.argtypes = [_PTR, _PTR]
            L.mojette_plan_config.argtypes = [_PTR, _PTR, _PTR]
            L.mojette_plan_info.argtypes = [_PTR, _PTR, _PTR, _PTR]
            L.mojette_encode.argtypes = [_PTR, _PTR, _PTR, _I64, _PTR]
            L.mojette_decode.argtypes = [_PTR, _PTR, _U32, _PTR, _I64, _PTR]
            L.mojette_decode_noalloc.argtypes = [_PTR, _PTR, _U32, _PTR, _I64, _PTR]
            L.mojette_sys_decode.argtypes = [_PTR, _PTR, _U32, _PTR, _I64, _PTR]
            L.mojette_stage_survivors.argtypes = [_PTR, _PTR, _U32, _PTR, _I64, _PTR, ctypes.POINTER(_I64)]
            L.mojette_decode_kernel.argtypes = [_PTR, _U32, _I64, ctypes.POINTER(ctypes.c_int32)]
            L.mojette_schedule.argtypes = [_PTR, _U32, _PTR, _PTR, _PTR, _PTR, _PTR, _I64, _PTR]
            L.mojette_schedule_layout.argtypes = [_PTR, _U32, _PTR, _PTR]
            L.mojette_batch_create.argtypes = [_PTR, _I64, _U32, ctypes.POINTER(_PTR)]
            L.mojette_batch_update.argtypes = [_PTR, _PTR, _I64, _PTR]
            L.mojette_batch_run.argtypes = [_PTR, _PTR]
            L.mojette_batch_tune.argtypes = [_PTR, _PTR, _INT]
            L.mojette_batch_info.argtypes = [_PTR, _PTR, _PTR, _PTR, _PTR]
            L.mojette_batch_destroy.argtypes = [_PTR]
            L.mojette_server_create.argtypes = [_I64, _INT, _I64, ctypes.POINTER(_PTR)]
            L.mojette_server_submit.argtypes = [_PTR, _PTR, _I64]
            L.mojette_server_poll.argtypes = [_PTR, _PTR, _I64, ctypes.POINTER(_I64)]
            L.mojette_server_now.argtypes = [_PTR, ctypes.POINTER(ctypes.c_double)]
            L.mojette_server_stats.argtypes = [_PTR] + [ctypes.POINTER(_I64)] * 6
            L.mojette_server_destroy.argtypes = [_PTR]
            L.mojette_selftest_wait.argtypes = [_I64, _PTR]
            L.mojette_device_status.argtypes = [ctypes.POINTER(_U32), _INT]
            L.mojette_strerror.argtypes = [_INT]
            L.mojette_strerror.restype = ctypes.c_char_p
            L.mojette_last_cuda_error.argtypes = []
            for name in ("mojette_plan", "mojette_plan_ex", "mojette_plan_bins", "mojette_plan_config",
                         "mojette_plan_destroy",
                         "mojette_plan_info",
                         "mojette_encode", "mojette_decode", "mojette_decode_noalloc", "mojette_sys_decode",
                         "mojette_stage_survivors", "mojette_decode_kernel",
                         "mojette_schedule", "mojette_schedule_layout", "mojette_batch_create",
                         "mojette_batch_update",
                         "mojette_batch_run", "mojette_batch_tune", "mojette_batch_info",
                         "mojette_batch_destroy", "mojette_server_create", "mojette_server_submit",
                         "mojette_server_poll", "mojette_server_now", "mojette_server_stats",
                         "mojette_server_destroy",
                         "mojette_selftest_wait", "mojette_device_status", "mojette_last_cuda_error"):
                getattr(L, name).restype = _INT
            _lib = L
    return _lib


def header_functions():
    """Names of the functions include/mojette.h declares."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:int|const char \*|void)\s*\*?\s*(mojette_\w+)\s*\(",
                                 text, flags=re.M)))


def mojette_strerror(code: int) -> str:
    return lib().mojette_strerror(int(code)).decode()


def _check(code: int, what: str):
    if code != 0:
        msg = mojette_strerror(code)
        if code == -errno.EIO:
            msg += f" [cudaError {lib().mojette_last_cuda_error()}]"
        raise MojetteError(code, what, msg)


def _addr(buf) -> int:
    if buf is None:
        return 0
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):
        if buf.element_size() != 8:
            raise TypeError("buffers hold 64-bit words (torch.int64 or torch.uint64)")
        if not buf.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return buf.data_ptr()
    raise TypeError(f"cannot take a device address of {type(buf).__name__}")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


MOJETTE_PLAN_TRIM_UNUSED = 1
MOJETTE_PLAN_SYSTEMATIC = 2


class Plan:
    """Owns a ``mojette_plan_t``; geometry (P, Q, p) and its bin layout.
    ``trim=True``: unused-bin removal (mojette_plan_ex); ``full_bin`` then
    maps each stored word of a stripe's block to its bin in the full
    projection (mojette_plan_bins). ``systematic=True``: the systematic form
    (the Q data lines are packets, ``p`` the parity projections; decode with
    mojette_sys_decode)."""

    def __init__(self, P: int, Q: int, p, trim: bool = False, systematic: bool = False):
        self.P, self.Q, self.p = int(P), int(Q), [int(v) for v in p]
        self.systematic = bool(systematic)
        arr = (ctypes.c_int * len(self.p))(*self.p)
        h = _PTR()
        flags = (MOJETTE_PLAN_TRIM_UNUSED if trim else 0) | (MOJETTE_PLAN_SYSTEMATIC if systematic else 0)
        _check(lib().mojette_plan_ex(self.P, self.Q, arr, len(self.p), flags, ctypes.byref(h)),
               "mojette_plan_ex")
        self.handle = h.value
        self._lib = lib()
        self.bins, self.offsets, self.total = mojette_plan_info(self)
        fb = np.zeros(max(1, self.total), dtype=np.int32)
        self.trimmed = lib().mojette_plan_bins(self.handle, fb.ctypes.data) == 1
        self.full_bin = fb[: self.total]

    @property
    def n(self) -> int:
        return len(self.p)

    def close(self):
        if getattr(self, "handle", None):
            self._lib.mojette_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mojette_plan(P: int, Q: int, p) -> Plan:
    return Plan(P, Q, p)


def mojette_plan_ex(P: int, Q: int, p, flags: int = 0) -> Plan:
    return Plan(P, Q, p, trim=bool(flags & MOJETTE_PLAN_TRIM_UNUSED),
                systematic=bool(flags & MOJETTE_PLAN_SYSTEMATIC))


def mojette_plan_destroy(plan: Plan) -> None:
    plan.close()


_CONFIG_KEYS = ("decode_tuned", "decode_kernel", "decode_gpc", "decode_persist", "decode_rowoff",
                "encode_tuned", "encode_tile_bytes", "reserved")


def mojette_plan_config(plan: Plan, config: dict | None = None) -> dict:
    """The plan's batch launch configuration as a dict; with ``config``,
    install that one first (keys as returned; missing keys keep their value)."""
    cur = np.zeros(8, dtype=np.int32)
    _check(lib().mojette_plan_config(plan.handle, cur.ctypes.data, None), "mojette_plan_config")
    if config is not None:
        new = cur.copy()
        for k, v in config.items():
            new[_CONFIG_KEYS.index(k)] = int(v)
        _check(lib().mojette_plan_config(plan.handle, None, new.ctypes.data), "mojette_plan_config")
        cur = new
    return {k: int(v) for k, v in zip(_CONFIG_KEYS, cur) if k != "reserved"}


def geometry_key(plan: Plan) -> str:
    return (f"P{plan.P}-Q{plan.Q}-p{','.join(str(v) for v in plan.p)}" + ("-trimmed" if plan.trimmed else "")
            + ("-systematic" if plan.systematic else ""))


def save_tuning(plans, path: str) -> None:
    """Write the launch configurations of ``plans`` to a JSON file keyed by
    geometry (merged into the file's existing entries)."""
    import json
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    for pl in plans:
        data[geometry_key(pl)] = mojette_plan_config(pl)
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


def load_tuning(plans, path: str) -> int:
    """Install the configurations stored for ``plans``' geometries; returns
    how many plans had one."""
    import json
    with open(path) as f:
        data = json.load(f)
    n = 0
    for pl in plans:
        cfg = data.get(geometry_key(pl))
        if cfg:
            mojette_plan_config(pl, cfg)
            n += 1
    return n


def mojette_plan_info(plan: Plan):
    n = len(plan.p)
    bins = (_I64 * n)()
    offs = (_I64 * n)()
    total = _I64()
    _check(lib().mojette_plan_info(plan.handle, bins, offs, ctypes.byref(total)), "mojette_plan_info")
    return list(bins), list(offs), int(total.value)


def mojette_encode(plan: Plan, d_img, d_proj, S: int | None = None, stream=None) -> None:
    """Encode S stripes: d_img [S][Q][P] -> d_proj [S][total] (64-bit words)."""
    if S is None:
        S = d_img.numel() // (plan.P * plan.Q)
    _check(lib().mojette_encode(plan.handle, _addr(d_img), _addr(d_proj), int(S), _stream(stream)),
           "mojette_encode")


def mojette_decode(plan: Plan, d_proj, erasure_mask: int, d_img, S: int | None = None,
                   stream=None) -> None:
    """Decode S stripes that lost the projections set in erasure_mask."""
    if S is None:
        S = d_img.numel() // (plan.P * plan.Q)
    _check(lib().mojette_decode(plan.handle, _addr(d_proj), int(erasure_mask) & 0xFFFFFFFF,
                                _addr(d_img), int(S), _stream(stream)), "mojette_decode")


def mojette_stage_survivors(plan: Plan, h_proj, erasure_mask: int, d_proj, S: int | None = None,
                            stream=None) -> int:
    """Copy to the device only the projections a decode under erasure_mask
    reads (h_proj [S][total] in host memory, pinned for an asynchronous
    copy, into d_proj [S][total]); returns the bytes copied."""
    if S is None:
        S = d_proj.numel() // max(1, plan.total)
    moved = _I64()
    _check(lib().mojette_stage_survivors(plan.handle, _addr(h_proj), int(erasure_mask) & 0xFFFFFFFF,
                                         _addr(d_proj), int(S), _stream(stream), ctypes.byref(moved)),
           "mojette_stage_survivors")
    return int(moved.value)


def mojette_sys_decode(plan: Plan, d_parity, erasure_mask: int, d_data, S: int | None = None,
                       stream=None) -> None:
    """Systematic plan: rebuild in place the data lines of d_data [S][Q][P]
    that erasure_mask marks lost (bits 0..Q-1; bits Q.. mark lost parity
    projections of d_parity [S][total])."""
    if S is None:
        S = d_data.numel() // (plan.P * plan.Q)
    _check(lib().mojette_sys_decode(plan.handle, _addr(d_parity), int(erasure_mask) & 0xFFFFFFFF,
                                    _addr(d_data), int(S), _stream(stream)), "mojette_sys_decode")


def mojette_decode_noalloc(plan: Plan, d_proj, erasure_mask: int, d_img, S: int | None = None,
                           stream=None) -> None:
    """mojette_decode without any device allocation (fixed in-library scratch;
    calls that overlap on the GPU race -- see include/mojette.h)."""
    if S is None:
        S = d_img.numel() // (plan.P * plan.Q)
    _check(lib().mojette_decode_noalloc(plan.handle, _addr(d_proj), int(erasure_mask) & 0xFFFFFFFF,
                                        _addr(d_img), int(S), _stream(stream)),
           "mojette_decode_noalloc")


DECODE_KERNELS = {-1: None, 0: "decode_lines", 1: "decode_fronts", 2: "decode_stream", 3: "decode_cols",
                  4: "decode_scan2", 5: "decode_vander", 6: "decode_ilv", 7: "decode_ring"}


def mojette_decode_kernel(plan: Plan, erasure_mask: int, S: int = 1 << 20) -> str | None:
    """Name of the decode kernel a decode of this mask over S stripes
    launches (None: none)."""
    k = ctypes.c_int32()
    _check(lib().mojette_decode_kernel(plan.handle, int(erasure_mask) & 0xFFFFFFFF, int(S), ctypes.byref(k)),
           "mojette_decode_kernel")
    return DECODE_KERNELS[int(k.value)]


def mojette_schedule(plan: Plan, erasure_mask: int) -> dict:
    """The cached reconstruction path for one mask (host data)."""
    Q = plan.Q
    nsteps = _I64()
    _check(lib().mojette_schedule(plan.handle, int(erasure_mask) & 0xFFFFFFFF, None, None, None,
                                  None, None, 0, ctypes.byref(nsteps)), "mojette_schedule")
    T = int(nsteps.value)
    left = (ctypes.c_int32 * Q)()
    right = (ctypes.c_int32 * Q)()
    split = (ctypes.c_int32 * Q)()
    steps = (ctypes.c_uint32 * max(T, 1))()
    forward = (ctypes.c_uint32 * max(T, 1))()
    _check(lib().mojette_schedule(plan.handle, int(erasure_mask) & 0xFFFFFFFF, left, right, split,
                                  steps, forward, T, ctypes.byref(nsteps)), "mojette_schedule")
    lines = Q
    if plan.systematic:   # one entry per lost data line
        lines = bin(int(erasure_mask) & ((1 << Q) - 1)).count("1")
    return {"left": list(left)[:lines], "right": list(right)[:lines], "split": list(split)[:lines],
            "steps": list(steps)[:T], "forward": list(forward)[:T], "T": T, "lines": lines}


def mojette_schedule_layout(plan: Plan, erasure_mask: int) -> dict:
    """decode_lines' shared-memory layout for one mask's path (host data):
    per-line row phases and per-front load orders (nibbles)."""
    lines = plan.Q
    if plan.systematic:
        lines = bin(int(erasure_mask) & ((1 << plan.Q) - 1)).count("1")
    n = max(lines, 1)
    phase = (ctypes.c_int32 * n)()
    order = (ctypes.c_uint32 * (2 * n))()
    _check(lib().mojette_schedule_layout(plan.handle, int(erasure_mask) & 0xFFFFFFFF, phase, order),
           "mojette_schedule_layout")
    return {"row_phase": list(phase)[:lines], "load_order": list(order)[:2 * lines], "lines": lines}


# ---- batches -----------------------------------------------------------------

MOJETTE_OP_ENCODE = 0
MOJETTE_OP_DECODE = 1
MOJETTE_BATCH_GRAPH = 1

# Layout of mojette_stripe_t (include/mojette.h): 32 bytes, no padding.
STRIPE_DTYPE = np.dtype([("plan", "<u8"), ("op", "<i4"), ("erasure_mask", "<u4"),
                         ("src", "<u8"), ("dst", "<u8")])
assert STRIPE_DTYPE.itemsize == 32


def stripe_table(plans, plan_index, op, erasure_mask, src, dst) -> np.ndarray:
    """A mojette_stripe_t array: stripe k uses plans[plan_index[k]], operation
    op[k], erasure_mask[k] and the device addresses src[k], dst[k] (integer
    arrays, or scalars broadcast over the stripes)."""
    plan_index = np.asarray(plan_index, dtype=np.int64)
    handles = np.array([pl.handle for pl in plans], dtype=np.uint64)
    t = np.zeros(len(plan_index), dtype=STRIPE_DTYPE)
    t["plan"] = handles[plan_index]
    t["op"] = op
    t["erasure_mask"] = np.asarray(erasure_mask, dtype=np.int64).astype(np.uint32)
    t["src"] = np.asarray(src, dtype=np.uint64)
    t["dst"] = np.asarray(dst, dtype=np.uint64)
    return t


class Batch:
    """Owns a ``mojette_batch_t``; keeps the plans it uses alive."""

    def __init__(self, table: np.ndarray, plans, flags: int = 0):
        table = np.ascontiguousarray(table, dtype=STRIPE_DTYPE)
        self.plans = list(plans)
        h = _PTR()
        _check(lib().mojette_batch_create(table.ctypes.data if len(table) else None, len(table),
                                          int(flags), ctypes.byref(h)), "mojette_batch_create")
        self.handle = h.value
        self._lib = lib()

    def close(self):
        if getattr(self, "handle", None):
            self._lib.mojette_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mojette_batch_create(table: np.ndarray, plans, flags: int = 0) -> Batch:
    """Build a batch from a stripe_table (``plans``: the Plan objects it uses)."""
    return Batch(table, plans, flags)


def mojette_batch_update(batch: Batch, table: np.ndarray, plans=None, stream=None) -> None:
    table = np.ascontiguousarray(table, dtype=STRIPE_DTYPE)
    if plans is not None:
        batch.plans = list(plans)
    _check(lib().mojette_batch_update(batch.handle, table.ctypes.data if len(table) else None,
                                      len(table), _stream(stream)), "mojette_batch_update")


def mojette_batch_run(batch: Batch, stream=None) -> None:
    _check(lib().mojette_batch_run(batch.handle, _stream(stream)), "mojette_batch_run")


def mojette_batch_tune(batch: Batch, stream=None, reps: int = 3) -> None:
    _check(lib().mojette_batch_tune(batch.handle, _stream(stream), int(reps)), "mojette_batch_tune")


def mojette_batch_info(batch: Batch) -> dict:
    launches, groups, work = _I64(), _I64(), _I64()
    _check(lib().mojette_batch_info(batch.handle, ctypes.byref(launches), ctypes.byref(groups),
                                    ctypes.byref(work), None), "mojette_batch_info")
    cfg = (ctypes.c_int32 * (6 * max(1, launches.value)))()
    _check(lib().mojette_batch_info(batch.handle, None, None, None, cfg), "mojette_batch_info")
    names = ("op", "Q", "P", "kernel", "param", "flags")
    configs = [dict(zip(names, cfg[6 * i: 6 * i + 6])) for i in range(launches.value)]
    return {"launches": int(launches.value), "groups": int(groups.value),
            "work_items": int(work.value), "configs": configs}


def mojette_batch_destroy(batch: Batch) -> None:
    batch.close()


# ---- request server -------------------------------------------------------

# Layouts of mojette_request_t (56 bytes) and mojette_completion_t (40 bytes).
REQUEST_DTYPE = np.dtype([("id", "<u8"), ("plan", "<u8"), ("op", "<i4"), ("erasure_mask", "<u4"),
                          ("stripes", "<i8"), ("host_src", "<u8"), ("host_dst", "<u8"),
                          ("arrival_s", "<f8")])
COMPLETION_DTYPE = np.dtype([("id", "<u8"), ("status", "<i4"), ("_pad", "<i4"), ("arrival_s", "<f8"),
                             ("admit_s", "<f8"), ("done_s", "<f8")])
assert REQUEST_DTYPE.itemsize == 56 and COMPLETION_DTYPE.itemsize == 40


class Server:
    """Owns a ``mojette_server_t``."""

    def __init__(self, budget_bytes: int, slots: int = 3, max_wave_stripes: int = 65536):
        h = _PTR()
        _check(lib().mojette_server_create(int(budget_bytes), int(slots), int(max_wave_stripes),
                                           ctypes.byref(h)), "mojette_server_create")
        self.handle = h.value
        self._lib = lib()
        self._buf = np.zeros(4096, dtype=COMPLETION_DTYPE)

    def close(self):
        if getattr(self, "handle", None):
            self._lib.mojette_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mojette_server_create(budget_bytes: int, slots: int = 3, max_wave_stripes: int = 65536) -> Server:
    return Server(budget_bytes, slots, max_wave_stripes)


def mojette_server_submit(server: Server, reqs: np.ndarray) -> None:
    reqs = np.ascontiguousarray(reqs, dtype=REQUEST_DTYPE)
    _check(lib().mojette_server_submit(server.handle, reqs.ctypes.data if len(reqs) else None, len(reqs)),
           "mojette_server_submit")


def mojette_server_poll(server: Server) -> np.ndarray:
    """Progress, then every completion available (a COMPLETION_DTYPE array)."""
    out = []
    n = _I64()
    while True:
        code = lib().mojette_server_poll(server.handle, server._buf.ctypes.data, len(server._buf),
                                         ctypes.byref(n))
        out.append(server._buf[: n.value].copy())
        _check(code, "mojette_server_poll")
        if n.value < len(server._buf):
            break
    return np.concatenate(out)


def mojette_server_now(server: Server) -> float:
    t = ctypes.c_double()
    _check(lib().mojette_server_now(server.handle, ctypes.byref(t)), "mojette_server_now")
    return t.value


def mojette_server_stats(server: Server) -> dict:
    v = [_I64() for _ in range(6)]
    _check(lib().mojette_server_stats(server.handle, *[ctypes.byref(x) for x in v]), "mojette_server_stats")
    names = ("queued", "in_flight", "waves", "completed", "pool_used", "pool_peak")
    return {k: int(x.value) for k, x in zip(names, v)}


def mojette_server_destroy(server: Server) -> None:
    server.close()


def mojette_selftest_wait(limit_ns: int = 20_000_000, stream=None) -> None:
    """Enqueue the bounded-wait self-test (mojette_device_status then reports
    -ETIMEDOUT)."""
    _check(lib().mojette_selftest_wait(int(limit_ns), _stream(stream)), "mojette_selftest_wait")


def mojette_device_status(clear: bool = True) -> int:
    """Synchronise and return the device status word (raises on a timeout bit)."""
    flags = _U32()
    code = lib().mojette_device_status(ctypes.byref(flags), 1 if clear else 0)
    _check(code, "mojette_device_status")
    return int(flags.value)


def mojette_last_cuda_error() -> int:
    return int(lib().mojette_last_cuda_error())
