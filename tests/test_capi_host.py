"""Host-side checks of libmojette that need no GPU.

The library must load and export every function include/mojette.h declares;
plans must have the layout of Eq. 2; and every reconstruction schedule the
library builds must be a valid path -- replayed here on the CPU, step by
step, with the gather rule of Sec. 2.2 on bins from the oracle's encoder, it
must rebuild the oracle's image exactly.
"""
import ctypes
import errno

import numpy as np
import pytest

import oracle
from paper_1504_07038_gb300 import binding as mj
from paper_1504_07038_gb300 import inputs

CONFIGS = [
    (128, 4, [-3, -2, -1, 1, 2, 3]),
    (256, 4, [-3, -2, -1, 1, 2, 3]),
    (64, 8, [v for v in range(-6, 7) if v]),
    (128, 8, [v for v in range(-6, 7) if v]),
    (256, 2, [-1, 1, 2]),
]


def test_library_exports_every_header_function():
    names = mj.header_functions()
    assert {"mojette_plan", "mojette_encode", "mojette_decode", "mojette_plan_destroy",
            "mojette_plan_info", "mojette_schedule", "mojette_device_status",
            "mojette_strerror", "mojette_last_cuda_error"} <= set(names)
    L = mj.lib()
    for n in names:
        assert hasattr(L, n), n
        assert ctypes.cast(getattr(L, n), ctypes.c_void_p).value


@pytest.mark.parametrize("P,Q,p", CONFIGS + [(5, 3, [0, 7, -9]), (1, 1, [4])])
def test_plan_layout_matches_eq2(P, Q, p):
    plan = mj.mojette_plan(P, Q, p)
    off, bins, _, total = oracle.offsets(p, P, Q)
    assert plan.bins == bins and plan.offsets == off and plan.total == total


@pytest.mark.parametrize("args", [
    (0, 4, [1]), (8, 0, [1]), (8, 4, []), (8, 4, [1, 1]), (8, 4, list(range(33))),
])
def test_plan_rejects_bad_geometry(args):
    with pytest.raises(mj.MojetteError) as e:
        mj.mojette_plan(*args)
    assert e.value.code == -errno.EINVAL


def test_calls_validate_arguments_without_a_device():
    plan = mj.mojette_plan(16, 4, [-2, -1, 1, 2])
    L = mj.lib()
    assert L.mojette_encode(None, 16, 16, 1, None) == -errno.EINVAL
    assert L.mojette_encode(plan.handle, 16, 16, -1, None) == -errno.EINVAL
    assert L.mojette_encode(plan.handle, 0, 16, 1, None) == -errno.EINVAL
    assert L.mojette_encode(plan.handle, 8, 16, 1, None) == -errno.ERANGE
    assert L.mojette_encode(plan.handle, 16, 16, 0, None) == 0          # S = 0: no-op
    assert L.mojette_decode(plan.handle, 16, 1 << 5, 16, 1, None) == -errno.EINVAL
    assert L.mojette_decode(plan.handle, 16, 0b0111, 16, 1, None) == -errno.ENOTRECOVERABLE
    assert L.mojette_decode(plan.handle, 16, 0, 24, 1, None) == -errno.ERANGE
    assert mj.mojette_strerror(-errno.ENOTRECOVERABLE).startswith("surviving")


def replay(sched, plan, proj, P, Q, p):
    """Run a schedule on the CPU for all stripes at once and return the image.

    Checks that it is a valid path: every pixel is rebuilt exactly once, from
    its front's dedicated projection, and every other in-image pixel of its
    bin line was rebuilt at an earlier step -- or, for line l + 1 only, by
    the same front earlier in the same step (fronts visit their lines from
    Q - 1 down to 0 and the device forwards that value in a register)."""
    S = proj.shape[0]
    img = np.zeros((S, Q, P), dtype=np.uint64)
    step_of = np.full((Q, P), -1)
    front_of = np.full((Q, P), -1)
    left, right, split = sched["left"], sched["right"], sched["split"]
    xa, xz = [0] * Q, [P - 1] * Q
    steady_mask = (1 << (2 * Q)) - 1
    steady_patterns = set()
    for t, w in enumerate(sched["steps"]):
        steady = Q <= 15 and bool(w >> 31 & 1)
        patt = {}
        if steady:
            assert w & steady_mask == steady_mask
        for side in (0, 1):
            for l in range(Q - 1, -1, -1):
                if not (w >> (2 * l + side) & 1):
                    continue
                x = xa[l] if side == 0 else xz[l]
                i = left[l] if side == 0 else right[l]
                assert (x < split[l]) == (side == 0)
                assert step_of[l, x] < 0
                pi = p[i]
                bmin = -(P - 1) + min(0, (Q - 1) * pi)
                v = proj[:, plan.offsets[i] + (l * pi - x - bmin)].copy()
                for l2 in range(Q):
                    x2 = x + (l2 - l) * pi
                    if l2 == l or not 0 <= x2 < P:
                        continue
                    done = step_of[l2, x2]
                    ok = 0 <= done < t or (done == t and l2 == l + 1 and front_of[l2, x2] == side)
                    assert ok, (t, side, l, x, l2, x2, done)
                    v ^= img[:, l2, x2]
                x2 = x + pi
                fwd_here = bool(l + 1 < Q and 0 <= x2 < P and step_of[l + 1, x2] == t
                                and front_of[l + 1, x2] == side)
                assert bool(sched["forward"][t] >> (2 * l + side) & 1) == fwd_here
                if steady and l + 1 < Q:
                    patt[(side, l)] = fwd_here
                img[:, l, x] = v
                step_of[l, x] = t
                front_of[l, x] = side
                if side == 0:
                    xa[l] += 1
                else:
                    xz[l] -= 1
        if steady:                      # every steady step follows one pattern
            key = tuple(sorted(patt.items()))
            steady_patterns.add(key)
            assert len(steady_patterns) == 1, steady_patterns
    assert (step_of >= 0).all()
    return img


@pytest.mark.parametrize("P,Q,p", CONFIGS)
def test_schedules_replay_to_the_oracle_image(P, Q, p):
    n = len(p)
    plan = mj.mojette_plan(P, Q, p)
    img = inputs.stripes(3, Q, P, seed=11)
    proj = oracle.encode(img, p)
    masks = []
    for e in range(0, n - Q + 1):
        ms = inputs.all_masks(n, e)
        masks += ms if len(ms) <= 40 else ms[:: len(ms) // 40]
    for m in masks:
        sched = mj.mojette_schedule(plan, m)
        used = set(sched["left"]) | set(sched["right"])
        assert all(not (m >> i & 1) for i in used)          # erased projections never read
        assert len(set(sched["left"])) == Q
        assert [p[i] for i in sched["left"]] == sorted(p[i] for i in sched["left"])
        assert sched["T"] <= P // 2 + 2 * Q * max(abs(v) for v in p)   # about P/2 steps
        assert (replay(sched, plan, proj, P, Q, p) == img).all(), m


def test_schedule_for_every_small_geometry():
    """Exhaustive over tiny geometries: every k-of-n mask yields a path that
    rebuilds the image (Eq. 3 says the image is unique; that the sweep never
    stalls is checked here rather than assumed)."""
    rng = np.random.default_rng(5)
    for P in range(1, 9):
        for Q in range(1, 5):
            for _ in range(2):
                n = int(rng.integers(Q, Q + 3))
                p = sorted(rng.choice(np.arange(-5, 6), size=n, replace=False).tolist())
                plan = mj.mojette_plan(P, Q, p)
                img = inputs.stripes(2, Q, P, seed=P * 10 + Q)
                proj = oracle.encode(img, p)
                for m in range(1 << n):
                    if n - bin(m).count("1") < Q:
                        continue
                    sched = mj.mojette_schedule(plan, m)
                    assert (replay(sched, plan, proj, P, Q, p) == img).all(), (P, Q, p, m)


TRIM_GEOMS = [(256, 4, [-3, -2, -1, 1, 2, 3]), (64, 8, [v for v in range(-6, 7) if v]),
              (20, 3, [-4, -1, 0, 2, 5, 6])]


@pytest.mark.parametrize("P,Q,p", TRIM_GEOMS)
def test_trimmed_plan_keeps_every_bin_a_path_reads(P, Q, p):
    """Unused-bin removal (Sec. 2.3): the stored bins of each projection are
    in increasing order, and for every recoverable mask every run of bins a
    front reads (bin l p - x - b_min, x over the front's pixels) is stored,
    at consecutive stored words -- what the decoder's base offsets assume."""
    from paper_1504_07038_gb300 import binding as mj
    full = mj.mojette_plan(P, Q, p)
    tr = mj.mojette_plan_ex(P, Q, p, mj.MOJETTE_PLAN_TRIM_UNUSED)
    assert tr.trimmed and not full.trimmed
    assert tr.total <= full.total and sum(tr.bins) == tr.total
    assert list(full.full_bin) == [j for i in range(len(p)) for j in range(full.bins[i])]
    where = {}
    for i in range(len(p)):
        fb = tr.full_bin[tr.offsets[i]: tr.offsets[i] + tr.bins[i]]
        assert all(0 <= j < full.bins[i] for j in fb)
        assert all(a < b for a, b in zip(fb, fb[1:]))
        where[i] = {int(j): s for s, j in enumerate(fb)}
    n = len(p)
    for e in range(0, n - Q + 1):
        for m in inputs.all_masks(n, e):
            sc = mj.mojette_schedule(tr, m)
            for l in range(Q):
                for side, i in ((0, sc["left"][l]), (1, sc["right"][l])):
                    xs = range(0, sc["split"][l]) if side == 0 else range(sc["split"][l], P)
                    bmin = oracle.bin_min(p[i], P, Q)
                    idx = [where[i].get(l * p[i] - x - bmin) for x in xs]
                    assert None not in idx, (m, l, side)
                    assert all(b == a - 1 for a, b in zip(idx, idx[1:])), (m, l, side)


def test_plan_config_round_trip(tmp_path):
    """Tuned launch configurations can be read, installed and kept in a JSON
    file keyed by geometry (host only)."""
    from paper_1504_07038_gb300 import binding as mj
    a = mj.mojette_plan(256, 4, [-3, -2, -1, 1, 2, 3])
    b = mj.mojette_plan(64, 8, [v for v in range(-6, 7) if v])
    assert mj.mojette_plan_config(a)["decode_tuned"] == 0
    mj.mojette_plan_config(a, {"decode_tuned": 1, "decode_kernel": 3, "decode_gpc": 2,
                               "encode_tuned": 1, "encode_tile_bytes": 16000})
    path = str(tmp_path / "tuning.json")
    mj.save_tuning([a, b], path)
    a2 = mj.mojette_plan(256, 4, [-3, -2, -1, 1, 2, 3])
    assert mj.load_tuning([a2], path) == 1
    c = mj.mojette_plan_config(a2)
    assert (c["decode_tuned"], c["decode_kernel"], c["decode_gpc"], c["encode_tile_bytes"]) == (1, 3, 2, 16000)
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_plan_config(b, {"decode_tuned": 1, "decode_kernel": 0, "decode_gpc": 0})
    assert ei.value.code == -errno.EINVAL


# ------------------------------------------------------- systematic form --

SYS_CONFIGS = [
    (128, 4, [-1, 1]),
    (256, 4, [-1, 1]),
    (64, 8, [-2, -1, 1, 2]),
    (128, 8, [-2, -1, 1, 2]),
]


def sys_replay(sched, plan, data, parity, P, Q, p, mask):
    """Run a systematic schedule on the CPU and return the rebuilt lost lines
    (uint64[S, lines, P]).

    The lost lines (image rows lpos) first get their dedicated bins with the
    known lines' pixels removed; then the steps rebuild each pixel from that
    residual bin XOR the other lost lines' pixels of its bin line, each
    rebuilt at an earlier step or -- for line l + 1 only -- by the same front
    earlier in the same step."""
    lpos = [l for l in range(Q) if mask >> l & 1]
    known = [l for l in range(Q) if not mask >> l & 1]
    L = len(lpos)
    assert sched["lines"] == L
    S = data.shape[0]
    left, right, split = sched["left"], sched["right"], sched["split"]
    for i in set(left) | set(right):
        assert not mask >> (Q + i) & 1                    # lost parity never read
    res = np.zeros((S, L, P), dtype=np.uint64)
    for j in range(L):
        for x in range(P):
            i = left[j] if x < split[j] else right[j]
            pi = p[i]
            bmin = -(P - 1) + min(0, (Q - 1) * pi)
            v = parity[:, plan.offsets[i] + (lpos[j] * pi - x - bmin)].copy()
            for l2 in known:
                x2 = x + (l2 - lpos[j]) * pi
                if 0 <= x2 < P:
                    v ^= data[:, l2, x2]
            res[:, j, x] = v
    out = np.zeros_like(res)
    step_of = np.full((L, P), -1)
    front_of = np.full((L, P), -1)
    xa, xz = [0] * L, [P - 1] * L
    if sched["T"] == 0:                  # one lost line: the residual bins are its pixels
        assert L == 1 and split[0] == P
        return res
    for t, w in enumerate(sched["steps"]):
        for side in (0, 1):
            for l in range(L - 1, -1, -1):
                if not (w >> (2 * l + side) & 1):
                    continue
                x = xa[l] if side == 0 else xz[l]
                pi = p[left[l] if side == 0 else right[l]]
                assert (x < split[l]) == (side == 0) and step_of[l, x] < 0
                v = res[:, l, x].copy()
                for l2 in range(L):
                    x2 = x + (lpos[l2] - lpos[l]) * pi
                    if l2 == l or not 0 <= x2 < P:
                        continue
                    done = step_of[l2, x2]
                    ok = 0 <= done < t or (done == t and l2 == l + 1 and front_of[l2, x2] == side)
                    assert ok, (t, side, l, x, l2, x2, done)
                    v ^= out[:, l2, x2]
                if l + 1 < L:
                    x2 = x + (lpos[l + 1] - lpos[l]) * pi
                    fwd_here = bool(0 <= x2 < P and step_of[l + 1, x2] == t and front_of[l + 1, x2] == side)
                    assert bool(sched["forward"][t] >> (2 * l + side) & 1) == fwd_here
                out[:, l, x] = v
                step_of[l, x] = t
                front_of[l, x] = side
                if side == 0:
                    xa[l] += 1
                else:
                    xz[l] -= 1
    assert (step_of >= 0).all()
    return out


def _sys_masks(Q, r, limit=None, seed=3):
    ms = [m for m in range(1 << (Q + r)) if bin(m).count("1") <= r and m & ((1 << Q) - 1)]
    if limit and len(ms) > limit:
        ms = [ms[i] for i in np.random.default_rng(seed).choice(len(ms), limit, replace=False)]
    return ms


@pytest.mark.parametrize("P,Q,p", SYS_CONFIGS)
def test_sys_schedules_replay_to_the_image(P, Q, p):
    plan = mj.Plan(P, Q, p, systematic=True)
    img = inputs.stripes(2, Q, P, seed=13)
    par = oracle.encode(img, p)
    for m in _sys_masks(Q, len(p), limit=60):
        sched = mj.mojette_schedule(plan, m)
        lost = [l for l in range(Q) if m >> l & 1]
        assert sched["T"] <= P // 2 + 2 * Q * max(abs(v) for v in p)
        data = img.copy()
        data[:, lost] = np.uint64(7)
        got = sys_replay(sched, plan, data, par, P, Q, p, m)
        assert (got == img[:, lost]).all(), m


def test_sys_schedule_for_every_small_geometry():
    """Exhaustive over tiny geometries: every mask losing e data lines with at
    least e parity projections left yields a path that rebuilds them."""
    rng = np.random.default_rng(17)
    for P in range(1, 9):
        for Q in range(1, 6):
            for _ in range(2):
                r = int(rng.integers(1, 4))
                p = sorted(rng.choice(np.arange(-5, 6), size=r, replace=False).tolist())
                plan = mj.Plan(P, Q, p, systematic=True)
                img = inputs.stripes(2, Q, P, seed=P * 10 + Q)
                par = oracle.encode(img, p)
                for m in range(1 << (Q + r)):
                    e = bin(m & ((1 << Q) - 1)).count("1")
                    surv = r - bin(m >> Q).count("1")
                    if e == 0 or e > surv:
                        continue
                    sched = mj.mojette_schedule(plan, m)
                    lost = [l for l in range(Q) if m >> l & 1]
                    got = sys_replay(sched, plan, img, par, P, Q, p, m)
                    assert (got == img[:, lost]).all(), (P, Q, p, m)


def test_sys_calls_validate_arguments_without_a_device():
    L = mj.lib()
    sysp = mj.Plan(16, 4, [-1, 1], systematic=True)
    plain = mj.mojette_plan(16, 4, [-2, -1, 1, 2])
    assert L.mojette_sys_decode(plain.handle, 16, 1, 16, 1, None) == -errno.EINVAL
    assert L.mojette_decode(sysp.handle, 16, 1, 16, 1, None) == -errno.EINVAL
    assert L.mojette_decode_noalloc(sysp.handle, 16, 1, 16, 1, None) == -errno.EINVAL
    assert L.mojette_sys_decode(sysp.handle, 16, 1 << 6, 16, 1, None) == -errno.EINVAL   # bit beyond Q + n
    assert L.mojette_sys_decode(sysp.handle, 16, 0b0111, 16, 1, None) == -errno.ENOTRECOVERABLE
    assert L.mojette_sys_decode(sysp.handle, 16, 0b0011 | 1 << 4, 16, 1, None) == -errno.ENOTRECOVERABLE
    assert L.mojette_sys_decode(sysp.handle, 16, 0b0101, 24, 1, None) == -errno.ERANGE
    assert L.mojette_sys_decode(sysp.handle, 0, 3 << 4, 0, 1, None) == 0     # no line lost: nothing to do
    assert L.mojette_sys_decode(sysp.handle, 16, 0b0001, 16, 0, None) == 0   # S = 0
    h = ctypes.c_void_p()
    arr = (ctypes.c_int * 2)(-1, 1)
    both = mj.MOJETTE_PLAN_SYSTEMATIC | mj.MOJETTE_PLAN_TRIM_UNUSED
    assert L.mojette_plan_ex(16, 4, arr, 2, both, ctypes.byref(h)) == -errno.EINVAL
    wide = (ctypes.c_int * 4)(-2, -1, 1, 2)
    assert L.mojette_plan_ex(16, 29, wide, 4, mj.MOJETTE_PLAN_SYSTEMATIC, ctypes.byref(h)) == -errno.EINVAL
    nine = (ctypes.c_int * 9)(*range(-4, 5))
    assert L.mojette_plan_ex(16, 12, nine, 9, mj.MOJETTE_PLAN_SYSTEMATIC, ctypes.byref(h)) == 0
    assert L.mojette_sys_decode(h.value, 16, (1 << 9) - 1, 16, 1, None) == -errno.EINVAL   # 9 lines lost
    L.mojette_plan_destroy(h.value)


def test_decode_kernel_choice():
    """The kernel a decode launches: the Sec. 2.2 path everywhere --
    decode_lines for Q <= 8 whatever P, S or the plan's trimming,
    decode_fronts beyond; a systematic decode runs the path over its lost
    lines (decode_lines), nothing when no data line is lost. The
    stripe-interleaved path kernel (decode_ilv), the closed forms
    (decode_vander, decode_scan2) and the other path kernels are opt-in
    through MOJETTE_DECODE_KERNEL, where they apply."""
    import os
    six = [-3, -2, -1, 1, 2, 3]
    twelve = [v for v in range(-6, 7) if v]
    for P, Q, p, m in [(256, 4, six, 0b11), (128, 4, six, 0b11), (256, 2, [-1, 1, 2], 0b1),
                       (512, 2, [-1, 1, 2], 0b1), (64, 8, twelve, 0xF), (128, 8, twelve, 0xF0)]:
        for S in (1, 1024, 1 << 20):
            assert mj.mojette_decode_kernel(mj.mojette_plan(P, Q, p), m, S=S) == "decode_lines", (P, Q, S)
    assert mj.mojette_decode_kernel(mj.mojette_plan(16, 9, list(range(-5, 5))), 0) == "decode_fronts"
    sysp = mj.Plan(128, 4, [-1, 1], systematic=True)
    assert mj.mojette_decode_kernel(sysp, 0b0110) == "decode_lines"
    assert mj.mojette_decode_kernel(sysp, 0b0100) == "decode_lines"
    assert mj.mojette_decode_kernel(sysp, 0b11 << 4) is None
    tr = mj.mojette_plan_ex(256, 4, six, mj.MOJETTE_PLAN_TRIM_UNUSED)
    assert mj.mojette_decode_kernel(tr, 0b11) == "decode_lines"
    for name, want in [("lines", "decode_lines"), ("vander", "decode_vander"), ("fronts", "decode_fronts"),
                       ("ilv", "decode_ilv")]:
        os.environ["MOJETTE_DECODE_KERNEL"] = name
        try:
            assert mj.mojette_decode_kernel(mj.mojette_plan(256, 4, six), 0b11) == want
        finally:
            del os.environ["MOJETTE_DECODE_KERNEL"]
    os.environ["MOJETTE_DECODE_KERNEL"] = "scan"
    try:
        assert mj.mojette_decode_kernel(mj.mojette_plan(256, 2, [-1, 1, 2]), 0b1) == "decode_scan2"
        assert mj.mojette_decode_kernel(sysp, 0b0110) == "decode_scan2"
    finally:
        del os.environ["MOJETTE_DECODE_KERNEL"]


def test_stage_survivors_argument_errors():
    """mojette_stage_survivors refuses NULL plans and buffers, systematic
    plans and mask bits beyond n, and an unrecoverable mask, before any copy;
    S = 0 copies nothing."""
    L = mj.lib()
    six = [-3, -2, -1, 1, 2, 3]
    plan = mj.mojette_plan(64, 4, six)
    n = ctypes.c_int64(-1)
    assert L.mojette_stage_survivors(None, 8, 0, 8, 1, None, ctypes.byref(n)) == -errno.EINVAL
    assert L.mojette_stage_survivors(plan.handle, 0, 0b11, 8, 1, None, ctypes.byref(n)) == -errno.EINVAL
    assert L.mojette_stage_survivors(plan.handle, 8, 0b11, 0, 1, None, None) == -errno.EINVAL
    assert L.mojette_stage_survivors(plan.handle, 8, 1 << 6, 8, 1, None, None) == -errno.EINVAL
    assert L.mojette_stage_survivors(plan.handle, 8, 0b111, 8, 1, None, None) == -errno.ENOTRECOVERABLE
    assert L.mojette_stage_survivors(plan.handle, 0, 0b11, 0, 0, None, ctypes.byref(n)) == 0 and n.value == 0
    sysp = mj.Plan(64, 4, [-1, 1], systematic=True)
    assert L.mojette_stage_survivors(sysp.handle, 8, 0b1, 8, 1, None, None) == -errno.EINVAL


def test_path_sync_marks_cover_every_cross_front_read():
    """decode_ilv runs the left and the right fronts in two warps that only
    synchronise at the steps the path marks (bit 31 of the forward word).
    Replaying each path: every read of a pixel the other front rebuilt
    must have a marked step after the pixel's step and no later than the
    read; and the marks are sparse (a few per path, not every step)."""
    six = [-3, -2, -1, 1, 2, 3]
    twelve = [v for v in range(-6, 7) if v]
    for P, Q, p, e in [(256, 4, six, 2), (64, 8, twelve, 4), (128, 8, twelve, 4), (20, 3, [-4, -1, 0, 2, 5, 6], 3),
                       (33, 6, [-4, -3, -1, 1, 2, 3, 5, 7], 2)]:
        plan = mj.mojette_plan(P, Q, p)
        masks = inputs.all_masks(len(p), e)
        for m in masks[:: max(1, len(masks) // 12)]:
            sc = mj.mojette_schedule(plan, m)
            T = sc["T"]
            marks = [t for t in range(T) if sc["forward"][t] >> 31 & 1]
            assert len(marks) <= max(8, T // 8), (P, Q, m, len(marks))
            pdir = [[p[i] for i in sc["left"]], [p[i] for i in sc["right"]]]
            by = {}
            x = [[0] * Q, [P - 1] * Q]
            for t in range(T):
                w = sc["steps"][t]
                moved = []
                for side in (0, 1):
                    for l in range(Q):
                        if not w >> (2 * l + side) & 1:
                            continue
                        xx = x[side][l]
                        for l2 in range(Q):
                            c = xx + (l2 - l) * pdir[side][l]
                            if l2 == l or not 0 <= c < P or (l2, c) not in by:
                                continue
                            s2, t2 = by[(l2, c)]
                            if s2 != side:
                                assert any(t2 < s <= t for s in marks), (P, Q, m, t, l, side)
                        moved.append((side, l, xx))
                for side, l, xx in moved:
                    by[(l, xx)] = (side, t)
                    x[side][l] += -1 if side else 1


def _steady_chain(sc, Q):
    """Longest run of same-step links (line l takes line l+1's value of the
    same step) in the path's steady pattern, either side."""
    steady = [t for t in range(sc["T"]) if sc["steps"][t] >> 31 & 1]
    if not steady:
        return 0
    fwd = sc["forward"][steady[0]]
    best = 0
    for side in (0, 1):
        run = 0
        for j in range(Q - 1):
            run = run + 1 if fwd >> (2 * j + side) & 1 else 0
            best = max(best, run)
    return best


def test_paths_prefer_short_same_step_chains():
    """Among the paths with the fewest steps the host keeps one whose
    same-step chains are short: decode_lines runs one shuffle round per
    link of a steady step's longest chain (Q <= 4) or per doubling round
    (Q > 4). At 8 KB (6,4) every two-erasure path links at most two lines in
    a row (three did on six masks before) and still takes at most 132 steps;
    at 8 KB (12,8) most four-erasure paths need at most two scan rounds
    (chains of at most 3 links)."""
    six = [-3, -2, -1, 1, 2, 3]
    plan = mj.mojette_plan(256, 4, six)
    for m in inputs.all_masks(6, 2):
        sc = mj.mojette_schedule(plan, m)
        assert _steady_chain(sc, 4) <= 2, m
        assert sc["T"] <= 132, (m, sc["T"])
    twelve = [v for v in range(-6, 7) if v]
    plan = mj.mojette_plan(128, 8, twelve)
    masks = inputs.all_masks(12, 4)[::3]
    short = sum(_steady_chain(mj.mojette_schedule(plan, m), 8) <= 3 for m in masks)
    assert short >= 0.7 * len(masks), (short, len(masks))


# ---- decode_lines' shared-memory layout (mojette_schedule_layout) ------------

def _bank_model_cost(P, Q, p, sched, phase, orders, rev):
    """Wavefronts of decode_lines' loads and stores under the half-warp bank
    model, replaying the path: a half-warp holds the fronts of one side; a
    load instruction of a half costs the largest number of distinct words
    one slot class (row phase + position, mod S) receives; a front that does
    not move loads nothing; a read outside the image is the zero word beside
    its row (column P)."""
    G = 32 // (2 * Q)
    S = 16 // G
    x = [[0] * Q, [P - 1] * Q]
    cost = 0
    for t in range(sched["T"]):
        w = sched["steps"][t]
        for side in (0, 1):
            per_k = [dict() for _ in range(Q)]
            store = {}
            for l in range(Q):
                if not (w >> (2 * l + side)) & 1:
                    continue
                pp = p[sched["right"][l] if side else sched["left"][l]]
                xx = x[side][l]
                words = [(l, xx)]
                for j in range(1, Q):
                    l2 = (l + j) % Q
                    c = xx + (l2 - l) * pp
                    words.append((l2, c if 0 <= c < P else P))

                def cls(word):
                    return (phase[word[0]] + (-word[1] if rev else word[1])) % S
                o = orders[2 * l + side]
                for k in range(Q):
                    word = words[(o >> (4 * k)) & 15]
                    per_k[k].setdefault(cls(word), set()).add(word)
                store.setdefault(cls(words[0]), set()).add(words[0])
            cost += sum(max(len(v) for v in d.values()) for d in per_k if d)
            cost += max((len(v) for v in store.values()), default=0)
        for l in range(Q):
            for side in (0, 1):
                if (w >> (2 * l + side)) & 1:
                    x[side][l] += -1 if side else 1
    return cost


def _run_parity(P, Q, p, plan, sched, l):
    """Parity of a row start that lets a bulk copy stage the longer of line
    l's two runs of bins (rows in bin order: pixel x at start + P - 1 - x;
    the left run of bins src - x, x < split, lands at start + P - split)."""
    _, offs, _ = mj.mojette_plan_info(plan)

    def src(i):
        bmin = -(P - 1) + min(0, (Q - 1) * p[i])
        return offs[i] + l * p[i] - bmin
    sp = sched["split"][l]
    parL = (src(sched["left"][l]) + 1 - P) & 1
    parR = (src(sched["right"][l]) + 1 - P) & 1
    return parL if sp >= P - sp else parR


@pytest.mark.parametrize("P,Q,p", CONFIGS)
def test_schedule_layout_invariants_and_bank_cost(P, Q, p):
    """The bank layout of every sampled mask: each front reads its own bin
    first and every other word of the step exactly once; row phases are
    slot classes with the parity that stages the longer run of each line by
    bulk copy; the search is deterministic, costs no more wavefronts (bank
    model; the search itself scores at most 96 evenly spaced steps) than
    plain orders with the same parities, and at Q = 8 at least 20% fewer."""
    plan = mj.mojette_plan(P, Q, p)
    n = len(p)
    G = 32 // (2 * Q)
    S = 16 // G
    masks = inputs.all_masks(n, n - Q)
    masks = masks[:: max(1, len(masks) // 12)]
    for m in masks:
        lay = mj.mojette_schedule_layout(plan, m)
        assert lay == mj.mojette_schedule_layout(plan, m)
        sched = mj.mojette_schedule(plan, m)
        for f, o in enumerate(lay["load_order"]):
            nib = [(o >> (4 * k)) & 15 for k in range(Q)]
            assert nib[0] == 0, (m, f)
            assert sorted(nib[1:]) == list(range(1, Q)), (m, f, nib)
        for l, e in enumerate(lay["row_phase"]):
            assert 0 <= e < S
            assert e % 2 == _run_parity(P, Q, p, plan, sched, l), (m, l)
        plain = [sum(k << (4 * k) for k in range(Q))] * (2 * Q)
        parity = [_run_parity(P, Q, p, plan, sched, l) for l in range(Q)]
        got = _bank_model_cost(P, Q, p, sched, lay["row_phase"], lay["load_order"], True)
        ref = _bank_model_cost(P, Q, p, sched, parity, plain, True)
        assert got <= 1.01 * ref, (m, got, ref)
        if Q == 8:
            assert got <= 0.8 * ref, (m, got, ref)


def test_schedule_layout_systematic_rows_even_and_no_bank_model_parity_only():
    """Systematic paths keep even row phases (their residual rows start at
    even words); a geometry with no bank model (Q = 3: five stripes per
    warp) gets only the staging parity and plain load orders."""
    sysplan = mj.mojette_plan_ex(128, 8, [-2, -1, 1, 2], mj.MOJETTE_PLAN_SYSTEMATIC)
    for lost in ([0, 3, 5], [1, 2, 6, 7], [2, 4]):
        m = sum(1 << i for i in lost)
        lay = mj.mojette_schedule_layout(sysplan, m)
        assert lay["lines"] == len(lost)
        assert all(e % 2 == 0 for e in lay["row_phase"]), lay
    p = [-2, -1, 1, 2, 3]
    plan = mj.mojette_plan(96, 3, p)
    for m in inputs.all_masks(len(p), 2):
        lay = mj.mojette_schedule_layout(plan, m)
        sched = mj.mojette_schedule(plan, m)
        assert lay["row_phase"] == [_run_parity(96, 3, p, plan, sched, l) for l in range(3)]
        assert all(o & 0xFFF == 0x210 for o in lay["load_order"]), lay


def test_schedule_layout_validates_arguments():
    plan = mj.mojette_plan(128, 4, [-3, -2, -1, 1, 2, 3])
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_schedule_layout(plan, 1 << 9)          # bit beyond n
    assert ei.value.code == -errno.EINVAL
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_schedule_layout(plan, 0b000111)        # three lost: two survivors short
    assert ei.value.code == -errno.ENOTRECOVERABLE
    assert mj.lib().mojette_schedule_layout(None, 0, None, None) == -errno.EINVAL
