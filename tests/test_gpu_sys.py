"""GPU parity of the systematic form against the CPU oracle, bit-exact.

The paper mentions a systematic Mojette code (Sec. 2.3, Sec. 4) without
defining it; the reading here: the Q data lines are Q of the packets and the
parity packets are Eq. 1 projections of the whole image (mojette_encode of a
MOJETTE_PLAN_SYSTEMATIC plan). mojette_sys_decode rebuilds the lost data
lines in place; every case is compared with oracle.sys_decode element by
element, and every word the call must not write is checked unchanged.
Integer XOR work: the tolerance is zero.
"""
import numpy as np
import pytest

import oracle
from paper_1504_07038_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1504_07038_gb300 import binding as mj


def dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


@pytest.fixture(autouse=True)
def clean_status():
    mj.mojette_device_status(clear=True)
    yield
    assert mj.mojette_device_status(clear=True) == 0


SYS_GEOMS = [
    ("4KB(6,4)", 128, 4, [-1, 1]),
    ("8KB(6,4)", 256, 4, [-1, 1]),
    ("4KB(12,8)", 64, 8, [-2, -1, 1, 2]),
    ("8KB(12,8)", 128, 8, [-2, -1, 1, 2]),
    ("8KB(10,8)", 128, 8, [-1, 1]),
    ("odd(7,4)", 37, 4, [-4, 0, 2]),
]
GARBAGE = np.uint64(0xA5A5A5A5A5A5A5A5)


def all_masks(Q, r, limit=None, seed=5):
    """Masks losing e >= 1 data lines and f parity packets, e + f <= r."""
    ms = [m for m in range(1 << (Q + r)) if bin(m).count("1") <= r and m & ((1 << Q) - 1)]
    if limit and len(ms) > limit:
        ms = [ms[i] for i in np.random.default_rng(seed).choice(len(ms), limit, replace=False)]
    return ms


def lost_lines(mask, Q):
    return [l for l in range(Q) if mask >> l & 1]


def sys_decode_gpu(plan, par_np, mask, img_np, guard=2):
    """Run mojette_sys_decode in place on a copy of img_np whose lost lines
    hold garbage, inside a buffer with `guard` stripes of garbage on both
    sides. Returns (stripes after the call, guard stripes after the call)."""
    S, Q, P = img_np.shape
    buf = np.full((S + 2 * guard, Q, P), GARBAGE, dtype=np.uint64)
    buf[guard:guard + S] = img_np
    buf[guard:guard + S, lost_lines(mask, Q)] = GARBAGE
    d = dev(buf)
    d_par = dev(par_np)
    mj.mojette_sys_decode(plan, d_par, mask, d[guard:guard + S], S)
    torch.cuda.synchronize()
    out = host(d)
    return out[guard:guard + S], np.concatenate([out[:guard], out[guard + S:]])


@pytest.mark.parametrize("name,P,Q,p", SYS_GEOMS)
def test_parity_encode_matches_oracle(name, P, Q, p):
    S = 300
    plan = mj.Plan(P, Q, p, systematic=True)
    img = inputs.stripes(S, Q, P, seed=P + Q)
    d_par = torch.empty((S, plan.total), dtype=torch.int64, device="cuda")
    mj.mojette_encode(plan, dev(img), d_par, S)
    torch.cuda.synchronize()
    assert (host(d_par) == oracle.encode(img, p, threads=8)).all()


@pytest.mark.parametrize("name,P,Q,p", SYS_GEOMS)
def test_sys_decode_every_mask(name, P, Q, p):
    """Every mask (a seeded sample of 40 at Q = 8) on 300 stripes: several
    work items per CTA and a ragged last warp. The lost lines equal the
    oracle's; the known lines and the guard stripes are untouched."""
    S = 300
    plan = mj.Plan(P, Q, p, systematic=True)
    img = inputs.stripes(S, Q, P, seed=3 * P + Q)
    par = oracle.encode(img, p, threads=8)
    for m in all_masks(Q, len(p), limit=40):
        data = img.copy()
        data[:, lost_lines(m, Q)] = GARBAGE
        ref = oracle.sys_decode(data, par, p, P, Q, m, threads=8)
        got, guard = sys_decode_gpu(plan, par, m, img)
        assert (got == ref).all(), m
        assert (ref == img).all()
        assert (guard == GARBAGE).all(), m


@pytest.mark.parametrize("name,P,Q,p", SYS_GEOMS)
def test_sys_two_lost_lines_sweep_and_closed_form(monkeypatch, name, P, Q, p):
    """Two lost data lines: the residual + decode_lines sweep (the default)
    and decode_scan2 (the closed form, opt-in) give the oracle's lines, for
    every pair of lines and every surviving parity set."""
    S = 67
    plan = mj.Plan(P, Q, p, systematic=True)
    img = inputs.stripes(S, Q, P, seed=5 * P + Q)
    par = oracle.encode(img, p, threads=8)
    r = len(p)
    masks = [m for m in range(1 << (Q + r))
             if bin(m & ((1 << Q) - 1)).count("1") == 2 and r - bin(m >> Q).count("1") >= 2]
    masks = masks[:: max(1, len(masks) // 30)]
    for kernel in ("scan", "lines"):
        monkeypatch.setenv("MOJETTE_DECODE_KERNEL", kernel)
        for m in masks:
            got, guard = sys_decode_gpu(plan, par, m, img)
            assert (got == img).all(), (kernel, m)
            assert (guard == GARBAGE).all()


@pytest.mark.parametrize("S", [1, 5, 31, 4096 + 13])
def test_sys_decode_sizes(S):
    """One stripe, a few, one warp's worth minus one, and enough stripes for
    the bank-phased row layout (launches of >= 4096 stripes)."""
    P, Q, p = 256, 4, [-1, 1]
    plan = mj.Plan(P, Q, p, systematic=True)
    img = inputs.stripes(S, Q, P, seed=S)
    par = oracle.encode(img, p, threads=8)
    for m in (0b0001, 0b1001, 0b0110, 0b0100 | 1 << 4, 0b1000 | 1 << 5):
        got, guard = sys_decode_gpu(plan, par, m, img)
        assert (got == img).all(), m
        assert (guard == GARBAGE).all()


def test_sys_decode_lost_parity_is_never_read():
    P, Q, p = 128, 8, [-2, -1, 1, 2]
    S = 100
    plan = mj.Plan(P, Q, p, systematic=True)
    img = inputs.stripes(S, Q, P, seed=8)
    par = oracle.encode(img, p, threads=8)
    off, bins = plan.offsets, plan.bins
    for m in (0b00010001 | 0b0101 << 8, 0b00000100 | 0b1110 << 8, 0b01000010 | 0b1001 << 8):
        junk = par.copy()
        for i in range(len(p)):
            if m >> (Q + i) & 1:
                junk[:, off[i]:off[i] + bins[i]] = GARBAGE
        got, _ = sys_decode_gpu(plan, junk, m, img)
        assert (got == img).all(), m


def test_sys_decode_no_lost_line_writes_nothing():
    P, Q, p = 128, 4, [-1, 1]
    S = 64
    plan = mj.Plan(P, Q, p, systematic=True)
    img = inputs.stripes(S, Q, P, seed=2)
    d = dev(img)
    for m in (0, 1 << 4, 3 << 4):
        mj.mojette_sys_decode(plan, d, m, d, S)     # parity pointer unused
    torch.cuda.synchronize()
    assert (host(d) == img).all()


def test_sys_decode_refusals():
    P, Q, p = 128, 4, [-1, 1]
    plan = mj.Plan(P, Q, p, systematic=True)
    d = torch.zeros((4, Q, P), dtype=torch.int64, device="cuda")
    par = torch.zeros((4, plan.total), dtype=torch.int64, device="cuda")
    with pytest.raises(mj.MojetteError):
        mj.mojette_sys_decode(plan, par, 0b0111, d, 4)          # 3 lost, 2 parity
    with pytest.raises(mj.MojetteError):
        mj.mojette_decode(plan, par, 0, d, 4)                   # not for systematic plans


def test_sys_batched_mixed_with_plain_decodes():
    """One batch (as a CUDA graph): systematic decodes of two geometries
    with per-stripe masks -- 0 to r lost lines, so several launches by lost
    count and stripes that launch nothing -- next to plain decodes and
    encodes. Every stripe equals the oracle; stripes with nothing lost are
    untouched."""
    rng = np.random.default_rng(21)
    geo = [(128, 4, [-1, 1]), (64, 8, [-2, -1, 1, 2])]
    splans = [mj.Plan(P, Q, p, systematic=True) for P, Q, p in geo]
    nplan = mj.mojette_plan(128, 4, [-3, -2, -1, 1, 2, 3])
    plans = splans + [nplan]
    S = 900
    which = rng.integers(0, 3, S)
    rows, expect = [], []
    for s in range(S):
        k = int(which[s])
        pl = plans[k]
        img = inputs.stripes(1, pl.Q, pl.P, seed=40 + s)
        if k < 2:
            r = len(pl.p)
            cand = [m for m in range(1 << (pl.Q + r)) if bin(m).count("1") <= r]
            m = int(cand[rng.integers(0, len(cand))])
            par = oracle.encode(img, pl.p)
            data = img.copy()
            data[:, lost_lines(m, pl.Q)] = GARBAGE
            d_src, d_dst = dev(par), dev(data)
            rows.append((k, mj.MOJETTE_OP_DECODE, m, d_src, d_dst))
            expect.append(oracle.sys_decode(data, par, pl.p, pl.P, pl.Q, m))
        else:
            m = int(inputs.erasure_masks(1, 6, int(rng.integers(0, 3)), first=s)[0])
            proj = oracle.encode(img, pl.p)
            d_src = dev(proj)
            d_dst = torch.zeros((1, pl.Q, pl.P), dtype=torch.int64, device="cuda")
            rows.append((k, mj.MOJETTE_OP_DECODE, m, d_src, d_dst))
            expect.append(oracle.decode(proj, pl.p, pl.P, pl.Q, m))
    table = mj.stripe_table(plans, np.array([r[0] for r in rows]), np.array([r[1] for r in rows]),
                            np.array([r[2] for r in rows], dtype=np.uint32),
                            np.array([r[3].data_ptr() for r in rows], dtype=np.uint64),
                            np.array([r[4].data_ptr() for r in rows], dtype=np.uint64))
    batch = mj.mojette_batch_create(table, plans, mj.MOJETTE_BATCH_GRAPH)
    info = mj.mojette_batch_info(batch)
    mj.mojette_batch_run(batch)
    torch.cuda.synchronize()
    for s, r in enumerate(rows):
        assert (host(r[4]) == expect[s]).all(), (s, r[0], r[2])
    # the tuner's candidates for the systematic launches are exact too
    mj.mojette_batch_tune(batch, reps=1)
    for s, r in enumerate(rows):
        if r[0] < 2:
            pl = plans[r[0]]
            data = expect[s].copy()
            data[:, lost_lines(r[2], pl.Q)] = GARBAGE
            r[4].copy_(dev(data))
    mj.mojette_batch_run(batch)
    torch.cuda.synchronize()
    for s, r in enumerate(rows):
        assert (host(r[4]) == expect[s]).all(), (s, r[0], r[2])
    assert info["launches"] >= 3
    batch.close()
