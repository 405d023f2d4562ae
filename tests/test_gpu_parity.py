"""GPU parity: the CUDA path against the CPU oracle, bit-exact.

Encode and decode run through the C ABI (ctypes binding) on cuda:0 and are
compared element by element with the oracle on the same seeded inputs: at
sizes spanning many tiles with ragged tails, on every erasure pattern of the
benchmark geometries, on edge cases (tiny, odd-sized and degenerate
geometries), and at the full benchmark sizes on sampled stripes plus the
size-independent property decode(encode(img)) == img on every stripe.
Integer XOR work: the tolerance is zero.
"""
import errno

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


def empty(shape, fill=0x5A5A5A5A5A5A5A5A):
    t = torch.empty(shape, dtype=torch.int64, device="cuda")
    t.fill_(fill - (1 << 64) if fill >= (1 << 63) else fill)
    return t


@pytest.fixture(autouse=True)
def clean_status():
    mj.mojette_device_status(clear=True)
    yield
    assert mj.mojette_device_status(clear=True) == 0


SIX = [-3, -2, -1, 1, 2, 3]
TWELVE = [v for v in range(-6, 7) if v]
GEOMS = [
    ("4KB(6,4)", 128, 4, SIX),
    ("8KB(6,4)", 256, 4, SIX),
    ("4KB(12,8)", 64, 8, TWELVE),
    ("8KB(12,8)", 128, 8, TWELVE),
    ("4KB(3,2)", 256, 2, [-1, 1, 2]),
    ("8KB(3,2)", 512, 2, [-1, 1, 2]),
]


def encode_gpu(plan, img_np):
    S = img_np.shape[0]
    out = empty((S, plan.total))
    mj.mojette_encode(plan, dev(img_np), out, S)
    torch.cuda.synchronize()
    return host(out)


def decode_gpu(plan, proj_np, mask, S=None):
    S = proj_np.shape[0] if S is None else S
    out = empty((S, plan.Q, plan.P))
    mj.mojette_decode(plan, dev(proj_np), mask, out, S)
    torch.cuda.synchronize()
    return host(out)


@pytest.mark.parametrize("name,P,Q,p", GEOMS)
@pytest.mark.parametrize("S", [1, 7, 1023, 1024])
def test_encode_matches_oracle(name, P, Q, p, S):
    img = inputs.stripes(S, Q, P, seed=S + P)
    plan = mj.mojette_plan(P, Q, p)
    assert (encode_gpu(plan, img) == oracle.encode(img, p, threads=8)).all()


@pytest.mark.parametrize("name,P,Q,p", GEOMS)
def test_decode_every_erasure_pattern(name, P, Q, p):
    """Every mask with n - Q erasures (all 15 / 495 / 3), and samples of the
    masks with fewer, decoded from oracle-made projections."""
    n = len(p)
    S = 67
    img = inputs.stripes(S, Q, P, seed=3)
    proj = oracle.encode(img, p, threads=8)
    plan = mj.mojette_plan(P, Q, p)
    d_proj = dev(proj)
    masks = inputs.all_masks(n, n - Q)
    for e in range(0, n - Q):
        ms = inputs.all_masks(n, e)
        masks += ms if len(ms) <= 24 else ms[:: len(ms) // 24]
    out = empty((S, Q, P))
    for m in masks:
        out.fill_(0x1234)
        mj.mojette_decode(plan, d_proj, m, out, S)
        got = host(out)
        assert (got == img).all(), (name, m)
    # the last mask also against the oracle's own decoder
    assert (host(out) == oracle.decode(proj, p, P, Q, masks[-1], threads=8)).all()


@pytest.mark.parametrize("name,P,Q,p", GEOMS[:4])
def test_round_trip_on_gpu_with_ragged_batches(name, P, Q, p):
    for S in [1, 5, 33, 1000]:
        img = inputs.stripes(S, Q, P, seed=S)
        plan = mj.mojette_plan(P, Q, p)
        d_img = dev(img)
        d_proj = empty((S, plan.total))
        mj.mojette_encode(plan, d_img, d_proj, S)
        mask = int(inputs.erasure_masks(1, len(p), len(p) - Q, seed=S)[0])
        out = empty((S, Q, P))
        mj.mojette_decode(plan, d_proj, mask, out, S)
        torch.cuda.synchronize()
        assert (host(out) == img).all()


def _tiny():
    rng = np.random.default_rng(77)
    cases = []
    for P in [1, 2, 3, 5, 8, 13]:
        for Q in [1, 2, 3, 4, 5, 16]:
            n = int(min(Q + int(rng.integers(0, 3)), 11))
            p = sorted(rng.choice(np.arange(-5, 6), size=n, replace=False).tolist())
            cases.append((P, Q, p))
    cases.append((9, 16, list(range(-9, 0)) + list(range(1, 9))))   # Q = 16, n = 17
    return cases


@pytest.mark.parametrize("P,Q,p", _tiny())
def test_edge_geometries(P, Q, p):
    """Tiny and odd geometries: Q*P odd (non-bulk staging), |p| > P (empty
    bins), p = 0, Q = 1, Q not a power of two, Q = 16 (largest decode)."""
    S = 45
    img = inputs.stripes(S, Q, P, seed=P * 31 + Q)
    plan = mj.mojette_plan(P, Q, p)
    proj = oracle.encode(img, p)
    assert (encode_gpu(plan, img) == proj).all()
    n = len(p)
    for e in range(0, n - Q + 1):
        for m in inputs.all_masks(n, e)[:6]:
            assert (decode_gpu(plan, proj, m) == img).all(), (P, Q, p, m)


def test_output_bounds_untouched():
    """Nothing is written outside [0, S) stripes (canaries on both sides)."""
    P, Q, p = 128, 8, TWELVE
    S = 301
    plan = mj.mojette_plan(P, Q, p)
    img = inputs.stripes(S, Q, P)
    pad = 64
    proj_buf = empty((S * plan.total + 2 * pad,), fill=0x0F0F)
    mj.mojette_encode(plan, dev(img), proj_buf[pad:pad + S * plan.total], S)
    h = host(proj_buf)
    assert (h[:pad] == 0x0F0F).all() and (h[-pad:] == 0x0F0F).all()
    assert (h[pad:-pad].reshape(S, -1) == oracle.encode(img, p, threads=8)).all()
    img_buf = empty((S * Q * P + 2 * pad,), fill=0x0F0F)
    mj.mojette_decode(plan, proj_buf[pad:pad + S * plan.total], 0b111100000000,
                      img_buf[pad:pad + S * Q * P], S)
    h = host(img_buf)
    assert (h[:pad] == 0x0F0F).all() and (h[-pad:] == 0x0F0F).all()
    assert (h[pad:-pad].reshape(S, Q, P) == img).all()


def test_too_few_survivors_refused_before_launch():
    plan = mj.mojette_plan(128, 4, SIX)
    buf = empty((8, plan.total))
    img = empty((8, 4, 128))
    with pytest.raises(mj.MojetteError):
        mj.mojette_decode(plan, buf, 0b000111, img, 8)


def _full_size(P, Q, p, S, masks, sample=48):
    """Full-size encode + decode in the benchmark's launch configuration:
    sampled stripes against the oracle, every stripe against the input."""
    plan = mj.mojette_plan(P, Q, p)
    img = inputs.stripes(S, Q, P)
    d_img = dev(img)
    d_proj = empty((S, plan.total))
    mj.mojette_encode(plan, d_img, d_proj, S)
    rng = np.random.default_rng(S)
    idx = np.unique(np.concatenate([[0, S - 1], rng.integers(0, S, sample)]))
    ref_img = inputs.stripe_rows(idx, Q, P)
    ref_proj = oracle.encode(ref_img, p, threads=8)
    got = host(d_proj[torch.from_numpy(idx).cuda()])
    assert (got == ref_proj).all()
    out = empty((S, Q, P))
    for m in masks:
        out.fill_(0)
        mj.mojette_decode(plan, d_proj, m, out, S)
        assert bool((out == d_img).all())
        assert (host(out[torch.from_numpy(idx).cuda()]) ==
                oracle.decode(ref_proj, p, P, Q, m, threads=8)).all()


def test_full_size_plain_at_scale_every_two_erasure_mask():
    """262144 stripes of 8 KB, (6,4): encode, then decode under all 15
    two-erasure patterns."""
    _full_size(256, 4, SIX, 262144, inputs.all_masks(6, 2))


def test_full_size_wide_geometry():
    """262144 stripes at 4 KB and 8 KB, (12,8), four erasures (a sample of the
    495 patterns at full size; all 495 run at small size above)."""
    ms = inputs.all_masks(12, 4)
    _full_size(64, 8, TWELVE, 262144, ms[::61])
    _full_size(128, 8, TWELVE, 262144, ms[7::83])


VARIANTS = [("ring", {}), ("ilv", {}), ("ilv", {"MOJETTE_DECODE_G": "5"}), ("ilv", {"MOJETTE_DECODE_G": "16"}),
            ("lines", {}), ("lines", {"MOJETTE_DECODE_ROWOFF": "0"}), ("fronts", {}), ("stream", {}),
            ("cols", {}), ("vander", {}), ("vander", {"MOJETTE_DECODE_GPC": "1"})]


@pytest.mark.parametrize("kernel,K", VARIANTS)
@pytest.mark.parametrize("name,P,Q,p", [GEOMS[0], GEOMS[2], GEOMS[3], GEOMS[4]]
                         + [("tiny(6,3)", 20, 3, [-4, -1, 0, 2, 5, 6]),
                            ("odd P(8,6)", 33, 6, [-4, -3, -1, 1, 2, 3, 5, 7])])
def test_every_decode_kernel_variant(monkeypatch, kernel, K, name, P, Q, p):
    """Each decode kernel (decode_ilv at several work-item widths,
    decode_lines with and without row phases, decode_fronts, decode_stream,
    decode_cols, decode_vander), every k-of-n mask (sampled at (12,8)),
    bit-exact."""
    monkeypatch.setenv("MOJETTE_DECODE_KERNEL", kernel)
    for k, v in K.items():
        monkeypatch.setenv(k, v)
    S = 53
    n = len(p)
    img = inputs.stripes(S, Q, P, seed=P + Q)
    proj = oracle.encode(img, p, threads=8)
    plan = mj.mojette_plan(P, Q, p)
    d_proj = dev(proj)
    out = empty((S, Q, P))
    masks = inputs.all_masks(n, n - Q)
    masks = masks if len(masks) <= 60 else masks[::9]
    masks += inputs.all_masks(n, 0)
    for m in masks:
        out.fill_(0x77)
        mj.mojette_decode(plan, d_proj, m, out, S)
        assert (host(out) == img).all(), (kernel, K, name, m)


@pytest.mark.parametrize("kernel", ["ring", "ilv", "lines"])
def test_path_kernels_8k_6x4_large_launch(monkeypatch, kernel):
    """The Sec. 2.2 path kernels at the headline geometry, 8 KB (6,4) (P = 256,
    Q = 4), in a launch of 4096 + 77 stripes -- large enough for decode_lines'
    searched row phases and per-front load orders and for decode_ilv's widest
    work items, with a ragged last item -- under every two-erasure mask and
    the no-erasure mask, element by element against the oracle."""
    monkeypatch.setenv("MOJETTE_DECODE_KERNEL", kernel)
    P, Q, p, S = 256, 4, SIX, 4096 + 77
    img = inputs.stripes(S, Q, P, seed=41)
    proj = oracle.encode(img, p, threads=8)
    plan = mj.mojette_plan(P, Q, p)
    assert mj.mojette_decode_kernel(plan, 0b11, S=S) == "decode_" + kernel
    d_proj = dev(proj)
    out = empty((S, Q, P))
    for m in inputs.all_masks(6, 2) + [0]:
        ref = oracle.decode(proj, p, P, Q, m, threads=8)
        out.fill_(0x5A)
        mj.mojette_decode(plan, d_proj, m, out, S)
        assert (host(out) == ref).all(), (kernel, m)


RING_GEOMS = [("4KB(6,4)", 128, 4, SIX), ("8KB(6,4)", 256, 4, SIX), ("16KB(6,4)", 512, 4, SIX),
              ("4KB(3,2)", 256, 2, [-1, 1, 2]), ("8KB(3,2)", 512, 2, [-1, 1, 2]),
              ("odd directions", 96, 3, [-5, -2, 1, 4, 7])]


@pytest.mark.parametrize("name,P,Q,p", RING_GEOMS)
@pytest.mark.parametrize("S", [1, 13, 2053])
def test_ring_decode_every_mask(monkeypatch, name, P, Q, p, S):
    """decode_ring (the one-sided path, each stripe's lines held as rings of
    64 or 128 words fed by 128-byte bulk copies): every k-of-n and every
    smaller erasure mask, ragged work items, against the oracle; the kernel
    really runs (the path fits a ring at these geometries)."""
    monkeypatch.setenv("MOJETTE_DECODE_KERNEL", "ring")
    n = len(p)
    img = inputs.stripes(S, Q, P, seed=13 * P + Q + S)
    proj = oracle.encode(img, p, threads=8)
    plan = mj.mojette_plan(P, Q, p)
    d_proj = dev(proj)
    out = empty((S, Q, P))
    masks = [m for m in range(1 << n) if n - bin(m).count("1") >= Q]
    masks = masks if S < 1000 else masks[:: max(1, len(masks) // 6)]
    for m in masks:
        assert mj.mojette_decode_kernel(plan, m, S) == "decode_ring", (name, m)
        out.fill_(0x66)
        mj.mojette_decode(plan, d_proj, m, out, S)
        assert (host(out) == img).all(), (name, m)


def test_stage_survivors_then_decode():
    """mojette_stage_survivors copies from pinned host memory exactly the Q
    projections the decode's path reads (their slices, every stripe) and
    nothing else: the other words of the device block keep their junk, the
    byte count is S * 8 * (sum of the used B_i), and the decode from that
    block gives the image."""
    P, Q, p, S = 128, 8, TWELVE, 777
    plan = mj.mojette_plan(P, Q, p)
    img = inputs.stripes(S, Q, P, seed=77)
    proj = oracle.encode(img, p, threads=8)
    h = torch.from_numpy(proj.view(np.int64)).pin_memory()
    offs, bins, _, _ = oracle.offsets(p, P, Q)
    for m in inputs.all_masks(len(p), 4)[::97] + inputs.all_masks(len(p), 1)[:2]:
        d = empty((S, plan.total), fill=0x0BAD)
        moved = mj.mojette_stage_survivors(plan, h, m, d, S)
        sc = mj.mojette_schedule(plan, m)
        used = set(sc["left"]) | set(sc["right"])
        assert len(used) == Q and not any(m >> i & 1 for i in used)
        assert moved == S * 8 * sum(bins[i] for i in used)
        got = host(d)
        for i, (o, B) in enumerate(zip(offs, bins)):
            want = proj[:, o:o + B] if i in used else np.uint64(0x0BAD)
            assert (got[:, o:o + B] == want).all(), (m, i)
        out = empty((S, Q, P))
        mj.mojette_decode(plan, d, m, out, S)
        assert (host(out) == img).all(), m


def test_decode_time_flat_across_masks():
    """Sec. 4 (Fig. 2-3): decode cost does not depend on which projections
    are lost. Every two-erasure mask of 8 KB (6,4) on 65536 stripes, timed
    with CUDA events (median of 3): the slowest mask within 1.3x of the
    median mask. (The paths of the 15 masks differ by at most a few steps;
    the default path kernel runs only the shuffle rounds a path's same-step
    chains need, so masks whose chains are short run faster than the rest:
    the bound is on how much slower any mask can be.)"""
    P, Q, p, S = 256, 4, [-3, -2, -1, 1, 2, 3], 65536
    plan = mj.mojette_plan(P, Q, p)
    img = torch.from_numpy(inputs.stripes(S, Q, P, seed=3).view(np.int64)).cuda()
    proj = torch.empty((S, plan.total), dtype=torch.int64, device="cuda")
    out = torch.empty_like(img)
    mj.mojette_encode(plan, img, proj, S)
    times = []
    for m in inputs.all_masks(len(p), 2):
        mj.mojette_decode(plan, proj, m, out, S)          # warm-up, path cached
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            mj.mojette_decode(plan, proj, m, out, S)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        times.append(sorted(ts)[1])
        assert torch.equal(out, img), bin(m)
    assert max(times) / sorted(times)[len(times) // 2] < 1.3, times


TRIM_CASES = [GEOMS[1], GEOMS[2], GEOMS[3], ("tiny(6,3)", 20, 3, [-4, -1, 0, 2, 5, 6])]


def trimmed_reference(plan, full_proj, p, P, Q):
    """The oracle's full projections gathered into a trimmed plan's layout."""
    offs, _, _, _ = oracle.offsets(p, P, Q)
    cols = [offs[i] + int(plan.full_bin[t]) for i in range(len(p))
            for t in range(plan.offsets[i], plan.offsets[i] + plan.bins[i])]
    return np.ascontiguousarray(full_proj[:, cols])


@pytest.mark.parametrize("name,P,Q,p", TRIM_CASES)
def test_trimmed_plan_encode_decode(name, P, Q, p):
    """Unused-bin removal: encode writes exactly the oracle's bins at the
    stored positions; decode from the stored bins alone (lost projections'
    slices junk) gives the image, for every mask (sampled at (12,8))."""
    tr = mj.mojette_plan_ex(P, Q, p, mj.MOJETTE_PLAN_TRIM_UNUSED)
    S = 301
    img = inputs.stripes(S, Q, P, seed=P * Q + 7)
    ref = trimmed_reference(tr, oracle.encode(img, p, threads=8), p, P, Q)
    assert ref.shape == (S, tr.total)
    assert (encode_gpu(tr, img) == ref).all()
    n = len(p)
    masks = [m for e in range(n - Q + 1) for m in inputs.all_masks(n, e)]
    masks = masks if len(masks) <= 80 else masks[::11]
    for m in masks:
        pr = ref.copy()
        for i in range(n):
            if (m >> i) & 1:
                pr[:, tr.offsets[i]: tr.offsets[i] + tr.bins[i]] = np.uint64(0xDEADBEEFDEADBEEF)
        assert (decode_gpu(tr, pr, m) == img).all(), (name, bin(m))


def test_trimmed_and_full_plans_in_one_batch():
    T12 = [v for v in range(-6, 7) if v]
    plans = [mj.mojette_plan_ex(64, 8, T12, mj.MOJETTE_PLAN_TRIM_UNUSED), mj.mojette_plan(256, 4, SIX)]
    geo = [(64, 8, T12), (256, 4, SIX)]
    S = [190, 70]
    imgs, d_proj, d_out, rows = [], [], [], []
    for k, ((P, Q, p), s) in enumerate(zip(geo, S)):
        img = inputs.stripes(s, Q, P, seed=31 + k)
        ref = oracle.encode(img, p, threads=8)
        if plans[k].trimmed:
            ref = trimmed_reference(plans[k], ref, p, P, Q)
        imgs.append(img)
        d_proj.append(dev(ref))
        d_out.append(empty((s, Q, P)))
    masks = [inputs.erasure_masks(s, len(g[2]), inputs.erasure_counts(s, len(g[2]) - g[1], seed=5), seed=6)
             for s, g in zip(S, geo)]
    ks = np.concatenate([np.full(s, k) for k, s in enumerate(S)])
    src = np.concatenate([d_proj[k].data_ptr() + np.arange(s, dtype=np.uint64) * np.uint64(plans[k].total * 8)
                          for k, s in enumerate(S)])
    dst = np.concatenate([d_out[k].data_ptr() + np.arange(s, dtype=np.uint64) * np.uint64(geo[k][0] * geo[k][1] * 8)
                          for k, s in enumerate(S)])
    table = mj.stripe_table(plans, ks, mj.MOJETTE_OP_DECODE, np.concatenate(masks), src, dst)
    b = mj.mojette_batch_create(table, plans, mj.MOJETTE_BATCH_GRAPH)
    mj.mojette_batch_run(b)
    torch.cuda.synchronize()
    for k in range(2):
        assert (host(d_out[k]) == imgs[k]).all()


@pytest.mark.parametrize("P,Q,p", [(2048, 4, SIX), (4096, 4, SIX), (1024, 8, TWELVE), (6000, 2, [-1, 1, 2])])
def test_large_stripes(P, Q, p):
    """Stripes far above the paper's blocks (16 KB to 94 KB): encode stages
    one stripe per tile, decode runs one or a few stripes per warp."""
    S = 37
    img = inputs.stripes(S, Q, P, seed=P + Q)
    plan = mj.mojette_plan(P, Q, p)
    proj = oracle.encode(img, p, threads=8)
    assert (encode_gpu(plan, img) == proj).all()
    n = len(p)
    for m in inputs.all_masks(n, n - Q)[:4] + [0]:
        assert (decode_gpu(plan, proj, m) == img).all(), (P, Q, bin(m))


def test_stripe_beyond_shared_memory_refused():
    """A stripe whose words cannot fit in one CTA's shared memory is refused
    before any launch."""
    P, Q, p = 16384, 4, SIX
    plan = mj.mojette_plan(P, Q, p)
    buf = empty((2, plan.total))
    out = empty((2, Q, P))
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_decode(plan, buf, 0b000011, out, 2)
    assert ei.value.code == -errno.EINVAL


def test_bounded_wait_reports_timeout():
    """Failure detection without a fault: a wait that nothing completes gives
    up after its limit, the status word says so (-ETIMEDOUT), the status is
    cleared, and the device still computes correctly."""
    mj.mojette_selftest_wait(20_000_000)
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_device_status(clear=True)
    assert ei.value.code == -errno.ETIMEDOUT
    assert mj.mojette_device_status(clear=True) == 0
    P, Q, p = 128, 4, SIX
    plan = mj.mojette_plan(P, Q, p)
    img = inputs.stripes(9, Q, P, seed=2)
    proj = oracle.encode(img, p)
    assert (encode_gpu(plan, img) == proj).all()
    assert (decode_gpu(plan, proj, 0b000101) == img).all()


TWO_LINE = [("4KB(3,2)", 256, 2, [-1, 1, 2]), ("8KB(3,2)", 512, 2, [-1, 1, 2]),
            ("wide gaps", 40, 2, [-7, -2, 0, 3, 9]), ("|p| > P", 3, 2, [-5, 1, 4]),
            ("one pixel", 1, 2, [-1, 2]), ("odd", 37, 2, [0, 5])]


@pytest.mark.parametrize("kernel", ["default", "scan", "lines", "ring"])
@pytest.mark.parametrize("name,P,Q,p", TWO_LINE)
@pytest.mark.parametrize("S", [1, 5, 4096 + 7])
def test_two_line_closed_form(monkeypatch, kernel, name, P, Q, p, S):
    """Two-line images: the default path kernel and, forced, decode_scan2
    (the chain recurrence of the two dedicated projections, evaluated by
    pointer doubling) and the sweep: every mask leaving >= 2 projections,
    ragged work items, bit-exact with the oracle."""
    if kernel != "default":
        monkeypatch.setenv("MOJETTE_DECODE_KERNEL", kernel)
    n = len(p)
    img = inputs.stripes(S, Q, P, seed=7 * P + S)
    proj = oracle.encode(img, p, threads=8)
    plan = mj.mojette_plan(P, Q, p)
    d_proj = dev(proj)
    out = empty((S, Q, P))
    masks = [m for m in range(1 << n) if n - bin(m).count("1") >= Q]
    if S > 100:
        masks = masks[:4]
    for m in masks:
        out.fill_(0x33)
        mj.mojette_decode(plan, d_proj, m, out, S)
        torch.cuda.synchronize()
        assert (host(out) == img).all(), (kernel, name, m)


VANDER_GEOMS = [("8KB(6,4)", 256, 4, SIX), ("4KB(12,8)", 64, 8, TWELVE), ("8KB(12,8)", 128, 8, TWELVE),
                ("tiny", 1, 3, [-2, 0, 5, 7]), ("|p| > P", 5, 4, [-7, -1, 3, 8, 9]),
                ("one-signed", 40, 5, [1, 2, 4, 5, 9, 11]), ("Q=2", 77, 2, [-3, 4, 6])]


@pytest.mark.parametrize("name,P,Q,p", VANDER_GEOMS)
@pytest.mark.parametrize("S", [1, 6, 4099])
def test_vandermonde_decode(monkeypatch, name, P, Q, p, S):
    """decode_vander (the Bjorck-Pereyra solve of Eq. 1's Vandermonde
    system) on every k-of-n mask (sampled at (12,8), four masks at the
    largest S), ragged work items, bit-exact."""
    monkeypatch.setenv("MOJETTE_DECODE_KERNEL", "vander")
    n = len(p)
    img = inputs.stripes(S, Q, P, seed=11 * P + Q + S)
    proj = oracle.encode(img, p, threads=8)
    plan = mj.mojette_plan(P, Q, p)
    d_proj = dev(proj)
    out = empty((S, Q, P))
    masks = [m for m in range(1 << n) if n - bin(m).count("1") >= Q]
    masks = masks[:: max(1, len(masks) // 40)] if S < 100 else masks[:4]
    for m in masks:
        out.fill_(0x55)
        mj.mojette_decode(plan, d_proj, m, out, S)
        torch.cuda.synchronize()
        assert (host(out) == img).all(), (name, m)
