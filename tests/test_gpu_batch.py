"""GPU parity of batched encode/decode (mojette_batch_*) against the oracle.

A batch mixes the six benchmark geometries -- 4 KB and 8 KB stripes at
(3,2), (6,4) and (12,8) -- in a seeded random order, each stripe with its own
seeded erasure pattern of 0..n-Q lost projections, with the slices of the
lost projections overwritten by junk before decoding. Every stripe's result
must equal the oracle's bit for bit, whatever the launch form (per-class
launches or one CUDA graph), after autotuning, after the stripe set changes,
and when encodes and decodes share a batch. Integer XOR work: tolerance zero.
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

SIX = [-3, -2, -1, 1, 2, 3]
TWELVE = [v for v in range(-6, 7) if v]
GEOMS = [  # (P, Q, p): 4 KB and 8 KB stripes of the three codes
    (256, 2, [-1, 1, 2]), (512, 2, [-1, 1, 2]),
    (128, 4, SIX), (256, 4, SIX),
    (64, 8, TWELVE), (128, 8, TWELVE),
]
JUNK = np.uint64(0xDEADBEEFCAFEF00D)


@pytest.fixture(autouse=True)
def clean_status():
    mj.mojette_device_status(clear=True)
    yield
    assert mj.mojette_device_status(clear=True) == 0


class Mixed:
    """Seeded stripes of every geometry, their buffers on the device, and
    the oracle's projections and decodes."""

    def __init__(self, counts, seed, oracle_decode=True):
        self.plans = [mj.mojette_plan(P, Q, p) for P, Q, p in GEOMS]
        self.counts = counts
        self.img, self.proj, self.masks = [], [], []
        self.d_img, self.d_proj, self.d_out = [], [], []
        self.ref_proj, self.ref_dec = [], []
        for k, ((P, Q, p), S) in enumerate(zip(GEOMS, counts)):
            img = inputs.stripes(S, Q, P, seed=seed + 101 * k)
            n = len(p)
            e = inputs.erasure_counts(S, n - Q, seed=seed + 7 * k)
            masks = inputs.erasure_masks(S, n, e, seed=seed + 13 * k)
            ref = oracle.encode(img, p, threads=8)
            self.img.append(img)
            self.masks.append(masks)
            self.ref_proj.append(ref)
            self.ref_dec.append(oracle.decode(ref, p, P, Q, masks, threads=8) if oracle_decode else img)
            self.d_img.append(torch.from_numpy(img.view(np.int64)).cuda())
            self.d_proj.append(torch.zeros((S, self.plans[k].total), dtype=torch.int64, device="cuda"))
            self.d_out.append(torch.full((S, Q, P), 0x5A5A, dtype=torch.int64, device="cuda"))

    def corrupt_erased(self):
        """Device projections = the oracle's, with every lost slice junk."""
        for k, ((P, Q, p), S) in enumerate(zip(GEOMS, self.counts)):
            pr = self.ref_proj[k].copy()
            offs, bins, _, _ = oracle.offsets(p, P, Q)
            for i, (off, B) in enumerate(zip(offs, bins)):
                lost = (self.masks[k] >> i) & 1 == 1
                pr[lost, off:off + B] = JUNK
            self.d_proj[k].copy_(torch.from_numpy(pr.view(np.int64)))

    def table(self, op, order_seed, select=None):
        """A stripe table over every stripe (or the (k, s) pairs in select), shuffled."""
        rows = []
        for k, S in enumerate(self.counts):
            for s in range(S):
                if select is None or (k, s) in select:
                    rows.append((k, s))
        rng = np.random.default_rng(order_seed)
        rows = [rows[i] for i in rng.permutation(len(rows))]
        ks = np.array([r[0] for r in rows], dtype=np.int64)
        ss = np.array([r[1] for r in rows], dtype=np.int64)
        src = np.zeros(len(rows), dtype=np.uint64)
        dst = np.zeros(len(rows), dtype=np.uint64)
        mask = np.zeros(len(rows), dtype=np.uint32)
        for k in range(len(self.counts)):
            sel = ks == k
            P, Q, _ = GEOMS[k]
            tot = self.plans[k].total
            if op == mj.MOJETTE_OP_ENCODE:
                src[sel] = self.d_img[k].data_ptr() + ss[sel] * (Q * P * 8)
                dst[sel] = self.d_proj[k].data_ptr() + ss[sel] * (tot * 8)
            else:
                src[sel] = self.d_proj[k].data_ptr() + ss[sel] * (tot * 8)
                dst[sel] = self.d_out[k].data_ptr() + ss[sel] * (Q * P * 8)
                mask[sel] = self.masks[k][ss[sel]]
        return mj.stripe_table(self.plans, ks, op, mask, src, dst)

    def check_proj(self):
        torch.cuda.synchronize()
        for k in range(len(self.counts)):
            got = self.d_proj[k].cpu().numpy().view(np.uint64)
            assert np.array_equal(got, self.ref_proj[k]), f"encode mismatch in geometry {GEOMS[k][:2]}"

    def check_out(self):
        torch.cuda.synchronize()
        for k in range(len(self.counts)):
            got = self.d_out[k].cpu().numpy().view(np.uint64)
            assert np.array_equal(got, self.ref_dec[k]), f"decode mismatch in geometry {GEOMS[k][:2]}"
            assert np.array_equal(got, self.img[k])


COUNTS = [37, 20, 301, 64, 517, 90]   # ragged: partial work items and tiles


@pytest.mark.parametrize("flags", [0, 1])
def test_batch_matches_oracle(flags):
    m = Mixed(COUNTS, seed=11)
    enc = mj.mojette_batch_create(m.table(mj.MOJETTE_OP_ENCODE, 1), m.plans, flags)
    mj.mojette_batch_run(enc)
    m.check_proj()
    m.corrupt_erased()
    dec = mj.mojette_batch_create(m.table(mj.MOJETTE_OP_DECODE, 2), m.plans, flags)
    info = mj.mojette_batch_info(dec)
    assert info["launches"] == len(GEOMS)
    assert info["groups"] == len({(k, int(x)) for k in range(len(GEOMS)) for x in m.masks[k]})
    mj.mojette_batch_run(dec)
    m.check_out()
    # a second run (graph replay) gives the same
    m.d_out[0].fill_(0)
    mj.mojette_batch_run(dec)
    m.check_out()


def test_batch_tune_keeps_results():
    m = Mixed([64, 16, 200, 40, 300, 50], seed=23)
    m.corrupt_erased()
    dec = mj.mojette_batch_create(m.table(mj.MOJETTE_OP_DECODE, 3), m.plans, mj.MOJETTE_BATCH_GRAPH)
    mj.mojette_batch_tune(dec, reps=1)
    info = mj.mojette_batch_info(dec)
    for c in info["configs"]:
        assert c["op"] == mj.MOJETTE_OP_DECODE and c["kernel"] in (0, 1, 2, 3, 4, 5, 6) and c["param"] >= 1
    for t in m.d_out:
        t.fill_(0)
    mj.mojette_batch_run(dec)
    m.check_out()
    enc = mj.mojette_batch_create(m.table(mj.MOJETTE_OP_ENCODE, 4), m.plans)
    mj.mojette_batch_tune(enc, reps=1)
    for t in m.d_proj:
        t.zero_()
    mj.mojette_batch_run(enc)
    m.check_proj()


def test_every_tuner_candidate_is_exact(monkeypatch):
    """Each decode configuration the tuner may pick gives the oracle's bytes:
    run plain decodes under every layout the environment can force."""
    P, Q, p = 128, 8, TWELVE
    plan = mj.mojette_plan(P, Q, p)
    img = inputs.stripes(133, Q, P, seed=5)
    proj = oracle.encode(img, p, threads=8)
    d_proj = torch.from_numpy(proj.view(np.int64)).cuda()
    mask = 0b000011000011
    cases = [(k, g, r) for k in ("lines", "ilv", "fronts", "stream", "cols", "vander") for g in ("1", "3", "8")
             for r in ("0", "1")]
    for kernel, gpc, rowoff in cases:
        monkeypatch.setenv("MOJETTE_DECODE_KERNEL", kernel)
        monkeypatch.setenv("MOJETTE_DECODE_GPC", gpc)
        monkeypatch.setenv("MOJETTE_DECODE_ROWOFF", rowoff)
        out = torch.zeros((133, Q, P), dtype=torch.int64, device="cuda")
        mj.mojette_decode(plan, d_proj, mask, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint64), img), (kernel, gpc, rowoff)


@pytest.mark.parametrize("kernel", [6, 0])
def test_batch_with_installed_kernel(kernel):
    """A decode configuration installed in every plan (mojette_plan_config)
    is the one each class launches -- decode_ilv (stripes across lanes) or
    decode_lines -- over the mixed geometries and per-stripe masks, and every
    stripe equals the oracle's decode."""
    m = Mixed(COUNTS, seed=19)
    for pl in m.plans:
        mj.mojette_plan_config(pl, {"decode_tuned": 1, "decode_kernel": kernel, "decode_gpc": 2,
                                    "decode_persist": 0, "decode_rowoff": 1})
    m.corrupt_erased()
    dec = mj.mojette_batch_create(m.table(mj.MOJETTE_OP_DECODE, 4), m.plans, mj.MOJETTE_BATCH_GRAPH)
    assert all(c["kernel"] == kernel for c in mj.mojette_batch_info(dec)["configs"])
    mj.mojette_batch_run(dec)
    m.check_out()


def test_batch_update_and_mixed_ops():
    m = Mixed([40, 30, 120, 60, 150, 45], seed=31)
    enc_sel = {(k, s) for k, S in enumerate(m.counts) for s in range(S) if s % 2 == 0}
    # decode stripes need their projections first
    for k in range(len(GEOMS)):
        m.d_proj[k].copy_(torch.from_numpy(m.ref_proj[k].view(np.int64)))
    m.corrupt_erased()
    dec_sel = {(k, s) for k, S in enumerate(m.counts) for s in range(S) if s % 2 == 1}
    t_enc = m.table(mj.MOJETTE_OP_ENCODE, 5, enc_sel)
    t_dec = m.table(mj.MOJETTE_OP_DECODE, 6, dec_sel)
    both = np.concatenate([t_enc, t_dec])[np.random.default_rng(7).permutation(len(t_enc) + len(t_dec))]
    b = mj.mojette_batch_create(both[:10], m.plans, mj.MOJETTE_BATCH_GRAPH)   # small first
    mj.mojette_batch_update(b, both)                                           # grows: realloc
    mj.mojette_batch_run(b)
    torch.cuda.synchronize()
    for k in range(len(GEOMS)):
        got_p = m.d_proj[k].cpu().numpy().view(np.uint64)
        got_o = m.d_out[k].cpu().numpy().view(np.uint64)
        for s in range(m.counts[k]):
            if s % 2 == 0:
                assert np.array_equal(got_p[s], m.ref_proj[k][s])
            else:
                assert np.array_equal(got_o[s], m.img[k][s])
    # shrink: the same batch, a third of the decode stripes only
    for t in m.d_out:
        t.zero_()
    mj.mojette_batch_update(b, t_dec[: len(t_dec) // 3])
    mj.mojette_batch_run(b)
    torch.cuda.synchronize()
    done = {(int(r["dst"]),) for r in t_dec[: len(t_dec) // 3]}
    for k in range(len(GEOMS)):
        P, Q, _ = GEOMS[k]
        got_o = m.d_out[k].cpu().numpy().view(np.uint64)
        base = m.d_out[k].data_ptr()
        for s in range(m.counts[k]):
            if (base + s * Q * P * 8,) in done:
                assert np.array_equal(got_o[s], m.img[k][s])
            else:
                assert not got_o[s].any()


def test_batch_errors():
    m = Mixed([4, 2, 4, 2, 4, 2], seed=41, oracle_decode=False)
    t = m.table(mj.MOJETTE_OP_DECODE, 8)
    k0 = int(np.nonzero(t["plan"] == m.plans[0].handle)[0][0])   # a (3,2) stripe
    bad = t.copy()
    bad["src"][0] += 4
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_batch_create(bad, m.plans)
    assert ei.value.code == -errno.ERANGE
    te = m.table(mj.MOJETTE_OP_ENCODE, 8)
    bad = te.copy()
    bad["src"][0] += 8       # P even: encode rows arrive by 16-byte bulk copies
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_batch_create(bad, m.plans)
    assert ei.value.code == -errno.ERANGE
    bad = t.copy()
    bad["erasure_mask"][k0] = 0b011   # two of three lost: one survivor, Q = 2
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_batch_create(bad, m.plans)
    assert ei.value.code == -errno.ENOTRECOVERABLE
    bad = t.copy()
    bad["op"][0] = 7
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_batch_create(bad, m.plans)
    assert ei.value.code == -errno.EINVAL
    bad = t.copy()
    bad["erasure_mask"][k0] = 1 << 5   # beyond n = 3
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_batch_create(bad, m.plans)
    assert ei.value.code == -errno.EINVAL
    empty = mj.mojette_batch_create(t[:0], m.plans, mj.MOJETTE_BATCH_GRAPH)
    mj.mojette_batch_run(empty)
    assert mj.mojette_batch_info(empty)["launches"] == 0


def test_batch_full_size_sampled():
    """500k mixed stripes in one decode batch (the batched workload's size):
    sampled stripes against the oracle, every stripe against its image."""
    S_total = 500_000
    rng = np.random.default_rng(1504)
    counts = np.bincount(rng.integers(0, len(GEOMS), S_total), minlength=len(GEOMS)).tolist()
    m = Mixed(counts, seed=77, oracle_decode=False)
    for k in range(len(GEOMS)):
        m.d_proj[k].copy_(torch.from_numpy(m.ref_proj[k].view(np.int64)))
    m.corrupt_erased()
    dec = mj.mojette_batch_create(m.table(mj.MOJETTE_OP_DECODE, 9), m.plans, mj.MOJETTE_BATCH_GRAPH)
    mj.mojette_batch_run(dec)
    torch.cuda.synchronize()
    for k, (P, Q, p) in enumerate(GEOMS):
        got = m.d_out[k].cpu().numpy().view(np.uint64)
        assert np.array_equal(got, m.img[k])
        idx = np.unique(rng.integers(0, counts[k], 64))
        ref = oracle.decode(m.ref_proj[k][idx], p, P, Q, m.masks[k][idx], threads=8)
        assert np.array_equal(got[idx], ref)


@pytest.mark.parametrize("P,Q,p", [(64, 8, TWELVE), (128, 8, TWELVE), (96, 6, [-4, -3, -2, -1, 1, 2, 3, 4])])
def test_batch_decode_stripes_at_odd_word_offsets(P, Q, p):
    """Decode stripes whose projection blocks and images start 8 bytes off a
    16-byte boundary (the batch API asks for 8-byte alignment only): every
    run of bins then disagrees mod 16 bytes with its place in shared memory
    in half the stripes, so decode_lines stages those runs with the warp's
    8-byte copies instead of bulk copies. Each stripe sits at its own odd or
    even word offset; results equal the oracle's."""
    S = 4500
    n = len(p)
    plan = mj.mojette_plan(P, Q, p)
    img = inputs.stripes(S, Q, P, seed=P * 7 + Q)
    ref = oracle.encode(img, p, threads=8)
    masks = inputs.erasure_masks(S, n, np.full(S, n - Q), seed=P + Q)
    masks[:4200] = masks[0]   # a group of 4200 stripes: its path's bank layout is searched
    tot = plan.total
    # stripe s at word s * (tot + 1) + 1 of its buffer: parities alternate
    # with s when tot is even, and the first stripe is 8 bytes off
    pw = tot + 1
    pr = ref.copy()
    offs, bins, _, _ = oracle.offsets(p, P, Q)
    for i, (off, B) in enumerate(zip(offs, bins)):
        pr[(masks >> i) & 1 == 1, off:off + B] = JUNK   # lost slices: junk
    flat = np.full(S * pw + 2, JUNK, dtype=np.uint64)
    for s in range(S):
        flat[s * pw + 1:s * pw + 1 + tot] = pr[s]
    d_src = torch.from_numpy(flat.view(np.int64)).cuda()
    iw = Q * P + 1
    d_out = torch.full((S * iw + 2,), 0x5A5A, dtype=torch.int64, device="cuda")
    st = np.arange(S, dtype=np.uint64)
    src = np.uint64(d_src.data_ptr()) + (st * np.uint64(pw) + np.uint64(1)) * np.uint64(8)
    dst = np.uint64(d_out.data_ptr()) + (st * np.uint64(iw) + np.uint64(1)) * np.uint64(8)
    table = mj.stripe_table([plan], np.zeros(S, dtype=np.int64), mj.MOJETTE_OP_DECODE, masks, src, dst)
    batch = mj.mojette_batch_create(table, [plan])
    assert mj.mojette_batch_info(batch)["launches"] >= 1
    mj.mojette_batch_run(batch)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy().view(np.uint64)
    out = np.stack([got[s * iw + 1:s * iw + 1 + Q * P] for s in range(S)]).reshape(S, Q, P)
    assert np.array_equal(out, img)
    idx = np.arange(0, S, 97)
    assert np.array_equal(out[idx], oracle.decode(ref[idx], p, P, Q, masks[idx], threads=8))
    # the words between stripes are untouched
    gaps = got[np.arange(S) * iw]
    assert (gaps == np.uint64(0x5A5A)).all()
    mj.mojette_batch_destroy(batch)
