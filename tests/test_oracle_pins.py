"""Pins of the CPU oracle to things other than itself.

Every check here compares the oracle with a fact the paper or the mathematics
fixes: hand-worked fixtures, closed forms, invariants, symmetries, and an
independent solver (Gaussian elimination over GF(2)) on tiny images.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_1504_07038_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _split(proj_row, p, P, Q):
    off, bins, _, _ = oracle.offsets(p, P, Q)
    return [proj_row[o:o + b] for o, b in zip(off, bins)]


# ---------------------------------------------------------------- fixtures --

@pytest.mark.parametrize("name", ["fig1_directions_3x3.json", "empty_bins_2x2.json"])
def test_hand_worked_fixture(name):
    g = _load(name)
    P, Q, p = g["P"], g["Q"], g["directions"]
    img = np.array(g["image_rows"], dtype=np.uint64)[None]
    assert [oracle.bin_count(pi, P, Q) for pi in p] == g["bin_counts_eq2"]
    got = _split(oracle.encode(img, p)[0], p, P, Q)
    for pi, proj in zip(p, got):
        assert proj.tolist() == g["projections"][str(pi)]["bins_b_ascending"], pi


def test_fig1_any_three_of_four_reconstruct():
    """Sec. 2.2: each subset of 3 of the 4 projections of Fig. 1 suffices."""
    g = _load("fig1_directions_3x3.json")
    P, Q, p = g["P"], g["Q"], g["directions"]
    img = np.array(g["image_rows"], dtype=np.uint64)[None]
    proj = oracle.encode(img, p)
    for lost in range(4):
        assert oracle.katz(p, P, Q, 1 << lost)
        assert (oracle.decode(proj, p, P, Q, 1 << lost) == img).all()


# ------------------------------------------------------------ closed forms --

@pytest.mark.parametrize("P", range(1, 10))
@pytest.mark.parametrize("Q", range(1, 6))
def test_eq2_bin_count_matches_lattice(P, Q):
    """Eq. 2 is the span of b = l p - x over the lattice; when |p| <= P every
    position in that span is reached (no empty bins)."""
    for p in range(-7, 8):
        bs = {l * p - x for l in range(Q) for x in range(P)}
        B = oracle.bin_count(p, P, Q)
        assert B == max(bs) - min(bs) + 1
        assert B == abs(p) * (Q - 1) + P
        if abs(p) <= P:
            assert B == len(bs)
        # storage origin: closed form -(P-1) + min(0, (Q-1) p)
        assert oracle.bin_min(p, P, Q) == -(P - 1) + min(0, (Q - 1) * p)


def test_config_bin_sizes():
    """Bins per stripe at the benchmark geometries (Eq. 2 by hand)."""
    cases = [
        (128, 4, [-3, -2, -1, 1, 2, 3], 804),
        (256, 4, [-3, -2, -1, 1, 2, 3], 1572),
        (64, 8, [p for p in range(-6, 7) if p], 1062),
        (128, 8, [p for p in range(-6, 7) if p], 1830),
        (256, 2, [-1, 1, 2], 772),
        (512, 2, [-1, 1, 2], 1540),
    ]
    for P, Q, p, total in cases:
        assert oracle.total_bins(p, P, Q) == total


# -------------------------------------------------------------- invariants --

def _rand_img(S, Q, P, seed=7):
    return inputs.stripes(S, Q, P, seed=seed)


@pytest.mark.parametrize("P,Q", [(1, 1), (5, 1), (1, 4), (7, 3), (16, 4), (9, 8)])
def test_impulse_response(P, Q):
    """A single set pixel (l, x) lands in exactly one bin per projection, at
    b = l p - x (Eq. 1)."""
    p = [-4, -1, 0, 2, 5]
    off, bins, _, total = oracle.offsets(p, P, Q)
    for l in range(Q):
        for x in range(P):
            img = np.zeros((1, Q, P), dtype=np.uint64)
            img[0, l, x] = np.uint64(0xA5A5_0000_0000_0001)
            pr = oracle.encode(img, p)[0]
            expect = np.zeros(total, dtype=np.uint64)
            for i, pi in enumerate(p):
                bmin = -(P - 1) + min(0, (Q - 1) * pi)
                expect[off[i] + (l * pi - x - bmin)] = img[0, l, x]
            assert (pr == expect).all()


def test_xor_of_bins_equals_xor_of_pixels():
    """Each pixel lies on exactly one line of each direction (Eq. 1), so the
    XOR of a projection's bins is the XOR of the whole image."""
    for P, Q, p in [(128, 4, [-3, -2, -1, 1, 2, 3]), (64, 8, list(range(-6, 0)) + list(range(1, 7))),
                    (13, 5, [0, 7, -9, 20])]:
        img = _rand_img(6, Q, P)
        for s, row in enumerate(oracle.encode(img, p)):
            want = np.bitwise_xor.reduce(img[s].ravel())
            for proj in _split(row, p, P, Q):
                assert np.bitwise_xor.reduce(proj) == want


def test_border_bins_are_pixel_copies():
    """Sec. 2.1: the border bins hold single pixels; for p > 0 the first is
    f(P-1, 0) and the last f(0, Q-1), mirrored for p < 0."""
    P, Q = 32, 5
    p = [-5, -2, -1, 1, 3, 4]
    img = _rand_img(3, Q, P)
    for s, row in enumerate(oracle.encode(img, p)):
        for pi, proj in zip(p, _split(row, p, P, Q)):
            if pi > 0:
                assert proj[0] == img[s, 0, P - 1] and proj[-1] == img[s, Q - 1, 0]
            else:
                assert proj[0] == img[s, Q - 1, P - 1] and proj[-1] == img[s, 0, 0]


def test_at_most_Q_pixels_per_bin():
    """Sec. 3: encoding needs at most k-1 XORs per bin (k = Q lines)."""
    for P, Q in [(128, 4), (64, 8)]:
        for p in range(-6, 7):
            counts = {}
            for l in range(Q):
                for x in range(P):
                    counts[l * p - x] = counts.get(l * p - x, 0) + 1
            assert max(counts.values()) <= Q
            # edges hold one pixel each when p != 0
            if p:
                assert counts[min(counts)] == 1 and counts[max(counts)] == 1


def test_linearity_over_gf2():
    P, Q, p = 40, 4, [-3, -2, -1, 1, 2, 3]
    a, b = _rand_img(2, Q, P, 1), _rand_img(2, Q, P, 2)
    assert (oracle.encode(a ^ b, p) == (oracle.encode(a, p) ^ oracle.encode(b, p))).all()


def test_mirror_symmetries():
    """Reversing the columns maps direction p to -p with the bins reversed;
    reversing the rows maps p to -p with the bins unchanged (Eq. 1 under
    x -> P-1-x and l -> Q-1-l)."""
    P, Q = 23, 5
    p = [-4, -3, -1, 0, 2, 5]
    neg = [-v for v in p]
    img = _rand_img(4, Q, P)
    pr = oracle.encode(img, p)
    pr_cols = oracle.encode(img[:, :, ::-1].copy(), neg)
    pr_rows = oracle.encode(img[:, ::-1, :].copy(), neg)
    for s in range(4):
        a = _split(pr[s], p, P, Q)
        c = _split(pr_cols[s], neg, P, Q)
        r = _split(pr_rows[s], neg, P, Q)
        for i in range(len(p)):
            assert (c[i] == a[i][::-1]).all()
            assert (r[i] == a[i]).all()


# ------------------------------------------------- GF(2) brute-force decode --

def _incidence(P, Q, p, survivors):
    """Rows: surviving bins; columns: pixels l*P + x (Eq. 1 as a 0/1 matrix)."""
    rows = []
    for i in survivors:
        B = abs(p[i]) * (Q - 1) + P
        bmin = -(P - 1) + min(0, (Q - 1) * p[i])
        M = np.zeros((B, P * Q), dtype=np.uint8)
        for l in range(Q):
            for x in range(P):
                M[l * p[i] - x - bmin, l * P + x] = 1
        rows.append(M)
    return np.concatenate(rows, axis=0)


def _gf2_solve(A, rhs):
    """Gaussian elimination over GF(2) with uint64 right-hand sides (64
    independent bit-planes at once). Returns (rank, solution or None)."""
    A = A.copy().astype(np.uint8)
    rhs = rhs.copy()
    nr, nc = A.shape
    r = 0
    pivots = []
    for c in range(nc):
        piv = None
        for k in range(r, nr):
            if A[k, c]:
                piv = k
                break
        if piv is None:
            continue
        if piv != r:
            A[[r, piv]] = A[[piv, r]]
            rhs[[r, piv]] = rhs[[piv, r]]
        for k in range(nr):
            if k != r and A[k, c]:
                A[k] ^= A[r]
                rhs[k] ^= rhs[r]
        pivots.append(c)
        r += 1
    if r < nc:
        return r, None
    x = np.zeros(nc, dtype=np.uint64)
    for k, c in enumerate(pivots):
        x[c] = rhs[k]
    return r, x


def _tiny_cases():
    rng = np.random.default_rng(1504)
    cases = []
    for P in range(1, 7):
        for Q in range(1, 5):
            for _ in range(3):
                n = int(rng.integers(Q, Q + 3))
                p = sorted(rng.choice(np.arange(-4, 5), size=min(n, 9), replace=False).tolist())
                cases.append((P, Q, p))
    return cases


@pytest.mark.parametrize("P,Q,p", _tiny_cases())
def test_decode_against_gf2_elimination(P, Q, p):
    """On tiny images, for every erasure mask: Eq. 3 true => the GF(2) system
    has full column rank (the image is unique, c11) and the oracle's peeling
    returns exactly the eliminated solution, which is the image; Eq. 3 false
    => the system is rank deficient and the oracle refuses."""
    n = len(p)
    img = _rand_img(1, Q, P, seed=P * 100 + Q)
    proj = oracle.encode(img, p)[0]
    off, bins, _, _ = oracle.offsets(p, P, Q)
    for mask in range(1 << n):
        surv = [i for i in range(n) if not mask >> i & 1]
        if not surv:
            continue
        A = _incidence(P, Q, p, surv)
        rhs = np.concatenate([proj[off[i]:off[i] + bins[i]] for i in surv])
        rank, sol = _gf2_solve(A, rhs)
        if oracle.katz(p, P, Q, mask):
            assert rank == P * Q, (mask, surv)
            assert (sol == img[0].ravel()).all()
            got = oracle.decode(proj[None], p, P, Q, mask)
            assert (got[0] == img[0]).all(), (mask, surv)
        else:
            assert rank < P * Q, (mask, surv)   # Eq. 3 is exact here: ghosts exist
            with pytest.raises(oracle.OracleError):
                oracle.decode(proj[None], p, P, Q, mask)


def test_katz_false_below_q_means_ghosts():
    """Fewer than Q projections with sum |p| < P: the GF(2) system is rank
    deficient, so a ghost (a nonzero image with all-zero projections) exists
    and refusing to decode is the only correct answer."""
    for P, Q, p in [(8, 4, [-2, 1, 3]), (10, 3, [1, -2]), (6, 2, [3])]:
        assert sum(abs(v) for v in p) < P and len(p) < Q
        rank, _ = _gf2_solve(_incidence(P, Q, p, list(range(len(p)))),
                             np.zeros(sum(abs(v) * (Q - 1) + P for v in p), dtype=np.uint64))
        assert rank < P * Q


# ------------------------------------------------- round trips at configs --

CONFIGS = [
    (128, 4, [-3, -2, -1, 1, 2, 3]),
    (256, 4, [-3, -2, -1, 1, 2, 3]),
    (64, 8, [v for v in range(-6, 7) if v]),
    (128, 8, [v for v in range(-6, 7) if v]),
    (256, 2, [-1, 1, 2]),
]


@pytest.mark.parametrize("P,Q,p", CONFIGS)
def test_round_trip_every_k_of_n_mask(P, Q, p):
    """Sec. 2.3: any Q of the n projections rebuild the image; also with
    fewer erasures (redundant projections take part in the peeling)."""
    n = len(p)
    img = _rand_img(2, Q, P, seed=P + Q)
    proj = oracle.encode(img, p)
    masks = []
    for e in range(0, n - Q + 1):
        ms = inputs.all_masks(n, e)
        if len(ms) > 60:                # (12,8): sample the C(12,e) patterns
            ms = ms[:: len(ms) // 60]
        masks += ms
    for m in masks:
        assert (oracle.decode(proj, p, P, Q, m) == img).all(), m
    # one erasure too many and Sigma|p| < P: refused
    for m in inputs.all_masks(n, n - Q + 1)[:5]:
        assert not oracle.katz(p, P, Q, m)
        with pytest.raises(oracle.OracleError):
            oracle.decode(proj, p, P, Q, m)


def test_per_stripe_masks_and_threads():
    P, Q, p = 64, 4, [-3, -2, -1, 1, 2, 3]
    S = 37
    img = _rand_img(S, Q, P)
    proj = oracle.encode(img, p, threads=3)
    assert (proj == oracle.encode(img, p)).all()
    masks = inputs.erasure_masks(S, 6, 2)
    assert (oracle.decode(proj, p, P, Q, masks, threads=4) == img).all()


def test_bad_arguments():
    with pytest.raises(oracle.OracleError):
        oracle.total_bins([1, 1], 8, 2)          # duplicate direction
    with pytest.raises(oracle.OracleError):
        oracle.total_bins([], 8, 2)
    with pytest.raises(oracle.OracleError):
        oracle.total_bins(list(range(33)), 64, 2)  # more than 32 projections


# ------------------------------------------------------------- generator --

def test_splitmix64_published_sequence():
    """SplitMix64 seeded with 0 starts 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4,
    0x06c45d188009454f (Vigna's reference splitmix64.c)."""
    got = inputs.splitmix64(0, np.arange(3)).tolist()
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_generator_is_counter_based():
    a = inputs.stripes(10, 4, 16, seed=3)
    b = inputs.stripe_rows(np.array([7, 2]), 4, 16, seed=3)
    c = inputs.stripes(3, 4, 16, seed=3, first=5)
    assert (b[0] == a[7]).all() and (b[1] == a[2]).all() and (c == a[5:8]).all()


def test_erasure_masks():
    m = inputs.erasure_masks(5000, 12, 4)
    assert all(bin(int(v)).count("1") == 4 for v in m)
    assert len(set(m.tolist())) > 400          # most of the C(12,4) = 495 patterns
    assert (inputs.erasure_masks(100, 6, 2, first=50) == inputs.erasure_masks(150, 6, 2)[50:]).all()
    assert len(inputs.all_masks(6, 2)) == 15 and len(inputs.all_masks(12, 4)) == 495


# ------------------------------------------- systematic form (next to Sec. 2.3) --
# The paper mentions a systematic Mojette code (Sec. 2.3, Sec. 4) without
# defining it. Reading used here: the Q data lines are Q of the packets and
# the r parity packets are Eq. 1 projections of the whole image; mask bit
# l < Q marks data line l lost, bit Q + i parity projection i lost.

SYS_CONFIGS = [
    (128, 4, [-1, 1]),                 # 4 KB (6,4) systematic
    (256, 4, [-1, 1]),                 # 8 KB (6,4)
    (64, 8, [-2, -1, 1, 2]),           # 4 KB (12,8)
    (128, 8, [-2, -1, 1, 2]),          # 8 KB (12,8)
]


def _sys_masks(Q, r):
    """Every mask losing e data lines and f parity packets with e + f <= r."""
    out = []
    for m in range(1 << (Q + r)):
        if bin(m).count("1") <= r:
            out.append(m)
    return out


def _sys_incidence(P, Q, p, mask):
    """GF(2) system of a systematic stripe over all Q*P pixels: one identity
    row per pixel of a surviving data line (the packet is the line itself)
    and the incidence rows of every surviving parity projection (Eq. 1)."""
    r = len(p)
    rows = []
    for l in range(Q):
        if not mask >> l & 1:
            M = np.zeros((P, P * Q), dtype=np.uint8)
            M[np.arange(P), l * P + np.arange(P)] = 1
            rows.append(M)
    surv = [i for i in range(r) if not mask >> (Q + i) & 1]
    if surv:
        rows.append(_incidence(P, Q, p, surv))
    if not rows:
        return np.zeros((0, P * Q), dtype=np.uint8), surv
    return np.concatenate(rows, axis=0), surv


def _sys_tiny_cases():
    rng = np.random.default_rng(15040)
    cases = []
    for P in range(1, 7):
        for Q in range(1, 5):
            for _ in range(2):
                r = int(rng.integers(1, 4))
                p = sorted(rng.choice(np.arange(-4, 5), size=r, replace=False).tolist())
                cases.append((P, Q, p))
    return cases


@pytest.mark.parametrize("P,Q,p", _sys_tiny_cases())
def test_sys_decode_against_gf2_elimination(P, Q, p):
    """Tiny images, every mask: whenever at least as many parity projections
    survive as data lines are lost, the GF(2) system of the surviving
    packets has full rank (any e distinct directions (p, 1) recover any e
    lines: the e x e matrix [u^(p_i l_j)] is a generalised Vandermonde
    matrix whose top monomial, matching sorted p to sorted l, occurs once,
    so its determinant is nonzero) and the oracle returns the eliminated
    solution, which is the image; a rank-deficient system is refused; and
    an oracle success is always the unique solution."""
    r = len(p)
    img = _rand_img(1, Q, P, seed=P * 31 + Q)
    par = oracle.encode(img, p)[0]
    off, bins, _, _ = oracle.offsets(p, P, Q)
    data = img.copy()
    for mask in range(1 << (Q + r)):
        lost = [l for l in range(Q) if mask >> l & 1]
        A, surv = _sys_incidence(P, Q, p, mask)
        rhs = np.concatenate([img[0, l] for l in range(Q) if l not in lost]
                             + [par[off[i]:off[i] + bins[i]] for i in surv]) \
            if A.shape[0] else np.zeros(0, np.uint64)
        rank, sol = _gf2_solve(A, rhs) if A.shape[0] else (0, None)
        garbage = data.copy()
        garbage[0, lost] = np.uint64(0xDEADBEEF)         # lost lines are never read
        try:
            got = oracle.sys_decode(garbage, par[None], p, P, Q, mask)
        except oracle.OracleError:
            got = None
        if len(surv) >= len(lost):
            assert rank == P * Q, (mask, lost, surv)
            assert (sol == img[0].ravel()).all()
            assert got is not None and (got[0] == img[0]).all(), mask
        if rank < P * Q:
            assert got is None, mask
        if got is not None:
            assert rank == P * Q and (got[0] == img[0]).all(), mask


@pytest.mark.parametrize("P,Q,p", SYS_CONFIGS)
def test_sys_round_trip_every_mask(P, Q, p):
    """Any e <= r lost data lines come back from any e surviving parity
    projections, whatever else is lost; with no data line lost the decode is
    the copy Sec. 4 expects of a systematic code."""
    r = len(p)
    img = _rand_img(2, Q, P, seed=P + 3 * Q)
    par = oracle.encode(img, p)
    masks = _sys_masks(Q, r)
    if len(masks) > 120:                       # (12,8): a seeded sample
        masks = [masks[i] for i in np.random.default_rng(8).choice(len(masks), 120, replace=False)]
    for m in masks:
        data = img.copy()
        lost = [l for l in range(Q) if m >> l & 1]
        data[:, lost] = np.uint64(0x0123456789ABCDEF)
        assert (oracle.sys_decode(data, par, p, P, Q, m) == img).all(), m


def test_sys_single_lost_line_closed_form():
    """One lost line l0 under projection p: Eq. 1 read backwards, pixel
    (l0, x) = bin l0 p - x XOR the other lines' pixels (l, x + (l - l0) p)
    inside the image -- no peeling order involved."""
    P, Q, p = 40, 5, [-2, 3]
    img = _rand_img(1, Q, P, seed=11)[0]
    par = oracle.encode(img[None], p)[0]
    off, _, bmins, _ = oracle.offsets(p, P, Q)
    for l0 in range(Q):
        for i, pi in enumerate(p):
            mask = (1 << l0) | (1 << (Q + 1 - i))    # the other projection lost too
            expect = np.empty(P, np.uint64)
            for x in range(P):
                v = par[off[i] + l0 * pi - x - bmins[i]]
                for l in range(Q):
                    x2 = x + (l - l0) * pi
                    if l != l0 and 0 <= x2 < P:
                        v ^= img[l, x2]
                expect[x] = v
            got = oracle.sys_decode(img[None], par[None], p, P, Q, mask)[0]
            assert (got[l0] == expect).all() and (expect == img[l0]).all()


def test_sys_no_lost_line_is_a_copy():
    """No data line lost: the output is the data, whatever the parity holds
    (it is not read)."""
    P, Q, p = 64, 4, [-1, 1]
    img = _rand_img(3, Q, P, seed=5)
    junk = np.full((3, oracle.total_bins(p, P, Q)), 0xFFFF, dtype=np.uint64)
    for m in (0, 1 << Q, 3 << Q):
        assert (oracle.sys_decode(img, junk, p, P, Q, m) == img).all()


def test_sys_too_many_losses_refused():
    """More lost lines than surviving parity with sum |p| < P: the GF(2)
    system is rank deficient, so the oracle must refuse."""
    P, Q, p = 32, 4, [-1, 1]
    img = _rand_img(1, Q, P, seed=9)
    par = oracle.encode(img, p)
    for m in (0b0111, 0b0011 | 1 << Q, 0b1000 | 3 << Q):
        A, _ = _sys_incidence(P, Q, p, m)
        assert _gf2_solve(A, np.zeros(A.shape[0], np.uint64))[0] < P * Q
        with pytest.raises(oracle.OracleError):
            oracle.sys_decode(img, par, p, P, Q, m)
