"""mojette_decode_noalloc against mojette_decode.

The no-allocation entry point serves callers that cannot call cudaMalloc --
for instance a storage server whose device memory all belongs to its own
buffer pool, or a request path that must not take cudaMalloc's device-wide
synchronisation. It keeps the reconstruction path in a fixed scratch array
inside the library. Calls in a row, on different geometries and erasure
masks whose paths all run through that scratch (each overwrites what the
previous one left there), must each give exactly what mojette_decode gives
on the same inputs; and a call allocates nothing on the device, even for a
mask it has not seen before.
"""
import errno

import numpy as np
import pytest

from paper_1504_07038_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIX = [-3, -2, -1, 1, 2, 3]
TWELVE = [v for v in range(-6, 7) if v]


def _case(mj, P, Q, p, S, mask, seed):
    plan = mj.mojette_plan(P, Q, p)
    img = torch.from_numpy(inputs.stripes(S, Q, P, seed=seed).view(np.int64)).cuda()
    proj = torch.empty((S, plan.total), dtype=torch.int64, device="cuda")
    mj.mojette_encode(plan, img, proj, S)
    want = torch.full((S, Q, P), 7, dtype=torch.int64, device="cuda")
    got = torch.full((S, Q, P), 9, dtype=torch.int64, device="cuda")
    mj.mojette_decode(plan, proj, mask, want, S)
    return plan, img, proj, want, got


def test_noalloc_decode_matches_decode_on_two_calls_in_a_row():
    from paper_1504_07038_gb300 import binding as mj

    a = _case(mj, 256, 4, SIX, 1001, 0b100100, seed=21)
    b = _case(mj, 128, 8, TWELVE, 777, 0b010100100001, seed=22)
    # both decodes follow a reconstruction path, read from the shared scratch
    assert mj.mojette_decode_kernel(a[0], 0b100100, 1001) == "decode_lines"
    assert mj.mojette_decode_kernel(b[0], 0b010100100001, 777) == "decode_lines"
    assert mj.mojette_schedule(a[0], 0b100100)["T"] != mj.mojette_schedule(b[0], 0b010100100001)["T"]
    mj.mojette_decode_noalloc(a[0], a[2], 0b100100, a[4], 1001)
    mj.mojette_decode_noalloc(b[0], b[2], 0b010100100001, b[4], 777)
    torch.cuda.synchronize()
    assert mj.mojette_device_status() == 0
    for plan, img, proj, want, got in (a, b):
        # bit-exact, the tolerance of every integer test here
        assert bool((got == want).all())
        assert bool((got == img).all())
    # the first path again, after the second overwrote the scratch
    a[4].fill_(3)
    mj.mojette_decode_noalloc(a[0], a[2], 0b100100, a[4], 1001)
    torch.cuda.synchronize()
    assert bool((a[4] == a[3]).all())


def test_noalloc_decode_allocates_no_device_memory():
    from paper_1504_07038_gb300 import binding as mj

    plan, img, proj, want, got = _case(mj, 128, 8, TWELVE, 513, 0b000011110000, seed=23)
    mj.mojette_decode_noalloc(plan, proj, 0b000011110000, got, 513)   # set-up on this device
    torch.cuda.synchronize()
    fresh = 0b110000000011                                            # a mask not decoded before
    free0 = torch.cuda.mem_get_info()[0]
    mj.mojette_decode_noalloc(plan, proj, fresh, got, 513)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    mj.mojette_decode(plan, proj, fresh, want, 513)
    torch.cuda.synchronize()
    assert bool((got == want).all()) and bool((got == img).all())


def test_noalloc_decode_refuses_an_oversized_schedule():
    from paper_1504_07038_gb300 import binding as mj

    # P = 40000 pixels per line gives about 20000 steps, over the scratch's 16384
    plan = mj.mojette_plan(40000, 2, [-1, 1, 2])
    buf = torch.empty((1, plan.total), dtype=torch.int64, device="cuda")
    out = torch.empty((1, 2, 40000), dtype=torch.int64, device="cuda")
    with pytest.raises(mj.MojetteError) as e:
        mj.mojette_decode_noalloc(plan, buf, 0b001, out, 1)
    assert e.value.code == -errno.ENOSPC
