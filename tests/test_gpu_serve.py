"""GPU tests of the request server (mojette_server_*): continuous batching of
object writes and reads under a device-memory budget.

Every write's projections must equal the oracle's, every read must return
the object; each request's output must be the same when it is served alone
as when it is served in the mix (tolerance zero: integer XOR work); the pool
never exceeds the budget; a budget that holds one request at a time still
drains the queue.
"""
import errno

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1504_07038_gb300 import binding as mj
    from paper_1504_07038_gb300 import serving


@pytest.fixture(autouse=True)
def clean_status():
    mj.mojette_device_status(clear=True)
    yield
    assert mj.mojette_device_status(clear=True) == 0


@pytest.fixture(scope="module")
def wl():
    return serving.Workload(240, seed=4242, max_bytes=256 << 10)


def check_outputs(wl, ids):
    for r in ids:
        P, Q, p = wl.geoms[wl.geom[r]]
        got = wl.output(r)
        if wl.write[r]:
            ref = oracle.encode(wl.images[r], p, threads=4).reshape(-1)
        else:
            ref = wl.images[r].reshape(-1)
        assert np.array_equal(got, ref), f"request {r} ({'write' if wl.write[r] else 'read'})"


def test_mix_matches_oracle_and_alone(wl):
    budget = 8 << 20                      # far below the workload's total: admission waits
    srv = mj.mojette_server_create(budget, slots=3, max_wave_stripes=512)
    wl.clear_outputs()
    comp, _ = serving.run_server(srv, wl, rate=None)
    assert sorted(comp["id"].tolist()) == list(range(len(wl)))
    st = mj.mojette_server_stats(srv)
    assert st["queued"] == 0 and st["in_flight"] == 0 and st["completed"] == len(wl)
    assert 0 < st["pool_peak"] <= budget and st["pool_used"] == 0
    assert st["waves"] > 3
    assert (comp["admit_s"] >= comp["arrival_s"]).all() and (comp["done_s"] >= comp["admit_s"]).all()
    check_outputs(wl, range(len(wl)))
    mixed = [wl.output(r).copy() for r in range(len(wl))]

    # the same requests, each alone on an idle server
    rng = np.random.default_rng(3)
    alone = mj.mojette_server_create(budget, slots=1, max_wave_stripes=512)
    for r in rng.choice(len(wl), 24, replace=False):
        wl.clear_outputs()
        serving.run_server(alone, wl, rate=None, order=[r])
        assert np.array_equal(wl.output(r), mixed[r]), f"request {r} differs alone vs in the mix"


def test_poisson_arrivals(wl):
    srv = mj.mojette_server_create(64 << 20, slots=4, max_wave_stripes=4096)
    wl.clear_outputs()
    comp, elapsed = serving.run_server(srv, wl, rate=4000.0, seed=9)
    assert len(comp) == len(wl) and elapsed > 0
    lat = serving.latency_stats(comp)
    assert 0 < lat["p50_ms"] <= lat["p99_ms"]
    check_outputs(wl, range(0, len(wl), 3))


def test_one_request_at_a_time_budget(wl):
    # room for the largest request only: waves of one request, still drains
    # each half of the pool holds the largest input / output
    need = 2 * int(max(max((wl.in_bytes + 15) // 16), max((wl.out_bytes + 15) // 16)) * 16)
    srv = mj.mojette_server_create(need, slots=2, max_wave_stripes=1 << 20)
    wl.clear_outputs()
    order = np.arange(0, len(wl), 4)
    comp, _ = serving.run_server(srv, wl, rate=None, order=order)
    assert len(comp) == len(order)
    check_outputs(wl, order)
    assert mj.mojette_server_stats(srv)["pool_peak"] <= need


def test_refusals(wl):
    srv = mj.mojette_server_create(1 << 20, slots=1, max_wave_stripes=8)
    big = int(np.argmax(wl.stripes))
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_server_submit(srv, wl.req[big:big + 1])
    assert ei.value.code == -errno.ENOSPC
    r = int(np.nonzero(~wl.write & (wl.stripes <= 8))[0][0])
    bad = wl.req[r:r + 1].copy()
    bad["erasure_mask"] = 0b111111 if wl.geom[r] < 2 else 0b11111         # too many lost
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_server_submit(srv, bad)
    assert ei.value.code == -errno.ENOTRECOVERABLE
    bad = wl.req[r:r + 1].copy()
    bad["stripes"] = 0
    with pytest.raises(mj.MojetteError) as ei:
        mj.mojette_server_submit(srv, bad)
    assert ei.value.code == -errno.EINVAL
    assert mj.mojette_server_stats(srv)["queued"] == 0
