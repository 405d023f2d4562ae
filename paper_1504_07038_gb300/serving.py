"""Client side of the request server (mojette_server_* in include/mojette.h):
a seeded object workload, Poisson arrivals, and the measurement loops.

The workload mirrors a hot-data storage node: 70% writes (encode an object)
and 30% reads (decode it from its projections with 0..n-k lost), objects of
4 KB to 1 MB (log-uniform) cut into 4 KB or 8 KB stripes of the (6,4) or
(12,8) code (the last stripe zero-padded), inputs and outputs in pinned host
memory. The server does the admission, batching and device work; this module
only decides when requests arrive and records what happens to them.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs

SIX = [-3, -2, -1, 1, 2, 3]
TWELVE = [v for v in range(-6, 7) if v]
# (P, Q, p): 4 KB and 8 KB stripes of the (6,4) and (12,8) codes
SERVE_GEOMS = [(128, 4, SIX), (256, 4, SIX), (64, 8, TWELVE), (128, 8, TWELVE)]


class Workload:
    """n seeded requests with their host buffers.

    Reads get valid projections: every object is encoded once on the device
    with the plain mojette_encode when the workload is built, outside any
    timed region. ``images[r]`` keeps each object's padded stripes, so a
    read's output can be checked against it.
    """

    def __init__(self, n: int, seed: int = inputs.DEFAULT_SEED, write_frac: float = 0.7,
                 min_bytes: int = 4096, max_bytes: int = 1 << 20, geoms=SERVE_GEOMS):
        import torch
        from . import binding as mj

        rng = np.random.default_rng(seed)
        self.plans = [mj.mojette_plan(P, Q, p) for P, Q, p in geoms]
        self.geoms = geoms
        g = rng.integers(0, len(geoms), n)
        write = rng.random(n) < write_frac
        size = np.exp(rng.uniform(np.log(min_bytes), np.log(max_bytes), n)).astype(np.int64)
        self.req = np.zeros(n, dtype=mj.REQUEST_DTYPE)
        self.user_bytes = size
        in_bytes = np.zeros(n, np.int64)
        out_bytes = np.zeros(n, np.int64)
        stripes = np.zeros(n, np.int64)
        masks = np.zeros(n, np.uint32)
        for k, (P, Q, p) in enumerate(geoms):
            sel = np.nonzero(g == k)[0]
            sb = Q * P * 8
            stripes[sel] = (size[sel] + sb - 1) // sb
            tot = self.plans[k].total * 8
            in_bytes[sel] = np.where(write[sel], stripes[sel] * sb, stripes[sel] * tot)
            out_bytes[sel] = np.where(write[sel], stripes[sel] * tot, stripes[sel] * sb)
            n_p = len(p)
            e = inputs.erasure_counts(len(sel), n_p - Q, seed=seed + k)
            masks[sel] = inputs.erasure_masks(len(sel), n_p, e, seed=seed + 31 * k)
        self.stripes, self.write, self.geom = stripes, write, g
        # pinned arenas, slices back to back (16-byte aligned), as a
        # receive ring would hold them
        al = lambda x: (x + 15) // 16 * 16
        in_off = np.concatenate([[0], np.cumsum(al(in_bytes))[:-1]])
        out_off = np.concatenate([[0], np.cumsum(al(out_bytes))[:-1]])
        self.h_in = torch.empty(int(al(in_bytes).sum()) // 8, dtype=torch.int64).pin_memory()
        self.h_out = torch.zeros(int(al(out_bytes).sum()) // 8, dtype=torch.int64).pin_memory()
        self.in_off, self.out_off = in_off, out_off
        self.in_bytes, self.out_bytes = in_bytes, out_bytes
        # objects: seeded stripes (whole stripes; bytes past the object are 0)
        self.images = []
        for r in range(n):
            P, Q, p = geoms[g[r]]
            img = inputs.stripes(int(stripes[r]), Q, P, seed=seed, first=int(in_off[r] // 8))
            flat = img.reshape(-1)
            flat[size[r] // 8:] = 0
            self.images.append(img)
        # reads: projections of the object, encoded on the device once
        for r in range(n):
            words = int(in_bytes[r] // 8)
            dst = self.h_in[in_off[r] // 8: in_off[r] // 8 + words]
            if write[r]:
                dst.copy_(torch.from_numpy(self.images[r].reshape(-1).view(np.int64)))
            else:
                d_img = torch.from_numpy(self.images[r].view(np.int64)).cuda()
                d_proj = torch.empty((int(stripes[r]), self.plans[g[r]].total), dtype=torch.int64,
                                     device="cuda")
                mj.mojette_encode(self.plans[g[r]], d_img, d_proj, int(stripes[r]))
                dst.copy_(d_proj.reshape(-1).cpu())
        torch.cuda.synchronize()
        base_in, base_out = self.h_in.data_ptr(), self.h_out.data_ptr()
        handles = np.array([pl.handle for pl in self.plans], dtype=np.uint64)
        self.req["id"] = np.arange(n, dtype=np.uint64)
        self.req["plan"] = handles[g]
        self.req["op"] = np.where(write, mj.MOJETTE_OP_ENCODE, mj.MOJETTE_OP_DECODE)
        self.req["erasure_mask"] = np.where(write, 0, masks)
        self.req["stripes"] = stripes
        self.req["host_src"] = base_in + in_off.astype(np.uint64)
        self.req["host_dst"] = base_out + out_off.astype(np.uint64)

    def __len__(self):
        return len(self.req)

    def output(self, r: int) -> np.ndarray:
        """Host bytes of request r's output (uint64 words)."""
        o = int(self.out_off[r] // 8)
        return self.h_out[o: o + int(self.out_bytes[r] // 8)].numpy().view(np.uint64)

    def clear_outputs(self):
        self.h_out.zero_()


def run_server(server, wl: Workload, rate: float | None = None, seed: int = 1, order=None):
    """Submit every request of ``wl`` (in ``order``) and wait for all.

    rate None: closed loop, every request submitted at once. Else open loop:
    Poisson arrivals at ``rate`` requests/s, each submitted when its arrival
    time comes (latency counts from that arrival even if submission runs
    late). Returns the completions (COMPLETION_DTYPE) and the elapsed seconds
    from the first arrival to the last completion.
    """
    from . import binding as mj

    idx = np.arange(len(wl)) if order is None else np.asarray(order)
    reqs = wl.req[idx].copy()
    done = []
    t0 = mj.mojette_server_now(server)
    if rate is None:
        reqs["arrival_s"] = t0
        mj.mojette_server_submit(server, reqs)
        i = len(reqs)
    else:
        gaps = np.random.default_rng(seed).exponential(1.0 / rate, len(reqs))
        arrival = t0 + np.cumsum(gaps)
        reqs["arrival_s"] = arrival
        i = 0
    n_done = 0
    while n_done < len(reqs):
        if i < len(reqs):
            now = mj.mojette_server_now(server)
            j = int(np.searchsorted(arrival, now, side="right"))
            if j > i:
                mj.mojette_server_submit(server, reqs[i:j])
                i = j
        c = mj.mojette_server_poll(server)
        if len(c):
            done.append(c)
            n_done += len(c)
        elif i >= len(reqs):
            time.sleep(20e-6)
    comp = np.concatenate(done) if done else np.zeros(0, dtype=mj.COMPLETION_DTYPE)
    if (comp["status"] != 0).any():
        raise RuntimeError(f"{int((comp['status'] != 0).sum())} requests failed")
    t_first = reqs["arrival_s"].min()
    return comp, float(comp["done_s"].max() - t_first)


def latency_stats(comp: np.ndarray) -> dict:
    lat = (comp["done_s"] - comp["arrival_s"]) * 1e3
    return {"p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3), "max_ms": round(float(lat.max()), 3)}


def run_plain(wl: Workload, order=None) -> float:
    """The same requests one at a time through the plain entry points: copy
    in, one mojette_encode / mojette_decode over the object's stripes, copy
    out, wait. Returns elapsed seconds."""
    import torch
    from . import binding as mj

    idx = np.arange(len(wl)) if order is None else np.asarray(order)
    cap_in = int(wl.in_bytes.max() // 8) + 1
    cap_out = int(wl.out_bytes.max() // 8) + 1
    d_in = torch.empty(cap_in, dtype=torch.int64, device="cuda")
    d_out = torch.empty(cap_out, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in idx:
        wi, wo = int(wl.in_bytes[r] // 8), int(wl.out_bytes[r] // 8)
        io, oo = int(wl.in_off[r] // 8), int(wl.out_off[r] // 8)
        d_in[:wi].copy_(wl.h_in[io: io + wi], non_blocking=True)
        plan = wl.plans[wl.geom[r]]
        S = int(wl.stripes[r])
        if wl.write[r]:
            mj.mojette_encode(plan, d_in, d_out, S, stream)
        else:
            mj.mojette_decode(plan, d_in, int(wl.req["erasure_mask"][r]), d_out, S, stream)
        wl.h_out[oo: oo + wo].copy_(d_out[:wo], non_blocking=True)
        stream.synchronize()
    return time.perf_counter() - t0
