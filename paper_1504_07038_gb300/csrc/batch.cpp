// Batched encode/decode: many stripes of mixed geometry, operation and
// erasure pattern in one submission (mojette_batch_* in include/mojette.h).
//
// Host side of the batch. Stripes are sorted by (operation, plan, mask);
// every (operation, plan) becomes one kernel launch (a "class"), and inside a
// decode class every erasure mask becomes one group with its own cached
// reconstruction path (Sec. 2.2, one path per surviving set). The kernels
// read per-stripe addresses, the groups and the work items from one device
// workspace, so a launch covers thousands of stripes of one geometry
// whatever their masks and wherever they live. Classes are independent:
// they run on side streams forked from the caller's stream (or as parallel
// nodes of one CUDA graph), so small classes fill the GPU together.
#include <algorithm>
#include <cerrno>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "mojette_internal.h"

namespace mojette {
namespace {

constexpr int kMaxSideStreams = 8;

struct Klass {
    int op = 0;                 // MOJETTE_OP_ENCODE / MOJETTE_OP_DECODE
    Plan *plan = nullptr;
    int64_t first = 0, count = 0;   // its stripes: srcp/dstp[first, first + count)
    // decode only
    std::vector<int64_t> gcount;    // stripes per group (groups in table order)
    int64_t gbase = 0;              // its first group in the group table
    int64_t wbase = 0, wcap = 0;    // its region of the work table
    int64_t nwork = 0;              // work items in use
    int maxp = 0, maxT = 0;
    int lines = 0;                  // lines rebuilt per stripe (systematic: lost lines)
    int span = 0;                   // widest row distance between two of them
    bool sys = false;               // systematic plan: in-place decode of the lost lines
    bool scan_ok = false;           // two lines and every group has the closed form (decode_scan2)
    bool van_ok = false;            // every group has the Vandermonde form (decode_vander)
    int van_maxp = 0;               //   and the largest |p| its paths use
    int32_t rowoff[kMaxLines] = {};   // row phases of its largest group
    DecodeConfig dcfg;
    EncodeConfig ecfg;
};

}  // namespace

struct Batch {
    int device = 0;
    uint32_t flags = 0;
    int64_t count = 0, ngroups = 0;
    std::vector<Klass> classes;
    // workspace, identical layout on the host (pinned staging) and device:
    // srcp[count], dstp[count], groups[ngroups], work[sum of wcap]
    char *host = nullptr, *dev = nullptr;
    size_t cap = 0, used = 0;
    size_t off_dst = 0, off_grp = 0, off_work = 0;
    cudaEvent_t staged = nullptr;   // the last upload has left the staging buffer
    bool staged_pending = false;
    cudaStream_t cap_stream = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool dirty = true;              // tables changed since the graph was captured
};

namespace {

const uint64_t **src_table(Batch &b, char *base) { return reinterpret_cast<const uint64_t **>(base); }
uint64_t **dst_table(Batch &b, char *base) { return reinterpret_cast<uint64_t **>(base + b.off_dst); }
DecGroup *group_table(Batch &b, char *base) { return reinterpret_cast<DecGroup *>(base + b.off_grp); }
DecWork *work_table(Batch &b, char *base) { return reinterpret_cast<DecWork *>(base + b.off_work); }

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
bool aligned8(const void *p) { return ((uintptr_t)p & 7u) == 0; }

void drop_graph(Batch &b)
{
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.graph) cudaGraphDestroy(b.graph);
    b.exec = nullptr;
    b.graph = nullptr;
    b.dirty = true;
}

// Work items of a decode class for the layout's G, written to the host
// staging copy of its work region.
int fill_work(Batch &b, Klass &k, int G)
{
    DecWork *w = work_table(b, b.host) + k.wbase;
    int64_t n = 0, first = k.first;
    for (size_t g = 0; g < k.gcount.size(); ++g) {
        for (int64_t i = 0; i < k.gcount[g]; i += G) {
            if (n >= k.wcap) return -EINVAL;
            w[n].group = (int32_t)(k.gbase + (int64_t)g);
            w[n].nst = (int32_t)std::min<int64_t>(G, k.gcount[g] - i);
            w[n].first = first + i;
            ++n;
        }
        first += k.gcount[g];
    }
    k.nwork = n;
    return 0;
}

int class_layout(const Klass &k, const DecodeConfig &cfg, DecodeLayout *L)
{
    if (k.sys && cfg.kernel != 0 && cfg.kernel != 4) return -EINVAL;   // decode_lines or decode_scan2
    if (cfg.kernel == 4 && !k.scan_ok) return -EINVAL;
    if (cfg.kernel == 5 && !k.van_ok) return -EINVAL;
    return decode_layout(k.plan->P, k.lines, k.span, cfg.kernel == 5 ? k.van_maxp : k.maxp, k.maxT, cfg,
                         k.rowoff, L);
}

// Lost data lines of a systematic decode stripe (0 otherwise).
int sys_lines(const mojette_stripe_t &d)
{
    const Plan *pl = reinterpret_cast<const Plan *>(d.plan);
    if (d.op != MOJETTE_OP_DECODE || !pl->systematic) return 0;
    const uint32_t data = pl->Q >= 32 ? 0xFFFFFFFFu : (1u << pl->Q) - 1u;
    return __builtin_popcount(d.erasure_mask & data);
}

int launch_class(Batch &b, const Klass &k, cudaStream_t st)
{
    if (k.op == MOJETTE_OP_ENCODE) {
        const Plan &pl = *k.plan;
        EncodeArgs a{};
        a.srcp = src_table(b, b.dev) + k.first;
        a.dstp = dst_table(b, b.dev) + k.first;
        a.tile_bytes = k.ecfg.tile_bytes;
        a.S = k.count;
        a.total = pl.total;
        a.P = pl.P;
        a.Q = pl.Q;
        a.n = pl.n;
        for (int i = 0; i < pl.n; ++i) {
            a.p[i] = pl.p[i];
            a.off[i] = pl.off[i];
            a.bmin[i] = pl.bmin[i];
        }
        int err = 0;
        a.status = device_status_ptr(&err);
        if (err) return err;
        if ((err = plan_full_bin_on_device(*k.plan, &a.full_bin))) return err;
        return launch_encode_batched(a, st);
    }
    DecBatchArgs a{};
    a.P = k.plan->P;
    a.Q = k.lines;
    a.sys = k.sys;
    a.Qd = k.plan->Q;
    a.span = k.span;
    a.van_maxp = k.van_maxp;
    a.maxp = k.maxp;
    a.maxT = k.maxT;
    for (int l = 0; l < kMaxLines; ++l) a.rowoff[l] = k.rowoff[l];
    a.groups = group_table(b, b.dev);
    a.work = work_table(b, b.dev) + k.wbase;
    a.nwork = k.nwork;
    a.srcp = src_table(b, b.dev);
    a.dstp = dst_table(b, b.dev);
    int err = 0;
    a.status = device_status_ptr(&err);
    if (err) return err;
    return launch_decode_batched(a, k.dcfg, st);
}

int ensure_streams(Batch &b, size_t n)
{
    n = std::min<size_t>(n, kMaxSideStreams);
    int err = 0;
    if (!b.fork && (err = record_cuda(cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming)))) return err;
    while (b.side.size() < n) {
        cudaStream_t s = nullptr;
        if ((err = record_cuda(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)))) return err;
        b.side.push_back(s);
        cudaEvent_t e = nullptr;
        if ((err = record_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming)))) return err;
        b.done.push_back(e);
    }
    return 0;
}

// Every class once, forked over side streams and joined back into `st`.
int launch_all(Batch &b, cudaStream_t st)
{
    int err = 0;
    if (b.classes.empty()) return 0;
    if (b.classes.size() == 1) return launch_class(b, b.classes[0], st);
    if ((err = ensure_streams(b, b.classes.size()))) return err;
    if ((err = record_cuda(cudaEventRecord(b.fork, st)))) return err;
    const size_t ns = b.side.size();
    for (size_t i = 0; i < ns && i < b.classes.size(); ++i)
        if ((err = record_cuda(cudaStreamWaitEvent(b.side[i], b.fork, 0)))) return err;
    // largest classes first, so the long launches start earliest
    std::vector<size_t> order(b.classes.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t x, size_t y) { return b.classes[x].count > b.classes[y].count; });
    for (size_t r = 0; r < order.size(); ++r)
        if ((err = launch_class(b, b.classes[order[r]], b.side[r % ns]))) return err;
    for (size_t i = 0; i < ns && i < b.classes.size(); ++i) {
        if ((err = record_cuda(cudaEventRecord(b.done[i], b.side[i])))) return err;
        if ((err = record_cuda(cudaStreamWaitEvent(st, b.done[i], 0)))) return err;
    }
    return 0;
}

int capture_graph(Batch &b)
{
    int err = 0;
    drop_graph(b);
    if (!b.cap_stream &&
        (err = record_cuda(cudaStreamCreateWithFlags(&b.cap_stream, cudaStreamNonBlocking))))
        return err;
    if ((err = record_cuda(cudaStreamBeginCapture(b.cap_stream, cudaStreamCaptureModeRelaxed)))) return err;
    const int lerr = launch_all(b, b.cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b.cap_stream, &g);
    if (lerr) {
        if (g) cudaGraphDestroy(g);
        return lerr;
    }
    if ((err = record_cuda(e))) return err;
    b.graph = g;
    if ((err = record_cuda(cudaGraphInstantiate(&b.exec, g, 0)))) return err;
    b.dirty = false;
    return 0;
}

// Build every table of the batch from `stripes` into the host staging copy
// and upload it on `st` (reallocating the workspace when it grows).
int build(Batch &b, const mojette_stripe_t *stripes, int64_t count, cudaStream_t st)
{
    int err = 0;
    // validate
    for (int64_t i = 0; i < count; ++i) {
        const mojette_stripe_t &d = stripes[i];
        if (!d.plan || !d.src || !d.dst) return -EINVAL;
        if (d.op != MOJETTE_OP_ENCODE && d.op != MOJETTE_OP_DECODE) return -EINVAL;
        const Plan *pl = reinterpret_cast<const Plan *>(d.plan);
        // 8-byte words everywhere; encode stages rows of even P by 16-byte
        // bulk copies
        if (!aligned8(d.src) || !aligned8(d.dst)) return -ERANGE;
        if (d.op == MOJETTE_OP_ENCODE && pl->P % 2 == 0 && !aligned16(d.src)) return -ERANGE;
        if (d.op == MOJETTE_OP_DECODE) {
            if (pl->Q > kMaxLines) return -EINVAL;
            const int bits = pl->systematic ? pl->Q + pl->n : pl->n;
            if (bits < 32 && (d.erasure_mask >> bits)) return -EINVAL;
        }
    }
    // order by (op, plan, lost data lines of a systematic decode, mask)
    std::vector<int64_t> idx(count);
    std::iota(idx.begin(), idx.end(), 0);
    auto key = [&](int64_t i) {
        const mojette_stripe_t &d = stripes[i];
        return std::make_tuple(d.op, (uintptr_t)d.plan, sys_lines(d),
                               d.op == MOJETTE_OP_DECODE ? d.erasure_mask : 0u);
    };
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return key(x) < key(y); });

    std::vector<Klass> classes;
    std::vector<DecGroup> groups;
    for (int64_t r = 0; r < count;) {
        const mojette_stripe_t &d0 = stripes[idx[r]];
        Klass k;
        k.op = d0.op;
        k.plan = reinterpret_cast<Plan *>(d0.plan);
        k.first = r;
        const int kl = sys_lines(d0);
        int64_t e = r;
        while (e < count && stripes[idx[e]].op == k.op && stripes[idx[e]].plan == d0.plan &&
               sys_lines(stripes[idx[e]]) == kl)
            ++e;
        k.count = e - r;
        k.sys = k.op == MOJETTE_OP_DECODE && k.plan->systematic;
        if (k.sys && kl == 0) {
            // systematic reads that lost no data line: the data is whole, no launch
            r = e;
            continue;
        }
        if (k.op == MOJETTE_OP_ENCODE) {
            k.ecfg = k.plan->tuned_enc ? k.plan->enc_cfg : EncodeConfig();
        } else {
            k.lines = k.sys ? kl : k.plan->Q;
            k.gbase = (int64_t)groups.size();
            k.scan_ok = k.lines == 2;
            k.van_ok = !k.sys && k.lines >= 2 && k.lines <= 8;
            int64_t big = 0;
            Schedule *big_sc = nullptr;
            int64_t big_grp = -1;
            for (int64_t g = r; g < e;) {
                const uint32_t mask = stripes[idx[g]].erasure_mask;
                int64_t h = g;
                while (h < e && stripes[idx[h]].erasure_mask == mask) ++h;
                Schedule *sc = get_schedule(*k.plan, mask, &err);
                if (!sc) return err;
                uint32_t *dsteps = nullptr;
                if ((err = schedule_on_device(*k.plan, *sc, &dsteps))) return err;
                DecGroup gr;
                std::memset(&gr, 0, sizeof(gr));
                gr.steps = dsteps;
                gr.T = sc->T;
                gr.fwd = sc->fwd;
                gr.known = sc->known;
                for (int l = 0; l < sc->lines; ++l) gr.lpos[l] = sc->lpos[l];
                k.scan_ok = k.scan_ok && sc->scan2;
                k.van_ok = k.van_ok && sc->vander;
                gr.van_E0 = sc->van_E0;
                gr.van_L = sc->van_L;
                for (int j = 0; j < kMaxLines; ++j) {
                    gr.van_q[j] = sc->van_q[j];
                    gr.van_base[j] = (int32_t)sc->van_base[j];
                    gr.van_lo[j] = sc->van_lo[j];
                    gr.van_hi[j] = sc->van_hi[j];
                    if (j < sc->lines) k.van_maxp = std::max(k.van_maxp, std::abs(sc->van_q[j]));
                }
                for (int j = 0; j < 2; ++j) {
                    gr.scan_p[j] = sc->scan_p[j];
                    gr.scan_src[j] = (int32_t)sc->scan_src[j];
                }
                k.span = std::max(k.span, sc->lines > 0 ? sc->lpos[sc->lines - 1] - sc->lpos[0] : 0);
                for (int l = 0; l < sc->lines; ++l) {
                    gr.p[2 * l] = sc->pL[l];
                    gr.p[2 * l + 1] = sc->pR[l];
                    gr.src[2 * l] = (int32_t)sc->srcL[l];
                    gr.src[2 * l + 1] = (int32_t)sc->srcR[l];
                    gr.split[l] = sc->split[l];
                    gr.order[2 * l] = kIdentityOrder;
                    gr.order[2 * l + 1] = kIdentityOrder;
                    gr.chunk_w = sc->chunk_w;
                    for (int c = 0; c < kStreamChunks; ++c) {
                        gr.chunk_wait[c] = sc->chunk_wait[c];
                        gr.chunk_done[c] = sc->chunk_done[c];
                    }
                    k.maxp = std::max(k.maxp, std::max(std::abs(sc->pL[l]), std::abs(sc->pR[l])));
                }
                k.maxT = std::max(k.maxT, sc->T);
                if (h - g > big) {   // the largest group sets the class's row phases
                    big = h - g;
                    big_sc = sc;
                    big_grp = (int64_t)groups.size();
                }
                groups.push_back(gr);
                k.gcount.push_back(h - g);
                g = h;
            }
            // configuration: the plan's tuned one where it applies, else the
            // closed form for two lines, else decode_lines
            DecodeConfig def;
            def.kernel = choose_decode_kernel(k.plan->P, k.lines, k.count, k.sys, k.scan_ok, k.van_ok, false);
            k.dcfg = k.plan->tuned_dec ? k.plan->dec_cfg : def;
            if ((k.sys && k.dcfg.kernel != 0 && k.dcfg.kernel != 4) || (k.dcfg.kernel == 4 && !k.scan_ok) ||
                (k.dcfg.kernel == 5 && !k.van_ok))
                k.dcfg = def;
            if (big_sc)   // bulk-staging parity of the largest group's rows
                for (int l = 0; l < kMaxLines; ++l) k.rowoff[l] = big_sc->rowpar[l];
            // the bank layout search serves the largest group's path: only
            // worth its host time when that group alone is a large launch
            if (big_sc && big >= kPhaseMinStripes) {
                const int32_t *ph = schedule_row_phases(*k.plan, *big_sc);
                for (int l = 0; l < kMaxLines; ++l) k.rowoff[l] = ph[l];
                // its load orders go with those phases; the other groups
                // keep the plain order
                for (int l = 0; l < big_sc->lines; ++l) {
                    groups[(size_t)big_grp].order[2 * l] = big_sc->order[2 * l];
                    groups[(size_t)big_grp].order[2 * l + 1] = big_sc->order[2 * l + 1];
                }
            }
            // room for the smallest G any configuration uses (1 stripe per item)
            k.wcap = k.count;
        }
        classes.push_back(std::move(k));
        r = e;
    }
    int64_t wtotal = 0;
    for (auto &k : classes)
        if (k.op == MOJETTE_OP_DECODE) {
            k.wbase = wtotal;
            wtotal += k.wcap;
        }

    // workspace layout
    const size_t off_dst = align256((size_t)count * 8);
    const size_t off_grp = off_dst + align256((size_t)count * 8);
    const size_t off_work = off_grp + align256(groups.size() * sizeof(DecGroup));
    const size_t used = off_work + align256((size_t)wtotal * sizeof(DecWork));

    // the staging buffer may still feed the previous upload
    if (b.staged_pending && (err = record_cuda(cudaEventSynchronize(b.staged)))) return err;
    b.staged_pending = false;
    if (used > b.cap) {
        // work enqueued before may still read the old tables
        if ((err = record_cuda(cudaStreamSynchronize(st)))) return err;
        if ((err = record_cuda(cudaDeviceSynchronize()))) return err;
        if (b.dev) cudaFree(b.dev);
        if (b.host) cudaFreeHost(b.host);
        b.dev = nullptr;
        b.host = nullptr;
        b.cap = 0;
        const size_t cap = std::max(used + used / 4, (size_t)4096);
        cudaError_t ce = cudaMalloc(&b.dev, cap);
        if (ce != cudaSuccess) {
            record_cuda(ce);
            return ce == cudaErrorMemoryAllocation ? -ENOMEM : -EIO;
        }
        ce = cudaHostAlloc(&b.host, cap, cudaHostAllocDefault);
        if (ce != cudaSuccess) {
            record_cuda(ce);
            cudaFree(b.dev);
            b.dev = nullptr;
            return ce == cudaErrorMemoryAllocation ? -ENOMEM : -EIO;
        }
        b.cap = cap;
        drop_graph(b);
    }
    b.off_dst = off_dst;
    b.off_grp = off_grp;
    b.off_work = off_work;
    b.used = used;
    b.count = count;
    b.ngroups = (int64_t)groups.size();
    b.classes = std::move(classes);

    const uint64_t **sp = src_table(b, b.host);
    uint64_t **dp = dst_table(b, b.host);
    for (int64_t r = 0; r < count; ++r) {
        sp[r] = stripes[idx[r]].src;
        dp[r] = stripes[idx[r]].dst;
    }
    if (!groups.empty()) std::memcpy(group_table(b, b.host), groups.data(), groups.size() * sizeof(DecGroup));
    for (auto &k : b.classes)
        if (k.op == MOJETTE_OP_DECODE) {
            DecodeLayout L;
            if ((err = class_layout(k, k.dcfg, &L))) {
                // a configuration that does not fit: decode_lines, else
                // decode_fronts (G down to one stripe; not for the
                // systematic form)
                k.dcfg = DecodeConfig();
                if ((err = class_layout(k, k.dcfg, &L))) {
                    if (k.sys) return err;
                    k.dcfg.kernel = 1;
                    if ((err = class_layout(k, k.dcfg, &L))) return err;
                }
            }
            if ((err = fill_work(b, k, L.G))) return err;
        }
    if (!b.staged && (err = record_cuda(cudaEventCreateWithFlags(&b.staged, cudaEventDisableTiming)))) return err;
    if (used) {
        if ((err = record_cuda(cudaMemcpyAsync(b.dev, b.host, used, cudaMemcpyHostToDevice, st)))) return err;
        if ((err = record_cuda(cudaEventRecord(b.staged, st)))) return err;
        b.staged_pending = true;
    }
    b.dirty = true;
    return 0;
}

// Upload one decode class's work region from the staging copy.
int upload_work(Batch &b, const Klass &k, cudaStream_t st)
{
    const size_t off = b.off_work + (size_t)k.wbase * sizeof(DecWork);
    const size_t bytes = (size_t)k.nwork * sizeof(DecWork);
    if (!bytes) return 0;
    return record_cuda(cudaMemcpyAsync(b.dev + off, b.host + off, bytes, cudaMemcpyHostToDevice, st));
}

// Mean milliseconds of `reps` launches of one class (after one untimed).
int time_class(Batch &b, const Klass &k, cudaStream_t st, int reps, cudaEvent_t e0, cudaEvent_t e1,
               float *ms)
{
    int err = 0;
    if ((err = launch_class(b, k, st))) return err;
    if ((err = record_cuda(cudaEventRecord(e0, st)))) return err;
    for (int r = 0; r < reps; ++r)
        if ((err = launch_class(b, k, st))) return err;
    if ((err = record_cuda(cudaEventRecord(e1, st)))) return err;
    if ((err = record_cuda(cudaEventSynchronize(e1)))) return err;
    float t = 0.f;
    if ((err = record_cuda(cudaEventElapsedTime(&t, e0, e1)))) return err;
    *ms = t / (float)std::max(reps, 1);
    return 0;
}

int tune(Batch &b, cudaStream_t st, int reps)
{
    int err = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((err = record_cuda(cudaEventCreate(&e0)))) return err;
    if ((err = record_cuda(cudaEventCreate(&e1)))) {
        cudaEventDestroy(e0);
        return err;
    }
    // the tables must be on the device before any class runs
    if (b.staged_pending && (err = record_cuda(cudaEventSynchronize(b.staged)))) goto out;
    b.staged_pending = false;
    for (auto &k : b.classes) {
        if (k.op == MOJETTE_OP_ENCODE) {
            // tile sizes from one stripe to several; candidates that give
            // the same stripes per tile are timed once
            const Plan &pl = *k.plan;
            int maxp = 0;
            for (int i = 0; i < pl.n; ++i) maxp = std::max(maxp, pl.p[i] < 0 ? -pl.p[i] : pl.p[i]);
            int pad = (pl.Q - 1) * maxp;
            pad += pad & 1;
            const int64_t sb = (int64_t)(pl.Q * (pl.P + pad) + pad) * 8;
            std::vector<int> tried_spt;
            float best = 1e30f;
            EncodeConfig best_cfg = k.ecfg;
            for (int64_t tb : {sb, (int64_t)9000, (int64_t)16000, (int64_t)24000, (int64_t)32000,
                               (int64_t)48000}) {
                const int spt = (int)std::max<int64_t>(1, tb / sb);
                if (std::find(tried_spt.begin(), tried_spt.end(), spt) != tried_spt.end()) continue;
                tried_spt.push_back(spt);
                k.ecfg.tile_bytes = (int)std::max<int64_t>(tb, sb);
                float ms = 0.f;
                if ((err = time_class(b, k, st, reps, e0, e1, &ms))) goto out;
                if (ms < best) {
                    best = ms;
                    best_cfg = k.ecfg;
                }
            }
            k.ecfg = best_cfg;
            k.plan->enc_cfg = best_cfg;
            k.plan->tuned_enc = true;
        } else {
            struct Cand { int kernel, gpc, persist, rowoff; };
            // the path kernels only: the closed forms (decode_scan2,
            // decode_vander) are not the paper's inverse and run only when a
            // configuration installed with mojette_plan_config names them
            std::vector<Cand> cands;
            if (k.sys) {
                for (int sp : {0, 1})
                    for (int g : {1, 2, 4, 8}) cands.push_back({0, g, 0, sp});
                cands.push_back({0, 4, 1, 1});
            } else if (k.plan->Q <= 8) {
                for (int g : {1, 2, 4, 8}) cands.push_back({6, g, 0, 0});
                cands.push_back({6, 4, 1, 0});
                for (int sp : {0, 1})
                    for (int g : {1, 2, 4, 8}) cands.push_back({0, g, 0, sp});
                for (int kern : {2, 3})
                    for (int g : {1, 2, 4, 8}) cands.push_back({kern, g, 0, 0});
                for (int kern : {0, 3}) cands.push_back({kern, 4, 1, 1});
            }
            if (!k.sys)
                for (int g : {1, 2, 4}) cands.push_back({1, g, 0, 0});
            float best = 1e30f;
            DecodeConfig best_cfg = k.dcfg;
            for (const Cand &c : cands) {
                DecodeConfig cfg;
                cfg.kernel = c.kernel;
                cfg.gpc = c.gpc;
                cfg.persist = c.persist;
                cfg.rowoff = c.rowoff;
                DecodeLayout L;
                if (class_layout(k, cfg, &L)) continue;      // does not fit: skip
                if (c.kernel != L.kernel) continue;           // Q > 8: decode_fronts only
                k.dcfg = cfg;
                if ((err = fill_work(b, k, L.G))) goto out;
                if ((err = upload_work(b, k, st))) goto out;
                float ms = 0.f;
                if ((err = time_class(b, k, st, reps, e0, e1, &ms))) goto out;
                if (ms < best) {
                    best = ms;
                    best_cfg = cfg;
                }
            }
            k.dcfg = best_cfg;
            k.plan->dec_cfg = best_cfg;
            k.plan->tuned_dec = true;
            DecodeLayout L;
            if ((err = class_layout(k, k.dcfg, &L))) goto out;
            if ((err = fill_work(b, k, L.G))) goto out;
            if ((err = upload_work(b, k, st))) goto out;
        }
    }
    err = record_cuda(cudaStreamSynchronize(st));
    b.dirty = true;
out:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err;
}

void release(Batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->dev || b->host) cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto s : b->side) cudaStreamDestroy(s);
    for (auto e : b->done) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->staged) cudaEventDestroy(b->staged);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->dev) cudaFree(b->dev);
    if (b->host) cudaFreeHost(b->host);
    delete b;
}

}  // namespace
}  // namespace mojette

using namespace mojette;

extern "C" {

int mojette_batch_create(const mojette_stripe_t *stripes, int64_t count, uint32_t flags,
                         mojette_batch_t *out)
{
    if (!out) return -EINVAL;
    *out = nullptr;
    if (count < 0 || (count > 0 && !stripes)) return -EINVAL;
    if (flags & ~(uint32_t)MOJETTE_BATCH_GRAPH) return -EINVAL;
    Batch *b = new (std::nothrow) Batch();
    if (!b) return -ENOMEM;
    b->flags = flags;
    int err = record_cuda(cudaGetDevice(&b->device));
    cudaStream_t st = nullptr;
    if (!err) err = record_cuda(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    if (!err) err = build(*b, stripes, count, st);
    if (!err) err = record_cuda(cudaStreamSynchronize(st));
    if (st) cudaStreamDestroy(st);
    b->staged_pending = false;
    if (err) {
        release(b);
        return err;
    }
    *out = reinterpret_cast<mojette_batch_t>(b);
    return 0;
}

int mojette_batch_update(mojette_batch_t batch, const mojette_stripe_t *stripes, int64_t count,
                         mojette_stream_t stream)
{
    if (!batch || count < 0 || (count > 0 && !stripes)) return -EINVAL;
    Batch *b = reinterpret_cast<Batch *>(batch);
    return build(*b, stripes, count, (cudaStream_t)stream);
}

int mojette_batch_run(mojette_batch_t batch, mojette_stream_t stream)
{
    if (!batch) return -EINVAL;
    Batch *b = reinterpret_cast<Batch *>(batch);
    if (b->count == 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    int err = 0;
    // the tables may have been uploaded on another stream
    if (b->staged_pending && (err = record_cuda(cudaStreamWaitEvent(st, b->staged, 0)))) return err;
    if (b->flags & MOJETTE_BATCH_GRAPH) {
        if (b->dirty || !b->exec) {
            // the capture stream must see the tables uploaded on other streams
            if (b->staged_pending && (err = record_cuda(cudaEventSynchronize(b->staged)))) return err;
            b->staged_pending = false;
            if ((err = capture_graph(*b))) return err;
        }
        return record_cuda(cudaGraphLaunch(b->exec, st));
    }
    return launch_all(*b, st);
}

int mojette_batch_tune(mojette_batch_t batch, mojette_stream_t stream, int reps)
{
    if (!batch || reps < 1) return -EINVAL;
    Batch *b = reinterpret_cast<Batch *>(batch);
    return tune(*b, (cudaStream_t)stream, reps);
}

int mojette_batch_info(mojette_batch_t batch, int64_t *launches, int64_t *groups, int64_t *work_items,
                       int32_t *configs)
{
    if (!batch) return -EINVAL;
    Batch *b = reinterpret_cast<Batch *>(batch);
    int64_t nw = 0;
    for (auto &k : b->classes) nw += k.op == MOJETTE_OP_DECODE ? k.nwork : 0;
    if (launches) *launches = (int64_t)b->classes.size();
    if (groups) *groups = b->ngroups;
    if (work_items) *work_items = nw;
    if (configs)
        for (size_t i = 0; i < b->classes.size(); ++i) {
            const Klass &k = b->classes[i];
            int32_t *c = configs + 6 * i;
            c[0] = k.op;
            c[1] = k.op == MOJETTE_OP_DECODE ? k.lines : k.plan->Q;
            c[2] = k.plan->P;
            c[3] = k.op == MOJETTE_OP_DECODE ? k.dcfg.kernel : 0;
            c[4] = k.op == MOJETTE_OP_DECODE ? k.dcfg.gpc : k.ecfg.tile_bytes;
            c[5] = k.op == MOJETTE_OP_DECODE ? (k.dcfg.persist | (k.dcfg.rowoff << 1)) : 0;
        }
    return 0;
}

int mojette_batch_destroy(mojette_batch_t batch)
{
    release(reinterpret_cast<Batch *>(batch));
    return 0;
}

}  // extern "C"
