// Request server: continuous batching of object writes (encode) and reads
// (decode) over a fixed device buffer pool (mojette_server_* in
// include/mojette.h). The paper measures one block at a time (Sec. 4); this
// is the storage-node side of a deployment and has no counterpart there.
//
// A request is an object of whole stripes of one geometry, with its input
// and output in pinned host memory. The server
//   - queues requests as they are submitted (never blocks);
//   - admits them first-come first-served into a wave while the wave's
//     device buffers fit the pool (the budget: one half for inputs, one for
//     outputs, each carved first-fit) and the wave stays under its stripe
//     cap; a request waits for memory rather than being skipped;
//   - copies a wave's inputs in and outputs out with one cudaMemcpyAsync per
//     run of requests whose host buffers and device buffers are both
//     back to back (first-fit keeps the device side so for a fresh pool), so
//     requests that arrive in a contiguous host ring move in a few large
//     copies instead of one per request;
//   - runs every wave on its own slot: a stream, a batch (one kernel per
//     (operation, plan), every stripe its own mask) and an event; up to
//     `slots` waves are in flight, so one wave's copies overlap another's
//     kernels, and requests that arrive while waves run join the next wave
//     as soon as a slot and memory free up;
//   - retires a wave when its event completes, frees its buffers and
//     reports each request's arrival, admission and completion times.
#include <algorithm>
#include <cerrno>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "mojette_internal.h"

namespace mojette {
namespace {

constexpr size_t kPoolAlign = 16;   // every buffer starts 16-byte aligned

// First-fit allocator over [0, size) with coalescing of free blocks.
class Pool {
public:
    void reset(size_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + kPoolAlign - 1) & ~(kPoolAlign - 1);
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + kPoolAlign - 1) & ~(kPoolAlign - 1);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct Req {
    mojette_request_t r;
    double arrival = 0, admit = 0;
    size_t in_off = 0, in_bytes = 0, out_off = 0, out_bytes = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    mojette_batch_t batch = nullptr;
    std::vector<Req> reqs;
    bool busy = false;
    std::vector<mojette_stripe_t> table;
};

}  // namespace

struct Server {
    int device = 0;
    char *pool_base = nullptr;
    size_t budget = 0, half = 0;
    Pool pin, pout;                  // [0, half): inputs, [half, budget): outputs
    int64_t max_wave_stripes = 0;
    std::vector<Slot> slots;
    std::deque<Req> queue;
    std::vector<mojette_completion_t> ready;
    std::chrono::steady_clock::time_point t0;
    int64_t waves = 0, completed = 0, peak_used = 0;
    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void request_bytes(const mojette_request_t &r, size_t *in, size_t *out)
{
    const Plan *pl = reinterpret_cast<const Plan *>(r.plan);
    const size_t img = (size_t)r.stripes * pl->Q * pl->P * 8;
    const size_t bins = (size_t)r.stripes * pl->total * 8;
    *in = r.op == MOJETTE_OP_ENCODE ? img : bins;
    *out = r.op == MOJETTE_OP_ENCODE ? bins : img;
}

// Complete the requests of a finished wave.
void retire(Server &s, Slot &sl, int status)
{
    const double t = s.now();
    for (const Req &q : sl.reqs) {
        s.pin.release(q.in_off, q.in_bytes);
        s.pout.release(q.out_off - s.half, q.out_bytes);
        mojette_completion_t c;
        c.id = q.r.id;
        c.status = status;
        c.arrival_s = q.arrival;
        c.admit_s = q.admit;
        c.done_s = t;
        s.ready.push_back(c);
        ++s.completed;
    }
    sl.reqs.clear();
    sl.busy = false;
}

// Admit queued requests into slot `sl` and launch the wave. Returns 0 when
// nothing was admitted or the wave was launched.
int launch_wave(Server &s, Slot &sl)
{
    int64_t stripes = 0;
    sl.reqs.clear();
    const double t = s.now();
    while (!s.queue.empty()) {
        Req &q = s.queue.front();
        if (!sl.reqs.empty() && stripes + q.r.stripes > s.max_wave_stripes) break;
        size_t in_off = 0, out_off = 0;
        if (!s.pin.alloc(q.in_bytes, &in_off)) break;
        if (!s.pout.alloc(q.out_bytes, &out_off)) {
            s.pin.release(in_off, q.in_bytes);
            break;
        }
        out_off += s.half;
        q.in_off = in_off;
        q.out_off = out_off;
        q.admit = t;
        stripes += q.r.stripes;
        sl.reqs.push_back(q);
        s.queue.pop_front();
    }
    if (sl.reqs.empty()) return 0;
    s.peak_used = std::max<int64_t>(s.peak_used, (int64_t)(s.pin.used() + s.pout.used()));
    int err = 0;
    // Copies of runs of requests whose host and device buffers both follow
    // each other exactly (no byte outside the requested ranges is copied).
    auto copy_runs = [&](bool in) -> int {
        const cudaMemcpyKind kind = in ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
        size_t i = 0;
        while (i < sl.reqs.size()) {
            const Req &q0 = sl.reqs[i];
            char *host0 = in ? (char *)q0.r.host_src : (char *)q0.r.host_dst;
            char *dev0 = s.pool_base + (in ? q0.in_off : q0.out_off);
            size_t len = in ? q0.in_bytes : q0.out_bytes;
            size_t j = i + 1;
            for (; j < sl.reqs.size(); ++j) {
                const Req &qj = sl.reqs[j];
                char *hj = in ? (char *)qj.r.host_src : (char *)qj.r.host_dst;
                char *dj = s.pool_base + (in ? qj.in_off : qj.out_off);
                if (hj != host0 + len || dj != dev0 + len) break;
                len += in ? qj.in_bytes : qj.out_bytes;
            }
            const int e = in ? record_cuda(cudaMemcpyAsync(dev0, host0, len, kind, sl.stream))
                             : record_cuda(cudaMemcpyAsync(host0, dev0, len, kind, sl.stream));
            if (e) return e;
            i = j;
        }
        return 0;
    };
    // inputs in (pinned host memory)
    if ((err = copy_runs(true))) return err;
    // one stripe table over the wave
    sl.table.clear();
    sl.table.reserve((size_t)stripes);
    for (const Req &q : sl.reqs) {
        const Plan *pl = reinterpret_cast<const Plan *>(q.r.plan);
        const size_t img = (size_t)pl->Q * pl->P * 8, bins = (size_t)pl->total * 8;
        const size_t si = q.r.op == MOJETTE_OP_ENCODE ? img : bins;
        const size_t so = q.r.op == MOJETTE_OP_ENCODE ? bins : img;
        for (int64_t k = 0; k < q.r.stripes; ++k) {
            mojette_stripe_t d;
            d.plan = q.r.plan;
            d.op = q.r.op;
            d.erasure_mask = q.r.op == MOJETTE_OP_DECODE ? q.r.erasure_mask : 0u;
            d.src = reinterpret_cast<const uint64_t *>(s.pool_base + q.in_off + (size_t)k * si);
            d.dst = reinterpret_cast<uint64_t *>(s.pool_base + q.out_off + (size_t)k * so);
            sl.table.push_back(d);
        }
    }
    if (!sl.batch) {
        if ((err = mojette_batch_create(sl.table.data(), (int64_t)sl.table.size(), 0, &sl.batch))) return err;
    } else if ((err = mojette_batch_update(sl.batch, sl.table.data(), (int64_t)sl.table.size(),
                                           (mojette_stream_t)sl.stream))) {
        return err;
    }
    if ((err = mojette_batch_run(sl.batch, (mojette_stream_t)sl.stream))) return err;
    // outputs back
    if ((err = copy_runs(false))) return err;
    if ((err = record_cuda(cudaEventRecord(sl.done, sl.stream)))) return err;
    sl.busy = true;
    ++s.waves;
    return 0;
}

// One round of progress: retire finished waves, then fill free slots.
int progress(Server &s)
{
    int err = 0;
    for (Slot &sl : s.slots) {
        if (!sl.busy) continue;
        const cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaSuccess) retire(s, sl, 0);
        else if (e != cudaErrorNotReady) {
            record_cuda(e);
            retire(s, sl, -EIO);
            return -EIO;
        }
    }
    for (Slot &sl : s.slots) {
        if (sl.busy) continue;
        if (s.queue.empty()) break;
        if ((err = launch_wave(s, sl))) {
            // the wave's requests fail; their buffers go back to the pool
            // once the copies already enqueued have finished
            cudaStreamSynchronize(sl.stream);
            retire(s, sl, err);
            return err;
        }
        if (!sl.busy) break;   // nothing fitted: wait for memory
    }
    return 0;
}

void release(Server *s)
{
    if (!s) return;
    cudaSetDevice(s->device);
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.batch) mojette_batch_destroy(sl.batch);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->pool_base) cudaFree(s->pool_base);
    delete s;
}

}  // namespace
}  // namespace mojette

using namespace mojette;

extern "C" {

int mojette_server_create(int64_t device_budget_bytes, int slots, int64_t max_wave_stripes,
                          mojette_server_t *out)
{
    if (!out) return -EINVAL;
    *out = nullptr;
    if (device_budget_bytes < (int64_t)kPoolAlign || slots < 1 || slots > 64 || max_wave_stripes < 1)
        return -EINVAL;
    Server *s = new (std::nothrow) Server();
    if (!s) return -ENOMEM;
    s->t0 = std::chrono::steady_clock::now();
    s->budget = (size_t)device_budget_bytes & ~(kPoolAlign - 1);
    s->half = (s->budget / 2) & ~(kPoolAlign - 1);
    s->max_wave_stripes = max_wave_stripes;
    int err = record_cuda(cudaGetDevice(&s->device));
    if (!err) {
        const cudaError_t e = cudaMalloc(&s->pool_base, s->budget);
        if (e != cudaSuccess) {
            record_cuda(e);
            s->pool_base = nullptr;
            err = e == cudaErrorMemoryAllocation ? -ENOMEM : -EIO;
        }
    }
    s->pin.reset(err ? 0 : s->half);
    s->pout.reset(err ? 0 : s->budget - s->half);
    s->slots.resize((size_t)slots);
    for (Slot &sl : s->slots) {
        if (err) break;
        err = record_cuda(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
        if (!err) err = record_cuda(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
    }
    if (err) {
        release(s);
        return err;
    }
    *out = reinterpret_cast<mojette_server_t>(s);
    return 0;
}

int mojette_server_submit(mojette_server_t server, const mojette_request_t *reqs, int64_t n)
{
    if (!server || n < 0 || (n > 0 && !reqs)) return -EINVAL;
    Server *s = reinterpret_cast<Server *>(server);
    // validate all first: a bad request rejects the whole call
    for (int64_t i = 0; i < n; ++i) {
        const mojette_request_t &r = reqs[i];
        if (!r.plan || !r.host_src || !r.host_dst || r.stripes < 1) return -EINVAL;
        if (r.op != MOJETTE_OP_ENCODE && r.op != MOJETTE_OP_DECODE) return -EINVAL;
        const Plan *pl = reinterpret_cast<const Plan *>(r.plan);
        if (r.op == MOJETTE_OP_DECODE) {
            // a systematic read rebuilds lines in place from two inputs
            // (data and parity): not a request of this server
            if (pl->Q > kMaxLines || pl->systematic) return -EINVAL;
            if (pl->n < 32 && (r.erasure_mask >> pl->n)) return -EINVAL;
            int err = 0;
            if (!get_schedule(*const_cast<Plan *>(pl), r.erasure_mask, &err)) return err;
        }
        size_t in = 0, out = 0;
        request_bytes(r, &in, &out);
        const size_t rin = (in + kPoolAlign - 1) & ~(kPoolAlign - 1);
        const size_t rout = (out + kPoolAlign - 1) & ~(kPoolAlign - 1);
        if (rin > s->half || rout > s->budget - s->half || r.stripes > s->max_wave_stripes) return -ENOSPC;
    }
    const double t = s->now();
    for (int64_t i = 0; i < n; ++i) {
        Req q;
        q.r = reqs[i];
        q.arrival = reqs[i].arrival_s > 0 ? reqs[i].arrival_s : t;
        request_bytes(q.r, &q.in_bytes, &q.out_bytes);
        s->queue.push_back(q);
    }
    return progress(*s);
}

int mojette_server_poll(mojette_server_t server, mojette_completion_t *out, int64_t max, int64_t *n_out)
{
    if (!server || max < 0 || (max > 0 && !out)) return -EINVAL;
    Server *s = reinterpret_cast<Server *>(server);
    const int err = progress(*s);
    const int64_t n = std::min<int64_t>(max, (int64_t)s->ready.size());
    for (int64_t i = 0; i < n; ++i) out[i] = s->ready[(size_t)i];
    s->ready.erase(s->ready.begin(), s->ready.begin() + n);
    if (n_out) *n_out = n;
    return err;
}

int mojette_server_now(mojette_server_t server, double *seconds)
{
    if (!server || !seconds) return -EINVAL;
    *seconds = reinterpret_cast<Server *>(server)->now();
    return 0;
}

int mojette_server_stats(mojette_server_t server, int64_t *queued, int64_t *in_flight, int64_t *waves,
                         int64_t *completed, int64_t *pool_used, int64_t *pool_peak)
{
    if (!server) return -EINVAL;
    Server *s = reinterpret_cast<Server *>(server);
    int64_t fl = 0;
    for (const Slot &sl : s->slots) fl += sl.busy ? (int64_t)sl.reqs.size() : 0;
    if (queued) *queued = (int64_t)s->queue.size();
    if (in_flight) *in_flight = fl;
    if (waves) *waves = s->waves;
    if (completed) *completed = s->completed;
    if (pool_used) *pool_used = (int64_t)(s->pin.used() + s->pout.used());
    if (pool_peak) *pool_peak = s->peak_used;
    return 0;
}

int mojette_server_destroy(mojette_server_t server)
{
    release(reinterpret_cast<Server *>(server));
    return 0;
}

}  // extern "C"
