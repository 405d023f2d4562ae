// extern "C" entry points of libmojette (declared in include/mojette.h).
#include <algorithm>
#include <cerrno>
#include <cstring>
#include <new>

#include "mojette_internal.h"

namespace mojette {

// Sticky status word the kernels OR their error bits into (one per device:
// a __device__ variable exists once in every context that loads the library).
__device__ uint32_t g_status;

namespace {
thread_local int t_last_cuda = 0;
std::mutex g_status_mu;
std::map<int, uint32_t *> g_status_ptr;
}  // namespace

int record_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return 0;
    t_last_cuda = (int)e;
    return -EIO;
}

uint32_t *device_status_ptr(int *err)
{
    int device = 0;
    if ((*err = record_cuda(cudaGetDevice(&device)))) return nullptr;
    std::lock_guard<std::mutex> g(g_status_mu);
    auto it = g_status_ptr.find(device);
    if (it != g_status_ptr.end()) return it->second;
    void *p = nullptr;
    if ((*err = record_cuda(cudaGetSymbolAddress(&p, g_status)))) return nullptr;
    g_status_ptr[device] = (uint32_t *)p;
    return (uint32_t *)p;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Decode arguments of one schedule (everything but the buffers, steps and status).
static void fill_decode_args(const Plan &pl, const Schedule &sc, int64_t S, DecodeArgs *a)
{
    std::memset(a, 0, sizeof(*a));
    a->S = S;
    a->total = pl.total;
    a->P = pl.P;
    a->Q = sc.lines;
    a->sys = pl.systematic;
    a->Qd = pl.Q;
    a->known = sc.known;
    a->T = sc.T;
    a->fwd = sc.fwd;
    for (int l = 0; l < sc.lines; ++l) {
        a->lpos[l] = sc.lpos[l];
        a->pL[l] = sc.pL[l];
        a->pR[l] = sc.pR[l];
        a->split[l] = sc.split[l];
        a->srcL[l] = sc.srcL[l];
        a->srcR[l] = sc.srcR[l];
    }
    a->chunk_w = sc.chunk_w;
    for (int c = 0; c < kStreamChunks; ++c) {
        a->chunk_wait[c] = sc.chunk_wait[c];
        a->chunk_done[c] = sc.chunk_done[c];
    }
    a->scan2 = sc.scan2;
    for (int j = 0; j < 2; ++j) {
        a->scan_p[j] = sc.scan_p[j];
        a->scan_src[j] = sc.scan_src[j];
    }
    a->vander = sc.vander;
    a->van_E0 = sc.van_E0;
    a->van_L = sc.van_L;
    a->ring_R = sc.one_sided ? sc.ring_R : 0;
    a->ring_D = sc.ring_D;
    for (int l = 0; l < kMaxLines; ++l) a->ring_delta[l] = sc.ring_delta[l];
    for (int j = 0; j < kMaxLines; ++j) {
        a->van_q[j] = sc.van_q[j];
        a->van_base[j] = sc.van_base[j];
        a->van_lo[j] = sc.van_lo[j];
        a->van_hi[j] = sc.van_hi[j];
    }
}

// Erasure mask bits a plan defines: n projections, or for a systematic plan
// Q data lines then n projections.
static bool mask_in_range(const Plan &pl, uint32_t mask)
{
    const int bits = pl.systematic ? pl.Q + pl.n : pl.n;
    return bits >= 32 || (mask >> bits) == 0;
}

}  // namespace mojette

using namespace mojette;

extern "C" {

int mojette_plan(int P, int Q, const int *p, int n, mojette_plan_t *out)
{
    if (!out || !p) return -EINVAL;
    *out = nullptr;
    if (P < 1 || Q < 1 || n < 1 || n > kMaxProj) return -EINVAL;
    // keep every index of a stripe (and every bin offset) within int32
    if ((int64_t)P * Q > (1 << 26)) return -EINVAL;
    for (int i = 0; i < n; ++i) {
        if (p[i] > (1 << 20) || p[i] < -(1 << 20)) return -EINVAL;
        for (int k = i + 1; k < n; ++k)
            if (p[i] == p[k]) return -EINVAL;
    }
    Plan *pl = new (std::nothrow) Plan();
    if (!pl) return -ENOMEM;
    pl->P = P;
    pl->Q = Q;
    pl->n = n;
    int64_t t = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t ap = p[i] < 0 ? -(int64_t)p[i] : p[i];
        pl->p[i] = p[i];
        pl->B[i] = ap * (Q - 1) + P;                           // Eq. 2, q = 1
        pl->bmin[i] = -(int64_t)(P - 1) + (p[i] < 0 ? (int64_t)(Q - 1) * p[i] : 0);
        pl->off[i] = t;
        t += pl->B[i];
    }
    if (t > (int64_t)1 << 30) {
        delete pl;
        return -EINVAL;
    }
    pl->total = t;
    *out = reinterpret_cast<mojette_plan_t>(pl);
    return 0;
}

int mojette_plan_ex(int P, int Q, const int *p, int n, uint32_t flags, mojette_plan_t *out)
{
    if (!out) return -EINVAL;
    *out = nullptr;
    if (flags & ~(uint32_t)(MOJETTE_PLAN_TRIM_UNUSED | MOJETTE_PLAN_SYSTEMATIC)) return -EINVAL;
    if (flags & MOJETTE_PLAN_SYSTEMATIC) {
        // mask bits: Q data lines then n parity projections
        if ((flags & MOJETTE_PLAN_TRIM_UNUSED) || Q < 1 || n < 1 || Q + n > 32) return -EINVAL;
    }
    int err = mojette_plan(P, Q, p, n, out);
    if (err) return err;
    if (flags & MOJETTE_PLAN_SYSTEMATIC) reinterpret_cast<Plan *>(*out)->systematic = true;
    if (flags & MOJETTE_PLAN_TRIM_UNUSED) {
        if ((err = trim_unused_bins(*reinterpret_cast<Plan *>(*out)))) {
            mojette_plan_destroy(*out);
            *out = nullptr;
            return err;
        }
    }
    return 0;
}

int mojette_plan_bins(mojette_plan_t plan, int32_t *full_bin)
{
    if (!plan) return -EINVAL;
    Plan *pl = reinterpret_cast<Plan *>(plan);
    if (full_bin) {
        if (pl->trimmed) {
            std::copy(pl->full_bin.begin(), pl->full_bin.end(), full_bin);
        } else {
            for (int i = 0; i < pl->n; ++i)
                for (int64_t j = 0; j < pl->B[i]; ++j) full_bin[pl->off[i] + j] = (int32_t)j;
        }
    }
    return pl->trimmed ? 1 : 0;
}

int mojette_plan_config(mojette_plan_t plan, int32_t *get, const int32_t *set)
{
    if (!plan) return -EINVAL;
    Plan *pl = reinterpret_cast<Plan *>(plan);
    std::lock_guard<std::mutex> g(pl->mu);
    if (get) {
        get[0] = pl->tuned_dec ? 1 : 0;
        get[1] = pl->dec_cfg.kernel;
        get[2] = pl->dec_cfg.gpc;
        get[3] = pl->dec_cfg.persist;
        get[4] = pl->dec_cfg.rowoff;
        get[5] = pl->tuned_enc ? 1 : 0;
        get[6] = pl->enc_cfg.tile_bytes;
        get[7] = 0;
    }
    if (set) {
        if (set[0]) {
            if (set[1] < 0 || set[1] > 6 || set[2] < 1 || set[2] > 64 || (set[3] & ~1) || (set[4] & ~1))
                return -EINVAL;
            if (set[1] == 5 && (pl->systematic || pl->trimmed || pl->Q < 2)) return -EINVAL;
            if (set[1] == 6 && pl->systematic) return -EINVAL;
            if (set[1] != 1 && pl->Q > 8) return -EINVAL;
            if (set[1] == 4 && pl->Q != 2 && !pl->systematic) return -EINVAL;
            pl->dec_cfg.kernel = set[1];
            pl->dec_cfg.gpc = set[2];
            pl->dec_cfg.persist = set[3];
            pl->dec_cfg.rowoff = set[4];
        }
        pl->tuned_dec = set[0] != 0;
        if (set[5] && set[6] < 0) return -EINVAL;
        if (set[5]) pl->enc_cfg.tile_bytes = set[6];
        pl->tuned_enc = set[5] != 0;
    }
    return 0;
}

int mojette_plan_destroy(mojette_plan_t plan)
{
    if (!plan) return 0;
    Plan *pl = reinterpret_cast<Plan *>(plan);
    int cur = 0;
    const bool have_device = cudaGetDevice(&cur) == cudaSuccess;
    for (auto &kv : pl->schedules)
        for (auto &d : kv.second->dev) {
            if (have_device && cudaSetDevice(d.first) == cudaSuccess) cudaFree(d.second);
        }
    for (auto &d : pl->full_bin_dev)
        if (have_device && cudaSetDevice(d.first) == cudaSuccess) cudaFree(d.second);
    if (have_device) cudaSetDevice(cur);
    delete pl;
    return 0;
}

int mojette_plan_info(mojette_plan_t plan, int64_t *bins, int64_t *offsets, int64_t *total)
{
    if (!plan) return -EINVAL;
    Plan *pl = reinterpret_cast<Plan *>(plan);
    for (int i = 0; i < pl->n; ++i) {
        if (bins) bins[i] = pl->B[i];
        if (offsets) offsets[i] = pl->off[i];
    }
    if (total) *total = pl->total;
    return 0;
}

int mojette_encode(mojette_plan_t plan, const uint64_t *d_img, uint64_t *d_proj,
                   int64_t S, mojette_stream_t stream)
{
    if (!plan || S < 0) return -EINVAL;
    if (S == 0) return 0;
    if (!d_img || !d_proj) return -EINVAL;
    if (!aligned16(d_img) || !aligned16(d_proj)) return -ERANGE;
    Plan *pl = reinterpret_cast<Plan *>(plan);
    int err = 0;
    EncodeArgs a{};
    a.img = d_img;
    a.proj = d_proj;
    a.S = S;
    a.total = pl->total;
    a.P = pl->P;
    a.Q = pl->Q;
    a.n = pl->n;
    for (int i = 0; i < pl->n; ++i) {
        a.p[i] = pl->p[i];
        a.off[i] = pl->off[i];
        a.bmin[i] = pl->bmin[i];
    }
    a.status = device_status_ptr(&err);
    if (err) return err;
    if ((err = plan_full_bin_on_device(*pl, &a.full_bin))) return err;
    return launch_encode(a, (cudaStream_t)stream);
}

int mojette_decode(mojette_plan_t plan, const uint64_t *d_proj, uint32_t erasure_mask,
                   uint64_t *d_img, int64_t S, mojette_stream_t stream)
{
    if (!plan || S < 0) return -EINVAL;
    Plan *pl = reinterpret_cast<Plan *>(plan);
    if (pl->Q > kMaxLines || pl->systematic) return -EINVAL;
    if (!mask_in_range(*pl, erasure_mask)) return -EINVAL;   // bits beyond n
    int err = 0;
    Schedule *sc = get_schedule(*pl, erasure_mask, &err);
    if (!sc) return err;
    if (S == 0) return 0;
    if (!d_img || !d_proj) return -EINVAL;
    if (!aligned16(d_img) || !aligned16(d_proj)) return -ERANGE;
    // decode_ring runs the mask's one-sided path, where it fits a ring
    if (choose_decode_kernel(pl->P, sc->lines, S, false, sc->scan2, sc->vander, true) == 7) {
        int e2 = 0;
        Schedule *rs = get_ring_schedule(*pl, erasure_mask, &e2);
        if (rs && rs->ring_R > 0) sc = rs;
    }
    uint32_t *dsteps = nullptr;
    if ((err = schedule_on_device(*pl, *sc, &dsteps))) return err;
    DecodeArgs a;
    fill_decode_args(*pl, *sc, S, &a);
    a.proj = d_proj;
    a.img = d_img;
    a.steps = dsteps;
    const int32_t *ph = S >= kPhaseMinStripes ? schedule_row_phases(*pl, *sc) : nullptr;
    for (int l = 0; l < kMaxLines; ++l) a.rowoff[l] = ph ? ph[l] : sc->rowpar[l];
    for (int f = 0; f < 2 * kMaxLines; ++f) a.order[f] = ph ? sc->order[f] : kIdentityOrder;
    a.status = device_status_ptr(&err);
    if (err) return err;
    return launch_decode(a, (cudaStream_t)stream);
}

int mojette_stage_survivors(mojette_plan_t plan, const uint64_t *h_proj, uint32_t erasure_mask,
                            uint64_t *d_proj, int64_t S, mojette_stream_t stream, int64_t *bytes)
{
    if (bytes) *bytes = 0;
    if (!plan || S < 0) return -EINVAL;
    Plan *pl = reinterpret_cast<Plan *>(plan);
    if (pl->systematic || pl->Q > kMaxLines) return -EINVAL;
    if (!mask_in_range(*pl, erasure_mask)) return -EINVAL;
    int err = 0;
    Schedule *sc = get_schedule(*pl, erasure_mask, &err);
    if (!sc) return err;
    if (S == 0) return 0;
    if (!h_proj || !d_proj) return -EINVAL;
    // the projections the path dedicates to a line, from either end
    uint32_t used = 0;
    for (int l = 0; l < sc->lines; ++l) used |= (1u << sc->projL[l]) | (1u << sc->projR[l]);
    const size_t pitch = (size_t)pl->total * sizeof(uint64_t);
    int64_t moved = 0;
    for (int i = 0; i < pl->n; ++i) {
        if (!(used >> i & 1u) || pl->B[i] == 0) continue;
        const size_t width = (size_t)pl->B[i] * sizeof(uint64_t);
        if ((err = record_cuda(cudaMemcpy2DAsync(d_proj + pl->off[i], pitch, h_proj + pl->off[i], pitch, width,
                                                 (size_t)S, cudaMemcpyHostToDevice, (cudaStream_t)stream))))
            return err;
        moved += (int64_t)width * S;
    }
    if (bytes) *bytes = moved;
    return 0;
}

int mojette_sys_decode(mojette_plan_t plan, const uint64_t *d_parity, uint32_t erasure_mask,
                       uint64_t *d_data, int64_t S, mojette_stream_t stream)
{
    if (!plan || S < 0) return -EINVAL;
    Plan *pl = reinterpret_cast<Plan *>(plan);
    if (!pl->systematic || pl->Q > kMaxLines) return -EINVAL;
    if (!mask_in_range(*pl, erasure_mask)) return -EINVAL;
    int err = 0;
    Schedule *sc = get_schedule(*pl, erasure_mask, &err);
    if (!sc) return err;
    if (S == 0 || sc->lines == 0) return 0;     // no data line lost: nothing to do
    if (!d_data || !d_parity) return -EINVAL;
    if (!aligned16(d_data) || !aligned16(d_parity)) return -ERANGE;
    uint32_t *dsteps = nullptr;
    if ((err = schedule_on_device(*pl, *sc, &dsteps))) return err;
    DecodeArgs a;
    fill_decode_args(*pl, *sc, S, &a);
    a.proj = d_parity;
    a.img = d_data;
    a.steps = dsteps;
    const int32_t *ph = S >= kPhaseMinStripes ? schedule_row_phases(*pl, *sc) : nullptr;
    for (int l = 0; l < kMaxLines; ++l) a.rowoff[l] = ph ? ph[l] : sc->rowpar[l];
    for (int f = 0; f < 2 * kMaxLines; ++f) a.order[f] = ph ? sc->order[f] : kIdentityOrder;
    a.status = device_status_ptr(&err);
    if (err) return err;
    return launch_decode(a, (cudaStream_t)stream);
}

int mojette_decode_noalloc(mojette_plan_t plan, const uint64_t *d_proj, uint32_t erasure_mask,
                           uint64_t *d_img, int64_t S, mojette_stream_t stream)
{
    if (!plan || S < 0) return -EINVAL;
    Plan *pl = reinterpret_cast<Plan *>(plan);
    if (pl->Q > kMaxLines || pl->systematic) return -EINVAL;
    if (!mask_in_range(*pl, erasure_mask)) return -EINVAL;
    int err = 0;
    Schedule *sc = get_schedule(*pl, erasure_mask, &err);   // host memory only
    if (!sc) return err;
    if (sc->T > kNoAllocMaxSteps) return -ENOSPC;
    if (S == 0) return 0;
    if (!d_img || !d_proj) return -EINVAL;
    if (!aligned16(d_img) || !aligned16(d_proj)) return -ERANGE;
    uint32_t *dsteps = nullptr;
    if ((err = noalloc_schedule_copy(*sc, (cudaStream_t)stream, &dsteps))) return err;
    DecodeArgs a;
    fill_decode_args(*pl, *sc, S, &a);
    a.proj = d_proj;
    a.img = d_img;
    a.steps = dsteps;
    const int32_t *ph = S >= kPhaseMinStripes ? schedule_row_phases(*pl, *sc) : nullptr;
    for (int l = 0; l < kMaxLines; ++l) a.rowoff[l] = ph ? ph[l] : sc->rowpar[l];
    for (int f = 0; f < 2 * kMaxLines; ++f) a.order[f] = ph ? sc->order[f] : kIdentityOrder;
    a.status = device_status_ptr(&err);
    if (err) return err;
    return launch_decode(a, (cudaStream_t)stream);
}

int mojette_decode_kernel(mojette_plan_t plan, uint32_t erasure_mask, int64_t S, int32_t *kernel)
{
    if (!plan || !kernel || S < 0) return -EINVAL;
    Plan *pl = reinterpret_cast<Plan *>(plan);
    if (pl->Q > kMaxLines) return -EINVAL;
    if (!mask_in_range(*pl, erasure_mask)) return -EINVAL;
    int err = 0;
    Schedule *sc = get_schedule(*pl, erasure_mask, &err);
    if (!sc) return err;
    if (sc->lines == 0) {
        *kernel = -1;                       // systematic, nothing lost: no launch
        return 0;
    }
    *kernel = choose_decode_kernel(pl->P, sc->lines, S, pl->systematic, sc->scan2, sc->vander, true);
    if (*kernel == 7) {
        int e2 = 0;
        Schedule *rs = get_ring_schedule(*pl, erasure_mask, &e2);
        if (!rs || rs->ring_R == 0 || pl->P % kRingChunk) *kernel = 0;   // no ring fits: decode_lines
    }
    return 0;
}

int mojette_schedule(mojette_plan_t plan, uint32_t erasure_mask, int32_t *survivors,
                     int32_t *survivors2, int32_t *split, uint32_t *steps,
                     uint32_t *forward, int64_t max_steps, int64_t *n_steps)
{
    if (!plan) return -EINVAL;
    Plan *pl = reinterpret_cast<Plan *>(plan);
    if (pl->Q > kMaxLines) return -EINVAL;
    if (!mask_in_range(*pl, erasure_mask)) return -EINVAL;
    int err = 0;
    Schedule *sc = get_schedule(*pl, erasure_mask, &err);
    if (!sc) return err;
    for (int l = 0; l < sc->lines; ++l) {
        if (survivors) survivors[l] = sc->projL[l];
        if (survivors2) survivors2[l] = sc->projR[l];
        if (split) split[l] = sc->split[l];
    }
    for (int64_t t = 0; t < sc->T && t < max_steps; ++t) {
        if (steps) steps[t] = sc->steps[(size_t)t];
        if (forward) forward[t] = sc->fwdw[(size_t)t];
    }
    if (n_steps) *n_steps = sc->T;
    return 0;
}

int mojette_schedule_layout(mojette_plan_t plan, uint32_t erasure_mask, int32_t *row_phase,
                            uint32_t *load_order)
{
    if (!plan) return -EINVAL;
    Plan *pl = reinterpret_cast<Plan *>(plan);
    if (pl->Q > kMaxLines) return -EINVAL;
    if (!mask_in_range(*pl, erasure_mask)) return -EINVAL;
    int err = 0;
    Schedule *sc = get_schedule(*pl, erasure_mask, &err);
    if (!sc) return err;
    // the search runs once per path and is kept with it; once done, the
    // phases and orders never change
    const int32_t *ph = schedule_row_phases(*pl, *sc);
    for (int l = 0; l < sc->lines; ++l) {
        if (row_phase) row_phase[l] = ph[l];
        if (load_order) {
            load_order[2 * l] = sc->order[2 * l];
            load_order[2 * l + 1] = sc->order[2 * l + 1];
        }
    }
    return 0;
}

int mojette_device_status(uint32_t *flags, int clear)
{
    int err = 0;
    uint32_t *d = device_status_ptr(&err);
    if (!d) return err;
    if ((err = record_cuda(cudaDeviceSynchronize()))) return err;
    uint32_t h = 0;
    if ((err = record_cuda(cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost)))) return err;
    if (clear && (err = record_cuda(cudaMemset(d, 0, sizeof(h))))) return err;
    if (flags) *flags = h;
    return (h & kStatusWaitTimeout) ? -ETIMEDOUT : 0;
}

const char *mojette_strerror(int status)
{
    switch (status) {
    case 0: return "success";
    case -EINVAL: return "invalid argument or geometry";
    case -ERANGE: return "device pointer not 16-byte aligned";
    case -ENOTRECOVERABLE: return "surviving projections cannot rebuild the image";
    case -ENOMEM: return "out of memory";
    case -EIO: return "CUDA runtime error (see mojette_last_cuda_error)";
    case -ETIMEDOUT: return "a bounded device-side wait expired";
    case -ENOSPC: return "schedule larger than the fixed scratch of mojette_decode_noalloc";
    default: return "unknown status";
    }
}

int mojette_last_cuda_error(void) { return t_last_cuda; }

}  // extern "C"
