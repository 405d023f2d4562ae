// Forward Mojette transform (encode), Sec. 2.1 Eq. 1 with XOR addition (Sec. 3).
//
// Bin b of projection (p, 1) is the XOR of the pixels f(x, l) with
// b = l p - x. Stored at j = b - b_min, so bin j of projection i collects
// pixel x = c + l p_i of every line l, with c = -(j + b_min_i), wherever
// 0 <= x < P: at most Q pixels, at most Q - 1 XORs (Sec. 3).
//
// GB300 design: the kernel is HBM-bound (every stripe is read once and its
// sum_i B_i bins written once; about 0.1 XOR per byte). Persistent CTAs walk
// tiles of whole stripes. Each tile arrives in shared memory by one 1-D TMA
// bulk copy (cp.async.bulk, completion on an mbarrier), several tiles in
// flight per CTA. Threads own fixed output words of the stripe (their
// (c, p) pairs live in registers for the whole kernel) and gather the
// pixels of each bin from shared memory, so the odd l p shifts never touch
// global addressing: global loads are whole-tile bulk copies and global
// stores are consecutive 8-byte words across the warp.
//
// Every kernel comes in two forms: plain (stripes back to back at fixed
// strides) and batched (stripe s read from srcp[s], its bins written to
// dstp[s]: stripes anywhere in memory, one launch per geometry).
#pragma once

#include <algorithm>
#include <cerrno>
#include <cstdlib>

#include "ptx.cuh"

namespace mojette {
namespace {

constexpr int kEncThreads = 256;
constexpr int kEncStages = 3;
// Target bytes of a tile (measured on GB300: one stripe per tile is best at
// Q <= 4, about two at Q = 8).
constexpr int kEncTileBytesNarrow = 9000;
constexpr int kEncTileBytesWide = 24000;

struct EncParams {
    const int32_t *full_bin;        // trimmed plan: full bin index of each stored word, else null
    const uint64_t *img;            // plain: stripe s at img + s * Q * P
    uint64_t *proj;                 // plain: its bins at proj + s * total
    const uint64_t *const *srcp;    // batched: stripe s at srcp[s]
    uint64_t *const *dstp;          //   its bins at dstp[s]
    int64_t S;
    int64_t ntiles;
    int total;
    int P, Q, n;
    int pad;      // zero words before, between and after the rows of a stripe
    int RP;       // row pitch in shared memory: P + pad (even when bulk)
    int SWs;      // shared words per stripe: Q * RP + pad
    int spt;      // stripes per tile
    int stages;   // tiles in flight per CTA (bulk path)
    int bulk;     // 1: one TMA bulk copy per row (P even); 0: 8-byte cp.async
    int align;    // output slots of a projection start on a multiple of this
    int32_t p[kMaxProj];
    int32_t off[kMaxProj];
    int32_t bmin[kMaxProj];
    uint32_t *status;
};

// Bin (c, p) of a stripe staged at byte address `a0` (its row 0, column c)
// collects the word at a0 + l * stepc on every line l; pixels outside the
// image read the zero pad columns.
template <int QT>
__device__ __forceinline__ uint64_t line_xor(const char *sbase, uint32_t a0, int stepc, int Q)
{
    uint64_t acc = 0;
    if (QT) {
#pragma unroll
        for (int l = 0; l < QT; ++l) acc ^= *reinterpret_cast<const uint64_t *>(sbase + a0 + l * stepc);
    } else {
        for (int l = 0; l < Q; ++l) acc ^= *reinterpret_cast<const uint64_t *>(sbase + a0 + l * stepc);
    }
    return acc;
}

// Address of stripe s's pixels and of its bins.
template <bool BATCHED>
__device__ __forceinline__ const uint64_t *stripe_in(const EncParams &a, int64_t s)
{
    if constexpr (BATCHED) return a.srcp[s];
    else return a.img + s * (int64_t)a.Q * a.P;
}
template <bool BATCHED>
__device__ __forceinline__ uint64_t *stripe_out(const EncParams &a, int64_t s)
{
    if constexpr (BATCHED) return a.dstp[s];
    else return a.proj + s * (int64_t)a.total;
}

template <int QT, int ITEMS, bool BATCHED>
__global__ void __launch_bounds__(kEncThreads, 2)
encode_tiles(const __grid_constant__ EncParams a)
{
    extern __shared__ __align__(128) uint64_t sm[];
    const int Q = QT ? QT : a.Q;
    const int P = a.P, RP = a.RP, SWs = a.SWs;
    const int tileWords = a.spt * SWs;
    uint64_t *bars = sm + (size_t)a.stages * tileWords;
    const int tid = threadIdx.x;
    const char *sbase = reinterpret_cast<const char *>(sm);

    // zero every pad column of every stage once; rows are always staged
    // before they are read, pads never written
    for (int st = 0; st < a.stages; ++st)
        for (int s = 0; s < a.spt; ++s) {
            uint64_t *w = sm + (size_t)st * tileWords + (size_t)s * SWs;
            for (int l = 0; l <= Q; ++l)
                for (int i = tid; i < a.pad; i += kEncThreads) w[l * RP + i] = 0;
        }

    // Output slots v = tid + k * kEncThreads: projection i's stored words
    // take slots [voff_i, voff_i + B_i), every projection starting on a
    // multiple of `align` slots: with align = 16 the 16 lanes of a half-warp
    // always gather consecutive bins of one projection (consecutive words of
    // every row: no bank conflicts) and store consecutive words; align = 1
    // packs the slots (fewer idle lanes; measured better at Q <= 4). Slot v holds
    // stored word t = off_i + (v - voff_i) (t = -1: an idle slot); the bin's
    // pixel on line l sits at column c + l p_i with c = -(j + b_min_i), i.e.
    // at byte a0 + l * stepc.
    uint32_t a0[ITEMS];
    int stepc[ITEMS], tw[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const int v = tid + k * kEncThreads;
        int i = -1, vo = 0;   // vo: the first slot of projection i
        for (int q = 0; q < a.n; ++q) {
            const int B = (q + 1 < a.n ? a.off[q + 1] : a.total) - a.off[q];
            if (v >= vo && v < vo + B) {
                i = q;
                break;
            }
            vo += (B + a.align - 1) / a.align * a.align;
        }
        int t = -1, j = 0, c = 0, p = 0;
        if (i >= 0) {
            t = a.off[i] + (v - vo);
            j = a.full_bin ? a.full_bin[t] : t - a.off[i];
            c = -j - a.bmin[i];
            p = a.p[i];
        }
        tw[k] = t;
        a0[k] = (uint32_t)((a.pad + c) * 8);
        stepc[k] = (RP + p) * 8;
    }
    __syncthreads();

    auto compute = [&](int stage, int64_t s0, int nst) {
        for (int s = 0; s < nst; ++s) {
            const uint32_t sb = (uint32_t)(((size_t)stage * tileWords + (size_t)s * SWs) * 8);
            uint64_t *out = stripe_out<BATCHED>(a, s0 + s);
#pragma unroll
            for (int k = 0; k < ITEMS; ++k)
                if (tw[k] >= 0) __stcs(out + tw[k], line_xor<QT>(sbase, sb + a0[k], stepc[k], Q));
        }
    };

    if (!a.bulk) {
        // odd P: 8-byte asynchronous copies into the padded rows, one tile at a time
        for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
            const int64_t s0 = tile * a.spt;
            const int nst = (int)min64(a.spt, a.S - s0);
            for (int w = tid; w < nst * Q * P; w += kEncThreads) {
                const int s = w / (Q * P), r = w - s * Q * P, l = r / P, x = r - l * P;
                cp_async8(sm + (size_t)s * SWs + a.pad + l * RP + x, stripe_in<BATCHED>(a, s0 + s) + r);
            }
            cp_async_wait_all();
            __syncthreads();
            compute(0, s0, nst);
            __syncthreads();
        }
        return;
    }

    if (tid == 0) {
        for (int s = 0; s < a.stages; ++s) mbar_init(smem_addr(bars + s), 1);
        mbar_init_fence();
    }
    __syncthreads();

    // One bulk copy per row of every stripe of the tile, all completing on
    // the stage's mbarrier.
    auto issue = [&](int64_t tile, int stage) {
        const int64_t s0 = tile * a.spt;
        const int nst = (int)min64(a.spt, a.S - s0);
        const uint32_t bar = smem_addr(bars + stage);
        mbar_arrive_expect_tx(bar, (uint32_t)nst * (uint32_t)Q * (uint32_t)P * 8u);
        for (int s = 0; s < nst; ++s) {
            const uint64_t *in = stripe_in<BATCHED>(a, s0 + s);
            for (int l = 0; l < Q; ++l)
                tma_load_1d(smem_addr(sm + (size_t)stage * tileWords + (size_t)s * SWs + a.pad + l * RP),
                            in + (int64_t)l * P, (uint32_t)P * 8u, bar);
        }
    };

    int64_t issued = 0;   // tiles issued by thread 0 (counted in this CTA's order)
    if (tid == 0)
        for (int s = 0; s < a.stages; ++s) {
            if ((int64_t)blockIdx.x + (int64_t)s * gridDim.x >= a.ntiles) break;
            issue(blockIdx.x + (int64_t)s * gridDim.x, s);
            ++issued;
        }

    int64_t k = 0;
    bool timed_out = false;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++k) {
        const int stage = (int)(k % a.stages);
        const uint32_t parity = (uint32_t)((k / a.stages) & 1);
        const bool ok = mbar_wait_bounded(smem_addr(bars + stage), parity);
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        // Every thread is past tile k-1: refill its stage with tile k-1+stages.
        if (tid == 0 && k > 0) {
            const int64_t nxt = tile + (int64_t)(a.stages - 1) * gridDim.x;
            if (nxt < a.ntiles) {
                issue(nxt, (int)((k - 1) % a.stages));
                ++issued;
            }
        }
        const int64_t s0 = tile * a.spt;
        compute(stage, s0, (int)min64(a.spt, a.S - s0));
    }
    if (timed_out && tid == 0) {
        atomicOr(a.status, kStatusWaitTimeout);
        // let the copies still in flight land before the CTA's shared memory goes away
        for (int64_t q = k; q < issued; ++q)
            mbar_wait_bounded(smem_addr(bars + (q % a.stages)), (uint32_t)((q / a.stages) & 1));
    }
}

// Stripes too large to stage in shared memory: one thread per bin, pixels
// read straight from global memory.
template <bool BATCHED>
__global__ void __launch_bounds__(256) encode_direct(const __grid_constant__ EncParams a)
{
    const int64_t nwords = a.S * (int64_t)a.total;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nwords;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = g / a.total;
        const int t = (int)(g - s * a.total);
        int i = 0;
        for (int q = 1; q < a.n; ++q)
            if (a.off[q] <= t) i = q;
        const int j = a.full_bin ? a.full_bin[t] : t - a.off[i];
        const int c = -j - a.bmin[i];
        const uint64_t *img = stripe_in<BATCHED>(a, s);
        uint64_t acc = 0;
        for (int l = 0; l < a.Q; ++l) {
            const int x = c + l * a.p[i];
            if ((unsigned)x < (unsigned)a.P) acc ^= img[(int64_t)l * a.P + x];
        }
        stripe_out<BATCHED>(a, s)[t] = acc;
    }
}

using EncKernel = void (*)(const EncParams);

template <int QT, bool BATCHED>
EncKernel pick_items(int items)
{
    switch (items) {
    case 2: return encode_tiles<QT, 2, BATCHED>;
    case 4: return encode_tiles<QT, 4, BATCHED>;
    case 8: return encode_tiles<QT, 8, BATCHED>;
    case 16: return encode_tiles<QT, 16, BATCHED>;
    default: return nullptr;
    }
}

template <bool BATCHED>
EncKernel pick_kernel(int Q, int items)
{
    switch (Q) {
    case 2: return pick_items<2, BATCHED>(items);
    case 4: return pick_items<4, BATCHED>(items);
    case 8: return pick_items<8, BATCHED>(items);
    default: return pick_items<0, BATCHED>(items);
    }
}

int device_sms(int *err)
{
    int dev = 0, sms = 0;
    if ((*err = record_cuda(cudaGetDevice(&dev)))) return 0;
    if ((*err = record_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))))
        return 0;
    return sms;
}

int max_dyn_smem(int *err)
{
    int dev = 0, v = 0;
    if ((*err = record_cuda(cudaGetDevice(&dev)))) return 0;
    if ((*err = record_cuda(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))))
        return 0;
    return v;
}

// Launch encode over e.S stripes (plain: img/proj; batched: srcp/dstp).
template <bool BATCHED>
int launch_encode_impl(const EncodeArgs &e, cudaStream_t st)
{
    EncParams a;
    a.full_bin = e.full_bin;
    a.img = e.img;
    a.proj = e.proj;
    a.srcp = e.srcp;
    a.dstp = e.dstp;
    a.S = e.S;
    a.total = (int)e.total;
    a.P = e.P;
    a.Q = e.Q;
    a.n = e.n;
    for (int i = 0; i < e.n; ++i) {
        a.p[i] = e.p[i];
        a.off[i] = (int32_t)e.off[i];
        a.bmin[i] = (int32_t)e.bmin[i];
    }
    a.status = e.status;

    int err = 0;
    const int sms = device_sms(&err);
    if (err) return err;
    const int smem_cap = max_dyn_smem(&err);
    if (err) return err;

    int maxp = 0;
    for (int i = 0; i < e.n; ++i) maxp = std::max(maxp, e.p[i] < 0 ? -e.p[i] : e.p[i]);
    // output slots: every projection's words from a multiple of `align`
    // (16 at Q >= 8, where a half-warp spanning two projections costs bank
    // conflicts: 1.100 -> 1.067 ms at 8 KB (12,8), 0.727 -> 0.700 ms at
    // 4 KB; 1 below, where the idle lanes cost more)
    a.align = e.Q >= 8 ? 16 : 1;
    int64_t slots = 0;
    for (int i = 0; i < e.n; ++i) {
        const int64_t B = (i + 1 < e.n ? e.off[i + 1] : e.total) - e.off[i];
        slots += (B + a.align - 1) / a.align * a.align;
    }
    const int64_t need = (slots + kEncThreads - 1) / kEncThreads;
    const int items = need <= 2 ? 2 : need <= 4 ? 4 : need <= 8 ? 8 : need <= 16 ? 16 : 0;
    a.bulk = (e.P % 2 == 0) ? 1 : 0;
    // Zero columns around the rows cover every offset l p of a bin line, so
    // no bounds test sits in the inner loop; with bulk copies the pad and row
    // pitch are even so that every row starts 16-byte aligned.
    a.pad = (e.Q - 1) * maxp;
    if (a.bulk && a.pad % 2) ++a.pad;
    a.RP = e.P + a.pad;
    a.SWs = e.Q * a.RP + a.pad;
    const int64_t stripe_bytes = (int64_t)a.SWs * 8;
    int64_t tile_bytes = e.Q <= 4 ? kEncTileBytesNarrow : kEncTileBytesWide;
    if (e.tile_bytes > 0) tile_bytes = e.tile_bytes;
    else if (const char *env = getenv("MOJETTE_ENCODE_TILE")) tile_bytes = std::max(1, atoi(env));   // tuning
    a.spt = (int)std::max<int64_t>(1, tile_bytes / stripe_bytes);
    a.stages = a.bulk ? kEncStages : 1;
    auto smem_of = [&](void) {
        return (int64_t)a.stages * a.spt * stripe_bytes + (a.bulk ? 8 * a.stages : 0);
    };
    while (a.bulk && a.stages > 1 && smem_of() > smem_cap) --a.stages;
    EncKernel fn = items ? pick_kernel<BATCHED>(e.Q, items) : nullptr;
    if (smem_of() > smem_cap) fn = nullptr;

    if (!fn) {
        const int64_t nwords = e.S * e.total;
        const int64_t blocks = std::min<int64_t>((nwords + 255) / 256, (int64_t)sms * 16);
        encode_direct<BATCHED><<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(a);
        return record_cuda(cudaGetLastError());
    }

    a.ntiles = (e.S + a.spt - 1) / a.spt;
    const int smem = (int)smem_of();
    if ((err = record_cuda(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))))
        return err;
    int per_sm = 0;
    if ((err = record_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kEncThreads, smem))))
        return err;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(a.ntiles, (int64_t)std::max(per_sm, 1) * sms));
    fn<<<(unsigned)grid, kEncThreads, smem, st>>>(a);
    return record_cuda(cudaGetLastError());
}

}  // namespace
}  // namespace mojette
