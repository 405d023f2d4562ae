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
#include <algorithm>
#include <cerrno>

#include "ptx.cuh"

namespace mojette {
namespace {

constexpr int kEncThreads = 256;
constexpr int kEncStages = 3;
constexpr int kEncTileBytes = 16384;

struct EncParams {
    const uint64_t *img;
    uint64_t *proj;
    int64_t S;
    int64_t ntiles;
    int total;
    int P, Q, n;
    int spt;      // stripes per tile
    int stages;   // tiles in flight per CTA (bulk path)
    int bulk;     // 1: TMA bulk copies; 0: 8-byte cp.async (odd Q*P)
    int32_t p[kMaxProj];
    int32_t off[kMaxProj];
    int32_t bmin[kMaxProj];
    uint32_t *status;
};

// XOR of the pixels on one discrete line: x = c + l p on line l.
template <int QT>
__device__ __forceinline__ uint64_t line_xor(const uint64_t *img, int Q, int P, int c, int p)
{
    uint64_t acc = 0;
    if (QT) {
#pragma unroll
        for (int l = 0; l < QT; ++l) {
            const int x = c + l * p;
            if ((unsigned)x < (unsigned)P) acc ^= img[l * P + x];
        }
    } else {
        for (int l = 0; l < Q; ++l) {
            const int x = c + l * p;
            if ((unsigned)x < (unsigned)P) acc ^= img[l * P + x];
        }
    }
    return acc;
}

template <int QT, int ITEMS>
__global__ void __launch_bounds__(kEncThreads)
encode_tiles(const __grid_constant__ EncParams a)
{
    extern __shared__ __align__(128) uint64_t sm[];
    const int Q = QT ? QT : a.Q;
    const int P = a.P;
    const int QP = Q * P;
    const int tileWords = a.spt * QP;
    uint64_t *bars = sm + (size_t)a.stages * tileWords;
    const int tid = threadIdx.x;

    // Output words t = tid + k * kEncThreads of every stripe: projection i
    // (the last with off_i <= t) and c = -(j + b_min_i).
    int c[ITEMS], pp[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const int t = tid + k * kEncThreads;
        int i = 0;
        for (int q = 1; q < a.n; ++q)
            if (a.off[q] <= t) i = q;
        c[k] = -(t - a.off[i]) - a.bmin[i];
        pp[k] = a.p[i];
    }

    auto compute = [&](const uint64_t *buf, int64_t s0, int nst) {
        for (int s = 0; s < nst; ++s) {
            const uint64_t *img = buf + s * QP;
            uint64_t *out = a.proj + (s0 + s) * (int64_t)a.total;
#pragma unroll
            for (int k = 0; k < ITEMS; ++k) {
                const int t = tid + k * kEncThreads;
                if (t < a.total) __stcs(out + t, line_xor<QT>(img, Q, P, c[k], pp[k]));
            }
        }
    };

    if (!a.bulk) {
        // Unaligned tiles (odd Q*P): 8-byte asynchronous copies, one tile at a time.
        for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
            const int64_t s0 = tile * a.spt;
            const int nst = (int)min64(a.spt, a.S - s0);
            const uint64_t *src = a.img + s0 * QP;
            for (int w = tid; w < nst * QP; w += kEncThreads) cp_async8(sm + w, src + w);
            cp_async_wait_all();
            __syncthreads();
            compute(sm, s0, nst);
            __syncthreads();
        }
        return;
    }

    if (tid == 0) {
        for (int s = 0; s < a.stages; ++s) mbar_init(smem_addr(bars + s), 1);
        mbar_init_fence();
    }
    __syncthreads();

    auto issue = [&](int64_t tile, int stage) {
        const int64_t s0 = tile * a.spt;
        const int nst = (int)min64(a.spt, a.S - s0);
        const uint32_t bytes = (uint32_t)nst * (uint32_t)QP * 8u;
        const uint32_t bar = smem_addr(bars + stage);
        mbar_arrive_expect_tx(bar, bytes);
        tma_load_1d(smem_addr(sm + (size_t)stage * tileWords), a.img + s0 * QP, bytes, bar);
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
        compute(sm + (size_t)stage * tileWords, s0, (int)min64(a.spt, a.S - s0));
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
__global__ void __launch_bounds__(256) encode_direct(const __grid_constant__ EncParams a)
{
    const int64_t QP = (int64_t)a.Q * a.P;
    const int64_t nwords = a.S * (int64_t)a.total;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nwords;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = g / a.total;
        const int t = (int)(g - s * a.total);
        int i = 0;
        for (int q = 1; q < a.n; ++q)
            if (a.off[q] <= t) i = q;
        const int c = -(t - a.off[i]) - a.bmin[i];
        const uint64_t *img = a.img + s * QP;
        uint64_t acc = 0;
        for (int l = 0; l < a.Q; ++l) {
            const int x = c + l * a.p[i];
            if ((unsigned)x < (unsigned)a.P) acc ^= img[(int64_t)l * a.P + x];
        }
        a.proj[g] = acc;
    }
}

using EncKernel = void (*)(const EncParams);

template <int QT>
EncKernel pick_items(int items)
{
    switch (items) {
    case 2: return encode_tiles<QT, 2>;
    case 4: return encode_tiles<QT, 4>;
    case 8: return encode_tiles<QT, 8>;
    case 16: return encode_tiles<QT, 16>;
    default: return nullptr;
    }
}

EncKernel pick_kernel(int Q, int items)
{
    switch (Q) {
    case 2: return pick_items<2>(items);
    case 4: return pick_items<4>(items);
    case 8: return pick_items<8>(items);
    default: return pick_items<0>(items);
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

}  // namespace

int launch_encode(const EncodeArgs &e, cudaStream_t st)
{
    EncParams a;
    a.img = e.img;
    a.proj = e.proj;
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

    const int64_t QP = (int64_t)e.Q * e.P;
    const int64_t stripe_bytes = QP * 8;
    const int64_t need = (e.total + kEncThreads - 1) / kEncThreads;
    const int items = need <= 2 ? 2 : need <= 4 ? 4 : need <= 8 ? 8 : need <= 16 ? 16 : 0;
    a.bulk = (QP % 2 == 0) ? 1 : 0;
    a.spt = (int)std::max<int64_t>(1, kEncTileBytes / stripe_bytes);
    a.stages = a.bulk ? kEncStages : 1;
    auto smem_of = [&](void) {
        return (int64_t)a.stages * a.spt * stripe_bytes + (a.bulk ? 8 * a.stages : 0);
    };
    while (a.bulk && a.stages > 1 && smem_of() > smem_cap) --a.stages;
    EncKernel fn = items ? pick_kernel(e.Q, items) : nullptr;
    if (smem_of() > smem_cap) fn = nullptr;

    if (!fn) {
        const int64_t nwords = e.S * e.total;
        const int64_t blocks = std::min<int64_t>((nwords + 255) / 256, (int64_t)sms * 16);
        encode_direct<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(a);
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

}  // namespace mojette
