// Inverse Mojette transform (decode), Sec. 2.2, along a pre-determined
// reconstruction path (one projection dedicated to each line, swept from
// both ends of the line; the path itself is built on the host, plan.cpp).
//
// Every pixel (l, x) is rebuilt in gather form: the bin of its dedicated
// projection (direction p) XOR the other pixels of that bin's discrete line,
// (l', x + (l' - l) p) for l' != l inside the image. The schedule
// guarantees those were rebuilt at earlier steps, so the result is the
// value the paper's "subtract its contribution from all projections"
// procedure reaches, at most Q - 1 XORs per pixel (Sec. 3).
//
// GB300 design: HBM-bound like encode, but with a sequential dependency
// along each line (about P steps). A warp holds 32/Q stripes and gives each
// (stripe, line) pair one lane, so a step rebuilds up to two pixels per lane
// with no divergence; steps are separated by __syncwarp only. The bins a
// stripe needs (exactly Q*P of them: pixel (l, x) uses one bin, at word
// src - x of the stripe's projection block) are staged into shared memory
// in pixel order by 8-byte cp.async copies -- coalesced, and the reversal
// of the bin order costs nothing -- and each rebuilt pixel overwrites its
// own bin in place, so a stripe needs Q*P words of shared memory. Rows
// have an odd pitch so that the lanes of different stripes at the same x
// fall in different banks. The finished image leaves as consecutive 8-byte
// stores. Many stripes per SM (one persistent CTA per SM, as many warps as
// shared memory holds) hide the per-step latency.
#include <algorithm>
#include <cerrno>

#include "ptx.cuh"

namespace mojette {
namespace {

struct DecParams {
    const uint64_t *proj;
    uint64_t *img;
    int64_t S;
    int64_t ngroups;
    int64_t total;
    int P, Q;
    int PP;       // shared-memory row pitch (odd)
    int G;        // stripes per warp
    int warps;    // warps per CTA
    int T;        // steps
    const uint32_t *steps;
    int32_t pL[kMaxLines], pR[kMaxLines], split[kMaxLines];
    int32_t srcL[kMaxLines], srcR[kMaxLines];
    uint32_t *status;
};

// Pixel (l, x) along direction p: its staged bin XOR the other pixels of
// the bin's line (all rebuilt at earlier steps).
template <int QT>
__device__ __forceinline__ uint64_t rebuild(const uint64_t *buf, int Q, int P, int PP, int l,
                                            int x, int p)
{
    uint64_t v = buf[l * PP + x];
    if (QT) {
#pragma unroll
        for (int l2 = 0; l2 < QT; ++l2) {
            const int x2 = x + (l2 - l) * p;
            if (l2 != l && (unsigned)x2 < (unsigned)P) v ^= buf[l2 * PP + x2];
        }
    } else {
        for (int l2 = 0; l2 < Q; ++l2) {
            const int x2 = x + (l2 - l) * p;
            if (l2 != l && (unsigned)x2 < (unsigned)P) v ^= buf[l2 * PP + x2];
        }
    }
    return v;
}

template <int QT>
__global__ void __launch_bounds__(1024) decode_lines(const __grid_constant__ DecParams a)
{
    extern __shared__ __align__(16) uint64_t sm[];
    const int Q = QT ? QT : a.Q;
    const int P = a.P, PP = a.PP, G = a.G;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int stripeWords = Q * PP;
    uint64_t *wbuf = sm + (size_t)warp * G * stripeWords;
    uint32_t *steps = reinterpret_cast<uint32_t *>(sm + (size_t)a.warps * G * stripeWords);
    for (int t = threadIdx.x; t < a.T; t += blockDim.x) steps[t] = a.steps[t];
    __syncthreads();

    const int g = lane / Q;
    const int l = lane - g * Q;
    const int pl = a.pL[l], pr = a.pR[l];
    uint64_t *mine = wbuf + g * stripeWords;

    for (int64_t grp = (int64_t)blockIdx.x * a.warps + warp; grp < a.ngroups;
         grp += (int64_t)gridDim.x * a.warps) {
        const int64_t s0 = grp * G;
        const int nst = (int)min64(G, a.S - s0);

        // stage the Q*P bins the path uses, in pixel order
        for (int gg = 0; gg < nst; ++gg) {
            const uint64_t *src = a.proj + (s0 + gg) * a.total;
            uint64_t *dst = wbuf + gg * stripeWords;
            for (int ll = 0; ll < Q; ++ll) {
                const int sp = a.split[ll];
                const int sl = a.srcL[ll], sr = a.srcR[ll];
                for (int x = lane; x < P; x += 32)
                    cp_async8(dst + ll * PP + x, src + ((x < sp ? sl : sr) - x));
            }
        }
        cp_async_wait_all();
        __syncwarp();

        // replay the path: bit 2l of step word t advances line l's left
        // front, bit 2l+1 its right front
        const bool work = g < nst;
        int xa = 0, xz = P - 1;
        uint32_t w = a.T > 0 ? steps[0] : 0u;
        for (int t = 0; t < a.T; ++t) {
            const uint32_t wn = (t + 1 < a.T) ? steps[t + 1] : 0u;
            const uint32_t bits = work ? (w >> (2 * l)) & 3u : 0u;
            uint64_t vl = 0, vr = 0;
            if (bits & 1u) vl = rebuild<QT>(mine, Q, P, PP, l, xa, pl);
            if (bits & 2u) vr = rebuild<QT>(mine, Q, P, PP, l, xz, pr);
            if (bits & 1u) mine[l * PP + xa++] = vl;
            if (bits & 2u) mine[l * PP + xz--] = vr;
            __syncwarp();
            w = wn;
        }

        // write the rebuilt image
        for (int gg = 0; gg < nst; ++gg) {
            uint64_t *out = a.img + (s0 + gg) * (int64_t)Q * P;
            const uint64_t *buf = wbuf + gg * stripeWords;
            for (int ll = 0; ll < Q; ++ll)
                for (int x = lane; x < P; x += 32) __stcs(out + ll * P + x, buf[ll * PP + x]);
        }
        __syncwarp();
    }
}

using DecKernel = void (*)(const DecParams);

DecKernel pick_kernel(int Q)
{
    switch (Q) {
    case 2: return decode_lines<2>;
    case 4: return decode_lines<4>;
    case 8: return decode_lines<8>;
    default: return decode_lines<0>;
    }
}

}  // namespace

int launch_decode(const DecodeArgs &d, cudaStream_t st)
{
    DecParams a;
    a.proj = d.proj;
    a.img = d.img;
    a.S = d.S;
    a.total = d.total;
    a.P = d.P;
    a.Q = d.Q;
    a.T = d.T;
    a.steps = d.steps;
    for (int l = 0; l < d.Q; ++l) {
        a.pL[l] = d.pL[l];
        a.pR[l] = d.pR[l];
        a.split[l] = d.split[l];
        a.srcL[l] = (int32_t)d.srcL[l];
        a.srcR[l] = (int32_t)d.srcR[l];
    }
    a.status = d.status;

    int err = 0, dev = 0, sms = 0, cap = 0;
    if ((err = record_cuda(cudaGetDevice(&dev)))) return err;
    if ((err = record_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))) return err;
    if ((err = record_cuda(cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))))
        return err;

    a.PP = (d.P % 2 == 0) ? d.P + 1 : d.P;
    const int64_t steps_bytes = ((int64_t)d.T * 4 + 15) / 16 * 16;
    int G = 32 / d.Q;
    int64_t warp_bytes = (int64_t)G * d.Q * a.PP * 8;
    while (G > 1 && warp_bytes + steps_bytes > cap) {
        --G;
        warp_bytes = (int64_t)G * d.Q * a.PP * 8;
    }
    if (warp_bytes + steps_bytes > cap) return -EINVAL;   // one stripe exceeds shared memory
    a.G = G;
    a.warps = (int)std::min<int64_t>(32, (cap - steps_bytes) / warp_bytes);
    a.ngroups = (d.S + G - 1) / G;
    a.warps = (int)std::max<int64_t>(1, std::min<int64_t>(a.warps, a.ngroups));
    const int smem = (int)(a.warps * warp_bytes + steps_bytes);
    DecKernel fn = pick_kernel(d.Q);
    if ((err = record_cuda(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))))
        return err;
    int per_sm = 0;
    if ((err = record_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, a.warps * 32, smem))))
        return err;
    const int64_t ctas = (a.ngroups + a.warps - 1) / a.warps;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ctas, (int64_t)std::max(per_sm, 1) * sms));
    fn<<<(unsigned)grid, a.warps * 32, smem, st>>>(a);
    return record_cuda(cudaGetLastError());
}

}  // namespace mojette
