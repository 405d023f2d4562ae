// Inverse Mojette transform (decode) kernels, Sec. 2.2, along a
// pre-determined reconstruction path (one projection dedicated to each line,
// swept from both ends of the line; the path itself is built on the host,
// plan.cpp).
//
// Every pixel (l, x) is rebuilt in gather form: the bin of its dedicated
// projection (direction p) XOR the other pixels of that bin's discrete line,
// (l', x + (l' - l) p) for l' != l inside the image. The schedule
// guarantees those are known when the pixel is rebuilt, so the result is
// the value the paper's "subtract its contribution from all projections"
// procedure reaches, with at most Q - 1 XORs per pixel (Sec. 3).
//
// GB300 design. Decode is HBM-bound in bytes but carries a sequential
// dependency along the lines (about P/2 steps per stripe with two fronts),
// so the kernels are built to keep that chain short and many stripes in
// flight:
//   - the pixel line l+1 rebuilt in the same step is forwarded through
//     registers (warp shuffles), so the only shared-memory round trip on the
//     critical path is one per step;
//   - the Q*P bins the path uses are staged in shared memory and each
//     rebuilt pixel overwrites its own bin, so a stripe needs about Q*P words
//     of shared memory;
//   - a pixel outside the image reads a zero word (the XOR identity), so no
//     bounds test sits in the inner loop.
// decode_lines, the default path kernel, keeps each stripe in its own region
// with rows in the order of the bins it stages (one bulk copy per front's run
// of bins), one zero word beside each row (at Q <= 4 operand columns outside
// the image are clamped to it; at Q > 4 such operands are not loaded), and
// a per-path bank layout chosen on the host (row phases and per-front load
// orders). decode_fronts, decode_cols and
// decode_stream interleave the G stripes of a warp word by word, staged by
// 8-byte cp.async into rows with zero columns around them.
//
// Every kernel comes in two forms: plain (one reconstruction path, stripes
// back to back at fixed strides) and batched (work items of G stripes, each
// with its own path from a device table, stripes anywhere in memory through
// per-stripe address arrays). Both run the same instructions per step.
#pragma once

#include <algorithm>
#include <cerrno>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>

#include "ptx.cuh"

namespace mojette {
namespace {

struct DecParams {
    // plain form
    const uint64_t *proj;   // stripe s at proj + s * total
    uint64_t *img;          // stripe s at img + s * Q * P
    int64_t S;
    DecGroup grp;           // its reconstruction path
    // batched form
    const DecGroup *groups;
    const DecWork *work;
    int64_t nwork;
    const uint64_t *const *srcp;
    uint64_t *const *dstp;
    // layout (both forms)
    int64_t total;
    int P, Q;     // Q: lines rebuilt (a systematic decode: the lost data lines)
    int Qd;       // systematic: data lines per stripe (img stripe pitch Qd * P)
    int reach;    // zero columns before, between and after the rows of a stripe
    int RP;       // row pitch in columns: P + reach (+ room for row phases)
    int SWc;      // columns per stripe slot
    int SWr;      // decode_lines: words per stripe region
    int rowbase[kMaxLines];   // decode_lines: first column of each line's row
    int G;        // stripes per work item (one warp)
    int GS;       // interleave stride (decode_lines: G; decode_fronts: G rounded to odd)
    int TS;       // words per step table in shared memory
    int gpc;      // work items per CTA (one warp per CTA)
    int persist;  // 1: grid-stride over chunks of gpc items
    int steady;   // decode_fronts: 1 to run steady steps on the short path
    uint32_t *status;   // device status word (bounded waits that time out)
};

__device__ __forceinline__ uint64_t ld_s64(uint32_t addr)
{
    uint64_t v;
    asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}

// Load when `pred` is nonzero, else 0.
__device__ __forceinline__ uint64_t ld_s64_if(uint32_t addr, uint32_t pred)
{
    uint64_t v;
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\tmov.b64 %0, 0;\n\t"
                 "@p ld.shared.u64 %0, [%1];\n\t}"
                 : "=l"(v) : "r"(addr), "r"(pred));
    return v;
}

__device__ __forceinline__ void st_s64(uint32_t addr, uint64_t v)
{
    asm volatile("st.shared.u64 [%0], %1;" ::"r"(addr), "l"(v));
}

// Store when `pred` is nonzero.
__device__ __forceinline__ void st_s64_if(uint32_t addr, uint64_t v, uint32_t pred)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.shared.u64 [%0], %1;\n\t}"
                 ::"r"(addr), "l"(v), "r"(pred));
}

// Walks the work items of one CTA: `body(item)` for item = base + k,
// k < gpc, base = blockIdx.x * gpc (+ gridDim.x * gpc when persistent).
template <typename F>
__device__ __forceinline__ void for_items(const DecParams &a, int64_t nitems, F &&body)
{
    const int64_t stride = a.persist ? (int64_t)gridDim.x * a.gpc : nitems;
    for (int64_t base = (int64_t)blockIdx.x * a.gpc; base < nitems; base += stride)
        for (int k = 0; k < a.gpc; ++k) {
            const int64_t item = base + k;
            if (item >= nitems) break;
            body(item);
        }
}

// ---------------------------------------------------------------------------
// decode_fronts: one lane runs one front (left or right) of one stripe, all Q
// lines, visiting the lines from Q-1 down to 0 each step. Lanes 0..15 are
// left fronts and 16..31 right fronts of the same G stripes.
// QT: number of lines at compile time (0: any Q up to kMaxLines, slower).
template <int QT, bool BATCHED>
__global__ void __launch_bounds__(32) decode_fronts(const __grid_constant__ DecParams a)
{
    constexpr int QA = QT ? QT : kMaxLines;   // register array extent
    extern __shared__ __align__(16) uint64_t sm[];
    const int Q = QT ? QT : a.Q;
    const int P = a.P, G = a.G, GS = a.GS;
    const int lane = threadIdx.x & 31;
    // Step words first, then the stripe slots; word (column c, slot g) sits
    // at c * GS + g.
    uint32_t *steps = reinterpret_cast<uint32_t *>(sm);
    uint64_t *wbuf = sm + a.TS / 2;
    // Zero columns stand for pixels outside the image (the XOR identity):
    // the reach columns before each row and after the last one. Rows are
    // always staged before they are read.
    for (int ll = 0; ll <= Q; ++ll)
        for (int i = lane; i < a.reach * GS; i += 32) wbuf[ll * a.RP * GS + i] = 0;
    const uint32_t wbase = smem_addr(wbuf);

    // Front lanes: lane = 16 * side + g. Lanes past G shadow stripe slot 0:
    // they load the same words and store the same values as lane g = 0 of
    // their side, so every lane runs the same instructions.
    const int side = lane >> 4;
    const int graw = lane & 15;
    const int g = graw < G ? graw : 0;
    const int stepb = (side ? -1 : 1) * GS * 8;

    // Per line: start address of this front's pixel, the bit of the step word
    // that moves it, whether a steady step forwards its line l+1 operand, and
    // the byte offsets from it to the other pixels of its bin line,
    // (l2, x + (l2 - l) p) -- the last three depend on the path.
    uint32_t start[QA], bit[QA], keep[QA];
    uint64_t fmask[QA];
    int dl[QA][QA];
#pragma unroll
    for (int l = 0; l < QA; ++l) {
        if (l >= Q) break;
        start[l] = wbase + ((a.reach + l * a.RP + (side ? P - 1 : 0)) * GS + g) * 8;
        bit[l] = 1u << (2 * l + side);
    }
    int T4 = 0;
    auto load_group = [&](const DecGroup &gr) {
        const int T = gr.T;
        T4 = (T + 3) & ~3;
        for (int t = lane; t < T4; t += 32) steps[t] = t < T ? gr.steps[t] : 0u;
#pragma unroll
        for (int l = 0; l < QA; ++l) {
            if (l >= Q) break;
            const int p = gr.p[2 * l + side];
            const uint32_t f = (l + 1 < Q) ? (gr.fwd >> (2 * l + side)) & 1u : 0u;
            keep[l] = f ^ 1u;
            fmask[l] = f ? ~0ull : 0ull;
#pragma unroll
            for (int l2 = 0; l2 < QA; ++l2) {
                if (l2 >= Q) break;
                dl[l][l2] = (l2 - l) * (a.RP + p) * GS * 8;
            }
        }
    };
    const DecGroup *gp = nullptr;   // batched: the current work item's path
    auto grp = [&]() -> const DecGroup & {
        if constexpr (BATCHED) return *gp;
        else return a.grp;
    };
    if constexpr (!BATCHED) load_group(a.grp);
    __syncwarp();

    // Copy lanes: lane = xk * G + gg covers XK columns of G stripes.
    const int XK = 32 / G;
    const int xk = lane / G, gg = lane - xk * G;
    const bool copy_ok = xk < XK;

    int cur = -1;
    const int64_t nitems = BATCHED ? a.nwork : (a.S + G - 1) / G;
    for_items(a, nitems, [&](int64_t item) {
        int nst;
        int64_t s0 = 0, first = 0;
        if constexpr (BATCHED) {
            const DecWork wk = a.work[item];
            nst = wk.nst;
            first = wk.first;
            if (wk.group != cur) {
                cur = wk.group;
                gp = a.groups + cur;
                __syncwarp();
                load_group(*gp);
                __syncwarp();
            }
        } else {
            s0 = item * G;
            nst = (int)min64(G, a.S - s0);
        }

        // stage the Q*P bins the path uses, in pixel order
        if (copy_ok && gg < nst) {
            const uint64_t *src = BATCHED ? a.srcp[first + gg] : a.proj + (s0 + gg) * a.total;
            for (int ll = 0; ll < Q; ++ll) {
                const int sp = grp().split[ll];
                const int sl = grp().src[2 * ll], sr = grp().src[2 * ll + 1];
                uint64_t *dst = wbuf + (a.reach + ll * a.RP) * GS + gg;
                for (int x = xk; x < P; x += XK)
                    cp_async8(dst + x * GS, src + ((x < sp ? sl : sr) - x));
            }
        }
        cp_async_wait_all();
        __syncwarp();

        // replay the path
        uint32_t pos[QA];
#pragma unroll
        for (int l = 0; l < QA; ++l)
            if (l < Q) pos[l] = start[l];

        // Steady step: every line moves; line l's operand on line l+1 is the
        // pixel rebuilt just before in this step exactly where fwd says so.
        auto steady = [&]() {
            uint64_t v[QA], own[QA], op[QA][QA];
#pragma unroll
            for (int l = QA - 1; l >= 0; --l) {
                if (l >= Q) continue;
                own[l] = ld_s64(pos[l]);
#pragma unroll
                for (int l2 = 0; l2 < QA; ++l2) {
                    if (l2 >= Q || l2 == l) continue;
                    if (l2 == l + 1) op[l][l2] = ld_s64_if(pos[l] + dl[l][l2], keep[l]);
                    else op[l][l2] = ld_s64(pos[l] + dl[l][l2]);
                }
            }
#pragma unroll
            for (int l = QA - 1; l >= 0; --l) {
                if (l >= Q) continue;
                uint64_t acc = own[l];
#pragma unroll
                for (int l2 = 0; l2 < QA; ++l2)
                    if (l2 < Q && l2 != l) acc ^= op[l][l2];
                if (l + 1 < Q) acc ^= v[l + 1] & fmask[l];
                v[l] = acc;
            }
#pragma unroll
            for (int l = 0; l < QA; ++l) {
                if (l >= Q) break;
                st_s64(pos[l], v[l]);
                pos[l] += stepb;
            }
            __syncwarp();
        };
        // Any step: per-line activity bits, forwarding where line l+1 moved
        // onto exactly the operand's pixel in this step.
        auto general = [&](uint32_t w) {
            uint64_t own[QA], op[QA][QA], v[QA];
            uint32_t act[QA];
#pragma unroll
            for (int l = QA - 1; l >= 0; --l) {
                if (l >= Q) continue;
                own[l] = ld_s64(pos[l]);
#pragma unroll
                for (int l2 = 0; l2 < QA; ++l2) {
                    if (l2 >= Q || l2 == l) continue;
                    op[l][l2] = ld_s64(pos[l] + dl[l][l2]);
                }
            }
#pragma unroll
            for (int l = QA - 1; l >= 0; --l) {
                if (l >= Q) continue;
                act[l] = w & bit[l];
                uint64_t acc = own[l];
#pragma unroll
                for (int l2 = 0; l2 < QA; ++l2) {
                    if (l2 >= Q || l2 == l) continue;
                    uint64_t o = op[l][l2];
                    if (l2 == l + 1 && act[l2] && pos[l2] == pos[l] + dl[l][l2]) o = v[l2];
                    acc ^= o;
                }
                v[l] = acc;
            }
#pragma unroll
            for (int l = 0; l < QA; ++l) {
                if (l >= Q) break;
                st_s64_if(pos[l], v[l], act[l]);
                pos[l] += act[l] ? stepb : 0;
            }
            __syncwarp();
        };
        const uint32_t steady_bit = (QT && QT <= kFastMaxLines && a.steady) ? kStepSteady : 0u;
        for (int t = 0; t < T4; ++t) {
            const uint32_t w = steps[t];
            if (w & steady_bit) steady();
            else general(w);
        }

        // write the rebuilt image
        if (copy_ok && gg < nst) {
            uint64_t *out = BATCHED ? a.dstp[first + gg] : a.img + (s0 + gg) * (int64_t)Q * P;
            for (int ll = 0; ll < Q; ++ll) {
                const uint64_t *buf = wbuf + (a.reach + ll * a.RP) * GS + gg;
                for (int x = xk; x < P; x += XK) __stcs(out + ll * P + x, buf[x * GS]);
            }
        }
        __syncwarp();
    });
}

// ---------------------------------------------------------------------------
// decode_lines: one lane per (stripe, line, front). A warp holds G = 32/(2Q)
// stripes; at every step each lane rebuilds the next pixel of its line's
// front (when the step word moves it), from its staged bin and the other
// pixels of the bin line read from shared memory -- except the value on
// line l+1, which line l+1 may rebuild in this same step. Those same-step
// links (bit 2l+side of the step's forward word) form chains l -> l+1 -> ...
// within a front; the chain values are a segmented suffix XOR over the lines,
// done with warp shuffles (only the rounds the path's chains need), so every
// lane of every line works at every step and a step costs one shared-memory
// round trip. At Q <= 4 a run of steady steps (every front moves, one link
// pattern) runs as an inner loop with no step-table reads. The layout, the
// staging and the addressing are described in the kernel.
//
// SYS: the systematic form. The lines rebuilt are the lost data lines (Q of
// them, at image rows lpos[]) of the data buffer (img, or dstp[s] batched, Qd
// lines per stripe), which sys_residual has already filled with their
// residual bins (the known lines removed); the rows are staged from there
// and the rebuilt lines written back in place.
template <int QT, bool BATCHED, bool SYS = false>
__global__ void __launch_bounds__(32) decode_lines(const __grid_constant__ DecParams a)
{
    extern __shared__ __align__(16) uint64_t sm[];
    constexpr int Q = QT;
    // Rows of the non-systematic form are kept in bin order (see below).
    constexpr bool REV = !SYS;
    const int P = a.P, G = a.G;
    const int lane = threadIdx.x & 31;
    // (step word, forward word) pairs (TS of them), the staging mbarrier,
    // then the stripes' regions
    uint2 *stw = reinterpret_cast<uint2 *>(sm);
    uint64_t *mbar = sm + a.TS;
    uint64_t *wbuf = sm + a.TS + 2;
    // Zero the regions once: rows are always staged before they are read,
    // and the word beside each row (a pixel outside the image, the XOR
    // identity) is never written.
    for (int i = lane; i < a.SWr * G; i += 32) wbuf[i] = 0;
    const uint32_t wbase = smem_addr(wbuf);
    const uint32_t bar = smem_addr(mbar);
    if (lane == 0) {
        mbar_init(bar, 32);   // every lane arrives once per item
        mbar_init_fence();
    }

    // Rebuild lanes: lane = side * 16 + l * G + g -- the left fronts in the
    // lower half-warp, the right fronts in the upper one (a 64-bit shared
    // load is served per half-warp, and fronts moving the same way keep
    // their relative bank slots); lanes past Q*G in a half shadow line 0 of
    // their side, load nothing and never store.
    const int hl = lane & 15, lq = hl / G;
    const bool ok = lq < Q;
    const int l = ok ? lq : 0, side = lane >> 4;
    const int g = ok ? hl - lq * G : 0;
    const int ls = 2 * l + side;   // front index in the step words
    const uint32_t bitmask = ok ? 1u << ls : 0u;
    const int myrow = a.rowbase[l];
    // Layout: each stripe has its own region of SWr words (SWr = S mod 16,
    // so the regions sit in different bank slots), row l starting at
    // rowbase[l]. The non-systematic form keeps a row in bin order -- pixel
    // x at rowbase[l] + P - 1 - x, the order of the dedicated projection's
    // bins, so that a front's run of bins is staged by one bulk copy -- and
    // the systematic form in pixel order (x at rowbase[l] + x), the order of
    // the residual rows it is staged from. One zero word sits beside each
    // row, at column P in the row's order; an operand column outside the
    // image is clamped to it (one unsigned min).
    const uint32_t start = wbase + (g * a.SWr + myrow + ((side == 0) == REV ? P - 1 : 0)) * 8;
    const int stepb = (side == 0) == REV ? -8 : 8;

    // Path-dependent state. A front reads Q words per step: its own bin
    // (first) and the pixels of the bin line on lines l + j (mod Q), j = 1 ..
    // Q-1, at column x + (row of l2 - row of l) p; j = 1 is line l+1, which
    // may be rebuilt by its front in this same step (forwarded), except for
    // l = Q-1 where it wraps to line 0. Operand k (the path's load order,
    // chosen with the row phases so that each load instruction meets
    // distinct bank slots) sits dk[k] columns from this front's pixel, on
    // the line whose column 0 is at byte address rk[k]. A forwarded word is
    // read all the same: it still holds line l+1's bin, which line l+1
    // reads as its own, so the chain runs over b = pixel ^ own bin -- b_l =
    // (XOR of l's operand words) ^ b_{l+1} while linked, pixel_l = b_l ^ own
    // bin_l -- and the stale bin cancels. For steady steps: this lane's link
    // (line l forwards from line l+1), the number of lines linked after it,
    // and the link state after each scan round, from the path's steady
    // pattern: after the round with stride d, line l is still linked iff it
    // was, and line l+d was too.
    int T4 = 0;
    int dk[Q > 1 ? Q - 1 : 1];
    uint32_t rk[Q > 1 ? Q - 1 : 1];
    uint32_t sfw = 0u;
    // steady steps, as all-ones / zero masks: Q <= 4, lm[d - 1] -- line
    // l + d is linked to this one (lines l+1 .. l+d all linked); Q > 4,
    // lm[r] -- this line is still linked after scan round r
    uint32_t lm[Q > 1 ? Q - 1 : 1];
    int smc = 0;
    auto load_group = [&](const DecGroup &gr) {
        const int T = gr.T;
        T4 = (T + 3) & ~3;
        // the table in shared memory: step word; forward word's links (bits
        // 0 .. 2Q-1) with the step's longest same-step chain (links l -> l+1
        // -> ... in a row, either side) in bits 24..27, so that a step runs
        // only the shuffle rounds some chain needs
        for (int t = lane; t < T4; t += 32) {
            uint32_t w = 0u, f = 0u;
            if (t < T) {
                w = gr.steps[t];
                f = gr.steps[T + t] & ((1u << (2 * Q)) - 1u);
            }
            uint32_t mc = 0u;
#pragma unroll
            for (int sd = 0; sd < 2; ++sd) {
                uint32_t run = 0u;
#pragma unroll
                for (int j = 0; j + 1 < Q; ++j) {
                    run = ((f >> (2 * j + sd)) & 1u) ? run + 1u : 0u;
                    mc = max(mc, run);
                }
            }
            stw[t] = make_uint2(w, f | (mc << 24));
        }
        // bits 16..30 of a steady step's word: the steady steps from it on,
        // 32 entries at a time from the end (the next non-steady entry by
        // ballot; the count carried in from the chunk after)
        __syncwarp();
        uint32_t carry = 0u;
        for (int base = ((T4 - 1) / 32) * 32; base >= 0; base -= 32) {
            const int t = base + lane;
            const bool in = t < T4;
            uint2 e = in ? stw[t] : make_uint2(0u, 0u);
            const bool st = in && (e.x & kStepSteady);
            const uint32_t above = __ballot_sync(0xffffffffu, !st) & ~((2u << lane) - 1u);
            uint32_t run = 0u;
            if (st) run = above ? (uint32_t)(__ffs(above) - 1 - lane) : 32u - lane + carry;
            run = min(run, 0x7fffu);
            if (in) {
                e.x = (e.x & ~(0x7fffu << 16)) | (run << 16);
                stw[t] = e;
            }
            carry = __shfl_sync(0xffffffffu, run, 0);
        }
        __syncwarp();
        const int p = gr.p[ls];
        const uint32_t ord = gr.order[ls];   // nibble 0 is the own bin
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const int l2 = (l + ((ord >> (4 * k)) & 15u)) % Q;
            dk[k - 1] = (gr.lpos[l2] - gr.lpos[l]) * p;
            rk[k - 1] = wbase + (uint32_t)(g * a.SWr + a.rowbase[l2] + (REV ? P - 1 : 0)) * 8u;
        }
        sfw = ok ? (gr.fwd >> ls) & 1u : 0u;
        smc = 0;   // the steady pattern's longest chain (the same in every lane)
        for (int sd = 0; sd < 2; ++sd)
            for (int j = 0, run = 0; j + 1 < Q; ++j) {
                run = ((gr.fwd >> (2 * j + sd)) & 1u) ? run + 1 : 0;
                smc = max(smc, run);
            }
        if constexpr (Q <= 4) {
            int chain = 0;   // lines l+1 .. l+chain are linked to this one
            if (ok)
                for (int j = l; j + 1 < Q && ((gr.fwd >> (2 * j + side)) & 1u); ++j) ++chain;
#pragma unroll
            for (int d = 1; d < Q; ++d) lm[d - 1] = d <= chain ? ~0u : 0u;
        } else {
            uint32_t c[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) c[j] = (j + 1 < Q) ? (gr.fwd >> (2 * j + side)) & 1u : 0u;
#pragma unroll
            for (int r = 0, d = 1; d < Q; ++r, d <<= 1) {
                lm[r] = ok && c[l] ? ~0u : 0u;
                uint32_t nc[Q];
#pragma unroll
                for (int j = 0; j < Q; ++j) nc[j] = (c[j] && j + d < Q) ? c[j + d] : 0u;
#pragma unroll
                for (int j = 0; j < Q; ++j) c[j] = nc[j];
            }
        }
    };
    const DecGroup *gp = nullptr;   // batched: the current work item's path
    auto grp = [&]() -> const DecGroup & {
        if constexpr (BATCHED) return *gp;
        else return a.grp;
    };
    if constexpr (!BATCHED) load_group(a.grp);
    __syncwarp();

    // Copy lanes (write-back): lane = xk * G + gg covers XK columns of G
    // stripes.
    const int XK = 32 / G;
    const int xk = lane / G, gg = lane - xk * G;
    const bool copy_ok = xk < XK;

    int cur = -1;
    uint32_t phase = 0;
    bool dead = false;   // a staging wait timed out: stop
    const int64_t nitems = BATCHED ? a.nwork : (a.S + G - 1) / G;
    for_items(a, nitems, [&](int64_t item) {
        if (dead) return;
        int nst;
        int64_t s0 = 0, first = 0;
        if constexpr (BATCHED) {
            const DecWork wk = a.work[item];
            nst = wk.nst;
            first = wk.first;
            if (wk.group != cur) {
                cur = wk.group;
                gp = a.groups + cur;
                __syncwarp();
                load_group(*gp);
                __syncwarp();
            }
        } else {
            s0 = item * G;
            nst = (int)min64(G, a.S - s0);
        }

        // Staging: each lane copies one run of n consecutive words in row
        // order -- non-systematic: its own front's run of bins of its
        // dedicated projection (bins src - x for the pixels x the front
        // rebuilds); systematic: the lanes of the left side each a whole
        // residual row. Where the run and its place in shared memory agree
        // mod 16 bytes, one bulk copy takes the aligned middle and 8-byte
        // cp.async the odd word at either end. Where they do not, the run's
        // first n - 1 words are staged the same way one word further on
        // (which makes them agree), its last word is loaded into a
        // register, and once the copies have landed the warp moves the run
        // down one word and puts the last word in place. The previous item's
        // reads and writes of the regions are ordered before the bulk
        // writes first.
        fence_proxy_async_smem();
        __syncwarp();
        int n = 0;
        const uint64_t *gsrc = nullptr;
        uint32_t sdst = 0;
        if (ok && g < nst) {
            if constexpr (SYS) {
                if (side == 0) {
                    const uint64_t *dat = BATCHED ? a.dstp[first + g] : a.img + (s0 + g) * (int64_t)a.Qd * P;
                    n = P;
                    gsrc = dat + (int64_t)grp().lpos[l] * P;
                    sdst = wbase + (g * a.SWr + myrow) * 8;
                }
            } else {
                const uint64_t *sb = BATCHED ? a.srcp[first + g] : a.proj + (s0 + g) * a.total;
                const int sp = grp().split[l];
                if (side == 0) {
                    n = sp;
                    gsrc = sb + (grp().src[2 * l] - (sp - 1));
                    sdst = wbase + (g * a.SWr + myrow + P - sp) * 8;
                } else {
                    n = P - sp;
                    gsrc = sb + (grp().src[2 * l + 1] - (P - 1));
                    sdst = wbase + (g * a.SWr + myrow) * 8;
                }
            }
        }
        const bool shifted = n > 0 && ((((uint32_t)(uintptr_t)gsrc) ^ sdst) & 8u) != 0;
        const int n1 = shifted ? n - 1 : n;                    // words staged by copies
        const uint32_t sd1 = shifted ? sdst + 8u : sdst;        // where they land
        const int head = n1 > 0 && ((uintptr_t)gsrc & 8u) ? 1 : 0;
        const int body = n1 > 0 ? ((n1 - head) & ~1) : 0;
        mbar_arrive_expect_tx(bar, (uint32_t)body * 8u);
        if (body > 0) tma_load_1d(sd1 + head * 8u, gsrc + head, (uint32_t)body * 8u, bar);
        if (head) cp_async8_s(sd1, gsrc);
        if (n1 - head - body > 0) cp_async8_s(sd1 + (uint32_t)(n1 - 1) * 8u, gsrc + (n1 - 1));
        const uint64_t lastw = shifted ? gsrc[n - 1] : 0ull;
        cp_async_wait_all();
        const bool arrived = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        if (__any_sync(0xffffffffu, !arrived)) {
            // the bulk copies did not land in time: report, let any still in
            // flight finish (bounded) and stop
            if (lane == 0) atomicOr(a.status, kStatusWaitTimeout);
            mbar_wait_bounded(bar, phase ^ 1u);
            dead = true;
            return;
        }
        __syncwarp();
        // the shifted runs, one at a time by the whole warp: every word read
        // before any is written
        uint32_t rest = __ballot_sync(0xffffffffu, shifted);
        while (rest) {
            const int src_lane = __ffs(rest) - 1;
            rest &= rest - 1;
            const int nn = __shfl_sync(0xffffffffu, n, src_lane);
            const uint32_t sd = __shfl_sync(0xffffffffu, sdst, src_lane);
            const uint64_t lw = __shfl_sync(0xffffffffu, (unsigned long long)lastw, src_lane);
            // K words per lane per round (K * 32 >= the run where it fits)
            auto shift_down = [&](auto kc) {
                constexpr int K = decltype(kc)::value;
                for (int i0 = 0; i0 < nn; i0 += 32 * K) {
                    uint64_t w[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const int i = i0 + k * 32 + lane;
                        w[k] = i + 1 < nn ? ld_s64(sd + (uint32_t)(i + 1) * 8u) : lw;
                    }
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const int i = i0 + k * 32 + lane;
                        if (i < nn) st_s64(sd + (uint32_t)i * 8u, w[k]);
                    }
                    __syncwarp();
                }
            };
            if (nn > 64) shift_down(std::integral_constant<int, 4>{});
            else if (nn > 32) shift_down(std::integral_constant<int, 2>{});
            else shift_down(std::integral_constant<int, 1>{});
        }

        uint32_t pos = start;
        int x = side ? P - 1 : 0;          // this front's column
        const int dx = side ? -1 : 1;
        // the word operand load k reads at this step
        auto opaddr = [&](int k) -> uint32_t {
            const uint32_t c = 8u * min((uint32_t)(x + dk[k]), (uint32_t)P);
            return REV ? rk[k] - c : rk[k] + c;
        };
        // Q <= 4: the operand addresses of the current step, computed as
        // soon as the column is known (in a steady step: while its loads are
        // in flight; measured 4-5% faster at 8 KB (6,4), no gain at Q = 8,
        // where the addresses are computed at the loads)
        constexpr bool PIPE = Q <= 4;
        uint32_t oa[Q > 1 ? Q - 1 : 1];
        auto set_oa = [&]() {
            if constexpr (PIPE) {
#pragma unroll
                for (int k = 0; k < Q - 1; ++k) oa[k] = opaddr(k);
            }
        };
        auto addr = [&](int k) -> uint32_t {
            if constexpr (PIPE) return oa[k];
            else return opaddr(k);
        };
        // Q > 4: an operand outside the image is not loaded at all (a zero),
        // instead of reading the zero word beside its row: fewer shared-memory
        // accesses and bank conflicts where the kernel is bound by them
        auto opload = [&](int k) -> uint64_t {
            if constexpr (PIPE) {
                return ld_s64(oa[k]);
            } else {
                const uint32_t c = (uint32_t)(x + dk[k]);
                return ld_s64_if(REV ? rk[k] - 8u * c : rk[k] + 8u * c, c < (uint32_t)P);
            }
        };
        set_oa();
        // The step loop, compiled once per bound MC on the steady pattern's
        // longest same-step chain (steady steps run only the shuffle rounds
        // d <= MC; a bound known at compile time costs no branch); other
        // steps skip the rounds their own longest chain does not need.
        auto run_steps = [&](auto mcc) {
            constexpr int MC = decltype(mcc)::value;
            // the next step's words are read one step ahead, as one 64-bit
            // word (the table holds T4 + 4 pairs, so the read past the last
            // step stays inside it)
            uint2 nx = stw[0];
            for (int t = 0; t < T4; ++t) {
                const uint32_t w = nx.x, f = nx.y;
                const int mc = (int)(f >> 24);   // longest same-step chain
                nx = stw[t + 1];
                if (w & kStepSteady) {
                    // steady: every line moves, links are the path's pattern
                    // FAST: every operand of every lane lies inside the
                    // image for the whole step, so the addresses just move
                    // with the front (no clamp); x is caught up afterwards
                    auto steady_step = [&](auto fastc) {
                        constexpr bool FAST = decltype(fastc)::value;
                        const uint64_t own = ld_s64(pos);
                        uint64_t lv[Q > 1 ? Q - 1 : 1];
#pragma unroll
                        for (int k = 0; k < Q - 1; ++k) lv[k] = opload(k);
                        const uint32_t at = pos;
                        pos += stepb;
                        if constexpr (FAST) {
#pragma unroll
                            for (int k = 0; k < Q - 1; ++k) oa[k] += stepb;
                        } else {
                            x += dx;
                            set_oa();
                        }
                        // in 32-bit halves: a masked XOR is one 3-input logic op
                        uint32_t xl = 0u, xh = 0u;
#pragma unroll
                        for (int k = 0; k < Q - 1; ++k) {
                            xl ^= (uint32_t)lv[k];
                            xh ^= (uint32_t)(lv[k] >> 32);
                        }
                        uint32_t vl, vh;
                        if constexpr (Q <= 4) {
                            // the linked lines' own values, all fetched at once: one
                            // shuffle latency instead of log2 Q dependent rounds
                            vl = xl ^ (uint32_t)own;
                            vh = xh ^ (uint32_t)(own >> 32);
#pragma unroll
                            for (int d = 1; d < Q; ++d) {
                                if (d <= MC) {   // a constant once unrolled
                                    vl ^= __shfl_down_sync(0xffffffffu, xl, d * G) & lm[d - 1];
                                    vh ^= __shfl_down_sync(0xffffffffu, xh, d * G) & lm[d - 1];
                                }
                            }
                        } else {
#pragma unroll
                            for (int r = 0, d = 1; d < Q; ++r, d <<= 1) {
                                if (d <= MC) {
                                    xl ^= __shfl_down_sync(0xffffffffu, xl, d * G) & lm[r];
                                    xh ^= __shfl_down_sync(0xffffffffu, xh, d * G) & lm[r];
                                }
                            }
                            vl = xl ^ (uint32_t)own;
                            vh = xh ^ (uint32_t)(own >> 32);
                        }
                        st_s64_if(at, ((uint64_t)vh << 32) | vl, ok);
                        __syncwarp();
                    };
                    if constexpr (Q <= 4) {
                        // a run of steady steps (its length in bits 16..30 of
                        // the step word), the table not read until it ends
                        // (at Q > 4 one step at a time measured faster)
                        const int run = (int)((w >> 16) & 0x7fffu);
                        // steps [s0, s1) of the run: every lane's operand
                        // columns x + dk (moving by dx per step) inside [0, P)
                        int lo = 0, hi = run;
                        if (ok) {
#pragma unroll
                            for (int k = 0; k < Q - 1; ++k) {
                                const int c = x + dk[k];
                                if (dx > 0) {
                                    lo = max(lo, -c);
                                    hi = min(hi, P - c);
                                } else {
                                    lo = max(lo, c - (P - 1));
                                    hi = min(hi, c + 1);
                                }
                            }
                        }
                        const int s0 = min(__reduce_max_sync(0xffffffffu, lo), run);
                        const int s1 = max(__reduce_min_sync(0xffffffffu, hi), s0);
                        for (int rs = 0; rs < s0; ++rs) steady_step(std::false_type{});
#pragma unroll 2
                        for (int rs = s0; rs < s1; ++rs) steady_step(std::true_type{});
                        x += dx * (s1 - s0);
                        for (int rs = s1; rs < run; ++rs) steady_step(std::false_type{});
                        t += run - 1;
                        nx = stw[t + 1];
                    } else {
                        steady_step(std::false_type{});
                    }
                    continue;
                }
                // a front that does not move this step loads nothing (its value
                // is not used: a link always points at a front that moves)
                const uint32_t act = w & bitmask;
                const uint32_t fw = ok ? (f >> ls) & 1u : 0u;
                uint64_t own = 0, v = 0;
                if (act) {
                    own = ld_s64(pos);
#pragma unroll
                    for (int k = 0; k < Q - 1; ++k) v ^= opload(k);
                }
                // segmented suffix XOR: v_l ^= v_{l+1} while linked (only the
                // rounds the step's longest chain needs)
                uint32_t c = fw;
#pragma unroll
                for (int d = 1; d < Q; d <<= 1) {
                    if (d <= mc) {
                        const uint64_t tv = __shfl_down_sync(0xffffffffu, v, d * G);
                        const uint32_t tc = __shfl_down_sync(0xffffffffu, c, d * G);
                        if (c) {
                            v ^= tv;
                            c = tc;
                        }
                    }
                }
                st_s64_if(pos, v ^ own, act);
                pos += act ? stepb : 0;
                x += act ? dx : 0;
                set_oa();
                __syncwarp();
            }
        };
        if constexpr (Q <= 4) {
            switch (smc) {
            case 0: run_steps(std::integral_constant<int, 0>{}); break;
            case 1: run_steps(std::integral_constant<int, 1>{}); break;
            case 2: run_steps(std::integral_constant<int, 2>{}); break;
            default: run_steps(std::integral_constant<int, 3>{}); break;
            }
        } else {
            // scan rounds of stride 1, 2, 4: a chain of length c needs those <= c
            if (smc == 0) run_steps(std::integral_constant<int, 0>{});
            else if (smc == 1) run_steps(std::integral_constant<int, 1>{});
            else if (smc <= 3) run_steps(std::integral_constant<int, 3>{});
            else run_steps(std::integral_constant<int, 7>{});
        }

        // write-back, coalesced along each row: the image's lines (the lost
        // data lines, in place, for the systematic form). The loop is
        // unrolled so that several shared loads are in flight at once (one
        // at a time, the write-back took about a quarter of an item's time
        // at 8 KB (6,4)); 16-byte stores of word pairs measured slower (a
        // half-warp's loads then span twice the banks). With 4 or more
        // stripes per warp (Q <= 4), each half-warp writes 16 consecutive
        // words -- a whole 128-byte line -- of one stripe, two stripes per
        // pass (8 KB (6,4): 1.062 -> 0.993 ms against 8 lanes per stripe);
        // with 2, the lanes alternate between the stripes (16 words of each
        // per store already; the blocked form measured 3% slower there).
        auto write_rows = [&](int gs, int x0, int xs) {
            uint64_t *out = BATCHED ? a.dstp[first + gs] : a.img + (s0 + gs) * (int64_t)(SYS ? a.Qd : Q) * P;
            for (int ll = 0; ll < Q; ++ll) {
                // column x of the row at row[dir * x]: pixel order (systematic)
                // or bin order from its last word
                const uint64_t *row = wbuf + gs * a.SWr + a.rowbase[ll] + (SYS ? 0 : P - 1);
                constexpr int dir = SYS ? 1 : -1;
                uint64_t *o = out + (int64_t)(SYS ? grp().lpos[ll] : ll) * P;
#pragma unroll 4
                for (int xx = x0; xx < P; xx += xs) __stcs(o + xx, row[dir * xx]);
            }
        };
        if constexpr (Q <= 4) {
            for (int gs = lane >> 4; gs < nst; gs += 2) write_rows(gs, lane & 15, 16);
        } else {
            if (copy_ok && gg < nst) write_rows(gg, xk, XK);
        }
        __syncwarp();
    });
}

// ---------------------------------------------------------------------------
// decode_ilv: the stripe-interleaved form of the path, one lane per stripe.
// A CTA of two warps rebuilds G <= 16 stripes at a time; word (column c of
// the stripe area, stripe g) sits at c * GS + g of its shared memory. Warp 0
// runs the left fronts and warp 1 the right fronts; lane h * 16 + g runs its
// side's front on lines h * H .. h * H + H - 1 (H = ceil(Q / 2)) of stripe g.
// The G lanes of a half-warp thus make the same access in G different stripes
// -- G consecutive words -- so every shared-memory load and store of the path
// is one wavefront per half-warp, with no bank planning and no dependence on
// the erasure pattern.
//
// Rows: PAD -- line l's pixels at columns rowbase[l] + [0, P), with a gap of
// `reach` zero columns between rows and at both ends, `reach` covering the
// widest offset (l2 - l) p of a bin line: the word of line l2 on a bin line
// is then at a fixed distance from the front's own word, whether inside the
// image or not (pixels outside the image are the XOR identity). Otherwise
// (no room for the gaps) rows of P + 1 columns, column P a zero word, and an
// operand column outside the image is clamped to it.
//
// A step, for each of the lane's lines: its own bin and the Q - 1 pixels of
// the bin line on the other lines, all loaded before anything is stored (a
// front that does not move this step loads as well, and stores nothing). The
// pixel line l+1 rebuilds in the same step (bit 2l+side of the forward word)
// is read as the bin it still holds, so line l takes the XOR of line l+1's
// other words on top: c_l = (words of l other than its bin) ^ (forwarded ?
// c_{l+1} : 0), pixel_l = bin_l ^ c_l. Within a lane that chain runs in
// registers; the link from the top line of the lower half-warp to the bottom
// line of the upper one is one warp shuffle. The two warps only meet where a
// front reads a pixel the other side rebuilt at an earlier step: the path
// marks such steps (kFwdSync) and the warps synchronise before their loads.
//
// Staging: every (stripe, line, front) run of consecutive bins is copied by
// 8-byte cp.async, 32 consecutive words per warp instruction (coalesced). The
// image goes back the same way, 32 consecutive words of a row per
// instruction.
template <int QT, bool BATCHED, bool PAD>
__global__ void __launch_bounds__(64) decode_ilv(const __grid_constant__ DecParams a)
{
    extern __shared__ __align__(16) uint64_t sm[];
    constexpr int Q = QT;
    constexpr int H = (Q + 1) / 2;   // lines per lane
    const int P = a.P, G = a.G, GS = a.GS;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int side = tid >> 5;       // 0: left fronts, 1: right fronts
    const int hh = lane >> 4;        // which half of the lines
    // stripe of the work item; lanes past G shadow stripe 0 (the same loads,
    // no stores), so that every address stays inside the CTA's stripes
    const bool gok = (lane & 15) < G;
    const int g = gok ? lane & 15 : 0;
    uint2 *stw = reinterpret_cast<uint2 *>(sm);   // (step word, forward word) pairs
    uint64_t *wbuf = sm + a.TS;
    for (int i = tid; i < a.SWc; i += 64) wbuf[i] = 0;
    const uint32_t wbase = smem_addr(wbuf);
    const uint32_t GSB = (uint32_t)GS * 8u;
    // shared-memory address of (line l, column c) of this lane's stripe
    auto at = [&](int l, int c) -> uint32_t {
        return wbase + ((uint32_t)(a.rowbase[l] + c) * (uint32_t)GS + (uint32_t)g) * 8u;
    };
    int sh[H];           // bit of line j in the step and forward words
    bool lv[H];          // line j exists
    int ln[H];           // its index
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const int l = hh * H + j;
        lv[j] = l < Q;
        ln[j] = lv[j] ? l : 0;
        sh[j] = 2 * ln[j] + side;
    }
    uint32_t rowa[Q];    // clamped rows: column 0 of every line
    if constexpr (!PAD) {
#pragma unroll
        for (int l = 0; l < Q; ++l) rowa[l] = at(l, 0);
    }

    // Path-dependent state: the word on line l2 of line j's bin line sits
    // dk = (lpos[l2] - lpos[l]) p columns from the front's column (0 for
    // l2 = l: its own bin); PAD keeps it as a byte offset from the front's
    // own word.
    int T4 = 0;
    int dk[H][Q];
    uint32_t off[H][Q];
    auto load_group = [&](const DecGroup &gr) {
        const int T = gr.T;
        T4 = (T + 3) & ~3;
        for (int t = tid; t < T4 + 4; t += 64)
            stw[t] = t < T ? make_uint2(gr.steps[t], gr.steps[T + t]) : make_uint2(0u, 0u);
#pragma unroll
        for (int j = 0; j < H; ++j) {
            const int p = gr.p[2 * ln[j] + side];
#pragma unroll
            for (int l2 = 0; l2 < Q; ++l2) {
                dk[j][l2] = (gr.lpos[l2] - gr.lpos[ln[j]]) * p;
                off[j][l2] = (uint32_t)((a.rowbase[l2] - a.rowbase[ln[j]] + dk[j][l2]) * GS) * 8u;
            }
        }
    };
    const DecGroup *gp = nullptr;   // batched: the current work item's path
    auto grp = [&]() -> const DecGroup & {
        if constexpr (BATCHED) return *gp;
        else return a.grp;
    };
    if constexpr (!BATCHED) load_group(a.grp);
    __syncthreads();

    int cur = -1;
    const int64_t nitems = BATCHED ? a.nwork : (a.S + G - 1) / G;
    for_items(a, nitems, [&](int64_t item) {
        int nst;
        int64_t s0 = 0, first = 0;
        if constexpr (BATCHED) {
            const DecWork wk = a.work[item];
            nst = wk.nst;
            first = wk.first;
            if (wk.group != cur) {
                cur = wk.group;
                gp = a.groups + cur;
                load_group(*gp);
            }
        } else {
            s0 = item * G;
            nst = (int)min64(G, a.S - s0);
        }

        // Staging: run r = (stripe gg, line ll, front sd), its bins in
        // consecutive words; word i of the left run is pixel sp - 1 - i, of
        // the right run pixel P - 1 - i.
        {
            const int nruns = nst * Q * 2;
            for (int r = side; r < nruns; r += 2) {
                const int gg = r / (2 * Q);
                const int rem = r - gg * 2 * Q;
                const int ll = rem >> 1, sd = rem & 1;
                const uint64_t *sb = BATCHED ? a.srcp[first + gg] : a.proj + (s0 + gg) * a.total;
                const int sp = grp().split[ll];
                const int n = sd ? P - sp : sp;
                const int xtop = sd ? P - 1 : sp - 1;
                const uint64_t *src = sb + (grp().src[2 * ll + sd] - xtop);
                const uint32_t d0 = wbase + ((uint32_t)(a.rowbase[ll] + xtop) * (uint32_t)GS + (uint32_t)gg) * 8u;
                for (int i = lane; i < n; i += 32) cp_async8_s(d0 - (uint32_t)i * GSB, src + i);
            }
            cp_async_wait_all();
        }
        __syncthreads();

        // replay the path
        const int x0 = side ? P - 1 : 0;
        int x[H];
        uint32_t pos[H];
#pragma unroll
        for (int j = 0; j < H; ++j) {
            x[j] = x0;
            pos[j] = at(ln[j], x0);
        }
        const int dx = side ? -1 : 1;
        const uint32_t stepb = side ? (uint32_t)(-(int32_t)GSB) : GSB;
        const uint32_t zcol = (uint32_t)P;
        uint2 nx = stw[0];
        for (int t = 0; t < T4; ++t) {
            const uint32_t w = nx.x, f = nx.y;
            nx = stw[t + 1];
            if (f & kFwdSync) named_barrier_sync(1, 64);
            uint64_t own[H], c[H];
#pragma unroll
            for (int j = 0; j < H; ++j) {
                uint64_t v[Q];
#pragma unroll
                for (int l2 = 0; l2 < Q; ++l2) {
                    uint32_t o;
                    if constexpr (PAD) o = pos[j] + off[j][l2];
                    else o = rowa[l2] + min((uint32_t)(x[j] + dk[j][l2]), zcol) * GSB;
                    v[l2] = ld_s64(o);
                }
                own[j] = hh ? v[(H + j) < Q ? H + j : 0] : v[j];
                uint64_t s = 0;
#pragma unroll
                for (int l2 = 0; l2 < Q; ++l2) s ^= v[l2];
                c[j] = s ^ own[j];   // the other words of the bin line
            }
            // same-step chain within the lane, top line down
            uint64_t fwm[H];
#pragma unroll
            for (int j = 0; j < H; ++j) fwm[j] = 0ull - (uint64_t)((f >> sh[j]) & (lv[j] ? 1u : 0u));
#pragma unroll
            for (int j = H - 2; j >= 0; --j) c[j] ^= c[j + 1] & fwm[j];
            // the lower half's top line links to the upper half's bottom line
            const uint64_t up = __shfl_down_sync(0xffffffffu, c[0], 16);
            uint64_t link = hh == 0 ? fwm[H - 1] : 0ull;
#pragma unroll
            for (int j = H - 1; j >= 0; --j) {
                if (j < H - 1) link &= fwm[j];
                c[j] ^= up & link;
            }
#pragma unroll
            for (int j = 0; j < H; ++j) {
                const uint32_t mv = (w >> sh[j]) & 1u;
                st_s64_if(pos[j], own[j] ^ c[j], (gok && lv[j]) ? mv : 0u);
                pos[j] += mv ? stepb : 0u;
                if constexpr (!PAD) x[j] += mv ? dx : 0;
            }
            __syncwarp();
        }
        __syncthreads();

        // write-back, 32 consecutive words of a row per instruction
        {
            const int nrows = nst * Q;
            for (int r = side; r < nrows; r += 2) {
                const int gg = r / Q, ll = r - gg * Q;
                uint64_t *out = BATCHED ? a.dstp[first + gg] : a.img + (s0 + gg) * (int64_t)Q * P;
                const uint64_t *row = wbuf + (int64_t)a.rowbase[ll] * GS + gg;
                for (int xx = lane; xx < P; xx += 32) __stcs(out + (int64_t)ll * P + xx, row[(int64_t)xx * GS]);
            }
        }
        __syncthreads();
    });
}

// ---------------------------------------------------------------------------
// decode_ring: the path of Sec. 2.2 swept from the left end of every line
// only (one front per line, the path built with split = P), each (stripe,
// line) keeping a ring of R words of shared memory instead of its whole row:
// for long lines the stripe's window -- the bins just ahead of the fronts
// and the pixels the other lines still read just behind them -- is a small
// part of the stripe, so several times more stripes fit on an SM.
//
// Lane = line * G + g (G = 32 / Q stripes per warp, one work item). Column c
// of line l sits at ring slot R - 1 - ((c + delta_l) mod R), in the order of
// the line's bins. Chunks of 16 columns (c + delta_l in [16 k, 16 k + 16))
// are fetched D chunks ahead of the line's front by one 128-byte bulk copy
// per (stripe, line) -- delta_l makes the chunk's bins 16-byte aligned --
// completing on an mbarrier of the line's chunk slot; chunks overlapping
// the image's ends take 8-byte cp.async copies for their in-image words and
// zeros for the others, chunks outside the image zeros only, so a word
// outside the image always reads 0 with no bounds test. A front entering
// chunk k fetches chunk k + D and waits for chunk k. A 16-column chunk of
// pixels is written back (all lanes, 128 consecutive bytes per half-warp)
// after the step that rebuilds its last pixel. The host marks both events
// in the path (Schedule::ringev) and replays the path under exactly these
// rules before choosing this kernel: every read meets its bin, pixel or
// zero, every pixel is still there when written back (ring_fits, plan.cpp).
//
// A step is decode_lines' step: own bin, the Q - 1 words of the bin line
// (read even by a front that does not move: its slots are valid, its result
// unused), the same-step chain over the lines by warp shuffles, the pixel
// stored.
template <int QT, bool BATCHED>
__global__ void __launch_bounds__(32) decode_ring(const __grid_constant__ DecParams a)
{
    extern __shared__ __align__(16) uint64_t sm[];
    constexpr int Q = QT;
    constexpr int CH = kRingChunk;
    const int P = a.P, G = a.G;
    const int R = a.RP, D = a.reach, NS = a.RP / CH;
    const uint32_t RM = (uint32_t)R - 1u;
    const int lane = threadIdx.x & 31;
    const int lq = lane / G;
    const bool ok = lq < Q;
    const int l = ok ? lq : 0;
    const int g = ok ? lane - lq * G : 0;
    // mbarriers (Q lines x NS chunk slots), then the stripes' regions of SWr
    // words, line l2's ring at rowbase[l2] of its region
    const uint32_t bar0 = smem_addr(sm);
    const uint32_t rings = bar0 + (uint32_t)a.SWc * 8u;
    const uint32_t rbase = rings + (uint32_t)g * (uint32_t)a.SWr * 8u;
    if (lane == 0) {
        for (int i = 0; i < Q * NS; ++i) mbar_init(bar0 + 8u * (uint32_t)i, (uint32_t)G);
        mbar_init_fence();
    }
    __syncwarp();

    const DecGroup &gr = a.grp;
    const int p = gr.p[2 * l];
    const int dl = gr.ring_delta[l];
    // ring slot address of column c of the line whose ring starts at base,
    // u = c + its delta
    auto slot = [&](uint32_t base, int u) -> uint32_t { return base + ((~(uint32_t)u) & RM) * 8u; };
    const uint32_t orb = rbase + (uint32_t)a.rowbase[l] * 8u;   // this lane's own ring
    // the other lines of this lane's bin line, l + 1 + k (mod Q): ring and
    // column offset (l2 - l) p + delta_l2 from the front's column
    int eo[Q > 1 ? Q - 1 : 1];
    uint32_t ro[Q > 1 ? Q - 1 : 1];
#pragma unroll
    for (int k = 0; k < Q - 1; ++k) {
        const int l2 = (l + 1 + k) % Q;
        eo[k] = (gr.lpos[l2] - gr.lpos[l]) * p + gr.ring_delta[l2];
        ro[k] = rbase + (uint32_t)a.rowbase[l2] * 8u;
    }
    // steady steps: the links of the path's steady pattern (as decode_lines)
    int chain = 0;
    uint32_t slink[4] = {0u, 0u, 0u, 0u};
    {
        if (ok)
            for (int j = l; j + 1 < Q && ((gr.fwd >> (2 * j)) & 1u); ++j) ++chain;
        uint32_t c[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) c[j] = (j + 1 < Q) ? (gr.fwd >> (2 * j)) & 1u : 0u;
#pragma unroll
        for (int r = 0, d = 1; d < Q; ++r, d <<= 1) {
            uint32_t cl = 0;
#pragma unroll
            for (int j = 0; j < Q; ++j)
                if (j == l) cl = c[j];
            slink[r] = ok ? cl : 0u;
            uint32_t nc[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) nc[j] = (c[j] && j + d < Q) ? c[j + d] : 0u;
#pragma unroll
            for (int j = 0; j < Q; ++j) c[j] = nc[j];
        }
    }
    const int T = gr.T;
    // (step, forward, event, 0) per step, from the next multiple of 4 words
    // after the step and forward words; one zero entry after the last
    const uint4 *sw4 = reinterpret_cast<const uint4 *>(gr.steps + ((2 * T + 3) & ~3));
    uint32_t fpar = 0;   // bit s: phase parity of the latest fill of this line's chunk slot s
    bool dead = false;

    const int64_t nitems = (a.S + G - 1) / G;
    for_items(a, nitems, [&](int64_t item) {
        if (dead) return;
        const int64_t s0 = item * G;
        const int nst = (int)min64(G, a.S - s0);
        const bool live = ok && g < nst;
        const uint64_t *sb = a.proj + (s0 + g) * a.total;
        const int64_t src = gr.src[2 * l];   // bin of column c at word src - c
        // fill chunk k of this lane's ring: columns [16 k - dl, 16 k + 16 - dl)
        auto fill = [&](int k) {
            const int sl = k & (NS - 1);
            const uint32_t bar = bar0 + 8u * (uint32_t)(l * NS + sl);
            const int c0 = CH * k - dl;
            // the chunk's slots: ascending addresses hold descending columns
            const uint32_t dst = slot(orb, c0 + dl + CH - 1);
            fpar ^= 1u << sl;
            if (!ok) return;
            const uint64_t *gs = sb + (src - (c0 + CH - 1));
            if (live && c0 >= 0 && c0 + CH <= P && ((uintptr_t)gs & 15u) == 0) {
                mbar_arrive_expect_tx(bar, CH * 8u);
                tma_load_1d(dst, gs, CH * 8u, bar);
            } else if (live && c0 + CH > 0 && c0 < P) {
                for (int i = 0; i < CH; ++i) {
                    const int c = c0 + CH - 1 - i;
                    if (c >= 0 && c < P) cp_async8_s(dst + 8u * (uint32_t)i, sb + (src - c));
                    else st_s64(dst + 8u * (uint32_t)i, 0ull);
                }
                cp_async_mbar_arrive(bar);
            } else {
                for (int i = 0; i < CH; ++i) st_s64(dst + 8u * (uint32_t)i, 0ull);
                mbar_arrive(bar);
            }
        };
        auto wait = [&](int k) -> bool {
            const int sl = k & (NS - 1);
            return !ok || mbar_wait_bounded(bar0 + 8u * (uint32_t)(l * NS + sl), (fpar >> sl & 1u) ^ 1u);
        };
        auto give_up = [&]() {
            // a fetch did not land in time: report, let the copies still in
            // flight land (bounded) before the CTA's shared memory goes away
            if (lane == 0) atomicOr(a.status, kStatusWaitTimeout);
            if (ok)
                for (int sl = 0; sl < NS; ++sl)
                    mbar_wait_bounded(bar0 + 8u * (uint32_t)(l * NS + sl), (fpar >> sl & 1u) ^ 1u);
            dead = true;
        };

        // the previous item's accesses of the rings before the bulk writes
        fence_proxy_async_smem();
        __syncwarp();
        for (int k = -1; k <= D; ++k) fill(k);
        if (__any_sync(0xffffffffu, !wait(0))) {
            give_up();
            return;
        }
        __syncwarp();

        int x = 0;
        uint4 nx = sw4[0];
        for (int t = 0; t < T; ++t) {
            const uint32_t w = nx.x, f = nx.y, ev = nx.z;
            nx = sw4[t + 1];
            if (ev & 0xFFu) {
                // fronts entering a chunk: fetch the one D ahead, wait for this one
                fence_proxy_async_smem();
                __syncwarp();
                bool okk = true;
                if (ok && (ev >> l & 1u)) {
                    const int k = (x + dl) / CH;
                    fill(k + D);
                    okk = wait(k);
                }
                if (__any_sync(0xffffffffu, !okk)) {
                    give_up();
                    return;
                }
                __syncwarp();
            }
            const uint32_t at = slot(orb, x + dl);
            const uint64_t own = ld_s64(at);
            uint64_t lv[Q > 1 ? Q - 1 : 1];
#pragma unroll
            for (int k = 0; k < Q - 1; ++k) lv[k] = ld_s64(slot(ro[k], x + eo[k]));
            uint64_t v = 0;
#pragma unroll
            for (int k = 0; k < Q - 1; ++k) v ^= lv[k];
            uint32_t act;
            if (w & kStepSteady) {
                act = ok ? 1u : 0u;
                if constexpr (Q <= 4) {
                    const uint64_t x0 = v;
#pragma unroll
                    for (int d = 1; d < Q; ++d) {
                        const uint64_t tv = __shfl_down_sync(0xffffffffu, x0, d * G);
                        if (d <= chain) v ^= tv;
                    }
                } else {
#pragma unroll
                    for (int r = 0, d = 1; d < Q; ++r, d <<= 1) {
                        const uint64_t tv = __shfl_down_sync(0xffffffffu, v, d * G);
                        if (slink[r]) v ^= tv;
                    }
                }
            } else {
                act = ok ? (w >> (2 * l)) & 1u : 0u;
                uint32_t c = (ok && act) ? (f >> (2 * l)) & 1u : 0u;
#pragma unroll
                for (int d = 1; d < Q; d <<= 1) {
                    const uint64_t tv = __shfl_down_sync(0xffffffffu, v, d * G);
                    const uint32_t tc = __shfl_down_sync(0xffffffffu, c, d * G);
                    if (c) {
                        v ^= tv;
                        c = tc;
                    }
                }
            }
            st_s64_if(at, own ^ v, act);
            x += act ? 1 : 0;
            __syncwarp();
            if (ev >> 8) {
                // write back the 16-column chunks just completed, a line at a time
                uint32_t lines = (ev >> 8) & 0xFFu;
                while (lines) {
                    const int l2 = __ffs(lines) - 1;
                    lines &= lines - 1;
                    const int xc = __shfl_sync(0xffffffffu, x, l2 * G) - 1;   // the chunk's last column
                    const int c = xc - (CH - 1) + (lane & (CH - 1));
                    const int u2 = c + gr.ring_delta[l2];
                    for (int gg = lane >> 4; gg < nst; gg += 2) {
                        const uint32_t rg = rings + (uint32_t)gg * (uint32_t)a.SWr * 8u + (uint32_t)a.rowbase[l2] * 8u;
                        __stcs(a.img + (s0 + gg) * (int64_t)Q * P + (int64_t)l2 * P + c, ld_s64(slot(rg, u2)));
                    }
                }
            }
        }
        __syncwarp();
    });
}

// ---------------------------------------------------------------------------
// decode_cols: decode_lines' arithmetic with the lines interleaved as well as
// the stripes. Word (line l, column c, stripe g) of a warp's slot sits at
// ((c + reach) * Q + l) * G + g: one column of all Q lines of the G stripes
// fills Q * G = 16 consecutive words (128 bytes, one shared-memory wavefront
// row), so the bank slot of a word is its line. The lanes are split by
// front: lanes 0..15 run the left fronts of lines 0..Q-1 (G lanes each),
// lanes 16..31 the right fronts. In every load of a step, the lanes of one
// front read Q different lines (their own, or line l+1+k mod Q for operand
// k), hence Q different bank slots, whatever their columns: a 64-bit load
// (served per half-warp) takes one wavefront per half instead of the
// several that colliding rows cost. Columns of zeros pad both ends of the
// rows (pixels outside the image, the XOR identity).
template <int QT, bool BATCHED>
__global__ void __launch_bounds__(32) decode_cols(const __grid_constant__ DecParams a)
{
    extern __shared__ __align__(16) uint64_t sm[];
    constexpr int Q = QT;
    const int P = a.P, G = a.G;
    const int CW = Q * G;            // words per column
    const int lane = threadIdx.x & 31;
    uint32_t *stepw = reinterpret_cast<uint32_t *>(sm);
    uint32_t *fwdw = stepw + a.TS;
    uint64_t *wbuf = sm + a.TS;
    for (int i = lane; i < a.SWc * G; i += 32) wbuf[i] = 0;
    const uint32_t wbase = smem_addr(wbuf);

    // Rebuild lanes: lane = 16 * side + l * G + g; lanes past Q*G in a half
    // shadow line 0 of their side (same loads, no stores).
    const int side = lane >> 4;
    const int r = lane & 15;
    const bool ok = r < CW;
    const int l = ok ? r / G : 0;
    const int g = ok ? r - (r / G) * G : 0;
    const int ls = 2 * l + side;
    const uint32_t bitmask = ok ? 1u << ls : 0u;
    const uint32_t start = wbase + (((a.reach + (side ? P - 1 : 0)) * Q + l) * G + g) * 8;
    const int stepb = (side ? -1 : 1) * CW * 8;
    const uint32_t has_next = (l + 1 < Q) ? 1u : 0u;

    int T4 = 0, d0 = 0;
    int dk[Q > 2 ? Q - 2 : 1];
    uint32_t sfw = 0u;
    uint32_t slink[4] = {0u, 0u, 0u, 0u};
    auto load_group = [&](const DecGroup &gr) {
        const int T = gr.T;
        T4 = (T + 3) & ~3;
        for (int t = lane; t < T4; t += 32) {
            stepw[t] = t < T ? gr.steps[t] : 0u;
            fwdw[t] = t < T ? gr.steps[T + t] : 0u;
        }
        // bytes from this lane's pixel to pixel (l2, x + (l2 - l) p)
        const int p = gr.p[ls];
        auto off = [&](int l2) { return ((l2 - l) * p * Q + (l2 - l)) * G * 8; };
        d0 = off(has_next ? l + 1 : 0);
#pragma unroll
        for (int k = 1; k < Q - 1; ++k) dk[k - 1] = off((l + 1 + k) % Q);
        sfw = ok ? (gr.fwd >> ls) & 1u : 0u;
        uint32_t c[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) c[j] = (j + 1 < Q) ? (gr.fwd >> (2 * j + side)) & 1u : 0u;
#pragma unroll
        for (int rr = 0, d = 1; d < Q; ++rr, d <<= 1) {
            slink[rr] = ok ? c[l] : 0u;
            uint32_t nc[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) nc[j] = (c[j] && j + d < Q) ? c[j + d] : 0u;
#pragma unroll
            for (int j = 0; j < Q; ++j) c[j] = nc[j];
        }
    };
    const DecGroup *gp = nullptr;
    auto grp = [&]() -> const DecGroup & {
        if constexpr (BATCHED) return *gp;
        else return a.grp;
    };
    if constexpr (!BATCHED) load_group(a.grp);
    __syncwarp();

    // Copy lanes: lane = (xk * Q + ll) * G + gg covers XC columns per pass,
    // so adjacent lanes touch adjacent shared-memory words.
    const int XC = 32 / CW;
    const int xk = lane / CW, rem = lane - xk * CW;
    const int ll = rem / G, gg = rem - (rem / G) * G;
    const bool copy_ok = xk < XC;

    int cur = -1;
    const int64_t nitems = BATCHED ? a.nwork : (a.S + G - 1) / G;
    for_items(a, nitems, [&](int64_t item) {
        int nst;
        int64_t s0 = 0, first = 0;
        if constexpr (BATCHED) {
            const DecWork wk = a.work[item];
            nst = wk.nst;
            first = wk.first;
            if (wk.group != cur) {
                cur = wk.group;
                gp = a.groups + cur;
                __syncwarp();
                load_group(*gp);
                __syncwarp();
            }
        } else {
            s0 = item * G;
            nst = (int)min64(G, a.S - s0);
        }

        if (copy_ok && gg < nst) {
            const uint64_t *src = BATCHED ? a.srcp[first + gg] : a.proj + (s0 + gg) * a.total;
            const int sp = grp().split[ll];
            const int sl = grp().src[2 * ll], sr = grp().src[2 * ll + 1];
            uint64_t *dst = wbuf + (a.reach * Q + ll) * G + gg;
            for (int x = xk; x < P; x += XC)
                cp_async8(dst + x * CW, src + ((x < sp ? sl : sr) - x));
        }
        cp_async_wait_all();
        __syncwarp();

        uint32_t pos = start;
        uint32_t w_next = stepw[0], f_next = fwdw[0];
        for (int t = 0; t < T4; ++t) {
            const uint32_t w = w_next, f = f_next;
            w_next = stepw[t + 1];
            f_next = fwdw[t + 1];
            if (w & kStepSteady) {
                uint64_t v = ld_s64(pos);
#pragma unroll
                for (int k2 = 0; k2 < Q - 2; ++k2) v ^= ld_s64(pos + dk[k2]);
                if (Q > 1) v ^= ld_s64_if(pos + d0, (sfw & has_next) ^ 1u);
#pragma unroll
                for (int rr = 0, d = 1; d < Q; ++rr, d <<= 1) {
                    const uint64_t tv = __shfl_down_sync(0xffffffffu, v, d * G);
                    if (slink[rr]) v ^= tv;
                }
                st_s64_if(pos, v, ok);
                pos += stepb;
                __syncwarp();
                continue;
            }
            const uint32_t act = w & bitmask;
            const uint32_t fw = ok ? (f >> ls) & 1u : 0u;
            uint64_t v = ld_s64(pos);
#pragma unroll
            for (int k2 = 0; k2 < Q - 2; ++k2) v ^= ld_s64(pos + dk[k2]);
            if (Q > 1) v ^= ld_s64_if(pos + d0, (fw & has_next) ^ 1u);
            uint32_t c = fw;
#pragma unroll
            for (int d = 1; d < Q; d <<= 1) {
                const uint64_t tv = __shfl_down_sync(0xffffffffu, v, d * G);
                const uint32_t tc = __shfl_down_sync(0xffffffffu, c, d * G);
                if (c) {
                    v ^= tv;
                    c = tc;
                }
            }
            st_s64_if(pos, v, act);
            pos += act ? stepb : 0;
            __syncwarp();
        }

        if (copy_ok && gg < nst) {
            uint64_t *out = BATCHED ? a.dstp[first + gg] : a.img + (s0 + gg) * (int64_t)Q * P;
            const uint64_t *buf = wbuf + (a.reach * Q + ll) * G + gg;
            for (int x = xk; x < P; x += XC) __stcs(out + ll * P + x, buf[x * CW]);
        }
        __syncwarp();
    });
}

// ---------------------------------------------------------------------------
// decode_stream: decode_lines' lanes and steps, with the stripe streamed
// through shared memory instead of staged and written whole:
//   - rows are packed at pitch RP (no zero columns between them); an operand
//     outside the image reads one zero column instead, chosen per operand
//     from the front's column, so a stripe takes Q*P words of shared memory
//     and more stripes fit on an SM;
//   - the bins arrive in kStreamChunks cp.async groups ordered by distance
//     from the ends where the fronts start; the step loop waits for chunk c
//     only before the first step that reaches it, so later chunks land
//     while the first ones are being rebuilt;
//   - each chunk goes back to global memory as soon as its last pixel is
//     rebuilt, so the write-out overlaps the remaining steps.
// The chunk steps come with the path (Schedule::chunk_wait, chunk_done).
template <int QT, bool BATCHED>
__global__ void __launch_bounds__(32) decode_stream(const __grid_constant__ DecParams a)
{
    extern __shared__ __align__(16) uint64_t sm[];
    constexpr int Q = QT;
    constexpr int NC = kStreamChunks;
    const int P = a.P, G = a.G, RP = a.RP;
    const int lane = threadIdx.x & 31;
    uint32_t *stepw = reinterpret_cast<uint32_t *>(sm);
    uint32_t *fwdw = stepw + a.TS;
    uint64_t *wbuf = sm + a.TS;
    // the zero column after the rows
    if (lane < G) wbuf[(size_t)Q * RP * G + lane] = 0;
    const uint32_t wbase = smem_addr(wbuf);

    // Rebuild lanes: lane = (2l + side) * G + g; lanes past 2Q*G shadow lane 0.
    const int lsr = lane / G;
    const bool ok = lsr < 2 * Q;
    const int ls = ok ? lsr : 0;
    const int g = ok ? lane - lsr * G : 0;
    const int l = ls >> 1, side = ls & 1;
    const uint32_t bitmask = ok ? 1u << ls : 0u;
    const uint32_t start = wbase + ((l * RP + (side ? P - 1 : 0)) * G + g) * 8;
    const uint32_t zaddr = wbase + ((Q * RP) * G + g) * 8;
    const int stepb = (side ? -1 : 1) * G * 8;
    const int dir = side ? -1 : 1;
    const uint32_t has_next = (l + 1 < Q) ? 1u : 0u;

    // Path-dependent state: for the operands on lines l2 = l+1+k (mod Q),
    // k = 0 .. Q-2, the column offset (l2 - l) p and the byte offset from
    // this lane's pixel; slink / sfw as in decode_lines.
    int T4 = 0;
    int ecol[Q > 1 ? Q - 1 : 1], eoff[Q > 1 ? Q - 1 : 1];
    uint32_t sfw = 0u;
    uint32_t slink[4] = {0u, 0u, 0u, 0u};
    int cw = 1, cwait[NC], cdone[NC];
    auto load_group = [&](const DecGroup &gr) {
        const int T = gr.T;
        T4 = (T + 3) & ~3;
        for (int t = lane; t < T4; t += 32) {
            stepw[t] = t < T ? gr.steps[t] : 0u;
            fwdw[t] = t < T ? gr.steps[T + t] : 0u;
        }
        const int p = gr.p[ls];
#pragma unroll
        for (int k = 0; k < Q - 1; ++k) {
            const int l2 = (l + 1 + k) % Q;
            ecol[k] = (l2 - l) * p;
            eoff[k] = (l2 - l) * (RP + p) * G * 8;
        }
        sfw = ok ? (gr.fwd >> ls) & 1u : 0u;
        uint32_t c[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) c[j] = (j + 1 < Q) ? (gr.fwd >> (2 * j + side)) & 1u : 0u;
#pragma unroll
        for (int r = 0, d = 1; d < Q; ++r, d <<= 1) {
            slink[r] = ok ? c[l] : 0u;
            uint32_t nc[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) nc[j] = (c[j] && j + d < Q) ? c[j + d] : 0u;
#pragma unroll
            for (int j = 0; j < Q; ++j) c[j] = nc[j];
        }
        cw = gr.chunk_w;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            cwait[q] = gr.chunk_wait[q];
            cdone[q] = gr.chunk_done[q];
        }
    };
    const DecGroup *gp = nullptr;
    auto grp = [&]() -> const DecGroup & {
        if constexpr (BATCHED) return *gp;
        else return a.grp;
    };
    if constexpr (!BATCHED) load_group(a.grp);
    __syncwarp();

    // Copy lanes: lane = xk * G + gg covers XK columns of G stripes.
    const int XK = 32 / G;
    const int xk = lane / G, gg = lane - xk * G;
    const bool copy_ok = xk < XK;

    // Columns of chunk q on line ll: the left front's x in [d0, min(d1, sp))
    // and the right front's x = P-1-d, d in [d0, min(d1, P - sp)).
    auto chunk_cols = [&](int q, int ll, auto &&fn) {
        const int d0 = q * cw, d1 = (q == NC - 1) ? P : (q + 1) * cw;
        const int sp = grp().split[ll];
        const int eL = min(d1, sp), eR = min(d1, P - sp);
        for (int x = d0 + xk; x < eL; x += XK) fn(x, 0);
        for (int d = d0 + xk; d < eR; d += XK) fn(P - 1 - d, 1);
    };

    int cur = -1;
    const int64_t nitems = BATCHED ? a.nwork : (a.S + G - 1) / G;
    for_items(a, nitems, [&](int64_t item) {
        int nst;
        int64_t s0 = 0, first = 0;
        if constexpr (BATCHED) {
            const DecWork wk = a.work[item];
            nst = wk.nst;
            first = wk.first;
            if (wk.group != cur) {
                cur = wk.group;
                gp = a.groups + cur;
                __syncwarp();
                load_group(*gp);
                __syncwarp();
            }
        } else {
            s0 = item * G;
            nst = (int)min64(G, a.S - s0);
        }
        const bool mine = copy_ok && gg < nst;
        const uint64_t *src = nullptr;
        uint64_t *out = nullptr;
        if (mine) {
            src = BATCHED ? a.srcp[first + gg] : a.proj + (s0 + gg) * a.total;
            out = BATCHED ? a.dstp[first + gg] : a.img + (s0 + gg) * (int64_t)Q * P;
        }

        // stage: one cp.async group per chunk (empty groups for idle lanes)
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            if (mine)
                for (int ll = 0; ll < Q; ++ll) {
                    const int sl = grp().src[2 * ll], sr = grp().src[2 * ll + 1];
                    uint64_t *dst = wbuf + (size_t)ll * RP * G + gg;
                    chunk_cols(q, ll, [&](int x, int right) {
                        cp_async8(dst + x * G, src + ((right ? sr : sl) - x));
                    });
                }
            cp_async_commit();
        }
        // write chunk q of every line back
        auto put = [&](int q) {
            if (mine)
                for (int ll = 0; ll < Q; ++ll) {
                    const uint64_t *buf = wbuf + (size_t)ll * RP * G + gg;
                    chunk_cols(q, ll, [&](int x, int) { __stcs(out + ll * P + x, buf[x * G]); });
                }
        };
        auto wait_chunk = [&](int q) {
            switch (q) {
            case 0: cp_async_wait_group<NC - 1>(); break;
            case 1: cp_async_wait_group<NC - 2 < 0 ? 0 : NC - 2>(); break;
            case 2: cp_async_wait_group<NC - 3 < 0 ? 0 : NC - 3>(); break;
            default: cp_async_wait_all(); break;
            }
            __syncwarp();
        };

        // chunk q's wait / done step, kept in registers (constant indices only)
        auto chunk_step = [&](const int (&tab)[NC], int q) {
            int v = 0x7fffffff;
#pragma unroll
            for (int i = 0; i < NC; ++i) v = (i == q) ? tab[i] : v;
            return v;
        };
        uint32_t pos = start;
        int x = side ? P - 1 : 0;   // this lane's front column
        int ev = 0, ov = 0;
        int next_wait = cwait[0], next_done = cdone[0];
        // operand address: its pixel, or the zero column outside the image
        auto opaddr = [&](int k) -> uint32_t {
            return (unsigned)(x + ecol[k]) < (unsigned)P ? pos + eoff[k] : zaddr;
        };
        for (int t = 0; t < T4; ++t) {
            while (t >= next_wait) {
                wait_chunk(ev++);
                next_wait = chunk_step(cwait, ev);
            }
            const uint32_t w = stepw[t];
            const bool steady = (w & kStepSteady) != 0;
            const uint32_t f = steady ? 0u : fwdw[t];
            const uint32_t fw = steady ? sfw : (ok ? (f >> ls) & 1u : 0u);
            uint64_t v = ld_s64(pos);
#pragma unroll
            for (int k = 1; k < Q - 1; ++k) v ^= ld_s64(opaddr(k));
            if (Q > 1) {
                const uint32_t a0 = opaddr(0);
                v ^= ld_s64_if(a0, (fw & has_next) ^ 1u);
            }
            uint32_t act;
            if (steady) {
#pragma unroll
                for (int r = 0, d = 1; d < Q; ++r, d <<= 1) {
                    const uint64_t tv = __shfl_down_sync(0xffffffffu, v, 2 * d * G);
                    if (slink[r]) v ^= tv;
                }
                act = ok ? 1u : 0u;
            } else {
                uint32_t c = fw;
#pragma unroll
                for (int d = 1; d < Q; d <<= 1) {
                    const uint64_t tv = __shfl_down_sync(0xffffffffu, v, 2 * d * G);
                    const uint32_t tc = __shfl_down_sync(0xffffffffu, c, 2 * d * G);
                    if (c) {
                        v ^= tv;
                        c = tc;
                    }
                }
                act = w & bitmask;
            }
            st_s64_if(pos, v, act);
            if (act) {
                pos += stepb;
                x += dir;
            }
            __syncwarp();
            while (t >= next_done) {
                put(ov++);
                next_done = chunk_step(cdone, ov);
            }
        }
        cp_async_wait_all();
        __syncwarp();
        while (ov < NC) put(ov++);
        __syncwarp();
    });
}

// ---------------------------------------------------------------------------
// decode_scan2: the inverse for exactly two unknown lines -- a two-line image
// (Q = 2), or a systematic stripe that lost two data lines -- in closed form
// instead of a step-by-step path. Lines u (image row l1) and v (row l2 =
// l1 + d) with projections a and b, p_a < p_b, each over its whole line.
// With the known lines removed (systematic), Eq. 1 leaves in the bin of
// pixel (l1, x) of projection a:  Ra(x) = u[x] ^ v[x + d p_a]  and in the
// bin of pixel (l2, y) of projection b:  Rb(y) = v[y] ^ u[y - d p_b]
// (a term outside the image absent). Substituting v gives
//     u[x] = c(x) ^ link(x) u[x - s],   s = d (p_b - p_a) >= 1,
// with c(x) = Ra(x) ^ Rb(x + d p_a) when x + d p_a is inside the image (else
// Ra(x), and no link), link(x) also needing x >= s: a prefix XOR along each
// chain x, x - s, x - 2s, ... cut where a link is missing. It is evaluated by
// pointer doubling -- round r joins each element to the one s 2^r before it
// while its chain continues, ceil(log2(P / s)) rounds -- and then
// v[y] = Rb(y) ^ u[y - d p_b]. The values are those of the Sec. 2.2 inverse
// (the image is unique); the work is independent per element, so the kernel
// is bound by memory traffic, not by a chain of ~P/2 dependent steps.
// One warp per stripe (kScanWarps stripes per work item and CTA); per warp
// the shared memory holds two copies of u (ping-pong), Rb, and two rows of
// chain flags.
__host__ __device__ inline int scan2_words(int P) { return 3 * P + (2 * P + 7) / 8; }
constexpr int kScanBatch = 8;

template <bool BATCHED, bool SYS>
__global__ void __launch_bounds__(32 * kScanWarps) decode_scan2(const __grid_constant__ DecParams a)
{
    extern __shared__ __align__(16) uint64_t sm[];
    const int P = a.P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *U0 = sm + (size_t)warp * scan2_words(P);
    uint64_t *U1 = U0 + P, *V = U1 + P;
    uint8_t *F0 = reinterpret_cast<uint8_t *>(V + P), *F1 = F0 + P;

    const int64_t nitems = BATCHED ? a.nwork : (a.S + a.G - 1) / a.G;
    for_items(a, nitems, [&](int64_t item) {
        const DecGroup *gr;
        int nst;
        int64_t s0 = 0, first = 0;
        if constexpr (BATCHED) {
            const DecWork wk = a.work[item];
            gr = a.groups + wk.group;
            nst = wk.nst;
            first = wk.first;
        } else {
            gr = &a.grp;
            s0 = item * a.G;
            nst = (int)min64(a.G, a.S - s0);
        }
        if (warp < nst) {
            const uint64_t *src = BATCHED ? a.srcp[first + warp] : a.proj + (s0 + warp) * a.total;
            uint64_t *out = BATCHED ? a.dstp[first + warp]
                                    : a.img + (s0 + warp) * (int64_t)(SYS ? a.Qd : 2) * P;
            const int l1 = SYS ? gr->lpos[0] : 0, l2 = SYS ? gr->lpos[1] : 1, d = l2 - l1;
            const int pa = gr->scan_p[0], pb = gr->scan_p[1];
            const int sa = gr->scan_src[0], sb = gr->scan_src[1];
            const int s = d * (pb - pa);
            const uint32_t known = SYS ? gr->known : 0u;
            // residual bins of both lines (the known lines removed), kScanBatch
            // columns per lane at a time so that each round of loads -- the
            // bins, then each known line -- is in flight together
            for (int x0 = lane; x0 < P; x0 += 32 * kScanBatch) {
                uint64_t ra[kScanBatch], rb[kScanBatch];
#pragma unroll
                for (int c = 0; c < kScanBatch; ++c) {
                    const int x = x0 + 32 * c;
                    const bool in = x < P;
                    ra[c] = in ? __ldcs(src + (sa - x)) : 0ull;
                    rb[c] = in ? __ldcs(src + (sb - x)) : 0ull;
                }
                if constexpr (SYS) {
                    for (uint32_t k = known; k; k &= k - 1) {
                        const int l = __ffs(k) - 1;
                        const uint64_t *row = out + (int64_t)l * P;
                        uint64_t ta[kScanBatch], tb[kScanBatch];
#pragma unroll
                        for (int c = 0; c < kScanBatch; ++c) {
                            const int x = x0 + 32 * c;
                            const int xa = x + (l - l1) * pa, xb = x + (l - l2) * pb;
                            ta[c] = (x < P && (unsigned)xa < (unsigned)P) ? row[xa] : 0ull;
                            tb[c] = (x < P && (unsigned)xb < (unsigned)P) ? row[xb] : 0ull;
                        }
#pragma unroll
                        for (int c = 0; c < kScanBatch; ++c) {
                            ra[c] ^= ta[c];
                            rb[c] ^= tb[c];
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < kScanBatch; ++c) {
                    const int x = x0 + 32 * c;
                    if (x < P) {
                        U1[x] = ra[c];
                        V[x] = rb[c];
                    }
                }
            }
            __syncwarp();
            // c(x) and the first links
            for (int x = lane; x < P; x += 32) {
                const int y = x + d * pa;
                const bool in = (unsigned)y < (unsigned)P;
                const uint64_t vy = V[in ? y : x];          // every index read is in range
                U0[x] = U1[x] ^ (in ? vy : 0ull);
                F0[x] = (in && x >= s) ? 1 : 0;
            }
            __syncwarp();
            // pointer doubling along the chains: an element whose chain still
            // continues (flag set, hence x >= k) takes the XOR of the span k
            // before it and inherits that span's flag
            uint64_t *Ui = U0, *Uo = U1;
            uint8_t *Fi = F0, *Fo = F1;
            for (int k = s; k < P; k <<= 1) {
                for (int x0 = lane; x0 < P; x0 += 32 * kScanBatch) {
                    // flags first, then every partner of the batch at once
                    bool f[kScanBatch];
#pragma unroll
                    for (int c = 0; c < kScanBatch; ++c) {
                        const int x = x0 + 32 * c;
                        f[c] = x < P && Fi[x] != 0;
                    }
                    uint64_t ux[kScanBatch], uk[kScanBatch];
                    uint8_t fk[kScanBatch];
#pragma unroll
                    for (int c = 0; c < kScanBatch; ++c) {
                        const int x = x0 + 32 * c;
                        const int xi = x < P ? x : 0;
                        const int xk = f[c] ? x - k : xi;
                        ux[c] = Ui[xi];
                        uk[c] = Ui[xk];
                        fk[c] = Fi[xk];
                    }
#pragma unroll
                    for (int c = 0; c < kScanBatch; ++c) {
                        const int x = x0 + 32 * c;
                        if (x < P) {
                            Uo[x] = f[c] ? ux[c] ^ uk[c] : ux[c];
                            Fo[x] = f[c] ? fk[c] : 0;
                        }
                    }
                }
                __syncwarp();
                uint64_t *tu = Ui; Ui = Uo; Uo = tu;
                uint8_t *tf = Fi; Fi = Fo; Fo = tf;
            }
            // u is final; v[y] = Rb(y) ^ u[y - d p_b]
            for (int x = lane; x < P; x += 32) {
                const int xu = x - d * pb;
                const bool in = (unsigned)xu < (unsigned)P;
                const uint64_t ux = Ui[in ? xu : x];
                __stcs(out + (int64_t)l1 * P + x, Ui[x]);
                __stcs(out + (int64_t)l2 * P + x, V[x] ^ (in ? ux : 0ull));
            }
            __syncwarp();
        }
    });
}

// ---------------------------------------------------------------------------
// decode_vander: every line at once, from the Vandermonde form of Eq. 1.
// Write line l as the Laurent polynomial U_l(z) = sum_x f(x, l) z^(-x) and
// projection i as R_i(z) = sum_b bin_b z^b; Eq. 1 with q = 1 says
//     R_i = sum_l U_l w_i^l,   w_i = z^(p_i),
// a Vandermonde system over GF(2)[z, 1/z] in the Q unknowns U_l, which has
// one solution when the Q directions differ (Eq. 3). It is solved by the
// Bjorck-Pereyra algorithm (Newton divided differences, then the Newton to
// monomial conversion), whose only non-trivial step is a division by
// w_i - w_j = z^(p_j) (1 + z^d), d = p_i - p_j > 0: a shift, then a prefix
// XOR with stride d (q[e] = a[e] ^ q[e - d], exact because the quotient is
// a polynomial). Over the Q chosen projections (ascending p):
//   for k = 0 .. Q-2, i = Q-1 down to k+1, j = i-k-1:
//       c_i <- (c_i ^ c_{i-1}) / (w_i - w_j)
//   for k = Q-2 down to 0, i = k .. Q-2:
//       c_i <- c_i ^ w_k c_{i+1}
// and then c_l = U_l. Every polynomial lives on one frame of positions
// [E0, E0 + L) (the bins' span plus one; no intermediate leaves it). A
// division's prefix runs along the d chains r, r + d, r + 2d, ... of the
// frame, each split into segments over several lanes: a pass for the
// segments' XOR totals, a segmented shuffle scan across the lanes of a
// chain, a pass writing the prefix with its carry. No step waits on
// another stripe or on a ~P/2-step path: the work is ~Q^2 / 2 parallel
// passes over the frame. One warp per stripe, kVanWarps per CTA; per warp
// Q + 1 frame arrays in shared memory (one spare for division outputs).
template <int QT, bool BATCHED>
__global__ void __launch_bounds__(32 * kVanWarps) decode_vander(const __grid_constant__ DecParams a)
{
    extern __shared__ __align__(16) uint64_t sm[];
    constexpr int Q = QT;
    constexpr int JMAX = 16;            // chain-segment values kept in registers
    const int P = a.P;
    const int L = a.RP;                 // frame words (the same for every path of the launch)
    const int PAD = a.reach;            // zero words on both sides of each array
    const int AS = L + 2 * PAD;         // array stride
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *wbase = sm + (size_t)warp * a.SWc;
    // the pads are never written: zero them once
    for (int j = 0; j <= Q; ++j)
        for (int t = lane; t < PAD; t += 32) {
            wbase[(size_t)j * AS + t] = 0ull;
            wbase[(size_t)j * AS + PAD + L + t] = 0ull;
        }
    uint64_t *base = wbase + PAD;

    const int64_t nitems = BATCHED ? a.nwork : (a.S + a.G - 1) / a.G;
    for_items(a, nitems, [&](int64_t item) {
        const DecGroup *gr;
        int nst;
        int64_t s0 = 0, first = 0;
        if constexpr (BATCHED) {
            const DecWork wk = a.work[item];
            gr = a.groups + wk.group;
            nst = wk.nst;
            first = wk.first;
        } else {
            gr = &a.grp;
            s0 = item * a.G;
            nst = (int)min64(a.G, a.S - s0);
        }
        if (warp < nst) {
            const uint64_t *src = BATCHED ? a.srcp[first + warp] : a.proj + (s0 + warp) * a.total;
            uint64_t *out = BATCHED ? a.dstp[first + warp] : a.img + (s0 + warp) * (int64_t)Q * P;
            const int E0 = gr->van_E0;
            int q[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) q[j] = gr->van_q[j];
            // physical array of each c_j, and the spare one
            int phys[Q + 1];
#pragma unroll
            for (int j = 0; j <= Q; ++j) phys[j] = j;
            auto arr = [&](int j) { return base + (size_t)phys[j] * AS; };

            // stage the bins: array j position e - E0 <- bin e of projection j
            // (0 outside the projection)
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const int lo = gr->van_lo[j] - E0, hi = gr->van_hi[j] - E0;
                const uint64_t *sj = src + (gr->van_base[j] + E0);
                uint64_t *c = base + (size_t)j * AS;
                for (int t = lane; t < L; t += 32) {
                    if (t >= lo && t < hi) cp_async8(c + t, sj + t);
                    else c[t] = 0ull;
                }
            }
            cp_async_wait_all();
            __syncwarp();

            // Newton divided differences: c_i <- (c_i ^ c_{i-1}) shifted by
            // -q_j, divided by 1 + z^d (prefix XOR along the d chains)
#pragma unroll
            for (int k = 0; k < Q - 1; ++k) {
#pragma unroll
                for (int i = Q - 1; i > k; --i) {
                    const int j = i - k - 1;
                    const int d = q[i] - q[j], sh = q[j];
                    const uint64_t *A = arr(i) + sh, *B = arr(i - 1) + sh;
                    uint64_t *O = arr(Q);
                    // chains r = 0 .. d-1 of the frame; cpp = 2^c >= d chains per
                    // pass, m = 32 / cpp lanes per chain (a power of two: lane
                    // -> (chain, segment) by mask and shift)
                    const int c = d <= 32 ? 32 - __clz(d - 1) : 5;
                    const int cpp = 1 << c, m = 32 >> c;
                    const int r0 = lane & (cpp - 1), sg = lane >> c;
                    for (int c0 = 0; c0 < d; c0 += cpp) {
                        const int r = c0 + r0;
                        // chain r holds positions r + d t, t < len_r
                        const int len0 = (L - c0 + d - 1) / d;        // warp-uniform
                        const int rem = L - c0 - (len0 - 1) * d;      // chains c0 .. c0+rem-1 have len0
                        const int J = (len0 + m - 1) >> (5 - c);
                        const int lenr = r < d ? (r0 < rem ? len0 : len0 - 1) : 0;
                        const int n = max(0, min(J, lenr - sg * J));
                        const int e0 = r + d * sg * J;
                        uint64_t nv[JMAX];
                        uint64_t tot = 0;
#pragma unroll
                        for (int t = 0; t < JMAX; ++t) {
                            if (t >= n) break;
                            nv[t] = A[e0 + t * d] ^ B[e0 + t * d];
                            tot ^= nv[t];
                        }
                        for (int t = JMAX; t < n; ++t) {
                            const int e = e0 + t * d;
                            tot ^= A[e] ^ B[e];
                        }
                        // inclusive scan over the segments of a chain (lanes cpp apart)
                        uint64_t inc = tot;
                        for (int w = 1; w < m; w <<= 1) {
                            const uint64_t o = __shfl_up_sync(0xffffffffu, inc, w << c);
                            if (sg >= w) inc ^= o;
                        }
                        uint64_t v = inc ^ tot;               // carry from earlier segments
#pragma unroll
                        for (int t = 0; t < JMAX; ++t) {
                            if (t >= n) break;
                            v ^= nv[t];
                            O[e0 + t * d] = v;
                        }
                        for (int t = JMAX; t < n; ++t) {
                            const int e = e0 + t * d;
                            v ^= A[e] ^ B[e];
                            O[e] = v;
                        }
                    }
                    __syncwarp();
                    const int tmp = phys[i];
                    phys[i] = phys[Q];
                    phys[Q] = tmp;
                }
            }
            // Newton form to the coefficients: c_i <- c_i ^ z^(q_k) c_{i+1};
            // the last level (k = 0) goes straight to the output
#pragma unroll
            for (int k = Q - 2; k >= 1; --k) {
#pragma unroll
                for (int i = k; i < Q - 1; ++i) {
                    uint64_t *C = arr(i);
                    const uint64_t *D = arr(i + 1) - q[k];
#pragma unroll 4
                    for (int t = lane; t < L; t += 32) C[t] ^= D[t];
                    __syncwarp();
                }
            }
            // line l = c_l ^ z^(q_0) c_{l+1} (c_{Q-1} as it is) at positions -x
#pragma unroll
            for (int l = 0; l < Q; ++l) {
                const uint64_t *C = arr(l) - E0;
                if (l + 1 < Q) {
                    const uint64_t *D = arr(l + 1) - E0 - q[0];
                    for (int x = lane; x < P; x += 32) __stcs(out + (int64_t)l * P + x, C[-x] ^ D[-x]);
                } else {
                    for (int x = lane; x < P; x += 32) __stcs(out + (int64_t)l * P + x, C[-x]);
                }
            }
            __syncwarp();
        }
    });
}

// ---------------------------------------------------------------------------
// sys_residual: first pass of a systematic decode. For every lost data line
// j (image row lpos[j]) and column x: the bin of the projection dedicated to
// the front that rebuilds x (direction pp), XOR the known lines' pixels of
// that bin's line, (l2, x + (l2 - lpos[j]) pp) -- Eq. 1's sum with the known
// pixels removed -- written into the lost line itself (its contents are
// garbage until rebuilt). With one lost line these are its pixels; with more,
// decode_lines<SYS> then runs the path on those rows. Memory-bound and
// independent per word: one warp per (stripe, lost line) row, lanes along x
// (coalesced loads of the bins, the known rows and the store).
template <bool BATCHED>
__global__ void __launch_bounds__(256) sys_residual(const __grid_constant__ DecParams a)
{
    const int P = a.P, E = a.Q;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t nitems = BATCHED ? a.nwork : (a.S + a.G - 1) / a.G;
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const DecGroup *gr;
        int nst;
        int64_t s0 = 0, first = 0;
        if constexpr (BATCHED) {
            const DecWork wk = a.work[item];
            gr = a.groups + wk.group;
            nst = wk.nst;
            first = wk.first;
        } else {
            gr = &a.grp;
            s0 = item * a.G;
            nst = (int)min64(a.G, a.S - s0);
        }
        const uint32_t known = gr->known;
        for (int row = warp; row < nst * E; row += nwarps) {
            const int g = row / E, j = row - g * E;
            const uint64_t *par = BATCHED ? a.srcp[first + g] : a.proj + (s0 + g) * a.total;
            uint64_t *dat = BATCHED ? a.dstp[first + g] : a.img + (s0 + g) * (int64_t)a.Qd * P;
            const int lp = gr->lpos[j], sp = gr->split[j];
            const int pa = gr->p[2 * j], pb = gr->p[2 * j + 1];
            const int sa = gr->src[2 * j], sb = gr->src[2 * j + 1];
            for (int x = lane; x < P; x += 32) {
                const bool left = x < sp;
                const int pp = left ? pa : pb;
                uint64_t v = __ldcs(par + ((left ? sa : sb) - x));
                for (uint32_t k = known; k; k &= k - 1) {
                    const int l2 = __ffs(k) - 1;
                    const int x2 = x + (l2 - lp) * pp;
                    if ((unsigned)x2 < (unsigned)P) v ^= dat[(int64_t)l2 * P + x2];
                }
                dat[(int64_t)lp * P + x] = v;
            }
        }
    }
}

// Launch sys_residual over the same work items as the decode that follows
// (L.G stripes each, plain form).
template <bool BATCHED>
int launch_sys_residual(DecParams &a, const DecodeLayout &L, int64_t nitems, cudaStream_t st)
{
    a.G = L.G;
    if (nitems <= 0) return 0;
    int dev = 0, sms = 0, err = 0;
    if ((err = record_cuda(cudaGetDevice(&dev)))) return err;
    if ((err = record_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))) return err;
    const int64_t grid = std::min<int64_t>(nitems, (int64_t)sms * 8);
    sys_residual<BATCHED><<<(unsigned)grid, 256, 0, st>>>(a);
    return record_cuda(cudaGetLastError());
}

using DecKernel = void (*)(const DecParams);

template <bool BATCHED>
DecKernel pick_fronts(int Q)
{
    switch (Q) {
    case 1: return decode_fronts<1, BATCHED>;
    case 2: return decode_fronts<2, BATCHED>;
    case 3: return decode_fronts<3, BATCHED>;
    case 4: return decode_fronts<4, BATCHED>;
    case 5: return decode_fronts<5, BATCHED>;
    case 6: return decode_fronts<6, BATCHED>;
    case 7: return decode_fronts<7, BATCHED>;
    case 8: return decode_fronts<8, BATCHED>;
    default: return decode_fronts<0, BATCHED>;
    }
}

template <bool BATCHED>
DecKernel pick_lines(int Q)
{
    switch (Q) {
    case 1: return decode_lines<1, BATCHED>;
    case 2: return decode_lines<2, BATCHED>;
    case 3: return decode_lines<3, BATCHED>;
    case 4: return decode_lines<4, BATCHED>;
    case 5: return decode_lines<5, BATCHED>;
    case 6: return decode_lines<6, BATCHED>;
    case 7: return decode_lines<7, BATCHED>;
    case 8: return decode_lines<8, BATCHED>;
    default: return nullptr;
    }
}

template <bool BATCHED>
DecKernel pick_ilv(int Q, bool pad)
{
    switch (Q) {
    case 1: return pad ? decode_ilv<1, BATCHED, true> : decode_ilv<1, BATCHED, false>;
    case 2: return pad ? decode_ilv<2, BATCHED, true> : decode_ilv<2, BATCHED, false>;
    case 3: return pad ? decode_ilv<3, BATCHED, true> : decode_ilv<3, BATCHED, false>;
    case 4: return pad ? decode_ilv<4, BATCHED, true> : decode_ilv<4, BATCHED, false>;
    case 5: return pad ? decode_ilv<5, BATCHED, true> : decode_ilv<5, BATCHED, false>;
    case 6: return pad ? decode_ilv<6, BATCHED, true> : decode_ilv<6, BATCHED, false>;
    case 7: return pad ? decode_ilv<7, BATCHED, true> : decode_ilv<7, BATCHED, false>;
    case 8: return pad ? decode_ilv<8, BATCHED, true> : decode_ilv<8, BATCHED, false>;
    default: return nullptr;
    }
}

template <bool BATCHED>
DecKernel pick_ring(int Q)
{
    if constexpr (BATCHED) {
        return nullptr;   // plain launches only
    } else {
        switch (Q) {
        case 1: return decode_ring<1, false>;
        case 2: return decode_ring<2, false>;
        case 3: return decode_ring<3, false>;
        case 4: return decode_ring<4, false>;
        case 5: return decode_ring<5, false>;
        case 6: return decode_ring<6, false>;
        case 7: return decode_ring<7, false>;
        case 8: return decode_ring<8, false>;
        default: return nullptr;
        }
    }
}

template <bool BATCHED>
DecKernel pick_lines_sys(int Q)
{
    switch (Q) {
    case 1: return decode_lines<1, BATCHED, true>;
    case 2: return decode_lines<2, BATCHED, true>;
    case 3: return decode_lines<3, BATCHED, true>;
    case 4: return decode_lines<4, BATCHED, true>;
    case 5: return decode_lines<5, BATCHED, true>;
    case 6: return decode_lines<6, BATCHED, true>;
    case 7: return decode_lines<7, BATCHED, true>;
    case 8: return decode_lines<8, BATCHED, true>;
    default: return nullptr;
    }
}

template <bool BATCHED>
DecKernel pick_vander(int Q)
{
    switch (Q) {
    case 2: return decode_vander<2, BATCHED>;
    case 3: return decode_vander<3, BATCHED>;
    case 4: return decode_vander<4, BATCHED>;
    case 5: return decode_vander<5, BATCHED>;
    case 6: return decode_vander<6, BATCHED>;
    case 7: return decode_vander<7, BATCHED>;
    case 8: return decode_vander<8, BATCHED>;
    default: return nullptr;
    }
}

template <bool BATCHED>
DecKernel pick_scan2(bool sys)
{
    return sys ? decode_scan2<BATCHED, true> : decode_scan2<BATCHED, false>;
}

template <bool BATCHED>
DecKernel pick_cols(int Q)
{
    switch (Q) {
    case 1: return decode_cols<1, BATCHED>;
    case 2: return decode_cols<2, BATCHED>;
    case 3: return decode_cols<3, BATCHED>;
    case 4: return decode_cols<4, BATCHED>;
    case 5: return decode_cols<5, BATCHED>;
    case 6: return decode_cols<6, BATCHED>;
    case 7: return decode_cols<7, BATCHED>;
    case 8: return decode_cols<8, BATCHED>;
    default: return nullptr;
    }
}

template <bool BATCHED>
DecKernel pick_stream(int Q)
{
    switch (Q) {
    case 1: return decode_stream<1, BATCHED>;
    case 2: return decode_stream<2, BATCHED>;
    case 3: return decode_stream<3, BATCHED>;
    case 4: return decode_stream<4, BATCHED>;
    case 5: return decode_stream<5, BATCHED>;
    case 6: return decode_stream<6, BATCHED>;
    case 7: return decode_stream<7, BATCHED>;
    case 8: return decode_stream<8, BATCHED>;
    default: return nullptr;
    }
}

// Launch a decode kernel over `nitems` work items with a layout from
// decode_layout; a's path and addressing fields are already set.
// sys: the systematic form (decode_lines only).
template <bool BATCHED>
int launch_decode_kernel(DecParams &a, const DecodeLayout &L, const DecodeConfig &cfg,
                         int64_t nitems, cudaStream_t st, bool sys = false)
{
    a.reach = L.reach;
    a.RP = L.RP;
    a.SWc = L.SWc;
    a.SWr = L.SWr;
    for (int l = 0; l < kMaxLines; ++l) a.rowbase[l] = L.rowbase[l];
    a.G = L.G;
    a.GS = L.GS;
    a.TS = L.TS;
    a.gpc = std::max(1, cfg.gpc);
    a.persist = cfg.persist ? 1 : 0;
    if (const char *e = getenv("MOJETTE_DECODE_STEADY")) a.steady = atoi(e) ? 1 : 0;
    else a.steady = 1;
    if (nitems <= 0) return 0;
    if (sys && L.kernel != 0 && L.kernel != 4) return -EINVAL;
    if (L.kernel == 4 && a.Q != 2) return -EINVAL;
    DecKernel fn = L.kernel == 5 ? pick_vander<BATCHED>(a.Q)
                 : L.kernel == 4 ? pick_scan2<BATCHED>(sys)
                 : sys ? pick_lines_sys<BATCHED>(a.Q)
                 : L.kernel == 0 ? pick_lines<BATCHED>(a.Q)
                 : L.kernel == 2 ? pick_stream<BATCHED>(a.Q)
                 : L.kernel == 3 ? pick_cols<BATCHED>(a.Q)
                 : L.kernel == 6 ? pick_ilv<BATCHED>(a.Q, L.reach > 1)
                 : L.kernel == 7 ? pick_ring<BATCHED>(a.Q)
                                 : pick_fronts<BATCHED>(a.Q);
    if (!fn) return -EINVAL;
    // decode_scan2 / decode_vander: one warp per stripe; decode_ilv: one warp
    // per side; the others: one warp
    const int block = (L.kernel == 4 || L.kernel == 5) ? 32 * L.G : L.kernel == 6 ? 64 : 32;
    int err = 0;
    if ((err = record_cuda(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)L.smem))))
        return err;
    // CTAs the device holds at once for this kernel and shared memory
    // (cached: the query costs host time on every launch otherwise)
    int slots = 0;
    {
        static std::mutex mu;
        static std::map<std::pair<const void *, int64_t>, int> cache;
        int dev = 0, sms = 0, per_sm = 0;
        if ((err = record_cuda(cudaGetDevice(&dev)))) return err;
        const auto key = std::make_pair((const void *)fn, L.smem * 64 + dev);
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            slots = it->second;
        } else {
            if ((err = record_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))) return err;
            if ((err = record_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block,
                                                                                 (size_t)L.smem))))
                return err;
            slots = std::max(per_sm, 1) * sms;
            cache[key] = slots;
        }
    }
    // a launch with fewer items than the device holds runs them all at once
    // (fewer items per CTA) instead of leaving SMs idle
    if (!a.persist && nitems < (int64_t)slots * a.gpc)
        a.gpc = (int)std::max<int64_t>(1, (nitems + slots - 1) / slots);
    int64_t grid = (nitems + a.gpc - 1) / a.gpc;
    if (a.persist) grid = std::min<int64_t>(grid, (int64_t)slots);
    fn<<<(unsigned)grid, block, (size_t)L.smem, st>>>(a);
    return record_cuda(cudaGetLastError());
}

}  // namespace
}  // namespace mojette
