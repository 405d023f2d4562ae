// Inverse Mojette transform (decode), Sec. 2.2, along a pre-determined
// reconstruction path (one projection dedicated to each line, swept from
// both ends of the line; the path itself is built on the host, plan.cpp).
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
// so the kernel is built to keep that chain short and many stripes in
// flight:
//   - one lane runs one front (left or right) of one stripe, all Q lines,
//     visiting the lines from Q-1 down to 0 each step; the pixel line l+1
//     rebuilt in the same step is forwarded in a register, so the only
//     shared-memory round trip on the critical path is one per step;
//   - lanes 0..15 are left fronts and 16..31 right fronts of the same G
//     stripes, whose 64-bit words are interleaved in shared memory, so each
//     half-warp reads one contiguous run: no bank conflicts;
//   - the Q*P bins the path uses are staged in pixel order by 8-byte
//     cp.async copies (coalesced; the descending bin order costs nothing)
//     and each rebuilt pixel overwrites its own bin, so a stripe needs Q*P
//     words of shared memory plus zero columns around the rows;
//   - the zero columns stand for pixels outside the image (the XOR
//     identity), so no bounds test sits in the inner loop.
#include <algorithm>
#include <cerrno>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include "ptx.cuh"

namespace mojette {
namespace {

struct DecParams {
    const uint64_t *proj;
    uint64_t *img;
    int64_t S;
    int64_t total;
    int P, Q;
    int reach;    // zero columns before, between and after the rows of a stripe
    int RP;       // row pitch in columns: P + reach
    int SWc;      // columns per stripe
    int G;        // stripes per warp (<= 15)
    int GS;       // interleave stride: G rounded up to an odd number
    int gpc;      // groups of G stripes per CTA (one warp per CTA)
    int steady;   // 1: run steady steps on the short path
    int T;        // steps
    int T4;       // steps, rounded up to a multiple of 4 (extra steps are empty)
    uint32_t fwd; // operand pattern of the steady steps (bit 2l + side)
    const uint32_t *steps;
    int32_t p[2 * kMaxLines];     // direction of front (l, side), index 2l + side
    int32_t src[2 * kMaxLines];   // bin of pixel x of that front: word src - x
    int32_t split[kMaxLines];     // x < split[l]: left front
    uint32_t *status;
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

// QT: number of lines at compile time (0: any Q up to kMaxLines, slower).
template <int QT>
__global__ void __launch_bounds__(32) decode_fronts(const __grid_constant__ DecParams a)
{
    constexpr int QA = QT ? QT : kMaxLines;   // register array extent
    extern __shared__ __align__(16) uint64_t sm[];
    const int Q = QT ? QT : a.Q;
    const int P = a.P, G = a.G, GS = a.GS;
    const int lane = threadIdx.x & 31;
    // Step words first (16-byte aligned for vector reads), then the stripe
    // slots; word (column c, slot g) sits at c * GS + g.
    uint32_t *steps = reinterpret_cast<uint32_t *>(sm);
    for (int t = lane; t < a.T4 + 4; t += 32) steps[t] = t < a.T ? a.steps[t] : 0u;
    uint64_t *wbuf = sm + (a.T4 + 4) / 2;
    // Zero columns stand for pixels outside the image (the XOR identity):
    // the reach columns before each row and after the last one. Rows are
    // always staged before they are read.
    for (int ll = 0; ll <= Q; ++ll)
        for (int i = lane; i < a.reach * GS; i += 32) wbuf[ll * a.RP * GS + i] = 0;
    __syncwarp();
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
    // (l2, x + (l2 - l) p).
    uint32_t start[QA], bit[QA], keep[QA];
    uint64_t fmask[QA];
    int dl[QA][QA];
#pragma unroll
    for (int l = 0; l < QA; ++l) {
        if (l >= Q) break;
        const int p = a.p[2 * l + side];
        start[l] = wbase + ((a.reach + l * a.RP + (side ? P - 1 : 0)) * GS + g) * 8;
        bit[l] = 1u << (2 * l + side);
        const uint32_t f = (l + 1 < Q) ? (a.fwd >> (2 * l + side)) & 1u : 0u;
        keep[l] = f ^ 1u;
        fmask[l] = f ? ~0ull : 0ull;
#pragma unroll
        for (int l2 = 0; l2 < QA; ++l2) {
            if (l2 >= Q) break;
            dl[l][l2] = (l2 - l) * (a.RP + p) * GS * 8;
        }
    }

    // Copy lanes: lane = xk * G + gg covers XK columns of G stripes.
    const int XK = 32 / G;
    const int xk = lane / G, gg = lane - xk * G;
    const bool copy_ok = xk < XK;

    for (int k = 0; k < a.gpc; ++k) {
        const int64_t s0 = ((int64_t)blockIdx.x * a.gpc + k) * G;
        if (s0 >= a.S) break;
        const int size = G;
        const int nst = (int)min64(size, a.S - s0);

        // stage the Q*P bins the path uses, in pixel order
        if (copy_ok && gg < nst) {
            const uint64_t *src = a.proj + (s0 + gg) * a.total;
            for (int ll = 0; ll < Q; ++ll) {
                const int sp = a.split[ll];
                const int sl = a.src[2 * ll], sr = a.src[2 * ll + 1];
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
        for (int t = 0; t < a.T4; ++t) {
            const uint32_t w = steps[t];
            if (w & steady_bit) steady();
            else general(w);
        }

        // write the rebuilt image
        if (copy_ok && gg < nst) {
            uint64_t *out = a.img + (s0 + gg) * (int64_t)Q * P;
            for (int ll = 0; ll < Q; ++ll) {
                const uint64_t *buf = wbuf + (a.reach + ll * a.RP) * GS + gg;
                for (int x = xk; x < P; x += XK) __stcs(out + ll * P + x, buf[x * GS]);
            }
        }
        __syncwarp();
    }
}

using DecKernel = void (*)(const DecParams);

DecKernel pick_kernel(int Q)
{
    switch (Q) {
    case 1: return decode_fronts<1>;
    case 2: return decode_fronts<2>;
    case 3: return decode_fronts<3>;
    case 4: return decode_fronts<4>;
    case 5: return decode_fronts<5>;
    case 6: return decode_fronts<6>;
    case 7: return decode_fronts<7>;
    case 8: return decode_fronts<8>;
    default: return decode_fronts<0>;
    }
}


// ---------------------------------------------------------------------------
// decode_lines: one lane per (stripe, line, front). A warp holds G = 32/(2Q)
// stripes; at every step each lane rebuilds the next pixel of its line's
// front (when the step word moves it), from its staged bin and the other
// pixels of the bin line read from shared memory -- except the operand on
// line l+1, which line l+1 may rebuild in this same step. Those same-step
// links (bit 2l+side of the step's forward word) form chains l -> l+1 -> ...
// within a front; the chain values are a segmented suffix XOR over the lines,
// done with log2(Q) rounds of warp shuffles, so every lane of every line
// works at every step and a step costs one shared-memory round trip.
struct LineParams {
    const uint64_t *proj;
    uint64_t *img;
    int64_t S;
    int64_t total;
    int P, Q;
    int reach, RP, SWc;   // layout as for decode_fronts
    int G;                // stripes per warp = 32 / (2Q); interleave stride G
    int gpc;              // groups of G stripes per CTA (one warp per CTA)
    int T4;               // steps, rounded up to a multiple of 4
    const uint32_t *steps;   // T step words, then T forward words
    int T;
    uint32_t fwd;            // forward pattern of the steady steps
    int32_t p[2 * kMaxLines];
    int32_t src[2 * kMaxLines];
    int32_t split[kMaxLines];
};

template <int QT>
__global__ void __launch_bounds__(32) decode_lines(const __grid_constant__ LineParams a)
{
    extern __shared__ __align__(16) uint64_t sm[];
    constexpr int Q = QT;
    const int P = a.P, G = a.G;
    const int lane = threadIdx.x & 31;
    // step words, forward words (each padded to T4 + 4), then the slots
    uint32_t *stepw = reinterpret_cast<uint32_t *>(sm);
    uint32_t *fwdw = stepw + a.T4 + 4;
    for (int t = lane; t < a.T4 + 4; t += 32) {
        stepw[t] = t < a.T ? a.steps[t] : 0u;
        fwdw[t] = t < a.T ? a.steps[a.T + t] : 0u;
    }
    uint64_t *wbuf = sm + (a.T4 + 4);
    for (int ll = 0; ll <= Q; ++ll)
        for (int i = lane; i < a.reach * G; i += 32) wbuf[ll * a.RP * G + i] = 0;
    __syncwarp();
    const uint32_t wbase = smem_addr(wbuf);

    // Rebuild lanes: lane = (2l + side) * G + g; lanes past 2Q*G shadow lane 0.
    const int lsr = lane / G;
    const bool ok = lsr < 2 * Q;
    const int ls = ok ? lsr : 0;
    const int g = ok ? lane - lsr * G : 0;
    const int l = ls >> 1, side = ls & 1;
    const int p = a.p[ls];
    const uint32_t bitmask = ok ? 1u << ls : 0u;   // shadow lanes never store
    const int colstep = (a.RP + p) * G * 8;    // bytes from line l to line l+1 on a bin line
    const uint32_t start = wbase + ((a.reach + l * a.RP + (side ? P - 1 : 0)) * G + g) * 8;
    const int stepb = (side ? -1 : 1) * G * 8;
    // The operands of line l sit on lines l2 = l+1+k (mod Q), k = 0 .. Q-2.
    // k = 0 is line l+1, which may be forwarded, except for l = Q-1 where it
    // wraps to line 0 and is always read.
    const uint32_t has_next = (l + 1 < Q) ? 1u : 0u;
    const int d0 = (has_next ? 1 : 1 - Q) * colstep;
    int dk[Q > 2 ? Q - 2 : 1];
#pragma unroll
    for (int k = 1; k < Q - 1; ++k) {
        const int l2 = (l + 1 + k) % Q;
        dk[k - 1] = (l2 - l) * colstep;
    }

    // Steady steps: this lane's link (line l forwards from line l+1) and the
    // link state after each scan round, from the schedule's steady pattern:
    // after the round with stride d, line l is still linked iff it was, and
    // line l+d was too.
    const uint32_t sfw = ok ? (a.fwd >> ls) & 1u : 0u;
    uint32_t slink[4] = {0u, 0u, 0u, 0u};
    {
        uint32_t c[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) c[j] = (j + 1 < Q) ? (a.fwd >> (2 * j + side)) & 1u : 0u;
#pragma unroll
        for (int r = 0, d = 1; d < Q; ++r, d <<= 1) {
            slink[r] = ok ? c[l] : 0u;
            uint32_t nc[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) nc[j] = (c[j] && j + d < Q) ? c[j + d] : (c[j] ? 0u : 0u);
#pragma unroll
            for (int j = 0; j < Q; ++j) c[j] = nc[j];
        }
    }

    // Copy lanes: lane = xk * G + gg covers XK columns of G stripes.
    const int XK = 32 / G;
    const int xk = lane / G, gg = lane - xk * G;
    const bool copy_ok = xk < XK;

    for (int k = 0; k < a.gpc; ++k) {
        const int64_t s0 = ((int64_t)blockIdx.x * a.gpc + k) * G;
        if (s0 >= a.S) break;
        const int nst = (int)min64(G, a.S - s0);

        if (copy_ok && gg < nst) {
            const uint64_t *src = a.proj + (s0 + gg) * a.total;
            for (int ll = 0; ll < Q; ++ll) {
                const int sp = a.split[ll];
                const int sl = a.src[2 * ll], sr = a.src[2 * ll + 1];
                uint64_t *dst = wbuf + (a.reach + ll * a.RP) * G + gg;
                for (int x = xk; x < P; x += XK)
                    cp_async8(dst + x * G, src + ((x < sp ? sl : sr) - x));
            }
        }
        cp_async_wait_all();
        __syncwarp();

        uint32_t pos = start;
        for (int t = 0; t < a.T4; ++t) {
            const uint32_t w = stepw[t];
            if (w & kStepSteady) {
                // steady: every line moves, links are the schedule's pattern
                uint64_t v = ld_s64(pos);
#pragma unroll
                for (int k2 = 0; k2 < Q - 2; ++k2) v ^= ld_s64(pos + dk[k2]);
                if (Q > 1) v ^= ld_s64_if(pos + d0, (sfw & has_next) ^ 1u);
#pragma unroll
                for (int r = 0, d = 1; d < Q; ++r, d <<= 1) {
                    const uint64_t tv = __shfl_down_sync(0xffffffffu, v, 2 * d * G);
                    if (slink[r]) v ^= tv;
                }
                st_s64_if(pos, v, ok);
                pos += stepb;
                __syncwarp();
                continue;
            }
            const uint32_t f = fwdw[t];
            const uint32_t act = w & bitmask;
            const uint32_t fw = ok ? (f >> ls) & 1u : 0u;
            uint64_t v = ld_s64(pos);
#pragma unroll
            for (int k2 = 0; k2 < Q - 2; ++k2) v ^= ld_s64(pos + dk[k2]);
            if (Q > 1) v ^= ld_s64_if(pos + d0, (fw & has_next) ^ 1u);
            // segmented suffix XOR: v_l ^= v_{l+1} while linked
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
            st_s64_if(pos, v, act);
            pos += act ? stepb : 0;
            __syncwarp();
        }

        if (copy_ok && gg < nst) {
            uint64_t *out = a.img + (s0 + gg) * (int64_t)Q * P;
            for (int ll = 0; ll < Q; ++ll) {
                const uint64_t *buf = wbuf + (a.reach + ll * a.RP) * G + gg;
                for (int x = xk; x < P; x += XK) __stcs(out + ll * P + x, buf[x * G]);
            }
        }
        __syncwarp();
    }
}

using LineKernel = void (*)(const LineParams);

LineKernel pick_lines(int Q)
{
    switch (Q) {
    case 1: return decode_lines<1>;
    case 2: return decode_lines<2>;
    case 3: return decode_lines<3>;
    case 4: return decode_lines<4>;
    case 5: return decode_lines<5>;
    case 6: return decode_lines<6>;
    case 7: return decode_lines<7>;
    case 8: return decode_lines<8>;
    default: return nullptr;
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
    a.T4 = (d.T + 3) / 4 * 4;
    a.steps = d.steps;
    int maxp = 0;
    for (int l = 0; l < d.Q; ++l) {
        a.p[2 * l] = d.pL[l];
        a.p[2 * l + 1] = d.pR[l];
        a.src[2 * l] = (int32_t)d.srcL[l];
        a.src[2 * l + 1] = (int32_t)d.srcR[l];
        a.split[l] = d.split[l];
        maxp = std::max(maxp, std::max(std::abs(d.pL[l]), std::abs(d.pR[l])));
    }
    a.status = d.status;

    int err = 0, dev = 0, cap = 0, cap_sm = 0;
    if ((err = record_cuda(cudaGetDevice(&dev)))) return err;
    if ((err = record_cuda(cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))))
        return err;
    if ((err = record_cuda(cudaDeviceGetAttribute(&cap_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev))))
        return err;

    // Zero columns between rows: one more than the widest offset (l2 - l) p
    // of a bin line, so that a front one step past its last pixel still
    // reads inside the stripe.
    a.reach = (d.Q - 1) * maxp + 1;
    a.RP = d.P + a.reach;
    a.SWc = d.Q * a.RP + a.reach;
    a.fwd = d.fwd;

    // decode_lines for Q <= 8 unless MOJETTE_DECODE_KERNEL=fronts
    const char *kenv = getenv("MOJETTE_DECODE_KERNEL");
    const bool want_lines = !(kenv && strcmp(kenv, "fronts") == 0);
    if (want_lines && d.Q <= 8) {
        LineParams b;
        b.proj = d.proj;
        b.img = d.img;
        b.S = d.S;
        b.total = d.total;
        b.P = d.P;
        b.Q = d.Q;
        b.reach = a.reach;
        b.RP = a.RP;
        b.SWc = a.SWc;
        b.G = std::max(1, 32 / (2 * d.Q));
        b.T = d.T;
        b.fwd = d.fwd;
        b.T4 = a.T4;
        b.steps = d.steps;
        for (int i = 0; i < 2 * d.Q; ++i) {
            b.p[i] = a.p[i];
            b.src[i] = a.src[i];
        }
        for (int l = 0; l < d.Q; ++l) b.split[l] = a.split[l];
        b.gpc = 4;
        if (const char *e = getenv("MOJETTE_DECODE_GPC")) b.gpc = std::max(1, atoi(e));
        const int64_t smem = (int64_t)(b.T4 + 4) * 8 + (int64_t)b.G * b.SWc * 8;
        if (smem > cap) return -EINVAL;   // one warp's stripes exceed shared memory
        LineKernel fl = pick_lines(d.Q);
        if ((err = record_cuda(cudaFuncSetAttribute(fl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem))))
            return err;
        const int64_t ngroups = (d.S + b.G - 1) / b.G;
        const int64_t grid = (ngroups + b.gpc - 1) / b.gpc;
        fl<<<(unsigned)grid, 32, (size_t)smem, st>>>(b);
        return record_cuda(cudaGetLastError());
    }
    const int64_t steps_bytes = (int64_t)(a.T4 + 4) * 4;
    const int64_t slot_bytes = (int64_t)a.SWc * 8;
    auto stride = [](int G) { return G | 1; };   // odd: conflict-free copies
    // One warp per CTA, several CTAs per SM: CTAs start and finish at
    // different times, so one CTA's staging and output overlap another's
    // reconstruction. G stripes per CTA: the most stripes resident per SM.
    int G = 0;
    int64_t best = 0;
    for (int g = 15; g >= 1; --g) {
        const int64_t per_cta = stride(g) * slot_bytes + steps_bytes + 1024;   // + reserved
        const int64_t ctas = std::min<int64_t>(cap_sm / per_cta, 32);
        if (per_cta - 1024 > cap) continue;
        if (ctas * g > best) { best = ctas * g; G = g; }
    }
    if (!G) return -EINVAL;   // one stripe exceeds shared memory
    if (const char *e = getenv("MOJETTE_DECODE_G")) {      // tuning override
        const int g = atoi(e);
        if (g >= 1 && g <= 15 && stride(g) * slot_bytes + steps_bytes <= cap) G = g;
    }
    a.G = G;
    a.GS = stride(G);
    const int64_t ngroups = (d.S + a.G - 1) / a.G;
    a.gpc = 4;
    if (const char *e = getenv("MOJETTE_DECODE_GPC")) a.gpc = std::max(1, atoi(e));
    a.steady = 1;
    if (const char *e = getenv("MOJETTE_DECODE_STEADY")) a.steady = atoi(e) ? 1 : 0;
    const int smem = (int)(a.GS * slot_bytes + steps_bytes);
    DecKernel fn = pick_kernel(d.Q);
    if ((err = record_cuda(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))))
        return err;
    const int64_t grid = (ngroups + a.gpc - 1) / a.gpc;
    fn<<<(unsigned)grid, 32, smem, st>>>(a);
    return record_cuda(cudaGetLastError());
}


// ---------------------------------------------------------------------------
// Scratch for mojette_decode_noalloc: the step words and forward words of one
// schedule, in a fixed array that every GPU loading the library holds until
// the process exits (2 * kNoAllocMaxSteps * 4 bytes = 128 KiB). In host code
// the name of the array is only a stand-in; the device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) uint32_t g_noalloc_steps[2 * kNoAllocMaxSteps];

namespace {
std::mutex g_noalloc_mu;
std::map<int, uint32_t *> g_noalloc_ptr;
}  // namespace

int noalloc_schedule_copy(const Schedule &sc, cudaStream_t st, uint32_t **dev)
{
    if (sc.T > kNoAllocMaxSteps) return -ENOSPC;
    int device = 0, err = 0;
    if ((err = record_cuda(cudaGetDevice(&device)))) return err;
    uint32_t *ptr = nullptr;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        auto it = g_noalloc_ptr.find(device);
        if (it != g_noalloc_ptr.end()) {
            ptr = it->second;
        } else {
            if ((err = record_cuda(cudaGetSymbolAddress((void **)&ptr, g_noalloc_steps)))) return err;
            g_noalloc_ptr[device] = ptr;
        }
    }
    // Step words then forward words, packed at stride T as the kernels read
    // them. Pageable host memory: the runtime has taken its own copy of both
    // vectors when cudaMemcpyAsync returns.
    const size_t bytes = sc.steps.size() * sizeof(uint32_t);
    if (bytes) {
        if ((err = record_cuda(cudaMemcpyAsync(ptr, sc.steps.data(), bytes, cudaMemcpyHostToDevice, st))))
            return err;
        if ((err = record_cuda(cudaMemcpyAsync(ptr + sc.steps.size(), sc.fwdw.data(), bytes,
                                               cudaMemcpyHostToDevice, st))))
            return err;
    }
    *dev = ptr;
    return 0;
}
}  // namespace mojette
