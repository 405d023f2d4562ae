// Plain decode launcher (one reconstruction path, stripes back to back), the
// shared-memory layout rule of every decode launch, and the fixed scratch of
// mojette_decode_noalloc. The kernels are in decode_kernels.cuh.
#include <map>
#include <mutex>

#include "decode_kernels.cuh"

namespace mojette {

int choose_decode_kernel(int P, int Q, int64_t S, bool sys, bool scan2, bool vander, bool env)
{
    // The Sec. 2.2 path: decode_lines (one warp per few stripes, one lane
    // per line and front) up to 8 lines, decode_fronts beyond; a systematic
    // decode runs the path over its lost lines. decode_ilv (stripes across
    // lanes) runs the same path; it (measured slower) and the closed forms
    // (decode_scan2, decode_vander: exact, but not the paper's inverse) are
    // opt-in alternatives (MOJETTE_DECODE_KERNEL, or a configuration
    // installed with mojette_plan_config).
    (void)P;
    (void)S;
    int k = 0;
    if (Q > 8) k = 1;
    if (env) {
        if (const char *e = getenv("MOJETTE_DECODE_KERNEL")) {
            if (strcmp(e, "ilv") == 0 && Q <= 8 && !sys) k = 6;
            else if (strcmp(e, "ring") == 0 && Q <= 8 && !sys) k = 7;
            else if (strcmp(e, "lines") == 0 && Q <= 8) k = 0;
            else if (strcmp(e, "fronts") == 0 && !sys) k = 1;
            else if (strcmp(e, "stream") == 0 && !sys && Q <= 8) k = 2;
            else if (strcmp(e, "cols") == 0 && !sys && Q <= 8) k = 3;
            else if (strcmp(e, "scan") == 0 && scan2) k = 4;
            else if (strcmp(e, "vander") == 0 && vander) k = 5;
        }
    }
    return k;
}

int decode_bank_slots(int Q)
{
    const int G = std::max(1, 32 / (2 * Q));
    return (16 % G == 0 && G < 16) ? 16 / G : 1;
}

int decode_layout(int P, int Q, int span, int maxp, int maxT, const DecodeConfig &cfg,
                  const int32_t *rowoff, DecodeLayout *L)
{
    int err = 0, dev = 0, cap = 0, cap_sm = 0;
    if ((err = record_cuda(cudaGetDevice(&dev)))) return err;
    if ((err = record_cuda(cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))))
        return err;
    if ((err = record_cuda(cudaDeviceGetAttribute(&cap_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev))))
        return err;
    // Zero columns between rows: one more than the widest offset (l2 - l) p
    // of a bin line (rows `span` apart at most), so that a front one step
    // past its last pixel still reads inside the stripe.
    L->reach = span * maxp + 1;
    L->RP = P + L->reach;
    L->TS = (maxT + 3) / 4 * 4 + 4;
    for (int l = 0; l < kMaxLines; ++l) L->rowbase[l] = L->reach + l * L->RP;
    const int want = (cfg.kernel == 1 || Q > 8) ? 1 : cfg.kernel;
    L->kernel = want;
    if (want == 5) {
        // decode_vander: one warp per stripe, kVanWarps per CTA; Q + 1 frame
        // arrays of RP = P + 2 (Q - 1) maxp + 2 words (a bound on every
        // path's frame; maxp over the directions it uses) with `reach` =
        // maxp zero words on both sides (the largest shift)
        if (Q < 2 || Q > 8) return -EINVAL;
        L->G = kVanWarps;
        L->GS = L->G;
        L->reach = std::max(1, maxp);
        L->RP = P + 2 * (Q - 1) * maxp + 2;
        L->TS = 0;
        L->SWc = (Q + 1) * (L->RP + 2 * L->reach);
        L->smem = (int64_t)L->G * L->SWc * 8;
        return L->smem > cap ? -EINVAL : 0;
    }
    if (want == 4) {
        // decode_scan2: two lines, one warp per stripe, kScanWarps per CTA
        if (Q != 2) return -EINVAL;
        L->G = kScanWarps;
        L->GS = L->G;
        L->reach = 0;
        L->RP = P;
        L->TS = 0;
        L->SWc = scan2_words(P);
        L->smem = (int64_t)L->G * L->SWc * 8;
        return L->smem > cap ? -EINVAL : 0;
    }
    if (want == 2) {
        // decode_stream: rows packed at pitch P (operands outside the image
        // read one zero column after the rows), step and forward words first
        L->G = std::max(1, 32 / (2 * Q));
        L->GS = L->G;
        L->reach = 0;
        L->RP = P;
        for (int l = 0; l < kMaxLines; ++l) L->rowbase[l] = l * L->RP;
        L->SWc = Q * L->RP + 1;
        L->smem = (int64_t)L->TS * 8 + (int64_t)L->G * L->SWc * 8;
        return L->smem > cap ? -EINVAL : 0;
    }
    if (want == 3) {
        // decode_cols: columns of Q lines x G stripes, reach zero columns at
        // both ends of the rows; step and forward words first
        L->G = std::max(1, 32 / (2 * Q));
        L->GS = L->G;
        L->RP = 0;
        L->SWc = (P + 2 * L->reach) * Q;
        L->smem = (int64_t)L->TS * 8 + (int64_t)L->G * L->SWc * 8;
        return L->smem > cap ? -EINVAL : 0;
    }
    if (want == 7) {
        // decode_ring: one warp, G = 32 / Q stripes; the mbarriers (Q lines
        // x R / 16 chunk slots), then each stripe's region of SWr words with
        // line l's ring of R words at l * R; SWr = 2 mod 16 so that the G
        // stripes' same slot falls in distinct bank pairs (G <= 8), regions
        // and rings 16-byte aligned for the bulk copies. RP = R, reach = D
        // (set by the caller, from the path; 0: no ring fits).
        L->RP = cfg.ring_R;
        L->reach = cfg.ring_D;
        if (Q > 8 || L->RP < 2 * kRingChunk || L->RP % kRingChunk || P % kRingChunk) return -EINVAL;
        L->G = std::max(1, 32 / Q);
        L->GS = L->G;
        const int NS = L->RP / kRingChunk;
        L->SWc = (Q * NS + 1) & ~1;
        for (int l = 0; l < kMaxLines; ++l) L->rowbase[l] = l * L->RP;
        L->SWr = Q * L->RP;
        while (L->SWr % 16 != 2) L->SWr += 2;
        L->TS = 0;
        L->smem = ((int64_t)L->SWc + (int64_t)L->G * L->SWr) * 8;
        return L->smem > cap ? -EINVAL : 0;
    }
    if (want == 6) {
        // decode_ilv: G stripes interleaved word by word at stride GS, the
        // (step, forward) word pairs first. Rows either with zero gaps of R
        // = (Q - 1) max|p| columns between them and at both ends, plus one
        // word at each end for a front one step past its line (PAD, signalled
        // by reach = R + 1 >= 2), or of P + 1 columns with column P the zero
        // word operands outside the image are clamped to (reach = 1). G: the
        // most stripes (up to 16, one per lane of a half-warp) for which two
        // CTAs fit on an SM, else one; a cap (cfg.gmax, or MOJETTE_DECODE_G)
        // spreads small launches over more CTAs. PAD unless the gaps cost
        // more than a quarter of the stripes a CTA holds
        // (MOJETTE_DECODE_PAD=0/1 forces it).
        if (Q > 8) return -EINVAL;
        const int R = std::max(0, span) * maxp;
        auto cols = [&](bool pad) -> int64_t {
            return pad ? 2 + R + (int64_t)Q * (P + R) : (int64_t)Q * (P + 1);
        };
        auto bytes = [&](bool pad, int g) { return (int64_t)L->TS * 8 + cols(pad) * (g | 1) * 8; };
        int gmax = 16;
        if (cfg.gmax > 0) gmax = std::min(gmax, cfg.gmax);
        if (const char *e = getenv("MOJETTE_DECODE_G")) {
            const int v = atoi(e);
            if (v >= 1 && v <= 16) gmax = v;
        }
        auto pick = [&](bool pad) {
            for (int want_ctas = 2; want_ctas >= 1; --want_ctas)
                for (int g = gmax; g >= 1; --g)
                    if (bytes(pad, g) <= cap && (bytes(pad, g) + 1024) * want_ctas <= cap_sm) return g;
            return 0;
        };
        const int Gc = pick(false), Gp = R > 0 ? pick(true) : 0;
        bool pad = Gp > 0 && 4 * Gp >= 3 * Gc;
        if (const char *e = getenv("MOJETTE_DECODE_PAD")) pad = atoi(e) != 0 && Gp > 0;
        const int G = pad ? Gp : Gc;
        if (!G) return -EINVAL;   // one stripe exceeds shared memory
        L->G = G;
        L->GS = G | 1;
        if (pad) {
            L->reach = R + 1;
            L->RP = P + R;
            for (int l = 0; l < kMaxLines; ++l) L->rowbase[l] = 1 + R + l * L->RP;
        } else {
            L->reach = 1;
            L->RP = P + 1;
            for (int l = 0; l < kMaxLines; ++l) L->rowbase[l] = l * L->RP;
        }
        L->SWc = (int)(cols(pad) * L->GS);
        L->smem = bytes(pad, G);
        return 0;
    }
    if (want == 0) {
        // decode_lines: 2Q lanes per stripe; step and forward words and the
        // staging mbarrier (16 bytes) first, then each stripe in a region
        // of SWr words, SWr = S mod 16 (stripe g's words g S bank slots
        // further on; even: 16-byte aligned regions). One zero word between
        // rows (before row 0, after the last): an operand column outside
        // the image is clamped to the word beside its row. With row phases,
        // line l's row starts at a column congruent to rowoff[l] mod M, M =
        // S (the bank slots of a group of G words), or 2 where no bank model
        // applies (only the parity that lets bulk copies stage the row): the
        // pitch gains M - 1 columns.
        L->G = std::max(1, 32 / (2 * Q));
        L->GS = L->G;
        const int S = decode_bank_slots(Q);
        const int M = S > 1 ? S : 2;
        L->reach = 1;
        L->RP = P + 1;
        for (int l = 0; l < kMaxLines; ++l) L->rowbase[l] = 1 + l * L->RP;
        if (cfg.rowoff && rowoff) {
            L->RP = P + 1 + (M - 1);
            for (int l = 0; l < Q; ++l) {
                const int base = 1 + l * L->RP;
                L->rowbase[l] = base + (((rowoff[l] - base) % M) + M) % M;
            }
        }
        L->SWc = Q * L->RP + 1;
        L->SWr = L->SWc;
        const int want_mod = (S > 1) ? S : 2;
        while (L->SWr % 16 != want_mod % 16 || L->SWr % 2) ++L->SWr;
        L->smem = (int64_t)L->TS * 8 + 16 + (int64_t)L->G * L->SWr * 8;
        return L->smem > cap ? -EINVAL : 0;   // one warp's stripes exceed shared memory
    }
    L->SWc = Q * L->RP + L->reach;
    const int64_t slot_bytes = (int64_t)L->SWc * 8;
    // decode_fronts: one warp per CTA, several CTAs per SM: CTAs start and
    // finish at different times, so one CTA's staging and output overlap
    // another's reconstruction. G stripes per CTA: the most stripes resident
    // per SM. The interleave stride is odd: conflict-free copies.
    const int64_t steps_bytes = (int64_t)L->TS * 4;
    auto stride = [](int g) { return g | 1; };
    int G = 0;
    int64_t best = 0;
    for (int g = 15; g >= 1; --g) {
        const int64_t per_cta = stride(g) * slot_bytes + steps_bytes + 1024;   // + reserved
        const int64_t ctas = std::min<int64_t>(cap_sm / per_cta, 32);
        if (per_cta - 1024 > cap) continue;
        if (ctas * g > best) {
            best = ctas * g;
            G = g;
        }
    }
    if (!G) return -EINVAL;   // one stripe exceeds shared memory
    if (const char *e = getenv("MOJETTE_DECODE_G")) {      // tuning override
        const int g = atoi(e);
        if (g >= 1 && g <= 15 && stride(g) * slot_bytes + steps_bytes <= cap) G = g;
    }
    L->G = G;
    L->GS = stride(G);
    L->smem = L->GS * slot_bytes + steps_bytes;
    return 0;
}

int launch_decode(const DecodeArgs &d, cudaStream_t st)
{
    DecParams a;
    std::memset(&a, 0, sizeof(a));
    a.proj = d.proj;
    a.img = d.img;
    a.S = d.S;
    a.total = d.total;
    a.P = d.P;
    a.Q = d.Q;
    a.Qd = d.Qd;
    a.grp.known = d.known;
    a.status = d.status;
    for (int l = 0; l < kMaxLines; ++l) a.grp.lpos[l] = d.lpos[l];
    a.grp.steps = d.steps;
    a.grp.T = d.T;
    a.grp.fwd = d.fwd;
    int maxp = 0;
    for (int l = 0; l < d.Q; ++l) {
        a.grp.p[2 * l] = d.pL[l];
        a.grp.p[2 * l + 1] = d.pR[l];
        a.grp.src[2 * l] = (int32_t)d.srcL[l];
        a.grp.src[2 * l + 1] = (int32_t)d.srcR[l];
        a.grp.split[l] = d.split[l];
        a.grp.order[2 * l] = d.order[2 * l];
        a.grp.order[2 * l + 1] = d.order[2 * l + 1];
        maxp = std::max(maxp, std::max(std::abs(d.pL[l]), std::abs(d.pR[l])));
    }
    a.grp.chunk_w = d.chunk_w;
    for (int c = 0; c < kStreamChunks; ++c) {
        a.grp.chunk_wait[c] = d.chunk_wait[c];
        a.grp.chunk_done[c] = d.chunk_done[c];
    }
    for (int j = 0; j < 2; ++j) {
        a.grp.scan_p[j] = d.scan_p[j];
        a.grp.scan_src[j] = (int32_t)d.scan_src[j];
    }
    int vmaxp = 0;
    a.grp.van_E0 = d.van_E0;
    a.grp.van_L = d.van_L;
    for (int j = 0; j < kMaxLines; ++j) {
        a.grp.van_q[j] = d.van_q[j];
        a.grp.van_base[j] = (int32_t)d.van_base[j];
        a.grp.van_lo[j] = d.van_lo[j];
        a.grp.van_hi[j] = d.van_hi[j];
        if (j < d.Q) vmaxp = std::max(vmaxp, std::abs(d.van_q[j]));
    }

    // the measured-fastest kernel that applies, unless MOJETTE_DECODE_KERNEL
    // names another
    DecodeConfig cfg;
    cfg.kernel = choose_decode_kernel(d.P, d.Q, d.S, d.sys, d.scan2, d.vander, true);
    if (const char *e = getenv("MOJETTE_DECODE_GPC")) cfg.gpc = std::max(1, atoi(e));
    if (const char *e = getenv("MOJETTE_DECODE_ROWOFF")) cfg.rowoff = atoi(e) ? 1 : 0;
    if (const char *e = getenv("MOJETTE_DECODE_PERSIST")) cfg.persist = atoi(e) ? 1 : 0;
    DecodeLayout L;
    if (d.sys) {
        // the systematic form: two lost lines in closed form (decode_scan2,
        // which removes the known lines itself); otherwise residual bins
        // into the lost rows, then the path on them (decode_lines; no path
        // for one lost line)
        const int span = d.lpos[d.Q - 1] - d.lpos[0];
        int err = decode_layout(d.P, d.Q, span, maxp, d.T, cfg, d.rowoff, &L);
        if (err == -EINVAL && cfg.kernel == 4) {
            cfg.kernel = 0;
            err = decode_layout(d.P, d.Q, span, maxp, d.T, cfg, d.rowoff, &L);
        }
        if (err) return err;
        const int64_t nitems = (d.S + L.G - 1) / L.G;
        if (L.kernel == 4) return launch_decode_kernel<false>(a, L, cfg, nitems, st, true);
        if ((err = launch_sys_residual<false>(a, L, nitems, st))) return err;
        if (d.T == 0) return 0;
        return launch_decode_kernel<false>(a, L, cfg, nitems, st, true);
    }
    if (cfg.kernel == 6) {
        // a launch too small to fill every SM twice at the widest work
        // items gets narrower ones, spread over more CTAs
        int dev = 0, sms = 0;
        if (record_cuda(cudaGetDevice(&dev)) == 0 &&
            record_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) == 0 && sms > 0) {
            const int64_t per = (d.S + 2 * (int64_t)sms - 1) / (2 * (int64_t)sms);
            if (per < 16) cfg.gmax = (int)std::max<int64_t>(1, per);
        }
    }
    if (cfg.kernel == 7 && (d.ring_R == 0 || d.P % kRingChunk)) cfg.kernel = 0;   // no ring for this path
    cfg.ring_R = d.ring_R;
    cfg.ring_D = d.ring_D;
    for (int l = 0; l < kMaxLines; ++l) a.grp.ring_delta[l] = d.ring_delta[l];
    int err = decode_layout(d.P, d.Q, d.Q - 1, cfg.kernel == 5 ? vmaxp : maxp, d.T, cfg, d.rowoff, &L);
    if (err == -EINVAL && (cfg.kernel == 2 || cfg.kernel == 3 || cfg.kernel == 4 || cfg.kernel == 5 ||
                           cfg.kernel == 6 || cfg.kernel == 7)) {
        cfg.kernel = 0;
        err = decode_layout(d.P, d.Q, d.Q - 1, maxp, d.T, cfg, d.rowoff, &L);
    }
    if (err == -EINVAL && cfg.kernel != 1) {
        // a warp's G stripes do not fit in shared memory: decode_fronts sizes
        // G to what fits, down to one stripe
        cfg.kernel = 1;
        err = decode_layout(d.P, d.Q, d.Q - 1, maxp, d.T, cfg, d.rowoff, &L);
    }
    if (err) return err;
    return launch_decode_kernel<false>(a, L, cfg, (d.S + L.G - 1) / L.G, st);
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
