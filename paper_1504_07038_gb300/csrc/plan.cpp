// Host side of libmojette: reconstruction schedules and their cache.
//
// Sec. 2.2 of the paper: reconstruction propagates from the image corners
// inward, and when one projection is dedicated to each line the
// reconstruction path can be fixed in advance (Normand et al., DGCI 2006).
// With directions (p, 1) this works as follows. Sort the Q projections used
// by p, ascending; line l takes the l-th one, p_(l). A pixel (l, x) is
// rebuilt from the bin b = l p_(l) - x of that projection: the bin's value
// XOR the other pixels of its discrete line, (l', x + (l' - l) p_(l)) for
// l' != l, that lie inside the image. Sweeping every line from left to
// right, those other pixels are already known once the lines are staggered
// suitably, because p_(l) increases with l. The mirror image of the same
// argument (directions -p) gives a right-to-left sweep in which line l takes
// the l-th largest p. Running both sweeps at once halves the number of
// sequential steps; the point where they meet on each line is where the
// greedy step-by-step simulation below finds them. Within a step a front
// visits its lines from Q-1 down to 0, so that line l may use the pixel
// line l + 1 rebuilt in the same step: the chain between lines with
// neighbouring directions then costs no extra step.
//
// A schedule records, for every step, which line fronts advance; the device
// replays it for every stripe that lost the same projections. Building it is
// the paper's excluded pre-computation (Sec. 3.1).
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cerrno>
#include <cstring>
#include <map>
#include <numeric>

#include "mojette_internal.h"

namespace mojette {

namespace {

// Left/right two-front sweep for one choice of Q projections (indices into
// the plan, sorted by ascending direction). At every step each front visits
// its lines from l = Q-1 down to 0 and rebuilds the next pixel of a line
// when every other in-image pixel of the pixel's bin line is known: rebuilt
// at an earlier step by either front, or -- for line l + 1 only -- by the
// same front earlier in the same step (the device keeps that value in a
// register). With the lines staggered by the dedicated directions this lets
// every front move one column per step, so a sweep takes about P/2 steps.
// Fills `out` and returns the number of steps, or -1 if the sweep stalls or
// reaches `limit` steps.
//
// The lines swept need not be all the image's rows: a systematic decode
// rebuilds only the lost data lines, after removing the known lines from the
// bins, so that the sweep runs over Q = `lines` lines at image rows pos[0] <
// pos[1] < ... (all rows 0 .. Q-1 otherwise); the other pixel of a bin line
// on line l2 is then (l2, x + (pos[l2] - pos[l]) p).
int sweep(const Plan &pl, const std::vector<int> &asc, const int *pos, int lines, int limit,
          Schedule *out, bool one_sided = false, int maxchain = kMaxLines)
{
    const int P = pl.P, Q = lines;
    const int sides = one_sided ? 1 : 2;
    int32_t pF[2][kMaxLines];
    for (int l = 0; l < Q; ++l) {
        pF[0][l] = pl.p[asc[l]];
        pF[1][l] = pl.p[asc[Q - 1 - l]];
    }
    std::vector<uint8_t> known((size_t)P * Q, 0);
    // front (0 left, 1 right) and step that rebuilt each known pixel
    std::vector<uint8_t> who((size_t)P * Q, 0);
    std::vector<int32_t> when((size_t)P * Q, 0);
    int last_sync = 0;   // a synchronisation before the loads of this step
    // chain[side][l]: how many lines l+1, l+2, ... line l's front reaches
    // through same-step values in the current step (at most `maxchain`)
    int a[kMaxLines], z[kMaxLines], took[2][kMaxLines], chain[2][kMaxLines];
    for (int l = 0; l < Q; ++l) { a[l] = 0; z[l] = P - 1; }
    int64_t remaining = (int64_t)P * Q;
    std::vector<uint32_t> steps, pattern;
    std::vector<uint8_t> syncs;

    while (remaining > 0) {
        if ((int)steps.size() >= limit) return -1;
        for (int l = 0; l < Q; ++l) took[1][l] = -1;
        uint32_t word = 0;
        for (int side = 0; side < sides; ++side) {
            for (int l = Q - 1; l >= 0; --l) {
                took[side][l] = -1;
                chain[side][l] = 0;
                if (a[l] > z[l]) continue;
                const int x = side ? z[l] : a[l];
                if (side == 1 && took[0][l] == x) continue;   // the fronts met on this pixel
                const int p = pF[side][l];
                bool ready = true, linked = false;
                for (int l2 = 0; l2 < Q && ready; ++l2) {
                    if (l2 == l) continue;
                    const int64_t x2 = (int64_t)x + (int64_t)(pos[l2] - pos[l]) * p;
                    if (x2 < 0 || x2 >= P) continue;
                    if (known[(size_t)l2 * P + x2]) continue;
                    if (l2 == l + 1 && took[side][l2] == x2 && chain[side][l2] < maxchain) {
                        linked = true;
                        continue;
                    }
                    ready = false;
                }
                if (ready) {
                    took[side][l] = x;
                    chain[side][l] = linked ? chain[side][l + 1] + 1 : 0;
                    word |= 1u << (2 * l + side);
                }
            }
        }
        if (!word) return -1;
        // Operand pattern of the step: bit 2l+side set when line l of that
        // front takes its line l+1 operand from the pixel line l+1 rebuilt
        // in this same step (otherwise the operand is an earlier pixel, or a
        // pixel outside the image, and is read from memory).
        uint32_t fwd = 0;
        for (int side = 0; side < 2; ++side)
            for (int l = 0; l + 1 < Q; ++l) {
                if (took[side][l] < 0) continue;
                const int64_t x2 = (int64_t)took[side][l] + (int64_t)(pos[l + 1] - pos[l]) * pF[side][l];
                if (x2 >= 0 && x2 < P && took[side][l + 1] == x2) fwd |= 1u << (2 * l + side);
            }
        // Cross-front reads: a front reading a pixel the other front rebuilt
        // at step when >= last_sync needs the two fronts synchronised before
        // this step (kernels that run the two sides in different warps).
        const int t = (int)steps.size();
        bool cross = false;
        for (int side = 0; side < 2 && !cross; ++side)
            for (int l = 0; l < Q && !cross; ++l) {
                if (took[side][l] < 0) continue;
                for (int l2 = 0; l2 < Q; ++l2) {
                    if (l2 == l) continue;
                    const int64_t x2 = (int64_t)took[side][l] + (int64_t)(pos[l2] - pos[l]) * pF[side][l];
                    if (x2 < 0 || x2 >= P) continue;
                    const size_t k = (size_t)l2 * P + x2;
                    if (known[k] && who[k] != side && when[k] >= last_sync) cross = true;
                }
            }
        if (cross) last_sync = t;
        syncs.push_back(cross ? 1 : 0);
        pattern.push_back(fwd);
        for (int l = 0; l < Q; ++l) {
            if (took[0][l] >= 0) {
                const size_t k = (size_t)l * P + a[l];
                known[k] = 1; who[k] = 0; when[k] = t; ++a[l]; --remaining;
            }
            if (took[1][l] >= 0) {
                const size_t k = (size_t)l * P + z[l];
                known[k] = 1; who[k] = 1; when[k] = t; --z[l]; --remaining;
            }
        }
        steps.push_back(word);
    }
    // Steady steps: every front of every line moves and the operand pattern
    // is the schedule's most common one among such steps. The device runs
    // those with no per-line tests, forwarding exactly where `fwd` says.
    uint32_t all = Q >= 16 ? 0xFFFFFFFFu : (1u << (2 * Q)) - 1u;
    if (one_sided) all &= 0x55555555u;   // the left fronts only
    uint32_t fwd = 0;
    if (Q <= kFastMaxLines) {
        std::map<uint32_t, int> count;
        int best = 0;
        for (size_t t = 0; t < steps.size(); ++t)
            if (steps[t] == all && ++count[pattern[t]] > best) {
                best = count[pattern[t]];
                fwd = pattern[t];
            }
        if (best > 0)
            for (size_t t = 0; t < steps.size(); ++t)
                if (steps[t] == all && pattern[t] == fwd) steps[t] |= kStepSteady;
    }
    // Streamed chunks: by distance from the end each front starts at.
    {
        int dmax = 1;
        for (int l = 0; l < Q; ++l) dmax = std::max(dmax, std::max(a[l], P - a[l]));
        const int cw = (dmax + kStreamChunks - 1) / kStreamChunks;
        const int T = (int)steps.size();
        int first[kStreamChunks], last[kStreamChunks];
        for (int c = 0; c < kStreamChunks; ++c) {
            first[c] = T;
            last[c] = -1;
        }
        int cl[kMaxLines] = {}, cr[kMaxLines] = {};
        for (int t = 0; t < T; ++t)
            for (int l = 0; l < Q; ++l)
                for (int side = 0; side < 2; ++side) {
                    if (!(steps[t] >> (2 * l + side) & 1u)) continue;
                    const int d = side ? cr[l]++ : cl[l]++;   // distance of the rebuilt pixel
                    const int c = std::min(d / cw, kStreamChunks - 1);
                    first[c] = std::min(first[c], t);
                    last[c] = std::max(last[c], t);
                }
        out->chunk_w = cw;
        // wait for chunk c before the first step that touches c or a later chunk
        int m = T;
        for (int c = kStreamChunks - 1; c >= 0; --c) {
            m = std::min(m, first[c]);
            out->chunk_wait[c] = m;
        }
        out->chunk_wait[0] = 0;
        // chunk c is final once it and every earlier chunk are
        int M = -1;
        for (int c = 0; c < kStreamChunks; ++c) {
            M = std::max(M, last[c]);
            out->chunk_done[c] = M;
        }
    }
    for (size_t t = 0; t < syncs.size(); ++t)
        if (syncs[t]) pattern[t] |= kFwdSync;
    out->fwd = fwd;
    out->lines = Q;
    out->known = 0;
    for (int l = 0; l < Q; ++l) out->lpos[l] = pos[l];
    out->T = (int)steps.size();
    out->steps = std::move(steps);
    out->fwdw = std::move(pattern);
    for (int l = 0; l < Q; ++l) {
        const int iL = asc[l], iR = asc[Q - 1 - l];
        out->projL[l] = iL;
        out->projR[l] = iR;
        out->pL[l] = pl.p[iL];
        out->pR[l] = pl.p[iR];
        out->split[l] = a[l];
        // bin j = l p - x - b_min at word off + j of the stripe block
        // bin j = l p - x - b_min of the projection holds pixel x; the
        // kernels read stored word src - x, so src is the stored word of the
        // front's first pixel plus that pixel's x (a front reads one run of
        // consecutive bins, all stored, hence consecutive stored words)
        if (!pl.trimmed) {
            out->srcL[l] = pl.off[iL] + (int64_t)pos[l] * pl.p[iL] - pl.bmin[iL];
            out->srcR[l] = pl.off[iR] + (int64_t)pos[l] * pl.p[iR] - pl.bmin[iR];
        } else {
            const int sp = a[l];
            auto stored = [&](int i, int64_t j) {
                return (int64_t)pl.stored_of[(size_t)(pl.fulloff[i] + j)];
            };
            out->srcL[l] = sp > 0 ? pl.off[iL] + stored(iL, (int64_t)l * pl.p[iL] - pl.bmin[iL]) : 0;
            out->srcR[l] = sp < P ? pl.off[iR] + stored(iR, (int64_t)l * pl.p[iR] - sp - pl.bmin[iR]) + sp : 0;
        }
        // Row parity for bulk staging (non-systematic decode_lines keeps a
        // row in bin order, pixel x at row start + P - 1 - x): a front's run
        // starts at bin src - x_last and lands at row start + P - 1 - x_last,
        // so it is bulk-copied when the row start has the parity of
        // src + 1 - P (stripe blocks of even length); the longer run decides.
        // A systematic decode stages whole residual rows, which start at
        // even words of the data buffer when P is even: even row starts.
        const int nL = a[l], nR = P - a[l];
        const int64_t parL = (out->srcL[l] + 1 - P) & 1, parR = (out->srcR[l] + 1 - P) & 1;
        out->rowpar[l] = pl.systematic ? 0 : (int32_t)(nL >= nR ? parL : parR);
    }
    return out->T;
}

// Shared-memory bank layout of decode_lines for one path: the row phases
// (line l's row starts at a column congruent to rowoff[l] mod S) and the
// order in which each front issues its loads.
//
// decode_lines runs one lane per (line, front, stripe): lane = side * 16 +
// l * G + g, so the left fronts fill the lower half-warp and the right fronts
// the upper one. The G stripes of a warp sit in regions that start S = 16 / G
// bank slots (8-byte words mod 16) apart, so the G lanes of a front that read
// the same position of their stripes fill one slot class of a 128-byte
// wavefront: class = (row start + position) mod S. A warp's 64-bit load is
// served per half-warp (measured on GB300: the count of load wavefronts
// follows this model, not a whole-warp one), and within a half, fronts that
// read different words of the same class serialise (a bank conflict). With
// each half holding fronts that move the same way, the classes of a half keep
// their relative positions in every step where all of its fronts move.
//
// Each front reads its own bin first, then XORs the other Q - 1 words of
// the step (the pixels of the bin line on the other lines; a word line l+1
// rebuilds in the same step is read too, and cancels on the device) in any
// order: order[2l + side] holds in nibble k the word that load instruction
// k reads (nibble 0 = 0, the own bin; j >= 1: the pixel on line l + j mod
// Q). Choosing phases and orders so that each instruction meets distinct
// slots is an edge colouring of the bipartite multigraph fronts x slots.
//
// This replays the path -- a front that does not move loads nothing, and
// every read of a line outside the image is one word, the zero word beside
// its row -- and costs a load instruction of a half the largest number of
// distinct words one class receives (its wavefronts); the store of the
// rebuilt pixels counts the same way. Phases by coordinate descent and
// orders by pairwise swaps, alternated, from three deterministic starts.
void choose_row_phases(const Plan &pl, Schedule *sc)
{
    sc->phases_done = true;
    const int P = pl.P, Q = sc->lines;
    for (int l = 0; l < kMaxLines; ++l) sc->rowoff[l] = sc->rowpar[l];
    for (int f = 0; f < 2 * kMaxLines; ++f) sc->order[f] = kIdentityOrder;
    if (Q < 2 || Q > 8) return;
    const int G = std::max(1, 32 / (2 * Q));
    if (16 % G != 0 || G >= 16) return;
    const int S = 16 / G;
    const int T = sc->T;
    // Non-systematic plans keep their rows in bin order (pixel x at row
    // start + P - 1 - x), systematic ones in pixel order. A row's phase
    // parity decides which of its runs are staged by bulk copies (rowpar:
    // from the path, or even for the residual rows of a systematic decode);
    // the search keeps that parity.
    const bool rev = !pl.systematic;
    const bool fixpar = S % 2 == 0;
    const int K = Q;          // words per front and step
    const int F = 2 * Q;      // fronts, index side * Q + l
    // Every step is replayed to track the fronts; the cost counts at most
    // 96 of them, evenly spaced.
    const int stride = std::max(1, (T + 95) / 96);
    const int TC = (T + stride - 1) / stride;
    // word j of front f at counted step c: (line << 16) | (column + 32768),
    // or -1 (no load); the front's store likewise
    auto key = [rev](int line, int col) {
        if (rev) col = -col;
        return (int32_t)((line << 16) | ((col + 32768) & 0xFFFF));
    };
    std::vector<int32_t> acc((size_t)TC * F * K, -1), sto((size_t)TC * F, -1);
    int x[2][kMaxLines];
    for (int l = 0; l < Q; ++l) { x[0][l] = 0; x[1][l] = P - 1; }
    for (int t = 0; t < T; ++t) {
        const uint32_t w = sc->steps[(size_t)t];
        if (t % stride == 0) {
            const int c = t / stride;
            for (int side = 0; side < 2; ++side)
                for (int l = 0; l < Q; ++l) {
                    const int bit = 2 * l + side;
                    if (!((w >> bit) & 1u)) continue;
                    const int f = side * Q + l;
                    const int p = side ? sc->pR[l] : sc->pL[l];
                    const int xx = x[side][l];
                    sto[(size_t)c * F + f] = key(l, xx);
                    int32_t *a = &acc[((size_t)c * F + f) * K];
                    a[0] = key(l, xx);
                    for (int j = 1; j < Q; ++j) {
                        const int l2 = (l + j) % Q;
                        int col = xx + (sc->lpos[l2] - sc->lpos[l]) * p;
                        if (col < 0 || col >= P) col = P;   // the zero word beside the row
                        a[j] = key(l2, col);
                    }
                }
        }
        for (int l = 0; l < Q; ++l)
            for (int side = 0; side < 2; ++side)
                if ((w >> (2 * l + side)) & 1u) x[side][l] += side ? -1 : 1;
    }
    int e[kMaxLines] = {};
    uint8_t ord[2 * kMaxLines][kMaxLines];
    // wavefronts of one set of words a half reads at once (k >= 0: load
    // instruction k; k < 0: the store)
    auto cost = [&](int h, int k) {
        int64_t c = 0;
        for (int t = 0; t < TC; ++t) {
            int cnt[16] = {};
            int32_t seen[16][kMaxLines];
            int worst = 0;
            for (int l = 0; l < Q; ++l) {
                const int f = h * Q + l;
                const int32_t kk = k < 0 ? sto[(size_t)t * F + f] : acc[((size_t)t * F + f) * K + ord[f][k]];
                if (kk < 0) continue;
                const int line = kk >> 16, col = (kk & 0xFFFF) - 32768;
                const int q = ((e[line] + col) % S + S) % S;
                bool dup = false;
                for (int i = 0; i < cnt[q]; ++i) dup = dup || seen[q][i] == kk;
                if (dup) continue;
                seen[q][cnt[q]++] = kk;
                worst = std::max(worst, cnt[q]);
            }
            c += worst;
        }
        return c;
    };
    int64_t part[2][kMaxLines + 1];
    auto total = [&]() {
        int64_t c = 0;
        for (int h = 0; h < 2; ++h)
            for (int k = -1; k < K; ++k) c += (part[h][k + 1] = cost(h, k));
        return c;
    };
    int best_e[kMaxLines] = {};
    uint8_t best_ord[2 * kMaxLines][kMaxLines];
    int64_t best_c = -1;
    uint32_t rng = 0x9E3779B9u ^ (uint32_t)(P * 131 + Q) ^ sc->mask;
    for (int start = 0; start < 3; ++start) {
        for (int l = 0; l < Q; ++l) {
            rng = rng * 1664525u + 1013904223u;
            e[l] = start == 0 ? 0 : (int)((rng >> 16) % (uint32_t)S);
            if (fixpar && ((e[l] ^ sc->rowpar[l]) & 1)) e[l] = (e[l] + 1) % S;
        }
        for (int f = 0; f < F; ++f)
            for (int k = 0; k < K; ++k) ord[f][k] = (uint8_t)k;
        int64_t c = total();
        for (int round = 0; round < 6; ++round) {
            bool improved = false;
            for (int l = 0; l < Q; ++l) {
                const int keep = e[l];
                int bestv = keep;
                for (int v = 0; v < S; ++v) {
                    if (v == keep || (fixpar && ((v ^ sc->rowpar[l]) & 1))) continue;
                    e[l] = v;
                    const int64_t cv = total();
                    if (cv < c) {
                        c = cv;
                        bestv = v;
                        improved = true;
                    }
                }
                e[l] = bestv;
                total();   // refresh the per-instruction parts
            }
            for (int h = 0; h < 2; ++h)
                for (int l = 0; l < Q; ++l) {
                    const int f = h * Q + l;
                    for (int a = 1; a < K; ++a)
                        for (int b = a + 1; b < K; ++b) {
                            std::swap(ord[f][a], ord[f][b]);
                            const int64_t ca = cost(h, a), cb = cost(h, b);
                            const int64_t d = ca + cb - part[h][a + 1] - part[h][b + 1];
                            if (d < 0) {
                                part[h][a + 1] = ca;
                                part[h][b + 1] = cb;
                                c += d;
                                improved = true;
                            } else {
                                std::swap(ord[f][a], ord[f][b]);
                            }
                        }
                }
            if (!improved) break;
        }
        if (best_c < 0 || c < best_c) {
            best_c = c;
            for (int l = 0; l < Q; ++l) best_e[l] = e[l];
            std::memcpy(best_ord, ord, sizeof(ord));
        }
    }
    for (int l = 0; l < Q; ++l) sc->rowoff[l] = best_e[l];
    for (int side = 0; side < 2; ++side)
        for (int l = 0; l < Q; ++l) {
            uint32_t o = 0;
            for (int k = 0; k < K; ++k) o |= (uint32_t)best_ord[side * Q + l][k] << (4 * k);
            sc->order[2 * l + side] = o;
        }
}

// Cap on the number of Q-subsets of the survivors tried per mask.
constexpr int kMaxCandidates = 512;

}  // namespace

int build_schedule(const Plan &pl, uint32_t mask, Schedule *out)
{
    if (pl.Q > kMaxLines) return -EINVAL;
    // Lines to rebuild (image rows, ascending) and surviving projections.
    // Non-systematic: every line, from any Q of the n projections.
    // Systematic: the lost data lines (mask bits 0 .. Q-1), each with one of
    // the surviving parity projections (mask bits Q .. Q+n-1).
    int pos[kMaxLines];
    int L = 0;
    std::vector<int> surv;
    if (pl.systematic) {
        for (int l = 0; l < pl.Q; ++l)
            if (mask >> l & 1u) pos[L++] = l;
        for (int i = 0; i < pl.n; ++i)
            if (!(mask >> (pl.Q + i) & 1u)) surv.push_back(i);
        if (L == 0) {
            // nothing lost: the data lines are the image, no path
            *out = Schedule();
            out->mask = mask;
            out->lines = 0;
            out->known = (pl.Q >= 32 ? 0xFFFFFFFFu : (1u << pl.Q) - 1u);
            out->phases_done = true;
            return 0;
        }
        if (L > kSysMaxLines) return -EINVAL;
    } else {
        for (int l = 0; l < pl.Q; ++l) pos[L++] = l;
        for (int i = 0; i < pl.n; ++i)
            if (!(mask >> i & 1u)) surv.push_back(i);
    }
    if ((int)surv.size() < L) return -ENOTRECOVERABLE;

    // Any L survivors rebuild the same lines (Eq. 3 gives uniqueness; for
    // the systematic form, the generalised Vandermonde argument of the
    // oracle's tests); pick the subset with the fewest steps. Candidates
    // are enumerated with the smallest |p| first.
    std::stable_sort(surv.begin(), surv.end(), [&](int x, int y) {
        const int ax = pl.p[x] < 0 ? -pl.p[x] : pl.p[x];
        const int ay = pl.p[y] < 0 ? -pl.p[y] : pl.p[y];
        return ax < ay;
    });
    const int m = (int)surv.size();
    std::vector<int> pick(L);
    std::iota(pick.begin(), pick.end(), 0);
    int best = -1;
    Schedule tmp;
    int tried = 0;
    while (true) {
        std::vector<int> asc(L);
        for (int k = 0; k < L; ++k) asc[k] = surv[pick[k]];
        std::sort(asc.begin(), asc.end(), [&](int x, int y) { return pl.p[x] < pl.p[y]; });
        if (pl.systematic && L == 1) {
            // one lost line: once the known lines are removed every bin of
            // the projection holds one lost pixel, so no step is needed
            tmp = Schedule();
            const int i = asc[0];
            tmp.lines = 1;
            tmp.lpos[0] = pos[0];
            tmp.projL[0] = tmp.projR[0] = i;
            tmp.pL[0] = tmp.pR[0] = pl.p[i];
            tmp.split[0] = pl.P;
            tmp.srcL[0] = tmp.srcR[0] = pl.off[i] + (int64_t)pos[0] * pl.p[i] - pl.bmin[i];
            tmp.T = 0;
            best = 0;
            *out = tmp;
            break;
        }
        const int limit = best < 0 ? (1 << 30) : best;
        int T = sweep(pl, asc, pos, L, limit, &tmp);
        if (T >= 0 && (best < 0 || T < best)) {
            best = T;
            *out = tmp;
            // The same path length with shorter same-step chains, where one
            // exists: decode_lines runs a shuffle round per chain link it may
            // meet in a steady step (Q <= 4: one per link of the longest
            // chain; Q > 4: rounds of stride 1, 2, 4), so prefer bound 1,
            // then 2 (Q <= 4) or 3 (Q > 4), never at the cost of a step.
            const int bounds[2] = {1, L <= 4 ? 2 : 3};
            for (int b : bounds) {
                if (b >= L - 1) break;
                Schedule alt;
                if (sweep(pl, asc, pos, L, best + 1, &alt, false, b) == best) {
                    *out = alt;
                    break;
                }
            }
        }
        if (++tried >= kMaxCandidates) break;
        // next combination of L out of m
        int k = L - 1;
        while (k >= 0 && pick[k] == m - L + k) --k;
        if (k < 0) break;
        ++pick[k];
        for (int r = k + 1; r < L; ++r) pick[r] = pick[r - 1] + 1;
    }
    if (best < 0) return -ENOTRECOVERABLE;
    out->mask = mask;
    out->scan2 = false;
    if (L == 2 && !pl.trimmed) {
        // the closed form for two lines: any two survivors with distinct
        // directions; the widest gap p_b - p_a gives the fewest scan rounds
        // (ties: the smaller directions)
        int ba = -1, bb = -1;
        for (int x = 0; x < m; ++x)
            for (int y = 0; y < m; ++y) {
                const int ia = surv[x], ib = surv[y];
                if (pl.p[ia] >= pl.p[ib]) continue;
                const int gap = pl.p[ib] - pl.p[ia];
                const int big = std::max(std::abs(pl.p[ia]), std::abs(pl.p[ib]));
                if (ba < 0 || gap > pl.p[bb] - pl.p[ba] ||
                    (gap == pl.p[bb] - pl.p[ba] && big < std::max(std::abs(pl.p[ba]), std::abs(pl.p[bb])))) {
                    ba = ia;
                    bb = ib;
                }
            }
        if (ba >= 0) {
            out->scan2 = true;
            const int idx[2] = {ba, bb};
            for (int j = 0; j < 2; ++j) {
                const int i = idx[j];
                out->scan_proj[j] = i;
                out->scan_p[j] = pl.p[i];
                out->scan_src[j] = pl.off[i] + (int64_t)pos[j] * pl.p[i] - pl.bmin[i];
            }
        }
    }
    out->vander = false;
    if (!pl.systematic && !pl.trimmed && L >= 2 && L <= 8) {
        // decode_vander: the first Q survivors by |p| (the narrowest frame),
        // ascending directions
        std::vector<int> v(surv.begin(), surv.begin() + L);
        std::sort(v.begin(), v.end(), [&](int x, int y) { return pl.p[x] < pl.p[y]; });
        const int64_t E0 = -(int64_t)(pl.P - 1) + std::min<int64_t>(0, (int64_t)(L - 1) * pl.p[v[0]]);
        const int64_t top = (int64_t)(L - 1) * std::max(0, pl.p[v[L - 1]]);
        const int64_t Lw = top - E0 + 2;
        if (Lw < (1 << 20)) {
            out->vander = true;
            out->van_E0 = (int32_t)E0;
            out->van_L = (int32_t)Lw;
            for (int j = 0; j < L; ++j) {
                const int i = v[j];
                out->van_proj[j] = i;
                out->van_q[j] = pl.p[i];
                out->van_base[j] = pl.off[i] - pl.bmin[i];
                out->van_lo[j] = (int32_t)pl.bmin[i];
                out->van_hi[j] = (int32_t)(pl.bmin[i] + pl.B[i]);
            }
        }
    }
    if (pl.systematic) {
        uint32_t known = 0;
        for (int l = 0; l < pl.Q; ++l)
            if (!(mask >> l & 1u)) known |= 1u << l;
        out->known = known;
    }
    out->dev.clear();
    return 0;
}

namespace {

// Replays a one-sided path the way decode_ring runs it -- line l's ring of R
// words holds column c at slot R - 1 - ((c + ring_delta[l]) mod R); at the
// start chunks -1 .. D are filled (bins inside the image, zeros outside);
// when a front enters chunk k (column c with c + ring_delta = 16 k > 0) it
// fills chunk k + D over the slots of chunk k + D - R / 16; a chunk of 16
// columns is written out at the end of the step that rebuilds its last
// pixel -- and checks that every word a front reads holds what the path
// needs at that moment: its own bin, the stale bin of a forwarded word, a
// pixel rebuilt earlier, or a zero outside the image; and that every pixel
// is still there when its chunk is written out.
bool ring_fits(const Plan &pl, const Schedule &sc, int R, int D)
{
    const int P = pl.P, Q = sc.lines;
    const int NS = R / kRingChunk;
    if (Q < 1 || P % kRingChunk || R % kRingChunk || NS <= D + 1) return false;
    struct Word {
        int32_t col;
        int8_t kind;   // 0 nothing, 1 bin, 2 pixel, 3 zero
    };
    std::vector<Word> ring((size_t)Q * R, Word{INT32_MIN, 0});
    auto slot = [&](int l, int c) -> Word & {
        const int u = ((c + sc.ring_delta[l]) % R + R) % R;
        return ring[(size_t)l * R + (R - 1 - u)];
    };
    auto fill = [&](int l, int k) {
        for (int i = 0; i < kRingChunk; ++i) {
            const int c = kRingChunk * k + i - sc.ring_delta[l];
            Word &w = slot(l, c);
            w.col = c;
            w.kind = (c >= 0 && c < P) ? 1 : 3;
        }
    };
    for (int l = 0; l < Q; ++l)
        for (int k = -1; k <= D; ++k) fill(l, k);
    std::vector<int> x(Q, 0);
    for (int t = 0; t < sc.T; ++t) {
        const uint32_t w = sc.steps[(size_t)t], f = sc.fwdw[(size_t)t];
        for (int l = 0; l < Q; ++l) {
            if (!(w >> (2 * l) & 1u)) continue;
            const int u = x[l] + sc.ring_delta[l];
            if (u > 0 && u % kRingChunk == 0) fill(l, u / kRingChunk + D);
        }
        for (int l = 0; l < Q; ++l) {
            if (!(w >> (2 * l) & 1u)) continue;
            for (int l2 = 0; l2 < Q; ++l2) {
                const int c = x[l] + (sc.lpos[l2] - sc.lpos[l]) * sc.pL[l];
                const Word &o = slot(l2, c);
                if (o.col != c) return false;
                if (l2 == l || (l2 == l + 1 && (f >> (2 * l) & 1u))) {
                    if (o.kind != 1) return false;   // own bin, or a forwarded word's stale bin
                } else if (c < 0 || c >= P) {
                    if (o.kind != 3) return false;
                } else if (o.kind != 2) {
                    return false;
                }
            }
        }
        for (int l = 0; l < Q; ++l) {
            if (!(w >> (2 * l) & 1u)) continue;
            Word &o = slot(l, x[l]);
            o.kind = 2;
            if (x[l] % kRingChunk == kRingChunk - 1)
                for (int c = x[l] - (kRingChunk - 1); c <= x[l]; ++c) {
                    const Word &q = slot(l, c);
                    if (q.col != c || q.kind != 2) return false;
                }
            ++x[l];
        }
    }
    for (int l = 0; l < Q; ++l)
        if (x[l] != P) return false;
    return true;
}

}  // namespace

int build_ring_schedule(const Plan &pl, uint32_t mask, Schedule *out)
{
    if (pl.systematic || pl.trimmed || pl.Q > kMaxLines) return -EINVAL;
    int pos[kMaxLines];
    const int L = pl.Q;
    for (int l = 0; l < L; ++l) pos[l] = l;
    std::vector<int> surv;
    for (int i = 0; i < pl.n; ++i)
        if (!(mask >> i & 1u)) surv.push_back(i);
    if ((int)surv.size() < L) return -ENOTRECOVERABLE;
    std::stable_sort(surv.begin(), surv.end(), [&](int a, int b) {
        return std::abs(pl.p[a]) < std::abs(pl.p[b]);
    });
    const int m = (int)surv.size();
    std::vector<int> pick(L);
    std::iota(pick.begin(), pick.end(), 0);
    int best = -1, tried = 0;
    Schedule tmp;
    while (true) {
        std::vector<int> asc(L);
        for (int k = 0; k < L; ++k) asc[k] = surv[pick[k]];
        std::sort(asc.begin(), asc.end(), [&](int a, int b) { return pl.p[a] < pl.p[b]; });
        const int T = sweep(pl, asc, pos, L, best < 0 ? (1 << 30) : best, &tmp, true);
        if (T >= 0 && (best < 0 || T < best)) {
            best = T;
            *out = tmp;
        }
        if (++tried >= kMaxCandidates) break;
        int k = L - 1;
        while (k >= 0 && pick[k] == m - L + k) --k;
        if (k < 0) break;
        ++pick[k];
        for (int r = k + 1; r < L; ++r) pick[r] = pick[r - 1] + 1;
    }
    if (best < 0) return -ENOTRECOVERABLE;
    out->mask = mask;
    out->one_sided = true;
    out->scan2 = out->vander = false;
    // chunk starts: a chunk's bins are 16 consecutive words ending at the
    // bin of its first column, src - (16 k - delta); a 16-byte aligned
    // source needs src - 16 k + delta - 15 even
    for (int l = 0; l < L; ++l) out->ring_delta[l] = (int32_t)((out->srcL[l] + 1) & 1);
    out->ring_R = out->ring_D = 0;
    const int RD[2][2] = {{64, 2}, {128, 3}};
    for (const auto &rd : RD)
        if (rd[0] < pl.P && ring_fits(pl, *out, rd[0], rd[1])) {
            out->ring_R = rd[0];
            out->ring_D = rd[1];
            break;
        }
    // chunk events per step (see Schedule::ringev)
    out->ringev.assign((size_t)out->T, 0u);
    std::vector<int> x(L, 0);
    for (int t = 0; t < out->T; ++t) {
        const uint32_t w = out->steps[(size_t)t];
        uint32_t ev = 0;
        for (int l = 0; l < L; ++l) {
            if (!(w >> (2 * l) & 1u)) continue;
            const int u = x[l] + out->ring_delta[l];
            if (u > 0 && u % kRingChunk == 0) ev |= 1u << l;
            if (x[l] % kRingChunk == kRingChunk - 1) ev |= 1u << (8 + l);
            ++x[l];
        }
        out->ringev[(size_t)t] = ev;
    }
    out->dev.clear();
    return 0;
}

Schedule *get_ring_schedule(Plan &pl, uint32_t mask, int *err)
{
    std::lock_guard<std::mutex> g(pl.mu);
    auto it = pl.ring_schedules.find(mask);
    if (it != pl.ring_schedules.end()) return it->second.get();
    std::unique_ptr<Schedule> sc(new (std::nothrow) Schedule());
    if (!sc) {
        *err = -ENOMEM;
        return nullptr;
    }
    const int r = build_ring_schedule(pl, mask, sc.get());
    if (r) {
        *err = r;
        return nullptr;
    }
    Schedule *raw = sc.get();
    pl.ring_schedules[mask] = std::move(sc);
    return raw;
}

Schedule *get_schedule(Plan &pl, uint32_t mask, int *err)
{
    std::lock_guard<std::mutex> g(pl.mu);
    auto it = pl.schedules.find(mask);
    if (it != pl.schedules.end()) return it->second.get();
    std::unique_ptr<Schedule> sc;
    try {
        sc.reset(new Schedule());
    } catch (...) {
        *err = -ENOMEM;
        return nullptr;
    }
    const int r = build_schedule(pl, mask, sc.get());
    if (r) {
        *err = r;
        return nullptr;
    }
    Schedule *raw = sc.get();
    pl.schedules[mask] = std::move(sc);
    return raw;
}

int schedule_on_device(Plan &pl, Schedule &sc, uint32_t **dev)
{
    int device = 0;
    int r = record_cuda(cudaGetDevice(&device));
    if (r) return r;
    std::lock_guard<std::mutex> g(pl.mu);
    auto it = sc.dev.find(device);
    if (it != sc.dev.end()) {
        *dev = it->second;
        return 0;
    }
    // device copy: the step words, then the forward words; a one-sided
    // path also (step, forward, chunk event, 0) per step from the next
    // multiple of 4 words, plus one zero entry
    uint32_t *d = nullptr;
    const size_t n = sc.steps.size();
    const size_t n4 = sc.one_sided ? (2 * n + 3) / 4 * 4 + 4 * (n + 1) : 2 * n;
    const size_t bytes = std::max<size_t>(4, n4 * sizeof(uint32_t));
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e == cudaErrorMemoryAllocation) {
        record_cuda(e);
        return -ENOMEM;
    }
    if ((r = record_cuda(e))) return r;
    std::vector<uint32_t> both(n4, 0u);
    std::copy(sc.steps.begin(), sc.steps.end(), both.begin());
    std::copy(sc.fwdw.begin(), sc.fwdw.end(), both.begin() + n);
    if (sc.one_sided) {
        const size_t b4 = (2 * n + 3) / 4 * 4;
        for (size_t t = 0; t < n; ++t) {
            both[b4 + 4 * t] = sc.steps[t];
            both[b4 + 4 * t + 1] = sc.fwdw[t];
            both[b4 + 4 * t + 2] = t < sc.ringev.size() ? sc.ringev[t] : 0u;
        }
    }
    if (n && (r = record_cuda(cudaMemcpy(d, both.data(), n4 * sizeof(uint32_t), cudaMemcpyHostToDevice)))) {
        cudaFree(d);
        return r;
    }
    sc.dev[device] = d;
    *dev = d;
    return 0;
}

const int32_t *schedule_row_phases(Plan &pl, Schedule &sc)
{
    std::lock_guard<std::mutex> g(pl.mu);
    if (!sc.phases_done) choose_row_phases(pl, &sc);
    return sc.rowoff;
}

// Unused-bin removal (Sec. 2.3 mentions that some bins need not be stored;
// the paper gives no rule). Here a bin is unused when no reconstruction path
// of this library reads it for any erasure mask that leaves at least Q
// projections: the decoder reads bin l p - x - b_min of the projection
// dedicated to line l for every pixel x of that line's front, one run of
// consecutive bins per (line, front). A trimmed projection stores the bins
// some path reads, in order; a run a path reads is then a run of
// consecutive stored words too, so the decoder is unchanged but for its
// base offsets, and the encoder computes each stored word from its full bin
// index (Plan::full_bin). The paths are the cached ones, built here for
// every mask; their offsets are rebuilt after the trim.
int trim_unused_bins(Plan &pl)
{
    const int n = pl.n, Q = pl.Q, P = pl.P;
    if (Q > kMaxLines || n > 20) return -EINVAL;
    int64_t full = 0;
    for (int i = 0; i < n; ++i) {
        pl.fulloff[i] = full;
        full += pl.B[i];
    }
    std::vector<uint8_t> used((size_t)full, 0);
    int err = 0;
    for (uint32_t mask = 0; mask < (1u << n); ++mask) {
        if (__builtin_popcount(mask) > n - Q) continue;
        Schedule *sc = get_schedule(pl, mask, &err);
        if (!sc) return err;
        for (int l = 0; l < Q; ++l) {
            const int sp = sc->split[l];
            for (int side = 0; side < 2; ++side) {
                const int i = side ? sc->projR[l] : sc->projL[l];
                const int x0 = side ? sp : 0, x1 = side ? P : sp;
                for (int x = x0; x < x1; ++x)
                    used[(size_t)(pl.fulloff[i] + (int64_t)l * pl.p[i] - x - pl.bmin[i])] = 1;
            }
        }
    }
    pl.stored_of.assign((size_t)full, -1);
    pl.full_bin.clear();
    int64_t t = 0;
    for (int i = 0; i < n; ++i) {
        pl.off[i] = t;
        int32_t s = 0;
        for (int64_t j = 0; j < pl.B[i]; ++j)
            if (used[(size_t)(pl.fulloff[i] + j)]) {
                pl.stored_of[(size_t)(pl.fulloff[i] + j)] = s++;
                pl.full_bin.push_back((int32_t)j);
            }
        pl.B[i] = s;
        t += s;
    }
    pl.total = t;
    pl.trimmed = true;
    std::lock_guard<std::mutex> g(pl.mu);
    pl.schedules.clear();        // their bin offsets follow the full layout
    return 0;
}

int plan_full_bin_on_device(Plan &pl, const int32_t **dev)
{
    *dev = nullptr;
    if (!pl.trimmed) return 0;
    int device = 0;
    int r = record_cuda(cudaGetDevice(&device));
    if (r) return r;
    std::lock_guard<std::mutex> g(pl.mu);
    auto it = pl.full_bin_dev.find(device);
    if (it != pl.full_bin_dev.end()) {
        *dev = it->second;
        return 0;
    }
    int32_t *d = nullptr;
    const size_t bytes = std::max<size_t>(4, pl.full_bin.size() * sizeof(int32_t));
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e == cudaErrorMemoryAllocation) {
        record_cuda(e);
        return -ENOMEM;
    }
    if ((r = record_cuda(e))) return r;
    if ((r = record_cuda(cudaMemcpy(d, pl.full_bin.data(), pl.full_bin.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice)))) {
        cudaFree(d);
        return r;
    }
    pl.full_bin_dev[device] = d;
    *dev = d;
    return 0;
}

}  // namespace mojette
