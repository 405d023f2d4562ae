/*
 * Mojette erasure code over GF(2): plain, slow CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do. It shares no code with the CUDA library.
 *
 * Conventions (the paper's notation, with the clash of "k" resolved):
 *   image      f(x, l), x in [0, P) the column (pixel index in a data line),
 *              l in [0, Q) the row (the paper's "k data lines", Sec. 2.3).
 *              Stored row-major: img[l * P + x], one uint64 word per pixel.
 *   direction  (p_i, q_i) with q_i = 1 for every projection (Sec. 2.3).
 *   bin        position b = l * p - x  (Eq. 1 with q = 1: b = -x q + l p).
 *              Stored at index j = b - b_min, b_min the smallest b that any
 *              pixel of the lattice reaches.
 *   addition   XOR of 64-bit words (Sec. 3, "Mojette" paragraph).
 *   stripe     one image; S stripes are stored back to back.
 *   output     proj[s][off_i + j], the n projections of a stripe concatenated
 *              in the order the directions are given.
 *
 * Error returns are negative errno values: -EINVAL for bad arguments,
 * -ENOTRECOVERABLE when the surviving projections cannot rebuild the image,
 * -ENOMEM when a work buffer cannot be allocated.
 *
 * parity pins (all in the CPU test-suite): Eq. 2 against enumeration of the
 * lattice, impulse images, the XOR-of-all-bins invariant, border bins equal
 * to single pixels, hand-worked 3x3 fixtures, brute-force GF(2) elimination,
 * and round trips through every erasure pattern.
 */
#include <errno.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_PROJ 32

/* Eq. 2 with q = 1: B(p, 1, P, Q) = |p| (Q - 1) + |1| (P - 1) + 1. */
int64_t oracle_bin_count(int p, int P, int Q)
{
    int64_t ap = p < 0 ? -(int64_t)p : (int64_t)p;
    return ap * (Q - 1) + (int64_t)(P - 1) + 1;
}

/* Smallest bin position b = l p - x over the whole lattice, by enumeration
 * (Eq. 1): the storage origin of a projection. */
int64_t oracle_bin_min(int p, int P, int Q)
{
    int64_t best = 0;
    int first = 1;
    for (int l = 0; l < Q; ++l)
        for (int x = 0; x < P; ++x) {
            int64_t b = (int64_t)l * p - x;
            if (first || b < best) { best = b; first = 0; }
        }
    return best;
}

static int check_geometry(int P, int Q, const int *p, int n)
{
    if (P < 1 || Q < 1 || n < 1 || n > ORACLE_MAX_PROJ || !p) return -EINVAL;
    for (int i = 0; i < n; ++i)
        for (int k = i + 1; k < n; ++k)
            if (p[i] == p[k]) return -EINVAL;  /* distinct directions */
    return 0;
}

/* Total number of bins of one stripe (all n projections). */
int64_t oracle_total_bins(int P, int Q, const int *p, int n)
{
    if (check_geometry(P, Q, p, n)) return -EINVAL;
    int64_t t = 0;
    for (int i = 0; i < n; ++i) t += oracle_bin_count(p[i], P, Q);
    return t;
}

/* Katz criterion, Eq. 3, for the projections whose bit is clear in mask:
 * P <= sum |p_i| or Q <= sum |q_i| (q_i = 1). Returns 1 if it holds. */
int oracle_katz(int P, int Q, const int *p, int n, uint32_t mask)
{
    int64_t sp = 0, sq = 0;
    for (int i = 0; i < n; ++i) {
        if (mask >> i & 1u) continue;
        sp += p[i] < 0 ? -(int64_t)p[i] : p[i];
        sq += 1;
    }
    return (P <= sp) || (Q <= sq);
}

/* Forward Mojette transform of one stripe, Eq. 1 read as a scatter: every
 * pixel f(x, l) is added (XOR) into the bin b = l p_i - x of every
 * projection i. */
static void encode_one(int P, int Q, const int *p, int n, const int64_t *off,
                       const int64_t *bmin, int64_t total, const uint64_t *img,
                       uint64_t *proj)
{
    memset(proj, 0, (size_t)total * sizeof(uint64_t));
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < Q; ++l)
            for (int x = 0; x < P; ++x) {
                int64_t b = (int64_t)l * p[i] - x;
                proj[off[i] + (b - bmin[i])] ^= img[(int64_t)l * P + x];
            }
}

struct layout {
    int64_t off[ORACLE_MAX_PROJ];
    int64_t bmin[ORACLE_MAX_PROJ];
    int64_t bins[ORACLE_MAX_PROJ];
    int64_t total;
};

static void make_layout(int P, int Q, const int *p, int n, struct layout *L)
{
    L->total = 0;
    for (int i = 0; i < n; ++i) {
        L->off[i] = L->total;
        L->bins[i] = oracle_bin_count(p[i], P, Q);
        L->bmin[i] = oracle_bin_min(p[i], P, Q);
        L->total += L->bins[i];
    }
}

/*
 * Peeling loop of the inverse Mojette transform (Sec. 2.2, "Inverse Mojette
 * Algorithm"), shared by both decoders below. On entry w holds the working
 * bins of the surviving projections (known pixels already removed), cnt the
 * number of unknown pixels in each bin, known the pixels already known, and
 * queue[0, tail) the bins with exactly one unknown pixel. Then, until
 * `want` pixels have been found:
 *   - a bin with exactly one unknown pixel is reconstructible;
 *   - its value is written to that pixel (back-projection);
 *   - the pixel's contribution is removed (XOR) from the bin it falls in,
 *     in every surviving projection, which may make further bins
 *     reconstructible.
 * Reconstructible bins are taken first-in first-out. Returns the number of
 * pixels found, or -ENOTRECOVERABLE if the counts fall out of step (a bug).
 */
static int64_t peel(int P, int Q, const int *p, int n, const struct layout *L,
                    uint32_t pmask, uint64_t *img, uint64_t *w, int32_t *cnt,
                    uint8_t *known, int64_t *queue, int64_t tail,
                    const uint8_t *pid, int64_t want)
{
    int64_t head = 0, found = 0;
    while (head < tail && found < want) {
        int64_t t = queue[head++];
        if (cnt[t] != 1) continue;
        int i = pid[t];
        int64_t b = (t - L->off[i]) + L->bmin[i];
        /* the single unknown pixel on the discrete line b = l p_i - x */
        int lu = -1;
        int64_t xu = -1;
        for (int l = 0; l < Q; ++l) {
            int64_t x = (int64_t)l * p[i] - b;
            if (x < 0 || x >= P) continue;
            if (!known[(int64_t)l * P + x]) { lu = l; xu = x; break; }
        }
        if (lu < 0) return -ENOTRECOVERABLE; /* counts out of step: a bug */
        uint64_t v = w[t];
        img[(int64_t)lu * P + xu] = v;
        known[(int64_t)lu * P + xu] = 1;
        found += 1;
        for (int i2 = 0; i2 < n; ++i2) {
            if (pmask >> i2 & 1u) continue;
            int64_t t2 = L->off[i2] + ((int64_t)lu * p[i2] - xu - L->bmin[i2]);
            w[t2] ^= v;
            cnt[t2] -= 1;
            if (cnt[t2] == 1) queue[tail++] = t2;
        }
    }
    return found;
}

/*
 * Inverse Mojette transform of one stripe (Sec. 2.2) with every surviving
 * projection taking part: all pixels start unknown, the working bins are
 * the surviving projections as stored, then peel(). Returns
 * -ENOTRECOVERABLE if no bin is reconstructible while pixels are unknown.
 * Work buffers are supplied by the caller (sized by the layout).
 */
static int decode_one(int P, int Q, const int *p, int n, const struct layout *L,
                      uint32_t mask, const uint64_t *proj, uint64_t *img,
                      uint64_t *w, int32_t *cnt, uint8_t *known, int64_t *queue,
                      uint8_t *pid)
{
    const int64_t npix = (int64_t)P * Q;

    /* working copies of the surviving bins and their unknown-pixel counts */
    for (int i = 0; i < n; ++i)
        for (int64_t j = 0; j < L->bins[i]; ++j) {
            w[L->off[i] + j] = (mask >> i & 1u) ? 0 : proj[L->off[i] + j];
            cnt[L->off[i] + j] = 0;
            pid[L->off[i] + j] = (uint8_t)i;
        }
    for (int i = 0; i < n; ++i) {
        if (mask >> i & 1u) continue;
        for (int l = 0; l < Q; ++l)
            for (int x = 0; x < P; ++x)
                cnt[L->off[i] + ((int64_t)l * p[i] - x - L->bmin[i])] += 1;
    }
    memset(known, 0, (size_t)npix);

    int64_t tail = 0;
    for (int i = 0; i < n; ++i) {
        if (mask >> i & 1u) continue;
        for (int64_t j = 0; j < L->bins[i]; ++j)
            if (cnt[L->off[i] + j] == 1) queue[tail++] = L->off[i] + j;
    }
    int64_t found = peel(P, Q, p, n, L, mask, img, w, cnt, known, queue, tail, pid, npix);
    if (found < 0) return (int)found;
    return found == npix ? 0 : -ENOTRECOVERABLE;
}

/*
 * Systematic form of the code (the paper mentions it in Sec. 2.3 and Sec. 4
 * without defining it; this is the reading used throughout): the Q data
 * lines are themselves Q of the packets, and r parity packets are the
 * projections of the whole image along the r directions p[0..r-1] (Eq. 1).
 * Erasure mask bit l (l < Q) marks data line l lost, bit Q + i parity
 * projection i lost. Decoding copies the surviving lines, removes (XOR)
 * their pixels from the surviving projections -- Eq. 1's sum over the
 * known pixels -- and peels the lost lines as in Sec. 2.2. With no line
 * lost it is a copy. Returns -ENOTRECOVERABLE if the peeling stalls.
 */
static int sys_decode_one(int P, int Q, const int *p, int r, const struct layout *L,
                          uint32_t mask, const uint64_t *data, const uint64_t *parity,
                          uint64_t *img, uint64_t *w, int32_t *cnt, uint8_t *known,
                          int64_t *queue, uint8_t *pid)
{
    const uint32_t pmask = mask >> Q;     /* parity projection i lost: bit i */
    int64_t unknown = 0;
    for (int l = 0; l < Q; ++l) {
        const int lost = (int)(mask >> l & 1u);
        for (int x = 0; x < P; ++x) {
            const int64_t k = (int64_t)l * P + x;
            known[k] = (uint8_t)!lost;
            img[k] = lost ? 0 : data[k];
        }
        if (lost) unknown += P;
    }
    if (unknown == 0) return 0;

    for (int i = 0; i < r; ++i)
        for (int64_t j = 0; j < L->bins[i]; ++j) {
            w[L->off[i] + j] = (pmask >> i & 1u) ? 0 : parity[L->off[i] + j];
            cnt[L->off[i] + j] = 0;
            pid[L->off[i] + j] = (uint8_t)i;
        }
    for (int i = 0; i < r; ++i) {
        if (pmask >> i & 1u) continue;
        for (int l = 0; l < Q; ++l)
            for (int x = 0; x < P; ++x) {
                const int64_t t = L->off[i] + ((int64_t)l * p[i] - x - L->bmin[i]);
                if (known[(int64_t)l * P + x]) w[t] ^= img[(int64_t)l * P + x];
                else cnt[t] += 1;
            }
    }
    int64_t tail = 0;
    for (int i = 0; i < r; ++i) {
        if (pmask >> i & 1u) continue;
        for (int64_t j = 0; j < L->bins[i]; ++j)
            if (cnt[L->off[i] + j] == 1) queue[tail++] = L->off[i] + j;
    }
    int64_t found = peel(P, Q, p, r, L, pmask, img, w, cnt, known, queue, tail, pid, unknown);
    if (found < 0) return (int)found;
    return found == unknown ? 0 : -ENOTRECOVERABLE;
}

/* ---- public entry points (stripes loop, optional threads) ---------------- */

struct job {
    int P, Q, n;
    const int *p;
    const struct layout *L;
    const uint64_t *in;
    const uint64_t *data;   /* systematic decode: the data lines */
    uint64_t *out;
    const uint32_t *masks;
    int64_t nmasks;
    int64_t s0, s1;
    int decode;             /* 0 encode, 1 decode, 2 systematic decode */
    int status;
};

static void *run_job(void *arg)
{
    struct job *J = (struct job *)arg;
    const int64_t npix = (int64_t)J->P * J->Q;
    const int64_t total = J->L->total;
    J->status = 0;
    if (!J->decode) {
        for (int64_t s = J->s0; s < J->s1; ++s)
            encode_one(J->P, J->Q, J->p, J->n, J->L->off, J->L->bmin, total,
                       J->in + s * npix, J->out + s * total);
        return NULL;
    }
    uint64_t *w = (uint64_t *)malloc((size_t)total * sizeof(uint64_t));
    int32_t *cnt = (int32_t *)malloc((size_t)total * sizeof(int32_t));
    uint8_t *known = (uint8_t *)malloc((size_t)npix);
    int64_t *queue = (int64_t *)malloc((size_t)(2 * total + 1) * sizeof(int64_t));
    uint8_t *pid = (uint8_t *)malloc((size_t)total);
    if (!w || !cnt || !known || !queue || !pid) {
        J->status = -ENOMEM;
    } else {
        for (int64_t s = J->s0; s < J->s1; ++s) {
            uint32_t m = J->nmasks == 1 ? J->masks[0] : J->masks[s];
            int r;
            if (J->decode == 2) {
                r = sys_decode_one(J->P, J->Q, J->p, J->n, J->L, m,
                                   J->data + s * npix, J->in + s * total,
                                   J->out + s * npix, w, cnt, known, queue, pid);
            } else {
                if (!oracle_katz(J->P, J->Q, J->p, J->n, m)) {
                    J->status = -ENOTRECOVERABLE;
                    break;
                }
                r = decode_one(J->P, J->Q, J->p, J->n, J->L, m,
                               J->in + s * total, J->out + s * npix, w, cnt,
                               known, queue, pid);
            }
            if (r) { J->status = r; break; }
        }
    }
    free(w); free(cnt); free(known); free(queue); free(pid);
    return NULL;
}

static int run(int P, int Q, const int *p, int n, const uint64_t *in,
               const uint64_t *data, uint64_t *out, int64_t S,
               const uint32_t *masks, int64_t nmasks, int decode, int nthreads)
{
    int r = check_geometry(P, Q, p, n);
    if (r) return r;
    if (S < 0 || (S > 0 && (!in || !out))) return -EINVAL;
    if (decode == 2 && (Q + n > 32 || (S > 0 && !data))) return -EINVAL;
    if (decode && (!masks || (nmasks != 1 && nmasks != S))) return -EINVAL;
    if (S == 0) return 0;
    struct layout L;
    make_layout(P, Q, p, n, &L);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > S) nthreads = (int)S;
    struct job *jobs = (struct job *)calloc((size_t)nthreads, sizeof(struct job));
    pthread_t *tid = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tid) { free(jobs); free(tid); return -ENOMEM; }
    for (int t = 0; t < nthreads; ++t) {
        struct job *J = &jobs[t];
        J->P = P; J->Q = Q; J->n = n; J->p = p; J->L = &L;
        J->in = in; J->data = data; J->out = out;
        J->masks = masks; J->nmasks = nmasks;
        J->s0 = S * t / nthreads; J->s1 = S * (t + 1) / nthreads;
        J->decode = decode;
    }
    if (nthreads == 1) {
        run_job(&jobs[0]);
    } else {
        int started = 0;
        for (int t = 0; t < nthreads; ++t) {
            if (pthread_create(&tid[t], NULL, run_job, &jobs[t]) != 0) break;
            started++;
        }
        for (int t = started; t < nthreads; ++t) run_job(&jobs[t]);
        for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    }
    int status = 0;
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].status && !status) status = jobs[t].status;
    free(jobs); free(tid);
    return status;
}

/* Encode S stripes img[S][Q][P] into proj[S][total_bins]. */
int oracle_encode(int P, int Q, const int *p, int n, const uint64_t *img,
                  uint64_t *proj, int64_t S, int nthreads)
{
    return run(P, Q, p, n, img, NULL, proj, S, NULL, 0, 0, nthreads);
}

/* Decode S stripes proj[S][total_bins] into img[S][Q][P]. masks holds one
 * erasure mask (bit i set: projection i lost) for all stripes when
 * nmasks == 1, or one per stripe when nmasks == S. The bins of erased
 * projections are never read. */
int oracle_decode(int P, int Q, const int *p, int n, const uint64_t *proj,
                  uint64_t *img, int64_t S, const uint32_t *masks,
                  int64_t nmasks, int nthreads)
{
    return run(P, Q, p, n, proj, NULL, img, S, masks, nmasks, 1, nthreads);
}

/* Systematic decode (see sys_decode_one) of S stripes: data[S][Q][P] holds
 * the data lines (lost lines are never read), parity[S][total_bins] the r
 * parity projections p[0..r-1]; img[S][Q][P] receives the whole image.
 * Erasure mask bit l < Q: data line l lost; bit Q + i: projection i lost
 * (Q + r <= 32). One mask for all stripes (nmasks == 1) or one per stripe. */
int oracle_sys_decode(int P, int Q, const int *p, int r, const uint64_t *data,
                      const uint64_t *parity, uint64_t *img, int64_t S,
                      const uint32_t *masks, int64_t nmasks, int nthreads)
{
    return run(P, Q, p, r, parity, data, img, S, masks, nmasks, 2, nthreads);
}
