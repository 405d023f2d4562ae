/*
 * mojette.h -- C ABI of libmojette, a GB300 (sm_103a) implementation of the
 * Mojette erasure code over GF(2): the forward Mojette transform (encode)
 * and its inverse (decode).
 *
 * Notation (Pertin et al., "Performance evaluation of the Mojette erasure
 * code for fault-tolerant distributed hot data storage"):
 *   - A stripe is a P x Q image f(x, l) of 64-bit pixels: Q data lines (the
 *     code's k, Sec. 2.3) of P pixels each, stored row-major as
 *     img[l * P + x] (x the column, l the line). S stripes lie back to back.
 *   - Projection i has direction (p_i, 1) (q_i = 1, Sec. 2.3). Its bin at
 *     position b is the XOR of the pixels on the discrete line b = l p_i - x
 *     (Eq. 1 with XOR as the addition, Sec. 3). It has
 *     B_i = |p_i| (Q - 1) + P bins (Eq. 2), stored at j = b - b_min_i with
 *     b_min_i = -(P - 1) + min(0, (Q - 1) p_i).
 *   - A stripe's projections are concatenated in the order the directions
 *     were given: proj[s * total + off_i + j], off_i = sum_{i' < i} B_i',
 *     total = sum_i B_i. A storage node would hold one projection slice.
 *
 * Conventions for every call:
 *   - Return value: 0 on success or a negative errno:
 *       -EINVAL           bad geometry or argument (P, Q, n out of range,
 *                         duplicate directions, null pointer, S < 0);
 *       -ERANGE           a device pointer that is not 16-byte aligned;
 *       -ENOTRECOVERABLE  the surviving projections cannot rebuild the image;
 *       -ENOMEM           host or device allocation failed;
 *       -EIO              a CUDA runtime error (see mojette_last_cuda_error);
 *       -ETIMEDOUT        a bounded device-side wait expired (reported by
 *                         mojette_device_status);
 *       -ENOSPC           a schedule too large for mojette_decode_noalloc.
 *   - Device buffers (d_*) are owned by the caller, live in the current
 *     device's memory, and must not overlap each other. Work is enqueued on
 *     `stream` (a cudaStream_t; NULL = legacy default stream) and is
 *     asynchronous: the caller synchronises before reading results.
 *   - Plans are owned by the library from mojette_plan until
 *     mojette_plan_destroy. A plan may be used from several host threads at
 *     once; its schedule cache is internally locked. Per-device resources
 *     (reconstruction schedules) are created on first use on each device,
 *     with a blocking copy: make that first call outside any stream capture.
 */
#ifndef MOJETTE_H
#define MOJETTE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so this header needs no CUDA
 * header. */
typedef struct CUstream_st *mojette_stream_t;

/* Opaque plan: geometry, bin layout and the reconstruction-schedule cache. */
typedef struct mojette_plan_s *mojette_plan_t;

/* Largest number of projections a plan may hold (erasure masks are 32-bit). */
#define MOJETTE_MAX_PROJECTIONS 32
/* Largest Q the decoder accepts (one lane per data line, Sec. 2.2). */
#define MOJETTE_MAX_DECODE_LINES 16

/*
 * mojette_plan -- validate a geometry and compute its bin layout.
 * Defines: Sec. 2.1 (Eq. 1, Eq. 2) for the layout, Sec. 2.3 for q_i = 1.
 *   P, Q   image width (pixels per line, >= 1) and number of lines (>= 1);
 *   p[n]   the directions p_i of the n projections (1 <= n <= 32), distinct
 *          integers (p = 0 allowed); read, not retained;
 *   out    receives the plan.
 * Host only: touches no device. Errors: -EINVAL, -ENOMEM.
 */
int mojette_plan(int P, int Q, const int *p, int n, mojette_plan_t *out);

/* mojette_plan_ex flag: unused-bin removal. */
#define MOJETTE_PLAN_TRIM_UNUSED 1u
/* mojette_plan_ex flag: the systematic form of the code. */
#define MOJETTE_PLAN_SYSTEMATIC 2u

/*
 * mojette_plan_ex -- mojette_plan with options (flags 0: the same plan).
 * MOJETTE_PLAN_TRIM_UNUSED: store in each projection only the bins some
 * reconstruction path of this library reads, over every erasure mask that
 * leaves at least Q projections (Sec. 2.3 notes that some bins need not be
 * stored and gives no rule; the rule here is that one). A trimmed
 * projection holds those bins in increasing order (mojette_plan_bins gives
 * each stored word's bin in the full projection of Eq. 2);
 * mojette_plan_info reports the trimmed B_i, offsets and total. Encode
 * writes exactly the stored bins; decode reads only them, for every mask
 * with at least Q survivors. Building the plan builds the reconstruction
 * path of every such mask (host only; a fraction of a second at n = 12);
 * it requires n <= 20.
 * MOJETTE_PLAN_SYSTEMATIC: the systematic form of the code, which the paper
 * mentions (Sec. 2.3: "a systematic version ... is currently under
 * development"; Sec. 4: such a code decodes a 0-erasure read by a copy)
 * without defining it. Here the Q data lines are themselves Q of the
 * packets and the n projections p[0..n-1] are the parity packets, each the
 * projection of the whole image (Eq. 1, encoded by mojette_encode as
 * usual). Erasure masks of such a plan have Q + n bits: bit l < Q marks data
 * line l lost, bit Q + i marks projection i lost; any e lost data lines come
 * back from any e surviving projections (mojette_sys_decode). Requires
 * Q + n <= 32; cannot be combined with MOJETTE_PLAN_TRIM_UNUSED.
 * Errors: as mojette_plan, -EINVAL for unknown flags, n > 20 with
 * MOJETTE_PLAN_TRIM_UNUSED, or Q + n > 32 (or both flags) with
 * MOJETTE_PLAN_SYSTEMATIC.
 */
int mojette_plan_ex(int P, int Q, const int *p, int n, uint32_t flags,
                    mojette_plan_t *out);

/*
 * mojette_plan_bins -- for each stored word of a stripe's projection block
 * (full_bin[total], may be NULL), the index of its bin in its projection's
 * full layout (Eq. 2: j = b - b_min); the identity j = word - off_i for a
 * plan that is not trimmed. Returns 1 for a trimmed plan, 0 for a full one,
 * -EINVAL for NULL.
 */
int mojette_plan_bins(mojette_plan_t plan, int32_t *full_bin);

/*
 * mojette_plan_config -- read (get, may be NULL) and then install (set, may
 * be NULL) the launch configuration batches of this plan use, as
 * mojette_batch_tune leaves it (so a tuned configuration can be saved and
 * restored across processes). 8 words each:
 *   [0] 1: decode configuration set (tuned), 0: library defaults;
 *   [1] decode kernel (0 decode_lines, 1 decode_fronts, 2 decode_stream,
 *       3 decode_cols, 4 decode_scan2 -- the closed form for two rebuilt
 *       lines, the default for a systematic plan's two-line decodes,
 *       5 decode_vander, 6 decode_ilv; Q > 8 allows 1 only, 4 needs Q = 2
 *       or a systematic plan and applies only to two-line decodes, 5 and 6
 *       need a plan that is not systematic, 5 one that is not trimmed);
 *   [2] work items per CTA (1 .. 64); [3] persistent grid (0/1);
 *   [4] decode_lines row phases (0/1);
 *   [5] 1: encode configuration set; [6] encode tile bytes (0: by Q);
 *   [7] reserved, 0.
 * Batches built after the call use it. Errors: -EINVAL (NULL plan, a value
 * out of range).
 */
int mojette_plan_config(mojette_plan_t plan, int32_t *get, const int32_t *set);

/* Release a plan and every host and device resource it holds. Must not be
 * called while work that uses the plan is still in flight. NULL is a no-op. */
int mojette_plan_destroy(mojette_plan_t plan);

/*
 * mojette_plan_info -- the bin layout (Eq. 2).
 *   bins[n], offsets[n]  receive B_i and off_i (either may be NULL);
 *   total                receives sum_i B_i, the words per encoded stripe
 *                        (may be NULL).
 */
int mojette_plan_info(mojette_plan_t plan, int64_t *bins, int64_t *offsets,
                      int64_t *total);

/*
 * mojette_encode -- forward Mojette transform of S stripes (Sec. 2.1, Eq. 1;
 * XOR addition, Sec. 3).
 *   d_img   [S][Q][P] uint64 pixels, read;
 *   d_proj  [S][total] uint64 bins, written (every bin, empty ones as 0);
 *   S       number of stripes (0 is a no-op).
 * Both pointers must be 16-byte aligned. Errors: -EINVAL, -ERANGE, -EIO.
 */
int mojette_encode(mojette_plan_t plan, const uint64_t *d_img, uint64_t *d_proj,
                   int64_t S, mojette_stream_t stream);

/*
 * mojette_decode -- inverse Mojette transform of S stripes that all lost the
 * same projections (Sec. 2.2; Sec. 2.3 for "any Q of the n projections").
 *   d_proj        [S][total] uint64 bins, read; the slices of erased
 *                 projections are never read (their contents do not matter);
 *   erasure_mask  bit i set: projection i is lost;
 *   d_img         [S][Q][P] uint64 pixels, written.
 * At least Q projections must survive, and Q <= MOJETTE_MAX_DECODE_LINES;
 * otherwise -ENOTRECOVERABLE (resp. -EINVAL). A stripe is rebuilt in shared
 * memory: its Q * P words plus zero columns must fit in one CTA's (about
 * 28000 words, e.g. 16 KB-wide lines at Q = 4); larger stripes get -EINVAL
 * before any launch (cut objects into smaller stripes). The reconstruction path for
 * the surviving set is computed on the host on first use and cached in the
 * plan (the paper's pre-determined path, Sec. 2.2 and Sec. 3.1). A
 * systematic plan decodes with mojette_sys_decode instead (-EINVAL here).
 * Errors: -EINVAL, -ERANGE, -ENOTRECOVERABLE, -ENOMEM, -EIO.
 */
int mojette_decode(mojette_plan_t plan, const uint64_t *d_proj,
                   uint32_t erasure_mask, uint64_t *d_img, int64_t S,
                   mojette_stream_t stream);

/*
 * mojette_stage_survivors -- copy to the device, from host memory, exactly
 * the projections a decode under `erasure_mask` reads: the Q surviving
 * projections its reconstruction path uses (any Q of the n rebuild the
 * block, Sec. 2.3; a storage read fetches only those packets), for S
 * stripes.
 *   h_proj  [S][total] uint64 bins in host memory, read (pinned memory for
 *           an asynchronous copy; pageable memory makes it synchronous);
 *           only the used projections' slices [off_i, off_i + B_i) are read;
 *   d_proj  [S][total] uint64 on the device: those slices written, every
 *           other word untouched (a following mojette_decode with the same
 *           mask reads nothing else);
 *   bytes   receives the number of bytes copied (may be NULL).
 * One strided 2-D copy (cudaMemcpy2DAsync, rows = stripes, pitch total * 8
 * bytes) per used projection, on `stream`; host only otherwise (the mask's
 * path is built and cached as for a decode). Not for systematic plans.
 * Errors: -EINVAL (NULL pointer, systematic plan, mask bits beyond n),
 * -ENOTRECOVERABLE, -ENOMEM, -EIO.
 */
int mojette_stage_survivors(mojette_plan_t plan, const uint64_t *h_proj,
                            uint32_t erasure_mask, uint64_t *d_proj, int64_t S,
                            mojette_stream_t stream, int64_t *bytes);

/*
 * mojette_sys_decode -- rebuild, in place, the lost data lines of S stripes
 * of a systematic plan (MOJETTE_PLAN_SYSTEMATIC) that all lost the same
 * packets. The paper leaves the systematic form undefined (Sec. 2.3,
 * Sec. 4); the decode here removes (XOR) the known lines' pixels from the
 * surviving projections' bins -- Eq. 1's sum split into known and lost
 * pixels -- and runs the inverse of Sec. 2.2 on the lost lines only, one
 * surviving projection dedicated to each.
 *   d_parity      [S][total] uint64 bins of the n parity projections, read;
 *                 the slices of lost projections are never read;
 *   erasure_mask  bit l < Q: data line l lost; bit Q + i: projection i lost;
 *   d_data        [S][Q][P] uint64 pixels: the surviving data lines are
 *                 read, the lost ones (any contents) are overwritten with
 *                 their values; no other word is written.
 * With no data line lost nothing is launched (the data is already whole:
 * the copy Sec. 4 expects of a systematic code). At most 8 data lines may
 * be lost per call (-EINVAL beyond), and at least as many projections must
 * survive as lines are lost, else -ENOTRECOVERABLE. The lost lines' bins
 * plus zero columns must fit in one CTA's shared memory (as for
 * mojette_decode), else -EINVAL. The path for the mask is computed on the
 * host on first use and cached in the plan.
 * Errors: -EINVAL (not a systematic plan, mask bits beyond Q + n, ...),
 * -ERANGE, -ENOTRECOVERABLE, -ENOMEM, -EIO.
 */
int mojette_sys_decode(mojette_plan_t plan, const uint64_t *d_parity,
                       uint32_t erasure_mask, uint64_t *d_data, int64_t S,
                       mojette_stream_t stream);

/*
 * mojette_decode_noalloc -- mojette_decode for callers that must not allocate
 * device memory. The paper has no counterpart: this is a library concern.
 * Some callers cannot call cudaMalloc: a storage server that hands all of its
 * device memory to its own buffer pool at start-up, or a request path that
 * must not take the device-wide synchronisation cudaMalloc may cause. This
 * call allocates nothing on the device (no cudaMalloc, cudaFree or
 * allocating library routine). The reconstruction path's step words go to a
 * fixed scratch array inside the library, 2 * 16384 words (128 KiB), that
 * every GPU loading the library holds until the process exits; schedules of
 * more than 16384 steps are refused with -ENOSPC. The caller still passes the
 * inputs and outputs, as for mojette_decode.
 * Systematic plans are refused (-EINVAL).
 * Every call shares that scratch and overwrites it (on `stream`, before the
 * kernel): calls that can overlap on the GPU -- on different streams without
 * ordering between them -- race and may decode with another call's path.
 * Order such calls on one stream, or use mojette_decode. The first call on a
 * device looks up the scratch's device address (cudaGetSymbolAddress), a
 * set-up step; make that first call outside any stream capture.
 * Errors: as mojette_decode, plus -ENOSPC.
 */
int mojette_decode_noalloc(mojette_plan_t plan, const uint64_t *d_proj,
                           uint32_t erasure_mask, uint64_t *d_img, int64_t S,
                           mojette_stream_t stream);

/*
 * mojette_decode_kernel -- which decode kernel mojette_decode (or, for a
 * systematic plan, mojette_sys_decode) launches for this mask and S stripes
 * (host only; builds and caches the mask's path like the decode would):
 *   0 decode_lines   the two-front path of Sec. 2.2, one lane per line and
 *                    front, a few stripes per warp (Q <= 8);
 *   1 decode_fronts  the same path, one lane per front (any Q);
 *   2 decode_stream, 3 decode_cols  variants of 0 (tuning candidates);
 *   4 decode_scan2   two rebuilt lines in closed form (a chain recurrence);
 *   5 decode_vander  every line at once: Eq. 1 as a Vandermonde system
 *                    solved by divided differences (non-systematic,
 *                    untrimmed plans; exact, but not the paper's inverse);
 *   6 decode_ilv     the path of Sec. 2.2 with the stripes across the lanes
 *                    (one lane per stripe, front and half of the lines;
 *                    non-systematic, Q <= 8);
 *   7 decode_ring    the path of Sec. 2.2 swept from the left end only, each
 *                    (stripe, line) held as a ring of 64 or 128 words
 *                    (non-systematic, untrimmed, Q <= 8, where the host's
 *                    replay of the path shows it fits a ring);
 *  -1                no launch (a systematic mask with no data line lost).
 * The default is the paper's inverse: decode_lines up to 8 lines,
 * decode_fronts beyond, and for a systematic plan decode_lines over the lost
 * lines or decode_scan2 for two of them. The MOJETTE_DECODE_KERNEL
 * environment variable may name another kernel (lines, ilv, ring, fronts,
 * stream, cols, scan, vander) where it applies; a stripe too wide for the chosen
 * kernel's shared memory falls back to decode_lines, then decode_fronts, at
 * launch. Errors: -EINVAL, -ENOTRECOVERABLE, -ENOMEM.
 */
int mojette_decode_kernel(mojette_plan_t plan, uint32_t erasure_mask, int64_t S,
                          int32_t *kernel);

/*
 * mojette_schedule -- the cached reconstruction path for one erasure mask,
 * copied out for inspection (host only, touches no device).
 *   survivors[Q]  receives the projection index dedicated to the left-to-
 *                 right front of each line l (ascending p), then
 *   survivors2[Q] the index dedicated to its right-to-left front;
 *   split[Q]      pixel x of line l comes from the left front iff x < split[l];
 *   steps         receives up to max_steps step words; bit 2l of word t set:
 *                 line l's left front rebuilds its next pixel at step t,
 *                 bit 2l+1: its right front does; for Q <= 15, bit 31 marks
 *                 a steady step (every front moves, and every line's operand
 *                 on line l+1 comes from the same step exactly where the
 *                 schedule's steady pattern says so);
 *   forward       receives up to max_steps words; bit 2l+side of word t set:
 *                 at step t, line l of that front (0 left, 1 right) takes
 *                 the pixel of its bin line on line l+1 from the pixel line
 *                 l+1 of the same front rebuilds in the same step (fronts
 *                 visit their lines from Q-1 down to 0 within a step);
 *   n_steps       receives the number of steps.
 * For a systematic plan the path rebuilds only the lost data lines: the
 * arrays get one entry per lost line, in increasing line order, line l of
 * the step and forward words being the l-th lost line (no entry and no
 * step when no line is lost; no step when one is).
 * Any output pointer may be NULL. Errors: -EINVAL, -ENOTRECOVERABLE, -ENOMEM.
 */
int mojette_schedule(mojette_plan_t plan, uint32_t erasure_mask,
                     int32_t *survivors, int32_t *survivors2, int32_t *split,
                     uint32_t *steps, uint32_t *forward, int64_t max_steps,
                     int64_t *n_steps);

/*
 * mojette_schedule_layout -- the shared-memory layout decode_lines uses for
 * the cached reconstruction path of one erasure mask in launches of 4096 or
 * more stripes, copied out for inspection (host only, touches no device; the
 * first call for a mask runs the search, tens of milliseconds at Q = 8, and
 * the result is kept with the path). The paper has no counterpart: this is
 * a GPU bank layout, not part of the inverse transform (Sec. 2.2), whose
 * result it does not change.
 *   row_phase[lines]   receives, per rebuilt line, the residue mod S of its
 *                      row's first shared-memory word (S = 16 / G bank-slot
 *                      classes, G = 32 / (2 Q) stripes per warp; where no
 *                      bank model applies, Q = 3, 5 or Q > 8, only a parity);
 *                      its parity lets bulk copies stage the row's bins;
 *   load_order[2*lines] receives, per front (index 2l + side, side 0: left
 *                      to right), its load order: nibble k = the word load
 *                      instruction k reads, 0 the front's own bin, j >= 1
 *                      the pixel on line l + j mod Q (nibble 0 is 0).
 * `lines` is Q (a systematic plan: the lost data lines, as mojette_schedule
 * counts them). Either pointer may be NULL. Errors: -EINVAL,
 * -ENOTRECOVERABLE, -ENOMEM.
 */
int mojette_schedule_layout(mojette_plan_t plan, uint32_t erasure_mask, int32_t *row_phase,
                            uint32_t *load_order);

/* ------------------------------------------------------------------------
 * Batches: many stripes of mixed geometry, operation (encode or decode) and
 * erasure pattern in one submission. The paper codes one block at a time
 * (Sec. 4); batching is a library concern with no counterpart there. Each
 * stripe's result is bit-identical to what mojette_encode / mojette_decode
 * give for it alone.
 * ------------------------------------------------------------------------ */

#define MOJETTE_OP_ENCODE 0
#define MOJETTE_OP_DECODE 1

/* One stripe of a batch. */
typedef struct mojette_stripe {
    mojette_plan_t plan;     /* its geometry; must outlive the batch */
    int32_t op;              /* MOJETTE_OP_ENCODE or MOJETTE_OP_DECODE */
    uint32_t erasure_mask;   /* decode: bit i set = projection i lost; else 0 */
    const uint64_t *src;     /* device, 8-byte aligned (16-byte for an
                                encode with P even): encode reads the
                                [Q][P] pixels, decode the [total] bins */
    uint64_t *dst;           /* device, 8-byte aligned: encode writes the
                                [total] bins, decode the [Q][P] pixels */
} mojette_stripe_t;
/* A decode stripe of a systematic plan is mojette_sys_decode's: src the
 * parity bins, dst the data lines, rebuilt in place; the mask has Q + n
 * bits. Such stripes with no data line lost launch nothing. */

/* Opaque batch: the stripes' device tables, side streams, an optional CUDA
 * graph. Not thread-safe: one host thread at a time per batch. */
typedef struct mojette_batch_s *mojette_batch_t;

/* mojette_batch_create flag: mojette_batch_run launches one CUDA graph
 * (captured on the first run after the stripes change) instead of one kernel
 * launch per (operation, plan). */
#define MOJETTE_BATCH_GRAPH 1u

/*
 * mojette_batch_create -- build a batch over count stripes (count >= 0).
 * Stripes are grouped by (operation, plan) -- one kernel launch each -- and,
 * for decode, by erasure mask -- one reconstruction path each (Sec. 2.2),
 * computed and cached in the plan as by mojette_decode. Builds the device
 * tables (per-stripe addresses, paths, work items: about 16 bytes per stripe
 * plus about 380 bytes per (plan, mask)) and uploads them; blocking. The stripes
 * array is read, not retained. Buffers must not overlap between stripes
 * whose writes could collide.
 * Errors: -EINVAL (null plan or pointer, bad op, mask bits beyond n, decode
 * with Q > MOJETTE_MAX_DECODE_LINES, unknown flag), -ERANGE (unaligned
 * pointer), -ENOTRECOVERABLE (a mask leaves fewer than Q projections),
 * -ENOMEM, -EIO.
 */
int mojette_batch_create(const mojette_stripe_t *stripes, int64_t count,
                         uint32_t flags, mojette_batch_t *out);

/*
 * mojette_batch_update -- replace the stripes of a batch (same rules as
 * mojette_batch_create). The tables are uploaded asynchronously on `stream`;
 * later runs on any stream wait for that upload. Waits on the host for the
 * previous update's upload to leave the pinned staging buffer. When the new
 * tables do not fit the workspace it is reallocated, which synchronises the
 * device. A batch must not be updated while one of its runs enqueued on
 * another stream can still be executing.
 */
int mojette_batch_update(mojette_batch_t batch, const mojette_stripe_t *stripes,
                         int64_t count, mojette_stream_t stream);

/*
 * mojette_batch_run -- enqueue every stripe of the batch on `stream`. The
 * launches of the different (operation, plan) classes run concurrently on
 * side streams (or graph branches) forked from and joined back into
 * `stream`. Within a batch, stripes are independent: a decode reads its
 * bins as they are when the run starts on the device.
 * Errors: -EINVAL, -EIO.
 */
int mojette_batch_run(mojette_batch_t batch, mojette_stream_t stream);

/*
 * mojette_batch_tune -- autotune the launch configuration of every class of
 * the batch: for decode the kernel (decode_lines, one lane per line and
 * front; decode_cols, the same lanes over a line-interleaved layout;
 * decode_stream, the same lanes with the stripe streamed through shared
 * memory in chunks; decode_ilv, one lane per stripe, front and half of the
 * lines; decode_fronts, one lane per front; decode_scan2 and decode_vander
 * where they apply), stripes per
 * CTA, persistent or one-shot grids and whether each line's row starts at
 * the bank phase chosen for the path; for encode the stripes per
 * shared-memory tile. Each
 * candidate runs 1 + reps times on `stream` (so the batch's outputs are
 * written, with their correct values) and is timed with CUDA events; the
 * fastest is kept in the batch and in the plan, where later batches of the
 * plan start from it. Synchronises `stream`. Errors: -EINVAL, -EIO.
 */
int mojette_batch_tune(mojette_batch_t batch, mojette_stream_t stream, int reps);

/*
 * mojette_batch_info -- the batch's shape (any pointer may be NULL):
 *   launches    kernel launches per run (one per (operation, plan), and
 *               for a systematic plan's decodes one per count of lost data
 *               lines, none for those that lost none);
 *   groups      (plan, mask) groups of the decode stripes;
 *   work_items  decode work items (one warp's stripes each);
 *   configs     6 words per launch: op, Q (decode: lines rebuilt per
 *               stripe, a systematic launch's lost lines), P, then for decode the kernel
 *               (0 decode_lines, 1 decode_fronts, 2 decode_stream,
 *               3 decode_cols, 4 decode_scan2, 5 decode_vander,
 *               6 decode_ilv), work
 *               items per CTA and
 *               flags (bit 0 persistent grid, bit 1 bank-phased rows),
 *               for encode 0, the tile bytes (0 = default) and 0. The array
 *               holds 6 * launches words.
 */
int mojette_batch_info(mojette_batch_t batch, int64_t *launches, int64_t *groups,
                       int64_t *work_items, int32_t *configs);

/* Release a batch (synchronises the device first). NULL is a no-op. */
int mojette_batch_destroy(mojette_batch_t batch);

/* ------------------------------------------------------------------------
 * Request server: continuous batching of object writes (encode) and reads
 * (decode) under a device-memory budget. Like batches, a library concern
 * with no counterpart in the paper. Each request's result is bit-identical
 * to mojette_encode / mojette_decode of its stripes alone.
 * ------------------------------------------------------------------------ */

/* One object write or read: `stripes` whole stripes of one plan. */
typedef struct mojette_request {
    uint64_t id;             /* caller's tag, returned in the completion */
    mojette_plan_t plan;     /* must outlive the server */
    int32_t op;              /* MOJETTE_OP_ENCODE (write) or _DECODE (read) */
    uint32_t erasure_mask;   /* read: projections lost; write: ignored */
    int64_t stripes;         /* >= 1 */
    const void *host_src;    /* pinned host memory: write [stripes][Q][P]
                                pixels, read [stripes][total] bins */
    void *host_dst;          /* pinned host memory: write [stripes][total]
                                bins, read [stripes][Q][P] pixels */
    double arrival_s;        /* arrival time on the server clock
                                (mojette_server_now); <= 0: at submission */
} mojette_request_t;

typedef struct mojette_completion {
    uint64_t id;
    int32_t status;          /* 0, or a negative errno for the request */
    double arrival_s;        /* as submitted (or the submission time) */
    double admit_s;          /* admitted into a wave: device memory reserved */
    double done_s;           /* its wave's event seen complete (output in
                                host_dst) */
} mojette_completion_t;

typedef struct mojette_server_s *mojette_server_t;

/*
 * mojette_server_create -- a server on the current device.
 *   device_budget_bytes  the device buffer pool, allocated here once (the
 *                        admission budget: a request holds its input stripes
 *                        in one half and its output stripes in the other
 *                        while it is in flight);
 *   slots                waves in flight at once (1..64), each with its own
 *                        stream and batch;
 *   max_wave_stripes     stripes per wave at most (bounds a wave's latency);
 *                        a larger request is refused at submission.
 * Errors: -EINVAL, -ENOMEM, -EIO.
 */
int mojette_server_create(int64_t device_budget_bytes, int slots,
                          int64_t max_wave_stripes, mojette_server_t *out);

/*
 * mojette_server_submit -- queue n requests (first come, first served) and
 * make progress. Never waits for the device. The request array is copied;
 * the host buffers must stay valid (and host_dst unread) until the request
 * completes. Admission: a wave takes queued requests in order while their
 * buffers fit the pool; a request that does not fit waits (later requests
 * wait behind it). A wave's requests whose host buffers follow each other
 * exactly (and whose device buffers do too) are copied in one transfer.
 * Errors (nothing is queued): -EINVAL (also a read of a systematic plan:
 * its decode takes data and parity in place, see mojette_sys_decode and
 * the batch calls), -ENOTRECOVERABLE (a read's mask
 * leaves fewer than Q projections), -ENOSPC (a request whose input or
 * output exceeds half the budget, or larger than max_wave_stripes), or an
 * error of a wave launched meanwhile (see mojette_server_poll).
 */
int mojette_server_submit(mojette_server_t server, const mojette_request_t *reqs,
                          int64_t n);

/*
 * mojette_server_poll -- make progress (retire finished waves, admit and
 * launch new ones into free slots) and return up to `max` completions in
 * completion order. A wave that fails completes its requests with the
 * error status, and the call returns that error too.
 */
int mojette_server_poll(mojette_server_t server, mojette_completion_t *out,
                        int64_t max, int64_t *n_out);

/* Seconds on the server's clock (steady, zero at creation). */
int mojette_server_now(mojette_server_t server, double *seconds);

/* Counters: requests queued and in flight, waves launched, requests
 * completed, pool bytes in use and the peak. Any pointer may be NULL. */
int mojette_server_stats(mojette_server_t server, int64_t *queued,
                         int64_t *in_flight, int64_t *waves, int64_t *completed,
                         int64_t *pool_used, int64_t *pool_peak);

/* Wait for the waves in flight, then release the server. NULL is a no-op. */
int mojette_server_destroy(mojette_server_t server);

/*
 * mojette_device_status -- synchronise the current device and return the
 * sticky status word the kernels set (0 = clean; bit 0: a bounded wait for
 * an asynchronous copy expired, so some outputs were not written).
 *   flags  receives the word (may be NULL);
 *   clear  nonzero: reset the word to 0 afterwards.
 * Returns 0, -ETIMEDOUT if bit 0 was set, or -EIO.
 */
int mojette_device_status(uint32_t *flags, int clear);

/*
 * mojette_selftest_wait -- failure-detection self-test (no counterpart in
 * the paper): enqueue on `stream` one warp that waits, through the bounded
 * mbarrier wait the encoder uses for its copies, for bytes that are never
 * sent. After limit_ns (1 us .. 1 s) the wait gives up, the kernel sets
 * status bit 0 and returns: a following mojette_device_status returns
 * -ETIMEDOUT, and the device stays usable. Errors: -EINVAL, -EIO.
 */
int mojette_selftest_wait(int64_t limit_ns, mojette_stream_t stream);

/* Text for a status code returned by any call above. */
const char *mojette_strerror(int status);

/* The last CUDA runtime error code seen by this library on this host thread
 * (a cudaError_t value; 0 = none). */
int mojette_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MOJETTE_H */
