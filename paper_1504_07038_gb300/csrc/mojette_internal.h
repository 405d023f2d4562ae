// Internal declarations of libmojette (host plan/schedule code and kernels).
#pragma once

#include <array>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mojette.h"

namespace mojette {

constexpr int kMaxProj = MOJETTE_MAX_PROJECTIONS;
constexpr int kMaxLines = MOJETTE_MAX_DECODE_LINES;

// Status bits the kernels OR into the device status word.
constexpr uint32_t kStatusWaitTimeout = 1u;

// Step word bit 31 marks a steady step: every front moves and the operand
// pattern is the schedule's `fwd` (see plan.cpp). Lines use bits 0..2Q-1, so
// the mark exists for Q <= 15.
constexpr uint32_t kStepSteady = 1u << 31;
constexpr int kFastMaxLines = 15;

// Forward word bit 31 marks a step at which some front reads a pixel the
// other front (the other side of the same line set) rebuilt at an earlier
// step since the last such mark: kernels that run the two sides in different
// warps synchronise them there. Line Q - 1 never forwards, so the bit is free
// for Q <= 16.
constexpr uint32_t kFwdSync = 1u << 31;

// Most lost data lines a systematic decode rebuilds in one stripe (one lane
// pair per lost line in decode_lines).
constexpr int kSysMaxLines = 8;

// decode_scan2: warps (one stripe each) per CTA.
constexpr int kScanWarps = 4;
// decode_vander: warps (one stripe each) per CTA.
constexpr int kVanWarps = 4;

// decode_stream stages and writes a stripe in this many chunks of columns,
// by distance from the nearer end of each line's front.
constexpr int kStreamChunks = 4;

// A bounded device-side wait gives up after this many nanoseconds.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Reconstruction path for one (geometry, erasure mask): Sec. 2.2's
// pre-determined path with one projection dedicated to each line, run from
// both ends of every line (a left-to-right and a right-to-left front).
// Load order of a front that reads its words as numbered: own bin, then the
// pixels on lines l + 1, l + 2, ... (mod Q).
constexpr uint32_t kIdentityOrder = 0x76543210u;
constexpr std::array<uint32_t, 2 * kMaxLines> identity_orders()
{
    std::array<uint32_t, 2 * kMaxLines> o{};
    for (auto &v : o) v = kIdentityOrder;
    return o;
}

struct Schedule {
    uint32_t mask = 0;
    int T = 0;                       // number of steps
    // Lines the path rebuilds: every line (lines = Q, lpos[l] = l), or for a
    // systematic plan the lost data lines (image rows lpos[0] < lpos[1] <
    // ...; line indices below count these), the rows in `known` being read
    // from the data instead. lines = 0: nothing to rebuild.
    int lines = 0;
    int32_t lpos[kMaxLines] = {};
    uint32_t known = 0;
    uint32_t fwd = 0;                // operand pattern of the steady steps
    int32_t projL[kMaxLines] = {};   // projection rebuilding line l left of split
    int32_t projR[kMaxLines] = {};   // ... and from split rightwards
    int32_t pL[kMaxLines] = {};      // their directions
    int32_t pR[kMaxLines] = {};
    int32_t split[kMaxLines] = {};   // x < split[l]: left front
    int64_t srcL[kMaxLines] = {};    // bin of pixel (l, x) sits at word srcL[l] - x
    int64_t srcR[kMaxLines] = {};    //   of the stripe's projection block
    std::vector<uint32_t> steps;     // T words, 2 bits per line
    std::vector<uint32_t> fwdw;      // T words: bit 2l+side set when line l of that
                                     // front uses line l+1's pixel of the same step
    // Chunks of a stripe for streamed staging and output: pixel (l, x) is in
    // chunk min(d / chunk_w, kStreamChunks - 1), d its distance from the end
    // its front starts at (x left of split[l], else P - 1 - x). Chunk c must
    // be staged before step chunk_wait[c] (non-decreasing, [0] = 0) and is
    // final after step chunk_done[c] (non-decreasing).
    int32_t chunk_w = 1;
    int32_t chunk_wait[kStreamChunks] = {};
    int32_t chunk_done[kStreamChunks] = {};
    // decode_lines: column offset of each line's row in shared memory (mod
    // the bank slots of its stripe groups), chosen so that the lanes of a
    // warp read different banks at the steps of this path (plan.cpp).
    int32_t rowoff[kMaxLines] = {};
    int32_t rowpar[kMaxLines] = {};  // decode_lines: row phase parity for bulk staging
    // decode_lines: load order of each front (index 2l + side), nibble k =
    // the word its load instruction k reads (0: own bin, j >= 1: the pixel
    // on line l + j mod Q); chosen with the row phases (plan.cpp).
    std::array<uint32_t, 2 * kMaxLines> order = identity_orders();
    bool phases_done = false;
    // Two lines rebuilt (lines == 2): the closed form decode_scan2 solves,
    // with projection scan_proj[0] (direction scan_p[0]) dedicated to line 0
    // and scan_proj[1] (scan_p[1] > scan_p[0]) to line 1 over the whole
    // line; the bin of pixel x of line j is stored word scan_src[j] - x.
    bool scan2 = false;
    int32_t scan_proj[2] = {};
    int32_t scan_p[2] = {};
    int64_t scan_src[2] = {};
    // decode_vander (every line at once, the Vandermonde form of Eq. 1): Q
    // survivors with ascending directions van_q, projection van_proj[j];
    // the bin at position b of projection j is stored word van_base[j] + b
    // for b in [van_lo[j], van_hi[j]); the solve runs over positions
    // [van_E0, van_E0 + van_L).
    bool vander = false;
    int32_t van_proj[kMaxLines] = {};
    int32_t van_q[kMaxLines] = {};
    int64_t van_base[kMaxLines] = {};
    int32_t van_lo[kMaxLines] = {};
    int32_t van_hi[kMaxLines] = {};
    int32_t van_E0 = 0, van_L = 0;
    // decode_ring: a one-sided path (left-to-right fronts only, split = P)
    // replayed with a ring of ring_R words per (stripe, line) in shared
    // memory, chunks of kRingChunk columns fetched ring_D chunks ahead of
    // each line's front; line l's chunks start at columns 16k - ring_delta[l]
    // (16-byte aligned sources). ring_R = 0: the path does not fit a ring.
    bool one_sided = false;
    int32_t ring_R = 0, ring_D = 0;
    int32_t ring_delta[kMaxLines] = {};
    // decode_ring events per step: bit l, line l's front enters a chunk
    // (fetch chunk k + D, wait for chunk k); bit 8 + l, it completes the
    // 16-column chunk its pixel ends (written back after the step). On the
    // device the schedule then also holds (step, forward, event, 0) words
    // per step, 16-byte aligned, after the step and forward words.
    std::vector<uint32_t> ringev;
    std::map<int, uint32_t *> dev;   // device copy of `steps` then `fwdw`, per device
};

// decode_ring chunk width in columns (one 128-byte bulk copy).
constexpr int kRingChunk = 16;

// Launch configuration of the decode kernels (chosen by the autotuner for a
// batch, else the defaults here).
struct DecodeConfig {
    int kernel = 0;    // 0: decode_lines, 1: decode_fronts, 2: decode_stream, 3: decode_cols
                       // (all but decode_fronts for Q <= 8 only), 4: decode_scan2
                       // (two lines rebuilt only; the default there), 5: decode_vander
                       // (non-systematic, untrimmed, 2 <= Q <= 8), 6: decode_ilv
                       // (non-systematic, Q <= 8), 7: decode_ring (non-systematic,
                       // untrimmed, Q <= 8, a one-sided path that fits a ring)
    int gpc = 4;       // work items (groups of G stripes) per CTA
    int gmax = 0;      // decode_ilv: most stripes per work item (0: up to 16)
    int ring_R = 0;    // decode_ring: ring words per (stripe, line), from the path
    int ring_D = 0;    //   and chunks fetched ahead
    int persist = 0;   // 1: grid capped at the resident CTAs, grid-stride over items
    int rowoff = 1;    // decode_lines: 1 to start each line's row at the path's
                       // bank phase (Schedule::rowoff), 0 at a uniform pitch
};

// Launch configuration of the encode kernel.
struct EncodeConfig {
    int tile_bytes = 0;   // target bytes of a tile of stripes; 0: by Q
};

struct Plan {
    int P = 0, Q = 0, n = 0;
    // Systematic form: the Q data lines are packets themselves and the n
    // projections are parity packets; erasure mask bit l < Q marks data
    // line l lost, bit Q + i projection i.
    bool systematic = false;
    int32_t p[kMaxProj] = {};
    int64_t B[kMaxProj] = {};
    int64_t off[kMaxProj] = {};
    int64_t bmin[kMaxProj] = {};   // Eq. 2's b_min: bin j of the full projection is b = j + b_min
    int64_t total = 0;             // stored words per stripe
    // Unused-bin removal: a trimmed plan stores, for projection i, only the
    // bins some reconstruction path reads, in order: stored word off_i + s
    // holds full bin full_bin[off_i + s]; stored_of[fulloff_i + j] is the
    // stored index s of full bin j (-1: not stored). Untrimmed: identity.
    bool trimmed = false;
    std::vector<int32_t> full_bin;     // total entries
    std::vector<int32_t> stored_of;    // sum of the full B_i entries
    int64_t fulloff[kMaxProj] = {};
    std::map<int, int32_t *> full_bin_dev;   // device copy of full_bin, per device
    std::mutex mu;
    std::map<uint32_t, std::unique_ptr<Schedule>> schedules;
    std::map<uint32_t, std::unique_ptr<Schedule>> ring_schedules;   // one-sided paths (decode_ring)
    // autotuned configurations (batch.cpp); used by batches of this plan
    bool tuned_dec = false, tuned_enc = false;
    DecodeConfig dec_cfg;
    EncodeConfig enc_cfg;
};

// Decode kernel a launch of S stripes uses by default (DecodeConfig::kernel
// numbering), before the shared-memory fit check: the measured-fastest
// kernel that applies (decode_vander for Q <= 3, Q = 4 with P >= 192, and
// Q = 4 or 5 in launches of at most kVanSmallLaunch stripes, where its
// shorter per-stripe latency wins; decode_scan2 for other two-line decodes;
// decode_lines up to 8 lines; decode_fronts beyond). `env`:
// MOJETTE_DECODE_KERNEL may name another kernel that applies.
constexpr int64_t kVanSmallLaunch = 4096;
int choose_decode_kernel(int P, int Q, int64_t S, bool sys, bool scan2, bool vander, bool env);

// ---- host helpers (plan.cpp) ---------------------------------------------
int build_schedule(const Plan &pl, uint32_t mask, Schedule *out);
// Returns the cached schedule (building it on a miss) or sets *err.
Schedule *get_schedule(Plan &pl, uint32_t mask, int *err);
// The one-sided path of a mask for decode_ring (cached; ring_R = 0 when no
// ring fits), or null with *err set (-EINVAL for systematic or trimmed plans).
Schedule *get_ring_schedule(Plan &pl, uint32_t mask, int *err);
// Unused-bin removal: keep in each projection only the bins some
// reconstruction path reads, over every recoverable erasure mask.
int trim_unused_bins(Plan &pl);
// Device copy of a trimmed plan's stored-word -> full-bin map (null, 0 for a
// plan that is not trimmed).
int plan_full_bin_on_device(Plan &pl, const int32_t **dev);
// decode_lines row phases of a schedule (computed on first use, cached; the
// search takes milliseconds, so launches of fewer than kPhaseMinStripes
// stripes use uniform rows instead, rowoff all zero).
const int32_t *schedule_row_phases(Plan &pl, Schedule &sc);
constexpr int64_t kPhaseMinStripes = 4096;
// Device copy of a schedule's step words on the current device.
int schedule_on_device(Plan &pl, Schedule &sc, uint32_t **dev);
int record_cuda(cudaError_t e);     // remembers e; returns 0 or -EIO
uint32_t *device_status_ptr(int *err);  // per-device status word

// ---- kernel launchers -------------------------------------------------------
struct EncodeArgs {
    const int32_t *full_bin;        // trimmed plan: full bin of each stored word (device), else null
    const uint64_t *img;            // plain: stripe s at img + s * Q * P
    uint64_t *proj;                 // plain: stripe s at proj + s * total
    const uint64_t *const *srcp;    // batched: stripe s at srcp[s] (device array)
    uint64_t *const *dstp;          //   and its bins at dstp[s]
    int tile_bytes;                 // 0: by Q
    int64_t S;
    int64_t total;
    int P, Q, n;
    int32_t p[kMaxProj];
    int64_t off[kMaxProj];
    int64_t bmin[kMaxProj];
    uint32_t *status;
};
int launch_encode(const EncodeArgs &a, cudaStream_t stream);           // img/proj
int launch_encode_batched(const EncodeArgs &a, cudaStream_t stream);   // srcp/dstp

struct DecodeArgs {
    const uint64_t *proj;
    uint64_t *img;
    int64_t S;
    int64_t total;
    int P, Q;                       // Q: lines rebuilt (systematic: lost lines)
    bool sys;                       // systematic: img holds the Qd data lines, in place
    int Qd;                         // data lines per stripe
    int32_t lpos[kMaxLines];        // image row of each rebuilt line
    uint32_t known;                 // systematic: rows read from img
    bool scan2;                     // two lines: the closed form is available
    int32_t scan_p[2];
    int64_t scan_src[2];
    bool vander;                    // decode_vander is available
    int32_t van_q[kMaxLines], van_lo[kMaxLines], van_hi[kMaxLines];
    int64_t van_base[kMaxLines];
    int32_t van_E0, van_L;
    int T;
    const uint32_t *steps;          // device
    uint32_t fwd;                   // operand pattern of the steady steps
    int32_t pL[kMaxLines], pR[kMaxLines], split[kMaxLines];
    int64_t srcL[kMaxLines], srcR[kMaxLines];
    int32_t chunk_w, chunk_wait[kStreamChunks], chunk_done[kStreamChunks];
    int32_t rowoff[kMaxLines];
    uint32_t order[2 * kMaxLines];  // decode_lines load orders (see Schedule)
    int32_t ring_R, ring_D;         // decode_ring (one-sided path): ring words, chunks ahead
    int32_t ring_delta[kMaxLines];
    uint32_t *status;
};
int launch_decode(const DecodeArgs &a, cudaStream_t stream);

// One (geometry, erasure mask) of a batch: its reconstruction path, as the
// decode kernels read it from device memory.
struct DecGroup {
    const uint32_t *steps;          // T step words then T forward words (device)
    int32_t T;
    uint32_t fwd;                   // operand pattern of the steady steps
    int32_t p[2 * kMaxLines];       // direction of front (l, side), index 2l + side
    int32_t src[2 * kMaxLines];     // bin of pixel x of that front: word src - x
    int32_t split[kMaxLines];       // x < split[l]: left front
    uint32_t order[2 * kMaxLines];  // decode_lines: load order of each front (see Schedule)
    int32_t chunk_w;                // streamed chunks (see Schedule)
    int32_t chunk_wait[kStreamChunks];
    int32_t chunk_done[kStreamChunks];
    int32_t lpos[kMaxLines];        // image row of each rebuilt line
    uint32_t known;                 // systematic: data rows read, not rebuilt
    int32_t scan_p[2];              // decode_scan2: directions of lines 0 and 1
    int32_t scan_src[2];            //   and their bins: pixel x at word scan_src - x
    int32_t van_q[kMaxLines];       // decode_vander (see Schedule)
    int32_t van_base[kMaxLines];
    int32_t van_lo[kMaxLines];
    int32_t van_hi[kMaxLines];
    int32_t van_E0, van_L;
    int32_t ring_delta[kMaxLines];  // decode_ring: chunk start shift of each line (see Schedule)
};

// One work item of a batched decode: nst (<= G) stripes of group `group`,
// whose addresses sit at srcp/dstp[first .. first + nst).
struct DecWork {
    int32_t group;
    int32_t nst;
    int64_t first;
};

// Shared-memory layout of a decode launch (one warp per CTA).
struct DecodeLayout {
    int kernel;         // 0: decode_lines, 1: decode_fronts, 2: decode_stream, 3: decode_cols
    int reach, RP, SWc; // zero columns, row pitch, columns per stripe
    int SWr = 0;        // decode_lines: words per stripe region
    int G, GS;          // stripes per work item, their interleave stride
    int TS;             // words per step table (>= every group's steps, rounded)
    int rowbase[kMaxLines];   // first column of each line's row
    int64_t smem;       // dynamic shared memory per CTA
};
// Q lines rebuilt whose image rows span `span` rows (Q - 1 unless
// systematic); rowoff: decode_lines row offsets (may be null: none).
int decode_layout(int P, int Q, int span, int maxp, int maxT, const DecodeConfig &cfg,
                  const int32_t *rowoff, DecodeLayout *L);
// Bank slots of one stripe group of decode_lines / decode_stream for Q lines.
int decode_bank_slots(int Q);

struct DecBatchArgs {
    int P, Q;                       // Q: lines rebuilt (systematic: lost lines)
    bool sys;                       // systematic: dstp[s] holds the Qd data lines, in place
    int Qd, span;
    int van_maxp;                   // decode_vander: largest |p| its groups use
    int maxp, maxT;                 // over the groups (layout)
    int32_t rowoff[kMaxLines];      // decode_lines row offsets for the launch
    const DecGroup *groups;         // device
    const DecWork *work;            // device
    int64_t nwork;
    const uint64_t *const *srcp;    // device: projection block of each stripe
    uint64_t *const *dstp;          // device: image of each stripe
    uint32_t *status;
};
int launch_decode_batched(const DecBatchArgs &a, const DecodeConfig &cfg, cudaStream_t stream);

// Largest schedule (in steps) mojette_decode_noalloc accepts.
constexpr int kNoAllocMaxSteps = 16384;
// Copy a schedule's words into the fixed device scratch of decode.cu (on
// `stream`) and return its device address; no device allocation.
int noalloc_schedule_copy(const Schedule &sc, cudaStream_t stream, uint32_t **dev);

}  // namespace mojette
