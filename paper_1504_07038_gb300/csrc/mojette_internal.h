// Internal declarations of libmojette (host plan/schedule code and kernels).
#pragma once

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

// A bounded device-side wait gives up after this many nanoseconds.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Reconstruction path for one (geometry, erasure mask): Sec. 2.2's
// pre-determined path with one projection dedicated to each line, run from
// both ends of every line (a left-to-right and a right-to-left front).
struct Schedule {
    uint32_t mask = 0;
    int T = 0;                       // number of steps
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
    std::map<int, uint32_t *> dev;   // device copy of `steps` then `fwdw`, per device
};

struct Plan {
    int P = 0, Q = 0, n = 0;
    int32_t p[kMaxProj] = {};
    int64_t B[kMaxProj] = {};
    int64_t off[kMaxProj] = {};
    int64_t bmin[kMaxProj] = {};
    int64_t total = 0;
    std::mutex mu;
    std::map<uint32_t, std::unique_ptr<Schedule>> schedules;
};

// ---- host helpers (plan.cpp) ---------------------------------------------
int build_schedule(const Plan &pl, uint32_t mask, Schedule *out);
// Returns the cached schedule (building it on a miss) or sets *err.
Schedule *get_schedule(Plan &pl, uint32_t mask, int *err);
// Device copy of a schedule's step words on the current device.
int schedule_on_device(Plan &pl, Schedule &sc, uint32_t **dev);
int record_cuda(cudaError_t e);     // remembers e; returns 0 or -EIO
uint32_t *device_status_ptr(int *err);  // per-device status word

// ---- kernel launchers -------------------------------------------------------
struct EncodeArgs {
    const uint64_t *img;
    uint64_t *proj;
    int64_t S;
    int64_t total;
    int P, Q, n;
    int32_t p[kMaxProj];
    int64_t off[kMaxProj];
    int64_t bmin[kMaxProj];
    uint32_t *status;
};
int launch_encode(const EncodeArgs &a, cudaStream_t stream);

struct DecodeArgs {
    const uint64_t *proj;
    uint64_t *img;
    int64_t S;
    int64_t total;
    int P, Q;
    int T;
    const uint32_t *steps;          // device
    uint32_t fwd;                   // operand pattern of the steady steps
    int32_t pL[kMaxLines], pR[kMaxLines], split[kMaxLines];
    int64_t srcL[kMaxLines], srcR[kMaxLines];
    uint32_t *status;
};
int launch_decode(const DecodeArgs &a, cudaStream_t stream);

// Largest schedule (in steps) mojette_decode_noalloc accepts.
constexpr int kNoAllocMaxSteps = 16384;
// Copy a schedule's words into the fixed device scratch of decode.cu (on
// `stream`) and return its device address; no device allocation.
int noalloc_schedule_copy(const Schedule &sc, cudaStream_t stream, uint32_t **dev);

}  // namespace mojette
