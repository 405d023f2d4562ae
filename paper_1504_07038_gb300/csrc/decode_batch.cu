// Batched decode launcher: work items of G stripes, each with its own
// reconstruction path (DecGroup) and per-stripe addresses, in one launch
// (the kernels are in decode_kernels.cuh; the tables are built by batch.cpp).
#include "decode_kernels.cuh"

namespace mojette {

int launch_decode_batched(const DecBatchArgs &b, const DecodeConfig &cfg, cudaStream_t st)
{
    DecodeLayout L;
    if (b.sys && cfg.kernel != 0 && cfg.kernel != 4) return -EINVAL;
    int err = decode_layout(b.P, b.Q, b.span, cfg.kernel == 5 ? b.van_maxp : b.maxp, b.maxT, cfg, b.rowoff, &L);
    if (err) return err;
    DecParams a;
    std::memset(&a, 0, sizeof(a));
    a.groups = b.groups;
    a.work = b.work;
    a.nwork = b.nwork;
    a.srcp = b.srcp;
    a.dstp = b.dstp;
    a.P = b.P;
    a.Q = b.Q;
    a.Qd = b.Qd;
    a.status = b.status;
    if (b.sys && L.kernel != 4) {
        // residual bins into the lost rows, then the path (none for one lost
        // line); decode_scan2 removes the known lines itself
        if ((err = launch_sys_residual<true>(a, L, b.nwork, st))) return err;
        if (b.maxT == 0) return 0;
    }
    return launch_decode_kernel<true>(a, L, cfg, b.nwork, st, b.sys);
}

}  // namespace mojette
