// Failure-detection self-test (mojette_selftest_wait in include/mojette.h):
// one warp waits, through the same bounded mbarrier wait the encoder's
// pipeline uses, for 16 bytes of asynchronous copy that are never issued.
// The wait gives up after the given limit, the kernel sets the status bit a
// real timeout would and returns, and the host reads it with
// mojette_device_status. Nothing faults, traps or hangs, and no copy is in
// flight when the kernel exits.
#include <cerrno>

#include "ptx.cuh"

namespace mojette {
namespace {

__global__ void __launch_bounds__(32) wait_selftest(uint32_t *status, uint64_t limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        mbar_init_fence();
        mbar_arrive_expect_tx(b, 16);   // 16 bytes nothing will deliver
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(b, 0, limit_ns);
    if (__any_sync(0xffffffffu, !ok) && threadIdx.x == 0) atomicOr(status, kStatusWaitTimeout);
}

}  // namespace
}  // namespace mojette

using namespace mojette;

extern "C" int mojette_selftest_wait(int64_t limit_ns, mojette_stream_t stream)
{
    if (limit_ns < 1000 || limit_ns > 1000000000) return -EINVAL;
    int err = 0;
    uint32_t *status = device_status_ptr(&err);
    if (err) return err;
    wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(status, (uint64_t)limit_ns);
    return record_cuda(cudaGetLastError());
}
