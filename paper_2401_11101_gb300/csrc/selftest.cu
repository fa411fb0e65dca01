// Self-test of the failure path of bounded device waits (no counterpart in
// the method). One CTA initialises an mbarrier that nothing ever arrives at
// and waits on it with the same bounded wait the TMA pipeline uses; when the
// limit passes, the wait returns false and the kernel records error code 4 in
// the plan's error word and returns. The kernel always ends: the wait reads
// %globaltimer, which advances whatever the barrier does.
#include "common.cuh"
#include "sync.cuh"

namespace lam {
namespace {

__global__ void __launch_bounds__(32) k_expired_wait(int* err, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // phase 0 of a fresh barrier completes only after one arrival: none comes
    const bool ok = mbar_wait(smem_addr(&bar), 0, limit_ns);
    if (!ok && threadIdx.x == 0) atomicExch(err, 4);
}

}  // namespace
}  // namespace lam

extern "C" int lamino_selftest_wait(lamino_plan_t p, unsigned int limit_us, cudaStream_t stream) {
    using namespace lam;
    if (!p) return fail(nullptr, LAMINO_EINVAL, "NULL plan");
    if (limit_us < 1 || limit_us > 5000000u)
        return fail(p, LAMINO_EINVAL, "lamino_selftest_wait: limit %u us outside [1, 5000000]", limit_us);
    int rc = set_device(p);
    if (rc) return rc;
    k_expired_wait<<<1, 32, 0, stream>>>(p->d_err, 1000ull * limit_us);
    LAM_CUDA(p, cudaGetLastError());
    return LAMINO_OK;
}
