// Self-test of the bounded device-side waits.  Every spin of the library (the look-back
// of the extraction, the mbarrier wait for staged pixels) gives up after a time limit,
// records kDevErrTimeout in an error word and returns, so that a lost predecessor or a
// lost copy surfaces as TOPOT_ERR_TIMEOUT instead of a hung GPU.  These kernels make
// such a wait run out on purpose -- a flag that nothing sets, an mbarrier whose phase
// never completes (no copy is issued) -- with a short limit, so that a test can check
// the status path and that the context stays usable afterwards.
#include "internal.cuh"

namespace topot {

__global__ void k_selftest_flag_wait(const unsigned long long* flag, unsigned long long limit_ns, unsigned* err) {
    const unsigned long long t0 = dev_time_ns();
    while (ld_relaxed_u64(flag) == 0ull) {
        if (dev_time_ns() - t0 > limit_ns) {
            if (threadIdx.x == 0) dev_set_error(err, kDevErrTimeout);
            return;
        }
    }
}

__global__ void k_selftest_mbar_wait(unsigned long long limit_ns, unsigned* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);          // two arrivals expected, one given: the phase never completes
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 0u);
    mbar_wait_bounded(&bar, 0, err, limit_ns);
}

cudaError_t launch_selftest_wait(int which, unsigned long long limit_ns, unsigned long long* flag, unsigned* err,
                                 cudaStream_t st) {
    if (which == 0) k_selftest_flag_wait<<<1, 32, 0, st>>>(flag, limit_ns, err);
    else k_selftest_mbar_wait<<<1, 64, 0, st>>>(limit_ns, err);
    return cudaGetLastError();
}

}  // namespace topot
