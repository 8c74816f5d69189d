// Diagnostic entry points: the device cube root cbrt_pow2 next to
// CUDA's cbrtf on the same inputs (see ising_selftest_cbrt in ising.h), and the
// lattice kernels' cube root with its log-domain offset (ising_selftest_cbrt_log).
#include <cmath>

#include "cbrt.cuh"
#include "internal.cuh"

namespace doch {
namespace {

__global__ void cbrt_pair(const float *__restrict__ z, float *__restrict__ ours,
                          float *__restrict__ ref, int64_t n, float zscale, float xscale) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        ours[i] = cbrt_pow2(z[i] * zscale) * xscale;
        ref[i] = cbrtf(z[i]);
    }
}

__global__ void cbrt_log_kernel(const float *__restrict__ z, float *__restrict__ out, int64_t n, float c3) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[i] = cbrt_log(z[i], c3);
}

}  // namespace
}  // namespace doch

extern "C" ising_status_t ising_selftest_cbrt_log(const float *z, float *out, int64_t n, float c3, void *stream) {
    return doch::guarded([&]() -> ising_status_t {
        using namespace doch;
        if (!z || !out || n < 0 || !std::isfinite(c3) || std::fabs(c3) > 64.f)
            return fail(ISING_ERR_INVALID_ARG, "selftest_cbrt_log: bad argument");
        if (n == 0) return ISING_OK;
        int dev = 0, sms = 1;
        DOCH_CUDA(cudaGetDevice(&dev));
        DOCH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int64_t blocks = (n + 255) / 256;
        if (blocks > 8LL * sms) blocks = 8LL * sms;
        cbrt_log_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(z, out, n, c3);
        DOCH_CUDA(cudaGetLastError());
        DOCH_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
        return ISING_OK;
    });
}

extern "C" ising_status_t ising_selftest_cbrt(const float *z, float *ours, float *ref, int64_t n,
                                              int32_t k, void *stream) {
    return doch::guarded([&]() -> ising_status_t {
        using namespace doch;
        if (!z || !ours || !ref || n < 0 || k < -40 || k > 40)
            return fail(ISING_ERR_INVALID_ARG, "selftest_cbrt: bad argument");
        if (n == 0) return ISING_OK;
        int dev = 0, sms = 1;
        DOCH_CUDA(cudaGetDevice(&dev));
        DOCH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int64_t blocks = (n + 255) / 256;
        if (blocks > 8LL * sms) blocks = 8LL * sms;
        cbrt_pair<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
            z, ours, ref, n, std::ldexp(1.0f, -3 * k), std::ldexp(1.0f, k));
        DOCH_CUDA(cudaGetLastError());
        DOCH_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
        return ISING_OK;
    });
}

// ---------------------------------------------------------------------------
// Bounded-wait self-test: one thread waits on a shared-memory mbarrier with
// the same bounded wait the tensor-core kernel uses. With arrive = 0 nobody
// arrives, so the wait runs out after limit_ns and sets DEV_ERR_TIMEOUT in the
// handle's error word; with arrive = 1 the thread arrives first and the wait
// completes at once. Nothing else is touched, so the context stays usable.
// ---------------------------------------------------------------------------
#include "mbar.cuh"

namespace doch {
namespace {

__global__ void wait_selftest(int *err, int arrive, uint64_t limit_ns) {
    __shared__ alignas(8) unsigned long long bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    abort_flag = 0;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&bar)) : "memory");
    mbar_wait(&bar, 0, err, &abort_flag, limit_ns);
}

}  // namespace

ising_status_t selftest_wait_launch(int *err, bool arrive, uint64_t limit_ns, cudaStream_t st) {
    wait_selftest<<<1, 32, 0, st>>>(err, arrive ? 1 : 0, limit_ns);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

}  // namespace doch
