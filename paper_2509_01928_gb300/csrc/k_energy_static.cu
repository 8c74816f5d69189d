// Energy and cut of a periodic lattice without any device allocation.
//
// Some callers cannot call cudaMalloc: code whose device memory is wholly
// owned by another allocator (a framework that has reserved the device for
// its own pool and forbids outside allocations), or a latency-critical loop
// in which an allocation, which may synchronise the device, is not
// acceptable. ising_energy needs a handle, and the handle allocates device
// copies of J plus scratch for the reduction partials. This entry point takes
// the lattice couplings, the iterates and the outputs as device arrays from
// the caller and keeps its reduction partials in a file-scope device array of
// fixed size, so it allocates nothing.
//
// Arithmetic: the same readout as ising_energy on a TORUS2D handle with FP32
// iterates: s = sign(x) with sign(0) = +1, E_r = -1/2 s^T J s (no field) and
// cut_r = 1/4 sum_ij (1 - s_i s_j) W_ij with W = -2J, exact in int64.
#include <climits>
#include <mutex>

#include "internal.cuh"

namespace doch {
namespace {

// Capacity of the static partials: 2 int64 per (replica, chunk).
constexpr int kStaticReplicas = 8192;
constexpr int kStaticSlots = 2 * kStaticReplicas;
constexpr int kThreadsS = 256;
constexpr int kWarpsS = kThreadsS / 32;

// One copy per device that loads the library; it stays allocated until the
// process exits. Every call shares it.
static __device__ __align__(256) long long g_energy_partials[kStaticSlots];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
long long *g_partials_addr[kMaxDevices] = {};

__device__ __forceinline__ int spin_f32(float v) { return v >= 0.f ? 1 : -1; }

// Lanes are (site, replica) pairs with the replica fastest: RT = the power of
// two >= min(R, 32) replicas per lane group, 32 / RT sites per warp step, so a
// warp's loads of x (and of the neighbours' x) are consecutive addresses.
// Block (ch, rt) covers the sites of chunk ch for replicas rt*RT .. rt*RT+RT-1.
// partials[(r * chunks + ch) * 2 + k]: k = 0 -> sum_{i,j} J_ij s_i s_j,
// k = 1 -> sum_{i,j} J_ij (1 - s_i s_j); each lattice edge enters twice.
// Integer sums are exact, so the result does not depend on the order.
__global__ void __launch_bounds__(kThreadsS)
torus_energy_partials_static(const int8_t *__restrict__ right, const int8_t *__restrict__ down,
                             int64_t Lr, int64_t Lc, const float *__restrict__ x, int R, int RT, int chunks,
                             long long *__restrict__ partials) {
    const int ch = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rl = lane % RT, sub = lane / RT, per_warp = 32 / RT;
    const int r = blockIdx.y * RT + rl;
    const int64_t n = Lr * Lc;
    const int64_t s0 = n * ch / chunks, s1 = n * (ch + 1) / chunks;
    long long q = 0, cw = 0;
    if (r < R) {
        for (int64_t i = s0 + static_cast<int64_t>(warp) * per_warp + sub; i < s1;
             i += static_cast<int64_t>(kWarpsS) * per_warp) {
            const int64_t rr = i / Lc, cc = i - rr * Lc;
            const int64_t jr = rr * Lc + (cc + 1 == Lc ? 0 : cc + 1);
            const int64_t jd = (rr + 1 == Lr ? 0 : rr + 1) * Lc + cc;
            const int s = spin_f32(x[i * R + r]);
            const int sr = spin_f32(x[jr * R + r]);
            const int sd = spin_f32(x[jd * R + r]);
            const int wr = right[i], wd = down[i];
            q += 2LL * (wr * s * sr + wd * s * sd);
            cw += 2LL * (wr * (1 - s * sr) + wd * (1 - s * sd));
        }
    }
    // lanes with the same replica differ by multiples of RT
    for (int o = 16; o >= RT; o >>= 1) {
        q += __shfl_xor_sync(0xffffffffu, q, o);
        cw += __shfl_xor_sync(0xffffffffu, cw, o);
    }
    __shared__ long long red[2][kWarpsS][32];
    if (lane < RT) { red[0][warp][lane] = q; red[1][warp][lane] = cw; }
    __syncthreads();
    if (threadIdx.x < RT && r < R) {
        long long tq = 0, tc = 0;
        for (int w = 0; w < kWarpsS; ++w) { tq += red[0][w][threadIdx.x]; tc += red[1][w][threadIdx.x]; }
        partials[(static_cast<int64_t>(r) * chunks + ch) * 2 + 0] = tq;
        partials[(static_cast<int64_t>(r) * chunks + ch) * 2 + 1] = tc;
    }
}

__global__ void torus_energy_finish_static(const long long *__restrict__ partials, int R, int chunks,
                                           int64_t *__restrict__ E, int64_t *__restrict__ cut) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    long long q = 0, cw = 0;
    for (int c = 0; c < chunks; ++c) {
        q += partials[(static_cast<int64_t>(r) * chunks + c) * 2 + 0];
        cw += partials[(static_cast<int64_t>(r) * chunks + c) * 2 + 1];
    }
    if (E) E[r] = -(q / 2);
    if (cut) cut[r] = -(cw / 2);
}

// device (or managed) memory of device `dev`, the current device
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Address of this device's copy of the static partials, looked up once per
// device (with that device current) and cached.
ising_status_t static_partials(long long **out) {
    int dev = 0;
    DOCH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(ISING_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void *p = nullptr;
        DOCH_CUDA(cudaGetSymbolAddress(&p, g_energy_partials));
        g_partials_addr[dev] = static_cast<long long *>(p);
    }
    *out = g_partials_addr[dev];
    return ISING_OK;
}

}  // namespace
}  // namespace doch

extern "C" ising_status_t ising_energy_torus_noalloc(const int8_t *right, const int8_t *down,
                                                     int64_t l_rows, int64_t l_cols, const float *x,
                                                     int32_t R, int64_t *E_out, int64_t *cut_out,
                                                     void *stream) {
    return doch::guarded([&]() -> ising_status_t {
        using namespace doch;
        if (!right || !down || !x || (!E_out && !cut_out))
            return fail(ISING_ERR_INVALID_ARG, "noalloc energy: NULL argument");
        if (l_rows < 2 || l_cols < 2) return fail(ISING_ERR_INVALID_ARG, "noalloc energy: l_rows, l_cols must be >= 2");
        if (R < 1) return fail(ISING_ERR_INVALID_ARG, "noalloc energy: R must be >= 1");
        if (R > kStaticReplicas)
            return fail(ISING_ERR_INVALID_ARG, "noalloc energy: R exceeds the static scratch capacity of " +
                                                   std::to_string(kStaticReplicas) + " replicas");
        if (l_rows > (int64_t(1) << 31) || l_cols > (int64_t(1) << 31) ||
            l_rows * l_cols > INT64_MAX / R)
            return fail(ISING_ERR_INVALID_ARG, "noalloc energy: lattice too large");
        int dev = 0, sms = 1;
        DOCH_CUDA(cudaGetDevice(&dev));
        if (!on_device(right, dev) || !on_device(down, dev) || !on_device(x, dev) ||
            (E_out && !on_device(E_out, dev)) || (cut_out && !on_device(cut_out, dev)))
            return fail(ISING_ERR_INVALID_ARG,
                        "noalloc energy: every array must be device memory of the current device");
        long long *partials = nullptr;
        DOCH_CHECK(static_partials(&partials));
        DOCH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int64_t n = l_rows * l_cols;
        int RT = 1;
        while (RT < R && RT < 32) RT <<= 1;
        const int64_t rtiles = (R + RT - 1) / RT;
        int64_t chunks = (4LL * sms + rtiles - 1) / rtiles;
        const int64_t cap_slots = kStaticReplicas / R;            // chunks whose partials fit
        const int64_t cap_sites = (n + (kThreadsS / RT) - 1) / (kThreadsS / RT);  // a block step of sites each
        if (chunks > cap_slots) chunks = cap_slots;
        if (chunks > cap_sites) chunks = cap_sites;
        if (chunks > 65535) chunks = 65535;
        if (chunks < 1) chunks = 1;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        // every partial read by the finisher is written by this call first: no clearing needed
        dim3 grid(static_cast<unsigned>(chunks), static_cast<unsigned>(rtiles));
        torus_energy_partials_static<<<grid, kThreadsS, 0, st>>>(right, down, l_rows, l_cols, x, R, RT,
                                                                static_cast<int>(chunks), partials);
        DOCH_CUDA(cudaGetLastError());
        torus_energy_finish_static<<<(R + 127) / 128, 128, 0, st>>>(partials, R, static_cast<int>(chunks),
                                                                   E_out, cut_out);
        DOCH_CUDA(cudaGetLastError());
        return ISING_OK;
    });
}
