// DOCH step on a periodic 2-D lattice (TORUS2D): x_out = T(x_in), Eq. FPE,
//   T(x)_i = cbrt( ( sum_j J_ij x_j + alpha x_i ) / beta ),
// with the four lattice neighbours j of site i and one int8 coupling per edge
// (right[r][c] couples (r,c)-(r,c+1), down[r][c] couples (r,c)-(r+1,c), both
// periodic). The lattice has no field term.
//
// Fast path (R = 1, FP32, l_cols % 4 == 0, 16-byte aligned rows): a CTA of
// 256 threads owns a tile of 1024 columns and a contiguous strip of rows.
// Each thread owns 4 columns (one float4 of x, one packed word of four int8
// couplings per row), walks down its strip keeping x rows r-1, r, r+1 and
// down rows r-1, r in registers, and prefetches the next row one step ahead.
// Horizontal neighbours come from the adjacent lanes by warp shuffles; the
// two edge lanes of a warp (and the lanes at the periodic seam) load their
// halo value from global memory. Per site and step the kernel reads x once
// (4 B), both couplings once (2 B) and writes x once (4 B), plus 2 extra x
// rows per strip.
#include "internal.cuh"

namespace doch {
namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int64_t wrap(int64_t i, int64_t L) {
    return i < 0 ? i + L : (i >= L ? i - L : i);
}

// sign-extended byte k (0..3) of a packed word of four int8
__device__ __forceinline__ float sbyte(int v, int k) {
    return static_cast<float>((v << (24 - 8 * k)) >> 24);
}

__global__ void __launch_bounds__(kThreads)
torus_f32_r1_vec4(const float *__restrict__ xi, float *__restrict__ xo,
                  const int8_t *__restrict__ right, const int8_t *__restrict__ down,
                  int64_t Lr, int64_t Lc, int tiles, int bpt, float alpha, float inv_beta) {
    const int tile = blockIdx.x % tiles;
    const int part = blockIdx.x / tiles;
    const int64_t r0 = Lr * part / bpt, r1 = Lr * (part + 1) / bpt;
    if (r0 >= r1) return;  // uniform over the block

    const int64_t ncol4 = Lc >> 2;
    const int64_t c4 = static_cast<int64_t>(tile) * kThreads + threadIdx.x;
    const bool active = c4 < ncol4;
    const int64_t c = c4 * 4;
    const int lane = threadIdx.x & 31;
    // halo columns: a lane whose neighbour lane does not hold them loads them
    const bool need_l = active && (lane == 0 || c == 0);
    const bool need_r = active && (lane == 31 || c + 4 >= Lc);
    const int64_t cl = (c == 0) ? Lc - 1 : c - 1;
    const int64_t cr = (c + 4 >= Lc) ? 0 : c + 4;

    auto ldx = [&](int64_t r) -> float4 {
        return active ? __ldg(reinterpret_cast<const float4 *>(xi + r * Lc) + c4)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto ldw = [&](const int8_t *p, int64_t r) -> int {
        return active ? __ldg(reinterpret_cast<const int *>(p + r * Lc) + c4) : 0;
    };
    auto ldhx = [&](bool need, int64_t r, int64_t cc) -> float {
        return need ? __ldg(xi + r * Lc + cc) : 0.f;
    };

    int64_t r = r0;
    float4 xu = ldx(wrap(r - 1, Lr));
    float4 xm = ldx(r);
    float hlm = ldhx(need_l, r, cl), hrm = ldhx(need_r, r, cr);
    int du = ldw(down, wrap(r - 1, Lr));
    // pending loads for row r: x row r+1 (+ halos), down row r, right row r (+ left halo)
    int64_t rp = wrap(r + 1, Lr);
    float4 xd_n = ldx(rp);
    float hld_n = ldhx(need_l, rp, cl), hrd_n = ldhx(need_r, rp, cr);
    int dm_n = ldw(down, r), rt_n = ldw(right, r);
    float wl_n = need_l ? static_cast<float>(__ldg(right + r * Lc + cl)) : 0.f;

    for (; r < r1; ++r) {
        const float4 xd = xd_n;
        const float hld = hld_n, hrd = hrd_n;
        const int dm = dm_n, rt = rt_n;
        const float wl = wl_n;
        if (r + 1 < r1) {  // prefetch the loads of row r+1
            const int64_t rn = r + 1, rnn = wrap(r + 2, Lr);
            xd_n = ldx(rnn);
            hld_n = ldhx(need_l, rnn, cl);
            hrd_n = ldhx(need_r, rnn, cr);
            dm_n = ldw(down, rn);
            rt_n = ldw(right, rn);
            wl_n = need_l ? static_cast<float>(__ldg(right + rn * Lc + cl)) : 0.f;
        }
        // horizontal neighbours of row r and the coupling to the left neighbour
        float xl = __shfl_up_sync(kFull, xm.w, 1);
        float xr = __shfl_down_sync(kFull, xm.x, 1);
        const int rt_left = __shfl_up_sync(kFull, rt, 1);
        float wleft = sbyte(rt_left, 3);
        if (need_l) { xl = hlm; wleft = wl; }
        if (need_r) xr = hrm;

        const float w0 = sbyte(rt, 0), w1 = sbyte(rt, 1), w2 = sbyte(rt, 2), w3 = sbyte(rt, 3);
        float u0 = w0 * xm.y + wleft * xl + sbyte(dm, 0) * xd.x + sbyte(du, 0) * xu.x;
        float u1 = w1 * xm.z + w0 * xm.x + sbyte(dm, 1) * xd.y + sbyte(du, 1) * xu.y;
        float u2 = w2 * xm.w + w1 * xm.y + sbyte(dm, 2) * xd.z + sbyte(du, 2) * xu.z;
        float u3 = w3 * xr + w2 * xm.z + sbyte(dm, 3) * xd.w + sbyte(du, 3) * xu.w;
        float4 out;
        out.x = cbrtf((u0 + alpha * xm.x) * inv_beta);
        out.y = cbrtf((u1 + alpha * xm.y) * inv_beta);
        out.z = cbrtf((u2 + alpha * xm.z) * inv_beta);
        out.w = cbrtf((u3 + alpha * xm.w) * inv_beta);
        if (active) __stcs(reinterpret_cast<float4 *>(xo + r * Lc) + c4, out);

        xu = xm; xm = xd; hlm = hld; hrm = hrd; du = dm;
    }
}

// Any R, float or double, any alignment: one thread per (site, replica).
template <typename T>
__global__ void torus_generic(const T *__restrict__ xi, T *__restrict__ xo,
                              const int8_t *__restrict__ right, const int8_t *__restrict__ down,
                              int64_t Lr, int64_t Lc, int R, T alpha, T beta) {
    const int64_t total = Lr * Lc * R;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t site = t / R;
        const int rep = static_cast<int>(t - site * R);
        const int64_t rr = site / Lc, cc = site - rr * Lc;
        const int64_t s_l = rr * Lc + (cc == 0 ? Lc - 1 : cc - 1);
        const int64_t s_r = rr * Lc + (cc + 1 == Lc ? 0 : cc + 1);
        const int64_t s_u = (rr == 0 ? Lr - 1 : rr - 1) * Lc + cc;
        const int64_t s_d = (rr + 1 == Lr ? 0 : rr + 1) * Lc + cc;
        const T u = static_cast<T>(right[site]) * xi[s_r * R + rep] +
                    static_cast<T>(right[s_l]) * xi[s_l * R + rep] +
                    static_cast<T>(down[site]) * xi[s_d * R + rep] +
                    static_cast<T>(down[s_u]) * xi[s_u * R + rep];
        const T z = (u + alpha * xi[t]);
        if constexpr (sizeof(T) == 4)
            xo[t] = cbrtf(z * beta);  // beta holds 1/beta for float
        else
            xo[t] = cbrt(z / beta);
    }
}

int vec4_blocks_per_sm() {
    static int occ = 0;
    if (!occ) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, torus_f32_r1_vec4, kThreads, 0) !=
                cudaSuccess || occ < 1)
            occ = 1;
    }
    return occ;
}

}  // namespace

ising_status_t torus_step_f32(const ising_context *c, const float *x_in, float *x_out, int R,
                              float alpha, float inv_beta, cudaStream_t st) {
    const int64_t Lr = c->l_rows, Lc = c->l_cols;
    const bool aligned = (reinterpret_cast<uintptr_t>(x_in) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(x_out) % 16 == 0);
    if (R == 1 && Lc % 4 == 0 && aligned) {
        const int64_t ncol4 = Lc / 4;
        const int tiles = static_cast<int>((ncol4 + kThreads - 1) / kThreads);
        const int64_t slots = static_cast<int64_t>(c->num_sms) * vec4_blocks_per_sm();
        int64_t bpt = slots / tiles;
        if (bpt < 1) bpt = 1;
        if (bpt > Lr / 4) bpt = Lr / 4 > 0 ? Lr / 4 : 1;
        const int64_t blocks = bpt * tiles;
        torus_f32_r1_vec4<<<static_cast<unsigned>(blocks), kThreads, 0, st>>>(
            x_in, x_out, c->right, c->down, Lr, Lc, tiles, static_cast<int>(bpt), alpha, inv_beta);
    } else {
        const int64_t total = Lr * Lc * R;
        int64_t blocks = (total + 255) / 256;
        const int64_t cap = static_cast<int64_t>(c->num_sms) * 16;
        if (blocks > cap) blocks = cap;
        torus_generic<float><<<static_cast<unsigned>(blocks), 256, 0, st>>>(
            x_in, x_out, c->right, c->down, Lr, Lc, R, alpha, inv_beta);
    }
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

ising_status_t torus_step_f64(const ising_context *c, const double *x_in, double *x_out, int R,
                              double alpha, double beta, cudaStream_t st) {
    const int64_t total = c->l_rows * c->l_cols * R;
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = static_cast<int64_t>(c->num_sms) * 16;
    if (blocks > cap) blocks = cap;
    torus_generic<double><<<static_cast<unsigned>(blocks), 256, 0, st>>>(
        x_in, x_out, c->right, c->down, c->l_rows, c->l_cols, R, alpha, beta);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

}  // namespace doch
