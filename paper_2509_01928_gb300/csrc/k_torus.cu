// DOCH step on a periodic 2-D lattice (TORUS2D): x_out = T(x_in), Eq. FPE,
//   T(x)_i = cbrt( ( sum_j J_ij x_j + alpha x_i ) / beta ),
// with the four lattice neighbours j of site i and one int8 coupling per edge
// (right[r][c] couples (r,c)-(r,c+1), down[r][c] couples (r,c)-(r+1,c), both
// periodic). The lattice has no field term.
//
// Fast path (R = 1, FP32, l_cols % 4 == 0, 16-byte aligned rows): a CTA of
// 256 threads owns a tile of 1024 columns and a contiguous strip of rows.
// Each thread owns 4 columns (one float4 of x, one packed word of four int8
// couplings per row), walks down its strip keeping x rows r-1, r, r+1 and the
// down couplings of row r-1 (already converted) in registers, and prefetches
// the loads of the next row one step ahead. Horizontal neighbours come from
// the adjacent lanes by warp shuffles; lane 0 loads the left halo (and the
// coupling to it), lane 31 the right halo. Lanes past the last column of the
// lattice read wrapped columns, so the shuffles at the periodic seam deliver
// column 0. Per site and step the kernel reads x once (4 B), both couplings
// once (2 B) and writes x once (4 B), plus 2 extra x rows per strip.
//
// Cube root: cbrt(z) = 2^(k) * exp2( log2(|z| 2^(-3k)) / 3 ) with sign, using
// the hardware base-2 logarithm/exponential approximations (PTX lg2.approx,
// ex2.approx). The exact power-of-two prescale 2^(-3k) is folded into 1/beta
// (k chosen on the host from beta) so |log2| stays small and the FP32 log
// keeps its precision; relative error ~2^-22.
#include <cmath>

#include "cbrt.cuh"
#include "internal.cuh"

namespace doch {
namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

// sign-extended byte k (0..3) of a packed word of four int8
__device__ __forceinline__ float sbyte(int v, int k) {
    return static_cast<float>((v << (24 - 8 * k)) >> 24);
}

// 40 registers: 6 CTAs (1536 threads) per SM keep enough loads in flight
__global__ void __launch_bounds__(kThreads, 6)
torus_f32_r1_vec4(const float *__restrict__ xi, float *__restrict__ xo,
                  const int8_t *__restrict__ right, const int8_t *__restrict__ down, int Lr, int Lc,
                  int tiles, int bpt, float alpha, float zscale, float xscale) {
    const int tile = blockIdx.x % tiles;
    const int part = blockIdx.x / tiles;
    const int r0 = static_cast<int>(static_cast<int64_t>(Lr) * part / bpt);
    const int r1 = static_cast<int>(static_cast<int64_t>(Lr) * (part + 1) / bpt);
    if (r0 >= r1) return;  // uniform over the block

    const int ncol4 = Lc >> 2;
    const int c4raw = tile * kThreads + threadIdx.x;
    const bool active = c4raw < ncol4;
    const int c4 = c4raw % ncol4;
    const int c = c4 * 4;
    const int lane = threadIdx.x & 31;
    const bool is_l = lane == 0, is_r = lane == 31;
    const int hcol = is_l ? (c == 0 ? Lc - 1 : c - 1) : (c + 4 >= Lc ? 0 : c + 4);
    const int64_t n = static_cast<int64_t>(Lr) * Lc;
    const float *xc = xi + c;
    const int8_t *rc = right + c, *dc = down + c;
    const float *hx = xi + hcol;
    const int8_t *hw = right + hcol;
    float *oc = xo + c;
    auto ldx = [&](int64_t o) -> float4 { return __ldg(reinterpret_cast<const float4 *>(xc + o)); };
    auto ldw = [&](const int8_t *p, int64_t o) -> int { return __ldg(reinterpret_cast<const int *>(p + o)); };
    auto ldh = [&](int64_t o) -> float { return (is_l || is_r) ? __ldg(hx + o) : 0.f; };

    int64_t o = static_cast<int64_t>(r0) * Lc;        // row r
    const int64_t ou = o == 0 ? n - Lc : o - Lc;       // row r-1
    int64_t od = o + Lc == n ? 0 : o + Lc;             // row r+1
    float4 xu = ldx(ou), xm = ldx(o);
    float hm = ldh(o);
    const int dup = ldw(dc, ou);
    float du0 = sbyte(dup, 0), du1 = sbyte(dup, 1), du2 = sbyte(dup, 2), du3 = sbyte(dup, 3);
    float4 xd = ldx(od);
    float hd = ldh(od);
    int dm = ldw(dc, o), rt = ldw(rc, o);
    float wl = is_l ? static_cast<float>(__ldg(hw + o)) : 0.f;
    for (int r = r0; r < r1; ++r) {
        const int64_t on = od;                            // row r+1
        const int64_t onn = on + Lc == n ? 0 : on + Lc;   // row r+2
        float4 xn = xd;
        float hn = hd, wn = wl;
        int dn = dm, rn = rt;
        if (r + 1 < r1) {  // prefetch the loads of row r+1
            xn = ldx(onn);
            hn = ldh(onn);
            dn = ldw(dc, on);
            rn = ldw(rc, on);
            wn = is_l ? static_cast<float>(__ldg(hw + on)) : 0.f;
        }
        // horizontal neighbours of row r and the coupling to the left neighbour
        float xl = __shfl_up_sync(kFull, xm.w, 1);
        float xr = __shfl_down_sync(kFull, xm.x, 1);
        const int rtl = __shfl_up_sync(kFull, rt, 1);
        float wleft = sbyte(rtl, 3);
        if (is_l) { xl = hm; wleft = wl; }
        if (is_r) xr = hm;

        const float w0 = sbyte(rt, 0), w1 = sbyte(rt, 1), w2 = sbyte(rt, 2), w3 = sbyte(rt, 3);
        const float d0 = sbyte(dm, 0), d1 = sbyte(dm, 1), d2 = sbyte(dm, 2), d3 = sbyte(dm, 3);
        const float u0 = w0 * xm.y + wleft * xl + d0 * xd.x + du0 * xu.x;
        const float u1 = w1 * xm.z + w0 * xm.x + d1 * xd.y + du1 * xu.y;
        const float u2 = w2 * xm.w + w1 * xm.y + d2 * xd.z + du2 * xu.z;
        const float u3 = w3 * xr + w2 * xm.z + d3 * xd.w + du3 * xu.w;
        float4 out;
        out.x = cbrt_pow2((u0 + alpha * xm.x) * zscale) * xscale;
        out.y = cbrt_pow2((u1 + alpha * xm.y) * zscale) * xscale;
        out.z = cbrt_pow2((u2 + alpha * xm.z) * zscale) * xscale;
        out.w = cbrt_pow2((u3 + alpha * xm.w) * zscale) * xscale;
        if (active) __stcs(reinterpret_cast<float4 *>(oc + o), out);

        xu = xm; xm = xd; hm = hd;
        du0 = d0; du1 = d1; du2 = d2; du3 = d3;
        xd = xn; hd = hn; dm = dn; rt = rn; wl = wn;
        o = on; od = onn;
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
                              float alpha, double inv_beta, cudaStream_t st) {
    const int64_t Lr = c->l_rows, Lc = c->l_cols;
    const bool aligned = (reinterpret_cast<uintptr_t>(x_in) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(x_out) % 16 == 0);
    if (R == 1 && Lc % 4 == 0 && aligned && Lr < (1LL << 31) && Lc < (1LL << 31)) {
        const int64_t ncol4 = Lc / 4;
        const int tiles = static_cast<int>((ncol4 + kThreads - 1) / kThreads);
        const int64_t slots = static_cast<int64_t>(c->num_sms) * vec4_blocks_per_sm();
        int64_t bpt = slots / tiles;
        if (bpt < 1) bpt = 1;
        if (bpt > Lr / 4) bpt = Lr / 4 > 0 ? Lr / 4 : 1;
        const int64_t blocks = bpt * tiles;
        const int k = cbrt_prescale_exp(inv_beta);
        const float zscale = static_cast<float>(std::ldexp(inv_beta, 3 * k));
        const float xscale = std::ldexp(1.0f, -k);
        torus_f32_r1_vec4<<<static_cast<unsigned>(blocks), kThreads, 0, st>>>(
            x_in, x_out, c->right, c->down, static_cast<int>(Lr), static_cast<int>(Lc), tiles,
            static_cast<int>(bpt), alpha, zscale, xscale);
    } else {
        const int64_t total = Lr * Lc * R;
        int64_t blocks = (total + 255) / 256;
        const int64_t cap = static_cast<int64_t>(c->num_sms) * 16;
        if (blocks > cap) blocks = cap;
        torus_generic<float><<<static_cast<unsigned>(blocks), 256, 0, st>>>(
            x_in, x_out, c->right, c->down, Lr, Lc, R, alpha, static_cast<float>(inv_beta));
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
