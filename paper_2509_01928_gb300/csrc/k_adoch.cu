// ADOCH (Algorithm 2): the DOCH map with a Nesterov-type extrapolation that
// is kept only when it passes a non-monotone test on the DC Hamiltonian H of
// Eq. Hamilton, H(x) = beta/4 sum x^4 - alpha/2 sum x^2 - 1/2 x^T J x - h^T x:
//   t_0 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, c_k = (t_k - 1) / t_{k+1},
//   y^k = x^k + c_k (x^k - x^{k-1})   (y^0 = x^0),
//   v^k = y^k if H(y^k) <= max(H(x^{max(0,k-q)}), ..., H(x^k)), else x^k,
//   x^{k+1} = T(v^k) = cbrt((J v^k + alpha v^k + h) / beta).
// One coupling product per step, by linearity: u^k = J x^k is formed once,
// J y^k = (1 + c_k) u^k - c_k u^{k-1}, and J v^k is u^k or J y^k. Each step is
//  (1) pass: u^k and, per (instance, replica, chunk) block, FP64 partial sums
//      of the terms of H(x^k) and H(y^k) in a fixed order;
//  (2) decide: one block per (instance, replica) adds the chunk partials in a
//      fixed order, forms H(x^k) and H(y^k), keeps the last q+1 values of H(x)
//      and sets the acceptance flag;
//  (3) update: x^{k+1} = T(v^k) element-wise.
// The coupling product and the update run in the iterate's precision (as the
// DOCH step kernels); H is reduced in FP64 across threads and blocks. With
// FP32 iterates each thread first sums its sites' terms in FP32 with Kahan
// compensation (FP64 arithmetic is a small fraction of the FP32 rate here),
// with FP64 iterates in FP64.
#include <algorithm>
#include <cmath>
#include <utility>

#include "cbrt.cuh"
#include "internal.cuh"

namespace doch {
namespace {

constexpr int kAThreads = 256;
constexpr int kTerms = 8;  // x^4, x^2, x u, h x, y^4, y^2, y Jy, h y

template <typename T>
__device__ __forceinline__ T acbrt(T z) {
    if constexpr (sizeof(T) == 4) return cbrtf(z);
    else return cbrt(z);
}

// scale by 1/beta: float tables hold 1/beta (multiply), double tables hold beta (divide)
template <typename T>
__device__ __forceinline__ T ascale(T v, T b) {
    if constexpr (sizeof(T) == 4) return v * b;
    else return v / b;
}

// u_i = (J x)_i for replica r, in the iterate's precision and the step kernels' order
template <typename XT, typename VT>
struct CsrProduct {
    const int64_t *row_ptr;
    const int32_t *col;
    const VT *val;
    static constexpr bool kGrid = false;
    static constexpr bool kStored = false;
    __device__ XT operator()(const XT *x, int64_t i, int64_t, int64_t, int r, int R) const {
        XT acc = XT(0);
        const int64_t e1 = row_ptr[i + 1];
        for (int64_t e = row_ptr[i]; e < e1; ++e)
            acc += static_cast<XT>(val[e]) * x[static_cast<int64_t>(col[e]) * R + r];
        return acc;
    }
};

template <typename XT>
struct TorusProduct {
    const int8_t *right, *down;
    int64_t Lr, Lc;
    static constexpr bool kGrid = true;  // wants the (row, column) of site i
    static constexpr bool kStored = false;
    __device__ XT operator()(const XT *x, int64_t i, int64_t rr, int64_t cc, int r, int R) const {
        const int64_t s_l = rr * Lc + (cc == 0 ? Lc - 1 : cc - 1);
        const int64_t s_r = rr * Lc + (cc + 1 == Lc ? 0 : cc + 1);
        const int64_t s_u = (rr == 0 ? Lr - 1 : rr - 1) * Lc + cc;
        const int64_t s_d = (rr + 1 == Lr ? 0 : rr + 1) * Lc + cc;
        return static_cast<XT>(right[i]) * x[s_r * R + r] + static_cast<XT>(right[s_l]) * x[s_l * R + r] +
               static_cast<XT>(down[i]) * x[s_d * R + r] + static_cast<XT>(down[s_u]) * x[s_u * R + r];
    }
};

// procedural couplings: u^k = J x^k is formed by the procedural product before the pass
// (the pass reads it from u1 instead of computing it)
struct ProcProduct {
    static constexpr bool kGrid = false;
    static constexpr bool kStored = true;
    __device__ float operator()(const float *, int64_t, int64_t, int64_t, int, int) const { return 0.f; }
};

template <typename Acc>
__device__ __forceinline__ Acc warp_sum(Acc v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// (1) grid (chunks, R, n_inst): rows of instance b in chunk ch, replica r
template <typename XT, typename Fn>
__global__ void __launch_bounds__(kAThreads)
adoch_pass(Fn fn, const XT *__restrict__ x1, const XT *__restrict__ x0, const XT *__restrict__ u0,
           XT *__restrict__ u1, const double *__restrict__ h, const int64_t *__restrict__ inst_off, int64_t n,
           int R, int chunks, XT c, double *__restrict__ partials) {
    const int ch = blockIdx.x, r = blockIdx.y, b = blockIdx.z;
    const int64_t lo = inst_off ? inst_off[b] : 0;
    const int64_t hi = inst_off ? inst_off[b + 1] : n;
    const int64_t len = hi - lo;
    const int64_t s0 = lo + len * ch / chunks, s1 = lo + len * (ch + 1) / chunks;
    // per-thread sums: FP32 with Kahan compensation for FP32 iterates, FP64 otherwise
    using Acc = XT;
    Acc acc[kTerms], cmp[kTerms];
#pragma unroll
    for (int k = 0; k < kTerms; ++k) acc[k] = cmp[k] = Acc(0);
    auto add = [&](int k, Acc v) {
        if constexpr (sizeof(XT) == 4) {
            const Acc y = v - cmp[k];
            const Acc t = acc[k] + y;
            cmp[k] = (t - acc[k]) - y;
            acc[k] = t;
        } else {
            acc[k] += v;
        }
    };
    // (row, column) of the site, advanced without division (lattice only)
    int64_t rr = 0, cc = 0, Lc = 1;
    if constexpr (Fn::kGrid) {
        Lc = fn.Lc;
        rr = (s0 + threadIdx.x) / Lc;
        cc = (s0 + threadIdx.x) - rr * Lc;
    }
    for (int64_t i = s0 + threadIdx.x; i < s1; i += kAThreads) {
        const int64_t at = i * R + r;
        XT u;
        if constexpr (Fn::kStored) {
            u = u1[at];
        } else {
            u = fn(x1, i, rr, cc, r, R);
            u1[at] = u;
        }
        const XT xv = x1[at];
        const XT y = xv + c * (xv - x0[at]);
        const XT jy = (XT(1) + c) * u - c * u0[at];
        const XT hv = h ? static_cast<XT>(h[i]) : XT(0);
        const XT x2 = xv * xv, y2 = y * y;
        add(0, x2 * x2);
        add(1, x2);
        add(2, xv * u);
        add(3, hv * xv);
        add(4, y2 * y2);
        add(5, y2);
        add(6, y * jy);
        add(7, hv * y);
        if constexpr (Fn::kGrid) {
            cc += kAThreads;
            while (cc >= Lc) {
                cc -= Lc;
                ++rr;
            }
        }
    }
    __shared__ double red[kAThreads / 32][kTerms];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < kTerms; ++k) {
        const double v = warp_sum(static_cast<double>(acc[k]) - static_cast<double>(cmp[k]));
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kTerms) {
        double t = 0.0;
        for (int w = 0; w < kAThreads / 32; ++w) t += red[w][threadIdx.x];
        partials[((static_cast<int64_t>(b) * R + r) * chunks + ch) * kTerms + threadIdx.x] = t;
    }
}

// (2) one block per (instance, replica) pair t = b R + r: the chunk partials
// are added by the block's threads in a fixed strided order and a fixed tree
constexpr int kDThreads = 128;
__global__ void __launch_bounds__(kDThreads)
adoch_decide(const double *__restrict__ partials, int n_inst, int R, int chunks,
             const double *__restrict__ alpha_tab, const double *__restrict__ beta_tab, int k, int q,
             double *__restrict__ hist, int *__restrict__ dec, int8_t *__restrict__ acc_out,
             double *__restrict__ H_out) {
    const int t = blockIdx.x;
    const int b = t / R;
    __shared__ double red[kDThreads][kTerms];
    double s[kTerms];
#pragma unroll
    for (int j = 0; j < kTerms; ++j) s[j] = 0.0;
    for (int ch = threadIdx.x; ch < chunks; ch += kDThreads)
#pragma unroll
        for (int j = 0; j < kTerms; ++j) s[j] += partials[(static_cast<int64_t>(t) * chunks + ch) * kTerms + j];
#pragma unroll
    for (int j = 0; j < kTerms; ++j) red[threadIdx.x][j] = s[j];
    __syncthreads();
    for (int w = kDThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int j = 0; j < kTerms; ++j) red[threadIdx.x][j] += red[threadIdx.x + w][j];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double a = alpha_tab[b], be = beta_tab[b];
    const double Hx = be / 4.0 * red[0][0] - a / 2.0 * red[0][1] - 0.5 * red[0][2] - red[0][3];
    const double Hy = be / 4.0 * red[0][4] - a / 2.0 * red[0][5] - 0.5 * red[0][6] - red[0][7];
    double *ht = hist + static_cast<int64_t>(t) * (q + 1);
    ht[k % (q + 1)] = Hx;
    double m = Hx;
    for (int j = (k > q ? k - q : 0); j <= k; ++j) m = fmax(m, ht[j % (q + 1)]);
    const int accept = Hy <= m ? 1 : 0;
    dec[t] = accept;
    if (acc_out) acc_out[static_cast<int64_t>(k) * n_inst * R + t] = static_cast<int8_t>(accept);
    if (H_out) H_out[static_cast<int64_t>(k) * n_inst * R + t] = Hx;
}

// (3) grid (chunks, R, n_inst): x^{k+1} = T(v^k)
template <typename XT>
__global__ void __launch_bounds__(kAThreads)
adoch_update(const XT *__restrict__ x1, const XT *__restrict__ x0, const XT *__restrict__ u1,
             const XT *__restrict__ u0, XT *__restrict__ x2, const XT *__restrict__ h,
             const int64_t *__restrict__ inst_off, int64_t n, int R, int chunks, XT c,
             const XT *__restrict__ alpha_tab, const XT *__restrict__ beta_tab, const int *__restrict__ dec) {
    const int ch = blockIdx.x, r = blockIdx.y, b = blockIdx.z;
    const int64_t lo = inst_off ? inst_off[b] : 0;
    const int64_t hi = inst_off ? inst_off[b + 1] : n;
    const int64_t len = hi - lo;
    const int64_t s0 = lo + len * ch / chunks, s1 = lo + len * (ch + 1) / chunks;
    const bool use_y = dec[b * R + r] != 0;
    const XT a = alpha_tab[b], bb = beta_tab[b];
    for (int64_t i = s0 + threadIdx.x; i < s1; i += kAThreads) {
        const int64_t at = i * R + r;
        const XT xv = x1[at], u = u1[at];
        XT v = xv, jv = u;
        if (use_y) {
            v = xv + c * (xv - x0[at]);
            jv = (XT(1) + c) * u - c * u0[at];
        }
        const XT hv = h ? h[i] : XT(0);
        x2[at] = acbrt(ascale(jv + a * v + hv, bb));
    }
}

int adoch_chunks(const ising_context *c, int R) {
    const int64_t pairs = static_cast<int64_t>(c->n_inst) * R;
    int64_t ch = (4LL * c->num_sms + pairs - 1) / pairs;
    const int64_t cap = (c->max_inst_n + kAThreads - 1) / kAThreads;
    if (ch > cap) ch = cap;
    if (ch < 1) ch = 1;
    if (ch > 65535) ch = 65535;
    return static_cast<int>(ch);
}

// ---- lattice fast path (R = 1, FP32, l_cols % 4 == 0, 16-byte aligned) ----
//
// Neither u^k nor u^{k-1} is stored: both passes recompute J x^k and
// J x^{k-1} from the two iterates (4 + 4 B per site) and the couplings (2 B),
// so a step reads 10 B per site twice and writes x^{k+1} once (24 B instead of
// 38 with the stored products). Layout as the DOCH lattice kernel: a CTA of
// 256 threads owns 1024 columns (4 per thread) and a strip of rows, keeps rows
// r-1, r, r+1 of both iterates in registers, takes horizontal neighbours by
// warp shuffles and the halos by lanes 0 and 31. The H terms of a row's four
// sites are summed plainly and then added with Kahan compensation; the update
// takes the prescaled fast cube root of the DOCH step kernels.

constexpr unsigned kFullMask = 0xffffffffu;

__device__ __forceinline__ float lat_byte(int v, int k) { return static_cast<float>((v << (24 - 8 * k)) >> 24); }

// u = right x_r + left x_l + down x_d + up x_u (the order of the lattice step kernels)
__device__ __forceinline__ float lat_sum(float wr, float xr, float wl, float xl, float wd, float xd, float wu,
                                         float xu) {
    return wr * xr + wl * xl + wd * xd + wu * xu;
}

// MODE 0: pass (H terms of step k); 1: update x^(k+1); 2: update and, from the new values, the H
// terms of step k+1 (x^T J x as twice the sum over right and down edges; the right edges of the
// last column of a warp and the down edges of the last row of a strip are left to
// adoch_lattice_bound)
template <int MODE>
__global__ void __launch_bounds__(kAThreads, 3)
adoch_lattice(const float *__restrict__ x1, const float *__restrict__ x0, float *__restrict__ x2,
              const int8_t *__restrict__ right, const int8_t *__restrict__ down, int Lr, int Lc, int tiles, int bpt,
              float c, float c_next, const float *__restrict__ alpha_tab, const float *__restrict__ zs_tab,
              const float *__restrict__ xsc_tab, const int *__restrict__ dec, double *__restrict__ partials) {
    constexpr bool UPDATE = MODE != 0;
    const int tile = blockIdx.x % tiles;
    const int part = blockIdx.x / tiles;
    const int r0 = static_cast<int>(static_cast<int64_t>(Lr) * part / bpt);
    const int r1 = static_cast<int>(static_cast<int64_t>(Lr) * (part + 1) / bpt);
    const int ncol4 = Lc >> 2;
    const int c4raw = tile * kAThreads + threadIdx.x;
    const bool active = c4raw < ncol4;
    const int c4 = c4raw % ncol4;
    const int col = c4 * 4;
    const int lane = threadIdx.x & 31;
    const bool is_l = lane == 0, is_r = lane == 31;
    const int hcol = is_l ? (col == 0 ? Lc - 1 : col - 1) : (col + 4 >= Lc ? 0 : col + 4);
    const int64_t n = static_cast<int64_t>(Lr) * Lc;
    auto ld4 = [&](const float *f, int64_t o) -> float4 { return __ldg(reinterpret_cast<const float4 *>(f + col + o)); };
    auto ldh = [&](const float *f, int64_t o) -> float { return (is_l || is_r) ? __ldg(f + hcol + o) : 0.f; };
    auto ldw = [&](const int8_t *p, int64_t o) -> int { return __ldg(reinterpret_cast<const int *>(p + col + o)); };
    const bool use_y = UPDATE ? dec[0] != 0 : false;
    const float alpha = UPDATE ? alpha_tab[0] : 0.f;
    const float zs = UPDATE ? zs_tab[0] : 0.f, xsc = UPDATE ? xsc_tab[0] : 0.f;  // prescaled cube root
    // FP32 sums with Kahan compensation: x^4, x^2, x u, y^4, y^2, y Jy
    float acc[6], cmp[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = cmp[k] = 0.f;
    auto add = [&](int k, float v) {
        const float y = v - cmp[k];
        const float t = acc[k] + y;
        cmp[k] = (t - acc[k]) - y;
        acc[k] = t;
    };
    if (r0 < r1) {
        int64_t o = static_cast<int64_t>(r0) * Lc;
        const int64_t ou = o == 0 ? n - Lc : o - Lc;
        int64_t od = o + Lc == n ? 0 : o + Lc;
        float4 au = ld4(x1, ou), am = ld4(x1, o), ad = ld4(x1, od);
        float4 bu = ld4(x0, ou), bm = ld4(x0, o), bd = ld4(x0, od);
        float ahm = ldh(x1, o), bhm = ldh(x0, o);
        float du[4];
        {
            const int w = ldw(down, ou);
#pragma unroll
            for (int q = 0; q < 4; ++q) du[q] = lat_byte(w, q);
        }
        int dm = ldw(down, o), rt = ldw(right, o);
        float wl_h = is_l ? static_cast<float>(__ldg(right + hcol + o)) : 0.f;
        float ahd = ldh(x1, od), bhd = ldh(x0, od);
        float pxn[4] = {0.f, 0.f, 0.f, 0.f}, pyn[4] = {0.f, 0.f, 0.f, 0.f};  // new values of the row above (MODE 2)
        for (int r = r0; r < r1; ++r) {
            const int64_t onn = od + Lc == n ? 0 : od + Lc;
            // loads of the next row, one row ahead
            float4 an = ad, bn = bd;
            int dn = dm, rn = rt;
            float wn = wl_h, ahn = ahd, bhn = bhd;
            if (r + 1 < r1) {
                an = ld4(x1, onn);
                bn = ld4(x0, onn);
                dn = ldw(down, od);
                rn = ldw(right, od);
                wn = is_l ? static_cast<float>(__ldg(right + hcol + od)) : 0.f;
                ahn = ldh(x1, onn);
                bhn = ldh(x0, onn);
            }
            float axl = __shfl_up_sync(kFullMask, am.w, 1), axr = __shfl_down_sync(kFullMask, am.x, 1);
            float bxl = __shfl_up_sync(kFullMask, bm.w, 1), bxr = __shfl_down_sync(kFullMask, bm.x, 1);
            const int rtl = __shfl_up_sync(kFullMask, rt, 1);
            float wleft = lat_byte(rtl, 3);
            if (is_l) {
                axl = ahm;
                bxl = bhm;
                wleft = wl_h;
            }
            if (is_r) {
                axr = ahm;
                bxr = bhm;
            }
            float wr[4], dd[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                wr[q] = lat_byte(rt, q);
                dd[q] = lat_byte(dm, q);
            }
            const float am_[4] = {am.x, am.y, am.z, am.w}, bm_[4] = {bm.x, bm.y, bm.z, bm.w};
            const float au_[4] = {au.x, au.y, au.z, au.w}, bu_[4] = {bu.x, bu.y, bu.z, bu.w};
            const float ad_[4] = {ad.x, ad.y, ad.z, ad.w}, bd_[4] = {bd.x, bd.y, bd.z, bd.w};
            float out[4], rs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // this row's four sites, then one compensated add
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float wlq = q == 0 ? wleft : wr[q - 1];
                const float axr_q = q == 3 ? axr : am_[q + 1], axl_q = q == 0 ? axl : am_[q - 1];
                const float bxr_q = q == 3 ? bxr : bm_[q + 1], bxl_q = q == 0 ? bxl : bm_[q - 1];
                const float u1 = lat_sum(wr[q], axr_q, wlq, axl_q, dd[q], ad_[q], du[q], au_[q]);
                const float u0 = lat_sum(wr[q], bxr_q, wlq, bxl_q, dd[q], bd_[q], du[q], bu_[q]);
                const float xv = am_[q];
                const float y = xv + c * (xv - bm_[q]);
                const float jy = (1.f + c) * u1 - c * u0;
                if (UPDATE) {
                    const float v = use_y ? y : xv, jv = use_y ? jy : u1;
                    out[q] = cbrt_pow2((jv + alpha * v) * zs) * xsc;
                } else {
                    const float x2v = xv * xv, y2 = y * y;
                    rs[0] += x2v * x2v;
                    rs[1] += x2v;
                    rs[2] += xv * u1;
                    rs[3] += y2 * y2;
                    rs[4] += y2;
                    rs[5] += y * jy;
                }
            }
            if (MODE == 2) {
                float yn[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    yn[q] = out[q] + c_next * (out[q] - am_[q]);
                    const float x2v = out[q] * out[q], y2 = yn[q] * yn[q];
                    rs[0] += x2v * x2v;
                    rs[1] += x2v;
                    rs[3] += y2 * y2;
                    rs[4] += y2;
                }
                // right edges of this row (the lane to the right holds the next four columns)
                const float xr_n = __shfl_down_sync(kFullMask, out[0], 1);
                const float yr_n = __shfl_down_sync(kFullMask, yn[0], 1);
                float ex = wr[0] * out[0] * out[1] + wr[1] * out[1] * out[2] + wr[2] * out[2] * out[3];
                float ey = wr[0] * yn[0] * yn[1] + wr[1] * yn[1] * yn[2] + wr[2] * yn[2] * yn[3];
                if (!is_r) {
                    ex += wr[3] * out[3] * xr_n;
                    ey += wr[3] * yn[3] * yr_n;
                }
                // down edges of the row above (its new values kept from the last pass of the walk)
                if (r > r0) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        ex += du[q] * pxn[q] * out[q];
                        ey += du[q] * pyn[q] * yn[q];
                    }
                }
                rs[2] = 2.f * ex;
                rs[5] = 2.f * ey;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    pxn[q] = out[q];
                    pyn[q] = yn[q];
                }
            }
            if (MODE != 1) {
#pragma unroll
                for (int k = 0; k < 6; ++k) add(k, rs[k]);
            }
            if (UPDATE && active) __stcs(reinterpret_cast<float4 *>(x2 + col + o), make_float4(out[0], out[1], out[2], out[3]));
            au = am;
            am = ad;
            ad = an;
            bu = bm;
            bm = bd;
            bd = bn;
            ahm = ahd;
            bhm = bhd;
            ahd = ahn;
            bhd = bhn;
            dm = dn;
            rt = rn;
            wl_h = wn;
#pragma unroll
            for (int q = 0; q < 4; ++q) du[q] = dd[q];
            o = od;
            od = onn;
        }
    }
    if (MODE == 1) return;
    // block sums in FP64 in a fixed order; inactive lanes (wrapped columns) add nothing
    __shared__ double red[kAThreads / 32][kTerms];
    const int warp = threadIdx.x >> 5;
    constexpr int kMap[6] = {0, 1, 2, 4, 5, 6};  // the terms of adoch_decide (no field on a lattice)
#pragma unroll
    for (int k = 0; k < kTerms; ++k) {
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < 6; ++j)
            if (kMap[j] == k && active) v = static_cast<double>(acc[j]) - static_cast<double>(cmp[j]);
        v = warp_sum(v);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kTerms) {
        double t = 0.0;
        for (int w = 0; w < kAThreads / 32; ++w) t += red[w][threadIdx.x];
        partials[static_cast<int64_t>(blockIdx.x) * kTerms + threadIdx.x] = t;
    }
}

// The edges adoch_lattice<2> leaves out: the right edge of every column c = 128 m + 127 (the last
// column of a warp) in every row, and the down edge of the last row of every strip, each adding
// 2 J x_i x_j of x^(k+1) and of y^(k+1) = x^(k+1) + c_next (x^(k+1) - x^k) to the H terms of step k+1.
__global__ void __launch_bounds__(kAThreads)
adoch_lattice_bound(const float *__restrict__ x1, const float *__restrict__ x2, const int8_t *__restrict__ right,
                    const int8_t *__restrict__ down, int Lr, int Lc, int bpt, float c_next,
                    double *__restrict__ partials) {
    const int nvb = Lc / 128;
    const int64_t nv = static_cast<int64_t>(Lr) * nvb;
    const int64_t total = nv + static_cast<int64_t>(bpt) * Lc;
    float ex = 0.f, ey = 0.f;
    for (int64_t idx = static_cast<int64_t>(blockIdx.x) * kAThreads + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * kAThreads) {
        int64_t a, b;
        float w;
        if (idx < nv) {
            const int64_t r = idx / nvb;
            const int64_t cc = (idx - r * nvb) * 128 + 127;
            const int64_t cn = cc + 1 == Lc ? 0 : cc + 1;
            a = r * Lc + cc;
            b = r * Lc + cn;
            w = static_cast<float>(right[a]);
        } else {
            const int64_t t = idx - nv;
            const int64_t p = t / Lc;
            const int64_t cc = t - p * Lc;
            const int64_t r = static_cast<int64_t>(Lr) * (p + 1) / bpt - 1;
            const int64_t rn = r + 1 == Lr ? 0 : r + 1;
            a = r * Lc + cc;
            b = rn * Lc + cc;
            w = static_cast<float>(down[a]);
        }
        const float xa = x2[a], xb = x2[b];
        const float ya = xa + c_next * (xa - x1[a]), yb = xb + c_next * (xb - x1[b]);
        ex += w * xa * xb;
        ey += w * ya * yb;
    }
    __shared__ double red[kAThreads / 32][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double vx = warp_sum(2.0 * static_cast<double>(ex)), vy = warp_sum(2.0 * static_cast<double>(ey));
    if (lane == 0) {
        red[warp][0] = vx;
        red[warp][1] = vy;
    }
    __syncthreads();
    if (threadIdx.x < kTerms) {
        double t = 0.0;
        if (threadIdx.x == 2 || threadIdx.x == 6)
            for (int w = 0; w < kAThreads / 32; ++w) t += red[w][threadIdx.x == 2 ? 0 : 1];
        partials[static_cast<int64_t>(blockIdx.x) * kTerms + threadIdx.x] = t;
    }
}

struct LatticeShape {
    int tiles = 0, bpt = 0, blocks = 0;
};

LatticeShape lattice_shape(const ising_context *c) {
    static int occ = 0;
    if (!occ && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adoch_lattice<2>, kAThreads, 0) !=
                     cudaSuccess || occ < 1))
        occ = 1;
    LatticeShape s;
    const int64_t ncol4 = c->l_cols / 4;
    s.tiles = static_cast<int>((ncol4 + kAThreads - 1) / kAThreads);
    int64_t bpt = static_cast<int64_t>(c->num_sms) * occ / s.tiles;
    if (bpt < 1) bpt = 1;
    if (bpt > c->l_rows) bpt = c->l_rows;
    s.bpt = static_cast<int>(bpt);
    s.blocks = static_cast<int>(bpt * s.tiles);
    return s;
}

bool lattice_fast_ok(const ising_context *c, const void *x, int R) {
    return c->format == ISING_FMT_TORUS2D && R == 1 && c->l_cols % 4 == 0 && c->l_rows >= 2 &&
           c->l_rows < (1LL << 31) && c->l_cols < (1LL << 31) && reinterpret_cast<uintptr_t>(x) % 16 == 0;
}

ising_status_t adoch_lattice_run(ising_context *c, float *x, const ParamTabs &p, int iters, int q, int8_t *acc_dev,
                                 double *H_dev, cudaStream_t st) {
    const int64_t count = c->n;
    const LatticeShape sh = lattice_shape(c);
    const int Lr = static_cast<int>(c->l_rows), Lc = static_cast<int>(c->l_cols);
    const int64_t bound_edges = static_cast<int64_t>(Lr) * (Lc / 128) + static_cast<int64_t>(sh.bpt) * Lc;
    const int nbb = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((bound_edges + kAThreads - 1) / kAThreads,
                                                                             2LL * c->num_sms)));
    auto al = [](size_t v) { return (v + 255) & ~static_cast<size_t>(255); };
    const size_t xb = al(sizeof(float) * count);
    const size_t pb = al(sizeof(double) * static_cast<size_t>(sh.blocks + nbb) * kTerms);
    const size_t hb = al(sizeof(double) * static_cast<size_t>(q + 1));
    const size_t db = al(sizeof(int));
    DOCH_CHECK(c->ckpt.ensure(2 * xb + pb + hb + db));
    unsigned char *base = c->ckpt.as<unsigned char>();
    float *x1 = x, *x0 = reinterpret_cast<float *>(base), *x2 = reinterpret_cast<float *>(base + xb);
    double *part = reinterpret_cast<double *>(base + 2 * xb);
    double *hist = reinterpret_cast<double *>(base + 2 * xb + pb);
    int *dec = reinterpret_cast<int *>(base + 2 * xb + pb + hb);
    DOCH_CUDA(cudaMemcpyAsync(x0, x1, sizeof(float) * count, cudaMemcpyDeviceToDevice, st));  // x^{-1} := x^0
    if (iters <= 0) return ISING_OK;
    // step 0: its H terms from a pass (y^0 = x^0)
    adoch_lattice<0><<<sh.blocks, kAThreads, 0, st>>>(x1, x0, nullptr, c->right, c->down, Lr, Lc, sh.tiles, sh.bpt,
                                                     0.f, 0.f, nullptr, nullptr, nullptr, nullptr, part);
    DOCH_CUDA(cudaGetLastError());
    adoch_decide<<<1, kDThreads, 0, st>>>(part, 1, 1, sh.blocks, p.alpha_d, p.beta_d, 0, q, hist, dec, acc_dev, H_dev);
    DOCH_CUDA(cudaGetLastError());
    auto t_after = [](double t) { return (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0; };
    double t = 1.0;  // t_k
    for (int k = 0; k < iters; ++k) {
        const double t1 = t_after(t), t2 = t_after(t1);  // t_(k+1), t_(k+2)
        const float ck = static_cast<float>(k >= 1 ? (t - 1.0) / t1 : 0.0);
        const float cn = static_cast<float>((t1 - 1.0) / t2);  // c_(k+1)
        if (k + 1 < iters) {
            // x^(k+1) and, from it, the H terms of step k+1
            adoch_lattice<2><<<sh.blocks, kAThreads, 0, st>>>(x1, x0, x2, c->right, c->down, Lr, Lc, sh.tiles,
                                                             sh.bpt, ck, cn, p.alpha_f, p.zscale_f, p.xscale_f, dec,
                                                             part);
            DOCH_CUDA(cudaGetLastError());
            adoch_lattice_bound<<<nbb, kAThreads, 0, st>>>(x1, x2, c->right, c->down, Lr, Lc, sh.bpt, cn,
                                                          part + static_cast<size_t>(sh.blocks) * kTerms);
            DOCH_CUDA(cudaGetLastError());
        } else {
            adoch_lattice<1><<<sh.blocks, kAThreads, 0, st>>>(x1, x0, x2, c->right, c->down, Lr, Lc, sh.tiles,
                                                             sh.bpt, ck, 0.f, p.alpha_f, p.zscale_f, p.xscale_f, dec,
                                                             nullptr);
            DOCH_CUDA(cudaGetLastError());
        }
        float *tx = x0;  // x^{k-1} <- x^k <- x^{k+1}
        x0 = x1;
        x1 = x2;
        x2 = tx;
        t = t1;
        if (k + 1 < iters) {
            adoch_decide<<<1, kDThreads, 0, st>>>(part, 1, 1, sh.blocks + nbb, p.alpha_d, p.beta_d, k + 1, q, hist,
                                                  dec, acc_dev, H_dev);
            DOCH_CUDA(cudaGetLastError());
        }
    }
    if (x1 != x) DOCH_CUDA(cudaMemcpyAsync(x, x1, sizeof(float) * count, cudaMemcpyDeviceToDevice, st));
    return ISING_OK;
}

template <typename XT, typename Fn>
ising_status_t adoch_run(ising_context *c, const Fn &fn, XT *x, int R, const ParamTabs &p, const XT *h_x,
                         int iters, int q, int8_t *acc_dev, double *H_dev, cudaStream_t st) {
    const int64_t count = c->n * R;
    const int pairs = c->n_inst * R;
    const int chunks = adoch_chunks(c, R);
    auto al = [](size_t v) { return (v + 255) & ~static_cast<size_t>(255); };
    const size_t xb = al(sizeof(XT) * count);
    const size_t pb = al(sizeof(double) * static_cast<size_t>(pairs) * chunks * kTerms);
    const size_t hb = al(sizeof(double) * static_cast<size_t>(pairs) * (q + 1));
    const size_t db = al(sizeof(int) * static_cast<size_t>(pairs));
    DOCH_CHECK(c->ckpt.ensure(4 * xb + pb + hb + db));
    unsigned char *base = c->ckpt.as<unsigned char>();
    XT *bx[3] = {x, reinterpret_cast<XT *>(base), reinterpret_cast<XT *>(base + xb)};  // x^k, x^{k-1}, x^{k+1}
    XT *bu[2] = {reinterpret_cast<XT *>(base + 2 * xb), reinterpret_cast<XT *>(base + 3 * xb)};  // u^{k-1}, u^k
    double *part = reinterpret_cast<double *>(base + 4 * xb);
    double *hist = reinterpret_cast<double *>(base + 4 * xb + pb);
    int *dec = reinterpret_cast<int *>(base + 4 * xb + pb + hb);
    XT *x1 = bx[0], *x0 = bx[1], *x2 = bx[2], *u0 = bu[0], *u1 = bu[1];
    DOCH_CUDA(cudaMemcpyAsync(x0, x1, sizeof(XT) * count, cudaMemcpyDeviceToDevice, st));  // x^{-1} := x^0
    DOCH_CUDA(cudaMemsetAsync(u0, 0, sizeof(XT) * count, st));
    const XT *alpha = nullptr, *beta = nullptr;
    if constexpr (sizeof(XT) == 4) {
        alpha = p.alpha_f;
        beta = p.inv_beta_f;
    } else {
        alpha = p.alpha_d;
        beta = p.beta_d;
    }
    const int64_t *off = c->n_inst > 1 ? c->inst_off : nullptr;
    const double *h_d = c->has_h ? c->h_f64 : nullptr;
    dim3 grid(static_cast<unsigned>(chunks), static_cast<unsigned>(R), static_cast<unsigned>(c->n_inst));
    double t = 1.0;
    for (int k = 0; k < iters; ++k) {
        const double t_next = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
        const XT ck = static_cast<XT>(k >= 1 ? (t - 1.0) / t_next : 0.0);
        if constexpr (Fn::kStored) {
            if constexpr (sizeof(XT) == 4) DOCH_CHECK(proc_product(c, x1, u1, R, st));
        }
        adoch_pass<XT, Fn><<<grid, kAThreads, 0, st>>>(fn, x1, x0, u0, u1, h_d, off, c->n, R, chunks, ck, part);
        DOCH_CUDA(cudaGetLastError());
        adoch_decide<<<pairs, kDThreads, 0, st>>>(part, c->n_inst, R, chunks, p.alpha_d, p.beta_d, k, q, hist,
                                                  dec, acc_dev, H_dev);
        DOCH_CUDA(cudaGetLastError());
        adoch_update<XT><<<grid, kAThreads, 0, st>>>(x1, x0, u1, u0, x2, h_x, off, c->n, R, chunks, ck, alpha,
                                                     beta, dec);
        DOCH_CUDA(cudaGetLastError());
        // rotate: x^{k-1} <- x^k <- x^{k+1}, u^{k-1} <- u^k
        XT *tx = x0;
        x0 = x1;
        x1 = x2;
        x2 = tx;
        std::swap(u0, u1);
        t = t_next;
    }
    if (x1 != x) DOCH_CUDA(cudaMemcpyAsync(x, x1, sizeof(XT) * count, cudaMemcpyDeviceToDevice, st));
    return ISING_OK;
}

template <typename XT>
ising_status_t adoch_dispatch(ising_context *c, XT *x, int R, const ParamTabs &p, const XT *h_x, int iters,
                              int q, int8_t *acc_dev, double *H_dev, cudaStream_t st) {
    if (c->format == ISING_FMT_TORUS2D)
        return adoch_run<XT>(c, TorusProduct<XT>{c->right, c->down, c->l_rows, c->l_cols}, x, R, p, h_x, iters,
                             q, acc_dev, H_dev, st);
    if (c->format == ISING_FMT_PROCEDURAL) {
        if constexpr (sizeof(XT) == 4)
            return adoch_run<XT>(c, ProcProduct{}, x, R, p, h_x, iters, q, acc_dev, H_dev, st);
        else
            return fail(ISING_ERR_INVALID_ARG, "PROCEDURAL iterates are F32");
    }
    if (c->format != ISING_FMT_CSR)
        return fail(ISING_ERR_UNSUPPORTED, "ADOCH runs on CSR, TORUS2D or PROCEDURAL couplings");
    switch (c->jtype) {
        case ISING_I8:
            return adoch_run<XT>(c, CsrProduct<XT, int8_t>{c->row_ptr, c->col, static_cast<const int8_t *>(c->val)},
                                 x, R, p, h_x, iters, q, acc_dev, H_dev, st);
        case ISING_I32:
            return adoch_run<XT>(c, CsrProduct<XT, int32_t>{c->row_ptr, c->col, static_cast<const int32_t *>(c->val)},
                                 x, R, p, h_x, iters, q, acc_dev, H_dev, st);
        case ISING_F32:
            return adoch_run<XT>(c, CsrProduct<XT, float>{c->row_ptr, c->col, static_cast<const float *>(c->val)},
                                 x, R, p, h_x, iters, q, acc_dev, H_dev, st);
        case ISING_F64:
            return adoch_run<XT>(c, CsrProduct<XT, double>{c->row_ptr, c->col, static_cast<const double *>(c->val)},
                                 x, R, p, h_x, iters, q, acc_dev, H_dev, st);
        default: return fail(ISING_ERR_UNSUPPORTED, "CSR value type not supported on the device");
    }
}

}  // namespace

ising_status_t adoch_iterate(ising_context *c, void *x, int xtype, int R, const ParamTabs &p, int iters, int q,
                             int8_t *acc_dev, double *H_dev, cudaStream_t st) {
    if (xtype == ISING_F32 && lattice_fast_ok(c, x, R))
        return adoch_lattice_run(c, static_cast<float *>(x), p, iters, q, acc_dev, H_dev, st);
    if (xtype == ISING_F32)
        return adoch_dispatch<float>(c, static_cast<float *>(x), R, p, c->has_h ? c->h_f32 : nullptr, iters, q,
                                     acc_dev, H_dev, st);
    if (xtype == ISING_F64)
        return adoch_dispatch<double>(c, static_cast<double *>(x), R, p, c->has_h ? c->h_f64 : nullptr, iters, q,
                                      acc_dev, H_dev, st);
    return fail(ISING_ERR_INVALID_ARG, "ADOCH iterates must be F32 or F64");
}

}  // namespace doch
