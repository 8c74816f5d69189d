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
// Cube root: cbrt(z / beta) = sign(z) exp2( log2|z| / 3 + c3 ), c3 = log2(1/beta) / 3
// from the host, with the hardware base-2 logarithm/exponential approximations
// (PTX lg2.approx, ex2.approx): cbrt_log of cbrt.cuh, one FMA between the two
// (relative error within 2^-21 + (0.25 |log2 z| + 0.75 |l|) 2^-24, l the
// exponent; near the attractor both logarithms are small).
#include <cmath>

#include "cbrt.cuh"
#include "hamsum.cuh"
#include "internal.cuh"

namespace doch {
namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

// Signed byte k (0..3) of a packed word of four int8, as a float, without an
// integer-to-float conversion: flipping the sign bit maps s to s + 128 in
// 0..255, which is placed in the low mantissa byte of 2^23; subtracting
// 2^23 + 128 leaves s exactly.
__device__ __forceinline__ float sbyte(int v, int k) {
    const unsigned b = static_cast<unsigned>(v) ^ 0x80808080u;
    return __uint_as_float(__byte_perm(b, 0x4B000000u, 0x7540u | static_cast<unsigned>(k))) - 8388736.0f;
}
// The same value by shifts and a conversion: fewer live constants, which the
// 40-register single-step kernel needs.
__device__ __forceinline__ float sbyte_cvt(int v, int k) {
    return static_cast<float>((v << (24 - 8 * k)) >> 24);
}

// One site of Eq. FPE: u = sum over the four neighbours (right, left, down,
// up -- always in this order), then cbrt((u + alpha x) / beta). Both stencil
// kernels use these two functions, so a fused two-step pass reproduces two
// single steps exactly.
__device__ __forceinline__ float site_sum(float wr, float xr, float wl, float xl, float wd, float xd,
                                          float wu, float xu) {
    return wr * xr + wl * xl + wd * xd + wu * xu;
}

__device__ __forceinline__ float site_new(float u, float x, float alpha, float c3) {
    return cbrt_log(u + alpha * x, c3);
}

// four consecutive sites c..c+3 of one row: xm row values, xl/xr the values
// left of c and right of c+3, xu/xd the rows above/below, rt the packed right
// couplings of the row, wleft the coupling to column c-1, dd/du the down
// couplings of this row / of the row above (as floats)
__device__ __forceinline__ float4 row4_new_w(float4 xm, float xl, float xr, float4 xu, float4 xd,
                                             const float (&wr)[4], float wleft, const float (&dd)[4],
                                             const float (&du)[4], float alpha, float c3) {
    const float w0 = wr[0], w1 = wr[1], w2 = wr[2], w3 = wr[3];
    float4 out;
    out.x = site_new(site_sum(w0, xm.y, wleft, xl, dd[0], xd.x, du[0], xu.x), xm.x, alpha, c3);
    out.y = site_new(site_sum(w1, xm.z, w0, xm.x, dd[1], xd.y, du[1], xu.y), xm.y, alpha, c3);
    out.z = site_new(site_sum(w2, xm.w, w1, xm.y, dd[2], xd.z, du[2], xu.z), xm.z, alpha, c3);
    out.w = site_new(site_sum(w3, xr, w2, xm.z, dd[3], xd.w, du[3], xu.w), xm.w, alpha, c3);
    return out;
}

__device__ __forceinline__ void unpack4(int v, float (&f)[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) f[k] = sbyte(v, k);
}
__device__ __forceinline__ void unpack4_cvt(int v, float (&f)[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) f[k] = sbyte_cvt(v, k);
}

__device__ __forceinline__ float4 row4_new(float4 xm, float xl, float xr, float4 xu, float4 xd, int rt,
                                           float wleft, const float (&dd)[4], const float (&du)[4], float alpha,
                                           float c3) {
    float wr[4];
    unpack4_cvt(rt, wr);
    return row4_new_w(xm, xl, xr, xu, xd, wr, wleft, dd, du, alpha, c3);
}

// u of four consecutive sites (the sums row4_new_w feeds to site_new)
__device__ __forceinline__ float4 row4_u(float4 xm, float xl, float xr, float4 xu, float4 xd, const float (&wr)[4],
                                         float wleft, const float (&dd)[4], const float (&du)[4]) {
    float4 u;
    u.x = site_sum(wr[0], xm.y, wleft, xl, dd[0], xd.x, du[0], xu.x);
    u.y = site_sum(wr[1], xm.z, wr[0], xm.x, dd[1], xd.y, du[1], xu.y);
    u.z = site_sum(wr[2], xm.w, wr[1], xm.y, dd[2], xd.z, du[2], xu.z);
    u.w = site_sum(wr[3], xr, wr[2], xm.z, dd[3], xd.w, du[3], xu.w);
    return u;
}

// block sum of the fused H monitor's three lattice terms into hpart[block][4]
// (x^4, x^2, x u; no field on a lattice), warps and threads in a fixed order
__device__ __forceinline__ void torus_ham_block(const HamSum<float> (&hs)[3], double *__restrict__ hpart) {
    __shared__ double red[kThreads / 32][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        double v = hs[m].value();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) red[warp][m] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        if (threadIdx.x < 3)
            for (int w = 0; w < kThreads / 32; ++w) t += red[w][threadIdx.x];
        hpart[static_cast<int64_t>(blockIdx.x) * 4 + threadIdx.x] = t;
    }
}

// 40 registers: 6 CTAs (1536 threads) per SM keep enough loads in flight.
// TRACE: also the terms of H(x_in) (Eq. Hamilton) for the fused monitor, from
// the same u = J x_in (same results for x_out).
template <bool TRACE>
__global__ void __launch_bounds__(kThreads, TRACE ? 4 : 6)
torus_f32_r1_vec4(const float *__restrict__ xi, float *__restrict__ xo,
                  const int8_t *__restrict__ right, const int8_t *__restrict__ down, int Lr, int Lc,
                  int tiles, int bpt, float alpha, float c3, double *__restrict__ hpart) {
    const int tile = blockIdx.x % tiles;
    const int part = blockIdx.x / tiles;
    const int r0 = static_cast<int>(static_cast<int64_t>(Lr) * part / bpt);
    const int r1 = static_cast<int>(static_cast<int64_t>(Lr) * (part + 1) / bpt);
    if (r0 >= r1) {  // uniform over the block
        if constexpr (TRACE) {
            const HamSum<float> none[3];
            torus_ham_block(none, hpart);
        }
        return;
    }
    HamSum<float> hs[TRACE ? 3 : 1];

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
    float du[4];
    unpack4_cvt(ldw(dc, ou), du);
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
        float wleft = sbyte_cvt(rtl, 3);
        if (is_l) { xl = hm; wleft = wl; }
        if (is_r) xr = hm;

        float dd[4];
        unpack4_cvt(dm, dd);
        if constexpr (TRACE) {
            float wr[4];
            unpack4_cvt(rt, wr);
            const float4 u = row4_u(xm, xl, xr, xu, xd, wr, wleft, dd, du);
            float4 out;
            out.x = site_new(u.x, xm.x, alpha, c3);
            out.y = site_new(u.y, xm.y, alpha, c3);
            out.z = site_new(u.z, xm.z, alpha, c3);
            out.w = site_new(u.w, xm.w, alpha, c3);
            if (active) {
                __stcs(reinterpret_cast<float4 *>(oc + o), out);
                const float xv[4] = {xm.x, xm.y, xm.z, xm.w}, uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float x2 = xv[q] * xv[q];
                    hs[0].add(x2 * x2);
                    hs[1].add(x2);
                    hs[2].add(xv[q] * uv[q]);
                }
            }
        } else {
            const float4 out = row4_new(xm, xl, xr, xu, xd, rt, wleft, dd, du, alpha, c3);
            if (active) __stcs(reinterpret_cast<float4 *>(oc + o), out);
        }

        xu = xm; xm = xd; hm = hd;
#pragma unroll
        for (int q = 0; q < 4; ++q) du[q] = dd[q];
        xd = xn; hd = hn; dm = dn; rt = rn; wl = wn;
        o = on; od = onn;
    }
    if constexpr (TRACE) torus_ham_block(hs, hpart);
}


__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Output column groups per warp of the two-step kernel: lanes 1..30. Lanes 0
// and 31 load the groups on either side and compute with the rest of the
// warp; their intermediate values at their three inner columns are exact
// (two steps need a halo of two columns, a lane holds four), their outer
// columns are wrong and never used, and they write nothing.
constexpr int kSeg = 30;

// Per-thread shared-memory ring of the two-step kernel: D slots, each holding
// one lattice row's loads of every thread (its float4 of x and its two packed
// coupling words).
template <int D>
struct T2Ring {
    float4 x[D][kThreads];
    int rw[D][kThreads];
    int dw[D][kThreads];
};

// Two DOCH steps per pass (temporal blocking): x^(k+2) from x^(k), with the
// intermediate x^(k+1) held in registers. Every warp is an independent unit
// owning kSeg column groups of 4 columns and a strip of rows [r0, r1); it
// walks down the strip computing y = x^(k+1) for row r from x rows r-1..r+1,
// then z = x^(k+2) for row r-1 from y rows r-2..r, reading x rows
// r0-2 .. r1+1. Loads are staged D rows ahead by cp.async into a per-thread
// ring in shared memory (no registers held by the prefetch); each thread reads
// only the slots it filled, so cp.async.wait_group is the only
// synchronisation. HBM traffic per site and step is about half that of the
// single-step kernel (the halo lanes add 2/30 to the reads); every site is
// computed by the same helpers, so the pass equals two single steps bit for
// bit.
template <int D>
__global__ void __launch_bounds__(kThreads, 3)
torus_f32_r1_vec4_t2(const float *__restrict__ xi, float *__restrict__ xo,
                     const int8_t *__restrict__ right, const int8_t *__restrict__ down, int Lr, int Lc,
                     int segs, int bpt, float alpha1, float alpha2, float c3) {
    extern __shared__ __align__(16) unsigned char t2_smem[];
    T2Ring<D> &ring = *reinterpret_cast<T2Ring<D> *>(t2_smem);
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = blockIdx.x * (kThreads / 32) + (t >> 5);
    const int seg = warp % segs;
    const int part = warp / segs;
    if (part >= bpt) return;  // uniform over the warp; nothing below synchronises the block
    const int r0 = static_cast<int>(static_cast<int64_t>(Lr) * part / bpt);
    const int r1 = static_cast<int>(static_cast<int64_t>(Lr) * (part + 1) / bpt);
    if (r0 >= r1) return;  // uniform over the warp

    // column group of this lane, wrapped periodically so that consecutive
    // lanes always hold consecutive groups of the torus
    const int ncol4 = Lc >> 2;
    const int g = seg * kSeg + lane - 1;
    const bool writes = lane >= 1 && lane <= kSeg && g < ncol4;
    const int c = (((g % ncol4) + ncol4) % ncol4) * 4;
    const int64_t n = static_cast<int64_t>(Lr) * Lc;
    const float *xc = xi + c;
    const int8_t *rc = right + c, *dc = down + c;
    auto wrap_up = [&](int64_t o) { return o == 0 ? n - Lc : o - Lc; };
    auto wrap_dn = [&](int64_t o) { o += Lc; return o == n ? int64_t(0) : o; };
    auto issue = [&](unsigned s, int64_t o) {
        cp_async16(&ring.x[s][t], xc + o);
        cp_async4(&ring.rw[s][t], rc + o);
        cp_async4(&ring.dw[s][t], dc + o);
    };

    // rows r0-2 and r0-1 are read directly; the ring then carries rows r0 .. r1+1
    const int64_t o0 = static_cast<int64_t>(r0) * Lc;
    const int64_t om = wrap_up(o0), omm = wrap_up(om);
    float4 xu = __ldg(reinterpret_cast<const float4 *>(xc + omm));
    float4 xm = __ldg(reinterpret_cast<const float4 *>(xc + om));
    float du[4];
    unpack4(__ldg(reinterpret_cast<const int *>(dc + omm)), du);
    int dm = __ldg(reinterpret_cast<const int *>(dc + om));
    int rt = __ldg(reinterpret_cast<const int *>(rc + om));
    const int rows = r1 - r0 + 2;  // ring bundles: rows r0 .. r1+1
    int64_t oi = o0;                // offset of the next row to stage
#pragma unroll
    for (int q = 0; q < D; ++q) {
        if (q < rows) {
            issue(q, oi);
            oi = wrap_dn(oi);
        }
        cp_async_commit();
    }
    int64_t os = o0;  // offset of the next output row of step 2 (rows r0, r0+1, ...)
    float4 ya = make_float4(0.f, 0.f, 0.f, 0.f), yb = ya;
    float wr_p[4] = {0.f, 0.f, 0.f, 0.f};
    float du_p[4] = {0.f, 0.f, 0.f, 0.f};

    // iteration i handles step-1 row r = r0-1+i and step-2 row r-1; unrolled
    // by 3 so the two-row histories (x, y, down couplings) rotate by renaming
#pragma unroll 3
    for (int i = 0; i < rows; ++i) {
        // the bundle of row r+1 (ring index i) has landed: older groups complete first
        cp_async_wait<D - 1>();
        const unsigned s = static_cast<unsigned>(i) % D;
        const float4 xd = ring.x[s][t];
        const int rt_n = ring.rw[s][t], dm_n = ring.dw[s][t];
        // every read of slot s is above; refill it with ring index i+D
        if (i + D < rows) {
            issue(s, oi);
            oi = wrap_dn(oi);
        }
        cp_async_commit();

        // ---- step 1: y row r
        float wr[4], dd[4];
        unpack4(rt, wr);
        unpack4(dm, dd);
        const float xl = __shfl_up_sync(kFull, xm.w, 1);
        const float xr = __shfl_down_sync(kFull, xm.x, 1);
        const float wleft = __shfl_up_sync(kFull, wr[3], 1);
        const float4 yc = row4_new_w(xm, xl, xr, xu, xd, wr, wleft, dd, du, alpha1, c3);

        // ---- step 2: z row r-1 from y rows r-2, r-1, r (once y row r0-1 is two rows back)
        if (i > 1) {
            const float yl = __shfl_up_sync(kFull, yb.w, 1);
            const float yr = __shfl_down_sync(kFull, yb.x, 1);
            const float wleftp = __shfl_up_sync(kFull, wr_p[3], 1);
            const float4 z = row4_new_w(yb, yl, yr, ya, yc, wr_p, wleftp, du, du_p, alpha2, c3);
            if (writes) __stcs(reinterpret_cast<float4 *>(xo + c + os), z);
            os = wrap_dn(os);
        }

        // ---- rotate
        ya = yb; yb = yc;
#pragma unroll
        for (int q = 0; q < 4; ++q) { wr_p[q] = wr[q]; du_p[q] = du[q]; du[q] = dd[q]; }
        xu = xm; xm = xd;
        dm = dm_n; rt = rt_n;
    }
    cp_async_wait<0>();
}

// Three DOCH steps per pass: x^(k+3) from x^(k), the intermediate iterates of
// steps k+1 and k+2 held in registers (two rows each). The layout is that of
// the two-step kernel: a warp owns kSeg column groups (lanes 1..30; lanes 0 and
// 31 hold the groups on either side, whose three inner columns stay exact for
// three steps, since a lane holds four columns) and a strip of rows [r0, r1).
// Iteration i computes level 1 (step k+1) for row r = r0-2+i from x rows
// r-1..r+1, level 2 for row r-1 from level-1 rows r-2..r, and level 3 for row
// r-2 from level-2 rows r-3..r-1, written out; x rows r0-3 .. r1+2 are read.
// The couplings of a row are unpacked once and kept for the three rows of
// history the levels need. Same helpers as the single step: the pass equals
// three single steps bit for bit.
template <int D>
__global__ void __launch_bounds__(kThreads, 2)
torus_f32_r1_vec4_t3(const float *__restrict__ xi, float *__restrict__ xo,
                     const int8_t *__restrict__ right, const int8_t *__restrict__ down, int Lr, int Lc,
                     int segs, int bpt, float alpha1, float alpha2, float alpha3, float c3) {
    extern __shared__ __align__(16) unsigned char t3_smem[];
    T2Ring<D> &ring = *reinterpret_cast<T2Ring<D> *>(t3_smem);
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = blockIdx.x * (kThreads / 32) + (t >> 5);
    const int seg = warp % segs;
    const int part = warp / segs;
    if (part >= bpt) return;  // uniform over the warp; nothing below synchronises the block
    const int r0 = static_cast<int>(static_cast<int64_t>(Lr) * part / bpt);
    const int r1 = static_cast<int>(static_cast<int64_t>(Lr) * (part + 1) / bpt);
    if (r0 >= r1) return;  // uniform over the warp

    const int ncol4 = Lc >> 2;
    const int g = seg * kSeg + lane - 1;
    const bool writes = lane >= 1 && lane <= kSeg && g < ncol4;
    const int c = (((g % ncol4) + ncol4) % ncol4) * 4;
    const int64_t n = static_cast<int64_t>(Lr) * Lc;
    const float *xc = xi + c;
    const int8_t *rc = right + c, *dc = down + c;
    auto wrap_up = [&](int64_t o) { return o == 0 ? n - Lc : o - Lc; };
    auto wrap_dn = [&](int64_t o) { o += Lc; return o == n ? int64_t(0) : o; };
    auto issue = [&](unsigned s, int64_t o) {
        cp_async16(&ring.x[s][t], xc + o);
        cp_async4(&ring.rw[s][t], rc + o);
        cp_async4(&ring.dw[s][t], dc + o);
    };

    // rows r0-3 and r0-2 are read directly; the ring then carries rows r0-1 .. r1+2
    const int64_t o0 = static_cast<int64_t>(r0) * Lc;
    const int64_t om = wrap_up(o0), omm = wrap_up(om), ommm = wrap_up(omm);
    float4 xu = __ldg(reinterpret_cast<const float4 *>(xc + ommm));
    float4 xm = __ldg(reinterpret_cast<const float4 *>(xc + omm));
    float d1[4], d2[4] = {0.f, 0.f, 0.f, 0.f}, d3[4] = {0.f, 0.f, 0.f, 0.f};  // down couplings of rows r-1, r-2, r-3
    unpack4(__ldg(reinterpret_cast<const int *>(dc + ommm)), d1);
    int dm = __ldg(reinterpret_cast<const int *>(dc + omm));
    int rt = __ldg(reinterpret_cast<const int *>(rc + omm));
    const int rows = r1 - r0 + 4;  // ring bundles: rows r0-1 .. r1+2
    int64_t oi = om;               // offset of the next row to stage
#pragma unroll
    for (int q = 0; q < D; ++q) {
        if (q < rows) {
            issue(q, oi);
            oi = wrap_dn(oi);
        }
        cp_async_commit();
    }
    int64_t os = o0;  // offset of the next output row (rows r0, r0+1, ...)
    float4 ya1 = make_float4(0.f, 0.f, 0.f, 0.f), yb1 = ya1, ya2 = ya1, yb2 = ya1;
    float w1[4] = {0.f, 0.f, 0.f, 0.f}, w2[4] = {0.f, 0.f, 0.f, 0.f};  // right couplings of rows r-1, r-2

    for (int i = 0; i < rows; ++i) {
        cp_async_wait<D - 1>();
        const unsigned s = static_cast<unsigned>(i) % D;
        const float4 xd = ring.x[s][t];
        const int rt_n = ring.rw[s][t], dm_n = ring.dw[s][t];
        if (i + D < rows) {
            issue(s, oi);
            oi = wrap_dn(oi);
        }
        cp_async_commit();

        // ---- level 1: row r
        float w0[4], d0[4];
        unpack4(rt, w0);
        unpack4(dm, d0);
        const float xl = __shfl_up_sync(kFull, xm.w, 1);
        const float xr = __shfl_down_sync(kFull, xm.x, 1);
        const float wl0 = __shfl_up_sync(kFull, w0[3], 1);
        const float4 y1 = row4_new_w(xm, xl, xr, xu, xd, w0, wl0, d0, d1, alpha1, c3);

        // ---- level 2: row r-1 from level-1 rows r-2, r-1, r
        float4 y2 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i >= 2) {
            const float yl = __shfl_up_sync(kFull, yb1.w, 1);
            const float yr = __shfl_down_sync(kFull, yb1.x, 1);
            const float wl1 = __shfl_up_sync(kFull, w1[3], 1);
            y2 = row4_new_w(yb1, yl, yr, ya1, y1, w1, wl1, d1, d2, alpha2, c3);
        }
        // ---- level 3: row r-2 from level-2 rows r-3, r-2, r-1, written out
        if (i >= 4) {
            const float zl = __shfl_up_sync(kFull, yb2.w, 1);
            const float zr = __shfl_down_sync(kFull, yb2.x, 1);
            const float wl2 = __shfl_up_sync(kFull, w2[3], 1);
            const float4 z = row4_new_w(yb2, zl, zr, ya2, y2, w2, wl2, d2, d3, alpha3, c3);
            if (writes) __stcs(reinterpret_cast<float4 *>(xo + c + os), z);
            os = wrap_dn(os);
        }

        // ---- rotate the histories by one row
        ya1 = yb1; yb1 = y1;
        ya2 = yb2; yb2 = y2;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            w2[q] = w1[q]; w1[q] = w0[q];
            d3[q] = d2[q]; d2[q] = d1[q]; d1[q] = d0[q];
        }
        xu = xm; xm = xd;
        dm = dm_n; rt = rt_n;
    }
    cp_async_wait<0>();
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

// ring depth of the two-step kernel: rows staged ahead of the one in use
constexpr int kT2Depth = 4;
constexpr size_t kT2Smem = sizeof(T2Ring<kT2Depth>);

int t2_blocks_per_sm() {
    static int occ = 0;
    if (!occ) {
        if (cudaFuncSetAttribute(torus_f32_r1_vec4_t2<kT2Depth>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kT2Smem)) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, torus_f32_r1_vec4_t2<kT2Depth>, kThreads,
                                                          kT2Smem) != cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    return occ;
}

int t3_blocks_per_sm() {
    static int occ = 0;
    if (!occ) {
        if (cudaFuncSetAttribute(torus_f32_r1_vec4_t3<kT2Depth>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kT2Smem)) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, torus_f32_r1_vec4_t3<kT2Depth>, kThreads,
                                                          kT2Smem) != cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    return occ;
}

int vec4_blocks_per_sm() {
    static int occ = 0;
    if (!occ) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, torus_f32_r1_vec4<false>, kThreads, 0) !=
                cudaSuccess || occ < 1)
            occ = 1;
    }
    return occ;
}

// launch shape of the single-step fast kernel: column tiles of 1024, bpt row strips per tile
struct Vec4Shape {
    int tiles = 0;
    int64_t bpt = 0;
    int64_t blocks() const { return bpt * tiles; }
};

Vec4Shape vec4_shape(const ising_context *c) {
    const int64_t Lr = c->l_rows, ncol4 = c->l_cols / 4;
    Vec4Shape v;
    v.tiles = static_cast<int>((ncol4 + kThreads - 1) / kThreads);
    const int64_t slots = static_cast<int64_t>(c->num_sms) * vec4_blocks_per_sm();
    v.bpt = slots / v.tiles;
    if (v.bpt < 1) v.bpt = 1;
    if (v.bpt > Lr / 4) v.bpt = Lr / 4 > 0 ? Lr / 4 : 1;
    return v;
}

bool vec4_ok(const ising_context *c, const float *x_in, const float *x_out, int R) {
    const bool aligned = (reinterpret_cast<uintptr_t>(x_in) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(x_out) % 16 == 0);
    return R == 1 && c->l_cols % 4 == 0 && aligned && c->l_rows < (1LL << 31) && c->l_cols < (1LL << 31);
}

}  // namespace

// the lattice cube root's offset c3 = log2(1 / beta) / 3 (cbrt_log)
static float lattice_c3(double inv_beta) { return static_cast<float>(std::log2(inv_beta) / 3.0); }

ising_status_t torus_step_f32_traced(ising_context *c, const float *x_in, float *x_out, int R, float alpha,
                                     double inv_beta, double alpha_k, double beta, double *H_out, cudaStream_t st) {
    if (!vec4_ok(c, x_in, x_out, R)) return ISING_ERR_UNSUPPORTED;
    const Vec4Shape v = vec4_shape(c);
    DOCH_CHECK(c->partials.ensure(sizeof(double) * 4 * static_cast<size_t>(v.blocks())));
    const float c3 = lattice_c3(inv_beta);
    torus_f32_r1_vec4<true><<<static_cast<unsigned>(v.blocks()), kThreads, 0, st>>>(
        x_in, x_out, c->right, c->down, static_cast<int>(c->l_rows), static_cast<int>(c->l_cols), v.tiles,
        static_cast<int>(v.bpt), alpha, c3, c->partials.as<double>());
    DOCH_CUDA(cudaGetLastError());
    return ham_fused_finish_launch(c->partials.as<double>(), static_cast<int>(v.blocks()), 1, alpha_k, beta, H_out, st);
}

ising_status_t torus_step_f32(const ising_context *c, const float *x_in, float *x_out, int R,
                              float alpha, double inv_beta, cudaStream_t st) {
    const int64_t Lr = c->l_rows, Lc = c->l_cols;
    if (vec4_ok(c, x_in, x_out, R)) {
        const Vec4Shape v = vec4_shape(c);
        const float c3 = lattice_c3(inv_beta);
        torus_f32_r1_vec4<false><<<static_cast<unsigned>(v.blocks()), kThreads, 0, st>>>(
            x_in, x_out, c->right, c->down, static_cast<int>(Lr), static_cast<int>(Lc), v.tiles,
            static_cast<int>(v.bpt), alpha, c3, nullptr);
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

bool torus_pair_ok(const ising_context *c, const float *x_in, const float *x_out, int R) {
    const bool aligned = (reinterpret_cast<uintptr_t>(x_in) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(x_out) % 16 == 0);
    return R == 1 && c->l_cols % 4 == 0 && aligned && c->l_rows >= 4 && c->l_rows < (1LL << 31) &&
           c->l_cols < (1LL << 31);
}

ising_status_t torus_pair_f32(const ising_context *c, const float *x_in, float *x_out, float alpha1,
                              float alpha2, double inv_beta, cudaStream_t st) {
    const int64_t Lr = c->l_rows, Lc = c->l_cols;
    const int64_t ncol4 = Lc / 4;
    const int64_t segs = (ncol4 + kSeg - 1) / kSeg;
    // one warp per (column segment, row strip); fill every warp slot of the GPU once
    const int64_t warp_slots = static_cast<int64_t>(c->num_sms) * t2_blocks_per_sm() * (kThreads / 32);
    int64_t bpt = warp_slots / segs;
    if (bpt < 1) bpt = 1;
    if (bpt > Lr / 4) bpt = Lr / 4 > 0 ? Lr / 4 : 1;
    const int64_t warps = segs * bpt;
    const int64_t blocks = (warps + kThreads / 32 - 1) / (kThreads / 32);
    if (blocks > INT32_MAX || segs > INT32_MAX) return fail(ISING_ERR_UNSUPPORTED, "lattice too large");
    const float c3 = lattice_c3(inv_beta);
    torus_f32_r1_vec4_t2<kT2Depth><<<static_cast<unsigned>(blocks), kThreads, kT2Smem, st>>>(
        x_in, x_out, c->right, c->down, static_cast<int>(Lr), static_cast<int>(Lc), static_cast<int>(segs),
        static_cast<int>(bpt), alpha1, alpha2, c3);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

ising_status_t torus_triple_f32(const ising_context *c, const float *x_in, float *x_out, float alpha1, float alpha2,
                                float alpha3, double inv_beta, cudaStream_t st) {
    const int64_t Lr = c->l_rows, Lc = c->l_cols;
    const int64_t ncol4 = Lc / 4;
    const int64_t segs = (ncol4 + kSeg - 1) / kSeg;
    const int64_t warp_slots = static_cast<int64_t>(c->num_sms) * t3_blocks_per_sm() * (kThreads / 32);
    int64_t bpt = warp_slots / segs;
    if (bpt < 1) bpt = 1;
    if (bpt > Lr / 6) bpt = Lr / 6 > 0 ? Lr / 6 : 1;
    const int64_t warps = segs * bpt;
    const int64_t blocks = (warps + kThreads / 32 - 1) / (kThreads / 32);
    if (blocks > INT32_MAX || segs > INT32_MAX) return fail(ISING_ERR_UNSUPPORTED, "lattice too large");
    const float c3 = lattice_c3(inv_beta);
    torus_f32_r1_vec4_t3<kT2Depth><<<static_cast<unsigned>(blocks), kThreads, kT2Smem, st>>>(
        x_in, x_out, c->right, c->down, static_cast<int>(Lr), static_cast<int>(Lc), static_cast<int>(segs),
        static_cast<int>(bpt), alpha1, alpha2, alpha3, c3);
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
