// Type-3 NUFFT sub-problems (Sect. 3, steps 1-4; Eq. 5-7 size the grids).
//
// For a block with pixel box centre C, baseline box centre D (wavelengths), per
// dimension: r~ = r - C, p~ = p - D, spread-grid scale a (cells per unit of r),
// spread grid n1, FFT grid n2. With s = isign:
//
//   f_k = Q_k sum_j G_j psi(v_k - j)                       (interpolate, n2 grid, periodic)
//   G   = FFT_s( pad( b_l / Psi(l) ) ),  l in [-n1/2, n1/2)  (deconvolve, zero-pad, FFT)
//   b_l = sum_n P_n c_n phi(l - g_n)                        (spread, n1 grid)
//   g_n = a r~_n + n1/2,  v_k = p~_k n2 / a,  tau_k = 2 pi p~_k / a
//   P_n = exp(s j 2 pi <D, r~_n>),  Q_k = exp(s j 2 pi <C, p_k>) / prod_d Phi(tau_kd)
//
// phi = psi = ES kernel of width w; Phi(tau) = int phi(z) cos(tau z) dz. Phi depends only
// on the kernel, so 1/Phi is one Chebyshev series in tau^2 per plan; Psi(l) = Phi(2 pi l/n2)
// is tabulated per block on the host. vis -> sky runs the exact transpose of every step
// (spread at baselines on n2, FFT_-s, crop and divide, gather at pixels).
//
// Grid positions and phases are computed on the fly for every (point, block): FP64 for
// the FP64 path; for the FP32 path from the float hi/lo splits of the coordinates and of
// C, D, a with exact differences and products, so no FP64 is used per point.
//
// Spreading: each CTA takes 128 consecutive points (chunk order is Morton order inside a
// chunk, in grid-cell units, so they are close on the grid), two threads per point each
// taking half of the window's z planes, accumulates the w^3 taps into a shared-memory
// tile that covers all their windows, then adds the tile to the grid with vector
// atomics; when the tile would not fit, the CTA adds its taps to the grid directly.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <mutex>
#include <vector>

#include "dfloat.cuh"
#include "hvox_internal.h"

namespace hvox {

namespace {

template <typename T> using cplx_t = typename CplxOf<T>::type;

constexpr int kSpreadThreads = 512;  // 16 warps: latency hiding at two CTAs per SM
constexpr int kSpreadPoints = 128;  // largest number of points per spreading CTA (the bin)

__device__ __forceinline__ float es_exp(float x) { return __expf(x); }
__device__ __forceinline__ double es_exp(double x) { return exp(x); }

// ES kernel phi(z) = exp(beta (sqrt(1 - (2 z / w)^2) - 1)) at z = j - fr, j = 0 .. W-1.
template <typename T, int W> __device__ __forceinline__ void es_weights(T fr, T beta, T *wt) {
    const T inv = T(2) / T(W);
#pragma unroll
    for (int j = 0; j < W; ++j) {
        T x = (T(j) - fr) * inv;
        T q = T(1) - x * x;
        wt[j] = q > T(0) ? es_exp(beta * (sqrt(q) - T(1))) : T(0);
    }
}

// The ES kernel weights of es_weights<double> in double-float arithmetic on the FP32 pipes
// (FP64 exp and sqrt cost ~30 FP64 instructions a weight, issued at 1/64 of the FP32 rate):
// x = (j - fr) 2 / W in FP64, then q = 1 - x^2, s = sqrt(q) (one Newton step on the float
// root), t = beta (s - 1) and exp(t) = 2^k exp(r), r = t - k ln 2 (|r| <= ln 2 / 2), by
// Horner's rule on the Taylor series to degree 11 (truncation below 7e-15). Absolute error
// ~2e-13 (the error of t, ~beta 2^-48, times the weight), which the FP64 kernels' weights
// share to within their own rounding.
struct DFConst {
    float h, l;
};
__host__ __device__ constexpr DFConst df_const(double x) { return {(float)x, (float)(x - (double)(float)x)}; }
__device__ __forceinline__ df::DF df_exp_es(df::DF t) {
    constexpr DFConst kLn2 = df_const(0.6931471805599453094);
    constexpr DFConst kInvFact[12] = {
        df_const(1.0),           df_const(1.0),           df_const(1.0 / 2),         df_const(1.0 / 6),
        df_const(1.0 / 24),      df_const(1.0 / 120),     df_const(1.0 / 720),       df_const(1.0 / 5040),
        df_const(1.0 / 40320),   df_const(1.0 / 362880),  df_const(1.0 / 3628800),   df_const(1.0 / 39916800)};
    const float k = rintf(__fmul_rn(t.h, 1.44269504088896341f));
    const df::DF r = df::dadd(t, df::dmul(df::DF{-k, 0.f}, df::DF{kLn2.h, kLn2.l}));
    df::DF p = {kInvFact[11].h, kInvFact[11].l};
#pragma unroll
    for (int i = 10; i >= 0; --i) p = df::dadd(df::dmul(p, r), df::DF{kInvFact[i].h, kInvFact[i].l});
    const float sc = __int_as_float((127 + (int)k) << 23);  // 2^k, k in [-64, 0]
    return {__fmul_rn(p.h, sc), __fmul_rn(p.l, sc)};
}

template <int W> __device__ __forceinline__ void es_weights_df(double fr, df::DF beta, df::DF *wt) {
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const df::DF x = df::split_bits(((double)j - fr) * (2.0 / W));
        const df::DF q = df::dadd(df::DF{1.f, 0.f}, df::dneg(df::dmul(x, x)));
        if (q.h <= 0.f) {
            wt[j] = {0.f, 0.f};
            continue;
        }
        // sqrt: s0 = fl(sqrt(q.h)), s1 = (q - s0^2) / (2 s0)
        const float s0 = __fsqrt_rn(q.h);
        const float pp = __fmul_rn(s0, s0);
        const float rr = __fadd_rn(__fsub_rn(__fsub_rn(q.h, pp), __fmaf_rn(s0, s0, -pp)), q.l);
        df::DF sq;
        df::fast_two_sum(s0, __fmul_rn(rr, __frcp_rn(__fmul_rn(2.f, s0))), sq.h, sq.l);
        const df::DF t = df::dmul(df::dadd(sq, df::DF{-1.f, 0.f}), beta);
        wt[j] = df_exp_es(t);
    }
}

// i mod n for i in [-n, 2n). Every caller indexes a window whose start geo_vis has
// checked to lie in [-n, 2n - w] (clamping it there and setting the device error word
// otherwise), and n2 >= 2w, so every argument is in that range.
__device__ __forceinline__ int wrap(int i, int n) {
    i += i < 0 ? n : 0;
    i -= i >= n ? n : 0;
    return i;
}

// Window start of a pixel on the n1 grid: inside [0, n1 - W] for every pixel of the
// sub-problem's box; anything else is clamped into the grid and reported.
template <int W> __device__ __forceinline__ int clamp_pix_window(int i0, int n1, int *err) {
    const int c = min(max(i0, 0), n1 - W);
    if (c != i0) atomicOr(err, kDevErrPixWindow);
    return c;
}

// Window start of a baseline on the periodic n2 grid: baselines of the sub-problem's box
// lie within n2/2 + W of the origin, so the start is in [-n2, 2 n2 - W]; anything else is
// clamped there and reported.
template <int W> __device__ __forceinline__ int check_vis_window(int i0, int n2, int *err) {
    const int c = min(max(i0, -n2), 2 * n2 - W);
    if (c != i0) atomicOr(err, kDevErrVisWindow);
    return c;
}

// ------------------------------------------------------------------ float helpers

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// (ah + al) - (bh + bl) as hi + lo with the leading difference exact.
__device__ __forceinline__ void df_sub(float ah, float al, float bh, float bl, float &rh, float &rl) {
    float s, e;
    two_sum(ah, -bh, s, e);
    rh = s;
    rl = __fadd_rn(e, __fsub_rn(al, bl));
}

// (ah + al)(bh + bl) as hi + lo.
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &p, float &lo) {
    two_prod(ah, bh, p, lo);
    lo = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, lo));
}

// Fraction of sum_d x_d y_d in turns (x, y as hi/lo splits), |error| ~ 1e-7 turn.
__device__ __forceinline__ float dot_frac_f32(const float *xh, const float *xl, const float *yh, const float *yl) {
    float f = 0.f, small = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float a, b;
        two_prod(xh[d], yh[d], a, b);
        a = __fsub_rn(a, rintf(a));
        f = __fadd_rn(f, a);
        small = __fadd_rn(small, __fmaf_rn(xh[d], yl[d], __fmaf_rn(xl[d], yh[d], b)));
    }
    f = __fadd_rn(f, small);
    return __fsub_rn(f, rintf(f));
}

// Window of a point at grid position g = s + off (s = sh + sl): start i0 = ceil(g - W/2)
// and offset fr = g - i0 in (W/2 - 1, W/2].
template <int W> __device__ __forceinline__ void window_f32(float sh, float sl, int off, int &i0, float &fr) {
    const float m = rintf(sh);
    const float f = __fadd_rn(__fsub_rn(sh, m), sl);
    const float cf = ceilf(__fsub_rn(f, 0.5f * W));
    i0 = (int)m + off + (int)cf;
    fr = __fsub_rn(f, cf);
}

template <int W> __device__ __forceinline__ void window_f64(double g, int &i0, double &fr) {
    const double c = ceil(g - 0.5 * W);
    i0 = (int)c;
    fr = g - c;
}

// 1 / Phi(tau): Chebyshev series in u = 2 (tau / tau_max)^2 - 1 (Clenshaw).
template <typename T> __device__ __forceinline__ T inv_phi(T tau, const T *__restrict__ cc, int deg, T inv_tmax2) {
    const T u = T(2) * tau * tau * inv_tmax2 - T(1);
    T b1 = 0, b2 = 0;
    for (int k = deg; k >= 1; --k) {
        T b0 = cc[k] + T(2) * u * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    return cc[0] + u * b1 - b2;
}

// ------------------------------------------------------------------ per-point geometry

// Pixel n (chunk position) in block b: window on the n1 grid and prephase P = exp(s j 2 pi <D, r~>).
template <int W>
__device__ __forceinline__ void geo_pix(const NufftDev &b, int64_t n, const float4 *__restrict__ rh,
                                        const float4 *__restrict__ rl, const double *, int64_t, int isign, int i0[3],
                                        float fr[3], float &pr, float &pim) {
    const float4 h = rh[n], l = rl[n];
    const float xh[3] = {h.x, h.y, h.z}, xl[3] = {l.x, l.y, l.z};
    float th[3], tl[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        df_sub(xh[d], xl[d], b.Ch[d], b.Cl[d], th[d], tl[d]);
        float sh, sl;
        df_mul(b.ah[d], b.al[d], th[d], tl[d], sh, sl);
        window_f32<W>(sh, sl, b.n1[d] / 2, i0[d], fr[d]);
        i0[d] = clamp_pix_window<W>(i0[d], b.n1[d], b.err);
    }
    const float f = dot_frac_f32(b.Dh, b.Dl, th, tl);
    float sn, cs;
    __sincosf(6.28318530717958648f * f, &sn, &cs);
    pr = cs;
    pim = isign * sn;
}

template <int W>
__device__ __forceinline__ void geo_pix(const NufftDev &b, int64_t n, const float4 *, const float4 *,
                                        const double *__restrict__ soa, int64_t n_all, int isign, int i0[3],
                                        double fr[3], double &pr, double &pim) {
    double t = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double r = soa[d * n_all + n] - b.C[d];
        window_f64<W>(b.a[d] * r + 0.5 * b.n1[d], i0[d], fr[d]);
        i0[d] = clamp_pix_window<W>(i0[d], b.n1[d], b.err);
        t = fma(b.D[d], r, t);
    }
    t -= rint(t);
    double sn, cs;
    sincospi(2.0 * t, &sn, &cs);
    pr = cs;
    pim = isign * sn;
}

// Baseline k (chunk position) in block b: window on the n2 grid (unwrapped start) and
// Q = exp(s j 2 pi <C, p>) / prod_d Phi(tau_d).
template <int W>
__device__ __forceinline__ void geo_vis(const NufftDev &b, int64_t k, const float4 *__restrict__ vh,
                                        const float4 *__restrict__ vl, const double *, int64_t, int isign,
                                        const float *__restrict__ cc, int deg, float inv_tmax2, int i0[3], float fr[3],
                                        float &qr, float &qi) {
    const float4 h = vh[k], l = vl[k];
    const float ph[3] = {h.x, h.y, h.z}, pl[3] = {l.x, l.y, l.z};
    float ip = 1.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float th, tl;
        df_sub(ph[d], pl[d], b.Dh[d], b.Dl[d], th, tl);
        float sh, sl;
        df_mul(b.n2ah[d], b.n2al[d], th, tl, sh, sl);
        window_f32<W>(sh, sl, 0, i0[d], fr[d]);
        i0[d] = check_vis_window<W>(i0[d], b.n2[d], b.err);
        ip *= inv_phi<float>(th * b.tpa[d], cc, deg, inv_tmax2);
    }
    const float f = dot_frac_f32(ph, pl, b.Ch, b.Cl);
    float sn, cs;
    __sincosf(6.28318530717958648f * f, &sn, &cs);
    qr = cs * ip;
    qi = isign * sn * ip;
}

template <int W>
__device__ __forceinline__ void geo_vis(const NufftDev &b, int64_t k, const float4 *, const float4 *,
                                        const double *__restrict__ soa, int64_t n_all, int isign,
                                        const double *__restrict__ cc, int deg, double inv_tmax2, int i0[3],
                                        double fr[3], double &qr, double &qi) {
    double t = 0.0, ip = 1.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double p = soa[d * n_all + k];
        const double pt = p - b.D[d];
        window_f64<W>(pt * b.n2a[d], i0[d], fr[d]);
        i0[d] = check_vis_window<W>(i0[d], b.n2[d], b.err);
        ip *= inv_phi<double>(pt * b.tpa64[d], cc, deg, inv_tmax2);
        t = fma(b.C[d], p, t);
    }
    t -= rint(t);
    double sn, cs;
    sincospi(2.0 * t, &sn, &cs);
    qr = cs * ip;
    qi = isign * sn * ip;
}

// ------------------------------------------------------------------ atomics

__device__ __forceinline__ void grid_add(float2 *g, float re, float im) { atomicAdd(g, make_float2(re, im)); }
__device__ __forceinline__ void grid_add(double2 *g, double re, double im) {
    atomicAdd(&g->x, re);
    atomicAdd(&g->y, im);
}
// ------------------------------------------------------------------ spreading (tiled)

// A CTA spreads up to 128 consecutive points (Morton order in grid-cell units, so they are
// close on the grid). Phase 1: threads 0..127 each take one point, compute its window
// start and value and stage them in shared memory; 384 threads evaluate the kernel weights
// (one per point and dimension); the window starts of each group of 8 points give a box,
// and consecutive groups are joined into sub-bins while their joint tile fits the shared
// memory (a group too wide alone goes to the grid directly). Phase 2, per sub-bin: each of
// the 16 warps takes its points one at a time; for a point, lane (g, j) (g = lane / 8,
// j = lane % 8) adds the taps of x offsets j (and j + 8 when w > 8) in the z planes g,
// g + 4, ... of the window, looping over its y rows. The taps go into a shared tile
// (separate real and imaginary planes) covering the union of the sub-bin's windows, whose
// plane stride is padded to 8 (mod 32) elements: the four groups of a warp then sit 8
// banks apart and their 8 lanes on consecutive banks, so every shared atomic of a warp
// touches 32 distinct banks. The tile is then added to the grid with vector atomics, one
// warp per tile row.
constexpr int kGroupLanes = 8;
constexpr int kZGroups = 32 / kGroupLanes;                        // lane groups along z
constexpr int kPointsPerWarp = kSpreadPoints / (kSpreadThreads / 32);
static_assert(kSpreadThreads % 32 == 0 && kPointsPerWarp * (kSpreadThreads / 32) == kSpreadPoints,
              "every point of a spreading CTA is taken by exactly one warp");
// Shared memory of a spreading CTA: two CTAs per SM for FP32 grids; one CTA per SM for
// FP64 grids (the w = 13 windows of eps <= 1e-9 need the larger tile to fit a bin at all).
template <typename T> __host__ __device__ constexpr int smem_per_cta() { return sizeof(T) == 4 ? 110 * 1024 : 224 * 1024; }

template <typename T, int W> struct SpreadShared {
    static constexpr int kWStride = 3 * W + 1;  // odd row stride: fewer bank conflicts
    T w[kSpreadPoints][kWStride];                // x, y, z weights of each point
    T v[kSpreadPoints][2];                       // complex value
    T fr[kSpreadPoints][3];                      // fractional window offsets
    int i0[kSpreadPoints][3];                    // window start (i0[.][0] = INT_MIN: no point)
};

// Kernel weights of the staged points: 3 x 128 rows (point, dimension), one per thread of
// the first 384, so the exponentials of a bin are spread over 12 warps instead of 4.
// DF = true (FP64 plans with fixed-point tiles): the weights in double-float arithmetic,
// stored as float pairs in the 8-byte slots (read back with weight_of).
template <typename T, int W, bool DF = false>
__device__ __forceinline__ void stage_weights(SpreadShared<T, W> &sh, T beta) {
    const int tid = threadIdx.x;
    static_assert(kSpreadThreads >= 3 * kSpreadPoints, "one thread per weight row");
    static_assert(!DF || sizeof(T) == 8, "float pairs fill FP64 slots");
    if (tid < 3 * kSpreadPoints) {
        const int p = tid % kSpreadPoints, d = tid / kSpreadPoints;
        if (sh.i0[p][0] != INT_MIN) {
            if constexpr (DF) {
                df::DF wv[W];
                es_weights_df<W>((double)sh.fr[p][d], df::split_bits((double)beta), wv);
#pragma unroll
                for (int j = 0; j < W; ++j)
                    *reinterpret_cast<float2 *>(&sh.w[p][d * W + j]) = make_float2(wv[j].h, wv[j].l);
            } else {
                T wv[W];
                es_weights<T, W>(sh.fr[p][d], beta, wv);
#pragma unroll
                for (int j = 0; j < W; ++j) sh.w[p][d * W + j] = wv[j];
            }
        }
    }
}

// A staged weight as T (DF: the float pair's value) and a staged weight or scaled value
// as a float pair.
template <typename T, bool DF> __device__ __forceinline__ T weight_of(const T &slot) {
    if constexpr (DF) {
        const float2 v = *reinterpret_cast<const float2 *>(&slot);
        return (T)df::to_double(df::DF{v.x, v.y});
    } else {
        return slot;
    }
}
template <typename T> __device__ __forceinline__ df::DF weight_df(const T &slot) {
    const float2 v = *reinterpret_cast<const float2 *>(&slot);
    return {v.x, v.y};
}

template <typename T, int W> __host__ __device__ constexpr int tile_bytes() {
    // the rest of the static shared memory of spread_cta (group boxes, sub-bins) < 1 KB
    return ((smem_per_cta<T>() - (int)sizeof(SpreadShared<T, W>) - (int)sizeof(NufftDev) - 1024) /
            (2 * (int)sizeof(T) * 32)) *
           (2 * (int)sizeof(T) * 32);
}

// The CTA's sub-problem descriptor, copied from the plan's device array into shared memory
// (every thread reads its fields; a shared broadcast instead of a global load each time).
__device__ __forceinline__ void load_desc(NufftDev &dst, const NufftDev *__restrict__ src) {
    static_assert(sizeof(NufftDev) % 4 == 0, "descriptor copied as 32-bit words");
    const int *from = reinterpret_cast<const int *>(src);
    int *to = reinterpret_cast<int *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(NufftDev) / 4); i += blockDim.x) to[i] = from[i];
    __syncthreads();
}

// Plane stride of a tile with tx * ty cells per plane: the next value = 8 (mod 32).
__device__ __forceinline__ int64_t tile_plane_stride(int64_t cells) { return cells + ((8 - cells) % 32 + 32) % 32; }

// The grid of a spreading CTA, read from its shared descriptor where it is used (the
// untiled path and the flush) rather than held in registers across the tap loop: the n1
// grid (pixels, contiguous) or the n2 grid (baselines, z planes zs2 apart).
// The lane's buffer arrives as a kernel parameter, so the compiler treats every grid
// address as global memory (fire-and-forget vector reductions in the flush).
template <typename T, bool PERIODIC> struct SpreadGrid {
    const NufftDev &b;
    cplx_t<T> *__restrict__ base;  // the lane's g1 (pixels) or g2 (baselines)
    __device__ __forceinline__ int n(int d) const { return PERIODIC ? b.n2[d] : b.n1[d]; }
    __device__ __forceinline__ cplx_t<T> *row(int64_t z, int64_t y) const {
        if (PERIODIC) return base + b.g2_off + z * b.zs2 + y * b.n2[0];
        return base + b.g1_off + (z * b.n1[1] + y) * b.n1[0];
    }
};

// Fixed-point tile (FP64 plans): the shared tile holds each cell's real and imaginary parts
// as fixed-point numbers in two 32-bit limbs, value = (H 2^22 + L) u with u = 2^(e - 43)
// per CTA and every |value| of the CTA's points below 2^e, so a tap costs no FP64
// instruction: its product in double-float arithmetic (FP32 pipes) splits into
// H = rint(x 2^-22) and L = rint(x - H 2^22) by FMA rounding against 1.5 2^23 (|H|, |L| <=
// 2^21; the at most 128 taps a cell receives from one CTA keep each limb below 2^28), added
// by native 32-bit shared integer atomics (FP64 shared atomics are compare-and-swap loops
// around an FP64 add). Sums are exact up to u / 2 = 2^-44 of the CTA's largest value per
// tap. The flush converts each cell back to FP64.
constexpr float kLimbMagic = 12582912.0f;  // 1.5 * 2^23

// q 2^k as a double for |q| < 2^52, exactly, by integer operations (no FP64 instruction:
// the flush of a large tile would otherwise spend two FP64 operations per part and cell).
__device__ __forceinline__ double i64_pow2(long long q, int k) {
    if (q == 0) return 0.0;
    const unsigned long long sign = q < 0 ? (1ull << 63) : 0ull;
    unsigned long long m = (unsigned long long)(q < 0 ? -q : q);
    const int msb = 63 - __clzll((long long)m);
    m <<= (52 - msb);  // leading one at bit 52 (msb <= 51)
    return __longlong_as_double((long long)(sign | ((unsigned long long)(msb + k + 1023) << 52) |
                                            (m & ((1ull << 52) - 1ull))));
}

__device__ __forceinline__ void limbs(df::DF x, int &H, int &L) {
    const float t = __fmaf_rn(x.h, 0x1p-22f, kLimbMagic);
    H = __float_as_int(t) - __float_as_int(kLimbMagic);
    const float hf = __fsub_rn(t, kLimbMagic);
    const float r = __fadd_rn(__fmaf_rn(-hf, 0x1p22f, x.h), x.l);
    L = __float_as_int(__fadd_rn(r, kLimbMagic)) - __float_as_int(kLimbMagic);
}

template <typename T, int W, bool PERIODIC>
__device__ __forceinline__ void spread_cta(bool act, const int i0[3], const T fr[3], T vr, T vi, T beta,
                                           const SpreadGrid<T, PERIODIC> grid, int ppc) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ SpreadShared<T, W> sh;
    __shared__ int s_lo[3], s_hi[3];
    constexpr int cap = tile_bytes<T, W>() / (2 * (int)sizeof(T));
    T *tre = reinterpret_cast<T *>(smem_raw);
    T *tim = tre + cap;
    const int tid = threadIdx.x;
    if (tid < 3) {
        s_lo[tid] = INT_MAX;
        s_hi[tid] = INT_MIN;
    }
    __syncthreads();
    if (tid < kSpreadPoints) {
        if (act) {
            sh.v[tid][0] = vr;
            sh.v[tid][1] = vi;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                sh.fr[tid][d] = fr[d];
                sh.i0[tid][d] = i0[d];
                atomicMin(&s_lo[d], i0[d]);
                atomicMax(&s_hi[d], i0[d]);
            }
        } else {
            sh.i0[tid][0] = INT_MIN;
        }
    }
    __syncthreads();
    if (s_hi[0] < s_lo[0]) return;  // no point in this CTA (uniform across the CTA)
    stage_weights<T, W>(sh, beta);
    const int lo0 = s_lo[0], lo1 = s_lo[1], lo2 = s_lo[2];
    const int64_t tx = (int64_t)s_hi[0] - lo0 + W, ty = (int64_t)s_hi[1] - lo1 + W,
                  tz = (int64_t)s_hi[2] - lo2 + W;
    const int64_t ps64 = tile_plane_stride(tx * ty);
    const bool tiled = tz * ps64 <= cap;
    const int txi = (int)tx, tyi = (int)ty, ps = tiled ? (int)ps64 : 0;
    if (tiled) {
        const int cells = (int)(tz * ps64);
        for (int j = tid; j < cells; j += blockDim.x) {
            tre[j] = T(0);
            tim[j] = T(0);
        }
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5, g = lane / kGroupLanes, jx0 = lane % kGroupLanes;
    constexpr int kXT = (W + kGroupLanes - 1) / kGroupLanes;  // x taps per lane (1 or 2)
    const int rounds = (ppc + kSpreadThreads / 32 - 1) / (kSpreadThreads / 32);
    for (int round = 0; round < rounds; ++round) {
        const int p = round * (kSpreadThreads / 32) + warp;  // warps take points 16 apart
        const int px0 = sh.i0[p][0];
        if (px0 == INT_MIN) continue;  // uniform across the warp
        const int py0 = sh.i0[p][1], pz0 = sh.i0[p][2];
        T ar[kXT], ai[kXT];
        int cx[kXT];
        bool on[kXT];
#pragma unroll
        for (int t = 0; t < kXT; ++t) {
            const int jx = jx0 + t * kGroupLanes;
            on[t] = jx < W;
            const T wxv = on[t] ? weight_of<T, false>(sh.w[p][jx]) : T(0);
            ar[t] = sh.v[p][0] * wxv;
            ai[t] = sh.v[p][1] * wxv;
            cx[t] = tiled ? px0 - lo0 + jx : (PERIODIC ? wrap(px0 + jx, grid.n(0)) : px0 + jx);
        }
        T wy[W];
#pragma unroll
        for (int j = 0; j < W; ++j) wy[j] = weight_of<T, false>(sh.w[p][W + j]);
        for (int jz = g; jz < W; jz += kZGroups) {
            const T wz = weight_of<T, false>(sh.w[p][2 * W + jz]);
            // Fold the z weight into the value once per plane: two multiplies per tap.
            T zr[kXT], zi[kXT];
#pragma unroll
            for (int t = 0; t < kXT; ++t) {
                zr[t] = ar[t] * wz;
                zi[t] = ai[t] * wz;
            }
            if (tiled) {
                const int zbase = (pz0 - lo2 + jz) * ps + (py0 - lo1) * txi;
#pragma unroll
                for (int jy = 0; jy < W; ++jy) {
                    const int base = zbase + jy * txi;
#pragma unroll
                    for (int t = 0; t < kXT; ++t)
                        if (on[t]) {
                            atomicAdd(tre + base + cx[t], zr[t] * wy[jy]);
                            atomicAdd(tim + base + cx[t], zi[t] * wy[jy]);
                        }
                }
            } else {
                const int64_t gz = PERIODIC ? wrap(pz0 + jz, grid.n(2)) : pz0 + jz;
                for (int jy = 0; jy < W; ++jy) {
                    const int64_t gy = PERIODIC ? wrap(py0 + jy, grid.n(1)) : py0 + jy;
                    cplx_t<T> *row = grid.row(gz, gy);
#pragma unroll
                    for (int t = 0; t < kXT; ++t)
                        if (on[t]) grid_add(row + cx[t], zr[t] * wy[jy], zi[t] * wy[jy]);
                }
            }
        }
    }
    if (!tiled) return;
    __syncthreads();
    // Flush: one warp per (y, z) row of the tile, lanes along x (coalesced vector atomics).
    const int rows = (int)(ty * tz);
    for (int r = warp; r < rows; r += blockDim.x >> 5) {
        const int y = r % tyi, z = r / tyi;
        int gy = lo1 + y, gz = lo2 + z;
        if (PERIODIC) {
            gy = wrap(gy, grid.n(1));
            gz = wrap(gz, grid.n(2));
        }
        cplx_t<T> *grow = grid.row(gz, gy);
        const int t0 = z * ps + y * txi;
        for (int x = lane; x < txi; x += 32) {
            const T re = tre[t0 + x], im = tim[t0 + x];
            if (re == T(0) && im == T(0)) continue;
            const int gx = PERIODIC ? wrap(lo0 + x, grid.n(0)) : lo0 + x;
            grid_add(grow + gx, re, im);
        }
    }
}

template <typename T, int W, bool PERIODIC>
__device__ __forceinline__ void spread_cta_fixed(bool act, const int i0[3], const T fr[3], T vr, T vi, T beta,
                                           const SpreadGrid<T, PERIODIC> grid, int ppc) {
    static_assert(sizeof(T) == 8, "the fixed-point tile serves FP64 grids");
    constexpr bool IT = true;
    constexpr int kGroup = 8;                           // points per bounding-box group
    constexpr int kGroups = kSpreadPoints / kGroup;
    extern __shared__ unsigned char smem_raw[];
    __shared__ SpreadShared<T, W> sh;
    __shared__ unsigned s_maxbits;
    __shared__ int s_gbox[kGroups][6];                  // per group: window-start min (3), max (3)
    __shared__ int s_sub[kGroups][8];                   // sub-bins: p0, p1, lo (3), tx, ty, tz (0: untiled)
    __shared__ int s_nsub;
    constexpr int cap = tile_bytes<T, W>() / (2 * (int)sizeof(T));  // cells (16 bytes each for FP64)
    T *tre = reinterpret_cast<T *>(smem_raw);
    T *tim = tre + cap;
    int *tHr = reinterpret_cast<int *>(smem_raw);  // fixed-point form: four int planes
    int *tLr = tHr + cap, *tHi = tLr + cap, *tLi = tHi + cap;
    const int tid = threadIdx.x;
    if (tid == 0) s_maxbits = 0u;
    __syncthreads();
    if (tid < kSpreadPoints) {
        if (act) {
            sh.v[tid][0] = vr;
            sh.v[tid][1] = vi;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                sh.fr[tid][d] = fr[d];
                sh.i0[tid][d] = i0[d];
            }
            if (IT) {
                // an upper bound of |vr|, |vi| as a float (non-negative floats order as integers)
                const double m = fmax(fabs((double)vr), fabs((double)vi));
                atomicMax(&s_maxbits, __float_as_uint(__double2float_ru(m)));
            }
        } else {
            sh.i0[tid][0] = INT_MIN;
        }
    }
    __syncthreads();
    stage_weights<T, W, IT>(sh, beta);
    // Bounding boxes of the window starts of each group of 8 consecutive points.
    const int ngroups = (ppc + kGroup - 1) / kGroup;
    if (tid < 3 * ngroups) {
        const int g = tid / 3, d = tid - 3 * g;
        int lo = INT_MAX, hi = INT_MIN;
#pragma unroll
        for (int q = 0; q < kGroup; ++q) {
            const int p = g * kGroup + q;
            if (p < kSpreadPoints && sh.i0[p][0] != INT_MIN) {
                lo = min(lo, sh.i0[p][d]);
                hi = max(hi, sh.i0[p][d]);
            }
        }
        s_gbox[g][d] = lo;
        s_gbox[g][3 + d] = hi;
    }
    __syncthreads();
    // Sub-bins: runs of consecutive groups whose joint tile fits (chunk order is Morton order,
    // so consecutive groups are close); a group too wide alone goes straight to the grid.
    // Only the fixed-point tile splits a bin (spread_cta keeps one tile per bin or none): with
    // float atomics (compare-and-swap loops) the taps of a bin too wide for the tile are
    // cheaper as vector reductions into the grid (splitting made FP32 spreading 1.4-1.7x
    // slower).
    if (tid == 0) {
        int n = 0, g0 = 0;
        int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
        auto cells_of = [&](const int *l, const int *h) -> int64_t {
            const int64_t tx = (int64_t)h[0] - l[0] + W, ty = (int64_t)h[1] - l[1] + W, tz = (int64_t)h[2] - l[2] + W;
            return tz * tile_plane_stride(tx * ty);
        };
        auto emit = [&](int ga, int gb, const int *l, const int *h, bool tiled) {
            int *e = s_sub[n++];
            e[0] = ga * kGroup;
            e[1] = min(gb * kGroup, kSpreadPoints);
            for (int d = 0; d < 3; ++d) e[2 + d] = l[d];
            e[5] = tiled ? h[0] - l[0] + W : 0;
            e[6] = h[1] - l[1] + W;
            e[7] = h[2] - l[2] + W;
        };
        for (int g = 0; g < ngroups; ++g) {
            if (s_gbox[g][0] == INT_MAX) continue;  // no point in this group
            int nl[3], nh[3];
            for (int d = 0; d < 3; ++d) {
                nl[d] = min(lo[d], s_gbox[g][d]);
                nh[d] = max(hi[d], s_gbox[g][3 + d]);
            }
            if (cells_of(nl, nh) <= cap) {
                for (int d = 0; d < 3; ++d) {
                    lo[d] = nl[d];
                    hi[d] = nh[d];
                }
                continue;
            }
            if (lo[0] != INT_MAX) emit(g0, g, lo, hi, true);
            g0 = g;
            for (int d = 0; d < 3; ++d) {
                lo[d] = s_gbox[g][d];
                hi[d] = s_gbox[g][3 + d];
            }
            if (cells_of(lo, hi) > cap) {  // this group alone does not fit
                emit(g, g + 1, lo, hi, false);
                g0 = g + 1;
                for (int d = 0; d < 3; ++d) {
                    lo[d] = INT_MAX;
                    hi[d] = INT_MIN;
                }
            }
        }
        if (lo[0] != INT_MAX) emit(g0, ngroups, lo, hi, true);
        s_nsub = n;
    }
    __syncthreads();
    const int nsub = s_nsub;
    if (nsub == 0) return;  // no point in this CTA (uniform across the CTA)
    const int e = (int)((s_maxbits >> 23) & 0xFFu) - 126;  // every |value| < 2^e
    const bool any_value = s_maxbits != 0u;
    if (IT && any_value) {
        // each point's value in units 2^(e - 43), as float pairs in place (once per point;
        // untiled sub-bins read it back as FP64 in the same units, scaled back at the add)
        if (tid < kSpreadPoints && sh.i0[tid][0] != INT_MIN) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const df::DF v = df::split_bits(ldexp((double)sh.v[tid][c], 43 - e));
                *reinterpret_cast<float2 *>(&sh.v[tid][c]) = make_float2(v.h, v.l);
            }
        }
    }
    const int lane = tid & 31, warp = tid >> 5, g = lane / kGroupLanes, jx0 = lane % kGroupLanes;
    constexpr int kXT = (W + kGroupLanes - 1) / kGroupLanes;  // x taps per lane (1 or 2)
    for (int sb = 0; sb < nsub; ++sb) {
        const int p0 = s_sub[sb][0], p1 = s_sub[sb][1];
        const int lo0 = s_sub[sb][2], lo1 = s_sub[sb][3], lo2 = s_sub[sb][4];
        const int txi = s_sub[sb][5], tyi = s_sub[sb][6], tzi = s_sub[sb][7];
        const bool tiled = txi > 0;
        const bool fixed = IT && tiled && any_value;  // fixed-point form of the tile
        const int ps = tiled ? (int)tile_plane_stride((int64_t)txi * tyi) : 0;
        if (tiled) {
            __syncthreads();  // the previous sub-bin's flush has read the tile
            const int cells = tzi * ps;
            if (fixed) {
                for (int j = tid; j < cells; j += blockDim.x) {
                    tHr[j] = 0;
                    tLr[j] = 0;
                    tHi[j] = 0;
                    tLi[j] = 0;
                }
            } else {
                for (int j = tid; j < cells; j += blockDim.x) {
                    tre[j] = T(0);
                    tim[j] = T(0);
                }
            }
        }
        __syncthreads();  // tile cleared; staged values, weights and scales visible
        const int rounds = (p1 - p0 + kSpreadThreads / 32 - 1) / (kSpreadThreads / 32);
        for (int round = 0; round < rounds; ++round) {
            const int p = p0 + round * (kSpreadThreads / 32) + warp;  // warps take points 16 apart
            if (p >= p1) continue;
            const int px0 = sh.i0[p][0];
            if (px0 == INT_MIN) continue;  // uniform across the warp
            const int py0 = sh.i0[p][1], pz0 = sh.i0[p][2];
            if constexpr (IT) {
                if (fixed) {
                    // taps in units 2^(e - 43), double-float products, two limbs, four int atomics
                    df::DF ar[kXT], ai[kXT];
                    int cx[kXT];
                    bool on[kXT];
                    const df::DF vr_ = weight_df(sh.v[p][0]), vi_ = weight_df(sh.v[p][1]);
#pragma unroll
                    for (int t = 0; t < kXT; ++t) {
                        const int jx = jx0 + t * kGroupLanes;
                        on[t] = jx < W;
                        const df::DF wxv = on[t] ? weight_df(sh.w[p][jx]) : df::DF{0.f, 0.f};
                        ar[t] = df::dmul(vr_, wxv);
                        ai[t] = df::dmul(vi_, wxv);
                        cx[t] = px0 - lo0 + jx;
                    }
                    df::DF wy[W];
#pragma unroll
                    for (int j = 0; j < W; ++j) wy[j] = weight_df(sh.w[p][W + j]);
                    for (int jz = g; jz < W; jz += kZGroups) {
                        const df::DF wz = weight_df(sh.w[p][2 * W + jz]);
                        df::DF zr[kXT], zi[kXT];
#pragma unroll
                        for (int t = 0; t < kXT; ++t) {
                            zr[t] = df::dmul(ar[t], wz);
                            zi[t] = df::dmul(ai[t], wz);
                        }
                        const int zbase = (pz0 - lo2 + jz) * ps + (py0 - lo1) * txi;
#pragma unroll
                        for (int jy = 0; jy < W; ++jy) {
                            const int base = zbase + jy * txi;
#pragma unroll
                            for (int t = 0; t < kXT; ++t)
                                if (on[t]) {
                                    int H, L;
                                    limbs(df::dmul(zr[t], wy[jy]), H, L);
                                    atomicAdd(tHr + base + cx[t], H);
                                    atomicAdd(tLr + base + cx[t], L);
                                    limbs(df::dmul(zi[t], wy[jy]), H, L);
                                    atomicAdd(tHi + base + cx[t], H);
                                    atomicAdd(tLi + base + cx[t], L);
                                }
                        }
                    }
                    continue;
                }
            }
            // T taps: into the T tile, or (untiled sub-bin) straight into the grid. With the
            // fixed-point form's scaled pairs staged, the values are read back as FP64 and the
            // unit applied once per point.
            T vr_, vi_;
            if (IT && any_value) {
                vr_ = (T)ldexp(df::to_double(weight_df(sh.v[p][0])), e - 43);
                vi_ = (T)ldexp(df::to_double(weight_df(sh.v[p][1])), e - 43);
            } else {
                vr_ = sh.v[p][0];
                vi_ = sh.v[p][1];
            }
            T ar[kXT], ai[kXT];
            int cx[kXT];
            bool on[kXT];
#pragma unroll
            for (int t = 0; t < kXT; ++t) {
                const int jx = jx0 + t * kGroupLanes;
                on[t] = jx < W;
                const T wxv = on[t] ? weight_of<T, IT>(sh.w[p][jx]) : T(0);
                ar[t] = vr_ * wxv;
                ai[t] = vi_ * wxv;
                cx[t] = tiled ? px0 - lo0 + jx : (PERIODIC ? wrap(px0 + jx, grid.n(0)) : px0 + jx);
            }
            T wy[W];
#pragma unroll
            for (int j = 0; j < W; ++j) wy[j] = weight_of<T, IT>(sh.w[p][W + j]);
            for (int jz = g; jz < W; jz += kZGroups) {
                const T wz = weight_of<T, IT>(sh.w[p][2 * W + jz]);
                // Fold the z weight into the value once per plane: two multiplies per tap.
                T zr[kXT], zi[kXT];
#pragma unroll
                for (int t = 0; t < kXT; ++t) {
                    zr[t] = ar[t] * wz;
                    zi[t] = ai[t] * wz;
                }
                if (tiled) {
                    const int zbase = (pz0 - lo2 + jz) * ps + (py0 - lo1) * txi;
#pragma unroll
                    for (int jy = 0; jy < W; ++jy) {
                        const int base = zbase + jy * txi;
#pragma unroll
                        for (int t = 0; t < kXT; ++t)
                            if (on[t]) {
                                atomicAdd(tre + base + cx[t], zr[t] * wy[jy]);
                                atomicAdd(tim + base + cx[t], zi[t] * wy[jy]);
                            }
                    }
                } else {
                    const int64_t gz = PERIODIC ? wrap(pz0 + jz, grid.n(2)) : pz0 + jz;
                    for (int jy = 0; jy < W; ++jy) {
                        const int64_t gy = PERIODIC ? wrap(py0 + jy, grid.n(1)) : py0 + jy;
                        cplx_t<T> *row = grid.row(gz, gy);
#pragma unroll
                        for (int t = 0; t < kXT; ++t)
                            if (on[t]) grid_add(row + cx[t], zr[t] * wy[jy], zi[t] * wy[jy]);
                    }
                }
            }
        }
        if (!tiled) continue;
        __syncthreads();
        // Flush: one warp per (y, z) row of the tile, lanes along x (coalesced vector atomics).
        const int rows = tyi * tzi;
        for (int r = warp; r < rows; r += blockDim.x >> 5) {
            const int y = r % tyi, z = r / tyi;
            int gy = lo1 + y, gz = lo2 + z;
            if (PERIODIC) {
                gy = wrap(gy, grid.n(1));
                gz = wrap(gz, grid.n(2));
            }
            cplx_t<T> *grow = grid.row(gz, gy);
            const int t0 = z * ps + y * txi;
            for (int x = lane; x < txi; x += 32) {
                T re, im;
                if (fixed) {
                    const int hr = tHr[t0 + x], lr = tLr[t0 + x], hi = tHi[t0 + x], li = tLi[t0 + x];
                    if ((hr | lr | hi | li) == 0) continue;
                    // (H 2^22 + L) exactly as a 64-bit integer (|.| < 2^51), times the unit
                    re = (T)i64_pow2(((long long)hr << 22) + lr, e - 43);
                    im = (T)i64_pow2(((long long)hi << 22) + li, e - 43);
                } else {
                    re = tre[t0 + x];
                    im = tim[t0 + x];
                    if (re == T(0) && im == T(0)) continue;
                }
                const int gx = PERIODIC ? wrap(lo0 + x, grid.n(0)) : lo0 + x;
                grid_add(grow + gx, re, im);
            }
        }
    }
}

// sky -> vis step 1: pixels (values c, prephase P) onto the n1 grids of a wave. blockIdx.y
// picks the sub-problem (descs[b0 + blockIdx.y]); a CTA takes ppc <= 128 consecutive points
// of it (the bin; the plan may tune it): thread t < ppc takes point blockIdx.x * ppc + t.
template <typename T, int W, bool IT>
__global__ void __launch_bounds__(kSpreadThreads, sizeof(T) == 4 ? 2 : 1)
    spread_pix_kernel(const NufftDev *__restrict__ descs, int b0, cplx_t<T> *__restrict__ G1,
                      const float4 *__restrict__ rh, const float4 *__restrict__ rl, const double *__restrict__ soa,
                      int64_t n_all, const T *__restrict__ c, T beta, int isign, int ppc) {
    __shared__ NufftDev sb;
    load_desc(sb, descs + b0 + blockIdx.y);
    const NufftDev &b = sb;
    if ((int64_t)blockIdx.x * ppc >= b.np) return;  // this sub-problem has fewer bins (uniform)
    const int64_t i = blockIdx.x * (int64_t)ppc + threadIdx.x;
    const bool act = threadIdx.x < ppc && i < b.np;
    int i0[3] = {0, 0, 0};
    T fr[3] = {0, 0, 0}, vr = 0, vi = 0;
    if (act) {
        T pr, pim;
        geo_pix<W>(b, b.p0 + i, rh, rl, soa, n_all, isign, i0, fr, pr, pim);
        const T cv = c[b.p0 + i];
        vr = cv * pr;
        vi = cv * pim;
    }
    if constexpr (IT)
        spread_cta_fixed<T, W, false>(act, i0, fr, vr, vi, beta, SpreadGrid<T, false>{b, G1}, ppc);
    else
        spread_cta<T, W, false>(act, i0, fr, vr, vi, beta, SpreadGrid<T, false>{b, G1}, ppc);
}

// vis -> sky step 1 (transpose of the interpolation): baselines u = conj(Q) V onto the n2
// grids of a wave (layout as for pixels).
template <typename T, int W, bool IT>
__global__ void __launch_bounds__(kSpreadThreads, sizeof(T) == 4 ? 2 : 1)
    spread_vis_kernel(const NufftDev *__restrict__ descs, int b0, cplx_t<T> *__restrict__ G2,
                      const float4 *__restrict__ vh, const float4 *__restrict__ vl, const double *__restrict__ soa,
                      int64_t n_all, const cplx_t<T> *__restrict__ V, const T *__restrict__ cc, int deg,
                      T inv_tmax2, T beta, int isign, int ppc) {
    __shared__ NufftDev sb;
    load_desc(sb, descs + b0 + blockIdx.y);
    const NufftDev &b = sb;
    if ((int64_t)blockIdx.x * ppc >= b.nv) return;
    const int64_t k = blockIdx.x * (int64_t)ppc + threadIdx.x;
    const bool act = threadIdx.x < ppc && k < b.nv;
    int i0[3] = {0, 0, 0};
    T fr[3] = {0, 0, 0}, ur = 0, ui = 0;
    if (act) {
        T qr, qi;
        geo_vis<W>(b, b.v0 + k, vh, vl, soa, n_all, isign, cc, deg, inv_tmax2, i0, fr, qr, qi);
        const cplx_t<T> v = V[b.v0 + k];
        ur = qr * v.x + qi * v.y;  // conj(Q) v
        ui = qr * v.y - qi * v.x;
    }
    if constexpr (IT)
        spread_cta_fixed<T, W, true>(act, i0, fr, ur, ui, beta, SpreadGrid<T, true>{b, G2}, ppc);
    else
        spread_cta<T, W, true>(act, i0, fr, ur, ui, beta, SpreadGrid<T, true>{b, G2}, ppc);
}

// ------------------------------------------------------------------ interpolation (gather)

// Baselines (sparse on the n2 grid): the mirror of the spreading layout. A CTA of 256
// threads takes 128 points; threads
// 0..127 stage each point's window start, kernel weights and output factor in shared
// memory; then 8 lanes per point sweep the window's x taps (lane j: taps j and j + 8), so a
// group's 8 loads of a grid row are one contiguous 64-byte (FP32) segment, and the group
// sums its partial results with shuffles.
constexpr int kGatherThreads = 256;

template <typename T, int W> struct GatherShared {
    static constexpr int kWStride = 3 * W + 1;
    T w[kSpreadPoints][kWStride];  // x, y, z weights of each point
    T q[kSpreadPoints][2];         // complex factor applied to the window sum
    int i0[kSpreadPoints][3];      // window start (i0[.][0] = INT_MIN: no point)
};

template <typename T, int W>
__device__ __forceinline__ void stage_point(GatherShared<T, W> &sh, int slot, bool act, const int i0[3],
                                            const T fr[3], T qr, T qi, T beta) {
    if (!act) {
        sh.i0[slot][0] = INT_MIN;
        return;
    }
    T wx[W], wy[W], wz[W];
    es_weights<T, W>(fr[0], beta, wx);
    es_weights<T, W>(fr[1], beta, wy);
    es_weights<T, W>(fr[2], beta, wz);
#pragma unroll
    for (int j = 0; j < W; ++j) {
        sh.w[slot][j] = wx[j];
        sh.w[slot][W + j] = wy[j];
        sh.w[slot][2 * W + j] = wz[j];
    }
    sh.q[slot][0] = qr;
    sh.q[slot][1] = qi;
#pragma unroll
    for (int d = 0; d < 3; ++d) sh.i0[slot][d] = i0[d];
}

// Window sum of point `slot` over grid G (this lane's x taps), reduced over the group's 8
// lanes: every lane of the group returns the full sum.
template <typename T, int W, bool PERIODIC>
__device__ __forceinline__ void gather_window(const GatherShared<T, W> &sh, int slot, int jx0, const int ng[3],
                                              int64_t zs, const cplx_t<T> *__restrict__ G, unsigned mask, T &sr,
                                              T &si) {
    constexpr int kXT = (W + kGroupLanes - 1) / kGroupLanes;
    const int px0 = sh.i0[slot][0], py0 = sh.i0[slot][1], pz0 = sh.i0[slot][2];
    const int64_t nx = ng[0];
    T wxv[kXT];
    int cx[kXT];
    bool on[kXT];
#pragma unroll
    for (int t = 0; t < kXT; ++t) {
        const int jx = jx0 + t * kGroupLanes;
        on[t] = jx < W;
        wxv[t] = on[t] ? sh.w[slot][jx] : T(0);
        cx[t] = on[t] ? (PERIODIC ? wrap(px0 + jx, ng[0]) : px0 + jx) : (PERIODIC ? 0 : px0);
    }
    int yrow[W];
#pragma unroll
    for (int j = 0; j < W; ++j) yrow[j] = PERIODIC ? wrap(py0 + j, ng[1]) : py0 + j;
    sr = T(0);
    si = T(0);
    for (int jz = 0; jz < W; ++jz) {
        const T wz = sh.w[slot][2 * W + jz];
        const int64_t zoff = (int64_t)(PERIODIC ? wrap(pz0 + jz, ng[2]) : pz0 + jz) * zs;
#pragma unroll
        for (int jy = 0; jy < W; ++jy) {
            const T c = sh.w[slot][W + jy] * wz;
            const cplx_t<T> *row = G + zoff + yrow[jy] * nx;
#pragma unroll
            for (int t = 0; t < kXT; ++t)
                if (on[t]) {
                    const cplx_t<T> g = row[cx[t]];
                    const T f = wxv[t] * c;
                    sr += g.x * f;
                    si += g.y * f;
                }
        }
    }
#pragma unroll
    for (int off = kGroupLanes / 2; off > 0; off >>= 1) {
        sr += __shfl_xor_sync(mask, sr, off, kGroupLanes);
        si += __shfl_xor_sync(mask, si, off, kGroupLanes);
    }
}

// sky -> vis steps 3-4: gather the n2 grids of a wave at the baselines, times Q; add into
// acc. blockIdx.y picks the sub-problem, blockIdx.x a tile of 128 of its baselines.
template <typename T, int W>
__global__ void __launch_bounds__(kGatherThreads)
    interp_vis_kernel(const NufftDev *__restrict__ descs, int b0, const cplx_t<T> *__restrict__ G2base,
                      const float4 *__restrict__ vh, const float4 *__restrict__ vl, const double *__restrict__ soa,
                      int64_t n_all, const T *__restrict__ cc, int deg, T inv_tmax2, cplx_t<T> *__restrict__ acc,
                      T beta, int isign) {
    __shared__ GatherShared<T, W> sh;
    __shared__ NufftDev sb;
    load_desc(sb, descs + b0 + blockIdx.y);
    const NufftDev &b = sb;
    const int tid = threadIdx.x;
    const int64_t base = blockIdx.x * (int64_t)kSpreadPoints;
    if (base >= b.nv) return;  // uniform
    if (tid < kSpreadPoints) {
        const int64_t k = base + tid;
        int i0[3] = {0, 0, 0};
        T fr[3] = {0, 0, 0}, qr = 0, qi = 0;
        const bool act = k < b.nv;
        if (act) geo_vis<W>(b, b.v0 + k, vh, vl, soa, n_all, isign, cc, deg, inv_tmax2, i0, fr, qr, qi);
        stage_point<T, W>(sh, tid, act, i0, fr, qr, qi, beta);
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5, g = lane / kGroupLanes, jx0 = lane % kGroupLanes;
    const unsigned mask = 0xFFu << (g * kGroupLanes);
    const int ng[3] = {b.n2[0], b.n2[1], b.n2[2]};
    const cplx_t<T> *G2 = G2base + b.g2_off;
    constexpr int kRounds = kSpreadPoints * kGroupLanes / kGatherThreads;
    for (int round = 0; round < kRounds; ++round) {
        const int p = g * 32 + warp * kRounds + round;
        if (sh.i0[p][0] == INT_MIN) continue;
        T sr, si;
        gather_window<T, W, true>(sh, p, jx0, ng, b.zs2, G2, mask, sr, si);
        if (jx0 == 0) {
            const T qr = sh.q[p][0], qi = sh.q[p][1];
            grid_add(acc + b.v0 + base + p, qr * sr - qi * si, qr * si + qi * sr);
        }
    }
}

// vis -> sky steps 3-4 (transpose of the spreading): gather the n1 grids of a wave at the
// pixels, times conj(P), real part into acc. One thread per pixel: neighbouring pixels'
// windows overlap on the n1 grid, so their row loads hit L1 (95 %), and this layout
// measured faster here than the 8-lanes-per-point one used for the baselines.
template <typename T, int W>
__global__ void __launch_bounds__(128)
    interp_pix_kernel(const NufftDev *__restrict__ descs, int b0, const cplx_t<T> *__restrict__ G1base,
                      const float4 *__restrict__ rh, const float4 *__restrict__ rl, const double *__restrict__ soa,
                      int64_t n_all, T *__restrict__ acc, T beta, int isign) {
    __shared__ NufftDev sb;
    load_desc(sb, descs + b0 + blockIdx.y);
    const NufftDev &b = sb;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= b.np) return;
    int i0[3];
    T fr[3], pr, pim;
    geo_pix<W>(b, b.p0 + i, rh, rl, soa, n_all, isign, i0, fr, pr, pim);
    T wx[W], wy[W], wz[W];
    es_weights<T, W>(fr[0], beta, wx);
    es_weights<T, W>(fr[1], beta, wy);
    es_weights<T, W>(fr[2], beta, wz);
    const int64_t nx = b.n1[0], ny = b.n1[1];
    const cplx_t<T> *G1 = G1base + b.g1_off;
    T sr = 0, si = 0;
    for (int jz = 0; jz < W; ++jz) {
        for (int jy = 0; jy < W; ++jy) {
            const cplx_t<T> *row = G1 + ((int64_t)(i0[2] + jz) * ny + (i0[1] + jy)) * nx + i0[0];
            T rr = 0, ri = 0;
#pragma unroll
            for (int jx = 0; jx < W; ++jx) {
                const cplx_t<T> g = row[jx];
                rr += g.x * wx[jx];
                ri += g.y * wx[jx];
            }
            const T wyz = wy[jy] * wz[jz];
            sr += rr * wyz;
            si += ri * wyz;
        }
    }
    atomicAdd(acc + b.p0 + i, pr * sr + pim * si);  // Re(conj(P) y)
}

// FP64 plans whose grids hold float pairs after the double-float FFT: the gathers in
// double-float arithmetic on the FP32 pipes. The kernel weights are evaluated in FP64 once
// per point and split into float pairs; every tap is a double-float product added to a
// lazy double-float sum (~24 FP32 instructions, where the FP64 form spends two FP64 FMAs
// issued at 1/64 of the FP32 rate). Layout as the FP64 kernels above.
template <int W> struct GatherSharedDF {
    static constexpr int kWStride = 3 * W + 1;
    float2 w[kSpreadPoints][kWStride];  // x, y, z weights of each point (hi, lo)
    double q[kSpreadPoints][2];         // complex factor applied to the window sum
    int i0[kSpreadPoints][3];           // window start (i0[.][0] = INT_MIN: no point)
};

template <int W>
__device__ __forceinline__ void stage_point_df(GatherSharedDF<W> &sh, int slot, bool act, const int i0[3],
                                               const double fr[3], double qr, double qi, double beta) {
    if (!act) {
        sh.i0[slot][0] = INT_MIN;
        return;
    }
    const df::DF bdf = df::split_bits(beta);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        df::DF t[W];
        es_weights_df<W>(fr[d], bdf, t);
#pragma unroll
        for (int j = 0; j < W; ++j) sh.w[slot][d * W + j] = make_float2(t[j].h, t[j].l);
    }
    sh.q[slot][0] = qr;
    sh.q[slot][1] = qi;
#pragma unroll
    for (int d = 0; d < 3; ++d) sh.i0[slot][d] = i0[d];
}

__device__ __forceinline__ df::DF df_of(float2 v) { return {v.x, v.y}; }

// Window sum of point `slot` over the double-float grid G (this lane's x taps), reduced
// over the group's 8 lanes: every lane of the group returns the full sum.
template <int W>
__device__ __forceinline__ void gather_window_df(const GatherSharedDF<W> &sh, int slot, int jx0, const int ng[3],
                                                 int64_t zs, const float4 *__restrict__ G, unsigned mask, double &sr,
                                                 double &si) {
    constexpr int kXT = (W + kGroupLanes - 1) / kGroupLanes;
    const int px0 = sh.i0[slot][0], py0 = sh.i0[slot][1], pz0 = sh.i0[slot][2];
    const int64_t nx = ng[0];
    df::DF wxv[kXT];
    int cx[kXT];
    bool on[kXT];
#pragma unroll
    for (int t = 0; t < kXT; ++t) {
        const int jx = jx0 + t * kGroupLanes;
        on[t] = jx < W;
        wxv[t] = on[t] ? df_of(sh.w[slot][jx]) : df::DF{0.f, 0.f};
        cx[t] = on[t] ? wrap(px0 + jx, ng[0]) : 0;
    }
    int yrow[W];
#pragma unroll
    for (int j = 0; j < W; ++j) yrow[j] = wrap(py0 + j, ng[1]);
    df::DAcc ar{0.f, 0.f}, ai{0.f, 0.f};
    for (int jz = 0; jz < W; ++jz) {
        const df::DF wz = df_of(sh.w[slot][2 * W + jz]);
        const int64_t zoff = (int64_t)wrap(pz0 + jz, ng[2]) * zs;
#pragma unroll
        for (int jy = 0; jy < W; ++jy) {
            const df::DF c = df::dmul(df_of(sh.w[slot][W + jy]), wz);
            const float4 *row = G + zoff + yrow[jy] * nx;
#pragma unroll
            for (int t = 0; t < kXT; ++t)
                if (on[t]) {
                    const float4 g = row[cx[t]];
                    const df::DF f = df::dmul(wxv[t], c);
                    df::acc_fma(ar, {g.x, g.y}, f);
                    df::acc_fma(ai, {g.z, g.w}, f);
                }
        }
    }
    df::DF a = df::acc_done(ar), b = df::acc_done(ai);
#pragma unroll
    for (int off = kGroupLanes / 2; off > 0; off >>= 1) {
        const df::DF oa = {__shfl_xor_sync(mask, a.h, off, kGroupLanes), __shfl_xor_sync(mask, a.l, off, kGroupLanes)};
        const df::DF ob = {__shfl_xor_sync(mask, b.h, off, kGroupLanes), __shfl_xor_sync(mask, b.l, off, kGroupLanes)};
        a = df::dadd(a, oa);
        b = df::dadd(b, ob);
    }
    sr = df::to_double(a);
    si = df::to_double(b);
}

template <int W>
__global__ void __launch_bounds__(kGatherThreads)
    interp_vis_df_kernel(const NufftDev *__restrict__ descs, int b0, const float4 *__restrict__ G2base,
                         const float4 *__restrict__ vh, const float4 *__restrict__ vl, const double *__restrict__ soa,
                         int64_t n_all, const double *__restrict__ cc, int deg, double inv_tmax2,
                         double2 *__restrict__ acc, double beta, int isign) {
    __shared__ GatherSharedDF<W> sh;
    __shared__ NufftDev sb;
    load_desc(sb, descs + b0 + blockIdx.y);
    const NufftDev &b = sb;
    const int tid = threadIdx.x;
    const int64_t base = blockIdx.x * (int64_t)kSpreadPoints;
    if (base >= b.nv) return;  // uniform
    if (tid < kSpreadPoints) {
        const int64_t k = base + tid;
        int i0[3] = {0, 0, 0};
        double fr[3] = {0, 0, 0}, qr = 0, qi = 0;
        const bool act = k < b.nv;
        if (act) geo_vis<W>(b, b.v0 + k, vh, vl, soa, n_all, isign, cc, deg, inv_tmax2, i0, fr, qr, qi);
        stage_point_df<W>(sh, tid, act, i0, fr, qr, qi, beta);
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5, g = lane / kGroupLanes, jx0 = lane % kGroupLanes;
    const unsigned mask = 0xFFu << (g * kGroupLanes);
    const int ng[3] = {b.n2[0], b.n2[1], b.n2[2]};
    const float4 *G2 = G2base + b.g2_off;
    constexpr int kRounds = kSpreadPoints * kGroupLanes / kGatherThreads;
    for (int round = 0; round < kRounds; ++round) {
        const int p = g * 32 + warp * kRounds + round;
        if (sh.i0[p][0] == INT_MIN) continue;
        double sr, si;
        gather_window_df<W>(sh, p, jx0, ng, b.zs2, G2, mask, sr, si);
        if (jx0 == 0) {
            const double qr = sh.q[p][0], qi = sh.q[p][1];
            grid_add(acc + b.v0 + base + p, qr * sr - qi * si, qr * si + qi * sr);
        }
    }
}

template <int W>
__global__ void __launch_bounds__(128)
    interp_pix_df_kernel(const NufftDev *__restrict__ descs, int b0, const float4 *__restrict__ G1base,
                         const float4 *__restrict__ rh, const float4 *__restrict__ rl, const double *__restrict__ soa,
                         int64_t n_all, double *__restrict__ acc, double beta, int isign) {
    __shared__ NufftDev sb;
    load_desc(sb, descs + b0 + blockIdx.y);
    const NufftDev &b = sb;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= b.np) return;
    int i0[3];
    double fr[3], pr, pim;
    geo_pix<W>(b, b.p0 + i, rh, rl, soa, n_all, isign, i0, fr, pr, pim);
    df::DF wx[W], wy[W], wz[W];
    const df::DF bdf = df::split_bits(beta);
    es_weights_df<W>(fr[0], bdf, wx);
    es_weights_df<W>(fr[1], bdf, wy);
    es_weights_df<W>(fr[2], bdf, wz);
    const int64_t nx = b.n1[0], ny = b.n1[1];
    const float4 *G1 = G1base + b.g1_off;
    df::DAcc sr{0.f, 0.f}, si{0.f, 0.f};
    for (int jz = 0; jz < W; ++jz) {
        for (int jy = 0; jy < W; ++jy) {
            const float4 *row = G1 + ((int64_t)(i0[2] + jz) * ny + (i0[1] + jy)) * nx + i0[0];
            df::DAcc rr{0.f, 0.f}, ri{0.f, 0.f};
#pragma unroll
            for (int jx = 0; jx < W; ++jx) {
                const float4 g = row[jx];
                df::acc_fma(rr, {g.x, g.y}, wx[jx]);
                df::acc_fma(ri, {g.z, g.w}, wx[jx]);
            }
            const df::DF wyz = df::dmul(wy[jy], wz[jz]);
            df::acc_fma(sr, df::acc_done(rr), wyz);
            df::acc_fma(si, df::acc_done(ri), wyz);
        }
    }
    // Re(conj(P) y)
    atomicAdd(acc + b.p0 + i, pr * df::to_double(df::acc_done(sr)) + pim * df::to_double(df::acc_done(si)));
}

// ------------------------------------------------------------------ deconvolution passes

// Row-wise passes over (y, z) rows of a grid: each warp takes a contiguous range of rows,
// its lanes sweep x with four independent elements in flight per lane (enough bytes in
// flight to keep HBM busy), and the row index advances without division.
constexpr int kRowThreads = 256;
constexpr int kRowUnroll = 4;

// CTAs per sub-problem of a row pass over a wave of nb sub-problems with at most `rows`
// rows each: at least two rows per warp, about 2,400 CTAs in all.
inline unsigned row_ctas(int64_t rows, int nb) {
    const int64_t warps = (rows + 1) / 2;
    const int64_t ctas = (warps + kRowThreads / 32 - 1) / (kRowThreads / 32);
    const int64_t cap = std::max<int64_t>(8, (152 * 16 + nb - 1) / nb);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ctas, cap));
}

// First row and row count of this warp for `rows` rows split over all warps of the grid.
__device__ __forceinline__ void warp_rows(int64_t rows, int64_t &r0, int64_t &cnt) {
    const int64_t nw = (int64_t)gridDim.x * (kRowThreads / 32);
    const int64_t gw = (int64_t)blockIdx.x * (kRowThreads / 32) + (threadIdx.x >> 5);
    const int64_t per = (rows + nw - 1) / nw;
    r0 = gw * per;
    cnt = r0 < rows ? (rows - r0 < per ? rows - r0 : per) : 0;
}

// G2[j] = G1[l + n1/2] / (Psi_x Psi_y Psi_z)(l) for the centred frequency l of FFT index j
// inside the n1 band, 0 elsewhere (rows of the n2 grid). blockIdx.y picks the sub-problem
// of the wave, whose rows are split over the gridDim.x CTAs.
template <typename T>
__global__ void __launch_bounds__(kRowThreads) deconv_pad_kernel(const NufftDev *__restrict__ descs, int b0,
                                                                 const cplx_t<T> *__restrict__ G1base,
                                                                 cplx_t<T> *__restrict__ G2base,
                                                                 const T *__restrict__ ipsi_all) {
    __shared__ NufftDev sb;
    load_desc(sb, descs + b0 + blockIdx.y);
    const NufftDev &b = sb;
    const int n2x = b.n2[0], n2y = b.n2[1], n2z = b.n2[2];
    const int n1x = b.n1[0], n1y = b.n1[1];
    const int h1x = b.n1[0] / 2, h1y = b.n1[1] / 2, h1z = b.n1[2] / 2;
    const T *ipsi = ipsi_all + b.psi_off;
    const T *px = ipsi, *py = ipsi + n1x, *pz = py + n1y;
    const cplx_t<T> *G1 = G1base + b.g1_off;
    cplx_t<T> *G2 = G2base + b.g2_off;
    int64_t r, cnt;
    warp_rows((int64_t)n2y * n2z, r, cnt);
    if (cnt == 0) return;
    int jy = (int)(r % n2y), jz = (int)(r / n2y);
    const int lane = threadIdx.x & 31;
    for (int64_t k = 0; k < cnt; ++k) {
        cplx_t<T> *out = G2 + (int64_t)jz * b.zs2 + (int64_t)jy * n2x;
        const int ly = jy < n2y / 2 ? jy : jy - n2y;
        const int lz = jz < n2z / 2 ? jz : jz - n2z;
        cplx_t<T> zero;
        zero.x = T(0);
        zero.y = T(0);
        if (ly >= -h1y && ly < h1y && lz >= -h1z && lz < h1z) {
            const int iy = ly + h1y, iz = lz + h1z;
            const T fyz = py[iy] * pz[iz];
            const cplx_t<T> *in = G1 + ((int64_t)iz * n1y + iy) * n1x;
            for (int x0 = lane; x0 < n2x; x0 += 32 * kRowUnroll) {
                cplx_t<T> v[kRowUnroll];
#pragma unroll
                for (int u = 0; u < kRowUnroll; ++u) {
                    const int jx = x0 + 32 * u;
                    const int lx = jx < n2x / 2 ? jx : jx - n2x;
                    v[u] = zero;
                    if (jx < n2x && lx >= -h1x && lx < h1x) {
                        const cplx_t<T> g = in[lx + h1x];
                        const T f = px[lx + h1x] * fyz;
                        v[u].x = g.x * f;
                        v[u].y = g.y * f;
                    }
                }
#pragma unroll
                for (int u = 0; u < kRowUnroll; ++u)
                    if (x0 + 32 * u < n2x) out[x0 + 32 * u] = v[u];
            }
        } else {
            for (int jx = lane; jx < n2x; jx += 32) out[jx] = zero;
        }
        if (++jy == n2y) {
            jy = 0;
            ++jz;
        }
    }
}

// G1[l + n1/2] = G2[l mod n2] / (Psi_x Psi_y Psi_z)(l), l in the n1 band (rows of the n1
// grid), for the sub-problem blockIdx.y of the wave.
template <typename T>
__global__ void __launch_bounds__(kRowThreads) crop_deconv_kernel(const NufftDev *__restrict__ descs, int b0,
                                                                  const cplx_t<T> *__restrict__ G2base,
                                                                  cplx_t<T> *__restrict__ G1base,
                                                                  const T *__restrict__ ipsi_all) {
    __shared__ NufftDev sb;
    load_desc(sb, descs + b0 + blockIdx.y);
    const NufftDev &b = sb;
    const int n1x = b.n1[0], n1y = b.n1[1], n1z = b.n1[2];
    const int n2x = b.n2[0], n2y = b.n2[1], n2z = b.n2[2];
    const T *ipsi = ipsi_all + b.psi_off;
    const T *px = ipsi, *py = ipsi + n1x, *pz = py + n1y;
    const cplx_t<T> *G2 = G2base + b.g2_off;
    cplx_t<T> *G1 = G1base + b.g1_off;
    int64_t r, cnt;
    warp_rows((int64_t)n1y * n1z, r, cnt);
    if (cnt == 0) return;
    int iy = (int)(r % n1y), iz = (int)(r / n1y);
    const int lane = threadIdx.x & 31;
    for (int64_t k = 0; k < cnt; ++k) {
        int jy = iy - n1y / 2, jz = iz - n1z / 2;
        jy += jy < 0 ? n2y : 0;
        jz += jz < 0 ? n2z : 0;
        const cplx_t<T> *in = G2 + (int64_t)jz * b.zs2 + (int64_t)jy * n2x;
        cplx_t<T> *out = G1 + ((int64_t)iz * n1y + iy) * n1x;
        const T fyz = py[iy] * pz[iz];
        for (int x0 = lane; x0 < n1x; x0 += 32 * kRowUnroll) {
            cplx_t<T> v[kRowUnroll];
#pragma unroll
            for (int u = 0; u < kRowUnroll; ++u) {
                const int ix = x0 + 32 * u;
                if (ix < n1x) {
                    int jx = ix - n1x / 2;
                    jx += jx < 0 ? n2x : 0;
                    const cplx_t<T> g = in[jx];
                    const T f = px[ix] * fyz;
                    v[u].x = g.x * f;
                    v[u].y = g.y * f;
                }
            }
#pragma unroll
            for (int u = 0; u < kRowUnroll; ++u)
                if (x0 + 32 * u < n1x) out[x0 + 32 * u] = v[u];
        }
        if (++iy == n1y) {
            iy = 0;
            ++iz;
        }
    }
}

// crop_deconv for double-float grids (after the double-float FFT): reads float-pair cells
// of the n2 band, writes the n1 grid as float pairs for interp_pix_df_kernel; the
// deconvolution factor is formed in FP64 once per cell and multiplied in double-float.
__global__ void __launch_bounds__(kRowThreads) crop_deconv_df_kernel(const NufftDev *__restrict__ descs, int b0,
                                                                     const float4 *__restrict__ G2base,
                                                                     float4 *__restrict__ G1base,
                                                                     const double *__restrict__ ipsi_all) {
    __shared__ NufftDev sb;
    load_desc(sb, descs + b0 + blockIdx.y);
    const NufftDev &b = sb;
    const int n1x = b.n1[0], n1y = b.n1[1], n1z = b.n1[2];
    const int n2x = b.n2[0], n2y = b.n2[1], n2z = b.n2[2];
    const double *ipsi = ipsi_all + b.psi_off;
    const double *px = ipsi, *py = ipsi + n1x, *pz = py + n1y;
    const float4 *G2 = G2base + b.g2_off;
    float4 *G1 = G1base + b.g1_off;
    int64_t r, cnt;
    warp_rows((int64_t)n1y * n1z, r, cnt);
    if (cnt == 0) return;
    int iy = (int)(r % n1y), iz = (int)(r / n1y);
    const int lane = threadIdx.x & 31;
    for (int64_t k = 0; k < cnt; ++k) {
        int jy = iy - n1y / 2, jz = iz - n1z / 2;
        jy += jy < 0 ? n2y : 0;
        jz += jz < 0 ? n2z : 0;
        const float4 *in = G2 + (int64_t)jz * b.zs2 + (int64_t)jy * n2x;
        float4 *out = G1 + ((int64_t)iz * n1y + iy) * n1x;
        const double fyz = py[iy] * pz[iz];
        for (int x0 = lane; x0 < n1x; x0 += 32 * kRowUnroll) {
            float4 v[kRowUnroll];
#pragma unroll
            for (int u = 0; u < kRowUnroll; ++u) {
                const int ix = x0 + 32 * u;
                if (ix < n1x) {
                    int jx = ix - n1x / 2;
                    jx += jx < 0 ? n2x : 0;
                    const float4 g = in[jx];
                    const df::DF f = df::split_bits(px[ix] * fyz);
                    const df::DF re = df::dmul({g.x, g.y}, f), im = df::dmul({g.z, g.w}, f);
                    v[u] = make_float4(re.h, re.l, im.h, im.l);
                }
            }
#pragma unroll
            for (int u = 0; u < kRowUnroll; ++u)
                if (x0 + 32 * u < n1x) out[x0 + 32 * u] = v[u];
        }
        if (++iy == n1y) {
            iy = 0;
            ++iz;
        }
    }
}

#define HVOX_W_SWITCH(w, CALL)                                         \
    switch (w) {                                                       \
        case 2: CALL(2); break;                                        \
        case 3: CALL(3); break;                                        \
        case 4: CALL(4); break;                                        \
        case 5: CALL(5); break;                                        \
        case 6: CALL(6); break;                                        \
        case 7: CALL(7); break;                                        \
        case 8: CALL(8); break;                                        \
        case 9: CALL(9); break;                                        \
        case 10: CALL(10); break;                                      \
        case 11: CALL(11); break;                                      \
        case 12: CALL(12); break;                                      \
        case 13: CALL(13); break;                                      \
        case 14: CALL(14); break;                                      \
        case 15: CALL(15); break;                                      \
        case 16: CALL(16); break;                                      \
        default: fail(HVOX_EUNSUPPORTED, "kernel width out of range"); \
    }

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }


// Dynamic shared memory of the spreading kernels: the tile (real and imaginary planes).
template <typename T, int W> void set_smem_attrs() {
    // Once per instantiation, also when plans are built and run on several host threads.
    static std::once_flag once;
    std::call_once(once, [] {
        for (auto k : {spread_pix_kernel<T, W, false>, spread_pix_kernel<T, W, sizeof(T) == 8>})
            check_cuda(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, tile_bytes<T, W>()),
                       "cudaFuncSetAttribute");
        for (auto k : {spread_vis_kernel<T, W, false>, spread_vis_kernel<T, W, sizeof(T) == 8>})
            check_cuda(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, tile_bytes<T, W>()),
                       "cudaFuncSetAttribute");
    });
}

}  // namespace

// ------------------------------------------------------------------ host launchers

// In-place transforms of one batch of FFT grids with sign dir. band_input: only the n1
// band's z planes are nonzero (sky -> vis: 2-D transforms of those planes, then z);
// otherwise only those planes are read afterwards (vis -> sky: z first, then 2-D).
// Returns the number of cuFFT executions.
template <typename T> int fft_batch(const FftBatch &f, int dir, bool band_input, cudaStream_t s) {
    if (f.df) return dfft_batch(f, dir, band_input, s);
    auto exec = [&](cufftHandle h, void *g) {
        check_cufft(cufftSetStream(h, s), "cufftSetStream");
        if constexpr (sizeof(T) == 4)
            check_cufft(cufftExecC2C(h, (cufftComplex *)g, (cufftComplex *)g, dir), "cufftExecC2C");
        else
            check_cufft(cufftExecZ2Z(h, (cufftDoubleComplex *)g, (cufftDoubleComplex *)g, dir), "cufftExecZ2Z");
    };
    if (f.plans.full) {
        exec(f.plans.full, f.g2);
        return 1;
    }
    const int64_t planes = f.n2[0] * f.n2[1] * f.K;  // one interleaved z plane of all K grids
    void *upper = static_cast<typename CplxOf<T>::type *>(f.g2) + (f.n2[2] - f.half) * planes;
    if (band_input) {
        exec(f.plans.xy, f.g2);
        exec(f.plans.xy, upper);
        exec(f.plans.z, f.g2);
    } else {
        exec(f.plans.z, f.g2);
        exec(f.plans.xy, f.g2);
        exec(f.plans.xy, upper);
    }
    return 3;
}

template <typename T>
void nufft_wave_s2v(const Wave &w, const NufftArgs<T> &a, void *g1, void *g2, const T *c, cplx_t<T> *acc,
                    cudaStream_t s, StageHook &hook) {
    const int wd = a.w;
    const T bt = (T)a.beta;
    const dim3 sgrid(blocks_for(w.max_np, a.ppc_pix), (unsigned)w.nb);
    const dim3 dgrid(row_ctas(w.max_rows2, w.nb), (unsigned)w.nb);
    const dim3 igrid(blocks_for(w.max_nv, kSpreadPoints), (unsigned)w.nb);
    hook.begin(HVOX_STAGE_ZERO, s);
    check_cuda(cudaMemsetAsync(g1, 0, sizeof(cplx_t<T>) * w.g1_cells, s), "memset G1");
    hook.end(HVOX_STAGE_ZERO, 1, s);
    hook.begin(HVOX_STAGE_SPREAD, s);
#define CALL(W)                                                                                                   \
    set_smem_attrs<T, W>();                                                                                       \
    (a.int_tile ? spread_pix_kernel<T, W, sizeof(T) == 8> : spread_pix_kernel<T, W, false>)<<<sgrid, kSpreadThreads, tile_bytes<T, W>(), s>>>(                                   \
        a.descs, w.b0, static_cast<cplx_t<T> *>(g1), a.pix_hi, a.pix_lo, a.pix_soa, a.n_pix, c, bt, a.isign,    \
        a.ppc_pix)
    HVOX_W_SWITCH(wd, CALL)
#undef CALL
    check_cuda(cudaGetLastError(), "spread_pix");
    hook.end(HVOX_STAGE_SPREAD, 1, s);
    hook.begin(HVOX_STAGE_DECONV, s);
    deconv_pad_kernel<T><<<dgrid, kRowThreads, 0, s>>>(a.descs, w.b0, static_cast<const cplx_t<T> *>(g1),
                                                       static_cast<cplx_t<T> *>(g2), a.ipsi);
    check_cuda(cudaGetLastError(), "deconv_pad");
    hook.end(HVOX_STAGE_DECONV, 1, s);
    hook.begin(HVOX_STAGE_FFT, s);
    int n_fft = 0;
    for (const FftBatch &f : w.ffts) n_fft += fft_batch<T>(f, a.isign < 0 ? CUFFT_FORWARD : CUFFT_INVERSE, true, s);
    hook.end(HVOX_STAGE_FFT, n_fft, s);
    hook.begin(HVOX_STAGE_INTERP, s);
    if constexpr (sizeof(T) == 8) {
        if (a.df_grids) {
#define CALL(W)                                                                                                   \
    interp_vis_df_kernel<W><<<igrid, kGatherThreads, 0, s>>>(a.descs, w.b0, static_cast<const float4 *>(g2),      \
                                                             a.vis_hi, a.vis_lo, a.vis_soa, a.n_vis, a.cheb, a.deg, \
                                                             a.inv_tmax2, acc, a.beta, a.isign)
            HVOX_W_SWITCH(wd, CALL)
#undef CALL
            check_cuda(cudaGetLastError(), "interp_vis_df");
            hook.end(HVOX_STAGE_INTERP, 1, s);
            return;
        }
    }
#define CALL(W)                                                                                                   \
    interp_vis_kernel<T, W><<<igrid, kGatherThreads, 0, s>>>(                                                \
        a.descs, w.b0, static_cast<const cplx_t<T> *>(g2), a.vis_hi, a.vis_lo, a.vis_soa, a.n_vis, a.cheb, a.deg, \
        (T)a.inv_tmax2, acc, bt, a.isign)
    HVOX_W_SWITCH(wd, CALL)
#undef CALL
    check_cuda(cudaGetLastError(), "interp_vis");
    hook.end(HVOX_STAGE_INTERP, 1, s);
}

template <typename T>
void nufft_wave_v2s(const Wave &w, const NufftArgs<T> &a, void *g1, void *g2, const cplx_t<T> *V, T *acc,
                    cudaStream_t s, StageHook &hook) {
    const int wd = a.w;
    const T bt = (T)a.beta;
    const dim3 sgrid(blocks_for(w.max_nv, a.ppc_vis), (unsigned)w.nb);
    const dim3 cgrid(row_ctas(w.max_rows1, w.nb), (unsigned)w.nb);
    const dim3 igrid(blocks_for(w.max_np, 128), (unsigned)w.nb);
    hook.begin(HVOX_STAGE_ZERO, s);
    check_cuda(cudaMemsetAsync(g2, 0, sizeof(cplx_t<T>) * w.g2_cells, s), "memset G2");
    hook.end(HVOX_STAGE_ZERO, 1, s);
    hook.begin(HVOX_STAGE_SPREAD, s);
#define CALL(W)                                                                                                   \
    set_smem_attrs<T, W>();                                                                                       \
    (a.int_tile ? spread_vis_kernel<T, W, sizeof(T) == 8> : spread_vis_kernel<T, W, false>)<<<sgrid, kSpreadThreads, tile_bytes<T, W>(), s>>>(                                   \
        a.descs, w.b0, static_cast<cplx_t<T> *>(g2), a.vis_hi, a.vis_lo, a.vis_soa, a.n_vis, V, a.cheb, a.deg,   \
        (T)a.inv_tmax2, bt, a.isign, a.ppc_vis)
    HVOX_W_SWITCH(wd, CALL)
#undef CALL
    check_cuda(cudaGetLastError(), "spread_vis");
    hook.end(HVOX_STAGE_SPREAD, 1, s);
    hook.begin(HVOX_STAGE_FFT, s);
    int n_fft = 0;
    for (const FftBatch &f : w.ffts)  // transpose: opposite sign
        n_fft += fft_batch<T>(f, a.isign < 0 ? CUFFT_INVERSE : CUFFT_FORWARD, false, s);
    hook.end(HVOX_STAGE_FFT, n_fft, s);
    if constexpr (sizeof(T) == 8) {
        if (a.df_grids) {
            hook.begin(HVOX_STAGE_DECONV, s);
            crop_deconv_df_kernel<<<cgrid, kRowThreads, 0, s>>>(a.descs, w.b0, static_cast<const float4 *>(g2),
                                                                static_cast<float4 *>(g1), a.ipsi);
            check_cuda(cudaGetLastError(), "crop_deconv_df");
            hook.end(HVOX_STAGE_DECONV, 1, s);
            hook.begin(HVOX_STAGE_INTERP, s);
#define CALL(W)                                                                                                   \
    interp_pix_df_kernel<W><<<igrid, 128, 0, s>>>(a.descs, w.b0, static_cast<const float4 *>(g1), a.pix_hi,      \
                                                  a.pix_lo, a.pix_soa, a.n_pix, acc, a.beta, a.isign)
            HVOX_W_SWITCH(wd, CALL)
#undef CALL
            check_cuda(cudaGetLastError(), "interp_pix_df");
            hook.end(HVOX_STAGE_INTERP, 1, s);
            return;
        }
    }
    hook.begin(HVOX_STAGE_DECONV, s);
    crop_deconv_kernel<T><<<cgrid, kRowThreads, 0, s>>>(a.descs, w.b0, static_cast<const cplx_t<T> *>(g2),
                                                        static_cast<cplx_t<T> *>(g1), a.ipsi);
    check_cuda(cudaGetLastError(), "crop_deconv");
    hook.end(HVOX_STAGE_DECONV, 1, s);
    hook.begin(HVOX_STAGE_INTERP, s);
#define CALL(W)                                                                                                   \
    interp_pix_kernel<T, W><<<igrid, 128, 0, s>>>(a.descs, w.b0, static_cast<const cplx_t<T> *>(g1), a.pix_hi,  \
                                                  a.pix_lo, a.pix_soa, a.n_pix, acc, bt, a.isign)
    HVOX_W_SWITCH(wd, CALL)
#undef CALL
    check_cuda(cudaGetLastError(), "interp_pix");
    hook.end(HVOX_STAGE_INTERP, 1, s);
}

template <typename T>
float time_spread(const Wave &w, const NufftArgs<T> &a, void *g1, void *g2, bool pix, const void *values, int ppc,
                  cudaStream_t s) {
    const int wd = a.w;
    const T bt = (T)a.beta;
    check_cuda(cudaMemsetAsync(pix ? g1 : g2, 0, sizeof(cplx_t<T>) * (pix ? w.g1_cells : w.g2_cells), s),
               "memset grid");
    cudaEvent_t e0, e1;
    check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
    check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
    check_cuda(cudaEventRecord(e0, s), "cudaEventRecord");
    const dim3 grid(blocks_for(pix ? w.max_np : w.max_nv, ppc), (unsigned)w.nb);
    if (pix) {
#define CALL(W)                                                                                                   \
    set_smem_attrs<T, W>();                                                                                       \
    (a.int_tile ? spread_pix_kernel<T, W, sizeof(T) == 8> : spread_pix_kernel<T, W, false>)<<<grid, kSpreadThreads, tile_bytes<T, W>(), s>>>(                                    \
        a.descs, w.b0, static_cast<cplx_t<T> *>(g1), a.pix_hi, a.pix_lo, a.pix_soa, a.n_pix, (const T *)values, \
        bt, a.isign, ppc)
        HVOX_W_SWITCH(wd, CALL)
#undef CALL
    } else {
#define CALL(W)                                                                                                   \
    set_smem_attrs<T, W>();                                                                                       \
    (a.int_tile ? spread_vis_kernel<T, W, sizeof(T) == 8> : spread_vis_kernel<T, W, false>)<<<grid, kSpreadThreads, tile_bytes<T, W>(), s>>>(                                    \
        a.descs, w.b0, static_cast<cplx_t<T> *>(g2), a.vis_hi, a.vis_lo, a.vis_soa, a.n_vis,                   \
        (const cplx_t<T> *)values, a.cheb, a.deg, (T)a.inv_tmax2, bt, a.isign, ppc)
        HVOX_W_SWITCH(wd, CALL)
#undef CALL
    }
    check_cuda(cudaGetLastError(), "spread (timing)");
    check_cuda(cudaEventRecord(e1, s), "cudaEventRecord");
    check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

template float time_spread<float>(const Wave &, const NufftArgs<float> &, void *, void *, bool, const void *, int,
                                  cudaStream_t);
template float time_spread<double>(const Wave &, const NufftArgs<double> &, void *, void *, bool, const void *, int,
                                   cudaStream_t);
template void nufft_wave_s2v<float>(const Wave &, const NufftArgs<float> &, void *, void *, const float *, float2 *,
                                    cudaStream_t, StageHook &);
template void nufft_wave_s2v<double>(const Wave &, const NufftArgs<double> &, void *, void *, const double *,
                                     double2 *, cudaStream_t, StageHook &);
template void nufft_wave_v2s<float>(const Wave &, const NufftArgs<float> &, void *, void *, const float2 *, float *,
                                    cudaStream_t, StageHook &);
template void nufft_wave_v2s<double>(const Wave &, const NufftArgs<double> &, void *, void *, const double2 *,
                                     double *, cudaStream_t, StageHook &);

}  // namespace hvox
