// Direct evaluation of sub-problems (Sect. 3.1: blocks below a size threshold are
// summed directly, O(n_pix n_vis), Sect. 2) and the point preparation kernels.
//
//   sky -> vis:  V_k += sum_n c_n exp(+isign j 2 pi <p_k, r_n>),  c_n = a_n I_n
//   vis -> sky:  I_n += Re sum_k V_k exp(-isign j 2 pi <p_k, r_n>)
//
// The phase <p, r> reaches ~1e5 turns, so it is never formed in plain FP32. Every
// coordinate is stored as a pair of floats hi + lo (hi = fl32(x), lo = fl32(x - hi)).
// Per pair the main products hi(p) hi(r) are split exactly (TwoProduct by fma), their
// integer turns dropped exactly, and only the fraction of a turn is carried on:
//  * FP32 path (eps >= 1e-6): fraction in FP32 (abs error ~1e-7 turn), hardware
//    sin/cos approximations, FP32 accumulation;
//  * double-float path (eps < 1e-6): fraction as an unevaluated float pair; exp(j 2 pi f)
//    as the hi parts of a periodic 2048-entry table of exp(j 2 pi m / 2048) plus a lo part
//    (the table's lo parts and a short series in the remainder, in plain float; error
//    2.7e-10); products and sums in double-float arithmetic (Dekker 1971);
//  * plain path: everything in FP64 (the reference form the optimised paths replace).
#include <cstdint>
#include <mutex>
#include <string>

#include "hvox_internal.h"

namespace hvox {

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 2;
constexpr int kTile = kThreads * kPerThread;  // owner points per work item

// ------------------------------------------------------------- point preparation

__global__ void prepare_points_kernel(const double *__restrict__ xyz, const int32_t *__restrict__ perm, int64_t n,
                                      double *__restrict__ soa, float4 *__restrict__ hi, float4 *__restrict__ lo) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t src = perm[i];
    float h[3], l[3];
    for (int d = 0; d < 3; ++d) {
        double x = xyz[3 * src + d];
        soa[d * n + i] = x;
        h[d] = (float)x;
        l[d] = (float)(x - (double)h[d]);
    }
    hi[i] = make_float4(h[0], h[1], h[2], 0.f);
    lo[i] = make_float4(l[0], l[1], l[2], 0.f);
}

__global__ void gather_weight_kernel(const double *__restrict__ w, const int32_t *__restrict__ perm, int64_t n,
                                     double *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = w[perm[i]];
}

// ------------------------------------------------------------- float helpers

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Round to nearest integer on the FMA pipe: adding and subtracting 1.5 * 2^23 leaves the
// integer part for |x| < 2^22 (rintf would use the XU pipe, which the sin/cos need).
constexpr float kRoundMagic = 12582912.0f;

__device__ __forceinline__ float round_fma(float x) { return __fsub_rn(__fadd_rn(x, kRoundMagic), kRoundMagic); }

// x - nearest integer, exact (the difference of a float and its rounding is exact).
__device__ __forceinline__ float frac_fma(float x) { return __fsub_rn(x, round_fma(x)); }

// Fraction of hi(p) hi(r) in turns for one dimension, in three FMA-pipe instructions:
// t = fl(p r + 1.5 * 2^23) carries n = round(p r) exactly (float spacing 1 there, for
// |p r| < 2^22), and fma(p, r, -n) forms the exact p r - n (|.| <= 1/2) with one rounding
// (<= 2^-25 turn).
__device__ __forceinline__ float prod_frac(float p, float r) {
    const float n = __fsub_rn(__fmaf_rn(p, r, kRoundMagic), kRoundMagic);
    return __fmaf_rn(p, r, -n);
}

// Fraction of <p, r> in turns, FP32 (|error| ~ 1e-7 turn), result in [-0.5, 0.5].
// Valid for |p_d r_d| < 2^22 turns per dimension.
__device__ __forceinline__ float phase_f32(const float3 &ph, const float3 &pl, const float4 &rh, const float4 &rl) {
    float small = __fmaf_rn(ph.x, rl.x, __fmul_rn(pl.x, rh.x));
    small = __fmaf_rn(ph.y, rl.y, __fmaf_rn(pl.y, rh.y, small));
    small = __fmaf_rn(ph.z, rl.z, __fmaf_rn(pl.z, rh.z, small));
    const float f = __fadd_rn(__fadd_rn(prod_frac(ph.x, rh.x), prod_frac(ph.y, rh.y)),
                              __fadd_rn(prod_frac(ph.z, rh.z), small));
    return frac_fma(f);
}

// Fraction of <p, r> in turns as an unevaluated float pair fh + fl with |fh| < 2
// (integer turns dropped exactly per dimension; the sum of the three fractions is kept
// exact with TwoSum), |error| ~ 1e-12 turn * |p| / 1e5.
__device__ __forceinline__ void phase_df(const float3 &ph, const float3 &pl, const float4 &rh, const float4 &rl,
                                         float &fh, float &fl) {
    float a0, b0, a1, b1, a2, b2;
    two_prod(ph.x, rh.x, a0, b0);
    two_prod(ph.y, rh.y, a1, b1);
    two_prod(ph.z, rh.z, a2, b2);
    a0 = __fsub_rn(a0, rintf(a0));
    a1 = __fsub_rn(a1, rintf(a1));
    a2 = __fsub_rn(a2, rintf(a2));
    float s1, e1, s2, e2;
    two_sum(a0, a1, s1, e1);
    two_sum(s1, a2, s2, e2);
    float small = __fadd_rn(__fadd_rn(b0, b1), __fadd_rn(b2, __fadd_rn(e1, e2)));
    small = __fmaf_rn(ph.x, rl.x, __fmaf_rn(pl.x, rh.x, small));
    small = __fmaf_rn(ph.y, rl.y, __fmaf_rn(pl.y, rh.y, small));
    small = __fmaf_rn(ph.z, rl.z, __fmaf_rn(pl.z, rh.z, small));
    fast_two_sum(s2, small, fh, fl);
}

constexpr int kTabN = 2048;    // table entries per turn; the table is periodic in m

// exp(j 2 pi f) for f = fh + fl (turns, |fh| < 1024) as re = reh + rel, im = imh + iml.
// (reh, imh) are the hi parts of cos and sin of 2 pi m / 2048 for m = round(2048 fh), read
// from T[m mod 2048] = (cos_h, cos_l, sin_h, sin_l). (rel, iml) collect the table's lo
// parts and the rotation by x = 2 pi (fh - m/2048 + fl), |x| <= pi/2048, through
// cos x - 1 = -x^2/2 and sin x = x - x^3/6 (dropped terms below 3e-13). Every term of a lo
// part is below 1.6e-3 in magnitude, so plain float arithmetic keeps the pair within
// ~2.5e-10 of exp(j 2 pi f); the hi parts need no error-free transformations.
__device__ __forceinline__ void cis_tab(float fh, float fl, const float4 *__restrict__ T, float &reh, float &rel,
                                        float &imh, float &iml) {
    const float t = __fmaf_rn(fh, (float)kTabN, kRoundMagic);  // 1.5 * 2^23 + m
    const int idx = __float_as_int(t) & (kTabN - 1);           // m mod 2048 (the magic's low bits are 0)
    const float d = __fmaf_rn(__fsub_rn(t, kRoundMagic), -1.0f / kTabN, fh);  // fh - m/2048, exact
    const float x = __fmul_rn(__fadd_rn(d, fl), 6.28318530717958648f);
    const float x2 = __fmul_rn(x, x);
    const float cm = __fmul_rn(x2, -0.5f);
    const float sx = __fmaf_rn(__fmul_rn(x2, x), -1.0f / 6.0f, x);
    const float4 tb = T[idx];
    reh = tb.x;
    rel = __fmaf_rn(-tb.z, sx, __fmaf_rn(tb.x, cm, tb.y));
    imh = tb.z;
    iml = __fmaf_rn(tb.x, sx, __fmaf_rn(tb.z, cm, tb.w));
}

__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &ph, float &pl) {
    float p, e;
    two_prod(ah, bh, p, e);
    e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
    ph = p;
    pl = e;
}

// Lazy double-float accumulation: hi carries an exact TwoSum, lo collects the errors.
__device__ __forceinline__ void df_acc(float &acc_h, float &acc_l, float th, float tl) {
    float s, e;
    two_sum(acc_h, th, s, e);
    acc_h = s;
    acc_l = __fadd_rn(acc_l, __fadd_rn(e, tl));
}

// Offset double-float accumulation of one streamed tile: the running high sum starts at a
// power of two M above twice the tile's sum of term magnitudes S, so it stays in
// [M - S, M + S], never below any term, and the rounding error of each add is recovered
// exactly by Fast2Sum (three instructions instead of TwoSum's six). The low part collects
// those errors and the terms' own low parts. At the tile's end hi - M is exact (Sterbenz).
__device__ __forceinline__ void df_acc_off(float &acc_h, float &acc_l, float th, float tl) {
    const float s = __fadd_rn(acc_h, th);
    const float e = __fsub_rn(th, __fsub_rn(s, acc_h));
    acc_h = s;
    acc_l = __fadd_rn(acc_l, __fadd_rn(e, tl));
}

// The offset for a tile whose term magnitudes sum to at most S: 2^(floor(log2 S) + 2) > 2 S
// (S from the block's own values; tiny or zero S gives 2^-100).
__device__ __forceinline__ float tile_offset(float S) {
    const unsigned e = __float_as_uint(fmaxf(S, 0x1p-102f)) & 0x7F800000u;
    return __uint_as_float(e + (2u << 23));
}

// Sum of x over the CTA (every thread gets it). red holds one float per warp; the caller
// has a __syncthreads() between this call and the previous use of red.
__device__ __forceinline__ float block_sum(float x, float *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    return t;
}

// Kahan-compensated accumulation of per-tile partial sums: the FP32 paths sum each
// 256-term shared-memory tile in registers and add the tile sums here, which keeps the
// rounding error of sums over millions of terms near that of a 256-term sum.
__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x) {
    const float y = __fsub_rn(x, comp);
    const float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

// Adds a tile's double-float partial sum (ih + il) into the running sum (oh + ol): the
// lazy accumulation's lo part rounds at ~2^-24 of itself, which over millions of terms
// (1.4M baselines per pixel) grows to ~5e-9 of the result; folding every 256 terms keeps
// that growth to one tile.
__device__ __forceinline__ void df_fold(float &oh, float &ol, float ih, float il) {
    float s, e;
    two_sum(oh, ih, s, e);
    e = __fadd_rn(e, __fadd_rn(ol, il));
    fast_two_sum(s, e, oh, ol);
}

// The next work item of this CTA, taken from the launch's counter (CTA b starts with
// item b; the counter is zero at launch): CTAs that finish early take more items, and
// with the items ordered largest first a launch ends within about one small item of its
// ideal time.
__device__ __forceinline__ int next_item(int *counter, int &s_next) {
    __syncthreads();  // every thread has read the previous s_next
    if (threadIdx.x == 0) s_next = (int)gridDim.x + atomicAdd(counter, 1);
    __syncthreads();
    return s_next;
}

__device__ __forceinline__ void load_tab(float4 *sT, const float4 *__restrict__ gT) {
    for (int i = threadIdx.x; i < kTabN; i += blockDim.x) sT[i] = gT[i];
}

// The pointers of one job of a direct launch: a plan's chunk-ordered buffers. A launch
// serves one job (BATCH false: the kernel parameter J0) or several (BATCH true: work item
// it belongs to job item_job[it] of the device table jobs, so the sums of several plans
// share one launch and its dynamic schedule).
template <bool BATCH>
__device__ __forceinline__ DirectJob job_of(const DirectJob &J0, const DirectJob *__restrict__ jobs,
                                            const int *__restrict__ item_job, int it) {
    if constexpr (BATCH)
        return jobs[item_job[it]];
    else
        return J0;
}

// ------------------------------------------------------------- sky -> vis

// FP32: owner = baselines, streamed = pixels (c real, chunk order).
template <int VPT, bool BATCH>
__global__ void __launch_bounds__(kThreads) direct_s2v_f32(const WorkItem *__restrict__ items, int n_items, int *__restrict__ counter,
    const DirectJob J0, const DirectJob *__restrict__ jobs, const int *__restrict__ item_job) {
    __shared__ float4 sh[kThreads];
    __shared__ float4 sl[kThreads];
    __shared__ int s_next;
    for (int it = blockIdx.x; it < n_items; it = next_item(counter, s_next)) {
        const WorkItem w = items[it];
        const DirectJob J = job_of<BATCH>(J0, jobs, item_job, it);
        const float4 *__restrict__ vh = J.own_hi, *__restrict__ vl = J.own_lo;
        const float4 *__restrict__ rh_g = J.str_hi, *__restrict__ rl_g = J.str_lo;
        const float *__restrict__ c = static_cast<const float *>(J.val);
        float2 *__restrict__ acc = static_cast<float2 *>(J.acc);
        const float sgn = J.sgn;
        float3 ph[VPT], pl[VPT];
        float are[VPT], aim[VPT], cre[VPT], cim[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int k = w.o0 + threadIdx.x + v * kThreads;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (k < w.o1) {
                a = vh[k];
                b = vl[k];
            }
            ph[v] = make_float3(a.x, a.y, a.z);
            pl[v] = make_float3(b.x, b.y, b.z);
            are[v] = aim[v] = cre[v] = cim[v] = 0.f;
        }
        for (int s0 = w.s0; s0 < w.s1; s0 += kThreads) {
            __syncthreads();
            int n = s0 + threadIdx.x;
            if (n < w.s1) {
                float4 a = rh_g[n];
                a.w = c[n];
                sh[threadIdx.x] = a;
                sl[threadIdx.x] = rl_g[n];
            } else {
                sh[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                sl[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();
            const int cnt = min(kThreads, w.s1 - s0);
            float tre[VPT], tim[VPT];
#pragma unroll
            for (int v = 0; v < VPT; ++v) tre[v] = tim[v] = 0.f;
#pragma unroll 4
            for (int q = 0; q < cnt; ++q) {
                const float4 rh = sh[q], rl = sl[q];
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    float f = phase_f32(ph[v], pl[v], rh, rl);
                    float sn, cs;
                    __sincosf(6.28318530717958648f * f, &sn, &cs);
                    tre[v] = __fmaf_rn(rh.w, cs, tre[v]);
                    tim[v] = __fmaf_rn(rh.w, sn, tim[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                kahan_add(are[v], cre[v], tre[v]);
                kahan_add(aim[v], cim[v], tim[v]);
            }
        }
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int k = w.o0 + threadIdx.x + v * kThreads;
            if (k < w.o1) {
                atomicAdd(&acc[k].x, __fsub_rn(are[v], cre[v]));
                atomicAdd(&acc[k].y, sgn * __fsub_rn(aim[v], cim[v]));
            }
        }
    }
}

// Double-float: c given in FP64, accumulation returned in FP64.
template <int VPT, bool BATCH>
__global__ void __launch_bounds__(kThreads, BATCH && VPT == 2 ? 4 : 0) direct_s2v_df(const WorkItem *__restrict__ items, int n_items, int *__restrict__ counter,
    const DirectJob J0, const DirectJob *__restrict__ jobs, const int *__restrict__ item_job, const float4 *__restrict__ gT) {
    __shared__ float4 sh[kThreads];
    __shared__ float4 sl[kThreads];
    __shared__ float2 sc[kThreads];
    __shared__ float4 sT[kTabN];
    __shared__ float red[kThreads / 32];
    load_tab(sT, gT);
    __shared__ int s_next;
    for (int it = blockIdx.x; it < n_items; it = next_item(counter, s_next)) {
        const WorkItem w = items[it];
        const DirectJob J = job_of<BATCH>(J0, jobs, item_job, it);
        const float4 *__restrict__ vh = J.own_hi, *__restrict__ vl = J.own_lo;
        const float4 *__restrict__ rh_g = J.str_hi, *__restrict__ rl_g = J.str_lo;
        const double *__restrict__ c = static_cast<const double *>(J.val);
        double2 *__restrict__ acc = static_cast<double2 *>(J.acc);
        const float sgn = J.sgn;
        float3 ph[VPT], pl[VPT];
        float arh[VPT], arl[VPT], aih[VPT], ail[VPT];  // tile sums, offset by M
        float orh[VPT], orl[VPT], oih[VPT], oil[VPT];  // running sums, folded per tile
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int k = w.o0 + threadIdx.x + v * kThreads;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (k < w.o1) {
                a = vh[k];
                b = vl[k];
            }
            ph[v] = make_float3(a.x, a.y, a.z);
            pl[v] = make_float3(b.x, b.y, b.z);
            arh[v] = arl[v] = aih[v] = ail[v] = 0.f;
            orh[v] = orl[v] = oih[v] = oil[v] = 0.f;
        }
        for (int s0 = w.s0; s0 < w.s1; s0 += kThreads) {
            __syncthreads();
            int n = s0 + threadIdx.x;
            float mag = 0.f;
            if (n < w.s1) {
                sh[threadIdx.x] = rh_g[n];
                sl[threadIdx.x] = rl_g[n];
                double cv = c[n];
                float chi = (float)cv;
                sc[threadIdx.x] = make_float2(chi, (float)(cv - (double)chi));
                mag = fabsf(chi);
            } else {
                sh[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                sl[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                sc[threadIdx.x] = make_float2(0.f, 0.f);
            }
            // |c (cos, sin)| <= |c| (1 + 2^-23): S = 1.01 sum |c| bounds each partial sum
            const float M = tile_offset(1.01f * block_sum(mag, red));
            const int cnt = min(kThreads, w.s1 - s0);
#pragma unroll
            for (int v = 0; v < VPT; ++v) arh[v] = aih[v] = M;
#pragma unroll 4
            for (int q = 0; q < cnt; ++q) {
                const float4 rh = sh[q], rl = sl[q];
                const float2 cv = sc[q];
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    float fh, fl, reh, rel, imh, iml;
                    phase_df(ph[v], pl[v], rh, rl, fh, fl);
                    cis_tab(fh, fl, sT, reh, rel, imh, iml);
                    float th, tl;
                    df_mul(cv.x, cv.y, reh, rel, th, tl);
                    df_acc_off(arh[v], arl[v], th, tl);
                    df_mul(cv.x, cv.y, imh, iml, th, tl);
                    df_acc_off(aih[v], ail[v], th, tl);
                }
            }
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                df_fold(orh[v], orl[v], __fsub_rn(arh[v], M), arl[v]);
                df_fold(oih[v], oil[v], __fsub_rn(aih[v], M), ail[v]);
                arl[v] = ail[v] = 0.f;
            }
        }
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int k = w.o0 + threadIdx.x + v * kThreads;
            if (k < w.o1) {
                atomicAdd(&acc[k].x, (double)orh[v] + (double)orl[v]);
                atomicAdd(&acc[k].y, (double)sgn * ((double)oih[v] + (double)oil[v]));
            }
        }
    }
}

// Plain FP64 reference form.
template <int VPT>
__global__ void __launch_bounds__(kThreads) direct_s2v_f64(const WorkItem *__restrict__ items, int n_items, int *__restrict__ counter,
                                                           const double *__restrict__ vxyz, int64_t nv_all,
                                                           const double *__restrict__ pxyz, int64_t np_all,
                                                           const double *__restrict__ c, double2 *__restrict__ acc,
                                                           double sgn) {
    __shared__ double sx[kThreads], sy[kThreads], sz[kThreads], sw[kThreads];
    __shared__ int s_next;
    for (int it = blockIdx.x; it < n_items; it = next_item(counter, s_next)) {
        const WorkItem w = items[it];
        double px[VPT], py[VPT], pz[VPT], are[VPT], aim[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int k = w.o0 + threadIdx.x + v * kThreads;
            bool ok = k < w.o1;
            px[v] = ok ? vxyz[k] : 0.0;
            py[v] = ok ? vxyz[nv_all + k] : 0.0;
            pz[v] = ok ? vxyz[2 * nv_all + k] : 0.0;
            are[v] = aim[v] = 0.0;
        }
        for (int s0 = w.s0; s0 < w.s1; s0 += kThreads) {
            __syncthreads();
            int n = s0 + threadIdx.x;
            bool ok = n < w.s1;
            sx[threadIdx.x] = ok ? pxyz[n] : 0.0;
            sy[threadIdx.x] = ok ? pxyz[np_all + n] : 0.0;
            sz[threadIdx.x] = ok ? pxyz[2 * np_all + n] : 0.0;
            sw[threadIdx.x] = ok ? c[n] : 0.0;
            __syncthreads();
            const int cnt = min(kThreads, w.s1 - s0);
            for (int q = 0; q < cnt; ++q) {
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    double t = fma(px[v], sx[q], fma(py[v], sy[q], pz[v] * sz[q]));
                    t -= rint(t);
                    double sn, cs;
                    sincospi(2.0 * t, &sn, &cs);
                    are[v] = fma(sw[q], cs, are[v]);
                    aim[v] = fma(sw[q], sn, aim[v]);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int k = w.o0 + threadIdx.x + v * kThreads;
            if (k < w.o1) {
                atomicAdd(&acc[k].x, are[v]);
                atomicAdd(&acc[k].y, sgn * aim[v]);
            }
        }
    }
}

// ------------------------------------------------------------- vis -> sky

// FP32: owner = pixels, streamed = baselines (V complex, chunk order). Output real.
template <int VPT, bool BATCH>
__global__ void __launch_bounds__(kThreads) direct_v2s_f32(const WorkItem *__restrict__ items, int n_items, int *__restrict__ counter,
    const DirectJob J0, const DirectJob *__restrict__ jobs, const int *__restrict__ item_job) {
    __shared__ float4 sh[kThreads];
    __shared__ float4 sl[kThreads];
    __shared__ int s_next;
    for (int it = blockIdx.x; it < n_items; it = next_item(counter, s_next)) {
        const WorkItem w = items[it];
        const DirectJob J = job_of<BATCH>(J0, jobs, item_job, it);
        const float4 *__restrict__ rh_g = J.own_hi, *__restrict__ rl_g = J.own_lo;
        const float4 *__restrict__ vh = J.str_hi, *__restrict__ vl = J.str_lo;
        const float2 *__restrict__ V = static_cast<const float2 *>(J.val);
        float *__restrict__ acc = static_cast<float *>(J.acc);
        const float sgn = J.sgn;
        float3 rh[VPT], rl[VPT];
        float a[VPT], ca[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int n = w.o0 + threadIdx.x + v * kThreads;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
            if (n < w.o1) {
                x = rh_g[n];
                y = rl_g[n];
            }
            rh[v] = make_float3(x.x, x.y, x.z);
            rl[v] = make_float3(y.x, y.y, y.z);
            a[v] = ca[v] = 0.f;
        }
        for (int s0 = w.s0; s0 < w.s1; s0 += kThreads) {
            __syncthreads();
            int k = s0 + threadIdx.x;
            if (k < w.s1) {
                float4 p = vh[k], q = vl[k];
                float2 val = V[k];
                p.w = val.x;
                q.w = sgn * val.y;
                sh[threadIdx.x] = p;
                sl[threadIdx.x] = q;
            } else {
                sh[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                sl[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();
            const int cnt = min(kThreads, w.s1 - s0);
            float ta[VPT];
#pragma unroll
            for (int v = 0; v < VPT; ++v) ta[v] = 0.f;
#pragma unroll 4
            for (int q = 0; q < cnt; ++q) {
                const float4 ph4 = sh[q], pl4 = sl[q];
                const float3 ph = make_float3(ph4.x, ph4.y, ph4.z), pl = make_float3(pl4.x, pl4.y, pl4.z);
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    float4 r4h = make_float4(rh[v].x, rh[v].y, rh[v].z, 0.f);
                    float4 r4l = make_float4(rl[v].x, rl[v].y, rl[v].z, 0.f);
                    float f = phase_f32(ph, pl, r4h, r4l);
                    float sn, cs;
                    __sincosf(6.28318530717958648f * f, &sn, &cs);
                    // Re(V e^{-isign j 2 pi t}) = Vr cos + isign Vi sin
                    ta[v] = __fmaf_rn(ph4.w, cs, __fmaf_rn(pl4.w, sn, ta[v]));
                }
            }
#pragma unroll
            for (int v = 0; v < VPT; ++v) kahan_add(a[v], ca[v], ta[v]);
        }
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int n = w.o0 + threadIdx.x + v * kThreads;
            if (n < w.o1) atomicAdd(&acc[n], __fsub_rn(a[v], ca[v]));
        }
    }
}

template <int VPT, bool BATCH>
__global__ void __launch_bounds__(kThreads) direct_v2s_df(const WorkItem *__restrict__ items, int n_items, int *__restrict__ counter,
    const DirectJob J0, const DirectJob *__restrict__ jobs, const int *__restrict__ item_job, const float4 *__restrict__ gT) {
    __shared__ float4 sh[kThreads];
    __shared__ float4 sl[kThreads];
    __shared__ float4 sv[kThreads];
    __shared__ float4 sT[kTabN];
    __shared__ float red[kThreads / 32];
    load_tab(sT, gT);
    __shared__ int s_next;
    for (int it = blockIdx.x; it < n_items; it = next_item(counter, s_next)) {
        const WorkItem w = items[it];
        const DirectJob J = job_of<BATCH>(J0, jobs, item_job, it);
        const float4 *__restrict__ rh_g = J.own_hi, *__restrict__ rl_g = J.own_lo;
        const float4 *__restrict__ vh = J.str_hi, *__restrict__ vl = J.str_lo;
        const double2 *__restrict__ V = static_cast<const double2 *>(J.val);
        double *__restrict__ acc = static_cast<double *>(J.acc);
        const float sgn = J.sgn;
        float4 rh[VPT], rl[VPT];
        float ah[VPT], al[VPT], oh[VPT], ol[VPT];  // tile sums (offset by M) and running sums
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int n = w.o0 + threadIdx.x + v * kThreads;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
            if (n < w.o1) {
                x = rh_g[n];
                y = rl_g[n];
            }
            rh[v] = x;
            rl[v] = y;
            ah[v] = al[v] = oh[v] = ol[v] = 0.f;
        }
        for (int s0 = w.s0; s0 < w.s1; s0 += kThreads) {
            __syncthreads();
            int k = s0 + threadIdx.x;
            float mag = 0.f;
            if (k < w.s1) {
                sh[threadIdx.x] = vh[k];
                sl[threadIdx.x] = vl[k];
                double2 val = V[k];
                double vi = (double)sgn * val.y;
                float rh_ = (float)val.x, ih_ = (float)vi;
                sv[threadIdx.x] = make_float4(rh_, (float)(val.x - (double)rh_), ih_, (float)(vi - (double)ih_));
                mag = fabsf(rh_) + fabsf(ih_);
            } else {
                sh[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                sl[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                sv[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            // each pair adds Vre cos + Vim sin: S = 1.01 sum (|Vre| + |Vim|) bounds the partial sums
            const float M = tile_offset(1.01f * block_sum(mag, red));
            const int cnt = min(kThreads, w.s1 - s0);
#pragma unroll
            for (int v = 0; v < VPT; ++v) ah[v] = M;
#pragma unroll 4
            for (int q = 0; q < cnt; ++q) {
                const float4 ph4 = sh[q], pl4 = sl[q], val = sv[q];
                const float3 ph = make_float3(ph4.x, ph4.y, ph4.z), pl = make_float3(pl4.x, pl4.y, pl4.z);
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    float fh, fl, reh, rel, imh, iml;
                    phase_df(ph, pl, rh[v], rl[v], fh, fl);
                    cis_tab(fh, fl, sT, reh, rel, imh, iml);
                    float th, tl;
                    df_mul(val.x, val.y, reh, rel, th, tl);
                    df_acc_off(ah[v], al[v], th, tl);
                    df_mul(val.z, val.w, imh, iml, th, tl);
                    df_acc_off(ah[v], al[v], th, tl);
                }
            }
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                df_fold(oh[v], ol[v], __fsub_rn(ah[v], M), al[v]);
                al[v] = 0.f;
            }
        }
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int n = w.o0 + threadIdx.x + v * kThreads;
            if (n < w.o1) atomicAdd(&acc[n], (double)oh[v] + (double)ol[v]);
        }
    }
}

template <int VPT>
__global__ void __launch_bounds__(kThreads) direct_v2s_f64(const WorkItem *__restrict__ items, int n_items, int *__restrict__ counter,
                                                           const double *__restrict__ pxyz, int64_t np_all,
                                                           const double *__restrict__ vxyz, int64_t nv_all,
                                                           const double2 *__restrict__ V, double *__restrict__ acc,
                                                           double sgn) {
    __shared__ double sx[kThreads], sy[kThreads], sz[kThreads], sr[kThreads], si[kThreads];
    __shared__ int s_next;
    for (int it = blockIdx.x; it < n_items; it = next_item(counter, s_next)) {
        const WorkItem w = items[it];
        double rx[VPT], ry[VPT], rz[VPT], a[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int n = w.o0 + threadIdx.x + v * kThreads;
            bool ok = n < w.o1;
            rx[v] = ok ? pxyz[n] : 0.0;
            ry[v] = ok ? pxyz[np_all + n] : 0.0;
            rz[v] = ok ? pxyz[2 * np_all + n] : 0.0;
            a[v] = 0.0;
        }
        for (int s0 = w.s0; s0 < w.s1; s0 += kThreads) {
            __syncthreads();
            int k = s0 + threadIdx.x;
            bool ok = k < w.s1;
            sx[threadIdx.x] = ok ? vxyz[k] : 0.0;
            sy[threadIdx.x] = ok ? vxyz[nv_all + k] : 0.0;
            sz[threadIdx.x] = ok ? vxyz[2 * nv_all + k] : 0.0;
            double2 val = ok ? V[k] : make_double2(0.0, 0.0);
            sr[threadIdx.x] = val.x;
            si[threadIdx.x] = sgn * val.y;
            __syncthreads();
            const int cnt = min(kThreads, w.s1 - s0);
            for (int q = 0; q < cnt; ++q) {
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    double t = fma(sx[q], rx[v], fma(sy[q], ry[v], sz[q] * rz[v]));
                    t -= rint(t);
                    double sn, cs;
                    sincospi(2.0 * t, &sn, &cs);
                    a[v] = fma(sr[q], cs, fma(si[q], sn, a[v]));
                }
            }
        }
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int n = w.o0 + threadIdx.x + v * kThreads;
            if (n < w.o1) atomicAdd(&acc[n], a[v]);
        }
    }
}

}  // namespace

// ------------------------------------------------------------- launchers

void launch_prepare_points(const double *xyz, const int32_t *perm, int64_t n, double *soa, float4 *hi, float4 *lo,
                           cudaStream_t s) {
    if (n <= 0) return;
    prepare_points_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xyz, perm, n, soa, hi, lo);
    check_cuda(cudaGetLastError(), "prepare_points");
}

void launch_gather_weight(const double *w, const int32_t *perm, int64_t n, double *out, cudaStream_t s) {
    if (n <= 0) return;
    gather_weight_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, perm, n, out);
    check_cuda(cudaGetLastError(), "gather_weight");
}

int direct_tile(int vpt) { return kThreads * vpt; }

static unsigned grid_for(int64_t n_items) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    int64_t g = std::min<int64_t>(n_items, (int64_t)sms * 4);
    return (unsigned)std::max<int64_t>(g, 1);
}

void launch_direct_s2v_f32(const WorkItem *items, int64_t n, int *counter, const float4 *vh, const float4 *vl, const float4 *rh,
                           const float4 *rl, const float *c, float2 *acc, int isign, int vpt, cudaStream_t s) {
    if (n <= 0) return;
    const DirectJob J{vh, vl, rh, rl, c, acc, (float)isign};
    if (vpt == 4)
        direct_s2v_f32<4, false><<<grid_for(n), kThreads, 0, s>>>(items, (int)n, counter, J, nullptr, nullptr);
    else
        direct_s2v_f32<2, false><<<grid_for(n), kThreads, 0, s>>>(items, (int)n, counter, J, nullptr, nullptr);
    check_cuda(cudaGetLastError(), "direct_s2v_f32");
}

void launch_direct_s2v_df(const WorkItem *items, int64_t n, int *counter, const float4 *vh, const float4 *vl, const float4 *rh,
                          const float4 *rl, const double *c, double2 *acc, const float4 *tab, int isign,
                          int vpt, cudaStream_t s) {
    if (n <= 0) return;
    const DirectJob J{vh, vl, rh, rl, c, acc, (float)isign};
    if (vpt == 4)
        direct_s2v_df<4, false><<<grid_for(n), kThreads, 0, s>>>(items, (int)n, counter, J, nullptr, nullptr, tab);
    else
        direct_s2v_df<2, false><<<grid_for(n), kThreads, 0, s>>>(items, (int)n, counter, J, nullptr, nullptr, tab);
    check_cuda(cudaGetLastError(), "direct_s2v_df");
}

void launch_direct_s2v_f64(const WorkItem *items, int64_t n, int *counter, const double *vxyz, int64_t nv, const double *pxyz,
                           int64_t np, const double *c, double2 *acc, int isign, int vpt, cudaStream_t s) {
    if (n <= 0) return;
    if (vpt == 4)
        direct_s2v_f64<4><<<grid_for(n), kThreads, 0, s>>>(items, (int)n, counter, vxyz, nv, pxyz, np, c, acc, (double)isign);
    else
        direct_s2v_f64<2><<<grid_for(n), kThreads, 0, s>>>(items, (int)n, counter, vxyz, nv, pxyz, np, c, acc, (double)isign);
    check_cuda(cudaGetLastError(), "direct_s2v_f64");
}

void launch_direct_v2s_f32(const WorkItem *items, int64_t n, int *counter, const float4 *rh, const float4 *rl, const float4 *vh,
                           const float4 *vl, const float2 *V, float *acc, int isign, int vpt, cudaStream_t s) {
    if (n <= 0) return;
    const DirectJob J{rh, rl, vh, vl, V, acc, (float)isign};
    if (vpt == 4)
        direct_v2s_f32<4, false><<<grid_for(n), kThreads, 0, s>>>(items, (int)n, counter, J, nullptr, nullptr);
    else
        direct_v2s_f32<2, false><<<grid_for(n), kThreads, 0, s>>>(items, (int)n, counter, J, nullptr, nullptr);
    check_cuda(cudaGetLastError(), "direct_v2s_f32");
}

void launch_direct_v2s_df(const WorkItem *items, int64_t n, int *counter, const float4 *rh, const float4 *rl, const float4 *vh,
                          const float4 *vl, const double2 *V, double *acc, const float4 *tab, int isign,
                          int vpt, cudaStream_t s) {
    if (n <= 0) return;
    const DirectJob J{rh, rl, vh, vl, V, acc, (float)isign};
    if (vpt == 4)
        direct_v2s_df<4, false><<<grid_for(n), kThreads, 0, s>>>(items, (int)n, counter, J, nullptr, nullptr, tab);
    else
        direct_v2s_df<2, false><<<grid_for(n), kThreads, 0, s>>>(items, (int)n, counter, J, nullptr, nullptr, tab);
    check_cuda(cudaGetLastError(), "direct_v2s_df");
}

// Several jobs' work items in one launch (kind 0 FP32, 1 double-float; dir 0 sky -> vis,
// 1 vis -> sky); jobs and item_job in device memory, items sorted largest first.
void launch_direct_batch(int kind, int dir, const WorkItem *items, int64_t n, int *counter, const DirectJob *jobs,
                         const int *item_job, const float4 *tab, int vpt, cudaStream_t s) {
    if (n <= 0) return;
    const DirectJob J0{};
    const unsigned g = grid_for(n);
#define HVOX_BATCH(KERNEL, ...)                                                                              \
    if (vpt == 4)                                                                                            \
        KERNEL<4, true><<<g, kThreads, 0, s>>>(items, (int)n, counter, J0, jobs, item_job __VA_ARGS__);      \
    else                                                                                                     \
        KERNEL<2, true><<<g, kThreads, 0, s>>>(items, (int)n, counter, J0, jobs, item_job __VA_ARGS__);
    if (kind == 0 && dir == 0) {
        HVOX_BATCH(direct_s2v_f32)
    } else if (kind == 0) {
        HVOX_BATCH(direct_v2s_f32)
    } else if (dir == 0) {
        HVOX_BATCH(direct_s2v_df, , tab)
    } else {
        HVOX_BATCH(direct_v2s_df, , tab)
    }
#undef HVOX_BATCH
    check_cuda(cudaGetLastError(), "direct_batch");
}

void launch_direct_v2s_f64(const WorkItem *items, int64_t n, int *counter, const double *pxyz, int64_t np, const double *vxyz,
                           int64_t nv, const double2 *V, double *acc, int isign, int vpt, cudaStream_t s) {
    if (n <= 0) return;
    if (vpt == 4)
        direct_v2s_f64<4><<<grid_for(n), kThreads, 0, s>>>(items, (int)n, counter, pxyz, np, vxyz, nv, V, acc, (double)isign);
    else
        direct_v2s_f64<2><<<grid_for(n), kThreads, 0, s>>>(items, (int)n, counter, pxyz, np, vxyz, nv, V, acc, (double)isign);
    check_cuda(cudaGetLastError(), "direct_v2s_f64");
}

}  // namespace hvox

// ============================================================================
// Direct sky -> vis evaluation that allocates nothing.
//
// For callers that cannot call cudaMalloc: code that runs inside another framework
// which has reserved the device's memory for its own pool (a cudaMalloc there fails or
// fragments that pool), and iteration loops such as calibration solvers that predict
// visibilities from a sky model every step, where an allocation (and the device
// synchronisation cudaFree brings) is not allowed. The caller passes device pointers
// for everything; the only working memory is the static array below. CUDA reserves it on
// a device when it loads this file's device code there (lazily by default: at the first
// call of the entry point or the first direct-sum launch of any plan on that device) and
// keeps it until the process exits.
// ============================================================================

namespace hvox {

namespace {

constexpr int64_t kNoAllocMaxPoints = int64_t(1) << 19;  // n_pix + n_vis <= 524,288

// hi and lo float splits of the pixel and baseline coordinates: 2 * 524,288 float4 = 16 MiB.
__device__ __align__(256) float4 g_noalloc_scratch[2 * kNoAllocMaxPoints];

__global__ void noalloc_split_kernel(const double *__restrict__ xyz, int64_t n, float4 *__restrict__ hi,
                                     float4 *__restrict__ lo) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h[3], l[3];
    for (int d = 0; d < 3; ++d) {
        double x = xyz[3 * i + d];
        h[d] = (float)x;
        l[d] = (float)(x - (double)h[d]);
    }
    hi[i] = make_float4(h[0], h[1], h[2], 0.f);
    lo[i] = make_float4(l[0], l[1], l[2], 0.f);
}

// The phase arithmetic and the two-level summation of direct_s2v_f32 (a register sum per
// 256-pixel shared-memory tile, tile sums added with Kahan compensation); the baseline
// tile comes from blockIdx.x and a segment of 4096 pixels from blockIdx.y instead of a
// work list, and the segments' sums meet in V through atomicAdd, so their order (and the
// last bits of the result) is not deterministic.
__global__ void __launch_bounds__(kThreads) direct_s2v_f32_noalloc(
    const float4 *__restrict__ vh, const float4 *__restrict__ vl, int n_vis, const float4 *__restrict__ rh_g,
    const float4 *__restrict__ rl_g, const float *__restrict__ c, int n_pix, int seg, float2 *__restrict__ V,
    float sgn) {
    __shared__ float4 sh[kThreads];
    __shared__ float4 sl[kThreads];
    const int o0 = blockIdx.x * kTile, o1 = min(o0 + kTile, n_vis);
    const int s_begin = blockIdx.y * seg, s_end = min(s_begin + seg, n_pix);
    float3 ph[kPerThread], pl[kPerThread];
    float are[kPerThread], aim[kPerThread], cre[kPerThread], cim[kPerThread];
#pragma unroll
    for (int v = 0; v < kPerThread; ++v) {
        int k = o0 + threadIdx.x + v * kThreads;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (k < o1) {
            a = vh[k];
            b = vl[k];
        }
        ph[v] = make_float3(a.x, a.y, a.z);
        pl[v] = make_float3(b.x, b.y, b.z);
        are[v] = aim[v] = cre[v] = cim[v] = 0.f;
    }
    for (int s0 = s_begin; s0 < s_end; s0 += kThreads) {
        __syncthreads();
        int n = s0 + threadIdx.x;
        if (n < s_end) {
            float4 a = rh_g[n];
            a.w = c[n];
            sh[threadIdx.x] = a;
            sl[threadIdx.x] = rl_g[n];
        } else {
            sh[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
            sl[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const int cnt = min(kThreads, s_end - s0);
        float tre[kPerThread], tim[kPerThread];
#pragma unroll
        for (int v = 0; v < kPerThread; ++v) tre[v] = tim[v] = 0.f;
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) {
            const float4 rh = sh[q], rl = sl[q];
#pragma unroll
            for (int v = 0; v < kPerThread; ++v) {
                float f = phase_f32(ph[v], pl[v], rh, rl);
                float sn, cs;
                __sincosf(6.28318530717958648f * f, &sn, &cs);
                tre[v] = __fmaf_rn(rh.w, cs, tre[v]);
                tim[v] = __fmaf_rn(rh.w, sn, tim[v]);
            }
        }
#pragma unroll
        for (int v = 0; v < kPerThread; ++v) {
            kahan_add(are[v], cre[v], tre[v]);
            kahan_add(aim[v], cim[v], tim[v]);
        }
    }
#pragma unroll
    for (int v = 0; v < kPerThread; ++v) {
        int k = o0 + threadIdx.x + v * kThreads;
        if (k < o1) {
            atomicAdd(&V[k].x, __fsub_rn(are[v], cre[v]));
            atomicAdd(&V[k].y, sgn * __fsub_rn(aim[v], cim[v]));
        }
    }
}

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[256] = {nullptr};

// Device address of the static scratch for the current device. The first call on a
// device looks it up (cudaGetSymbolAddress, no allocation) with that device current.
float4 *noalloc_scratch_for_current_device() {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 256) fail(HVOX_EUNSUPPORTED, "hvox_direct_synthesize_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        check_cuda(cudaGetSymbolAddress(&ptr, g_noalloc_scratch), "cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = ptr;
    }
    return static_cast<float4 *>(g_noalloc_ptr[dev]);
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace hvox

extern "C" hvox_status hvox_direct_synthesize_noalloc(const double *pix_xyz, int64_t n_pix, const double *uvw,
                                                      int64_t n_vis, const float *I, float *V, int isign,
                                                      void *stream) {
    using namespace hvox;
    try {
        if (!pix_xyz || !uvw || !I || !V) fail(HVOX_EINVAL, "hvox_direct_synthesize_noalloc: NULL pointer");
        if (n_pix < 1 || n_vis < 1) fail(HVOX_EINVAL, "hvox_direct_synthesize_noalloc: need n_pix, n_vis >= 1");
        if (n_pix + n_vis > kNoAllocMaxPoints)
            fail(HVOX_EINVAL, "hvox_direct_synthesize_noalloc: n_pix + n_vis = " + std::to_string(n_pix + n_vis) +
                                  " exceeds the static limit of " + std::to_string(kNoAllocMaxPoints) + " points");
        if (isign != 1 && isign != -1) fail(HVOX_EINVAL, "hvox_direct_synthesize_noalloc: isign must be +1 or -1");
        if (!on_device(pix_xyz) || !on_device(uvw) || !on_device(I) || !on_device(V))
            fail(HVOX_EINVAL, "hvox_direct_synthesize_noalloc: every pointer must be device memory");
        cudaStream_t s = (cudaStream_t)stream;
        float4 *scratch = noalloc_scratch_for_current_device();
        float4 *rh = scratch, *rl = scratch + n_pix;
        float4 *vh = scratch + 2 * n_pix, *vl = vh + n_vis;
        noalloc_split_kernel<<<(unsigned)((n_pix + 255) / 256), 256, 0, s>>>(pix_xyz, n_pix, rh, rl);
        check_cuda(cudaGetLastError(), "noalloc_split pixels");
        noalloc_split_kernel<<<(unsigned)((n_vis + 255) / 256), 256, 0, s>>>(uvw, n_vis, vh, vl);
        check_cuda(cudaGetLastError(), "noalloc_split baselines");
        check_cuda(cudaMemsetAsync(V, 0, sizeof(float) * 2 * (size_t)n_vis, s), "clear V");
        const int seg = 4096;
        dim3 grid((unsigned)((n_vis + kTile - 1) / kTile), (unsigned)((n_pix + seg - 1) / seg));
        direct_s2v_f32_noalloc<<<grid, kThreads, 0, s>>>(vh, vl, (int)n_vis, rh, rl, I, (int)n_pix, seg,
                                                          reinterpret_cast<float2 *>(V), (float)isign);
        check_cuda(cudaGetLastError(), "direct_s2v_f32_noalloc");
        set_error("");
        return HVOX_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::exception &e) {
        set_error(std::string("internal error: ") + e.what());
        return HVOX_EINTERNAL;
    }
}
