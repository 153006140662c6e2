// Double-float FFT for the FP64 grids of NUFFT sub-problems (eps < 1e-6), the uniform FFT of
// step 2 of the type-3 transform (Sect. 3).
//
// GB300 runs FP64 at 1/63 of its FP32 rate, and cuFFT's Z2Z transforms of these grids are
// bound by the FP64 units (~17x the C2C time per cell). Here every value is an unevaluated
// pair of floats (hi + lo, ~48 bits; Dekker 1971 with FMA products) and every 1-D transform
// runs in shared memory on the FP32 pipes: Stockham auto-sorting stages of radix 4, 2, 3, 5
// and 7 (the odd radices through the symmetric form X_k, X_{r-k} = A_k +- s i B_k, half the
// multiplications of a plain DFT), with twiddles exp(2 pi i q / n) computed in FP64 on the
// host and stored as float pairs. One pass per dimension reads the FP64 grid, transforms
// and writes it back in place:
//   rows (x): one row per CTA, only the rows that the pruned transform needs;
//   columns (y): two adjacent columns per CTA (32-byte sectors), every column of a plane;
//   columns (z): 64 adjacent columns per CTA, the planes of a batch interleaved.
// Transforms are unnormalised, sign s = -1 or +1: X_k = sum_q x_q exp(s 2 pi i q k / n).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "hvox_internal.h"

namespace hvox {

namespace {

constexpr int kFftThreads = 256;

struct DF {
    float h, l;
};
struct DC {
    DF re, im;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Accurate double-float sum (both parts summed with error-free transformations).
__device__ __forceinline__ DF dadd(DF a, DF b) {
    float s, e, t, f;
    two_sum(a.h, b.h, s, e);
    two_sum(a.l, b.l, t, f);
    e = __fadd_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    fast_two_sum(s, e, s, e);
    return {s, e};
}

__device__ __forceinline__ DF dneg(DF a) { return {-a.h, -a.l}; }

__device__ __forceinline__ DF dmul(DF a, DF b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    float s;
    fast_two_sum(p, e, s, e);
    return {s, e};
}

__device__ __forceinline__ DC cadd(const DC &a, const DC &b) { return {dadd(a.re, b.re), dadd(a.im, b.im)}; }
__device__ __forceinline__ DC csub(const DC &a, const DC &b) { return {dadd(a.re, dneg(b.re)), dadd(a.im, dneg(b.im))}; }

// a * (c + j s) for real double-float c, s.
__device__ __forceinline__ DC cmul(const DC &a, DF c, DF s) {
    return {dadd(dmul(a.re, c), dneg(dmul(a.im, s))), dadd(dmul(a.re, s), dmul(a.im, c))};
}

// a * (j sg) for sg = +-1.
__device__ __forceinline__ DC times_j(const DC &a, float sg) {
    return {{-sg * a.im.h, -sg * a.im.l}, {sg * a.re.h, sg * a.re.l}};
}

__device__ __forceinline__ DC from4(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 to4(const DC &c) { return make_float4(c.re.h, c.re.l, c.im.h, c.im.l); }

__device__ __forceinline__ DF split(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ float4 load_cell(const double2 *p) {
    const double2 v = *p;
    const DF re = split(v.x), im = split(v.y);
    return make_float4(re.h, re.l, im.h, im.l);
}
__device__ __forceinline__ void store_cell(double2 *p, float4 v) {
    *p = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

// Twiddle exp(s 2 pi i e / n) from the table of exp(2 pi i q / n) (cos h, cos l, sin h, sin l).
__device__ __forceinline__ void twiddle(const float4 *__restrict__ tw, int e, float sg, DF &c, DF &s) {
    const float4 t = __ldg(tw + e);
    c = {t.x, t.y};
    s = {sg * t.z, sg * t.w};
}

// One Stockham stage of radix R over TX interleaved sequences: butterfly j (of n / R) reads
// elements j + q n / R, twiddles them by exp(s 2 pi i q k span / n) (k = j mod Ns) and writes
// the R outputs to (j / Ns) Ns R + k + q Ns. q k span < n, so the table index needs no wrap.
template <int R, int TX>
__device__ __forceinline__ void stage(const float4 *__restrict__ a, float4 *__restrict__ b, const DfftDev &d, int Ns,
                                      float sg) {
    const int n = d.n, m = n / R, span = n / (Ns * R);
    for (int wk = threadIdx.x; wk < m * TX; wk += blockDim.x) {
        const int j = wk / TX, t = wk - j * TX;
        DC v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = from4(a[(j + q * m) * TX + t]);
        const int jn = j / Ns, k = j - jn * Ns;
        if (k != 0) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                DF c, s;
                twiddle(d.tw, q * k * span, sg, c, s);
                v[q] = cmul(v[q], c, s);
            }
        }
        DC y[R];
        if constexpr (R == 2) {
            y[0] = cadd(v[0], v[1]);
            y[1] = csub(v[0], v[1]);
        } else if constexpr (R == 4) {
            const DC a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
            const DC b0 = cadd(v[1], v[3]), b1 = times_j(csub(v[1], v[3]), sg);
            y[0] = cadd(a0, b0);
            y[1] = cadd(a1, b1);
            y[2] = csub(a0, b0);
            y[3] = csub(a1, b1);
        } else {
            // odd R: s_q = v_q + v_{R-q}, d_q = v_q - v_{R-q} (q = 1 .. H); X_0 = v_0 + sum s_q;
            // A_k = v_0 + sum s_q cos(2 pi q k / R), B_k = sum d_q sin(2 pi q k / R);
            // X_k = A_k + s j B_k, X_{R-k} = A_k - s j B_k.
            constexpr int H = R / 2;
            const int rstep = n / R;
            DC sq[H], dq[H];
            y[0] = v[0];
#pragma unroll
            for (int q = 1; q <= H; ++q) {
                sq[q - 1] = cadd(v[q], v[R - q]);
                dq[q - 1] = csub(v[q], v[R - q]);
                y[0] = cadd(y[0], sq[q - 1]);
            }
#pragma unroll
            for (int kk = 1; kk <= H; ++kk) {
                DC A = v[0], B = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
                for (int q = 1; q <= H; ++q) {
                    DF c, s;
                    twiddle(d.tw, ((q * kk) % R) * rstep, 1.f, c, s);
                    A = cadd(A, {dmul(sq[q - 1].re, c), dmul(sq[q - 1].im, c)});
                    B = cadd(B, {dmul(dq[q - 1].re, s), dmul(dq[q - 1].im, s)});
                }
                const DC jb = times_j(B, sg);
                y[kk] = cadd(A, jb);
                y[R - kk] = csub(A, jb);
            }
        }
        const int base = jn * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) b[(base + q * Ns) * TX + t] = to4(y[q]);
    }
}

// In-place transforms of TX interleaved sequences of length n in shared memory (element q of
// sequence t at a[q TX + t]); b is the second buffer of the Stockham ping-pong. Returns the
// buffer holding the result.
template <int TX>
__device__ float4 *fft_smem(float4 *a, float4 *b, const DfftDev &d, float sg) {
    int Ns = 1;
    for (int st = 0; st < d.stages; ++st) {
        const int r = d.radix[st];
        switch (r) {
            case 4: stage<4, TX>(a, b, d, Ns, sg); break;
            case 2: stage<2, TX>(a, b, d, Ns, sg); break;
            case 3: stage<3, TX>(a, b, d, Ns, sg); break;
            case 5: stage<5, TX>(a, b, d, Ns, sg); break;
            default: stage<7, TX>(a, b, d, Ns, sg); break;
        }
        __syncthreads();
        float4 *tmp = a;
        a = b;
        b = tmp;
        Ns *= r;
    }
    return a;
}

// Linear index of a band plane (the n1 band's z planes of a batch: the lower slab's
// half K planes, then the upper slab's) -> plane number in the interleaved layout.
__device__ __forceinline__ int64_t band_plane(int64_t P, int64_t halfK, int64_t n2z, int64_t K, int64_t half) {
    return P < halfK ? P : (n2z - half) * K + (P - halfK);
}

// Rows (x): sequence s = (band plane P, row R) with R over all n2y rows or only the band rows.
__global__ void __launch_bounds__(kFftThreads) dfft_rows_kernel(double2 *__restrict__ g, DfftDev d, int64_t n2y,
                                                                 int64_t halfK, int64_t n2z, int64_t K, int64_t half,
                                                                 int64_t rows, int64_t h1y, float sg) {
    extern __shared__ float4 smem[];
    const int n = d.n;
    const int64_t s = blockIdx.x;
    const int64_t P = s / rows, R = s - P * rows;
    const int64_t y = h1y > 0 ? (R < h1y ? R : n2y - h1y + (R - h1y)) : R;
    double2 *row = g + (band_plane(P, halfK, n2z, K, half) * n2y + y) * n;
    float4 *a = smem, *b = smem + n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = load_cell(row + i);
    __syncthreads();
    const float4 *out = fft_smem<1>(a, b, d, sg);
    for (int i = threadIdx.x; i < n; i += blockDim.x) store_cell(row + i, out[i]);
}

// Columns: TX adjacent columns starting at column c0 of a plane (y: columns of one band plane,
// stride n2x; z: every column of the batch, stride K n2x n2y), element q at c + q * stride.
template <int TX>
__global__ void __launch_bounds__(kFftThreads) dfft_cols_kernel(double2 *__restrict__ g, DfftDev d, int64_t stride,
                                                                 int64_t ncols, int64_t plane_cells, int64_t halfK,
                                                                 int64_t n2z, int64_t K, int64_t half, int band,
                                                                 float sg) {
    extern __shared__ float4 smem[];
    const int n = d.n;
    const int64_t tiles = (ncols + TX - 1) / TX;
    const int64_t P = blockIdx.x / tiles, c0 = (blockIdx.x - P * tiles) * TX;
    double2 *base = g + (band ? band_plane(P, halfK, n2z, K, half) * plane_cells : 0) + c0;
    const int valid = ncols - c0 < TX ? (int)(ncols - c0) : TX;
    float4 *a = smem, *b = smem + (size_t)n * TX;
    for (int e = threadIdx.x; e < n * TX; e += blockDim.x) {
        const int q = e / TX, t = e - q * TX;
        a[e] = t < valid ? load_cell(base + q * stride + t) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const float4 *out = fft_smem<TX>(a, b, d, sg);
    for (int e = threadIdx.x; e < n * TX; e += blockDim.x) {
        const int q = e / TX, t = e - q * TX;
        if (t < valid) store_cell(base + q * stride + t, out[e]);
    }
}

constexpr size_t kFftSmemMax = 220 * 1024;

template <typename K> void allow_smem(K kernel) {
    check_cuda(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFftSmemMax),
               "cudaFuncSetAttribute");
}

void set_fft_attrs() {
    static std::once_flag once;
    std::call_once(once, [] {
        allow_smem(dfft_rows_kernel);
        allow_smem(dfft_cols_kernel<1>);
        allow_smem(dfft_cols_kernel<2>);
        allow_smem(dfft_cols_kernel<8>);
        allow_smem(dfft_cols_kernel<64>);
    });
}

// Columns per CTA for a column transform of length n: as many as the shared memory holds
// (two buffers of n TX cells of 16 bytes), at most `want`.
int cols_per_cta(int n, int want) {
    for (int tx : {64, 8, 2, 1})
        if (tx <= want && (size_t)2 * n * tx * 16 <= kFftSmemMax) return tx;
    return 0;
}

template <int TX>
void launch_cols(double2 *g, const DfftDev &d, int64_t stride, int64_t ncols, int64_t plane_cells, int64_t planes,
                 int64_t halfK, int64_t n2z, int64_t K, int64_t half, int band, float sg, cudaStream_t s) {
    const int64_t tiles = (ncols + TX - 1) / TX;
    const size_t smem = (size_t)2 * d.n * TX * sizeof(float4);
    dfft_cols_kernel<TX><<<(unsigned)(planes * tiles), kFftThreads, smem, s>>>(g, d, stride, ncols, plane_cells, halfK,
                                                                               n2z, K, half, band, sg);
    check_cuda(cudaGetLastError(), "dfft_cols");
}

void cols(int tx, double2 *g, const DfftDev &d, int64_t stride, int64_t ncols, int64_t plane_cells, int64_t planes,
          int64_t halfK, int64_t n2z, int64_t K, int64_t half, int band, float sg, cudaStream_t s) {
    switch (tx) {
        case 64: launch_cols<64>(g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, sg, s); break;
        case 8: launch_cols<8>(g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, sg, s); break;
        case 2: launch_cols<2>(g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, sg, s); break;
        default: launch_cols<1>(g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, sg, s); break;
    }
}

}  // namespace

bool dfft_factor(int n, DfftDev &d) {
    d.n = n;
    d.stages = 0;
    int m = n;
    for (int r : {4, 2, 3, 5, 7})
        while (m % r == 0) {
            if (d.stages == kDfftMaxStages) return false;
            d.radix[d.stages++] = r;
            m /= r;
        }
    return m == 1 && n >= 2;
}

bool dfft_supported(const int64_t n2[3]) {
    DfftDev d;
    for (int k = 0; k < 3; ++k)
        if (n2[k] > (int64_t)(kFftSmemMax / 32) || !dfft_factor((int)n2[k], d)) return false;
    return cols_per_cta((int)n2[1], 2) > 0 && cols_per_cta((int)n2[2], 64) > 0;
}

void dfft_twiddles(int n, std::vector<float> &tab) {
    tab.resize(4 * (size_t)n);
    for (int q = 0; q < n; ++q) {
        const double ang = 2.0 * M_PI * (double)q / (double)n;
        const double c = std::cos(ang), s = std::sin(ang);
        const float ch = (float)c, sh = (float)s;
        tab[4 * q + 0] = ch;
        tab[4 * q + 1] = (float)(c - (double)ch);
        tab[4 * q + 2] = sh;
        tab[4 * q + 3] = (float)(s - (double)sh);
    }
}

int dfft_batch(const FftBatch &f, int sign, bool band_input, cudaStream_t s) {
    set_fft_attrs();
    double2 *g = static_cast<double2 *>(f.g2);
    const int64_t n2x = f.n2[0], n2y = f.n2[1], n2z = f.n2[2], K = f.K, half = f.half;
    const int64_t halfK = half * K, band_planes = 2 * halfK, plane = n2x * n2y;
    const float sg = (float)sign;
    auto rows = [&](bool band_rows) {
        const int64_t r = band_rows ? 2 * f.h1y : n2y;
        const size_t smem = (size_t)2 * n2x * sizeof(float4);
        dfft_rows_kernel<<<(unsigned)(band_planes * r), kFftThreads, smem, s>>>(
            g, f.dx, n2y, halfK, n2z, K, half, r, band_rows ? f.h1y : 0, sg);
        check_cuda(cudaGetLastError(), "dfft_rows");
    };
    auto ycols = [&] {
        cols(cols_per_cta((int)n2y, 2), g, f.dy, n2x, n2x, plane, band_planes, halfK, n2z, K, half, 1, sg, s);
    };
    auto zcols = [&] {
        cols(cols_per_cta((int)n2z, 64), g, f.dz, K * plane, K * plane, 0, 1, halfK, n2z, K, half, 0, sg, s);
    };
    if (band_input) {  // only the band rows of the band planes are nonzero
        rows(true);
        ycols();
        zcols();
    } else {  // only the band rows of the band planes are read afterwards
        zcols();
        ycols();
        rows(true);
    }
    return 3;
}

}  // namespace hvox
