// Double-float FFT for the FP64 grids of NUFFT sub-problems (eps < 1e-6), the uniform FFT of
// step 2 of the type-3 transform (Sect. 3).
//
// GB300 runs FP64 at 1/63 of its FP32 rate, and cuFFT's Z2Z transforms of these grids are
// bound by the FP64 units (~17x the C2C time per cell). Here every value is an unevaluated
// pair of floats (hi + lo, ~48 bits; Dekker 1971 with FMA products) and every 1-D transform
// runs in shared memory on the FP32 pipes: Stockham auto-sorting stages of radix 4, 2, 3, 5
// and 7 (the odd radices through the symmetric form X_k, X_{r-k} = A_k +- s i B_k, half the
// multiplications of a plain DFT), with twiddles exp(2 pi i q / n) computed in FP64 on the
// host and stored as float pairs. One pass per dimension transforms the grid in place; the
// first reads FP64 cells, every pass writes float pairs (the same 16 bytes per cell):
//   rows (x): one row per CTA, only the rows that the pruned transform needs;
//   columns (y): two adjacent columns per CTA (32-byte sectors), every column of a plane;
//   columns (z): 64 adjacent columns per CTA, the planes of a batch interleaved; these short
//   transforms (two stages for most grids) read the grid in their first stage and write it
//   in their last, so they need one shared buffer and one barrier.
// Transforms are unnormalised, sign s = -1 or +1: X_k = sum_q x_q exp(s 2 pi i q k / n).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "dfloat.cuh"
#include "hvox_internal.h"

namespace hvox {

namespace {

using namespace df;

// 256 threads per CTA, held to 64 registers so that four CTAs fit an SM where shared memory
// allows (a fourth CTA hides more of each CTA's load phase and stage barriers).
constexpr int kFftThreads = 256;

struct DC {
    DF re, im;
};

__device__ __forceinline__ DC cadd(const DC &a, const DC &b) { return {dadd(a.re, b.re), dadd(a.im, b.im)}; }
__device__ __forceinline__ DC csub(const DC &a, const DC &b) { return {dadd(a.re, dneg(b.re)), dadd(a.im, dneg(b.im))}; }

// Sums and products whose results only feed further sums (within one butterfly) skip their
// renormalisation (dadd_lazy); the outputs a butterfly stores are renormalised.
__device__ __forceinline__ DC cadd_lazy(const DC &a, const DC &b) {
    return {dadd_lazy(a.re, b.re), dadd_lazy(a.im, b.im)};
}
__device__ __forceinline__ DC csub_lazy(const DC &a, const DC &b) {
    return {dadd_lazy(a.re, dneg(b.re)), dadd_lazy(a.im, dneg(b.im))};
}

// a * (c + j s) for real double-float c, s (unnormalised, it feeds the butterfly's sums).
__device__ __forceinline__ DC cmul_lazy(const DC &a, DF c, DF s) {
    return {dmul2_lazy(a.re, c, a.im, s, -1.f), dmul2_lazy(a.re, s, a.im, c, 1.f)};
}

// a * (j SG) for SG = +-1 (sign flips only).
template <int SG> __device__ __forceinline__ DC times_j(const DC &a) {
    if constexpr (SG > 0) return {dneg(a.im), a.re};
    else return {a.im, dneg(a.re)};
}

__device__ __forceinline__ DC from4(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 to4(const DC &c) { return make_float4(c.re.h, c.re.l, c.im.h, c.im.l); }

__device__ __forceinline__ float4 load_f64(const double2 *p) {
    const double2 v = *p;
    const DF re = split_bits(v.x), im = split_bits(v.y);
    return make_float4(re.h, re.l, im.h, im.l);
}
__device__ __forceinline__ void store_f64(double2 *p, float4 v) {
    *p = make_double2(f2d_bits(v.x) + f2d_bits(v.y), f2d_bits(v.z) + f2d_bits(v.w));
}

// A grid cell in either format: FP64 (double2) or, between the passes of one transform, the
// double-float form itself (float4 of the same 16 bytes; zero is all-zero bits in both).
template <bool F64> __device__ __forceinline__ float4 load_cell(double2 *p) {
    if constexpr (F64) return load_f64(p);
    else return *reinterpret_cast<const float4 *>(p);
}
template <bool F64> __device__ __forceinline__ void store_cell(double2 *p, float4 v) {
    if constexpr (F64) store_f64(p, v);
    else *reinterpret_cast<float4 *>(p) = v;
}

// Twiddle exp(SG 2 pi i e / n) from the table of exp(2 pi i q / n) (cos h, cos l, sin h, sin l).
template <int SG> __device__ __forceinline__ void twiddle(const float4 *__restrict__ tw, int e, DF &c, DF &s) {
    const float4 t = __ldg(tw + e);
    c = {t.x, t.y};
    s = SG > 0 ? DF{t.z, t.w} : DF{-t.z, -t.w};
}

// One Stockham stage of radix R over TX interleaved sequences: butterfly j (of n / R) reads
// elements j + q n / R, twiddles them by exp(s 2 pi i q k span / n) (k = j mod Ns) and writes
// the R outputs to (j / Ns) Ns R + k + q Ns. q k span < n, so the table index needs no wrap.
// The sign SG of the exponent is a template parameter: its flips fold into the operands.
// ld(e, t) reads element e of sequence t, st(e, t, v) writes it: shared memory between
// stages; the grid itself in the first and the last stage of a z-column pass.
template <int R, int TX, int SG, class Ld, class St>
__device__ __forceinline__ void stage(Ld ld, St st, const DfftDev &d, int Ns, unsigned magic) {
    const int n = d.n, m = n / R, span = n / (Ns * R);
    for (int wk = threadIdx.x; wk < m * TX; wk += blockDim.x) {
        const int j = wk / TX, t = wk - j * TX;
        DC v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = from4(ld(j + q * m, t));
        const int jn = Ns == 1 ? j : (int)__umulhi((unsigned)j, magic), k = j - jn * Ns;
        if (k != 0) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                DF c, s;
                twiddle<SG>(d.tw, q * k * span, c, s);
                v[q] = cmul_lazy(v[q], c, s);
            }
        }
        DC y[R];
        if constexpr (R == 2) {
            y[0] = cadd(v[0], v[1]);
            y[1] = csub(v[0], v[1]);
        } else if constexpr (R == 4) {
            const DC a0 = cadd_lazy(v[0], v[2]), a1 = csub_lazy(v[0], v[2]);
            const DC b0 = cadd_lazy(v[1], v[3]), b1 = times_j<SG>(csub_lazy(v[1], v[3]));
            y[0] = cadd(a0, b0);
            y[1] = cadd(a1, b1);
            y[2] = csub(a0, b0);
            y[3] = csub(a1, b1);
        } else {
            // odd R: s_q = v_q + v_{R-q}, d_q = v_q - v_{R-q} (q = 1 .. H); X_0 = v_0 + sum s_q;
            // A_k = v_0 + sum s_q cos(2 pi q k / R), B_k = sum d_q sin(2 pi q k / R);
            // X_k = A_k + s j B_k, X_{R-k} = A_k - s j B_k. The coefficients come from the
            // kernel parameters at compile-time offsets (constant-bank operands).
            constexpr int H = R / 2;
            constexpr int off = R == 3 ? 0 : (R == 5 ? 1 : 5);
            DC sq[H], dq[H];
#pragma unroll
            for (int q = 1; q <= H; ++q) {
                sq[q - 1] = cadd_lazy(v[q], v[R - q]);
                dq[q - 1] = csub_lazy(v[q], v[R - q]);
            }
            {
                DAcc re = acc_of(v[0].re), im = acc_of(v[0].im);
#pragma unroll
                for (int q = 0; q < H; ++q) {
                    acc_add(re, sq[q].re.h, sq[q].re.l);
                    acc_add(im, sq[q].im.h, sq[q].im.l);
                }
                y[0] = {acc_done(re), acc_done(im)};
            }
#pragma unroll
            for (int kk = 1; kk <= H; ++kk) {
                DAcc ar = acc_of(v[0].re), ai = acc_of(v[0].im), br, bi;
#pragma unroll
                for (int q = 1; q <= H; ++q) {
                    const float4 cs = d.odd[off + (q - 1) * H + (kk - 1)];
                    const DF c = {cs.x, cs.y}, sn = {cs.z, cs.w};
                    acc_fma(ar, sq[q - 1].re, c);
                    acc_fma(ai, sq[q - 1].im, c);
                    if (q == 1) {
                        br = acc_mul(dq[0].re, sn);
                        bi = acc_mul(dq[0].im, sn);
                    } else {
                        acc_fma(br, dq[q - 1].re, sn);
                        acc_fma(bi, dq[q - 1].im, sn);
                    }
                }
                const DC A = {acc_lazy(ar), acc_lazy(ai)};
                const DC jb = times_j<SG>({acc_lazy(br), acc_lazy(bi)});
                y[kk] = cadd(A, jb);
                y[R - kk] = csub(A, jb);
            }
        }
        const int base = jn * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) st(base + q * Ns, t, to4(y[q]));
    }
}

// Element accessors: shared memory (element e of sequence t at e TX + t) and a tile of TX
// grid columns (columns t >= valid of a ragged tile read as 0, never written).
template <int TX> struct SmemLd {
    const float4 *a;
    __device__ __forceinline__ float4 operator()(int e, int t) const { return a[e * TX + t]; }
};
template <int TX> struct SmemSt {
    float4 *b;
    __device__ __forceinline__ void operator()(int e, int t, float4 v) const { b[e * TX + t] = v; }
};
template <bool F64> struct ColLd {
    double2 *base;
    int64_t stride;
    int valid;
    __device__ __forceinline__ float4 operator()(int e, int t) const {
        return t < valid ? load_cell<F64>(base + e * stride + t) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
};
template <bool F64> struct ColSt {
    double2 *base;
    int64_t stride;
    int valid;
    __device__ __forceinline__ void operator()(int e, int t, float4 v) const {
        if (t < valid) store_cell<F64>(base + e * stride + t, v);
    }
};

template <int TX, int SG, class Ld, class St>
__device__ __forceinline__ void run_stage(int r, Ld ld, St st, const DfftDev &d, int Ns, unsigned mg) {
    switch (r) {
        case 4: stage<4, TX, SG>(ld, st, d, Ns, mg); break;
        case 2: stage<2, TX, SG>(ld, st, d, Ns, mg); break;
        case 3: stage<3, TX, SG>(ld, st, d, Ns, mg); break;
        case 5: stage<5, TX, SG>(ld, st, d, Ns, mg); break;
        default: stage<7, TX, SG>(ld, st, d, Ns, mg); break;
    }
}

// Transforms of TX interleaved sequences of length n held in the grid: the first stage
// reads the grid, the last writes it back, the stages between ping-pong through the
// shared buffers a and b (a only for two stages, none for one). The grid is read only in
// the first stage and written only in the last, with a barrier between them (one stage:
// each thread reads every input of the butterflies it writes), so in-place is safe.
template <int TX, int SG, class GLd, class GSt>
__device__ __forceinline__ void fft_pass(float4 *a, float4 *b, const DfftDev &d, GLd gld, GSt gst) {
    const int S = d.stages;
    if (S == 1) {
        run_stage<TX, SG>(d.radix[0], gld, gst, d, 1, d.ns_magic[0]);
        return;
    }
    run_stage<TX, SG>(d.radix[0], gld, SmemSt<TX>{a}, d, 1, d.ns_magic[0]);
    __syncthreads();
    int Ns = d.radix[0];
    for (int st = 1; st < S - 1; ++st) {
        run_stage<TX, SG>(d.radix[st], SmemLd<TX>{a}, SmemSt<TX>{b}, d, Ns, d.ns_magic[st]);
        __syncthreads();
        float4 *tmp = a;
        a = b;
        b = tmp;
        Ns *= d.radix[st];
    }
    run_stage<TX, SG>(d.radix[S - 1], SmemLd<TX>{a}, gst, d, Ns, d.ns_magic[S - 1]);
}

// Shared buffers a pass needs for a transform of s stages (see fft_pass).
inline int pass_buffers(int s) { return s >= 3 ? 2 : s - 1; }

// In-place transforms of TX interleaved sequences of length n in shared memory (element q of
// sequence t at a[q TX + t]); b is the second buffer of the Stockham ping-pong. Returns the
// buffer holding the result.
template <int TX, int SG>
__device__ float4 *fft_smem(float4 *a, float4 *b, const DfftDev &d) {
    int Ns = 1;
    for (int st = 0; st < d.stages; ++st) {
        run_stage<TX, SG>(d.radix[st], SmemLd<TX>{a}, SmemSt<TX>{b}, d, Ns, d.ns_magic[st]);
        __syncthreads();
        float4 *tmp = a;
        a = b;
        b = tmp;
        Ns *= d.radix[st];
    }
    return a;
}

// Linear index of a band plane (the n1 band's z planes of a batch: the lower slab's
// half K planes, then the upper slab's) -> plane number in the interleaved layout.
__device__ __forceinline__ int64_t band_plane(int64_t P, int64_t halfK, int64_t n2z, int64_t K, int64_t half) {
    return P < halfK ? P : (n2z - half) * K + (P - halfK);
}

// Rows (x): sequence s = (band plane P, row R) with R over all n2y rows or only the band rows.
// IN64 / OUT64: the grid holds FP64 values before / after the pass (else double-float).
template <int SG, bool IN64, bool OUT64>
__global__ void __launch_bounds__(kFftThreads, 4) dfft_rows_kernel(double2 *__restrict__ g, DfftDev d, int64_t n2y,
                                                                 int64_t halfK, int64_t n2z, int64_t K, int64_t half,
                                                                 int64_t rows, int64_t h1y) {
    extern __shared__ float4 smem[];
    const int n = d.n;
    const int64_t s = blockIdx.x;
    const int64_t P = s / rows, R = s - P * rows;
    const int64_t y = h1y > 0 ? (R < h1y ? R : n2y - h1y + (R - h1y)) : R;
    double2 *row = g + (band_plane(P, halfK, n2z, K, half) * n2y + y) * n;
    float4 *a = smem, *b = smem + n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = load_cell<IN64>(row + i);
    __syncthreads();
    const float4 *out = fft_smem<1, SG>(a, b, d);
    for (int i = threadIdx.x; i < n; i += blockDim.x) store_cell<OUT64>(row + i, out[i]);
}

// Columns: TX adjacent columns starting at column c0 of a plane (y: columns of one band plane,
// stride n2x; z: every column of the batch, stride K n2x n2y), element q at c + q * stride.
template <int TX, int SG, bool IN64, bool OUT64>
__global__ void __launch_bounds__(kFftThreads, 4) dfft_cols_kernel(double2 *__restrict__ g, DfftDev d, int64_t stride,
                                                                 int64_t ncols, int64_t plane_cells, int64_t halfK,
                                                                 int64_t n2z, int64_t K, int64_t half, int band) {
    extern __shared__ float4 smem[];
    const int n = d.n;
    const int64_t tiles = (ncols + TX - 1) / TX;
    const int64_t P = blockIdx.x / tiles, c0 = (blockIdx.x - P * tiles) * TX;
    double2 *base = g + (band ? band_plane(P, halfK, n2z, K, half) * plane_cells : 0) + c0;
    const int valid = ncols - c0 < TX ? (int)(ncols - c0) : TX;
    float4 *a = smem, *b = smem + (size_t)n * TX;
    if constexpr (TX == 64) {  // the short z columns: first and last stage on the grid
        fft_pass<TX, SG>(a, b, d, ColLd<IN64>{base, stride, valid}, ColSt<OUT64>{base, stride, valid});
    } else {
        for (int e = threadIdx.x; e < n * TX; e += blockDim.x) {
            const int q = e / TX, t = e - q * TX;
            a[e] = t < valid ? load_cell<IN64>(base + q * stride + t) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const float4 *out = fft_smem<TX, SG>(a, b, d);
        for (int e = threadIdx.x; e < n * TX; e += blockDim.x) {
            const int q = e / TX, t = e - q * TX;
            if (t < valid) store_cell<OUT64>(base + q * stride + t, out[e]);
        }
    }
}

constexpr size_t kFftSmemMax = 220 * 1024;

template <typename K> void allow_smem(K kernel) {
    check_cuda(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFftSmemMax),
               "cudaFuncSetAttribute");
}

// Cell formats of a pass: kDD double-float in and out, kFD FP64 in, kDF FP64 out.
enum Io { kDD = 0, kFD = 1, kDF = 2 };

template <int TX, int SG> void allow_cols() {
    allow_smem(dfft_cols_kernel<TX, SG, false, false>);
    allow_smem(dfft_cols_kernel<TX, SG, true, false>);
    allow_smem(dfft_cols_kernel<TX, SG, false, true>);
}

template <int SG> void allow_sign() {
    allow_smem(dfft_rows_kernel<SG, true, false>);
    allow_smem(dfft_rows_kernel<SG, false, false>);
    allow_cols<1, SG>();
    allow_cols<2, SG>();
    allow_cols<8, SG>();
    allow_cols<64, SG>();
}

void set_fft_attrs() {
    static std::once_flag once;
    std::call_once(once, [] {
        allow_sign<1>();
        allow_sign<-1>();
    });
}

// Columns per CTA for a column transform of length n: as many as the shared memory holds
// (two buffers of n TX cells of 16 bytes), at most `want`.
int cols_per_cta(int n, int want) {
    for (int tx : {64, 8, 2, 1})
        if (tx <= want && (size_t)2 * n * tx * 16 <= kFftSmemMax) return tx;
    return 0;
}

template <int TX, int SG, bool IN64, bool OUT64>
void launch_cols(double2 *g, const DfftDev &d, int64_t stride, int64_t ncols, int64_t plane_cells, int64_t planes,
                 int64_t halfK, int64_t n2z, int64_t K, int64_t half, int band, cudaStream_t s) {
    const int64_t tiles = (ncols + TX - 1) / TX;
    const size_t smem = (size_t)(TX == 64 ? pass_buffers(d.stages) : 2) * d.n * TX * sizeof(float4);
    dfft_cols_kernel<TX, SG, IN64, OUT64><<<(unsigned)(planes * tiles), kFftThreads, smem, s>>>(
        g, d, stride, ncols, plane_cells, halfK, n2z, K, half, band);
    check_cuda(cudaGetLastError(), "dfft_cols");
}

template <int TX, int SG>
void launch_cols_io(Io io, double2 *g, const DfftDev &d, int64_t stride, int64_t ncols, int64_t plane_cells,
                    int64_t planes, int64_t halfK, int64_t n2z, int64_t K, int64_t half, int band, cudaStream_t s) {
    if (io == kFD) launch_cols<TX, SG, true, false>(g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, s);
    else if (io == kDF) launch_cols<TX, SG, false, true>(g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, s);
    else launch_cols<TX, SG, false, false>(g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, s);
}

template <int SG>
void cols_sign(int tx, Io io, double2 *g, const DfftDev &d, int64_t stride, int64_t ncols, int64_t plane_cells,
               int64_t planes, int64_t halfK, int64_t n2z, int64_t K, int64_t half, int band, cudaStream_t s) {
    switch (tx) {
        case 64: launch_cols_io<64, SG>(io, g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, s); break;
        case 8: launch_cols_io<8, SG>(io, g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, s); break;
        case 2: launch_cols_io<2, SG>(io, g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, s); break;
        default: launch_cols_io<1, SG>(io, g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, s); break;
    }
}

void cols(int tx, Io io, double2 *g, const DfftDev &d, int64_t stride, int64_t ncols, int64_t plane_cells,
          int64_t planes, int64_t halfK, int64_t n2z, int64_t K, int64_t half, int band, int sign, cudaStream_t s) {
    if (sign > 0) cols_sign<1>(tx, io, g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, s);
    else cols_sign<-1>(tx, io, g, d, stride, ncols, plane_cells, planes, halfK, n2z, K, half, band, s);
}

template <int SG>
void launch_rows(Io io, unsigned grid, size_t smem, double2 *g, const DfftDev &d, int64_t n2y, int64_t halfK,
                 int64_t n2z, int64_t K, int64_t half, int64_t rows, int64_t h1y, cudaStream_t s) {
    if (io == kFD)
        dfft_rows_kernel<SG, true, false><<<grid, kFftThreads, smem, s>>>(g, d, n2y, halfK, n2z, K, half, rows, h1y);
    else
        dfft_rows_kernel<SG, false, false><<<grid, kFftThreads, smem, s>>>(g, d, n2y, halfK, n2z, K, half, rows, h1y);
    check_cuda(cudaGetLastError(), "dfft_rows");
}

}  // namespace

namespace {
float4 cis_pair(int m, int r) {
    const double ang = 2.0 * M_PI * (double)m / (double)r;
    const double c = std::cos(ang), s = std::sin(ang);
    const float ch = (float)c, sh = (float)s;
    return make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
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
    long long Ns = 1;
    for (int st = 0; st < d.stages; ++st) {
        d.ns_magic[st] = Ns >= 2 ? (unsigned)((1ull << 32) / (unsigned long long)Ns + 1) : 0u;
        Ns *= d.radix[st];
    }
    int at = 0;
    for (int r : {3, 5, 7})
        for (int q = 1; q <= r / 2; ++q)
            for (int k = 1; k <= r / 2; ++k) d.odd[at++] = cis_pair((q * k) % r, r);
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
    // The grid is FP64 before the first pass (written by the deconvolution or the spreading)
    // and holds double-float values after it: the last pass leaves them for the
    // double-float gathers (sky -> vis) or crop (vis -> sky).
    auto rows = [&](Io io) {
        const int64_t r = 2 * f.h1y;  // band rows only
        const size_t smem = (size_t)2 * n2x * sizeof(float4);
        const unsigned grid = (unsigned)(band_planes * r);
        if (sign > 0) launch_rows<1>(io, grid, smem, g, f.dx, n2y, halfK, n2z, K, half, r, f.h1y, s);
        else launch_rows<-1>(io, grid, smem, g, f.dx, n2y, halfK, n2z, K, half, r, f.h1y, s);
    };
    // y columns: two adjacent columns per CTA (32-byte segments) unless that leaves fewer than
    // two CTAs per SM (long columns), then one (twice the DRAM sectors, at ~15 % of HBM).
    const int ty = (size_t)2 * n2y * 2 * sizeof(float4) <= kFftSmemMax / 2 ? 2 : 1;
    auto ycols = [&] {
        cols(cols_per_cta((int)n2y, ty), kDD, g, f.dy, n2x, n2x, plane, band_planes, halfK, n2z, K, half, 1, sign, s);
    };
    auto zcols = [&](Io io) {
        cols(cols_per_cta((int)n2z, 64), io, g, f.dz, K * plane, K * plane, 0, 1, halfK, n2z, K, half, 0, sign, s);
    };
    if (band_input) {  // only the band rows of the band planes are nonzero
        rows(kFD);
        ycols();
        zcols(kDD);
    } else {  // only the band rows of the band planes are read afterwards
        zcols(kFD);
        ycols();
        rows(kDD);
    }
    return 3;
}

}  // namespace hvox
