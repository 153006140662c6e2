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
// Spreading: each CTA takes 256 consecutive points (chunk order is Morton order inside a
// chunk, so they are close in space), accumulates their w^3 taps into a shared-memory
// tile that covers all their windows, then adds the tile to the grid with vector
// atomics; when the tile would not fit, the CTA adds its taps to the grid directly.
#include <climits>
#include <cstdint>
#include <vector>

#include "hvox_internal.h"

namespace hvox {

namespace {

template <typename T> using cplx_t = typename CplxOf<T>::type;

constexpr int kSpreadThreads = 256;

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

// Same weights with the tap order rotated: wt[j] = phi((j + rot) mod W - fr).
template <typename T, int W> __device__ __forceinline__ void es_weights_rot(T fr, T beta, int rot, T *wt) {
    const T inv = T(2) / T(W);
#pragma unroll
    for (int j = 0; j < W; ++j) {
        int jr = j + rot;
        jr = jr >= W ? jr - W : jr;
        T x = (T(jr) - fr) * inv;
        T q = T(1) - x * x;
        wt[j] = q > T(0) ? es_exp(beta * (sqrt(q) - T(1))) : T(0);
    }
}

// i mod n for i in [-n, 2n): window cells of points inside a sub-problem's band lie within
// n2/2 + w of the origin and n2 >= 2w. The clamp keeps any index inside the grid.
__device__ __forceinline__ int wrap(int i, int n) {
    i += i < 0 ? n : 0;
    i -= i >= n ? n : 0;
    return min(max(i, 0), n - 1);
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
        i0[d] = min(max(i0[d], 0), b.n1[d] - W);
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
        i0[d] = min(max(i0[d], 0), b.n1[d] - W);
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
__device__ __forceinline__ void tile_add(float2 *t, float re, float im) {
    atomicAdd(&t->x, re);
    atomicAdd(&t->y, im);
}
__device__ __forceinline__ void tile_add(double2 *t, double re, double im) {
    atomicAdd(&t->x, re);
    atomicAdd(&t->y, im);
}

// ------------------------------------------------------------------ spreading (tiled)

// Shared-memory tile over the union of the CTA's windows, then vector-atomic flush.
// PERIODIC: grid indices wrap (n2 grid) instead of lying inside (n1 grid).
template <typename T, int W, bool PERIODIC>
__device__ __forceinline__ void spread_tiled(bool act, const int i0[3], const T fr[3], T vr, T vi, T beta,
                                             const int ng[3], cplx_t<T> *__restrict__ G, int tile_cap) {
    extern __shared__ unsigned char smem_raw[];
    cplx_t<T> *tile = reinterpret_cast<cplx_t<T> *>(smem_raw);
    __shared__ int s_lo[3], s_hi[3];
    if (threadIdx.x < 3) {
        s_lo[threadIdx.x] = INT_MAX;
        s_hi[threadIdx.x] = INT_MIN;
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            atomicMin(&s_lo[d], i0[d]);
            atomicMax(&s_hi[d], i0[d]);
        }
    }
    __syncthreads();
    const int lo0 = s_lo[0], lo1 = s_lo[1], lo2 = s_lo[2];
    const int64_t tx = (int64_t)s_hi[0] - lo0 + W, ty = (int64_t)s_hi[1] - lo1 + W, tz = (int64_t)s_hi[2] - lo2 + W;
    const int64_t cells = tx * ty * tz;
    // Lanes whose windows coincide (clustered points) would add to the same cell in the
    // same instruction; rotating the z order of the taps by lane spreads those adds.
    const int rot = (threadIdx.x & 31) % W;
    T wx[W], wy[W], wz[W];
    if (act) {
        es_weights<T, W>(fr[0], beta, wx);
        es_weights<T, W>(fr[1], beta, wy);
        es_weights_rot<T, W>(fr[2], beta, rot, wz);
    }
    if (s_hi[0] >= lo0 && cells <= tile_cap) {
        for (int64_t j = threadIdx.x; j < cells; j += blockDim.x) {
            tile[j].x = T(0);
            tile[j].y = T(0);
        }
        __syncthreads();
        if (act) {
            for (int jz = 0; jz < W; ++jz) {
                int jzr = jz + rot;
                jzr = jzr >= W ? jzr - W : jzr;
                for (int jy = 0; jy < W; ++jy) {
                    const T wyz = wy[jy] * wz[jz];
                    const T ar = vr * wyz, ai = vi * wyz;
                    cplx_t<T> *row = tile + ((int64_t)(i0[2] - lo2 + jzr) * ty + (i0[1] - lo1 + jy)) * tx + (i0[0] - lo0);
#pragma unroll
                    for (int jx = 0; jx < W; ++jx) tile_add(row + jx, ar * wx[jx], ai * wx[jx]);
                }
            }
        }
        __syncthreads();
        // Flush: one warp per (y, z) row of the tile, lanes along x (coalesced atomics).
        const int txi = (int)tx, tyi = (int)ty, rows = (int)(ty * tz);
        const int lane = threadIdx.x & 31;
        for (int r = threadIdx.x >> 5; r < rows; r += blockDim.x >> 5) {
            const int y = r % tyi, z = r / tyi;
            int gy = lo1 + y, gz = lo2 + z;
            if (PERIODIC) {
                gy = wrap(gy, ng[1]);
                gz = wrap(gz, ng[2]);
            }
            cplx_t<T> *grow = G + ((int64_t)gz * ng[1] + gy) * ng[0];
            const cplx_t<T> *trow = tile + (int64_t)r * txi;
            for (int x = lane; x < txi; x += 32) {
                const cplx_t<T> v = trow[x];
                if (v.x == T(0) && v.y == T(0)) continue;
                const int gx = PERIODIC ? wrap(lo0 + x, ng[0]) : lo0 + x;
                grid_add(grow + gx, v.x, v.y);
            }
        }
    } else if (act) {
        int64_t ix[W];
#pragma unroll
        for (int j = 0; j < W; ++j) ix[j] = PERIODIC ? wrap(i0[0] + j, ng[0]) : i0[0] + j;
        for (int jz = 0; jz < W; ++jz) {
            int jzr = jz + rot;
            jzr = jzr >= W ? jzr - W : jzr;
            const int64_t gz = PERIODIC ? wrap(i0[2] + jzr, ng[2]) : i0[2] + jzr;
            for (int jy = 0; jy < W; ++jy) {
                const int64_t gy = PERIODIC ? wrap(i0[1] + jy, ng[1]) : i0[1] + jy;
                const T wyz = wy[jy] * wz[jz];
                const T ar = vr * wyz, ai = vi * wyz;
                cplx_t<T> *row = G + (gz * ng[1] + gy) * ng[0];
#pragma unroll
                for (int jx = 0; jx < W; ++jx) grid_add(row + ix[jx], ar * wx[jx], ai * wx[jx]);
            }
        }
    }
}

// Point of the CTA's 256 handled by this thread: warp w takes points w, w + 8, w + 16, ...
// so that the 32 lanes of a warp are spread over the CTA's (spatially ordered) points.
__device__ __forceinline__ int cta_slot() { return (threadIdx.x & 31) * (kSpreadThreads / 32) + (threadIdx.x >> 5); }

// sky -> vis step 1: pixels (values c, prephase P) onto the n1 grid.
template <typename T, int W>
__global__ void __launch_bounds__(kSpreadThreads) spread_pix_kernel(NufftDev b, const float4 *__restrict__ rh,
                                                                     const float4 *__restrict__ rl,
                                                                     const double *__restrict__ soa, int64_t n_all,
                                                                     const T *__restrict__ c, cplx_t<T> *__restrict__ G1,
                                                                     T beta, int isign, int tile_cap) {
    const int64_t i = blockIdx.x * (int64_t)kSpreadThreads + cta_slot();
    const bool act = i < b.np;
    int i0[3] = {0, 0, 0};
    T fr[3] = {0, 0, 0}, vr = 0, vi = 0;
    if (act) {
        T pr, pim;
        geo_pix<W>(b, b.p0 + i, rh, rl, soa, n_all, isign, i0, fr, pr, pim);
        const T cv = c[b.p0 + i];
        vr = cv * pr;
        vi = cv * pim;
    }
    const int ng[3] = {b.n1[0], b.n1[1], b.n1[2]};
    spread_tiled<T, W, false>(act, i0, fr, vr, vi, beta, ng, G1, tile_cap);
}

// vis -> sky step 1 (transpose of the interpolation): baselines u = conj(Q) V onto the n2 grid.
template <typename T, int W>
__global__ void __launch_bounds__(kSpreadThreads) spread_vis_kernel(NufftDev b, const float4 *__restrict__ vh,
                                                                     const float4 *__restrict__ vl,
                                                                     const double *__restrict__ soa, int64_t n_all,
                                                                     const cplx_t<T> *__restrict__ V,
                                                                     const T *__restrict__ cc, int deg, T inv_tmax2,
                                                                     cplx_t<T> *__restrict__ G2, T beta, int isign,
                                                                     int tile_cap) {
    const int64_t k = blockIdx.x * (int64_t)kSpreadThreads + cta_slot();
    const bool act = k < b.nv;
    int i0[3] = {0, 0, 0};
    T fr[3] = {0, 0, 0}, ur = 0, ui = 0;
    if (act) {
        T qr, qi;
        geo_vis<W>(b, b.v0 + k, vh, vl, soa, n_all, isign, cc, deg, inv_tmax2, i0, fr, qr, qi);
        const cplx_t<T> v = V[b.v0 + k];
        ur = qr * v.x + qi * v.y;  // conj(Q) v
        ui = qr * v.y - qi * v.x;
    }
    const int ng[3] = {b.n2[0], b.n2[1], b.n2[2]};
    spread_tiled<T, W, true>(act, i0, fr, ur, ui, beta, ng, G2, tile_cap);
}

// ------------------------------------------------------------------ interpolation (gather)

// sky -> vis steps 3-4: gather the n2 grid at the baselines, times Q; add into acc.
template <typename T, int W>
__global__ void __launch_bounds__(128) interp_vis_kernel(NufftDev b, const float4 *__restrict__ vh,
                                                          const float4 *__restrict__ vl, const double *__restrict__ soa,
                                                          int64_t n_all, const cplx_t<T> *__restrict__ G2,
                                                          const T *__restrict__ cc, int deg, T inv_tmax2,
                                                          cplx_t<T> *__restrict__ acc, T beta, int isign) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= b.nv) return;
    int i0[3];
    T fr[3], qr, qi;
    geo_vis<W>(b, b.v0 + k, vh, vl, soa, n_all, isign, cc, deg, inv_tmax2, i0, fr, qr, qi);
    T wx[W], wy[W], wz[W];
    es_weights<T, W>(fr[0], beta, wx);
    es_weights<T, W>(fr[1], beta, wy);
    es_weights<T, W>(fr[2], beta, wz);
    const int64_t nx = b.n2[0], ny = b.n2[1], nz = b.n2[2];
    int64_t ix[W], iy[W], iz[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
        ix[j] = wrap(i0[0] + j, (int)nx);
        iy[j] = (int64_t)wrap(i0[1] + j, (int)ny) * nx;
        iz[j] = (int64_t)wrap(i0[2] + j, (int)nz) * ny * nx;
    }
    T sr = 0, si = 0;
    for (int jz = 0; jz < W; ++jz) {
        for (int jy = 0; jy < W; ++jy) {
            const cplx_t<T> *row = G2 + iz[jz] + iy[jy];
            T rr = 0, ri = 0;
#pragma unroll
            for (int jx = 0; jx < W; ++jx) {
                const cplx_t<T> g = row[ix[jx]];
                rr += g.x * wx[jx];
                ri += g.y * wx[jx];
            }
            const T wyz = wy[jy] * wz[jz];
            sr += rr * wyz;
            si += ri * wyz;
        }
    }
    grid_add(acc + b.v0 + k, qr * sr - qi * si, qr * si + qi * sr);
}

// vis -> sky steps 3-4 (transpose of the spreading): gather the n1 grid at the pixels,
// times conj(P), real part into acc.
template <typename T, int W>
__global__ void __launch_bounds__(128) interp_pix_kernel(NufftDev b, const float4 *__restrict__ rh,
                                                          const float4 *__restrict__ rl, const double *__restrict__ soa,
                                                          int64_t n_all, const cplx_t<T> *__restrict__ G1,
                                                          T *__restrict__ acc, T beta, int isign) {
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

// ------------------------------------------------------------------ deconvolution passes

// G2[j] = G1[l + n1/2] / (Psi_x Psi_y Psi_z)(l) for the centred frequency l of FFT index j
// inside the n1 band, 0 elsewhere. One thread per x index of a (y, z) row: coalesced rows,
// no integer division.
template <typename T>
__global__ void deconv_pad_kernel(NufftDev b, const cplx_t<T> *__restrict__ G1, const T *__restrict__ ipsi,
                                  cplx_t<T> *__restrict__ G2) {
    const int jx = blockIdx.x * blockDim.x + threadIdx.x;
    const int jy = blockIdx.y, jz = blockIdx.z;
    const int n2x = b.n2[0], n2y = b.n2[1], n2z = b.n2[2];
    if (jx >= n2x) return;
    const int h1x = b.n1[0] / 2, h1y = b.n1[1] / 2, h1z = b.n1[2] / 2;
    const int lx = jx < n2x / 2 ? jx : jx - n2x;
    const int ly = jy < n2y / 2 ? jy : jy - n2y;
    const int lz = jz < n2z / 2 ? jz : jz - n2z;
    cplx_t<T> out;
    out.x = T(0);
    out.y = T(0);
    if (lx >= -h1x && lx < h1x && ly >= -h1y && ly < h1y && lz >= -h1z && lz < h1z) {
        const int ix = lx + h1x, iy = ly + h1y, iz = lz + h1z;
        const T *px = ipsi, *py = ipsi + b.n1[0], *pz = py + b.n1[1];
        const T f = px[ix] * py[iy] * pz[iz];
        const cplx_t<T> g = G1[((int64_t)iz * b.n1[1] + iy) * b.n1[0] + ix];
        out.x = g.x * f;
        out.y = g.y * f;
    }
    G2[((int64_t)jz * n2y + jy) * n2x + jx] = out;
}

// G1[l + n1/2] = G2[l mod n2] / (Psi_x Psi_y Psi_z)(l), l in the n1 band (row-wise, as above).
template <typename T>
__global__ void crop_deconv_kernel(NufftDev b, const cplx_t<T> *__restrict__ G2, const T *__restrict__ ipsi,
                                   cplx_t<T> *__restrict__ G1) {
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iy = blockIdx.y, iz = blockIdx.z;
    const int n1x = b.n1[0], n1y = b.n1[1], n1z = b.n1[2];
    if (ix >= n1x) return;
    const int n2x = b.n2[0], n2y = b.n2[1], n2z = b.n2[2];
    int jx = ix - n1x / 2, jy = iy - n1y / 2, jz = iz - n1z / 2;
    jx += jx < 0 ? n2x : 0;
    jy += jy < 0 ? n2y : 0;
    jz += jz < 0 ? n2z : 0;
    const cplx_t<T> g = G2[((int64_t)jz * n2y + jy) * n2x + jx];
    const T *px = ipsi, *py = ipsi + n1x, *pz = py + n1y;
    const T f = px[ix] * py[iy] * pz[iz];
    cplx_t<T> out;
    out.x = g.x * f;
    out.y = g.y * f;
    G1[((int64_t)iz * n1y + iy) * n1x + ix] = out;
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


// Dynamic shared memory of the spreading kernels (tile capacity in cells).
constexpr int kTileBytes = 96 * 1024;

template <typename T, int W> void set_smem_attrs() {
    static bool done = false;
    if (done) return;
    check_cuda(cudaFuncSetAttribute(spread_pix_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileBytes),
               "cudaFuncSetAttribute");
    check_cuda(cudaFuncSetAttribute(spread_vis_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileBytes),
               "cudaFuncSetAttribute");
    done = true;
}

}  // namespace

// ------------------------------------------------------------------ host launchers

template <typename T>
void nufft_block_s2v(const NufftDev &b, const NufftArgs<T> &a, const T *c, cplx_t<T> *acc, cudaStream_t s,
                     StageHook &hook) {
    const int w = a.w;
    const T bt = (T)a.beta;
    const int64_t m1 = (int64_t)b.n1[0] * b.n1[1] * b.n1[2];
    hook.begin(HVOX_STAGE_ZERO, s);
    check_cuda(cudaMemsetAsync(a.G1, 0, sizeof(cplx_t<T>) * m1, s), "memset G1");
    hook.end(HVOX_STAGE_ZERO, 1, s);
    const int cap = kTileBytes / (int)sizeof(cplx_t<T>);
    if (b.np > 0) {
        hook.begin(HVOX_STAGE_SPREAD, s);
#define CALL(W)                                                                                                   \
    set_smem_attrs<T, W>();                                                                                       \
    spread_pix_kernel<T, W><<<blocks_for(b.np, kSpreadThreads), kSpreadThreads, kTileBytes, s>>>(                 \
        b, a.pix_hi, a.pix_lo, a.pix_soa, a.n_pix, c, a.G1, bt, a.isign, cap)
        HVOX_W_SWITCH(w, CALL)
#undef CALL
        check_cuda(cudaGetLastError(), "spread_pix");
        hook.end(HVOX_STAGE_SPREAD, 1, s);
    }
    const int64_t m2 = (int64_t)b.n2[0] * b.n2[1] * b.n2[2];
    hook.begin(HVOX_STAGE_DECONV, s);
    deconv_pad_kernel<T><<<dim3((unsigned)((b.n2[0] + 127) / 128), (unsigned)b.n2[1], (unsigned)b.n2[2]), 128, 0, s>>>(
        b, a.G1, a.ipsi + b.psi_off, a.G2);
    check_cuda(cudaGetLastError(), "deconv_pad");
    hook.end(HVOX_STAGE_DECONV, 1, s);
    hook.begin(HVOX_STAGE_FFT, s);
    check_cufft(cufftSetStream(a.fft, s), "cufftSetStream");
    const int dir = a.isign < 0 ? CUFFT_FORWARD : CUFFT_INVERSE;
    if constexpr (sizeof(T) == 4)
        check_cufft(cufftExecC2C(a.fft, (cufftComplex *)a.G2, (cufftComplex *)a.G2, dir), "cufftExecC2C");
    else
        check_cufft(cufftExecZ2Z(a.fft, (cufftDoubleComplex *)a.G2, (cufftDoubleComplex *)a.G2, dir), "cufftExecZ2Z");
    hook.end(HVOX_STAGE_FFT, 1, s);
    if (b.nv > 0) {
        hook.begin(HVOX_STAGE_INTERP, s);
#define CALL(W)                                                                                                   \
    interp_vis_kernel<T, W><<<blocks_for(b.nv, 128), 128, 0, s>>>(b, a.vis_hi, a.vis_lo, a.vis_soa, a.n_vis, a.G2, \
                                                                  a.cheb, a.deg, (T)a.inv_tmax2, acc, bt, a.isign)
        HVOX_W_SWITCH(w, CALL)
#undef CALL
        check_cuda(cudaGetLastError(), "interp_vis");
        hook.end(HVOX_STAGE_INTERP, 1, s);
    }
}

template <typename T>
void nufft_block_v2s(const NufftDev &b, const NufftArgs<T> &a, const cplx_t<T> *V, T *acc, cudaStream_t s,
                     StageHook &hook) {
    const int w = a.w;
    const T bt = (T)a.beta;
    const int64_t m2 = (int64_t)b.n2[0] * b.n2[1] * b.n2[2];
    hook.begin(HVOX_STAGE_ZERO, s);
    check_cuda(cudaMemsetAsync(a.G2, 0, sizeof(cplx_t<T>) * m2, s), "memset G2");
    hook.end(HVOX_STAGE_ZERO, 1, s);
    const int cap = kTileBytes / (int)sizeof(cplx_t<T>);
    if (b.nv > 0) {
        hook.begin(HVOX_STAGE_SPREAD, s);
#define CALL(W)                                                                                                   \
    set_smem_attrs<T, W>();                                                                                       \
    spread_vis_kernel<T, W><<<blocks_for(b.nv, kSpreadThreads), kSpreadThreads, kTileBytes, s>>>(                 \
        b, a.vis_hi, a.vis_lo, a.vis_soa, a.n_vis, V, a.cheb, a.deg, (T)a.inv_tmax2, a.G2, bt, a.isign, cap)
        HVOX_W_SWITCH(w, CALL)
#undef CALL
        check_cuda(cudaGetLastError(), "spread_vis");
        hook.end(HVOX_STAGE_SPREAD, 1, s);
    }
    hook.begin(HVOX_STAGE_FFT, s);
    check_cufft(cufftSetStream(a.fft, s), "cufftSetStream");
    const int dir = a.isign < 0 ? CUFFT_INVERSE : CUFFT_FORWARD;  // transpose: opposite sign
    if constexpr (sizeof(T) == 4)
        check_cufft(cufftExecC2C(a.fft, (cufftComplex *)a.G2, (cufftComplex *)a.G2, dir), "cufftExecC2C");
    else
        check_cufft(cufftExecZ2Z(a.fft, (cufftDoubleComplex *)a.G2, (cufftDoubleComplex *)a.G2, dir), "cufftExecZ2Z");
    hook.end(HVOX_STAGE_FFT, 1, s);
    const int64_t m1 = (int64_t)b.n1[0] * b.n1[1] * b.n1[2];
    hook.begin(HVOX_STAGE_DECONV, s);
    crop_deconv_kernel<T><<<dim3((unsigned)((b.n1[0] + 127) / 128), (unsigned)b.n1[1], (unsigned)b.n1[2]), 128, 0, s>>>(
        b, a.G2, a.ipsi + b.psi_off, a.G1);
    check_cuda(cudaGetLastError(), "crop_deconv");
    hook.end(HVOX_STAGE_DECONV, 1, s);
    if (b.np > 0) {
        hook.begin(HVOX_STAGE_INTERP, s);
#define CALL(W)                                                                                                   \
    interp_pix_kernel<T, W><<<blocks_for(b.np, 128), 128, 0, s>>>(b, a.pix_hi, a.pix_lo, a.pix_soa, a.n_pix, a.G1, \
                                                                  acc, bt, a.isign)
        HVOX_W_SWITCH(w, CALL)
#undef CALL
        check_cuda(cudaGetLastError(), "interp_pix");
        hook.end(HVOX_STAGE_INTERP, 1, s);
    }
}

template void nufft_block_s2v<float>(const NufftDev &, const NufftArgs<float> &, const float *, float2 *,
                                     cudaStream_t, StageHook &);
template void nufft_block_s2v<double>(const NufftDev &, const NufftArgs<double> &, const double *, double2 *,
                                      cudaStream_t, StageHook &);
template void nufft_block_v2s<float>(const NufftDev &, const NufftArgs<float> &, const float2 *, float *,
                                     cudaStream_t, StageHook &);
template void nufft_block_v2s<double>(const NufftDev &, const NufftArgs<double> &, const double2 *, double *,
                                      cudaStream_t, StageHook &);

}  // namespace hvox
