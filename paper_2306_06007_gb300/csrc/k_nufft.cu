// Type-3 NUFFT sub-problems (Sect. 3, steps 1-4; Eq. 5-7 size the grids).
//
// For a block with pixel box centre C, baseline box centre D (wavelengths), per
// dimension: r~ = r - C, p~ = p - D, spread-grid scale a (cells per unit of r),
// spread grid n1, FFT grid n2. With s = isign:
//
//   f_k = Q_k sum_j G_j psi(v_k - j)                      (interpolate, n2 grid, periodic)
//   G   = FFT_s( pad( b_l / Psi(l) ) ),  l in [-n1/2, n1/2)  (deconvolve, zero-pad, FFT)
//   b_l = sum_n P_n c_n phi(l - g_n)                       (spread, n1 grid)
//   g_n = a r~_n + n1/2,  v_k = p~_k n2 / a,  tau_k = 2 pi p~_k / a
//   P_n = exp(s j 2 pi <D, r~_n>),  Q_k = exp(s j 2 pi <C, p_k>) / prod_d Phi(tau_kd)
//
// phi = psi = ES kernel of width w; Phi(tau) = int phi(z) cos(tau z) dz on the n1 grid,
// Psi(l) = int psi(z) cos(2 pi l z / n2) dz on the n2 grid. vis -> sky runs the exact
// transpose of every step (spread at baselines on n2, FFT_-s, crop and divide, gather
// at pixels), so the pair is adjoint to rounding.
#include <cstdint>
#include <vector>

#include "hvox_internal.h"

namespace hvox {

namespace {

template <typename T> using cplx_t = typename CplxOf<T>::type;

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

// ------------------------------------------------------------------ sky -> vis

template <typename T, int W>
__global__ void spread_pix_kernel(DevBlock b, const T *__restrict__ c, const GridRec<T> *__restrict__ rec,
                                  const cplx_t<T> *__restrict__ ph, cplx_t<T> *__restrict__ G1, T beta) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= b.np) return;
    const GridRec<T> r = rec[b.prec_off + i];
    const cplx_t<T> P = ph[b.prec_off + i];
    const T cv = c[b.p0 + i];
    const T vr = cv * P.x, vi = cv * P.y;
    T wx[W], wy[W], wz[W];
    es_weights<T, W>(r.fr[0], beta, wx);
    es_weights<T, W>(r.fr[1], beta, wy);
    es_weights<T, W>(r.fr[2], beta, wz);
    const int64_t nx = b.n1[0], ny = b.n1[1];
    for (int jz = 0; jz < W; ++jz) {
        for (int jy = 0; jy < W; ++jy) {
            const T wyz = wy[jy] * wz[jz];
            const int64_t base = ((int64_t)(r.i0[2] + jz) * ny + (r.i0[1] + jy)) * nx + r.i0[0];
            const T ar = vr * wyz, ai = vi * wyz;
#pragma unroll
            for (int jx = 0; jx < W; ++jx) {
                atomicAdd(&G1[base + jx].x, ar * wx[jx]);
                atomicAdd(&G1[base + jx].y, ai * wx[jx]);
            }
        }
    }
}

// G2[j] = G1[l + n1/2] / (Psi_x Psi_y Psi_z)(l) for the centred frequency l of FFT index j
// inside the n1 band, 0 elsewhere.
template <typename T>
__global__ void deconv_pad_kernel(DevBlock b, const cplx_t<T> *__restrict__ G1, const T *__restrict__ ipsi,
                                  cplx_t<T> *__restrict__ G2) {
    const int64_t n2x = b.n2[0], n2y = b.n2[1], n2z = b.n2[2];
    const int64_t total = n2x * n2y * n2z;
    const T *px = ipsi, *py = ipsi + b.n1[0], *pz = py + b.n1[1];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
        int64_t jx = j % n2x, t = j / n2x;
        int64_t jy = t % n2y, jz = t / n2y;
        int64_t lx = jx < n2x / 2 ? jx : jx - n2x;
        int64_t ly = jy < n2y / 2 ? jy : jy - n2y;
        int64_t lz = jz < n2z / 2 ? jz : jz - n2z;
        cplx_t<T> out;
        out.x = T(0);
        out.y = T(0);
        if (lx >= -b.n1[0] / 2 && lx < b.n1[0] / 2 && ly >= -b.n1[1] / 2 && ly < b.n1[1] / 2 && lz >= -b.n1[2] / 2 &&
            lz < b.n1[2] / 2) {
            int64_t ix = lx + b.n1[0] / 2, iy = ly + b.n1[1] / 2, iz = lz + b.n1[2] / 2;
            T f = px[ix] * py[iy] * pz[iz];
            cplx_t<T> g = G1[(iz * b.n1[1] + iy) * b.n1[0] + ix];
            out.x = g.x * f;
            out.y = g.y * f;
        }
        G2[j] = out;
    }
}

__device__ __forceinline__ int64_t wrap(int64_t i, int64_t n) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

template <typename T, int W>
__global__ void interp_vis_kernel(DevBlock b, const cplx_t<T> *__restrict__ G2, const GridRec<T> *__restrict__ rec,
                                  const cplx_t<T> *__restrict__ q, cplx_t<T> *__restrict__ acc, T beta) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= b.nv) return;
    const GridRec<T> r = rec[b.vrec_off + k];
    T wx[W], wy[W], wz[W];
    es_weights<T, W>(r.fr[0], beta, wx);
    es_weights<T, W>(r.fr[1], beta, wy);
    es_weights<T, W>(r.fr[2], beta, wz);
    const int64_t nx = b.n2[0], ny = b.n2[1], nz = b.n2[2];
    int64_t ix[W];
#pragma unroll
    for (int j = 0; j < W; ++j) ix[j] = wrap((int64_t)r.i0[0] + j, nx);
    T sr = 0, si = 0;
    for (int jz = 0; jz < W; ++jz) {
        const int64_t iz = wrap((int64_t)r.i0[2] + jz, nz);
        for (int jy = 0; jy < W; ++jy) {
            const int64_t iy = wrap((int64_t)r.i0[1] + jy, ny);
            const cplx_t<T> *row = G2 + (iz * ny + iy) * nx;
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
    const cplx_t<T> Q = q[b.vrec_off + k];
    atomicAdd(&acc[b.v0 + k].x, Q.x * sr - Q.y * si);
    atomicAdd(&acc[b.v0 + k].y, Q.x * si + Q.y * sr);
}

// ------------------------------------------------------------------ vis -> sky (transposes)

template <typename T, int W>
__global__ void spread_vis_kernel(DevBlock b, const cplx_t<T> *__restrict__ V, const GridRec<T> *__restrict__ rec,
                                  const cplx_t<T> *__restrict__ q, cplx_t<T> *__restrict__ G2, T beta) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= b.nv) return;
    const GridRec<T> r = rec[b.vrec_off + k];
    const cplx_t<T> Q = q[b.vrec_off + k];
    const cplx_t<T> v = V[b.v0 + k];
    // u = conj(Q) v
    const T ur = Q.x * v.x + Q.y * v.y, ui = Q.x * v.y - Q.y * v.x;
    T wx[W], wy[W], wz[W];
    es_weights<T, W>(r.fr[0], beta, wx);
    es_weights<T, W>(r.fr[1], beta, wy);
    es_weights<T, W>(r.fr[2], beta, wz);
    const int64_t nx = b.n2[0], ny = b.n2[1], nz = b.n2[2];
    int64_t ix[W];
#pragma unroll
    for (int j = 0; j < W; ++j) ix[j] = wrap((int64_t)r.i0[0] + j, nx);
    for (int jz = 0; jz < W; ++jz) {
        const int64_t iz = wrap((int64_t)r.i0[2] + jz, nz);
        for (int jy = 0; jy < W; ++jy) {
            const int64_t iy = wrap((int64_t)r.i0[1] + jy, ny);
            cplx_t<T> *row = G2 + (iz * ny + iy) * nx;
            const T wyz = wy[jy] * wz[jz];
            const T ar = ur * wyz, ai = ui * wyz;
#pragma unroll
            for (int jx = 0; jx < W; ++jx) {
                atomicAdd(&row[ix[jx]].x, ar * wx[jx]);
                atomicAdd(&row[ix[jx]].y, ai * wx[jx]);
            }
        }
    }
}

// G1[l + n1/2] = G2[l mod n2] / (Psi_x Psi_y Psi_z)(l), l in the n1 band.
template <typename T>
__global__ void crop_deconv_kernel(DevBlock b, const cplx_t<T> *__restrict__ G2, const T *__restrict__ ipsi,
                                   cplx_t<T> *__restrict__ G1) {
    const int64_t n1x = b.n1[0], n1y = b.n1[1], n1z = b.n1[2];
    const int64_t total = n1x * n1y * n1z;
    const T *px = ipsi, *py = ipsi + n1x, *pz = py + n1y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t ix = i % n1x, t = i / n1x;
        int64_t iy = t % n1y, iz = t / n1y;
        int64_t jx = wrap(ix - n1x / 2, b.n2[0]), jy = wrap(iy - n1y / 2, b.n2[1]), jz = wrap(iz - n1z / 2, b.n2[2]);
        cplx_t<T> g = G2[(jz * b.n2[1] + jy) * b.n2[0] + jx];
        T f = px[ix] * py[iy] * pz[iz];
        cplx_t<T> out;
        out.x = g.x * f;
        out.y = g.y * f;
        G1[i] = out;
    }
}

template <typename T, int W>
__global__ void interp_pix_kernel(DevBlock b, const cplx_t<T> *__restrict__ G1, const GridRec<T> *__restrict__ rec,
                                  const cplx_t<T> *__restrict__ ph, T *__restrict__ acc, T beta) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= b.np) return;
    const GridRec<T> r = rec[b.prec_off + i];
    T wx[W], wy[W], wz[W];
    es_weights<T, W>(r.fr[0], beta, wx);
    es_weights<T, W>(r.fr[1], beta, wy);
    es_weights<T, W>(r.fr[2], beta, wz);
    const int64_t nx = b.n1[0], ny = b.n1[1];
    T sr = 0, si = 0;
    for (int jz = 0; jz < W; ++jz) {
        for (int jy = 0; jy < W; ++jy) {
            const cplx_t<T> *row = G1 + ((int64_t)(r.i0[2] + jz) * ny + (r.i0[1] + jy)) * nx + r.i0[0];
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
    const cplx_t<T> P = ph[b.prec_off + i];
    // Re(conj(P) y)
    atomicAdd(&acc[b.p0 + i], P.x * sr + P.y * si);
}

// ------------------------------------------------------------------ plan-time tables

// Pixel-side records: window start, offset, prephase exp(s j 2 pi <D, r~>).
template <typename T>
__global__ void pix_tables_kernel(int64_t np, const double *__restrict__ xyz, int64_t n_all, int64_t p0, double3 C,
                                  double3 D, double3 a, int3 n1, int w, int isign, GridRec<T> *__restrict__ rec,
                                  cplx_t<T> *__restrict__ ph, int *__restrict__ err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const double r[3] = {xyz[p0 + i] - C.x, xyz[n_all + p0 + i] - C.y, xyz[2 * n_all + p0 + i] - C.z};
    const double aa[3] = {a.x, a.y, a.z};
    const int nn[3] = {n1.x, n1.y, n1.z};
    GridRec<T> R;
    R.pad = 0;
    R.pad2 = T(0);
    for (int d = 0; d < 3; ++d) {
        double g = aa[d] * r[d] + 0.5 * nn[d];
        double i0 = ceil(g - 0.5 * w);
        if (i0 < 0.0 || i0 + w > nn[d]) {
            atomicExch(err, 1);
            i0 = fmin(fmax(i0, 0.0), (double)(nn[d] - w));
        }
        R.i0[d] = (int32_t)i0;
        R.fr[d] = (T)(g - i0);
    }
    rec[i] = R;
    double t = fma(D.x, r[0], fma(D.y, r[1], D.z * r[2]));
    t -= rint(t);
    double s, c;
    sincospi(2.0 * t, &s, &c);
    cplx_t<T> P;
    P.x = (T)c;
    P.y = (T)(isign * s);
    ph[i] = P;
}

// Baseline-side records: window start and offset on the n2 grid, and
// Q = exp(s j 2 pi <C, p>) / prod_d Phi(tau_d) with Phi by Gauss-Legendre quadrature.
template <typename T>
__global__ void vis_tables_kernel(int64_t nv, const double *__restrict__ xyz, int64_t n_all, int64_t v0, double3 C,
                                  double3 D, double3 a, int3 n2, int w, int isign, const double *__restrict__ qz,
                                  const double *__restrict__ qf, int nq, GridRec<T> *__restrict__ rec,
                                  cplx_t<T> *__restrict__ q) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nv) return;
    const double p[3] = {xyz[v0 + k], xyz[n_all + v0 + k], xyz[2 * n_all + v0 + k]};
    const double pt[3] = {p[0] - D.x, p[1] - D.y, p[2] - D.z};
    const double aa[3] = {a.x, a.y, a.z};
    const int nn[3] = {n2.x, n2.y, n2.z};
    GridRec<T> R;
    R.pad = 0;
    R.pad2 = T(0);
    double phiprod = 1.0;
    for (int d = 0; d < 3; ++d) {
        double v = aa[d] > 0.0 ? pt[d] * nn[d] / aa[d] : 0.0;
        double j0 = ceil(v - 0.5 * w);
        R.i0[d] = (int32_t)j0;
        R.fr[d] = (T)(v - j0);
        double tau = aa[d] > 0.0 ? 2.0 * M_PI * pt[d] / aa[d] : 0.0;
        double s = 0.0;
        for (int m = 0; m < nq; ++m) s += qf[m] * cos(tau * qz[m]);
        phiprod *= s;
    }
    rec[k] = R;
    double t = fma(C.x, p[0], fma(C.y, p[1], C.z * p[2]));
    t -= rint(t);
    double s, c;
    sincospi(2.0 * t, &s, &c);
    cplx_t<T> Q;
    Q.x = (T)(c / phiprod);
    Q.y = (T)(isign * s / phiprod);
    q[k] = Q;
}

// ------------------------------------------------------------------ dispatch on W

#define HVOX_W_SWITCH(w, CALL)                       \
    switch (w) {                                     \
        case 2: CALL(2); break;                      \
        case 3: CALL(3); break;                      \
        case 4: CALL(4); break;                      \
        case 5: CALL(5); break;                      \
        case 6: CALL(6); break;                      \
        case 7: CALL(7); break;                      \
        case 8: CALL(8); break;                      \
        case 9: CALL(9); break;                      \
        case 10: CALL(10); break;                    \
        case 11: CALL(11); break;                    \
        case 12: CALL(12); break;                    \
        case 13: CALL(13); break;                    \
        case 14: CALL(14); break;                    \
        case 15: CALL(15); break;                    \
        case 16: CALL(16); break;                    \
        default: fail(HVOX_EUNSUPPORTED, "kernel width out of range"); \
    }

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

inline unsigned grid_stride_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

}  // namespace

// ------------------------------------------------------------------ host launchers

template <typename T>
void nufft_block_s2v(const DevBlock &b, int w, double beta, const T *c, const GridRec<T> *prec,
                     const cplx_t<T> *pph, const GridRec<T> *vrec, const cplx_t<T> *vq, const T *ipsi, cplx_t<T> *G1,
                     cplx_t<T> *G2, cufftHandle plan, int isign, cplx_t<T> *acc, cudaStream_t s, StageHook &hook) {
    const int64_t m1 = (int64_t)b.n1[0] * b.n1[1] * b.n1[2];
    hook.begin(HVOX_STAGE_ZERO);
    check_cuda(cudaMemsetAsync(G1, 0, sizeof(cplx_t<T>) * m1, s), "memset G1");
    hook.end(HVOX_STAGE_ZERO, 1);
    const T bt = (T)beta;
    if (b.np > 0) {
        hook.begin(HVOX_STAGE_SPREAD);
#define CALL(W) spread_pix_kernel<T, W><<<blocks_for(b.np, 128), 128, 0, s>>>(b, c, prec, pph, G1, bt)
        HVOX_W_SWITCH(w, CALL)
#undef CALL
        check_cuda(cudaGetLastError(), "spread_pix");
        hook.end(HVOX_STAGE_SPREAD, 1);
    }
    const int64_t m2 = (int64_t)b.n2[0] * b.n2[1] * b.n2[2];
    hook.begin(HVOX_STAGE_DECONV);
    deconv_pad_kernel<T><<<grid_stride_blocks(m2), 256, 0, s>>>(b, G1, ipsi, G2);
    check_cuda(cudaGetLastError(), "deconv_pad");
    hook.end(HVOX_STAGE_DECONV, 1);
    hook.begin(HVOX_STAGE_FFT);
    check_cufft(cufftSetStream(plan, s), "cufftSetStream");
    const int dir = isign < 0 ? CUFFT_FORWARD : CUFFT_INVERSE;
    if constexpr (sizeof(T) == 4)
        check_cufft(cufftExecC2C(plan, (cufftComplex *)G2, (cufftComplex *)G2, dir), "cufftExecC2C");
    else
        check_cufft(cufftExecZ2Z(plan, (cufftDoubleComplex *)G2, (cufftDoubleComplex *)G2, dir), "cufftExecZ2Z");
    hook.end(HVOX_STAGE_FFT, 1);
    if (b.nv > 0) {
        hook.begin(HVOX_STAGE_INTERP);
#define CALL(W) interp_vis_kernel<T, W><<<blocks_for(b.nv, 128), 128, 0, s>>>(b, G2, vrec, vq, acc, bt)
        HVOX_W_SWITCH(w, CALL)
#undef CALL
        check_cuda(cudaGetLastError(), "interp_vis");
        hook.end(HVOX_STAGE_INTERP, 1);
    }
}

template <typename T>
void nufft_block_v2s(const DevBlock &b, int w, double beta, const cplx_t<T> *V, const GridRec<T> *prec,
                     const cplx_t<T> *pph, const GridRec<T> *vrec, const cplx_t<T> *vq, const T *ipsi, cplx_t<T> *G1,
                     cplx_t<T> *G2, cufftHandle plan, int isign, T *acc, cudaStream_t s, StageHook &hook) {
    const int64_t m2 = (int64_t)b.n2[0] * b.n2[1] * b.n2[2];
    hook.begin(HVOX_STAGE_ZERO);
    check_cuda(cudaMemsetAsync(G2, 0, sizeof(cplx_t<T>) * m2, s), "memset G2");
    hook.end(HVOX_STAGE_ZERO, 1);
    const T bt = (T)beta;
    if (b.nv > 0) {
        hook.begin(HVOX_STAGE_SPREAD);
#define CALL(W) spread_vis_kernel<T, W><<<blocks_for(b.nv, 128), 128, 0, s>>>(b, V, vrec, vq, G2, bt)
        HVOX_W_SWITCH(w, CALL)
#undef CALL
        check_cuda(cudaGetLastError(), "spread_vis");
        hook.end(HVOX_STAGE_SPREAD, 1);
    }
    hook.begin(HVOX_STAGE_FFT);
    check_cufft(cufftSetStream(plan, s), "cufftSetStream");
    const int dir = isign < 0 ? CUFFT_INVERSE : CUFFT_FORWARD;  // transpose: opposite sign
    if constexpr (sizeof(T) == 4)
        check_cufft(cufftExecC2C(plan, (cufftComplex *)G2, (cufftComplex *)G2, dir), "cufftExecC2C");
    else
        check_cufft(cufftExecZ2Z(plan, (cufftDoubleComplex *)G2, (cufftDoubleComplex *)G2, dir), "cufftExecZ2Z");
    hook.end(HVOX_STAGE_FFT, 1);
    const int64_t m1 = (int64_t)b.n1[0] * b.n1[1] * b.n1[2];
    hook.begin(HVOX_STAGE_DECONV);
    crop_deconv_kernel<T><<<grid_stride_blocks(m1), 256, 0, s>>>(b, G2, ipsi, G1);
    check_cuda(cudaGetLastError(), "crop_deconv");
    hook.end(HVOX_STAGE_DECONV, 1);
    if (b.np > 0) {
        hook.begin(HVOX_STAGE_INTERP);
#define CALL(W) interp_pix_kernel<T, W><<<blocks_for(b.np, 128), 128, 0, s>>>(b, G1, prec, pph, acc, bt)
        HVOX_W_SWITCH(w, CALL)
#undef CALL
        check_cuda(cudaGetLastError(), "interp_pix");
        hook.end(HVOX_STAGE_INTERP, 1);
    }
}

template void nufft_block_s2v<float>(const DevBlock &, int, double, const float *, const GridRec<float> *,
                                     const float2 *, const GridRec<float> *, const float2 *, const float *, float2 *,
                                     float2 *, cufftHandle, int, float2 *, cudaStream_t, StageHook &);
template void nufft_block_s2v<double>(const DevBlock &, int, double, const double *, const GridRec<double> *,
                                      const double2 *, const GridRec<double> *, const double2 *, const double *,
                                      double2 *, double2 *, cufftHandle, int, double2 *, cudaStream_t, StageHook &);
template void nufft_block_v2s<float>(const DevBlock &, int, double, const float2 *, const GridRec<float> *,
                                     const float2 *, const GridRec<float> *, const float2 *, const float *, float2 *,
                                     float2 *, cufftHandle, int, float *, cudaStream_t, StageHook &);
template void nufft_block_v2s<double>(const DevBlock &, int, double, const double2 *, const GridRec<double> *,
                                      const double2 *, const GridRec<double> *, const double2 *, const double *,
                                      double2 *, double2 *, cufftHandle, int, double *, cudaStream_t, StageHook &);

template <typename T>
void nufft_tables(const NufftBlock &b, const double *pix_soa, int64_t n_pix, const double *vis_soa, int64_t n_vis,
                  int w, int isign, const double *qz, const double *qf, int nq, GridRec<T> *prec, cplx_t<T> *pph,
                  GridRec<T> *vrec, cplx_t<T> *vq, int *err, cudaStream_t s) {
    double3 C = make_double3(b.C[0], b.C[1], b.C[2]);
    double3 D = make_double3(b.D[0], b.D[1], b.D[2]);
    double3 a = make_double3(b.a[0], b.a[1], b.a[2]);
    int3 n1 = make_int3((int)b.n1[0], (int)b.n1[1], (int)b.n1[2]);
    int3 n2 = make_int3((int)b.n2[0], (int)b.n2[1], (int)b.n2[2]);
    int64_t np = b.p1 - b.p0, nv = b.v1 - b.v0;
    if (np > 0) {
        pix_tables_kernel<T><<<blocks_for(np, 256), 256, 0, s>>>(np, pix_soa, n_pix, b.p0, C, D, a, n1, w, isign,
                                                                   prec + b.prec_off, pph + b.prec_off, err);
        check_cuda(cudaGetLastError(), "pix_tables");
    }
    if (nv > 0) {
        vis_tables_kernel<T><<<blocks_for(nv, 128), 128, 0, s>>>(nv, vis_soa, n_vis, b.v0, C, D, a, n2, w, isign, qz,
                                                                   qf, nq, vrec + b.vrec_off, vq + b.vrec_off);
        check_cuda(cudaGetLastError(), "vis_tables");
    }
}

template void nufft_tables<float>(const NufftBlock &, const double *, int64_t, const double *, int64_t, int, int,
                                  const double *, const double *, int, GridRec<float> *, float2 *, GridRec<float> *,
                                  float2 *, int *, cudaStream_t);
template void nufft_tables<double>(const NufftBlock &, const double *, int64_t, const double *, int64_t, int, int,
                                   const double *, const double *, int, GridRec<double> *, double2 *,
                                   GridRec<double> *, double2 *, int *, cudaStream_t);

}  // namespace hvox
