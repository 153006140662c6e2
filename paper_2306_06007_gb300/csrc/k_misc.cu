// Permutations between the caller's point order and the plan's chunk order (Sect. 4:
// inputs and outputs are reordered so that every sub-problem reads contiguous
// slices), with the tessellation weights a_n of Eq. 2 applied on the pixel side. A null
// permutation means the caller's data is already in chunk order.
#include <cstdint>

#include "hvox_internal.h"

namespace hvox {

namespace {

template <typename TI, typename TO>
__global__ void s2v_in_kernel(const TI *__restrict__ I, const int32_t *__restrict__ perm, const double *__restrict__ w,
                              int64_t n, TO *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = (double)I[perm ? perm[i] : i];
    if (w) v *= w[i];
    out[i] = (TO)v;
}

template <typename C>
__global__ void scatter_complex_kernel(const C *__restrict__ acc, const int32_t *__restrict__ perm, int64_t n,
                                       C *__restrict__ V) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) V[perm ? perm[i] : i] = acc[i];
}

template <typename C>
__global__ void gather_complex_kernel(const C *__restrict__ V, const int32_t *__restrict__ perm, int64_t n,
                                      C *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = V[perm ? perm[i] : i];
}

template <typename T>
__global__ void v2s_out_kernel(const T *__restrict__ acc, const int32_t *__restrict__ perm,
                               const double *__restrict__ w, int64_t n, T *__restrict__ I) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = (double)acc[i];
    if (w) v *= w[i];
    I[perm ? perm[i] : i] = (T)v;
}

// Complex sky <-> two real skies, and the complex combinations that give a complex-sky
// transform from two real ones (linearity): A (x + j y) = A x + j A y and
// A^H v = Re(A^H v) + j Re(A^H (-j v)).
template <typename T, typename C>
__global__ void split_complex_kernel(const C *__restrict__ z, int64_t n, T *__restrict__ re, T *__restrict__ im) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const C v = z[i];
    re[i] = v.x;
    im[i] = v.y;
}

template <typename T, typename C>
__global__ void join_complex_kernel(const T *__restrict__ re, const T *__restrict__ im, int64_t n, C *__restrict__ z) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    C v;
    v.x = re[i];
    v.y = im[i];
    z[i] = v;
}

template <typename C> __global__ void add_j_kernel(C *__restrict__ a, const C *__restrict__ b, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const C u = a[i], v = b[i];
    C r;
    r.x = u.x - v.y;
    r.y = u.y + v.x;
    a[i] = r;
}

template <typename C> __global__ void times_mj_kernel(const C *__restrict__ a, int64_t n, C *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const C u = a[i];
    C r;
    r.x = u.y;
    r.y = -u.x;
    out[i] = r;
}

inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

void launch_s2v_in(int prec, const void *I, const int32_t *perm, const double *w, int64_t n, void *src,
                   cudaStream_t s) {
    if (prec == 1)
        s2v_in_kernel<float, float><<<nb(n), 256, 0, s>>>((const float *)I, perm, w, n, (float *)src);
    else
        s2v_in_kernel<double, double><<<nb(n), 256, 0, s>>>((const double *)I, perm, w, n, (double *)src);
    check_cuda(cudaGetLastError(), "s2v_in");
}

void launch_s2v_out(int prec, const void *acc, const int32_t *perm, int64_t n, void *V, cudaStream_t s) {
    if (prec == 1)
        scatter_complex_kernel<float2><<<nb(n), 256, 0, s>>>((const float2 *)acc, perm, n, (float2 *)V);
    else
        scatter_complex_kernel<double2><<<nb(n), 256, 0, s>>>((const double2 *)acc, perm, n, (double2 *)V);
    check_cuda(cudaGetLastError(), "s2v_out");
}

void launch_v2s_in(int prec, const void *V, const int32_t *perm, int64_t n, void *src, cudaStream_t s) {
    if (prec == 1)
        gather_complex_kernel<float2><<<nb(n), 256, 0, s>>>((const float2 *)V, perm, n, (float2 *)src);
    else
        gather_complex_kernel<double2><<<nb(n), 256, 0, s>>>((const double2 *)V, perm, n, (double2 *)src);
    check_cuda(cudaGetLastError(), "v2s_in");
}

void launch_v2s_out(int prec, const void *acc, const int32_t *perm, const double *w, int64_t n, void *I,
                    cudaStream_t s) {
    if (prec == 1)
        v2s_out_kernel<float><<<nb(n), 256, 0, s>>>((const float *)acc, perm, w, n, (float *)I);
    else
        v2s_out_kernel<double><<<nb(n), 256, 0, s>>>((const double *)acc, perm, w, n, (double *)I);
    check_cuda(cudaGetLastError(), "v2s_out");
}

void launch_split_complex(int prec, const void *z, int64_t n, void *re, void *im, cudaStream_t s) {
    if (prec == 1)
        split_complex_kernel<float, float2><<<nb(n), 256, 0, s>>>((const float2 *)z, n, (float *)re, (float *)im);
    else
        split_complex_kernel<double, double2><<<nb(n), 256, 0, s>>>((const double2 *)z, n, (double *)re, (double *)im);
    check_cuda(cudaGetLastError(), "split_complex");
}

void launch_join_complex(int prec, const void *re, const void *im, int64_t n, void *z, cudaStream_t s) {
    if (prec == 1)
        join_complex_kernel<float, float2><<<nb(n), 256, 0, s>>>((const float *)re, (const float *)im, n, (float2 *)z);
    else
        join_complex_kernel<double, double2><<<nb(n), 256, 0, s>>>((const double *)re, (const double *)im, n,
                                                                    (double2 *)z);
    check_cuda(cudaGetLastError(), "join_complex");
}

void launch_add_j(int prec, void *a, const void *b, int64_t n, cudaStream_t s) {
    if (prec == 1)
        add_j_kernel<float2><<<nb(n), 256, 0, s>>>((float2 *)a, (const float2 *)b, n);
    else
        add_j_kernel<double2><<<nb(n), 256, 0, s>>>((double2 *)a, (const double2 *)b, n);
    check_cuda(cudaGetLastError(), "add_j");
}

void launch_times_mj(int prec, const void *a, int64_t n, void *out, cudaStream_t s) {
    if (prec == 1)
        times_mj_kernel<float2><<<nb(n), 256, 0, s>>>((const float2 *)a, n, (float2 *)out);
    else
        times_mj_kernel<double2><<<nb(n), 256, 0, s>>>((const double2 *)a, n, (double2 *)out);
    check_cuda(cudaGetLastError(), "times_mj");
}

}  // namespace hvox
