// Permutations between the caller's point order and the plan's chunk order (Sect. 4:
// inputs and outputs are reordered so that every sub-problem reads contiguous
// slices), with the tessellation weights a_n of Eq. 2 applied on the pixel side.
#include <cstdint>

#include "hvox_internal.h"

namespace hvox {

namespace {

template <typename TI, typename TO>
__global__ void s2v_in_kernel(const TI *__restrict__ I, const int32_t *__restrict__ perm, const double *__restrict__ w,
                              int64_t n, TO *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = (double)I[perm[i]];
    if (w) v *= w[i];
    out[i] = (TO)v;
}

template <typename C>
__global__ void scatter_complex_kernel(const C *__restrict__ acc, const int32_t *__restrict__ perm, int64_t n,
                                       C *__restrict__ V) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) V[perm[i]] = acc[i];
}

template <typename C>
__global__ void gather_complex_kernel(const C *__restrict__ V, const int32_t *__restrict__ perm, int64_t n,
                                      C *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = V[perm[i]];
}

template <typename T>
__global__ void v2s_out_kernel(const T *__restrict__ acc, const int32_t *__restrict__ perm,
                               const double *__restrict__ w, int64_t n, T *__restrict__ I) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = (double)acc[i];
    if (w) v *= w[i];
    I[perm[i]] = (T)v;
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

}  // namespace hvox
