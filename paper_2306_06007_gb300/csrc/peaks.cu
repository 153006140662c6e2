// Throughput probes for the roofline denominators that the driver's measured peaks do not
// cover (they hold HBM copy bandwidth and dense bf16 only): FP32 and FP64 FMA issue, float
// atomicAdd into shared memory (the pipe the spreading kernels are bound by) and L1 load
// bandwidth (the interpolation kernels' gathers). Built as its own library
// (libhvox_peaks.so) for the benchmark; nothing in libhvox.so uses it.
//
// Every kernel runs a fixed number of iterations over registers or a small, fixed
// buffer: no waits, every index inside its buffer.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kChains = 8;

template <typename T> __global__ void fma_kernel(T *out, int iters, T a, T b) {
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == (T)-1.2345) out[blockIdx.x] = s;  // never true for these inputs; keeps the loop
}

// Each warp adds into its own 32 x 8 floats; lane j always hits bank j (no conflicts).
constexpr int kAtomThreads = 512;
__global__ void __launch_bounds__(kAtomThreads) shared_atomic_kernel(float *out, int iters) {
    __shared__ float buf[kAtomThreads / 32][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kAtomThreads / 32) * 256; i += blockDim.x) (&buf[0][0])[i] = 0.f;
    __syncthreads();
    for (int i = 0; i < iters; ++i) atomicAdd(&buf[warp][((i & 7) << 5) + lane], 1.0f);
    __syncthreads();
    if (threadIdx.x == 0 && buf[0][0] == -1.0f) out[blockIdx.x] = buf[0][1];
}

// The same pattern with 32-bit integer atomics, and with a plain read-modify-write of
// lane-private words (load, add, store; no atomic): the alternatives a spreading kernel
// could use for its shared tile.
__global__ void __launch_bounds__(kAtomThreads) shared_int_atomic_kernel(float *out, int iters) {
    __shared__ int buf[kAtomThreads / 32][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kAtomThreads / 32) * 256; i += blockDim.x) (&buf[0][0])[i] = 0;
    __syncthreads();
    for (int i = 0; i < iters; ++i) atomicAdd(&buf[warp][((i & 7) << 5) + lane], 3);
    __syncthreads();
    if (threadIdx.x == 0 && buf[0][0] == -1) out[blockIdx.x] = (float)buf[0][1];
}

__global__ void __launch_bounds__(kAtomThreads) shared_rmw_kernel(float *out, int iters) {
    __shared__ float buf[kAtomThreads / 32][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kAtomThreads / 32) * 256; i += blockDim.x) (&buf[0][0])[i] = 0.f;
    __syncthreads();
    volatile float *b = &buf[warp][0];
    for (int i = 0; i < iters; ++i) {
        const int k = ((i & 7) << 5) + lane;  // lane-private words: no two lanes share one
        b[k] = b[k] + 1.0f;
    }
    __syncthreads();
    if (threadIdx.x == 0 && buf[0][0] == -1.0f) out[blockIdx.x] = buf[0][1];
}

// Every CTA reads the same 16 KiB (float2, lane-consecutive), which stays in each SM's L1.
constexpr int kL1Elems = 2048;
__global__ void l1_load_kernel(const float2 *__restrict__ src, float *out, int iters) {
    float sx = 0.f, sy = 0.f;
    int j = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
        const float2 v = src[j];
        sx += v.x;
        sy += v.y;
        j += blockDim.x;
        j &= kL1Elems - 1;
    }
    if (sx + sy == -1.0f) out[blockIdx.x] = sx;
}

template <typename F> double time_ms(F &&launch) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch();  // warm-up
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

}  // namespace

// out[0] FP32 FMA flop/s, out[1] FP64 FMA flop/s, out[2] shared-memory float atomicAdd/s,
// out[3] L1 load bytes/s, out[4] shared-memory int atomicAdd/s, out[5] shared-memory
// float read-modify-writes/s (no atomic). Returns 0, or the CUDA error code of the first
// failing call.
extern "C" int hvox_probe_peaks(double *out) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float *sink = nullptr;
    float2 *src = nullptr;
    double *dsink = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * 65536) != cudaSuccess) return (int)cudaGetLastError();
    if (cudaMalloc(&dsink, sizeof(double) * 65536) != cudaSuccess) return (int)cudaGetLastError();
    if (cudaMalloc(&src, sizeof(float2) * kL1Elems) != cudaSuccess) return (int)cudaGetLastError();
    cudaMemset(src, 0, sizeof(float2) * kL1Elems);
    const unsigned blocks = (unsigned)sms * 8;  // 8 x 256 threads per SM: full occupancy
    {
        const int iters = 1 << 16;
        double ms = time_ms([&] { fma_kernel<float><<<blocks, 256>>>(sink, iters, 0.999f, 1e-3f); });
        out[0] = 2.0 * kChains * (double)iters * blocks * 256 / (ms * 1e-3);
    }
    {
        const int iters = 1 << 9;
        double ms = time_ms([&] { fma_kernel<double><<<blocks, 256>>>(dsink, iters, 0.999, 1e-3); });
        out[1] = 2.0 * kChains * (double)iters * blocks * 256 / (ms * 1e-3);
    }
    {
        const int iters = 1 << 15;
        const unsigned ab = (unsigned)sms * 4;  // 4 x 512 threads per SM
        double ms = time_ms([&] { shared_atomic_kernel<<<ab, kAtomThreads>>>(sink, iters); });
        out[2] = (double)iters * ab * kAtomThreads / (ms * 1e-3);
    }
    {
        const int iters = 1 << 15;
        double ms = time_ms([&] { l1_load_kernel<<<blocks, 256>>>(src, sink, iters); });
        out[3] = 8.0 * (double)iters * blocks * 256 / (ms * 1e-3);
    }
    {
        const int iters = 1 << 15;
        const unsigned ab = (unsigned)sms * 4;
        double ms = time_ms([&] { shared_int_atomic_kernel<<<ab, kAtomThreads>>>(sink, iters); });
        out[4] = (double)iters * ab * kAtomThreads / (ms * 1e-3);
        ms = time_ms([&] { shared_rmw_kernel<<<ab, kAtomThreads>>>(sink, iters); });
        out[5] = (double)iters * ab * kAtomThreads / (ms * 1e-3);
    }
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(sink);
    cudaFree(dsink);
    cudaFree(src);
    return (int)e;
}
