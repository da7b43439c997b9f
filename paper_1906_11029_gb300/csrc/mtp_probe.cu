// Arithmetic-rate probes of the current GPU (roofline denominators that no library measures
// for us): FP32 and FP64 FMA loops, and warp-level tensor-core MMA loops (TF32 m16n8k8 and
// BF16 m16n8k16, FP32 accumulate).  Each kernel runs independent dependency chains per
// thread so the pipe, not latency, is the limit; the results are stored so nothing is
// optimised away.
#include <string>

#include <cuda_runtime.h>

#include "mtp_internal.h"

namespace mtp {

constexpr int kProbeIters = 4096;

template <typename T>
__global__ void probe_fma_kernel(T* out, T seed) {
    T a[8], b = seed * T(0.999), c = T(1e-3);
    for (int i = 0; i < 8; ++i) a[i] = seed + T(threadIdx.x + i);
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = a[i] * b + c;
    }
    T s = 0;
    for (int i = 0; i < 8; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_mma_tf32_kernel(float* out, unsigned seed) {
    float c[4][4] = {};
    const unsigned a0 = seed ^ threadIdx.x, a1 = a0 * 3u, a2 = a0 * 5u, a3 = a0 * 7u;
    const unsigned b0 = seed + threadIdx.x, b1 = b0 * 11u;
    for (int it = 0; it < kProbeIters / 4; ++it) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            asm volatile(
                "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(c[q][0]), "+f"(c[q][1]), "+f"(c[q][2]), "+f"(c[q][3])
                : "r"(a0 & 0x3f7fffffu), "r"(a1 & 0x3f7fffffu), "r"(a2 & 0x3f7fffffu), "r"(a3 & 0x3f7fffffu),
                  "r"(b0 & 0x3f7fffffu), "r"(b1 & 0x3f7fffffu));
    }
    float s = 0;
    for (int q = 0; q < 4; ++q)
        for (int i = 0; i < 4; ++i) s += c[q][i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_mma_bf16_kernel(float* out, unsigned seed) {
    float c[4][4] = {};
    const unsigned a0 = (seed ^ threadIdx.x) & 0x3f003f00u, a1 = a0 ^ 0x00100010u, a2 = a0 ^ 0x00200020u,
                   a3 = a0 ^ 0x00300030u;
    const unsigned b0 = (seed + threadIdx.x) & 0x3f003f00u, b1 = b0 ^ 0x00400040u;
    for (int it = 0; it < kProbeIters / 4; ++it) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(c[q][0]), "+f"(c[q][1]), "+f"(c[q][2]), "+f"(c[q][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    float s = 0;
    for (int q = 0; q < 4; ++q)
        for (int i = 0; i < 4; ++i) s += c[q][i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace mtp

using namespace mtp;

#define PROBE_TRY(call)                                                                              \
    do {                                                                                             \
        cudaError_t _e = (call);                                                                     \
        if (_e != cudaSuccess) return set_error(MTP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)

extern "C" int mtp_probe_rates(double* out_tflops, void* stream) {
    if (!out_tflops) return set_error(MTP_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int dev, nsm;
    PROBE_TRY(cudaGetDevice(&dev));
    PROBE_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = nsm * 8;
    void* buf = nullptr;
    PROBE_TRY(cudaMalloc(&buf, sizeof(double) * threads * blocks));
    cudaEvent_t e0, e1;
    PROBE_TRY(cudaEventCreate(&e0));
    PROBE_TRY(cudaEventCreate(&e1));
    const double nthreads = (double)threads * blocks;
    // flops per kernel: FMA loops 2 * 8 * iters per thread; MMA loops (iters/4)*4 MMAs per warp
    const double fl[4] = {2.0 * 8 * kProbeIters * nthreads, 2.0 * 8 * kProbeIters * nthreads,
                          (double)kProbeIters * (nthreads / 32) * 2048.0,
                          (double)kProbeIters * (nthreads / 32) * 4096.0};
    for (int k = 0; k < 4; ++k) {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {   // first repetition warms up
            PROBE_TRY(cudaEventRecord(e0, st));
            if (k == 0) probe_fma_kernel<float><<<blocks, threads, 0, st>>>((float*)buf, 1.0001f);
            if (k == 1) probe_fma_kernel<double><<<blocks, threads, 0, st>>>((double*)buf, 1.0001);
            if (k == 2) probe_mma_tf32_kernel<<<blocks, threads, 0, st>>>((float*)buf, 12345u);
            if (k == 3) probe_mma_bf16_kernel<<<blocks, threads, 0, st>>>((float*)buf, 12345u);
            PROBE_TRY(cudaGetLastError());
            PROBE_TRY(cudaEventRecord(e1, st));
            PROBE_TRY(cudaEventSynchronize(e1));
            float ms;
            PROBE_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0 && ms < best) best = ms;
        }
        out_tflops[k] = fl[k] / (best * 1e-3) / 1e12;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return MTP_OK;
}
