// FMA throughput probes: the denominators of the ALU rooflines (FP64 for the
// FP64 stage kernels; FP32 for the double-float and FP32 ones).  Eight
// independent FMA chains per thread, 8 blocks of 256 threads per SM.
#include <cuda_runtime.h>

__global__ void dfma_probe_kernel(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// Runs the probe `reps` times on the current device and returns the best
// rate in FP64 FMA lane-operations per second.  0 on success.
extern "C" int hho_probe_dfma_rate(int iters, int reps, double* fma_per_s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int blocks = sms * 8, threads = 256;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    int rc = 0;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        dfma_probe_kernel<<<blocks, threads>>>(out, iters, 1.0000001, 1e-9);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = 1; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double rate = (double)blocks * threads * iters * 8 / (ms * 1e-3);
        if (rate > best) best = rate;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *fma_per_s = best;
    return rc;
}

__global__ void ffma_probe_kernel(float* out, int iters, float a, float b) {
    float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
        x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// The same for FP32 FMAs: best rate in FP32 FMA lane-operations per second.
extern "C" int hho_probe_ffma_rate(int iters, int reps, double* fma_per_s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int blocks = sms * 8, threads = 256;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    int rc = 0;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        ffma_probe_kernel<<<blocks, threads>>>(out, iters, 1.0000001f, 1e-9f);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = 1; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double rate = (double)blocks * threads * iters * 8 / (ms * 1e-3);
        if (rate > best) best = rate;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *fma_per_s = best;
    return rc;
}

// FP64 tensor-core (DMMA) throughput: the only FP64 matrix instruction is the
// warp-wide mma.sync m8n8k4 (D = A B + C, 8x4 by 4x8, FP64 throughout; each
// thread holds one element of A and B and two of C/D).  tcgen05.mma has no
// FP64 kind.  Eight independent accumulator tiles per warp, 8 blocks of 256
// threads per SM, as the FMA probes.
__global__ void dmma_probe_kernel(double* out, int iters, double a0, double b0) {
    const double a = a0 + 1e-12 * threadIdx.x, b = b0;
    double c[8][2];
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = 0.0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c[j][0]), "+d"(c[j][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += c[j][0] + c[j][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best DMMA rate over `reps` runs, in FP64 multiply-add operations per second
// (one m8n8k4 is 256 of them), the unit of the FMA probes.  0 on success.
extern "C" int hho_probe_dmma_rate(int iters, int reps, double* fma_per_s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int blocks = sms * 8, threads = 256;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    int rc = 0;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        dmma_probe_kernel<<<blocks, threads>>>(out, iters, 1e-3, 1e-3);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = 1; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double warps = (double)blocks * threads / 32;
        const double rate = warps * iters * 8 * 256 / (ms * 1e-3);
        if (rate > best) best = rate;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *fma_per_s = best;
    return rc;
}

// DFMA and DMMA issued together: each thread runs the eight DFMA chains of
// dfma_probe_kernel and the eight mma.sync accumulators of dmma_probe_kernel
// in the same loop.  If the two use separate hardware the loop takes about as
// long as the slower half alone; if they share it, as long as both halves one
// after the other.
__global__ void mixed_probe_kernel(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    const double am = 1e-3 + 1e-12 * threadIdx.x, bm = 1e-3;
    double c[8][2];
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = 0.0;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c[j][0]), "+d"(c[j][1])
                         : "d"(am), "d"(bm));
    }
    double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += c[j][0] + c[j][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best time per loop iteration of the mixed probe over `reps` runs, in
// seconds, with the same launch as the other probes.  0 on success.
extern "C" int hho_probe_mixed_time(int iters, int reps, double* seconds_per_iter) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int blocks = sms * 8, threads = 256;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    int rc = 0;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        mixed_probe_kernel<<<blocks, threads>>>(out, iters, 1.0000001, 1e-9);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = 1; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double t = ms * 1e-3 / iters;
        if (t < best) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *seconds_per_iter = best;
    return rc;
}
