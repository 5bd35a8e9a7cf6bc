// Device self-check of the double-float arithmetic (f2x.cuh) that the
// double-float stage kernels use: each double-word operation, and a Horner
// chain of multiply-adds like the square-face traces, applied on the GPU to
// pairs given by the caller.  The caller compares the results with exact
// arithmetic; the operations must stay within their published error bounds
// however the compiler schedules them.
#include <cuda_runtime.h>

#include "f2x.cuh"
#include "hho_internal.h"

namespace {

constexpr int F2X_CHECK_OUT = 6;   // results per item

// in: [n][3] pairs (x, y, z); out: [n][6] pairs:
//   x + y, x - y, x * y, x * y + z, x / y, ((x z + y) z + x) z + y
__global__ void f2x_check_kernel(int n, const float2* __restrict__ in, float2* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 a = in[3 * i], b = in[3 * i + 1], c = in[3 * i + 2];
    const f2x x(a.x, a.y), y(b.x, b.y), z(c.x, c.y);
    f2x r[F2X_CHECK_OUT];
    r[0] = x + y;
    r[1] = x - y;
    r[2] = x * y;
    r[3] = fma(x, y, z);
    r[4] = x / y;
    r[5] = fma(fma(fma(x, z, y), z, x), z, y);
    for (int k = 0; k < F2X_CHECK_OUT; ++k) out[F2X_CHECK_OUT * i + k] = make_float2(r[k].hi, r[k].lo);
}

}  // namespace

extern "C" int hho_f2x_check(int32_t n, const float* h_in, float* h_out) {
    if (n < 1 || !h_in || !h_out) {
        hho_set_error("hho_f2x_check: bad arguments (n >= 1, non-null buffers)");
        return HHO_EINVAL;
    }
    float2 *in = nullptr, *out = nullptr;
    int rc = HHO_OK;
    const size_t bin = sizeof(float2) * 3 * (size_t)n, bout = sizeof(float2) * F2X_CHECK_OUT * (size_t)n;
    if (cudaMalloc(&in, bin) != cudaSuccess || cudaMalloc(&out, bout) != cudaSuccess) {
        hho_set_error("hho_f2x_check: device allocation failed");
        rc = HHO_ENOMEM;
    }
    if (!rc && cudaMemcpy(in, h_in, bin, cudaMemcpyHostToDevice) != cudaSuccess) {
        hho_set_error("hho_f2x_check: upload failed");
        rc = HHO_ECUDA;
    }
    if (!rc) {
        f2x_check_kernel<<<(n + 127) / 128, 128>>>(n, in, out);
        if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(h_out, out, bout, cudaMemcpyDeviceToHost) != cudaSuccess) {
            hho_set_error("hho_f2x_check: kernel failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = HHO_ECUDA;
        }
    }
    cudaFree(in);
    cudaFree(out);
    return rc;
}
