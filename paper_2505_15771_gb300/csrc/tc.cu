// Split-BF16 GEMM on the tcgen05 tensor cores: a self-check of the
// descriptors, the tensor-memory handling and the MMA/commit/wait protocol
// that the tensor-core stage products use (tc.cuh), on one 128-row tile.
#include <cuda_runtime.h>

#include <cstring>

#include "hho_internal.h"
#include "tc.cuh"

namespace {

// D[128][N] = A[128][K] B[K][N]: three products per K step (hi hi, hi lo,
// lo hi) accumulated in FP32 in tensor memory.  One CTA of 128 threads;
// thread t owns row t of A and of D.
__global__ void __launch_bounds__(128) tc_gemm_kernel(int K, int N, const float* __restrict__ A,
                                                      const float* __restrict__ B, float* __restrict__ D,
                                                      int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t bar;
    __shared__ uint32_t taddr_s;
    const int t = threadIdx.x, warp = t >> 5;
    __nv_bfloat16* Ahi = reinterpret_cast<__nv_bfloat16*>(sm);
    __nv_bfloat16* Alo = Ahi + 128 * K;
    __nv_bfloat16* Bhi = Alo + 128 * K;
    __nv_bfloat16* Blo = Bhi + N * K;
    for (int k = 0; k < K; ++k) {
        __nv_bfloat16 h, l;
        tc::split_bf16(A[t * K + k], h, l);
        Ahi[tc::tile_off(t, k, K) / 2] = h;
        Alo[tc::tile_off(t, k, K) / 2] = l;
    }
    for (int n = t; n < N; n += 128)
        for (int k = 0; k < K; ++k) {   // B stored transposed: row n of B^T
            __nv_bfloat16 h, l;
            tc::split_bf16(B[k * N + n], h, l);
            Bhi[tc::tile_off(n, k, K) / 2] = h;
            Blo[tc::tile_off(n, k, K) / 2] = l;
        }
    uint32_t ncols = 32;
    while (ncols < (uint32_t)N) ncols <<= 1;
    if (warp == 0) tc::tmem_alloc(&taddr_s, ncols);
    if (t == 0) tc::mbar_init(&bar, 1);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = taddr_s;
    if (t == 0) {
        const uint32_t idesc = tc::idesc_bf16(128, N);
        const uint32_t sbo = (uint32_t)(K / 8) * 128;
        const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo), bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint32_t off = (uint32_t)ks * 256;
            const uint64_t dah = tc::smem_desc(ah + off, 128, sbo), dal = tc::smem_desc(al + off, 128, sbo);
            const uint64_t dbh = tc::smem_desc(bh + off, 128, sbo), dbl = tc::smem_desc(bl + off, 128, sbo);
            tc::mma_bf16(tmem, dah, dbh, idesc, ks > 0 ? 1u : 0u);
            tc::mma_bf16(tmem, dah, dbl, idesc, 1u);
            tc::mma_bf16(tmem, dal, dbh, idesc, 1u);
        }
        tc::mma_commit(&bar);
    }
    const bool ok = tc::mbar_wait(&bar, 0, 1 << 22);
    tc::fence_after_sync();
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            for (int i = 0; i < 16; ++i) D[t * N + c0 + i] = v[i];
        }
    } else if (t == 0) {
        atomicExch(status, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

}  // namespace

extern "C" int hho_tc_gemm_check(int32_t K, int32_t N, const float* h_A, const float* h_B, float* h_D,
                                 int32_t* h_status) {
    if (!h_A || !h_B || !h_D || !h_status || K < 16 || K > 64 || K % 16 || N < 16 || N > 128 || N % 16) {
        hho_set_error("hho_tc_gemm_check: bad arguments (16 <= K <= 64, 16 <= N <= 128, multiples of 16)");
        return HHO_EINVAL;
    }
    float *A = nullptr, *B = nullptr, *D = nullptr;
    int* st = nullptr;
    const size_t smem = (size_t)2 * 2 * (128 + N) * K;
    int rc = HHO_OK;
    if (cudaMalloc(&A, sizeof(float) * 128 * K) != cudaSuccess || cudaMalloc(&B, sizeof(float) * K * N) != cudaSuccess ||
        cudaMalloc(&D, sizeof(float) * 128 * N) != cudaSuccess || cudaMalloc(&st, sizeof(int)) != cudaSuccess) {
        hho_set_error("hho_tc_gemm_check: device allocation failed");
        rc = HHO_ENOMEM;
    }
    if (!rc && (cudaMemcpy(A, h_A, sizeof(float) * 128 * K, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(B, h_B, sizeof(float) * K * N, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemset(st, 0, sizeof(int)) != cudaSuccess ||
                cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                    cudaSuccess)) {
        hho_set_error("hho_tc_gemm_check: set-up failed");
        rc = HHO_ECUDA;
    }
    if (!rc) {
        tc_gemm_kernel<<<1, 128, smem>>>(K, N, A, B, D, st);
        if (cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(h_D, D, sizeof(float) * 128 * N, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(h_status, st, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            hho_set_error("hho_tc_gemm_check: kernel failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = HHO_ECUDA;
        }
    }
    cudaFree(A);
    cudaFree(B);
    cudaFree(D);
    cudaFree(st);
    return rc;
}
