// Batched FP32 stage with its dense local products on the tcgen05 tensor
// cores in split BF16 (HHO_BF16X3).  Included by stage.cu (uses its cell
// helpers, in its anonymous namespace).
//
// A block is 128 (cell, shot) rows: C = 32 consecutive cells of one class
// (class runs are padded to 32 cells, so they share a class and a domain)
// times 4 shots; thread t owns row t = (cell t % 32, shot t / 32), which is
// also tensor-memory lane t.  Per
// stage, with the class's operand tiles (tc_tiles in operators.cpp) staged
// in shared memory:
//   1. each row forms its exact derivative terms in registers and its face
//      jumps (own omega plus the neighbour's w, as the FP32 kernel does);
//   2. GEMM 1: the jumps of all faces (4 columns per face, split into BF16
//      hi + lo; one 8-byte store per face and tile) times the
//      n_F-weighted lifting matrices gives every face's lifted contribution
//      to every rate accumulator at once (three MMAs per K step: hi hi,
//      hi lo, lo hi, FP32 accumulation in tensor memory);
//   3. the rows add it (the tau-scaled blocks times tau), apply sources and
//      write the ERK targets (FP32, as the FP32 kernel);
//   4. GEMM 2: the new stage value's fields times the trace matrices gives
//      every face's traces of p and m.n (fluid) or v and s n (solid);
//   5. the rows publish w and omega per face.
// One elected thread issues the MMAs and commits them to an mbarrier that
// the block waits on (bounded; a wait that gives up sets the error flag).

struct TcArgs {
    const uint4* tiles;      // per-class operand tiles (meta[4] in 16-byte units)
    const int32_t* meta;     // [n_classes][6]: K1, N1, K2, N2, tile offset, tile bytes
    int C;                   // cells per block
    int S_blk;               // shots per block (128 / C)
    int n_shots;
    int kmax;                // width of the A tile in shared memory
    uint32_t cols;           // tensor-memory columns allocated per block
    int* error;              // set to 1 when an MMA wait gives up
};

constexpr int TC_WAIT_LIMIT = 1 << 22;

// Four consecutive columns k0..k0+3 (k0 a multiple of 4) of one row of the
// A tile, split into BF16 hi / lo: one 8-byte store per tile.
__device__ __forceinline__ void tc_put4(__nv_bfloat16* hi, __nv_bfloat16* lo, int row, int k0, int K, float a,
                                        float b, float c, float d) {
    __nv_bfloat16 h[4], l[4];
    tc::split_bf16(a, h[0], l[0]);
    tc::split_bf16(b, h[1], l[1]);
    tc::split_bf16(c, h[2], l[2]);
    tc::split_bf16(d, h[3], l[3]);
    const uint32_t o = tc::tile_off(row, k0, K);
    *reinterpret_cast<uint2*>(reinterpret_cast<char*>(hi) + o) = *reinterpret_cast<const uint2*>(h);
    *reinterpret_cast<uint2*>(reinterpret_cast<char*>(lo) + o) = *reinterpret_cast<const uint2*>(l);
}

// A row of the A tile: values[0..NV) at columns 0..NV, zeros up to K
// (inactive rows: zeros)
template <int NV>
__device__ __forceinline__ void tc_put_row(__nv_bfloat16* hi, __nv_bfloat16* lo, int row, int K, const float* v,
                                           bool active) {
    auto val = [&](int k) { return (active && k < NV) ? v[k] : 0.0f; };
#pragma unroll
    for (int k0 = 0; k0 < (NV + 3) / 4 * 4; k0 += 4) tc_put4(hi, lo, row, k0, K, val(k0), val(k0 + 1), val(k0 + 2), val(k0 + 3));
    for (int k0 = (NV + 3) / 4 * 4; k0 < K; k0 += 4) tc_put4(hi, lo, row, k0, K, 0.0f, 0.0f, 0.0f, 0.0f);
}

// the f <= 4 jump coefficients of one face at columns k0..k0+3
template <int F>
__device__ __forceinline__ void tc_put_jump(__nv_bfloat16* hi, __nv_bfloat16* lo, int row, int k0, int K,
                                            const float* j, bool active) {
    auto val = [&](int l) { return (active && l < F) ? j[l] : 0.0f; };
    tc_put4(hi, lo, row, k0, K, val(0), val(1), val(2), val(3));
}

// Block-wide: make the A tile visible to the tensor cores, issue D = A B
// (split BF16, K / 16 steps) from thread 0, wait for its completion.
__device__ __forceinline__ bool tc_gemm(uint32_t tmem, uint64_t* bar, uint32_t& phase, const __nv_bfloat16* Ahi,
                                        const __nv_bfloat16* Alo, const __nv_bfloat16* Bhi,
                                        const __nv_bfloat16* Blo, int K, int N) {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
        const uint32_t idesc = tc::idesc_bf16(128, N);
        const uint32_t sboA = (uint32_t)(K / 8) * 128, sboB = sboA;
        const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo), bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint32_t o = (uint32_t)ks * 256;
            const uint64_t dah = tc::smem_desc(ah + o, 128, sboA), dal = tc::smem_desc(al + o, 128, sboA);
            const uint64_t dbh = tc::smem_desc(bh + o, 128, sboB), dbl = tc::smem_desc(bl + o, 128, sboB);
            tc::mma_bf16(tmem, dah, dbh, idesc, ks > 0 ? 1u : 0u);
            tc::mma_bf16(tmem, dah, dbl, idesc, 1u);
            tc::mma_bf16(tmem, dal, dbh, idesc, 1u);
        }
        tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait(bar, phase & 1u, TC_WAIT_LIMIT);
    ++phase;
    tc::fence_after_sync();
    return ok;
}

template <int K, int MODE>
__global__ void __launch_bounds__(128) stage_tc_kernel(const StageArgsT<float> A, const TcArgs T) {
    constexpr int n = Dims<K>::n, f = Dims<K>::f;
    extern __shared__ __align__(1024) unsigned char tc_sm[];
    __shared__ uint64_t bar;
    __shared__ uint32_t taddr_s;
    const int t = threadIdx.x, warp = t >> 5;
    const DevOps& op = A.op;
    const int gq0 = blockIdx.x * T.C;
    const bool fluid = gq0 < op.Nf;
    const int q = (fluid ? gq0 : gq0 - op.Nf) + t % T.C;
    const int shot = blockIdx.y * T.S_blk + t / T.C;
    const int cls = __ldg(op.warp_class + (fluid ? 0 : op.n_warps_f) + (q >> 5));
    const int* ci = op.cls_int + cls * CI_STRIDE;
    const int32_t* mt = T.meta + 6 * cls;
    const int K1 = mt[0], N1 = mt[1], K2 = mt[2], N2 = mt[3];
    __nv_bfloat16* Ahi = reinterpret_cast<__nv_bfloat16*>(tc_sm);
    __nv_bfloat16* Alo = Ahi + 128 * T.kmax;
    uint4* Bs = reinterpret_cast<uint4*>(Alo + 128 * T.kmax);
    {
        const int nv = mt[5] / 16;
        const uint4* src = T.tiles + mt[4];
        for (int e = t; e < nv; e += 128) Bs[e] = __ldg(src + e);
    }
    const __nv_bfloat16* B1h = reinterpret_cast<const __nv_bfloat16*>(Bs);
    const __nv_bfloat16* B1l = B1h + N1 * K1;
    const __nv_bfloat16* B2h = B1l + N1 * K1;
    const __nv_bfloat16* B2l = B2h + N2 * K2;
    if (warp == 0) tc::tmem_alloc(&taddr_s, T.cols);
    if (t == 0) tc::mbar_init(&bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = taddr_s;
    const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    bool ok = true;

    CellCtx<float> c;
    c.q = q;
    c.lq = q - __ldg(ci + CI_START);
    const bool active = c.lq < __ldg(ci + CI_COUNT) && shot < T.n_shots;
    const int sh = active ? shot : 0;
    c.nF = __ldg(ci + CI_NF);
    c.npad = __ldg(ci + CI_NPAD);
    c.sbase = __ldg(ci + CI_SLOT);
    c.cd = OpData<float>::cls(op) + __ldg(ci + CI_DOFF) + Dims<K>::M0P;
    c.N = fluid ? op.Nf : op.Ns;
    c.SF = op.SF;
    c.SS = op.SS;
    c.tau = __ldg((fluid ? OpData<float>::scal_f(op) + SF_TAU * c.N : OpData<float>::scal_s(op) + SS_TAU * c.N) + q);
    const size_t toff = (size_t)sh * A.trace_stride;
    c.trf_in = A.tr_in + toff;
    c.trs_in = A.tr_in + toff + (size_t)2 * f * c.SF;
    c.trf_out = A.tr_out + toff;
    c.trs_out = A.tr_out + toff + (size_t)2 * f * c.SF;
    const size_t soff = (size_t)sh * A.state_stride + (fluid ? 0 : (size_t)3 * n * op.Nf);
    constexpr int NVMAX = 5 * n;
    float U[NVMAX];

    if constexpr (MODE == MODE_TRACES) {
        if (active) {
            if (fluid) load_state<3 * n>(A.inp + soff, c.N, q, 0, U);
            else load_state<5 * n>(A.inp + soff, c.N, q, 0, U);
        }
    } else {
        // 1. derivative terms and face jumps
        if (fluid) {
            float* kmx = U;
            float* kmy = U + n;
            float* kp = U + 2 * n;
            if (active) {
                float u[n];
                load_state<n>(A.inp + soff, c.N, q, 2 * n, u);
                ddx<float, K>(u, kmx);
                ddy<float, K>(u, kmy);
                load_state<n>(A.inp + soff, c.N, q, 0, u);
                ddx<float, K>(u, kp);
                load_state<n>(A.inp + soff, c.N, q, n, u);
                add_ddy<float, K>(u, kp);
            }
            for (int j = 0; j < c.nF; ++j) {
                float jm[f];
                if (active) fluid_face_jump<float, K>(A, c, j, jm);
                tc_put_jump<f>(Ahi, Alo, t, 4 * j, K1, jm, active);
            }
            for (int k0 = 4 * c.nF; k0 < K1; k0 += 4) tc_put4(Ahi, Alo, t, k0, K1, 0.0f, 0.0f, 0.0f, 0.0f);
        } else {
            float* exx = U;
            float* eyy = U + n;
            float* exy = U + 2 * n;
            float* kvx = U + 3 * n;
            float* kvy = U + 4 * n;
            if (active) {
                const float* inp = A.inp + soff;
                float u[n];
                load_state<n>(inp, c.N, q, 3 * n, u);
                ddx<float, K>(u, exx);
                ddy<float, K>(u, exy);
                load_state<n>(inp, c.N, q, 4 * n, u);
                ddy<float, K>(u, eyy);
                add_ddx<float, K>(u, exy);
                load_state<n>(inp, c.N, q, 0, u);
                ddx<float, K>(u, kvx);
                load_state<n>(inp, c.N, q, n, u);
                ddy<float, K>(u, kvy);
                load_state<n>(inp, c.N, q, 2 * n, u);
                add_ddy<float, K>(u, kvx);
                add_ddx<float, K>(u, kvy);
            }
            for (int j = 0; j < c.nF; ++j) {
                float jx[f], jy[f];
                if (active) solid_face_jump<float, K>(A, c, j, jx, jy);
                tc_put_jump<f>(Ahi, Alo, t, 4 * j, K1, jx, active);
                tc_put_jump<f>(Ahi, Alo, t, 4 * (c.nF + j), K1, jy, active);
            }
            for (int k0 = 8 * c.nF; k0 < K1; k0 += 4) tc_put4(Ahi, Alo, t, k0, K1, 0.0f, 0.0f, 0.0f, 0.0f);
        }
        // 2. all faces' lifted jumps: 16-column block b of D1 is accumulator block b
        ok = tc_gemm(tmem, &bar, phase, Ahi, Alo, B1h, B1l, K1, N1) && ok;
        const int nblk = fluid ? 3 : 5, ntau = fluid ? 2 : 3;   // blocks from ntau on are times tau
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            if (b < nblk) {   // block-uniform
                float d[16];
                tc::tmem_ld16(lane + (uint32_t)(b * 16), d);
                if (active) {
                    const float s = b >= ntau ? c.tau : 1.0f;
#pragma unroll
                    for (int i = 0; i < n; ++i) U[b * n + i] = fmaf(s, d[i], U[b * n + i]);
                }
            }
        }
        // 3. sources and ERK targets (as the FP32 kernel)
        if (active) {
            if (fluid) {
                float* kp = U + 2 * n;
                const float Am = __ldg(OpData<float>::scal_f(op) + SF_AM * c.N + q);
                const float Ap = __ldg(OpData<float>::scal_f(op) + SF_AP * c.N + q);
                for (int s = 0; s < A.n_src; ++s)
                    if (A.src_dom[s] == 0 && A.src_q[s] == q) {
                        const float w = src_value(A, s) / Ap;
                        const float* g = A.src_g + (size_t)s * 2 * n;
                        for (int i = 0; i < n; ++i) kp[i] = fmaf(w, g[i], kp[i]);
                    }
                if (A.shot_src_q && A.shot_src_dom[shot] == 0 && A.shot_src_q[shot] == q) {
                    const float w = shot_src_value(A) / Ap;
                    const float* g = A.shot_src_g + (size_t)shot * 2 * n;
                    for (int i = 0; i < n; ++i) kp[i] = fmaf(w, g[i], kp[i]);
                }
                const float sc[3] = {Am, Ap, 0.0f};
                write_targets<3 * n, FluidGroups<n>>(A, c.N, soff, q, U, sc);
            } else {
                float* exx = U;
                float* eyy = U + n;
                float* kvx = U + 3 * n;
                float* kvy = U + 4 * n;
                const float r = __ldg(OpData<float>::scal_s(op) + SS_R * c.N + q);
                for (int i = 0; i < n; ++i) {
                    const float a = exx[i], b = eyy[i];
                    exx[i] = fmaf(r, b, a);
                    eyy[i] = fmaf(r, a, b);
                }
                const float Av = __ldg(OpData<float>::scal_s(op) + SS_AV * c.N + q);
                for (int s = 0; s < A.n_src; ++s)
                    if (A.src_dom[s] == 1 && A.src_q[s] == q) {
                        const float w = src_value(A, s) / Av;
                        const float* g = A.src_g + (size_t)s * 2 * n;
                        for (int i = 0; i < n; ++i) {
                            kvx[i] = fmaf(w, g[i], kvx[i]);
                            kvy[i] = fmaf(w, g[n + i], kvy[i]);
                        }
                    }
                if (A.shot_src_q && A.shot_src_dom[shot] == 1 && A.shot_src_q[shot] == q) {
                    const float w = shot_src_value(A) / Av;
                    const float* g = A.shot_src_g + (size_t)shot * 2 * n;
                    for (int i = 0; i < n; ++i) {
                        kvx[i] = fmaf(w, g[i], kvx[i]);
                        kvy[i] = fmaf(w, g[n + i], kvy[i]);
                    }
                }
                const float sc[3] = {__ldg(OpData<float>::scal_s(op) + SS_C1 * c.N + q),
                                     __ldg(OpData<float>::scal_s(op) + SS_C3 * c.N + q), Av};
                write_targets<5 * n, SolidGroups<n>>(A, c.N, soff, q, U, sc);
            }
        }
    }
    // 4. traces of the stage value U: 16-column block F of D2 is face F
    if (fluid) tc_put_row<3 * n>(Ahi, Alo, t, K2, U, active);
    else tc_put_row<5 * n>(Ahi, Alo, t, K2, U, active);
    ok = tc_gemm(tmem, &bar, phase, Ahi, Alo, B2h, B2l, K2, N2) && ok;
    for (int j = 0; j < c.nF; ++j) {
        float d[16];
        tc::tmem_ld16(lane + (uint32_t)(j * 16), d);
        if (!active) continue;
        // 5. publish w = tau u|_F - (flux)|_F and omega = alpha w - u|_F
        const int slot = c.sbase + j * c.npad + c.lq;
        if (fluid) {
            const int nb = __ldg(op.nb_f + slot);
            const float al = (nb >= NB_BOUNDARY) ? __ldg(OpData<float>::beta_f(op) + slot)
                                                 : __ldg(OpData<float>::if_coef(op) + 6 * (-2 - nb));
#pragma unroll
            for (int l = 0; l < f; ++l) {
                const float w = fmaf(c.tau, d[l], -d[f + l]);
                c.trf_out[(size_t)l * c.SF + slot] = w;
                c.trf_out[(size_t)(f + l) * c.SF + slot] = fmaf(al, w, -d[l]);
            }
        } else {
            const int nb = __ldg(op.nb_s + slot);
            float* TWS = c.trs_out;
#pragma unroll
            for (int l = 0; l < f; ++l) {
                const float tvx = d[l], tvy = d[f + l], tsx = d[2 * f + l], tsy = d[3 * f + l];
                const float wx = fmaf(c.tau, tvx, -tsx), wy = fmaf(c.tau, tvy, -tsy);
                TWS[(size_t)l * c.SS + slot] = wx;
                TWS[(size_t)(f + l) * c.SS + slot] = wy;
                if (nb >= NB_BOUNDARY) {
                    const float be = __ldg(OpData<float>::beta_s(op) + slot);
                    TWS[(size_t)(2 * f + l) * c.SS + slot] = fmaf(be, wx, -tvx);
                    TWS[(size_t)(3 * f + l) * c.SS + slot] = fmaf(be, wy, -tvy);
                } else {
                    const float* co = OpData<float>::if_coef(op) + 6 * (-2 - nb);
                    TWS[(size_t)(2 * f + l) * c.SS + slot] = fmaf(__ldg(co), wx, fmaf(__ldg(co + 1), wy, -tvx));
                    TWS[(size_t)(3 * f + l) * c.SS + slot] = fmaf(__ldg(co + 2), wx, fmaf(__ldg(co + 3), wy, -tvy));
                }
            }
        }
    }
    if (!ok && t == 0) atomicExch(T.error, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, T.cols);
}
