// ERK stage kernels for GB300 (sm_103a) and the time-stepping entry points.
//
// One stage of Eq. ex_solve (Sec. 4.2) is ONE kernel.  Thread q owns cell q of
// its domain (cells sorted by class, so a warp shares one class and its class
// matrices are read with warp-uniform loads).  The face unknowns are never
// stored: every cell publishes, per local face, two small vectors in the face
// basis psi_l = (rho0 xi)^l (xi along the face in the cell's own
// counter-clockwise orientation; operators.cpp):
//     w     = tau u_T|_F - (dual flux of T on F)      (what the neighbour needs)
//     omega = alpha w - u_T|_F                         (what the cell itself needs)
// where u is p (fluid) or v (solid) and the dual flux is m.n_T or s n_T.  The
// face solve of Eq. ex_solve is block-diagonal; its closed form per
// coefficient is
//     interior:  u_F = (w_T + w_N) / (tau_T + tau_N)
//     boundary:  u_F = 0
//     interface: [p_F; v_F] = A^-1 [w_f; w_s],  A = [tau_f, n^T; -n, tau_s I]
// (rows of the face block of the compact system, Eq. compact_AR, divided by
// the face mass matrix).  So the jump u_F - u_T|_F a cell needs is
// omega + beta * flip(w_N), flip = (-1)^l because the neighbour traverses
// the face in the opposite direction.
//
// A stage thread then: reads its state; forms the exact derivatives of its
// polynomials (sparse, compile-time); lifts each face jump with the class
// matrix Lift_F; scales by the per-cell material factors (inverse mass,
// Eq. mass, folded in); adds point sources; writes the ERK partial sums
// (Eq. ERK_compact with a_{s+1,j} = b_j); and publishes w, omega of the new
// stage value for the next stage (double-buffered traces).
//
// The kernels are templated on the arithmetic: FP64; double-float pairs on
// the FP32 pipes (f2x.cuh, FP64-class accuracy, the single-shot default of
// the benchmark); FP32 for batched shots (shots on blockIdx.y).  Their
// launch parameters (resident blocks, accumulator placement, prefetch hints)
// come from the table in stage_tuning.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "f2x.cuh"
#include "tc.cuh"
#include "hho_internal.h"
#include "stage_tuning.h"

namespace {

__host__ __device__ constexpr int deg_of(int i) {
    int d = 0;
    while ((d + 1) * (d + 2) / 2 <= i) ++d;
    return d;
}
__host__ __device__ constexpr int ea(int i) { return deg_of(i) - (i - deg_of(i) * (deg_of(i) + 1) / 2); }
__host__ __device__ constexpr int eb(int i) { return i - deg_of(i) * (deg_of(i) + 1) / 2; }
__host__ __device__ constexpr int eidx(int a, int b) { return (a + b) * (a + b + 1) / 2 + b; }

template <int K>
struct Dims {
    static constexpr int n = (K + 1) * (K + 2) / 2;
    static constexpr int f = K + 1;
    static constexpr int nP = (n + 3) / 4 * 4;            // padded row lengths (16-byte rows)
    static constexpr int fP = (f + 3) / 4 * 4;
    static constexpr int M0P = (n * n + 3) / 4 * 4;       // class mass block, padded
    static constexpr int FS = 4 + f * nP + n * fP;        // per-face stride: [nx ny 0 0 | Tr | Lift]
    static constexpr int TR = 4;                          // offset of Tr in a face block
    static constexpr int LI = 4 + f * nP;                 // offset of Lift
};

// 16-byte vector loads of class-matrix rows (two doubles or four floats).
template <class T>
struct Vec16;
template <>
struct Vec16<double> {
    static constexpr int w = 2;
    __device__ static void load(const double* p, double* o) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = v.x;
        o[1] = v.y;
    }
};
template <>
struct Vec16<float> {
    static constexpr int w = 4;
    __device__ static void load(const float* p, float* o) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
};

template <>
struct Vec16<f2x> {
    static constexpr int w = 2;
    __device__ static void load(const f2x* p, f2x* o) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = f2x(v.x, v.y);
        o[1] = f2x(v.z, v.w);
    }
};

// Operator data in the arithmetic type T (FP64, its FP32 copy, or its
// double-float copy).
template <class T>
struct OpData;
template <>
struct OpData<double> {
    __device__ static const double* cls(const DevOps& o) { return o.cls_dbl; }
    __device__ static const double* scal_f(const DevOps& o) { return o.scal_f; }
    __device__ static const double* scal_s(const DevOps& o) { return o.scal_s; }
    __device__ static const double* beta_f(const DevOps& o) { return o.beta_f; }
    __device__ static const double* beta_s(const DevOps& o) { return o.beta_s; }
    __device__ static const double* if_coef(const DevOps& o) { return o.if_coef; }
};
template <>
struct OpData<float> {
    __device__ static const float* cls(const DevOps& o) { return o.cls_f32; }
    __device__ static const float* scal_f(const DevOps& o) { return o.scal_f_f32; }
    __device__ static const float* scal_s(const DevOps& o) { return o.scal_s_f32; }
    __device__ static const float* beta_f(const DevOps& o) { return o.beta_f_f32; }
    __device__ static const float* beta_s(const DevOps& o) { return o.beta_s_f32; }
    __device__ static const float* if_coef(const DevOps& o) { return o.if_coef_f32; }
};

template <>
struct OpData<f2x> {
    __device__ static const f2x* cls(const DevOps& o) { return o.cls_x; }
    __device__ static const f2x* scal_f(const DevOps& o) { return o.scal_f_x; }
    __device__ static const f2x* scal_s(const DevOps& o) { return o.scal_s_x; }
    __device__ static const f2x* beta_f(const DevOps& o) { return o.beta_f_x; }
    __device__ static const f2x* beta_s(const DevOps& o) { return o.beta_s_x; }
    __device__ static const f2x* if_coef(const DevOps& o) { return o.if_coef_x; }
};

// d/dX of a polynomial in the scaled-monomial basis (exact, compile-time sparse).
template <class T, int K>
__device__ __forceinline__ void ddx(const T* u, T* out) {
#pragma unroll
    for (int i = 0; i < Dims<K>::n; ++i) {
        const int a = ea(i), b = eb(i);
        if (a + 1 + b <= K) {
            const int s = eidx(a + 1, b);
            out[i] = (a == 0) ? u[s] : mulc(float(a + 1), u[s]);
        } else {
            out[i] = T(0);
        }
    }
}
template <class T, int K>
__device__ __forceinline__ void ddy(const T* u, T* out) {
#pragma unroll
    for (int i = 0; i < Dims<K>::n; ++i) {
        const int a = ea(i), b = eb(i);
        if (a + b + 1 <= K) {
            const int s = eidx(a, b + 1);
            out[i] = (b == 0) ? u[s] : mulc(float(b + 1), u[s]);
        } else {
            out[i] = T(0);
        }
    }
}
// out += d/dX u  (or d/dY u)
template <class T, int K>
__device__ __forceinline__ void add_ddx(const T* u, T* out) {
#pragma unroll
    for (int i = 0; i < Dims<K>::n; ++i) {
        const int a = ea(i), b = eb(i);
        if (a + 1 + b <= K) {
            const int s = eidx(a + 1, b);
            out[i] = (a == 0) ? out[i] + u[s] : fmac(float(a + 1), u[s], out[i]);
        }
    }
}
template <class T, int K>
__device__ __forceinline__ void add_ddy(const T* u, T* out) {
#pragma unroll
    for (int i = 0; i < Dims<K>::n; ++i) {
        const int a = ea(i), b = eb(i);
        if (a + b + 1 <= K) {
            const int s = eidx(a, b + 1);
            out[i] = (b == 0) ? out[i] + u[s] : fmac(float(b + 1), u[s], out[i]);
        }
    }
}

// ---- face policies ---------------------------------------------------------------
// GenericFace: any polygon face; normals and class matrices read at run time,
// every matrix entry used (no run-time tests on floating-point values).
// RectAxis<A>: the faces of an axis-aligned rectangle with one orientation,
// A = 0 horizontal (faces 0 bottom and 2 top, normal (0, s)), A = 1 vertical
// (faces 1 right and 3 left, normal (s, 0)); the sign s = +-1 is a run-time
// argument, the parity sparsity of Tr and Lift is compile-time and entries
// outside the pattern are never loaded.  One body per orientation, looped
// over its two faces, keeps the kernel's instruction footprint small.
// SquareAxis<A>: the faces of a square cell; their traces are Horner sums
// with compile-time coefficients (trace_square) and Tr is never read, and
// their lifting matrices also vanish where the exponent along the face
// exceeds the face coefficient's degree by 2 (checked when the class is
// built, up to k = 3).
struct GenericFace {
    static constexpr bool rect = false;
    static constexpr bool square = false;
    static constexpr bool horiz = false;
    __host__ __device__ static constexpr bool tr_nz(int, int) { return true; }
    __host__ __device__ static constexpr bool lift_nz(int, int) { return true; }
};
template <int AX>
struct RectAxis {
    static constexpr bool rect = true;
    static constexpr bool square = false;
    static constexpr bool horiz = AX == 0;
    __host__ __device__ static constexpr int e(int i) { return horiz ? ea(i) : eb(i); }
    __host__ __device__ static constexpr bool tr_nz(int l, int i) { return e(i) == l; }
    __host__ __device__ static constexpr bool lift_nz(int i, int l) { return ((e(i) + l) % 2) == 0; }
};
template <int AX>
struct SquareAxis : RectAxis<AX> {
    static constexpr bool square = true;
    __host__ __device__ static constexpr bool lift_nz(int i, int l) {
        return RectAxis<AX>::lift_nz(i, l) && RectAxis<AX>::e(i) - l != 2;
    }
};

// Class matrices of the double-float kernel are read from a per-warp copy in
// shared memory (its many FP32 instructions per matrix entry would otherwise
// wait on L1 misses: the streamed state and traces evict the class rows); the
// FP64 and FP32 kernels read them through the read-only data path.
template <class T>
struct ClsSmem {
    static constexpr bool value = false;
};
template <>
struct ClsSmem<f2x> {
    static constexpr bool value = true;
};
template <class T>
__device__ __forceinline__ void cls_row(const T* p, T* o) {
    if constexpr (ClsSmem<T>::value) {
        const float4 v = *reinterpret_cast<const float4*>(p);   // two pairs
        o[0] = T(v.x, v.y);
        o[1] = T(v.z, v.w);
    } else {
        Vec16<T>::load(p, o);
    }
}
template <class T>
__device__ __forceinline__ T cls_val(const T* p) {
    if constexpr (ClsSmem<T>::value) return *p;
    else return __ldg(p);
}

// y[l] = sum_i Tr[l][i] x[i] over the policy's pattern.  Each row is read in
// 16-byte chunks; a chunk with no entry in the pattern is not loaded.
template <class T, int K, class P>
__device__ __forceinline__ void trace_apply(const T* __restrict__ Tr, const T* x, T* y) {
    constexpr int n = Dims<K>::n, f = Dims<K>::f, nP = Dims<K>::nP, w = Vec16<T>::w;
#pragma unroll
    for (int l = 0; l < f; ++l) {
        T row[nP];
#pragma unroll
        for (int c0 = 0; c0 < nP; c0 += w) {
            bool need = false;
#pragma unroll
            for (int e = 0; e < w; ++e) need = need || (c0 + e < n && P::tr_nz(l, c0 + e));
            if (need) cls_row<T>(Tr + l * nP + c0, row + c0);
        }
        T acc = T(0);
#pragma unroll
        for (int i = 0; i < n; ++i)
            if (P::tr_nz(l, i)) acc = fma(row[i], x[i], acc);
        y[l] = acc;
    }
}
// Traces on a square's face with outward normal sign sg (faces 0 and 3:
// -1, faces 1 and 2: +1): the monomial with exponent l along the face and m
// across it traces to s_t^l (sg rho0)^m psi_l, s_t = -sg on horizontal and
// sg on vertical faces, so y[l] = s_t^l sum_m (sg rho0)^m x[(l, m)] by
// Horner's rule (K - l multiply-adds).
// sg * rho0 in T; the double-float split is formed at compile time (a
// run-time split would issue FP64 instructions on the slow FP64 pipe)
template <class T>
__device__ __forceinline__ T signed_face_rho(int sg) {
    return T(sg > 0 ? FACE_RHO : -FACE_RHO);
}
template <>
__device__ __forceinline__ f2x signed_face_rho<f2x>(int sg) {
    constexpr float hi = (float)FACE_RHO;
    constexpr float lo = (float)(FACE_RHO - (double)hi);
    return sg > 0 ? f2x(hi, lo) : f2x(-hi, -lo);
}
template <class T, int K, bool HORIZ>
__device__ __forceinline__ void trace_square(const T* x, T* y, int sg) {
    const T c = signed_face_rho<T>(sg);
    const bool flip = HORIZ ? sg > 0 : sg < 0;   // s_t = -1
#pragma unroll
    for (int l = 0; l <= K; ++l) {
        T acc = x[HORIZ ? eidx(l, K - l) : eidx(K - l, l)];
#pragma unroll
        for (int m = K - l - 1; m >= 0; --m) acc = fma(c, acc, x[HORIZ ? eidx(l, m) : eidx(m, l)]);
        y[l] = ((l & 1) && flip) ? -acc : acc;
    }
}
template <class T, int K, class P>
__device__ __forceinline__ void face_trace_apply(const T* __restrict__ Tr, const T* x, T* y, int sg) {
    if constexpr (P::square) trace_square<T, K, P::horiz>(x, y, sg);
    else trace_apply<T, K, P>(Tr, x, y);
}
// y[i] = sum_l L[i][l] j[l] over the policy's pattern (rows of fP entries).
template <class T, int K, class P>
__device__ __forceinline__ void lift_apply(const T* __restrict__ L, const T* j, T* y) {
    constexpr int n = Dims<K>::n, f = Dims<K>::f, fP = Dims<K>::fP, w = Vec16<T>::w;
#pragma unroll
    for (int i = 0; i < n; ++i) {
        T row[fP];
#pragma unroll
        for (int c0 = 0; c0 < fP; c0 += w) {
            bool need = false;
#pragma unroll
            for (int e = 0; e < w; ++e) need = need || (c0 + e < f && P::lift_nz(i, c0 + e));
            if (need) cls_row<T>(L + i * fP + c0, row + c0);
        }
        T acc = T(0);
#pragma unroll
        for (int l = 0; l < f; ++l)
            if (P::lift_nz(i, l)) acc = fma(row[l], j[l], acc);
        y[i] = acc;
    }
}
// Rectangle faces: one body per orientation looped over its two faces
// (compact code: the double-float kernel is bound by instruction fetch
// otherwise), or the four faces unrolled with constant signs (the FP64
// kernel schedules better fully unrolled); per arithmetic and k from the
// tuning table.

// Where a stage thread keeps its 3n (fluid) or 5n (solid) accumulators.  In
// registers they do not fit the 64-register budget of 8 resident blocks and
// spill to local memory, whose footprint (over 400 bytes a thread) exceeds
// L1.  With AccSmem the block's dynamic shared memory holds them instead,
// thread-major with an odd stride in elements (no bank conflicts).  That
// makes the FP32 kernel about 20 % faster at k = 3 (still 8 blocks).  For
// 8-byte values the shared memory allows at most 6 blocks: the double-float
// k = 2 kernel at 5 blocks (96 registers, no spills) with prefetched target
// sources is 7 % faster than with 8 blocks and spills; the FP64 kernel, bound
// by its FP64 pipe, and double-float k = 3 (4 blocks) gain nothing.
template <class T>
struct Tuned;
template <>
struct Tuned<double> {
    static constexpr StageTuning t = TUNED_F64;
};
template <>
struct Tuned<float> {
    static constexpr StageTuning t = TUNED_F32;
};
template <>
struct Tuned<f2x> {
    static constexpr StageTuning t = TUNED_F2X;
};
template <class T, int K>
struct RectLoop {
    static constexpr bool value = Tuned<T>::t.rect_loop[K - 1] != 0;
};
template <class T, int K>
struct AccSmem {
    static constexpr bool value = Tuned<T>::t.acc_smem[K - 1] != 0;
};
template <int K>
__host__ __device__ constexpr int acc_stride() {
    return (5 * Dims<K>::n) | 1;
}

// y += s * x for a run-time sign s = +-1
template <int NN, class T>
__device__ __forceinline__ void add_signed(const T* x, T* y, int s) {
#pragma unroll
    for (int i = 0; i < NN; ++i) y[i] += (s > 0) ? x[i] : -x[i];
}

template <int NV, class T>
__device__ __forceinline__ void load_state(const T* __restrict__ src, int N, int q, int first, T* u) {
#pragma unroll
    for (int i = 0; i < NV; ++i) u[i] = src[(size_t)(first + i) * N + q];
}

// ERK targets: dst = src + coef * scale_g * k, where g = GRP(i) picks the
// per-cell material factor of value i (the inverse mass, folded into the
// target coefficient).  Target 0 is kept in `k` (overwritten).  `off` is the
// offset of this shot's domain block.
template <int NV, class GRP, class T>
__device__ __forceinline__ void write_targets(const StageArgsT<T>& A, int N, size_t off, int q, T* k, const T* sc) {
    for (int t = A.n_tgt - 1; t >= 1; --t) {
        const TargetT<T> G = A.tgt[t];
        const T c[3] = {G.coef * sc[0], G.coef * sc[1], G.coef * sc[2]};
        T* dst = G.dst + off;
        if (G.src) {
            const T* src = G.src + off;
#pragma unroll
            for (int i = 0; i < NV; ++i) dst[(size_t)i * N + q] = norm(fma(c[GRP::g(i)], k[i], src[(size_t)i * N + q]));
        } else {
#pragma unroll
            for (int i = 0; i < NV; ++i) dst[(size_t)i * N + q] = norm(c[GRP::g(i)] * k[i]);
        }
    }
    const TargetT<T> G = A.tgt[0];
    const T c[3] = {G.coef * sc[0], G.coef * sc[1], G.coef * sc[2]};
    T* dst = G.dst + off;
    if (G.src) {
        const T* src = G.src + off;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            k[i] = norm(fma(c[GRP::g(i)], k[i], src[(size_t)i * N + q]));
            dst[(size_t)i * N + q] = k[i];
        }
    } else {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            k[i] = norm(c[GRP::g(i)] * k[i]);
            dst[(size_t)i * N + q] = k[i];
        }
    }
}
template <int n>
struct FluidGroups {   // [m_x, m_y | p]
    __host__ __device__ static constexpr int g(int i) { return i < 2 * n ? 0 : 1; }
};
template <int n>
struct SolidGroups {   // [s_xx, s_yy | s_xy | v_x, v_y]
    __host__ __device__ static constexpr int g(int i) { return i < 2 * n ? 0 : (i < 3 * n ? 1 : 2); }
};

// Per-thread view of one (cell, shot): class layout and this shot's buffers.
template <class T>
struct CellCtx {
    int q, lq, nF, npad, sbase, N, SF, SS;
    const T* cd;       // class face blocks
    T tau;
    const T* trf_in;   // this shot's trace buffers (fluid part, solid part)
    const T* trs_in;
    T* trf_out;
    T* trs_out;
};

// ---- L2 prefetch hints -------------------------------------------------------------
// A stage thread reads its cell's state, its faces' own traces, its
// neighbours' traces and the targets' sources in about twenty dependent
// rounds, and with 64 registers it cannot hold more of them in flight.
// Prefetch hints take no register and bring the lines of later rounds into
// L2 early.  Mask bits: 1 state, 2 own traces and face tables, 4 neighbour
// traces, 8 target sources, all at the start of the cell; 16 target sources
// and 32 neighbour traces just before the face loop.  The FP32 kernel gains
// about 20 % from them (mask 50, the best of a sweep on GB300).  The 8-byte
// kernels with register accumulators (spilled) lost with every mask; the
// 8-byte k = 2 kernels with shared-memory accumulators gain from mask 50 too
// (double-float about 10 % over no hints, FP64 a few per cent).
template <class T, int K>
struct L2Prefetch {
    static constexpr int mask = Tuned<T>::t.prefetch[K - 1];
};

__device__ __forceinline__ void pf_l2(const void* p) { asm volatile("prefetch.L2 [%0];" ::"l"(p)); }

// The warp's 32-element runs base + a * stride (a < narr), spread over the
// lanes: every 128-byte line a run touches, unaligned runs included.
template <class E>
__device__ __forceinline__ void pf_runs(const E* base, size_t stride, int narr, int lane) {
    constexpr int BYTES = 32 * (int)sizeof(E), LINES = BYTES / 128 + 1;
    for (int e = lane; e < narr * LINES; e += 32) {
        const int a = e / LINES, m = e - a * LINES;
        pf_l2(reinterpret_cast<const char*>(base + (size_t)a * stride) + min(m * 128, BYTES - 1));
    }
}

// WHERE 0: at the start of the cell; 1: before the face loop.  NV state
// values per cell, NW published traces per face slot (w first, then omega).
template <class T, int K, int NV, int NW, int WHERE, bool TARGETS>
__device__ __forceinline__ void prefetch_cell(const StageArgsT<T>& A, const CellCtx<T>& c, size_t soff, const T* tr,
                                              int S, const int* nbt, const T* bet, int nfaces) {
    constexpr int PF = L2Prefetch<T, K>::mask;
    const int lane = c.q & 31;
    if constexpr (WHERE == 0 && (PF & 1)) pf_runs(A.inp + soff + (c.q - lane), c.N, NV, lane);
    if constexpr (WHERE == 0 && (PF & 2)) {
        for (int j = 0; j < nfaces; ++j) {
            const int s0 = c.sbase + j * c.npad + c.lq - lane;
            pf_runs(tr + (size_t)NW * S + s0, S, NW, lane);
            pf_runs(nbt + s0, 0, 1, lane);
            pf_runs(bet + s0, 0, 1, lane);
        }
    }
    if constexpr ((WHERE == 0 && (PF & 4)) || (WHERE == 1 && (PF & 32))) {
        for (int j = 0; j < nfaces; ++j) {
            const int nb = __ldg(nbt + c.sbase + j * c.npad + c.lq);
            if (nb >= 0)
                for (int l = 0; l < NW; ++l) pf_l2(tr + (size_t)l * S + nb);
        }
    }
    if constexpr (TARGETS && ((WHERE == 0 && (PF & 8)) || (WHERE == 1 && (PF & 16)))) {
        for (int t = 0; t < A.n_tgt; ++t)
            if (A.tgt[t].src) pf_runs(A.tgt[t].src + soff + (c.q - lane), c.N, NV, lane);
    }
}

// ---- point-source wavelets ----------------------------------------------------------
// Ricker wavelet amp (1 - 2 a^2) exp(-a^2), a = pi f0 (t - t0), at the stage
// time.  With a device clock (graph replay) the time is (t0 + n dt) + c dt
// formed with rounded operations in the host's order, and the wavelet is
// evaluated here; otherwise the host's values are used.
__device__ __forceinline__ double stage_time(const StageClock* clk, double dt, double c) {
    const double tn = __dadd_rn(clk->t0, __dmul_rn((double)clk->step, dt));
    return __dadd_rn(tn, __dmul_rn(c, dt));
}
__device__ __forceinline__ double ricker_dev(double t, double f0, double t0, double amp) {
    const double a = __dmul_rn(__dmul_rn(M_PI, f0), __dadd_rn(t, -t0));
    const double a2 = __dmul_rn(a, a);
    return __dmul_rn(__dmul_rn(amp, __dadd_rn(1.0, -__dmul_rn(2.0, a2))), exp(-a2));
}
template <class T>
__device__ __forceinline__ T src_value(const StageArgsT<T>& A, int s) {
    if (!A.clock) return A.src_w[s];
    return T(ricker_dev(stage_time(A.clock, A.dt, A.c_stage), A.src_f0[s], A.src_t0[s], A.src_amp[s]));
}
template <class T>
__device__ __forceinline__ T shot_src_value(const StageArgsT<T>& A) {
    if (!A.clock) return A.shot_src_w;
    return T(ricker_dev(stage_time(A.clock, A.dt, A.c_stage), A.shot_f0, A.shot_t0, A.shot_amp));
}

// ---- fluid cells -------------------------------------------------------------------
// Lift the face jump of one face into the raw rate accumulators
// (kmx, kmy: grad p part; kp: div m part, tau folded).
// The jump p_F - p|_F on local face j (face-basis coefficients, the cell's
// orientation): own omega plus the neighbour's w (interior), or the
// interface combination of the solid neighbour's traces.
template <class T, int K>
__device__ __forceinline__ void fluid_face_jump(const StageArgsT<T>& A, const CellCtx<T>& c, int j, T* jmp) {
    constexpr int f = Dims<K>::f;
    const DevOps& op = A.op;
    const int slot = c.sbase + j * c.npad + c.lq;
    const int nb = __ldg(op.nb_f + slot);
#pragma unroll
    for (int l = 0; l < f; ++l) jmp[l] = __ldg(c.trf_in + (size_t)(f + l) * c.SF + slot);
    if (nb >= 0) {
        const T be = __ldg(OpData<T>::beta_f(op) + slot);
#pragma unroll
        for (int l = 0; l < f; ++l) {
            const T w = __ldg(c.trf_in + (size_t)l * c.SF + nb);
            jmp[l] = (l & 1) ? fma(-be, w, jmp[l]) : fma(be, w, jmp[l]);
        }
    } else if (nb < NB_BOUNDARY) {
        const int r = -2 - nb;
        const int ns = __ldg(op.if_nb + r);
        const T* co = OpData<T>::if_coef(op) + 6 * r;
        const T bx = __ldg(co + 1), by = __ldg(co + 2);
#pragma unroll
        for (int l = 0; l < f; ++l) {
            const T ws = fma(bx, __ldg(c.trs_in + (size_t)l * c.SS + ns), by * __ldg(c.trs_in + (size_t)(f + l) * c.SS + ns));
            jmp[l] = (l & 1) ? jmp[l] - ws : jmp[l] + ws;
        }
    }
}

// Both faces of one orientation of a rectangle (AX = 0: faces 0 and 2,
// normals -/+ e_y; AX = 1: faces 1 and 3, normals +/- e_x), lifted with the
// first face's matrix L.  The mirror through the centroid maps face AX to
// face AX + 2 with Lift_{AX+2} = P L F (P: (-1)^(exponent along the normal)
// on the rows, F: (-1)^l on the face coefficients; checked when the class is
// built).  With s the first face's normal sign, jb, jp the two jumps and
// jh = F jp, sigma = jb + jh and delta = jb - jh:
//     normal accumulator  += s L delta (rows with P = +1), s L sigma (P = -1)
//     tau accumulator     += tau L sigma (P = +1), tau L delta (P = -1)
// Each lifted row is accumulated straight into its target: 4f + 2 nnz(L)
// operations per pair instead of 2 (nnz(L) + 2n) for two separate lifts.
template <class T, int K, int AX, bool SQ = false>
__device__ __forceinline__ void lift_pair(const T* __restrict__ L, const T* jb, const T* jp, T tau, T* ke, T* kt) {
    constexpr int n = Dims<K>::n, f = Dims<K>::f, fP = Dims<K>::fP, w = Vec16<T>::w;
    using P = typename std::conditional<SQ, SquareAxis<AX>, RectAxis<AX>>::type;
    constexpr bool neg = AX == 0;   // face 0 has normal -e_y, face 1 +e_x
    T sg[f], dl[f], ts[f], td[f];
#pragma unroll
    for (int l = 0; l < f; ++l) {
        const T jh = (l & 1) ? -jp[l] : jp[l];
        sg[l] = jb[l] + jh;
        dl[l] = jb[l] - jh;
        ts[l] = tau * sg[l];
        td[l] = tau * dl[l];
    }
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const int en = AX == 0 ? eb(i) : ea(i);   // exponent along the normal
        const bool even = (en & 1) == 0;
        T row[fP];
#pragma unroll
        for (int c0 = 0; c0 < fP; c0 += w) {
            bool need = false;
#pragma unroll
            for (int e = 0; e < w; ++e) need = need || (c0 + e < f && P::lift_nz(i, c0 + e));
            if (need) cls_row<T>(L + i * fP + c0, row + c0);
        }
        T e = ke[i], k = kt[i];
#pragma unroll
        for (int l = 0; l < f; ++l)
            if (P::lift_nz(i, l)) {
                const T a = even ? dl[l] : sg[l];
                e = neg ? fma(-row[l], a, e) : fma(row[l], a, e);
                k = fma(row[l], even ? ts[l] : td[l], k);
            }
        ke[i] = e;
        kt[i] = k;
    }
}

template <class T, int K, int AX, bool SQ = false>
__device__ __forceinline__ void fluid_pair_rate(const StageArgsT<T>& A, const CellCtx<T>& c, T* kmx, T* kmy, T* kp) {
    constexpr int f = Dims<K>::f, FS = Dims<K>::FS;
    T jb[f], jp[f];
    fluid_face_jump<T, K>(A, c, AX, jb);
    fluid_face_jump<T, K>(A, c, AX + 2, jp);
    lift_pair<T, K, AX, SQ>(c.cd + AX * FS + Dims<K>::LI, jb, jp, c.tau, AX == 0 ? kmy : kmx, kp);
}

template <class T, int K, class P>
__device__ __forceinline__ void fluid_face_rate(const StageArgsT<T>& A, const CellCtx<T>& c, int j, int sg, T* kmx,
                                                T* kmy, T* kp) {
    constexpr int n = Dims<K>::n, f = Dims<K>::f, FS = Dims<K>::FS;
    const DevOps& op = A.op;
    const T* fm = c.cd + j * FS;
    T jmp[f];
    fluid_face_jump<T, K>(A, c, j, jmp);
    T lv[n];
    lift_apply<T, K, P>(fm + Dims<K>::LI, jmp, lv);
    if constexpr (P::rect) {
        add_signed<n>(lv, P::horiz ? kmy : kmx, sg);
    } else {
        const T nx = cls_val(fm), ny = cls_val(fm + 1);
#pragma unroll
        for (int i = 0; i < n; ++i) {
            kmx[i] = fma(nx, lv[i], kmx[i]);
            kmy[i] = fma(ny, lv[i], kmy[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < n; ++i) kp[i] = fma(c.tau, lv[i], kp[i]);
}

// Publish w = tau p|_F - (m.n)|_F and omega = alpha w - p|_F for one face.
template <class T, int K, class P>
__device__ __forceinline__ void fluid_face_trace(const StageArgsT<T>& A, const CellCtx<T>& c, int j, int sg,
                                                 const T* U) {
    constexpr int n = Dims<K>::n, f = Dims<K>::f, FS = Dims<K>::FS;
    const DevOps& op = A.op;
    const T* fm = c.cd + j * FS;
    const T* Tr = fm + Dims<K>::TR;
    const T* mx = U;
    const T* my = U + n;
    const T* p = U + 2 * n;
    T tp[f], tm[f];
    face_trace_apply<T, K, P>(Tr, p, tp, sg);
    if constexpr (P::rect) {
        face_trace_apply<T, K, P>(Tr, P::horiz ? my : mx, tm, sg);
    } else {
        const T nx = cls_val(fm), ny = cls_val(fm + 1);
        T mn[n];
#pragma unroll
        for (int i = 0; i < n; ++i) mn[i] = fma(nx, mx[i], ny * my[i]);
        face_trace_apply<T, K, P>(Tr, mn, tm, sg);
    }
    const int sgn = P::rect ? sg : 1;   // rect: tm holds the unsigned trace
    const int slot = c.sbase + j * c.npad + c.lq;
    const int nb = __ldg(op.nb_f + slot);
    const T al = (nb >= NB_BOUNDARY) ? __ldg(OpData<T>::beta_f(op) + slot) : __ldg(OpData<T>::if_coef(op) + 6 * (-2 - nb));
#pragma unroll
    for (int l = 0; l < f; ++l) {
        const T w = fma(c.tau, tp[l], (sgn > 0) ? -tm[l] : tm[l]);
        c.trf_out[(size_t)l * c.SF + slot] = norm(w);
        c.trf_out[(size_t)(f + l) * c.SF + slot] = norm(fma(al, w, -tp[l]));
    }
}

// The four faces of a rectangle: one body per orientation looped over its
// two faces (RectLoop), or unrolled with constant signs.
template <class T, int K, class PH, class PV>
__device__ __forceinline__ void fluid_rect_traces(const StageArgsT<T>& A, const CellCtx<T>& c, const T* U) {
    if constexpr (RectLoop<T, K>::value) {
#pragma unroll 1
        for (int h = 0; h < 2; ++h) fluid_face_trace<T, K, PH>(A, c, 2 * h, 2 * h - 1, U);
#pragma unroll 1
        for (int v = 0; v < 2; ++v) fluid_face_trace<T, K, PV>(A, c, 1 + 2 * v, 1 - 2 * v, U);
    } else {
        fluid_face_trace<T, K, PH>(A, c, 0, -1, U);
        fluid_face_trace<T, K, PV>(A, c, 1, 1, U);
        fluid_face_trace<T, K, PH>(A, c, 2, 1, U);
        fluid_face_trace<T, K, PV>(A, c, 3, -1, U);
    }
}

template <class T, int K, int MODE>
__device__ __forceinline__ void fluid_cell(const StageArgsT<T>& A, int q, int shot, const T* cd_smem, T* acc_smem) {
    constexpr int n = Dims<K>::n, f = Dims<K>::f;
    const DevOps& op = A.op;
    const int cls = __ldg(op.warp_class + (q >> 5));
    const int* ci = op.cls_int + cls * CI_STRIDE;
    CellCtx<T> c;
    c.q = q;
    c.lq = q - __ldg(ci + CI_START);
    if (c.lq >= __ldg(ci + CI_COUNT)) return;   // class padding
    c.nF = __ldg(ci + CI_NF);
    c.npad = __ldg(ci + CI_NPAD);
    c.sbase = __ldg(ci + CI_SLOT);
    c.cd = ClsSmem<T>::value ? cd_smem : OpData<T>::cls(op) + __ldg(ci + CI_DOFF) + Dims<K>::M0P;
    c.N = op.Nf;
    c.SF = op.SF;
    c.SS = op.SS;
    c.tau = __ldg(OpData<T>::scal_f(op) + SF_TAU * c.N + q);
    const size_t toff = (size_t)shot * A.trace_stride;
    c.trf_in = A.tr_in + toff;
    c.trs_in = A.tr_in + toff + (size_t)2 * f * c.SF;
    c.trf_out = A.tr_out + toff;
    c.trs_out = A.tr_out + toff + (size_t)2 * f * c.SF;
    const size_t soff = (size_t)shot * A.state_stride;
    const int kind = __ldg(ci + CI_KIND);
    const bool rect = kind != KIND_GENERIC;
    T Ureg[AccSmem<T, K>::value ? 1 : 3 * n];
    T* U = AccSmem<T, K>::value ? acc_smem : Ureg;   // [m_x | m_y | p]
    if constexpr (MODE == MODE_TRACES) {
        load_state<3 * n>(A.inp + soff, c.N, q, 0, U);
    } else {
        T* kmx = U;
        T* kmy = U + n;
        T* kp = U + 2 * n;
        if constexpr (L2Prefetch<T, K>::mask != 0)
            prefetch_cell<T, K, 3 * n, f, 0, MODE != MODE_RAW>(A, c, soff, c.trf_in, c.SF, op.nb_f,
                                                            OpData<T>::beta_f(op), rect ? 4 : c.nF);
        {
            T u[n];
            load_state<n>(A.inp + soff, c.N, q, 2 * n, u);      // p
            ddx<T, K>(u, kmx);
            ddy<T, K>(u, kmy);
            load_state<n>(A.inp + soff, c.N, q, 0, u);          // m_x
            ddx<T, K>(u, kp);
            load_state<n>(A.inp + soff, c.N, q, n, u);          // m_y
            add_ddy<T, K>(u, kp);
        }
        if constexpr (L2Prefetch<T, K>::mask != 0)
            prefetch_cell<T, K, 3 * n, f, 1, MODE != MODE_RAW>(A, c, soff, c.trf_in, c.SF, op.nb_f,
                                                            OpData<T>::beta_f(op), rect ? 4 : c.nF);
        if (rect) {
            // faces 0 (s = -1) and 2 (s = +1) are horizontal, 1 (s = +1) and 3 (s = -1) vertical
            if (kind == KIND_SQUARE) {
                fluid_pair_rate<T, K, 0, true>(A, c, kmx, kmy, kp);   // faces 0 and 2
                fluid_pair_rate<T, K, 1, true>(A, c, kmx, kmy, kp);   // faces 1 and 3
            } else {
                fluid_pair_rate<T, K, 0>(A, c, kmx, kmy, kp);
                fluid_pair_rate<T, K, 1>(A, c, kmx, kmy, kp);
            }
        } else {
#pragma unroll 1
            for (int j = 0; j < c.nF; ++j) fluid_face_rate<T, K, GenericFace>(A, c, j, 1, kmx, kmy, kp);
        }
        const T Am = __ldg(OpData<T>::scal_f(op) + SF_AM * c.N + q), Ap = __ldg(OpData<T>::scal_f(op) + SF_AP * c.N + q);
        // Point sources: the stored vector is kappa/h^2 M0^-1 phi(x_s); the
        // raw rate is multiplied by A_p = kappa/h in the targets.
        for (int s = 0; s < A.n_src; ++s) {
            if (A.src_dom[s] == 0 && A.src_q[s] == q) {
                const T w = src_value(A, s) / Ap;
                const T* g = A.src_g + (size_t)s * 2 * n;
#pragma unroll
                for (int i = 0; i < n; ++i) kp[i] = fma(w, g[i], kp[i]);
            }
        }
        if (A.shot_src_q && A.shot_src_dom[shot] == 0 && A.shot_src_q[shot] == q) {
            const T w = shot_src_value(A) / Ap;
            const T* g = A.shot_src_g + (size_t)shot * 2 * n;
#pragma unroll
            for (int i = 0; i < n; ++i) kp[i] = fma(w, g[i], kp[i]);
        }
        if constexpr (MODE == MODE_RAW) {
            T* dst = A.tgt[0].dst + soff;
#pragma unroll
            for (int i = 0; i < 3 * n; ++i) dst[(size_t)i * c.N + q] = norm(U[i]);
            return;
        }
        const T sc[3] = {Am, Ap, T(0)};
        write_targets<3 * n, FluidGroups<n>>(A, c.N, soff, q, U, sc);
        if constexpr (MODE == MODE_APPLY) return;
    }
    if (kind == KIND_SQUARE) {
        fluid_rect_traces<T, K, SquareAxis<0>, SquareAxis<1>>(A, c, U);
    } else if (rect) {
        fluid_rect_traces<T, K, RectAxis<0>, RectAxis<1>>(A, c, U);
    } else {
#pragma unroll 1
        for (int j = 0; j < c.nF; ++j) fluid_face_trace<T, K, GenericFace>(A, c, j, 1, U);
    }
}

// ---- solid cells -------------------------------------------------------------------
// The velocity jump v_F - v|_F on local face j (components x, y).
template <class T, int K>
__device__ __forceinline__ void solid_face_jump(const StageArgsT<T>& A, const CellCtx<T>& c, int j, T* jx, T* jy) {
    constexpr int f = Dims<K>::f;
    const DevOps& op = A.op;
    const int slot = c.sbase + j * c.npad + c.lq;
    const int nb = __ldg(op.nb_s + slot);
#pragma unroll
    for (int l = 0; l < f; ++l) {
        jx[l] = __ldg(c.trs_in + (size_t)(2 * f + l) * c.SS + slot);
        jy[l] = __ldg(c.trs_in + (size_t)(3 * f + l) * c.SS + slot);
    }
    if (nb >= 0) {
        const T be = __ldg(OpData<T>::beta_s(op) + slot);
#pragma unroll
        for (int l = 0; l < f; ++l) {
            const T wx = __ldg(c.trs_in + (size_t)l * c.SS + nb);
            const T wy = __ldg(c.trs_in + (size_t)(f + l) * c.SS + nb);
            jx[l] = (l & 1) ? fma(-be, wx, jx[l]) : fma(be, wx, jx[l]);
            jy[l] = (l & 1) ? fma(-be, wy, jy[l]) : fma(be, wy, jy[l]);
        }
    } else if (nb < NB_BOUNDARY) {
        const int r = -2 - nb;
        const int nfs = __ldg(op.if_nb + r);
        const T* co = OpData<T>::if_coef(op) + 6 * r;
        const T b0 = __ldg(co + 4), b1 = __ldg(co + 5);
#pragma unroll
        for (int l = 0; l < f; ++l) {
            const T wf = __ldg(c.trf_in + (size_t)l * c.SF + nfs);
            jx[l] = (l & 1) ? fma(-b0, wf, jx[l]) : fma(b0, wf, jx[l]);
            jy[l] = (l & 1) ? fma(-b1, wf, jy[l]) : fma(b1, wf, jy[l]);
        }
    }
}

// Lift one face's velocity jump into the raw accumulators: e (strain rate,
// symmetric-gradient part) and kv (div s part, tau folded).
template <class T, int K, class P>
__device__ __forceinline__ void solid_face_rate(const StageArgsT<T>& A, const CellCtx<T>& c, int j, int sg, T* exx,
                                                T* eyy, T* exy, T* kvx, T* kvy) {
    constexpr int n = Dims<K>::n, f = Dims<K>::f, FS = Dims<K>::FS;
    const DevOps& op = A.op;
    const T* fm = c.cd + j * FS;
    T jx[f], jy[f];
    solid_face_jump<T, K>(A, c, j, jx, jy);
    const T* L = fm + Dims<K>::LI;
    T lx[n], ly[n];
    lift_apply<T, K, P>(L, jx, lx);
    lift_apply<T, K, P>(L, jy, ly);
    if constexpr (P::rect) {
        if constexpr (P::horiz) {
            add_signed<n>(ly, eyy, sg);
            add_signed<n>(lx, exy, sg);
        } else {
            add_signed<n>(lx, exx, sg);
            add_signed<n>(ly, exy, sg);
        }
    } else {
        const T nx = cls_val(fm), ny = cls_val(fm + 1);
#pragma unroll
        for (int i = 0; i < n; ++i) {
            exx[i] = fma(nx, lx[i], exx[i]);
            eyy[i] = fma(ny, ly[i], eyy[i]);
            exy[i] = fma(nx, ly[i], fma(ny, lx[i], exy[i]));
        }
    }
#pragma unroll
    for (int i = 0; i < n; ++i) {
        kvx[i] = fma(c.tau, lx[i], kvx[i]);
        kvy[i] = fma(c.tau, ly[i], kvy[i]);
    }
}

// Both faces of one rectangle orientation (see lift_pair): horizontal faces
// feed e_yy (y component) and e_xy (x component), vertical ones e_xx (x) and
// e_xy (y); tau times both components feeds kv.
template <class T, int K, int AX, bool SQ = false>
__device__ __forceinline__ void solid_pair_rate(const StageArgsT<T>& A, const CellCtx<T>& c, T* exx, T* eyy, T* exy,
                                                T* kvx, T* kvy) {
    constexpr int f = Dims<K>::f, FS = Dims<K>::FS;
    T bx[f], by[f], px[f], py[f];
    solid_face_jump<T, K>(A, c, AX, bx, by);
    solid_face_jump<T, K>(A, c, AX + 2, px, py);
    const T* L = c.cd + AX * FS + Dims<K>::LI;
    lift_pair<T, K, AX, SQ>(L, bx, px, c.tau, AX == 0 ? exy : exx, kvx);
    lift_pair<T, K, AX, SQ>(L, by, py, c.tau, AX == 0 ? eyy : exy, kvy);
}

// Publish w = tau v|_F - (s n)|_F and omega = alpha w - v|_F for one face.
template <class T, int K, class P>
__device__ __forceinline__ void solid_face_trace(const StageArgsT<T>& A, const CellCtx<T>& c, int j, int sg,
                                                 const T* U) {
    constexpr int n = Dims<K>::n, f = Dims<K>::f, FS = Dims<K>::FS;
    const DevOps& op = A.op;
    const T* fm = c.cd + j * FS;
    const T* Tr = fm + Dims<K>::TR;
    const T* sxx = U;
    const T* syy = U + n;
    const T* sxy = U + 2 * n;
    const T* vx = U + 3 * n;
    const T* vy = U + 4 * n;
    T tvx[f], tvy[f], tsx[f], tsy[f];
    face_trace_apply<T, K, P>(Tr, vx, tvx, sg);
    face_trace_apply<T, K, P>(Tr, vy, tvy, sg);
    if constexpr (P::rect) {
        // s n = (nx s_xx + ny s_xy, nx s_xy + ny s_yy) with one of nx, ny = +-1
        if constexpr (!P::horiz) {
            face_trace_apply<T, K, P>(Tr, sxx, tsx, sg);
            face_trace_apply<T, K, P>(Tr, sxy, tsy, sg);
        } else {
            face_trace_apply<T, K, P>(Tr, sxy, tsx, sg);
            face_trace_apply<T, K, P>(Tr, syy, tsy, sg);
        }
    } else {
        const T nx = cls_val(fm), ny = cls_val(fm + 1);
        T snx[n], sny[n];
#pragma unroll
        for (int i = 0; i < n; ++i) {
            snx[i] = fma(nx, sxx[i], ny * sxy[i]);
            sny[i] = fma(nx, sxy[i], ny * syy[i]);
        }
        face_trace_apply<T, K, P>(Tr, snx, tsx, sg);
        face_trace_apply<T, K, P>(Tr, sny, tsy, sg);
    }
    const int sgn = P::rect ? sg : 1;
    const int slot = c.sbase + j * c.npad + c.lq;
    const int nb = __ldg(op.nb_s + slot);
    T* TWS = c.trs_out;
    if (nb >= NB_BOUNDARY) {
        const T be = __ldg(OpData<T>::beta_s(op) + slot);
#pragma unroll
        for (int l = 0; l < f; ++l) {
            const T wx = fma(c.tau, tvx[l], (sgn > 0) ? -tsx[l] : tsx[l]);
            const T wy = fma(c.tau, tvy[l], (sgn > 0) ? -tsy[l] : tsy[l]);
            TWS[(size_t)l * c.SS + slot] = norm(wx);
            TWS[(size_t)(f + l) * c.SS + slot] = norm(wy);
            TWS[(size_t)(2 * f + l) * c.SS + slot] = norm(fma(be, wx, -tvx[l]));
            TWS[(size_t)(3 * f + l) * c.SS + slot] = norm(fma(be, wy, -tvy[l]));
        }
    } else {
        const T* co = OpData<T>::if_coef(op) + 6 * (-2 - nb);
        const T a00 = __ldg(co), a01 = __ldg(co + 1), a10 = __ldg(co + 2), a11 = __ldg(co + 3);
#pragma unroll
        for (int l = 0; l < f; ++l) {
            const T wx = fma(c.tau, tvx[l], (sgn > 0) ? -tsx[l] : tsx[l]);
            const T wy = fma(c.tau, tvy[l], (sgn > 0) ? -tsy[l] : tsy[l]);
            TWS[(size_t)l * c.SS + slot] = norm(wx);
            TWS[(size_t)(f + l) * c.SS + slot] = norm(wy);
            TWS[(size_t)(2 * f + l) * c.SS + slot] = norm(fma(a00, wx, fma(a01, wy, -tvx[l])));
            TWS[(size_t)(3 * f + l) * c.SS + slot] = norm(fma(a10, wx, fma(a11, wy, -tvy[l])));
        }
    }
}

// The four faces of a rectangle: one body per orientation looped over its
// two faces (RectLoop), or unrolled with constant signs.
template <class T, int K, class PH, class PV>
__device__ __forceinline__ void solid_rect_traces(const StageArgsT<T>& A, const CellCtx<T>& c, const T* U) {
    if constexpr (RectLoop<T, K>::value) {
#pragma unroll 1
        for (int h = 0; h < 2; ++h) solid_face_trace<T, K, PH>(A, c, 2 * h, 2 * h - 1, U);
#pragma unroll 1
        for (int v = 0; v < 2; ++v) solid_face_trace<T, K, PV>(A, c, 1 + 2 * v, 1 - 2 * v, U);
    } else {
        solid_face_trace<T, K, PH>(A, c, 0, -1, U);
        solid_face_trace<T, K, PV>(A, c, 1, 1, U);
        solid_face_trace<T, K, PH>(A, c, 2, 1, U);
        solid_face_trace<T, K, PV>(A, c, 3, -1, U);
    }
}

template <class T, int K, int MODE>
__device__ __forceinline__ void solid_cell(const StageArgsT<T>& A, int q, int shot, const T* cd_smem, T* acc_smem) {
    constexpr int n = Dims<K>::n, f = Dims<K>::f;
    const DevOps& op = A.op;
    const int cls = __ldg(op.warp_class + op.n_warps_f + (q >> 5));
    const int* ci = op.cls_int + cls * CI_STRIDE;
    CellCtx<T> c;
    c.q = q;
    c.lq = q - __ldg(ci + CI_START);
    if (c.lq >= __ldg(ci + CI_COUNT)) return;
    c.nF = __ldg(ci + CI_NF);
    c.npad = __ldg(ci + CI_NPAD);
    c.sbase = __ldg(ci + CI_SLOT);
    c.cd = ClsSmem<T>::value ? cd_smem : OpData<T>::cls(op) + __ldg(ci + CI_DOFF) + Dims<K>::M0P;
    c.N = op.Ns;
    c.SF = op.SF;
    c.SS = op.SS;
    c.tau = __ldg(OpData<T>::scal_s(op) + SS_TAU * c.N + q);
    const size_t toff = (size_t)shot * A.trace_stride;
    c.trf_in = A.tr_in + toff;
    c.trs_in = A.tr_in + toff + (size_t)2 * f * c.SF;
    c.trf_out = A.tr_out + toff;
    c.trs_out = A.tr_out + toff + (size_t)2 * f * c.SF;
    const int kind = __ldg(ci + CI_KIND);
    const bool rect = kind != KIND_GENERIC;
    const size_t soff = (size_t)shot * A.state_stride + (size_t)3 * n * op.Nf;
    const T* inp = A.inp + soff;
    T Ureg[AccSmem<T, K>::value ? 1 : 5 * n];
    T* U = AccSmem<T, K>::value ? acc_smem : Ureg;   // [s_xx | s_yy | s_xy | v_x | v_y]
    if constexpr (MODE == MODE_TRACES) {
        load_state<5 * n>(inp, c.N, q, 0, U);
    } else {
        T* exx = U;
        T* eyy = U + n;
        T* exy = U + 2 * n;
        T* kvx = U + 3 * n;
        T* kvy = U + 4 * n;
        if constexpr (L2Prefetch<T, K>::mask != 0)
            prefetch_cell<T, K, 5 * n, 2 * f, 0, MODE != MODE_RAW>(A, c, soff, c.trs_in, c.SS, op.nb_s,
                                                                OpData<T>::beta_s(op), rect ? 4 : c.nF);
        {
            T u[n];
            load_state<n>(inp, c.N, q, 3 * n, u);    // v_x
            ddx<T, K>(u, exx);
            ddy<T, K>(u, exy);
            load_state<n>(inp, c.N, q, 4 * n, u);    // v_y
            ddy<T, K>(u, eyy);
            add_ddx<T, K>(u, exy);
            load_state<n>(inp, c.N, q, 0, u);        // s_xx
            ddx<T, K>(u, kvx);
            load_state<n>(inp, c.N, q, n, u);        // s_yy
            ddy<T, K>(u, kvy);
            load_state<n>(inp, c.N, q, 2 * n, u);    // s_xy
            add_ddy<T, K>(u, kvx);
            add_ddx<T, K>(u, kvy);
        }
        if constexpr (L2Prefetch<T, K>::mask != 0)
            prefetch_cell<T, K, 5 * n, 2 * f, 1, MODE != MODE_RAW>(A, c, soff, c.trs_in, c.SS, op.nb_s,
                                                                OpData<T>::beta_s(op), rect ? 4 : c.nF);
        if (rect) {
            if (kind == KIND_SQUARE) {
                solid_pair_rate<T, K, 0, true>(A, c, exx, eyy, exy, kvx, kvy);   // faces 0 and 2
                solid_pair_rate<T, K, 1, true>(A, c, exx, eyy, exy, kvx, kvy);   // faces 1 and 3
            } else {
                solid_pair_rate<T, K, 0>(A, c, exx, eyy, exy, kvx, kvy);
                solid_pair_rate<T, K, 1>(A, c, exx, eyy, exy, kvx, kvy);
            }
        } else {
#pragma unroll 1
            for (int j = 0; j < c.nF; ++j) solid_face_rate<T, K, GenericFace>(A, c, j, 1, exx, eyy, exy, kvx, kvy);
        }
        // stress rate = C e = c1 [(e_xx + r e_yy), (e_yy + r e_xx)], c3 e_xy; c1, c3 folded into targets
        const T r = __ldg(OpData<T>::scal_s(op) + SS_R * c.N + q);
        if constexpr (MODE != MODE_RAW) {
#pragma unroll
            for (int i = 0; i < n; ++i) {
                const T a = exx[i], b = eyy[i];
                exx[i] = fma(r, b, a);
                eyy[i] = fma(r, a, b);
            }
        }
        const T Av = __ldg(OpData<T>::scal_s(op) + SS_AV * c.N + q);
        for (int s = 0; s < A.n_src; ++s) {
            if (A.src_dom[s] == 1 && A.src_q[s] == q) {
                const T w = src_value(A, s) / Av;
                const T* g = A.src_g + (size_t)s * 2 * n;
#pragma unroll
                for (int i = 0; i < n; ++i) {
                    kvx[i] = fma(w, g[i], kvx[i]);
                    kvy[i] = fma(w, g[n + i], kvy[i]);
                }
            }
        }
        if (A.shot_src_q && A.shot_src_dom[shot] == 1 && A.shot_src_q[shot] == q) {
            const T w = shot_src_value(A) / Av;
            const T* g = A.shot_src_g + (size_t)shot * 2 * n;
#pragma unroll
            for (int i = 0; i < n; ++i) {
                kvx[i] = fma(w, g[i], kvx[i]);
                kvy[i] = fma(w, g[n + i], kvy[i]);
            }
        }
        if constexpr (MODE == MODE_RAW) {
            T* dst = A.tgt[0].dst + soff;
#pragma unroll
            for (int i = 0; i < 5 * n; ++i) dst[(size_t)i * c.N + q] = norm(U[i]);
            return;
        }
        const T sc[3] = {__ldg(OpData<T>::scal_s(op) + SS_C1 * c.N + q), __ldg(OpData<T>::scal_s(op) + SS_C3 * c.N + q), Av};
        write_targets<5 * n, SolidGroups<n>>(A, c.N, soff, q, U, sc);
        if constexpr (MODE == MODE_APPLY) return;
    }
    if (kind == KIND_SQUARE) {
        solid_rect_traces<T, K, SquareAxis<0>, SquareAxis<1>>(A, c, U);
    } else if (rect) {
        solid_rect_traces<T, K, RectAxis<0>, RectAxis<1>>(A, c, U);
    } else {
#pragma unroll 1
        for (int j = 0; j < c.nF; ++j) solid_face_trace<T, K, GenericFace>(A, c, j, 1, U);
    }
}

#include "stage_tc.cuh"

// Resident blocks per SM asked of the register allocator (128 threads a
// block): 2 blocks allow 255 registers, 3 allow 168, 4 allow 128, 5 allow 96,
// 6 allow 80, 8 allow 64.  The stage kernels are bound by load latency, so
// occupancy pays even at the price of spills to local memory; where the
// accumulators sit in shared memory (AccSmem) the shared memory may cap the
// resident blocks below this count.  The values are the fastest of sweeps
// on the 1024 x 512 bilayer (and, for FP32, the 1.2 M-cell hybrid mesh) on
// GB300.
template <class T, int K>
struct MinBlocks {
    static constexpr int value = Tuned<T>::t.min_blocks[K - 1];
};

// Dynamic shared memory of a stage block: the per-warp class copies
// (max_nf face blocks of Dims<K>::FS values per warp) when ClsSmem<T>.
template <class T, int K>
__host__ __device__ size_t stage_cls_smem_bytes(int max_nf) {
    return ClsSmem<T>::value ? sizeof(T) * (128 / 32) * (size_t)max_nf * Dims<K>::FS : 0;
}
template <class T, int K>
size_t stage_smem_bytes(int max_nf) {
    return stage_cls_smem_bytes<T, K>(max_nf) + (AccSmem<T, K>::value ? sizeof(T) * 128 * acc_stride<K>() : 0);
}

// Grid: x over the padded cells of both domains (fluid warps, then solid
// warps; a warp lies in one class), y over shots; 128 threads.
template <class T, int K, int MODE>
__global__ void __launch_bounds__(128, MinBlocks<T, K>::value) stage_kernel(const StageArgsT<T> A) {
    const int gq = blockIdx.x * blockDim.x + threadIdx.x;
    const int shot = blockIdx.y;
    const T* cd = nullptr;
    extern __shared__ __align__(16) unsigned char stage_smem[];
    T* acc = nullptr;
    if constexpr (AccSmem<T, K>::value)
        acc = reinterpret_cast<T*>(stage_smem + stage_cls_smem_bytes<T, K>(A.op.max_nf)) + threadIdx.x * acc_stride<K>();
    if constexpr (ClsSmem<T>::value) {
        constexpr int FS = Dims<K>::FS;
        const int gw = gq >> 5;
        if (gw >= A.op.n_warps_f + A.op.n_warps_s) return;   // the whole warp is past the last class
        T* dst = reinterpret_cast<T*>(stage_smem) + (threadIdx.x >> 5) * A.op.max_nf * FS;
        const int* ci = A.op.cls_int + __ldg(A.op.warp_class + gw) * CI_STRIDE;
        const int nv = __ldg(ci + CI_NF) * FS * (int)sizeof(T) / 16;
        const float4* src =
            reinterpret_cast<const float4*>(OpData<T>::cls(A.op) + __ldg(ci + CI_DOFF) + Dims<K>::M0P);
        float4* d4 = reinterpret_cast<float4*>(dst);
        for (int e = threadIdx.x & 31; e < nv; e += 32) d4[e] = __ldg(src + e);
        __syncwarp();
        cd = dst;
    }
    if (gq < A.op.Nf)
        fluid_cell<T, K, MODE>(A, gq, shot, cd, acc);
    else if (gq < A.op.Nf + A.op.Ns)
        solid_cell<T, K, MODE>(A, gq - A.op.Nf, shot, cd, acc);
}

// canonical (AoS, input cell order, FP64) <-> device layout (SoA by class, T);
// y = shot: canonical shot stride n_canon, state shot stride n_state.
template <class T>
__global__ void pack_kernel(const int32_t* __restrict__ dev2orig, const int64_t* __restrict__ canon_off, int Nf,
                            int Ns, int n, int64_t n_canon, int64_t n_state, const double* __restrict__ canon,
                            T* __restrict__ state) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Nf + Ns) return;
    const bool fl = g < Nf;
    const int q = fl ? g : g - Nf;
    const int N = fl ? Nf : Ns;
    const int nv = (fl ? 3 : 5) * n;
    T* st = state + (size_t)blockIdx.y * n_state + (fl ? 0 : (size_t)3 * n * Nf);
    const int c = dev2orig[g];
    if (c < 0) {
        for (int i = 0; i < nv; ++i) st[(size_t)i * N + q] = T(0);
        return;
    }
    const double* cv = canon + (size_t)blockIdx.y * n_canon + canon_off[c];
    for (int i = 0; i < nv; ++i) st[(size_t)i * N + q] = T(cv[i]);
}
template <class T>
__global__ void unpack_kernel(const int32_t* __restrict__ dev2orig, const int64_t* __restrict__ canon_off, int Nf,
                              int Ns, int n, int64_t n_canon, int64_t n_state, const T* __restrict__ state,
                              double* __restrict__ canon) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Nf + Ns) return;
    const bool fl = g < Nf;
    const int q = fl ? g : g - Nf;
    const int N = fl ? Nf : Ns;
    const int nv = (fl ? 3 : 5) * n;
    const T* st = state + (size_t)blockIdx.y * n_state + (fl ? 0 : (size_t)3 * n * Nf);
    const int c = dev2orig[g];
    if (c < 0) return;
    double* cv = canon + (size_t)blockIdx.y * n_canon + canon_off[c];
    for (int i = 0; i < nv; ++i) cv[i] = double(st[(size_t)i * N + q]);
}

// Canonical vector in host memory (pinned, mapped into the device's address
// space) <-> device-layout state of type T.  A block of 64 threads takes 64
// consecutive canonical cells, whose values form one contiguous run: the run
// crosses the host link in coalesced 8-byte accesses (eight in flight per
// thread) and is reordered through shared memory, one thread per cell on the
// device side.  Padding slots of the state are not touched.
constexpr int STAGED_CELLS = 64;
template <class T>
__global__ void __launch_bounds__(STAGED_CELLS) pack_host_kernel(const int32_t* __restrict__ cell_dom,
                                                                 const int32_t* __restrict__ cell_pos,
                                                                 const int64_t* __restrict__ canon_off, int nc,
                                                                 int64_t n_canon, int Nf, int Ns, int n,
                                                                 const double* __restrict__ canon,
                                                                 T* __restrict__ state) {
    extern __shared__ double run[];
    const int c0 = blockIdx.x * STAGED_CELLS;
    const int c1 = min(c0 + STAGED_CELLS, nc);
    const int64_t e0 = canon_off[c0];
    const int len = (int)((c1 < nc ? canon_off[c1] : n_canon) - e0);
    constexpr int U = 8;
    for (int b = 0; b < len; b += U * STAGED_CELLS) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = b + u * STAGED_CELLS + threadIdx.x;
            v[u] = e < len ? canon[e0 + e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = b + u * STAGED_CELLS + threadIdx.x;
            if (e < len) run[e] = v[u];
        }
    }
    __syncthreads();
    const int c = c0 + threadIdx.x;
    if (c >= c1) return;
    const bool fl = cell_dom[c] == 0;
    const int q = cell_pos[c];
    const int N = fl ? Nf : Ns;
    T* st = state + (fl ? 0 : (size_t)3 * n * Nf);
    const double* v = run + (canon_off[c] - e0);
    const int nv = (fl ? 3 : 5) * n;
    for (int i = 0; i < nv; ++i) st[(size_t)i * N + q] = T(v[i]);
}
template <class T>
__global__ void __launch_bounds__(STAGED_CELLS) unpack_host_kernel(const int32_t* __restrict__ cell_dom,
                                                                   const int32_t* __restrict__ cell_pos,
                                                                   const int64_t* __restrict__ canon_off, int nc,
                                                                   int64_t n_canon, int Nf, int Ns, int n,
                                                                   const T* __restrict__ state,
                                                                   double* __restrict__ canon) {
    extern __shared__ double run[];
    const int c0 = blockIdx.x * STAGED_CELLS;
    const int c1 = min(c0 + STAGED_CELLS, nc);
    const int64_t e0 = canon_off[c0];
    const int len = (int)((c1 < nc ? canon_off[c1] : n_canon) - e0);
    const int c = c0 + threadIdx.x;
    if (c < c1) {
        const bool fl = cell_dom[c] == 0;
        const int q = cell_pos[c];
        const int N = fl ? Nf : Ns;
        const T* st = state + (fl ? 0 : (size_t)3 * n * Nf);
        double* v = run + (canon_off[c] - e0);
        const int nv = (fl ? 3 : 5) * n;
        for (int i = 0; i < nv; ++i) v[i] = double(st[(size_t)i * N + q]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < len; e += STAGED_CELLS) canon[e0 + e] = run[e];
}

// Energy 1/2 U^T M U (Sec. 5.1) with M = h^2 (material) x M0_ref per cell.
template <int K>
__global__ void __launch_bounds__(256) energy_kernel(DevOps op, const double* __restrict__ state,
                                                    const double* __restrict__ mass_f,
                                                    const double* __restrict__ mass_s, double* partial) {
    constexpr int n = Dims<K>::n;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (g < op.Nf + op.Ns) {
        const bool fl = g < op.Nf;
        const int q = fl ? g : g - op.Nf;
        const int cls = op.warp_class[(fl ? 0 : op.n_warps_f) + (q >> 5)];
        const int* ci = op.cls_int + cls * CI_STRIDE;
        if (q - ci[CI_START] < ci[CI_COUNT]) {
            const double* M0 = op.cls_dbl + ci[CI_DOFF];
            const int N = fl ? op.Nf : op.Ns;
            const double* st = state + (fl ? 0 : (size_t)3 * n * op.Nf);
            auto quad = [&](int fa, int fb) {
                double s = 0.0;
                for (int i = 0; i < n; ++i) {
                    double r = 0.0;
                    for (int j = 0; j < n; ++j) r = fma(M0[i * n + j], st[(size_t)(fb * n + j) * N + q], r);
                    s = fma(st[(size_t)(fa * n + i) * N + q], r, s);
                }
                return s;
            };
            if (fl) {
                e = 0.5 * (mass_f[q] * (quad(0, 0) + quad(1, 1)) + mass_f[N + q] * quad(2, 2));
            } else {
                const double d0 = mass_s[q], d1 = mass_s[N + q], d2 = mass_s[2 * N + q], r = mass_s[3 * N + q];
                e = 0.5 * (d0 * (quad(0, 0) + quad(1, 1)) + 2.0 * d1 * quad(0, 1) + d2 * quad(2, 2) +
                           r * (quad(3, 3) + quad(4, 4)));
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    __shared__ double ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
        partial[blockIdx.x] = s;
    }
}

__global__ void sum_kernel(const double* __restrict__ partial, int np, double* out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// Receivers: fluid [p, m_x, m_y, 0, 0]; solid [v_x, v_y, s_xx, s_yy, s_xy];
// interface [p_F, v_Fx, v_Fy, 0, 0] from the pointwise face solve.
// y = shot: state shot stride n_state, output shot stride 5 n_rec.
template <class T, class TO = T>
__global__ void record_kernel(DevOps op, int n_rec, const int32_t* __restrict__ ri, const double* __restrict__ rd,
                              const T* __restrict__ state, int64_t n_state, TO* out,
                              const StageClock* clock = nullptr) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rec) return;
    const int n = op.n;
    const int stride = 2 * n + 15;
    const double* d = rd + (size_t)r * stride;
    const int kind = ri[4 * r], qf = ri[4 * r + 1], qs = ri[4 * r + 2];
    const T* sf = state + (size_t)blockIdx.y * n_state;
    const T* ss = sf + (size_t)3 * n * op.Nf;
    auto ev = [&](const T* base, int N, int q, int field, const double* phi) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s = fma(phi[i], double(base[(size_t)(field * n + i) * N + q]), s);
        return s;
    };
    double o[5] = {0, 0, 0, 0, 0};
    if (kind == 0) {
        o[0] = ev(sf, op.Nf, qf, 2, d);
        o[1] = ev(sf, op.Nf, qf, 0, d);
        o[2] = ev(sf, op.Nf, qf, 1, d);
    } else if (kind == 1) {
        o[0] = ev(ss, op.Ns, qs, 3, d);
        o[1] = ev(ss, op.Ns, qs, 4, d);
        o[2] = ev(ss, op.Ns, qs, 0, d);
        o[3] = ev(ss, op.Ns, qs, 1, d);
        o[4] = ev(ss, op.Ns, qs, 2, d);
    } else {
        const double* pf = d;
        const double* ps = d + n;
        const double tf = d[2 * n], ts = d[2 * n + 1];
        const double nfx = d[2 * n + 2], nfy = d[2 * n + 3], nsx = d[2 * n + 4], nsy = d[2 * n + 5];
        const double* Ai = d + 2 * n + 6;
        const double p = ev(sf, op.Nf, qf, 2, pf), mx = ev(sf, op.Nf, qf, 0, pf), my = ev(sf, op.Nf, qf, 1, pf);
        const double sxx = ev(ss, op.Ns, qs, 0, ps), syy = ev(ss, op.Ns, qs, 1, ps), sxy = ev(ss, op.Ns, qs, 2, ps);
        const double vx = ev(ss, op.Ns, qs, 3, ps), vy = ev(ss, op.Ns, qs, 4, ps);
        const double wf = tf * p - (mx * nfx + my * nfy);
        const double wsx = ts * vx - (sxx * nsx + sxy * nsy);
        const double wsy = ts * vy - (sxy * nsx + syy * nsy);
        o[0] = Ai[0] * wf + Ai[1] * wsx + Ai[2] * wsy;
        o[1] = Ai[3] * wf + Ai[4] * wsx + Ai[5] * wsy;
        o[2] = Ai[6] * wf + Ai[7] * wsx + Ai[8] * wsy;
    }
    // with a device clock (graph replay) out is the trace base, offset by the step
    if (clock) out += (size_t)clock->step * 5 * n_rec * gridDim.y;
    TO* ob = out + (size_t)blockIdx.y * 5 * n_rec + 5 * r;
    for (int j = 0; j < 5; ++j) ob[j] = TO(o[j]);
}

template <class T, int K, int MODE>
void launch_kk(const StageArgsT<T>& a, dim3 grid, cudaStream_t s) {
    const size_t smem = stage_smem_bytes<T, K>(a.op.max_nf);
    if (smem > 48 * 1024) {
        // the opt-in is per function and device; remember the largest size set
        static size_t opted[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64 || opted[dev] < smem) {
            cudaFuncSetAttribute(stage_kernel<T, K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (dev >= 0 && dev < 64) opted[dev] = smem;
        }
    }
    if constexpr (AccSmem<T, K>::value) {
        // the accumulators need the largest shared-memory carveout for the
        // resident blocks the register budget allows
        static bool carved[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64 || !carved[dev]) {
            cudaFuncSetAttribute(stage_kernel<T, K, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
            if (dev >= 0 && dev < 64) carved[dev] = true;
        }
    }
    stage_kernel<T, K, MODE><<<grid, 128, smem, s>>>(a);
}

template <class T, int MODE>
void launch_k(int k, const StageArgsT<T>& a, dim3 grid, cudaStream_t s) {
    if (k == 1) launch_kk<T, 1, MODE>(a, grid, s);
    else if (k == 2) launch_kk<T, 2, MODE>(a, grid, s);
    else launch_kk<T, 3, MODE>(a, grid, s);
}

// The tensor-core stage (HHO_BF16X3): 32 consecutive cells of one class
// (a class run is padded to 32 cells) times 4 shots per block, so that each
// warp reads 32 consecutive cells of one shot, as the FP32 kernel does.
template <int K, int MODE>
void launch_tc_k(const hho_ops* ops, const StageArgsT<float>& a, int n_shots, cudaStream_t s) {
    const int C = 32, S_blk = 128 / C;
    const dim3 grid((unsigned)((ops->dev.Nf + ops->dev.Ns) / C), (unsigned)((n_shots + S_blk - 1) / S_blk));
    if (grid.x == 0) return;
    TcArgs T;
    T.tiles = (const uint4*)ops->d_tc_b;
    T.meta = ops->d_tc_meta;
    T.C = C;
    T.S_blk = S_blk;
    T.n_shots = n_shots;
    T.kmax = ops->tc_kmax;
    T.cols = ops->tc_cols;
    T.error = ops->d_tc_err;
    const size_t smem = (size_t)2 * 2 * 128 * ops->tc_kmax + (size_t)ops->tc_bmax;
    static size_t opted[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (smem > 48 * 1024 && (dev < 0 || dev >= 64 || opted[dev] < smem)) {
        cudaFuncSetAttribute(stage_tc_kernel<K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (dev >= 0 && dev < 64) opted[dev] = smem;
    }
    stage_tc_kernel<K, MODE><<<grid, 128, smem, s>>>(a, T);
}

// A stage launch of erk_run: the tensor-core stage when the batched call
// asked for HHO_BF16X3, else the stage kernel of the arithmetic.
template <class T, int MODE>
void launch_stage(const hho_ops* ops, const StageArgsT<T>& a, dim3 grid, int n_shots, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        if (ops->tc_on) {
            if (ops->k == 1) launch_tc_k<1, MODE>(ops, a, n_shots, s);
            else if (ops->k == 2) launch_tc_k<2, MODE>(ops, a, n_shots, s);
            else launch_tc_k<3, MODE>(ops, a, n_shots, s);
            return;
        }
    }
    launch_k<T, MODE>(ops->k, a, grid, s);
}

}  // namespace

int build_plan(const hho_tableau* tab, std::vector<StagePlan>& plan, int* n_buf) {
    const int s = tab->s;
    if (s < 1 || s > 6) return HHO_EINVAL;
    auto coef = [&](int i, int j) { return i == s ? tab->b[j] : tab->a[i][j]; };
    std::vector<int> buf(s + 1, -1);      // row -> buffer index
    std::vector<bool> touched(s + 1, false);
    int nb = 0;
    plan.assign(s, StagePlan{});
    for (int j = 0; j < s; ++j) {
        StagePlan& P = plan[j];
        P.n_tgt = 0;
        const int r0 = j + 1;
        TargetPlan t0;
        t0.src = touched[r0] ? buf[r0] : SRC_STATE;
        t0.dst = (r0 == s) ? SRC_STATE : SRC_X;
        t0.a = coef(r0, j);
        P.t[P.n_tgt++] = t0;
        for (int i = j + 2; i <= s; ++i) {
            const double a = coef(i, j);
            if (a == 0.0) continue;
            if (P.n_tgt >= MAX_TARGETS) return HHO_EINVAL;
            if (buf[i] < 0) buf[i] = nb++;
            TargetPlan t;
            t.src = touched[i] ? buf[i] : SRC_STATE;
            t.dst = buf[i];
            t.a = a;
            touched[i] = true;
            P.t[P.n_tgt++] = t;
        }
    }
    *n_buf = nb;
    return HHO_OK;
}

namespace {

int64_t n_energy_blocks(const hho_ops* ops) { return ((int64_t)ops->dev.Nf + ops->dev.Ns + 255) / 256 + 1; }

double ricker(double t, double f0, double t0, double amp) {
    const double a = M_PI * f0 * (t - t0);
    const double a2 = a * a;
    return amp * (1.0 - 2.0 * a2) * std::exp(-a2);
}

int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        hho_set_error("%s: %s", what, cudaGetErrorString(e));
        return HHO_ECUDA;
    }
    return HHO_OK;
}

template <class T>
const T* src_g_of(const hho_ops* ops);
template <>
const double* src_g_of<double>(const hho_ops* ops) { return ops->d_src_g; }
template <>
const float* src_g_of<float>(const hho_ops* ops) { return ops->d_src_g32; }
template <>
const f2x* src_g_of<f2x>(const hho_ops* ops) { return ops->d_src_gx; }
template <class T>
const T* shot_g_of(const hho_ops* ops);
template <>
const double* shot_g_of<double>(const hho_ops* ops) { return ops->d_shot_src_g; }
template <>
const float* shot_g_of<float>(const hho_ops* ops) { return ops->d_shot_src_g32; }
template <>
const f2x* shot_g_of<f2x>(const hho_ops* ops) { return ops->d_shot_src_gx; }

// Value of point source s for the stage of step time tn, stage j (time
// tn + cdt): its Ricker wavelet, or, for a sampled time function, the sample
// of step round((tn - t_start) / dt) and stage j (zero outside the sampled
// steps and for j < 0, a call with no stage index).
double source_value(const hho_ops* ops, int s, double tn, int j, double cdt) {
    if (!ops->src_sampled) return ricker(tn + cdt, ops->src_f0[s], ops->src_t0[s], ops->src_amp[s]);
    if (j < 0 || j >= ops->samp_s) return 0.0;
    const int64_t n = std::llround((tn - ops->samp_t0) / ops->samp_dt);
    if (n < 0 || n >= ops->samp_n) return 0.0;
    return ops->src_samples[((size_t)s * ops->samp_n + n) * ops->samp_s + j];
}

template <class T>
void fill_sources(const hho_ops* ops, StageArgsT<T>& a, double tn, int j, double cdt, int n_shots) {
    a.n_src = ops->n_src;
    a.src_g = src_g_of<T>(ops);
    for (int s = 0; s < ops->n_src; ++s) {
        a.src_dom[s] = ops->src_dom[s];
        a.src_q[s] = ops->src_q[s];
        a.src_w[s] = T(source_value(ops, s, tn, j, cdt));
    }
    if (ops->n_shot_src > 0 && n_shots <= ops->n_shot_src) {
        a.shot_src_dom = ops->d_shot_src_dom;
        a.shot_src_q = ops->d_shot_src_q;
        a.shot_src_g = shot_g_of<T>(ops);
        a.shot_src_w = T(ricker(tn + cdt, ops->shot_f0, ops->shot_t0, ops->shot_amp));
    } else {
        a.shot_src_dom = nullptr;
        a.shot_src_q = nullptr;
        a.shot_src_g = nullptr;
        a.shot_src_w = T(0);
    }
}

}  // namespace

extern "C" int hho_ricker_samples(const hho_tableau* tab, double t_start, double dt, int64_t nsteps, double f0,
                                  double t0, double amp, double* h_out) {
    if (!tab || tab->s < 1 || tab->s > 6 || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt) ||
        !std::isfinite(t_start) || !(f0 > 0.0) || (nsteps > 0 && !h_out)) {
        hho_set_error("hho_ricker_samples: bad arguments");
        return HHO_EINVAL;
    }
    // the same rounded stage times as the ERK loops: (t_start + n dt) + c_j dt
    for (int64_t n = 0; n < nsteps; ++n) {
        const double tn = t_start + (double)n * dt;
        for (int j = 0; j < tab->s; ++j) h_out[n * tab->s + j] = ricker(tn + tab->c[j] * dt, f0, t0, amp);
    }
    return HHO_OK;
}

extern "C" int hho_work_size(const hho_ops* ops, const hho_tableau* tab, int64_t* out) {
    if (!ops || !tab || !out) {
        hho_set_error("hho_work_size: null pointer");
        return HHO_EINVAL;
    }
    std::vector<StagePlan> plan;
    int nb = 0;
    if (build_plan(tab, plan, &nb) != HHO_OK) {
        hho_set_error("hho_work_size: unsupported tableau");
        return HHO_EINVAL;
    }
    *out = ops->n_state * (2 + nb) + 2 * ops->trace_doubles + n_energy_blocks(ops) + 8;
    return HHO_OK;
}

namespace {
__global__ void clock_set_kernel(StageClock* c, double t0) {
    c->t0 = t0;
    c->step = 0;
}
__global__ void clock_advance_kernel(StageClock* c) { c->step += 1; }

// Sources for a stage evaluated from the device clock (graph replay).
template <class T>
void fill_sources_clock(const hho_ops* ops, StageArgsT<T>& a, double c_stage, double dt, int n_shots) {
    fill_sources<T>(ops, a, 0.0, -1, 0.0, n_shots);   // cells, vectors and pointers
    for (int s = 0; s < MAX_SOURCES; ++s) a.src_w[s] = T(0);
    a.shot_src_w = T(0);
    a.clock = ops->d_clock;
    a.dt = dt;
    a.c_stage = c_stage;
    for (int s = 0; s < ops->n_src; ++s) {
        a.src_f0[s] = ops->src_f0[s];
        a.src_t0[s] = ops->src_t0[s];
        a.src_amp[s] = ops->src_amp[s];
    }
    if (a.shot_src_q) {
        a.shot_f0 = ops->shot_f0;
        a.shot_t0 = ops->shot_t0;
        a.shot_amp = ops->shot_amp;
    }
}

template <class V>
void append_bytes(std::vector<unsigned char>& key, const V& v) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    key.insert(key.end(), p, p + sizeof(V));
}
}  // namespace

// Time stepping for n_shots states of element type T.  Work layout (elements
// of T): [X: S n_state][partial sums: nb S n_state][traces: 2 x S trace].
template <class T>
struct SeisOf {   // element type of recorded traces: the state's, FP64 for double-float
    using type = T;
};
template <>
struct SeisOf<f2x> {
    using type = double;
};

template <class T>
static int erk_run(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps, int n_shots,
                   T* d_state, T* d_work, void* d_seis_v, void* stream, const char* who) {
    using TS = typename SeisOf<T>::type;
    TS* d_seis = (TS*)d_seis_v;
    if (!ops || !tab || !d_state || !d_work || nsteps < 0 || n_shots < 1 || n_shots > 65535 || !std::isfinite(dt) ||
        !std::isfinite(t0)) {
        hho_set_error("%s: bad arguments", who);
        return HHO_EINVAL;
    }
    std::vector<StagePlan> plan;
    int nb = 0;
    if (build_plan(tab, plan, &nb) != HHO_OK) {
        hho_set_error("%s: unsupported tableau (s <= 6, at most %d partial sums per stage)", who, MAX_TARGETS);
        return HHO_EINVAL;
    }
    if (nsteps == 0) return HHO_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t S = ops->n_state * n_shots;
    const int64_t TRS = ops->trace_doubles * n_shots;
    T* X = d_work;
    T* bufs = d_work + S;
    T* tr[2] = {d_work + S * (1 + nb), d_work + S * (1 + nb) + TRS};
    const dim3 grid((ops->dev.Nf + ops->dev.Ns + 127) / 128, n_shots);
    if (grid.x == 0) return HHO_OK;
    auto resolve = [&](int code) -> T* {
        if (code == SRC_STATE) return d_state;
        if (code == SRC_X) return X;
        if (code == SRC_ZERO) return nullptr;
        return bufs + S * code;
    };
    StageArgsT<T> a;
    memset(&a, 0, sizeof(a));
    a.op = ops->dev;
    a.state_stride = ops->n_state;
    a.trace_stride = ops->trace_doubles;
    a.inp = d_state;
    a.tr_out = tr[0];
    a.n_tgt = 0;
    const bool use_graph =
        !ops->prof_on && ops->d_clock && !ops->src_sampled &&
        (ops->launch_mode == HHO_LAUNCH_GRAPH ||
         (ops->launch_mode == HHO_LAUNCH_AUTO && (int64_t)grid.x * n_shots <= 2048 && nsteps >= 8));
    launch_stage<T, MODE_TRACES>(ops, a, grid, n_shots, st);
    int rc = check_launch(who);
    if (rc) return rc;
    int cur = 0;
    if (use_graph) {
        // One step = its stage kernels, the receiver record and the clock
        // increment, captured once per distinct set of arguments (two sets
        // when an odd stage count alternates the trace buffers) and replayed.
        clock_set_kernel<<<1, 1, 0, st>>>(ops->d_clock, t0);
        rc = check_launch(who);
        if (rc) return rc;
        const bool rec = d_seis && ops->n_rec > 0;
        const dim3 rgrid((ops->n_rec + 63) / 64, n_shots);
        cudaGraphExec_t execs[2] = {nullptr, nullptr};
        for (int par = 0; par < ((tab->s & 1) ? 2 : 1); ++par) {
            std::vector<StageArgsT<T>> args(tab->s);
            int c2 = par;
            std::vector<unsigned char> key;
            append_bytes(key, (int)sizeof(T));
            append_bytes(key, ops->tc_on);
            append_bytes(key, grid);
            for (int j = 0; j < tab->s; ++j) {
                StageArgsT<T>& b = args[j];
                b = a;
                const StagePlan& P = plan[j];
                b.inp = (j == 0) ? d_state : X;
                b.tr_in = tr[c2];
                b.tr_out = tr[c2 ^ 1];
                b.n_tgt = P.n_tgt;
                for (int t = 0; t < P.n_tgt; ++t) {
                    b.tgt[t].src = resolve(P.t[t].src);
                    b.tgt[t].dst = resolve(P.t[t].dst);
                    b.tgt[t].coef = T(P.t[t].a * dt);
                }
                fill_sources_clock<T>(ops, b, tab->c[j], dt, n_shots);
                append_bytes(key, b);
                c2 ^= 1;
            }
            append_bytes(key, rec ? (const void*)d_seis : nullptr);
            append_bytes(key, ops->d_rec_int);
            append_bytes(key, ops->d_rec_dbl);
            append_bytes(key, ops->n_rec);
            cudaGraphExec_t found = nullptr;
            for (auto& g : ops->graphs)
                if (g.key == key) found = (cudaGraphExec_t)g.exec;
            if (!found) {
                if (!ops->cap_stream) {
                    cudaStream_t cs;
                    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
                        hho_set_error("%s: capture stream creation failed", who);
                        return HHO_ECUDA;
                    }
                    ops->cap_stream = (void*)cs;
                }
                cudaStream_t cs = (cudaStream_t)ops->cap_stream;
                cudaGraph_t graph = nullptr;
                if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                    hho_set_error("%s: stream capture failed to start", who);
                    return HHO_ECUDA;
                }
                for (int j = 0; j < tab->s; ++j) launch_stage<T, MODE_STAGE>(ops, args[j], grid, n_shots, cs);
                if (rec)
                    record_kernel<T, TS><<<rgrid, 64, 0, cs>>>(ops->dev, ops->n_rec, ops->d_rec_int, ops->d_rec_dbl,
                                                             d_state, ops->n_state, d_seis, ops->d_clock);
                clock_advance_kernel<<<1, 1, 0, cs>>>(ops->d_clock);
                const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
                if (ce != cudaSuccess || !graph || cudaGraphInstantiate(&found, graph, 0) != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    cudaGetLastError();
                    hho_set_error("%s: step graph capture or instantiation failed", who);
                    return HHO_ECUDA;
                }
                cudaGraphDestroy(graph);
                if (ops->graphs.size() >= 8) {
                    cudaGraphExecDestroy((cudaGraphExec_t)ops->graphs.front().exec);
                    ops->graphs.erase(ops->graphs.begin());
                }
                ops->graphs.push_back({key, (void*)found});
            }
            execs[par] = found;
        }
        for (int64_t step = 0; step < nsteps; ++step) {
            if (cudaGraphLaunch(execs[(tab->s & 1) ? (int)(step & 1) : 0], st) != cudaSuccess) {
                hho_set_error("%s: graph launch failed", who);
                return HHO_ECUDA;
            }
        }
        return check_launch(who);
    }
    for (int64_t step = 0; step < nsteps; ++step) {
        const double tn = t0 + (double)step * dt;
        for (int j = 0; j < tab->s; ++j) {
            const StagePlan& P = plan[j];
            a.inp = (j == 0) ? d_state : X;
            a.tr_in = tr[cur];
            a.tr_out = tr[cur ^ 1];
            a.n_tgt = P.n_tgt;
            for (int t = 0; t < P.n_tgt; ++t) {
                a.tgt[t].src = resolve(P.t[t].src);
                a.tgt[t].dst = resolve(P.t[t].dst);
                a.tgt[t].coef = T(P.t[t].a * dt);
            }
            fill_sources<T>(ops, a, tn, j, tab->c[j] * dt, n_shots);
            const bool prof = ops->prof_on && 2 * ops->prof_n + 1 < (int)ops->prof_events.size();
            if (prof) cudaEventRecord((cudaEvent_t)ops->prof_events[2 * ops->prof_n], st);
            launch_stage<T, MODE_STAGE>(ops, a, grid, n_shots, st);
            if (prof) cudaEventRecord((cudaEvent_t)ops->prof_events[2 * ops->prof_n++ + 1], st);
            rc = check_launch(who);
            if (rc) return rc;
            cur ^= 1;
        }
        if (d_seis && ops->n_rec > 0) {
            record_kernel<T, TS><<<dim3((ops->n_rec + 63) / 64, n_shots), 64, 0, st>>>(
                ops->dev, ops->n_rec, ops->d_rec_int, ops->d_rec_dbl, d_state, ops->n_state,
                d_seis + (size_t)step * 5 * ops->n_rec * n_shots);
            rc = check_launch(who);
            if (rc) return rc;
        }
    }
    return HHO_OK;
}

// Doubles of the FP64 work layout [X][partial sums][2 traces][energy scratch];
// hho_work_size adds one state of double-float pairs after it.
static int64_t work_f64_part(const hho_ops* ops, int nb) {
    return ops->n_state * (1 + nb) + 2 * ops->trace_doubles + n_energy_blocks(ops) + 8;
}

namespace {
__global__ void to_pairs_kernel(const double* __restrict__ x, f2x* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = f2x(x[i]);
}
__global__ void from_pairs_kernel(const f2x* __restrict__ x, double* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = double(x[i]);
}
int pairs_grid(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }
}  // namespace

// Single-shot stepping: FP64, or double-float on a pair copy of the state
// kept at the end of the work buffer (converted in and out once per call).
static int erk_single(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps, double* d_state,
                      double* d_work, double* d_seis, void* stream, const char* who) {
    if (!ops || ops->arith != HHO_F32X2)
        return erk_run<double>(ops, tab, t0, dt, nsteps, 1, d_state, d_work, d_seis, stream, who);
    std::vector<StagePlan> plan;
    int nb = 0;
    if (!tab || !d_state || !d_work || build_plan(tab, plan, &nb) != HHO_OK) {
        hho_set_error("%s: bad arguments", who);
        return HHO_EINVAL;
    }
    if (nsteps <= 0 || ops->n_state == 0)
        return erk_run<f2x>(ops, tab, t0, dt, nsteps, 1, (f2x*)d_state, (f2x*)d_work, d_seis, stream, who);
    cudaStream_t st = (cudaStream_t)stream;
    f2x* ux = (f2x*)(d_work + work_f64_part(ops, nb));
    to_pairs_kernel<<<pairs_grid(ops->n_state), 256, 0, st>>>(d_state, ux, ops->n_state);
    int rc = check_launch(who);
    if (rc) return rc;
    rc = erk_run<f2x>(ops, tab, t0, dt, nsteps, 1, ux, (f2x*)d_work, d_seis, stream, who);
    if (rc) return rc;
    from_pairs_kernel<<<pairs_grid(ops->n_state), 256, 0, st>>>(ux, d_state, ops->n_state);
    return check_launch(who);
}

// hho_erk_run_host on a pinned, mapped host buffer: the state is packed
// from the host buffer straight into the arithmetic's device state (the
// double-float pair copy, or the FP64 state), stepped, and unpacked
// straight back, with no device copy of the canonical vector.
static int erk_run_mapped(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps,
                          double* m_canonical, cudaStream_t st) {
    const char* who = "hho_erk_run_host";
    std::vector<StagePlan> plan;
    int nb = 0;
    if (build_plan(tab, plan, &nb) != HHO_OK) {
        hho_set_error("%s: unsupported tableau", who);
        return HHO_EINVAL;
    }
    const int nc = (int)ops->nc;
    if (nc == 0) return HHO_OK;
    const int blocks = (nc + STAGED_CELLS - 1) / STAGED_CELLS;
    const size_t smem = sizeof(double) * STAGED_CELLS * 5 * ops->n;
    const bool pairs = ops->arith == HHO_F32X2;
    void* dst = pairs ? (void*)(ops->d_host_work + work_f64_part(ops, nb)) : (void*)ops->d_host_state;
    if (pairs)
        pack_host_kernel<f2x><<<blocks, STAGED_CELLS, smem, st>>>(ops->d_cell_dom, ops->d_cell_pos, ops->d_canon_off, nc,
                                                                   ops->n_canonical, ops->dev.Nf, ops->dev.Ns, ops->n,
                                                                   m_canonical, (f2x*)dst);
    else
        pack_host_kernel<double><<<blocks, STAGED_CELLS, smem, st>>>(ops->d_cell_dom, ops->d_cell_pos, ops->d_canon_off,
                                                                      nc, ops->n_canonical, ops->dev.Nf, ops->dev.Ns,
                                                                      ops->n, m_canonical, (double*)dst);
    int rc = check_launch(who);
    if (rc) return rc;
    rc = pairs ? erk_run<f2x>(ops, tab, t0, dt, nsteps, 1, (f2x*)dst, (f2x*)ops->d_host_work, nullptr, st, who)
               : erk_run<double>(ops, tab, t0, dt, nsteps, 1, (double*)dst, ops->d_host_work, nullptr, st, who);
    if (rc) return rc;
    if (pairs)
        unpack_host_kernel<f2x><<<blocks, STAGED_CELLS, smem, st>>>(ops->d_cell_dom, ops->d_cell_pos, ops->d_canon_off,
                                                                     nc, ops->n_canonical, ops->dev.Nf, ops->dev.Ns,
                                                                     ops->n, (const f2x*)dst, m_canonical);
    else
        unpack_host_kernel<double><<<blocks, STAGED_CELLS, smem, st>>>(ops->d_cell_dom, ops->d_cell_pos,
                                                                        ops->d_canon_off, nc, ops->n_canonical,
                                                                        ops->dev.Nf, ops->dev.Ns, ops->n,
                                                                        (const double*)dst, m_canonical);
    return check_launch(who);
}

extern "C" int hho_set_launch_mode(hho_ops* ops, int32_t mode) {
    if (!ops || (mode != HHO_LAUNCH_STREAM && mode != HHO_LAUNCH_GRAPH && mode != HHO_LAUNCH_AUTO)) {
        hho_set_error("hho_set_launch_mode: mode must be HHO_LAUNCH_STREAM, HHO_LAUNCH_GRAPH or HHO_LAUNCH_AUTO");
        return HHO_EINVAL;
    }
    ops->launch_mode = mode;
    return HHO_OK;
}

extern "C" int hho_set_arithmetic(hho_ops* ops, int32_t arith) {
    if (!ops || (arith != HHO_F64 && arith != HHO_F32X2)) {
        hho_set_error("hho_set_arithmetic: arith must be HHO_F64 or HHO_F32X2");
        return HHO_EINVAL;
    }
    ops->arith = arith;
    return HHO_OK;
}

extern "C" int hho_erk_step(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps,
                            double* d_state, double* d_work, void* stream) {
    return erk_single(ops, tab, t0, dt, nsteps, d_state, d_work, nullptr, stream, "hho_erk_step");
}

extern "C" int hho_erk_step_record(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps,
                                   double* d_state, double* d_work, double* d_seismogram, void* stream) {
    if (ops && ops->n_rec > 0 && !d_seismogram) {
        hho_set_error("hho_erk_step_record: null seismogram buffer");
        return HHO_EINVAL;
    }
    return erk_single(ops, tab, t0, dt, nsteps, d_state, d_work, d_seismogram, stream, "hho_erk_step_record");
}

// ---- one stage at a time (drivers that exchange halos between stages) ---------------
// The same kernel arguments as erk_run's stream path, so a sequence
// hho_erk_traces, hho_erk_stage(n, j) for n < nsteps, j < s reproduces
// hho_erk_step in stream launch mode bit for bit.

namespace {
__global__ void halo_gather_kernel(const double* __restrict__ src, const int64_t* __restrict__ idx, int64_t n,
                                   double* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}
__global__ void halo_scatter_kernel(const double* __restrict__ src, const int64_t* __restrict__ idx, int64_t n,
                                    double* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[idx[i]] = src[i];
}
}  // namespace

static int stage_api_check(const hho_ops* ops, const hho_tableau* tab, const void* d_state, const void* d_work,
                           std::vector<StagePlan>& plan, int* nb, const char* who) {
    if (!ops || !tab || !d_state || !d_work) {
        hho_set_error("%s: null pointer", who);
        return HHO_EINVAL;
    }
    if (ops->arith != HHO_F64) {
        hho_set_error("%s: the stage-at-a-time entry points run the FP64 arithmetic only", who);
        return HHO_EINVAL;
    }
    if (build_plan(tab, plan, nb) != HHO_OK) {
        hho_set_error("%s: unsupported tableau", who);
        return HHO_EINVAL;
    }
    return HHO_OK;
}

extern "C" int hho_trace_buffer_offset(const hho_ops* ops, const hho_tableau* tab, int32_t which, int64_t* offset) {
    std::vector<StagePlan> plan;
    int nb = 0;
    if (!ops || !tab || !offset || (which != 0 && which != 1) || build_plan(tab, plan, &nb) != HHO_OK) {
        hho_set_error("hho_trace_buffer_offset: bad arguments");
        return HHO_EINVAL;
    }
    *offset = ops->n_state * (1 + nb) + (int64_t)which * ops->trace_doubles;
    return HHO_OK;
}

extern "C" int hho_erk_traces(hho_ops* ops, const hho_tableau* tab, const double* d_state, double* d_work,
                              void* stream) {
    std::vector<StagePlan> plan;
    int nb = 0;
    int rc = stage_api_check(ops, tab, d_state, d_work, plan, &nb, "hho_erk_traces");
    if (rc) return rc;
    const dim3 grid((ops->dev.Nf + ops->dev.Ns + 127) / 128, 1);
    if (grid.x == 0) return HHO_OK;
    StageArgsT<double> a;
    memset(&a, 0, sizeof(a));
    a.op = ops->dev;
    a.state_stride = ops->n_state;
    a.trace_stride = ops->trace_doubles;
    a.inp = d_state;
    a.tr_out = d_work + ops->n_state * (1 + nb);
    launch_k<double, MODE_TRACES>(ops->k, a, grid, (cudaStream_t)stream);
    return check_launch("hho_erk_traces");
}

extern "C" int hho_erk_stage(hho_ops* ops, const hho_tableau* tab, int64_t n, int32_t j, double tn, double dt,
                             double* d_state, double* d_work, void* stream) {
    std::vector<StagePlan> plan;
    int nb = 0;
    int rc = stage_api_check(ops, tab, d_state, d_work, plan, &nb, "hho_erk_stage");
    if (rc) return rc;
    if (n < 0 || j < 0 || j >= tab->s || !std::isfinite(tn) || !std::isfinite(dt)) {
        hho_set_error("hho_erk_stage: bad step or stage index");
        return HHO_EINVAL;
    }
    const dim3 grid((ops->dev.Nf + ops->dev.Ns + 127) / 128, 1);
    if (grid.x == 0) return HHO_OK;
    const int64_t S = ops->n_state;
    double* X = d_work;
    double* bufs = d_work + S;
    double* tr[2] = {d_work + S * (1 + nb), d_work + S * (1 + nb) + ops->trace_doubles};
    const int cur = (int)((n * tab->s + j) & 1);
    auto resolve = [&](int code) -> double* {
        if (code == SRC_STATE) return d_state;
        if (code == SRC_X) return X;
        if (code == SRC_ZERO) return nullptr;
        return bufs + S * code;
    };
    StageArgsT<double> a;
    memset(&a, 0, sizeof(a));
    a.op = ops->dev;
    a.state_stride = ops->n_state;
    a.trace_stride = ops->trace_doubles;
    const StagePlan& P = plan[j];
    a.inp = (j == 0) ? d_state : X;
    a.tr_in = tr[cur];
    a.tr_out = tr[cur ^ 1];
    a.n_tgt = P.n_tgt;
    for (int t = 0; t < P.n_tgt; ++t) {
        a.tgt[t].src = resolve(P.t[t].src);
        a.tgt[t].dst = resolve(P.t[t].dst);
        a.tgt[t].coef = P.t[t].a * dt;
    }
    fill_sources<double>(ops, a, tn, j, tab->c[j] * dt, 1);
    launch_k<double, MODE_STAGE>(ops->k, a, grid, (cudaStream_t)stream);
    return check_launch("hho_erk_stage");
}

extern "C" int hho_trace_offsets(const hho_ops* ops, int64_t n, const int64_t* h_cells, const int32_t* h_faces,
                                 int64_t* h_out) {
    if (!ops || n < 0 || (n > 0 && (!h_cells || !h_faces || !h_out))) {
        hho_set_error("hho_trace_offsets: bad arguments");
        return HHO_EINVAL;
    }
    const int f = ops->f;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t c = h_cells[i];
        if (c < 0 || c >= ops->nc) {
            hho_set_error("hho_trace_offsets: cell %lld out of range", (long long)c);
            return HHO_EINVAL;
        }
        const int32_t* ci = &ops->h_cls_int[ops->cell_class_of[c] * CI_STRIDE];
        const int j = h_faces[i];
        if (j < 0 || j >= ci[CI_NF]) {
            hho_set_error("hho_trace_offsets: cell %lld has no local face %d", (long long)c, j);
            return HHO_EINVAL;
        }
        const int64_t slot = ci[CI_SLOT] + (int64_t)j * ci[CI_NPAD] + (ops->cell_pos[c] - ci[CI_START]);
        int64_t* o = h_out + i * 2 * f;
        if (ops->cell_dom[c] == 0) {
            for (int l = 0; l < f; ++l) o[l] = (int64_t)l * ops->dev.SF + slot;
            for (int l = f; l < 2 * f; ++l) o[l] = -1;
        } else {
            const int64_t base = (int64_t)2 * f * ops->dev.SF;
            for (int l = 0; l < 2 * f; ++l) o[l] = base + (int64_t)l * ops->dev.SS + slot;
        }
    }
    return HHO_OK;
}

extern "C" int hho_halo_gather(const double* d_src, const int64_t* d_idx, int64_t n, double* d_dst, void* stream) {
    if (n < 0 || (n > 0 && (!d_src || !d_idx || !d_dst))) {
        hho_set_error("hho_halo_gather: bad arguments");
        return HHO_EINVAL;
    }
    if (n == 0) return HHO_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    halo_gather_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d_src, d_idx, n, d_dst);
    return check_launch("hho_halo_gather");
}

extern "C" int hho_halo_scatter(const double* d_src, const int64_t* d_idx, int64_t n, double* d_dst, void* stream) {
    if (n < 0 || (n > 0 && (!d_src || !d_idx || !d_dst))) {
        hho_set_error("hho_halo_scatter: bad arguments");
        return HHO_EINVAL;
    }
    if (n == 0) return HHO_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    halo_scatter_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d_src, d_idx, n, d_dst);
    return check_launch("hho_halo_scatter");
}

// ---- batched shots -----------------------------------------------------------------

static bool batch_args_ok(const hho_ops* ops, int32_t n_shots, int32_t precision, const char* who) {
    if (!ops || n_shots < 1 || n_shots > 65535 ||
        (precision != HHO_F64 && precision != HHO_F32 && precision != HHO_F32X2 && precision != HHO_BF16X3)) {
        hho_set_error("%s: bad arguments (1 <= n_shots <= 65535, precision HHO_F64, HHO_F32, HHO_F32X2 or HHO_BF16X3)",
                      who);
        return false;
    }
    return true;
}

extern "C" int hho_batch_sizes(const hho_ops* ops, const hho_tableau* tab, int32_t n_shots, int32_t precision,
                               int64_t* state_elems, int64_t* work_elems) {
    if (!batch_args_ok(ops, n_shots, precision, "hho_batch_sizes") || !tab) {
        if (!tab) hho_set_error("hho_batch_sizes: null tableau");
        return HHO_EINVAL;
    }
    std::vector<StagePlan> plan;
    int nb = 0;
    if (build_plan(tab, plan, &nb) != HHO_OK) {
        hho_set_error("hho_batch_sizes: unsupported tableau");
        return HHO_EINVAL;
    }
    if (state_elems) *state_elems = ops->n_state * n_shots;
    if (work_elems) *work_elems = (ops->n_state * (1 + nb) + 2 * ops->trace_doubles) * n_shots;
    return HHO_OK;
}

extern "C" int hho_batch_pack(const hho_ops* ops, int32_t n_shots, int32_t precision, const double* d_canonical,
                              void* d_state, void* stream) {
    if (!batch_args_ok(ops, n_shots, precision, "hho_batch_pack") || !d_canonical || !d_state) {
        if (ops) hho_set_error("hho_batch_pack: bad arguments");
        return HHO_EINVAL;
    }
    const int tot = ops->dev.Nf + ops->dev.Ns;
    if (tot == 0) return HHO_OK;
    const dim3 grid((tot + 127) / 128, n_shots);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == HHO_F64)
        pack_kernel<double><<<grid, 128, 0, st>>>(ops->d_dev2orig, ops->d_canon_off, ops->dev.Nf, ops->dev.Ns, ops->n,
                                                  ops->n_canonical, ops->n_state, d_canonical, (double*)d_state);
    else if (precision == HHO_F32X2)
        pack_kernel<f2x><<<grid, 128, 0, st>>>(ops->d_dev2orig, ops->d_canon_off, ops->dev.Nf, ops->dev.Ns, ops->n,
                                               ops->n_canonical, ops->n_state, d_canonical, (f2x*)d_state);
    else
        pack_kernel<float><<<grid, 128, 0, st>>>(ops->d_dev2orig, ops->d_canon_off, ops->dev.Nf, ops->dev.Ns, ops->n,
                                                 ops->n_canonical, ops->n_state, d_canonical, (float*)d_state);
    return check_launch("hho_batch_pack");
}

extern "C" int hho_batch_unpack(const hho_ops* ops, int32_t n_shots, int32_t precision, const void* d_state,
                                double* d_canonical, void* stream) {
    if (!batch_args_ok(ops, n_shots, precision, "hho_batch_unpack") || !d_canonical || !d_state) {
        if (ops) hho_set_error("hho_batch_unpack: bad arguments");
        return HHO_EINVAL;
    }
    const int tot = ops->dev.Nf + ops->dev.Ns;
    if (tot == 0) return HHO_OK;
    const dim3 grid((tot + 127) / 128, n_shots);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == HHO_F64)
        unpack_kernel<double><<<grid, 128, 0, st>>>(ops->d_dev2orig, ops->d_canon_off, ops->dev.Nf, ops->dev.Ns, ops->n,
                                                    ops->n_canonical, ops->n_state, (const double*)d_state, d_canonical);
    else if (precision == HHO_F32X2)
        unpack_kernel<f2x><<<grid, 128, 0, st>>>(ops->d_dev2orig, ops->d_canon_off, ops->dev.Nf, ops->dev.Ns, ops->n,
                                                 ops->n_canonical, ops->n_state, (const f2x*)d_state, d_canonical);
    else
        unpack_kernel<float><<<grid, 128, 0, st>>>(ops->d_dev2orig, ops->d_canon_off, ops->dev.Nf, ops->dev.Ns, ops->n,
                                                   ops->n_canonical, ops->n_state, (const float*)d_state, d_canonical);
    return check_launch("hho_batch_unpack");
}

extern "C" int hho_batch_erk_step(hho_ops* ops, const hho_tableau* tab, int32_t n_shots, int32_t precision, double t0,
                                  double dt, int64_t nsteps, void* d_state, void* d_work, void* d_seismogram,
                                  void* stream) {
    if (!batch_args_ok(ops, n_shots, precision, "hho_batch_erk_step")) return HHO_EINVAL;
    if (ops->n_shot_src > 0 && ops->n_shot_src < n_shots) {
        hho_set_error("hho_batch_erk_step: %d shot sources set for %d shots", ops->n_shot_src, n_shots);
        return HHO_EINVAL;
    }
    if (precision == HHO_F64)
        return erk_run<double>(ops, tab, t0, dt, nsteps, n_shots, (double*)d_state, (double*)d_work, d_seismogram,
                               stream, "hho_batch_erk_step");
    if (precision == HHO_F32X2)
        return erk_run<f2x>(ops, tab, t0, dt, nsteps, n_shots, (f2x*)d_state, (f2x*)d_work, d_seismogram, stream,
                            "hho_batch_erk_step");
    ops->tc_on = precision == HHO_BF16X3;
    const int rc = erk_run<float>(ops, tab, t0, dt, nsteps, n_shots, (float*)d_state, (float*)d_work, d_seismogram,
                                  stream, "hho_batch_erk_step");
    ops->tc_on = false;
    return rc;
}

extern "C" int hho_tc_error(hho_ops* ops, int32_t* h_flag) {
    if (!ops || !h_flag) {
        hho_set_error("hho_tc_error: null pointer");
        return HHO_EINVAL;
    }
    int32_t v = 0;
    if (cudaMemcpy(&v, ops->d_tc_err, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(ops->d_tc_err, 0, sizeof(v)) != cudaSuccess) {
        hho_set_error("hho_tc_error: copy failed");
        return HHO_ECUDA;
    }
    *h_flag = v;
    return HHO_OK;
}

extern "C" int hho_profile_enable(hho_ops* ops, int32_t on) {
    if (!ops) {
        hho_set_error("hho_profile_enable: null ops");
        return HHO_EINVAL;
    }
    if (on && ops->prof_events.empty()) {
        for (int i = 0; i < 8192; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) {
                hho_set_error("hho_profile_enable: cudaEventCreate failed");
                return HHO_ECUDA;
            }
            ops->prof_events.push_back((void*)e);
        }
    }
    ops->prof_on = on != 0;
    ops->prof_n = 0;
    return HHO_OK;
}

extern "C" int hho_profile_read(hho_ops* ops, double* ms, int64_t* n) {
    if (!ops || !ms || !n) {
        hho_set_error("hho_profile_read: null pointer");
        return HHO_EINVAL;
    }
    double tot = 0.0;
    for (int i = 0; i < ops->prof_n; ++i) {
        float t = 0.0f;
        if (cudaEventSynchronize((cudaEvent_t)ops->prof_events[2 * i + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&t, (cudaEvent_t)ops->prof_events[2 * i], (cudaEvent_t)ops->prof_events[2 * i + 1]) !=
                cudaSuccess) {
            hho_set_error("hho_profile_read: event query failed");
            return HHO_ECUDA;
        }
        tot += t;
    }
    *ms = tot;
    *n = ops->prof_n;
    ops->prof_n = 0;
    return HHO_OK;
}

// FP64 lane-ops of one stage thread, mirroring fluid_cell / solid_cell.
extern "C" int hho_stage_cost(const hho_ops* ops, const hho_tableau* tab, int64_t* fp64_ops, int64_t* bytes_min,
                              int64_t* bytes_kernel) {
    if (!ops || !tab) {
        hho_set_error("hho_stage_cost: null pointer");
        return HHO_EINVAL;
    }
    std::vector<StagePlan> plan;
    int nbuf = 0;
    if (build_plan(tab, plan, &nbuf) != HHO_OK) {
        hho_set_error("hho_stage_cost: unsupported tableau");
        return HHO_EINVAL;
    }
    const int K = ops->k, n = ops->n, f = ops->f;
    const int64_t dsm = (int64_t)K * (K - 1) / 2, dvalid = (int64_t)K * (K + 1) / 2;
    // entries of the rectangle parity patterns (the same count on every face);
    // a square's trace takes K(K+1)/2 multiply-adds (trace_square)
    int64_t rect_tr = 0, rect_lift = 0, square_lift = 0;
    const int64_t square_tr = (int64_t)K * (K + 1) / 2;
    for (int i = 0; i < n; ++i) {
        const int e = ea(i);
        for (int l = 0; l < f; ++l) {
            rect_tr += (e == l);
            rect_lift += (((e + l) % 2) == 0);
            square_lift += (((e + l) % 2) == 0) && e - l != 2;
        }
    }
    int64_t ops_total = 0, bytes_k = 0, dofs = 0;
    for (int cl = 0; cl < ops->n_classes; ++cl) {
        const int32_t* ci = &ops->h_cls_int[cl * CI_STRIDE];
        const int dom = ci[CI_DOMAIN], nF = ci[CI_NF], count = ci[CI_COUNT];
        const int npad = ci[CI_NPAD], sbase = ci[CI_SLOT];
        const bool rect = ci[CI_KIND] != KIND_GENERIC;
        const int nv = (dom ? 5 : 3) * n, pc = dom ? 2 : 1;   // state values, primal components
        const int64_t nnzT = ci[CI_KIND] == KIND_SQUARE ? square_tr : rect ? rect_tr : (int64_t)f * n;
        const int64_t nnzL = ci[CI_KIND] == KIND_SQUARE ? square_lift : rect ? rect_lift : (int64_t)f * n;
        dofs += (int64_t)count * nv;
        for (int r = 0; r < count; ++r) {
            int64_t rate = dom ? 5 * dsm + 3 * dvalid + 2 * n : 3 * dsm + dvalid;   // derivatives (+ stress mix)
            int64_t traces = 0, bytes_faces = 0;
            for (int j = 0; j < nF; ++j) {
                const int32_t nb = (dom ? ops->h_nb_s : ops->h_nb_f)[sbase + j * npad + r];
                const bool bnd = nb == NB_BOUNDARY, ifc = nb < NB_BOUNDARY;
                rate += bnd ? 0 : (ifc && !dom ? 3 * f : pc * f);                  // jump
                // lift and the normal / tau combinations; rectangles lift each mirror
                // pair of faces at once (lift_pair: 4f + 2 nnz(L) per pair and component)
                rate += rect ? pc * (nnzL + 2 * f) : pc * nnzL + (dom ? 6 * n : 3 * n);
                traces += dom ? (rect ? 4 * nnzT : 4 * n + 4 * nnzT) + 2 * f + (ifc ? 4 * f : 2 * f)
                              : (rect ? 2 * nnzT : 2 * n + 2 * nnzT) + 2 * f;
                bytes_faces += 8 * (int64_t)pc * f * (1 + (bnd ? 0 : 1) + 2) + 4 + 8;
            }
            for (int j = 0; j < tab->s; ++j) {
                const StagePlan& P = plan[j];
                ops_total += rate + (int64_t)P.n_tgt * (nv + 3) + traces;
                int64_t passes = 1;   // stage input
                for (int t = 0; t < P.n_tgt; ++t) passes += 1 + (P.t[t].src != SRC_ZERO ? 1 : 0);
                bytes_k += 8 * passes * nv + bytes_faces + 8 * (dom ? SCS : SCF);
            }
        }
    }
    int64_t passes_min = 0;
    for (int j = 0; j < tab->s; ++j) {
        const StagePlan& P = plan[j];
        std::vector<int> reads, writes;
        reads.push_back(j == 0 ? SRC_STATE : SRC_X);
        for (int t = 0; t < P.n_tgt; ++t) {
            if (P.t[t].src != SRC_ZERO) reads.push_back(P.t[t].src);
            writes.push_back(P.t[t].dst);
        }
        std::sort(reads.begin(), reads.end());
        reads.erase(std::unique(reads.begin(), reads.end()), reads.end());
        passes_min += (int64_t)reads.size() + (int64_t)writes.size();
    }
    if (fp64_ops) *fp64_ops = ops_total;
    if (bytes_min) *bytes_min = 8 * passes_min * dofs;
    if (bytes_kernel) *bytes_kernel = bytes_k;
    return HHO_OK;
}

template <class T>
static int apply_t(hho_ops* ops, double t, const T* d_state, T* d_rate, T* d_traces, cudaStream_t st) {
    const dim3 grid((ops->dev.Nf + ops->dev.Ns + 127) / 128, 1);
    if (grid.x == 0) return HHO_OK;
    StageArgsT<T> a;
    memset(&a, 0, sizeof(a));
    a.op = ops->dev;
    a.state_stride = ops->n_state;
    a.trace_stride = ops->trace_doubles;
    a.inp = d_state;
    a.tr_out = d_traces;
    launch_k<T, MODE_TRACES>(ops->k, a, grid, st);
    int rc = check_launch("hho_apply (trace kernel)");
    if (rc) return rc;
    a.tr_in = d_traces;
    a.tr_out = nullptr;
    a.n_tgt = 1;
    a.tgt[0].src = nullptr;
    a.tgt[0].dst = d_rate;
    a.tgt[0].coef = T(1.0);
    fill_sources<T>(ops, a, t, -1, 0.0, 1);
    launch_k<T, MODE_APPLY>(ops->k, a, grid, st);
    return check_launch("hho_apply (stage kernel)");
}

extern "C" int hho_apply(hho_ops* ops, double t, const double* d_state, double* d_rate, double* d_work,
                         void* stream) {
    if (!ops || !d_state || !d_rate || !d_work) {
        hho_set_error("hho_apply: null pointer");
        return HHO_EINVAL;
    }
    if (ops->src_sampled) {
        hho_set_error("hho_apply: sampled source time functions are indexed by ERK stages, not by time");
        return HHO_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (ops->arith != HHO_F32X2) return apply_t<double>(ops, t, d_state, d_rate, d_work, st);
    // double-float: [traces][state pairs][rate pairs] inside the work buffer
    if (ops->n_state == 0) return HHO_OK;
    f2x* tr = (f2x*)d_work;
    f2x* ux = (f2x*)(d_work + ops->trace_doubles);
    f2x* rx = ux + ops->n_state;
    to_pairs_kernel<<<pairs_grid(ops->n_state), 256, 0, st>>>(d_state, ux, ops->n_state);
    int rc = check_launch("hho_apply");
    if (rc) return rc;
    rc = apply_t<f2x>(ops, t, ux, rx, tr, st);
    if (rc) return rc;
    from_pairs_kernel<<<pairs_grid(ops->n_state), 256, 0, st>>>(rx, d_rate, ops->n_state);
    return check_launch("hho_apply");
}

extern "C" int hho_state_pack(const hho_ops* ops, const double* d_canonical, double* d_state, void* stream) {
    if (!ops || !d_canonical || !d_state) {
        hho_set_error("hho_state_pack: null pointer");
        return HHO_EINVAL;
    }
    return hho_batch_pack(ops, 1, HHO_F64, d_canonical, d_state, stream);
}

extern "C" int hho_state_unpack(const hho_ops* ops, const double* d_state, double* d_canonical, void* stream) {
    if (!ops || !d_canonical || !d_state) {
        hho_set_error("hho_state_unpack: null pointer");
        return HHO_EINVAL;
    }
    return hho_batch_unpack(ops, 1, HHO_F64, d_state, d_canonical, stream);
}

extern "C" int hho_energy(hho_ops* ops, const double* d_state, double* d_work, double* h_energy, void* stream) {
    if (!ops || !d_state || !d_work || !h_energy) {
        hho_set_error("hho_energy: null pointer");
        return HHO_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int tot = ops->dev.Nf + ops->dev.Ns;
    const int nblk = (tot + 255) / 256;
    double* partial = d_work;
    double* result = d_work + nblk;
    if (nblk > 0) {
        if (ops->k == 1) energy_kernel<1><<<nblk, 256, 0, st>>>(ops->dev, d_state, ops->d_mass_f, ops->d_mass_s, partial);
        else if (ops->k == 2) energy_kernel<2><<<nblk, 256, 0, st>>>(ops->dev, d_state, ops->d_mass_f, ops->d_mass_s, partial);
        else energy_kernel<3><<<nblk, 256, 0, st>>>(ops->dev, d_state, ops->d_mass_f, ops->d_mass_s, partial);
    }
    sum_kernel<<<1, 256, 0, st>>>(partial, nblk, result);
    int rc = check_launch("hho_energy");
    if (rc) return rc;
    double e = 0.0;
    if (cudaMemcpyAsync(&e, result, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        hho_set_error("hho_energy: copy failed");
        return HHO_ECUDA;
    }
    *h_energy = e;
    if (!std::isfinite(e)) {
        hho_set_error("hho_energy: non-finite energy");
        return HHO_EUNSTABLE;
    }
    return HHO_OK;
}

extern "C" int hho_record(hho_ops* ops, const double* d_state, double* d_out, void* stream) {
    if (!ops || !d_state || (ops->n_rec > 0 && !d_out)) {
        hho_set_error("hho_record: null pointer");
        return HHO_EINVAL;
    }
    if (ops->n_rec == 0) return HHO_OK;
    record_kernel<double><<<dim3((ops->n_rec + 63) / 64, 1), 64, 0, (cudaStream_t)stream>>>(
        ops->dev, ops->n_rec, ops->d_rec_int, ops->d_rec_dbl, d_state, ops->n_state, d_out);
    return check_launch("hho_record");
}

extern "C" int hho_erk_run_host(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps,
                                double* h_canonical, void* stream) {
    if (!ops || !tab || !h_canonical) {
        hho_set_error("hho_erk_run_host: null pointer");
        return HHO_EINVAL;
    }
    int64_t wsz = 0;
    int rc = hho_work_size(ops, tab, &wsz);
    if (rc) return rc;
    if (!ops->d_host_state) {
        if (cudaMalloc((void**)&ops->d_host_state, sizeof(double) * ops->n_state) != cudaSuccess ||
            cudaMalloc((void**)&ops->d_host_canon, sizeof(double) * ops->n_canonical) != cudaSuccess) {
            hho_set_error("hho_erk_run_host: device allocation failed");
            return HHO_ENOMEM;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (ops->host_work_size < wsz) {
        if (ops->d_host_work) cudaFree(ops->d_host_work);
        ops->d_host_work = nullptr;
        if (cudaMalloc((void**)&ops->d_host_work, sizeof(double) * wsz) != cudaSuccess) {
            hho_set_error("hho_erk_run_host: device allocation failed");
            return HHO_ENOMEM;
        }
        ops->host_work_size = wsz;
        // the mapped path leaves padding slots of its states unwritten
        if (cudaMemsetAsync(ops->d_host_work, 0, sizeof(double) * wsz, st) != cudaSuccess ||
            cudaMemsetAsync(ops->d_host_state, 0, sizeof(double) * ops->n_state, st) != cudaSuccess) {
            hho_set_error("hho_erk_run_host: device memset failed");
            return HHO_ECUDA;
        }
    }
    // A pinned host buffer mapped into the device's address space is read
    // and written by the pack kernels directly (over NVLink-C2C on GB300);
    // any other host memory goes through a staging copy.
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, h_canonical) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer) {
        rc = erk_run_mapped(ops, tab, t0, dt, nsteps, (double*)pa.devicePointer, st);
        if (rc) return rc;
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            hho_set_error("hho_erk_run_host: %s", cudaGetErrorString(cudaGetLastError()));
            return HHO_ECUDA;
        }
        return HHO_OK;
    }
    cudaGetLastError();   // an unregistered pointer leaves an error on some drivers
    if (cudaMemcpyAsync(ops->d_host_canon, h_canonical, sizeof(double) * ops->n_canonical, cudaMemcpyHostToDevice,
                        st) != cudaSuccess) {
        hho_set_error("hho_erk_run_host: host-to-device copy failed");
        return HHO_ECUDA;
    }
    rc = hho_state_pack(ops, ops->d_host_canon, ops->d_host_state, stream);
    if (rc) return rc;
    rc = hho_erk_step(ops, tab, t0, dt, nsteps, ops->d_host_state, ops->d_host_work, stream);
    if (rc) return rc;
    rc = hho_state_unpack(ops, ops->d_host_state, ops->d_host_canon, stream);
    if (rc) return rc;
    if (cudaMemcpyAsync(h_canonical, ops->d_host_canon, sizeof(double) * ops->n_canonical, cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        hho_set_error("hho_erk_run_host: device-to-host copy failed");
        return HHO_ECUDA;
    }
    return HHO_OK;
}

extern "C" int hho_cfl_bracket(hho_ops* ops, const hho_tableau* tab, const double* d_state0, double T_f,
                               int64_t N0, double eps, double delta, int64_t max_trials, double* d_state,
                               double* d_work, int64_t* n_stable, int64_t* n_unstable, void* stream) {
    if (!ops || !tab || !d_state0 || !d_state || !d_work || !n_stable || !n_unstable || !(T_f > 0.0) || N0 < 1 ||
        !(eps > 0.0) || !(delta > 0.0) || max_trials < 1) {
        hho_set_error("hho_cfl_bracket: bad arguments");
        return HHO_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int saved_src = ops->n_src, saved_shot = ops->n_shot_src;
    ops->n_src = 0;        // Algorithm 1 runs without sources
    ops->n_shot_src = 0;
    int rc = HHO_OK;
    int64_t N = N0, last = -1, first_unstable = -1;
    for (int64_t trial = 0; trial < max_trials && N >= 1 && rc == HHO_OK; ++trial) {
        const double dt = T_f / (double)N;
        if (cudaMemcpyAsync(d_state, d_state0, sizeof(double) * ops->n_state, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess) {
            hho_set_error("hho_cfl_bracket: copy failed");
            rc = HHO_ECUDA;
            break;
        }
        double E0 = 0.0;
        rc = hho_energy(ops, d_state, d_work, &E0, stream);
        if (rc) break;
        if (!(E0 > 0.0) || !std::isfinite(E0)) {   // the relative increases below divide by E0
            hho_set_error("hho_cfl_bracket: the initial energy must be positive and finite (got %g)", E0);
            rc = HHO_EINVAL;
            break;
        }
        double Eprev = E0;
        bool stable = true;
        for (int64_t n = 0; n < N; ++n) {
            rc = hho_erk_step(ops, tab, (double)n * dt, dt, 1, d_state, d_work, stream);
            if (rc) break;
            double E = 0.0;
            rc = hho_energy(ops, d_state, d_work, &E, stream);
            if (rc == HHO_EUNSTABLE) {   // non-finite energy: the trial is unstable
                rc = HHO_OK;
                stable = false;
                break;
            }
            if (rc) break;
            if ((E - E0) / E0 > eps || (E - Eprev) / Eprev > eps) {
                stable = false;
                break;
            }
            Eprev = E;
        }
        if (rc) break;
        if (!stable) {
            first_unstable = N;
            break;
        }
        last = N;
        int64_t dec = (int64_t)std::floor(delta * (double)N);
        N -= dec < 1 ? 1 : dec;
    }
    ops->n_src = saved_src;
    ops->n_shot_src = saved_shot;
    *n_stable = last;
    *n_unstable = first_unstable;
    return rc;
}

// ---- energy without allocation ------------------------------------------------------
// Block partial sums of hho_energy_static live in this fixed array instead of
// a caller buffer.  Host code must not take its address directly (the host
// symbol is only a stand-in for the device variable); the device address is
// looked up with cudaGetSymbolAddress, with the device current, on every
// call.  The lookup allocates nothing and is cheap, and an address kept from
// an earlier call would go stale after a device reset.
namespace {
constexpr int kEnergyStaticMaxBlocks = (int)(HHO_ENERGY_STATIC_MAX_CELLS / 256);
static __device__ __align__(256) double g_energy_partials[kEnergyStaticMaxBlocks];

// Device address of g_energy_partials on the current device.
int energy_scratch(double** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_energy_partials);
    if (e != cudaSuccess || !p) {
        hho_set_error("hho_energy_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return HHO_ECUDA;
    }
    *out = (double*)p;
    return HHO_OK;
}
}  // namespace

extern "C" int hho_energy_static(hho_ops* ops, const double* d_state, double* d_energy, void* stream) {
    if (!ops || !d_state || !d_energy) {
        hho_set_error("hho_energy_static: null pointer");
        return HHO_EINVAL;
    }
    const int64_t tot = (int64_t)ops->dev.Nf + ops->dev.Ns;
    if (tot > HHO_ENERGY_STATIC_MAX_CELLS) {
        hho_set_error("hho_energy_static: %lld padded cell slots exceed the fixed scratch limit of %lld; use hho_energy",
                      (long long)tot, (long long)HHO_ENERGY_STATIC_MAX_CELLS);
        return HHO_EINVAL;
    }
    double* partial = nullptr;
    int rc = energy_scratch(&partial);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nblk = (int)((tot + 255) / 256);
    // energy_kernel writes every partial[0..nblk) before sum_kernel reads it,
    // so the array's previous contents never matter.
    if (nblk > 0) {
        if (ops->k == 1) energy_kernel<1><<<nblk, 256, 0, st>>>(ops->dev, d_state, ops->d_mass_f, ops->d_mass_s, partial);
        else if (ops->k == 2) energy_kernel<2><<<nblk, 256, 0, st>>>(ops->dev, d_state, ops->d_mass_f, ops->d_mass_s, partial);
        else energy_kernel<3><<<nblk, 256, 0, st>>>(ops->dev, d_state, ops->d_mass_f, ops->d_mass_s, partial);
    }
    sum_kernel<<<1, 256, 0, st>>>(partial, nblk, d_energy);
    return check_launch("hho_energy_static");
}

// ---- launchers for the adjoint driver (adjoint.cu) -----------------------------------
void launch_stage_f64(const hho_ops* ops, int mode, StageArgsT<double>& a, int n_shots, double tn, int j, double cdt,
                      bool sources, void* stream) {
    const dim3 grid((ops->dev.Nf + ops->dev.Ns + 127) / 128, n_shots);
    if (grid.x == 0) return;
    a.state_stride = ops->n_state;
    a.trace_stride = ops->trace_doubles;
    if (sources) {
        fill_sources<double>(ops, a, tn, j, cdt, n_shots);
    } else {
        a.n_src = 0;
        a.shot_src_q = nullptr;
        a.shot_src_dom = nullptr;
        a.shot_src_g = nullptr;
    }
    cudaStream_t st = (cudaStream_t)stream;
    switch (mode) {
        case MODE_TRACES: launch_k<double, MODE_TRACES>(ops->k, a, grid, st); break;
        case MODE_STAGE: launch_k<double, MODE_STAGE>(ops->k, a, grid, st); break;
        case MODE_APPLY: launch_k<double, MODE_APPLY>(ops->k, a, grid, st); break;
        default: launch_k<double, MODE_RAW>(ops->k, a, grid, st); break;
    }
}

void launch_stage_f32(const hho_ops* ops, int mode, StageArgsT<float>& a, int n_shots, double tn, int j, double cdt,
                      bool sources, void* stream) {
    const dim3 grid((ops->dev.Nf + ops->dev.Ns + 127) / 128, n_shots);
    if (grid.x == 0) return;
    a.state_stride = ops->n_state;
    a.trace_stride = ops->trace_doubles;
    if (sources) {
        fill_sources<float>(ops, a, tn, j, cdt, n_shots);
    } else {
        a.n_src = 0;
        a.shot_src_q = nullptr;
        a.shot_src_dom = nullptr;
        a.shot_src_g = nullptr;
    }
    cudaStream_t st = (cudaStream_t)stream;
    switch (mode) {
        case MODE_TRACES: launch_k<float, MODE_TRACES>(ops->k, a, grid, st); break;
        case MODE_STAGE: launch_k<float, MODE_STAGE>(ops->k, a, grid, st); break;
        case MODE_APPLY: launch_k<float, MODE_APPLY>(ops->k, a, grid, st); break;
        default: launch_k<float, MODE_RAW>(ops->k, a, grid, st); break;
    }
}

int erk_steps_f32(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps, float* d_state,
                  float* d_work, void* stream) {
    return erk_run<float>(ops, tab, t0, dt, nsteps, 1, d_state, d_work, nullptr, stream, "hho_adjoint_vjp_f32");
}

void launch_record_f64(const hho_ops* ops, const double* state, double* out, void* stream) {
    if (ops->n_rec == 0) return;
    record_kernel<double><<<dim3((ops->n_rec + 63) / 64, 1), 64, 0, (cudaStream_t)stream>>>(
        ops->dev, ops->n_rec, ops->d_rec_int, ops->d_rec_dbl, state, ops->n_state, out);
}

int check_cuda(const char* what) { return check_launch(what); }
