// Implicit SDIRK stepping (Sec. 4.1, Eq. SDIRK_compact, Eq. cp_dirk) on GB300.
//
// Every stage of Eq. cp_dirk keeps the face rows K_FT U_T + K_F U_F = 0 (the
// first stage has a zero face right-hand side and the later ones inherit
// it), so the cell part of stage i is the stage of the condensed ODE
//     (I - a* dt J) Y_i = Z_i + a* dt s(t_i),
//     J = -M^-1 (K_T - K_TF K_F^-1 K_FT),   s(t) = M^-1 F(t),
//     Z_i = U^{n-1} + dt sum_{j<i} a_ij k_j,   k_j = J Y_j + s(t_j),
// and the last stage (a_{s+1,j} = b_j) is the mass-matrix-only update
//     U^n = U^{n-1} + dt sum_j b_j k_j.
// The paper condenses the cell unknowns and solves a global face system.
// Here each stage system is solved matrix-free on the cell unknowns by
// restarted GMRES, right-preconditioned by the exact cell blocks
// (I - a* dt J_TT)^-1, the local solves of Eq. sc2 (block Jacobi; see
// build_block_jacobi).  One operator application is the ERK stage kernel (the
// closed-form face solve on every face, reconstruction, stabilisation and
// inverse mass) with the target v - a* dt J v, so no global matrix is
// assembled or stored and the implicit path reuses the explicit one's
// kernels.  Orthogonalisation is classical Gram-Schmidt applied twice, with
// its coefficients kept on the device; one copy to the host and one stream
// synchronisation per Krylov vector.  All reductions are block-partial sums
// added in a fixed order, so results are deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hho_internal.h"

namespace {

constexpr int RED_BLOCKS = 608;   // 4 x 152 SMs
constexpr int RED_THREADS = 256;
constexpr int MAX_RESTART = 64;

// partial[b * nv + l] = block b's share of sum_i V_l[i] w[i], l < nv
// (V_l = V + l * stride).  Four vectors per pass over i (independent FP64
// chains), then one fixed tree over the block for the four sums.
constexpr int MD_W = 4;
__global__ void multidot_kernel(const double* __restrict__ V, int64_t stride, int nv, const double* __restrict__ w,
                                int64_t n, double* __restrict__ partial) {
    __shared__ double sh[MD_W][RED_THREADS];
    for (int l0 = 0; l0 < nv; l0 += MD_W) {
        const int nl = min(MD_W, nv - l0);
        double acc[MD_W] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t i = blockIdx.x * (int64_t)RED_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * RED_THREADS) {
            const double wi = w[i];
#pragma unroll
            for (int l = 0; l < MD_W; ++l)
                if (l < nl) acc[l] = fma(V[(size_t)(l0 + l) * stride + i], wi, acc[l]);
        }
#pragma unroll
        for (int l = 0; l < MD_W; ++l) sh[l][threadIdx.x] = acc[l];
        __syncthreads();
        for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o)
                for (int l = 0; l < nl; ++l) sh[l][threadIdx.x] += sh[l][threadIdx.x + o];
            __syncthreads();
        }
        if ((int)threadIdx.x < nl) partial[(size_t)blockIdx.x * nv + l0 + threadIdx.x] = sh[threadIdx.x][0];
        __syncthreads();
    }
}

// out[l] = sum over blocks of partial[b * nv + l]: block l; thread t adds
// b = t, t + 256, ... in increasing order, then a fixed tree over the
// threads.  (A single dependent chain over the 608 partials took about
// 50 us a call on GB300, whose FP64 add latency is long.)
__global__ void sum_partials_kernel(const double* __restrict__ partial, int nb, int nv, double* __restrict__ out) {
    __shared__ double sh[RED_THREADS];
    const int l = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += RED_THREADS) s += partial[(size_t)b * nv + l];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[l] = sh[0];
}

// y = alpha y + beta sum_l coef[l] V_l  (coef in device memory; y may be
// one of the V_l: each element is read before the same thread writes it)
__global__ void lincomb_kernel(double* y, double alpha, double beta, const double* V, int64_t stride, int nv,
                               const double* __restrict__ coef, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int l = 0; l < nv; ++l) v = fma(coef[l], V[(size_t)l * stride + i], v);
        y[i] = fma(beta, v, alpha * y[i]);
    }
}

// y *= c
__global__ void scale_kernel(double* y, double c, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] *= c;
}

// Up to 8 terms with coefficients passed by value: y = sum_l c_l x_l.
struct Terms {
    int n;
    const double* x[8];
    double c[8];
};
__global__ void terms_kernel(double* y, Terms T, int64_t n) {   // y may be one of the x_l
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int l = 0; l < T.n; ++l) v = fma(T.c[l], T.x[l][i], v);
        y[i] = v;
    }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

extern "C" int hho_tableau_sdirk(int32_t s, hho_tableau* out) {
    if (!out) {
        hho_set_error("hho_tableau_sdirk: null pointer");
        return HHO_EINVAL;
    }
    hho_tableau t;
    memset(&t, 0, sizeof(t));
    if (s == 1) {
        t.s = 1;
        t.a[0][0] = 0.5;
        t.b[0] = 1.0;
        t.c[0] = 0.5;
    } else if (s == 2) {   // as printed: a* = 1/4 (order 2)
        t.s = 2;
        t.a[0][0] = 0.25;
        t.a[1][0] = 0.5;
        t.a[1][1] = 0.25;
        t.b[0] = t.b[1] = 0.5;
        t.c[0] = 0.25;
        t.c[1] = 0.75;
    } else if (s == 23) {   // the order-3 member of the same family
        const double g = (3.0 + std::sqrt(3.0)) / 6.0;
        t.s = 2;
        t.a[0][0] = g;
        t.a[1][0] = 1.0 - 2.0 * g;
        t.a[1][1] = g;
        t.b[0] = t.b[1] = 0.5;
        t.c[0] = g;
        t.c[1] = 1.0 - g;
    } else if (s == 3) {
        const double nu = std::cos(M_PI / 18.0) / std::sqrt(3.0) + 0.5;
        const double xi = 1.0 / (6.0 * (2.0 * nu - 1.0) * (2.0 * nu - 1.0));
        t.s = 3;
        t.a[0][0] = nu;
        t.a[1][0] = 0.5 - nu;
        t.a[1][1] = nu;
        t.a[2][0] = 2.0 * nu;
        t.a[2][1] = 1.0 - 4.0 * nu;
        t.a[2][2] = nu;
        t.b[0] = xi;
        t.b[1] = 1.0 - 2.0 * xi;
        t.b[2] = xi;
        t.c[0] = nu;
        t.c[1] = 0.5;
        t.c[2] = 1.0 - nu;
    } else {
        hho_set_error("hho_tableau_sdirk: s must be 1, 2, 3 or 23");
        return HHO_EINVAL;
    }
    *out = t;
    return HHO_OK;
}

namespace {

bool sdirk_tableau_ok(const hho_tableau* tab) {
    if (!tab || tab->s < 1 || tab->s > 6) return false;
    const double a = tab->a[0][0];
    if (!(a > 0.0)) return false;
    for (int i = 0; i < tab->s; ++i) {
        if (tab->a[i][i] != a) return false;
        for (int j = i + 1; j < tab->s; ++j)
            if (tab->a[i][j] != 0.0) return false;
    }
    return true;
}

// Work layout (doubles; vectors of n_state): Z | Y | T | W | K[s] |
// V[restart + 1] | zero | traces | reduction partials | reduction sums | coefficients |
// preconditioned vector
struct SdirkWork {
    double *Z, *Y, *T, *W, *K, *V, *zero, *tr, *partial, *sums, *coef, *PZ;
    int64_t n;
};

int64_t sdirk_layout(const hho_ops* ops, int s, int m, SdirkWork* w, double* base) {
    const int64_t n = ops->n_state;
    int64_t off = 0;
    auto take = [&](int64_t cnt) {
        double* p = base ? base + off : nullptr;
        off += (cnt + 31) / 32 * 32;
        return p;
    };
    SdirkWork W;
    W.n = n;
    W.Z = take(n);
    W.Y = take(n);
    W.T = take(n);
    W.W = take(n);
    W.K = take(n * s);
    W.V = take(n * (m + 1));
    W.zero = take(n);
    W.tr = take(ops->trace_doubles);
    W.partial = take((int64_t)RED_BLOCKS * (m + 1));
    W.sums = take(2 * (m + 1) + 2);
    W.coef = take(m + 1);
    W.PZ = take(n);
    if (w) *w = W;
    return off;
}

// out = v - a_dt J v (sources off), or out = J v + s(t) when rate is true
void apply_op(hho_ops* ops, const double* v, double* out, double* tr, double a_dt, bool rate, double t,
              cudaStream_t st) {
    StageArgsT<double> a;
    memset(&a, 0, sizeof(a));
    a.op = ops->dev;
    a.inp = v;
    a.tr_out = tr;
    launch_stage_f64(ops, MODE_TRACES, a, 1, 0.0, -1, 0.0, false, st);
    a.tr_in = tr;
    a.tr_out = nullptr;
    a.n_tgt = 1;
    a.tgt[0].src = rate ? nullptr : v;
    a.tgt[0].dst = out;
    a.tgt[0].coef = rate ? 1.0 : -a_dt;
    launch_stage_f64(ops, MODE_APPLY, a, 1, t, -1, 0.0, rate, st);
}

// ---- block-Jacobi preconditioner --------------------------------------------------
// The stage system's cell-diagonal blocks P_T = I - a* dt J_TT (J_TT: the
// rate of cell T's unknowns with every other cell at zero, its own face
// terms included) are the local solves of Eq. sc2.  Their columns come from
// the stage operator itself: on a state that is the unit vector e_i in every
// cell of one colour and zero elsewhere, v - a* dt J v restricted to a cell of
// that colour is column i of its block, because no two cells of a colour
// share a face (nor an interface face).  The blocks are inverted in place
// (Gauss-Jordan with partial pivoting, one CTA per cell) and applied as
// y = P^-1 x, one thread per (row, cell), coalesced over cells.

// Greedy colouring of the cells (fluid slots 0..Nf-1, solid Nf..Nf+Ns-1;
// padding slots -1) so that face neighbours, across an interface too,
// differ.
std::vector<int32_t> cell_colours(const hho_ops* ops, int* n_colours) {
    const int Nf = ops->dev.Nf, Ns = ops->dev.Ns;
    std::vector<int32_t> slot_cell[2] = {std::vector<int32_t>(ops->dev.SF, -1), std::vector<int32_t>(ops->dev.SS, -1)};
    std::vector<std::vector<int32_t>> adj(Nf + Ns);
    for (int pass = 0; pass < 2; ++pass)
        for (int cl = 0; cl < ops->n_classes; ++cl) {
            const int32_t* ci = &ops->h_cls_int[cl * CI_STRIDE];
            const int d = ci[CI_DOMAIN], base = d ? Nf : 0;
            const std::vector<int32_t>& nbt = d ? ops->h_nb_s : ops->h_nb_f;
            for (int j = 0; j < ci[CI_NF]; ++j)
                for (int lq = 0; lq < ci[CI_COUNT]; ++lq) {
                    const int slot = ci[CI_SLOT] + j * ci[CI_NPAD] + lq;
                    const int g = base + ci[CI_START] + lq;
                    if (pass == 0) {
                        slot_cell[d][slot] = g;
                        continue;
                    }
                    const int nb = nbt[slot];
                    int other = -1;
                    if (nb >= 0) other = slot_cell[d][nb];
                    else if (nb < NB_BOUNDARY) other = slot_cell[1 - d][ops->h_if_nb[-2 - nb]];
                    if (other >= 0) adj[g].push_back(other);
                }
        }
    std::vector<int32_t> colour(Nf + Ns, -1);
    int nc = 0;
    for (int g = 0; g < Nf + Ns; ++g) {
        if (adj[g].empty()) {
            bool real = false;   // a cell with no neighbour (one-cell mesh) is still a cell
            for (int cl = 0; cl < ops->n_classes && !real; ++cl) {
                const int32_t* ci = &ops->h_cls_int[cl * CI_STRIDE];
                const int start = (ci[CI_DOMAIN] ? Nf : 0) + ci[CI_START];
                real = g >= start && g < start + ci[CI_COUNT];
            }
            if (!real) continue;
        }
        std::vector<bool> used(nc + 1, false);
        for (int o : adj[g])
            if (colour[o] >= 0) used[colour[o]] = true;
        int c = 0;
        while (used[c]) ++c;
        colour[g] = c;
        nc = std::max(nc, c + 1);
    }
    *n_colours = nc;
    return colour;
}

// x = e_i on every cell of colour c, 0 elsewhere (device state layout)
__global__ void unit_state_kernel(double* __restrict__ x, const int32_t* __restrict__ colour, int c, int i, int Nf,
                                  int Ns, int n) {
    const int64_t nf = (int64_t)3 * n * Nf, tot = nf + (int64_t)5 * n * Ns;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const bool fl = e < nf;
        const int64_t e2 = fl ? e : e - nf;
        const int N = fl ? Nf : Ns;
        const int field = (int)(e2 / N), q = (int)(e2 % N);
        x[e] = (field == i && colour[fl ? q : Nf + q] == c) ? 1.0 : 0.0;
    }
}

// column i of the block of every cell of colour c from y = x - a* dt J x
__global__ void bj_column_kernel(const double* __restrict__ y, const int32_t* __restrict__ colour, int c, int i,
                                 int Nf, int Ns, int n, double* __restrict__ bj) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Nf + Ns || colour[g] != c) return;
    const bool fl = g < Nf;
    const int q = fl ? g : g - Nf, N = fl ? Nf : Ns, nv = (fl ? 3 : 5) * n;
    if (i >= nv) return;
    const double* yb = fl ? y : y + (size_t)3 * n * Nf;
    double* b = fl ? bj : bj + (size_t)9 * n * n * Nf;
    for (int r = 0; r < nv; ++r) b[((size_t)r * nv + i) * N + q] = yb[(size_t)r * N + q];
}

// In-place inverse of every cell's block; one CTA of 64 threads per cell,
// [P | I] in shared memory (2 nv^2 doubles).  Padding slots get zeros.
__global__ void bj_invert_kernel(double* __restrict__ bj, const int32_t* __restrict__ colour, int Nf, int Ns, int n,
                                 int* __restrict__ status) {
    extern __shared__ double A[];
    __shared__ double fac[5 * 10];   // column k of every row (nv <= 5n <= 50)
    __shared__ int piv;
    const int g = blockIdx.x;
    const bool fl = g < Nf;
    const int q = fl ? g : g - Nf, N = fl ? Nf : Ns, nv = (fl ? 3 : 5) * n, w = 2 * nv;
    double* b = fl ? bj : bj + (size_t)9 * n * n * Nf;
    if (colour[g] < 0) {
        for (int e = threadIdx.x; e < nv * nv; e += blockDim.x) b[(size_t)e * N + q] = 0.0;
        return;
    }
    for (int e = threadIdx.x; e < nv * w; e += blockDim.x) {
        const int r = e / w, c = e % w;
        A[e] = c < nv ? b[((size_t)r * nv + c) * N + q] : (c - nv == r ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int k = 0; k < nv; ++k) {
        if (threadIdx.x == 0) {
            int p = k;
            for (int r = k + 1; r < nv; ++r)
                if (fabs(A[r * w + k]) > fabs(A[p * w + k])) p = r;
            piv = p;
            if (A[p * w + k] == 0.0) atomicExch(status, 1);
        }
        __syncthreads();
        const int p = piv;
        if (p != k)
            for (int c = threadIdx.x; c < w; c += blockDim.x) {
                const double t = A[k * w + c];
                A[k * w + c] = A[p * w + c];
                A[p * w + c] = t;
            }
        __syncthreads();
        const double d = A[k * w + k];
        __syncthreads();
        for (int c = threadIdx.x; c < w; c += blockDim.x) A[k * w + c] = d != 0.0 ? A[k * w + c] / d : 0.0;
        for (int r = threadIdx.x; r < nv; r += blockDim.x) fac[r] = A[r * w + k];
        __syncthreads();
        for (int e = threadIdx.x; e < nv * w; e += blockDim.x) {
            const int r = e / w, c = e % w;
            if (r != k) A[e] = fma(-fac[r], A[k * w + c], A[e]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nv * nv; e += blockDim.x) {
        const int r = e / nv, c = e % nv;
        b[((size_t)r * nv + c) * N + q] = A[r * w + nv + c];
    }
}

// y = P^-1 x (accumulate: y += P^-1 x); one thread per state entry (row r of
// cell q at r N + q)
__global__ void bj_apply_kernel(const double* __restrict__ bj, const double* __restrict__ x, double* __restrict__ y,
                                int accumulate, int Nf, int Ns, int n) {
    const int64_t nf = (int64_t)3 * n * Nf, tot = nf + (int64_t)5 * n * Ns;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const bool fl = e < nf;
        const int64_t e2 = fl ? e : e - nf;
        const int N = fl ? Nf : Ns, nv = (fl ? 3 : 5) * n;
        const int r = (int)(e2 / N), q = (int)(e2 % N);
        const double* b = (fl ? bj : bj + (size_t)9 * n * n * Nf) + (size_t)r * nv * N + q;
        const double* xb = (fl ? x : x + nf) + q;
        double s = 0.0;
        for (int c = 0; c < nv; ++c) s = fma(b[(size_t)c * N], xb[(size_t)c * N], s);
        y[e] = accumulate ? y[e] + s : s;
    }
}

// Builds (or reuses, for the same a* dt) the inverse blocks; scratch: x, y, tr.
int build_block_jacobi(hho_ops* ops, double a_dt, double* x, double* y, double* tr, cudaStream_t st) {
    const int Nf = ops->dev.Nf, Ns = ops->dev.Ns, n = ops->n;
    if (ops->d_bj && ops->bj_adt == a_dt) return HHO_OK;
    if (!ops->d_bj_colour) {
        int nc = 0;
        std::vector<int32_t> col = cell_colours(ops, &nc);
        if (cudaMalloc((void**)&ops->d_bj_colour, sizeof(int32_t) * std::max<size_t>(col.size(), 1)) != cudaSuccess ||
            cudaMemcpy(ops->d_bj_colour, col.data(), sizeof(int32_t) * col.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            hho_set_error("hho_sdirk_step: preconditioner colouring upload failed");
            return HHO_ECUDA;
        }
        ops->bj_colours = nc;
    }
    const size_t nbj = (size_t)9 * n * n * Nf + (size_t)25 * n * n * Ns;
    if (!ops->d_bj && cudaMalloc((void**)&ops->d_bj, sizeof(double) * std::max<size_t>(nbj, 1)) != cudaSuccess) {
        ops->d_bj = nullptr;
        hho_set_error("hho_sdirk_step: preconditioner allocation failed (%zu doubles)", nbj);
        return HHO_ENOMEM;
    }
    const int cells = Nf + Ns;
    for (int c = 0; c < ops->bj_colours; ++c)
        for (int i = 0; i < 5 * n; ++i) {
            if (i >= 3 * n && Ns == 0) break;
            unit_state_kernel<<<grid_for(ops->n_state), 256, 0, st>>>(x, ops->d_bj_colour, c, i, Nf, Ns, n);
            apply_op(ops, x, y, tr, a_dt, false, 0.0, st);
            bj_column_kernel<<<(cells + 127) / 128, 128, 0, st>>>(y, ops->d_bj_colour, c, i, Nf, Ns, n, ops->d_bj);
        }
    int* status = nullptr;
    if (cudaMalloc((void**)&status, sizeof(int)) != cudaSuccess) {
        hho_set_error("hho_sdirk_step: preconditioner status allocation failed");
        return HHO_ECUDA;
    }
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) {
        cudaFree(status);
        hho_set_error("hho_sdirk_step: preconditioner status initialisation failed");
        return HHO_ECUDA;
    }
    const size_t smem = sizeof(double) * 2 * (5 * n) * (5 * n);
    bj_invert_kernel<<<cells, 64, smem, st>>>(ops->d_bj, ops->d_bj_colour, Nf, Ns, n, status);
    int h_status = 0;
    const bool ok = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                    cudaStreamSynchronize(st) == cudaSuccess;
    cudaFree(status);
    if (!ok) {
        hho_set_error("hho_sdirk_step: preconditioner build failed: %s", cudaGetErrorString(cudaGetLastError()));
        return HHO_ECUDA;
    }
    if (h_status) {
        hho_set_error("hho_sdirk_step: a cell block I - a* dt J_TT is singular");
        return HHO_EUNSTABLE;
    }
    ops->bj_adt = a_dt;
    return HHO_OK;
}

// dst[l] = V_l . w for l < nv, on the device (no synchronisation)
void dots_dev(const SdirkWork& W, const double* V, int nv, const double* w, double* dst, cudaStream_t st) {
    multidot_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(V, W.n, nv, w, W.n, W.partial);
    sum_partials_kernel<<<nv, RED_THREADS, 0, st>>>(W.partial, RED_BLOCKS, nv, dst);
}

// the same, copied to the host (synchronises)
int dots(const SdirkWork& W, const double* V, int nv, const double* w, double* h, cudaStream_t st) {
    dots_dev(W, V, nv, w, W.sums, st);
    if (cudaMemcpyAsync(h, W.sums, sizeof(double) * nv, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        hho_set_error("hho_sdirk_step: reduction failed");
        return HHO_ECUDA;
    }
    return HHO_OK;
}

// y = alpha y + sum_l c[l] V_l with host coefficients (a copy from pageable
// memory returns once the source is staged, so c may be reused at once)
int combine(const SdirkWork& W, double* y, double alpha, const double* V, int nv, const double* c, cudaStream_t st) {
    if (cudaMemcpyAsync(W.coef, c, sizeof(double) * nv, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        hho_set_error("hho_sdirk_step: coefficient upload failed");
        return HHO_ECUDA;
    }
    lincomb_kernel<<<grid_for(W.n), 256, 0, st>>>(y, alpha, 1.0, V, W.n, nv, W.coef, W.n);
    return HHO_OK;
}

// Restarted GMRES for (I - a_dt J) x = b, x holding the initial guess; with
// bj, right-preconditioned (the Krylov space of A P^-1, x = x0 + P^-1 V y).
// Applying the inverted blocks rounds at a level set by their condition
// (about 1e-14 relative at k = 3), so when a preconditioned restart cycle
// does not halve the true residual the remaining cycles run without the
// preconditioner, which reaches the FP64 floor.  Adds its operator
// applications to *its; HHO_ENOCONV if tol is missed.
int gmres(hho_ops* ops, const SdirkWork& W, const double* b, double* x, double a_dt, double tol, int m,
          int max_iter, const double* bj, int64_t* its, cudaStream_t st) {
    const int Nf = ops->dev.Nf, Ns = ops->dev.Ns, nn = ops->n;
    double bn = 0.0;
    int rc = dots(W, b, 1, b, &bn, st);
    if (rc) return rc;
    bn = std::sqrt(bn);
    if (bn == 0.0) {
        cudaMemsetAsync(x, 0, sizeof(double) * W.n, st);
        return HHO_OK;
    }
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), hs(2 * (m + 1) + 1);
    int used = 0;
    double rn = 0.0, rn_prev = 0.0;
    while (true) {
        // r = b - A x into V_0; the true residual decides convergence
        apply_op(ops, x, W.W, W.tr, a_dt, false, 0.0, st);
        ++used;
        Terms T;
        T.n = 2;
        T.x[0] = b;
        T.c[0] = 1.0;
        T.x[1] = W.W;
        T.c[1] = -1.0;
        terms_kernel<<<grid_for(W.n), 256, 0, st>>>(W.V, T, W.n);
        double r2 = 0.0;
        rc = dots(W, W.V, 1, W.V, &r2, st);
        if (rc) return rc;
        rn = std::sqrt(r2);
        if (!std::isfinite(rn)) {
            hho_set_error("hho_sdirk_step: non-finite residual");
            return HHO_EUNSTABLE;
        }
        if (rn <= tol * bn || used >= max_iter) break;
        if (bj && rn_prev > 0.0 && rn > 0.5 * rn_prev) bj = nullptr;   // stagnation: finish unpreconditioned
        rn_prev = rn;
        scale_kernel<<<grid_for(W.n), 256, 0, st>>>(W.V, 1.0 / rn, W.n);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = rn;
        int j = 0;
        for (; j < m && used < max_iter; ++j) {
            double* vj1 = W.V + (size_t)(j + 1) * W.n;
            if (bj) {
                bj_apply_kernel<<<grid_for(W.n), 256, 0, st>>>(bj, W.V + (size_t)j * W.n, W.PZ, 0, Nf, Ns, nn);
                apply_op(ops, W.PZ, vj1, W.tr, a_dt, false, 0.0, st);
            } else {
                apply_op(ops, W.V + (size_t)j * W.n, vj1, W.tr, a_dt, false, 0.0, st);
            }
            ++used;
            // classical Gram-Schmidt twice, coefficients kept on the device
            double* S1 = W.sums;
            double* S2 = W.sums + (m + 1);
            double* S3 = W.sums + 2 * (m + 1);
            dots_dev(W, W.V, j + 1, vj1, S1, st);
            lincomb_kernel<<<grid_for(W.n), 256, 0, st>>>(vj1, 1.0, -1.0, W.V, W.n, j + 1, S1, W.n);
            dots_dev(W, W.V, j + 1, vj1, S2, st);
            lincomb_kernel<<<grid_for(W.n), 256, 0, st>>>(vj1, 1.0, -1.0, W.V, W.n, j + 1, S2, W.n);
            dots_dev(W, vj1, 1, vj1, S3, st);
            if (cudaMemcpyAsync(hs.data(), W.sums, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                hho_set_error("hho_sdirk_step: reduction failed");
                return HHO_ECUDA;
            }
            const double hn = std::sqrt(hs[2 * (m + 1)]);
            double* col = &H[(size_t)j * (m + 1)];
            for (int l = 0; l <= j; ++l) col[l] = hs[l] + hs[m + 1 + l];
            col[j + 1] = hn;
            for (int l = 0; l < j; ++l) {   // earlier rotations
                const double t0 = cs[l] * col[l] + sn[l] * col[l + 1];
                col[l + 1] = -sn[l] * col[l] + cs[l] * col[l + 1];
                col[l] = t0;
            }
            const double den = std::hypot(col[j], col[j + 1]);
            cs[j] = den > 0.0 ? col[j] / den : 1.0;
            sn[j] = den > 0.0 ? col[j + 1] / den : 0.0;
            col[j] = den;
            col[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (std::fabs(g[j + 1]) <= tol * bn || hn == 0.0) {
                ++j;
                break;
            }
            scale_kernel<<<grid_for(W.n), 256, 0, st>>>(vj1, 1.0 / hn, W.n);
        }
        // x += V y with H y = g (upper triangular, j x j)
        for (int r = j - 1; r >= 0; --r) {
            double v = g[r];
            for (int c2 = r + 1; c2 < j; ++c2) v -= H[(size_t)c2 * (m + 1) + r] * y[c2];
            y[r] = v / H[(size_t)r * (m + 1) + r];
        }
        if (j > 0 && bj) {   // x += P^-1 (V y)
            cudaMemsetAsync(W.W, 0, sizeof(double) * W.n, st);
            rc = combine(W, W.W, 0.0, W.V, j, y.data(), st);
            if (rc) return rc;
            bj_apply_kernel<<<grid_for(W.n), 256, 0, st>>>(bj, W.W, x, 1, Nf, Ns, nn);
        } else if (j > 0) {
            rc = combine(W, x, 1.0, W.V, j, y.data(), st);
            if (rc) return rc;
        }
    }
    *its += used;
    if (rn > tol * bn) {
        hho_set_error("hho_sdirk_step: GMRES reached %d operator applications with ||r||/||b|| = %.3e > %.3e",
                      used, rn / bn, tol);
        return HHO_ENOCONV;
    }
    return HHO_OK;
}

}  // namespace

extern "C" int hho_sdirk_work_size(const hho_ops* ops, const hho_tableau* tab, int32_t restart, int64_t* n_doubles) {
    if (!ops || !n_doubles || !sdirk_tableau_ok(tab) || restart < 1 || restart > MAX_RESTART) {
        hho_set_error("hho_sdirk_work_size: bad arguments (SDIRK tableau, 1 <= restart <= %d)", MAX_RESTART);
        return HHO_EINVAL;
    }
    *n_doubles = sdirk_layout(ops, tab->s, restart, nullptr, nullptr);
    return HHO_OK;
}

extern "C" int hho_sdirk_step(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps, double tol,
                              int32_t restart, int32_t max_iter, double* d_state, double* d_work,
                              int64_t* h_iterations, void* stream) {
    if (!ops || !d_state || !d_work || !sdirk_tableau_ok(tab) || restart < 1 || restart > MAX_RESTART ||
        max_iter < 1 || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(t0) || !(tol > 0.0)) {
        hho_set_error("hho_sdirk_step: bad arguments (SDIRK tableau, dt > 0, tol > 0, 1 <= restart <= %d, "
                      "max_iter >= 1)", MAX_RESTART);
        return HHO_EINVAL;
    }
    if (ops->src_sampled) {
        hho_set_error("hho_sdirk_step: sampled source time functions are indexed by ERK stages; use "
                      "hho_sources_set for the implicit path");
        return HHO_EINVAL;
    }
    int64_t its = 0;
    if (h_iterations) *h_iterations = 0;
    if (nsteps == 0 || ops->n_state == 0) return HHO_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int s = tab->s;
    SdirkWork W;
    const int64_t total = sdirk_layout(ops, s, restart, &W, d_work);
    // padding slots stay zero: the stage kernel never writes them
    if (cudaMemsetAsync(d_work, 0, sizeof(double) * total, st) != cudaSuccess) {
        hho_set_error("hho_sdirk_step: work initialisation failed");
        return HHO_ECUDA;
    }
    const double a_dt = tab->a[0][0] * dt;
    const int64_t n = W.n;
    int rc = HHO_OK;
    bool precond = ops->sdirk_precond != 0;
    if (precond) {
        rc = build_block_jacobi(ops, a_dt, W.Z, W.W, W.tr, st);
        if (rc == HHO_ENOMEM) {   // no room for the blocks: the same solve, unpreconditioned
            cudaGetLastError();
            precond = false;
            rc = HHO_OK;
        }
        if (rc) return rc;
    }
    const double* bj = precond ? ops->d_bj : nullptr;
    for (int64_t step = 0; step < nsteps && rc == HHO_OK; ++step) {
        const double tn = t0 + (double)step * dt;
        for (int i = 0; i < s && rc == HHO_OK; ++i) {
            const double ti = tn + tab->c[i] * dt;
            // Z_i = U^{n-1} + dt sum_{j<i} a_ij k_j
            Terms T;
            T.n = 1;
            T.x[0] = d_state;
            T.c[0] = 1.0;
            for (int j = 0; j < i; ++j) {
                if (tab->a[i][j] == 0.0) continue;
                T.x[T.n] = W.K + (size_t)j * n;
                T.c[T.n] = dt * tab->a[i][j];
                ++T.n;
            }
            terms_kernel<<<grid_for(n), 256, 0, st>>>(W.Z, T, n);
            // right-hand side Z_i + a* dt s(t_i): s(t) is the rate of the zero state
            apply_op(ops, W.zero, W.T, W.tr, 0.0, true, ti, st);
            Terms R;
            R.n = 2;
            R.x[0] = W.Z;
            R.c[0] = 1.0;
            R.x[1] = W.T;
            R.c[1] = a_dt;
            terms_kernel<<<grid_for(n), 256, 0, st>>>(W.T, R, n);
            // initial guess: Z_i + a* dt k_{i-1} (the previous stage's rate), else Z_i
            Terms G;
            G.n = 1;
            G.x[0] = W.Z;
            G.c[0] = 1.0;
            if (i > 0) {
                G.x[1] = W.K + (size_t)(i - 1) * n;
                G.c[1] = a_dt;
                G.n = 2;
            }
            terms_kernel<<<grid_for(n), 256, 0, st>>>(W.Y, G, n);
            rc = check_cuda("hho_sdirk_step");
            if (rc) break;
            rc = gmres(ops, W, W.T, W.Y, a_dt, tol, restart, max_iter, bj, &its, st);
            if (rc) break;
            // k_i = J Y_i + s(t_i)
            apply_op(ops, W.Y, W.K + (size_t)i * n, W.tr, 0.0, true, ti, st);
        }
        if (rc) break;
        // U^n = U^{n-1} + dt sum_j b_j k_j
        Terms U;
        U.n = 1;
        U.x[0] = d_state;
        U.c[0] = 1.0;
        for (int j = 0; j < s; ++j) {
            U.x[U.n] = W.K + (size_t)j * n;
            U.c[U.n] = dt * tab->b[j];
            ++U.n;
        }
        terms_kernel<<<grid_for(n), 256, 0, st>>>(d_state, U, n);
        rc = check_cuda("hho_sdirk_step");
    }
    if (h_iterations) *h_iterations = its;
    return rc;
}

extern "C" int hho_sdirk_set_preconditioner(hho_ops* ops, int32_t kind) {
    if (!ops || kind < 0 || kind > 1) {
        hho_set_error("hho_sdirk_set_preconditioner: bad arguments (kind 0: none, 1: block Jacobi)");
        return HHO_EINVAL;
    }
    ops->sdirk_precond = kind;
    return HHO_OK;
}
