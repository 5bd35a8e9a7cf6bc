// Discrete adjoint of the ERK time stepping (vector-Jacobian product of the
// receiver traces with respect to the materials and the source wavelet).
//
// Forward: k_i = A Y_i + w(t_i) g (A = -M^-1 K_cond, Eq. ex_solve), Y_i the
// stage values of Eq. ERK_compact, U^n = U^{n-1} + dt sum_i b_i k_i, and the
// traces d^n = R U^n (hho_record after every step).
// Backward, for a cotangent G^n = dL/dd^n: lambda^n += R^T G^n, then for the
// stages in reverse order
//     mu_i = dt (b_i lambda^n + sum_{l>i} a_li nu_l),   nu_i = A^T mu_i,
//     lambda^{n-1} = lambda^n + sum_i nu_i,
//     dL/dtheta += mu_i^T dk_i/dtheta,   dL/dw(t_i) += mu_i^T g.
// A^T is applied without a transposed kernel: the block structure of the
// paper's system (Sec. 3.3) gives A^T = S M A' M^-1 S, where S flips the
// signs of the dual fields (m, s) and A' is the same operator with the sign
// of the interface coupling block reversed.  So A^T = mass kernel, forward
// stage kernel on A' (traces + apply), mass kernel.
//
// Parameters.  (1) The per-cell factors of the inverse mass, theta =
// (1/(rho h), kappa/h) in fluid cells and ((lambda+2mu)/h, lambda/(lambda+2mu),
// mu/h, 1/(rho h)) in solid cells; dk/dtheta is the raw rate (MODE_RAW).
// (2) The stabilisation weights tau (Sec. 3.3: tau^f = eta_f/(rho c_P),
// tau^s = eta_s rho c^s).  The full stiffness is affine in tau: dK/dtau_c is
// cell c's least-squares stabilisation (Eq. stab) without its weight, so
//     d(eta^T K_cond Y)/dtau_c = sum_{F of c} (eta_c - eta_F, Y_c - Y_F)_F
// on the primal unknowns, with Y_F the face values of the stage value Y and
// eta_F = -K_F^-T K_TF^T eta the adjoint face values of eta = M^-1 mu.  By the
// same block structure eta_F are the face values of the coupling-reversed
// operator A' applied to x = S eta, which the backward stage computes anyway:
// tau_grad_kernel takes the products of both jumps from the two trace
// buffers.  The interface receivers read face values, which depend on tau
// too (rec_tau_kernel).  The host maps dL/dtheta and dL/dtau to
// dL/d(rho, kappa, lambda, mu); with tau given explicitly
// (hho_operators_build_tau) tau is a constant and only (1) remains.
//
// Checkpointing: U is stored every `checkpoint_every` steps in the forward
// pass; each segment is recomputed, keeping its stage values and their face
// traces, before its backward sweep.
//
// Arithmetic: the driver and its kernels are templates on the state type,
// FP64 (hho_adjoint_vjp) or FP32 (hho_adjoint_vjp_f32: the FP32 stage
// kernels, states, traces and adjoint vectors in FP32); the gradient sums
// are accumulated in FP64 in both.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hho_internal.h"

namespace {

constexpr int MAX_STAGES = 6;   // the largest tableau build_plan accepts

// The operand of the mass kernel: in = a1 in1 + a2 in2 (in2 may be null),
// rounded as axpby_kernel does; stored to `keep` when that is not null.
template <class T>
struct MassIn {
    const T* in1;
    double a1;
    const T* in2;
    double a2;
    T* keep;
};
// Where the result v = S M in (or S M^-1 in) goes: `out` (may be null), and
// the ERK adjoint accumulations acc += v, pend[l] += a[l] v.
template <class T>
struct MassOut {
    T* out;
    T* acc;
    int n_pend;
    T* pend[MAX_STAGES];
    double a[MAX_STAGES];
};

// v = S M in (inverse = 0) or S M^-1 in (inverse = 1) per cell; S = -1 on the
// dual fields (m_x, m_y / s_xx, s_yy, s_xy), +1 on the primal fields.  One
// thread per cell; the operand combination and the accumulations of the
// adjoint stage recursion are fused in (MassIn, MassOut).
template <class T>
__global__ void mass_kernel(DevOps op, const double* __restrict__ mass_f, const double* __restrict__ mass_s,
                            const double* __restrict__ cls_minv, MassIn<T> I, MassOut<T> O, int inverse) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= op.Nf + op.Ns) return;
    const bool fl = g < op.Nf;
    const int q = fl ? g : g - op.Nf;
    const int n = op.n;
    const int cls = op.warp_class[(fl ? 0 : op.n_warps_f) + (q >> 5)];
    const int* ci = op.cls_int + cls * CI_STRIDE;
    if (q - ci[CI_START] >= ci[CI_COUNT]) return;
    const double* Mat = inverse ? cls_minv + (size_t)cls * n * n : op.cls_dbl + ci[CI_DOFF];
    const int N = fl ? op.Nf : op.Ns;
    const size_t off = fl ? 0 : (size_t)3 * n * op.Nf;
    auto idx = [&](int field, int i) { return off + (size_t)(field * n + i) * N + q; };
    T u[10], r[10];
    auto matvec = [&](int field) {
        for (int i = 0; i < n; ++i) {
            const size_t e = idx(field, i);
            T v = T(I.a1) * I.in1[e];
            if (I.in2) v = fma(T(I.a2), I.in2[e], v);
            if (I.keep) I.keep[e] = v;
            u[i] = v;
        }
        for (int i = 0; i < n; ++i) {
            T s = T(0);
            for (int j = 0; j < n; ++j) s = fma(T(Mat[i * n + j]), u[j], s);
            r[i] = s;
        }
    };
    auto emit = [&](int field, int i, T v) {
        const size_t e = idx(field, i);
        if (O.out) O.out[e] = v;
        if (O.acc) O.acc[e] = O.acc[e] + v;
        for (int l = 0; l < O.n_pend; ++l) O.pend[l][e] = fma(T(O.a[l]), v, O.pend[l][e]);
    };
    if (fl) {
        const T cm = T(inverse ? 1.0 / mass_f[q] : mass_f[q]);                 // rho h^2
        const T cp = T(inverse ? 1.0 / mass_f[N + q] : mass_f[N + q]);         // h^2 / kappa
        for (int fld = 0; fld < 3; ++fld) {
            matvec(fld);
            const T c = fld < 2 ? -cm : cp;                                    // S: m negated
            for (int i = 0; i < n; ++i) emit(fld, i, c * r[i]);
        }
    } else {
        // s block: (h^2 D) (x) M0 with D = [[d0, d1, 0], [d1, d0, 0], [0, 0, d2]]
        double d0 = mass_s[q], d1 = mass_s[N + q], d2 = mass_s[2 * N + q];
        const double rv = inverse ? 1.0 / mass_s[3 * N + q] : mass_s[3 * N + q];
        if (inverse) {
            const double det = d0 * d0 - d1 * d1;
            const double e0 = d0 / det, e1 = -d1 / det;
            d0 = e0;
            d1 = e1;
            d2 = 1.0 / d2;
        }
        const T D0 = T(d0), D1 = T(d1), D2 = T(d2), RV = T(rv);
        T t0[10], t1[10];
        matvec(0);
        for (int i = 0; i < n; ++i) t0[i] = r[i];
        matvec(1);
        for (int i = 0; i < n; ++i) t1[i] = r[i];
        for (int i = 0; i < n; ++i) {
            emit(0, i, -(D0 * t0[i] + D1 * t1[i]));
            emit(1, i, -(D1 * t0[i] + D0 * t1[i]));
        }
        matvec(2);
        for (int i = 0; i < n; ++i) emit(2, i, -D2 * r[i]);
        for (int fld = 3; fld < 5; ++fld) {
            matvec(fld);
            for (int i = 0; i < n; ++i) emit(fld, i, RV * r[i]);
        }
    }
}

// out = a x + b y over n values (x or y may be null: treated as zero; out may
// alias x or y, each element is read before it is written by the same thread).
template <class T>
__global__ void axpby_kernel(int64_t n, double a, const T* x, double b, const T* y, T* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v = T(0);
        if (x) v = T(a) * x[i];
        if (y) v = fma(T(b), y[i], v);
        out[i] = v;
    }
}

// lambda += R^T G for one time node: the transpose of record_kernel.  Block t
// owns the t-th cell read by the receivers; thread (field, i) adds the
// contributions of that cell's receivers to lambda[field, i] in increasing
// receiver order, so each entry receives the same sums in the same order as a
// walk over the receivers one by one.  blockDim >= 5 n.
template <class T>
__global__ void inject_kernel(DevOps op, int n_inj, const int32_t* __restrict__ inj, const int32_t* __restrict__ ri,
                              const double* __restrict__ rd, const T* __restrict__ G, T* lam) {
    const int t = blockIdx.x;
    const int n = op.n;
    const int fld = threadIdx.x / n, i = threadIdx.x - fld * n;
    if (t >= n_inj) return;
    const int dom = inj[n_inj + 1 + 2 * t], q = inj[n_inj + 1 + 2 * t + 1];
    if (fld >= (dom == 0 ? 3 : 5)) return;
    const int32_t* recs = inj + 3 * n_inj + 1;
    const int stride = 2 * n + 15;
    const int N = dom == 0 ? op.Nf : op.Ns;
    T* base = dom == 0 ? lam : lam + (size_t)3 * n * op.Nf;
    const size_t idx = (size_t)(fld * n + i) * N + q;
    double acc = base[idx];
    for (int e = inj[t]; e < inj[t + 1]; ++e) {
        const int r = recs[e];
        const double* d = rd + (size_t)r * stride;
        const int kind = ri[4 * r];
        double g[5];
        for (int j = 0; j < 5; ++j) g[j] = (double)G[5 * r + j];
        double v;
        const double* phi = d;
        if (kind == 0) {          // [p, m_x, m_y]
            v = fld == 2 ? g[0] : (fld == 0 ? g[1] : g[2]);
        } else if (kind == 1) {   // [v_x, v_y, s_xx, s_yy, s_xy]
            v = fld == 3 ? g[0] : fld == 4 ? g[1] : fld == 0 ? g[2] : fld == 1 ? g[3] : g[4];
        } else {                  // interface: [p_F, v_F] = Ai [w_f, w_sx, w_sy]
            const double tf = d[2 * n], ts = d[2 * n + 1];
            const double nfx = d[2 * n + 2], nfy = d[2 * n + 3], nsx = d[2 * n + 4], nsy = d[2 * n + 5];
            const double* Ai = d + 2 * n + 6;
            if (dom == 0) {
                const double hf = Ai[0] * g[0] + Ai[3] * g[1] + Ai[6] * g[2];
                v = fld == 2 ? tf * hf : (fld == 0 ? -nfx * hf : -nfy * hf);
            } else {
                const double hx = Ai[1] * g[0] + Ai[4] * g[1] + Ai[7] * g[2];
                const double hy = Ai[2] * g[0] + Ai[5] * g[1] + Ai[8] * g[2];
                phi = d + n;
                v = fld == 3 ? ts * hx
                    : fld == 4 ? ts * hy
                    : fld == 0 ? -nsx * hx
                    : fld == 2 ? -(nsy * hx + nsx * hy)
                               : -nsy * hy;
            }
        }
        if (v != 0.0) acc += v * phi[i];
    }
    base[idx] = T(acc);
}

// dL/dtheta += mu^T dk/dtheta with dk/dtheta from the raw rate (MODE_RAW).
// grad: fluid [2][Nf] (1/(rho h), kappa/h), solid [4][Ns] (c1, r, c3, 1/(rho h)).
template <class T>
__global__ void grad_kernel(DevOps op, const T* __restrict__ mu, const T* __restrict__ raw,
                            double* __restrict__ grad_f, double* __restrict__ grad_s) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= op.Nf + op.Ns) return;
    const bool fl = g < op.Nf;
    const int q = fl ? g : g - op.Nf;
    const int n = op.n;
    const int cls = op.warp_class[(fl ? 0 : op.n_warps_f) + (q >> 5)];
    const int* ci = op.cls_int + cls * CI_STRIDE;
    if (q - ci[CI_START] >= ci[CI_COUNT]) return;
    const int N = fl ? op.Nf : op.Ns;
    const size_t off = fl ? 0 : (size_t)3 * n * op.Nf;
    auto dot = [&](int fa, int fb) {
        double s = 0.0;
        for (int i = 0; i < n; ++i)
            s = fma((double)mu[off + (size_t)(fa * n + i) * N + q], (double)raw[off + (size_t)(fb * n + i) * N + q], s);
        return s;
    };
    if (fl) {
        grad_f[q] += dot(0, 0) + dot(1, 1);
        grad_f[N + q] += dot(2, 2);
    } else {
        const double c1 = op.scal_s[SS_C1 * N + q], r = op.scal_s[SS_R * N + q];
        const double sxx_exx = dot(0, 0), sxx_eyy = dot(0, 1), syy_exx = dot(1, 0), syy_eyy = dot(1, 1);
        grad_s[q] += sxx_exx + r * sxx_eyy + syy_eyy + r * syy_exx;      // d/dc1
        grad_s[N + q] += c1 * (sxx_eyy + syy_exx);                      // d/dr
        grad_s[2 * N + q] += dot(2, 2);                                  // d/dc3
        grad_s[3 * N + q] += dot(3, 3) + dot(4, 4);                      // d/d(1/(rho h))
    }
}

// (psi_l, psi_m) over a face of unit length: the face basis
// psi_l = (rho0 xi)^l, xi in [-1, 1], gives rho0^(l+m) / (l+m+1) for even
// l + m and 0 otherwise.
__device__ __forceinline__ double face_gram(int l, int m) {
    if ((l + m) & 1) return 0.0;
    double r = 1.0;
    for (int e = 0; e < l + m; ++e) r *= FACE_RHO;
    return r / (l + m + 1);
}

// Stabilisation-weight part of one backward stage: for every cell,
// gstab += sum_F |F|/h jY^T G jX, the face integrals (G = face_gram) of the
// products of the primal jumps u_F - u|_F of the
// forward stage value (traces trY, coefficients of op) and of x = S M^-1 mu
// (traces trX under the coupling-reversed operator opx).  The host multiplies
// by -h per cell.  Same jump formulas as the stage kernel's face rates.
template <class T>
__global__ void tau_grad_kernel(DevOps op, DevOps opx, const T* __restrict__ trY, const T* __restrict__ trX,
                                double* __restrict__ gstab) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= op.Nf + op.Ns) return;
    const bool fl = g < op.Nf;
    const int q = fl ? g : g - op.Nf;
    const int n = op.n, f = op.f;
    const int cls = op.warp_class[(fl ? 0 : op.n_warps_f) + (q >> 5)];
    const int* ci = op.cls_int + cls * CI_STRIDE;
    const int lq = q - ci[CI_START];
    if (lq >= ci[CI_COUNT]) return;
    const int nF = ci[CI_NF], npad = ci[CI_NPAD], sbase = ci[CI_SLOT];
    const int nP = (n + 3) / 4 * 4, fP = (f + 3) / 4 * 4, M0P = (n * n + 3) / 4 * 4, FS = 4 + f * nP + n * fP;
    const double* cd = op.cls_dbl + ci[CI_DOFF] + M0P;
    const int SF = op.SF, SS = op.SS;
    const T* yf = trY;
    const T* ys = trY + (size_t)2 * f * SF;
    const T* xf = trX;
    const T* xs = trX + (size_t)2 * f * SF;
    double acc = 0.0;
    for (int j = 0; j < nF; ++j) {
        const double rel = cd[j * FS + 2];   // |F| / h
        const int slot = sbase + j * npad + lq;
        double sum = 0.0;
        double ja[2][4], jb[2][4];   // jumps (Y, X) of up to two components
        if (fl) {
            const int nb = op.nb_f[slot];
            for (int l = 0; l < f; ++l) {
                const double sg = (l & 1) ? -1.0 : 1.0;
                double jy = (double)yf[(size_t)(f + l) * SF + slot], jx = (double)xf[(size_t)(f + l) * SF + slot];
                if (nb >= 0) {
                    const double be = op.beta_f[slot];
                    jy += sg * be * yf[(size_t)l * SF + nb];
                    jx += sg * be * xf[(size_t)l * SF + nb];
                } else if (nb < NB_BOUNDARY) {
                    const int r = -2 - nb, ns = op.if_nb[r];
                    const double* cy = op.if_coef + 6 * r;
                    const double* cx = opx.if_coef + 6 * r;
                    jy += sg * (cy[1] * ys[(size_t)l * SS + ns] + cy[2] * ys[(size_t)(f + l) * SS + ns]);
                    jx += sg * (cx[1] * xs[(size_t)l * SS + ns] + cx[2] * xs[(size_t)(f + l) * SS + ns]);
                }
                ja[0][l] = jy;
                jb[0][l] = jx;
            }
            for (int l = 0; l < f; ++l)
                for (int m = 0; m < f; ++m) sum += ja[0][l] * face_gram(l, m) * jb[0][m];
        } else {
            const int nb = op.nb_s[slot];
            for (int l = 0; l < f; ++l) {
                const double sg = (l & 1) ? -1.0 : 1.0;
                double jyx = (double)ys[(size_t)(2 * f + l) * SS + slot], jyy = (double)ys[(size_t)(3 * f + l) * SS + slot];
                double jxx = (double)xs[(size_t)(2 * f + l) * SS + slot], jxy = (double)xs[(size_t)(3 * f + l) * SS + slot];
                if (nb >= 0) {
                    const double be = op.beta_s[slot];
                    jyx += sg * be * ys[(size_t)l * SS + nb];
                    jyy += sg * be * ys[(size_t)(f + l) * SS + nb];
                    jxx += sg * be * xs[(size_t)l * SS + nb];
                    jxy += sg * be * xs[(size_t)(f + l) * SS + nb];
                } else if (nb < NB_BOUNDARY) {
                    const int r = -2 - nb, nfs = op.if_nb[r];
                    const double* cy = op.if_coef + 6 * r;
                    const double* cx = opx.if_coef + 6 * r;
                    const double wy = (double)yf[(size_t)l * SF + nfs], wx = (double)xf[(size_t)l * SF + nfs];
                    jyx += sg * cy[4] * wy;
                    jyy += sg * cy[5] * wy;
                    jxx += sg * cx[4] * wx;
                    jxy += sg * cx[5] * wx;
                }
                ja[0][l] = jyx;
                ja[1][l] = jyy;
                jb[0][l] = jxx;
                jb[1][l] = jxy;
            }
            for (int l = 0; l < f; ++l)
                for (int m = 0; m < f; ++m)
                    sum += (ja[0][l] * jb[0][m] + ja[1][l] * jb[1][m]) * face_gram(l, m);
        }
        acc += rel * sum;
    }
    gstab[g] += acc;
}

// d(G^T d)/dtau of the interface receivers at one time node.  Such a
// receiver records [p_F, v_F] = Ai w at its point, w = (tau_f p - m.n_f,
// tau_s v - s n_s) from the two cells' values there and A = [tau_f, n^T;
// -n, tau_s I]; so dd/dtau_f = Ai e_0 (p - p_F) and dd/dtau_s = Ai [0; v - v_F].
// grec[2r] (the fluid cell's tau) and grec[2r + 1] (the solid cell's) sum
// these over the time nodes; other receivers do not depend on tau.
template <class T>
__global__ void rec_tau_kernel(DevOps op, int n_rec, const int32_t* __restrict__ ri, const double* __restrict__ rd,
                               const T* __restrict__ state, const T* __restrict__ G, double* grec) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rec || ri[4 * r] != 2) return;
    const int n = op.n;
    const double* d = rd + (size_t)r * (2 * n + 15);
    const int qf = ri[4 * r + 1], qs = ri[4 * r + 2];
    const T* sf = state;
    const T* ss = state + (size_t)3 * n * op.Nf;
    auto ev = [&](const T* base, int N, int q, int field, const double* phi) {
        double v = 0.0;
        for (int i = 0; i < n; ++i) v = fma(phi[i], (double)base[(size_t)(field * n + i) * N + q], v);
        return v;
    };
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
    const double o0 = Ai[0] * wf + Ai[1] * wsx + Ai[2] * wsy;
    const double o1 = Ai[3] * wf + Ai[4] * wsx + Ai[5] * wsy;
    const double o2 = Ai[6] * wf + Ai[7] * wsx + Ai[8] * wsy;
    double g[3];
    for (int j = 0; j < 3; ++j) g[j] = (double)G[5 * r + j];
    const double hf = Ai[0] * g[0] + Ai[3] * g[1] + Ai[6] * g[2];   // (Ai^T g)
    const double hx = Ai[1] * g[0] + Ai[4] * g[1] + Ai[7] * g[2];
    const double hy = Ai[2] * g[0] + Ai[5] * g[1] + Ai[8] * g[2];
    grec[2 * r] += hf * (p - o0);
    grec[2 * r + 1] += hx * (vx - o1) + hy * (vy - o2);
}

// dL/dw for each point source: mu^T g over the source cell's coefficients
// (the stage rate carries w(t) g, g the source's lifted load vector).
struct SrcMeta {
    int n;
    int dom[MAX_SOURCES];
    int q[MAX_SOURCES];
};
template <class T>
__global__ void wavelet_grad_kernel(DevOps op, SrcMeta meta, const T* __restrict__ g, const T* __restrict__ mu,
                                    double* out) {
    const int s = threadIdx.x;
    if (s >= meta.n) return;
    const int n = op.n;
    const int q = meta.q[s];
    double acc = 0.0;
    if (meta.dom[s] == 0) {
        for (int i = 0; i < n; ++i)
            acc = fma((double)mu[(size_t)(2 * n + i) * op.Nf + q], (double)g[(size_t)s * 2 * n + i], acc);
    } else {
        const T* ms = mu + (size_t)3 * n * op.Nf;
        for (int i = 0; i < n; ++i) {
            acc = fma((double)ms[(size_t)(3 * n + i) * op.Ns + q], (double)g[(size_t)s * 2 * n + i], acc);
            acc = fma((double)ms[(size_t)(4 * n + i) * op.Ns + q], (double)g[(size_t)s * 2 * n + n + i], acc);
        }
    }
    out[s] = acc;
}

template <class E>
struct AdjBuffers {
    int64_t S, T;           // state and trace sizes
    E *ckpt, *stages, *stage_tr, *erk_work, *lam, *mu, *x, *y, *acc, *pend, *raw, *tr;
    double *grad_f, *grad_s, *wgrad;
    double *gstab, *grec;   // tau parts: per device cell slot; per receiver (fluid, solid)
};

// Work layout in elements of E; the FP64 gradient sums take 8 / sizeof(E)
// elements per value (every piece starts on a 128-byte boundary).
template <class E>
int64_t adjoint_layout(const hho_ops* ops, const hho_tableau* tab, int64_t nsteps, int64_t C, AdjBuffers<E>* b,
                       E* base) {
    const int s = tab->s;
    const int64_t S = ops->n_state, T = ops->trace_doubles;
    const int64_t n_ckpt = (nsteps + C - 1) / C + 1;
    int64_t erk = 0;
    hho_work_size(ops, tab, &erk);
    int64_t off = 0;
    auto take = [&](int64_t n) {
        E* p = base ? base + off : nullptr;
        off += (n + 31) / 32 * 32;
        return p;
    };
    constexpr int64_t DW = (int64_t)(sizeof(double) / sizeof(E));
    auto take_d = [&](int64_t n) { return reinterpret_cast<double*>(take(n * DW)); };
    AdjBuffers<E> B;
    B.S = S;
    B.T = T;
    B.ckpt = take(n_ckpt * S);
    B.stages = take((C * s + 1) * S);     // stage inputs of a segment, then its end state
    B.stage_tr = take((C * s + 1) * T);   // their face traces
    B.erk_work = take(erk);
    B.lam = take(S);
    B.mu = take(S);
    B.x = take(S);
    B.y = take(S);
    B.acc = take(S);
    B.pend = take(s * S);
    B.raw = take(S);
    B.tr = take(T);
    B.grad_f = take_d(2 * (int64_t)ops->dev.Nf);
    B.grad_s = take_d(4 * (int64_t)ops->dev.Ns);
    B.wgrad = take_d(nsteps * s * MAX_SOURCES);
    B.gstab = take_d((int64_t)ops->dev.Nf + ops->dev.Ns);
    B.grec = take_d(2 * (int64_t)std::max(ops->n_rec, 1));
    if (b) *b = B;
    return off;
}

int64_t grid1(int64_t n) {
    int64_t g = (n + 255) / 256;
    return g > 4096 ? 4096 : (g < 1 ? 1 : g);
}

// the stage launcher and the operator data of the arithmetic
template <class E>
void launch_stage_t(const hho_ops* ops, int mode, StageArgsT<E>& a, double tn, int j, double cdt, bool sources,
                    void* stream);
template <>
void launch_stage_t<double>(const hho_ops* ops, int mode, StageArgsT<double>& a, double tn, int j, double cdt,
                            bool sources, void* stream) {
    launch_stage_f64(ops, mode, a, 1, tn, j, cdt, sources, stream);
}
template <>
void launch_stage_t<float>(const hho_ops* ops, int mode, StageArgsT<float>& a, double tn, int j, double cdt,
                           bool sources, void* stream) {
    launch_stage_f32(ops, mode, a, 1, tn, j, cdt, sources, stream);
}
int forward_steps(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t n, double* x, double* w,
                  void* stream) {
    return hho_erk_step(ops, tab, t0, dt, n, x, w, stream);
}
int forward_steps(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t n, float* x, float* w,
                  void* stream) {
    return erk_steps_f32(ops, tab, t0, dt, n, x, w, stream);
}
const double* src_vectors(const hho_ops* ops, const double*) { return ops->d_src_g; }
const float* src_vectors(const hho_ops* ops, const float*) { return ops->d_src_g32; }

template <class E>
int adjoint_vjp_t(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps, int64_t checkpoint_every,
                  const E* d_state0, const E* d_cotangent, E* d_work, int64_t work_elems, double* h_grad_cell,
                  double* h_grad_wavelet, double* h_grad_tau, void* stream, const char* who);

}  // namespace

extern "C" int hho_adjoint_work_size(const hho_ops* ops, const hho_tableau* tab, int64_t nsteps,
                                     int64_t checkpoint_every, int64_t* n_doubles) {
    if (!ops || !tab || !n_doubles || nsteps < 1 || checkpoint_every < 1) {
        hho_set_error("hho_adjoint_work_size: bad arguments");
        return HHO_EINVAL;
    }
    *n_doubles = adjoint_layout<double>(ops, tab, nsteps, checkpoint_every, nullptr, nullptr);
    return HHO_OK;
}

extern "C" int hho_adjoint_work_size_f32(const hho_ops* ops, const hho_tableau* tab, int64_t nsteps,
                                         int64_t checkpoint_every, int64_t* n_floats) {
    if (!ops || !tab || !n_floats || nsteps < 1 || checkpoint_every < 1) {
        hho_set_error("hho_adjoint_work_size_f32: bad arguments");
        return HHO_EINVAL;
    }
    *n_floats = adjoint_layout<float>(ops, tab, nsteps, checkpoint_every, nullptr, nullptr);
    return HHO_OK;
}

extern "C" int hho_adjoint_vjp(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps,
                               int64_t checkpoint_every, const double* d_state0, const double* d_cotangent,
                               double* d_work, int64_t work_doubles, double* h_grad_cell, double* h_grad_wavelet,
                               double* h_grad_tau, void* stream) {
    return adjoint_vjp_t<double>(ops, tab, t0, dt, nsteps, checkpoint_every, d_state0, d_cotangent, d_work,
                                 work_doubles, h_grad_cell, h_grad_wavelet, h_grad_tau, stream, "hho_adjoint_vjp");
}

extern "C" int hho_adjoint_vjp_f32(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps,
                                   int64_t checkpoint_every, const float* d_state0, const float* d_cotangent,
                                   float* d_work, int64_t work_floats, double* h_grad_cell, double* h_grad_wavelet,
                                   double* h_grad_tau, void* stream) {
    return adjoint_vjp_t<float>(ops, tab, t0, dt, nsteps, checkpoint_every, d_state0, d_cotangent, d_work,
                                work_floats, h_grad_cell, h_grad_wavelet, h_grad_tau, stream, "hho_adjoint_vjp_f32");
}

namespace {
template <class E>
int adjoint_vjp_t(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps, int64_t checkpoint_every,
                  const E* d_state0, const E* d_cotangent, E* d_work, int64_t work_doubles, double* h_grad_cell,
                  double* h_grad_wavelet, double* h_grad_tau, void* stream, const char* who) {
    if (!ops || !tab || !d_state0 || !d_cotangent || !d_work || !h_grad_cell || nsteps < 1 || checkpoint_every < 1 ||
        !std::isfinite(dt)) {
        hho_set_error("%s: bad arguments", who);
        return HHO_EINVAL;
    }
    std::vector<StagePlan> plan;
    int nb = 0;
    if (build_plan(tab, plan, &nb) != HHO_OK) {
        hho_set_error("%s: unsupported tableau", who);
        return HHO_EINVAL;
    }
    const int64_t C = checkpoint_every;
    const int s = tab->s;
    AdjBuffers<E> B;
    const int64_t need = adjoint_layout<E>(ops, tab, nsteps, C, &B, d_work);
    if (work_doubles < need) {
        hho_set_error("%s: work buffer has %lld elements, needs %lld", who, (long long)work_doubles, (long long)need);
        return HHO_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t S = B.S;
    const int nthr = ops->dev.Nf + ops->dev.Ns;
    const int cblk = (nthr + 127) / 128;
    int rc = HHO_OK;
    auto copy = [&](E* dst, const E* src, int64_t n) {
        return cudaMemcpyAsync(dst, src, sizeof(E) * n, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    };
    // the ERK partial-sum buffers of the segment recompute, laid out as in
    // erk_run ([X][partial sums][2 traces]; X and the traces live in the
    // segment store here)
    E* bufs = B.erk_work + S;
    auto partial = [&](int code) -> E* { return code == SRC_ZERO ? nullptr : bufs + S * code; };
    DevOps adj = ops->dev;
    adj.if_coef = ops->d_if_coef_adj;
    adj.if_coef_f32 = ops->d_if_coef_adj_f32;

    // ---- forward pass: checkpoints ------------------------------------------------
    if (!copy(B.ckpt, d_state0, S)) {
        hho_set_error("%s: copy failed", who);
        return HHO_ECUDA;
    }
    const int64_t n_ckpt = (nsteps + C - 1) / C;
    for (int64_t c = 1; c < n_ckpt + 1 && c * C <= nsteps; ++c) {
        if (!copy(B.ckpt + c * S, B.ckpt + (c - 1) * S, S)) return HHO_ECUDA;
        rc = forward_steps(ops, tab, t0 + (double)((c - 1) * C) * dt, dt, C, B.ckpt + c * S, B.erk_work, stream);
        if (rc) return rc;
    }

    // ---- backward sweep ---------------------------------------------------------------
    axpby_kernel<E><<<grid1(S), 256, 0, st>>>(S, 0.0, nullptr, 0.0, nullptr, B.lam);
    if (ops->dev.Nf > 0)
        axpby_kernel<double><<<grid1(2 * (int64_t)ops->dev.Nf), 256, 0, st>>>(2 * (int64_t)ops->dev.Nf, 0.0, nullptr,
                                                                               0.0, nullptr, B.grad_f);
    if (ops->dev.Ns > 0)
        axpby_kernel<double><<<grid1(4 * (int64_t)ops->dev.Ns), 256, 0, st>>>(4 * (int64_t)ops->dev.Ns, 0.0, nullptr,
                                                                               0.0, nullptr, B.grad_s);
    axpby_kernel<double><<<grid1((int64_t)nthr), 256, 0, st>>>((int64_t)nthr, 0.0, nullptr, 0.0, nullptr, B.gstab);
    axpby_kernel<double><<<1, 256, 0, st>>>(2 * (int64_t)std::max(ops->n_rec, 1), 0.0, nullptr, 0.0, nullptr, B.grec);
    const int64_t n_segments = (nsteps + C - 1) / C;
    for (int64_t seg = n_segments - 1; seg >= 0; --seg) {
        const int64_t n0 = seg * C;                                   // segment starts at U^{n0}
        const int64_t nst = (n0 + C <= nsteps) ? C : nsteps - n0;
        // Recompute the segment.  Stage j of step m reads its input Y_{m,j}
        // and that input's face traces from slot m s + j of the segment store
        // and writes the next stage input (slot m s + j + 1, or the next
        // step's state in slot (m + 1) s) with its traces straight into the
        // store: no copies, and the backward sweep needs no trace launch for
        // the forward stage values.
        auto Y = [&](int64_t m, int j) { return B.stages + (m * s + j) * S; };
        auto TY = [&](int64_t m, int j) { return B.stage_tr + (m * s + j) * B.T; };
        if (!copy(Y(0, 0), B.ckpt + seg * S, S)) return HHO_ECUDA;
        StageArgsT<E> a;
        memset(&a, 0, sizeof(a));
        a.op = ops->dev;
        a.inp = Y(0, 0);
        a.tr_out = TY(0, 0);
        launch_stage_t<E>(ops, MODE_TRACES, a, 0.0, -1, 0.0, false, stream);
        for (int64_t m = 0; m < nst; ++m) {
            const double tn = t0 + (double)(n0 + m) * dt;
            for (int j = 0; j < s; ++j) {
                const StagePlan& P = plan[j];
                const bool last = j + 1 == s;
                a.inp = Y(m, j);
                a.tr_in = TY(m, j);
                a.tr_out = last ? TY(m + 1, 0) : TY(m, j + 1);
                a.n_tgt = P.n_tgt;
                for (int t = 0; t < P.n_tgt; ++t) {
                    const int sc = P.t[t].src, dc = P.t[t].dst;
                    a.tgt[t].src = sc == SRC_STATE ? Y(m, 0) : partial(sc);
                    a.tgt[t].dst = dc == SRC_STATE ? Y(m + 1, 0) : dc == SRC_X ? Y(m, j + 1) : partial(dc);
                    a.tgt[t].coef = E(P.t[t].a * dt);
                }
                launch_stage_t<E>(ops, MODE_STAGE, a, tn, j, tab->c[j] * dt, true, stream);
            }
        }
        rc = check_cuda(who);
        if (rc) return rc;
        // backward through the segment
        for (int64_t m = nst - 1; m >= 0; --m) {
            const int64_t n = n0 + m + 1;                            // step n: U^{n-1} -> U^n
            const double tn = t0 + (double)(n - 1) * dt;
            if (ops->n_inj > 0)
                inject_kernel<E><<<ops->n_inj, (5 * ops->n + 31) / 32 * 32, 0, st>>>(
                    ops->dev, ops->n_inj, ops->d_inj, ops->d_rec_int, ops->d_rec_dbl,
                    d_cotangent + (size_t)(n - 1) * 5 * ops->n_rec, B.lam);
            if (ops->n_rec > 0)   // U^n is the next step's first stage value in the store
                rec_tau_kernel<E><<<(ops->n_rec + 63) / 64, 64, 0, st>>>(ops->dev, ops->n_rec, ops->d_rec_int,
                                                                     ops->d_rec_dbl, Y(m + 1, 0),
                                                                     d_cotangent + (size_t)(n - 1) * 5 * ops->n_rec,
                                                                     B.grec);
            if (!copy(B.acc, B.lam, S)) return HHO_ECUDA;
            axpby_kernel<E><<<grid1(s * S), 256, 0, st>>>(s * S, 0.0, nullptr, 0.0, nullptr, B.pend);
            for (int j = s - 1; j >= 0; --j) {
                // mu_j = dt (b_j lambda + P_j), x = M^-1 S mu_j
                const MassIn<E> mi = {B.lam, dt * tab->b[j], B.pend + j * S, dt, B.mu};
                MassOut<E> mo;
                memset(&mo, 0, sizeof(mo));
                mo.out = B.x;
                mass_kernel<E><<<cblk, 128, 0, st>>>(ops->dev, ops->d_mass_f, ops->d_mass_s, ops->d_cls_minv, mi, mo, 1);
                // nu_j = S M A' x, accumulated into acc and the pending sums P_l (l < j)
                StageArgsT<E> b;
                memset(&b, 0, sizeof(b));
                b.op = adj;
                b.inp = B.x;
                b.tr_out = B.tr;
                launch_stage_t<E>(ops, MODE_TRACES, b, 0.0, -1, 0.0, false, stream);
                b.tr_in = B.tr;
                b.tr_out = nullptr;
                b.n_tgt = 1;
                b.tgt[0].src = nullptr;
                b.tgt[0].dst = B.y;
                b.tgt[0].coef = E(1.0);
                launch_stage_t<E>(ops, MODE_APPLY, b, 0.0, -1, 0.0, false, stream);
                // the stabilisation weights' part: forward jumps of Y_{m,j} against those of x under A'
                tau_grad_kernel<E><<<cblk, 128, 0, st>>>(ops->dev, adj, TY(m, j), B.tr, B.gstab);
                const MassIn<E> ni = {B.y, 1.0, nullptr, 0.0, nullptr};
                MassOut<E> no;
                memset(&no, 0, sizeof(no));
                no.acc = B.acc;
                for (int l = 0; l < j; ++l)
                    if (tab->a[j][l] != 0.0) {
                        no.pend[no.n_pend] = B.pend + l * S;
                        no.a[no.n_pend++] = tab->a[j][l];
                    }
                mass_kernel<E><<<cblk, 128, 0, st>>>(ops->dev, ops->d_mass_f, ops->d_mass_s, ops->d_cls_minv, ni, no, 0);
                // parameter and wavelet gradients of stage j (the forward traces of Y_{m,j} are stored)
                StageArgsT<E> r;
                memset(&r, 0, sizeof(r));
                r.op = ops->dev;
                r.inp = Y(m, j);
                r.tr_in = TY(m, j);
                r.tr_out = nullptr;
                r.n_tgt = 1;
                r.tgt[0].src = nullptr;
                r.tgt[0].dst = B.raw;
                r.tgt[0].coef = E(1.0);
                launch_stage_t<E>(ops, MODE_RAW, r, tn, j, tab->c[j] * dt, true, stream);
                grad_kernel<E><<<cblk, 128, 0, st>>>(ops->dev, B.mu, B.raw, B.grad_f, B.grad_s);
                if (ops->n_src > 0 && h_grad_wavelet) {
                    SrcMeta meta;
                    meta.n = ops->n_src;
                    for (int k2 = 0; k2 < ops->n_src; ++k2) {
                        meta.dom[k2] = ops->src_dom[k2];
                        meta.q[k2] = ops->src_q[k2];
                    }
                    wavelet_grad_kernel<E><<<1, 32, 0, st>>>(ops->dev, meta, src_vectors(ops, (const E*)nullptr), B.mu,
                                                             B.wgrad + ((n - 1) * s + j) * MAX_SOURCES);
                }
                rc = check_cuda(who);
                if (rc) return rc;
            }
            if (!copy(B.lam, B.acc, S)) return HHO_ECUDA;
        }
    }
    // ---- gradients to the host, mapped to the materials ----------------------------------------
    std::vector<double> gf(2 * (size_t)ops->dev.Nf), gs(4 * (size_t)ops->dev.Ns);
    std::vector<double> gstab((size_t)nthr), grec(2 * (size_t)std::max(ops->n_rec, 1));
    if ((!gf.empty() && cudaMemcpyAsync(gf.data(), B.grad_f, sizeof(double) * gf.size(), cudaMemcpyDeviceToHost, st) !=
                            cudaSuccess) ||
        (!gs.empty() && cudaMemcpyAsync(gs.data(), B.grad_s, sizeof(double) * gs.size(), cudaMemcpyDeviceToHost, st) !=
                            cudaSuccess) ||
        (!gstab.empty() &&
         cudaMemcpyAsync(gstab.data(), B.gstab, sizeof(double) * gstab.size(), cudaMemcpyDeviceToHost, st) !=
             cudaSuccess) ||
        cudaMemcpyAsync(grec.data(), B.grec, sizeof(double) * grec.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        hho_set_error("%s: gradient copy failed", who);
        return HHO_ECUDA;
    }
    if (ops->n_src > 0 && h_grad_wavelet) {
        std::vector<double> wg((size_t)nsteps * s * MAX_SOURCES);
        if (cudaMemcpy(wg.data(), B.wgrad, sizeof(double) * wg.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
            hho_set_error("%s: wavelet gradient copy failed", who);
            return HHO_ECUDA;
        }
        for (int64_t n = 0; n < nsteps; ++n)
            for (int j = 0; j < s; ++j)
                for (int k2 = 0; k2 < ops->n_src; ++k2)
                    h_grad_wavelet[(n * s + j) * ops->n_src + k2] = wg[(n * s + j) * MAX_SOURCES + k2];
    }
    const int Nf = ops->dev.Nf, Ns = ops->dev.Ns;
    // dL/dtau per cell: the stage part (face integrals scale with h) and the
    // interface receivers' part, mapped from device positions to cell ids
    std::vector<double> gtau((size_t)ops->nc, 0.0);
    std::vector<int64_t> orig_f((size_t)Nf, -1), orig_s((size_t)Ns, -1);
    for (int64_t c = 0; c < ops->nc; ++c) {
        const int q = ops->cell_pos[c];
        (ops->cell_dom[c] == 0 ? orig_f : orig_s)[q] = c;
        gtau[c] = -ops->diam[c] * gstab[(ops->cell_dom[c] == 0 ? 0 : Nf) + q];
    }
    {
        std::vector<int32_t> ri(4 * (size_t)std::max(ops->n_rec, 1));
        if (ops->n_rec > 0 &&
            cudaMemcpy(ri.data(), ops->d_rec_int, sizeof(int32_t) * 4 * ops->n_rec, cudaMemcpyDeviceToHost) !=
                cudaSuccess) {
            hho_set_error("%s: receiver table copy failed", who);
            return HHO_ECUDA;
        }
        for (int r = 0; r < ops->n_rec; ++r)
            if (ri[4 * r] == 2) {
                gtau[orig_f[ri[4 * r + 1]]] += grec[2 * r];
                gtau[orig_s[ri[4 * r + 2]]] += grec[2 * r + 1];
            }
    }
    if (h_grad_tau)
        for (int64_t c = 0; c < ops->nc; ++c) h_grad_tau[c] = gtau[c];
    for (int64_t c = 0; c < ops->nc; ++c) {
        double* o = h_grad_cell + 4 * c;   // [rho, kappa, lambda, mu]
        o[0] = o[1] = o[2] = o[3] = 0.0;
        const int q = ops->cell_pos[c];
        const double h = ops->diam[c], rho = ops->rho[c];
        if (ops->cell_dom[c] == 0) {
            o[0] = gf[q] * (-1.0 / (rho * rho * h));                       // A_m = 1/(rho h)
            o[1] = gf[Nf + q] / h;                                          // A_p = kappa/h
        } else {
            const double lam = ops->lam[c], mu = ops->mu[c], l2m = lam + 2.0 * mu;
            const double gc1 = gs[q], gr = gs[Ns + q], gc3 = gs[2 * Ns + q], gav = gs[3 * Ns + q];
            o[0] = gav * (-1.0 / (rho * rho * h));                          // A_v = 1/(rho h)
            o[2] = gc1 / h + gr * (2.0 * mu / (l2m * l2m));                 // c1 = (lambda+2mu)/h, r = lambda/(lambda+2mu)
            o[3] = gc1 * 2.0 / h + gr * (-2.0 * lam / (l2m * l2m)) + gc3 / h;   // c3 = mu/h
        }
        if (ops->tau_explicit) continue;
        // tau^f = eta_f (rho kappa)^-1/2; tau^s = eta_s (rho (lambda + 2 mu))^1/2 or eta_s (rho mu)^1/2
        // (an optional 1/k factor cancels in these logarithmic derivatives)
        const double t = ops->tau[c], gt = gtau[c];
        if (ops->cell_dom[c] == 0) {
            o[0] += gt * (-0.5 * t / rho);
            o[1] += gt * (-0.5 * t / ops->kappa[c]);
        } else if (ops->stab_speed == 0) {
            const double l2m = ops->lam[c] + 2.0 * ops->mu[c];
            o[0] += gt * (0.5 * t / rho);
            o[2] += gt * (0.5 * t / l2m);
            o[3] += gt * (t / l2m);
        } else {
            o[0] += gt * (0.5 * t / rho);
            o[3] += gt * (0.5 * t / ops->mu[c]);
        }
    }
    return HHO_OK;
}
}  // namespace
