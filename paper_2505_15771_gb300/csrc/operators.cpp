// Operator build (Sec. 3.3): per-class reference matrices in FP64, the device
// layout, per-cell scalars and the face-side exchange tables.
//
// What a stage needs, per cell T of diameter h (all matrices dimensionless, in
// the scaled-monomial basis phi_(a,b) = X^a Y^b, X = (x - x_T)/h):
//   * the trace of a cell polynomial on local face j in the face basis
//     psi_l = (rho0 xi)^l, l <= k, rho0 = 1/(2 sqrt 2) (FACE_RHO), with xi in
//     [-1, 1] running along the counter-clockwise edge: Tr_j (f x n);
//   * the lifting of a face polynomial, Lift_j = M0^-1 B_j (n x f), where
//     M0 = (phi_j, phi_i)_T and B_j = (psi_l, phi_i)_F in scaled coordinates;
//   * the outward unit normal n_j.
// With these, the weak form (Eq. rec, Eq. stab, mass Eq. mass) gives, for the
// jump J_F = u_F - u_T|_F on each face:
//   dm/dt = 1/(rho h) [ grad^ p + sum_F n_F Lift_F J_F ]
//   dp/dt = kappa/h   [ div^ m  + tau sum_F Lift_F J_F ]
//   ds/dt = C/h       [ grad_sym^ v + sum_F sym(n_F (x) Lift_F J_F) ]
//   dv/dt = 1/(rho h) [ div^ s  + tau sum_F Lift_F J_F ]
// (hats: derivatives in scaled coordinates), which is the condensed operator
// of Eq. ex_solve applied cell by cell.
//
// Any basis of P_k(F) serves the face solve (Eq. ex_solve): the trace of a
// cell polynomial on a straight face is a polynomial of degree k, so both
// sides' traces, fluxes and the face unknown are exact coefficient vectors
// and the face equations hold coefficient by coefficient.  The scaled
// monomials psi_l make the traces of a square cell (X, Y = +-rho0 on its
// faces) single terms: X^a Y^b traces to (+-rho0)^b psi_a on a horizontal
// face, so the square kernels evaluate them by Horner's rule in +-rho0
// without reading a matrix.
//
// Integration route: fan of triangles from the centroid, each integrated with
// a collapsed (Duffy) Gauss-Legendre rule; Legendre nodes by Newton's method.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "hho_internal.h"

namespace {

void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
    x.assign(q, 0.0);
    w.assign(q, 0.0);
    for (int i = 0; i < q; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= q; ++l) {
                double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_q(z), p0 = P_{q-1}(z)
            double dp = q * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        double p0 = 1.0, p1 = z;
        for (int l = 2; l <= q; ++l) {
            double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
            p0 = p1;
            p1 = p2;
        }
        double dp = q * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// psi_l(xi) = (rho0 xi)^l, l < f
void face_basis_values(int f, double xi, double* P) {
    P[0] = 1.0;
    for (int l = 1; l < f; ++l) P[l] = P[l - 1] * (FACE_RHO * xi);
}

double ipow(double x, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

double binom(int a, int p) {
    double r = 1.0;
    for (int i = 1; i <= p; ++i) r = r * (a - p + i) / i;
    return r;
}

// Trace of X^a Y^b on the edge (X, Y) = (Xm + Xd xi, Ym + Yd xi), xi in
// [-1, 1], in the basis psi_l: the binomial expansion of both factors,
// coefficient of xi^m divided by rho0^m.
void face_trace_row(int a, int b, double Xm, double Xd, double Ym, double Yd, int f, double* tr) {
    for (int m = 0; m < f; ++m) {
        double c = 0.0;
        for (int p = 0; p <= a && p <= m; ++p) {
            const int q = m - p;
            if (q > b) continue;
            c += binom(a, p) * ipow(Xm, a - p) * ipow(Xd, p) * binom(b, q) * ipow(Ym, b - q) * ipow(Yd, q);
        }
        tr[m] = c / ipow(FACE_RHO, m);
    }
}

void exponents(int k, std::vector<int>& A, std::vector<int>& B) {
    A.clear();
    B.clear();
    for (int d = 0; d <= k; ++d)
        for (int a = d; a >= 0; --a) {
            A.push_back(a);
            B.push_back(d - a);
        }
}

void basis_values(const std::vector<int>& A, const std::vector<int>& B, double X, double Y, double* out) {
    for (size_t i = 0; i < A.size(); ++i) out[i] = std::pow(X, A[i]) * std::pow(Y, B[i]);
}

// Inverse of an SPD matrix by Cholesky (row-major n x n).
bool spd_inverse(int n, const std::vector<double>& M, std::vector<double>& inv) {
    std::vector<double> L(n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = M[j * n + j];
        for (int p = 0; p < j; ++p) d -= L[j * n + p] * L[j * n + p];
        if (!(d > 0.0)) return false;
        L[j * n + j] = std::sqrt(d);
        for (int i = j + 1; i < n; ++i) {
            double s = M[i * n + j];
            for (int p = 0; p < j; ++p) s -= L[i * n + p] * L[j * n + p];
            L[i * n + j] = s / L[j * n + j];
        }
    }
    inv.assign(n * n, 0.0);
    std::vector<double> y(n), x(n);
    for (int col = 0; col < n; ++col) {
        for (int i = 0; i < n; ++i) {
            double s = (i == col) ? 1.0 : 0.0;
            for (int p = 0; p < i; ++p) s -= L[i * n + p] * y[p];
            y[i] = s / L[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = y[i];
            for (int p = i + 1; p < n; ++p) s -= L[p * n + i] * x[p];
            x[i] = s / L[i * n + i];
        }
        for (int i = 0; i < n; ++i) inv[i * n + col] = x[i];
    }
    return true;
}

bool inverse3(const double A[9], double out[9]) {
    double c00 = A[4] * A[8] - A[5] * A[7];
    double c01 = A[5] * A[6] - A[3] * A[8];
    double c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(std::fabs(det) > 0.0)) return false;
    double id = 1.0 / det;
    out[0] = c00 * id;
    out[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    out[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    out[3] = c01 * id;
    out[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    out[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    out[6] = c02 * id;
    out[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    out[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return true;
}

template <class T>
T* dev_upload(hho_ops* ops, const std::vector<T>& h, int* err) {
    if (h.empty()) return nullptr;
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * h.size()) != cudaSuccess) {
        *err = HHO_ENOMEM;
        return nullptr;
    }
    ops->allocations.push_back(p);
    if (cudaMemcpy(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        *err = HHO_ECUDA;
        return nullptr;
    }
    return (T*)p;
}

bool point_in_cell(const std::vector<double>& xy, const int64_t* vtx, int nv, double x, double y) {
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int i = 0; i < nv; ++i) {
        double px = xy[2 * vtx[i]], py = xy[2 * vtx[i] + 1];
        xmin = std::min(xmin, px); xmax = std::max(xmax, px);
        ymin = std::min(ymin, py); ymax = std::max(ymax, py);
    }
    double scale = std::max(xmax - xmin, ymax - ymin);
    for (int i = 0; i < nv; ++i) {
        int j = (i + 1) % nv;
        double ax = xy[2 * vtx[i]], ay = xy[2 * vtx[i] + 1];
        double ex = xy[2 * vtx[j]] - ax, ey = xy[2 * vtx[j] + 1] - ay;
        double cr = ex * (y - ay) - ey * (x - ax);
        if (cr < -1e-12 * scale * scale) return false;
    }
    return true;
}

// Bucket grid for locate(): about one bucket per cell over the mesh's
// bounding box; each cell is listed in every bucket its bounding box
// (enlarged by 1e-9 of its size, beyond point_in_cell's tolerance) meets.
void build_locator(hho_ops* ops) {
    const int64_t nc = ops->nc;
    ops->loc_gx = ops->loc_gy = 0;
    if (nc <= 0) return;
    std::vector<double> bb((size_t)4 * nc);
    double X0 = 1e300, X1 = -1e300, Y0 = 1e300, Y1 = -1e300;
    for (int64_t c = 0; c < nc; ++c) {
        double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
        for (int64_t e = ops->poly_ptr[c]; e < ops->poly_ptr[c + 1]; ++e) {
            const double px = ops->poly_xy[2 * ops->poly_vtx[e]], py = ops->poly_xy[2 * ops->poly_vtx[e] + 1];
            xmin = std::min(xmin, px); xmax = std::max(xmax, px);
            ymin = std::min(ymin, py); ymax = std::max(ymax, py);
        }
        const double pad = 1e-9 * std::max(xmax - xmin, ymax - ymin);
        bb[4 * c + 0] = xmin - pad; bb[4 * c + 1] = xmax + pad;
        bb[4 * c + 2] = ymin - pad; bb[4 * c + 3] = ymax + pad;
        X0 = std::min(X0, bb[4 * c]); X1 = std::max(X1, bb[4 * c + 1]);
        Y0 = std::min(Y0, bb[4 * c + 2]); Y1 = std::max(Y1, bb[4 * c + 3]);
    }
    const double W = std::max(X1 - X0, 1e-300), H = std::max(Y1 - Y0, 1e-300);
    const double target = (double)std::min<int64_t>(nc, (int64_t)1 << 22);
    int64_t gx = std::max<int64_t>(1, std::min<int64_t>(1 << 14, (int64_t)std::llround(std::sqrt(target * W / H))));
    int64_t gy = std::max<int64_t>(1, std::min<int64_t>(1 << 14, (int64_t)std::llround(target / (double)gx)));
    ops->loc_gx = (int32_t)gx;
    ops->loc_gy = (int32_t)gy;
    ops->loc_x0 = X0;
    ops->loc_y0 = Y0;
    ops->loc_dx = W / (double)gx;
    ops->loc_dy = H / (double)gy;
    auto range = [&](double lo, double hi, double o, double d, int64_t g, int64_t* a, int64_t* b) {
        *a = std::min<int64_t>(std::max<int64_t>((int64_t)std::floor((lo - o) / d), 0), g - 1);
        *b = std::min<int64_t>(std::max<int64_t>((int64_t)std::floor((hi - o) / d), 0), g - 1);
    };
    std::vector<int64_t> cnt((size_t)gx * gy + 1, 0);
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            for (size_t i = 1; i < cnt.size(); ++i) cnt[i] += cnt[i - 1];
            ops->loc_ptr.assign(cnt.size(), 0);
            for (size_t i = 1; i < cnt.size(); ++i) ops->loc_ptr[i] = cnt[i - 1];
            ops->loc_ids.assign((size_t)cnt.back(), 0);
            cnt.assign(ops->loc_ptr.begin(), ops->loc_ptr.end());
        }
        for (int64_t c = 0; c < nc; ++c) {
            int64_t ax, bx, ay, by;
            range(bb[4 * c], bb[4 * c + 1], X0, ops->loc_dx, gx, &ax, &bx);
            range(bb[4 * c + 2], bb[4 * c + 3], Y0, ops->loc_dy, gy, &ay, &by);
            for (int64_t j = ay; j <= by; ++j)
                for (int64_t i = ax; i <= bx; ++i) {
                    const int64_t k = j * gx + i;
                    if (pass == 0) ++cnt[k];
                    else ops->loc_ids[(size_t)cnt[k]++] = c;
                }
        }
    }
}

}  // namespace

// BF16 value nearest to x (ties to even), as raw bits
static uint16_t bf16_bits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;   // NaN
    const uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(r >> 16);
}
static float bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}
static int pad16(int v) { return (v + 15) / 16 * 16; }

// Operand tiles of the tensor-core batched stage, per class.  With one
// 128-row block of (cell, shot) pairs of the class:
//   GEMM 1 (lifts):  D1 = J B1, J the face jumps at columns 4 face + l
//     (fluid: p; solid: x components, then y components from column
//     4 n_F), D1's column blocks of 16 the rate
//     accumulators (fluid: m_x, m_y, p before tau; solid: e_xx, e_yy, e_xy,
//     v_x, v_y before tau): B1 = n_F-weighted Lift_F (Eq. rec lifted by M0^-1).
//   GEMM 2 (traces): D2 = X B2, X the stage value's fields, D2's 16-column
//     block per face holding that face's traces (fluid: p, m.n; solid: v_x,
//     v_y, (s n)_x, (s n)_y), f face-basis coefficients each.
// Each B is stored transposed (N x K) in the K-major core-matrix layout of
// tc.cuh, as two BF16 tiles hi and lo with B = hi + lo.
static int tc_tiles(hho_ops* ops, const std::vector<double>& cls_dbl, const std::vector<int32_t>& doff,
                    const std::vector<int32_t>& nfs, const std::vector<int32_t>& doms) {
    const int n = ops->n, f = ops->f, NCL = ops->n_classes;
    const int nP = (n + 3) / 4 * 4, fP = (f + 3) / 4 * 4, M0P = (n * n + 3) / 4 * 4, FS = 4 + f * nP + n * fP;
    std::vector<uint16_t> tiles;
    std::vector<int32_t> meta(6 * (size_t)NCL);
    int kmax = 16, cols = 32;
    int64_t bmax = 0;
    auto off = [](int r, int k, int K) { return (size_t)((r >> 3) * (K >> 3) * 64 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7)); };
    for (int cl = 0; cl < NCL; ++cl) {
        const int nF = nfs[cl];
        const bool sol = doms[cl] != 0;
        // jumps: 4 columns per face (f <= 4), x components then y components
        const int K1 = pad16(sol ? 8 * nF : 4 * nF), N1 = (sol ? 5 : 3) * 16;
        const int K2 = pad16((sol ? 5 : 3) * n), N2 = nF * 16;
        std::vector<double> B1((size_t)N1 * K1, 0.0), B2((size_t)N2 * K2, 0.0);   // transposed: [col][k]
        const double* cd = &cls_dbl[doff[cl] + M0P];
        for (int F = 0; F < nF; ++F) {
            const double* fm = cd + F * FS;
            const double nx = fm[0], ny = fm[1];
            const double* Tr = fm + 4;
            const double* L = fm + 4 + f * nP;
            for (int l = 0; l < f; ++l)
                for (int i = 0; i < n; ++i) {
                    const double lift = L[i * fP + l], tr = Tr[l * nP + i];
                    if (!sol) {
                        const int k = 4 * F + l;
                        B1[(size_t)(0 * 16 + i) * K1 + k] = nx * lift;   // m_x rate
                        B1[(size_t)(1 * 16 + i) * K1 + k] = ny * lift;   // m_y rate
                        B1[(size_t)(2 * 16 + i) * K1 + k] = lift;        // p rate, times tau
                        B2[(size_t)(F * 16 + l) * K2 + 2 * n + i] = tr;                // trace of p
                        B2[(size_t)(F * 16 + f + l) * K2 + i] = nx * tr;               // trace of m.n
                        B2[(size_t)(F * 16 + f + l) * K2 + n + i] = ny * tr;
                    } else {
                        const int kx = 4 * F + l, ky = 4 * nF + 4 * F + l;
                        B1[(size_t)(0 * 16 + i) * K1 + kx] = nx * lift;  // e_xx
                        B1[(size_t)(1 * 16 + i) * K1 + ky] = ny * lift;  // e_yy
                        B1[(size_t)(2 * 16 + i) * K1 + kx] = ny * lift;  // e_xy
                        B1[(size_t)(2 * 16 + i) * K1 + ky] = nx * lift;
                        B1[(size_t)(3 * 16 + i) * K1 + kx] = lift;       // v_x rate, times tau
                        B1[(size_t)(4 * 16 + i) * K1 + ky] = lift;       // v_y rate, times tau
                        B2[(size_t)(F * 16 + l) * K2 + 3 * n + i] = tr;          // v_x
                        B2[(size_t)(F * 16 + f + l) * K2 + 4 * n + i] = tr;      // v_y
                        B2[(size_t)(F * 16 + 2 * f + l) * K2 + i] = nx * tr;     // (s n)_x = nx s_xx + ny s_xy
                        B2[(size_t)(F * 16 + 2 * f + l) * K2 + 2 * n + i] = ny * tr;
                        B2[(size_t)(F * 16 + 3 * f + l) * K2 + 2 * n + i] = nx * tr;   // (s n)_y = nx s_xy + ny s_yy
                        B2[(size_t)(F * 16 + 3 * f + l) * K2 + n + i] = ny * tr;
                    }
                }
        }
        const size_t base = tiles.size();
        meta[6 * cl + 0] = K1;
        meta[6 * cl + 1] = N1;
        meta[6 * cl + 2] = K2;
        meta[6 * cl + 3] = N2;
        meta[6 * cl + 4] = (int32_t)(base * 2 / 16);
        const size_t s1 = (size_t)N1 * K1, s2 = (size_t)N2 * K2;
        meta[6 * cl + 5] = (int32_t)(2 * (2 * s1 + 2 * s2));
        tiles.resize(base + 2 * s1 + 2 * s2, 0);
        uint16_t* t1h = &tiles[base];
        uint16_t* t1l = t1h + s1;
        uint16_t* t2h = t1l + s1;
        uint16_t* t2l = t2h + s2;
        auto put = [&](const std::vector<double>& B, int N, int K, uint16_t* hi, uint16_t* lo) {
            for (int r = 0; r < N; ++r)
                for (int k = 0; k < K; ++k) {
                    const float v = (float)B[(size_t)r * K + k];
                    const uint16_t h = bf16_bits(v);
                    hi[off(r, k, K)] = h;
                    lo[off(r, k, K)] = bf16_bits(v - bf16_value(h));
                }
        };
        put(B1, N1, K1, t1h, t1l);
        put(B2, N2, K2, t2h, t2l);
        kmax = std::max(kmax, std::max(K1, K2));
        bmax = std::max<int64_t>(bmax, meta[6 * cl + 5]);
        while (cols < std::max(N1, N2)) cols <<= 1;
    }
    int err = HHO_OK;
    ops->d_tc_b = dev_upload(ops, tiles, &err);
    if (err) return err;
    ops->d_tc_meta = dev_upload(ops, meta, &err);
    if (err) return err;
    ops->d_tc_err = dev_upload(ops, std::vector<int32_t>(1, 0), &err);
    ops->tc_kmax = kmax;
    ops->tc_bmax = bmax;
    ops->tc_cols = (uint32_t)cols;
    return err;
}

extern "C" void hho_params_default(hho_params* p) {
    if (!p) return;
    p->eta_f = 0.8;
    p->eta_s = 1.5;
    p->stab_speed = 0;
    p->tau_over_k = 0;
}

extern "C" int hho_tableau_erk(int32_t s, hho_tableau* t) {
    if (!t || s < 2 || s > 4) {
        hho_set_error("hho_tableau_erk: s must be 2, 3 or 4");
        return HHO_EINVAL;
    }
    memset(t, 0, sizeof(*t));
    t->s = s;
    if (s == 2) {            // explicit midpoint (Eq. ERK, left)
        t->a[1][0] = 0.5;
        t->b[0] = 0.0; t->b[1] = 1.0;
        t->c[1] = 0.5;
    } else if (s == 3) {     // Eq. ERK, middle
        t->a[1][0] = 0.5;
        t->a[2][0] = -1.0; t->a[2][1] = 2.0;
        t->b[0] = 1.0 / 6.0; t->b[1] = 2.0 / 3.0; t->b[2] = 1.0 / 6.0;
        t->c[1] = 0.5; t->c[2] = 1.0;
    } else {                 // classical ERK(4), Eq. ERK, right
        t->a[1][0] = 0.5; t->a[2][1] = 0.5; t->a[3][2] = 1.0;
        t->b[0] = 1.0 / 6.0; t->b[1] = 1.0 / 3.0; t->b[2] = 1.0 / 3.0; t->b[3] = 1.0 / 6.0;
        t->c[1] = 0.5; t->c[2] = 0.5; t->c[3] = 1.0;
    }
    return HHO_OK;
}

extern "C" int hho_operators_build(const hho_mesh* m, int32_t k, const double* rho, const double* lam,
                                   const double* mu, const double* kappa, const hho_params* params,
                                   hho_ops** out) {
    return hho_operators_build_tau(m, k, rho, lam, mu, kappa, params, nullptr, out);
}

extern "C" int hho_ops_tau(const hho_ops* ops, double* h_tau) {
    if (!ops || !h_tau) {
        hho_set_error("hho_ops_tau: null pointer");
        return HHO_EINVAL;
    }
    memcpy(h_tau, ops->tau.data(), sizeof(double) * ops->nc);
    return HHO_OK;
}

extern "C" int hho_operators_build_tau(const hho_mesh* m, int32_t k, const double* rho, const double* lam,
                                       const double* mu, const double* kappa, const hho_params* params,
                                       const double* h_tau, hho_ops** out) {
    if (!m || !rho || !lam || !mu || !kappa || !out) {
        hho_set_error("hho_operators_build: null pointer");
        return HHO_EINVAL;
    }
    *out = nullptr;
    if (k < 1 || k > 3) {
        hho_set_error("hho_operators_build: k = %d, must be 1, 2 or 3", (int)k);
        return HHO_EDEGREE;
    }
    hho_params P;
    hho_params_default(&P);
    if (params) P = *params;
    if (!(P.eta_f > 0.0) || !(P.eta_s > 0.0) || (P.stab_speed != 0 && P.stab_speed != 1)) {
        hho_set_error("hho_operators_build: bad stabilisation parameters");
        return HHO_EINVAL;
    }
    const int64_t nc = m->nc;
    std::vector<double> tau(nc), cmax(nc);
    for (int64_t c = 0; c < nc; ++c) {
        if (m->domain[c] == 0) {
            if (!(rho[c] > 0.0) || !(kappa[c] > 0.0)) {
                hho_set_error("hho_operators_build: fluid cell %lld has rho = %g, kappa = %g", (long long)c, rho[c], kappa[c]);
                return HHO_EMATERIAL;
            }
            double cp = std::sqrt(kappa[c] / rho[c]);
            tau[c] = P.eta_f / (rho[c] * cp);
            cmax[c] = cp;
        } else {
            if (!(rho[c] > 0.0) || !(mu[c] > 0.0) || !(lam[c] + mu[c] > 0.0)) {
                hho_set_error("hho_operators_build: solid cell %lld has rho = %g, lambda = %g, mu = %g",
                              (long long)c, rho[c], lam[c], mu[c]);
                return HHO_EMATERIAL;
            }
            double cp = std::sqrt((lam[c] + 2.0 * mu[c]) / rho[c]);
            double cs = std::sqrt(mu[c] / rho[c]);
            tau[c] = P.eta_s * rho[c] * (P.stab_speed == 0 ? cp : cs);
            cmax[c] = cp;
        }
        if (P.tau_over_k) tau[c] /= k;
        if (h_tau) {
            if (!(h_tau[c] > 0.0)) {
                hho_set_error("hho_operators_build_tau: tau[%lld] = %g must be positive", (long long)c, h_tau[c]);
                return HHO_EINVAL;
            }
            tau[c] = h_tau[c];
        }
    }

    hho_ops* ops = new (std::nothrow) hho_ops();
    if (!ops) {
        hho_set_error("hho_operators_build: out of host memory");
        return HHO_ENOMEM;
    }
    const int n = (k + 1) * (k + 2) / 2, f = k + 1;
    ops->k = k;
    ops->n = n;
    ops->f = f;
    ops->nc = nc;
    ops->n_classes = m->n_classes;
    std::vector<int> EA, EB;
    exponents(k, EA, EB);

    // ---- class reference matrices ------------------------------------------------
    const int NCL = m->n_classes;
    std::vector<int32_t> cls_nf(NCL), cls_dom(NCL);
    std::vector<int32_t> cls_doff(NCL);
    std::vector<double> cls_dbl;
    ops->class_M0inv.resize(NCL);
    ops->class_normals.resize(NCL);
    std::vector<double> gx, gw, fx, fw;
    gauss_legendre(k + 3, gx, gw);
    gauss_legendre(k + 2, fx, fw);
    std::vector<double> phi(n), Pl(f);
    for (int cl = 0; cl < NCL; ++cl) {
        int64_t c = m->class_first[cl];
        int nv = (int)(m->class_ref_off[cl + 1] - m->class_ref_off[cl]) / 2;
        std::vector<double> X(nv), Y(nv);
        for (int i = 0; i < nv; ++i) {   // the class reference geometry (relative to centroid, over diameter)
            X[i] = m->class_ref[m->class_ref_off[cl] + 2 * i];
            Y[i] = m->class_ref[m->class_ref_off[cl] + 2 * i + 1];
        }
        cls_nf[cl] = nv;
        cls_dom[cl] = m->domain[c];
        // M0 by fan triangles from the origin (the centroid) with a collapsed rule.
        std::vector<double> M0(n * n, 0.0);
        for (int t = 0; t < nv; ++t) {
            int t1 = (t + 1) % nv;
            double ax = X[t], ay = Y[t], bx = X[t1] - X[t], by = Y[t1] - Y[t];
            double det = ax * by - ay * bx;
            for (size_t iu = 0; iu < gx.size(); ++iu)
                for (size_t iv = 0; iv < gx.size(); ++iv) {
                    double u = 0.5 * (gx[iu] + 1.0), v = 0.5 * (gx[iv] + 1.0);
                    double wt = 0.25 * gw[iu] * gw[iv] * u * det;
                    basis_values(EA, EB, u * ax + u * v * bx, u * ay + u * v * by, phi.data());
                    for (int i = 0; i < n; ++i)
                        for (int j = 0; j < n; ++j) M0[i * n + j] += wt * phi[i] * phi[j];
                }
        }
        std::vector<double> M0inv;
        if (!spd_inverse(n, M0, M0inv)) {
            hho_set_error("hho_operators_build: class %d mass matrix is not positive definite", cl);
            hho_ops_destroy(ops);
            return HHO_EMESH;
        }
        ops->class_M0inv[cl] = M0inv;
        // Class block: M0 (n x n, padded to a multiple of 4 entries), then per
        // face [nx, ny, |F|/h_T, 0 | Tr rows of nP | Lift rows of fP] with nP,
        // fP the row lengths n, f rounded up to multiples of 4, so that every
        // row starts on a 16-byte boundary (vector loads in the kernels).  The
        // stage kernels read only the normal; the adjoint reads the relative
        // face length for face integrals (|F| = h_T times it).
        cls_doff[cl] = (int32_t)cls_dbl.size();
        for (double v : M0) cls_dbl.push_back(v);
        while (cls_dbl.size() % 4) cls_dbl.push_back(0.0);
        for (int j = 0; j < nv; ++j) {
            int j1 = (j + 1) % nv;
            double ex = X[j1] - X[j], ey = Y[j1] - Y[j];
            double L = std::sqrt(ex * ex + ey * ey);
            double nx = ey / L, ny = -ex / L;
            if (std::fabs(nx) < 1e-15) nx = 0.0;
            if (std::fabs(ny) < 1e-15) ny = 0.0;
            ops->class_normals[cl].push_back(nx);
            ops->class_normals[cl].push_back(ny);
            std::vector<double> Tr(f * n, 0.0), Bm(n * f, 0.0), row(f);
            for (int i = 0; i < n; ++i) {
                face_trace_row(EA[i], EB[i], 0.5 * (X[j] + X[j1]), 0.5 * ex, 0.5 * (Y[j] + Y[j1]), 0.5 * ey, f,
                               row.data());
                for (int l = 0; l < f; ++l) Tr[l * n + i] = row[l];
            }
            for (size_t g = 0; g < fx.size(); ++g) {   // k + 2 points: exact for degree 2k
                double xi = fx[g];
                double s = 0.5 * (xi + 1.0);
                basis_values(EA, EB, X[j] + s * ex, Y[j] + s * ey, phi.data());
                face_basis_values(f, xi, Pl.data());
                for (int l = 0; l < f; ++l)
                    for (int i = 0; i < n; ++i) Bm[i * f + l] += 0.5 * L * fw[g] * phi[i] * Pl[l];
            }
            std::vector<double> Lift(n * f, 0.0);
            for (int i = 0; i < n; ++i)
                for (int l = 0; l < f; ++l) {
                    double s = 0.0;
                    for (int p = 0; p < n; ++p) s += M0inv[i * n + p] * Bm[p * f + l];
                    Lift[i * f + l] = s;
                }
            // Entries that vanish by symmetry come out of the quadrature as
            // rounding noise (below 1e-15 of the largest entry); store them as
            // exact zeros so the kernels can skip them.
            double tmax = 0.0, lmax = 0.0;
            for (double v : Tr) tmax = std::max(tmax, std::fabs(v));
            for (double v : Lift) lmax = std::max(lmax, std::fabs(v));
            const int nP = (n + 3) / 4 * 4, fP = (f + 3) / 4 * 4;
            cls_dbl.push_back(nx);
            cls_dbl.push_back(ny);
            cls_dbl.push_back(L);
            cls_dbl.push_back(0.0);
            for (int l = 0; l < f; ++l)
                for (int i = 0; i < nP; ++i) {
                    const double v = i < n ? Tr[l * n + i] : 0.0;
                    cls_dbl.push_back(std::fabs(v) < 1e-13 * tmax ? 0.0 : v);
                }
            for (int i = 0; i < n; ++i)
                for (int l = 0; l < fP; ++l) {
                    const double v = l < f ? Lift[i * f + l] : 0.0;
                    cls_dbl.push_back(std::fabs(v) < 1e-13 * lmax ? 0.0 : v);
                }
        }
    }

    // ---- class kinds: axis-aligned rectangles (faces bottom, right, top, left) ----
    // The rectangle kernels skip, at compile time, the entries that vanish by
    // parity: on a horizontal face a cell monomial X^a Y^b traces to a
    // multiple of xi^a, so Tr[l][i] = 0 unless l = a;
    // Lift[i][l] = 0 unless a_i = l (mod 2) (M0 couples only equal parities);
    // vertical faces use b.  The pattern is checked against the computed
    // matrices before a class is marked.
    std::vector<int32_t> cls_kind(NCL, KIND_GENERIC);
    for (int cl = 0; cl < NCL; ++cl) {
        if (cls_nf[cl] != 4) continue;
        const double want[4][2] = {{0.0, -1.0}, {1.0, 0.0}, {0.0, 1.0}, {-1.0, 0.0}};
        const int nP = (n + 3) / 4 * 4, fP = (f + 3) / 4 * 4;
        const double* cd = &cls_dbl[cls_doff[cl] + (n * n + 3) / 4 * 4];
        const int FS = 4 + f * nP + n * fP;
        bool ok = true;
        for (int j = 0; j < 4 && ok; ++j) {
            const double* fm = cd + j * FS;
            if (fm[0] != want[j][0] || fm[1] != want[j][1]) ok = false;
            for (int l = 0; l < f && ok; ++l)
                for (int i = 0; i < n && ok; ++i) {
                    int e = (j % 2 == 0) ? EA[i] : EB[i];
                    bool tr_nz = e == l;
                    bool li_nz = ((e + l) % 2) == 0;
                    if (!tr_nz && fm[4 + l * nP + i] != 0.0) ok = false;
                    if (!li_nz && fm[4 + f * nP + i * fP + l] != 0.0) ok = false;
                }
        }
        // the kernels lift both faces of an orientation pair with the first
        // face's matrix: the mirror through the centroid maps face j to
        // face j + 2 with Lift_{j+2} = P Lift_j F, P = (-1)^(exponent along
        // the normal) on the rows, F = (-1)^l on the columns
        double lmax = 0.0;
        for (int j = 0; j < 4 && ok; ++j)
            for (int i = 0; i < n; ++i)
                for (int l = 0; l < f; ++l) lmax = std::max(lmax, std::fabs(cd[j * FS + 4 + f * nP + i * fP + l]));
        for (int j = 0; j < 2 && ok; ++j)
            for (int i = 0; i < n && ok; ++i)
                for (int l = 0; l < f && ok; ++l) {
                    const int en = (j == 0) ? EB[i] : EA[i];
                    const double sgn = (((en + l) & 1) ? -1.0 : 1.0);
                    const double a = cd[j * FS + 4 + f * nP + i * fP + l];
                    const double b = cd[(j + 2) * FS + 4 + f * nP + i * fP + l];
                    if (std::fabs(b - sgn * a) > 1e-12 * lmax) ok = false;
                }
        if (!ok) continue;
        cls_kind[cl] = KIND_RECT;
        // A square (X, Y in [-rho0, rho0]) traces X^a Y^b on face j to
        // s_t^l (s_n rho0)^(e_n) psi_l, l = e_t, with e_t / e_n the exponent
        // along / across the face, s_n the sign of the face's normal
        // coordinate and s_t of its direction: (s_n, s_t) = (-1, 1), (1, 1),
        // (1, -1), (-1, -1) for faces 0..3.  The square kernels use these
        // values instead of the stored rows.
        const int sn[4] = {-1, 1, 1, -1}, st[4] = {1, 1, -1, -1};
        bool sq = true;
        for (int j = 0; j < 4 && sq; ++j)
            for (int l = 0; l < f && sq; ++l)
                for (int i = 0; i < n && sq; ++i) {
                    const int et = (j % 2 == 0) ? EA[i] : EB[i], en = (j % 2 == 0) ? EB[i] : EA[i];
                    const double want = et != l ? 0.0 : ((l & 1) && st[j] < 0 ? -1.0 : 1.0) * ipow(sn[j] * FACE_RHO, en);
                    if (std::fabs(cd[j * FS + 4 + l * nP + i] - want) > 1e-14) sq = false;
                    // the square kernels skip Lift[i][l] for e_t - l = 2 (zero for
                    // squares at k <= 3; stored as an exact zero by the noise cut)
                    if (et - l == 2 && cd[j * FS + 4 + f * nP + i * fP + l] != 0.0) sq = false;
                }
        if (sq) cls_kind[cl] = KIND_SQUARE;
    }

    // ---- device layout: cells sorted by (domain, class), classes padded to 32 ----
    std::vector<std::vector<int64_t>> members(NCL);
    for (int64_t c = 0; c < nc; ++c) members[m->cell_class[c]].push_back(c);
    std::vector<int32_t> cls_start(NCL), cls_count(NCL), cls_npad(NCL), cls_slot(NCL);
    int64_t Nd[2] = {0, 0}, Sd[2] = {0, 0};
    for (int d = 0; d < 2; ++d)
        for (int cl = 0; cl < NCL; ++cl) {
            if (cls_dom[cl] != d) continue;
            int64_t cnt = (int64_t)members[cl].size();
            int64_t npad = (cnt + 31) / 32 * 32;
            cls_start[cl] = (int32_t)Nd[d];
            cls_count[cl] = (int32_t)cnt;
            cls_npad[cl] = (int32_t)npad;
            cls_slot[cl] = (int32_t)Sd[d];
            Nd[d] += npad;
            Sd[d] += npad * cls_nf[cl];
        }
    if (Nd[0] * 5 * n > INT32_MAX || Nd[1] * 5 * n > INT32_MAX || Sd[0] * 4 * f > INT32_MAX ||
        Sd[1] * 4 * f > INT32_MAX) {
        hho_set_error("hho_operators_build: mesh too large for 32-bit device offsets");
        hho_ops_destroy(ops);
        return HHO_EINVAL;
    }
    const int32_t Nf = (int32_t)Nd[0], Ns = (int32_t)Nd[1], SF = (int32_t)Sd[0], SS = (int32_t)Sd[1];
    ops->cell_dom.resize(nc);
    ops->cell_pos.resize(nc);
    ops->cell_class_of.assign(m->cell_class.begin(), m->cell_class.end());
    std::vector<int32_t> dev2orig(Nf + Ns, -1);
    for (int cl = 0; cl < NCL; ++cl)
        for (size_t r = 0; r < members[cl].size(); ++r) {
            int64_t c = members[cl][r];
            int32_t q = cls_start[cl] + (int32_t)r;
            ops->cell_dom[c] = cls_dom[cl];
            ops->cell_pos[c] = q;
            dev2orig[(cls_dom[cl] ? Nf : 0) + q] = (int32_t)c;
        }
    std::vector<int32_t> warp_class((Nf + Ns) / 32, 0);
    for (int cl = 0; cl < NCL; ++cl) {
        int32_t base = (cls_dom[cl] ? Nf : 0) + cls_start[cl];
        for (int32_t w = 0; w < cls_npad[cl] / 32; ++w) warp_class[base / 32 + w] = cl;
    }
    std::vector<int32_t> cls_int(NCL * CI_STRIDE, 0);
    for (int cl = 0; cl < NCL; ++cl) {
        int32_t* r = &cls_int[cl * CI_STRIDE];
        r[CI_DOMAIN] = cls_dom[cl];
        r[CI_NF] = cls_nf[cl];
        r[CI_START] = cls_start[cl];
        r[CI_COUNT] = cls_count[cl];
        r[CI_NPAD] = cls_npad[cl];
        r[CI_SLOT] = cls_slot[cl];
        r[CI_DOFF] = cls_doff[cl];
        r[CI_KIND] = cls_kind[cl];
    }

    // ---- per-cell scalars ----------------------------------------------------------
    std::vector<double> scal_f((size_t)SCF * Nf, 0.0), scal_s((size_t)SCS * Ns, 0.0);
    std::vector<double> mass_f((size_t)2 * Nf, 0.0), mass_s((size_t)4 * Ns, 0.0);
    for (int64_t c = 0; c < nc; ++c) {
        int32_t q = ops->cell_pos[c];
        double h = m->diam[c];
        if (m->domain[c] == 0) {
            scal_f[SF_AM * (size_t)Nf + q] = 1.0 / (rho[c] * h);
            scal_f[SF_AP * (size_t)Nf + q] = kappa[c] / h;
            scal_f[SF_TAU * (size_t)Nf + q] = tau[c];
            mass_f[0 * (size_t)Nf + q] = rho[c] * h * h;
            mass_f[1 * (size_t)Nf + q] = h * h / kappa[c];
        } else {
            scal_s[SS_C1 * (size_t)Ns + q] = (lam[c] + 2.0 * mu[c]) / h;
            scal_s[SS_R * (size_t)Ns + q] = lam[c] / (lam[c] + 2.0 * mu[c]);
            scal_s[SS_C3 * (size_t)Ns + q] = mu[c] / h;
            scal_s[SS_AV * (size_t)Ns + q] = 1.0 / (rho[c] * h);
            scal_s[SS_TAU * (size_t)Ns + q] = tau[c];
            // plane-strain compliance in the (E_xx, E_yy, E_xy) basis times h^2:
            // D = [[1-beta, -beta, 0], [-beta, 1-beta, 0], [0, 0, 2]] / (2 mu)
            double beta = lam[c] / (2.0 * (lam[c] + mu[c]));
            mass_s[0 * (size_t)Ns + q] = h * h * (1.0 - beta) / (2.0 * mu[c]);
            mass_s[1 * (size_t)Ns + q] = -h * h * beta / (2.0 * mu[c]);
            mass_s[2 * (size_t)Ns + q] = h * h / mu[c];
            mass_s[3 * (size_t)Ns + q] = rho[c] * h * h;
        }
    }

    // ---- face-side exchange tables -------------------------------------------------
    auto slot_of = [&](int64_t c, int j) -> int32_t {
        int cl = m->cell_class[c];
        return cls_slot[cl] + j * cls_npad[cl] + (ops->cell_pos[c] - cls_start[cl]);
    };
    std::vector<int32_t> nb_f(SF, NB_BOUNDARY), nb_s(SS, NB_BOUNDARY);
    std::vector<double> beta_f(SF, 0.0), beta_s(SS, 0.0);
    std::vector<int32_t> if_nb;
    std::vector<double> if_coef, if_coef_adj;
    for (int64_t c = 0; c < nc; ++c) {
        int64_t b = m->cell_ptr[c];
        int nv = (int)(m->cell_ptr[c + 1] - b);
        int d = m->domain[c];
        for (int j = 0; j < nv; ++j) {
            int64_t F = m->cell_faces[b + j];
            int32_t own = slot_of(c, j);
            int side = (m->face_cells[2 * F] == c) ? 0 : 1;
            int64_t c2 = m->face_cells[2 * F + 1 - side];
            int32_t* nbt = d ? nb_s.data() : nb_f.data();
            double* bet = d ? beta_s.data() : beta_f.data();
            if (c2 < 0) {
                nbt[own] = NB_BOUNDARY;
                bet[own] = 0.0;
                continue;
            }
            int j2 = m->face_local[2 * F + 1 - side];
            int32_t other = slot_of(c2, j2);
            if (m->domain[c2] == d) {
                nbt[own] = other;
                bet[own] = 1.0 / (tau[c] + tau[c2]);
                continue;
            }
            // Interface face: [tau_f, n^T; -n, tau_s I] [p_F; v_F] = [w_f; w_s],
            // n = n_Gamma, outward normal of the solid cell (coupling block, Sec. 3.3).
            int64_t cf = d == 0 ? c : c2, cs = d == 0 ? c2 : c;
            int js = d == 0 ? j2 : j;
            const std::vector<double>& ns = ops->class_normals[m->cell_class[cs]];
            double nx = ns[2 * js], ny = ns[2 * js + 1];
            double Am[9] = {tau[cf], nx, ny, -nx, tau[cs], 0.0, -ny, 0.0, tau[cs]};
            double Ai[9];
            if (!inverse3(Am, Ai)) {
                hho_set_error("hho_operators_build: singular interface block");
                hho_ops_destroy(ops);
                return HHO_EMATERIAL;
            }
            // the adjoint operator reverses the sign of the coupling block
            double Amt[9] = {tau[cf], -nx, -ny, nx, tau[cs], 0.0, ny, 0.0, tau[cs]};
            double Ait[9];
            inverse3(Amt, Ait);
            if (d == 0)
                for (double v : {Ait[0], Ait[1], Ait[2], 0.0, 0.0, 0.0}) if_coef_adj.push_back(v);
            else
                for (double v : {Ait[4], Ait[5], Ait[7], Ait[8], Ait[3], Ait[6]}) if_coef_adj.push_back(v);
            int32_t r = (int32_t)if_nb.size();
            if_nb.push_back(other);
            if (d == 0)   // fluid side: p_F = a w_f + b_x w_sx + b_y w_sy
                for (double v : {Ai[0], Ai[1], Ai[2], 0.0, 0.0, 0.0}) if_coef.push_back(v);
            else          // solid side: v_F = alpha (2x2) w_s + beta w_f
                for (double v : {Ai[4], Ai[5], Ai[7], Ai[8], Ai[3], Ai[6]}) if_coef.push_back(v);
            nbt[own] = -2 - r;
            bet[own] = 0.0;
        }
    }

    // ---- canonical offsets ----------------------------------------------------------
    ops->canon_off.resize(nc);
    int64_t off = 0;
    for (int64_t c = 0; c < nc; ++c) {
        ops->canon_off[c] = off;
        off += (m->domain[c] == 0 ? 3 : 5) * n;
    }
    ops->n_canonical = off;

    // ---- host copies for sources, receivers, CFL ---------------------------------------
    ops->centroid = m->centroid;
    ops->diam = m->diam;
    ops->rho.assign(rho, rho + nc);
    ops->kappa.assign(kappa, kappa + nc);
    ops->lam.assign(lam, lam + nc);
    ops->mu.assign(mu, mu + nc);
    ops->tau = tau;
    ops->tau_explicit = h_tau != nullptr;
    ops->stab_speed = P.stab_speed;
    ops->poly_xy = m->xy;
    ops->poly_ptr = m->cell_ptr;
    ops->poly_vtx = m->cell_vtx;
    ops->poly_dom = m->domain;
    ops->face_cells = m->face_cells;
    ops->cell_faces = m->cell_faces;
    ops->face_type = m->face_type;
    ops->face_local = m->face_local;
    for (int64_t F = 0; F < (int64_t)m->face_type.size(); ++F)
        if (m->face_type[F] == FT_IFACE) ops->iface_faces.push_back(F);
    build_locator(ops);
    double hmin = 1e300, cm = 0.0;
    for (int64_t c = 0; c < nc; ++c) {
        int64_t b = m->cell_ptr[c];
        int nv = (int)(m->cell_ptr[c + 1] - b);
        for (int j = 0; j < nv; ++j) {
            int64_t va = m->cell_vtx[b + j], vb = m->cell_vtx[b + (j + 1) % nv];
            double ex = m->xy[2 * vb] - m->xy[2 * va], ey = m->xy[2 * vb + 1] - m->xy[2 * va + 1];
            hmin = std::min(hmin, std::sqrt(ex * ex + ey * ey));
        }
        cm = std::max(cm, cmax[c]);
    }
    ops->h_min = hmin;
    ops->c_max = cm;

    // ---- upload ------------------------------------------------------------------------
    int err = HHO_OK;
    DevOps& D = ops->dev;
    D.k = k;
    D.n = n;
    D.f = f;
    D.Nf = Nf;
    D.Ns = Ns;
    D.SF = SF;
    D.SS = SS;
    D.n_warps_f = Nf / 32;
    D.n_warps_s = Ns / 32;
    {
        std::vector<StageClock> clk(1, StageClock{0.0, 0});
        ops->d_clock = dev_upload(ops, clk, &err);
    }
    D.max_nf = 0;
    for (int32_t cl = 0; cl < (int32_t)(cls_int.size() / CI_STRIDE); ++cl)
        D.max_nf = std::max(D.max_nf, cls_int[(size_t)cl * CI_STRIDE + CI_NF]);
    D.warp_class = dev_upload(ops, warp_class, &err);
    D.cls_int = dev_upload(ops, cls_int, &err);
    D.cls_dbl = dev_upload(ops, cls_dbl, &err);
    D.scal_f = dev_upload(ops, scal_f, &err);
    D.scal_s = dev_upload(ops, scal_s, &err);
    D.nb_f = dev_upload(ops, nb_f, &err);
    D.nb_s = dev_upload(ops, nb_s, &err);
    D.beta_f = dev_upload(ops, beta_f, &err);
    D.beta_s = dev_upload(ops, beta_s, &err);
    D.if_nb = dev_upload(ops, if_nb, &err);
    D.if_coef = dev_upload(ops, if_coef, &err);
    auto to_f32 = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
    D.cls_f32 = dev_upload(ops, to_f32(cls_dbl), &err);
    D.scal_f_f32 = dev_upload(ops, to_f32(scal_f), &err);
    D.scal_s_f32 = dev_upload(ops, to_f32(scal_s), &err);
    D.beta_f_f32 = dev_upload(ops, to_f32(beta_f), &err);
    D.beta_s_f32 = dev_upload(ops, to_f32(beta_s), &err);
    D.if_coef_f32 = dev_upload(ops, to_f32(if_coef), &err);
    auto to_x = [](const std::vector<double>& v) {
        std::vector<f2x> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) o[i] = f2x(v[i]);
        return o;
    };
    D.cls_x = dev_upload(ops, to_x(cls_dbl), &err);
    D.scal_f_x = dev_upload(ops, to_x(scal_f), &err);
    D.scal_s_x = dev_upload(ops, to_x(scal_s), &err);
    D.beta_f_x = dev_upload(ops, to_x(beta_f), &err);
    D.beta_s_x = dev_upload(ops, to_x(beta_s), &err);
    D.if_coef_x = dev_upload(ops, to_x(if_coef), &err);
    ops->d_if_coef_adj = dev_upload(ops, if_coef_adj, &err);
    ops->d_if_coef_adj_f32 = dev_upload(ops, to_f32(if_coef_adj), &err);
    {
        std::vector<double> minv;
        for (int cl = 0; cl < NCL; ++cl)
            for (double v : ops->class_M0inv[cl]) minv.push_back(v);
        ops->d_cls_minv = dev_upload(ops, minv, &err);
    }
    ops->d_dev2orig = dev_upload(ops, dev2orig, &err);
    ops->d_canon_off = dev_upload(ops, ops->canon_off, &err);
    ops->d_cell_dom = dev_upload(ops, ops->cell_dom, &err);
    ops->d_cell_pos = dev_upload(ops, ops->cell_pos, &err);
    ops->d_mass_f = dev_upload(ops, mass_f, &err);
    ops->d_mass_s = dev_upload(ops, mass_s, &err);
    if (err != HHO_OK) {
        hho_set_error("hho_operators_build: device allocation or upload failed");
        hho_ops_destroy(ops);
        return err;
    }
    err = tc_tiles(ops, cls_dbl, cls_doff, cls_nf, cls_dom);
    if (err) {
        hho_set_error("hho_operators_build: tensor-core tile upload failed");
        hho_ops_destroy(ops);
        return err;
    }
    ops->h_cls_dbl = cls_dbl;
    ops->h_cls_int = cls_int;
    ops->h_nb_f = nb_f;
    ops->h_nb_s = nb_s;
    ops->h_if_nb = if_nb;
    ops->n_state = (int64_t)3 * n * Nf + (int64_t)5 * n * Ns;
    ops->trace_doubles = (int64_t)2 * f * SF + (int64_t)4 * f * SS;
    *out = ops;
    return HHO_OK;
}

extern "C" void hho_ops_destroy(hho_ops* ops) {
    if (!ops) return;
    for (void* p : ops->allocations) cudaFree(p);
    if (ops->d_src_g) cudaFree(ops->d_src_g);
    if (ops->d_src_g32) cudaFree(ops->d_src_g32);
    if (ops->d_src_gx) cudaFree(ops->d_src_gx);
    if (ops->d_shot_src_gx) cudaFree(ops->d_shot_src_gx);
    if (ops->d_shot_src_dom) cudaFree(ops->d_shot_src_dom);
    if (ops->d_shot_src_q) cudaFree(ops->d_shot_src_q);
    if (ops->d_shot_src_g) cudaFree(ops->d_shot_src_g);
    if (ops->d_shot_src_g32) cudaFree(ops->d_shot_src_g32);
    if (ops->d_rec_int) cudaFree(ops->d_rec_int);
    if (ops->d_inj) cudaFree(ops->d_inj);
    if (ops->d_rec_dbl) cudaFree(ops->d_rec_dbl);
    if (ops->d_host_state) cudaFree(ops->d_host_state);
    if (ops->d_host_canon) cudaFree(ops->d_host_canon);
    if (ops->d_host_work) cudaFree(ops->d_host_work);
    if (ops->d_bj) cudaFree(ops->d_bj);
    if (ops->d_bj_colour) cudaFree(ops->d_bj_colour);
    for (void* e : ops->prof_events) cudaEventDestroy((cudaEvent_t)e);
    for (auto& g : ops->graphs)
        if (g.exec) cudaGraphExecDestroy((cudaGraphExec_t)g.exec);
    if (ops->cap_stream) cudaStreamDestroy((cudaStream_t)ops->cap_stream);
    delete ops;
}

extern "C" int hho_state_layout(const hho_ops* ops, hho_layout* out) {
    if (!ops || !out) {
        hho_set_error("hho_state_layout: null pointer");
        return HHO_EINVAL;
    }
    memset(out, 0, sizeof(*out));
    out->n_state = ops->n_state;
    out->n_canonical = ops->n_canonical;
    out->n_fluid_pad = ops->dev.Nf;
    out->n_solid_pad = ops->dev.Ns;
    out->n = ops->n;
    out->f = ops->f;
    out->n_classes = ops->n_classes;
    return HHO_OK;
}

// Lowest-index cell containing the point (boundary inclusive), or -1.
// The lowest-numbered cell containing (x, y), or -1.  Candidates come from
// the point's bucket (every cell whose slightly enlarged bounding box meets
// the bucket), tested in increasing order: the same answer as testing every
// cell in order.
static int64_t locate(const hho_ops* ops, double x, double y) {
    if (ops->loc_gx <= 0 || !std::isfinite(x) || !std::isfinite(y)) return -1;
    const double fx = std::floor((x - ops->loc_x0) / ops->loc_dx), fy = std::floor((y - ops->loc_y0) / ops->loc_dy);
    if (fx < -1.0 || fy < -1.0 || fx > ops->loc_gx || fy > ops->loc_gy) return -1;
    const int64_t bx = std::min<int64_t>(std::max<int64_t>((int64_t)fx, 0), ops->loc_gx - 1);
    const int64_t by = std::min<int64_t>(std::max<int64_t>((int64_t)fy, 0), ops->loc_gy - 1);
    const int64_t bk = by * ops->loc_gx + bx;
    for (int64_t e = ops->loc_ptr[bk]; e < ops->loc_ptr[bk + 1]; ++e) {
        const int64_t c = ops->loc_ids[e];
        int64_t b = ops->poly_ptr[c];
        int nv = (int)(ops->poly_ptr[c + 1] - b);
        if (point_in_cell(ops->poly_xy, &ops->poly_vtx[b], nv, x, y)) return c;
    }
    return -1;
}

static void cell_basis_at(const hho_ops* ops, int64_t c, double x, double y, double* phi) {
    std::vector<int> EA, EB;
    exponents(ops->k, EA, EB);
    double h = ops->diam[c];
    basis_values(EA, EB, (x - ops->centroid[2 * c]) / h, (y - ops->centroid[2 * c + 1]) / h, phi);
}

extern "C" int hho_sources_set(hho_ops* ops, int32_t n_src, const double* xy, const double* dir,
                               const double* f0, const double* t0, const double* amp) {
    if (!ops || n_src < 0 || n_src > MAX_SOURCES || (n_src > 0 && (!xy || !dir || !f0 || !t0 || !amp))) {
        hho_set_error("hho_sources_set: bad arguments (at most %d sources)", MAX_SOURCES);
        return HHO_EINVAL;
    }
    ops->src_sampled = false;
    const int n = ops->n;
    std::vector<double> g((size_t)n_src * 2 * n, 0.0);
    std::vector<double> phi(n);
    for (int s = 0; s < n_src; ++s) {
        int64_t c = locate(ops, xy[2 * s], xy[2 * s + 1]);
        if (c < 0) {
            hho_set_error("hho_sources_set: source %d at (%g, %g) is outside the mesh", s, xy[2 * s], xy[2 * s + 1]);
            return HHO_EINVAL;
        }
        cell_basis_at(ops, c, xy[2 * s], xy[2 * s + 1], phi.data());
        const std::vector<double>& Mi = ops->class_M0inv[ops->cell_class_of[c]];
        double h = ops->diam[c];
        // M0 = h^2 M0_ref; the load vector w(t) phi(x_s) e enters M^-1 b.
        double scale = ops->poly_dom[c] == 0 ? ops->kappa[c] / (h * h) : 1.0 / (ops->rho[c] * h * h);
        for (int i = 0; i < n; ++i) {
            double s_i = 0.0;
            for (int p = 0; p < n; ++p) s_i += Mi[i * n + p] * phi[p];
            s_i *= scale;
            if (ops->poly_dom[c] == 0) {
                g[((size_t)s * 2 + 0) * n + i] = s_i;
            } else {
                g[((size_t)s * 2 + 0) * n + i] = dir[2 * s] * s_i;
                g[((size_t)s * 2 + 1) * n + i] = dir[2 * s + 1] * s_i;
            }
        }
        ops->src_dom[s] = ops->cell_dom[c];
        ops->src_q[s] = ops->cell_pos[c];
        ops->src_f0[s] = f0[s];
        ops->src_t0[s] = t0[s];
        ops->src_amp[s] = amp[s];
    }
    if (ops->d_src_g) {
        cudaFree(ops->d_src_g);
        ops->d_src_g = nullptr;
    }
    if (ops->d_src_g32) {
        cudaFree(ops->d_src_g32);
        ops->d_src_g32 = nullptr;
    }
    if (ops->d_src_gx) {
        cudaFree(ops->d_src_gx);
        ops->d_src_gx = nullptr;
    }
    ops->n_src = 0;
    if (n_src > 0) {
        std::vector<float> g32(g.begin(), g.end());
        std::vector<f2x> gx(g.size());
        for (size_t i = 0; i < g.size(); ++i) gx[i] = f2x(g[i]);
        if (cudaMalloc((void**)&ops->d_src_g, sizeof(double) * g.size()) != cudaSuccess ||
            cudaMalloc((void**)&ops->d_src_g32, sizeof(float) * g.size()) != cudaSuccess ||
            cudaMalloc((void**)&ops->d_src_gx, sizeof(f2x) * g.size()) != cudaSuccess) {
            hho_set_error("hho_sources_set: device allocation failed");
            return HHO_ENOMEM;
        }
        if (cudaMemcpy(ops->d_src_g, g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ops->d_src_gx, gx.data(), sizeof(f2x) * g.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ops->d_src_g32, g32.data(), sizeof(float) * g.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            hho_set_error("hho_sources_set: upload failed");
            return HHO_ECUDA;
        }
    }
    ops->n_src = n_src;
    return HHO_OK;
}

extern "C" int hho_locate_points(const hho_ops* ops, int64_t n, const double* h_xy, int64_t* h_cells) {
    if (!ops || n < 0 || (n > 0 && (!h_xy || !h_cells))) {
        hho_set_error("hho_locate_points: bad arguments");
        return HHO_EINVAL;
    }
    for (int64_t i = 0; i < n; ++i) h_cells[i] = locate(ops, h_xy[2 * i], h_xy[2 * i + 1]);
    return HHO_OK;
}

extern "C" int hho_sources_set_samples(hho_ops* ops, int32_t n_src, const double* xy, const double* dir,
                                       double t_start, double dt, int64_t nsteps, int32_t s,
                                       const double* samples) {
    if (!ops || n_src < 0 || n_src > MAX_SOURCES || nsteps < 0 || s < 1 || s > 6 || !(dt > 0.0) ||
        !std::isfinite(dt) || !std::isfinite(t_start) || (n_src > 0 && nsteps > 0 && !samples)) {
        hho_set_error("hho_sources_set_samples: bad arguments (at most %d sources, 1 <= s <= 6, dt > 0)",
                      MAX_SOURCES);
        return HHO_EINVAL;
    }
    const std::vector<double> f0(n_src, 1.0), t0(n_src, 0.0), amp(n_src, 0.0);
    const int rc = hho_sources_set(ops, n_src, xy, dir, f0.data(), t0.data(), amp.data());
    if (rc) return rc;
    const size_t cnt = (size_t)n_src * (size_t)nsteps * (size_t)s;
    for (size_t i = 0; i < cnt; ++i)
        if (!std::isfinite(samples[i])) {
            hho_set_error("hho_sources_set_samples: sample %zu is not finite", i);
            return HHO_EINVAL;
        }
    ops->src_samples.assign(samples, samples + cnt);
    ops->samp_t0 = t_start;
    ops->samp_dt = dt;
    ops->samp_n = nsteps;
    ops->samp_s = s;
    ops->src_sampled = n_src > 0;
    return HHO_OK;
}

// Receiver record on the device: ints [kind, q_fluid, q_solid, pad];
// doubles [phi_fluid (n), phi_solid (n), tau_f, tau_s, nf_x, nf_y, ns_x, ns_y, Ainv (9)].
int receiver_dbl_stride(int n) { return 2 * n + 6 + 9; }

extern "C" int hho_receivers_set(hho_ops* ops, int32_t n_rec, const double* xy) {
    if (!ops || n_rec < 0 || (n_rec > 0 && !xy)) {
        hho_set_error("hho_receivers_set: bad arguments");
        return HHO_EINVAL;
    }
    const int n = ops->n, stride = receiver_dbl_stride(n);
    std::vector<int32_t> ri((size_t)n_rec * 4, 0);
    std::vector<double> rd((size_t)n_rec * stride, 0.0);
    for (int r = 0; r < n_rec; ++r) {
        double x = xy[2 * r], y = xy[2 * r + 1];
        // interface face containing the point?
        int64_t found = -1;
        for (size_t e = 0; e < ops->iface_faces.size() && found < 0; ++e) {
            const int64_t F = ops->iface_faces[e];
            int64_t c0 = ops->face_cells[2 * F];
            int j = ops->face_local[2 * F];
            int64_t b = ops->poly_ptr[c0];
            int nv = (int)(ops->poly_ptr[c0 + 1] - b);
            int64_t va = ops->poly_vtx[b + j], vb = ops->poly_vtx[b + (j + 1) % nv];
            double ax = ops->poly_xy[2 * va], ay = ops->poly_xy[2 * va + 1];
            double tx = ops->poly_xy[2 * vb] - ax, ty = ops->poly_xy[2 * vb + 1] - ay;
            double L2 = tx * tx + ty * ty;
            double s = ((x - ax) * tx + (y - ay) * ty) / L2;
            double dist = std::fabs(tx * (y - ay) - ty * (x - ax)) / std::sqrt(L2);
            if (s >= -1e-10 && s <= 1.0 + 1e-10 && dist <= 1e-10 * std::sqrt(L2)) found = F;
        }
        double* d = &rd[(size_t)r * stride];
        if (found >= 0) {
            int64_t c0 = ops->face_cells[2 * found], c1 = ops->face_cells[2 * found + 1];
            int64_t cf = ops->poly_dom[c0] == 0 ? c0 : c1, cs = ops->poly_dom[c0] == 0 ? c1 : c0;
            int jf = ops->poly_dom[c0] == 0 ? ops->face_local[2 * found] : ops->face_local[2 * found + 1];
            int js = ops->poly_dom[c0] == 0 ? ops->face_local[2 * found + 1] : ops->face_local[2 * found];
            ri[r * 4 + 0] = 2;
            ri[r * 4 + 1] = ops->cell_pos[cf];
            ri[r * 4 + 2] = ops->cell_pos[cs];
            cell_basis_at(ops, cf, x, y, d);
            cell_basis_at(ops, cs, x, y, d + n);
            const std::vector<double>& nfv = ops->class_normals[ops->cell_class_of[cf]];
            const std::vector<double>& nsv = ops->class_normals[ops->cell_class_of[cs]];
            d[2 * n + 0] = ops->tau[cf];
            d[2 * n + 1] = ops->tau[cs];
            d[2 * n + 2] = nfv[2 * jf];
            d[2 * n + 3] = nfv[2 * jf + 1];
            d[2 * n + 4] = nsv[2 * js];
            d[2 * n + 5] = nsv[2 * js + 1];
            double nx = nsv[2 * js], ny = nsv[2 * js + 1];
            double Am[9] = {ops->tau[cf], nx, ny, -nx, ops->tau[cs], 0.0, -ny, 0.0, ops->tau[cs]};
            inverse3(Am, d + 2 * n + 6);
            continue;
        }
        int64_t c = locate(ops, x, y);
        if (c < 0) {
            hho_set_error("hho_receivers_set: receiver %d at (%g, %g) is outside the mesh", r, x, y);
            return HHO_EINVAL;
        }
        ri[r * 4 + 0] = ops->poly_dom[c];
        ri[r * 4 + 1] = ops->cell_pos[c];
        ri[r * 4 + 2] = ops->cell_pos[c];
        cell_basis_at(ops, c, x, y, d);
    }
    // cells read by the receivers (an interface receiver reads two), each with
    // its receivers in increasing order
    std::map<std::pair<int32_t, int32_t>, std::vector<int32_t>> reads;
    for (int r = 0; r < n_rec; ++r) {
        const int kind = ri[r * 4 + 0];
        if (kind == 0 || kind == 2) reads[{0, ri[r * 4 + 1]}].push_back(r);
        if (kind == 1 || kind == 2) reads[{1, ri[r * 4 + 2]}].push_back(r);
    }
    std::vector<int32_t> inj;
    {
        const int32_t nt = (int32_t)reads.size();
        inj.assign((size_t)3 * nt + 1, 0);
        int32_t t = 0;
        for (const auto& kv : reads) {
            inj[t + 1] = inj[t] + (int32_t)kv.second.size();
            inj[nt + 1 + 2 * t] = kv.first.first;
            inj[nt + 1 + 2 * t + 1] = kv.first.second;
            inj.insert(inj.end(), kv.second.begin(), kv.second.end());
            ++t;
        }
    }
    if (ops->d_rec_int) { cudaFree(ops->d_rec_int); ops->d_rec_int = nullptr; }
    if (ops->d_rec_dbl) { cudaFree(ops->d_rec_dbl); ops->d_rec_dbl = nullptr; }
    if (ops->d_inj) { cudaFree(ops->d_inj); ops->d_inj = nullptr; }
    ops->n_rec = 0;
    ops->n_inj = 0;
    if (n_rec > 0) {
        if (cudaMalloc((void**)&ops->d_rec_int, sizeof(int32_t) * ri.size()) != cudaSuccess ||
            cudaMalloc((void**)&ops->d_rec_dbl, sizeof(double) * rd.size()) != cudaSuccess ||
            cudaMalloc((void**)&ops->d_inj, sizeof(int32_t) * inj.size()) != cudaSuccess) {
            hho_set_error("hho_receivers_set: device allocation failed");
            return HHO_ENOMEM;
        }
        if (cudaMemcpy(ops->d_rec_int, ri.data(), sizeof(int32_t) * ri.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ops->d_rec_dbl, rd.data(), sizeof(double) * rd.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ops->d_inj, inj.data(), sizeof(int32_t) * inj.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            hho_set_error("hho_receivers_set: upload failed");
            return HHO_ECUDA;
        }
        ops->n_inj = (int32_t)reads.size();
    }
    ops->n_rec = n_rec;
    return HHO_OK;
}

extern "C" int hho_project_field(const hho_ops* ops, int32_t kind, const double* params, int32_t n_params,
                                 double* h_canonical) {
    if (!ops || !h_canonical || !params || kind != HHO_FIELD_RICKER || n_params != 4 || !(params[3] > 0.0) ||
        !std::isfinite(params[0]) || !std::isfinite(params[1]) || !std::isfinite(params[2])) {
        hho_set_error("hho_project_field: bad arguments (kind HHO_FIELD_RICKER, params {x_c, y_c, theta, lambda > 0})");
        return HHO_EINVAL;
    }
    const double xc = params[0], yc = params[1], theta = params[2], lam = params[3];
    const int n = ops->n;
    std::vector<int> EA, EB;
    exponents(ops->k, EA, EB);
    std::vector<double> gx, gw;
    gauss_legendre(16, gx, gw);
    std::fill(h_canonical, h_canonical + ops->n_canonical, 0.0);
    std::vector<double> phi(n), mx(n), my(n), X, Y;
    for (int64_t c = 0; c < ops->nc; ++c) {
        if (ops->poly_dom[c] != 0) continue;   // the pulse lives on the fluid unknown m
        const int64_t b = ops->poly_ptr[c];
        const int nv = (int)(ops->poly_ptr[c + 1] - b);
        const double h = ops->diam[c], cx = ops->centroid[2 * c], cy = ops->centroid[2 * c + 1];
        X.assign(nv, 0.0);
        Y.assign(nv, 0.0);
        for (int i = 0; i < nv; ++i) {
            X[i] = (ops->poly_xy[2 * ops->poly_vtx[b + i]] - cx) / h;
            Y[i] = (ops->poly_xy[2 * ops->poly_vtx[b + i] + 1] - cy) / h;
        }
        std::fill(mx.begin(), mx.end(), 0.0);
        std::fill(my.begin(), my.end(), 0.0);
        // moments in the scaled coordinates X = (x - x_T)/h: M0 = h^2 M0_ref
        // and (f, phi)_T = h^2 (f, phi)_ref, so M0^-1 (f, phi)_T = M0_ref^-1 (f, phi)_ref
        for (int t = 0; t < nv; ++t) {
            const int t1 = (t + 1) % nv;
            const double ax = X[t], ay = Y[t], bx = X[t1] - X[t], by = Y[t1] - Y[t];
            const double det = ax * by - ay * bx;
            for (size_t iu = 0; iu < gx.size(); ++iu)
                for (size_t iv = 0; iv < gx.size(); ++iv) {
                    const double u = 0.5 * (gx[iu] + 1.0), v = 0.5 * (gx[iv] + 1.0);
                    const double wt = 0.25 * gw[iu] * gw[iv] * u * det;
                    const double Xp = u * ax + u * v * bx, Yp = u * ay + u * v * by;
                    const double x = cx + h * Xp, y = cy + h * Yp;
                    const double r2 = (x - xc) * (x - xc) + (y - yc) * (y - yc);
                    const double g = theta * std::exp(-M_PI * M_PI * r2 / (lam * lam));
                    basis_values(EA, EB, Xp, Yp, phi.data());
                    for (int i = 0; i < n; ++i) {
                        mx[i] += wt * g * (x - xc) * phi[i];
                        my[i] += wt * g * (y - yc) * phi[i];
                    }
                }
        }
        const std::vector<double>& Mi = ops->class_M0inv[ops->cell_class_of[c]];
        double* out = h_canonical + ops->canon_off[c];   // fluid block [m_x | m_y | p]
        for (int i = 0; i < n; ++i) {
            double sx = 0.0, sy = 0.0;
            for (int q = 0; q < n; ++q) {
                sx += Mi[i * n + q] * mx[q];
                sy += Mi[i * n + q] * my[q];
            }
            out[i] = sx;
            out[n + i] = sy;
        }
    }
    return HHO_OK;
}

extern "C" int hho_cfl_dt(const hho_ops* ops, double cfl_star, double safety, double* dt_out) {
    if (!ops || !dt_out || !(cfl_star > 0.0) || !(safety > 0.0)) {
        hho_set_error("hho_cfl_dt: bad arguments");
        return HHO_EINVAL;
    }
    *dt_out = safety * cfl_star * ops->h_min / ops->c_max;
    return HHO_OK;
}

extern "C" int hho_batch_sources_set(hho_ops* ops, int32_t n_shots, const double* xy, const double* dir, double f0,
                                     double t0, double amp) {
    if (!ops || n_shots < 0 || (n_shots > 0 && (!xy || !dir))) {
        hho_set_error("hho_batch_sources_set: bad arguments");
        return HHO_EINVAL;
    }
    const int n = ops->n;
    std::vector<int32_t> dom(n_shots), q(n_shots);
    std::vector<double> g((size_t)n_shots * 2 * n, 0.0);
    std::vector<double> phi(n);
    for (int s = 0; s < n_shots; ++s) {
        int64_t c = locate(ops, xy[2 * s], xy[2 * s + 1]);
        if (c < 0) {
            hho_set_error("hho_batch_sources_set: shot %d source at (%g, %g) is outside the mesh", s, xy[2 * s],
                          xy[2 * s + 1]);
            return HHO_EINVAL;
        }
        cell_basis_at(ops, c, xy[2 * s], xy[2 * s + 1], phi.data());
        const std::vector<double>& Mi = ops->class_M0inv[ops->cell_class_of[c]];
        double h = ops->diam[c];
        double scale = ops->poly_dom[c] == 0 ? ops->kappa[c] / (h * h) : 1.0 / (ops->rho[c] * h * h);
        for (int i = 0; i < n; ++i) {
            double v = 0.0;
            for (int p = 0; p < n; ++p) v += Mi[i * n + p] * phi[p];
            v *= scale;
            if (ops->poly_dom[c] == 0) {
                g[((size_t)s * 2 + 0) * n + i] = v;
            } else {
                g[((size_t)s * 2 + 0) * n + i] = dir[2 * s] * v;
                g[((size_t)s * 2 + 1) * n + i] = dir[2 * s + 1] * v;
            }
        }
        dom[s] = ops->cell_dom[c];
        q[s] = ops->cell_pos[c];
    }
    for (void** p : {(void**)&ops->d_shot_src_dom, (void**)&ops->d_shot_src_q, (void**)&ops->d_shot_src_g,
                     (void**)&ops->d_shot_src_g32, (void**)&ops->d_shot_src_gx}) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    ops->n_shot_src = 0;
    if (n_shots == 0) return HHO_OK;
    std::vector<float> g32(g.begin(), g.end());
    std::vector<f2x> gx(g.size());
    for (size_t i = 0; i < g.size(); ++i) gx[i] = f2x(g[i]);
    if (cudaMalloc((void**)&ops->d_shot_src_dom, sizeof(int32_t) * n_shots) != cudaSuccess ||
        cudaMalloc((void**)&ops->d_shot_src_q, sizeof(int32_t) * n_shots) != cudaSuccess ||
        cudaMalloc((void**)&ops->d_shot_src_g, sizeof(double) * g.size()) != cudaSuccess ||
        cudaMalloc((void**)&ops->d_shot_src_g32, sizeof(float) * g.size()) != cudaSuccess ||
        cudaMalloc((void**)&ops->d_shot_src_gx, sizeof(f2x) * g.size()) != cudaSuccess) {
        hho_set_error("hho_batch_sources_set: device allocation failed");
        return HHO_ENOMEM;
    }
    if (cudaMemcpy(ops->d_shot_src_gx, gx.data(), sizeof(f2x) * g.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ops->d_shot_src_dom, dom.data(), sizeof(int32_t) * n_shots, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ops->d_shot_src_q, q.data(), sizeof(int32_t) * n_shots, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ops->d_shot_src_g, g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ops->d_shot_src_g32, g32.data(), sizeof(float) * g.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        hho_set_error("hho_batch_sources_set: upload failed");
        return HHO_ECUDA;
    }
    ops->n_shot_src = n_shots;
    ops->shot_f0 = f0;
    ops->shot_t0 = t0;
    ops->shot_amp = amp;
    return HHO_OK;
}
