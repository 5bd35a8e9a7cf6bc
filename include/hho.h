/*
 * hho.h -- C ABI of the GB300 library for the explicit Runge-Kutta stage
 * operator of the hybrid high-order (HHO) first-order elasto-acoustic scheme
 * on 2D general meshes (Mottier, Ern, Guillot, "Elasto-acoustic wave
 * propagation in geophysical media using hybrid high-order methods on general
 * meshes").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an int status (HHO_OK = 0 on success); on failure
 *   hho_last_error() returns a one-line message (thread-local).
 * - Pointers named h_* are host memory; pointers named d_* are device memory
 *   of the current CUDA device; all sizes are element counts.
 * - Handles (hho_mesh, hho_ops) are opaque and owned by the library.  They are
 *   freed by the matching *_destroy call.  A handle is not thread-safe.
 * - Device state and work buffers are owned by the caller.  Their sizes come
 *   from hho_state_layout() and hho_work_size().  The stage path (hho_erk_step,
 *   hho_apply) allocates nothing.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Device work is stream-ordered; calls return once work is
 *   enqueued, except where a host result is documented.
 *
 * Canonical cell-DOF layout (host or device "canonical" vectors): cells in
 * input order; per cell its coefficients in the local scaled-monomial basis
 * phi_(a,b) = ((x - x_T)/h_T)^a ((y - y_T)/h_T)^b (x_T area centroid, h_T
 * diameter; ordered by total degree, then decreasing a).  A fluid cell holds
 * [m_x, m_y, p] and a solid cell [s_xx, s_yy, s_xy, v_x, v_y], n = (k+1)(k+2)/2
 * coefficients each.  This is the row order of the paper's block system
 * (Sec. 3.3, "algebraic_system").  The dual unknowns m and s use the sign of the
 * weak form (Eq. HHO1/HHO2).
 */
#ifndef HHO_H
#define HHO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define HHO_OK         0
#define HHO_EINVAL     1  /* bad argument, null pointer, size out of range          */
#define HHO_EMESH      2  /* non-manifold edge, clockwise/degenerate cell, bad id  */
#define HHO_EMATERIAL  3  /* rho <= 0, kappa <= 0, mu <= 0 or lambda + mu <= 0     */
#define HHO_EDEGREE    4  /* k not in {1, 2, 3} (k >= 1 is required in the solid)   */
#define HHO_ECFL       5  /* reserved: time step above a stated CFL limit          */
#define HHO_EUNSTABLE  6  /* non-finite or growing energy detected on the host      */
#define HHO_ECUDA      7  /* a CUDA runtime call failed                             */
#define HHO_ENOMEM     8  /* host or device allocation failed                       */
#define HHO_ENOCONV    9  /* an implicit stage solve missed its tolerance           */

typedef struct hho_mesh hho_mesh;
typedef struct hho_ops hho_ops;

/* Copies the last error message of the calling thread into buf (always
 * NUL-terminated when len > 0).  Returns the message length. */
int hho_last_error(char* buf, size_t len);

/* ------------------------------------------------------------------------- */
/* Mesh (Sec. 3.1: polygonal cells aligned with the fluid/solid partition;   */
/* hanging nodes are ordinary polygon vertices).                              */
/* ------------------------------------------------------------------------- */

/* Builds a mesh from n_vertices points h_xy[2*v] = (x, y) and n_cells
 * counter-clockwise polygons: cell c has vertices h_cell_vtx[h_cell_ptr[c] ..
 * h_cell_ptr[c+1]-1].  h_cell_domain[c] is 0 (fluid) or 1 (solid).
 * h_vertex_rep (may be NULL) maps each vertex to a representative id used to
 * match faces, which identifies periodic images.  A periodic direction needs
 * at least three cells.
 * Faces, face types, colours and cell classes follow the canonical rules:
 *  1 faces numbered by first encounter (cells in order, local edge j joins
 *    vertex j to j+1), keyed by the unordered pair of representative ids;
 *  2 a face's cell 0 is the first cell meeting it, cell 1 the other or -1;
 *  3 tangent from the smaller to the larger representative id (cell 0's
 *    coordinates), normal (t_y, -t_x);
 *  4 colours: greedy in face order, the smallest colour unused by an earlier
 *    face sharing a cell;
 *  5 classes: key (domain, number of vertices, vertex coordinates relative to
 *    the centroid divided by the diameter, scaled by 2^40 and rounded half to
 *    even), numbered by first appearance; centroid = p_0 + cx / (3 A2) from
 *    coordinates relative to vertex 0, no fused multiply-add.
 * Errors: HHO_EINVAL (null/negative sizes, vertex id out of range, domain not
 * 0/1), HHO_EMESH (fewer than 3 vertices, non-positive area, an edge shared
 * by more than two cells).  The input arrays are copied; *out is owned by
 * the caller and freed with hho_mesh_destroy. */
int hho_mesh_create(const double* h_xy, int64_t n_vertices,
                    const int64_t* h_cell_ptr, const int64_t* h_cell_vtx, int64_t n_cells,
                    const uint8_t* h_cell_domain, const int64_t* h_vertex_rep,
                    hho_mesh** out);

typedef struct {
    int64_t n_vertices, n_cells, n_faces;
    int64_t n_fluid_cells, n_solid_cells;
    int64_t n_faces_by_type[5];     /* 0 fluid, 1 solid, 2 interface, 3 fluid bnd, 4 solid bnd */
    int32_t n_classes, n_colours, max_faces_per_cell, reserved;
} hho_mesh_info;

int hho_mesh_query(const hho_mesh* mesh, hho_mesh_info* out);

/* Writes the canonical integer tables (each pointer may be NULL to skip):
 * h_face_cells[2*n_faces], h_cell_faces_ptr[n_cells+1],
 * h_cell_faces[sum of cell sizes] (local order), h_face_type[n_faces],
 * h_face_colour[n_faces], h_cell_class[n_cells]. */
int hho_mesh_tables(const hho_mesh* mesh, int64_t* h_face_cells, int64_t* h_cell_faces_ptr,
                    int64_t* h_cell_faces, int32_t* h_face_type, int32_t* h_face_colour,
                    int32_t* h_cell_class);

void hho_mesh_destroy(hho_mesh* mesh);

/* The sub-mesh of the listed cells of `parent` (h_cells: n_cells distinct
 * parent cell ids; the sub-mesh numbers them 0..n_cells-1 in that order), for
 * a subdomain of a partition: the owned cells plus one layer of ghost cells.
 * Faces whose other cell is not listed become boundary faces.  Each class
 * keeps the reference geometry of the parent's class (the parent's first
 * cell of that class), so operators built on the sub-mesh use the parent's
 * class matrices bit for bit and a cell's stage arithmetic is the same in
 * both.  Periodic vertex identifications are kept.  Host only. */
int hho_mesh_submesh(const hho_mesh* parent, int64_t n_cells, const int64_t* h_cells, hho_mesh** out);

/* ------------------------------------------------------------------------- */
/* Operators (Sec. 3.3: Eq. mass, Eq. rec, Eq. stab, coupling, Eq. rhs).      */
/* ------------------------------------------------------------------------- */

typedef struct {
    double  eta_f;        /* weight of the fluid stabilisation, default 0.8 (Sec. 5.1)  */
    double  eta_s;        /* weight of the solid stabilisation, default 1.5 (Sec. 5.1)  */
    int32_t stab_speed;   /* c^s in tau^s = eta_s rho c^s: 0 = c_P (default), 1 = c_S   */
    int32_t tau_over_k;   /* 1: divide both tau by k (Sec. 3.3, optional scaling)       */
} hho_params;

void hho_params_default(hho_params* p);

/* Builds the stage operator on the current CUDA device for polynomial degree
 * k in {1,2,3} (equal order, least-squares stabilisation, alpha = 0):
 * tau^f = eta_f / (rho c_P^f), tau^s = eta_s rho c^s (Sec. 3.3).
 * Per-cell materials (host arrays of n_cells): h_rho; h_lambda, h_mu (used in
 * solid cells, plane strain); h_kappa (used in fluid cells, kappa = rho c^2).
 * Class matrices are computed in FP64 on the host by quadrature and uploaded
 * with synchronous copies.  The mesh may be destroyed afterwards.
 * Errors: HHO_EDEGREE, HHO_EMATERIAL, HHO_EINVAL, HHO_ENOMEM, HHO_ECUDA. */
int hho_operators_build(const hho_mesh* mesh, int32_t k,
                        const double* h_rho, const double* h_lambda, const double* h_mu,
                        const double* h_kappa, const hho_params* params, hho_ops** out);

/* As hho_operators_build, with the stabilisation weights given per cell in
 * h_tau (n_cells values, > 0) instead of derived from the materials.  With
 * h_tau = NULL it is hho_operators_build.  Used to evaluate gradients and
 * finite differences with the stabilisation frozen (see hho_adjoint_vjp). */
int hho_operators_build_tau(const hho_mesh* mesh, int32_t k, const double* h_rho, const double* h_lambda,
                            const double* h_mu, const double* h_kappa, const hho_params* params,
                            const double* h_tau, hho_ops** out);

/* Writes the per-cell stabilisation weights tau used by ops (n_cells values,
 * input cell order) into h_tau. */
int hho_ops_tau(const hho_ops* ops, double* h_tau);

void hho_ops_destroy(hho_ops* ops);

typedef struct {
    int64_t n_state;       /* doubles in a device-layout state vector                   */
    int64_t n_canonical;   /* doubles in a canonical vector (sum of 3n / 5n per cell)    */
    int64_t n_fluid_pad;   /* padded fluid cell slots (multiple of 32)                   */
    int64_t n_solid_pad;   /* padded solid cell slots (multiple of 32)                   */
    int32_t n;             /* dim P^k(T) = (k+1)(k+2)/2                                   */
    int32_t f;             /* dim P^k(F) = k+1                                            */
    int32_t n_classes;
    int32_t reserved;
} hho_layout;

int hho_state_layout(const hho_ops* ops, hho_layout* out);

/* Device-layout state: fluid block [3n][n_fluid_pad] then solid block
 * [5n][n_solid_pad], i.e. one array per (field, coefficient), cells sorted by
 * (domain, class) with each class padded to a multiple of 32.  Padding slots
 * are zero.  pack: canonical -> device layout; unpack: the reverse.  Both
 * pointers are device memory of the stated sizes; stream-ordered. */
int hho_state_pack(const hho_ops* ops, const double* d_canonical, double* d_state, void* stream);
int hho_state_unpack(const hho_ops* ops, const double* d_state, double* d_canonical, void* stream);

/* Initial fields, L2-projected onto the cell spaces P^k(T) (host, FP64).
 *   HHO_FIELD_RICKER: the Ricker pulse of Sec. 5.2, Eq. ricker_ic, on the
 *     fluid dual variable m:
 *       m_0(x, y) = theta exp(-pi^2 r^2 / lambda^2) (x - x_c, y - y_c),
 *       r^2 = (x - x_c)^2 + (y - y_c)^2,
 *     params = {x_c, y_c, theta, lambda} (n_params = 4); every other field
 *     (p, and all solid fields) is zero.
 * Writes the whole canonical vector h_canonical (n_canonical doubles, host):
 * per cell M0^-1 of the moments (f, phi_i)_T computed with a collapsed
 * Gauss-Legendre rule of 16 x 16 points on each triangle of the cell's fan
 * from its centroid.  HHO_EINVAL for an unknown kind or bad params.  No
 * device work. */
#define HHO_FIELD_RICKER 0
int hho_project_field(const hho_ops* ops, int32_t kind, const double* params, int32_t n_params, double* h_canonical);

/* ------------------------------------------------------------------------- */
/* Time stepping (Sec. 4.2: Eq. ERK_compact, face elimination Eq. ex_solve,   */
/* tableaux Eq. ERK).                                                         */
/* ------------------------------------------------------------------------- */

/* An explicit tableau with s <= 6 stages: a[i][j] (strictly lower
 * triangular), b[j], c[i]; rows and columns beyond s are ignored. */
typedef struct {
    int32_t s;
    int32_t reserved;
    double a[6][6];
    double b[6];
    double c[6];
} hho_tableau;

/* Fills *out with ERK(s) of Eq. ERK for s = 2 (explicit midpoint), 3 or 4
 * (classical).  HHO_EINVAL for other s. */
int hho_tableau_erk(int32_t s, hho_tableau* out);

/* Size in doubles of the caller-owned work buffer that hho_erk_step needs
 * for this tableau (stage vector, partial sums, two trace buffers, energy
 * scratch, and room for a double-float copy of the state). */
int hho_work_size(const hho_ops* ops, const hho_tableau* tab, int64_t* n_doubles);

/* Arithmetic of hho_erk_step, hho_erk_step_record, hho_erk_run_host and
 * hho_apply on this operator: HHO_F64 (default, FP64 instructions) or
 * HHO_F32X2 (double-float pairs on the FP32 pipes, about 48 significant bits;
 * see HHO_F32X2 below).  With HHO_F32X2 the FP64 device state is split into a
 * pair copy inside d_work at the start of each call and rounded back at the
 * end; the stage operator itself is unchanged (Eq. ex_solve).  HHO_EINVAL
 * for other values.  No counterpart in the paper: GB300 issues FP64 at a
 * small fraction of its FP32 rate. */
int hho_set_arithmetic(hho_ops* ops, int32_t arith);

/* How the ERK loops of hho_erk_step, hho_erk_step_record, hho_erk_run_host
 * and hho_batch_erk_step issue their kernels:
 *   HHO_LAUNCH_STREAM: each stage, record and trace kernel launched on the
 *     caller's stream, with the stage times computed on the host;
 *   HHO_LAUNCH_GRAPH: one step (its stage kernels, the receiver record and a
 *     clock increment) captured once as a CUDA graph on a stream of ops and
 *     replayed on the caller's stream for every step; the stage times and the
 *     Ricker wavelets come from a clock in device memory, so the replayed
 *     kernels have identical arguments.  The graph is captured again when the
 *     arguments of a step change (buffers, tableau, dt, sources, receivers);
 *   HHO_LAUNCH_AUTO (default): graphs when a stage grid has at most 2048
 *     blocks (about 260,000 cells x shots) and a call has at least 8 steps,
 *     where launch overhead matters, else stream launches.
 * Stage profiling (hho_profile_enable) always uses stream launches.  Device
 * and host evaluate the wavelet's exponential separately, so the two modes
 * agree to rounding (about 1e-16 relative), not bit for bit.  HHO_EINVAL for
 * other values.  No counterpart in the paper. */
#define HHO_LAUNCH_STREAM 0
#define HHO_LAUNCH_GRAPH  1
#define HHO_LAUNCH_AUTO   2
int hho_set_launch_mode(hho_ops* ops, int32_t mode);

/* Point sources with a Ricker wavelet
 * w(t) = amp (1 - 2 pi^2 f0^2 (t - t0)^2) exp(-pi^2 f0^2 (t - t0)^2):
 * in a solid cell a point force along h_dir (load vector w(t) phi_i(x_s) e_dir
 * in the velocity equation); in a fluid cell a pressure source w(t) phi_i(x_s)
 * (Eq. rhs, read as a load vector).  Arrays of n_src entries (h_xy and h_dir
 * of 2*n_src).  Replaces any previous set; n_src = 0 clears.  At most 8.
 * The owning cell is the lowest-index cell containing the point. */
int hho_sources_set(hho_ops* ops, int32_t n_src, const double* h_xy, const double* h_dir,
                    const double* h_f0, const double* h_t0, const double* h_amp);

/* Point sources with sampled time functions: the same load vectors as
 * hho_sources_set, with source s taking the value
 * h_samples[(s nsteps + n) s_stages + j] in stage j of step n, for steps of
 * size dt from t_start (stage time t_start + n dt + c_j dt) of an ERK tableau
 * with s_stages stages; zero outside those nsteps steps.  A step is located by
 * rounding (t - t_start) / dt, so the stepping calls must use the same dt and
 * a start time on that grid.  The samples of stages sharing a time may
 * differ (they are independent inputs, e.g. for the wavelet gradient of
 * hho_adjoint_vjp, whose h_grad_wavelet has this layout for t0 = t_start).
 * Replaces any previous set.  The ERK entry points use stream launches
 * while sampled sources are set; hho_apply and hho_sdirk_step, which have
 * no stage index, return HHO_EINVAL.  At most 8 sources. */
int hho_sources_set_samples(hho_ops* ops, int32_t n_src, const double* h_xy, const double* h_dir, double t_start,
                            double dt, int64_t nsteps, int32_t s_stages, const double* h_samples);

/* The cell (input order) that sources and receivers at the points h_xy
 * (2 n values) belong to: the lowest-index cell containing the point, or -1
 * outside the mesh.  Host only. */
int hho_locate_points(const hho_ops* ops, int64_t n, const double* h_xy, int64_t* h_cells);

/* Ricker wavelet samples at the stage times of the tableau:
 * h_out[n s + j] = w(t_start + n dt + c_j dt) with the wavelet of
 * hho_sources_set, the times rounded as the ERK loops round them.
 * So hho_sources_set_samples with these samples steps exactly like
 * hho_sources_set with (f0, t0, amp). */
int hho_ricker_samples(const hho_tableau* tab, double t_start, double dt, int64_t nsteps, double f0, double t0,
                       double amp, double* h_out);

/* Advances d_state (device layout, in/out) by nsteps steps of size dt from
 * time t0 with the tableau.  Each stage is one fused kernel (face values from
 * neighbour traces, reconstruction, stabilisation, coupling, inverse mass,
 * ERK accumulation, traces for the next stage), plus one trace kernel per
 * call.  d_work: caller-owned device buffer of hho_work_size doubles.
 * No allocation, no host synchronisation.  Errors: HHO_EINVAL, HHO_ECUDA
 * (launch failure). */
int hho_erk_step(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps,
                 double* d_state, double* d_work, void* stream);

/* hho_erk_step followed, after every step, by hho_record into
 * d_seismogram + 5 * n_rec * step (device, nsteps * n_rec * 5 doubles): the
 * sensor traces of Sec. 5.2 sampled at every time node. */
int hho_erk_step_record(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps,
                        double* d_state, double* d_work, double* d_seismogram, void* stream);

/* Same as hho_erk_step, end to end from host memory: the canonical host
 * vector h_canonical (n_canonical doubles) is packed into the device layout,
 * stepped, unpacked back into h_canonical, and the stream is synchronised.
 * Pinned host memory (cudaHostAlloc, or a pinned torch tensor) mapped into
 * the device's address space is read and written by the pack kernels
 * directly; other host memory is staged through a device copy.  Both give
 * the same bits as hho_state_pack, hho_erk_step and hho_state_unpack.  The
 * device buffers it needs are allocated on the first call and kept with
 * ops. */
int hho_erk_run_host(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps,
                     double* h_canonical, void* stream);

/* Semi-discrete rate d_rate = M^-1 (F(t) - (K_T - K_TF K_F^-1 K_FT) U) for the
 * device-layout state d_state: the operator inside every stage of Eq. ex_solve.
 * d_work: at least hho_work_size(ops, ERK2) doubles. */
int hho_apply(hho_ops* ops, double t, const double* d_state, double* d_rate, double* d_work,
              void* stream);

/* ------------------------------------------------------------------------- */
/* Implicit stepping: SDIRK (Sec. 4.1, Eq. SDIRK_compact, Eq. cp_dirk).        */
/* ------------------------------------------------------------------------- */

/* Fills *out with an SDIRK tableau (lower triangular a, constant diagonal
 * a_*): s = 1 the implicit midpoint rule (a_* = 1/2); s = 2 Eq. SDIRK's
 * 2-stage tableau as printed (a_* = 1/4, order 2); s = 3 Eq. SDIRK's
 * SDIRK(3,4) (nu = cos(pi/18)/sqrt 3 + 1/2, xi = 1/(6 (2 nu - 1)^2));
 * s = 23 the order-3 2-stage member a_* = (3 + sqrt 3)/6.  HHO_EINVAL
 * otherwise. */
int hho_tableau_sdirk(int32_t s, hho_tableau* out);

/* Doubles of the caller-owned device work buffer hho_sdirk_step needs for
 * this tableau and GMRES restart length (1 <= restart <= 64). */
int hho_sdirk_work_size(const hho_ops* ops, const hho_tableau* tab, int32_t restart, int64_t* n_doubles);

/* Advances d_state (device layout, FP64, in/out) by nsteps SDIRK steps.
 * Every stage of Eq. cp_dirk keeps K_FT U_T + K_F U_F = 0, so its cell part
 * is (I - a_* dt J) Y_i = U^{n-1} + dt sum_{j<i} a_ij k_j + a_* dt M^-1 F(t_i)
 * with J = -M^-1 (K_T - K_TF K_F^-1 K_FT) and k_j = J Y_j + M^-1 F(t_j); the
 * last stage is U^n = U^{n-1} + dt sum_j b_j k_j.  Each stage system is
 * solved matrix-free by restarted GMRES (restart vectors, at most max_iter
 * operator applications per stage) to ||r|| <= tol ||rhs||; the operator is
 * the stage kernel of hho_erk_step in FP64 (hho_set_arithmetic does not
 * apply).  h_iterations (host, may be NULL) receives the total number of
 * operator applications inside GMRES.  Synchronises the stream once per
 * Krylov vector (the Hessenberg matrix and the Givens rotations live on the
 * host).  HHO_ENOCONV if a stage misses tol within max_iter (d_state then
 * holds the steps completed so far); HHO_EINVAL for a tableau that is not
 * lower triangular with a constant positive diagonal. */
int hho_sdirk_step(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps, double tol,
                   int32_t restart, int32_t max_iter, double* d_state, double* d_work, int64_t* h_iterations,
                   void* stream);

/* Preconditioner of hho_sdirk_step's GMRES (no counterpart in the paper's
 * direct solves): kind 1 (the default) = block Jacobi, right
 * preconditioning by the exact cell blocks (I - a* dt J_TT)^-1, which are the
 * local cell solves of Eq. sc2; kind 0 = none.  The blocks (9n^2 doubles a
 * fluid cell, 25n^2 a solid cell, owned by ops) are built on the first step
 * with a new a* dt from the stage operator applied to unit vectors on one
 * colour of cells at a time, and inverted on the GPU; HHO_EUNSTABLE if a
 * block is singular.  Where the device has no room for the blocks the step
 * runs unpreconditioned (same solution, more iterations).  HHO_EINVAL for
 * another kind. */
int hho_sdirk_set_preconditioner(hho_ops* ops, int32_t kind);

/* ------------------------------------------------------------------------- */
/* Batched shots: S independent states (right-hand sides, e.g. one point     */
/* source each) on the same mesh, advanced by the same stage kernels with    */
/* the shot index as the second grid dimension, in FP64 or FP32.  Each shot  */
/* follows Eq. ERK_compact / Eq. ex_solve exactly as the single-shot path.   */
/* ------------------------------------------------------------------------- */

#define HHO_F64 0   /* state, traces and arithmetic in FP64 */
#define HHO_F32 1   /* state, traces and arithmetic in FP32; operators built in FP64 and rounded */
#define HHO_F32X2 2 /* double-float: every value a pair of FP32 numbers hi + lo (about 48
                       significant bits, 8 bytes), arithmetic by error-free transforms on
                       the FP32 pipes; operators built in FP64 and split into pairs;
                       seismograms in FP64 */
#define HHO_BF16X3 3 /* state, traces and seismograms in FP32 as HHO_F32, with the dense local
                        products (every face's lifted jump, every face's traces) on the
                        tcgen05 tensor cores: operands split into two BF16 numbers each,
                        three products (hi hi + hi lo + lo hi) accumulated in FP32 in tensor
                        memory; blocks of 128 (cell, shot) rows of one class */

/* Element counts (of the precision's type) of a batched state
 * (n_shots x n_state, shot-major) and of the work buffer hho_batch_erk_step
 * needs for this tableau. */
int hho_batch_sizes(const hho_ops* ops, const hho_tableau* tab, int32_t n_shots, int32_t precision,
                    int64_t* state_elems, int64_t* work_elems);

/* Canonical FP64 vectors [n_shots][n_canonical] (device) <-> batched device
 * state of the given precision (rounded to FP32 for HHO_F32). */
int hho_batch_pack(const hho_ops* ops, int32_t n_shots, int32_t precision, const double* d_canonical,
                   void* d_state, void* stream);
int hho_batch_unpack(const hho_ops* ops, int32_t n_shots, int32_t precision, const void* d_state,
                     double* d_canonical, void* stream);

/* One point source per shot: shot s has its source at h_xy[2s..2s+1] with
 * direction h_dir[2s..2s+1] (solid cells; pressure source in fluid cells),
 * all shots sharing the Ricker wavelet (f0, t0, amp) of hho_sources_set.
 * Sources set with hho_sources_set still act on every shot.  n_shots = 0
 * clears. */
int hho_batch_sources_set(hho_ops* ops, int32_t n_shots, const double* h_xy, const double* h_dir, double f0,
                          double t0, double amp);

/* Advances n_shots batched states by nsteps ERK steps (one launch per stage
 * for all shots).  d_seismogram (may be NULL): receiver traces
 * [nsteps][n_shots][n_rec][5] in the state's precision, recorded after
 * every step.  No allocation, no host synchronisation. */
int hho_batch_erk_step(hho_ops* ops, const hho_tableau* tab, int32_t n_shots, int32_t precision, double t0,
                       double dt, int64_t nsteps, void* d_state, void* d_work, void* d_seismogram, void* stream);

/* Reads and clears the tensor-core stage's error flag (HHO_BF16X3): *h_flag
 * = 1 if a block's wait for its MMAs gave up since the last call (its
 * results are then invalid), else 0.  Synchronises the device. */
int hho_tc_error(hho_ops* ops, int32_t* h_flag);

/* ------------------------------------------------------------------------- */
/* One stage at a time, for subdomain drivers (a mesh partition with a halo   */
/* exchange of the published face traces between stages; no counterpart in   */
/* the paper, whose implementation is serial).                                */
/* ------------------------------------------------------------------------- */

/* hho_erk_traces publishes the face traces of d_state into trace buffer 0 of
 * d_work (as hho_erk_step does at the start of a call).  hho_erk_stage runs
 * stage j of step n (step time tn, sources at tn + c_j dt): it reads trace
 * buffer (n s + j) % 2 and writes the traces of its result into buffer
 * (n s + j + 1) % 2; stage s-1 writes the new state into d_state.  The
 * sequence traces, stage(0, 0), ..., stage(nsteps-1, s-1) gives the same bits
 * as hho_erk_step in stream launch mode (HHO_LAUNCH_STREAM).  d_work as for
 * hho_erk_step; FP64 arithmetic only (HHO_EINVAL otherwise).  No receivers
 * are recorded (hho_record).  Stream-ordered, no synchronisation. */
int hho_erk_traces(hho_ops* ops, const hho_tableau* tab, const double* d_state, double* d_work, void* stream);
int hho_erk_stage(hho_ops* ops, const hho_tableau* tab, int64_t n, int32_t j, double tn, double dt, double* d_state,
                  double* d_work, void* stream);

/* Offset, in doubles from d_work, of trace buffer `which` (0 or 1). */
int hho_trace_buffer_offset(const hho_ops* ops, const hho_tableau* tab, int32_t which, int64_t* offset);

/* Offsets within one trace buffer of the traces w that cell h_cells[i]
 * (mesh input order) publishes on its local face h_faces[i] (the face from
 * its vertex i to vertex i+1), which is what the neighbour across that face
 * reads: f values in a fluid cell, 2f (x then y components) in a solid
 * cell, coefficients in the face basis (rho0 xi)^l, rho0 = 1/(2 sqrt 2),
 * xi in [-1, 1] along the face in the publishing cell's counter-clockwise
 * direction.  h_out: [n][2f], unused entries -1.  Host. */
int hho_trace_offsets(const hho_ops* ops, int64_t n, const int64_t* h_cells, const int32_t* h_faces,
                      int64_t* h_out);

/* d_dst[i] = d_src[d_idx[i]] (gather), d_dst[d_idx[i]] = d_src[i] (scatter),
 * i < n, on the device: the halo exchange's packing of trace entries. */
int hho_halo_gather(const double* d_src, const int64_t* d_idx, int64_t n, double* d_dst, void* stream);
int hho_halo_scatter(const double* d_src, const int64_t* d_idx, int64_t n, double* d_dst, void* stream);

/* ------------------------------------------------------------------------- */
/* Tensor cores (tcgen05).                                                    */
/* ------------------------------------------------------------------------- */

/* Self-check of the split-BF16 tensor-core products (no counterpart in the
 * paper): D = A B for one 128-row tile on the tcgen05 tensor cores, each
 * operand split as x = hi + lo (two BF16 numbers), three products
 * (hi hi + hi lo + lo hi) accumulated in FP32 in tensor memory, read back
 * with tcgen05.ld.  Host buffers, row-major: h_A [128][K], h_B [K][N],
 * h_D [128][N]; 16 <= K <= 64 and 16 <= N <= 128, multiples of 16.
 * *h_status = 0, or 1 if the MMA completion wait gave up.  Allocates its
 * own device buffers and synchronises. */
int hho_tc_gemm_check(int32_t K, int32_t N, const float* h_A, const float* h_B, float* h_D, int32_t* h_status);

/* ------------------------------------------------------------------------- */
/* Double-float arithmetic.                                                   */
/* ------------------------------------------------------------------------- */

/* Self-check of the double-float (FP32 pair) arithmetic of the HHO_F32X2
 * kernels (no counterpart in the paper): for each of n items, pairs
 * x = (hi, lo), y, z given as h_in [n][3][2] floats (value hi + lo), the
 * GPU computes x + y, x - y, x * y, x * y + z, x / y and the Horner chain
 * ((x z + y) z + x) z + y with the kernels' operations and writes the
 * resulting pairs, unnormalised (value hi + lo), to h_out [n][6][2].  The
 * caller compares them with exact arithmetic.  Allocates its own device
 * buffers and synchronises; HHO_EINVAL for n < 1 or null buffers. */
int hho_f2x_check(int32_t n, const float* h_in, float* h_out);

/* ------------------------------------------------------------------------- */
/* Discrete adjoint (vector-Jacobian product of the receiver traces).         */
/* ------------------------------------------------------------------------- */

/* Doubles of device work that hho_adjoint_vjp needs: checkpoints every
 * checkpoint_every steps, the stage values of one segment with their face
 * traces, the ERK work buffer and a few state-sized vectors. */
int hho_adjoint_work_size(const hho_ops* ops, const hho_tableau* tab, int64_t nsteps, int64_t checkpoint_every,
                          int64_t* n_doubles);

/* Reverse mode through nsteps ERK steps (Eq. ERK_compact / Eq. ex_solve)
 * from the device state d_state0 at time t0, with the sources and receivers
 * set on ops.  d_cotangent (device, [nsteps][n_rec][5]) is dL/d of the
 * traces that hho_erk_step_record writes after every step.  Outputs:
 *   h_grad_cell[4 c + (0,1,2,3)] = dL/d(rho, kappa, lambda, mu) of cell c
 *     (input order; kappa only in fluid cells, lambda and mu only in solid
 *     cells).  The materials enter through the mass matrix (Eq. mass) and
 *     through the stabilisation weights tau (Sec. 3.3, tau^f = eta_f/(rho c_P),
 *     tau^s = eta_s rho c^s), which scale each cell's stabilisation (Eq. stab)
 *     and with it the face solve: both parts are included for operators from
 *     hho_operators_build.  For operators from hho_operators_build_tau the
 *     weights are the caller's constants and only the mass part remains (the
 *     gradient with tau frozen);
 *   h_grad_wavelet (may be NULL): [nsteps][s][n_src] dL/dw at every stage time
 *     t_{n-1} + c_j dt of every hho_sources_set source;
 *   h_grad_tau (may be NULL): [nc] dL/dtau_c, the partial derivative with the
 *     weights as independent parameters (stage and interface-receiver parts).
 * The adjoint uses A^T = S M A' M^-1 S (S: sign flip of the dual fields, A':
 * the stage operator with the interface coupling reversed) on the forward
 * kernels; the adjoint face values needed by the tau part are those of A'.
 * Segments between checkpoints are recomputed.  Synchronises. */
int hho_adjoint_vjp(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps,
                    int64_t checkpoint_every, const double* d_state0, const double* d_cotangent, double* d_work,
                    int64_t work_doubles, double* h_grad_cell, double* h_grad_wavelet, double* h_grad_tau,
                    void* stream);

/* The same reverse mode in FP32: the FP32
 * stage kernels (the batched FP32 path with one shot) for the forward
 * checkpoints, the segment recompute and the transposed stages; states,
 * traces, adjoint vectors, d_state0 and d_cotangent ([nsteps][n_rec][5]) in
 * FP32; the gradient sums in FP64; outputs as hho_adjoint_vjp.  d_work:
 * hho_adjoint_work_size_f32 floats. */
int hho_adjoint_work_size_f32(const hho_ops* ops, const hho_tableau* tab, int64_t nsteps, int64_t checkpoint_every,
                              int64_t* n_floats);
int hho_adjoint_vjp_f32(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps,
                        int64_t checkpoint_every, const float* d_state0, const float* d_cotangent, float* d_work,
                        int64_t work_floats, double* h_grad_cell, double* h_grad_wavelet, double* h_grad_tau,
                        void* stream);

/* ------------------------------------------------------------------------- */
/* Sensors and energy (Sec. 5).                                               */
/* ------------------------------------------------------------------------- */

/* Sets n_rec receiver points h_xy[2*n_rec].  A point on an interface face
 * records the face unknowns; otherwise the lowest-index containing cell. */
int hho_receivers_set(hho_ops* ops, int32_t n_rec, const double* h_xy);

/* d_out[5*r + j] for each receiver r: fluid [p, m_x, m_y, 0, 0]; solid
 * [v_x, v_y, s_xx, s_yy, s_xy]; interface [p_F, v_Fx, v_Fy, 0, 0] (the face
 * solve of Eq. ex_solve evaluated at the point). */
int hho_record(hho_ops* ops, const double* d_state, double* d_out, void* stream);

/* Discrete energy E = 1/2 U^T M U (Sec. 5.1) of a device-layout state,
 * returned in *h_energy after synchronising the stream.  d_work: at least
 * hho_work_size(ops, ERK2) doubles (block partial sums).  A non-finite
 * result returns HHO_EUNSTABLE. */
int hho_energy(hho_ops* ops, const double* d_state, double* d_work, double* h_energy, void* stream);

/* ------------------------------------------------------------------------- */
/* Cost model and stage timing (measurement support; no counterpart in the   */
/* paper, which reports only CPU seconds, Table 4).                           */
/* ------------------------------------------------------------------------- */

/* Per ERK step with this tableau, summed over all cells (padding excluded):
 * *fp64_ops = FP64 instructions the stage kernels execute per thread-lane
 * (FMA, ADD and MUL each count 1), from the class-matrix sparsity and the face
 * kinds; *bytes_min = 8 bytes x cell DOFs x state-vector passes of the fused
 * design, counting per stage the distinct vectors read (stage input, U^{n-1},
 * partial sums) and written (classical ERK4: 16 passes per step, i.e. 32
 * bytes per cell DOF per stage); *bytes_kernel = bytes the stage kernels move
 * by design (those passes plus face traces, exchange tables and per-cell
 * scalars).  Any output pointer may be NULL. */
int hho_stage_cost(const hho_ops* ops, const hho_tableau* tab, int64_t* fp64_ops, int64_t* bytes_min,
                   int64_t* bytes_kernel);

/* When on != 0, hho_erk_step brackets every stage-kernel launch with CUDA
 * events on the launch stream (up to 4096 launches are kept).  hho_profile_read
 * synchronises those events and returns the summed stage-kernel time in
 * milliseconds and the number of launches since the last enable, then resets. */
int hho_profile_enable(hho_ops* ops, int32_t on);
int hho_profile_read(hho_ops* ops, double* ms_stage_total, int64_t* n_launches);

/* Energy without any allocation, for callers that must not allocate device
 * memory: for example a check that runs between time steps inside a
 * framework whose caching allocator already owns the device memory, or code
 * with a fixed memory budget.  cudaFree also synchronises the whole device,
 * which a per-step check must not do.  The paper has no counterpart to this
 * entry point.
 *
 * Same result as hho_energy (E = 1/2 U^T M U) but written to d_energy (one
 * device double, caller-owned) instead of host memory, stream-ordered and
 * without synchronising.  Its scratch (one partial sum per 256 cells) lives
 * in a fixed array inside the library, so it handles at most
 * HHO_ENERGY_STATIC_MAX_CELLS padded cell slots (n_fluid_pad + n_solid_pad);
 * larger meshes return HHO_EINVAL.  Every GPU that loads the library holds
 * this array (512 KiB) until the process exits.
 * Every call looks up the array's address on the current device (which
 * allocates nothing); the first call on a device may load the library's
 * device code, so make it before any stream capture.
 * Each device holds its own copy of the array.  All calls on one device
 * share it: calls on the same device that overlap on the GPU (different
 * streams) race and must be serialised by the caller; calls on different
 * devices do not interact.  Nothing in the array needs to start at zero. */
#define HHO_ENERGY_STATIC_MAX_CELLS (65536LL * 256LL)
int hho_energy_static(hho_ops* ops, const double* d_state, double* d_energy, void* stream);

/* Empirical CFL bracketing, Algorithm 1 of Sec. 5.1, on the GPU stage.
 * Starting from N = N0 steps over [0, T_f] (dt = T_f / N), each trial copies
 * d_state0 into the scratch d_state and steps without sources, reading the
 * energy after every step.  A trial is unstable at the first step whose
 * energy exceeds (1 + eps) E^0 or (1 + eps) E^{n-1} (read as the signed
 * relative increase), or is not finite.  After a stable trial, N decreases by
 * max(1, floor(delta N)).  *n_stable receives the last stable N (-1 if N0 is
 * unstable) and *n_unstable the first unstable N (-1 if none within
 * max_trials).  d_state: n_state doubles; d_work: hho_work_size(tab) doubles.
 * The energy of d_state0 must be positive and finite (the test divides by
 * it): a zero state returns HHO_EINVAL. 
 * Synchronises the stream after every step. */
int hho_cfl_bracket(hho_ops* ops, const hho_tableau* tab, const double* d_state0, double T_f, int64_t N0,
                    double eps, double delta, int64_t max_trials, double* d_state, double* d_work,
                    int64_t* n_stable, int64_t* n_unstable, void* stream);

/* CFL-limited step (Eq. CFL): dt = safety * cfl_star * h_min / c_max, with
 * h_min the shortest cell edge and c_max the largest wave speed. */
int hho_cfl_dt(const hho_ops* ops, double cfl_star, double safety, double* dt_out);

#ifdef __cplusplus
}
#endif

#endif /* HHO_H */
