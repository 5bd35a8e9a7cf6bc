// Internal declarations shared by the host C++ sources and the CUDA sources.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "hho.h"

void hho_set_error(const char* fmt, ...);

#if defined(__CUDACC__)
#define HHO_HD __host__ __device__
#else
#define HHO_HD
#endif

// A double-float value hi + lo: two FP32 numbers with hi = RN(hi + lo),
// about 48 significant bits (arithmetic in f2x.cuh).  8 bytes: arrays of it
// have the layout of FP64 arrays.
struct alignas(8) f2x {
    float hi, lo;
    f2x() = default;
    HHO_HD constexpr f2x(float h, float l) : hi(h), lo(l) {}
    HHO_HD constexpr explicit f2x(int v) : hi((float)v), lo(0.0f) {}
    // split of an FP64 value: hi = RN(v), lo = RN(v - hi) (v - hi is exact)
    HHO_HD explicit f2x(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    HHO_HD explicit operator double() const { return (double)hi + (double)lo; }
};

// Face types (Sec. 3.1 face sets).
enum { FT_FLUID = 0, FT_SOLID = 1, FT_IFACE = 2, FT_BND_FLUID = 3, FT_BND_SOLID = 4 };

struct hho_mesh {
    int64_t nv = 0, nc = 0, nf = 0;
    std::vector<double> xy;            // 2 nv
    std::vector<int64_t> cell_ptr;     // nc + 1
    std::vector<int64_t> cell_vtx;
    std::vector<uint8_t> domain;       // nc
    std::vector<int64_t> rep;          // nv
    std::vector<int64_t> face_cells;   // 2 nf
    std::vector<int32_t> face_local;   // 2 nf: local edge index in cell 0 / cell 1
    std::vector<int64_t> cell_faces;   // indexed by cell_ptr
    std::vector<int32_t> face_type, face_colour, cell_class;
    std::vector<double> centroid;      // 2 nc
    std::vector<double> diam, area;    // nc
    int32_t n_classes = 0, n_colours = 0, max_nf = 0;
    std::vector<int64_t> class_first;  // first cell of each class
    // per class: vertex coordinates relative to the reference cell's centroid
    // over its diameter, [x_0, y_0, x_1, ...] from class_ref_off[cl]; the
    // class matrices are built from these.  A sub-mesh inherits them from its
    // parent mesh, so its operators use the same class matrices bit for bit.
    std::vector<double> class_ref;
    std::vector<int64_t> class_ref_off;
};

// Per-class integer record on the device (stride CI_STRIDE ints).
enum { CI_DOMAIN = 0, CI_NF, CI_START, CI_COUNT, CI_NPAD, CI_SLOT, CI_DOFF, CI_KIND, CI_STRIDE };

// Class kinds: generic polygon (dense class matrices) or axis-aligned
// rectangle with faces ordered bottom, right, top, left, whose trace and
// lifting matrices have a sparsity pattern fixed by monomial parity; a
// square rectangle's traces are known in closed form (operators.cpp).
enum { KIND_GENERIC = 0, KIND_RECT = 1, KIND_SQUARE = 2 };

// Scale of the face basis psi_l = (FACE_RHO xi)^l, xi in [-1, 1] along a
// face: 1/(2 sqrt 2), the half side over the diameter of a square, so that a
// square cell's scaled coordinates are +-FACE_RHO on its faces.
#define FACE_RHO 0.35355339059327376220

// Device-side description of one stage launch and the static operator data.
struct DevOps {
    int32_t k, n, f;
    int32_t Nf, Ns;          // padded cell slots per domain (multiples of 32)
    int32_t SF, SS;          // face-side slots per domain
    int32_t n_warps_f, n_warps_s;
    int32_t max_nf;              // most faces of any class
    const int32_t* warp_class;   // [n_warps_f + n_warps_s]
    const int32_t* cls_int;      // [n_classes][CI_STRIDE]
    const double* cls_dbl;       // class matrices, see operators.cpp
    const double* scal_f;        // fluid per-cell scalars [SCF][Nf]
    const double* scal_s;        // solid per-cell scalars [SCS][Ns]
    const int32_t* nb_f;         // face-side neighbour slot, fluid [SF]
    const int32_t* nb_s;         // solid [SS]
    const double* beta_f;        // face-side coefficient, fluid [SF]
    const double* beta_s;        // solid [SS]
    const int32_t* if_nb;        // interface records: neighbour slot in the other domain
    const double* if_coef;       // interface records: 6 coefficients each
    // FP32 copies of the same data, for the FP32 batched path
    const float* cls_f32;
    const float* scal_f_f32;
    const float* scal_s_f32;
    const float* beta_f_f32;
    const float* beta_s_f32;
    const float* if_coef_f32;
    // double-float copies, for the double-float path
    const f2x* cls_x;
    const f2x* scal_f_x;
    const f2x* scal_s_x;
    const f2x* beta_f_x;
    const f2x* beta_s_x;
    const f2x* if_coef_x;
};

// Fluid scalars: A_m = 1/(rho h), A_p = kappa/h, tau.  Solid: c1 = (lambda+2mu)/h,
// r = lambda/(lambda+2mu), c3 = mu/h, A_v = 1/(rho h), tau.
enum { SF_AM = 0, SF_AP, SF_TAU, SCF };
enum { SS_C1 = 0, SS_R, SS_C3, SS_AV, SS_TAU, SCS };

// Face-side neighbour encoding: >= 0 same-domain neighbour slot, -1 boundary,
// <= -2 interface record (-2 - r).
constexpr int32_t NB_BOUNDARY = -1;

constexpr int MAX_TARGETS = 4;
constexpr int MAX_SOURCES = 8;

// Simulation clock read by graph-replayed stage kernels: the time of stage
// j of step n of a call is (t0 + n dt) + c_j dt.
struct StageClock {
    double t0;
    int64_t step;
};

template <class T>
struct TargetT {
    const T* src;   // nullptr: zero
    T* dst;
    T coef;
};

// One stage launch.  Shots are blockIdx.y; every state, trace and target
// pointer is the base of shot 0 and advances by state_stride / trace_stride
// elements per shot.
template <class T>
struct StageArgsT {
    DevOps op;
    const T* inp;            // device-layout state read by the stage
    const T* tr_in;          // traces of inp: fluid [2f][SF] then solid [4f][SS]
    T* tr_out;               // traces of the target-0 result (same layout)
    TargetT<T> tgt[MAX_TARGETS];
    int32_t n_tgt;
    int32_t pad0;
    int64_t state_stride, trace_stride;
    // point sources applied to every shot
    int32_t n_src;
    int32_t src_dom[MAX_SOURCES];
    int32_t src_q[MAX_SOURCES];
    T src_w[MAX_SOURCES];            // wavelet value at the stage time
    const T* src_g;                  // [n_src][2][n] lifted load vectors
    // one point source per shot (batched shots); shot_src_q == nullptr: none
    const int32_t* shot_src_dom;
    const int32_t* shot_src_q;
    const T* shot_src_g;             // [shots][2][n]
    T shot_src_w;
    // graph replay: with clock set the stage time comes from the device clock
    // and the wavelets are evaluated in the kernel from these parameters
    const StageClock* clock;
    double dt, c_stage;
    double src_f0[MAX_SOURCES], src_t0[MAX_SOURCES], src_amp[MAX_SOURCES];
    double shot_f0, shot_t0, shot_amp;
};

// MODE_RAW writes the rate before the per-cell material factors (and, in
// solids, before the stress mixing): the derivative of the rate with respect
// to those factors, used by the adjoint gradient.
enum { MODE_TRACES = 0, MODE_STAGE = 1, MODE_APPLY = 2, MODE_RAW = 3 };

// ERK plan (stage.cu): row i of the extended tableau (a_{s+1,:} = b) is the
// partial sum P_i = U^{n-1} + dt sum_j a_ij k_j.
enum { SRC_ZERO = -3, SRC_STATE = -2, SRC_X = -1 };   // >= 0: row buffer index
struct TargetPlan {
    int src, dst;
    double a;
};
struct StagePlan {
    int n_tgt;
    TargetPlan t[MAX_TARGETS];
};
int build_plan(const hho_tableau* tab, std::vector<StagePlan>& plan, int* n_buf);

// Launches one stage-kernel pass (FP64) over n_shots shots; and the receiver
// kernel.  Defined in stage.cu, used by the adjoint driver.
struct hho_ops;
// Stage launch for the adjoint and SDIRK drivers.  Sources (when `sources`)
// are evaluated for step time tn, stage j (time tn + cdt); j < 0 for calls
// that have no stage index (sampled source time functions are then zero).
void launch_stage_f64(const hho_ops* ops, int mode, StageArgsT<double>& a, int n_shots, double tn, int j, double cdt,
                      bool sources, void* stream);
void launch_stage_f32(const hho_ops* ops, int mode, StageArgsT<float>& a, int n_shots, double tn, int j, double cdt,
                      bool sources, void* stream);
void launch_record_f64(const hho_ops* ops, const double* state, double* out, void* stream);
// nsteps ERK steps of one FP32 state (the batched FP32 path with one shot)
int erk_steps_f32(hho_ops* ops, const hho_tableau* tab, double t0, double dt, int64_t nsteps, float* d_state,
                  float* d_work, void* stream);
int check_cuda(const char* what);

struct hho_ops {
    int32_t k = 0, n = 0, f = 0;
    int64_t nc = 0;
    int32_t n_classes = 0;
    DevOps dev{};
    // device allocations owned by ops
    std::vector<void*> allocations;
    // host copies needed later
    std::vector<int32_t> cell_dom, cell_pos;   // per original cell: domain, device position
    std::vector<int64_t> canon_off;            // per original cell: offset in canonical vector
    int64_t n_canonical = 0;
    int32_t* d_dev2orig = nullptr;             // [Nf + Ns]: original cell id or -1 (padding)
    int64_t* d_canon_off = nullptr;            // [nc]
    int32_t* d_cell_dom = nullptr;             // [nc]: 0 fluid, 1 solid
    int32_t* d_cell_pos = nullptr;             // [nc]: device position within the cell's domain
    double c_max = 0.0, h_min = 0.0;
    // host-side per-cell data kept for sources/receivers
    std::vector<double> centroid, diam, rho, tau;
    bool tau_explicit = false;   // tau given by the caller (hho_operators_build_tau): not a function of the materials
    int32_t stab_speed = 0;      // c^s in tau^s: 0 = c_P, 1 = c_S
    std::vector<int32_t> cell_class_of;
    std::vector<std::vector<double>> class_M0inv;     // per class, n x n
    std::vector<std::vector<double>> class_normals;   // per class, 2 per face
    std::vector<double> kappa, lam, mu;
    std::vector<double> poly_xy;                      // copy of vertex coordinates for location
    std::vector<int64_t> poly_ptr, poly_vtx;
    std::vector<uint8_t> poly_dom;
    std::vector<int64_t> face_cells, cell_faces;
    std::vector<int32_t> face_type, face_local;
    std::vector<int64_t> iface_faces;                 // the fluid-solid interface faces
    // point location: uniform bucket grid over the cells' bounding boxes,
    // each bucket listing its cells in increasing order
    int32_t loc_gx = 0, loc_gy = 0;
    double loc_x0 = 0.0, loc_y0 = 0.0, loc_dx = 1.0, loc_dy = 1.0;
    std::vector<int64_t> loc_ptr, loc_ids;
    // per-shot sources of the batched path
    int32_t n_shot_src = 0;
    int32_t* d_shot_src_dom = nullptr;
    int32_t* d_shot_src_q = nullptr;
    double* d_shot_src_g = nullptr;
    float* d_shot_src_g32 = nullptr;
    double shot_f0 = 0.0, shot_t0 = 0.0, shot_amp = 0.0;
    float* d_src_g32 = nullptr;
    f2x* d_src_gx = nullptr;
    f2x* d_shot_src_gx = nullptr;
    // arithmetic of the single-shot stepping entry points (HHO_F64 or HHO_F32X2)
    int32_t arith = HHO_F64;
    // launch mode of the ERK loops and the captured steps (stage.cu)
    int32_t launch_mode = HHO_LAUNCH_AUTO;
    StageClock* d_clock = nullptr;
    void* cap_stream = nullptr;                      // cudaStream_t used for capture
    struct StepGraph {
        std::vector<unsigned char> key;              // byte image of the step's kernel arguments
        void* exec = nullptr;                        // cudaGraphExec_t
    };
    std::vector<StepGraph> graphs;
    // sampled source time functions (hho_sources_set_samples): the value of
    // source s at step n, stage j is src_samples[(s samp_n + n) samp_s + j]
    bool src_sampled = false;
    std::vector<double> src_samples;
    double samp_t0 = 0.0, samp_dt = 0.0;
    int64_t samp_n = 0;
    int32_t samp_s = 0;
    // sources
    int32_t n_src = 0;
    int32_t src_dom[MAX_SOURCES], src_q[MAX_SOURCES];
    double src_f0[MAX_SOURCES], src_t0[MAX_SOURCES], src_amp[MAX_SOURCES];
    double* d_src_g = nullptr;
    // receivers
    int32_t n_rec = 0;
    int32_t* d_rec_int = nullptr;
    double* d_rec_dbl = nullptr;
    // transpose of recording (adjoint): the cells the receivers read, each with
    // its receivers in increasing order.  One int block:
    // [ptr: n_inj + 1][cell: 2 n_inj (domain, position)][receiver ids]
    int32_t n_inj = 0;
    int32_t* d_inj = nullptr;
    // energy
    double* d_mass_f = nullptr;   // per fluid cell: rho h^2, h^2/kappa
    double* d_mass_s = nullptr;   // per solid cell: h^2 * compliance (3), rho h^2
    // host-buffer entry point scratch
    double* d_host_state = nullptr;
    double* d_host_canon = nullptr;
    double* d_host_work = nullptr;
    int64_t host_work_size = 0;
    int64_t n_state = 0;
    int64_t trace_doubles = 0;    // one trace buffer (fluid + solid parts)
    // tensor-core batched stage (HHO_BF16X3): per class the split-BF16
    // operand tiles of its two GEMMs (all faces' lifts, all faces' traces),
    // see tc_tiles in operators.cpp; meta [n_classes][6] = K1, N1, K2, N2,
    // offset of the class's tiles (16-byte units), tile bytes
    void* d_tc_b = nullptr;
    int32_t* d_tc_meta = nullptr;
    int32_t tc_kmax = 0;          // widest A tile (K) over the classes
    int64_t tc_bmax = 0;          // largest tile bytes of one class
    uint32_t tc_cols = 32;        // tensor-memory columns a block allocates
    int32_t* d_tc_err = nullptr;  // set by a tensor-core block whose MMA wait gave up
    bool tc_on = false;           // the current batched call runs the tensor-core stage
    // adjoint support: interface coefficients of the operator with the
    // coupling sign reversed, and per-class M0^-1 (n x n each)
    double* d_if_coef_adj = nullptr;
    float* d_if_coef_adj_f32 = nullptr;   // its FP32 copy (the FP32 adjoint)
    double* d_cls_minv = nullptr;
    // host copies for the cost model and the SDIRK preconditioner's colouring
    std::vector<double> h_cls_dbl;
    std::vector<int32_t> h_cls_int, h_nb_f, h_nb_s, h_if_nb;
    // SDIRK block-Jacobi preconditioner: (I - a* dt J_TT)^-1 of every cell,
    // entry (r, c) of a fluid cell q at d_bj[(r 3n + c) Nf + q], of a solid
    // cell at d_bj[9n^2 Nf + (r 5n + c) Ns + q], built for a* dt = bj_adt
    int32_t sdirk_precond = 1;
    double* d_bj = nullptr;
    double bj_adt = 0.0;
    int32_t* d_bj_colour = nullptr;   // cell colouring, fluid then solid slots
    int32_t bj_colours = 0;
    // stage-kernel timing (hho_profile_*)
    bool prof_on = false;
    int32_t prof_n = 0;
    std::vector<void*> prof_events;   // cudaEvent_t pairs
};
