// Internal declarations of the crhyb library (not part of the C interface).
//
// Device data layout (all arrays in HBM, allocated once per handle):
//   mesh    coords f64 [nv][d], elems i32 [ne][d+1], elem_face i32 [ne][d+1]
//           (-1: exterior face), elem_side u8 [ne][d+1] (0: the simplex owns
//           the face, C = +1; 1: C = -1), face_elems / face_local i32 [nf][2],
//           cols i32 sliced like G below, 2d planes (ELL columns of slots 1..2d).
//   G       block ELL with NSLOT = 2d+1 slots per face row.  Slot 0 is the
//           diagonal block; slots 1..d are the other local faces of the
//           owner simplex of the row face, in increasing local index; slots
//           d+1..2d those of the second simplex.  A slot whose face is
//           exterior keeps col = row and zero values.  Sliced ELL: the face
//           rows are cut into slices of 256; a slice stores its planes q =
//           (slot*d + i)*d + j one after the other, 256 rows each, so element
//           (f, q) is at ((f/256)*nplanes + q)*256 + f%256.  Consecutive rows
//           are consecutive in memory in every plane (coalesced loads), and a
//           slice is one contiguous run that one bulk copy stages.  The rows
//           of the last slice beyond nf hold zero values and column 0.
//   vectors [nf][d], face major, component fastest.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <initializer_list>
#include <string>
#include <vector>

#include "../../include/crhyb.h"

struct cr_mesh;

namespace crhyb {

constexpr int kSlice = 256;   // face rows per slice of the sliced ELL

// Index of row f in plane q of a sliced-ELL array with nplanes planes.
__host__ __device__ __forceinline__ size_t sell(int64_t f, int q, int nplanes) {
    return (size_t(f >> 8) * size_t(nplanes) + size_t(q)) * kSlice + size_t(f & (kSlice - 1));
}

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define CR_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return ::crhyb::cuda_fail(_e, #call);    \
    } while (0)

#define CR_TRY(call)                                                    \
    do {                                                                \
        int _rc = (call);                                               \
        if (_rc != CR_OK) return _rc;                                   \
    } while (0)

// Where an array argument lives: 1 device memory of the current GPU (or
// managed memory), 0 host memory, -1 device memory of another GPU (*owner
// receives that GPU).  is_device_pointer(p) is pointer_place(p) == 1.
// place_of is the decision from the attributes the driver reports.
inline int place_of(cudaMemoryType type, int owner, int current) {
    if (type == cudaMemoryTypeManaged) return 1;
    if (type != cudaMemoryTypeDevice) return 0;
    return owner == current ? 1 : -1;
}
int pointer_place(const void* p, int* owner);
bool is_device_pointer(const void* p);
// Argument check of an entry point: the handle's mesh (may be NULL) was
// loaded on the current GPU, and no pointer is device memory of another GPU
// (the library launches on the current GPU and enables no peer access).
int check_call(const cr_mesh* m, const char* fn, std::initializer_list<const void*> ptrs);

// Device allocation helper: records the pointer for release by the owner.
struct DevArena {
    std::vector<void*> ptrs;
    int alloc(void** p, size_t bytes);
    template <typename T>
    int alloc_n(T** p, size_t n) { return alloc(reinterpret_cast<void**>(p), n * sizeof(T)); }
    void release();
};

// Deterministic two-level reductions: per-block partial sums, then the last
// block to finish sums the partials in block order.
constexpr int kRedSlots = 4;          // up to 4 simultaneous dot products
constexpr int kMaxRedBlocks = 65536;  // capacity of the partial-sum buffer (blocks per reduction)

struct RedBuf {
    double* partial;      // [kRedSlots][kMaxRedBlocks]
    unsigned int* count;  // completion counter (reset by the last block)
};

// Workspace of the flexible GMRES of cr_solve_steady, kept with the
// preconditioning hybrid (so that the steps of a Newton loop share it): Arnoldi vectors V [m+1][n] and preconditioned
// vectors Z [m][n] over the coupled unknowns (n = nf d + ne), the iterate x,
// b = [R; 0], a residual r; per face unknown the previous level up, the lumped
// mass, the inner solve's W and S; the two-sided S scratch [2][d][nf]; the
// Krylov scalars and a reduction buffer.
struct SteadyWork {
    DevArena arena;
    int m = 0;
    int64_t n = 0;
    double *V = nullptr, *Z = nullptr, *x = nullptr, *b = nullptr, *r = nullptr;
    double *up = nullptr, *mass = nullptr, *W = nullptr, *S = nullptr, *spart = nullptr;
    void* scal = nullptr;
    void* h_scal = nullptr;
    RedBuf red{};
    void release() {
        arena.release();
        if (h_scal) cudaFreeHost(h_scal);
        h_scal = nullptr;
        m = 0;
        n = 0;
    }
};

}  // namespace crhyb

struct cr_mesh {
    int d = 0;
    int device = 0;    // the GPU that was current at cr_mesh_load; every later call on it must run there
    int64_t ne = 0, nv = 0, nf = 0, nf_ext = 0;
    int64_t nfp = 0;   // face rows rounded up to whole slices of the sliced ELL (a multiple of 256)
    int k0 = 0;
    bool has_mis = false;
    cudaStream_t user_stream = nullptr;  // the caller's stream
    cudaStream_t stream = nullptr;       // library-owned stream (graph capture needs a non-default stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // host copies for export
    std::vector<int32_t> h_face_vertices, h_face_elems, h_face_local;
    std::vector<uint8_t> h_mis;
    // device
    crhyb::DevArena arena;
    double* coords = nullptr;
    int32_t* elems = nullptr;
    int32_t* elem_face = nullptr;
    uint8_t* elem_side = nullptr;
    int32_t* face_elems = nullptr;
    int32_t* face_local = nullptr;
    int32_t* cols = nullptr;
    uint8_t* mis = nullptr;
};

struct cr_system {
    cr_mesh* m = nullptr;
    double nu = 0, mu = 0, lam_scale = 2.0;
    int conv = CR_CONV_NONE;
    int nrhs = 1;
    crhyb::DevArena arena;
    double* fbar = nullptr;   // [nrhs][ne][d]
    double* w = nullptr;      // [nf][d] or null
    double* uprev = nullptr;  // [nrhs][nf][d]: previous time level (implicit Euler), used when uprev_on
    bool uprev_on = false;
    cr_coupled* steady_op = nullptr;   // coupled operator of a steady system (cr_solve_steady), made on first use
};

namespace crhyb {
constexpr int kMaxDefl = 16;           // deflation vectors at most
constexpr int kMaxDeflBlocks = 1024;   // blocks of the deflation dot products
// what the deflation kernels read and write
struct DeflDev {
    int k;
    const double* L;     // [k][k] Cholesky factor of E = V^t G V, row-major lower
    double* c;           // [kMaxDefl] coefficients of the last dot-product solve
    float* cf;           // the same in FP32
    double* partial;     // [kMaxDefl][kMaxDeflBlocks] per-block partial sums
    unsigned* count;     // completion counter of the dot products
};
}  // namespace crhyb

// A deflation space (deflate.cu): k vectors V, rounded to FP32, of the G shared by
// every Stokes system of one mesh with one nu and mu; G V, M^{-1} G V (FP64), V in
// FP32, and the Cholesky factor of E = V^t G V.
struct cr_deflation {
    cr_mesh* m = nullptr;
    int dim = 0, k = 0;
    int64_t n = 0;
    double nu = 0, mu = 0;
    uint64_t serial = 0;              // distinguishes spaces in the solvers' graph caches
    std::vector<int> kept;            // indices of the given vectors kept
    crhyb::DevArena arena;
    double *V64 = nullptr, *GV64 = nullptr, *W64 = nullptr;   // [k][n]
    float* V32 = nullptr;                                     // [k][n]
    double* L = nullptr;
    double* c = nullptr;
    float* cf = nullptr;
    double* partial = nullptr;
    unsigned* count = nullptr;
};

struct cr_hybrid {
    cr_system* s = nullptr;
    cr_mesh* m = nullptr;
    int nslot = 0;
    crhyb::DevArena arena;
    double* val64 = nullptr;
    float* val32 = nullptr;
    __nv_bfloat16* val16 = nullptr;
    float2* vff = nullptr;        // float-float values interleaved: (fl32(g), fl32(g - fl32(g)))
    __nv_bfloat16* vlo16 = nullptr; // the same rounded to BF16
    double* S = nullptr;          // [nrhs][nf][d]
    double* minv64 = nullptr;     // [nf*d]
    float* minv32 = nullptr;
    double* lam = nullptr;        // [ne] lambda_K on M_1 (mu = 0)
    double* dpart = nullptr;      // [2][d][d][nf] diagonal contributions per side
    double* spart = nullptr;      // [nrhs][2][d][nf] S contributions per side
    int32_t* status = nullptr;    // device status word
    crhyb::RedBuf red{};
    // Krylov workspace (allocated on first solve)
    bool ws_ready = false;
    int ws_restart = 0;
    double *x64 = nullptr, *r64 = nullptr, *p64 = nullptr, *q64 = nullptr, *b64 = nullptr;
    float *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    float2 *xf = nullptr, *rf = nullptr, *pf = nullptr, *qf = nullptr;  // float-float PCG vectors
    double *bs_rh = nullptr, *bs_v = nullptr, *bs_y = nullptr, *bs_s = nullptr, *bs_z = nullptr,
           *bs_t = nullptr;       // BiCGStab: shadow residual, A y, M p, s, M s, A z
    float* V32 = nullptr;         // GMRES basis [restart+1][N]
    double* V64 = nullptr;        // GMRES basis FP64 [restart+1][N]
    float* Z32 = nullptr;         // GMRES scratch vector
    double* Z64 = nullptr;
    double* cheb = nullptr;       // Chebyshev preconditioner: z (two buffers), d [3][N], lmax slot
    float2* chebf = nullptr;      // the same vectors in float-float [3][N]
    double cheb_lmax = -1.0;      // Gershgorin bound of M^{-1} G (computed on first use)
    double* fgz = nullptr;        // flexible GMRES: preconditioned vectors FP64 [restart][N]
    int fgz_m = 0;
    void* scal = nullptr;         // device Krylov scalars
    void* h_scal = nullptr;       // pinned host mirror
    double* pvol = nullptr;       // recovery scratch
    double* ualt = nullptr;       // recovery: velocity from the non-owner side
    double* stage = nullptr;      // host<->device staging
    size_t stage_bytes = 0;
    static constexpr int kGraphs = 8;   // one captured iteration chunk per solver variant
    cudaGraphExec_t graph_exec[kGraphs] = {};
    std::vector<cudaEvent_t> prof_ev;   // profile = 1: event pairs around SpMV launches
    double prof_ms = 0.0;
    int prof_n = 0;
    int64_t graph_key[kGraphs] = {-1, -1, -1, -1, -1, -1, -1, -1};
    uint64_t graph_tag[kGraphs] = {};   // the deflation space a captured chunk uses (its serial; 0: none)
    int64_t graph_launches[kGraphs] = {};   // kernels in each captured chunk
    void* pplan[3] = {nullptr, nullptr, nullptr};   // persistent PCG plans (FP64, FF, FF_BF16), solve.cu
    crhyb::SteadyWork steady;     // cr_solve_steady with this hybrid as preconditioner (first use)
};

namespace crhyb {

// ---- kernels launched from the API layer (defined in the .cu files) ----
int launch_assemble_export(cr_system* s, double* blocks, cudaStream_t st);
int launch_hybridise(cr_hybrid* h, cudaStream_t st);
int launch_recover(cr_hybrid* h, int rhs, const double* W, double* U, double* P, int normalise,
                   double* jump_dev, cudaStream_t st);
int launch_spmv64(cr_hybrid* h, const double* x, double* y, cudaStream_t st);
int launch_assemble_A(cr_system* s, double* val64, int npl, double* dpart, double* spart, double* R,
                      double* minv64, double* DK, cudaStream_t st);
int solve_impl(cr_hybrid* h, int rhs, const cr_solve_opts* o, double* Wdev, cr_solve_stats* st);
int solve_fgmres_impl(cr_hybrid* h, int rhs, cr_hybrid* pre, const cr_solve_opts* o, double* Wdev,
                      cr_solve_stats* st);
// steady problems: the coupled operator of any system, y = K x or b - K x, b = [R_rhs; 0]
int coupled_build(cr_system* s, cr_coupled** out, bool minres);
int launch_coupled_apply(cr_coupled* c, const double* x, const double* b, double* y, cudaStream_t st);
int launch_coupled_rhs(cr_coupled* c, int rhs, double* b, cudaStream_t st);
// the transient Stokes step of h as a preconditioner: S from the previous level up alone
// (no source) and a divergence gdiv per simplex (D_K^t U_K = gdiv_K; NULL: 0), the
// recovery of U and P (P_{K_0} = 0, not normalised) from W, up and gdiv, the lumped face
// mass m_sigma per face unknown
int launch_rhs_previous(cr_hybrid* h, const double* up, const double* gdiv, double* spart, double* S,
                        cudaStream_t st);
int launch_recover_previous(cr_hybrid* h, const double* up, const double* gdiv, const double* W, double* U,
                            double* P, cudaStream_t st);
int launch_face_mass(cr_mesh* m, double* mass, cudaStream_t st);
int solve_steady_impl(cr_coupled* c, cr_mesh* m, cr_hybrid* pre, int rhs, const cr_solve_opts* o, double* U,
                      double* P, cr_solve_stats* st);
int solve_newton_impl(cr_mesh* m, double nu, const double* fbar, cr_hybrid* pre, const cr_solve_opts* lin, double ntol,
                      int maxn, double* U, double* P, cr_newton_stats* st);
int cheb_step_form_impl(int d, int poly_prec);
// deflation (deflate.cu): dot products g = Y^t v over the space's k vectors (with
// solve: c = E^{-1} g into the space's coefficient slots), x += sign Y c, p -= V c,
// skipped while *done (when given) is set; the space's build and allocation; the
// Lanczos-vector store q = z / sqrt(rz) and the Ritz vectors Y = Q S (the eigenpairs of
// the Lanczos matrix: tridiag.h)
int defl_dots64(const cr_deflation* d, const double* Y, const double* v, bool solve, const int* done, cudaStream_t st);
int defl_dots64f(const cr_deflation* d, const double* Y, const float* v, const int* done, cudaStream_t st);
int defl_dots64ff(const cr_deflation* d, const double* Y, const float2* v, const int* done, cudaStream_t st);
int defl_axpy64(const cr_deflation* d, const double* Y, double sign, double* x, cudaStream_t st);
int defl_project64(const cr_deflation* d, double* p, const int* done, cudaStream_t st);
int defl_projectff(const cr_deflation* d, float2* p, const int* done, cudaStream_t st);
int defl_alloc(cr_hybrid* h, int k, cr_deflation** out);
int defl_build(cr_deflation* d, cr_hybrid* h, cudaStream_t st);
int lanczos_store(int64_t n, const double* z, const double* minv, const double* r, const double* rz, float* q,
                  cudaStream_t st);
int ritz_vectors(int64_t n, int m, int k, const float* Q, const float* S, double* Y, cudaStream_t st);
int lanczos_impl(cr_hybrid* h, int rhs, const cr_solve_opts* o, int m, int k, double* theta, cr_deflation** out);
int solve_ritz_impl(cr_hybrid* h, int rhs, const cr_solve_opts* o, double* W, cr_solve_stats* st, int m, int k,
                    double* theta, cr_deflation** out);
void destroy_persistent_plans(cr_hybrid* h);
size_t kscal_bytes();

// staging buffer for host arguments (api.cu)
int ensure_stage(cr_hybrid* h, size_t bytes);

// Orders the library stream after the caller's stream on entry and the
// caller's stream after the library stream on exit.
struct StreamScope {
    cr_mesh* m;
    explicit StreamScope(cr_mesh* mm) : m(mm) {
        cudaEventRecord(m->ev_in, m->user_stream);
        cudaStreamWaitEvent(m->stream, m->ev_in, 0);
    }
    ~StreamScope() {
        cudaEventRecord(m->ev_out, m->stream);
        cudaStreamWaitEvent(m->user_stream, m->ev_out, 0);
    }
};

}  // namespace crhyb
