/*
 * crhyb.h - C interface of the GB300 library for the exact pressure
 * elimination (algebraic hybridisation) of the Crouzeix-Raviart P1
 * nonconforming / P0 discretisation of the Stokes and Navier-Stokes problems
 * (Chenier & Eymard, "Exact pressure elimination for the Crouzeix-Raviart
 * scheme applied to the Stokes and Navier-Stokes problems", arXiv 2101.03777).
 *
 * The library computes, on one GPU:
 *   1. the element blocks S_K, A_K, D_K, R_K of the coupled system
 *      [A D^t; D 0][U; P] = [R; 0]                       (Section 3.1, Eq. 10)
 *   2. the hybridised face system G W = S, element by element
 *      (Section 3.2, items 4 and 5):
 *        B_K = D_K^t Â_K^{-1} D_K,
 *        G_K = C_K (Â_K^{-1} - Â_K^{-1} D_K D_K^t Â_K^{-1} / B_K) C_K, K != K_0,
 *        G_{K_0} = C_{K_0} Â_{K_0}^{-1} C_{K_0},
 *        G = sum_K H_K G_K H_K^t,  S = sum_K H_K C_K M_K R_K;
 *   3. the Krylov solve of G W = S (Jacobi-PCG when G is symmetric positive
 *      definite, Section 3.2 item 6; restarted GMRES otherwise, Section 4.3),
 *      in FP64 or in FP32 inside FP64 iterative refinement;
 *   4. the element-local recovery of P and U (Section 3.2, items 2 and 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns CR_OK (0) or a negative CR_ERR_* code; the text of
 *   the last error of the calling thread is returned by cr_last_error().  No
 *   C++ exception crosses this interface.
 * - Handles (cr_mesh, cr_system, cr_hybrid) are owned by the library and
 *   released by the matching cr_destroy_* call; destroying a handle that
 *   others were created from is the caller's error (destroy in reverse order).
 * - Array arguments are owned by the caller.  Unless stated otherwise an array
 *   argument may be a device pointer or a host pointer: the library asks the
 *   CUDA driver which one it is and copies host data through its own staging
 *   buffers (the copies are part of the call and are stream ordered).  Device
 *   arrays must live on the GPU that is current during the call; device
 *   memory of another GPU is rejected with CR_ERR_ARG before any device work
 *   (the library enables no peer access).
 * - A mesh and every handle made from it belong to the GPU that was current
 *   at cr_mesh_load: a call with another GPU current fails with CR_ERR_ARG.
 * - All device work is ordered on the CUDA stream given to cr_mesh_load (NULL
 *   = the legacy default stream).  Calls that return results to the host
 *   (statistics, host output arrays) synchronise that stream before returning.
 * - Faces: only interior faces carry unknowns (homogeneous Dirichlet, Section
 *   2).  They are numbered in the lexicographic order of their sorted vertex
 *   tuples; cr_mesh_faces reports that order.  Velocity-like arrays U, W, S are
 *   laid out [nrhs][nf_int][d] (face major, component fastest), pressures
 *   [nrhs][ne], element sources fbar [nrhs][ne][d].
 * - Local face l of a simplex is the face opposite its local vertex l.
 */
#ifndef CRHYB_H
#define CRHYB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define CR_OK                  0
#define CR_ERR_ARG            -1  /* invalid argument (NULL handle, bad size, bad option) */
#define CR_ERR_MESH           -2  /* invalid mesh: index out of range, face in > 2 simplices, flat simplex */
#define CR_ERR_SINGULAR       -3  /* an element matrix Â_K or B_K is singular (Section 3.2, item 3) */
#define CR_ERR_NOT_CONVERGED  -4  /* the solve hit its iteration limit before the tolerance */
#define CR_ERR_BREAKDOWN      -5  /* Krylov breakdown: p.Gp <= 0 in PCG, NaN, zero Arnoldi norm */
#define CR_ERR_TIMEOUT        -6  /* a bounded device wait gave up */
#define CR_ERR_CUDA           -7  /* a CUDA runtime call failed (text in cr_last_error) */
#define CR_ERR_OOM            -8  /* device allocation failed */

/* ---- opaque handles ----------------------------------------------------- */
typedef struct cr_mesh cr_mesh;
typedef struct cr_system cr_system;
typedef struct cr_hybrid cr_hybrid;
typedef struct cr_deflation cr_deflation;

/* ---- options and parameters --------------------------------------------- */
typedef struct cr_mesh_opts {
    int32_t k0;        /* index of the simplex K_0 whose pressure is fixed to 0 (Section 2, item 5); default 0 */
    int32_t need_mis;  /* 1: build the maximal independent set M_1 used for E_K when mu = 0 (Section 3.2, item 7) */
} cr_mesh_opts;

enum cr_conv { CR_CONV_NONE = 0, CR_CONV_NEWTON = 1, CR_CONV_OSEEN = 2 };

typedef struct cr_params {
    double nu;         /* viscosity, the inverse of the Reynolds number (Eq. 1) */
    double mu;         /* 1/dt for a transient step, 0 for a steady problem (Eq. 1) */
    int32_t conv;      /* enum cr_conv: b_h = 0 (Stokes), Newton or Oseen linearisation of Eq. 9 */
    double lambda_scale; /* mu = 0 only: lambda_K = lambda_scale * ||A_K||_inf on M_1 (Section 3.2, item 7); <= 0 selects 2 */
} cr_params;

/* Precision of the Krylov solve (every path returns an FP64 W whose FP64 residual is checked):
 *   FP64        native FP64 iteration;
 *   MIXED_FP32  FP32 PCG/GMRES on FP32 values of G, restarted inside FP64 iterative refinement;
 *   MIXED_BF16  the same on BF16 values of G (kept only where the refinement still converges);
 *   FF          float-float PCG: G = hi + lo with FP32 hi and lo planes, vectors as FP32 pairs
 *               (about 48 significant bits), all iteration arithmetic on FP32 units, with FP64
 *               reliable updates (the FP64 true residual, rescaled to unit norm, replaces the
 *               iterated one each time the latter has fallen by inner_tol);
 *   FF_BF16     the same with the low plane of G stored in BF16 (6 bytes per value). */
enum cr_prec { CR_PREC_FP64 = 0, CR_PREC_MIXED_FP32 = 1, CR_PREC_MIXED_BF16 = 2, CR_PREC_FF = 3,
               CR_PREC_FF_BF16 = 4 };
/* Krylov method: PCG (G symmetric positive definite: mu > 0, b_h = 0, Section 3.2 item 6);
 * restarted GMRES(m) with right Jacobi preconditioning (Section 4.3); BiCGStab with right
 * Jacobi preconditioning (van der Vorst), FP64, for nonsymmetric G where restarted GMRES with
 * a Jacobi preconditioner stalls (the Newton/Oseen steps on fine meshes). */
enum cr_method { CR_METHOD_PCG = 0, CR_METHOD_GMRES = 1, CR_METHOD_BICGSTAB = 2 };

/* Preconditioner of PCG.  JACOBI: z = M^{-1} r, M = diag(G).  CHEBYSHEV: z is
 * poly_degree steps of the Jacobi-preconditioned Chebyshev iteration on G z = r
 * from z = 0 (Saad, Iterative Methods for Sparse Linear Systems, Algorithm
 * 12.1) over the interval [lmax/poly_ratio, lmax], lmax the Gershgorin bound
 * of M^{-1} G (largest absolute row sum of M^{-1} G, computed once per
 * hybridised system).  lmax bounds the spectrum, so the preconditioner is a
 * symmetric positive definite polynomial in M^{-1} G times M^{-1}: CG keeps
 * its guarantees and takes about poly_degree times fewer iterations, each
 * applying G poly_degree times. */
enum cr_precond { CR_PRECOND_JACOBI = 0, CR_PRECOND_CHEBYSHEV = 1 };
#define CR_MAX_POLY_DEGREE 32

typedef struct cr_hyb_opts {
    int32_t keep_fp32;  /* also keep FP32 values of G (needed by CR_PREC_MIXED_FP32) */
    int32_t keep_bf16;  /* also keep BF16 values of G (needed by CR_PREC_MIXED_BF16) */
    int32_t keep_lo_fp32; /* also keep the FP32 plane and the FP32 low plane G - fp32(G) (CR_PREC_FF) */
    int32_t keep_lo_bf16; /* also keep the FP32 plane and the BF16 low plane (CR_PREC_FF_BF16) */
} cr_hyb_opts;

typedef struct cr_solve_opts {
    int32_t method;     /* enum cr_method */
    int32_t prec;       /* enum cr_prec */
    double tol;         /* stop when ||S - G W||_2 <= tol ||S||_2 (FP64 residual for the mixed paths,
                           the recursively updated residual for plain FP64 PCG/GMRES) */
    int32_t max_iter;   /* limit on Krylov iterations (inner iterations summed for the mixed paths) */
    int32_t restart;    /* GMRES restart length m (1..CR_MAX_RESTART) */
    double inner_tol;   /* MIXED_*: relative residual of each inner FP32 solve (1e-4 if <= 0);
                           FF*: residual reduction between reliable updates (if <= 0 or >= 1:
                           0.01 for FF, 0.1 for FF_BF16, whose rounded low parts need more
                           frequent updates) */
    int32_t max_outer;  /* mixed paths: limit on refinement steps */
    int32_t use_x0;     /* 1: W holds the initial guess on entry; 0: start from W = 0 */
    int32_t check_every;/* iterations between host convergence checks (0 selects 16) */
    int32_t use_graph;  /* 1: replay the iteration chunk as a captured CUDA graph */
    int32_t profile;    /* 1: time every SpMV launch of the iteration with CUDA events (no graph) */
    int32_t persistent; /* PCG in FP64, FF or FF_BF16 only: 1 runs the iteration in one cooperative
                           persistent launch (grid barriers with bounded waits between its phases;
                           up to check_every*64 iterations per launch) instead of three launches
                           per iteration; profile and use_graph are ignored then */
    int32_t precond;    /* enum cr_precond (0: Jacobi).  CHEBYSHEV is implemented for PCG in FP64, FF and
                           FF_BF16 on the multi-kernel path (persistent is ignored): an iteration is the
                           SpMV of CG, the update, poly_degree - 1 Chebyshev steps (each one SpMV fused
                           with its vector update) and the direction; the float-float forms take FP64
                           reliable updates as their Jacobi forms do; profile = 1 times the Chebyshev
                           steps.  cr_solve_preconditioned, cr_solve_steady, cr_solve_coupled and
                           cr_solve_batched take Jacobi only */
    int32_t poly_degree;/* CHEBYSHEV: polynomial degree, 2..CR_MAX_POLY_DEGREE (0 selects 4) */
    double poly_ratio;  /* CHEBYSHEV: lmax / (lower end of the interval), > 1 (<= 0 selects 100) */
    int32_t poly_prec;  /* CHEBYSHEV with prec FF or FF_BF16: the arithmetic of the Chebyshev steps
                           (the preconditioner only; the CG keeps its precision and its FP64 reliable
                           updates).  enum cr_poly_prec: SAME (the CG's), FP32 (FP32 values of G,
                           kept with keep_fp32 or keep_lo_bf16, FP32 vectors and FMAs), BF16 (BF16
                           values, kept with keep_bf16, FP32 vectors).  A polynomial in M^{-1} G~
                           for the rounded, still symmetric G~ is a fixed symmetric positive definite
                           operator under the same Gershgorin bound, so CG keeps its guarantees up to
                           the FP32 rounding of the steps, which the reliable updates absorb */
    const cr_deflation* deflation; /* NULL, or a deflation space of this G (cr_deflation_create or
                           cr_deflation_lanczos) for deflated PCG: x starts at x + V E^{-1} V^t r
                           (E = V^t G V) and every search direction is made G-orthogonal to V,
                           p = z + beta p - V E^{-1} (G V)^t z, so V^t r = 0 throughout and the
                           eigenvalues of the preconditioned operator on span(V) leave the
                           convergence.  PCG in FP64 (Jacobi or Chebyshev, persistent ignored) or
                           FF with the Chebyshev preconditioner (the dot products with G V in FP64,
                           the projection with V in FP32; every reliable update repeats the
                           deflated start, removing the components along V that the FP32
                           projection lets into r).  The space must come from a system of
                           the same mesh, nu and mu without convection (the same G) */
} cr_solve_opts;

enum cr_poly_prec { CR_POLY_SAME = 0, CR_POLY_FP32 = 1, CR_POLY_BF16 = 2 };

#define CR_MAX_RESTART 64

typedef struct cr_solve_stats {
    int32_t iterations;  /* Krylov iterations (inner iterations summed for the mixed paths) */
    int32_t outer;       /* refinement steps (0 for plain FP64) */
    double relres;       /* final ||S - G W||_2 / ||S||_2 computed in FP64 from the returned W */
    int32_t status;      /* CR_OK or the error code the solve returned */
    int32_t spmv_launches; /* profile = 1: SpMV launches timed (persistent: PCG iterations run by
                              the timed persistent launches) */
    double spmv_ms;      /* profile = 1: their summed device time in ms (persistent: of those launches) */
    int64_t kernel_launches; /* kernels this solve launched (iterations after convergence return at once
                                but still count) */
} cr_solve_stats;

/* ---- mesh --------------------------------------------------------------- */

/* Build the mesh topology (Section 2, item 1): faces from sorted vertex tuples,
 * interior/exterior faces, for each interior face its two simplices (owner =
 * lower simplex index, C = +1; the other C = -1; Section 3.2, Eq. 12), K_0,
 * the block ELL structure of G (stencil of A, Section 3.2 item 5) and, if
 * asked, the maximal independent set M_1 (greedy in increasing simplex index).
 *   dim     2 (triangles) or 3 (tetrahedra)
 *   coords  host, float64 [nv][dim]
 *   elems   host, int32 [ne][dim+1], vertex indices in [0, nv)
 *   opts    may be NULL (defaults)
 *   stream  cudaStream_t on which all later work of this mesh is ordered
 * Errors: CR_ERR_ARG, CR_ERR_MESH (index out of range, a face shared by more
 * than two simplices, a simplex of zero measure), CR_ERR_OOM, CR_ERR_CUDA. */
int cr_mesh_load(int dim, const double* coords, int64_t nv, const int32_t* elems, int64_t ne,
                 const cr_mesh_opts* opts, void* stream, cr_mesh** out);

/* Sizes of a loaded mesh (any output pointer may be NULL). */
int cr_mesh_info(const cr_mesh* m, int32_t* dim, int64_t* ne, int64_t* nf_int, int64_t* nf_ext);

/* Sorted vertex tuples of the interior faces, int32 [nf_int][dim], in the
 * face order used by every face array; host or device pointer. */
int cr_mesh_faces(const cr_mesh* m, int32_t* face_vertices);

/* Face-adjacency structure: per interior face its two simplices (owner first)
 * and its local face index in each, int32 [nf_int][2] each; host or device. */
int cr_mesh_face_elements(const cr_mesh* m, int32_t* face_elems, int32_t* face_local);

/* M_1 flags (uint8 [ne], 1 = in M_1); CR_ERR_ARG if the mesh was loaded without need_mis. */
int cr_mesh_mis(const cr_mesh* m, uint8_t* in_m1);

void cr_destroy_mesh(cr_mesh* m);

/* ---- coupled system ----------------------------------------------------- */

/* Record the coefficients and sources of the coupled system (Section 3.1) and,
 * if blocks_out is not NULL, export its element blocks.
 *   fbar        float64 [nrhs][ne][dim]: element means of the source,
 *               (1/|K|) int_K f, as used by R_K (Eq. 8); copied by the library
 *   nrhs        >= 1 right-hand sides sharing the matrix
 *   w           float64 [nf_int][dim] face velocities about which the convection
 *               term is linearised (conv != NONE), else NULL; copied
 *   blocks_out  NULL or float64 [ne][L*L + L + nrhs*L], L = (dim+1)*dim, per
 *               simplex: A_K (row major), D_K, then R_K per right-hand side,
 *               local unknown (l, i) at l*dim + i, zero rows/columns on exterior
 *               faces; with conv = NEWTON, R_K includes the Newton term c_K(w)
 * Errors: CR_ERR_ARG, CR_ERR_OOM, CR_ERR_CUDA. */
int cr_assemble_coupled(cr_mesh* m, const cr_params* p, const double* fbar, int nrhs,
                        const double* w, cr_system** out, double* blocks_out);

/* Implicit Euler time stepping of the transient problem (mu = 1/dt): make the
 * right-hand side of the next step carry the previous time level,
 *   R_K,(sigma, i) += mu |K|/(d+1) u_prev(sigma, i)   for every interior face sigma of K,
 * the lumped mass that S_K already holds (Section 3.1, with mu = 1/dt as in
 * Section 2), so that the step solves (u^{n+1} - u^n)/dt - nu Lap u^{n+1} + grad p = f.
 *   u_prev  float64 [nrhs][nf_int][dim], host or device; copied.  NULL turns the
 *           term off again.
 * The term enters every later cr_hybridise (S), cr_recover_up (R_K) and export of
 * a hybrid of this system: keep u_prev unchanged between the cr_hybridise and the
 * cr_recover_up of one step.  Errors: CR_ERR_ARG (NULL system, mu <= 0),
 * CR_ERR_OOM, CR_ERR_CUDA. */
int cr_system_set_previous(cr_system* s, const double* u_prev);

void cr_destroy_system(cr_system* s);

/* ---- hybridisation ------------------------------------------------------ */

/* Compute G (block ELL, FP64 plus the FP32/BF16 copies asked for), S for every
 * right-hand side and the Jacobi preconditioner 1/diag(G) (Section 3.2, items
 * 4, 5, 7).  Atomic free: every off-diagonal block of G belongs to one simplex;
 * the two contributions to a diagonal block and to S are summed per face.
 * Errors: CR_ERR_SINGULAR (an Â_K or B_K with a vanishing pivot; the
 * handle is not created), CR_ERR_ARG (mu = 0 on a mesh loaded without
 * need_mis), CR_ERR_OOM, CR_ERR_CUDA. */
int cr_hybridise(cr_system* s, const cr_hyb_opts* o, cr_hybrid** out);

/* Export G as block ELL: cols int32 [nslot][nf_int] (slot 0 is the diagonal),
 * vals float64 [nslot][dim][dim][nf_int], nslot = 2*dim + 1; padding slots have
 * col = row and zero values.  S float64 [nrhs][nf_int][dim].  Any pointer may
 * be NULL; host or device pointers. */
int cr_hybrid_export(const cr_hybrid* h, int32_t* cols, double* vals, double* S);

/* Solve G W = S for right-hand side `rhs` (0 <= rhs < nrhs).
 *   W   float64 [nf_int][dim]: initial guess on entry if opts->use_x0, solution
 *       on exit.  Host or device pointer.
 *   st  host, may be NULL.
 * Returns CR_OK, CR_ERR_NOT_CONVERGED (W holds the last iterate),
 * CR_ERR_BREAKDOWN, CR_ERR_ARG (e.g. a precision whose values were not kept),
 * CR_ERR_CUDA. */
int cr_solve(cr_hybrid* h, int rhs, const cr_solve_opts* opts, double* W, cr_solve_stats* st);

/* ---- deflation spaces ----------------------------------------------------
 * Deflated CG (Saad, Yeung, Erhel and Guyomarc'h, SIAM J. Sci. Comput. 21,
 * 2000) for repeated solves with one G: the steps of a time loop (Section 3.1,
 * implicit Euler: G depends on nu, mu and the mesh, not on the previous level)
 * and several right-hand sides.  The paper has no counterpart: it compares
 * algebraic multigrid and ILU preconditioners instead (Section 4).  A space
 * holds at most CR_MAX_DEFLATION vectors V of length n = dim * nf_int, rounded
 * to FP32 on entry (the FP64 and float-float solvers then deflate the same
 * space), with G V and M^{-1} G V in FP64 and the Cholesky factor of
 * E = V^t G V on the device.  A vector whose Cholesky pivot falls below 1e-2 of its diagonal
 * entry (the sine of its G-angle to the span of those before it below 0.1) is
 * dropped, which keeps E well conditioned for the FP32 dot products of the
 * float-float solves: Ritz vectors are G-orthogonal and pass, while the
 * near-copies that the loss of orthogonality of Lanczos produces do not;
 * cr_deflation_info gives the count kept.  The space serves every system of
 * the same mesh, nu and mu without convection.  Destroy it before its mesh. */
#define CR_MAX_DEFLATION 16
#define CR_MAX_LANCZOS 4096

/* A space from k given vectors V, float64 [k][n], host or device.
 * Errors: CR_ERR_ARG (k out of range, h not the SPD G of a transient Stokes
 * system, no vector with V^t G V > 0), CR_ERR_OOM, CR_ERR_CUDA. */
int cr_deflation_create(cr_hybrid* h, int k, const double* V, cr_deflation** out);

/* A space of Ritz vectors: m steps of FP64 PCG on right-hand side rhs of h from
 * W = 0, with the preconditioner of opts (Jacobi, or Chebyshev with its degree
 * and ratio; opts->prec is not used), storing the normalised preconditioned
 * residuals q_j = z_j / sqrt(r_j . z_j) (FP32, m * n * 4 bytes of scratch).
 * They are orthonormal in the inner product of M (the preconditioner's
 * inverse), and Q^t G Q is the Lanczos matrix T with diagonal 1/alpha_j +
 * beta_{j-1}/alpha_{j-1} and off-diagonal -sqrt(beta_j)/alpha_j from the CG
 * coefficients (Saad, Iterative Methods for Sparse Linear Systems, Section
 * 6.7.3).  The k smallest eigenpairs (theta, s) of T (bisection and inverse
 * iteration on the host) give the Ritz vectors y = Q s, approximate
 * eigenvectors of the preconditioned operator for its smallest eigenvalues.
 *   theta  host, float64 [k]: the Ritz values of the vectors kept, in order (0 after them)
 * Stops early when the residual vanishes.  Errors: CR_ERR_ARG (1 <= k <=
 * CR_MAX_DEFLATION and k <= m <= CR_MAX_LANCZOS, a zero right-hand side),
 * CR_ERR_BREAKDOWN, CR_ERR_OOM, CR_ERR_CUDA. */
int cr_deflation_lanczos(cr_hybrid* h, int rhs, const cr_solve_opts* opts, int m, int k, double* theta,
                         cr_deflation** out);

/* cr_solve that also returns a space of Ritz vectors from its own iterations:
 * the first m iterations of the solve record q_j = z_j / sqrt(r_j . z_j) (FP32,
 * m * n * 4 bytes of scratch) and the CG coefficients on the device, inside the
 * solve's (graph-replayed) launch sequence, and the space follows from them as
 * in cr_deflation_lanczos.  In the float-float form a reliable update rewrites
 * the current vector with the one of the true residual and records the
 * continued beta; a restarted direction (beta = 0) ends the record.  The first
 * solve of a time loop thus yields the space for the later ones at the cost of
 * writing m vectors.  PCG in FP64 (Jacobi or Chebyshev) or FF with the
 * Chebyshev preconditioner, on the multi-kernel path (persistent is ignored),
 * without deflation.  W, st, the return codes as for cr_solve (with
 * CR_ERR_NOT_CONVERGED the space is still formed); theta and out as for
 * cr_deflation_lanczos. */
int cr_solve_ritz(cr_hybrid* h, int rhs, const cr_solve_opts* opts, double* W, cr_solve_stats* st, int m, int k,
                  double* theta, cr_deflation** out);

/* Vectors kept and their length. */
int cr_deflation_info(const cr_deflation* d, int32_t* k, int64_t* n);

/* The space's vectors (as rounded to FP32), float64 [k][n], host or device. */
int cr_deflation_export(const cr_deflation* d, double* V);

void cr_destroy_deflation(cr_deflation* d);

/* Which form of the reduced-precision Chebyshev step kernel (poly_prec FP32 or
 * BF16) cr_solve runs on a dim-dimensional mesh.  An introspection call of the
 * library; the paper has no counterpart.  Every form computes the same step
 * (the SpMV of G on z fused with d <- c1 d + c2 M^{-1}(r - G z), z <- z + d), each
 * face row's sums in the same order:
 *   0  one face row per thread;
 *   1  two adjacent face rows per thread (paired value and column loads);
 *   2  one slice of the sliced ELL per block, its values and columns copied into
 *      shared memory by TMA bulk copies (cp.async.bulk) while the rows' own
 *      vector entries load.
 * The default depends on dim and poly_prec; the environment variable
 * CRHYB_CHEB_KERNEL (rows1, rows2, staged), read once per process, overrides it.
 * Returns the form, or CR_ERR_ARG (dim not 2 or 3, poly_prec not FP32 or BF16). */
int cr_chebyshev_step_form(int dim, int poly_prec);

/* Solve G W = S (right-hand side `rhs` of h) by flexible GMRES(m) in FP64
 * (Saad, Iterative Methods for Sparse Linear Systems, Algorithm 9.6), right-
 * preconditioned by an inner PCG solve with the SPD matrix G_pre of `pre`
 * (the persistent Jacobi-PCG kernel of cr_solve, or its Chebyshev-preconditioned
 * PCG):
 *   z_j = PCG(G_pre, v_j) to relative residual inner_tol,  v_{j+1} from G z_j,
 *   W = W_0 + Z y  (y minimises ||S - G W|| over the cycle).
 * For the nonsymmetric Newton/Oseen systems (Section 4.3) `pre` is the
 * transient Stokes system with the same mu and nu on the same mesh: G_pre^{-1} G
 * departs from the identity only by the convection term, so the number of
 * GMRES steps does not grow as the mesh is refined (Jacobi-preconditioned
 * GMRES(30) stagnates on these systems beyond about 64x64 squares).
 *   h     the system to solve (any conv, mu > 0 or mu = 0)
 *   pre   hybridised on the same mesh handle with conv = NONE and mu > 0;
 *         FF and FF_BF16 need the float-float values kept (keep_lo_fp32 or
 *         keep_lo_bf16); its own S and W are untouched
 *   opts  method GMRES; prec is the precision of the inner PCG (FP64, FF or
 *         FF_BF16); precond JACOBI (the persistent PCG) or CHEBYSHEV (the
 *         Chebyshev-preconditioned PCG of cr_solve, with poly_degree, poly_ratio
 *         and poly_prec as there; FP64 or FF); deflation: a space of pre's G
 *         (the inner solves then run on the multi-kernel path); restart m
 *         (default 30); tol on ||S - G W|| / ||S||; inner_tol (default 0.1);
 *         max_iter caps the GMRES steps (default 1000); use_x0 as for cr_solve;
 *         check_every x 64 inner iterations per persistent launch
 *   W     as for cr_solve
 *   st    iterations = inner PCG iterations in total, outer = GMRES steps,
 *         relres = FP64 relative residual of the returned W; with opts->profile,
 *         spmv_ms and spmv_launches receive the inner persistent launches' time
 *         and the PCG iterations they ran
 * Returns CR_OK, CR_ERR_NOT_CONVERGED, CR_ERR_BREAKDOWN, CR_ERR_ARG, CR_ERR_CUDA. */
int cr_solve_preconditioned(cr_hybrid* h, int rhs, cr_hybrid* pre, const cr_solve_opts* opts, double* W,
                            cr_solve_stats* st);

/* The steady problem (mu = 0) solved without the indefinite G of its E_K
 * elimination: flexible GMRES(m) (Saad, Iterative Methods for Sparse Linear
 * Systems, Algorithm 9.6) on the steady coupled system of Eq. 10,
 *   K_s [U; P] = [R; 0],  K_s = [A_0 D^t; D 0],  P_{K_0} = 0,
 * right-preconditioned by the transient Stokes step of `pre`: each
 * preconditioner application solves K_mu [z_u; z_p] = [v; g] by the hybrid
 * method (Section 3.2: the SPD G_mu of `pre`, persistent Jacobi-PCG, then the
 * element-wise recovery), v entering as the previous level v/(mu m) of an
 * implicit Euler step with no source (m_sigma = sum_{K ni sigma} |K|/(d+1),
 * the lumped mass of S_K) and g as a divergence D_K^t U_K = g_K that the
 * element-wise elimination carries (P_K = (D_K^t Â^{-1} y - g_K)/B_K).  On divergence-free fields K_s K_mu^{-1} has the
 * eigenvalues lambda/(lambda + mu), so the number of steps does not grow with
 * the mesh.  The minimised residual is that of K_s.
 *   sys   assembled with mu = 0 (conv NONE, NEWTON or OSEEN with its field w);
 *         its mesh need not hold M_1; the coupled operator is built on the
 *         first call and kept with sys
 *   pre   hybridised on the same mesh handle, conv = NONE, mu > 0 (e.g. mu = 30
 *         for nu = 1, mu = 1 for nu = 0.01); its own S and W are untouched
 *   opts  method GMRES; prec: precision of the inner PCG (FP64, FF, FF_BF16;
 *         FF needs keep_lo_fp32 on pre); precond: JACOBI (inner solves by the
 *         persistent Jacobi-PCG) or CHEBYSHEV (the Chebyshev-preconditioned PCG
 *         of cr_solve, poly_degree and poly_ratio as there); restart m (default
 *         30); tol on the FP64 residual ||[R;0] - K_s [U;P]|| / ||R||;
 *         inner_tol: relative residual of each inner PCG (default 1e-6; looser
 *         inner solves cost fewer inner iterations on small meshes but let the
 *         outer steps stall from about 384x384 squares on; an inner solve that
 *         stagnates stops at four times the iterations of the first one);
 *         max_iter caps the GMRES steps (default 1000); use_x0: U, P hold the
 *         start; check_every x 64 inner iterations per persistent launch;
 *         deflation: a space of pre's G (cr_deflation_lanczos on pre) deflates
 *         every inner solve (G_mu does not change across the outer steps; the
 *         inner solves then run on the multi-kernel path: FP64 with either
 *         preconditioner, FF with CHEBYSHEV)
 *   U     device float64 [nf_int][dim]; P device float64 [ne] (P_{K_0} = 0, not
 *         normalised)
 *   st    iterations = inner PCG iterations in total, outer = GMRES steps,
 *         relres = the FP64 coupled residual of the returned U, P
 * Returns CR_OK, CR_ERR_NOT_CONVERGED, CR_ERR_BREAKDOWN, CR_ERR_ARG, CR_ERR_CUDA. */
int cr_solve_steady(cr_system* sys, cr_hybrid* pre, int rhs, const cr_solve_opts* opts, double* U, double* P,
                    cr_solve_stats* st);

/* Newton's method for the steady Navier-Stokes problem (Section 3.1: the
 * scheme with the convection term b_h of Eq. 9, mu = 0, homogeneous Dirichlet
 * data), each step a steady linear solve by cr_solve_steady:
 *   U_0 = U on entry (zeros: the first step is the steady Stokes problem);
 *   step k: the coupled system linearised about w = U_k (conv = NEWTON:
 *   Jacobian of b_h at w, right-hand side R + c_K(w)) solved from [U_k; P_k]
 *   to lin->tol, giving U_{k+1}, P_{k+1};
 *   stop when ||U_{k+1} - U_k||_2 <= newton_tol ||U_{k+1}||_2.
 *   m           2D mesh; nu = 1/Re
 *   fbar        float64 [ne][2] element means of the source, host or device
 *   pre         transient Stokes hybrid of the same mesh (as for cr_solve_steady)
 *   lin         options of every linear solve (as for cr_solve_steady; use_x0 is implied)
 *   U, P        device float64 [nf_int][2] (in: U_0; out: the last iterate) and [ne]
 *               (in: P_0; out: P with P_{K_0} = 0)
 *   st          host, may be NULL: Newton steps, GMRES steps and inner PCG
 *               iterations summed, the last increment, the nonlinear relative
 *               residual ||[R + c(U); 0] - K(U)[U; P]|| / ||[R + c(U); 0]|| at
 *               the returned U, P and at U_0
 * Returns CR_OK, CR_ERR_NOT_CONVERGED (max_newton steps without meeting
 * newton_tol), or the error of a linear solve.  */
typedef struct cr_newton_stats {
    int32_t iterations;        /* Newton steps taken */
    int32_t linear_steps;      /* flexible GMRES steps over all Newton steps */
    int64_t inner_iterations;  /* inner PCG iterations over all Newton steps */
    double increment;          /* ||U_{k+1} - U_k|| / ||U_{k+1}|| of the last step */
    double residual;           /* nonlinear relative residual at the returned U, P */
    double first_residual;     /* the same at U_0, P_0 */
    int32_t status;
} cr_newton_stats;

int cr_solve_newton(cr_mesh* m, double nu, const double* fbar, cr_hybrid* pre, const cr_solve_opts* lin,
                    double newton_tol, int max_newton, double* U, double* P, cr_newton_stats* st);

/* y = G x in FP64 (x, y float64 [nf_int][dim], device pointers). */
int cr_apply_G(cr_hybrid* h, const double* x, double* y);

/* Recover P and U from W for right-hand side `rhs` (Section 3.2, items 2, 4):
 * y_K = R_K - C_K W_K, P_K = D_K^t Â_K^{-1} y_K / B_K (K != K_0), P_{K_0} = 0,
 * Û_K = Â_K^{-1}(y_K - D_K P_K), U_sigma = Û_{K,sigma} from the owner K.
 *   W  float64 [nf_int][dim]; U float64 [nf_int][dim]; P float64 [ne]
 *   normalise_p  1: return P - (1/|Omega|) int P (zero mean, Section 2 item 5)
 *   jump  NULL, or host double receiving max |Û_K - Û_L| over interior faces
 *         (Eq. 15 makes it vanish for the exact W)
 * Host or device pointers. */
int cr_recover_up(cr_hybrid* h, int rhs, const double* W, double* U, double* P, int normalise_p,
                  double* jump);

void cr_destroy_hybrid(cr_hybrid* h);

/* ---- the coupled system without hybridisation ------------------------- */

/* The comparison the paper draws against the hybrid method (Section 4): the
 * coupled system of Eq. 10, [A D^t; D 0][U; P] = [R; 0] with P_{K_0} = 0,
 * solved directly by preconditioned MINRES (Paige and Saunders) in FP64,
 * without eliminating the pressure.  A = sum_K H_K A_K H_K^t (A_K = S_K (x) Id,
 * the velocity stencil, stored like G), D_K = -a_{K,sigma}, R as for the hybrid
 * method (including a previous time level set by cr_system_set_previous).
 * The preconditioner is diagonal: 1/diag(A) on U and the inverse diagonal of
 * D diag(A)^{-1} D^t on P (0 at K_0).
 * Only symmetric systems (conv = NONE); mu >= 0. */
typedef struct cr_coupled cr_coupled;

/* Assemble A, R, D_K and the preconditioner of system s (which must outlive
 * the handle).  Errors: CR_ERR_ARG (NULL, conv != NONE), CR_ERR_OOM, CR_ERR_CUDA. */
int cr_coupled_create(cr_system* s, cr_coupled** out);

/* MINRES for right-hand side rhs until ||[R;0] - K [U;P]||_2 <= tol ||R||_2.
 * Each cycle runs until its preconditioned residual estimate |eta| has fallen
 * by a tenth of what the 2-norm still needs; the FP64 true residual then
 * decides, and a shortfall restarts MINRES from the iterate (up to max_outer).
 *   opts  prec FP64; tol; max_iter (MINRES steps in total); max_outer (cycles,
 *         default 20); use_x0 (U, P hold the initial guess); check_every (steps
 *         between host checks)
 *   U     device float64 [nf_int][dim]; P device float64 [ne] (P_{K_0} = 0)
 *   st    iterations = MINRES steps, outer = cycles, relres = the true relative
 *         residual of the returned U, P
 * Returns CR_OK, CR_ERR_NOT_CONVERGED, CR_ERR_BREAKDOWN, CR_ERR_ARG, CR_ERR_CUDA. */
int cr_solve_coupled(cr_coupled* c, int rhs, const cr_solve_opts* opts, double* U, double* P, cr_solve_stats* st);

void cr_destroy_coupled(cr_coupled* c);

/* ---- batched solves ------------------------------------------------------ */

/* Many transient Stokes systems (mu > 0, b_h = 0, so G is SPD: Section 3.2,
 * item 6) of uneven size, each with up to 4 right-hand sides (the nrhs of its
 * cr_assemble_coupled), solved by Jacobi-PCG in one persistent cooperative
 * launch: the face rows of all problems are cut into tiles of 256 rows that
 * the resident blocks sweep in every phase of an iteration, and the
 * right-hand sides of a problem share each pass over its G.  Every
 * (problem, right-hand side) pair has its own scalars and stops on its own
 * FP64 true residual. */
typedef struct cr_batch cr_batch;

typedef struct cr_batch_opts {
    int32_t prec;          /* CR_PREC_FP64, CR_PREC_FF or CR_PREC_FF_BF16 (values kept by cr_hybridise) */
    int32_t autotune;      /* 1: the first solve times the right-hand-side groupings and 1..7 resident
                              blocks per SM (64 iterations each, from the start state) and keeps the
                              fastest for every later solve */
    int32_t blocks_per_sm; /* > 0: cap on the resident blocks per SM (default: the occupancy limit) */
    int32_t rhs_grouping;  /* 0 or 1: the right-hand sides of a problem share each pass over its G (one
                              system per problem); 2: one system per (problem, right-hand side) pair,
                              G read once per right-hand side by the single-right-hand-side kernel;
                              3: one system per two right-hand sides.  With autotune = 1 the three
                              groupings are timed and the fastest is kept */
} cr_batch_opts;

/* Plan a batch over nprob hybridised systems of one dimension.  The handles
 * stay owned by the caller and must outlive the batch; all work is ordered on
 * the stream of the first problem's mesh.  The plan holds the iteration
 * vectors of every problem.  Errors: CR_ERR_ARG (mu = 0 or a convection term,
 * more than 4 right-hand sides, values not kept, dimensions differ), CR_ERR_OOM. */
int cr_batch_create(cr_hybrid* const* probs, int nprob, const cr_batch_opts* o, cr_batch** out);

/* Launch shape of a plan (any output may be NULL): systems of the grouping in use (problems, or
 * (problem, rhs) pairs), tiles, grid and resident blocks per SM. */
int cr_batch_info(const cr_batch* b, int32_t* nsys, int32_t* ntiles, int32_t* grid, int32_t* blocks_per_sm);

/* Solve every (problem, right-hand side) pair.
 *   opts  method PCG; tol, max_iter, inner_tol and use_x0 as for cr_solve; check_every x 8
 *         iterations per launch (between launches the plan drops the converged problems
 *         and spreads the others over the resident blocks); profile = 1 reports the
 *         persistent launches' time
 *   W     nprob device pointers, W[k] float64 [nrhs_k][nf_k][dim] (initial guess on entry
 *         if use_x0, solution on exit)
 *   st    NULL or host [sum_k nrhs_k], pair order problem-major
 * Returns CR_OK, or the first failing pair's status (its W holds the last iterate). */
int cr_solve_batched(cr_batch* b, const cr_solve_opts* opts, double* const* W, cr_solve_stats* st);

void cr_destroy_batch(cr_batch* b);

/* ---- allocation-free residual ------------------------------------------- */

/* The paper has no counterpart to these two entry points.  They serve
 * callers that cannot allocate device memory: a host application whose own
 * pool owns every allocation, code that must avoid the device-wide
 * synchronisation cudaMalloc/cudaFree can cause on its hot path, or a checker
 * that must leave the device's memory exactly as it found it.
 *
 * cr_residual_noalloc computes r = b - G x and the squared norms
 * norms2[0] = ||r||_2^2, norms2[1] = ||b||_2^2 for G in the block ELL layout
 * that cr_hybrid_export writes, without allocating anything.  Its only scratch
 * (per-tile partial sums and two counters, 262,208 bytes) is a fixed device
 * array inside the library, which every GPU that loads the library holds
 * until the process exits.
 *   dim     2 or 3
 *   nf      face rows, 0 <= nf <= cr_residual_noalloc_max_rows() (4,194,304);
 *           larger sizes fail with CR_ERR_ARG before any device work
 *   nslot   block slots per row, 1..2*dim+1 (the export's 2*dim+1)
 *   cols    int32 [nslot][nf] block column of each slot (slot 0 may be the row itself),
 *           device; a column outside [0, nf) is skipped and the call fails with CR_ERR_ARG
 *   vals    float64 [nslot][dim][dim][nf], device
 *   b, x    float64 [nf][dim], device
 *   r       float64 [nf][dim], device, or NULL (norms only)
 *   norms2  float64 [2], host or device
 *   stream  cudaStream_t (NULL = the legacy default stream); every call, nf = 0
 *           included, synchronises it before returning
 * Every call reads its results back to the host and synchronises its stream,
 * so it cannot be recorded inside a CUDA stream capture.  The first call on a
 * device looks up the device address of the scratch array (cudaGetSymbolAddress,
 * once per device, with that device current).  Every call shares the one
 * scratch array, whose counters the call clears first: calls that overlap on
 * the same GPU (from several threads or streams) race and must be serialised
 * by the caller.  Arrays on another GPU than the current one are rejected with
 * CR_ERR_ARG.  Errors: CR_ERR_ARG, CR_ERR_CUDA. */
int cr_residual_noalloc(int dim, int64_t nf, int nslot, const int32_t* cols, const double* vals, const double* b,
                        const double* x, double* r, double* norms2, void* stream);

/* The largest nf that cr_residual_noalloc accepts (its fixed scratch capacity). */
int64_t cr_residual_noalloc_max_rows(void);

/* ---- errors ------------------------------------------------------------- */
const char* cr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CRHYB_H */
