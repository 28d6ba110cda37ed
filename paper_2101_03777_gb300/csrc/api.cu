// C interface of the crhyb library: handles, argument checks, host/device
// staging, stream ordering and error reporting.  The numerical work is in
// hybridise.cu (element kernels) and solve.cu (Krylov kernels).

#include <cstdio>
#include <initializer_list>
#include <cstring>
#include <string>

#include "internal.h"

namespace crhyb {

size_t kscal_bytes();

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    const int code = (e == cudaErrorMemoryAllocation) ? CR_ERR_OOM : CR_ERR_CUDA;
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return code;
}

int pointer_place(const void* p, int* owner) {
    if (owner) *owner = -1;
    if (!p) return 0;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // clear the sticky-free error of an unknown pointer
        return 0;
    }
    int cur = -1;
    if (a.type == cudaMemoryTypeDevice && cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (owner && a.type == cudaMemoryTypeDevice) *owner = a.device;
    return place_of(a.type, a.device, cur);
}

bool is_device_pointer(const void* p) { return pointer_place(p, nullptr) == 1; }

int check_call(const cr_mesh* m, const char* fn, std::initializer_list<const void*> ptrs) {
    int cur = -1;
    CR_CUDA(cudaGetDevice(&cur));
    if (m && m->device != cur)
        return fail(CR_ERR_ARG, std::string(fn) + ": the handle belongs to GPU " + std::to_string(m->device) +
                                    " but GPU " + std::to_string(cur) + " is current");
    for (const void* p : ptrs) {
        int owner = -1;
        if (pointer_place(p, &owner) < 0)
            return fail(CR_ERR_ARG, std::string(fn) + ": an array argument is device memory of GPU " +
                                        std::to_string(owner) + " but GPU " + std::to_string(cur) +
                                        " is current (no peer access is set up)");
    }
    return CR_OK;
}

int DevArena::alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc");
    }
    ptrs.push_back(*p);
    return CR_OK;
}

void DevArena::release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
}

int ensure_stage(cr_hybrid* h, size_t bytes) {
    if (h->stage_bytes >= bytes) return CR_OK;
    if (h->stage) cudaFree(h->stage);
    h->stage = nullptr;
    h->stage_bytes = 0;
    CR_CUDA(cudaMalloc(&h->stage, bytes));
    h->stage_bytes = bytes;
    return CR_OK;
}

namespace {

// Copy n doubles from a host or device source into a device buffer.
int copy_in(double* dst, const double* src, size_t n, cudaStream_t st) {
    CR_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, st));
    return CR_OK;
}

int ensure_workspace(cr_hybrid* h, bool gmres, int restart, int prec) {
    cr_mesh* m = h->m;
    const size_t n = size_t(m->nf) * m->d;
    if (!h->ws_ready) {
        CR_TRY(h->arena.alloc_n(&h->x64, n));
        CR_TRY(h->arena.alloc_n(&h->r64, n));
        CR_TRY(h->arena.alloc_n(&h->p64, n));
        CR_TRY(h->arena.alloc_n(&h->q64, n));
        CR_TRY(h->arena.alloc_n(&h->x32, n));
        CR_TRY(h->arena.alloc_n(&h->r32, n));
        CR_TRY(h->arena.alloc_n(&h->p32, n));
        CR_TRY(h->arena.alloc_n(&h->q32, n));
        CR_TRY(h->arena.alloc(&h->scal, kscal_bytes()));
        CR_CUDA(cudaMallocHost(&h->h_scal, kscal_bytes()));
        h->ws_ready = true;
    }
    if (gmres && restart > h->ws_restart) {
        if (h->V32) cudaFree(h->V32);
        if (h->V64) cudaFree(h->V64);
        if (h->Z32) cudaFree(h->Z32);
        if (h->Z64) cudaFree(h->Z64);
        h->V32 = nullptr;
        h->V64 = nullptr;
        h->Z32 = nullptr;
        h->Z64 = nullptr;
        h->ws_restart = 0;
        CR_CUDA(cudaMalloc(&h->V32, sizeof(float) * n * (restart + 1)));
        CR_CUDA(cudaMalloc(&h->Z32, sizeof(float) * n));
        CR_CUDA(cudaMalloc(&h->Z64, sizeof(double) * n));
        h->ws_restart = restart;
    }
    if (prec == -1 && !h->bs_rh) {   // BiCGStab
        CR_TRY(h->arena.alloc_n(&h->bs_rh, n));
        CR_TRY(h->arena.alloc_n(&h->bs_v, n));
        CR_TRY(h->arena.alloc_n(&h->bs_y, n));
        CR_TRY(h->arena.alloc_n(&h->bs_s, n));
        CR_TRY(h->arena.alloc_n(&h->bs_z, n));
        CR_TRY(h->arena.alloc_n(&h->bs_t, n));
    }
    if ((prec == CR_PREC_FF || prec == CR_PREC_FF_BF16) && !h->xf) {
        CR_TRY(h->arena.alloc_n(&h->xf, n));
        CR_TRY(h->arena.alloc_n(&h->rf, n));
        CR_TRY(h->arena.alloc_n(&h->pf, n));
        CR_TRY(h->arena.alloc_n(&h->qf, n));
    }
    if (gmres && prec == CR_PREC_FP64 && !h->V64)
        CR_CUDA(cudaMalloc(&h->V64, sizeof(double) * n * (h->ws_restart + 1)));
    return CR_OK;
}

}  // namespace
}  // namespace crhyb

using namespace crhyb;

extern "C" const char* cr_last_error(void) { return g_last_error.c_str(); }

extern "C" int cr_chebyshev_step_form(int dim, int poly_prec) {
    if ((dim != 2 && dim != 3) || (poly_prec != CR_POLY_FP32 && poly_prec != CR_POLY_BF16))
        return fail(CR_ERR_ARG, "cr_chebyshev_step_form: dim must be 2 or 3 and poly_prec FP32 or BF16");
    return cheb_step_form_impl(dim, poly_prec);
}

// ---------------------------------------------------------------------------
extern "C" int cr_assemble_coupled(cr_mesh* m, const cr_params* p, const double* fbar, int nrhs, const double* w,
                                   cr_system** out, double* blocks_out) {
    if (!out) return fail(CR_ERR_ARG, "cr_assemble_coupled: out is NULL");
    *out = nullptr;
    if (!m || !p || !fbar) return fail(CR_ERR_ARG, "cr_assemble_coupled: NULL argument");
    if (nrhs < 1) return fail(CR_ERR_ARG, "cr_assemble_coupled: nrhs must be >= 1");
    if (!(p->nu > 0.0) || !(p->mu >= 0.0)) return fail(CR_ERR_ARG, "cr_assemble_coupled: need nu > 0 and mu >= 0");
    if (p->conv != CR_CONV_NONE && p->conv != CR_CONV_NEWTON && p->conv != CR_CONV_OSEEN)
        return fail(CR_ERR_ARG, "cr_assemble_coupled: unknown convection option");
    if (p->conv != CR_CONV_NONE && (m->d != 2 || !w))
        return fail(CR_ERR_ARG, "cr_assemble_coupled: the convection term needs dim 2 and the field w");
    CR_TRY(check_call(m, "cr_assemble_coupled", {fbar, w, blocks_out}));
    cr_system* s = new cr_system();
    s->m = m;
    s->nu = p->nu;
    s->mu = p->mu;
    s->conv = p->conv;
    s->lam_scale = p->lambda_scale > 0 ? p->lambda_scale : 2.0;
    s->nrhs = nrhs;
    StreamScope scope(m);
    const size_t nfb = size_t(nrhs) * m->ne * m->d;
    int rc;
    if ((rc = s->arena.alloc_n(&s->fbar, nfb)) || (rc = copy_in(s->fbar, fbar, nfb, m->stream))) {
        cr_destroy_system(s);
        return rc;
    }
    if (p->conv != CR_CONV_NONE) {
        const size_t nw = size_t(m->nf) * m->d;
        if ((rc = s->arena.alloc_n(&s->w, nw)) || (rc = copy_in(s->w, w, nw, m->stream))) {
            cr_destroy_system(s);
            return rc;
        }
    }
    if (blocks_out) {
        const int L = (m->d + 1) * m->d;
        const size_t nb = size_t(m->ne) * (size_t(L) * L + L + size_t(nrhs) * L);
        double* dst = blocks_out;
        const bool dev = is_device_pointer(blocks_out);
        if (!dev && (rc = s->arena.alloc_n(&dst, nb))) {
            cr_destroy_system(s);
            return rc;
        }
        if ((rc = launch_assemble_export(s, dst, m->stream))) {
            cr_destroy_system(s);
            return rc;
        }
        if (!dev) {
            cudaError_t e = cudaMemcpyAsync(blocks_out, dst, nb * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
            if (e != cudaSuccess) {
                cr_destroy_system(s);
                return cuda_fail(e, "cr_assemble_coupled: export copy");
            }
        }
    }
    *out = s;
    return CR_OK;
}

extern "C" int cr_system_set_previous(cr_system* s, const double* u_prev) {
    if (!s) return fail(CR_ERR_ARG, "cr_system_set_previous: NULL system");
    if (!u_prev) {
        s->uprev_on = false;
        return CR_OK;
    }
    if (!(s->mu > 0.0)) return fail(CR_ERR_ARG, "cr_system_set_previous: an implicit Euler step needs mu = 1/dt > 0");
    CR_TRY(check_call(s->m, "cr_system_set_previous", {u_prev}));
    cr_mesh* m = s->m;
    const size_t n = size_t(s->nrhs) * m->nf * m->d;
    StreamScope scope(m);
    if (!s->uprev) CR_TRY(s->arena.alloc_n(&s->uprev, n));
    CR_TRY(copy_in(s->uprev, u_prev, n, m->stream));
    s->uprev_on = true;
    return CR_OK;
}

extern "C" void cr_destroy_system(cr_system* s) {
    if (!s) return;
    if (s->steady_op) cr_destroy_coupled(s->steady_op);
    s->arena.release();
    delete s;
}

// ---------------------------------------------------------------------------
extern "C" int cr_hybridise(cr_system* s, const cr_hyb_opts* o, cr_hybrid** out) {
    if (!out) return fail(CR_ERR_ARG, "cr_hybridise: out is NULL");
    *out = nullptr;
    if (!s) return fail(CR_ERR_ARG, "cr_hybridise: NULL system");
    CR_TRY(check_call(s->m, "cr_hybridise", {}));
    if (s->mu == 0.0 && !s->m->has_mis)
        return fail(CR_ERR_ARG, "cr_hybridise: mu = 0 needs the set M_1 of a mesh loaded with need_mis = 1");
    cr_mesh* m = s->m;
    const int d = m->d;
    cr_hybrid* h = new cr_hybrid();
    h->s = s;
    h->m = m;
    h->nslot = 2 * d + 1;
    const size_t nv = size_t(h->nslot) * d * d * m->nfp;   // sliced ELL: whole slices of 256 rows
    const size_t n = size_t(m->nf) * d;
    StreamScope scope(m);
    DevArena tmp;
    int rc = CR_OK;
    auto bail = [&](int code) {
        tmp.release();
        cr_destroy_hybrid(h);
        return code;
    };
    if ((rc = h->arena.alloc_n(&h->val64, nv))) return bail(rc);
    const bool lo32 = o && o->keep_lo_fp32, lo16 = o && o->keep_lo_bf16;
    if (o && (o->keep_fp32 || lo16) && (rc = h->arena.alloc_n(&h->val32, nv))) return bail(rc);
    if (o && o->keep_bf16 && (rc = h->arena.alloc_n(&h->val16, nv))) return bail(rc);
    if (lo32 && (rc = h->arena.alloc_n(&h->vff, nv))) return bail(rc);
    if (lo16 && (rc = h->arena.alloc_n(&h->vlo16, nv))) return bail(rc);
    if ((rc = h->arena.alloc_n(&h->S, n * s->nrhs)) || (rc = h->arena.alloc_n(&h->minv64, n)) ||
        (rc = h->arena.alloc_n(&h->minv32, n)) || (rc = h->arena.alloc_n(&h->status, 1)) ||
        (rc = h->arena.alloc_n(&h->red.partial, size_t(kRedSlots) * kMaxRedBlocks)) ||
        (rc = h->arena.alloc_n(&h->red.count, 1)) || (rc = h->arena.alloc_n(&h->pvol, 4)) ||
        (rc = h->arena.alloc_n(&h->ualt, n)))
        return bail(rc);
    if (s->mu == 0.0 && (rc = h->arena.alloc_n(&h->lam, size_t(m->ne)))) return bail(rc);
    if ((rc = tmp.alloc_n(&h->dpart, size_t(2) * d * d * m->nf)) ||
        (rc = tmp.alloc_n(&h->spart, size_t(s->nrhs) * 2 * d * m->nf)))
        return bail(rc);
    cudaError_t e;
    if ((e = cudaMemsetAsync(h->status, 0, sizeof(int32_t), m->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->red.count, 0, sizeof(unsigned), m->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMemsetAsync"));
    // zero the last slice of every value array: its rows beyond nf are staged, never used
    if (m->nfp > m->nf) {
        const size_t npl = size_t(h->nslot) * d * d, off = size_t(m->nfp - kSlice) * npl;
        auto zero_last = [&](void* base, size_t es) {
            if (!base) return cudaSuccess;
            return cudaMemsetAsync(static_cast<char*>(base) + off * es, 0, npl * kSlice * es, m->stream);
        };
        if ((e = zero_last(h->val64, 8)) != cudaSuccess || (e = zero_last(h->val32, 4)) != cudaSuccess ||
            (e = zero_last(h->val16, 2)) != cudaSuccess || (e = zero_last(h->vff, 8)) != cudaSuccess ||
            (e = zero_last(h->vlo16, 2)) != cudaSuccess)
            return bail(cuda_fail(e, "cudaMemsetAsync"));
    }
    if ((rc = launch_hybridise(h, m->stream))) return bail(rc);
    int32_t status = 0;
    if ((e = cudaMemcpyAsync(&status, h->status, sizeof(int32_t), cudaMemcpyDeviceToHost, m->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(m->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "cr_hybridise"));
    tmp.release();
    h->dpart = nullptr;
    h->spart = nullptr;
    if (status != 0) return bail(fail(CR_ERR_SINGULAR, "cr_hybridise: a singular element matrix (A_K or B_K)"));
    *out = h;
    return CR_OK;
}

extern "C" int cr_hybrid_export(const cr_hybrid* h, int32_t* cols, double* vals, double* S) {
    if (!h) return fail(CR_ERR_ARG, "cr_hybrid_export: NULL handle");
    CR_TRY(check_call(h->m, "cr_hybrid_export", {cols, vals, S}));
    cr_mesh* m = h->m;
    const size_t nf = size_t(m->nf);
    cudaError_t e;
    if ((e = cudaStreamSynchronize(m->stream)) != cudaSuccess) return cuda_fail(e, "cr_hybrid_export");
    // the library keeps G sliced (see internal.h); the export is plane-major with stride nf
    const int npl = h->nslot * m->d * m->d, ncol = 2 * m->d;
    if (cols) {
        std::vector<int32_t> sl(size_t(ncol) * m->nfp), out(size_t(h->nslot) * nf);
        if ((e = cudaMemcpy(sl.data(), m->cols, sl.size() * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "cr_hybrid_export (cols)");
        for (size_t f = 0; f < nf; ++f) out[f] = int32_t(f);   // slot 0 is the diagonal
        for (int q = 0; q < ncol; ++q)
            for (size_t f = 0; f < nf; ++f) out[(q + 1) * nf + f] = sl[sell(int64_t(f), q, ncol)];
        if ((e = cudaMemcpy(cols, out.data(), out.size() * sizeof(int32_t), cudaMemcpyDefault)) != cudaSuccess)
            return cuda_fail(e, "cr_hybrid_export (cols)");
    }
    if (vals) {
        std::vector<double> sl(size_t(npl) * m->nfp), out(size_t(npl) * nf);
        if ((e = cudaMemcpy(sl.data(), h->val64, sl.size() * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "cr_hybrid_export (vals)");
        for (int q = 0; q < npl; ++q)
            for (size_t f = 0; f < nf; ++f) out[q * nf + f] = sl[sell(int64_t(f), q, npl)];
        if ((e = cudaMemcpy(vals, out.data(), out.size() * sizeof(double), cudaMemcpyDefault)) != cudaSuccess)
            return cuda_fail(e, "cr_hybrid_export (vals)");
    }
    if (S && (e = cudaMemcpy(S, h->S, size_t(h->s->nrhs) * nf * m->d * sizeof(double), cudaMemcpyDefault)) !=
                 cudaSuccess)
        return cuda_fail(e, "cr_hybrid_export (S)");
    return CR_OK;
}

extern "C" int cr_apply_G(cr_hybrid* h, const double* x, double* y) {
    if (!h || !x || !y) return fail(CR_ERR_ARG, "cr_apply_G: NULL argument");
    CR_TRY(check_call(h->m, "cr_apply_G", {x, y}));
    if (!is_device_pointer(x) || !is_device_pointer(y)) return fail(CR_ERR_ARG, "cr_apply_G: device pointers expected");
    StreamScope scope(h->m);
    return launch_spmv64(h, x, y, h->m->stream);
}

// A deflation space serves the solves whose G is the one it was built from: the same
// mesh, nu and mu, no convection; PCG in FP64 (Jacobi or Chebyshev) or float-float
// (Chebyshev).
static int check_deflation(const cr_deflation* d, const cr_hybrid* h, const cr_solve_opts* o, const char* fn) {
    const std::string f(fn);
    if (d->m != h->m || d->nu != h->s->nu || d->mu != h->s->mu || h->s->conv != CR_CONV_NONE)
        return fail(CR_ERR_ARG, f + ": the deflation space belongs to another G (mesh, nu, mu or convection)");
    if (o->method != CR_METHOD_PCG) return fail(CR_ERR_ARG, f + ": deflation applies to PCG");
    const bool ok = (o->prec == CR_PREC_FP64) || (o->prec == CR_PREC_FF && o->precond == CR_PRECOND_CHEBYSHEV);
    if (!ok)
        return fail(CR_ERR_ARG, f + ": deflation runs in FP64 PCG (Jacobi or Chebyshev) or float-float Chebyshev PCG");
    return CR_OK;
}

// The checks, the workspace and the staging of a host W shared by cr_solve and
// cr_solve_ritz; `run` solves on the device copy.
template <typename Run>
static int solve_entry(const char* fn, cr_hybrid* h, int rhs, const cr_solve_opts* o, double* W, cr_solve_stats* st,
                       Run run) {
    const std::string f(fn);
    if (st) std::memset(st, 0, sizeof(*st));
    if (!h || !o || !W) return fail(CR_ERR_ARG, f + ": NULL argument");
    CR_TRY(check_call(h->m, fn, {W}));
    if (rhs < 0 || rhs >= h->s->nrhs) return fail(CR_ERR_ARG, f + ": rhs out of range");
    if (o->method != CR_METHOD_PCG && o->method != CR_METHOD_GMRES && o->method != CR_METHOD_BICGSTAB)
        return fail(CR_ERR_ARG, f + ": bad method");
    if (o->method == CR_METHOD_BICGSTAB && o->prec != CR_PREC_FP64)
        return fail(CR_ERR_ARG, f + ": BiCGStab runs in FP64");
    if (o->prec != CR_PREC_FP64 && o->prec != CR_PREC_MIXED_FP32 && o->prec != CR_PREC_MIXED_BF16 &&
        o->prec != CR_PREC_FF && o->prec != CR_PREC_FF_BF16)
        return fail(CR_ERR_ARG, f + ": bad precision");
    if (!(o->tol > 0.0)) return fail(CR_ERR_ARG, f + ": tol must be > 0");
    const int restart = o->restart > 0 ? o->restart : 30;
    if (o->method == CR_METHOD_GMRES && (restart < 1 || restart > CR_MAX_RESTART))
        return fail(CR_ERR_ARG, f + ": restart must be in [1, CR_MAX_RESTART]");
    if (o->precond != CR_PRECOND_JACOBI && o->precond != CR_PRECOND_CHEBYSHEV)
        return fail(CR_ERR_ARG, f + ": bad preconditioner");
    if (o->precond == CR_PRECOND_CHEBYSHEV) {
        if (o->method != CR_METHOD_PCG ||
            (o->prec != CR_PREC_FP64 && o->prec != CR_PREC_FF && o->prec != CR_PREC_FF_BF16))
            return fail(CR_ERR_ARG, f + ": the Chebyshev preconditioner is implemented for PCG in FP64, FF and "
                                        "FF_BF16");
        const int deg = o->poly_degree > 0 ? o->poly_degree : 4;
        if (deg < 2 || deg > CR_MAX_POLY_DEGREE)
            return fail(CR_ERR_ARG, f + ": poly_degree must be in [2, CR_MAX_POLY_DEGREE]");
        if (!(o->poly_ratio <= 0.0 || o->poly_ratio > 1.0))
            return fail(CR_ERR_ARG, f + ": poly_ratio must be > 1 (or <= 0 for the default)");
        if (o->poly_prec != CR_POLY_SAME && o->poly_prec != CR_POLY_FP32 && o->poly_prec != CR_POLY_BF16)
            return fail(CR_ERR_ARG, f + ": bad poly_prec");
        if (o->poly_prec != CR_POLY_SAME && o->prec == CR_PREC_FP64)
            return fail(CR_ERR_ARG, f + ": poly_prec applies to the float-float Chebyshev PCG");
    }
    if (o->deflation) CR_TRY(check_deflation(o->deflation, h, o, fn));
    cr_mesh* m = h->m;
    const size_t n = size_t(m->nf) * m->d;
    StreamScope scope(m);
    CR_TRY(ensure_workspace(h, o->method == CR_METHOD_GMRES, restart, o->prec));
    if (o->method == CR_METHOD_BICGSTAB) CR_TRY(ensure_workspace(h, false, restart, -1));
    if (o->precond == CR_PRECOND_CHEBYSHEV && !h->cheb) CR_TRY(h->arena.alloc_n(&h->cheb, 3 * n + 1));
    if (o->precond == CR_PRECOND_CHEBYSHEV && o->prec != CR_PREC_FP64 && !h->chebf)
        CR_TRY(h->arena.alloc_n(&h->chebf, 3 * n));
    double* Wd = W;
    const bool host = !is_device_pointer(W);
    if (host) {
        CR_TRY(ensure_stage(h, n * sizeof(double)));
        Wd = h->stage;
        if (o->use_x0) CR_CUDA(cudaMemcpyAsync(Wd, W, n * sizeof(double), cudaMemcpyHostToDevice, m->stream));
    }
    int rc = run(Wd);
    if (host) {
        cudaError_t e = cudaMemcpyAsync(W, Wd, n * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess && rc == CR_OK) rc = cuda_fail(e, (f + ": copy of W").c_str());
    }
    return rc;
}

extern "C" int cr_solve(cr_hybrid* h, int rhs, const cr_solve_opts* o, double* W, cr_solve_stats* st) {
    return solve_entry("cr_solve", h, rhs, o, W, st, [&](double* Wd) { return solve_impl(h, rhs, o, Wd, st); });
}

extern "C" int cr_solve_ritz(cr_hybrid* h, int rhs, const cr_solve_opts* o, double* W, cr_solve_stats* st, int m,
                             int k, double* theta, cr_deflation** out) {
    if (!theta || !out) return fail(CR_ERR_ARG, "cr_solve_ritz: NULL argument");
    *out = nullptr;
    if (!h || !o) return fail(CR_ERR_ARG, "cr_solve_ritz: NULL argument");
    if (k < 1 || k > CR_MAX_DEFLATION || m < k || m > CR_MAX_LANCZOS)
        return fail(CR_ERR_ARG, "cr_solve_ritz: need 1 <= k <= CR_MAX_DEFLATION and k <= m <= CR_MAX_LANCZOS");
    if (o->method != CR_METHOD_PCG || o->deflation ||
        !(o->prec == CR_PREC_FP64 || (o->prec == CR_PREC_FF && o->precond == CR_PRECOND_CHEBYSHEV)))
        return fail(CR_ERR_ARG, "cr_solve_ritz: records PCG in FP64 (Jacobi or Chebyshev) or float-float Chebyshev "
                                "PCG, without deflation");
    if (h->s->conv != CR_CONV_NONE || !(h->s->mu > 0.0))
        return fail(CR_ERR_ARG, "cr_solve_ritz: needs the SPD G of a transient Stokes system");
    return solve_entry("cr_solve_ritz", h, rhs, o, W, st,
                       [&](double* Wd) { return solve_ritz_impl(h, rhs, o, Wd, st, m, k, theta, out); });
}

// ---- deflation spaces ---------------------------------------------------------

extern "C" int cr_deflation_create(cr_hybrid* h, int k, const double* V, cr_deflation** out) {
    if (!h || !V || !out) return fail(CR_ERR_ARG, "cr_deflation_create: NULL argument");
    *out = nullptr;
    CR_TRY(check_call(h->m, "cr_deflation_create", {V}));
    if (k < 1 || k > CR_MAX_DEFLATION) return fail(CR_ERR_ARG, "cr_deflation_create: k must be in [1, CR_MAX_DEFLATION]");
    if (h->s->conv != CR_CONV_NONE || !(h->s->mu > 0.0))
        return fail(CR_ERR_ARG, "cr_deflation_create: deflated CG needs the SPD G of a transient Stokes system");
    StreamScope scope(h->m);
    cr_deflation* d = nullptr;
    CR_TRY(defl_alloc(h, k, &d));
    const size_t bytes = sizeof(double) * size_t(k) * size_t(d->n);
    cudaError_t e = cudaMemcpyAsync(d->V64, V, bytes, cudaMemcpyDefault, h->m->stream);
    int rc = e == cudaSuccess ? defl_build(d, h, h->m->stream) : cuda_fail(e, "cr_deflation_create: copy of V");
    if (rc != CR_OK) {
        d->arena.release();
        delete d;
        return rc;
    }
    *out = d;
    return CR_OK;
}

extern "C" int cr_deflation_lanczos(cr_hybrid* h, int rhs, const cr_solve_opts* o, int m, int k, double* theta,
                                    cr_deflation** out) {
    if (!h || !o || !theta || !out) return fail(CR_ERR_ARG, "cr_deflation_lanczos: NULL argument");
    *out = nullptr;
    CR_TRY(check_call(h->m, "cr_deflation_lanczos", {}));
    if (rhs < 0 || rhs >= h->s->nrhs) return fail(CR_ERR_ARG, "cr_deflation_lanczos: rhs out of range");
    if (k < 1 || k > CR_MAX_DEFLATION || m < k || m > CR_MAX_LANCZOS)
        return fail(CR_ERR_ARG, "cr_deflation_lanczos: need 1 <= k <= CR_MAX_DEFLATION and k <= m <= CR_MAX_LANCZOS");
    if (h->s->conv != CR_CONV_NONE || !(h->s->mu > 0.0))
        return fail(CR_ERR_ARG, "cr_deflation_lanczos: deflated CG needs the SPD G of a transient Stokes system");
    if (o->precond != CR_PRECOND_JACOBI && o->precond != CR_PRECOND_CHEBYSHEV)
        return fail(CR_ERR_ARG, "cr_deflation_lanczos: bad preconditioner");
    if (o->precond == CR_PRECOND_CHEBYSHEV) {
        const int deg = o->poly_degree > 0 ? o->poly_degree : 4;
        if (deg < 2 || deg > CR_MAX_POLY_DEGREE || !(o->poly_ratio <= 0.0 || o->poly_ratio > 1.0))
            return fail(CR_ERR_ARG, "cr_deflation_lanczos: bad poly_degree or poly_ratio");
    }
    const size_t n = size_t(h->m->nf) * h->m->d;
    StreamScope scope(h->m);
    CR_TRY(ensure_workspace(h, false, 0, CR_PREC_FP64));
    if (o->precond == CR_PRECOND_CHEBYSHEV && !h->cheb) CR_TRY(h->arena.alloc_n(&h->cheb, 3 * n + 1));
    return lanczos_impl(h, rhs, o, m, k, theta, out);
}

extern "C" int cr_deflation_info(const cr_deflation* d, int32_t* k, int64_t* n) {
    if (!d) return fail(CR_ERR_ARG, "cr_deflation_info: NULL deflation");
    if (k) *k = d->k;
    if (n) *n = d->n;
    return CR_OK;
}

extern "C" int cr_deflation_export(const cr_deflation* d, double* V) {
    if (!d || !V) return fail(CR_ERR_ARG, "cr_deflation_export: NULL argument");
    CR_TRY(check_call(d->m, "cr_deflation_export", {V}));
    StreamScope scope(d->m);
    CR_CUDA(cudaMemcpyAsync(V, d->V64, sizeof(double) * size_t(d->k) * size_t(d->n), cudaMemcpyDefault, d->m->stream));
    CR_CUDA(cudaStreamSynchronize(d->m->stream));
    return CR_OK;
}

extern "C" void cr_destroy_deflation(cr_deflation* d) {
    if (!d) return;
    // cudaFree waits for the device; the mesh (and its stream), which may be gone
    // already, is not touched here
    d->arena.release();
    delete d;
}

extern "C" int cr_solve_preconditioned(cr_hybrid* h, int rhs, cr_hybrid* pre, const cr_solve_opts* o, double* W,
                                       cr_solve_stats* st) {
    if (st) std::memset(st, 0, sizeof(*st));
    if (!h || !pre || !o || !W) return fail(CR_ERR_ARG, "cr_solve_preconditioned: NULL argument");
    CR_TRY(check_call(h->m, "cr_solve_preconditioned", {W}));
    if (rhs < 0 || rhs >= h->s->nrhs) return fail(CR_ERR_ARG, "cr_solve_preconditioned: rhs out of range");
    if (pre->m != h->m) return fail(CR_ERR_ARG, "cr_solve_preconditioned: pre must be hybridised on the same mesh");
    if (pre->s->mu <= 0.0 || pre->s->conv != CR_CONV_NONE)
        return fail(CR_ERR_ARG, "cr_solve_preconditioned: pre needs a transient Stokes system (mu > 0, b_h = 0), "
                                "whose G is SPD");
    if (o->method != CR_METHOD_GMRES) return fail(CR_ERR_ARG, "cr_solve_preconditioned: the outer method is GMRES");
    if (o->precond != CR_PRECOND_JACOBI && o->precond != CR_PRECOND_CHEBYSHEV)
        return fail(CR_ERR_ARG, "cr_solve_preconditioned: bad preconditioner of the inner PCG");
    if (o->prec != CR_PREC_FP64 && o->prec != CR_PREC_FF && o->prec != CR_PREC_FF_BF16)
        return fail(CR_ERR_ARG, "cr_solve_preconditioned: the inner PCG runs in FP64, FF or FF_BF16");
    if ((o->prec == CR_PREC_FF && !pre->vff) || (o->prec == CR_PREC_FF_BF16 && (!pre->val32 || !pre->vlo16)))
        return fail(CR_ERR_ARG, "cr_solve_preconditioned: the float-float values of pre were not kept");
    if (o->precond == CR_PRECOND_CHEBYSHEV) {
        const int deg = o->poly_degree > 0 ? o->poly_degree : 4;
        if (deg < 2 || deg > CR_MAX_POLY_DEGREE || !(o->poly_ratio <= 0.0 || o->poly_ratio > 1.0))
            return fail(CR_ERR_ARG, "cr_solve_preconditioned: bad poly_degree or poly_ratio");
        if (o->poly_prec != CR_POLY_SAME && o->poly_prec != CR_POLY_FP32 && o->poly_prec != CR_POLY_BF16)
            return fail(CR_ERR_ARG, "cr_solve_preconditioned: bad poly_prec");
        if (o->poly_prec != CR_POLY_SAME && o->prec == CR_PREC_FP64)
            return fail(CR_ERR_ARG, "cr_solve_preconditioned: poly_prec applies to the float-float Chebyshev PCG");
    }
    if (o->deflation) {   // a space of pre's G deflates every inner solve
        cr_solve_opts io = *o;
        io.method = CR_METHOD_PCG;
        CR_TRY(check_deflation(o->deflation, pre, &io, "cr_solve_preconditioned"));
    }
    if (!(o->tol > 0.0)) return fail(CR_ERR_ARG, "cr_solve_preconditioned: tol must be > 0");
    const int restart = o->restart > 0 ? o->restart : 30;
    if (restart < 1 || restart > CR_MAX_RESTART)
        return fail(CR_ERR_ARG, "cr_solve_preconditioned: restart must be in [1, CR_MAX_RESTART]");
    cr_mesh* m = h->m;
    const size_t n = size_t(m->nf) * m->d;
    StreamScope scope(m);
    CR_TRY(ensure_workspace(h, true, restart, CR_PREC_FP64));
    CR_TRY(ensure_workspace(pre, false, 0, o->prec));
    if (o->precond == CR_PRECOND_CHEBYSHEV && !pre->cheb) CR_TRY(pre->arena.alloc_n(&pre->cheb, 3 * n + 1));
    if (o->precond == CR_PRECOND_CHEBYSHEV && o->prec != CR_PREC_FP64 && !pre->chebf)
        CR_TRY(pre->arena.alloc_n(&pre->chebf, 3 * n));
    if (restart > h->fgz_m) {
        if (h->fgz) cudaFree(h->fgz);
        h->fgz = nullptr;
        h->fgz_m = 0;
        CR_CUDA(cudaMalloc(&h->fgz, sizeof(double) * n * restart));
        h->fgz_m = restart;
    }
    double* Wd = W;
    const bool host = !is_device_pointer(W);
    if (host) {
        CR_TRY(ensure_stage(h, n * sizeof(double)));
        Wd = h->stage;
        if (o->use_x0) CR_CUDA(cudaMemcpyAsync(Wd, W, n * sizeof(double), cudaMemcpyHostToDevice, m->stream));
    }
    int rc = solve_fgmres_impl(h, rhs, pre, o, Wd, st);
    if (host) {
        cudaError_t e = cudaMemcpyAsync(W, Wd, n * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess && rc == CR_OK) rc = cuda_fail(e, "cr_solve_preconditioned: copy of W");
    }
    return rc;
}

extern "C" int cr_solve_steady(cr_system* sys, cr_hybrid* pre, int rhs, const cr_solve_opts* o, double* U, double* P,
                               cr_solve_stats* st) {
    if (st) std::memset(st, 0, sizeof(*st));
    if (!sys || !pre || !o || !U || !P) return fail(CR_ERR_ARG, "cr_solve_steady: NULL argument");
    CR_TRY(check_call(sys->m, "cr_solve_steady", {U, P}));
    if (rhs < 0 || rhs >= sys->nrhs) return fail(CR_ERR_ARG, "cr_solve_steady: rhs out of range");
    if (sys->mu != 0.0) return fail(CR_ERR_ARG, "cr_solve_steady: the system to solve is steady (mu = 0)");
    if (pre->m != sys->m) return fail(CR_ERR_ARG, "cr_solve_steady: pre must be hybridised on the same mesh");
    if (!(pre->s->mu > 0.0) || pre->s->conv != CR_CONV_NONE)
        return fail(CR_ERR_ARG, "cr_solve_steady: pre needs a transient Stokes system (mu > 0, b_h = 0), whose G is SPD");
    if (o->method != CR_METHOD_GMRES) return fail(CR_ERR_ARG, "cr_solve_steady: the outer method is (flexible) GMRES");
    if (o->precond != CR_PRECOND_JACOBI && o->precond != CR_PRECOND_CHEBYSHEV)
        return fail(CR_ERR_ARG, "cr_solve_steady: bad preconditioner of the inner PCG");
    if (o->precond == CR_PRECOND_CHEBYSHEV) {
        const int deg = o->poly_degree > 0 ? o->poly_degree : 4;
        if (deg < 2 || deg > CR_MAX_POLY_DEGREE || !(o->poly_ratio <= 0.0 || o->poly_ratio > 1.0))
            return fail(CR_ERR_ARG, "cr_solve_steady: bad poly_degree or poly_ratio");
    }
    if (o->prec != CR_PREC_FP64 && o->prec != CR_PREC_FF && o->prec != CR_PREC_FF_BF16)
        return fail(CR_ERR_ARG, "cr_solve_steady: the inner PCG runs in FP64, FF or FF_BF16");
    if ((o->prec == CR_PREC_FF && !pre->vff) || (o->prec == CR_PREC_FF_BF16 && (!pre->val32 || !pre->vlo16)))
        return fail(CR_ERR_ARG, "cr_solve_steady: the float-float values of pre were not kept");
    if (!(o->tol > 0.0)) return fail(CR_ERR_ARG, "cr_solve_steady: tol must be > 0");
    const int restart = o->restart > 0 ? o->restart : 30;
    if (restart < 1 || restart > CR_MAX_RESTART)
        return fail(CR_ERR_ARG, "cr_solve_steady: restart must be in [1, CR_MAX_RESTART]");
    if (!is_device_pointer(U) || !is_device_pointer(P))
        return fail(CR_ERR_ARG, "cr_solve_steady: U and P must be device pointers");
    if (o->deflation) {   // a space of pre's G deflates every inner solve
        cr_solve_opts io = *o;
        io.method = CR_METHOD_PCG;
        CR_TRY(check_deflation(o->deflation, pre, &io, "cr_solve_steady"));
    }
    cr_mesh* m = sys->m;
    StreamScope scope(m);
    CR_TRY(ensure_workspace(pre, false, 0, o->prec));
    if (o->precond == CR_PRECOND_CHEBYSHEV) {
        const size_t n = size_t(m->nf) * m->d;
        if (!pre->cheb) CR_TRY(pre->arena.alloc_n(&pre->cheb, 3 * n + 1));
        if (o->prec != CR_PREC_FP64 && !pre->chebf) CR_TRY(pre->arena.alloc_n(&pre->chebf, 3 * n));
    }
    if (!sys->steady_op) CR_TRY(coupled_build(sys, &sys->steady_op, false));
    return solve_steady_impl(sys->steady_op, m, pre, rhs, o, U, P, st);
}

extern "C" int cr_solve_newton(cr_mesh* m, double nu, const double* fbar, cr_hybrid* pre, const cr_solve_opts* lin,
                               double newton_tol, int max_newton, double* U, double* P, cr_newton_stats* st) {
    if (st) std::memset(st, 0, sizeof(*st));
    if (!m || !fbar || !pre || !lin || !U || !P) return fail(CR_ERR_ARG, "cr_solve_newton: NULL argument");
    CR_TRY(check_call(m, "cr_solve_newton", {fbar, U, P}));
    if (m->d != 2) return fail(CR_ERR_ARG, "cr_solve_newton: the convection term is implemented in 2D");
    if (!(nu > 0.0)) return fail(CR_ERR_ARG, "cr_solve_newton: nu must be > 0");
    if (!(newton_tol > 0.0) || max_newton < 1)
        return fail(CR_ERR_ARG, "cr_solve_newton: need newton_tol > 0 and max_newton >= 1");
    if (pre->m != m) return fail(CR_ERR_ARG, "cr_solve_newton: pre must be hybridised on the same mesh");
    if (!(pre->s->mu > 0.0) || pre->s->conv != CR_CONV_NONE)
        return fail(CR_ERR_ARG, "cr_solve_newton: pre needs a transient Stokes system (mu > 0, b_h = 0)");
    if (lin->method != CR_METHOD_GMRES || lin->precond != CR_PRECOND_JACOBI)
        return fail(CR_ERR_ARG, "cr_solve_newton: the linear solves are cr_solve_steady's flexible GMRES");
    if (lin->prec != CR_PREC_FP64 && lin->prec != CR_PREC_FF && lin->prec != CR_PREC_FF_BF16)
        return fail(CR_ERR_ARG, "cr_solve_newton: the inner PCG runs in FP64, FF or FF_BF16");
    if ((lin->prec == CR_PREC_FF && !pre->vff) || (lin->prec == CR_PREC_FF_BF16 && (!pre->val32 || !pre->vlo16)))
        return fail(CR_ERR_ARG, "cr_solve_newton: the float-float values of pre were not kept");
    const int restart = lin->restart > 0 ? lin->restart : 30;
    if (!(lin->tol > 0.0) || restart < 1 || restart > CR_MAX_RESTART)
        return fail(CR_ERR_ARG, "cr_solve_newton: bad tol or restart of the linear solves");
    if (!is_device_pointer(U) || !is_device_pointer(P))
        return fail(CR_ERR_ARG, "cr_solve_newton: U and P must be device pointers");
    if (lin->deflation) {   // a space of pre's G deflates the inner solves (FP64 Jacobi PCG)
        cr_solve_opts io = *lin;
        io.method = CR_METHOD_PCG;
        CR_TRY(check_deflation(lin->deflation, pre, &io, "cr_solve_newton"));
    }
    StreamScope scope(m);
    CR_TRY(ensure_workspace(pre, false, 0, lin->prec));
    return solve_newton_impl(m, nu, fbar, pre, lin, newton_tol, max_newton, U, P, st);
}

extern "C" int cr_recover_up(cr_hybrid* h, int rhs, const double* W, double* U, double* P, int normalise_p,
                             double* jump) {
    if (!h || !W || !U || !P) return fail(CR_ERR_ARG, "cr_recover_up: NULL argument");
    CR_TRY(check_call(h->m, "cr_recover_up", {W, U, P}));
    if (rhs < 0 || rhs >= h->s->nrhs) return fail(CR_ERR_ARG, "cr_recover_up: rhs out of range");
    cr_mesh* m = h->m;
    const size_t n = size_t(m->nf) * m->d, ne = size_t(m->ne);
    StreamScope scope(m);
    const bool hw = !is_device_pointer(W), hu = !is_device_pointer(U), hp = !is_device_pointer(P);
    size_t need = 0;
    if (hw) need += n;
    if (hu) need += n;
    if (hp) need += ne;
    need += 1;   // jump
    CR_TRY(ensure_stage(h, need * sizeof(double)));
    double* cur = h->stage;
    const double* Wd = W;
    double* Ud = U;
    double* Pd = P;
    if (hw) {
        CR_CUDA(cudaMemcpyAsync(cur, W, n * sizeof(double), cudaMemcpyHostToDevice, m->stream));
        Wd = cur;
        cur += n;
    }
    if (hu) { Ud = cur; cur += n; }
    if (hp) { Pd = cur; cur += ne; }
    double* jd = jump ? cur : nullptr;
    CR_TRY(launch_recover(h, rhs, Wd, Ud, Pd, normalise_p, jd, m->stream));
    if (hu) CR_CUDA(cudaMemcpyAsync(U, Ud, n * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    if (hp) CR_CUDA(cudaMemcpyAsync(P, Pd, ne * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    if (jump) CR_CUDA(cudaMemcpyAsync(jump, jd, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    if (hu || hp || jump) CR_CUDA(cudaStreamSynchronize(m->stream));
    return CR_OK;
}

extern "C" void cr_destroy_hybrid(cr_hybrid* h) {
    if (!h) return;
    // cudaFree waits for the device; the mesh (and its stream) is not touched here,
    // so handles may be destroyed in any order.
    for (auto& g : h->graph_exec)
        if (g) cudaGraphExecDestroy(g);
    destroy_persistent_plans(h);
    h->steady.release();
    for (auto e : h->prof_ev) cudaEventDestroy(e);
    h->arena.release();
    if (h->V32) cudaFree(h->V32);
    if (h->V64) cudaFree(h->V64);
    if (h->Z32) cudaFree(h->Z32);
    if (h->Z64) cudaFree(h->Z64);
    if (h->fgz) cudaFree(h->fgz);
    if (h->stage) cudaFree(h->stage);
    if (h->h_scal) cudaFreeHost(h->h_scal);
    delete h;
}
