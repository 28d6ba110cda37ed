// Batched hybridised solves: many meshes of uneven size, each with several
// right-hand sides (time or Newton steps sharing one matrix), solved by
// Jacobi-PCG (hybrid method, step 2; Section 3.2, item 6) in one persistent
// cooperative launch (persist.cu).  The right-hand sides of a mesh share
// every pass over its G.
//
// The plan lays the problems' tiles end to end.  Three groupings of the
// right-hand sides: one system per problem (its right-hand sides share each
// pass over G, a block SpMM), one system per pair of right-hand sides, or one
// system per (problem, right-hand side) (G read once per right-hand side by the
// leanest kernel).  Fewer right-hand sides per system need fewer registers and
// let more blocks reside on an SM; more share more of G's traffic.  An
// autotuner times the groupings and the resident blocks per SM on the first
// solve and keeps the fastest.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "persist.h"

struct cr_batch {
    std::vector<cr_hybrid*> probs;
    int d = 2, mode = 0;
    crhyb::PersistPlan plan;
    crhyb::DevArena arena;
    std::vector<int> nrhs;          // per problem
    std::vector<int64_t> n;         // unknowns per problem
    std::vector<double*> x64, r64;  // per problem [nrhs][n]
    std::vector<void*> x, r, p, q;
    std::vector<crhyb::PSys> sys[3];  // [0]: one system per problem; [1]: one per right-hand side;
                                      // [2]: one per two right-hand sides
    std::vector<int2> pair[3];        // per (problem, rhs) pair: (system, right-hand side within it)
    int group = 0;                    // the grouping in use
    cudaStream_t stream = nullptr;
    bool tuned = false;
    int bps = 0;                      // chosen resident blocks per SM
    double tune_ms[3][8] = {};        // autotuner: time per PCG iteration of each candidate
};

namespace crhyb {
namespace {

int zero_vectors(cr_batch* b, cudaStream_t st) {
    const bool ff = b->mode != 0;
    for (size_t k = 0; k < b->probs.size(); ++k) {
        const size_t len = size_t(b->nrhs[k]) * b->n[k];
        const size_t vb = ff ? sizeof(float2) : sizeof(double);
        CR_CUDA(cudaMemsetAsync(b->p[k], 0, vb * len, st));
        if (ff) CR_CUDA(cudaMemsetAsync(b->x[k], 0, vb * len, st));
    }
    return CR_OK;
}

}  // namespace
}  // namespace crhyb

using namespace crhyb;

extern "C" int cr_batch_create(cr_hybrid* const* probs, int nprob, const cr_batch_opts* o, cr_batch** out) {
    if (!out) return fail(CR_ERR_ARG, "cr_batch_create: out is NULL");
    *out = nullptr;
    if (!probs || nprob < 1) return fail(CR_ERR_ARG, "cr_batch_create: no problems");
    const int prec = o ? o->prec : CR_PREC_FF;
    if (prec != CR_PREC_FP64 && prec != CR_PREC_FF && prec != CR_PREC_FF_BF16)
        return fail(CR_ERR_ARG, "cr_batch_create: the batched solve runs in FP64, FF or FF_BF16");
    for (int k = 0; k < nprob; ++k)
        if (probs[k]) CR_TRY(check_call(probs[k]->m, "cr_batch_create", {}));
    cr_batch* b = new cr_batch();
    auto bail = [&](int rc) {
        cr_destroy_batch(b);
        return rc;
    };
    b->mode = prec == CR_PREC_FP64 ? 0 : (prec == CR_PREC_FF ? 1 : 2);
    const bool ff = b->mode != 0;
    b->tuned = !(o && o->autotune);
    b->bps = o && o->blocks_per_sm > 0 ? o->blocks_per_sm : 0;
    b->group = (o && o->rhs_grouping == 2) ? 1 : ((o && o->rhs_grouping == 3) ? 2 : 0);
    for (int k = 0; k < nprob; ++k) {
        cr_hybrid* h = probs[k];
        if (!h) return bail(fail(CR_ERR_ARG, "cr_batch_create: NULL problem"));
        if (k == 0) {
            b->d = h->m->d;
            b->stream = h->m->stream;
        }
        if (h->m->d != b->d) return bail(fail(CR_ERR_ARG, "cr_batch_create: problems of different dimension"));
        if (h->s->mu <= 0.0 || h->s->conv != CR_CONV_NONE)
            return bail(fail(CR_ERR_ARG, "cr_batch_create: PCG needs a transient Stokes system (mu > 0, b_h = 0)"));
        if (h->s->nrhs > kPMaxRhs) return bail(fail(CR_ERR_ARG, "cr_batch_create: more than 4 right-hand sides"));
        if (h->m->nf < 1) return bail(fail(CR_ERR_ARG, "cr_batch_create: a mesh without interior faces"));
        if ((b->mode == 1 && !h->vff) || (b->mode == 2 && (!h->val32 || !h->vlo16)))
            return bail(fail(CR_ERR_ARG, "cr_batch_create: the float-float values were not kept by cr_hybridise"));
        b->probs.push_back(h);
        const int R = h->s->nrhs;
        const int64_t n = h->m->nf * b->d;
        const size_t len = size_t(R) * n;
        b->nrhs.push_back(R);
        b->n.push_back(n);
        double *x64 = nullptr, *r64 = nullptr;
        void *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
        const size_t vb = ff ? sizeof(float2) : sizeof(double);
        int rc;
        if ((rc = b->arena.alloc_n(&x64, len)) || (rc = b->arena.alloc_n(&r64, len)) ||
            (rc = b->arena.alloc(&p, vb * len)) || (rc = b->arena.alloc(&q, vb * len)))
            return bail(rc);
        if (ff && ((rc = b->arena.alloc(&x, vb * len)) || (rc = b->arena.alloc(&r, vb * len)))) return bail(rc);
        if (!ff) {
            x = x64;
            r = r64;
        }
        b->x64.push_back(x64);
        b->r64.push_back(r64);
        b->x.push_back(x);
        b->r.push_back(r);
        b->p.push_back(p);
        b->q.push_back(q);
        PSys sy{};
        sy.nf = h->m->nf;
        sy.R = R;
        sy.cols = h->m->cols;
        sy.vh = h->val32;
        sy.vl = b->mode == 2 ? static_cast<const void*>(h->vlo16) : static_cast<const void*>(h->vff);
        sy.v64 = h->val64;
        sy.minv32 = h->minv32;
        sy.minv64 = h->minv64;
        sy.b = h->S;
        sy.x64 = x64;
        sy.r64 = r64;
        sy.x = x;
        sy.r = r;
        sy.p = p;
        sy.q = q;
        for (int r = 0; r < R; ++r) b->pair[0].push_back(make_int2(int(b->sys[0].size()), r));
        b->sys[0].push_back(sy);
        // the same problem as R single-right-hand-side systems
        const size_t vb1 = ff ? sizeof(float2) : sizeof(double);
        for (int k2 = 0; k2 < R; ++k2) {
            PSys y = sy;
            const size_t off = size_t(k2) * n;
            y.R = 1;
            y.b = h->S + off;
            y.x64 = x64 + off;
            y.r64 = r64 + off;
            y.x = static_cast<char*>(x) + off * vb1;
            y.r = static_cast<char*>(r) + off * vb1;
            y.p = static_cast<char*>(p) + off * vb1;
            y.q = static_cast<char*>(q) + off * vb1;
            b->pair[1].push_back(make_int2(int(b->sys[1].size()), 0));
            b->sys[1].push_back(y);
        }
        // and as systems of two right-hand sides (the last may have one)
        for (int k2 = 0; k2 < R; k2 += 2) {
            PSys y = sy;
            const size_t off = size_t(k2) * n;
            y.R = std::min(2, R - k2);
            y.b = h->S + off;
            y.x64 = x64 + off;
            y.r64 = r64 + off;
            y.x = static_cast<char*>(x) + off * vb1;
            y.r = static_cast<char*>(r) + off * vb1;
            y.p = static_cast<char*>(p) + off * vb1;
            y.q = static_cast<char*>(q) + off * vb1;
            for (int j2 = 0; j2 < y.R; ++j2) b->pair[2].push_back(make_int2(int(b->sys[2].size()), j2));
            b->sys[2].push_back(y);
        }
    }
    int rc = b->plan.build(b->sys[b->group], b->d, b->mode, b->bps);
    if (rc) return bail(rc);
    *out = b;
    return CR_OK;
}

extern "C" int cr_batch_info(const cr_batch* b, int32_t* nsys, int32_t* ntiles, int32_t* grid,
                             int32_t* blocks_per_sm) {
    if (!b) return fail(CR_ERR_ARG, "cr_batch_info: NULL batch");
    // nsys: systems of the grouping in use (problems, or (problem, rhs) pairs)
    if (nsys) *nsys = b->plan.nsys;
    if (ntiles) *ntiles = b->plan.ntiles;
    if (grid) *grid = b->plan.grid;
    if (blocks_per_sm) *blocks_per_sm = b->plan.blocks_per_sm;
    return CR_OK;
}

extern "C" int cr_solve_batched(cr_batch* b, const cr_solve_opts* o, double* const* W, cr_solve_stats* st) {
    if (!b || !o || !W) return fail(CR_ERR_ARG, "cr_solve_batched: NULL argument");
    if (o->method != CR_METHOD_PCG) return fail(CR_ERR_ARG, "cr_solve_batched: the batched solve is PCG");
    if (o->precond != CR_PRECOND_JACOBI) return fail(CR_ERR_ARG, "cr_solve_batched: the batched PCG is Jacobi-preconditioned");
    const int np = int(b->probs.size());
    CR_TRY(check_call(b->probs[0]->m, "cr_solve_batched", {}));
    for (int k = 0; k < np; ++k)
        if (!W[k] || !is_device_pointer(W[k]))
            return fail(CR_ERR_ARG, "cr_solve_batched: W[k] must be device memory of the current GPU");
    cudaStream_t s = b->stream;
    StreamScope scope(b->probs[0]->m);
    const double delta = o->inner_tol > 0 && o->inner_tol < 1 ? o->inner_tol : (b->mode == 2 ? 0.1 : 0.01);
    const int gmax = o->max_iter > 0 ? o->max_iter : 100000;
    // shorter launches than a single solve: between launches the plan drops the
    // problems that have converged and spreads the rest over the resident blocks
    const int per_launch = (o->check_every > 0 ? o->check_every : 16) * 8;
    auto start = [&]() -> int {
        for (int k = 0; k < np; ++k) {
            const size_t len = size_t(b->nrhs[k]) * b->n[k];
            if (o->use_x0) CR_CUDA(cudaMemcpyAsync(b->x64[k], W[k], sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
            else CR_CUDA(cudaMemsetAsync(b->x64[k], 0, sizeof(double) * len, s));
        }
        return zero_vectors(b, s);
    };
    if (!b->tuned) {
        // autotune the grouping of the right-hand sides and the resident blocks per SM:
        // a short run of each candidate from the start state, timed per PCG iteration;
        // the fastest is kept for every later solve
        double best = 1e30;
        int best_g = b->group, best_b = 1;
        for (int g = 0; g < 3; ++g) {
            CR_TRY(b->plan.build(b->sys[g], b->d, b->mode, 0));
            const int maxb = std::min(b->plan.blocks_per_sm, 7);
            for (int cand = 1; cand <= maxb; ++cand) {
                CR_TRY(b->plan.build(b->sys[g], b->d, b->mode, cand));
                CR_TRY(start());
                double ms = 0.0;
                int64_t pit = 0;
                CR_TRY(b->plan.run(o->tol, delta, 64, 64, s, nullptr, true, &ms, &pit));
                const double per = pit > 0 ? ms / double(pit) : 1e30;
                b->tune_ms[g][cand] = per;
                if (per < best) {
                    best = per;
                    best_g = g;
                    best_b = cand;
                }
            }
        }
        b->group = best_g;
        b->bps = best_b;
        CR_TRY(b->plan.build(b->sys[best_g], b->d, b->mode, best_b));
        b->tuned = true;
    }
    CR_TRY(start());
    int64_t launches = 0;
    double kms = 0.0;
    int64_t kit = 0;
    CR_TRY(b->plan.run(o->tol, delta, gmax, per_launch, s, &launches, o->profile != 0, &kms, &kit));
    for (int k = 0; k < np; ++k) {
        const size_t len = size_t(b->nrhs[k]) * b->n[k];
        CR_CUDA(cudaMemcpyAsync(W[k], b->x64[k], sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    }
    CR_CUDA(cudaStreamSynchronize(s));
    int worst = CR_OK;
    int j = 0;
    for (int k = 0; k < np; ++k)
        for (int r = 0; r < b->nrhs[k]; ++r, ++j) {
            const int2 pr = b->pair[b->group][size_t(j)];
            const PScal& P = b->plan.h_scal[size_t(pr.x) * kPMaxRhs + pr.y];
            int status = P.status;
            if (status == CR_OK && !P.conv) status = CR_ERR_NOT_CONVERGED;
            if (status != CR_OK && worst == CR_OK) worst = status;
            if (st) {
                st[j].iterations = P.it;
                st[j].outer = P.outer;
                st[j].relres = P.bb > 0 ? std::sqrt(P.orr / P.bb) : 0.0;
                st[j].status = status;
                st[j].spmv_launches = int32_t(kit);
                st[j].spmv_ms = kms;
                st[j].kernel_launches = launches;
            }
        }
    if (worst == CR_ERR_NOT_CONVERGED) return fail(worst, "cr_solve_batched: a system hit the iteration limit");
    if (worst == CR_ERR_BREAKDOWN) return fail(worst, "cr_solve_batched: Krylov breakdown in a system");
    return worst;
}

extern "C" void cr_destroy_batch(cr_batch* b) {
    if (!b) return;
    b->plan.release();
    b->arena.release();
    delete b;
}
