// The coupled system of Eq. 10 solved without hybridisation: preconditioned
// MINRES (Paige and Saunders) on
//     [A D^t; D 0] [U; P] = [R; 0],   P_{K_0} = 0,
// the comparison the paper draws against the hybrid method (Section 4).
//
// A (velocity stencil, A_K = S_K (x) Id) lives in the sliced ELL of G with
// the same columns; D_K = -a_{K,sigma} is kept per simplex.  The unknowns are
// one vector [U (nf d) | P (ne)]; the preconditioner is diagonal: 1/diag(A) on
// U and 1/diag(D diag(A)^{-1} D^t) on P, with 0 at K_0, which removes that
// pressure from the Krylov space (P_{K_0} stays 0).
//
// One MINRES step is three kernels: the operator q = K z with the dot z.q;
// the Lanczos vector v_{j+1} = q - (delta/gamma) v_j - (gamma/gamma_{j-1}) v_{j-1}
// with z_{j+1} = M^{-1} v_{j+1}, gamma_{j+1}^2 = z_{j+1}.v_{j+1} and the Givens
// rotation (last block); the direction w_{j+1} and x += c eta w_{j+1}.  The
// step index is a launch argument; a step whose index is past the one at
// which the residual estimate met the tolerance returns at once.

#include <cmath>
#include <cstring>

#include "device_common.cuh"

struct cr_coupled {
    cr_system* s = nullptr;
    cr_mesh* m = nullptr;
    crhyb::DevArena arena;
    int npl = 0;
    double* A = nullptr;       // sliced ELL values, (2d+1) d^2 planes
    double* R = nullptr;       // [nrhs][nf][d]
    double* DK = nullptr;      // [ne][d+1][d]
    double* minv = nullptr;    // [nf d + ne] preconditioner (velocity part first)
    double* dpart = nullptr;   // assembly scratch
    double* spart = nullptr;
    // MINRES workspace, each [nf d + ne]
    double *x = nullptr, *b = nullptr, *q = nullptr, *V = nullptr /*3*/, *W = nullptr /*3*/, *Z = nullptr /*2*/;
    void* scal = nullptr;      // device MScal
    void* h_scal = nullptr;    // pinned mirror
    crhyb::RedBuf red{};
};

namespace crhyb {
namespace {

struct MScal {
    double gamma, gamma_old, gamma1, delta, eta, c, c_old, s, s_old, a1, a2, a3, ceta;
    double inv_g;    // 1/gamma_j of the next operator step
    double inv_gz;   // 1/gamma_j of the direction kernel of the step just rotated
    double rr, bb;   // ||b - K x||^2 and ||b||^2 of the last true-residual check
    int stop_it, status, pad0, pad1;
};

int grid_vec(int64_t n) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    const int64_t want = (n + kBlock - 1) / kBlock, cap = int64_t(sms) * 8;
    return int(want < 1 ? 1 : (want < cap ? want : cap));
}

struct Op {
    int64_t nf, ne;
    int npl;
    const int32_t* cols;
    const double* A;
    const double* DK;
    const int32_t* elem_face;
    const int32_t* face_elems;
    const int32_t* face_local;
};

// y = K (scale z) on one face row (all d components) or one simplex row.
template <int D>
__device__ __forceinline__ void op_face(const Op& o, int64_t f, const double* __restrict__ z, double scale,
                                        double (&y)[D]) {
    constexpr int NS = 2 * D + 1;
    const int64_t N = o.nf * D;
#pragma unroll
    for (int i = 0; i < D; ++i) y[i] = 0.0;
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) {
        const int64_t c = sl == 0 ? f : int64_t(__ldg(o.cols + sell(f, sl - 1, 2 * D)));
        double xv[D];
#pragma unroll
        for (int j = 0; j < D; ++j) xv[j] = z[c * D + j];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) y[i] = fma(__ldcs(o.A + sell(f, (sl * D + i) * D + j, o.npl)), xv[j], y[i]);
    }
    // D^t p: the two simplices of the face
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int64_t K = __ldg(o.face_elems + f * 2 + k);
        const int l = __ldg(o.face_local + f * 2 + k);
        const double p = z[N + K];
#pragma unroll
        for (int i = 0; i < D; ++i) y[i] += __ldg(o.DK + (K * (D + 1) + l) * D + i) * p;
    }
#pragma unroll
    for (int i = 0; i < D; ++i) y[i] *= scale;
}

template <int D>
__device__ __forceinline__ double op_elem(const Op& o, int64_t K, const double* __restrict__ z, double scale) {
    double y = 0.0;
#pragma unroll
    for (int l = 0; l <= D; ++l) {
        const int64_t f = __ldg(o.elem_face + K * (D + 1) + l);
        if (f < 0) continue;
#pragma unroll
        for (int i = 0; i < D; ++i) y = fma(__ldg(o.DK + (K * (D + 1) + l) * D + i), z[f * D + i], y);
    }
    return y * scale;
}

// y = K x, or y = b - K x when b is given (no reductions).  Blocks [0, nbf)
// take face rows, the rest simplices.
template <int D>
__global__ void __launch_bounds__(kBlock) k_cp_apply(Op o, int nbf, const double* __restrict__ x,
                                                     const double* __restrict__ b, double* __restrict__ y) {
    const int64_t N = o.nf * D;
    if (int(blockIdx.x) < nbf) {
        const int64_t f = int64_t(blockIdx.x) * kBlock + threadIdx.x;
        if (f >= o.nf) return;
        double v[D];
        op_face<D>(o, f, x, 1.0, v);
#pragma unroll
        for (int i = 0; i < D; ++i) y[f * D + i] = b ? b[f * D + i] - v[i] : v[i];
    } else {
        const int64_t K = int64_t(blockIdx.x - nbf) * kBlock + threadIdx.x;
        if (K >= o.ne) return;
        const double v = op_elem<D>(o, K, x, 1.0);
        y[N + K] = b ? b[N + K] - v : v;
    }
}

// Blocks [0, nbf) take face rows, the rest simplices.  mode 0: q = K (z/gamma),
// delta = q.(z/gamma) (a MINRES step j, skipped past stop_it); mode 1: q = b - K x
// with ||q||^2 and ||b||^2 (true residual; z = x, b given).
template <int D>
__global__ void __launch_bounds__(kBlock) k_mr_op(Op o, int nbf, const double* __restrict__ z,
                                                  const double* __restrict__ b, double* __restrict__ q, MScal* sc,
                                                  RedBuf red, int mode, int j) {
    if (mode == 0 && j > sc->stop_it) return;
    const double scale = mode == 0 ? sc->inv_g : 1.0;
    const int64_t N = o.nf * D;
    double part[2] = {0.0, 0.0};
    if (int(blockIdx.x) < nbf) {
        const int64_t f = int64_t(blockIdx.x) * kBlock + threadIdx.x;
        if (f < o.nf) {
            double y[D];
            op_face<D>(o, f, z, scale, y);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const int64_t k = f * D + i;
                if (mode == 0) {
                    q[k] = y[i];
                    part[0] += y[i] * z[k] * scale;
                } else {
                    const double r = b[k] - y[i];
                    q[k] = r;
                    part[0] += r * r;
                    part[1] += b[k] * b[k];
                }
            }
        }
    } else {
        const int64_t K = int64_t(blockIdx.x - nbf) * kBlock + threadIdx.x;
        if (K < o.ne) {
            const double y = op_elem<D>(o, K, z, scale);
            if (mode == 0) {
                q[N + K] = y;
                part[0] += y * z[N + K] * scale;
            } else {
                const double r = b[N + K] - y;
                q[N + K] = r;
                part[0] += r * r;
                part[1] += b[N + K] * b[N + K];
            }
        }
    }
    double tot[2];
    if (grid_sum<2>(part, red, tot) && threadIdx.x == 0) {
        if (mode == 0) sc->delta = tot[0];
        else {
            sc->rr = tot[0];
            sc->bb = tot[1];
        }
    }
}

// Start of a MINRES cycle from the residual r (in q): v_1 = r, v_0 = 0,
// z_1 = M^{-1} r, gamma_1 = sqrt(z_1.r); w_0 = w_1 = 0.
__global__ void __launch_bounds__(kBlock) k_mr_start(int64_t n, const double* __restrict__ r,
                                                     const double* __restrict__ minv, double* __restrict__ V,
                                                     double* __restrict__ W, double* __restrict__ Z, MScal* sc,
                                                     RedBuf red) {
    double part[1] = {0.0};
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const double v = r[k], z = minv[k] * v;
        V[k] = 0.0;            // v_0 (ring slot 0)
        V[n + k] = v;          // v_1 (ring slot 1)
        W[k] = 0.0;
        W[n + k] = 0.0;
        Z[k] = z;              // z_1 (slot 0)
        part[0] += z * v;
    }
    double tot[1];
    if (grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        const double g = sqrt(fmax(tot[0], 0.0));
        sc->gamma = g;
        sc->gamma1 = g;
        sc->gamma_old = 1.0;
        sc->eta = g;
        sc->c = sc->c_old = 1.0;
        sc->s = sc->s_old = 0.0;
        sc->inv_g = g > 0.0 ? 1.0 / g : 0.0;
        sc->status = isfinite(g) ? CR_OK : CR_ERR_BREAKDOWN;
        sc->stop_it = (g > 0.0 && isfinite(g)) ? 0x7fffffff : -1;
    }
}

// Step j: v_{j+1} = q - (delta/gamma) v_j - (gamma/gamma_old) v_{j-1},
// z_{j+1} = M^{-1} v_{j+1}, gamma_{j+1}; last block: the rotation.
// Ring slots: v_{j-1} = V[j % 3], v_j = V[(j+1) % 3], v_{j+1} = V[(j+2) % 3];
// z_j = Z[j % 2], z_{j+1} = Z[(j+1) % 2].
__global__ void __launch_bounds__(kBlock) k_mr_lanczos(int64_t n, const double* __restrict__ q,
                                                       const double* __restrict__ minv, double* __restrict__ V,
                                                       double* __restrict__ Z, MScal* sc, RedBuf red, int j,
                                                       double tol, int max_it) {
    if (j > sc->stop_it) return;
    const double g = sc->gamma, dg = sc->delta / g, go = g / sc->gamma_old;
    const double* vo = V + size_t(j % 3) * n;
    const double* vj = V + size_t((j + 1) % 3) * n;
    double* vn = V + size_t((j + 2) % 3) * n;
    double* zn = Z + size_t((j + 1) % 2) * n;
    double part[1] = {0.0};
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const double v = q[k] - dg * vj[k] - go * vo[k];
        const double z = minv[k] * v;
        vn[k] = v;
        zn[k] = z;
        part[0] += z * v;
    }
    double tot[1];
    if (grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        const double gn = sqrt(fmax(tot[0], 0.0));
        const double delta = sc->delta, c = sc->c, s = sc->s, co = sc->c_old, so = sc->s_old;
        const double a0 = c * delta - co * s * g;
        const double a1 = hypot(a0, gn);
        sc->a1 = a1;
        sc->a2 = s * delta + co * c * g;
        sc->a3 = so * g;
        const double cn = a1 > 0.0 ? a0 / a1 : 1.0, sn = a1 > 0.0 ? gn / a1 : 0.0;
        sc->ceta = cn * sc->eta;
        sc->eta = -sn * sc->eta;
        sc->c_old = c;
        sc->s_old = s;
        sc->c = cn;
        sc->s = sn;
        sc->inv_gz = 1.0 / g;          // the scale of z_j, used by the direction kernel of step j
        sc->inv_g = gn > 0.0 ? 1.0 / gn : 0.0;
        sc->gamma_old = g;
        sc->gamma = gn;
        if (!isfinite(gn) || !isfinite(a1) || !(a1 > 0.0)) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->stop_it = j;
        } else if (fabs(sc->eta) <= tol * sc->gamma1 || gn == 0.0 || j + 1 >= max_it) {
            sc->stop_it = j;           // this step's direction kernel still runs
        }
    }
}

// Step j: w_{j+1} = (z_j/gamma_j - a3 w_{j-1} - a2 w_j) / a1, x += c eta w_{j+1}.
// Ring slots: w_{j-1} = W[j % 3], w_j = W[(j+1) % 3], w_{j+1} = W[(j+2) % 3].
__global__ void __launch_bounds__(kBlock) k_mr_update(int64_t n, const double* __restrict__ Z,
                                                      double* __restrict__ W, double* __restrict__ x, MScal* sc,
                                                      int j) {
    if (j > sc->stop_it) return;
    const double ig = sc->inv_gz, a1 = sc->a1, a2 = sc->a2, a3 = sc->a3, ce = sc->ceta;
    const double* zj = Z + size_t(j % 2) * n;
    const double* wo = W + size_t(j % 3) * n;
    const double* wj = W + size_t((j + 1) % 3) * n;
    double* wn = W + size_t((j + 2) % 3) * n;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const double w = (zj[k] * ig - a3 * wo[k] - a2 * wj[k]) / a1;
        wn[k] = w;
        x[k] += ce * w;
    }
}

// Pressure preconditioner: 1/sum_{l, i} a_{K,l,i}^2 / A_{(l,i),(l,i)}, 0 at K_0.
template <int D>
__global__ void __launch_bounds__(kBlock) k_mr_schur(int64_t ne, int k0, const int32_t* __restrict__ elem_face,
                                                     const double* __restrict__ DK, double* __restrict__ minv,
                                                     int64_t N) {
    const int64_t K = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (K >= ne) return;
    double s = 0.0;
#pragma unroll
    for (int l = 0; l <= D; ++l) {
        const int64_t f = elem_face[K * (D + 1) + l];
        if (f < 0) continue;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const double a = DK[(K * (D + 1) + l) * D + i];
            s += a * a * minv[f * D + i];
        }
    }
    minv[N + K] = (K == k0 || !(s > 0.0)) ? 0.0 : 1.0 / s;
}

// b = [R_rhs; 0]
__global__ void k_mr_rhs(int64_t N, int64_t ne, const double* __restrict__ R, double* __restrict__ b) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < N + ne; k += int64_t(gridDim.x) * blockDim.x)
        b[k] = k < N ? R[k] : 0.0;
}

template <int D>
int solve_coupled_dim(cr_coupled* c, int rhs, const cr_solve_opts* o, double* U, double* P, cr_solve_stats* st) {
    cr_mesh* m = c->m;
    cudaStream_t s = m->stream;
    const int64_t N = m->nf * D, ne = m->ne, n = N + ne;
    MScal* sc = static_cast<MScal*>(c->scal);
    MScal* hs = static_cast<MScal*>(c->h_scal);
    Op op{m->nf, ne, c->npl, m->cols, c->A, c->DK, m->elem_face, m->face_elems, m->face_local};
    const int nbf = int((m->nf + kBlock - 1) / kBlock), nbe = int((ne + kBlock - 1) / kBlock);
    if (nbf + nbe > kMaxRedBlocks) return fail(CR_ERR_ARG, "cr_solve_coupled: mesh too large for one reduction pass");
    const int gv = grid_vec(n);
    const int max_it = o->max_iter > 0 ? o->max_iter : 1000000;
    const int max_outer = o->max_outer > 0 ? o->max_outer : 20;
    const int chunk = o->check_every > 0 ? o->check_every : 16;
    int64_t launches = 0;
    k_mr_rhs<<<gv, kBlock, 0, s>>>(N, ne, c->R + size_t(rhs) * N, c->b);
    ++launches;
    if (o->use_x0) {
        CR_CUDA(cudaMemcpyAsync(c->x, U, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        CR_CUDA(cudaMemcpyAsync(c->x + N, P, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
    } else {
        CR_CUDA(cudaMemsetAsync(c->x, 0, sizeof(double) * n, s));
    }
    auto read = [&]() -> int {
        CR_CUDA(cudaMemcpyAsync(hs, sc, sizeof(MScal), cudaMemcpyDeviceToHost, s));
        CR_CUDA(cudaStreamSynchronize(s));
        return CR_OK;
    };
    int status = CR_OK, it = 0, outer = 0;
    double relres = 0.0;
    for (;;) {
        // true residual of the iterate; it starts each MINRES cycle
        k_mr_op<D><<<nbf + nbe, kBlock, 0, s>>>(op, nbf, c->x, c->b, c->q, sc, c->red, 1, 0);
        ++launches;
        CR_CUDA(cudaGetLastError());
        CR_TRY(read());
        relres = hs->bb > 0.0 ? std::sqrt(hs->rr / hs->bb) : 0.0;
        if (!std::isfinite(relres)) { status = CR_ERR_BREAKDOWN; break; }
        if (relres <= o->tol) break;
        if (it >= max_it || outer >= max_outer) { status = CR_ERR_NOT_CONVERGED; break; }
        k_mr_start<<<gv, kBlock, 0, s>>>(n, c->q, c->minv, c->V, c->W, c->Z, sc, c->red);
        ++launches;
        CR_CUDA(cudaGetLastError());
        // the cycle runs until its M^{-1}-norm residual estimate has fallen by the factor
        // the 2-norm still needs, with a margin of 10 (the 2-norm check above decides)
        const double itol = 0.1 * o->tol / relres;
        int j = 0;
        for (;;) {
            for (int k = 0; k < chunk; ++k, ++j) {
                k_mr_op<D><<<nbf + nbe, kBlock, 0, s>>>(op, nbf, c->Z + size_t(j % 2) * n, nullptr, c->q, sc, c->red,
                                                        0, j);
                k_mr_lanczos<<<gv, kBlock, 0, s>>>(n, c->q, c->minv, c->V, c->Z, sc, c->red, j, itol, max_it - it);
                k_mr_update<<<gv, kBlock, 0, s>>>(n, c->Z, c->W, c->x, sc, j);
                launches += 3;
            }
            CR_CUDA(cudaGetLastError());
            CR_TRY(read());
            if (hs->stop_it < 0x7fffffff) break;
        }
        it += hs->stop_it + 1;
        ++outer;
        if (hs->status != CR_OK) { status = hs->status; break; }
    }
    // U and P (P_{K_0} = 0 by construction)
    CR_CUDA(cudaMemcpyAsync(U, c->x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    CR_CUDA(cudaMemcpyAsync(P, c->x + N, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
    CR_CUDA(cudaStreamSynchronize(s));
    if (st) {
        st->iterations = it;
        st->outer = outer;
        st->relres = relres;
        st->status = status;
        st->kernel_launches = launches;
    }
    if (status == CR_ERR_NOT_CONVERGED) return fail(status, "cr_solve_coupled: iteration limit reached before the tolerance");
    if (status == CR_ERR_BREAKDOWN) return fail(status, "cr_solve_coupled: MINRES breakdown (NaN or a zero rotation)");
    return status;
}

}  // namespace
}  // namespace crhyb

using namespace crhyb;

namespace crhyb {

// The coupled operator [A D^t; D 0] of system s (any convection option), its
// right-hand sides and, when `minres`, the MINRES workspace.
int coupled_build(cr_system* s, cr_coupled** out, bool minres) {
    *out = nullptr;
    cr_mesh* m = s->m;
    StreamScope scope(m);
    cr_coupled* c = new cr_coupled();
    c->s = s;
    c->m = m;
    const int d = m->d;
    c->npl = (2 * d + 1) * d * d;
    const size_t N = size_t(m->nf) * d, ne = size_t(m->ne), n = N + ne;
    DevArena tmp;
    auto bail = [&](int rc) {
        tmp.release();
        cr_destroy_coupled(c);
        return rc;
    };
    int rc;
    if ((rc = c->arena.alloc_n(&c->A, size_t(c->npl) * m->nfp)) || (rc = c->arena.alloc_n(&c->R, N * s->nrhs)) ||
        (rc = c->arena.alloc_n(&c->DK, ne * (d + 1) * d)) || (rc = c->arena.alloc_n(&c->minv, n)) ||
        (rc = tmp.alloc_n(&c->dpart, size_t(2) * d * d * m->nf)) ||
        (rc = tmp.alloc_n(&c->spart, size_t(s->nrhs) * 2 * d * m->nf)))
        return bail(rc);
    if (minres &&
        ((rc = c->arena.alloc_n(&c->x, n)) || (rc = c->arena.alloc_n(&c->b, n)) || (rc = c->arena.alloc_n(&c->q, n)) ||
         (rc = c->arena.alloc_n(&c->V, 3 * n)) || (rc = c->arena.alloc_n(&c->W, 3 * n)) ||
         (rc = c->arena.alloc_n(&c->Z, 2 * n)) || (rc = c->arena.alloc(&c->scal, sizeof(MScal))) ||
         (rc = c->arena.alloc_n(&c->red.partial, size_t(kRedSlots) * kMaxRedBlocks)) ||
         (rc = c->arena.alloc_n(&c->red.count, 1))))
        return bail(rc);
    cudaError_t e;
    if (minres) {
        if ((e = cudaMallocHost(&c->h_scal, sizeof(MScal))) != cudaSuccess)
            return bail(cuda_fail(e, "cudaMallocHost"));
        if ((e = cudaMemsetAsync(c->red.count, 0, sizeof(unsigned), m->stream)) != cudaSuccess)
            return bail(cuda_fail(e, "cudaMemsetAsync"));
    }
    if ((e = cudaMemsetAsync(c->A, 0, sizeof(double) * c->npl * m->nfp, m->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMemsetAsync"));
    if ((rc = launch_assemble_A(s, c->A, c->npl, c->dpart, c->spart, c->R, c->minv, c->DK, m->stream))) return bail(rc);
    const unsigned nb = unsigned((ne + kBlock - 1) / kBlock);
    if (d == 2) k_mr_schur<2><<<nb, kBlock, 0, m->stream>>>(ne, m->k0, m->elem_face, c->DK, c->minv, int64_t(N));
    else k_mr_schur<3><<<nb, kBlock, 0, m->stream>>>(ne, m->k0, m->elem_face, c->DK, c->minv, int64_t(N));
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(e, "k_mr_schur"));
    if ((e = cudaStreamSynchronize(m->stream)) != cudaSuccess) return bail(cuda_fail(e, "cr_coupled_create"));
    tmp.release();
    c->dpart = c->spart = nullptr;
    *out = c;
    return CR_OK;
}

int launch_coupled_apply(cr_coupled* c, const double* x, const double* b, double* y, cudaStream_t st) {
    cr_mesh* m = c->m;
    Op op{m->nf, m->ne, c->npl, m->cols, c->A, c->DK, m->elem_face, m->face_elems, m->face_local};
    const int nbf = int((m->nf + kBlock - 1) / kBlock), nbe = int((m->ne + kBlock - 1) / kBlock);
    if (m->d == 2) k_cp_apply<2><<<nbf + nbe, kBlock, 0, st>>>(op, nbf, x, b, y);
    else k_cp_apply<3><<<nbf + nbe, kBlock, 0, st>>>(op, nbf, x, b, y);
    CR_CUDA(cudaGetLastError());
    return CR_OK;
}

int launch_coupled_rhs(cr_coupled* c, int rhs, double* b, cudaStream_t st) {
    cr_mesh* m = c->m;
    const int64_t N = m->nf * m->d, ne = m->ne;
    k_mr_rhs<<<grid_vec(N + ne), kBlock, 0, st>>>(N, ne, c->R + size_t(rhs) * N, b);
    CR_CUDA(cudaGetLastError());
    return CR_OK;
}

}  // namespace crhyb

extern "C" int cr_coupled_create(cr_system* s, cr_coupled** out) {
    if (!out) return fail(CR_ERR_ARG, "cr_coupled_create: out is NULL");
    *out = nullptr;
    if (!s) return fail(CR_ERR_ARG, "cr_coupled_create: NULL system");
    CR_TRY(check_call(s->m, "cr_coupled_create", {}));
    if (s->conv != CR_CONV_NONE)
        return fail(CR_ERR_ARG, "cr_coupled_create: MINRES needs the symmetric (Stokes) system, conv = NONE");
    return coupled_build(s, out, true);
}

extern "C" int cr_solve_coupled(cr_coupled* c, int rhs, const cr_solve_opts* o, double* U, double* P,
                                cr_solve_stats* st) {
    if (st) std::memset(st, 0, sizeof(*st));
    if (!c || !o || !U || !P) return fail(CR_ERR_ARG, "cr_solve_coupled: NULL argument");
    CR_TRY(check_call(c->m, "cr_solve_coupled", {U, P}));
    if (rhs < 0 || rhs >= c->s->nrhs) return fail(CR_ERR_ARG, "cr_solve_coupled: rhs out of range");
    if (o->prec != CR_PREC_FP64) return fail(CR_ERR_ARG, "cr_solve_coupled: MINRES runs in FP64");
    if (o->precond != CR_PRECOND_JACOBI)
        return fail(CR_ERR_ARG, "cr_solve_coupled: MINRES takes its own diagonal preconditioner (precond 0)");
    if (!(o->tol > 0.0)) return fail(CR_ERR_ARG, "cr_solve_coupled: tol must be > 0");
    cr_mesh* m = c->m;
    if (!is_device_pointer(U) || !is_device_pointer(P))
        return fail(CR_ERR_ARG, "cr_solve_coupled: U and P must be device pointers");
    StreamScope scope(m);
    return m->d == 2 ? solve_coupled_dim<2>(c, rhs, o, U, P, st) : solve_coupled_dim<3>(c, rhs, o, U, P, st);
}

extern "C" void cr_destroy_coupled(cr_coupled* c) {
    if (!c) return;
    c->arena.release();
    if (c->h_scal) cudaFreeHost(c->h_scal);
    delete c;
}
