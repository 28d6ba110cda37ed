// Deflation of the CG for G W = S: a space of k vectors V whose G-components
// the iteration keeps out of its search directions (deflated CG: Saad, Yeung,
// Erhel and Guyomarc'h, SIAM J. Sci. Comput. 21, 2000).  With E = V^t G V,
//   x_0 = x + V E^{-1} V^t (b - G x),   p_j = z_j + beta_j p_{j-1} - V E^{-1} (G V)^t z_j,
// every residual stays orthogonal to V and the eigenvalues of the preconditioned
// operator on span(V) drop out of the convergence.  The paper has no counterpart
// (it compares algebraic multigrid and ILU preconditioners, Section 4); this is
// the library's way to cut the iterations of repeated solves with one G (the
// steps of a time loop, several right-hand sides).
//
// This file holds the space (cr_deflation), its kernels and the host linear
// algebra of its small matrices: the Cholesky factor of E, and the eigenpairs of
// the Lanczos matrix T from which cr_deflation_lanczos takes Ritz vectors.

#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "ff.cuh"
#include "internal.h"
#include "tridiag.h"

namespace crhyb {
namespace {

constexpr int kDeflBlock = 256;
constexpr double kDeflPivot = 1e-2;   // kept: sine of the G-angle to the span before it >= 0.1

__device__ __forceinline__ double as_double(double v) { return v; }
__device__ __forceinline__ double as_double(float v) { return double(v); }
__device__ __forceinline__ double as_double(float2 v) { return double(v.x) + double(v.y); }

__device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    return a;
}

// g = Y^t v (k sums, Y [k][n]); the last block sums the per-block partials in
// block order and, with solve, forms c = E^{-1} g from the Cholesky factor
// L (row-major, E = L L^t).  Nothing runs when *done is set (a converged solve).
template <typename YT, typename VT>
__global__ void __launch_bounds__(kDeflBlock) k_defl_dots(int64_t n, const YT* __restrict__ Y,
                                                          const VT* __restrict__ v, DeflDev dd, int solve,
                                                          const int* done) {
    if (done && *done) return;
    const int k = dd.k;
    double acc[kMaxDefl];
#pragma unroll
    for (int i = 0; i < kMaxDefl; ++i) acc[i] = 0.0;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        const double vj = as_double(v[j]);
#pragma unroll
        for (int i = 0; i < kMaxDefl; ++i)
            if (i < k) acc[i] = fma(as_double(Y[size_t(i) * n + j]), vj, acc[i]);
    }
    __shared__ double sh[kMaxDefl][kDeflBlock / 32];
    __shared__ double tot[kMaxDefl];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kMaxDefl; ++i) {
        if (i >= k) break;
        const double a = warp_sum(acc[i]);
        if (lane == 0) sh[i][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < k) {
        double s = 0.0;
        for (int w = 0; w < kDeflBlock / 32; ++w) s += sh[threadIdx.x][w];
        dd.partial[size_t(threadIdx.x) * kMaxDeflBlocks + blockIdx.x] = s;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(dd.count, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the per-block partials summed by the whole block (fixed order: deterministic)
#pragma unroll
    for (int i = 0; i < kMaxDefl; ++i) acc[i] = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int i = 0; i < kMaxDefl; ++i)
            if (i < k) acc[i] += __ldcg(dd.partial + size_t(i) * kMaxDeflBlocks + b);
    }
#pragma unroll
    for (int i = 0; i < kMaxDefl; ++i) {
        if (i >= k) break;
        const double a = warp_sum(acc[i]);
        if (lane == 0) sh[i][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < k) {
        double s = 0.0;
        for (int w = 0; w < kDeflBlock / 32; ++w) s += sh[threadIdx.x][w];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *dd.count = 0u;
        double c[kMaxDefl];
        for (int i = 0; i < k; ++i) c[i] = tot[i];
        if (solve) {
            for (int i = 0; i < k; ++i) {   // L y = g
                double s = c[i];
                for (int j = 0; j < i; ++j) s -= dd.L[i * k + j] * c[j];
                c[i] = s / dd.L[i * k + i];
            }
            for (int i = k - 1; i >= 0; --i) {   // L^t c = y
                double s = c[i];
                for (int j = i + 1; j < k; ++j) s -= dd.L[j * k + i] * c[j];
                c[i] = s / dd.L[i * k + i];
            }
        }
        for (int i = 0; i < k; ++i) {
            dd.c[i] = c[i];
            dd.cf[i] = float(c[i]);
        }
    }
}

// x += sign * Y c (FP64)
template <typename YT>
__global__ void __launch_bounds__(kDeflBlock) k_defl_axpy(int64_t n, const YT* __restrict__ Y, DeflDev dd,
                                                          double sign, double* __restrict__ x) {
    const int k = dd.k;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s = fma(dd.c[i], as_double(Y[size_t(i) * n + j]), s);
        x[j] = fma(sign, s, x[j]);
    }
}

// p -= V c: FP64 p, or float-float p with the FP32 vectors (the sum in FP32)
__global__ void __launch_bounds__(kDeflBlock) k_defl_project64(int64_t n, const double* __restrict__ V, DeflDev dd,
                                                               double* __restrict__ p, const int* done) {
    if (done && *done) return;
    const int k = dd.k;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s = fma(dd.c[i], V[size_t(i) * n + j], s);
        p[j] -= s;
    }
}

// The float-float form: V is FP32-representable, so V c is formed exactly enough in FP64
// from the FP32 copy (FP64 products and sums) and subtracted from p as a float-float
// pair.  A sum in FP32 does not do: with a mode of r outside span(V) amplified in z by
// the polynomial preconditioner, its rounding feeds components along V back into every
// direction (measured on 64x64 squares: no fewer iterations than without deflation).
__global__ void __launch_bounds__(kDeflBlock) k_defl_projectff(int64_t n, const float* __restrict__ V, DeflDev dd,
                                                               float2* __restrict__ p, const int* done) {
    if (done && *done) return;
    const int k = dd.k;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s = fma(dd.c[i], double(V[size_t(i) * n + j]), s);
        p[j] = ff_add(p[j], ff_from_double(-s));
    }
}

// V rounded to FP32 (in place in FP64, and its FP32 copy)
__global__ void __launch_bounds__(kDeflBlock) k_defl_round(int64_t n, double* __restrict__ v, float* __restrict__ v32) {
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        const float f = __double2float_rn(v[j]);
        v[j] = double(f);
        v32[j] = f;
    }
}

// w = M^{-1} g (FP64)
__global__ void __launch_bounds__(kDeflBlock) k_defl_scale(int64_t n, const double* __restrict__ g,
                                                           const double* __restrict__ minv, double* __restrict__ w) {
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x)
        w[j] = minv[j] * g[j];
}

// q = z / sqrt(rz), z = zin or (zin = null) M^{-1} r; rz read from the device
__global__ void __launch_bounds__(kDeflBlock) k_lanczos_store(int64_t n, const double* __restrict__ zin,
                                                              const double* __restrict__ minv,
                                                              const double* __restrict__ r, const double* rz,
                                                              float* __restrict__ q) {
    const double s = 1.0 / sqrt(*rz);
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        const double z = zin ? zin[j] : minv[j] * r[j];
        q[j] = __double2float_rn(z * s);
    }
}

// Y [k][n] = Q S: Q [m][n] (FP32 Lanczos vectors), S [m][k] (FP32, column l the
// eigenvector of T for Ritz value l).  FP32 products and sums: the vectors are
// rounded to FP32 when the space is built, and the FP64 pipe would bound m k n FMAs.
__global__ void __launch_bounds__(kDeflBlock) k_ritz(int64_t n, int m, int k, const float* __restrict__ Q,
                                                     const float* __restrict__ S, double* __restrict__ Y) {
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        float y[kMaxDefl];
#pragma unroll
        for (int l = 0; l < kMaxDefl; ++l) y[l] = 0.f;
        for (int t = 0; t < m; ++t) {
            const float qv = Q[size_t(t) * n + j];
#pragma unroll
            for (int l = 0; l < kMaxDefl; ++l)
                if (l < k) y[l] = fmaf(qv, __ldg(S + size_t(t) * k + l), y[l]);
        }
#pragma unroll
        for (int l = 0; l < kMaxDefl; ++l)
            if (l < k) Y[size_t(l) * n + j] = double(y[l]);
    }
}

int defl_grid(int64_t n) {
    const int64_t g = (n + kDeflBlock - 1) / kDeflBlock;
    return int(g < 1 ? 1 : (g > kMaxDeflBlocks ? kMaxDeflBlocks : g));
}

// ---- host linear algebra of the small matrices ----------------------------------

}  // namespace

DeflDev cr_deflation_dev(const cr_deflation* d) {
    DeflDev dd;
    dd.k = d->k;
    dd.L = d->L;
    dd.c = d->c;
    dd.cf = d->cf;
    dd.partial = d->partial;
    dd.count = d->count;
    return dd;
}

int defl_dots64(const cr_deflation* d, const double* Y, const double* v, bool solve, const int* done, cudaStream_t st) {
    k_defl_dots<double, double><<<defl_grid(d->n), kDeflBlock, 0, st>>>(d->n, Y, v, cr_deflation_dev(d), solve, done);
    return CR_OK;
}

// c = E^{-1} (G V)^t z for the float-float solves' z (FP32, or float-float pairs):
// G V in FP64, FP64 products (exact for an FP32 z) and sums.  G V rounded to FP32
// would not do: the polynomial preconditioner amplifies the low modes of r in z by
// up to the inverse of their eigenvalue, and when such a mode lies outside span(V)
// the rounding error of (G V)^t z (2^-24 of |G V| |z|) swamps the small true value;
// the projection then feeds components along V back into every direction, which CG
// cannot remove (measured on 64x64 squares: no fewer iterations than without
// deflation, against 320 -> 244 with exact dot products).
int defl_dots64f(const cr_deflation* d, const double* Y, const float* v, const int* done, cudaStream_t st) {
    k_defl_dots<double, float><<<defl_grid(d->n), kDeflBlock, 0, st>>>(d->n, Y, v, cr_deflation_dev(d), 1, done);
    return CR_OK;
}

int defl_dots64ff(const cr_deflation* d, const double* Y, const float2* v, const int* done, cudaStream_t st) {
    k_defl_dots<double, float2><<<defl_grid(d->n), kDeflBlock, 0, st>>>(d->n, Y, v, cr_deflation_dev(d), 1, done);
    return CR_OK;
}

int defl_axpy64(const cr_deflation* d, const double* Y, double sign, double* x, cudaStream_t st) {
    k_defl_axpy<double><<<defl_grid(d->n), kDeflBlock, 0, st>>>(d->n, Y, cr_deflation_dev(d), sign, x);
    return CR_OK;
}

int defl_project64(const cr_deflation* d, double* p, const int* done, cudaStream_t st) {
    k_defl_project64<<<defl_grid(d->n), kDeflBlock, 0, st>>>(d->n, d->V64, cr_deflation_dev(d), p, done);
    return CR_OK;
}

int defl_projectff(const cr_deflation* d, float2* p, const int* done, cudaStream_t st) {
    k_defl_projectff<<<defl_grid(d->n), kDeflBlock, 0, st>>>(d->n, d->V32, cr_deflation_dev(d), p, done);
    return CR_OK;
}

int lanczos_store(int64_t n, const double* z, const double* minv, const double* r, const double* rz, float* q,
                  cudaStream_t st) {
    k_lanczos_store<<<defl_grid(n), kDeflBlock, 0, st>>>(n, z, minv, r, rz, q);
    return CR_OK;
}

int ritz_vectors(int64_t n, int m, int k, const float* Q, const float* S, double* Y, cudaStream_t st) {
    k_ritz<<<defl_grid(n), kDeflBlock, 0, st>>>(n, m, k, Q, S, Y);
    return CR_OK;
}

// Build the space from the k vectors in d->V64 (device, [k][n]) for the G of h:
// V rounded to FP32, G V, M^{-1} G V, E = V^t G V, and the vectors kept greedily
// in order while the Cholesky pivot of E stays above kDeflPivot of its diagonal
// entry (d->k becomes the count).  The pivot over the diagonal entry is the squared
// sine of the G-angle between a vector and the span of those before it: Ritz
// vectors are G-orthogonal (pivots near 1), while the near-copies that the loss of
// orthogonality of Lanczos produces, and dependent vectors, fall far below.  A
// nearly dependent set would make E ill-conditioned, and the float-float solves,
// whose dot products use G V in FP32, would lose their projection to it.
int defl_build(cr_deflation* d, cr_hybrid* h, cudaStream_t st) {
    const int64_t n = d->n;
    const int k = d->k;
    const int g = defl_grid(n);
    for (int i = 0; i < k; ++i) {
        k_defl_round<<<g, kDeflBlock, 0, st>>>(n, d->V64 + size_t(i) * n, d->V32 + size_t(i) * n);
        CR_TRY(launch_spmv64(h, d->V64 + size_t(i) * n, d->GV64 + size_t(i) * n, st));
        k_defl_scale<<<g, kDeflBlock, 0, st>>>(n, d->GV64 + size_t(i) * n, h->minv64, d->W64 + size_t(i) * n);
    }
    CR_CUDA(cudaGetLastError());
    // E column by column: E_ij = V_i . (G V)_j
    std::vector<double> E(size_t(k) * k);
    std::vector<double> col(kMaxDefl);
    for (int j = 0; j < k; ++j) {
        CR_TRY(defl_dots64(d, d->V64, d->GV64 + size_t(j) * n, false, nullptr, st));
        CR_CUDA(cudaMemcpyAsync(col.data(), d->c, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CR_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < k; ++i) E[size_t(i) * k + j] = col[i];
    }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < i; ++j) E[size_t(i) * k + j] = E[size_t(j) * k + i] = 0.5 * (E[size_t(i) * k + j] + E[size_t(j) * k + i]);
    // greedy Cholesky over the vectors in order
    std::vector<int> keep;
    std::vector<double> L;   // row-major over the kept vectors
    for (int i = 0; i < k; ++i) {
        const int r = int(keep.size());
        std::vector<double> row(r + 1, 0.0);
        bool ok = E[size_t(i) * k + i] > 0.0 && std::isfinite(E[size_t(i) * k + i]);
        for (int a = 0; ok && a < r; ++a) {
            double s = E[size_t(i) * k + keep[a]];
            for (int b = 0; b < a; ++b) s -= row[b] * L[size_t(a) * (k) + b];
            row[a] = s / L[size_t(a) * k + a];
        }
        double piv = ok ? E[size_t(i) * k + i] : 0.0;
        for (int a = 0; ok && a < r; ++a) piv -= row[a] * row[a];
        if (!ok || !(piv > kDeflPivot * E[size_t(i) * k + i])) continue;
        row[r] = std::sqrt(piv);
        L.resize(size_t(r + 1) * k, 0.0);
        for (int a = 0; a <= r; ++a) L[size_t(r) * k + a] = row[a];
        keep.push_back(i);
    }
    if (keep.empty()) return fail(CR_ERR_ARG, "deflation: no vector with V^t G V > 0");
    // compact the kept vectors to the front
    for (int a = 0; a < int(keep.size()); ++a) {
        const int i = keep[a];
        if (i == a) continue;
        const size_t dst = size_t(a) * n, src = size_t(i) * n;
        CR_CUDA(cudaMemcpyAsync(d->V64 + dst, d->V64 + src, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        CR_CUDA(cudaMemcpyAsync(d->GV64 + dst, d->GV64 + src, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        CR_CUDA(cudaMemcpyAsync(d->W64 + dst, d->W64 + src, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        CR_CUDA(cudaMemcpyAsync(d->V32 + dst, d->V32 + src, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    }
    const int kk = int(keep.size());
    std::vector<double> Lk(size_t(kk) * kk, 0.0);
    for (int a = 0; a < kk; ++a)
        for (int b = 0; b <= a; ++b) Lk[size_t(a) * kk + b] = L[size_t(a) * k + b];
    d->k = kk;
    d->kept = keep;
    CR_CUDA(cudaMemcpyAsync(d->L, Lk.data(), sizeof(double) * kk * kk, cudaMemcpyHostToDevice, st));
    CR_CUDA(cudaStreamSynchronize(st));
    return CR_OK;
}

// Allocate a space for up to k vectors of the G of h (mesh, nu, mu recorded).
int defl_alloc(cr_hybrid* h, int k, cr_deflation** out) {
    auto* d = new cr_deflation();
    static std::atomic<uint64_t> serial{0};
    d->m = h->m;
    d->dim = h->m->d;
    d->n = h->m->nf * h->m->d;
    d->k = k;
    d->nu = h->s->nu;
    d->mu = h->s->mu;
    d->serial = ++serial;
    const size_t kn = size_t(k) * size_t(d->n);
    int rc;
    if ((rc = d->arena.alloc_n(&d->V64, kn)) || (rc = d->arena.alloc_n(&d->GV64, kn)) ||
        (rc = d->arena.alloc_n(&d->W64, kn)) || (rc = d->arena.alloc_n(&d->V32, kn)) ||
        (rc = d->arena.alloc_n(&d->L, size_t(kMaxDefl) * kMaxDefl)) ||
        (rc = d->arena.alloc_n(&d->c, size_t(kMaxDefl))) || (rc = d->arena.alloc_n(&d->cf, size_t(kMaxDefl))) ||
        (rc = d->arena.alloc_n(&d->partial, size_t(kMaxDefl) * kMaxDeflBlocks)) ||
        (rc = d->arena.alloc_n(&d->count, 1))) {
        d->arena.release();
        delete d;
        return rc;
    }
    cudaError_t e = cudaMemsetAsync(d->count, 0, sizeof(unsigned), h->m->stream);
    if (e != cudaSuccess) {
        d->arena.release();
        delete d;
        return cuda_fail(e, "cudaMemsetAsync");
    }
    *out = d;
    return CR_OK;
}

}  // namespace crhyb
