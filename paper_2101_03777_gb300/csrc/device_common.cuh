// Device helpers shared by the crhyb kernels: deterministic block reductions
// and the per-simplex geometry of the CR scheme.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace crhyb {

constexpr int kBlock = 256;  // threads per block of every reduction kernel

// Sum NV values over the block; thread 0 receives the totals in out[].
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* [NV][32] */, double (&out)[NV]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[k * 32 + warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = lane < nw ? sh[k * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            out[k] = x;
        }
    }
    __syncthreads();
}

// Two-level deterministic reduction.  Every block writes its partial sums;
// the last block to arrive sums all partials in block order and returns true
// (in every thread of that block) with the totals in tot[] (valid in thread 0).
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], RedBuf red, double (&tot)[NV]) {
    __shared__ double sh[NV * 32];
    __shared__ bool last;
    double bs[NV];
    block_sum<NV>(v, sh, bs);
    const int nb = gridDim.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) red.partial[k * kMaxRedBlocks + blockIdx.x] = bs[k];
        __threadfence();
        const unsigned t = atomicAdd(red.count, 1u);
        last = (t == unsigned(nb - 1));
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double a = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) a += __ldcg(red.partial + k * kMaxRedBlocks + b);
        acc[k] = a;
    }
    block_sum<NV>(acc, sh, tot);
    if (threadIdx.x == 0) *red.count = 0u;
    return true;
}

// Geometry of a simplex (Section 2, item 1).  Local face l is opposite local
// vertex l.  a_l = |sigma_l| n_l = -d |K| grad(lambda_l), where lambda_l is
// the barycentric coordinate of vertex l; x_l - x_K = (x_K - X_l)/d.
template <int D>
struct Geom {
    static constexpr int NF = D + 1;
    double vol;
    double a[NF][D];
    double dx[NF][D];   // x_sigma - x_K
};

template <int D>
__device__ __forceinline__ void simplex_geometry(const double* __restrict__ coords, const int32_t* __restrict__ ev,
                                                 Geom<D>& g) {
    constexpr int NF = D + 1;
    double X[NF][D];
#pragma unroll
    for (int l = 0; l < NF; ++l) {
        const int v = __ldg(ev + l);
#pragma unroll
        for (int b = 0; b < D; ++b) X[l][b] = __ldg(coords + size_t(v) * D + b);
    }
    if constexpr (D == 2) {
        const double e1x = X[1][0] - X[0][0], e1y = X[1][1] - X[0][1];
        const double e2x = X[2][0] - X[0][0], e2y = X[2][1] - X[0][1];
        const double det = e1x * e2y - e2x * e1y;
        const double s = det > 0.0 ? 1.0 : -1.0;
        // grad lambda_1 = (e2y, -e2x)/det, grad lambda_2 = (-e1y, e1x)/det; d|K| = |det|
        g.a[1][0] = -s * e2y;
        g.a[1][1] = s * e2x;
        g.a[2][0] = s * e1y;
        g.a[2][1] = -s * e1x;
        g.a[0][0] = -(g.a[1][0] + g.a[2][0]);
        g.a[0][1] = -(g.a[1][1] + g.a[2][1]);
        g.vol = 0.5 * fabs(det);
    } else {
        double e[3][3];
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int b = 0; b < 3; ++b) e[q][b] = X[q + 1][b] - X[0][b];
        // rows of the inverse Jacobian times det: e2 x e3, e3 x e1, e1 x e2
        double c[3][3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double* u = e[(q + 1) % 3];
            const double* w = e[(q + 2) % 3];
            c[q][0] = u[1] * w[2] - u[2] * w[1];
            c[q][1] = u[2] * w[0] - u[0] * w[2];
            c[q][2] = u[0] * w[1] - u[1] * w[0];
        }
        const double det = e[0][0] * c[0][0] + e[0][1] * c[0][1] + e[0][2] * c[0][2];
        const double h = det > 0.0 ? -0.5 : 0.5;   // d|K| = |det|/2
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int b = 0; b < 3; ++b) g.a[q + 1][b] = h * c[q][b];
#pragma unroll
        for (int b = 0; b < 3; ++b) g.a[0][b] = -(g.a[1][b] + g.a[2][b] + g.a[3][b]);
        g.vol = fabs(det) / 6.0;
    }
    double xK[D];
#pragma unroll
    for (int b = 0; b < D; ++b) {
        double t = 0.0;
#pragma unroll
        for (int l = 0; l < NF; ++l) t += X[l][b];
        xK[b] = t / NF;
    }
#pragma unroll
    for (int l = 0; l < NF; ++l)
#pragma unroll
        for (int b = 0; b < D; ++b) g.dx[l][b] = (xK[b] - X[l][b]) / D;
}

}  // namespace crhyb
