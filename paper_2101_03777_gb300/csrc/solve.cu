// Krylov solve of the hybridised system G W = S (hybrid method, step 2).
//
//   * Jacobi-PCG (G symmetric positive definite for mu > 0, b_h = 0,
//     Section 3.2 item 6) in FP64, or in FP32 (FP32 or BF16 matrix values)
//     inside FP64 iterative refinement;
//   * restarted GMRES(m) with right Jacobi preconditioning for the
//     nonsymmetric or indefinite systems (Section 4.3), same precisions;
//   * PCG in FP64 with a Chebyshev polynomial preconditioner (Jacobi-
//     preconditioned Chebyshev steps under a Gershgorin bound of the
//     spectrum), which trades CG iterations, and their reductions, for
//     SpMVs fused with the Chebyshev vector update.
//
// Every scalar of the iteration lives in device memory; the host only reads
// a status record every `check_every` iterations.  Kernels of an iteration
// return at once when the solve has finished, so a chunk of iterations may be
// launched (or replayed as a CUDA graph) without knowing where it stops, and
// the iteration count stays exact.  All dot products are deterministic
// two-level reductions (no floating-point atomics).

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <string>

#include "device_common.cuh"
#include "tridiag.h"
#include "ff.cuh"
#include "persist.h"

namespace crhyb {

// Scalars of a solve, in device memory (mirrored to pinned host memory).
struct KScal {
    double rz, alpha, beta, rr, bb, tol2, pq;   // inner Krylov state
    double orr, obb;                            // FP64 residual of the outer iteration
    double rz_prev;                             // r.M^{-1}r before the last update
    int it, max_it, done, status;
    int conv;                                   // the FP64 true residual met the tolerance
    // GMRES
    double beta0;                               // ||r0|| of the current cycle
    int j;                                      // Arnoldi step within the cycle
    int m;                                      // restart length
    int stop;                                   // the current GMRES cycle has ended
    int pad_;
    float2 alpha_ff, beta_ff;                   // alpha and beta in float-float for the FF iteration
    double sigma;                               // FF vectors hold sigma * (the FP64 quantities)
    double omega, rho_old;                      // BiCGStab
    double cheb[2 * CR_MAX_POLY_DEGREE];        // Chebyshev preconditioner: 1/theta, then (c1_j, c2_j)
    double hb[CR_MAX_RESTART + 1];              // Gram-Schmidt coefficients of the current step
    double H[(CR_MAX_RESTART + 1) * CR_MAX_RESTART];
    double cs[CR_MAX_RESTART], sn[CR_MAX_RESTART], g[CR_MAX_RESTART + 1];
    double y[CR_MAX_RESTART];
};

namespace {

int g_num_sms = 0;

int grid_for(int64_t n) {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    const int64_t want = (n + kBlock - 1) / kBlock;
    const int64_t cap = int64_t(g_num_sms) * 8;   // 8 resident 256-thread blocks per SM
    return int(want < cap ? (want > 0 ? want : 1) : cap);
}

// Grid of a grid-stride kernel over n rows: one row per thread, capped at the
// blocks that all SMs hold at once for this kernel (its occupancy), so that a
// kernel whose registers allow fewer than 8 resident blocks per SM runs in one
// wave instead of a full wave and a partial one.
template <typename K>
int grid_occ(K kernel, int64_t n) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> per_sm_of;
    if (g_num_sms == 0) grid_for(1);
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = per_sm_of.find(reinterpret_cast<const void*>(kernel));
        if (it != per_sm_of.end()) {
            per_sm = it->second;
        } else {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess) {
                cudaGetLastError();
                per_sm = 0;
            }
            if (per_sm <= 0 || per_sm > 8) per_sm = 8;
            per_sm_of[reinterpret_cast<const void*>(kernel)] = per_sm;
        }
    }
    const int64_t want = (n + kBlock - 1) / kBlock;
    const int64_t cap = int64_t(g_num_sms) * per_sm;
    return int(want < cap ? (want > 0 ? want : 1) : cap);
}

// streaming (evict-first) loads of matrix data
__device__ __forceinline__ double ld_val(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_val(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_val(const __nv_bfloat16* p) {
    const unsigned short u = __ldcs(reinterpret_cast<const unsigned short*>(p));
    return __uint_as_float(unsigned(u) << 16);
}

// y_f = sum over the 2d+1 slots of block(slot) * x[col(slot)]  (one face row)
template <int D, typename VT, typename XT, typename AT>
__device__ __forceinline__ void ell_row(int64_t f, const int32_t* __restrict__ cols,
                                        const VT* __restrict__ vals, const XT* __restrict__ x, AT (&y)[D]) {
    constexpr int NS = 2 * D + 1;
#pragma unroll
    for (int i = 0; i < D; ++i) y[i] = AT(0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int64_t c = s == 0 ? f : int64_t(__ldcs(cols + sell(f, s - 1, 2 * D)));
        AT xv[D];
#pragma unroll
        for (int j = 0; j < D; ++j) xv[j] = AT(__ldg(x + c * D + j));
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j)
                y[i] = fma(AT(ld_val(vals + sell(f, (s * D + i) * D + j, NS * D * D))), xv[j], y[i]);
    }
}

// ---------------------------------------------------------------------------
// PCG kernels
// ---------------------------------------------------------------------------

// q = G p, pq = p.q; last block: alpha = rz/pq (breakdown if pq <= 0 or NaN).
template <int D, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_pcg_spmv(int64_t nf, const int32_t* __restrict__ cols,
                                                     const VT* __restrict__ vals, const XT* __restrict__ p,
                                                     XT* __restrict__ q, KScal* sc, RedBuf red) {
    if (sc->done) return;
    double part[1] = {0.0};
    for (int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < nf; f += int64_t(gridDim.x) * blockDim.x) {
        XT y[D];
        ell_row<D, VT, XT, XT>(f, cols, vals, p, y);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            q[f * D + i] = y[i];
            part[0] += double(p[f * D + i]) * double(y[i]);
        }
    }
    double tot[1];
    if (grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        sc->pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else {
            sc->alpha = sc->rz / pq;
        }
    }
}

// x += alpha p, r -= alpha q, rz' = r.M^{-1}r, rr = r.r; last block: beta,
// iteration count, convergence (rr <= tol2) and the iteration limit.
template <int D, typename XT>
__global__ void __launch_bounds__(kBlock) k_pcg_update(int64_t n, XT* __restrict__ x, XT* __restrict__ r,
                                                       const XT* __restrict__ p, const XT* __restrict__ q,
                                                       const XT* __restrict__ minv, KScal* sc, RedBuf red) {
    if (sc->done) return;
    const XT alpha = XT(sc->alpha);
    double part[2] = {0.0, 0.0};
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const XT xn = fma(alpha, p[k], x[k]);
        const XT rn = fma(-alpha, q[k], r[k]);
        x[k] = xn;
        r[k] = rn;
        const double rd = double(rn);
        part[0] += rd * double(minv[k]) * rd;
        part[1] += rd * rd;
    }
    double tot[2];
    if (grid_sum<2>(part, red, tot) && threadIdx.x == 0) {
        const double rz = tot[0];
        sc->rz_prev = sc->rz;
        sc->beta = rz / sc->rz;
        sc->rz = rz;
        sc->rr = tot[1];
        sc->it += 1;
        if (!isfinite(tot[1])) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else if (tot[1] <= sc->tol2) {
            sc->done = 1;
        } else if (sc->it >= sc->max_it) {
            sc->status = CR_ERR_NOT_CONVERGED;
            sc->done = 1;
        }
    }
}

// p = M^{-1} r + beta p   (first: p = M^{-1} r)
template <typename XT>
__global__ void __launch_bounds__(kBlock) k_pcg_dir(int64_t n, XT* __restrict__ p, const XT* __restrict__ r,
                                                    const XT* __restrict__ minv, const KScal* sc, int first) {
    if (sc->done) return;
    const XT beta = XT(first ? 0.0 : sc->beta);
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const XT z = minv[k] * r[k];
        p[k] = first ? z : fma(beta, p[k], z);
    }
}

// ---------------------------------------------------------------------------
// Chebyshev-preconditioned CG (FP64).  The preconditioner z = P(r) is
// `degree` steps of the Chebyshev iteration on M^{-1} G z = M^{-1} r from
// z = 0 over [lmax/ratio, lmax] (Saad, Algorithm 12.1), lmax the Gershgorin
// bound of M^{-1} G.  With theta, delta the interval's centre and half width:
//   d_0 = M^{-1} r / theta,  z_1 = d_0;
//   step j = 1 .. degree-1:  d_j = c1_j d_{j-1} + c2_j M^{-1} (r - G z_j),
//                            z_{j+1} = z_j + d_j,
// with rho_0 = delta/theta, rho_j = 1/(2 theta/delta - rho_{j-1}),
// c1_j = rho_j rho_{j-1}, c2_j = 2 rho_j / delta (host-computed, in KScal).
// The first step is fused into the CG update, every later one into its SpMV
// (z double-buffered: the SpMV gathers z_j while z_{j+1} is written).
// ---------------------------------------------------------------------------

// lmax = max over rows of sum_j |G_ij| / G_ii; the non-negative maximum is
// taken on the bit pattern (integer order = numeric order for doubles >= 0).
template <int D>
__global__ void __launch_bounds__(kBlock) k_gershgorin(int64_t nf, const double* __restrict__ vals,
                                                       const double* __restrict__ minv, unsigned long long* out) {
    constexpr int NS = 2 * D + 1;
    double mx = 0.0;
    for (int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < nf; f += int64_t(gridDim.x) * blockDim.x) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double rs = 0.0;
#pragma unroll
            for (int sl = 0; sl < NS; ++sl)
#pragma unroll
                for (int j = 0; j < D; ++j) rs += fabs(vals[sell(f, (sl * D + i) * D + j, NS * D * D)]);
            mx = fmax(mx, rs * fabs(minv[f * D + i]));
        }
    }
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if (lane == 0) sh[warp] = mx;
    __syncthreads();
    if (warp == 0) {
        mx = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        if (lane == 0) atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(mx)));
    }
}

// z = d = M^{-1} r / theta (the first Chebyshev step)
__global__ void __launch_bounds__(kBlock) k_cheb_start(int64_t n, const double* __restrict__ r,
                                                      const double* __restrict__ minv, double* __restrict__ z,
                                                      double* __restrict__ d, const KScal* sc) {
    if (sc->done) return;
    const double c0 = sc->cheb[0];
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const double v = c0 * minv[k] * r[k];
        z[k] = v;
        d[k] = v;
    }
}

// Chebyshev step j: zout = zin + d_j, d_j = c1_j d + c2_j M^{-1} (r - G zin);
// on the last step r.z and, in the last block, beta = r.z / r.z(previous).
template <int D>
__global__ void __launch_bounds__(kBlock) k_cheb_step(int64_t nf, const int32_t* __restrict__ cols,
                                                     const double* __restrict__ vals, const double* __restrict__ minv,
                                                     const double* __restrict__ r, const double* __restrict__ zin,
                                                     double* __restrict__ zout, double* __restrict__ d, KScal* sc,
                                                     RedBuf red, int j, int last) {
    if (sc->done) return;
    const double c1 = sc->cheb[2 * j - 1], c2 = sc->cheb[2 * j];
    double part[1] = {0.0};
    for (int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < nf; f += int64_t(gridDim.x) * blockDim.x) {
        double y[D];
        ell_row<D, double, double, double>(f, cols, vals, zin, y);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int64_t k = f * D + i;
            const double rk = r[k];
            const double dn = fma(c1, d[k], c2 * minv[k] * (rk - y[i]));
            const double zn = zin[k] + dn;
            d[k] = dn;
            zout[k] = zn;
            part[0] += rk * zn;
        }
    }
    if (!last) return;
    double tot[1];
    if (grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        const double rz = tot[0];
        if (!(rz > 0.0) || !isfinite(rz)) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else {
            sc->rz_prev = sc->rz;
            sc->beta = rz / sc->rz;
            sc->rz = rz;
        }
    }
}

// x += alpha p, r -= alpha q, r.r; then the first Chebyshev step z = d =
// M^{-1} r / theta.  Last block: iteration count, convergence, the limit.
__global__ void __launch_bounds__(kBlock) k_cpcg_update(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                       const double* __restrict__ p, const double* __restrict__ q,
                                                       const double* __restrict__ minv, double* __restrict__ z,
                                                       double* __restrict__ d, KScal* sc, RedBuf red) {
    if (sc->done) return;
    const double alpha = sc->alpha, c0 = sc->cheb[0];
    double part[1] = {0.0};
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        x[k] = fma(alpha, p[k], x[k]);
        const double rn = fma(-alpha, q[k], r[k]);
        r[k] = rn;
        const double v = c0 * minv[k] * rn;
        z[k] = v;
        d[k] = v;
        part[0] += rn * rn;
    }
    double tot[1];
    if (grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        sc->rr = tot[0];
        sc->it += 1;
        if (!isfinite(tot[0])) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else if (tot[0] <= sc->tol2) {
            sc->done = 1;
        } else if (sc->it >= sc->max_it) {
            sc->status = CR_ERR_NOT_CONVERGED;
            sc->done = 1;
        }
    }
}

// p = z + beta p   (first: p = z)
__global__ void __launch_bounds__(kBlock) k_cpcg_dir(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                                                    const KScal* sc, int first) {
    if (sc->done) return;
    const double beta = first ? 0.0 : sc->beta;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        p[k] = first ? z[k] : fma(beta, p[k], z[k]);
}

// r = b - G x in FP64 (x optional: NULL means x = 0), optionally r32 = float(r);
// sums rr, bb, r.M^{-1}r.  Last block:
//   mode 0: outer residual only (orr, obb);
//   mode 1: start of a PCG solve: rz, rr, bb, tol2 = tol^2 bb, done;
//   mode 2: reliable update of the float-float PCG, whose vectors carry the
//           scale sigma (r_ff = sigma r): the new scale makes ||r_ff|| = 1;
//           beta = r.z(true) / r.z(previous, unscaled) continues the search
//           direction (times sigma_new / sigma_old for the rescaled p); the
//           next update is due after a reduction by `delta` or at the target
//           (tol2 = max(delta^2 rr, (tol/2)^2 bb), scaled); conv/done when the
//           true residual meets the tolerance.
//   minv32 (optional) replaces minv in r.M^{-1}r so that it matches the
//   float-float iteration's preconditioner.
template <int D>
__global__ void __launch_bounds__(kBlock) k_residual64(int64_t nf, const int32_t* __restrict__ cols,
                                                       const double* __restrict__ vals, const double* __restrict__ b,
                                                       const double* __restrict__ x, double* __restrict__ r,
                                                       float* __restrict__ r32, const double* __restrict__ minv,
                                                       KScal* sc, RedBuf red, int mode, double tol, double delta,
                                                       const float* __restrict__ minv32 = nullptr) {
    double part[3] = {0.0, 0.0, 0.0};
    for (int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < nf; f += int64_t(gridDim.x) * blockDim.x) {
        double y[D];
        if (x) ell_row<D, double, double, double>(f, cols, vals, x, y);
        else {
#pragma unroll
            for (int i = 0; i < D; ++i) y[i] = 0.0;
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const double bi = b[f * D + i];
            const double ri = bi - y[i];
            if (r) r[f * D + i] = ri;
            if (r32) r32[f * D + i] = __double2float_rn(ri);
            part[0] += ri * ri;
            part[1] += bi * bi;
            part[2] += ri * (minv32 ? double(minv32[f * D + i]) : minv[f * D + i]) * ri;
        }
    }
    double tot[3];
    if (grid_sum<3>(part, red, tot) && threadIdx.x == 0) {
        sc->orr = tot[0];
        sc->obb = tot[1];
        if (mode == 1) {
            sc->rr = tot[0];
            sc->bb = tot[1];
            sc->rz = tot[2];
            sc->tol2 = tol * tol * tot[1];
            sc->status = CR_OK;
            sc->done = (tot[0] <= sc->tol2) ? 1 : 0;
            if (!isfinite(tot[0])) {
                sc->done = 1;
                sc->status = CR_ERR_BREAKDOWN;
            }
        } else if (mode == 3) {
            // reliable update of the Chebyshev float-float PCG: the new scale; r.z of the
            // last direction moved to the new scale's continuation (beta = r.z(new) /
            // (r.z(old) sigma_new / sigma_old) gives p = z + beta_true (sigma_new/sigma_old) p)
            const double rr = tot[0], bb = tot[1];
            const double target = tol * tol * bb;
            const double s_old = sc->sigma > 0.0 ? sc->sigma : 1.0;
            const double s_new = rr > 0.0 && isfinite(rr) ? 1.0 / sqrt(rr) : s_old;
            sc->bb = bb;
            sc->rz = sc->rz * (s_new / s_old);
            sc->rr = rr * s_new * s_new;
            sc->tol2 = fmax(delta * delta * rr, 0.25 * target) * s_new * s_new;
            sc->sigma = s_new;
            sc->conv = (rr <= target) ? 1 : 0;
            sc->done = sc->conv;
            sc->status = CR_OK;
            if (!isfinite(rr)) {
                sc->done = 1;
                sc->status = CR_ERR_BREAKDOWN;
            }
        } else if (mode == 2) {
            const double rr = tot[0], bb = tot[1], rz = tot[2];
            const double target = tol * tol * bb;
            const double s_old = sc->sigma > 0.0 ? sc->sigma : 1.0;
            const double s_new = rr > 0.0 && isfinite(rr) ? 1.0 / sqrt(rr) : s_old;
            const double rz_prev = sc->rz_prev / (s_old * s_old);
            sc->bb = bb;
            sc->beta = rz_prev > 0.0 ? rz / rz_prev * (s_new / s_old) : 0.0;
            sc->beta_ff = ff_from_double(sc->beta);
            sc->rz = rz * s_new * s_new;
            sc->rr = rr * s_new * s_new;
            sc->tol2 = fmax(delta * delta * rr, 0.25 * target) * s_new * s_new;
            sc->sigma = s_new;
            sc->conv = (rr <= target) ? 1 : 0;
            sc->done = sc->conv;
            sc->status = CR_OK;
            if (!isfinite(rr)) {
                sc->done = 1;
                sc->status = CR_ERR_BREAKDOWN;
            }
        }
    }
}

// Inner FP32 solve start for refinement: x = 0, p = M^{-1} r; rz, rr; the
// inner target is ||r_k|| <= inner_tol ||r_0||.
template <typename XT>
__global__ void __launch_bounds__(kBlock) k_inner_start(int64_t n, XT* __restrict__ x, const XT* __restrict__ r,
                                                        XT* __restrict__ p, const XT* __restrict__ minv, KScal* sc,
                                                        RedBuf red, double inner_tol) {
    double part[2] = {0.0, 0.0};
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        x[k] = XT(0);
        const XT z = minv[k] * r[k];
        if (p) p[k] = z;
        part[0] += double(r[k]) * double(z);
        part[1] += double(r[k]) * double(r[k]);
    }
    double tot[2];
    if (grid_sum<2>(part, red, tot) && threadIdx.x == 0) {
        sc->rz = tot[0];
        sc->rr = tot[1];
        sc->bb = tot[1];
        sc->tol2 = inner_tol * inner_tol * tot[1];
        sc->status = CR_OK;
        sc->done = (tot[1] == 0.0) ? 1 : 0;
        if (sc->it >= sc->max_it) {
            sc->done = 1;
            sc->status = CR_ERR_NOT_CONVERGED;
        }
    }
}

// x64 += x32
__global__ void __launch_bounds__(kBlock) k_add32(int64_t n, double* __restrict__ x, const float* __restrict__ d) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        x[k] += double(d[k]);
}

// plain FP64 SpMV (no reduction)
template <int D>
__global__ void __launch_bounds__(kBlock) k_spmv64(int64_t nf, const int32_t* __restrict__ cols,
                                                   const double* __restrict__ vals, const double* __restrict__ x,
                                                   double* __restrict__ y) {
    for (int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < nf; f += int64_t(gridDim.x) * blockDim.x) {
        double v[D];
        ell_row<D, double, double, double>(f, cols, vals, x, v);
#pragma unroll
        for (int i = 0; i < D; ++i) y[f * D + i] = v[i];
    }
}

// ---------------------------------------------------------------------------
// Lanczos record of a PCG solve (cr_solve_ritz): after the direction of
// iteration `it` (sc->it CG steps done, z_it and r_it.z_it = sc->rz in place), the
// normalised preconditioned residual q_it = z_it / sqrt(r_it.z_it) goes to slot it
// of Q (FP32) and the step's alpha_{it-1}, beta_{it-1} to the history.  The
// quantities are those of the scaled float-float vectors where they are scaled (q is
// scale-invariant).  A reliable update rewrites slot it with the z of the true
// residual and the continued beta; a restarted direction (beta = 0) ends the record.
// ---------------------------------------------------------------------------
struct LanczosRec {
    float* Q = nullptr;      // [m][n]
    double* ab = nullptr;    // [2][m]: alpha_j, then beta_j
    int* count = nullptr;    // slots written (q_0 .. q_{count-1})
    int* stop = nullptr;     // set: the record has ended
    int m = 0;
};

__device__ __forceinline__ double rec_val(double v) { return v; }
__device__ __forceinline__ double rec_val(float v) { return double(v); }
__device__ __forceinline__ double rec_val(float2 v) { return double(v.x) + double(v.y); }

template <typename ZT>
__global__ void __launch_bounds__(kBlock) k_lanczos_record(int64_t n, const ZT* __restrict__ z,
                                                           const double* __restrict__ minv,
                                                           const double* __restrict__ r, const KScal* sc,
                                                           LanczosRec rec) {
    if (sc->done || *rec.stop) return;
    const int it = sc->it;
    if (it >= rec.m || !(sc->rz > 0.0)) return;
    const double scale = 1.0 / sqrt(sc->rz);
    float* q = rec.Q + size_t(it) * n;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        const double zj = z ? rec_val(z[j]) : minv[j] * r[j];
        q[j] = __double2float_rn(zj * scale);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (it > 0) {
            rec.ab[it - 1] = sc->alpha;
            rec.ab[rec.m + it - 1] = sc->beta;
        }
        *rec.count = it + 1;
    }
}

// ---------------------------------------------------------------------------
// Float-float PCG kernels.  Vectors are float2 (hi, lo) per unknown; G is the
// FP32 plane val32 (hi) plus a low plane (FP32 or BF16) holding G - hi.
// Dot products are Dot2 sums reduced in float-float through the block and
// across blocks; only the last block converts its totals to FP64.
// ---------------------------------------------------------------------------

// Sum NV float-float values over the grid (two-level, deterministic, like
// grid_sum); the last block returns true with the FP64 totals in thread 0.
template <int NV>
__device__ __forceinline__ bool ff_grid_sum(float2 (&v)[NV], RedBuf red, double (&tot)[NV]) {
    __shared__ float2 sh[NV * 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    auto warp_reduce = [&](float2 a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float2 b;
            b.x = __shfl_down_sync(0xffffffffu, a.x, o);
            b.y = __shfl_down_sync(0xffffffffu, a.y, o);
            a = ff_add(a, b);
        }
        return a;
    };
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const float2 a = warp_reduce(v[k]);
        if (lane == 0) sh[k * 32 + warp] = a;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float2 a = warp_reduce(lane < nw ? sh[k * 32 + lane] : make_float2(0.f, 0.f));
            if (lane == 0) reinterpret_cast<float2*>(red.partial)[k * kMaxRedBlocks + blockIdx.x] = a;
        }
        if (lane == 0) {
            __threadfence();
            const unsigned t = atomicAdd(red.count, 1u);
            last = (t == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    const float2* part = reinterpret_cast<const float2*>(red.partial);
    float2 acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        float2 a = make_float2(0.f, 0.f);
        for (int b = threadIdx.x; b < int(gridDim.x); b += blockDim.x) a = ff_add(a, __ldcg(part + k * kMaxRedBlocks + b));
        acc[k] = warp_reduce(a);
    }
    __syncthreads();   // sh is reused below
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + warp] = acc[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float2 a = warp_reduce(lane < nw ? sh[k * 32 + lane] : make_float2(0.f, 0.f));
            if (lane == 0) tot[k] = ff_to_double(a);
        }
        if (lane == 0) *red.count = 0u;
    }
    return true;
}

// y_f = sum over the 2d+1 slots of block(slot) * x[col(slot)], float-float
template <int D, typename LT>
__device__ __forceinline__ void ff_ell_row(int64_t f, const int32_t* __restrict__ cols,
                                           const float* __restrict__ vh, const LT* __restrict__ vl,
                                           const float2* __restrict__ x, float2 (&y)[D]) {
    constexpr int NS = 2 * D + 1;
    FFAcc acc[D];
#pragma unroll
    for (int i = 0; i < D; ++i) acc[i].zero();
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int64_t c = s == 0 ? f : int64_t(__ldcs(cols + sell(f, s - 1, 2 * D)));
        float2 xv[D];
#pragma unroll
        for (int j = 0; j < D; ++j) xv[j] = __ldg(x + c * D + j);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const size_t idx = sell(f, (s * D + i) * D + j, NS * D * D);
                float h, l;
                hl_val(vh, vl, idx, h, l);
                acc[i].mad(h, l, xv[j].x, xv[j].y);
            }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) y[i] = acc[i].result();
}

// q = G p, pq = p.q; last block: alpha = rz/pq (breakdown if pq <= 0 or NaN).
template <int D, typename LT>
__global__ void __launch_bounds__(kBlock) kf_spmv(int64_t nf, const int32_t* __restrict__ cols,
                                                  const float* __restrict__ vh, const LT* __restrict__ vl,
                                                  const float2* __restrict__ p, float2* __restrict__ q, KScal* sc,
                                                  RedBuf red) {
    if (sc->done) return;
    FFAcc dot;
    dot.zero();
    for (int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < nf; f += int64_t(gridDim.x) * blockDim.x) {
        float2 y[D];
        ff_ell_row<D, LT>(f, cols, vh, vl, p, y);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            q[f * D + i] = y[i];
            const float2 pi = p[f * D + i];
            dot.mad(pi.x, pi.y, y[i].x, y[i].y);
        }
    }
    float2 part[1] = {dot.result()};
    double tot[1];
    if (ff_grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        sc->pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else {
            sc->alpha = sc->rz / pq;
            sc->alpha_ff = ff_from_double(sc->alpha);
        }
    }
}

// x += alpha p, r -= alpha q, rz' = r.M^{-1}r, rr = r.r; last block: beta,
// iteration count, the reliable-update target (rr <= tol2) and the limit.
__global__ void __launch_bounds__(kBlock) kf_update(int64_t n, float2* __restrict__ x, float2* __restrict__ r,
                                                   const float2* __restrict__ p, const float2* __restrict__ q,
                                                   const float* __restrict__ minv, KScal* sc, RedBuf red) {
    if (sc->done) return;
    const float2 alpha = sc->alpha_ff;
    FFAcc rz, rr;
    rz.zero();
    rr.zero();
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const float2 xn = ff_add(x[k], ff_mul(alpha, p[k]));
        const float2 rn = ff_add(r[k], ff_neg(ff_mul(alpha, q[k])));
        x[k] = xn;
        r[k] = rn;
        const float2 z = ff_mul1(minv[k], rn);
        rz.mad(rn.x, rn.y, z.x, z.y);
        rr.mad(rn.x, rn.y, rn.x, rn.y);
    }
    float2 part[2] = {rz.result(), rr.result()};
    double tot[2];
    if (ff_grid_sum<2>(part, red, tot) && threadIdx.x == 0) {
        const double rzn = tot[0];
        sc->rz_prev = sc->rz;
        sc->beta = rzn / sc->rz;
        sc->beta_ff = ff_from_double(sc->beta);
        sc->rz = rzn;
        sc->rr = tot[1];
        sc->it += 1;
        if (!isfinite(tot[1])) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else if (tot[1] <= sc->tol2) {
            sc->done = 1;
        } else if (sc->it >= sc->max_it) {
            sc->status = CR_ERR_NOT_CONVERGED;
            sc->done = 1;
        }
    }
}

// p = M^{-1} r + beta p   (first: p = M^{-1} r)
__global__ void __launch_bounds__(kBlock) kf_dir(int64_t n, float2* __restrict__ p, const float2* __restrict__ r,
                                                const float* __restrict__ minv, const KScal* sc, int first) {
    if (sc->done) return;
    const float2 beta = sc->beta_ff;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const float2 z = ff_mul1(minv[k], r[k]);
        p[k] = first ? z : ff_add(z, ff_mul(beta, p[k]));
    }
}

// ---------------------------------------------------------------------------
// Chebyshev-preconditioned CG in float-float (the FP64 form above with every
// vector and matrix operation on the FP32 pipes; FP64 reliable updates as for
// the Jacobi form).  Vectors carry the scale sigma of the last update.
// ---------------------------------------------------------------------------

// x += alpha p, r -= alpha q, r.r; then the first Chebyshev step z = d = M^{-1} r / theta.
// Last block: iteration count, the reliable-update target (rr <= tol2), the limit.
__global__ void __launch_bounds__(kBlock) kf_cpcg_update(int64_t n, float2* __restrict__ x, float2* __restrict__ r,
                                                        const float2* __restrict__ p, const float2* __restrict__ q,
                                                        const float* __restrict__ minv, float2* __restrict__ z,
                                                        float2* __restrict__ d, KScal* sc, RedBuf red) {
    if (sc->done) return;
    const float2 alpha = sc->alpha_ff;
    const float2 c0 = ff_from_double(sc->cheb[0]);
    FFAcc rr;
    rr.zero();
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        x[k] = ff_add(x[k], ff_mul(alpha, p[k]));
        const float2 rn = ff_add(r[k], ff_neg(ff_mul(alpha, q[k])));
        r[k] = rn;
        const float2 v = ff_mul(c0, ff_mul1(minv[k], rn));
        z[k] = v;
        d[k] = v;
        rr.mad(rn.x, rn.y, rn.x, rn.y);
    }
    float2 part[1] = {rr.result()};
    double tot[1];
    if (ff_grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        sc->rr = tot[0];
        sc->it += 1;
        if (!isfinite(tot[0])) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else if (tot[0] <= sc->tol2) {
            sc->done = 1;
        } else if (sc->it >= sc->max_it) {
            sc->status = CR_ERR_NOT_CONVERGED;
            sc->done = 1;
        }
    }
}

// z = d = M^{-1} r / theta (the first Chebyshev step after a reliable update)
__global__ void __launch_bounds__(kBlock) kf_cheb_start(int64_t n, const float2* __restrict__ r,
                                                       const float* __restrict__ minv, float2* __restrict__ z,
                                                       float2* __restrict__ d, const KScal* sc) {
    if (sc->done) return;
    const float2 c0 = ff_from_double(sc->cheb[0]);
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const float2 v = ff_mul(c0, ff_mul1(minv[k], r[k]));
        z[k] = v;
        d[k] = v;
    }
}

// Chebyshev step j: zout = zin + d_j, d_j = c1_j d + c2_j M^{-1} (r - G zin); on the
// last step r.z and, in the last block, beta = r.z / r.z(previous).
template <int D, typename LT>
__global__ void __launch_bounds__(kBlock) kf_cheb_step(int64_t nf, const int32_t* __restrict__ cols,
                                                      const float* __restrict__ vh, const LT* __restrict__ vl,
                                                      const float* __restrict__ minv, const float2* __restrict__ r,
                                                      const float2* __restrict__ zin, float2* __restrict__ zout,
                                                      float2* __restrict__ d, KScal* sc, RedBuf red, int j, int last) {
    if (sc->done) return;
    const float2 c1 = ff_from_double(sc->cheb[2 * j - 1]), c2 = ff_from_double(sc->cheb[2 * j]);
    FFAcc rz;
    rz.zero();
    for (int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < nf; f += int64_t(gridDim.x) * blockDim.x) {
        float2 y[D];
        ff_ell_row<D, LT>(f, cols, vh, vl, zin, y);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int64_t k = f * D + i;
            const float2 rk = r[k];
            const float2 res = ff_add(rk, ff_neg(y[i]));
            const float2 dn = ff_add(ff_mul(c1, d[k]), ff_mul(c2, ff_mul1(minv[k], res)));
            const float2 zn = ff_add(zin[k], dn);
            d[k] = dn;
            zout[k] = zn;
            rz.mad(rk.x, rk.y, zn.x, zn.y);
        }
    }
    if (!last) return;
    float2 part[1] = {rz.result()};
    double tot[1];
    if (ff_grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        const double rzn = tot[0];
        if (!(rzn > 0.0) || !isfinite(rzn)) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else {
            sc->rz_prev = sc->rz;
            sc->beta = rzn / sc->rz;
            sc->beta_ff = ff_from_double(sc->beta);
            sc->rz = rzn;
        }
    }
}

// p = z + beta p   (first: p = z)
__global__ void __launch_bounds__(kBlock) kf_cpcg_dir(int64_t n, float2* __restrict__ p, const float2* __restrict__ z,
                                                     const KScal* sc, int first) {
    if (sc->done) return;
    const float2 beta = sc->beta_ff;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        p[k] = first ? z[k] : ff_add(z[k], ff_mul(beta, p[k]));
}

// The same preconditioner with its Chebyshev steps in FP32 (FP32 or BF16 values
// of G, FP32 z and d): a fixed polynomial in M^{-1} G~ for the rounded G~, which
// stays positive near 0 and below the Gershgorin bound, so the preconditioner is
// symmetric positive definite; the CG around it stays in float-float.

// x += alpha p, r -= alpha q, r.r (float-float); z = d = M^{-1} r / theta (FP32).
__global__ void __launch_bounds__(kBlock) kf_cpcg_update32(int64_t n, float2* __restrict__ x, float2* __restrict__ r,
                                                          const float2* __restrict__ p, const float2* __restrict__ q,
                                                          const float* __restrict__ minv, float* __restrict__ z,
                                                          float* __restrict__ d, KScal* sc, RedBuf red) {
    if (sc->done) return;
    const float2 alpha = sc->alpha_ff;
    const float c0 = float(sc->cheb[0]);
    FFAcc rr;
    rr.zero();
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        x[k] = ff_add(x[k], ff_mul(alpha, p[k]));
        const float2 rn = ff_add(r[k], ff_neg(ff_mul(alpha, q[k])));
        r[k] = rn;
        const float v = c0 * minv[k] * (rn.x + rn.y);
        z[k] = v;
        d[k] = v;
        rr.mad(rn.x, rn.y, rn.x, rn.y);
    }
    float2 part[1] = {rr.result()};
    double tot[1];
    if (ff_grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        sc->rr = tot[0];
        sc->it += 1;
        if (!isfinite(tot[0])) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else if (tot[0] <= sc->tol2) {
            sc->done = 1;
        } else if (sc->it >= sc->max_it) {
            sc->status = CR_ERR_NOT_CONVERGED;
            sc->done = 1;
        }
    }
}

__global__ void __launch_bounds__(kBlock) kf_cheb_start32(int64_t n, const float2* __restrict__ r,
                                                         const float* __restrict__ minv, float* __restrict__ z,
                                                         float* __restrict__ d, const KScal* sc) {
    if (sc->done) return;
    const float c0 = float(sc->cheb[0]);
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const float v = c0 * minv[k] * (r[k].x + r[k].y);
        z[k] = v;
        d[k] = v;
    }
}

// Chebyshev step j in FP32 on the FP32 (or BF16) values of G; the last step forms
// r.z in float-float and beta = r.z / r.z(previous).
template <int D, typename VT>
__global__ void __launch_bounds__(kBlock) k32_cheb_step(int64_t nf, const int32_t* __restrict__ cols,
                                                       const VT* __restrict__ vals, const float* __restrict__ minv,
                                                       const float2* __restrict__ r, const float* __restrict__ zin,
                                                       float* __restrict__ zout, float* __restrict__ d, KScal* sc,
                                                       RedBuf red, int j, int last) {
    if (sc->done) return;
    const float c1 = float(sc->cheb[2 * j - 1]), c2 = float(sc->cheb[2 * j]);
    FFAcc rz;
    rz.zero();
    for (int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < nf; f += int64_t(gridDim.x) * blockDim.x) {
        float y[D];
        ell_row<D, VT, float, float>(f, cols, vals, zin, y);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int64_t k = f * D + i;
            const float2 rk = r[k];
            const float dn = fmaf(c1, d[k], c2 * minv[k] * ((rk.x + rk.y) - y[i]));
            const float zn = zin[k] + dn;
            d[k] = dn;
            zout[k] = zn;
            if (last) rz.mad(rk.x, rk.y, zn, 0.f);
        }
    }
    if (!last) return;
    float2 part[1] = {rz.result()};
    double tot[1];
    if (ff_grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        const double rzn = tot[0];
        if (!(rzn > 0.0) || !isfinite(rzn)) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else {
            sc->rz_prev = sc->rz;
            sc->beta = rzn / sc->rz;
            sc->beta_ff = ff_from_double(sc->beta);
            sc->rz = rzn;
        }
    }
}

// ---- the FP32-step Chebyshev kernel, two rows per thread ----
//
// Every thread takes two adjacent rows: two independent gather chains, and one
// load instruction for the values (and for the columns) of both rows, which are
// adjacent in every plane of the sliced ELL.

// values of rows f and f+1 (f even) of one plane, as FP32
__device__ __forceinline__ float2 ld_val2(const float* p) { return __ldcs(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ float2 ld_val2(const __nv_bfloat16* p) {
    const unsigned u = __ldcs(reinterpret_cast<const unsigned*>(p));
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

// The Chebyshev step of k32_cheb_step on rows (2t, 2t+1) per thread.  The rows
// of the last slice beyond nf hold zero values and column 0 (in bounds); their
// vectors are neither read nor written.
template <int D, typename VT>
__global__ void __launch_bounds__(kBlock) k32_cheb_step2(int64_t nf, const int32_t* __restrict__ cols,
                                                        const VT* __restrict__ vals, const float* __restrict__ minv,
                                                        const float2* __restrict__ r, const float* __restrict__ zin,
                                                        float* __restrict__ zout, float* __restrict__ d, KScal* sc,
                                                        RedBuf red, int j, int last) {
    if (sc->done) return;
    constexpr int NS = 2 * D + 1, NPL = NS * D * D;
    const float c1 = float(sc->cheb[2 * j - 1]), c2 = float(sc->cheb[2 * j]);
    FFAcc rz;
    rz.zero();
    const int64_t npair = (nf + 1) / 2;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < npair; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t f0 = 2 * t;
        const bool two = f0 + 1 < nf;
        float y0[D], y1[D];
#pragma unroll
        for (int i = 0; i < D; ++i) y0[i] = y1[i] = 0.f;
#pragma unroll
        for (int sl = 0; sl < NS; ++sl) {
            int64_t c0 = f0, cb = f0 + 1;
            if (sl > 0) {
                const int2 cc = __ldcs(reinterpret_cast<const int2*>(cols + sell(f0, sl - 1, 2 * D)));
                c0 = cc.x;
                cb = cc.y;
            }
            if (!two) cb = c0;   // the padding row: any in-bounds column, its values are 0
            float x0[D], x1[D];
#pragma unroll
            for (int jj = 0; jj < D; ++jj) {
                x0[jj] = __ldg(zin + c0 * D + jj);
                x1[jj] = __ldg(zin + cb * D + jj);
            }
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int jj = 0; jj < D; ++jj) {
                    const float2 v = ld_val2(vals + sell(f0, (sl * D + i) * D + jj, NPL));
                    y0[i] = fmaf(v.x, x0[jj], y0[i]);
                    y1[i] = fmaf(v.y, x1[jj], y1[i]);
                }
        }
#pragma unroll
        for (int row = 0; row < 2; ++row) {
            if (row == 1 && !two) break;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const int64_t k = (f0 + row) * D + i;
                const float2 rk = r[k];
                const float yi = row == 0 ? y0[i] : y1[i];
                const float dn = fmaf(c1, d[k], c2 * minv[k] * ((rk.x + rk.y) - yi));
                const float zn = zin[k] + dn;
                d[k] = dn;
                zout[k] = zn;
                if (last) rz.mad(rk.x, rk.y, zn, 0.f);
            }
        }
    }
    if (!last) return;
    float2 part[1] = {rz.result()};
    double tot[1];
    if (ff_grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        const double rzn = tot[0];
        if (!(rzn > 0.0) || !isfinite(rzn)) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else {
            sc->rz_prev = sc->rz;
            sc->beta = rzn / sc->rz;
            sc->beta_ff = ff_from_double(sc->beta);
            sc->rz = rzn;
        }
    }
}

// ---- the FP32-step Chebyshev kernel on slices staged in shared memory ----
//
// Every block takes whole slices of the sliced ELL (256 rows, one row per
// thread) and has the TMA engine copy the slice's values and
// columns (one contiguous run each) into shared memory with cp.async.bulk,
// completion counted in bytes on one mbarrier.  The rows' own vector entries
// are loaded while the copy runs; only the gathers of z at the neighbours stay
// per-thread global loads.  A slice of an array starts at a multiple of 256 rows
// times 2-8 bytes per entry, so both copies are 16-byte aligned and a multiple of
// 16 bytes long; the last slice is copied whole (its rows beyond nf are zero).
constexpr long long kStageWaitLimit = 1ll << 22;   // bounded mbarrier waits

template <int D, typename VT>
struct ChebStage {
    static constexpr int NPL = (2 * D + 1) * D * D, NC = 2 * D;
    static constexpr uint32_t VB = uint32_t(NPL) * kSlice * sizeof(VT);   // bytes of a slice's values
    static constexpr uint32_t CB = uint32_t(NC) * kSlice * 4;             // bytes of its columns
    static constexpr uint32_t SMEM = VB + CB + 16;                        // + the mbarrier
    static_assert(VB % 16 == 0 && CB % 16 == 0, "bulk copies are whole 16-byte units");
};

__device__ __forceinline__ uint32_t cta_smem(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ bool stage_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(cta_smem(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool stage_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (long long n = 0; n < kStageWaitLimit; ++n)
        if (stage_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ float smem_val(const float* p) { return *p; }
__device__ __forceinline__ float smem_val(const __nv_bfloat16* p) { return __bfloat162float(*p); }

template <int D, typename VT>
__global__ void __launch_bounds__(kBlock) k32_cheb_step_staged(int64_t nf, const int32_t* __restrict__ cols,
                                                              const VT* __restrict__ vals,
                                                              const float* __restrict__ minv,
                                                              const float2* __restrict__ r,
                                                              const float* __restrict__ zin, float* __restrict__ zout,
                                                              float* __restrict__ d, KScal* sc, RedBuf red, int j,
                                                              int last) {
    static_assert(kBlock == kSlice, "one row of the slice per thread");
    if (sc->done) return;
    using G = ChebStage<D, VT>;
    constexpr int NS = 2 * D + 1;
    extern __shared__ __align__(128) unsigned char stage[];
    const VT* sv = reinterpret_cast<const VT*>(stage);
    const int32_t* scol = reinterpret_cast<const int32_t*>(stage + G::VB);
    uint64_t* bar = reinterpret_cast<uint64_t*>(stage + G::VB + G::CB);
    const int tid = threadIdx.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cta_smem(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const float c1 = float(sc->cheb[2 * j - 1]), c2 = float(sc->cheb[2 * j]);
    FFAcc rz;
    rz.zero();
    const int64_t nsl = (nf + kSlice - 1) / kSlice;
    uint32_t parity = 0;
    for (int64_t sl = blockIdx.x; sl < nsl; sl += gridDim.x) {
        if (tid == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cta_smem(bar)),
                         "r"(G::VB + G::CB)
                         : "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads before the new writes
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                             "r"(cta_smem(stage)),
                         "l"(vals + size_t(sl) * G::NPL * kSlice), "r"(G::VB), "r"(cta_smem(bar))
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                             "r"(cta_smem(stage + G::VB)),
                         "l"(cols + size_t(sl) * G::NC * kSlice), "r"(G::CB), "r"(cta_smem(bar))
                         : "memory");
        }
        const int64_t f = sl * kSlice + tid;
        const bool act = f < nf;
        float2 rk[D];
        float mk[D], dk[D], zk[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int64_t k = act ? f * D + i : 0;
            rk[i] = r[k];
            mk[i] = minv[k];
            dk[i] = d[k];
            zk[i] = zin[k];
        }
        const bool ok = stage_wait_bounded(bar, parity);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            // the copies never completed: wait (bounded) once more so that none is
            // left in flight, report the time-out and leave the sweep
            if (tid == 0) {
                stage_wait_bounded(bar, parity ^ 1u);
                sc->status = CR_ERR_TIMEOUT;
                sc->done = 1;
            }
            break;
        }
        if (act) {
            float y[D];
#pragma unroll
            for (int i = 0; i < D; ++i) y[i] = 0.f;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int64_t c = s == 0 ? f : int64_t(scol[(s - 1) * kSlice + tid]);
                float xv[D];
#pragma unroll
                for (int jj = 0; jj < D; ++jj) xv[jj] = __ldg(zin + c * D + jj);
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int jj = 0; jj < D; ++jj)
                        y[i] = fmaf(smem_val(sv + ((s * D + i) * D + jj) * kSlice + tid), xv[jj], y[i]);
            }
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const int64_t k = f * D + i;
                const float dn = fmaf(c1, dk[i], c2 * mk[i] * ((rk[i].x + rk[i].y) - y[i]));
                const float zn = zk[i] + dn;
                d[k] = dn;
                zout[k] = zn;
                if (last) rz.mad(rk[i].x, rk[i].y, zn, 0.f);
            }
        }
        __syncthreads();   // every read of this slice ends before the next copy overwrites it
    }
    if (!last) return;
    float2 part[1] = {rz.result()};
    double tot[1];
    if (ff_grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        const double rzn = tot[0];
        if (sc->status == CR_ERR_TIMEOUT) return;
        if (!(rzn > 0.0) || !isfinite(rzn)) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else {
            sc->rz_prev = sc->rz;
            sc->beta = rzn / sc->rz;
            sc->beta_ff = ff_from_double(sc->beta);
            sc->rz = rzn;
        }
    }
}

// Grid of the staged kernel: resident blocks per SM (shared memory and registers)
// x SMs, at most one block per slice; the first call per instantiation raises the
// kernel's dynamic shared-memory limit (it runs before any graph capture).
template <int D, typename VT>
int staged_grid(int64_t nf) {
    static std::once_flag once;
    static int per_sm = 1;
    std::call_once(once, [] {
        auto kern = k32_cheb_step_staged<D, VT>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ChebStage<D, VT>::SMEM)) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, ChebStage<D, VT>::SMEM) !=
                cudaSuccess) {
            cudaGetLastError();
            per_sm = 1;
        }
        if (per_sm <= 0) per_sm = 1;
        if (per_sm > 8) per_sm = 8;
    });
    if (g_num_sms == 0) grid_for(1);
    const int64_t want = (nf + kSlice - 1) / kSlice, cap = int64_t(g_num_sms) * per_sm;
    return int(want < cap ? (want > 0 ? want : 1) : cap);
}

// Which form of the FP32 Chebyshev step runs: 2 staged, 1 two rows per thread,
// 0 one row per thread.  Defaults, from timing each form on GB300 (2D 512^2 and
// 3D 64^3 meshes): staged for BF16 values (its slice, 32 KB in 3D, leaves five
// blocks per SM); for FP32 values, whose slice leaves three, two rows per thread
// in 3D and one in 2D.  The environment variable CRHYB_CHEB_KERNEL (staged,
// rows2, rows1) overrides the default for a process.
int cheb32_form(int d, bool bf16) {
    static const int forced = [] {
        const char* e = std::getenv("CRHYB_CHEB_KERNEL");
        if (e && !std::strcmp(e, "staged")) return 2;
        if (e && !std::strcmp(e, "rows2")) return 1;
        if (e && !std::strcmp(e, "rows1")) return 0;
        return -1;
    }();
    if (forced >= 0) return forced;
    return bf16 ? 2 : (d == 3 ? 1 : 0);
}

// One FP32 Chebyshev step on FP32 or BF16 values, in the form cheb32_form() names.
template <int D, typename VT>
void launch_cheb32(int64_t nf, const int32_t* cols, const VT* vals, const float* minv, const float2* r,
                   const float* zin, float* zout, float* d, KScal* sc, RedBuf red, int j, int last, cudaStream_t st) {
    const int form = cheb32_form(D, std::is_same<VT, __nv_bfloat16>::value);
    if (form == 2) {
        // the dynamic shared-memory limit is a per-device attribute: raise it on every GPU
        // this thread launches on (the first launch on a device is never inside a capture)
        static thread_local int raised_on = -1;
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && dev != raised_on &&
            cudaFuncSetAttribute(k32_cheb_step_staged<D, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(ChebStage<D, VT>::SMEM)) == cudaSuccess)
            raised_on = dev;
    }
    if (form == 2)
        k32_cheb_step_staged<D, VT><<<staged_grid<D, VT>(nf), kBlock, ChebStage<D, VT>::SMEM, st>>>(
            nf, cols, vals, minv, r, zin, zout, d, sc, red, j, last);
    else if (form == 1)
        k32_cheb_step2<D, VT><<<grid_occ(k32_cheb_step2<D, VT>, (nf + 1) / 2), kBlock, 0, st>>>(
            nf, cols, vals, minv, r, zin, zout, d, sc, red, j, last);
    else
        k32_cheb_step<D, VT><<<grid_occ(k32_cheb_step<D, VT>, nf), kBlock, 0, st>>>(nf, cols, vals, minv, r, zin, zout,
                                                                                   d, sc, red, j, last);
}

// p = z + beta p (float-float p, FP32 z)
__global__ void __launch_bounds__(kBlock) kf_cpcg_dir32(int64_t n, float2* __restrict__ p, const float* __restrict__ z,
                                                       const KScal* sc, int first) {
    if (sc->done) return;
    const float2 beta = sc->beta_ff;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const float2 zk = make_float2(z[k], 0.f);
        p[k] = first ? zk : ff_add(zk, ff_mul(beta, p[k]));
    }
}

// x64 += x_ff / sigma; x_ff = 0   (the reliable update of the iterate)
__global__ void __launch_bounds__(kBlock) k_add_ff(int64_t n, double* __restrict__ x, float2* __restrict__ d,
                                                  const KScal* sc) {
    const double inv = 1.0 / sc->sigma;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        x[k] += ff_to_double(d[k]) * inv;
        d[k] = make_float2(0.f, 0.f);
    }
}

// r_ff = sigma r64 in float-float (after a reliable update set sigma)
__global__ void __launch_bounds__(kBlock) k_ff_from64(int64_t n, const double* __restrict__ r, float2* __restrict__ rf,
                                                     const KScal* sc) {
    const double s = sc->sigma;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        rf[k] = ff_from_double(r[k] * s);
}

// ---------------------------------------------------------------------------
// BiCGStab (van der Vorst 1992) with right Jacobi preconditioning, FP64:
//   rho = rh.r, beta = (rho/rho_old)(alpha/omega), p = r + beta (p - omega v),
//   y = M^{-1} p, v = G y, alpha = rho / rh.v, s = r - alpha v, z = M^{-1} s,
//   t = G z, omega = t.s / t.t, x += alpha y + omega z, r = s - omega t.
// ---------------------------------------------------------------------------

// rh = r (the shadow residual), p = v = 0; rho = r.r, rho_old = alpha = omega = 1.
__global__ void __launch_bounds__(kBlock) k_bs_init(int64_t n, const double* __restrict__ r, double* __restrict__ rh,
                                                   double* __restrict__ p, double* __restrict__ v, KScal* sc,
                                                   RedBuf red) {
    double part[1] = {0.0};
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const double rk = r[k];
        rh[k] = rk;
        p[k] = 0.0;
        v[k] = 0.0;
        part[0] += rk * rk;
    }
    double tot[1];
    if (grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        sc->rz = tot[0];
        sc->rho_old = 1.0;
        sc->alpha = 1.0;
        sc->omega = 1.0;
    }
}

// p = r + beta (p - omega v), y = M^{-1} p
__global__ void __launch_bounds__(kBlock) k_bs_dir(int64_t n, const double* __restrict__ r, double* __restrict__ p,
                                                  const double* __restrict__ v, const double* __restrict__ minv,
                                                  double* __restrict__ y, const KScal* sc) {
    if (sc->done) return;
    const double omega = sc->omega, beta = (sc->rz / sc->rho_old) * (sc->alpha / omega);
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const double pk = fma(beta, p[k] - omega * v[k], r[k]);
        p[k] = pk;
        y[k] = minv[k] * pk;
    }
}

// out = G in and its dot products.  which = 0: rh.out -> alpha = rho / rh.out;
// which = 1: out.s and out.out -> omega = out.s / out.out.
template <int D>
__global__ void __launch_bounds__(kBlock) k_bs_spmv(int64_t nf, const int32_t* __restrict__ cols,
                                                   const double* __restrict__ vals, const double* __restrict__ in,
                                                   double* __restrict__ out, const double* __restrict__ w,
                                                   KScal* sc, RedBuf red, int which) {
    if (sc->done) return;
    double part[2] = {0.0, 0.0};
    for (int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < nf; f += int64_t(gridDim.x) * blockDim.x) {
        double y[D];
        ell_row<D, double, double, double>(f, cols, vals, in, y);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            out[f * D + i] = y[i];
            part[0] += w[f * D + i] * y[i];
            part[1] += y[i] * y[i];
        }
    }
    double tot[2];
    if (grid_sum<2>(part, red, tot) && threadIdx.x == 0) {
        if (which == 0) {
            if (!(tot[0] != 0.0) || !isfinite(tot[0])) {
                sc->status = CR_ERR_BREAKDOWN;
                sc->done = 1;
            } else {
                sc->alpha = sc->rz / tot[0];
            }
        } else {
            sc->omega = tot[1] > 0.0 ? tot[0] / tot[1] : 0.0;
            if (!isfinite(sc->omega)) {
                sc->status = CR_ERR_BREAKDOWN;
                sc->done = 1;
            }
        }
    }
}

// s = r - alpha v, z = M^{-1} s
__global__ void __launch_bounds__(kBlock) k_bs_s(int64_t n, const double* __restrict__ r, const double* __restrict__ v,
                                                const double* __restrict__ minv, double* __restrict__ sv,
                                                double* __restrict__ z, const KScal* sc) {
    if (sc->done) return;
    const double alpha = sc->alpha;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const double s = fma(-alpha, v[k], r[k]);
        sv[k] = s;
        z[k] = minv[k] * s;
    }
}

// x += alpha y + omega z, r = s - omega t; rho' = rh.r, r.r; last block: the
// iteration count, convergence, the limit, and breakdown (rho' or omega zero).
__global__ void __launch_bounds__(kBlock) k_bs_update(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                     const double* __restrict__ y, const double* __restrict__ z,
                                                     const double* __restrict__ sv, const double* __restrict__ t,
                                                     const double* __restrict__ rh, KScal* sc, RedBuf red) {
    if (sc->done) return;
    const double alpha = sc->alpha, omega = sc->omega;
    double part[2] = {0.0, 0.0};
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        x[k] = fma(omega, z[k], fma(alpha, y[k], x[k]));
        const double rk = fma(-omega, t[k], sv[k]);
        r[k] = rk;
        part[0] += rh[k] * rk;
        part[1] += rk * rk;
    }
    double tot[2];
    if (grid_sum<2>(part, red, tot) && threadIdx.x == 0) {
        sc->rho_old = sc->rz;
        sc->rz = tot[0];
        sc->rr = tot[1];
        sc->it += 1;
        if (!isfinite(tot[1])) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        } else if (tot[1] <= sc->tol2) {
            sc->done = 1;
        } else if (sc->it >= sc->max_it) {
            sc->status = CR_ERR_NOT_CONVERGED;
            sc->done = 1;
        } else if (!(tot[0] != 0.0) || !(sc->omega != 0.0)) {
            sc->status = CR_ERR_BREAKDOWN;
            sc->done = 1;
        }
    }
}

// ---------------------------------------------------------------------------
// GMRES(m) kernels: Arnoldi with classical Gram-Schmidt applied twice (CGS2),
// right Jacobi preconditioning: G M^{-1} z_j, x = x0 + M^{-1} V y.
// ---------------------------------------------------------------------------

// V_0 = r / ||r||; beta0 = ||r||, g = (beta0, 0, ...), j = 0.  r holds r0.
template <typename XT>
__global__ void __launch_bounds__(kBlock) k_gm_norm_start(int64_t n, const XT* __restrict__ r, KScal* sc,
                                                          RedBuf red) {
    if (sc->done) return;
    double part[1] = {0.0};
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        part[0] += double(r[k]) * double(r[k]);
    double tot[1];
    if (grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        const double b = sqrt(tot[0]);
        sc->beta0 = b;
        sc->g[0] = b;
        sc->j = 0;
        sc->stop = 0;
        sc->rr = tot[0];
        if (!isfinite(b)) { sc->status = CR_ERR_BREAKDOWN; sc->done = 1; }
        else if (tot[0] <= sc->tol2) sc->done = 1;
        else if (sc->it >= sc->max_it) { sc->status = CR_ERR_NOT_CONVERGED; sc->done = 1; }
    }
}

template <typename XT>
__global__ void __launch_bounds__(kBlock) k_gm_scale_v0(int64_t n, const XT* __restrict__ r, XT* __restrict__ V,
                                                        const KScal* sc) {
    if (sc->done) return;
    const double inv = 1.0 / sc->beta0;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        V[k] = XT(double(r[k]) * inv);
}

// w = G (M^{-1} V_j) into V_{j+1} (unnormalised)
template <int D, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_gm_precond(int64_t n, const XT* __restrict__ V, const XT* __restrict__ minv,
                                                       XT* __restrict__ z, const KScal* sc) {
    if (sc->done || sc->stop) return;
    const XT* vj = V + size_t(sc->j) * n;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        z[k] = minv[k] * vj[k];
}

template <int D, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_gm_spmv(int64_t nf, const int32_t* __restrict__ cols,
                                                    const VT* __restrict__ vals, const XT* __restrict__ z,
                                                    XT* __restrict__ V, const KScal* sc) {
    if (sc->done || sc->stop) return;
    XT* w = V + size_t(sc->j + 1) * nf * D;
    for (int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < nf; f += int64_t(gridDim.x) * blockDim.x) {
        XT y[D];
        ell_row<D, VT, XT, XT>(f, cols, vals, z, y);
#pragma unroll
        for (int i = 0; i < D; ++i) w[f * D + i] = y[i];
    }
}

// h_i = V_i . w for i = 0..j (one pass over w and V_0..V_j); `pass` 0 or 1 (CGS2).
// The (j+1) dots go through the partial buffer in groups of kRedSlots.
template <typename XT>
__global__ void __launch_bounds__(kBlock) k_gm_dots(int64_t n, const XT* __restrict__ V, int i0, KScal* sc,
                                                    RedBuf red) {
    if (sc->done || sc->stop) return;
    const int j = sc->j;
    if (i0 > j) return;
    const XT* w = V + size_t(j + 1) * n;
    double part[kRedSlots] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const double wk = double(w[k]);
#pragma unroll
        for (int t = 0; t < kRedSlots; ++t)
            if (i0 + t <= j) part[t] += double(V[size_t(i0 + t) * n + k]) * wk;
    }
    double tot[kRedSlots];
    if (grid_sum<kRedSlots>(part, red, tot) && threadIdx.x == 0) {
#pragma unroll
        for (int t = 0; t < kRedSlots; ++t)
            if (i0 + t <= j) sc->hb[i0 + t] = tot[t];
    }
}

// w -= sum_i h_i V_i; accumulate h into H(:, j); ||w||^2 on the second pass.
template <typename XT>
__global__ void __launch_bounds__(kBlock) k_gm_orth(int64_t n, XT* __restrict__ V, KScal* sc, RedBuf red, int pass) {
    if (sc->done || sc->stop) return;
    const int j = sc->j;
    XT* w = V + size_t(j + 1) * n;
    double part[1] = {0.0};
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        double wk = double(w[k]);
        for (int i = 0; i <= j; ++i) wk -= sc->hb[i] * double(V[size_t(i) * n + k]);
        w[k] = XT(wk);
        part[0] += wk * wk;
    }
    double tot[1];
    if (grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        const int m = sc->m;
        for (int i = 0; i <= j; ++i) sc->H[i * m + j] = (pass == 0 ? 0.0 : sc->H[i * m + j]) + sc->hb[i];
        if (pass == 1) {
            // H(j+1, j) = ||w||; Givens rotations; residual estimate |g_{j+1}|
            const double hn = sqrt(tot[0]);
            sc->H[(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {
                const double a = sc->H[i * m + j], b = sc->H[(i + 1) * m + j];
                sc->H[i * m + j] = sc->cs[i] * a + sc->sn[i] * b;
                sc->H[(i + 1) * m + j] = -sc->sn[i] * a + sc->cs[i] * b;
            }
            const double a = sc->H[j * m + j], b = sc->H[(j + 1) * m + j];
            const double den = hypot(a, b);
            const double c = den > 0.0 ? a / den : 1.0, s = den > 0.0 ? b / den : 0.0;
            sc->cs[j] = c;
            sc->sn[j] = s;
            sc->H[j * m + j] = den;
            sc->H[(j + 1) * m + j] = 0.0;
            sc->g[j + 1] = -s * sc->g[j];
            sc->g[j] = c * sc->g[j];
            sc->it += 1;
            sc->rr = sc->g[j + 1] * sc->g[j + 1];
            sc->j = j + 1;
            sc->pq = hn;   // ||w|| before normalisation
            if (!isfinite(hn) || !(den > 0.0)) { sc->status = CR_ERR_BREAKDOWN; sc->done = 1; }
            if (sc->rr <= sc->tol2 || sc->it >= sc->max_it || j + 1 == m) sc->stop = 1;
        }
    }
}

// V_{j} /= H(j, j-1) (j already advanced); skipped on a happy breakdown.
template <typename XT>
__global__ void __launch_bounds__(kBlock) k_gm_normalise(int64_t n, XT* __restrict__ V, const KScal* sc) {
    if (sc->done || sc->stop) return;   // the last vector of a cycle is never used
    const double hn = sc->pq;
    if (!(hn > 0.0)) return;
    XT* w = V + size_t(sc->j) * n;
    const double inv = 1.0 / hn;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        w[k] = XT(double(w[k]) * inv);
}

// Back substitution H y = g (upper triangular, size j) by one thread.
__global__ void k_gm_solve_y(KScal* sc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (sc->status != CR_OK) { sc->j = 0; return; }
    const int k = sc->j, m = sc->m;
    for (int i = k - 1; i >= 0; --i) {
        double s = sc->g[i];
        for (int t = i + 1; t < k; ++t) s -= sc->H[i * m + t] * sc->y[t];
        sc->y[i] = s / sc->H[i * m + i];
    }
}

// x += M^{-1} V y
template <typename XT>
__global__ void __launch_bounds__(kBlock) k_gm_update(int64_t n, XT* __restrict__ x, const XT* __restrict__ V,
                                                      const XT* __restrict__ minv, const KScal* sc) {
    const int k = sc->j;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += sc->y[i] * double(V[size_t(i) * n + q]);
        x[q] = XT(double(x[q]) + double(minv[q]) * s);
    }
}

// x += Z y (flexible GMRES: the preconditioned vectors are stored)
__global__ void __launch_bounds__(kBlock) k_fgm_update(int64_t n, double* __restrict__ x, const double* __restrict__ Z,
                                                       const KScal* sc) {
    const int k = sc->j;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += sc->y[i] * Z[size_t(i) * n + q];
        x[q] += s;
    }
}

// r = b - G x in the working precision (for GMRES restarts)
template <int D, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_residual_w(int64_t nf, const int32_t* __restrict__ cols,
                                                       const VT* __restrict__ vals, const XT* __restrict__ b,
                                                       const XT* __restrict__ x, XT* __restrict__ r, const KScal* sc) {
    if (sc->done) return;
    for (int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < nf; f += int64_t(gridDim.x) * blockDim.x) {
        XT y[D];
        ell_row<D, VT, XT, XT>(f, cols, vals, x, y);
#pragma unroll
        for (int i = 0; i < D; ++i) r[f * D + i] = b[f * D + i] - y[i];
    }
}

// ---------------------------------------------------------------------------
// Steady problems: flexible GMRES on the coupled system, preconditioned by
// transient hybridised solves (cr_solve_steady)
// ---------------------------------------------------------------------------

// up = v / (mu m): the previous level whose lumped mass term mu m up is the
// velocity block v of an Arnoldi vector
__global__ void __launch_bounds__(kBlock) k_prev_from_residual(int64_t N, const double* __restrict__ v,
                                                             const double* __restrict__ mass, double mu,
                                                             double* __restrict__ up) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < N; k += int64_t(gridDim.x) * blockDim.x)
        up[k] = v[k] / (mu * mass[k]);
}

// sum of squares of r into sc->orr (slot 0) or sc->obb (slot 1)
__global__ void __launch_bounds__(kBlock) k_sumsq(int64_t n, const double* __restrict__ r, KScal* sc, RedBuf red,
                                                int slot) {
    double part[1] = {0.0};
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        part[0] += r[k] * r[k];
    double tot[1];
    if (grid_sum<1>(part, red, tot) && threadIdx.x == 0) {
        if (slot == 0) sc->orr = tot[0];
        else sc->obb = tot[0];
    }
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
struct Ctx {
    cr_hybrid* h;
    cudaStream_t st;
    KScal* sc;    // device
    KScal* hs;    // pinned host
    int64_t nf, n;
    int d;
    bool profile;
    int64_t launches = 0;   // kernels launched by this solve (graph replays counted per kernel)
};

int read_scal(Ctx& c) {
    CR_CUDA(cudaMemcpyAsync(c.hs, c.sc, offsetof(KScal, H), cudaMemcpyDeviceToHost, c.st));
    CR_CUDA(cudaStreamSynchronize(c.st));
    return CR_OK;
}

// One PCG iteration: SpMV (+ p.q), update (+ r.z, r.r), new direction.
// e0/e1 (optional) bracket the SpMV launch for the profile mode.
template <int D, typename VT, typename XT>
void pcg_iteration(Ctx& c, const VT* vals, const XT* minv, XT* x, XT* r, XT* p, XT* q, cudaEvent_t e0,
                   cudaEvent_t e1) {
    const int g = grid_for(c.nf), gn = grid_for(c.n);
    if (e0) cudaEventRecord(e0, c.st);
    k_pcg_spmv<D, VT, XT><<<g, kBlock, 0, c.st>>>(c.nf, c.h->m->cols, vals, p, q, c.sc, c.h->red);
    if (e1) cudaEventRecord(e1, c.st);
    k_pcg_update<D, XT><<<gn, kBlock, 0, c.st>>>(c.n, x, r, p, q, minv, c.sc, c.h->red);
    k_pcg_dir<XT><<<gn, kBlock, 0, c.st>>>(c.n, p, r, minv, c.sc, 0);
    c.launches += 3;
}

// The same iteration in float-float (values hi = val32, lo = vl).
template <int D, typename LT>
void ff_iteration(Ctx& c, const LT* vl, float2* x, float2* r, float2* p, float2* q, cudaEvent_t e0, cudaEvent_t e1) {
    const int g = grid_for(c.nf), gn = grid_for(c.n);
    if (e0) cudaEventRecord(e0, c.st);
    kf_spmv<D, LT><<<g, kBlock, 0, c.st>>>(c.nf, c.h->m->cols, c.h->val32, vl, p, q, c.sc, c.h->red);
    if (e1) cudaEventRecord(e1, c.st);
    kf_update<<<gn, kBlock, 0, c.st>>>(c.n, x, r, p, q, c.h->minv32, c.sc, c.h->red);
    kf_dir<<<gn, kBlock, 0, c.st>>>(c.n, p, r, c.h->minv32, c.sc, 0);
    c.launches += 3;
}

// Run PCG iterations until sc->done, in chunks of `chunk` iterations,
// replayed as a CUDA graph when asked.  `iter(e0, e1)` launches one
// iteration.  Assumes x, r, p, rz, tol2 are set.  `variant` distinguishes
// iterations with different launch sequences under the same graph slot.
template <typename Iter>
int pcg_loop(Ctx& c, Iter iter, int chunk, bool graph, int gkey, int variant = 0, uint64_t tag = 0) {
    cr_hybrid* h = c.h;
    const int64_t key = int64_t(chunk) + (int64_t(variant) << 20);
    if (graph && (h->graph_key[gkey] != key || h->graph_tag[gkey] != tag || !h->graph_exec[gkey])) {
        if (h->graph_exec[gkey]) { cudaGraphExecDestroy(h->graph_exec[gkey]); h->graph_exec[gkey] = nullptr; }
        cudaGraph_t gr;
        const int64_t before = c.launches;
        CR_CUDA(cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < chunk; ++k) iter(nullptr, nullptr);
        CR_CUDA(cudaStreamEndCapture(c.st, &gr));
        h->graph_launches[gkey] = c.launches - before;
        c.launches = before;
        cudaError_t e = cudaGraphInstantiate(&h->graph_exec[gkey], gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        h->graph_key[gkey] = key;
        h->graph_tag[gkey] = tag;
    }
    const bool prof = c.profile && !graph;
    if (prof && int(h->prof_ev.size()) < 2 * chunk) {
        for (int k = int(h->prof_ev.size()); k < 2 * chunk; ++k) {
            cudaEvent_t e;
            CR_CUDA(cudaEventCreate(&e));
            h->prof_ev.push_back(e);
        }
    }
    int it_before = -1;
    for (;;) {
        CR_TRY(read_scal(c));
        if (prof && it_before >= 0) {
            // the SpMV of an iteration runs in full exactly when that iteration is counted
            const int ran = c.hs->it - it_before + (c.hs->status == CR_ERR_BREAKDOWN ? 1 : 0);
            for (int k = 0; k < ran && k < chunk; ++k) {
                float ms = 0.f;
                CR_CUDA(cudaEventElapsedTime(&ms, h->prof_ev[2 * k], h->prof_ev[2 * k + 1]));
                h->prof_ms += ms;
                h->prof_n += 1;
            }
        }
        if (c.hs->done) break;
        it_before = c.hs->it;
        if (graph) {
            CR_CUDA(cudaGraphLaunch(h->graph_exec[gkey], c.st));
            c.launches += h->graph_launches[gkey];
        } else {
            for (int k = 0; k < chunk; ++k) {
                if (prof) iter(h->prof_ev[2 * k], h->prof_ev[2 * k + 1]);
                else iter(nullptr, nullptr);
            }
            CR_CUDA(cudaGetLastError());
        }
    }
    return CR_OK;
}

// One GMRES(m) cycle set: iterate until the residual target or the limit.
// b, x, r, V, z in the working precision; the recursive residual estimate
// |g_{j+1}| drives the inner stop, the true residual is recomputed per cycle.
template <int D, typename VT, typename XT>
int gmres_loop(Ctx& c, const VT* vals, const XT* minv, const XT* b, XT* x, XT* r, XT* V, XT* z) {
    cr_hybrid* h = c.h;
    const int g = grid_for(c.nf), gn = grid_for(c.n);
    for (;;) {
        // true residual of the current iterate starts every cycle
        k_residual_w<D, VT, XT><<<g, kBlock, 0, c.st>>>(c.nf, h->m->cols, vals, b, x, r, c.sc);
        ++c.launches;
        k_gm_norm_start<XT><<<gn, kBlock, 0, c.st>>>(c.n, r, c.sc, h->red);
        ++c.launches;
        k_gm_scale_v0<XT><<<gn, kBlock, 0, c.st>>>(c.n, r, V, c.sc);
        ++c.launches;
        CR_CUDA(cudaGetLastError());
        CR_TRY(read_scal(c));
        if (c.hs->done) break;
        const int m = c.hs->m;
        for (int j = 0; j < m; ++j) {
            k_gm_precond<D, VT, XT><<<gn, kBlock, 0, c.st>>>(c.n, V, minv, z, c.sc);
            ++c.launches;
            k_gm_spmv<D, VT, XT><<<g, kBlock, 0, c.st>>>(c.nf, h->m->cols, vals, z, V, c.sc);
            ++c.launches;
            for (int pass = 0; pass < 2; ++pass) {
                for (int i0 = 0; i0 <= j; i0 += kRedSlots) {
                    k_gm_dots<XT><<<gn, kBlock, 0, c.st>>>(c.n, V, i0, c.sc, h->red);
                    ++c.launches;
                }
                k_gm_orth<XT><<<gn, kBlock, 0, c.st>>>(c.n, V, c.sc, h->red, pass);
                ++c.launches;
            }
            k_gm_normalise<XT><<<gn, kBlock, 0, c.st>>>(c.n, V, c.sc);
            ++c.launches;
            CR_CUDA(cudaGetLastError());
            if ((j + 1) % 8 == 0 || j + 1 == m) {
                CR_TRY(read_scal(c));
                if (c.hs->done || c.hs->stop) break;
            }
        }
        // x += M^{-1} V y over the steps taken in this cycle
        k_gm_solve_y<<<1, 32, 0, c.st>>>(c.sc);
        ++c.launches;
        k_gm_update<XT><<<gn, kBlock, 0, c.st>>>(c.n, x, V, minv, c.sc);
        ++c.launches;
        CR_CUDA(cudaGetLastError());
        CR_TRY(read_scal(c));
        if (c.hs->status != CR_OK) break;
    }
    return CR_OK;
}

// PCG in one cooperative persistent launch per chunk of iterations
// (persist.cu): FP64 (mode 0), or float-float with FP64 reliable updates
// (mode 1: FP32 low plane, mode 2: BF16 low plane).  Solves G x = b for one
// right-hand side b (device, FP64 [nf][d]) from x0 (or 0) and writes the FP64
// iterate to x; *out receives the pair's final scalars.
template <int D>
int persistent_pcg(Ctx& c, const double* b, const double* x0, double* x, int mode, double tol, double delta,
                   int max_it, int per_launch, bool profile, PScal* out, double* kms, int64_t* kit) {
    cr_hybrid* h = c.h;
    cr_mesh* m = h->m;
    const bool ff = mode != 0;
    if ((mode == 2 && (!h->val32 || !h->vlo16)) || (mode == 1 && !h->vff))
        return fail(CR_ERR_ARG, "cr_solve: the float-float values were not kept by cr_hybridise");
    PSys sy{};
    sy.nf = m->nf;
    sy.R = 1;
    sy.cols = m->cols;
    sy.vh = h->val32;
    sy.vl = mode == 2 ? static_cast<const void*>(h->vlo16) : static_cast<const void*>(h->vff);
    sy.v64 = h->val64;
    sy.minv32 = h->minv32;
    sy.minv64 = h->minv64;
    sy.b = b;
    sy.x64 = h->x64;
    sy.r64 = h->r64;
    if (ff) { sy.x = h->xf; sy.r = h->rf; sy.p = h->pf; sy.q = h->qf; }
    else { sy.x = h->x64; sy.r = h->r64; sy.p = h->p64; sy.q = h->q64; }
    PersistPlan*& plan = reinterpret_cast<PersistPlan*&>(h->pplan[mode]);
    if (!plan) plan = new PersistPlan();
    if (!plan->built()) CR_TRY(plan->build({sy}, D, mode, 0));
    else CR_TRY(plan->update_systems({sy}, c.st));
    // start: x64 = x0 (or 0), iteration vectors zero
    if (x0) CR_CUDA(cudaMemcpyAsync(h->x64, x0, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.st));
    else CR_CUDA(cudaMemsetAsync(h->x64, 0, sizeof(double) * c.n, c.st));
    if (ff) {
        CR_CUDA(cudaMemsetAsync(h->xf, 0, sizeof(float2) * c.n, c.st));
        CR_CUDA(cudaMemsetAsync(h->pf, 0, sizeof(float2) * c.n, c.st));
    } else {
        CR_CUDA(cudaMemsetAsync(h->p64, 0, sizeof(double) * c.n, c.st));
    }
    CR_TRY(plan->run(tol, delta, max_it, per_launch, c.st, &c.launches, profile, kms, kit));
    *out = plan->h_scal[0];
    // x = x64, whose FP64 residual the last update phase computed
    CR_CUDA(cudaMemcpyAsync(x, h->x64, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.st));
    return CR_OK;
}

double default_delta(int mode) { return mode == 2 ? 0.1 : 0.01; }
int persistent_mode(int prec) { return prec == CR_PREC_FP64 ? 0 : (prec == CR_PREC_FF ? 1 : 2); }

template <int D>
int solve_persistent(cr_hybrid* h, int rhs, const cr_solve_opts* o, double* W, cr_solve_stats* st) {
    cr_mesh* m = h->m;
    Ctx c{h, m->stream, static_cast<KScal*>(h->scal), static_cast<KScal*>(h->h_scal), m->nf, m->nf * D, D, false};
    const int mode = persistent_mode(o->prec);
    const double delta = o->inner_tol > 0 && o->inner_tol < 1 ? o->inner_tol : default_delta(mode);
    const int gmax = o->max_iter > 0 ? o->max_iter : 100000;
    const int per_launch = (o->check_every > 0 ? o->check_every : 16) * 64;
    double kms = 0.0;
    int64_t kit = 0;
    PScal P{};
    CR_TRY(persistent_pcg<D>(c, h->S + size_t(rhs) * c.n, o->use_x0 ? W : nullptr, W, mode, o->tol, delta, gmax,
                             per_launch, o->profile != 0, &P, &kms, &kit));
    CR_CUDA(cudaStreamSynchronize(c.st));
    int status = P.status;
    if (status == CR_OK && !P.conv) status = CR_ERR_NOT_CONVERGED;
    const double relres = P.bb > 0 ? std::sqrt(P.orr / P.bb) : 0.0;
    if (status == CR_OK && !(relres <= o->tol)) status = CR_ERR_NOT_CONVERGED;
    if (st) {
        st->iterations = P.it;
        st->outer = P.outer;
        st->relres = relres;
        st->status = status;
        // profile: the persistent launches' time and the PCG iterations they ran
        st->spmv_launches = int32_t(kit);
        st->spmv_ms = kms;
        st->kernel_launches = c.launches;
    }
    if (status == CR_ERR_NOT_CONVERGED) return fail(status, "cr_solve: iteration limit reached before the tolerance");
    if (status == CR_ERR_BREAKDOWN) return fail(status, "cr_solve: Krylov breakdown (p.Gp <= 0 or NaN)");
    return status;
}

// Flexible GMRES(m) in FP64 (Saad, Iterative Methods for Sparse Linear
// Systems, Algorithm 9.6) on G W = S, right-preconditioned by an inner
// Jacobi-PCG solve with the SPD matrix of `pre` (persistent kernel, FP64 or
// float-float), each to the relative residual inner_tol:
//   z_j = PCG(G_pre, v_j),  v_{j+1} = G z_j orthogonalised (CGS2),  x = x0 + Z y.
// A preconditioner that changes from step to step is what the flexible form
// allows; the minimised residual is still that of G.
// the multi-kernel solver of cr_solve (defined below): G W = S of h, or = b_override,
// with the Lanczos record when rec is given
template <int D>
int solve_dim(cr_hybrid* h, int rhs, const cr_solve_opts* o, double* W, cr_solve_stats* st,
              const double* b_override = nullptr, const LanczosRec* rec = nullptr);

template <int D>
int solve_fgmres(cr_hybrid* h, int rhs, cr_hybrid* pre, const cr_solve_opts* o, double* W, cr_solve_stats* st) {
    cr_mesh* m = h->m;
    Ctx c{h, m->stream, static_cast<KScal*>(h->scal), static_cast<KScal*>(h->h_scal), m->nf, m->nf * D, D, false};
    Ctx cp{pre, m->stream, static_cast<KScal*>(pre->scal), static_cast<KScal*>(pre->h_scal), m->nf, m->nf * D, D,
           false};
    const double* b = h->S + size_t(rhs) * c.n;
    const int g = grid_for(c.nf), gn = grid_for(c.n);
    const int mode = persistent_mode(o->prec);
    const double itol = o->inner_tol > 0 && o->inner_tol < 1 ? o->inner_tol : 0.1;
    const int gmax = o->max_iter > 0 ? o->max_iter : 1000;
    const int per_launch = (o->check_every > 0 ? o->check_every : 16) * 64;
    double* V = h->V64;
    double* Z = h->fgz;
    std::memset(c.hs, 0, sizeof(KScal));
    c.hs->max_it = gmax;
    c.hs->m = o->restart > 0 ? o->restart : 30;
    CR_CUDA(cudaMemcpyAsync(c.sc, c.hs, sizeof(KScal), cudaMemcpyHostToDevice, c.st));
    if (o->use_x0) CR_CUDA(cudaMemcpyAsync(h->x64, W, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.st));
    else CR_CUDA(cudaMemsetAsync(h->x64, 0, sizeof(double) * c.n, c.st));
    // tol2 = tol^2 ||b||^2 from the FP64 residual of the start
    k_residual64<D><<<g, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, b, h->x64, h->r64, nullptr, h->minv64, c.sc,
                                            h->red, 1, o->tol, 0.0);
    ++c.launches;
    CR_CUDA(cudaGetLastError());
    int64_t inner_its = 0, prof_it = 0;
    double prof_ms = 0.0;
    int status = CR_OK;
    for (;;) {
        k_residual_w<D, double, double><<<g, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, b, h->x64, h->r64, c.sc);
        k_gm_norm_start<double><<<gn, kBlock, 0, c.st>>>(c.n, h->r64, c.sc, h->red);
        k_gm_scale_v0<double><<<gn, kBlock, 0, c.st>>>(c.n, h->r64, V, c.sc);
        c.launches += 3;
        CR_CUDA(cudaGetLastError());
        CR_TRY(read_scal(c));
        if (c.hs->done) break;
        const int mr = c.hs->m;
        for (int j = 0; j < mr; ++j) {
            if (o->precond == CR_PRECOND_CHEBYSHEV || o->deflation) {
                // z_j by the Chebyshev-preconditioned (or deflated) PCG of cr_solve on G_pre,
                // multi-kernel and graph-replayed, with v_j as its right-hand side
                cr_solve_opts io = *o;
                io.method = CR_METHOD_PCG;
                io.tol = itol;
                io.max_iter = 100000;
                io.use_x0 = 0;
                io.use_graph = o->profile ? 0 : 1;
                io.persistent = 0;
                io.inner_tol = 0.0;
                cr_solve_stats ist{};
                const int rc = solve_dim<D>(pre, 0, &io, Z + size_t(j) * c.n, &ist, V + size_t(j) * c.n);
                if (rc != CR_OK && rc != CR_ERR_NOT_CONVERGED && rc != CR_ERR_BREAKDOWN) return rc;
                inner_its += ist.iterations;
                prof_ms += ist.spmv_ms;
                prof_it += ist.spmv_launches;
                cp.launches += ist.kernel_launches;
                if (ist.status == CR_ERR_BREAKDOWN) { status = CR_ERR_BREAKDOWN; break; }
            } else {
                PScal P{};
                double kms = 0.0;
                int64_t kit = 0;
                CR_TRY(persistent_pcg<D>(cp, V + size_t(j) * c.n, nullptr, Z + size_t(j) * c.n, mode, itol,
                                         default_delta(mode), 100000, per_launch, o->profile != 0, &P, &kms, &kit));
                inner_its += P.it;
                prof_ms += kms;
                prof_it += kit;
                if (P.status == CR_ERR_BREAKDOWN) { status = CR_ERR_BREAKDOWN; break; }
            }
            k_gm_spmv<D, double, double><<<g, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, Z + size_t(j) * c.n, V,
                                                                 c.sc);
            ++c.launches;
            for (int pass = 0; pass < 2; ++pass) {
                for (int i0 = 0; i0 <= j; i0 += kRedSlots) {
                    k_gm_dots<double><<<gn, kBlock, 0, c.st>>>(c.n, V, i0, c.sc, h->red);
                    ++c.launches;
                }
                k_gm_orth<double><<<gn, kBlock, 0, c.st>>>(c.n, V, c.sc, h->red, pass);
                ++c.launches;
            }
            k_gm_normalise<double><<<gn, kBlock, 0, c.st>>>(c.n, V, c.sc);
            ++c.launches;
            CR_CUDA(cudaGetLastError());
            CR_TRY(read_scal(c));
            if (c.hs->done || c.hs->stop) break;
        }
        if (status != CR_OK) break;
        // x += Z y over the steps taken in this cycle
        k_gm_solve_y<<<1, 32, 0, c.st>>>(c.sc);
        k_fgm_update<<<gn, kBlock, 0, c.st>>>(c.n, h->x64, Z, c.sc);
        c.launches += 2;
        CR_CUDA(cudaGetLastError());
        CR_TRY(read_scal(c));
        if (c.hs->status != CR_OK) break;
    }
    c.launches += cp.launches;
    CR_TRY(read_scal(c));
    if (status == CR_OK) status = c.hs->status;
    const int steps = c.hs->it;
    // W = x; final FP64 residual of the returned W
    CR_CUDA(cudaMemcpyAsync(W, h->x64, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.st));
    k_residual64<D><<<g, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, b, h->x64, nullptr, nullptr, h->minv64, c.sc,
                                            h->red, 0, o->tol, 0.0);
    ++c.launches;
    CR_CUDA(cudaGetLastError());
    CR_TRY(read_scal(c));
    const double relres = c.hs->obb > 0 ? std::sqrt(c.hs->orr / c.hs->obb) : 0.0;
    if (status == CR_OK && !(relres <= o->tol)) status = CR_ERR_NOT_CONVERGED;
    if (st) {
        st->iterations = int32_t(inner_its);
        st->outer = steps;
        st->relres = relres;
        st->status = status;
        // profile: the inner persistent launches' time and the PCG iterations they ran
        st->spmv_launches = int32_t(prof_it);
        st->spmv_ms = prof_ms;
        st->kernel_launches = c.launches;
    }
    if (status == CR_ERR_NOT_CONVERGED) return fail(status, "cr_solve_preconditioned: step limit reached before the tolerance");
    if (status == CR_ERR_BREAKDOWN) return fail(status, "cr_solve_preconditioned: breakdown (zero Arnoldi vector, NaN, or p.Gp <= 0 in the inner PCG)");
    return status;
}

// FP64 PCG whose recursively updated residual decides the stop: once it meets
// the tolerance, the FP64 true residual b - G x decides.  A true residual still
// above the tolerance (the recursive one drifts from it on ill-conditioned
// systems) restarts CG from the iterate with r = b - G x, up to max_outer
// times, so that CR_OK always means ||b - G x|| <= tol ||b||.  `start` forms
// the first direction from r; `run` iterates until the device flags done.
// With a deflation space dfl every cycle first moves x to x + V E^{-1} V^t r and
// recomputes r (the deflated start: V^t r = 0).
template <int D, typename Start, typename Run>
int restarted_pcg(Ctx& c, Start start, Run run, const double* b, int max_outer, double tol, int& outer,
                  const cr_deflation* dfl = nullptr) {
    cr_hybrid* h = c.h;
    const int ggrid = grid_for(c.nf);
    for (;;) {
        CR_TRY(read_scal(c));
        if (c.hs->done) return CR_OK;   // the start (true) residual already meets the tolerance
        if (dfl) {
            CR_TRY(defl_dots64(dfl, dfl->V64, h->r64, true, nullptr, c.st));
            CR_TRY(defl_axpy64(dfl, dfl->V64, 1.0, h->x64, c.st));
            k_residual64<D><<<ggrid, kBlock, 0, c.st>>>(c.nf, h->m->cols, h->val64, b, h->x64, h->r64, nullptr,
                                                        h->minv64, c.sc, h->red, 1, tol, 0.0);
            c.launches += 3;
            CR_CUDA(cudaGetLastError());
            CR_TRY(read_scal(c));
            if (c.hs->done) return CR_OK;
        }
        start();
        CR_CUDA(cudaGetLastError());
        CR_TRY(run());
        CR_TRY(read_scal(c));
        if (c.hs->status != CR_OK) return CR_OK;
        // mode 1: r = b - G x, rz, rr, tol2; done when the true residual meets tol
        k_residual64<D><<<ggrid, kBlock, 0, c.st>>>(c.nf, h->m->cols, h->val64, b, h->x64, h->r64, nullptr,
                                                    h->minv64, c.sc, h->red, 1, tol, 0.0);
        ++c.launches;
        CR_CUDA(cudaGetLastError());
        CR_TRY(read_scal(c));
        if (c.hs->done) return CR_OK;
        if (outer >= max_outer || c.hs->it >= c.hs->max_it) {
            c.hs->status = CR_ERR_NOT_CONVERGED;
            return CR_OK;
        }
        ++outer;
    }
}

// The Chebyshev preconditioner's coefficients for this solve (into hs->cheb):
// the Gershgorin bound lmax of M^{-1} G is computed once per hybridised system.
template <int D>
int chebyshev_setup(cr_hybrid* h, const cr_solve_opts* o, cudaStream_t st, KScal* hs) {
    const int64_t n = h->m->nf * D;
    if (n == 0) h->cheb_lmax = 1.0;   // no unknowns: any interval will do
    if (h->cheb_lmax < 0.0) {
        unsigned long long* slot = reinterpret_cast<unsigned long long*>(h->cheb + 3 * n);
        CR_CUDA(cudaMemsetAsync(slot, 0, sizeof(unsigned long long), st));
        k_gershgorin<D><<<grid_for(h->m->nf), kBlock, 0, st>>>(h->m->nf, h->val64, h->minv64, slot);
        CR_CUDA(cudaGetLastError());
        double lmax = 0.0;
        CR_CUDA(cudaMemcpyAsync(&lmax, slot, sizeof(double), cudaMemcpyDeviceToHost, st));
        CR_CUDA(cudaStreamSynchronize(st));
        if (!(lmax > 0.0) || !std::isfinite(lmax))
            return fail(CR_ERR_BREAKDOWN, "cr_solve: no positive Gershgorin bound for the Chebyshev preconditioner");
        h->cheb_lmax = lmax;
    }
    const int deg = o->poly_degree > 0 ? o->poly_degree : 4;
    const double ratio = o->poly_ratio > 0.0 ? o->poly_ratio : 100.0;
    const double b = h->cheb_lmax, a = b / ratio;
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a);
    double rho = delta / theta;
    hs->cheb[0] = 1.0 / theta;
    for (int j = 1; j < deg; ++j) {
        const double rn = 1.0 / (2.0 * theta / delta - rho);
        hs->cheb[2 * j - 1] = rn * rho;
        hs->cheb[2 * j] = 2.0 * rn / delta;
        rho = rn;
    }
    return CR_OK;
}

template <int D>
int solve_dim(cr_hybrid* h, int rhs, const cr_solve_opts* o, double* W, cr_solve_stats* st,
              const double* b_override, const LanczosRec* rec) {
    cr_mesh* m = h->m;
    Ctx c{h, m->stream, static_cast<KScal*>(h->scal), static_cast<KScal*>(h->h_scal), m->nf, m->nf * D, D,
          o->profile != 0};
    h->prof_ms = 0.0;
    h->prof_n = 0;
    // the right-hand side: S of h, or (inner solves of the steady preconditioner) a given vector
    const double* b = b_override ? b_override : h->S + size_t(rhs) * c.n;
    const int chunk = o->check_every > 0 ? o->check_every : 16;
    const bool graph = o->use_graph != 0;
    const int gmax = o->max_iter > 0 ? o->max_iter : 100000;
    const int max_outer = o->max_outer > 0 ? o->max_outer : 60;
    const int ggrid = grid_for(c.nf), gn = grid_for(c.n);
    const double* x0 = o->use_x0 ? h->x64 : nullptr;
    const cr_deflation* dfl = o->deflation;   // checked against h by the caller
    const int* done = &c.sc->done;            // device flag: the deflation kernels skip a finished solve
    const uint64_t dtag = dfl ? dfl->serial : 0;
    // the Lanczos record: after every direction; a restarted direction after the first ends it
    bool rec_started = false;
    auto record = [&](const void* z, int kind, bool restart) {   // kind 0: FP64 z (null: M^{-1} r), 1: FP32, 2: FF
        if (!rec) return;
        if (restart && rec_started) cudaMemsetAsync(rec->stop, 0xff, sizeof(int), c.st);
        rec_started = true;
        const int g = grid_for(c.n);
        if (kind == 1)
            k_lanczos_record<float><<<g, kBlock, 0, c.st>>>(c.n, static_cast<const float*>(z), h->minv64, h->r64,
                                                            c.sc, *rec);
        else if (kind == 2)
            k_lanczos_record<float2><<<g, kBlock, 0, c.st>>>(c.n, static_cast<const float2*>(z), h->minv64,
                                                             h->r64, c.sc, *rec);
        else
            k_lanczos_record<double><<<g, kBlock, 0, c.st>>>(c.n, static_cast<const double*>(z), h->minv64,
                                                             h->r64, c.sc, *rec);
        ++c.launches;
    };
    const int rtag = rec ? 1 << 11 : 0;   // graph variant of recording iterations

    std::memset(c.hs, 0, sizeof(KScal));
    c.hs->max_it = gmax;
    c.hs->m = o->restart > 0 ? o->restart : 30;
    const bool cheb = o->precond == CR_PRECOND_CHEBYSHEV;
    if (cheb) CR_TRY(chebyshev_setup<D>(h, o, c.st, c.hs));
    CR_CUDA(cudaMemcpyAsync(c.sc, c.hs, sizeof(KScal), cudaMemcpyHostToDevice, c.st));
    if (o->use_x0) CR_CUDA(cudaMemcpyAsync(h->x64, W, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.st));
    else CR_CUDA(cudaMemsetAsync(h->x64, 0, sizeof(double) * c.n, c.st));

    int status = CR_OK;   // decided on the host; device statuses are folded in below
    int outer = 0;
    std::string why;      // which exit of a refinement loop ended an unsuccessful solve
    if (o->prec == CR_PREC_FP64) {
        k_residual64<D><<<ggrid, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, b, x0, h->r64, nullptr, h->minv64, c.sc,
                                                    h->red, 1, o->tol, 0.0);
        ++c.launches;
        CR_CUDA(cudaGetLastError());
        if (o->method == CR_METHOD_BICGSTAB) {
            auto iter = [&](cudaEvent_t e0, cudaEvent_t e1) {
                const int g = grid_for(c.nf);
                k_bs_dir<<<gn, kBlock, 0, c.st>>>(c.n, h->r64, h->p64, h->bs_v, h->minv64, h->bs_y, c.sc);
                if (e0) cudaEventRecord(e0, c.st);
                k_bs_spmv<D><<<g, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, h->bs_y, h->bs_v, h->bs_rh, c.sc, h->red, 0);
                if (e1) cudaEventRecord(e1, c.st);
                k_bs_s<<<gn, kBlock, 0, c.st>>>(c.n, h->r64, h->bs_v, h->minv64, h->bs_s, h->bs_z, c.sc);
                k_bs_spmv<D><<<g, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, h->bs_z, h->bs_t, h->bs_s, c.sc, h->red, 1);
                k_bs_update<<<gn, kBlock, 0, c.st>>>(c.n, h->x64, h->r64, h->bs_y, h->bs_z, h->bs_s, h->bs_t, h->bs_rh,
                                                     c.sc, h->red);
                c.launches += 5;
            };
            // The recursive residual of BiCGStab drifts from the true one on these
            // ill-conditioned systems: when it meets the tolerance the FP64 true
            // residual decides, and a shortfall restarts BiCGStab from the iterate
            // (shadow residual = the true residual), up to max_outer times.
            for (int restart = 0;; ++restart) {
                k_bs_init<<<gn, kBlock, 0, c.st>>>(c.n, h->r64, h->bs_rh, h->p64, h->bs_v, c.sc, h->red);
                ++c.launches;
                CR_TRY(pcg_loop(c, iter, chunk, graph, 5));
                CR_TRY(read_scal(c));
                if (c.hs->status != CR_OK) break;
                k_residual64<D><<<ggrid, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, b, h->x64, h->r64, nullptr,
                                                            h->minv64, c.sc, h->red, 1, o->tol, 0.0);
                ++c.launches;
                CR_TRY(read_scal(c));
                if (c.hs->done || restart >= max_outer) break;
                ++outer;
            }
        } else if (o->method == CR_METHOD_PCG && cheb) {
            // CG iteration: SpMV + p.q, update + r.r + first Chebyshev step, the
            // remaining degree - 1 steps (SpMV each; the last one forms r.z and
            // beta), direction.  profile = 1 brackets the Chebyshev steps.
            const int deg = o->poly_degree > 0 ? o->poly_degree : 4;
            double* zb[2] = {h->cheb, h->cheb + c.n};
            double* dv = h->cheb + 2 * c.n;
            auto cheb_steps = [&](cudaEvent_t e0, cudaEvent_t e1) {
                if (e0) cudaEventRecord(e0, c.st);
                for (int j = 1; j < deg; ++j)
                    k_cheb_step<D><<<grid_occ(k_cheb_step<D>, c.nf), kBlock, 0, c.st>>>(c.nf, m->cols, h->val64,
                                                                                       h->minv64, h->r64,
                                                               zb[(j - 1) & 1], zb[j & 1], dv, c.sc, h->red, j,
                                                               j == deg - 1);
                if (e1) cudaEventRecord(e1, c.st);
                c.launches += deg - 1;
            };
            // deflated: c = E^{-1} (G V)^t z before the direction, p -= V c after it
            auto direction = [&](int first) {
                if (dfl) defl_dots64(dfl, dfl->GV64, zb[(deg - 1) & 1], true, done, c.st);
                k_cpcg_dir<<<gn, kBlock, 0, c.st>>>(c.n, h->p64, zb[(deg - 1) & 1], c.sc, first);
                if (dfl) defl_project64(dfl, h->p64, done, c.st);
                c.launches += dfl ? 3 : 1;
                record(zb[(deg - 1) & 1], 0, first != 0);
            };
            auto start = [&]() {
                k_cheb_start<<<gn, kBlock, 0, c.st>>>(c.n, h->r64, h->minv64, zb[0], dv, c.sc);
                ++c.launches;
                cheb_steps(nullptr, nullptr);
                direction(1);
            };
            auto iter = [&](cudaEvent_t e0, cudaEvent_t e1) {
                k_pcg_spmv<D, double, double><<<grid_occ(k_pcg_spmv<D, double, double>, c.nf), kBlock, 0, c.st>>>(
                    c.nf, m->cols, h->val64, h->p64, h->q64,
                                                                          c.sc, h->red);
                k_cpcg_update<<<gn, kBlock, 0, c.st>>>(c.n, h->x64, h->r64, h->p64, h->q64, h->minv64, zb[0], dv,
                                                       c.sc, h->red);
                cheb_steps(e0, e1);
                direction(0);
                c.launches += 2;
            };
            CR_TRY(restarted_pcg<D>(
                c, start, [&]() { return pcg_loop(c, iter, chunk, graph, 6, deg + (dfl ? 512 : 0) + rtag, dtag); },
                b, max_outer, o->tol, outer, dfl));
        } else if (o->method == CR_METHOD_PCG) {
            // deflated (Jacobi): c = E^{-1} (M^{-1} G V)^t r = E^{-1} (G V)^t z, p -= V c
            auto start = [&]() {
                k_pcg_dir<double><<<gn, kBlock, 0, c.st>>>(c.n, h->p64, h->r64, h->minv64, c.sc, 1);
                ++c.launches;
                if (dfl) {
                    defl_dots64(dfl, dfl->W64, h->r64, true, done, c.st);
                    defl_project64(dfl, h->p64, done, c.st);
                    c.launches += 2;
                }
                record(nullptr, 0, true);
            };
            auto iter = [&](cudaEvent_t e0, cudaEvent_t e1) {
                if (!dfl) {
                    pcg_iteration<D, double, double>(c, h->val64, h->minv64, h->x64, h->r64, h->p64, h->q64, e0, e1);
                    record(nullptr, 0, false);
                    return;
                }
                if (e0) cudaEventRecord(e0, c.st);
                k_pcg_spmv<D, double, double><<<ggrid, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, h->p64, h->q64,
                                                                           c.sc, h->red);
                if (e1) cudaEventRecord(e1, c.st);
                k_pcg_update<D, double><<<gn, kBlock, 0, c.st>>>(c.n, h->x64, h->r64, h->p64, h->q64, h->minv64,
                                                                 c.sc, h->red);
                defl_dots64(dfl, dfl->W64, h->r64, true, done, c.st);
                k_pcg_dir<double><<<gn, kBlock, 0, c.st>>>(c.n, h->p64, h->r64, h->minv64, c.sc, 0);
                defl_project64(dfl, h->p64, done, c.st);
                c.launches += 5;
            };
            CR_TRY(restarted_pcg<D>(
                c, start, [&]() { return pcg_loop(c, iter, chunk, graph, 0, (dfl ? 512 : 0) + rtag, dtag); }, b,
                max_outer, o->tol, outer, dfl));
        } else {
            CR_TRY((gmres_loop<D, double, double>(c, h->val64, h->minv64, b, h->x64, h->r64, h->V64, h->Z64)));
        }
        const int restart_status = c.hs->status;   // restarted_pcg may have set it on the host
        CR_TRY(read_scal(c));
        status = restart_status != CR_OK ? restart_status : c.hs->status;
    } else if (o->prec == CR_PREC_FF || o->prec == CR_PREC_FF_BF16) {
        // Float-float PCG with reliable updates (FP32 pipes only inside the
        // iteration).  Each time the iterated residual has fallen by `delta`,
        // the correction is added to the FP64 iterate, the residual is
        // replaced by the FP64 true residual b - G x (FP64 values), and the
        // search direction is continued with beta = r.z(true) / r.z(previous).
        if (o->method != CR_METHOD_PCG)
            return fail(CR_ERR_ARG, "cr_solve: the float-float precisions are implemented for PCG");
        const bool bf = o->prec == CR_PREC_FF_BF16;
        if ((bf && (!h->val32 || !h->vlo16)) || (!bf && !h->vff))
            return fail(CR_ERR_ARG, "cr_solve: the float-float values were not kept by cr_hybridise");
        const double delta = o->inner_tol > 0 && o->inner_tol < 1 ? o->inner_tol : (bf ? 0.1 : 0.01);
        const bool trace = std::getenv("CRHYB_TRACE") != nullptr;
        c.hs->sigma = 1.0;
        CR_CUDA(cudaMemcpyAsync(&c.sc->sigma, &c.hs->sigma, sizeof(double), cudaMemcpyHostToDevice, c.st));
        CR_CUDA(cudaMemsetAsync(h->xf, 0, sizeof(float2) * c.n, c.st));
        if (cheb) {
            // Chebyshev-preconditioned CG in float-float: per iteration the SpMV (+ p.q),
            // the update with the first Chebyshev step (+ r.r), degree - 1 Chebyshev steps
            // (SpMV each; the last forms r.z and beta) and the direction.  Reliable updates
            // as for the Jacobi form: the FP64 true residual, a new scale, and the
            // direction continued with r.z moved to the new scale.
            const int deg = o->poly_degree > 0 ? o->poly_degree : 4;
            float2* zb[2] = {h->chebf, h->chebf + c.n};
            float2* dv = h->chebf + 2 * c.n;
            // reduced-precision steps (poly_prec): FP32 z (two buffers) and d in the same storage
            const int pp = o->poly_prec;
            float* zs[2] = {reinterpret_cast<float*>(h->chebf), reinterpret_cast<float*>(h->chebf) + c.n};
            float* ds = reinterpret_cast<float*>(h->chebf) + 2 * c.n;
            if ((pp == CR_POLY_FP32 && !h->val32) || (pp == CR_POLY_BF16 && !h->val16))
                return fail(CR_ERR_ARG, "cr_solve: the values for poly_prec were not kept by cr_hybridise");
            auto cheb_steps = [&](cudaEvent_t e0, cudaEvent_t e1) {
                if (e0) cudaEventRecord(e0, c.st);
                for (int j = 1; j < deg; ++j) {
                    if (pp == CR_POLY_FP32)
                        launch_cheb32<D, float>(c.nf, m->cols, h->val32, h->minv32, h->rf, zs[(j - 1) & 1], zs[j & 1],
                                                ds, c.sc, h->red, j, j == deg - 1, c.st);
                    else if (pp == CR_POLY_BF16)
                        launch_cheb32<D, __nv_bfloat16>(c.nf, m->cols, h->val16, h->minv32, h->rf, zs[(j - 1) & 1],
                                                        zs[j & 1], ds, c.sc, h->red, j, j == deg - 1, c.st);
                    else if (bf)
                        kf_cheb_step<D, __nv_bfloat16>
                            <<<grid_occ(kf_cheb_step<D, __nv_bfloat16>, c.nf), kBlock, 0, c.st>>>(
                                c.nf, m->cols, h->val32, h->vlo16, h->minv32, h->rf, zb[(j - 1) & 1], zb[j & 1], dv,
                                c.sc, h->red, j, j == deg - 1);
                    else
                        kf_cheb_step<D, float2><<<grid_occ(kf_cheb_step<D, float2>, c.nf), kBlock, 0, c.st>>>(
                            c.nf, m->cols, h->val32, h->vff, h->minv32, h->rf, zb[(j - 1) & 1], zb[j & 1], dv, c.sc,
                            h->red, j, j == deg - 1);
                }
                if (e1) cudaEventRecord(e1, c.st);
                c.launches += deg - 1;
            };
            // the direction p = z + beta p; deflated: c = E^{-1} (G V)^t z (FP64 G V, FP64
            // products) before, p -= V c (FP32 V) after
            auto direction = [&](int first) {
                if (dfl) {
                    if (pp != CR_POLY_SAME) defl_dots64f(dfl, dfl->GV64, zs[(deg - 1) & 1], done, c.st);
                    else defl_dots64ff(dfl, dfl->GV64, zb[(deg - 1) & 1], done, c.st);
                }
                if (pp != CR_POLY_SAME)
                    kf_cpcg_dir32<<<gn, kBlock, 0, c.st>>>(c.n, h->pf, zs[(deg - 1) & 1], c.sc, first);
                else kf_cpcg_dir<<<gn, kBlock, 0, c.st>>>(c.n, h->pf, zb[(deg - 1) & 1], c.sc, first);
                if (dfl) defl_projectff(dfl, h->pf, done, c.st);
                c.launches += dfl ? 3 : 1;
                if (pp != CR_POLY_SAME) record(zs[(deg - 1) & 1], 1, first != 0);
                else record(zb[(deg - 1) & 1], 2, first != 0);
            };
            auto restart_direction = [&](int first) {
                if (pp != CR_POLY_SAME) kf_cheb_start32<<<gn, kBlock, 0, c.st>>>(c.n, h->rf, h->minv32, zs[0], ds, c.sc);
                else kf_cheb_start<<<gn, kBlock, 0, c.st>>>(c.n, h->rf, h->minv32, zb[0], dv, c.sc);
                ++c.launches;
                cheb_steps(nullptr, nullptr);
                direction(first);
            };
            // deflated start (and the same at every reliable update, which also removes the
            // components along V that the FP32 projection lets into r):
            // x64 += V E^{-1} V^t (b - G x64)
            auto deflate_x = [&](const double* x) {
                k_residual64<D><<<ggrid, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, b, x, h->r64, nullptr,
                                                            h->minv64, c.sc, h->red, 0, o->tol, 0.0);
                defl_dots64(dfl, dfl->V64, h->r64, true, nullptr, c.st);
                defl_axpy64(dfl, dfl->V64, 1.0, h->x64, c.st);
                c.launches += 3;
            };
            auto true_residual3 = [&](const double* x) {
                k_residual64<D><<<ggrid, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, b, x, h->r64, nullptr, h->minv64,
                                                            c.sc, h->red, 3, o->tol, delta, h->minv32);
                k_ff_from64<<<gn, kBlock, 0, c.st>>>(c.n, h->r64, h->rf, c.sc);
                c.launches += 2;
            };
            if (dfl) {
                deflate_x(x0);
                true_residual3(h->x64);
            } else {
                true_residual3(x0);
            }
            restart_direction(1);
            CR_CUDA(cudaGetLastError());
            CR_TRY(read_scal(c));
            if (c.hs->status == CR_ERR_BREAKDOWN) status = CR_ERR_BREAKDOWN;
            double last_rr = c.hs->orr;
            int it_mark = 0;
            auto iter = [&](cudaEvent_t e0, cudaEvent_t e1) {
                if (bf)
                    kf_spmv<D, __nv_bfloat16><<<grid_occ(kf_spmv<D, __nv_bfloat16>, c.nf), kBlock, 0, c.st>>>(
                        c.nf, m->cols, h->val32, h->vlo16, h->pf, h->qf, c.sc, h->red);
                else
                    kf_spmv<D, float2><<<grid_occ(kf_spmv<D, float2>, c.nf), kBlock, 0, c.st>>>(
                        c.nf, m->cols, h->val32, h->vff, h->pf, h->qf, c.sc, h->red);
                if (pp != CR_POLY_SAME)
                    kf_cpcg_update32<<<gn, kBlock, 0, c.st>>>(c.n, h->xf, h->rf, h->pf, h->qf, h->minv32, zs[0], ds,
                                                              c.sc, h->red);
                else
                    kf_cpcg_update<<<gn, kBlock, 0, c.st>>>(c.n, h->xf, h->rf, h->pf, h->qf, h->minv32, zb[0], dv,
                                                            c.sc, h->red);
                cheb_steps(e0, e1);
                direction(0);
                c.launches += 2;
            };
            while (status == CR_OK && !c.hs->conv) {
                CR_TRY(pcg_loop(c, iter, chunk, graph, 7, deg + (bf ? 100 : 0) + 1000 * pp + (dfl ? 4096 : 0) + 4 * rtag,
                                dtag));
                CR_TRY(read_scal(c));
                const int dev_status = c.hs->status;
                if (dev_status == CR_ERR_TIMEOUT) { status = CR_ERR_TIMEOUT; break; }
                if (dev_status == CR_ERR_BREAKDOWN && c.hs->it == it_mark) { status = CR_ERR_BREAKDOWN; break; }
                k_add_ff<<<gn, kBlock, 0, c.st>>>(c.n, h->x64, h->xf, c.sc);
                ++c.launches;
                if (dfl) deflate_x(h->x64);
                true_residual3(h->x64);
                CR_CUDA(cudaGetLastError());
                CR_TRY(read_scal(c));
                ++outer;
                if (trace)
                    std::fprintf(stderr, "[crhyb] ff chebyshev update %d: it %d, true relres %.3e, status %d\n", outer,
                                 c.hs->it, std::sqrt(c.hs->orr / c.hs->obb), dev_status);
                it_mark = c.hs->it;
                if (c.hs->status == CR_ERR_BREAKDOWN) { status = CR_ERR_BREAKDOWN; break; }
                if (c.hs->conv) break;
                if (c.hs->it >= gmax) { status = CR_ERR_NOT_CONVERGED; break; }
                if (c.hs->orr > 100.0 * last_rr) { status = CR_ERR_BREAKDOWN; break; }   // diverging
                last_rr = c.hs->orr;
                restart_direction(dev_status == CR_OK ? 0 : 1);
                CR_CUDA(cudaGetLastError());
            }
        } else {
        // the reliable update: r64 = b - G x64 (FP64), new scale, r_ff = sigma r64
        auto true_residual = [&](const double* x) {
            k_residual64<D><<<ggrid, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, b, x, h->r64, nullptr, h->minv64,
                                                        c.sc, h->red, 2, o->tol, delta, h->minv32);
            k_ff_from64<<<gn, kBlock, 0, c.st>>>(c.n, h->r64, h->rf, c.sc);
            c.launches += 2;
        };
        true_residual(x0);
        kf_dir<<<gn, kBlock, 0, c.st>>>(c.n, h->pf, h->rf, h->minv32, c.sc, 1);
        ++c.launches;
        CR_CUDA(cudaGetLastError());
        CR_TRY(read_scal(c));
        if (c.hs->status == CR_ERR_BREAKDOWN) status = CR_ERR_BREAKDOWN;
        double last_rr = c.hs->orr;
        int it_mark = 0;
        auto iter = [&](cudaEvent_t e0, cudaEvent_t e1) {
            if (bf) ff_iteration<D, __nv_bfloat16>(c, h->vlo16, h->xf, h->rf, h->pf, h->qf, e0, e1);
            else ff_iteration<D, float2>(c, h->vff, h->xf, h->rf, h->pf, h->qf, e0, e1);
        };
        while (status == CR_OK && !c.hs->conv) {
            CR_TRY(pcg_loop(c, iter, chunk, graph, bf ? 4 : 3));
            CR_TRY(read_scal(c));
            const int dev_status = c.hs->status;
            const double it_rr = c.hs->rr / (c.hs->sigma * c.hs->sigma);
            if (dev_status == CR_ERR_BREAKDOWN && c.hs->it == it_mark) { status = CR_ERR_BREAKDOWN; break; }
            // reliable update
            k_add_ff<<<gn, kBlock, 0, c.st>>>(c.n, h->x64, h->xf, c.sc);
            ++c.launches;
            true_residual(h->x64);
            CR_CUDA(cudaGetLastError());
            CR_TRY(read_scal(c));
            ++outer;
            if (trace)
                std::fprintf(stderr, "[crhyb] ff update %d: it %d, iterated relres %.3e, true relres %.3e, status %d\n",
                             outer, c.hs->it, std::sqrt(it_rr / c.hs->obb), std::sqrt(c.hs->orr / c.hs->obb),
                             dev_status);
            it_mark = c.hs->it;
            if (c.hs->status == CR_ERR_BREAKDOWN) { status = CR_ERR_BREAKDOWN; break; }
            if (c.hs->conv) break;
            if (c.hs->it >= gmax) { status = CR_ERR_NOT_CONVERGED; break; }
            if (c.hs->orr > 100.0 * last_rr) { status = CR_ERR_BREAKDOWN; break; }   // diverging
            last_rr = c.hs->orr;
            kf_dir<<<gn, kBlock, 0, c.st>>>(c.n, h->pf, h->rf, h->minv32, c.sc, dev_status == CR_OK ? 0 : 1);
            ++c.launches;
            CR_CUDA(cudaGetLastError());
        }
        }
    } else if (o->method == CR_METHOD_PCG) {
        // FP32 PCG (FP32 or BF16 matrix values) inside FP64 iterative
        // refinement: r = b - G x in FP64, an inner FP32 solve G d = r to the
        // relative residual inner_tol from d = 0, x += d; repeated until the
        // FP64 residual meets the tolerance.
        const bool bf = o->prec == CR_PREC_MIXED_BF16;
        if ((bf && !h->val16) || (!bf && !h->val32))
            return fail(CR_ERR_ARG, "cr_solve: the values for this precision were not kept by cr_hybridise");
        const double itol = o->inner_tol > 0 ? o->inner_tol : 1e-4;
        const bool trace = std::getenv("CRHYB_TRACE") != nullptr;
        auto iter = [&](cudaEvent_t e0, cudaEvent_t e1) {
            if (bf) pcg_iteration<D, __nv_bfloat16, float>(c, h->val16, h->minv32, h->x32, h->r32, h->p32, h->q32, e0, e1);
            else pcg_iteration<D, float, float>(c, h->val32, h->minv32, h->x32, h->r32, h->p32, h->q32, e0, e1);
        };
        double last = -1.0;
        const char* exit_reason = "converged";
        for (;;) {
            k_residual64<D><<<ggrid, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, b, x0, h->r64, h->r32, h->minv64,
                                                        c.sc, h->red, 0, o->tol, 0.0);
            ++c.launches;
            x0 = h->x64;
            CR_CUDA(cudaGetLastError());
            CR_TRY(read_scal(c));
            const double rel2 = c.hs->obb > 0 ? c.hs->orr / c.hs->obb : 0.0;
            if (trace)
                std::fprintf(stderr, "[crhyb] fp32 refinement step %d: FP64 relres %.3e, inner iterations so far %d\n",
                             outer, std::sqrt(rel2), c.hs->it);
            if (!std::isfinite(rel2)) { status = CR_ERR_BREAKDOWN; exit_reason = "non-finite FP64 residual"; break; }
            if (rel2 <= o->tol * o->tol) break;
            if (outer >= max_outer || c.hs->it >= gmax) {
                status = CR_ERR_NOT_CONVERGED;
                exit_reason = outer >= max_outer ? "refinement step limit" : "inner iteration limit";
                break;
            }
            if (last >= 0.0 && rel2 > 100.0 * last) {   // diverging
                status = CR_ERR_BREAKDOWN;
                exit_reason = "divergence guard: the FP64 residual grew more than 100-fold in one step";
                break;
            }
            last = rel2;
            const int it_start = c.hs->it;
            k_inner_start<float><<<gn, kBlock, 0, c.st>>>(c.n, h->x32, h->r32, h->p32, h->minv32, c.sc, h->red, itol);
            ++c.launches;
            CR_CUDA(cudaGetLastError());
            CR_TRY(pcg_loop(c, iter, chunk, graph, bf ? 2 : 1));
            CR_TRY(read_scal(c));
            if (trace)
                std::fprintf(stderr, "[crhyb]   inner FP32 PCG: %d iterations, inner relres %.3e, status %d\n",
                             c.hs->it - it_start, c.hs->bb > 0 ? std::sqrt(c.hs->rr / c.hs->bb) : 0.0,
                             c.hs->status);
            if (c.hs->status == CR_ERR_BREAKDOWN && c.hs->it == it_start) {
                status = CR_ERR_BREAKDOWN;
                exit_reason = "inner FP32 PCG broke down in its first iteration (p.Gp <= 0 or NaN)";
                break;
            }
            k_add32<<<gn, kBlock, 0, c.st>>>(c.n, h->x64, h->x32);
            ++c.launches;
            CR_CUDA(cudaGetLastError());
            ++outer;
        }
        if (trace) std::fprintf(stderr, "[crhyb] fp32 refinement exit: %s\n", exit_reason);
        if (status != CR_OK) why = exit_reason;
    } else {
        // GMRES in FP32 (or BF16 values) inside FP64 iterative refinement
        const bool bf = o->prec == CR_PREC_MIXED_BF16;
        if ((bf && !h->val16) || (!bf && !h->val32))
            return fail(CR_ERR_ARG, "cr_solve: the values for this precision were not kept by cr_hybridise");
        const double itol = o->inner_tol > 0 ? o->inner_tol : 1e-4;
        double last = -1.0;
        for (;;) {
            k_residual64<D><<<ggrid, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, b, h->x64, h->r64, h->r32, h->minv64,
                                                        c.sc, h->red, 0, o->tol, 0.0);
            ++c.launches;
            CR_CUDA(cudaGetLastError());
            CR_TRY(read_scal(c));
            const double rel2 = c.hs->obb > 0 ? c.hs->orr / c.hs->obb : 0.0;
            if (!std::isfinite(rel2)) { status = CR_ERR_BREAKDOWN; break; }
            if (rel2 <= o->tol * o->tol) break;
            if (outer >= max_outer || c.hs->it >= gmax) { status = CR_ERR_NOT_CONVERGED; break; }
            if (last >= 0.0 && rel2 > 100.0 * last) { status = CR_ERR_BREAKDOWN; break; }
            last = rel2;
            const int it_start = c.hs->it;
            k_inner_start<float><<<gn, kBlock, 0, c.st>>>(c.n, h->x32, h->r32, nullptr, h->minv32, c.sc, h->red, itol);
            ++c.launches;
            CR_CUDA(cudaMemcpyAsync(h->q32, h->r32, sizeof(float) * c.n, cudaMemcpyDeviceToDevice, c.st));
            CR_CUDA(cudaGetLastError());
            if (bf) CR_TRY((gmres_loop<D, __nv_bfloat16, float>(c, h->val16, h->minv32, h->q32, h->x32, h->r32, h->V32, h->Z32)));
            else CR_TRY((gmres_loop<D, float, float>(c, h->val32, h->minv32, h->q32, h->x32, h->r32, h->V32, h->Z32)));
            CR_TRY(read_scal(c));
            if (c.hs->status == CR_ERR_BREAKDOWN && c.hs->it == it_start) { status = CR_ERR_BREAKDOWN; break; }
            k_add32<<<gn, kBlock, 0, c.st>>>(c.n, h->x64, h->x32);
            ++c.launches;
            CR_CUDA(cudaGetLastError());
            ++outer;
        }
    }
    CR_TRY(read_scal(c));
    const int iters = c.hs->it;
    // W = x; final FP64 residual of the returned W
    CR_CUDA(cudaMemcpyAsync(W, h->x64, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.st));
    k_residual64<D><<<ggrid, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, b, h->x64, nullptr, nullptr, h->minv64, c.sc,
                                                h->red, 0, o->tol, 0.0);
    ++c.launches;
    CR_CUDA(cudaGetLastError());
    CR_TRY(read_scal(c));
    const double relres = c.hs->obb > 0 ? std::sqrt(c.hs->orr / c.hs->obb) : 0.0;
    // CR_OK means the FP64 true residual of the returned W meets the tolerance
    if (status == CR_OK && !(relres <= o->tol)) status = CR_ERR_NOT_CONVERGED;
    if (st) {
        st->iterations = iters;
        st->outer = outer;
        st->relres = relres;
        st->status = status;
        st->spmv_launches = h->prof_n;
        st->spmv_ms = h->prof_ms;
        st->kernel_launches = c.launches;
    }
    const std::string detail = why.empty() ? std::string() : " [" + why + "]";
    if (status == CR_ERR_NOT_CONVERGED)
        return fail(status, "cr_solve: iteration limit reached before the tolerance" + detail);
    if (status == CR_ERR_BREAKDOWN)
        return fail(status, "cr_solve: Krylov breakdown or divergence (p.Gp <= 0, NaN, zero Arnoldi vector, "
                            "or the low-precision values made the iteration diverge)" + detail);
    return status;
}

// Flexible GMRES(m) (Saad, Algorithm 9.6) on the steady coupled system
// K_s [U; P] = [R; 0] (Eq. 10 with mu = 0), right-preconditioned by the
// transient Stokes step of `pre` (mu_pre > 0): z = K_mu^{-1} [v; g] is one
// hybridised solve (PCG on G_mu to inner_tol, FP64 or float-float: the
// persistent Jacobi-PCG, or the Chebyshev-preconditioned PCG)
// whose right-hand side is the previous level v / (mu m) with no source and
// the divergence g per simplex, followed by the element-wise recovery.  The Arnoldi vectors, the minimised
// residual and the update x += Z y are those of K_s, so the result is the
// steady solution whatever the inner solves return; only the number of
// steps depends on them (on divergence-free fields K_s K_mu^{-1} has the
// eigenvalues lambda / (lambda + mu), lambda those of the steady operator).
template <int D>
int solve_steady(cr_coupled* cpl, cr_mesh* m, cr_hybrid* pre, int rhs, const cr_solve_opts* o, double* U, double* P,
                 cr_solve_stats* st, double* res0 = nullptr) {
    const int64_t N = m->nf * D, ne = m->ne, n = N + ne;
    const cudaStream_t s = m->stream;
    const int mr = o->restart > 0 ? o->restart : 30;
    SteadyWork& w = pre->steady;
    if (w.m < mr || w.n != n) {
        w.release();
        CR_TRY(w.arena.alloc_n(&w.V, size_t(mr + 1) * n));
        CR_TRY(w.arena.alloc_n(&w.Z, size_t(mr) * n));
        CR_TRY(w.arena.alloc_n(&w.x, size_t(n)));
        CR_TRY(w.arena.alloc_n(&w.b, size_t(n)));
        CR_TRY(w.arena.alloc_n(&w.r, size_t(n)));
        CR_TRY(w.arena.alloc_n(&w.up, size_t(N)));
        CR_TRY(w.arena.alloc_n(&w.mass, size_t(N)));
        CR_TRY(w.arena.alloc_n(&w.W, size_t(N)));
        CR_TRY(w.arena.alloc_n(&w.S, size_t(N)));
        CR_TRY(w.arena.alloc_n(&w.spart, size_t(2) * N));
        CR_TRY(w.arena.alloc(&w.scal, sizeof(KScal)));
        CR_TRY(w.arena.alloc_n(&w.red.partial, size_t(kRedSlots) * kMaxRedBlocks));
        CR_TRY(w.arena.alloc_n(&w.red.count, 1));
        CR_CUDA(cudaMemsetAsync(w.red.count, 0, sizeof(unsigned), s));
        CR_CUDA(cudaMallocHost(&w.h_scal, sizeof(KScal)));
        w.m = mr;
        w.n = n;
    }
    Ctx c{pre, s, static_cast<KScal*>(w.scal), static_cast<KScal*>(w.h_scal), m->nf, n, D, false};
    Ctx cp{pre, s, static_cast<KScal*>(pre->scal), static_cast<KScal*>(pre->h_scal), m->nf, N, D, false};
    const int g = grid_for(n), gN = grid_for(N);
    const int mode = persistent_mode(o->prec);
    const double itol = o->inner_tol > 0 && o->inner_tol < 1 ? o->inner_tol : 1e-6;
    // the multi-kernel inner PCG: Chebyshev-preconditioned, or deflated (a space of G_mu serves
    // every inner solve: G_mu does not change across the outer steps)
    const bool cheb_inner = o->precond == CR_PRECOND_CHEBYSHEV || o->deflation;
    const int gmax = o->max_iter > 0 ? o->max_iter : 1000;
    const int per_launch = (o->check_every > 0 ? o->check_every : 16) * 64;
    const double mu = pre->s->mu;
    std::memset(c.hs, 0, sizeof(KScal));
    c.hs->max_it = gmax;
    c.hs->m = mr;
    CR_CUDA(cudaMemcpyAsync(c.sc, c.hs, sizeof(KScal), cudaMemcpyHostToDevice, s));
    CR_TRY(launch_face_mass(m, w.mass, s));
    CR_TRY(launch_coupled_rhs(cpl, rhs, w.b, s));
    if (o->use_x0) {
        CR_CUDA(cudaMemcpyAsync(w.x, U, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        CR_CUDA(cudaMemcpyAsync(w.x + N, P, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
    } else {
        CR_CUDA(cudaMemsetAsync(w.x, 0, sizeof(double) * n, s));
    }
    // tol2 = tol^2 ||[R; 0]||^2
    k_sumsq<<<g, kBlock, 0, s>>>(n, w.b, c.sc, w.red, 1);
    ++c.launches;
    CR_CUDA(cudaGetLastError());
    CR_TRY(read_scal(c));
    const double bb = c.hs->obb;
    c.hs->tol2 = o->tol * o->tol * bb;
    CR_CUDA(cudaMemcpyAsync(&c.sc->tol2, &c.hs->tol2, sizeof(double), cudaMemcpyHostToDevice, s));
    int64_t inner_its = 0, prof_it = 0;
    double prof_ms = 0.0;
    int status = CR_OK;
    int first_inner = -1, inner_cap = 200000;
    bool first_cycle = true;
    if (res0) *res0 = 0.0;
    if (bb > 0.0) {
        for (;;) {
            CR_TRY(launch_coupled_apply(cpl, w.x, w.b, w.r, s));   // r = b - K x
            k_gm_norm_start<double><<<g, kBlock, 0, s>>>(n, w.r, c.sc, w.red);
            k_gm_scale_v0<double><<<g, kBlock, 0, s>>>(n, w.r, w.V, c.sc);
            c.launches += 3;
            CR_CUDA(cudaGetLastError());
            CR_TRY(read_scal(c));
            if (res0 && first_cycle) *res0 = std::sqrt(c.hs->rr / bb);
            first_cycle = false;
            if (c.hs->done) break;
            for (int j = 0; j < mr; ++j) {
                double* z = w.Z + size_t(j) * n;
                // z_j = K_mu^{-1} [v_j; 0]: previous level, S, inner PCG, recovery
                k_prev_from_residual<<<gN, kBlock, 0, s>>>(N, w.V + size_t(j) * n, w.mass, mu, w.up);
                ++c.launches;
                const double* gdiv = w.V + size_t(j) * n + N;   // the divergence block of v_j
                CR_TRY(launch_rhs_previous(pre, w.up, gdiv, w.spart, w.S, s));
                c.launches += 2;
                // an inner solve that stagnates above inner_tol (its attainable accuracy) stops at
                // four times the first one's iterations; the flexible outer step takes what it returns
                int inner_it = 0, inner_status = CR_OK;
                if (cheb_inner) {
                    // Chebyshev-preconditioned or deflated PCG (multi-kernel, graph-replayed) on G_mu
                    cr_solve_opts io = *o;
                    io.method = CR_METHOD_PCG;
                    io.tol = itol;
                    io.max_iter = inner_cap;
                    io.use_x0 = 0;
                    io.use_graph = o->profile ? 0 : 1;
                    io.persistent = 0;
                    io.inner_tol = 0.0;
                    cr_solve_stats ist{};
                    const int rc = solve_dim<D>(pre, 0, &io, w.W, &ist, w.S);
                    if (rc != CR_OK && rc != CR_ERR_NOT_CONVERGED && rc != CR_ERR_BREAKDOWN) return rc;
                    inner_it = ist.iterations;
                    inner_status = ist.status;
                    cp.launches += ist.kernel_launches;
                    prof_ms += ist.spmv_ms;
                    prof_it += ist.spmv_launches;
                } else {
                    PScal Pst{};
                    double kms = 0.0;
                    int64_t kit = 0;
                    CR_TRY(persistent_pcg<D>(cp, w.S, nullptr, w.W, mode, itol, default_delta(mode), inner_cap,
                                             per_launch, o->profile != 0, &Pst, &kms, &kit));
                    inner_it = Pst.it;
                    inner_status = Pst.status;
                    prof_ms += kms;
                    prof_it += kit;
                }
                if (first_inner < 0) {
                    first_inner = inner_it;
                    inner_cap = int(std::min<int64_t>(int64_t(4) * std::max(first_inner, 64), 1000000));
                }
                inner_its += inner_it;
                if (inner_status == CR_ERR_BREAKDOWN) { status = CR_ERR_BREAKDOWN; break; }
                CR_TRY(launch_recover_previous(pre, w.up, gdiv, w.W, z, z + N, s));
                ++c.launches;
                // v_{j+1} = K_s z_j, orthogonalised (CGS2) and normalised
                CR_TRY(launch_coupled_apply(cpl, z, nullptr, w.V + size_t(j + 1) * n, s));
                ++c.launches;
                for (int pass = 0; pass < 2; ++pass) {
                    for (int i0 = 0; i0 <= j; i0 += kRedSlots) {
                        k_gm_dots<double><<<g, kBlock, 0, s>>>(n, w.V, i0, c.sc, w.red);
                        ++c.launches;
                    }
                    k_gm_orth<double><<<g, kBlock, 0, s>>>(n, w.V, c.sc, w.red, pass);
                    ++c.launches;
                }
                k_gm_normalise<double><<<g, kBlock, 0, s>>>(n, w.V, c.sc);
                ++c.launches;
                CR_CUDA(cudaGetLastError());
                CR_TRY(read_scal(c));
                if (c.hs->done || c.hs->stop) break;
            }
            if (status != CR_OK) break;
            k_gm_solve_y<<<1, 32, 0, s>>>(c.sc);
            k_fgm_update<<<g, kBlock, 0, s>>>(n, w.x, w.Z, c.sc);
            c.launches += 2;
            CR_CUDA(cudaGetLastError());
            CR_TRY(read_scal(c));
            if (c.hs->status != CR_OK) break;
        }
    }
    c.launches += cp.launches;
    CR_TRY(read_scal(c));
    if (status == CR_OK) status = c.hs->status;
    const int steps = c.hs->it;
    // U, P and the FP64 residual of the coupled system they satisfy
    CR_CUDA(cudaMemcpyAsync(U, w.x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    CR_CUDA(cudaMemcpyAsync(P, w.x + N, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
    CR_TRY(launch_coupled_apply(cpl, w.x, w.b, w.r, s));
    k_sumsq<<<g, kBlock, 0, s>>>(n, w.r, c.sc, w.red, 0);
    c.launches += 2;
    CR_CUDA(cudaGetLastError());
    CR_TRY(read_scal(c));
    const double relres = bb > 0.0 ? std::sqrt(c.hs->orr / bb) : 0.0;
    if (status == CR_OK && !(relres <= o->tol)) status = CR_ERR_NOT_CONVERGED;
    if (st) {
        st->iterations = int32_t(inner_its);
        st->outer = steps;
        st->relres = relres;
        st->status = status;
        st->spmv_launches = int32_t(prof_it);
        st->spmv_ms = prof_ms;
        st->kernel_launches = c.launches;
    }
    if (status == CR_ERR_NOT_CONVERGED) return fail(status, "cr_solve_steady: step limit reached before the tolerance");
    if (status == CR_ERR_BREAKDOWN)
        return fail(status, "cr_solve_steady: breakdown (zero Arnoldi vector, NaN, or p.Gp <= 0 in an inner PCG)");
    return status;
}

// sc->orr = sum (a - b)^2, sc->obb = sum a^2
__global__ void __launch_bounds__(kBlock) k_diff_sumsq(int64_t n, const double* __restrict__ a,
                                                     const double* __restrict__ b, KScal* sc, RedBuf red) {
    double part[2] = {0.0, 0.0};
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const double d = a[k] - b[k];
        part[0] += d * d;
        part[1] += a[k] * a[k];
    }
    double tot[2];
    if (grid_sum<2>(part, red, tot) && threadIdx.x == 0) {
        sc->orr = tot[0];
        sc->obb = tot[1];
    }
}

// Newton's method for the steady Navier-Stokes problem (Section 3.1 with
// b_h != 0, mu = 0): from U_0 (the caller's U), step k solves the steady
// coupled system linearised about w = U_k (the Newton Jacobian and its
// right-hand side R + c_K(w), cr_assemble_coupled with conv = NEWTON) by
// cr_solve_steady's flexible GMRES from [U_k; P_k], whose first residual is
// the nonlinear residual at (U_k, P_k); the solution is U_{k+1}.  It stops
// when ||U_{k+1} - U_k|| <= newton_tol ||U_{k+1}||.
template <int D>
int solve_newton(cr_mesh* m, double nu, const double* fbar, cr_hybrid* pre, const cr_solve_opts* lin, double ntol,
                 int maxn, double* U, double* P, cr_newton_stats* st) {
    const int64_t N = m->nf * D, ne = m->ne;
    const cudaStream_t s = m->stream;
    DevArena tmp;
    double *Un = nullptr, *Pn = nullptr;
    CR_TRY(tmp.alloc_n(&Un, size_t(N)));
    CR_TRY(tmp.alloc_n(&Pn, size_t(ne)));
    cr_solve_opts o = *lin;
    o.use_x0 = 1;
    int status = CR_ERR_NOT_CONVERGED, k = 0, steps = 0;
    int64_t inner = 0;
    double incr = 0.0, res_first = 0.0;
    for (; k < maxn;) {
        cr_params p{nu, 0.0, CR_CONV_NEWTON, 0.0};
        cr_system* sys = nullptr;
        int rc = cr_assemble_coupled(m, &p, fbar, 1, U, &sys, nullptr);
        if (rc != CR_OK) { tmp.release(); return rc; }
        rc = coupled_build(sys, &sys->steady_op, false);
        cr_solve_stats lst{};
        double res0 = 0.0;
        if (rc == CR_OK) {
            CR_CUDA(cudaMemcpyAsync(Un, U, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
            CR_CUDA(cudaMemcpyAsync(Pn, P, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
            rc = solve_steady<D>(sys->steady_op, m, pre, 0, &o, Un, Pn, &lst, &res0);
        }
        cr_destroy_system(sys);
        ++k;
        steps += lst.outer;
        inner += lst.iterations;
        if (k == 1) res_first = res0;
        if (rc != CR_OK) { status = rc; break; }
        // the increment, then U_{k+1}, P_{k+1}
        SteadyWork& w = pre->steady;
        Ctx c{pre, s, static_cast<KScal*>(w.scal), static_cast<KScal*>(w.h_scal), m->nf, N, D, false};
        k_diff_sumsq<<<grid_for(N), kBlock, 0, s>>>(N, Un, U, c.sc, w.red);
        CR_CUDA(cudaGetLastError());
        CR_TRY(read_scal(c));
        incr = c.hs->obb > 0.0 ? std::sqrt(c.hs->orr / c.hs->obb) : 0.0;
        CR_CUDA(cudaMemcpyAsync(U, Un, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        CR_CUDA(cudaMemcpyAsync(P, Pn, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
        if (!std::isfinite(incr)) { status = CR_ERR_BREAKDOWN; break; }
        if (incr <= ntol) { status = CR_OK; break; }
    }
    // the nonlinear residual at the returned (U, P): the Newton system linearised about U
    // evaluated at [U; P] (b_h is quadratic: J(U) U - c(U) = b_h(U, U))
    double resid = 0.0;
    {
        cr_params p{nu, 0.0, CR_CONV_NEWTON, 0.0};
        cr_system* sys = nullptr;
        int rc = cr_assemble_coupled(m, &p, fbar, 1, U, &sys, nullptr);
        if (rc == CR_OK) rc = coupled_build(sys, &sys->steady_op, false);
        if (rc == CR_OK) {
            SteadyWork& w = pre->steady;
            Ctx c{pre, s, static_cast<KScal*>(w.scal), static_cast<KScal*>(w.h_scal), m->nf, N + ne, D, false};
            CR_CUDA(cudaMemcpyAsync(w.x, U, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
            CR_CUDA(cudaMemcpyAsync(w.x + N, P, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
            rc = launch_coupled_rhs(sys->steady_op, 0, w.b, s);
            if (rc == CR_OK) rc = launch_coupled_apply(sys->steady_op, w.x, w.b, w.r, s);
            if (rc == CR_OK) {
                k_sumsq<<<grid_for(N + ne), kBlock, 0, s>>>(N + ne, w.r, c.sc, w.red, 0);
                k_sumsq<<<grid_for(N + ne), kBlock, 0, s>>>(N + ne, w.b, c.sc, w.red, 1);
                CR_CUDA(cudaGetLastError());
                CR_TRY(read_scal(c));
                resid = c.hs->obb > 0.0 ? std::sqrt(c.hs->orr / c.hs->obb) : 0.0;
            }
        }
        cr_destroy_system(sys);
        if (rc != CR_OK) { tmp.release(); return rc; }
    }
    CR_CUDA(cudaStreamSynchronize(s));
    tmp.release();
    if (st) {
        st->iterations = k;
        st->linear_steps = steps;
        st->inner_iterations = inner;
        st->increment = incr;
        st->residual = resid;
        st->first_residual = res_first;
        st->status = status;
    }
    if (status == CR_ERR_NOT_CONVERGED)
        return fail(status, "cr_solve_newton: Newton iteration limit reached before the increment tolerance");
    if (status != CR_OK) return status;
    return CR_OK;
}

}  // namespace

size_t kscal_bytes() { return sizeof(KScal); }

int launch_spmv64(cr_hybrid* h, const double* x, double* y, cudaStream_t st) {
    const int g = grid_for(h->m->nf);
    if (h->m->d == 2) k_spmv64<2><<<g, kBlock, 0, st>>>(h->m->nf, h->m->cols, h->val64, x, y);
    else k_spmv64<3><<<g, kBlock, 0, st>>>(h->m->nf, h->m->cols, h->val64, x, y);
    CR_CUDA(cudaGetLastError());
    return CR_OK;
}

int solve_fgmres_impl(cr_hybrid* h, int rhs, cr_hybrid* pre, const cr_solve_opts* o, double* Wdev,
                      cr_solve_stats* st) {
    return h->m->d == 2 ? solve_fgmres<2>(h, rhs, pre, o, Wdev, st) : solve_fgmres<3>(h, rhs, pre, o, Wdev, st);
}

int solve_steady_impl(cr_coupled* c, cr_mesh* m, cr_hybrid* pre, int rhs, const cr_solve_opts* o, double* U,
                      double* P, cr_solve_stats* st) {
    return m->d == 2 ? solve_steady<2>(c, m, pre, rhs, o, U, P, st) : solve_steady<3>(c, m, pre, rhs, o, U, P, st);
}

int solve_newton_impl(cr_mesh* m, double nu, const double* fbar, cr_hybrid* pre, const cr_solve_opts* lin, double ntol,
                      int maxn, double* U, double* P, cr_newton_stats* st) {
    return m->d == 2 ? solve_newton<2>(m, nu, fbar, pre, lin, ntol, maxn, U, P, st)
                     : solve_newton<3>(m, nu, fbar, pre, lin, ntol, maxn, U, P, st);
}

int solve_impl(cr_hybrid* h, int rhs, const cr_solve_opts* o, double* Wdev, cr_solve_stats* st) {
    if (o->persistent && o->method == CR_METHOD_PCG && o->precond == CR_PRECOND_JACOBI && !o->deflation &&
        (o->prec == CR_PREC_FP64 || o->prec == CR_PREC_FF || o->prec == CR_PREC_FF_BF16))
        return h->m->d == 2 ? solve_persistent<2>(h, rhs, o, Wdev, st) : solve_persistent<3>(h, rhs, o, Wdev, st);
    return h->m->d == 2 ? solve_dim<2>(h, rhs, o, Wdev, st) : solve_dim<3>(h, rhs, o, Wdev, st);
}

// A deflation space of Ritz vectors from the Lanczos data of a PCG run: T with
// diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1} and off-diagonal -sqrt(beta_j)/alpha_j
// (j < mm = alpha.size(); Saad, Iterative Methods for Sparse Linear Systems, Section
// 6.7.3), its k smallest eigenpairs on the host, Y = Q S on the device (Q: the mm
// FP32 vectors q_j), then the space (defl_build).  theta [k] gets the Ritz values of
// the vectors kept (0 after them).
int ritz_space(cr_hybrid* h, const float* Q, const std::vector<double>& alpha, const std::vector<double>& beta, int k,
               double* theta, cr_deflation** out, cudaStream_t st) {
    const int mm = int(alpha.size());
    const int64_t n = h->m->nf * h->m->d;
    std::vector<double> ta(mm), tb(mm > 1 ? mm - 1 : 0);
    for (int j = 0; j < mm; ++j) {
        ta[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
        if (j + 1 < mm) tb[j] = -std::sqrt(beta[j]) / alpha[j];
    }
    std::vector<double> th, S;
    tridiag_smallest_eigen(ta, tb, k, th, S);
    const int kk = int(th.size());
    struct Tmp {
        DevArena a;
        ~Tmp() { a.release(); }
    } tmp;
    std::vector<float> S32(S.begin(), S.end());
    float* Sd = nullptr;
    CR_TRY(tmp.a.alloc_n(&Sd, S32.size()));
    CR_CUDA(cudaMemcpyAsync(Sd, S32.data(), sizeof(float) * S32.size(), cudaMemcpyHostToDevice, st));
    CR_CUDA(cudaStreamSynchronize(st));   // S32 is a host temporary
    cr_deflation* d = nullptr;
    CR_TRY(defl_alloc(h, kk, &d));
    CR_TRY(ritz_vectors(n, mm, kk, Q, Sd, d->V64, st));
    CR_CUDA(cudaGetLastError());
    int rc = defl_build(d, h, st);
    if (rc != CR_OK) {
        d->arena.release();
        delete d;
        return rc;
    }
    for (int a = 0; a < k; ++a) theta[a] = a < d->k ? th[d->kept[a]] : 0.0;
    *out = d;
    return CR_OK;
}

// Ritz vectors for a deflation space from m steps of FP64 PCG (Jacobi or Chebyshev,
// as opts says) on right-hand side rhs from x = 0: the normalised preconditioned
// residuals q_j = z_j / sqrt(r_j.z_j) are stored in FP32, the Lanczos matrix T (its
// diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal -sqrt(beta_j)/alpha_j
// from the CG coefficients; Saad, Iterative Methods for Sparse Linear Systems,
// Section 6.7.3) gives its k smallest eigenpairs on the host, and Y = Q S.  One
// iteration per launch sequence, its coefficients read back after each.
template <int D>
int lanczos_dim(cr_hybrid* h, int rhs, const cr_solve_opts* o, int mmax, int k, double* theta,
                cr_deflation** out) {
    cr_mesh* m = h->m;
    Ctx c{h, m->stream, static_cast<KScal*>(h->scal), static_cast<KScal*>(h->h_scal), m->nf, m->nf * D, D, false};
    const double* b = h->S + size_t(rhs) * c.n;
    const int ggrid = grid_for(c.nf), gn = grid_for(c.n);
    std::memset(c.hs, 0, sizeof(KScal));
    c.hs->max_it = 1 << 30;
    const bool cheb = o->precond == CR_PRECOND_CHEBYSHEV;
    if (cheb) CR_TRY(chebyshev_setup<D>(h, o, c.st, c.hs));
    CR_CUDA(cudaMemcpyAsync(c.sc, c.hs, sizeof(KScal), cudaMemcpyHostToDevice, c.st));
    CR_CUDA(cudaMemsetAsync(h->x64, 0, sizeof(double) * c.n, c.st));
    struct Tmp {
        DevArena a;
        ~Tmp() { a.release(); }
    } tmp;
    float* Q = nullptr;
    CR_TRY(tmp.a.alloc_n(&Q, size_t(mmax) * size_t(c.n)));
    // r = b with r.M^{-1}r; tolerance 0: the flag stays down unless r is exactly zero
    k_residual64<D><<<ggrid, kBlock, 0, c.st>>>(c.nf, m->cols, h->val64, b, nullptr, h->r64, nullptr, h->minv64, c.sc,
                                                h->red, 1, 0.0, 0.0);
    const int deg = o->poly_degree > 0 ? o->poly_degree : 4;
    double* zb[2] = {h->cheb, h->cheb ? h->cheb + c.n : nullptr};
    double* dv = h->cheb ? h->cheb + 2 * c.n : nullptr;
    auto cheb_steps = [&]() {
        for (int j = 1; j < deg; ++j)
            k_cheb_step<D><<<grid_occ(k_cheb_step<D>, c.nf), kBlock, 0, c.st>>>(
                c.nf, m->cols, h->val64, h->minv64, h->r64, zb[(j - 1) & 1], zb[j & 1], dv, c.sc, h->red, j,
                j == deg - 1);
    };
    const double* zcur = cheb ? zb[(deg - 1) & 1] : nullptr;   // null: z = M^{-1} r
    if (cheb) {
        k_cheb_start<<<gn, kBlock, 0, c.st>>>(c.n, h->r64, h->minv64, zb[0], dv, c.sc);
        cheb_steps();
        k_cpcg_dir<<<gn, kBlock, 0, c.st>>>(c.n, h->p64, zb[(deg - 1) & 1], c.sc, 1);
    } else {
        k_pcg_dir<double><<<gn, kBlock, 0, c.st>>>(c.n, h->p64, h->r64, h->minv64, c.sc, 1);
    }
    CR_CUDA(cudaGetLastError());
    CR_TRY(read_scal(c));
    if (c.hs->done || !(c.hs->rz > 0.0)) return fail(CR_ERR_ARG, "cr_deflation_lanczos: zero right-hand side");
    CR_TRY(lanczos_store(c.n, zcur, h->minv64, h->r64, &c.sc->rz, Q, c.st));
    std::vector<double> alpha, beta;
    for (int j = 0; j < mmax; ++j) {
        if (cheb) {
            k_pcg_spmv<D, double, double><<<grid_occ(k_pcg_spmv<D, double, double>, c.nf), kBlock, 0, c.st>>>(
                c.nf, m->cols, h->val64, h->p64, h->q64, c.sc, h->red);
            k_cpcg_update<<<gn, kBlock, 0, c.st>>>(c.n, h->x64, h->r64, h->p64, h->q64, h->minv64, zb[0], dv, c.sc,
                                                   h->red);
            cheb_steps();
            k_cpcg_dir<<<gn, kBlock, 0, c.st>>>(c.n, h->p64, zb[(deg - 1) & 1], c.sc, 0);
        } else {
            pcg_iteration<D, double, double>(c, h->val64, h->minv64, h->x64, h->r64, h->p64, h->q64, nullptr,
                                             nullptr);
        }
        CR_CUDA(cudaGetLastError());
        CR_TRY(read_scal(c));
        if (c.hs->status == CR_ERR_BREAKDOWN || !(c.hs->alpha > 0.0) || !std::isfinite(c.hs->alpha)) break;
        alpha.push_back(c.hs->alpha);
        beta.push_back(c.hs->beta);
        if (c.hs->done || !(c.hs->rz > 0.0) || !std::isfinite(c.hs->beta)) break;   // r = 0: the space is exact
        if (j + 1 < mmax) CR_TRY(lanczos_store(c.n, zcur, h->minv64, h->r64, &c.sc->rz, Q + size_t(j + 1) * c.n, c.st));
    }
    if (alpha.empty()) return fail(CR_ERR_BREAKDOWN, "cr_deflation_lanczos: the first CG step broke down");
    return ritz_space(h, Q, alpha, beta, k, theta, out, c.st);
}

// cr_solve on the multi-kernel path with the Lanczos record of its first m
// iterations, then the space of k Ritz vectors from it.
template <int D>
int solve_ritz_dim(cr_hybrid* h, int rhs, const cr_solve_opts* o, double* W, cr_solve_stats* st, int m, int k,
                   double* theta, cr_deflation** out) {
    const int64_t n = h->m->nf * D;
    cudaStream_t s = h->m->stream;
    struct Tmp {
        DevArena a;
        ~Tmp() { a.release(); }
    } tmp;
    LanczosRec rec;
    rec.m = m;
    CR_TRY(tmp.a.alloc_n(&rec.Q, size_t(m) * size_t(n)));
    CR_TRY(tmp.a.alloc_n(&rec.ab, size_t(2) * m));
    CR_TRY(tmp.a.alloc_n(&rec.count, 2));
    rec.stop = rec.count + 1;
    CR_CUDA(cudaMemsetAsync(rec.count, 0, 2 * sizeof(int), s));
    const int rc = solve_dim<D>(h, rhs, o, W, st, nullptr, &rec);
    if (rc != CR_OK && rc != CR_ERR_NOT_CONVERGED) return rc;
    int cnt = 0;
    std::vector<double> ab(size_t(2) * m);
    CR_CUDA(cudaMemcpyAsync(&cnt, rec.count, sizeof(int), cudaMemcpyDeviceToHost, s));
    CR_CUDA(cudaMemcpyAsync(ab.data(), rec.ab, sizeof(double) * ab.size(), cudaMemcpyDeviceToHost, s));
    CR_CUDA(cudaStreamSynchronize(s));
    // q_0 .. q_{cnt-1} and the steps between them: alpha_j, beta_j for j < cnt - 1, and
    // T of size cnt - 1 (the last vector closes no step)
    const int mm = cnt - 1;
    if (mm < 1) return fail(CR_ERR_ARG, "cr_solve_ritz: the solve ended before its first CG step");
    std::vector<double> alpha(ab.begin(), ab.begin() + mm), beta(ab.begin() + m, ab.begin() + m + mm);
    const int rs = ritz_space(h, rec.Q, alpha, beta, k, theta, out, s);
    return rs != CR_OK ? rs : rc;
}

int solve_ritz_impl(cr_hybrid* h, int rhs, const cr_solve_opts* o, double* W, cr_solve_stats* st, int m, int k,
                    double* theta, cr_deflation** out) {
    return h->m->d == 2 ? solve_ritz_dim<2>(h, rhs, o, W, st, m, k, theta, out)
                        : solve_ritz_dim<3>(h, rhs, o, W, st, m, k, theta, out);
}

int lanczos_impl(cr_hybrid* h, int rhs, const cr_solve_opts* o, int m, int k, double* theta, cr_deflation** out) {
    return h->m->d == 2 ? lanczos_dim<2>(h, rhs, o, m, k, theta, out) : lanczos_dim<3>(h, rhs, o, m, k, theta, out);
}

int cheb_step_form_impl(int d, int poly_prec) { return cheb32_form(d, poly_prec == CR_POLY_BF16); }

void destroy_persistent_plans(cr_hybrid* h) {
    for (void*& p : h->pplan) {
        delete static_cast<PersistPlan*>(p);
        p = nullptr;
    }
}

}  // namespace crhyb
