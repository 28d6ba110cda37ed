// Persistent Jacobi-PCG over a batch of hybridised systems (hybrid method,
// step 2; Section 3.2, item 6: G is symmetric positive definite for mu > 0
// and b_h = 0).
//
// One cooperative launch runs many PCG iterations for a list of systems.  A
// system is one matrix G with up to kPMaxRhs right-hand sides, which share
// every load of G (the SpMV is a block SpMM).  Face rows are cut into tiles of
// one thread block each; the persistent blocks sweep the tile list in every
// phase, and the phases of an iteration are separated by a grid barrier:
//   P1  q = G p and p.q per right-hand side; the block that completes a
//       system's last tile sums the tile partials in tile order and sets alpha;
//   P2  x += alpha p, r -= alpha q, r.M^{-1}r and r.r; the same block sets beta
//       and decides convergence (or that a reliable update is due);
//   P3  p = M^{-1} r + beta p.
// Reliable updates (float-float arithmetic) take three more phases:
//   U1  x64 += x / sigma, x = 0;
//   U2  r64 = b - G x64 in FP64 with the FP64 values; r.r, b.b, r.M^{-1}r;
//       new scale sigma = 1/||r64||, beta continues the search direction;
//   U3  r = sigma r64 (float-float), p = M^{-1} r + beta p.
// The same update phases start every solve (from x64 = x0, beta = 0) and end
// it: convergence is always decided on the FP64 true residual of the iterate.
// In plain FP64 arithmetic U1 has nothing to do and U2 writes r itself.
//
// Every barrier wait is bounded: a wait that runs out sets an error flag,
// after which every block returns; the host reports CR_ERR_TIMEOUT.  Loop
// decisions are taken from a snapshot of the control counters that the block
// releasing the barrier at the end of an iteration (P3, U3) writes, so that
// every block takes the same branch.

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "ff.cuh"
#include "persist.h"

namespace crhyb {
namespace {

// Build knobs (defaults are the measured best on cfg2): blocks per SM the
// register allocation aims at for single-right-hand-side d = 2 kernels, and
// how d = 2 tiles reach the SpMV phase: 0 per-thread loads, 1 one shared-memory
// stage per block filled by TMA bulk copies, 2 two stages (the next tile is
// copied in while the current one is computed).  Staging (two 45 KB
// stages per block) limits a block of 256 threads to 2 per SM; measured per
// iteration on cfg2 (float-float): 95.6 us staged at 2 blocks/SM against
// 75.4 us with per-thread coalesced loads at 3 blocks/SM, the update and
// direction phases losing more to the lower occupancy than the SpMV phase gains.
#ifndef CRHYB_PERSIST_MINB
#define CRHYB_PERSIST_MINB 3
#endif
#ifndef CRHYB_STAGE_D2
#define CRHYB_STAGE_D2 0
#endif
// blocks per SM the register allocation of the two- and four-right-hand-side kernels aims at
// (measured on the 64-mesh batch: 3 for R = 2, 1.52 s against 1.82 s at 2)
#ifndef CRHYB_R2_MINB
#define CRHYB_R2_MINB 3
#endif
#ifndef CRHYB_R4_MINB
#define CRHYB_R4_MINB 2
#endif
// blocks per SM of the 3D one-right-hand-side kernel, FP64 and float-float apart
#ifndef CRHYB_3D_MINB
#define CRHYB_3D_MINB 3
#endif
#ifndef CRHYB_3D_FF_MINB
#define CRHYB_3D_FF_MINB 2
#endif
// SpMV phase with per-thread loads: how many tiles ahead of the sweep one
// thread of the block asks L2 to fetch the tile's values and columns (bulk L2
// prefetch, no completion to wait for); 0 turns it off.
#ifndef CRHYB_L2_PREFETCH
#define CRHYB_L2_PREFETCH 0
#endif

constexpr int kPBlock = 256;   // rows per tile = threads per block
static_assert(kPBlock == kSlice, "a tile is one slice of the sliced ELL");
constexpr long long kSpinLimit = 1ll << 22;   // bounded barrier wait (about 0.3-1 s with the sleeps)

enum PMode { kModeFP64 = 0, kModeFF32 = 1, kModeFFBF16 = 2 };

__device__ __forceinline__ int ld_vol(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Per-pair scalars are written during the kernel by the block that completes
// a system's last tile: read them from L2 (the L1 of another SM may be stale).
__device__ __forceinline__ int sc_i(const int& v) { return __ldcg(&v); }
__device__ __forceinline__ double sc_d(const double& v) { return __ldcg(&v); }
__device__ __forceinline__ float2 sc_f2(const float2& v) { return __ldcg(&v); }

// The d components of a face are adjacent: in 2D one 16-byte access moves both
// (float-float pairs or FP64 values; the arrays are 16-byte aligned).
//
// Vectors written by other blocks in an earlier phase (the gathered p, x64)
// are read with ordinary coherent loads, which may hit in L1: the grid barrier
// orders them after those writes (release by the writers' fence and atomic,
// acquire by the waiting thread's fence, then bar.sync for its block), the
// same ordering a cooperative-groups grid sync gives.  Only the non-coherent
// read-only path (ld.global.nc) would be unsafe here, and it is not used.
__device__ __forceinline__ void ld2(const float2* p, float2 (&v)[2]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = make_float2(t.x, t.y);
    v[1] = make_float2(t.z, t.w);
}
__device__ __forceinline__ void ld2(const double* p, double (&v)[2]) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x;
    v[1] = t.y;
}
__device__ __forceinline__ void ld2(const float* p, float (&v)[2]) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x;
    v[1] = t.y;
}
__device__ __forceinline__ void ld2cg(const float2* p, float2 (&v)[2]) {
    const float4 t = __ldcg(reinterpret_cast<const float4*>(p));
    v[0] = make_float2(t.x, t.y);
    v[1] = make_float2(t.z, t.w);
}
__device__ __forceinline__ void ld2cg(const double* p, double (&v)[2]) {
    const double2 t = __ldcg(reinterpret_cast<const double2*>(p));
    v[0] = t.x;
    v[1] = t.y;
}
__device__ __forceinline__ void st2(float2* p, const float2 (&v)[2]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
}
__device__ __forceinline__ void st2(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}
template <int D, typename V>
__device__ __forceinline__ void ldrow(const V* p, V (&v)[D]) {
    if constexpr (D == 2) ld2(p, v);
    else
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] = p[j];
}
template <int D, typename V>
__device__ __forceinline__ void ldrow_cg(const V* p, V (&v)[D]) {
    if constexpr (D == 2) ld2cg(p, v);
    else
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] = __ldcg(p + j);
}
template <int D, typename V>
__device__ __forceinline__ void strow(V* p, const V (&v)[D]) {
    if constexpr (D == 2) st2(p, v);
    else
#pragma unroll
        for (int j = 0; j < D; ++j) p[j] = v[j];
}

// Grid barrier with a bounded wait, on one 64-bit word: arrivals in the low
// half, the generation in bits 32-62, an error bit on top.  An arrival's
// atomic returns the generation it waits to see change, and the last arrival
// bumps it and clears the count in one atomic, so a barrier costs one atomic
// round trip per block.  With snap, the last arrival first copies the loop
// control counters, which every block reads at the top of the next iteration.
// A wait that runs out sets the error bit, which ends every other wait.
// Returns false in every block once any wait has run out.
constexpr unsigned long long kBarErr = 1ull << 63;
__device__ __forceinline__ bool pbar(PCtl* ctl, bool snap) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long old = atomicAdd(&ctl->bar, 1ull);
        const unsigned gen = unsigned(old >> 32);
        int ok = (old & kBarErr) == 0;
        if (unsigned(old) == gridDim.x - 1) {
            if (snap) {
                ctl->snap_active = ld_vol(&ctl->active);
                ctl->snap_upd = ld_vol(&ctl->upd);
                __threadfence();
            }
            atomicAdd(&ctl->bar, (1ull << 32) - gridDim.x);
        } else if (ok) {
            const volatile unsigned long long* w = &ctl->bar;
            long long n = 0;
            for (;;) {
                const unsigned long long v = *w;
                if (unsigned(v >> 32) != gen) {
                    if (v & kBarErr) ok = 0;
                    break;
                }
                if (++n > kSpinLimit) {
                    atomicExch(&ctl->err, 1);
                    atomicOr(&ctl->bar, kBarErr);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Phase timing (profile runs only): block 0 adds the time since the previous
// barrier to the phase's total, read from the global nanosecond timer.
__device__ __forceinline__ void phase_mark(const PArgs& a, int phase, unsigned long long& t_last) {
    if (a.phase_ns && blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        a.phase_ns[phase] += t - t_last;
        t_last = t;
    }
}

// Sum of NV doubles over the block (thread 0 gets the totals).
template <int NV>
__device__ __forceinline__ void bsum(double (&v)[NV], double (&out)[NV]) {
    __shared__ double sh[NV * 32];
    block_sum<NV>(v, sh, out);
}

// Float-float block sum, converted to FP64 by thread 0.
template <int NV>
__device__ __forceinline__ void bsum_ff(float2 (&v)[NV], double (&out)[NV]) {
    __shared__ float2 sh[NV * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    auto wred = [&](float2 a) {
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
        const float2 a = wred(v[k]);
        if (lane == 0) sh[k * 32 + warp] = a;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float2 a = wred(lane < nw ? sh[k * 32 + lane] : make_float2(0.f, 0.f));
            if (lane == 0) out[k] = ff_to_double(a);
        }
    }
    __syncthreads();
}

// Block partials -> per-system totals.  Each block sums its rows of system s
// (all of them, over its contiguous tile range) into mine[][]; the block that
// delivers the system's last partial returns true, with tot[k][q] (thread 0)
// the sum of the partials in block order: deterministic, and one atomic per
// block and system.
template <int R, int NQ>
__device__ __forceinline__ bool system_flush(const PArgs& a, const PSys& S, int s, const double (&mine)[R][NQ],
                                             double (&tot)[R][NQ]) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        double* tp = a.tpart + size_t(S.slot0 + int(blockIdx.x) - S.blk0) * kPMaxRhs * 4;
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int q = 0; q < NQ; ++q) tp[k * 4 + q] = mine[k][q];
        __threadfence();
        last = atomicAdd(a.syscnt + s, 1u) == unsigned(S.nblk - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[R * NQ];
#pragma unroll
    for (int k = 0; k < R * NQ; ++k) acc[k] = 0.0;
    for (int u = threadIdx.x; u < S.nblk; u += blockDim.x) {
        const double* src = a.tpart + size_t(S.slot0 + u) * kPMaxRhs * 4;
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[k * NQ + q] += __ldcg(src + k * 4 + q);
    }
    double out[R * NQ];
    bsum<R * NQ>(acc, out);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int q = 0; q < NQ; ++q) tot[k][q] = out[k * NQ + q];
        a.syscnt[s] = 0u;
    }
    return true;
}

// Block sum of per-thread partials (float-float or FP64) into a [R][NQ] FP64 array.
template <int R, int NQ, bool FF>
__device__ __forceinline__ void block_partials(FFAcc (&af)[R][NQ], double (&ad)[R][NQ], double (&out)[R][NQ]) {
    double flat[R * NQ];
    if (FF) {
        float2 v[R * NQ];
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int q = 0; q < NQ; ++q) v[k * NQ + q] = af[k][q].result();
        bsum_ff<R * NQ>(v, flat);
    } else {
        double v[R * NQ];
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int q = 0; q < NQ; ++q) v[k * NQ + q] = ad[k][q];
        bsum<R * NQ>(v, flat);
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
        for (int q = 0; q < NQ; ++q) out[k][q] = flat[k * NQ + q];
}

// ---- row kernels ---------------------------------------------------------

// y_k = G p_k for the right-hand sides in amask, float-float (one face row).
template <int D, int R, typename LT>
__device__ __forceinline__ void ff_row(const PSys& S, int64_t f, unsigned amask, const float2* p,
                                       float2 (&y)[R][D]) {
    constexpr int NS = 2 * D + 1;
    constexpr int NPV = NS * D * D;
    const int64_t N = S.nf * D;
    const float* vh = S.vh;
    const LT* vl = static_cast<const LT*>(S.vl);
    FFAcc acc[R][D];
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
        for (int i = 0; i < D; ++i) acc[k][i].zero();
#pragma unroll(R == 1 ? NS : 1)
    for (int s = 0; s < NS; ++s) {
        const int64_t c = s == 0 ? f : int64_t(__ldcs(S.cols + sell(f, s - 1, 2 * D)));
        float h[D][D], l[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const size_t idx = sell(f, (s * D + i) * D + j, NPV);
                hl_val(vh, vl, idx, h[i][j], l[i][j]);
            }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (!((amask >> k) & 1u)) continue;
            float2 xv[D];
            ldrow<D>(p + k * N + c * D, xv);
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) acc[k][i].mad(h[i][j], l[i][j], xv[j].x, xv[j].y);
        }
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
        for (int i = 0; i < D; ++i) y[k][i] = acc[k][i].result();
}

// y_k = G x_k in FP64 with the FP64 values (one face row).
template <int D, int R>
__device__ __forceinline__ void d_row(const PSys& S, int64_t f, unsigned amask, const double* x,
                                      double (&y)[R][D]) {
    constexpr int NS = 2 * D + 1;
    constexpr int NPV = NS * D * D;
    const int64_t N = S.nf * D;
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
        for (int i = 0; i < D; ++i) y[k][i] = 0.0;
#pragma unroll(R == 1 ? NS : 1)
    for (int s = 0; s < NS; ++s) {
        const int64_t c = s == 0 ? f : int64_t(__ldcs(S.cols + sell(f, s - 1, 2 * D)));
        double v[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) v[i][j] = __ldcs(S.v64 + sell(f, (s * D + i) * D + j, NPV));
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (!((amask >> k) & 1u)) continue;
            double xv[D];
            ldrow<D>(x + k * N + c * D, xv);
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) y[k][i] = fma(v[i][j], xv[j], y[k][i]);
        }
    }
}

// ---- tile staging (TMA bulk copies) ------------------------------------------
//
// For d = 2 the SpMV phase stages each tile (one slice of the sliced ELL: its
// high values, low values and columns are three contiguous runs) into shared
// memory with cp.async.bulk (the TMA engine's 1D mode) while the block
// computes the previous tile: two stages, one mbarrier each, completion counted
// in bytes.  A slice starts at a multiple of 256 rows times 2-8 bytes per
// value, so every copy is 16-byte aligned and a multiple of 16 bytes long; the
// last slice is copied whole (its rows beyond nf are zero).

template <int D, int MODE>
struct Stage {
    // d = 3 tiles would not fit twice; interleaved float-float values (FF32) are not staged
    static constexpr bool kOn = D == 2 && CRHYB_STAGE_D2 != 0 && MODE != kModeFF32;
    static constexpr int NST = CRHYB_STAGE_D2 >= 2 ? 2 : 1;    // stages per block (2: prefetch the next tile)
    static constexpr int NS = 2 * D + 1, NPV = NS * D * D, NC = 2 * D;
    static constexpr int VB = MODE == kModeFP64 ? 8 : 4;      // bytes of a (high) value
    static constexpr int LB = MODE == kModeFF32 ? 4 : (MODE == kModeFFBF16 ? 2 : 0);
    static constexpr int HI = 0;                              // offsets inside a stage
    static constexpr int LO = NPV * kPBlock * VB;
    static constexpr int CO = LO + NPV * kPBlock * LB;
    static constexpr int BYTES = CO + NC * kPBlock * 4;
    static constexpr int SMEM = kOn ? NST * BYTES + 16 : 0;   // the stages and two mbarriers
};

constexpr long long kWaitLimit = 1ll << 22;   // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Warp 0 stages the slice that starts at row r0 of system S into buf.
template <int D, int MODE>
__device__ __forceinline__ void stage_issue(const PSys& S, int64_t r0, unsigned char* buf, uint64_t* bar) {
    using G = Stage<D, MODE>;
    const int lane = threadIdx.x & 31;
    constexpr uint32_t HB = uint32_t(G::NPV) * kPBlock * G::VB, LBY = uint32_t(G::NPV) * kPBlock * G::LB,
                       CB = uint32_t(G::NC) * kPBlock * 4;
    const size_t slice = size_t(r0 / kPBlock);
    if (lane == 0) {
        mbar_expect_tx(bar, HB + LBY + CB);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads of buf before the new writes
        const char* vh = MODE == kModeFP64 ? reinterpret_cast<const char*>(S.v64) : reinterpret_cast<const char*>(S.vh);
        bulk_g2s(buf + G::HI, vh + slice * HB, HB, bar);
        if (G::LB) bulk_g2s(buf + G::LO, static_cast<const char*>(S.vl) + slice * LBY, LBY, bar);
        bulk_g2s(buf + G::CO, reinterpret_cast<const char*>(S.cols) + slice * CB, CB, bar);
    }
}

// Every thread waits for the stage; a wait that runs out sets the error flag.
__device__ __forceinline__ bool stage_wait(uint64_t* bar, uint32_t parity, PCtl* ctl) {
    for (long long n = 0; n < kWaitLimit; ++n)
        if (mbar_try_wait(bar, parity)) return true;
    atomicExch(&ctl->err, 3);
    return false;
}

// q = G p for one row from a staged tile (row r of the stage), float-float.
// Right-hand sides outermost: only one right-hand side's gathers of p are live
// at a time; the values of G are re-read from shared memory for each.
template <int D, int R, int MODE>
__device__ __forceinline__ void ff_row_staged(const unsigned char* buf, int r, int64_t f, unsigned amask,
                                              const float2* p, int64_t N, float2 (&y)[R][D]) {
    using G = Stage<D, MODE>;
    constexpr int NS = 2 * D + 1;
    const float* hi = reinterpret_cast<const float*>(buf + G::HI);
    const int32_t* co = reinterpret_cast<const int32_t*>(buf + G::CO);
#pragma unroll
    for (int k = 0; k < R; ++k) {
        FFAcc acc[D];
#pragma unroll
        for (int i = 0; i < D; ++i) acc[i].zero();
        if ((amask >> k) & 1u) {
            float2 xv[NS][D];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int64_t c = s == 0 ? f : int64_t(co[(s - 1) * kPBlock + r]);
#pragma unroll
                for (int j = 0; j < D; ++j) xv[s][j] = p[k * N + c * D + j];
            }
#pragma unroll
            for (int s = 0; s < NS; ++s)
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        const int q = (s * D + i) * D + j;
                        float l;
                        if (MODE == kModeFFBF16)
                            l = __uint_as_float(
                                unsigned(reinterpret_cast<const unsigned short*>(buf + G::LO)[q * kPBlock + r]) << 16);
                        else
                            l = reinterpret_cast<const float*>(buf + G::LO)[q * kPBlock + r];
                        acc[i].mad(hi[q * kPBlock + r], l, xv[s][j].x, xv[s][j].y);
                    }
        }
#pragma unroll
        for (int i = 0; i < D; ++i) y[k][i] = acc[i].result();
    }
}

// q = G x for one row from a staged tile, FP64 (right-hand sides outermost).
template <int D, int R, int MODE>
__device__ __forceinline__ void d_row_staged(const unsigned char* buf, int r, int64_t f, unsigned amask,
                                             const double* x, int64_t N, double (&y)[R][D]) {
    using G = Stage<D, MODE>;
    constexpr int NS = 2 * D + 1;
    const double* v = reinterpret_cast<const double*>(buf + G::HI);
    const int32_t* co = reinterpret_cast<const int32_t*>(buf + G::CO);
#pragma unroll
    for (int k = 0; k < R; ++k) {
#pragma unroll
        for (int i = 0; i < D; ++i) y[k][i] = 0.0;
        if (!((amask >> k) & 1u)) continue;
        double xv[NS][D];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int64_t c = s == 0 ? f : int64_t(co[(s - 1) * kPBlock + r]);
#pragma unroll
            for (int j = 0; j < D; ++j) xv[s][j] = x[k * N + c * D + j];
        }
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) y[k][i] = fma(v[((s * D + i) * D + j) * kPBlock + r], xv[s][j], y[k][i]);
    }
}

// ---- the persistent kernel -------------------------------------------------

// active-pair mask of system s: pairs that are neither done nor waiting for an update
__device__ __forceinline__ unsigned active_mask(const PArgs& a, const PSys& S, int s) {
    unsigned m = 0;
    for (int k = 0; k < S.R; ++k) {
        const PScal& P = a.scal[s * kPMaxRhs + k];
        if (!sc_i(P.done) && !sc_i(P.upd)) m |= 1u << k;
    }
    return m;
}

__device__ __forceinline__ unsigned update_mask(const PArgs& a, const PSys& S, int s) {
    unsigned m = 0;
    for (int k = 0; k < S.R; ++k)
        if (sc_i(a.scal[s * kPMaxRhs + k].upd)) m |= 1u << k;
    return m;
}

// Ask L2 for the sliced-ELL data of tile t (its values and columns: one
// contiguous run each, 16-byte aligned, whole slices allocated).
__device__ __forceinline__ void l2_prefetch(const void* ptr, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ptr), "r"(bytes) : "memory");
}

template <int D, bool FF, typename LT>
__device__ __forceinline__ void prefetch_tile(const PArgs& a, int t) {
    constexpr int NPV = (2 * D + 1) * D * D;
    const int2 td = a.tiles[t];
    const PSys& S = a.sys[td.x];
    const size_t sl = size_t(td.y) / kSlice;
    if (FF) {
        if (!std::is_same<LT, float2>::value) l2_prefetch(S.vh + sl * NPV * kSlice, NPV * kSlice * sizeof(float));
        l2_prefetch(static_cast<const LT*>(S.vl) + sl * NPV * kSlice, NPV * kSlice * sizeof(LT));
    } else {
        l2_prefetch(S.v64 + sl * NPV * kSlice, NPV * kSlice * sizeof(double));
    }
    l2_prefetch(S.cols + sl * 2 * D * kSlice, 2 * D * kSlice * sizeof(int32_t));
}

// the register budget each instantiation is compiled for, as blocks per SM
constexpr int persist_min_blocks(int D, int R, int MODE) {
    return R == 1 ? (D == 3 ? (MODE == kModeFP64 ? CRHYB_3D_MINB : CRHYB_3D_FF_MINB) : CRHYB_PERSIST_MINB)
                  : (R == 2 ? CRHYB_R2_MINB : CRHYB_R4_MINB);
}

template <int D, int R, int MODE>
__global__ void __launch_bounds__(kPBlock, persist_min_blocks(D, R, MODE)) k_pcg_persist(PArgs a) {
    constexpr bool FF = MODE != kModeFP64;
    using LT = typename std::conditional<MODE == kModeFFBF16, __nv_bfloat16, float2>::type;
    PCtl* ctl = a.ctl;
    if (int(blockIdx.x) == a.stall_block) return;   // testing hook (failure detection), see PArgs
    const int t0 = int(blockIdx.x) * a.tpb, t1 = min(t0 + a.tpb, a.ntiles);
    int piters = 0, epoch = a.epoch0;
    int ph[2] = {0, 0};   // phase parity of the two staging mbarriers
    unsigned long long t_last = 0;
    if (a.phase_ns && blockIdx.x == 0 && threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_last));
    if constexpr (Stage<D, MODE>::kOn) {
        extern __shared__ __align__(128) unsigned char dsm[];
        uint64_t* bars = reinterpret_cast<uint64_t*>(dsm + Stage<D, MODE>::NST * Stage<D, MODE>::BYTES);
        if (threadIdx.x == 0) {
            mbar_init(bars);
            mbar_init(bars + 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    bool after_update = false;
    for (;;) {
        const int active = ld_vol(&ctl->snap_active), upd = ld_vol(&ctl->snap_upd);
        if (active == 0) break;
        if (upd == 0 && piters >= a.iters) break;
        if (upd != 0) {
            // One update pass clears every flag it finds; a flag that survives
            // it means a system whose tiles never ran: stop instead of looping.
            if (after_update) {
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&ctl->err, 2);
                break;
            }
            after_update = true;
            ++epoch;
            // ---------------- U1: x64 += x / sigma, x = 0 ----------------
            if (FF) {
                for (int t = t0; t < t1; ++t) {
                    const int2 td = a.tiles[t];
                    const PSys& S = a.sys[td.x];
                    const int64_t N = S.nf * D;
                    const int64_t f = td.y + threadIdx.x;
                    if (f >= S.nf) continue;
                    for (int k = 0; k < S.R; ++k) {
                        const PScal& P = a.scal[td.x * kPMaxRhs + k];
                        if (!sc_i(P.upd)) continue;
                        const double inv = 1.0 / sc_d(P.sigma);
                        float2* xv = static_cast<float2*>(S.x);
#pragma unroll
                        for (int i = 0; i < D; ++i) {
                            const int64_t q = k * N + f * D + i;
                            S.x64[q] += ff_to_double(xv[q]) * inv;
                            xv[q] = make_float2(0.f, 0.f);
                        }
                    }
                }
                if (!pbar(ctl, false)) return;
                phase_mark(a, 0, t_last);
            }
            // ---------------- U2: r64 = b - G x64 (FP64); r.r, b.b, r.M^{-1}r ----------------
            {
                int cur = -1;
                unsigned umask = 0;
                FFAcc af[R][3];
                double ad[R][3];
                auto flush = [&]() {
                    const PSys& S = a.sys[cur];
                    double bs[R][3], tot[R][3];
                    block_partials<R, 3, false>(af, ad, bs);
                    if (system_flush<R, 3>(a, S, cur, bs, tot) && threadIdx.x == 0) {
#pragma unroll
                        for (int k = 0; k < R; ++k) {
                            if (k >= S.R || !((umask >> k) & 1u)) continue;
                            PScal& P = a.scal[cur * kPMaxRhs + k];
                            const double rr = tot[k][0], bb = tot[k][1], rz = tot[k][2];
                            const double target = a.tol * a.tol * bb;
                            P.orr = rr;
                            P.bb = bb;
                            P.upd = 0;
                            const int first = sc_i(P.first);
                            P.outer = sc_i(P.outer) + (FF && !first ? 1 : 0);
                            atomicSub(&ctl->upd, 1);
                            if (!isfinite(rr)) {
                                P.status = CR_ERR_BREAKDOWN;
                                P.done = 1;
                                atomicSub(&ctl->active, 1);
                                continue;
                            }
                            if (rr <= target) {
                                P.conv = 1;
                                P.done = 1;
                                atomicSub(&ctl->active, 1);
                                continue;
                            }
                            if (sc_i(P.it) >= a.max_it) {
                                P.status = CR_ERR_NOT_CONVERGED;
                                P.done = 1;
                                atomicSub(&ctl->active, 1);
                                continue;
                            }
                            if (FF) {
                                const double s_old = sc_d(P.sigma), s_new = 1.0 / sqrt(rr);
                                const double rz_prev = sc_d(P.rz_prev) / (s_old * s_old);
                                P.beta = (first || !(rz_prev > 0.0)) ? 0.0 : rz / rz_prev * (s_new / s_old);
                                P.rz = rz * s_new * s_new;
                                P.rr = rr * s_new * s_new;
                                P.tol2 = fmax(a.delta * a.delta * rr, 0.25 * target) * s_new * s_new;
                                P.sigma = s_new;
                            } else {   // FP64: the true residual replaces the recursive one
                                const double rz_prev = sc_d(P.rz_prev);
                                P.beta = (first || !(rz_prev > 0.0)) ? 0.0 : rz / rz_prev;
                                P.rz = rz;
                                P.rr = rr;
                                P.tol2 = target;
                            }
                            P.beta_ff = ff_from_double(P.beta);
                            P.first = 0;
                            P.epoch = epoch;
                        }
                    }
                };
                for (int t = t0; t < t1; ++t) {
                    const int2 td = a.tiles[t];
                    if (td.x != cur) {
                        if (cur >= 0 && umask) flush();
                        cur = td.x;
                        umask = update_mask(a, a.sys[cur], cur);
#pragma unroll
                        for (int k = 0; k < R; ++k)
#pragma unroll
                            for (int q = 0; q < 3; ++q) ad[k][q] = 0.0;
                    }
                    if (!umask) continue;
                    const PSys& S = a.sys[cur];
                    const int64_t N = S.nf * D;
                    const int64_t f = td.y + threadIdx.x;
                    if (f >= S.nf) continue;
                    double y[R][D];
                    d_row<D, R>(S, f, umask, FF ? S.x64 : static_cast<const double*>(S.x), y);
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        if (!((umask >> k) & 1u)) continue;
#pragma unroll
                        for (int i = 0; i < D; ++i) {
                            const int64_t q = k * N + f * D + i;
                            const double bi = S.b[q];
                            const double ri = bi - y[k][i];
                            if (FF) S.r64[q] = ri;
                            else static_cast<double*>(S.r)[q] = ri;
                            const double mi = FF ? double(S.minv32[f * D + i]) : S.minv64[f * D + i];
                            ad[k][0] += ri * ri;
                            ad[k][1] += bi * bi;
                            ad[k][2] += ri * mi * ri;
                        }
                    }
                }
                if (cur >= 0 && umask) flush();
            }
            if (!pbar(ctl, false)) return;
            phase_mark(a, 1, t_last);
            // ---------------- U3: r = sigma r64 (float-float); p = M^{-1} r + beta p ----------------
            for (int t = t0; t < t1; ++t) {
                const int2 td = a.tiles[t];
                const PSys& S = a.sys[td.x];
                const int64_t N = S.nf * D;
                const int64_t f = td.y + threadIdx.x;
                if (f >= S.nf) continue;
                for (int k = 0; k < S.R; ++k) {
                    const PScal& P = a.scal[td.x * kPMaxRhs + k];
                    if (sc_i(P.epoch) != epoch || sc_i(P.done)) continue;
                    const double beta = sc_d(P.beta), sigma = sc_d(P.sigma);
                    const float2 beta_ff = sc_f2(P.beta_ff);
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        const int64_t q = k * N + f * D + i;
                        if (FF) {
                            const float2 rv = ff_from_double(S.r64[q] * sigma);
                            static_cast<float2*>(S.r)[q] = rv;
                            const float2 z = ff_mul1(S.minv32[f * D + i], rv);
                            float2* pv = static_cast<float2*>(S.p);
                            pv[q] = ff_add(z, ff_mul(beta_ff, pv[q]));
                        } else {
                            const double z = S.minv64[f * D + i] * static_cast<double*>(S.r)[q];
                            double* pv = static_cast<double*>(S.p);
                            pv[q] = fma(beta, pv[q], z);
                        }
                    }
                }
            }
            if (!pbar(ctl, true)) return;
            phase_mark(a, 2, t_last);
            continue;
        }
        // ---------------- P1: q = G p, p.q ----------------
        {
            int cur = -1;
            unsigned amask = 0;
            FFAcc af[R][1];
            double ad[R][1];
            auto flush = [&]() {
                const PSys& S = a.sys[cur];
                double bs[R][1], tot[R][1];
                block_partials<R, 1, FF>(af, ad, bs);
                if (system_flush<R, 1>(a, S, cur, bs, tot) && threadIdx.x == 0) {
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        if (k >= S.R || !((amask >> k) & 1u)) continue;
                        PScal& P = a.scal[cur * kPMaxRhs + k];
                        const double pq = tot[k][0];
                        if (!(pq > 0.0) || !isfinite(pq)) {
                            P.status = CR_ERR_BREAKDOWN;
                            P.done = 1;
                            atomicSub(&ctl->active, 1);
                        } else {
                            P.alpha = sc_d(P.rz) / pq;
                            P.alpha_ff = ff_from_double(P.alpha);
                        }
                    }
                }
            };
            // accumulate one row's q = G p and p.q (y computed by the caller)
            auto row_out = [&](const PSys& S, int64_t f, const void* yv) {
                const int64_t N = S.nf * D;
                if (FF) {
                    const float2(&y)[R][D] = *static_cast<const float2(*)[R][D]>(yv);
                    const float2* p = static_cast<const float2*>(S.p);
                    float2* q = static_cast<float2*>(S.q);
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        if (!((amask >> k) & 1u)) continue;
                        float2 pv[D];
                        ldrow<D>(p + k * N + f * D, pv);
                        strow<D>(q + k * N + f * D, y[k]);
#pragma unroll
                        for (int i = 0; i < D; ++i) af[k][0].mad(pv[i].x, pv[i].y, y[k][i].x, y[k][i].y);
                    }
                } else {
                    const double(&y)[R][D] = *static_cast<const double(*)[R][D]>(yv);
                    const double* p = static_cast<const double*>(S.p);
                    double* q = static_cast<double*>(S.q);
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        if (!((amask >> k) & 1u)) continue;
                        double pv[D];
                        ldrow<D>(p + k * N + f * D, pv);
                        strow<D>(q + k * N + f * D, y[k]);
#pragma unroll
                        for (int i = 0; i < D; ++i) ad[k][0] += pv[i] * y[k][i];
                    }
                }
            };
            auto new_system = [&](int s) {
                cur = s;
                amask = active_mask(a, a.sys[cur], cur);
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    af[k][0].zero();
                    ad[k][0] = 0.0;
                }
            };
            if constexpr (Stage<D, MODE>::kOn) {
                // staged: tile t + 1 is copied in while tile t is computed
                extern __shared__ __align__(128) unsigned char dsm[];   // the same dynamic buffer
                using G = Stage<D, MODE>;
                uint64_t* bars = reinterpret_cast<uint64_t*>(dsm + G::NST * G::BYTES);
                auto work = [&](int t) {   // is tile t one with rows to compute?
                    const int sidx = a.tiles[t].x;
                    return active_mask(a, a.sys[sidx], sidx) != 0u;
                };
                auto issue = [&](int t, int stage) {
                    const int2 td = a.tiles[t];
                    stage_issue<D, MODE>(a.sys[td.x], td.y, dsm + stage * G::BYTES, bars + stage);
                };
                int u = 0;         // work tiles seen in this phase
                int issued = -1;   // the last tile whose copies were issued
                for (int t = t0; t < t1; ++t) {
                    const int2 td = a.tiles[t];
                    if (td.x != cur) {
                        if (cur >= 0 && amask) flush();
                        new_system(td.x);
                    }
                    if (!amask) continue;
                    const int stage = G::NST == 2 ? (u & 1) : 0;
                    if (issued < t) {   // not prefetched (single stage, or the previous tile was not a work tile)
                        if (threadIdx.x < 32) issue(t, stage);
                        issued = t;
                    }
                    // prefetch the next work tile into the other stage (read last by tile t - 1)
                    if (G::NST == 2 && t + 1 < t1 && work(t + 1)) {
                        if (threadIdx.x < 32) issue(t + 1, stage ^ 1);
                        issued = t + 1;
                    }
                    if (!stage_wait(bars + stage, uint32_t(ph[stage]), ctl)) {
                        stage_wait(bars + stage, uint32_t(ph[stage]), ctl);   // bounded, then give up
                        return;
                    }
                    ph[stage] ^= 1;
                    const PSys& S = a.sys[cur];
                    const int64_t f = td.y + threadIdx.x;
                    if (f < S.nf) {
                        const int64_t N = S.nf * D;
                        if (FF) {
                            float2 y[R][D];
                            ff_row_staged<D, R, MODE>(dsm + stage * G::BYTES, threadIdx.x, f, amask,
                                                      static_cast<const float2*>(S.p), N, y);
                            row_out(S, f, &y);
                        } else {
                            double y[R][D];
                            d_row_staged<D, R, MODE>(dsm + stage * G::BYTES, threadIdx.x, f, amask,
                                                     static_cast<const double*>(S.p), N, y);
                            row_out(S, f, &y);
                        }
                    }
                    __syncthreads();   // the stage may be refilled
                    ++u;
                }
            } else {
                constexpr int PF = CRHYB_L2_PREFETCH;
                if (PF > 0 && threadIdx.x == 0)
                    for (int t = t0; t < t0 + PF && t < t1; ++t) prefetch_tile<D, FF, LT>(a, t);
                for (int t = t0; t < t1; ++t) {
                    if (PF > 0 && threadIdx.x == 0 && t + PF < t1) prefetch_tile<D, FF, LT>(a, t + PF);
                    const int2 td = a.tiles[t];
                    if (td.x != cur) {
                        if (cur >= 0 && amask) flush();
                        new_system(td.x);
                    }
                    if (!amask) continue;
                    const PSys& S = a.sys[cur];
                    const int64_t N = S.nf * D;
                    const int64_t f = td.y + threadIdx.x;
                    if (f >= S.nf) continue;
                    if (FF) {
                        float2 y[R][D];
                        ff_row<D, R, LT>(S, f, amask, static_cast<const float2*>(S.p), y);
                        row_out(S, f, &y);
                    } else {
                        double y[R][D];
                        d_row<D, R>(S, f, amask, static_cast<const double*>(S.p), y);
                        row_out(S, f, &y);
                    }
                }
            }
            if (cur >= 0 && amask) flush();
        }
        if (!pbar(ctl, false)) return;
        phase_mark(a, 3, t_last);
        // ---------------- P2: x += alpha p, r -= alpha q; r.z, r.r ----------------
        {
            int cur = -1;
            unsigned amask = 0;
            FFAcc af[R][2];
            double ad[R][2];
            float2 al_ff[R];
            double al[R];
            auto flush = [&]() {
                const PSys& S = a.sys[cur];
                double bs[R][2], tot[R][2];
                block_partials<R, 2, FF>(af, ad, bs);
                if (system_flush<R, 2>(a, S, cur, bs, tot) && threadIdx.x == 0) {
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        if (k >= S.R || !((amask >> k) & 1u)) continue;
                        PScal& P = a.scal[cur * kPMaxRhs + k];
                        const double rz = tot[k][0], rr = tot[k][1];
                        const double rz_old = sc_d(P.rz);
                        P.rz_prev = rz_old;
                        P.beta = rz / rz_old;
                        P.beta_ff = ff_from_double(P.beta);
                        P.rz = rz;
                        P.rr = rr;
                        const int it = sc_i(P.it) + 1;
                        P.it = it;
                        if (!isfinite(rr)) {
                            P.status = CR_ERR_BREAKDOWN;
                            P.done = 1;
                            atomicSub(&ctl->active, 1);
                        } else if (rr <= sc_d(P.tol2) || it >= a.max_it) {
                            // the iterated residual reached this update's target (float-float),
                            // or the tolerance (FP64), or the limit: the true residual of the
                            // iterate decides in the update phases
                            P.upd = 1;
                            atomicAdd(&ctl->upd, 1);
                        }
                    }
                }
            };
            for (int t = t0; t < t1; ++t) {
                const int2 td = a.tiles[t];
                if (td.x != cur) {
                    if (cur >= 0 && amask) flush();
                    cur = td.x;
                    const PSys& S0 = a.sys[cur];
                    amask = active_mask(a, S0, cur);
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        af[k][0].zero();
                        af[k][1].zero();
                        ad[k][0] = ad[k][1] = 0.0;
                        if (k < S0.R) {
                            al_ff[k] = sc_f2(a.scal[cur * kPMaxRhs + k].alpha_ff);
                            al[k] = sc_d(a.scal[cur * kPMaxRhs + k].alpha);
                        }
                    }
                }
                if (!amask) continue;
                const PSys& S = a.sys[cur];
                const int64_t N = S.nf * D;
                const int64_t f = td.y + threadIdx.x;
                if (f >= S.nf) continue;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    if (!((amask >> k) & 1u)) continue;
                    const int64_t o = k * N + f * D;
                    if (FF) {
                        float2* x = static_cast<float2*>(S.x);
                        float2* r = static_cast<float2*>(S.r);
                        float2 xv[D], rv[D], pv[D], qv[D];
                        float mv[D];
                        ldrow<D>(x + o, xv);
                        ldrow<D>(r + o, rv);
                        ldrow<D>(static_cast<const float2*>(S.p) + o, pv);
                        ldrow<D>(static_cast<const float2*>(S.q) + o, qv);
                        ldrow<D>(S.minv32 + f * D, mv);
#pragma unroll
                        for (int i = 0; i < D; ++i) {
                            xv[i] = ff_add(xv[i], ff_mul(al_ff[k], pv[i]));
                            rv[i] = ff_add(rv[i], ff_neg(ff_mul(al_ff[k], qv[i])));
                            const float2 z = ff_mul1(mv[i], rv[i]);
                            af[k][0].mad(rv[i].x, rv[i].y, z.x, z.y);
                            af[k][1].mad(rv[i].x, rv[i].y, rv[i].x, rv[i].y);
                        }
                        strow<D>(x + o, xv);
                        strow<D>(r + o, rv);
                    } else {
                        double* x = static_cast<double*>(S.x);
                        double* r = static_cast<double*>(S.r);
                        double xv[D], rv[D], pv[D], qv[D], mv[D];
                        ldrow<D>(x + o, xv);
                        ldrow<D>(r + o, rv);
                        ldrow<D>(static_cast<const double*>(S.p) + o, pv);
                        ldrow<D>(static_cast<const double*>(S.q) + o, qv);
                        ldrow<D>(S.minv64 + f * D, mv);
#pragma unroll
                        for (int i = 0; i < D; ++i) {
                            xv[i] = fma(al[k], pv[i], xv[i]);
                            rv[i] = fma(-al[k], qv[i], rv[i]);
                            ad[k][0] += rv[i] * mv[i] * rv[i];
                            ad[k][1] += rv[i] * rv[i];
                        }
                        strow<D>(x + o, xv);
                        strow<D>(r + o, rv);
                    }
                }
            }
            if (cur >= 0 && amask) flush();
        }
        if (!pbar(ctl, false)) return;
        phase_mark(a, 4, t_last);
        // ---------------- P3: p = M^{-1} r + beta p ----------------
        {
            int cur = -1;
            unsigned amask = 0;
            float2 be_ff[R];
            double be[R];
            for (int t = t0; t < t1; ++t) {
                const int2 td = a.tiles[t];
                if (td.x != cur) {
                    cur = td.x;
                    const PSys& S0 = a.sys[cur];
                    amask = active_mask(a, S0, cur);
#pragma unroll
                    for (int k = 0; k < R; ++k)
                        if (k < S0.R) {
                            be_ff[k] = sc_f2(a.scal[cur * kPMaxRhs + k].beta_ff);
                            be[k] = sc_d(a.scal[cur * kPMaxRhs + k].beta);
                        }
                }
                if (!amask) continue;
                const PSys& S = a.sys[cur];
                const int64_t N = S.nf * D;
                const int64_t f = td.y + threadIdx.x;
                if (f >= S.nf) continue;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    if (!((amask >> k) & 1u)) continue;
                    const int64_t o = k * N + f * D;
                    if (FF) {
                        float2* p = static_cast<float2*>(S.p);
                        float2 pv[D], rv[D];
                        float mv[D];
                        ldrow<D>(p + o, pv);
                        ldrow<D>(static_cast<const float2*>(S.r) + o, rv);
                        ldrow<D>(S.minv32 + f * D, mv);
#pragma unroll
                        for (int i = 0; i < D; ++i) pv[i] = ff_add(ff_mul1(mv[i], rv[i]), ff_mul(be_ff[k], pv[i]));
                        strow<D>(p + o, pv);
                    } else {
                        double* p = static_cast<double*>(S.p);
                        double pv[D], rv[D], mv[D];
                        ldrow<D>(p + o, pv);
                        ldrow<D>(static_cast<const double*>(S.r) + o, rv);
                        ldrow<D>(S.minv64 + f * D, mv);
#pragma unroll
                        for (int i = 0; i < D; ++i) pv[i] = fma(be[k], pv[i], mv[i] * rv[i]);
                        strow<D>(p + o, pv);
                    }
                }
            }
        }
        if (!pbar(ctl, true)) return;
        phase_mark(a, 5, t_last);
        ++piters;
        after_update = false;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->epoch = epoch;
        a.ctl->piters = piters;
    }
}

template <int D, int R, int MODE>
int launch_one(const PArgs& a, int grid, cudaStream_t st) {
    void* args[] = {const_cast<PArgs*>(&a)};
    CR_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_pcg_persist<D, R, MODE>), dim3(grid),
                                        dim3(kPBlock), args, size_t(Stage<D, MODE>::SMEM), st));
    return CR_OK;
}

template <int D, int R, int MODE>
int occupancy(int* blocks_per_sm) {
    constexpr int smem = Stage<D, MODE>::SMEM;
    if (smem > 48 * 1024)
        CR_CUDA(cudaFuncSetAttribute(&k_pcg_persist<D, R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, &k_pcg_persist<D, R, MODE>, kPBlock, smem));
    return CR_OK;
}

using LaunchFn = int (*)(const PArgs&, int, cudaStream_t);
using OccFn = int (*)(int*);

template <int D, int R>
void pick(int mode, LaunchFn* l, OccFn* o) {
    if (mode == kModeFP64) { *l = launch_one<D, R, kModeFP64>; *o = occupancy<D, R, kModeFP64>; }
    else if (mode == kModeFF32) { *l = launch_one<D, R, kModeFF32>; *o = occupancy<D, R, kModeFF32>; }
    else { *l = launch_one<D, R, kModeFFBF16>; *o = occupancy<D, R, kModeFFBF16>; }
}

int g_sms = 0;

}  // namespace

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------

int PersistPlan::build(const std::vector<PSys>& systems, int d_, int mode_, int blocks_per_sm_cap) {
    release();
    d = d_;
    mode = mode_;
    nsys = int(systems.size());
    rmax = 1;
    for (const PSys& s : systems) rmax = std::max(rmax, s.R);
    // tiles
    std::vector<int2> tl;
    std::vector<PSys> sy = systems;
    for (int s = 0; s < nsys; ++s) {
        if (sy[s].nf <= 0 || sy[s].R < 1 || sy[s].R > kPMaxRhs)
            return fail(CR_ERR_ARG, "persistent PCG: a system without face rows or with a bad number of right-hand sides");
        sy[s].tile0 = int(tl.size());
        const int64_t nt = (sy[s].nf + kPBlock - 1) / kPBlock;
        sy[s].ntiles = int(nt);
        for (int64_t t = 0; t < nt; ++t) tl.push_back(make_int2(s, int(t * kPBlock)));
    }
    ntiles = int(tl.size());
    // kernels for 1, 2 or 4 right-hand sides per system
    const int R = rmax <= 1 ? 1 : (rmax <= 2 ? 2 : kPMaxRhs);
    LaunchFn l = nullptr;
    OccFn o = nullptr;
    if (d == 2) {
        if (R == 1) pick<2, 1>(mode, &l, &o);
        else if (R == 2) pick<2, 2>(mode, &l, &o);
        else pick<2, kPMaxRhs>(mode, &l, &o);
    } else {
        if (R == 1) pick<3, 1>(mode, &l, &o);
        else if (R == 2) pick<3, 2>(mode, &l, &o);
        else pick<3, kPMaxRhs>(mode, &l, &o);
    }
    launch = reinterpret_cast<void*>(l);
    int bps = 0;
    CR_TRY(o(&bps));
    if (g_sms == 0) {
        int dev = 0;
        CR_CUDA(cudaGetDevice(&dev));
        CR_CUDA(cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    if (bps <= 0) return fail(CR_ERR_CUDA, "persistent PCG: the kernel does not fit on an SM");
    if (blocks_per_sm_cap > 0) bps = std::min(bps, blocks_per_sm_cap);
    grid = std::min(g_sms * bps, std::max(ntiles, 1));
    blocks_per_sm = bps;
    CR_TRY(arena.alloc_n(&d_sys, size_t(nsys)));
    CR_TRY(arena.alloc_n(&d_tiles, size_t(std::max(ntiles, 1))));
    CR_TRY(arena.alloc_n(&d_scal, size_t(nsys) * kPMaxRhs));
    CR_TRY(arena.alloc_n(&d_tpart, size_t(nsys + grid) * kPMaxRhs * 4));   // slots never exceed nsys + grid
    CR_TRY(arena.alloc_n(&d_syscnt, size_t(nsys)));
    CR_TRY(arena.alloc_n(&d_ctl, 1));
    CR_TRY(arena.alloc_n(&d_phase, 8));
    CR_CUDA(cudaMallocHost(&h_scal, sizeof(PScal) * nsys * kPMaxRhs));
    CR_CUDA(cudaMallocHost(&h_ctl, sizeof(PCtl)));
    CR_CUDA(cudaMallocHost(&h_sys, sizeof(PSys) * nsys));
    CR_CUDA(cudaMallocHost(&h_tiles, sizeof(int2) * std::max(ntiles, 1)));
    CR_CUDA(cudaMemset(d_syscnt, 0, sizeof(unsigned) * nsys));
    sys_host = sy;
    live.assign(size_t(nsys), 1);
    CR_TRY(layout(nullptr));
    CR_CUDA(cudaDeviceSynchronize());
    return CR_OK;
}

// Lay the tiles of the live systems out over the blocks: block b sweeps the
// contiguous range [b tpb, (b+1) tpb); per system the blocks that cover it and
// their partial-sum slots.  Systems whose pairs are all done get no tiles, so
// the resident blocks spread over the work that is left.
int PersistPlan::layout(cudaStream_t st) {
    int nt = 0;
    for (int s = 0; s < nsys; ++s) {
        PSys& y = sys_host[s];
        y.tile0 = nt;
        y.ntiles = live[s] ? int((y.nf + kPBlock - 1) / kPBlock) : 0;
        for (int t = 0; t < y.ntiles; ++t) h_tiles[nt + t] = make_int2(s, t * kPBlock);
        nt += y.ntiles;
    }
    ntiles_live = nt;
    tpb = std::max((nt + grid - 1) / grid, 1);
    nslots = 0;
    for (int s = 0; s < nsys; ++s) {
        PSys& y = sys_host[s];
        if (y.ntiles == 0) {
            y.blk0 = y.nblk = 0;
            y.slot0 = nslots;
        } else {
            y.blk0 = y.tile0 / tpb;
            y.nblk = (y.tile0 + y.ntiles - 1) / tpb - y.blk0 + 1;
            y.slot0 = nslots;
            nslots += y.nblk;
        }
        h_sys[s] = y;
    }
    CR_CUDA(cudaMemcpyAsync(d_tiles, h_tiles, sizeof(int2) * std::max(nt, 1), cudaMemcpyHostToDevice, st));
    CR_CUDA(cudaMemcpyAsync(d_sys, h_sys, sizeof(PSys) * nsys, cudaMemcpyHostToDevice, st));
    return CR_OK;
}

int PersistPlan::update_systems(const std::vector<PSys>& systems, cudaStream_t st) {
    if (int(systems.size()) != nsys) return fail(CR_ERR_ARG, "persistent PCG: system count changed");
    CR_CUDA(cudaStreamSynchronize(st));   // the staging buffer may still feed an earlier copy
    for (int s = 0; s < nsys; ++s) {
        PSys y = systems[s];
        y.tile0 = sys_host[s].tile0;
        y.ntiles = sys_host[s].ntiles;
        y.blk0 = sys_host[s].blk0;
        y.nblk = sys_host[s].nblk;
        y.slot0 = sys_host[s].slot0;
        if (y.nf != sys_host[s].nf || y.R != sys_host[s].R)
            return fail(CR_ERR_ARG, "persistent PCG: system sizes changed");
        sys_host[s] = y;
        h_sys[s] = y;
    }
    CR_CUDA(cudaMemcpyAsync(d_sys, h_sys, sizeof(PSys) * nsys, cudaMemcpyHostToDevice, st));
    return CR_OK;
}

void PersistPlan::release() {
    arena.release();
    for (cudaEvent_t& e : ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    if (h_scal) cudaFreeHost(h_scal);
    if (h_ctl) cudaFreeHost(h_ctl);
    if (h_sys) cudaFreeHost(h_sys);
    if (h_tiles) cudaFreeHost(h_tiles);
    h_tiles = nullptr;
    h_scal = nullptr;
    h_ctl = nullptr;
    h_sys = nullptr;
    d_sys = nullptr;
    d_tiles = nullptr;
    d_scal = nullptr;
    d_tpart = nullptr;
    d_syscnt = nullptr;
    d_ctl = nullptr;
    d_phase = nullptr;
}

// Run the solve to completion: every (system, rhs) pair starts from x64
// (FF) or x (FP64) as set by the caller.  `iters` bounds the iterations of
// one launch; the host reads the control block between launches.
int PersistPlan::run(double tol, double delta, int max_it, int iters, cudaStream_t st, int64_t* launches,
                     bool profile, double* ms, int64_t* piters) {
    if (profile && !ev[0]) {
        CR_CUDA(cudaEventCreate(&ev[0]));
        CR_CUDA(cudaEventCreate(&ev[1]));
    }
    if (ms) *ms = 0.0;
    if (piters) *piters = 0;
    // start: every pair has a (start) update due
    std::vector<PScal> sc(size_t(nsys) * kPMaxRhs);
    int npairs = 0;
    for (int s = 0; s < nsys; ++s)
        for (int k = 0; k < kPMaxRhs; ++k) {
            PScal& P = sc[size_t(s) * kPMaxRhs + k];
            std::memset(&P, 0, sizeof(PScal));
            P.sigma = 1.0;
            P.first = 1;
            if (k < sys_host[s].R) {
                P.upd = 1;
                ++npairs;
            } else {
                P.done = 1;
            }
        }
    PCtl c{};
    c.active = c.snap_active = npairs;
    c.upd = c.snap_upd = npairs;
    std::memcpy(h_scal, sc.data(), sizeof(PScal) * sc.size());
    std::memcpy(h_ctl, &c, sizeof(PCtl));
    CR_CUDA(cudaMemcpyAsync(d_scal, h_scal, sizeof(PScal) * sc.size(), cudaMemcpyHostToDevice, st));
    CR_CUDA(cudaMemcpyAsync(d_ctl, h_ctl, sizeof(PCtl), cudaMemcpyHostToDevice, st));
    CR_CUDA(cudaMemsetAsync(d_syscnt, 0, sizeof(unsigned) * nsys, st));
    if (std::find(live.begin(), live.end(), 0) != live.end()) {
        std::fill(live.begin(), live.end(), 1);
        CR_CUDA(cudaStreamSynchronize(st));   // the pinned staging buffers may feed an earlier copy
        CR_TRY(layout(st));
    }
    PArgs a{};
    a.sys = d_sys;
    a.tiles = d_tiles;
    a.scal = d_scal;
    a.tpart = d_tpart;
    a.syscnt = d_syscnt;
    a.ctl = d_ctl;
    a.ntiles = ntiles_live;
    a.tpb = tpb;
    a.tol = tol;
    a.delta = delta;
    a.max_it = max_it;
    a.iters = iters > 0 ? iters : 1 << 30;
    a.epoch0 = 0;
    a.phase_ns = profile ? d_phase : nullptr;
    // Failure-detection test hook: CRHYB_TEST_STALL_BLOCK=<block> makes that block skip the
    // solve; every other block's barrier wait then runs out (bounded) and the call returns
    // CR_ERR_TIMEOUT with the context intact.  Nothing faults or hangs.
    a.stall_block = -1;
    if (const char* sb = std::getenv("CRHYB_TEST_STALL_BLOCK")) a.stall_block = std::atoi(sb);
    if (profile) CR_CUDA(cudaMemsetAsync(d_phase, 0, sizeof(unsigned long long) * 8, st));
    LaunchFn l = reinterpret_cast<LaunchFn>(launch);
    int idle = 0;
    for (;;) {
        if (profile) CR_CUDA(cudaEventRecord(ev[0], st));
        CR_TRY(l(a, grid, st));
        if (profile) CR_CUDA(cudaEventRecord(ev[1], st));
        if (launches) ++*launches;
        CR_CUDA(cudaMemcpyAsync(h_ctl, d_ctl, sizeof(PCtl), cudaMemcpyDeviceToHost, st));
        CR_CUDA(cudaStreamSynchronize(st));
        if (h_ctl->err == 2) return fail(CR_ERR_ARG, "persistent PCG: a reliable update found no tiles to run on");
        if (h_ctl->err) return fail(CR_ERR_TIMEOUT, "persistent PCG: a bounded grid-barrier wait ran out");
        if (profile) {
            float t = 0.f;
            CR_CUDA(cudaEventElapsedTime(&t, ev[0], ev[1]));
            if (ms) *ms += t;
            if (piters) *piters += h_ctl->piters;
        }
        if (h_ctl->snap_active == 0 || h_ctl->active == 0) break;
        if (nsys > 1) {
            // drop the systems whose pairs are all done and spread the rest over the blocks
            CR_CUDA(cudaMemcpyAsync(h_scal, d_scal, sizeof(PScal) * sc.size(), cudaMemcpyDeviceToHost, st));
            CR_CUDA(cudaStreamSynchronize(st));
            bool changed = false;
            for (int s2 = 0; s2 < nsys; ++s2) {
                if (!live[s2]) continue;
                bool any = false;
                for (int k = 0; k < sys_host[s2].R; ++k) any |= !h_scal[size_t(s2) * kPMaxRhs + k].done;
                if (!any) {
                    live[s2] = 0;
                    changed = true;
                }
            }
            if (changed) {
                CR_TRY(layout(st));
                a.ntiles = ntiles_live;
                a.tpb = tpb;
            }
        }
        if (h_ctl->piters == 0 && ++idle > 2)
            return fail(CR_ERR_BREAKDOWN, "persistent PCG: launches make no progress");
        if (h_ctl->piters > 0) idle = 0;
        a.epoch0 = h_ctl->epoch;
    }
    CR_CUDA(cudaMemcpyAsync(h_scal, d_scal, sizeof(PScal) * sc.size(), cudaMemcpyDeviceToHost, st));
    if (profile) CR_CUDA(cudaMemcpyAsync(h_phase, d_phase, sizeof(h_phase), cudaMemcpyDeviceToHost, st));
    CR_CUDA(cudaStreamSynchronize(st));
    if (profile && std::getenv("CRHYB_TRACE")) {
        static const char* names[6] = {"U1", "U2", "U3", "P1", "P2", "P3"};
        for (int k = 0; k < 6; ++k)
            std::fprintf(stderr, "[crhyb] persistent phase %s: %.3f ms\n", names[k], h_phase[k] * 1e-6);
    }
    return CR_OK;
}

}  // namespace crhyb
