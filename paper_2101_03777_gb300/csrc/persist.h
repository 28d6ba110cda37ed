// Persistent batched Jacobi-PCG: data structures shared by the persistent
// kernel (persist.cu) and its callers (solve.cu, batch.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "internal.h"

namespace crhyb {

constexpr int kPMaxRhs = 4;   // right-hand sides sharing one pass over G

// One system: a hybridised matrix G and R right-hand sides.  Vectors are laid
// out [R][nf][d]; x, r, p, q are float2 (float-float) or double (FP64).
struct PSys {
    int64_t nf;
    int R;
    int tile0, ntiles;          // its tiles in the tile list (set by PersistPlan::build)
    int blk0, nblk, slot0;      // the blocks whose tile ranges cover it, and its partial-sum slots
    const int32_t* cols;        // sliced ELL columns of slots 1..2d
    const float* vh;            // float-float high values, sliced ELL
    const void* vl;             // low plane (float or bf16)
    const double* v64;          // FP64 values
    const float* minv32;        // 1 / diag(G)
    const double* minv64;
    const double* b;            // [R][nf][d] right-hand sides
    double* x64;                // [R][nf][d] FP64 iterate (float-float runs)
    double* r64;                // [R][nf][d] FP64 residual of the reliable updates
    void *x, *r, *p, *q;        // [R][nf][d] iteration vectors
};

// Scalars of one (system, right-hand side) pair.
struct PScal {
    double rz, rz_prev, alpha, beta, rr, orr, bb, tol2, sigma;
    float2 alpha_ff, beta_ff;
    int it, done, conv, status, upd, first, epoch, outer;
};

// Control block: barrier state and loop-control counters.
struct PCtl {
    unsigned long long bar;     // grid barrier: arrivals (bits 0-31), generation (32-62), error (63)
    int err;                    // a bounded barrier wait ran out
    int active;                 // pairs not done
    int upd;                    // pairs with a reliable update due
    int snap_active, snap_upd;  // snapshot taken by the block that opened the last barrier
    int epoch, piters;          // state handed from one launch to the next
};

struct PArgs {
    const PSys* sys;
    const int2* tiles;          // (system, first row) per tile
    PScal* scal;                // [nsys][kPMaxRhs]
    double* tpart;              // [slots][kPMaxRhs][4] partial sums, one slot per (block, system)
    unsigned* syscnt;           // [nsys] tiles completed in the current phase
    PCtl* ctl;
    int ntiles, tpb;            // tiles, tiles per block (contiguous ranges)
    double tol, delta;
    int max_it, iters, epoch0;
    unsigned long long* phase_ns;   // profile runs: time per phase (U1 U2 U3 P1 P2 P3), else NULL
    int stall_block;                // testing hook: this block leaves at once (-1: none), so that the
                                    // others' bounded barrier waits run out
};

// A launch plan for one list of systems (all with the same d and arithmetic).
struct PersistPlan {
    int d = 2, mode = 0, nsys = 0, rmax = 1, ntiles = 0, grid = 0, blocks_per_sm = 0, tpb = 1, nslots = 0;
    int ntiles_live = 0;        // tiles of the systems that still have pairs to solve
    std::vector<char> live;     // per system: some pair not done
    void* launch = nullptr;
    DevArena arena;
    PSys* d_sys = nullptr;
    int2* d_tiles = nullptr;
    PScal* d_scal = nullptr;
    double* d_tpart = nullptr;
    unsigned* d_syscnt = nullptr;
    PCtl* d_ctl = nullptr;
    PScal* h_scal = nullptr;    // pinned
    PCtl* h_ctl = nullptr;      // pinned
    PSys* h_sys = nullptr;      // pinned staging of the system table
    int2* h_tiles = nullptr;    // pinned staging of the tile list
    std::vector<PSys> sys_host;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    unsigned long long* d_phase = nullptr;   // [8] phase times of the profile runs
    unsigned long long h_phase[8] = {};

    // mode: 0 FP64, 1 float-float (FP32 low plane), 2 float-float (BF16 low plane)
    int build(const std::vector<PSys>& systems, int d, int mode, int blocks_per_sm_cap);
    // replace the systems' pointers (same sizes and tiles as at build), stream ordered
    int update_systems(const std::vector<PSys>& systems, cudaStream_t st);
    bool built() const { return d_sys != nullptr; }
    int layout(cudaStream_t st);
    // profile: time every launch with CUDA events; *ms and *piters receive the summed
    // kernel time and the PCG iterations those launches ran
    int run(double tol, double delta, int max_it, int iters, cudaStream_t st, int64_t* launches,
            bool profile = false, double* ms = nullptr, int64_t* piters = nullptr);
    void release();
    ~PersistPlan() { release(); }
};

}  // namespace crhyb
