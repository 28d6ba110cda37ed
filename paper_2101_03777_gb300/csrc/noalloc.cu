// Residual of a block-ELL system with no device allocation at all.
//
// The paper has no counterpart to this entry point.  It serves callers that
// cannot allocate device memory themselves or through the library: code
// running inside a host that owns every allocation (a memory-pool manager or
// a framework that forbids cudaMalloc on its hot path), code that must not
// take the allocator's implicit synchronisation, and checkers that must
// leave the device's memory state exactly as they found it.  The caller
// passes every input and output; the only scratch (per-tile partial sums and
// the completion counter of the reduction) is a fixed file-scope device array
// that every GPU loading the library holds until the process exits.

#include <mutex>

#include "device_common.cuh"

namespace crhyb {
namespace {

constexpr int kNaTile = 256;                              // face rows per block (one per thread)
constexpr int64_t kNaMaxTiles = 16384;                    // scratch capacity in tiles
constexpr int64_t kNaMaxRows = kNaTile * kNaMaxTiles;     // 4,194,304 face rows
constexpr int kNaMaxDevices = 64;

// Layout of the scratch array (doubles):
//   [0, kNaMaxTiles)                 partial ||r||^2 per tile
//   [kNaMaxTiles, 2 kNaMaxTiles)     partial ||b||^2 per tile
//   [2 kNaMaxTiles + 0..1]           results ||r||^2, ||b||^2
//   [2 kNaMaxTiles + 2]              number of out-of-range column indices (as a double)
//   [2 kNaMaxTiles + 3]              completion counter (its low 32 bits, as unsigned)
//   [2 kNaMaxTiles + 4]              out-of-range counter (its low 32 bits, as unsigned)
constexpr int64_t kNaResult = 2 * kNaMaxTiles;
constexpr int64_t kNaScratchDoubles = 2 * kNaMaxTiles + 8;   // 262,208 bytes
static __device__ __align__(256) double g_noalloc_scratch[kNaScratchDoubles];

template <int D>
__global__ void __launch_bounds__(kNaTile) k_residual_noalloc(int64_t nf, int nslot, const int32_t* __restrict__ cols,
                                                              const double* __restrict__ vals,
                                                              const double* __restrict__ b,
                                                              const double* __restrict__ x, double* __restrict__ r,
                                                              double* __restrict__ scratch) {
    unsigned* count = reinterpret_cast<unsigned*>(scratch + kNaResult + 3);
    unsigned* bad = reinterpret_cast<unsigned*>(scratch + kNaResult + 4);
    const int64_t f = int64_t(blockIdx.x) * kNaTile + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (f < nf) {
        double y[D];
#pragma unroll
        for (int i = 0; i < D; ++i) y[i] = 0.0;
        for (int s = 0; s < nslot; ++s) {
            const int64_t c = cols[size_t(s) * nf + f];
            if (c < 0 || c >= nf) {   // reject the column: count it, skip the access
                atomicAdd(bad, 1u);
                continue;
            }
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) y[i] = fma(vals[((size_t(s) * D + i) * D + j) * nf + f], x[c * D + j], y[i]);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const double bi = b[f * D + i];
            const double ri = bi - y[i];
            if (r) r[f * D + i] = ri;
            v[0] += ri * ri;
            v[1] += bi * bi;
        }
    }
    __shared__ double sh[2 * 32];
    __shared__ bool last;
    double bs[2];
    block_sum<2>(v, sh, bs);
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = bs[0];
        scratch[kNaMaxTiles + blockIdx.x] = bs[1];
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block sums the tiles in order: the result does not depend on scheduling
    double acc[2] = {0.0, 0.0};
    for (int t = threadIdx.x; t < int(gridDim.x); t += blockDim.x) {
        acc[0] += __ldcg(scratch + t);
        acc[1] += __ldcg(scratch + kNaMaxTiles + t);
    }
    double tot[2];
    block_sum<2>(acc, sh, tot);
    if (threadIdx.x == 0) {
        scratch[kNaResult + 0] = tot[0];
        scratch[kNaResult + 1] = tot[1];
        scratch[kNaResult + 2] = double(atomicAdd(bad, 0u));
        *count = 0u;
    }
}

std::mutex g_na_mutex;
double* g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (in host code the symbol's name is only a host-side stand-in).
int noalloc_scratch(double** out) {
    int dev = 0;
    CR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) return fail(CR_ERR_ARG, "cr_residual_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        CR_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_na_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_na_ptr[dev];
    return CR_OK;
}

}  // namespace
}  // namespace crhyb

using namespace crhyb;

extern "C" int64_t cr_residual_noalloc_max_rows(void) { return kNaMaxRows; }

extern "C" int cr_residual_noalloc(int dim, int64_t nf, int nslot, const int32_t* cols, const double* vals,
                                   const double* b, const double* x, double* r, double* norms2, void* stream) {
    if (dim != 2 && dim != 3) return fail(CR_ERR_ARG, "cr_residual_noalloc: dim must be 2 or 3");
    if (nf < 0) return fail(CR_ERR_ARG, "cr_residual_noalloc: negative number of face rows");
    if (nf > kNaMaxRows)
        return fail(CR_ERR_ARG, "cr_residual_noalloc: " + std::to_string(nf) + " face rows exceed the fixed scratch "
                                "capacity of " + std::to_string(kNaMaxRows) + " rows");
    if (nslot < 1 || nslot > 2 * dim + 1) return fail(CR_ERR_ARG, "cr_residual_noalloc: nslot must be in [1, 2*dim+1]");
    if (!norms2) return fail(CR_ERR_ARG, "cr_residual_noalloc: norms2 is NULL");
    CR_TRY(check_call(nullptr, "cr_residual_noalloc", {cols, vals, b, x, r, norms2}));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool dev_out = is_device_pointer(norms2);
    if (nf == 0) {
        if (dev_out) {
            CR_CUDA(cudaMemsetAsync(norms2, 0, 2 * sizeof(double), st));
            CR_CUDA(cudaStreamSynchronize(st));
        } else {
            norms2[0] = norms2[1] = 0.0;
        }
        return CR_OK;
    }
    if (!is_device_pointer(cols) || !is_device_pointer(vals) || !is_device_pointer(b) || !is_device_pointer(x) ||
        (r && !is_device_pointer(r)))
        return fail(CR_ERR_ARG, "cr_residual_noalloc: cols, vals, b, x and r must be device pointers");
    double* scratch = nullptr;
    CR_TRY(noalloc_scratch(&scratch));
    // the completion and out-of-range counters start at zero on every call
    CR_CUDA(cudaMemsetAsync(scratch + kNaResult + 3, 0, 2 * sizeof(double), st));
    const unsigned grid = unsigned((nf + kNaTile - 1) / kNaTile);
    if (dim == 2) k_residual_noalloc<2><<<grid, kNaTile, 0, st>>>(nf, nslot, cols, vals, b, x, r, scratch);
    else k_residual_noalloc<3><<<grid, kNaTile, 0, st>>>(nf, nslot, cols, vals, b, x, r, scratch);
    CR_CUDA(cudaGetLastError());
    double res[3];
    CR_CUDA(cudaMemcpyAsync(res, scratch + kNaResult, sizeof(res), cudaMemcpyDeviceToHost, st));
    CR_CUDA(cudaStreamSynchronize(st));
    if (res[2] != 0.0) return fail(CR_ERR_ARG, "cr_residual_noalloc: column index out of range in cols");
    if (dev_out) {
        CR_CUDA(cudaMemcpyAsync(norms2, scratch + kNaResult, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CR_CUDA(cudaStreamSynchronize(st));
    } else {
        norms2[0] = res[0];
        norms2[1] = res[1];
    }
    return CR_OK;
}
