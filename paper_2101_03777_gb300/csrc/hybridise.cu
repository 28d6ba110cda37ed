// Element-local kernels of the hybrid method (Section 3.2): condensation of
// each simplex into its G_K and S_K contributions, the per-face merge of the
// two contributions to diagonal blocks and to S, the export of the coupled
// element blocks (Section 3.1), and the element-local recovery of P and U.
//
// One thread handles one simplex.  Stokes (b_h = 0): Â_K = (S_K + diag(e)) (x)
// Id_d, so only the (d+1)x(d+1) matrix T = S_K + diag(e) is inverted and
//   Â^{-1} D = v with v[l][i] = sum_m T^{-1}[l][m] D[m][i],
//   M_K((l,i),(m,j)) = T^{-1}[l][m] delta_ij - v[l][i] v[m][j] / B_K.
// Navier-Stokes (2D): Â_K is a full nonsymmetric 6x6 matrix inverted by
// Gauss-Jordan elimination with partial pivoting in registers.

#include <cuda_bf16.h>

#include "device_common.cuh"

namespace crhyb {
namespace {

constexpr int kElemBlock = 128;

struct MeshView {
    int64_t ne, nf;
    const double* coords;
    const int32_t* elems;
    const int32_t* elem_face;
    const uint8_t* elem_side;
    const int32_t* face_elems;
    const uint8_t* mis;
    int k0;
    // previous time level of an implicit Euler step, or NULL: [nrhs][nf][d] in the
    // condensation and export kernels, the recovered right-hand side's [nf][d] in recovery
    const double* uprev;
};

MeshView view(const cr_mesh* m) {
    return MeshView{m->ne, m->nf, m->coords, m->elems, m->elem_face, m->elem_side, m->face_elems, m->mis, m->k0,
                    nullptr};
}

struct Outputs {
    double* val64;
    float* val32;
    __nv_bfloat16* val16;
    float2* vff;
    __nv_bfloat16* vlo16;
    int npl;             // value planes of the sliced ELL: (2d+1) d^2
    double* dpart;
    double* spart;
    int32_t* status;
};

template <int D>
struct Topo {
    int face[D + 1];
    int side[D + 1];
    bool in[D + 1];
    double c[D + 1];   // C_K diagonal: +1 owner, -1 other, 0 exterior
};

template <int D>
__device__ __forceinline__ void load_topo(const MeshView& mv, int64_t K, Topo<D>& t) {
#pragma unroll
    for (int l = 0; l <= D; ++l) {
        t.face[l] = __ldg(mv.elem_face + K * (D + 1) + l);
        t.side[l] = __ldg(mv.elem_side + K * (D + 1) + l);
        t.in[l] = t.face[l] >= 0;
        t.c[l] = t.in[l] ? (t.side[l] == 0 ? 1.0 : -1.0) : 0.0;
    }
}

// S_K restricted to interior faces (Section 3.1):
//   (S_K)_{lm} = nu a_l.a_m/|K| + mu |K|/(d+1) delta_lm.
template <int D>
__device__ __forceinline__ double s_entry(const Geom<D>& g, int l, int m, double nu, double mu) {
    double dot = 0.0;
#pragma unroll
    for (int b = 0; b < D; ++b) dot += g.a[l][b] * g.a[m][b];
    double s = nu * dot / g.vol;
    if (l == m) s += mu * g.vol / (D + 1);
    return s;
}

// Diagonal of E_K per local face (Section 3.2, item 7): -lambda_K on M_1,
// +lambda_L on a face shared with L in M_1, else 0.  Zero when mu > 0.
template <int D>
__device__ __forceinline__ void e_diag(const MeshView& mv, const double* __restrict__ lam, int64_t K,
                                       const Topo<D>& t, double (&e)[D + 1]) {
#pragma unroll
    for (int l = 0; l <= D; ++l) e[l] = 0.0;
    if (!lam) return;
    if (mv.mis[K]) {
        const double lk = lam[K];
#pragma unroll
        for (int l = 0; l <= D; ++l) e[l] = t.in[l] ? -lk : 0.0;
    } else {
#pragma unroll
        for (int l = 0; l <= D; ++l) {
            if (!t.in[l]) continue;
            const int L = __ldg(mv.face_elems + 2 * t.face[l] + (1 - t.side[l]));
            if (mv.mis[L]) e[l] = lam[L];
        }
    }
}

// In-place Gauss-Jordan inverse without pivoting (T definite: SPD, or
// negative definite on M_1).  Returns false on a vanishing pivot.
template <int N>
__device__ __forceinline__ bool invert_nopivot(double (&A)[N][N]) {
    double scale = 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) scale = fmax(scale, fabs(A[k][k]));
    bool ok = scale > 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const double piv = A[k][k];
        ok = ok && (fabs(piv) > 1e-15 * scale);
        const double ip = 1.0 / piv;
        A[k][k] = 1.0;
#pragma unroll
        for (int j = 0; j < N; ++j) A[k][j] *= ip;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (i == k) continue;
            const double f = A[i][k];
            A[i][k] = 0.0;
#pragma unroll
            for (int j = 0; j < N; ++j) A[i][j] -= f * A[k][j];
        }
    }
    return ok;
}

// Gauss-Jordan inverse with partial pivoting, all indices compile-time so the
// matrix stays in registers (row swaps are done by selects).
template <int N>
__device__ __forceinline__ bool invert_pivot(const double (&A0)[N][N], double (&X)[N][N]) {
    double A[N][N];
    double scale = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            A[i][j] = A0[i][j];
            X[i][j] = i == j ? 1.0 : 0.0;
            scale = fmax(scale, fabs(A0[i][j]));
        }
    bool ok = scale > 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int p = k;
        double best = fabs(A[k][k]);
#pragma unroll
        for (int r = k + 1; r < N; ++r) {
            const double v = fabs(A[r][k]);
            if (v > best) { best = v; p = r; }
        }
#pragma unroll
        for (int r = k + 1; r < N; ++r) {
            const bool sw = (r == p);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const double a = A[k][j], b = A[r][j];
                A[k][j] = sw ? b : a;
                A[r][j] = sw ? a : b;
                const double x = X[k][j], y = X[r][j];
                X[k][j] = sw ? y : x;
                X[r][j] = sw ? x : y;
            }
        }
        const double piv = A[k][k];
        ok = ok && (fabs(piv) > 1e-15 * scale);
        const double ip = 1.0 / piv;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            A[k][j] *= ip;
            X[k][j] *= ip;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (i == k) continue;
            const double f = A[i][k];
#pragma unroll
            for (int j = 0; j < N; ++j) {
                A[i][j] -= f * A[k][j];
                X[i][j] -= f * X[k][j];
            }
        }
    }
    return ok;
}

// ---------------------------------------------------------------------------
// Stokes element: T^{-1}, v = Â^{-1} D_K, B_K
// ---------------------------------------------------------------------------
template <int D>
struct StokesLocal {
    double Ti[D + 1][D + 1];
    double v[D + 1][D];
    double Dm[D + 1][D];
    double B, invB;
    bool ok;
};

template <int D>
__device__ __forceinline__ void stokes_local(const Geom<D>& g, const Topo<D>& t, const double (&e)[D + 1], double nu,
                                             double mu, bool isK0, StokesLocal<D>& L) {
    constexpr int NF = D + 1;
#pragma unroll
    for (int l = 0; l < NF; ++l)
#pragma unroll
        for (int m = 0; m < NF; ++m)
            L.Ti[l][m] = (t.in[l] && t.in[m]) ? s_entry<D>(g, l, m, nu, mu) + (l == m ? e[l] : 0.0)
                                              : (l == m ? 1.0 : 0.0);
    L.ok = invert_nopivot<NF>(L.Ti);
#pragma unroll
    for (int l = 0; l < NF; ++l)
#pragma unroll
        for (int i = 0; i < D; ++i) L.Dm[l][i] = t.in[l] ? -g.a[l][i] : 0.0;
    double B = 0.0;
#pragma unroll
    for (int l = 0; l < NF; ++l)
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double s = 0.0;
#pragma unroll
            for (int m = 0; m < NF; ++m) s += L.Ti[l][m] * L.Dm[m][i];
            L.v[l][i] = s;
            B += L.Dm[l][i] * s;
        }
    L.B = B;
    L.ok = L.ok && (fabs(B) > 0.0) && isfinite(B);
    L.invB = isK0 ? 0.0 : 1.0 / B;
}

// R_K (Eq. 8, Section 3.1): (R_K)_{l,i} = a_l^(i) fbar_K . (x_l - x_K).
template <int D>
__device__ __forceinline__ void rhs_local(const Geom<D>& g, const Topo<D>& t, const double* __restrict__ fb,
                                          double (&R)[D + 1][D], const double* __restrict__ up = nullptr,
                                          double mu = 0.0) {
    double f[D];   // fb == NULL: no source (the right-hand side is the previous level alone)
#pragma unroll
    for (int b = 0; b < D; ++b) f[b] = fb ? __ldg(fb + b) : 0.0;
#pragma unroll
    for (int l = 0; l <= D; ++l) {
        double rho = 0.0;
#pragma unroll
        for (int b = 0; b < D; ++b) rho += f[b] * g.dx[l][b];
#pragma unroll
        for (int i = 0; i < D; ++i) R[l][i] = t.in[l] ? g.a[l][i] * rho : 0.0;
    }
    // implicit Euler (mu = 1/dt): the lumped mass of the previous time level,
    // mu |K|/(d+1) u^n on each interior face, the same mass as in S_K
    if (up) {
        const double m = mu * g.vol / double(D + 1);
#pragma unroll
        for (int l = 0; l <= D; ++l)
            if (t.in[l])
#pragma unroll
                for (int i = 0; i < D; ++i) R[l][i] += m * __ldg(up + size_t(t.face[l]) * D + i);
    }
}

// The previous time level of right-hand side r (NULL if none).
__device__ __forceinline__ const double* uprev_of(const MeshView& mv, int r, int d) {
    return mv.uprev ? mv.uprev + size_t(r) * mv.nf * d : nullptr;
}

__device__ __forceinline__ void store_val(const Outputs& o, size_t idx, double v) {
    o.val64[idx] = v;
    const float hi = __double2float_rn(v);
    if (o.val32) o.val32[idx] = hi;
    if (o.val16) o.val16[idx] = __double2bfloat16(v);
    // float-float low parts: v - hi is exact in FP64, then rounded once
    if (o.vff) o.vff[idx] = make_float2(hi, __double2float_rn(v - double(hi)));
    if (o.vlo16) o.vlo16[idx] = __double2bfloat16(v - double(hi));
}

// lambda_K = scale * ||A_K||_inf on M_1 (Stokes: A_K = S_K (x) Id).
template <int D>
__global__ void __launch_bounds__(kElemBlock) k_lambda_stokes(MeshView mv, double nu, double mu, double scale,
                                                              double* __restrict__ lam) {
    const int64_t K = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (K >= mv.ne) return;
    if (!mv.mis[K]) { lam[K] = 0.0; return; }
    Geom<D> g;
    simplex_geometry<D>(mv.coords, mv.elems + K * (D + 1), g);
    Topo<D> t;
    load_topo<D>(mv, K, t);
    double best = 0.0;
#pragma unroll
    for (int l = 0; l <= D; ++l) {
        if (!t.in[l]) continue;
        double s = 0.0;
#pragma unroll
        for (int m = 0; m <= D; ++m)
            if (t.in[m]) s += fabs(s_entry<D>(g, l, m, nu, mu));
        best = fmax(best, s);
    }
    lam[K] = scale * best;
}

template <int D>
__global__ void __launch_bounds__(kElemBlock) k_condense_stokes(MeshView mv, double nu, double mu,
                                                                const double* __restrict__ lam,
                                                                const double* __restrict__ fbar, int nrhs,
                                                                Outputs o) {
    constexpr int NF = D + 1;
    const int64_t K = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (K >= mv.ne) return;
    const int64_t nf = mv.nf;
    Geom<D> g;
    simplex_geometry<D>(mv.coords, mv.elems + K * NF, g);
    Topo<D> t;
    load_topo<D>(mv, K, t);
    double e[NF];
    e_diag<D>(mv, lam, K, t, e);
    StokesLocal<D> L;
    stokes_local<D>(g, t, e, nu, mu, K == mv.k0, L);
    if (!L.ok) atomicExch(o.status, CR_ERR_SINGULAR);

    // G_K blocks: off-diagonal into their ELL slots, diagonal into dpart
#pragma unroll
    for (int l = 0; l < NF; ++l) {
        if (!t.in[l]) continue;
        const int64_t f = t.face[l];
        const int s = t.side[l];
#pragma unroll
        for (int m = 0; m < NF; ++m) {
            if (m == l) {
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        const double gv = (i == j ? L.Ti[l][l] : 0.0) - L.v[l][i] * L.v[l][j] * L.invB;
                        o.dpart[((size_t(s) * D + i) * D + j) * nf + f] = gv;
                    }
            } else {
                const int slot = 1 + s * D + (m < l ? m : m - 1);
                const double cc = t.c[l] * t.c[m];   // 0 when m is exterior
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        const double gv = cc * ((i == j ? L.Ti[l][m] : 0.0) - L.v[l][i] * L.v[m][j] * L.invB);
                        store_val(o, sell(f, (slot * D + i) * D + j, o.npl), gv);
                    }
            }
        }
    }
    // S_K = C_K M_K R_K, M_K R = T^{-1} R - v (v.R)/B
    for (int r = 0; r < nrhs; ++r) {
        double R[NF][D];
        rhs_local<D>(g, t, fbar + (size_t(r) * mv.ne + K) * D, R, uprev_of(mv, r, D), mu);
        double vR = 0.0;
#pragma unroll
        for (int m = 0; m < NF; ++m)
#pragma unroll
            for (int j = 0; j < D; ++j) vR += L.v[m][j] * R[m][j];
#pragma unroll
        for (int l = 0; l < NF; ++l) {
            if (!t.in[l]) continue;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                double s = 0.0;
#pragma unroll
                for (int m = 0; m < NF; ++m) s += L.Ti[l][m] * R[m][i];
                s -= L.v[l][i] * vR * L.invB;
                o.spart[((size_t(r) * 2 + t.side[l]) * D + i) * nf + t.face[l]] = t.c[l] * s;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Navier-Stokes element (2D): A_K = S_K (x) Id + N_K(w) (Oseen) or the Newton
// derivative of the co-volume convection (Eq. 9) at w, R_K += c_K(w) (Newton).
//   F_lm(w) = (W_l + W_m - Wbar) . (a_m - a_l)/(d+1)
//   c_l(w)  = 1/2 sum_{m != l} F_lm (W_m - W_l)
// ---------------------------------------------------------------------------
constexpr int kL2 = 6;   // local unknowns of a triangle

__device__ __forceinline__ void conv_matrix2(const Geom<2>& g, const Topo<2>& t, const double* __restrict__ w,
                                             double nu, double mu, int conv, double (&A)[kL2][kL2],
                                             double (&cw)[kL2]) {
    double W[3][2];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int i = 0; i < 2; ++i) W[l][i] = t.in[l] ? __ldg(w + size_t(t.face[l]) * 2 + i) : 0.0;
    double Wb[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) Wb[i] = (W[0][i] + W[1][i] + W[2][i]) / 3.0;
    double gg[3][3][2], F[3][3];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            double f = 0.0;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                gg[l][m][i] = (g.a[m][i] - g.a[l][i]) / 3.0;
                f += (W[l][i] + W[m][i] - Wb[i]) * gg[l][m][i];
            }
            F[l][m] = f;
        }
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            const double snm = s_entry<2>(g, l, n, nu, mu);
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    double v = (i == j) ? snm : 0.0;
                    if (conv != CR_CONV_NONE) {
                        double acc = 0.0;
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            if (m == l) continue;
                            const double dnm = (n == m ? 1.0 : 0.0) - (n == l ? 1.0 : 0.0);
                            if (i == j) acc += F[l][m] * dnm;
                            if (conv == CR_CONV_NEWTON) {
                                const double coef = (n == l ? 1.0 : 0.0) + (n == m ? 1.0 : 0.0) - 1.0 / 3.0;
                                acc += (W[m][i] - W[l][i]) * gg[l][m][j] * coef;
                            }
                        }
                        v += 0.5 * acc;
                    }
                    A[l * 2 + i][n * 2 + j] = (t.in[l] && t.in[n]) ? v : 0.0;
                }
        }
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            double c = 0.0;
#pragma unroll
            for (int m = 0; m < 3; ++m)
                if (m != l) c += F[l][m] * (W[m][i] - W[l][i]);
            cw[l * 2 + i] = (conv == CR_CONV_NEWTON && t.in[l]) ? 0.5 * c : 0.0;
        }
}

struct ConvLocal {
    double Ai[kL2][kL2];
    double u[kL2];    // Â^{-1} D
    double wt[kL2];   // D^t Â^{-1}
    double Dm[kL2];
    double invB;
    bool ok;
};

__device__ __forceinline__ void conv_local(const Geom<2>& g, const Topo<2>& t, const double (&e)[3],
                                           const double (&A)[kL2][kL2], bool isK0, ConvLocal& L) {
    double Ah[kL2][kL2];
#pragma unroll
    for (int p = 0; p < kL2; ++p)
#pragma unroll
        for (int q = 0; q < kL2; ++q) {
            const bool inp = t.in[p / 2], inq = t.in[q / 2];
            Ah[p][q] = (inp && inq) ? A[p][q] + (p == q ? e[p / 2] : 0.0) : (p == q ? 1.0 : 0.0);
        }
    L.ok = invert_pivot<kL2>(Ah, L.Ai);
#pragma unroll
    for (int p = 0; p < kL2; ++p) L.Dm[p] = t.in[p / 2] ? -g.a[p / 2][p % 2] : 0.0;
    double B = 0.0;
#pragma unroll
    for (int p = 0; p < kL2; ++p) {
        double s = 0.0, r = 0.0;
#pragma unroll
        for (int q = 0; q < kL2; ++q) {
            s += L.Ai[p][q] * L.Dm[q];
            r += L.Dm[q] * L.Ai[q][p];
        }
        L.u[p] = s;
        L.wt[p] = r;
        B += L.Dm[p] * s;
    }
    L.ok = L.ok && (fabs(B) > 0.0) && isfinite(B);
    L.invB = isK0 ? 0.0 : 1.0 / B;
}

__global__ void __launch_bounds__(kElemBlock) k_lambda_conv2(MeshView mv, double nu, double mu, int conv,
                                                             const double* __restrict__ w, double scale,
                                                             double* __restrict__ lam) {
    const int64_t K = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (K >= mv.ne) return;
    if (!mv.mis[K]) { lam[K] = 0.0; return; }
    Geom<2> g;
    simplex_geometry<2>(mv.coords, mv.elems + K * 3, g);
    Topo<2> t;
    load_topo<2>(mv, K, t);
    double A[kL2][kL2], cw[kL2];
    conv_matrix2(g, t, w, nu, mu, conv, A, cw);
    double best = 0.0;
#pragma unroll
    for (int p = 0; p < kL2; ++p) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < kL2; ++q) s += fabs(A[p][q]);
        best = fmax(best, s);
    }
    lam[K] = scale * best;
}

__global__ void __launch_bounds__(kElemBlock) k_condense_conv2(MeshView mv, double nu, double mu, int conv,
                                                               const double* __restrict__ w,
                                                               const double* __restrict__ lam,
                                                               const double* __restrict__ fbar, int nrhs, Outputs o) {
    const int64_t K = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (K >= mv.ne) return;
    const int64_t nf = mv.nf;
    Geom<2> g;
    simplex_geometry<2>(mv.coords, mv.elems + K * 3, g);
    Topo<2> t;
    load_topo<2>(mv, K, t);
    double e[3];
    e_diag<2>(mv, lam, K, t, e);
    double A[kL2][kL2], cw[kL2];
    conv_matrix2(g, t, w, nu, mu, conv, A, cw);
    ConvLocal L;
    conv_local(g, t, e, A, K == mv.k0, L);
    if (!L.ok) atomicExch(o.status, CR_ERR_SINGULAR);
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        if (!t.in[l]) continue;
        const int64_t f = t.face[l];
        const int s = t.side[l];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const double cc = t.c[l] * t.c[m];
            const int slot = 1 + s * 2 + (m < l ? m : m - 1);
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int p = l * 2 + i, q = m * 2 + j;
                    const double gv = cc * (L.Ai[p][q] - L.u[p] * L.wt[q] * L.invB);
                    if (m == l) o.dpart[((size_t(s) * 2 + i) * 2 + j) * nf + f] = gv;
                    else store_val(o, sell(f, (slot * 2 + i) * 2 + j, o.npl), gv);
                }
        }
    }
    for (int r = 0; r < nrhs; ++r) {
        double R[3][2];
        rhs_local<2>(g, t, fbar + (size_t(r) * mv.ne + K) * 2, R, uprev_of(mv, r, 2), mu);
        double Rv[kL2];
#pragma unroll
        for (int p = 0; p < kL2; ++p) Rv[p] = R[p / 2][p % 2] + cw[p];
        double wR = 0.0;
#pragma unroll
        for (int q = 0; q < kL2; ++q) wR += L.wt[q] * Rv[q];
#pragma unroll
        for (int p = 0; p < kL2; ++p) {
            if (!t.in[p / 2]) continue;
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < kL2; ++q) s += L.Ai[p][q] * Rv[q];
            s -= L.u[p] * wR * L.invB;
            o.spart[((size_t(r) * 2 + t.side[p / 2]) * 2 + (p % 2)) * nf + t.face[p / 2]] = t.c[p / 2] * s;
        }
    }
}

// ---------------------------------------------------------------------------
// Per-face merge: diagonal block and S are the sums of the two sides; the
// Jacobi preconditioner is the inverse of the scalar diagonal of G.
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256) k_merge(int64_t nf, int nrhs, const double* __restrict__ dpart,
                                               const double* __restrict__ spart, Outputs o, double* __restrict__ S,
                                               double* __restrict__ minv64, float* __restrict__ minv32) {
    const int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (f >= nf) return;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const double gv = dpart[((size_t(0) * D + i) * D + j) * nf + f] + dpart[((size_t(1) * D + i) * D + j) * nf + f];
            store_val(o, sell(f, i * D + j, o.npl), gv);
            if (i == j) {
                minv64[f * D + i] = 1.0 / gv;
                if (minv32) minv32[f * D + i] = __double2float_rn(1.0 / gv);
            }
        }
    for (int r = 0; r < nrhs; ++r)
#pragma unroll
        for (int i = 0; i < D; ++i)
            S[(size_t(r) * nf + f) * D + i] = spart[((size_t(r) * 2 + 0) * D + i) * nf + f] +
                                              spart[((size_t(r) * 2 + 1) * D + i) * nf + f];
}

// ---------------------------------------------------------------------------
// The coupled system without elimination (Eq. 10, Section 3.1), for the
// non-hybrid comparison solve: A = sum_K H_K A_K H_K^t with A_K = S_K (x) Id in
// the sliced ELL of G (the same stencil: the faces of one simplex), the
// diagonal blocks and R = sum_K H_K R_K summed per face by k_merge, and
// D_K = -a_{K, sigma} kept per simplex [ne][d+1][d] (zero on exterior faces).
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kElemBlock) k_assemble_A(MeshView mv, double nu, double mu, int conv,
                                                           const double* __restrict__ w,
                                                           const double* __restrict__ fbar, int nrhs, Outputs o,
                                                           double* __restrict__ DK) {
    constexpr int NF = D + 1, L = NF * D;
    const int64_t K = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (K >= mv.ne) return;
    const int64_t nf = mv.nf;
    Geom<D> g;
    simplex_geometry<D>(mv.coords, mv.elems + K * NF, g);
    Topo<D> t;
    load_topo<D>(mv, K, t);
    // A_K: S_K (x) Id, completed with the linearised convection N_K(w) (2D, Newton or
    // Oseen), whose Newton form also adds c_K(w) to R_K (Section 3.1)
    double A2[kL2][kL2], cw[L];   // A2: the 2D convective A_K (used when conv != NONE)
#pragma unroll
    for (int p = 0; p < L; ++p) cw[p] = 0.0;
    const bool use_conv = D == 2 && conv != CR_CONV_NONE;
    if constexpr (D == 2) {
        if (use_conv) conv_matrix2(g, t, w, nu, mu, conv, A2, cw);
    }
    auto aval = [&](int l, int i, int m, int j) -> double {
        if constexpr (D == 2) {
            if (use_conv) return A2[l * 2 + i][m * 2 + j];
        }
        return (t.in[l] && t.in[m] && i == j) ? s_entry<D>(g, l, m, nu, mu) : 0.0;
    };
#pragma unroll
    for (int l = 0; l < NF; ++l) {
#pragma unroll
        for (int i = 0; i < D; ++i) DK[(K * NF + l) * D + i] = t.in[l] ? -g.a[l][i] : 0.0;
        if (!t.in[l]) continue;
        const int64_t f = t.face[l];
        const int s = t.side[l];
#pragma unroll
        for (int m = 0; m < NF; ++m) {
            if (m == l) {
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int j = 0; j < D; ++j) o.dpart[((size_t(s) * D + i) * D + j) * nf + f] = aval(l, i, l, j);
            } else {
                const int slot = 1 + s * D + (m < l ? m : m - 1);
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int j = 0; j < D; ++j)
                        store_val(o, sell(f, (slot * D + i) * D + j, o.npl), aval(l, i, m, j));
            }
        }
    }
    for (int r = 0; r < nrhs; ++r) {
        double R[NF][D];
        rhs_local<D>(g, t, fbar + (size_t(r) * mv.ne + K) * D, R, uprev_of(mv, r, D), mu);
#pragma unroll
        for (int l = 0; l < NF; ++l) {
            if (!t.in[l]) continue;
#pragma unroll
            for (int i = 0; i < D; ++i)
                o.spart[((size_t(r) * 2 + t.side[l]) * D + i) * nf + t.face[l]] = R[l][i] + cw[l * D + i];
        }
    }
}

// ---------------------------------------------------------------------------
// Transient Stokes steps used as a preconditioner (steady problems): the
// hybridised right-hand side S of a step with no source and the previous
// level `up` alone (R_K = mu |K|/(d+1) up on the interior faces of K), and the
// lumped face mass m_sigma = sum_{K ni sigma} |K|/(d+1) that turns a velocity
// residual v into that previous level, up = v / (mu m).
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kElemBlock) k_rhs_previous(MeshView mv, double nu, double mu,
                                                             const double* __restrict__ up,
                                                             const double* __restrict__ gdiv,
                                                             double* __restrict__ spart, int32_t* status) {
    constexpr int NF = D + 1;
    const int64_t K = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (K >= mv.ne) return;
    const int64_t nf = mv.nf;
    Geom<D> g;
    simplex_geometry<D>(mv.coords, mv.elems + K * NF, g);
    Topo<D> t;
    load_topo<D>(mv, K, t);
    double e[NF];
#pragma unroll
    for (int l = 0; l < NF; ++l) e[l] = 0.0;
    StokesLocal<D> L;
    stokes_local<D>(g, t, e, nu, mu, K == mv.k0, L);
    if (!L.ok) atomicExch(status, CR_ERR_SINGULAR);
    double R[NF][D];
    rhs_local<D>(g, t, nullptr, R, up, mu);
    double vR = 0.0;
#pragma unroll
    for (int m = 0; m < NF; ++m)
#pragma unroll
        for (int j = 0; j < D; ++j) vR += L.v[m][j] * R[m][j];
    // a divergence D_K^t U_K = g_K adds Â^{-1} D_K g_K / B_K (invB = 0 on K_0)
    const double gK = gdiv ? gdiv[K] : 0.0;
#pragma unroll
    for (int l = 0; l < NF; ++l) {
        if (!t.in[l]) continue;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double s = 0.0;
#pragma unroll
            for (int m = 0; m < NF; ++m) s += L.Ti[l][m] * R[m][i];
            s += L.v[l][i] * (gK - vR) * L.invB;
            spart[(size_t(t.side[l]) * D + i) * nf + t.face[l]] = t.c[l] * s;
        }
    }
}

template <int D>
__global__ void __launch_bounds__(256) k_merge_rhs(int64_t nf, const double* __restrict__ spart,
                                                   double* __restrict__ S) {
    const int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (f >= nf) return;
#pragma unroll
    for (int i = 0; i < D; ++i)
        S[f * D + i] = spart[(size_t(0) * D + i) * nf + f] + spart[(size_t(1) * D + i) * nf + f];
}

template <int D>
__global__ void __launch_bounds__(256) k_face_mass(MeshView mv, double* __restrict__ mass) {
    const int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (f >= mv.nf) return;
    double m = 0.0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int64_t K = __ldg(mv.face_elems + 2 * f + k);
        Geom<D> g;
        simplex_geometry<D>(mv.coords, mv.elems + K * (D + 1), g);
        m += g.vol / double(D + 1);
    }
#pragma unroll
    for (int i = 0; i < D; ++i) mass[f * D + i] = m;
}

// ---------------------------------------------------------------------------
// Export of the coupled element blocks A_K, D_K, R_K (Section 3.1)
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kElemBlock) k_export(MeshView mv, double nu, double mu, int conv,
                                                       const double* __restrict__ w,
                                                       const double* __restrict__ fbar, int nrhs,
                                                       double* __restrict__ out) {
    constexpr int NF = D + 1, L = NF * D;
    const int64_t K = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (K >= mv.ne) return;
    Geom<D> g;
    simplex_geometry<D>(mv.coords, mv.elems + K * NF, g);
    Topo<D> t;
    load_topo<D>(mv, K, t);
    double* o = out + size_t(K) * (L * L + L + size_t(nrhs) * L);
    double cw[L];
#pragma unroll
    for (int p = 0; p < L; ++p) cw[p] = 0.0;
    if constexpr (D == 2) {
        if (conv != CR_CONV_NONE) {
            double A[kL2][kL2];
            conv_matrix2(g, t, w, nu, mu, conv, A, cw);
            for (int p = 0; p < L; ++p)
                for (int q = 0; q < L; ++q) o[p * L + q] = A[p][q];
        }
    }
    if (conv == CR_CONV_NONE || D != 2) {
        for (int p = 0; p < L; ++p)
            for (int q = 0; q < L; ++q) {
                const int l = p / D, i = p % D, m = q / D, j = q % D;
                o[p * L + q] = (t.in[l] && t.in[m] && i == j) ? s_entry<D>(g, l, m, nu, mu) : 0.0;
            }
    }
    for (int p = 0; p < L; ++p) o[L * L + p] = t.in[p / D] ? -g.a[p / D][p % D] : 0.0;
    for (int r = 0; r < nrhs; ++r) {
        double R[NF][D];
        rhs_local<D>(g, t, fbar + (size_t(r) * mv.ne + K) * D, R, uprev_of(mv, r, D), mu);
        for (int p = 0; p < L; ++p) o[L * L + L + size_t(r) * L + p] = R[p / D][p % D] + cw[p];
    }
}

// ---------------------------------------------------------------------------
// Recovery (Section 3.2, items 2 and 4)
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kBlock) k_recover_stokes(MeshView mv, double nu, double mu,
                                                           const double* __restrict__ lam,
                                                           const double* __restrict__ fb, const double* __restrict__ W,
                                                           double* __restrict__ U, double* __restrict__ ualt,
                                                           double* __restrict__ P, RedBuf red,
                                                           double* __restrict__ mean_out,
                                                           const double* __restrict__ gdiv = nullptr) {
    constexpr int NF = D + 1;
    const int64_t K = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    double vals[2] = {0.0, 0.0};
    if (K < mv.ne) {
        Geom<D> g;
        simplex_geometry<D>(mv.coords, mv.elems + K * NF, g);
        Topo<D> t;
        load_topo<D>(mv, K, t);
        double e[NF];
        e_diag<D>(mv, lam, K, t, e);
        StokesLocal<D> L;
        stokes_local<D>(g, t, e, nu, mu, K == mv.k0, L);
        double R[NF][D];
        rhs_local<D>(g, t, fb ? fb + size_t(K) * D : nullptr, R, mv.uprev, mu);
        double y[NF][D];
#pragma unroll
        for (int l = 0; l < NF; ++l)
#pragma unroll
            for (int i = 0; i < D; ++i)
                y[l][i] = t.in[l] ? R[l][i] - t.c[l] * W[size_t(t.face[l]) * D + i] : 0.0;
        // P_K = (D^t Â^{-1} y - g_K) / B = (v . y - g_K) / B (Â symmetric; g = 0 but in a
        // preconditioner solve with a divergence residual)
        double vy = 0.0;
#pragma unroll
        for (int l = 0; l < NF; ++l)
#pragma unroll
            for (int i = 0; i < D; ++i) vy += L.v[l][i] * y[l][i];
        const double PK = (vy - (gdiv ? gdiv[K] : 0.0)) * L.invB;
#pragma unroll
        for (int l = 0; l < NF; ++l) {
            if (!t.in[l]) continue;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                double s = 0.0;
#pragma unroll
                for (int m = 0; m < NF; ++m) s += L.Ti[l][m] * y[m][i];
                const double uh = s - L.v[l][i] * PK;
                if (t.side[l] == 0) U[size_t(t.face[l]) * D + i] = uh;
                else if (ualt) ualt[size_t(t.face[l]) * D + i] = uh;
            }
        }
        P[K] = PK;
        vals[0] = g.vol * PK;
        vals[1] = g.vol;
    }
    double tot[2];
    if (grid_sum<2>(vals, red, tot) && threadIdx.x == 0) *mean_out = tot[0] / tot[1];
}

__global__ void __launch_bounds__(kBlock) k_recover_conv2(MeshView mv, double nu, double mu, int conv,
                                                          const double* __restrict__ w,
                                                          const double* __restrict__ lam,
                                                          const double* __restrict__ fb, const double* __restrict__ W,
                                                          double* __restrict__ U, double* __restrict__ ualt,
                                                          double* __restrict__ P, RedBuf red,
                                                          double* __restrict__ mean_out) {
    const int64_t K = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    double vals[2] = {0.0, 0.0};
    if (K < mv.ne) {
        Geom<2> g;
        simplex_geometry<2>(mv.coords, mv.elems + K * 3, g);
        Topo<2> t;
        load_topo<2>(mv, K, t);
        double e[3];
        e_diag<2>(mv, lam, K, t, e);
        double A[kL2][kL2], cw[kL2];
        conv_matrix2(g, t, w, nu, mu, conv, A, cw);
        ConvLocal L;
        conv_local(g, t, e, A, K == mv.k0, L);
        double R[3][2];
        rhs_local<2>(g, t, fb + size_t(K) * 2, R, mv.uprev, mu);
        double y[kL2];
#pragma unroll
        for (int p = 0; p < kL2; ++p) {
            const int l = p / 2, i = p % 2;
            y[p] = t.in[l] ? R[l][i] + cw[p] - t.c[l] * W[size_t(t.face[l]) * 2 + i] : 0.0;
        }
        double wy = 0.0;
#pragma unroll
        for (int p = 0; p < kL2; ++p) wy += L.wt[p] * y[p];
        const double PK = wy * L.invB;
#pragma unroll
        for (int p = 0; p < kL2; ++p) {
            const int l = p / 2, i = p % 2;
            if (!t.in[l]) continue;
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < kL2; ++q) s += L.Ai[p][q] * y[q];
            const double uh = s - L.u[p] * PK;
            if (t.side[l] == 0) U[size_t(t.face[l]) * 2 + i] = uh;
            else if (ualt) ualt[size_t(t.face[l]) * 2 + i] = uh;
        }
        P[K] = PK;
        vals[0] = g.vol * PK;
        vals[1] = g.vol;
    }
    double tot[2];
    if (grid_sum<2>(vals, red, tot) && threadIdx.x == 0) *mean_out = tot[0] / tot[1];
}

__global__ void __launch_bounds__(256) k_subtract_mean(int64_t n, const double* __restrict__ mean,
                                                       double* __restrict__ P) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k < n) P[k] -= *mean;
}

__global__ void __launch_bounds__(kBlock) k_jump(int64_t n, const double* __restrict__ U,
                                                 const double* __restrict__ ualt, RedBuf red, double* out) {
    __shared__ double sh[32];
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    double v = k < n ? fabs(U[k] - ualt[k]) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) {
            // max is order independent: a plain atomic max on the bit pattern of a non-negative double
            atomicMax(reinterpret_cast<unsigned long long*>(out), __double_as_longlong(v));
        }
    }
}

inline unsigned blocks_for(int64_t n, int b) { return unsigned((n + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int launch_assemble_export(cr_system* s, double* blocks, cudaStream_t st) {
    cr_mesh* m = s->m;
    MeshView mv = view(m);
    mv.uprev = s->uprev_on ? s->uprev : nullptr;
    const unsigned nb = blocks_for(m->ne, kElemBlock);
    if (m->d == 2) k_export<2><<<nb, kElemBlock, 0, st>>>(mv, s->nu, s->mu, s->conv, s->w, s->fbar, s->nrhs, blocks);
    else k_export<3><<<nb, kElemBlock, 0, st>>>(mv, s->nu, s->mu, s->conv, s->w, s->fbar, s->nrhs, blocks);
    CR_CUDA(cudaGetLastError());
    return CR_OK;
}

int launch_hybridise(cr_hybrid* h, cudaStream_t st) {
    cr_system* s = h->s;
    cr_mesh* m = h->m;
    MeshView mv = view(m);
    mv.uprev = s->uprev_on ? s->uprev : nullptr;
    const unsigned nbe = blocks_for(m->ne, kElemBlock);
    const double* lam = nullptr;
    if (s->mu == 0.0) {
        const double sc = s->lam_scale > 0 ? s->lam_scale : 2.0;
        if (s->conv != CR_CONV_NONE)
            k_lambda_conv2<<<nbe, kElemBlock, 0, st>>>(mv, s->nu, s->mu, s->conv, s->w, sc, h->lam);
        else if (m->d == 2)
            k_lambda_stokes<2><<<nbe, kElemBlock, 0, st>>>(mv, s->nu, s->mu, sc, h->lam);
        else
            k_lambda_stokes<3><<<nbe, kElemBlock, 0, st>>>(mv, s->nu, s->mu, sc, h->lam);
        CR_CUDA(cudaGetLastError());
        lam = h->lam;
    }
    Outputs o{h->val64, h->val32, h->val16, h->vff, h->vlo16, h->nslot * m->d * m->d, h->dpart, h->spart,
              h->status};
    if (s->conv != CR_CONV_NONE)
        k_condense_conv2<<<nbe, kElemBlock, 0, st>>>(mv, s->nu, s->mu, s->conv, s->w, lam, s->fbar, s->nrhs, o);
    else if (m->d == 2)
        k_condense_stokes<2><<<nbe, kElemBlock, 0, st>>>(mv, s->nu, s->mu, lam, s->fbar, s->nrhs, o);
    else
        k_condense_stokes<3><<<nbe, kElemBlock, 0, st>>>(mv, s->nu, s->mu, lam, s->fbar, s->nrhs, o);
    CR_CUDA(cudaGetLastError());
    const unsigned nbf = blocks_for(m->nf, 256);
    if (m->d == 2) k_merge<2><<<nbf, 256, 0, st>>>(m->nf, s->nrhs, h->dpart, h->spart, o, h->S, h->minv64, h->minv32);
    else k_merge<3><<<nbf, 256, 0, st>>>(m->nf, s->nrhs, h->dpart, h->spart, o, h->S, h->minv64, h->minv32);
    CR_CUDA(cudaGetLastError());
    return CR_OK;
}

int launch_assemble_A(cr_system* s, double* val64, int npl, double* dpart, double* spart, double* R,
                      double* minv64, double* DK, cudaStream_t st) {
    cr_mesh* m = s->m;
    MeshView mv = view(m);
    mv.uprev = s->uprev_on ? s->uprev : nullptr;
    Outputs o{val64, nullptr, nullptr, nullptr, nullptr, npl, dpart, spart, nullptr};
    const unsigned nbe = blocks_for(m->ne, kElemBlock);
    if (m->d == 2) k_assemble_A<2><<<nbe, kElemBlock, 0, st>>>(mv, s->nu, s->mu, s->conv, s->w, s->fbar, s->nrhs, o, DK);
    else k_assemble_A<3><<<nbe, kElemBlock, 0, st>>>(mv, s->nu, s->mu, s->conv, s->w, s->fbar, s->nrhs, o, DK);
    CR_CUDA(cudaGetLastError());
    const unsigned nbf = blocks_for(m->nf, 256);
    if (m->d == 2) k_merge<2><<<nbf, 256, 0, st>>>(m->nf, s->nrhs, dpart, spart, o, R, minv64, nullptr);
    else k_merge<3><<<nbf, 256, 0, st>>>(m->nf, s->nrhs, dpart, spart, o, R, minv64, nullptr);
    CR_CUDA(cudaGetLastError());
    return CR_OK;
}

int launch_rhs_previous(cr_hybrid* h, const double* up, const double* gdiv, double* spart, double* S,
                        cudaStream_t st) {
    cr_system* s = h->s;
    cr_mesh* m = h->m;
    if (s->conv != CR_CONV_NONE || !(s->mu > 0.0))
        return fail(CR_ERR_ARG, "transient preconditioner: needs a Stokes system with mu > 0");
    MeshView mv = view(m);
    const unsigned nbe = blocks_for(m->ne, kElemBlock), nbf = blocks_for(m->nf, 256);
    if (m->d == 2) {
        k_rhs_previous<2><<<nbe, kElemBlock, 0, st>>>(mv, s->nu, s->mu, up, gdiv, spart, h->status);
        k_merge_rhs<2><<<nbf, 256, 0, st>>>(m->nf, spart, S);
    } else {
        k_rhs_previous<3><<<nbe, kElemBlock, 0, st>>>(mv, s->nu, s->mu, up, gdiv, spart, h->status);
        k_merge_rhs<3><<<nbf, 256, 0, st>>>(m->nf, spart, S);
    }
    CR_CUDA(cudaGetLastError());
    return CR_OK;
}

int launch_recover_previous(cr_hybrid* h, const double* up, const double* gdiv, const double* W, double* U,
                            double* P, cudaStream_t st) {
    cr_system* s = h->s;
    cr_mesh* m = h->m;
    if (s->conv != CR_CONV_NONE || !(s->mu > 0.0))
        return fail(CR_ERR_ARG, "transient preconditioner: needs a Stokes system with mu > 0");
    MeshView mv = view(m);
    mv.uprev = up;
    const unsigned nb = blocks_for(m->ne, kBlock);
    if (nb > unsigned(kMaxRedBlocks)) return fail(CR_ERR_ARG, "mesh too large for one reduction pass");
    if (m->d == 2)
        k_recover_stokes<2><<<nb, kBlock, 0, st>>>(mv, s->nu, s->mu, nullptr, nullptr, W, U, nullptr, P, h->red, h->pvol,
                                                   gdiv);
    else
        k_recover_stokes<3><<<nb, kBlock, 0, st>>>(mv, s->nu, s->mu, nullptr, nullptr, W, U, nullptr, P, h->red, h->pvol,
                                                   gdiv);
    CR_CUDA(cudaGetLastError());
    return CR_OK;
}

int launch_face_mass(cr_mesh* m, double* mass, cudaStream_t st) {
    MeshView mv = view(m);
    const unsigned nbf = blocks_for(m->nf, 256);
    if (m->d == 2) k_face_mass<2><<<nbf, 256, 0, st>>>(mv, mass);
    else k_face_mass<3><<<nbf, 256, 0, st>>>(mv, mass);
    CR_CUDA(cudaGetLastError());
    return CR_OK;
}

int launch_recover(cr_hybrid* h, int rhs, const double* W, double* U, double* P, int normalise, double* jump_dev,
                   cudaStream_t st) {
    cr_system* s = h->s;
    cr_mesh* m = h->m;
    MeshView mv = view(m);
    mv.uprev = s->uprev_on ? s->uprev + size_t(rhs) * m->nf * m->d : nullptr;
    const unsigned nb = blocks_for(m->ne, kBlock);
    const double* lam = s->mu == 0.0 ? h->lam : nullptr;
    const double* fb = s->fbar + size_t(rhs) * m->ne * m->d;
    double* ualt = jump_dev ? h->ualt : nullptr;
    double* mean = h->pvol;
    if (nb > unsigned(kMaxRedBlocks)) return fail(CR_ERR_ARG, "mesh too large for one reduction pass");
    if (s->conv != CR_CONV_NONE)
        k_recover_conv2<<<nb, kBlock, 0, st>>>(mv, s->nu, s->mu, s->conv, s->w, lam, fb, W, U, ualt, P, h->red, mean);
    else if (m->d == 2)
        k_recover_stokes<2><<<nb, kBlock, 0, st>>>(mv, s->nu, s->mu, lam, fb, W, U, ualt, P, h->red, mean);
    else
        k_recover_stokes<3><<<nb, kBlock, 0, st>>>(mv, s->nu, s->mu, lam, fb, W, U, ualt, P, h->red, mean);
    CR_CUDA(cudaGetLastError());
    if (normalise) {
        k_subtract_mean<<<blocks_for(m->ne, 256), 256, 0, st>>>(m->ne, mean, P);
        CR_CUDA(cudaGetLastError());
    }
    if (jump_dev) {
        const int64_t n = m->nf * m->d;
        CR_CUDA(cudaMemsetAsync(jump_dev, 0, sizeof(double), st));
        k_jump<<<blocks_for(n, kBlock), kBlock, 0, st>>>(n, U, ualt, h->red, jump_dev);
        CR_CUDA(cudaGetLastError());
    }
    return CR_OK;
}

}  // namespace crhyb
