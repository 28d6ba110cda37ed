// Host-side mesh topology for the CR scheme (Section 2, item 1; Section 3.2).
//
// Faces are identified by their sorted vertex tuples.  All (simplex, local
// face) incidences are sorted by that tuple with a stable LSD radix sort, so
// equal faces become adjacent runs in increasing simplex order: a run of two
// is an interior face (the lower simplex owns it, C = +1, Eq. 12), a run of
// one an exterior face, a longer run an invalid mesh.  Interior faces are
// numbered in run order, i.e. in lexicographic order of their vertex tuples.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace {

// Stable LSD radix sort of (key, index) pairs by key, 16-bit digits.
void radix_sort_pairs(std::vector<uint64_t>& key, std::vector<uint32_t>& idx, int key_bits) {
    const size_t n = key.size();
    std::vector<uint64_t> k2(n);
    std::vector<uint32_t> i2(n);
    std::vector<size_t> cnt(1 << 16);
    for (int shift = 0; shift < key_bits; shift += 16) {
        std::fill(cnt.begin(), cnt.end(), 0);
        for (size_t t = 0; t < n; ++t) cnt[(key[t] >> shift) & 0xFFFF]++;
        size_t sum = 0;
        for (auto& c : cnt) { size_t v = c; c = sum; sum += v; }
        for (size_t t = 0; t < n; ++t) {
            size_t pos = cnt[(key[t] >> shift) & 0xFFFF]++;
            k2[pos] = key[t];
            i2[pos] = idx[t];
        }
        key.swap(k2);
        idx.swap(i2);
    }
}

}  // namespace

extern "C" int cr_mesh_load(int dim, const double* coords, int64_t nv, const int32_t* elems, int64_t ne,
                            const cr_mesh_opts* opts, void* stream, cr_mesh** out) {
    using namespace crhyb;
    if (!out) return fail(CR_ERR_ARG, "cr_mesh_load: out is NULL");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(CR_ERR_ARG, "cr_mesh_load: dim must be 2 or 3");
    if (!coords || !elems || nv <= 0 || ne <= 1) return fail(CR_ERR_ARG, "cr_mesh_load: empty mesh");
    if (ne >= (int64_t(1) << 31) / (dim + 1)) return fail(CR_ERR_ARG, "cr_mesh_load: too many simplices");
    if (pointer_place(coords, nullptr) != 0 || pointer_place(elems, nullptr) != 0)
        return fail(CR_ERR_ARG, "cr_mesh_load: coords and elems must be host arrays");
    const int d = dim, dp1 = dim + 1;
    int k0 = opts ? opts->k0 : 0;
    if (k0 < 0 || k0 >= ne) return fail(CR_ERR_ARG, "cr_mesh_load: k0 out of range");

    // ---- validate indices and measures ----
    for (int64_t t = 0; t < ne * dp1; ++t)
        if (elems[t] < 0 || elems[t] >= nv) return fail(CR_ERR_MESH, "cr_mesh_load: vertex index out of range");
    {
        double vmax = 0.0;
        std::vector<double> det(ne);
        for (int64_t K = 0; K < ne; ++K) {
            const int32_t* e = elems + K * dp1;
            double J[3][3] = {{0}};
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) J[b][a] = coords[e[a + 1] * d + b] - coords[e[0] * d + b];
            double dt;
            if (d == 2) dt = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            else dt = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                      J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
            det[K] = std::fabs(dt);
            vmax = std::max(vmax, det[K]);
        }
        for (int64_t K = 0; K < ne; ++K)
            if (!(det[K] > 1e-13 * vmax)) return fail(CR_ERR_MESH, "cr_mesh_load: simplex " + std::to_string(K) + " has zero measure");
    }

    // ---- face keys ----
    const int64_t ninc = ne * dp1;
    const bool packed = (d == 2) ? (nv <= (int64_t(1) << 32)) : (nv <= (int64_t(1) << 21));
    if (!packed) return fail(CR_ERR_ARG, "cr_mesh_load: too many vertices for the face-key packing");
    std::vector<uint64_t> key(ninc);
    std::vector<uint32_t> idx(ninc);
    for (int64_t K = 0; K < ne; ++K) {
        const int32_t* e = elems + K * dp1;
        for (int l = 0; l < dp1; ++l) {
            uint32_t v[3];
            int c = 0;
            for (int m = 0; m < dp1; ++m)
                if (m != l) v[c++] = uint32_t(e[m]);
            std::sort(v, v + d);
            uint64_t k = (d == 2) ? ((uint64_t(v[0]) << 32) | v[1])
                                  : ((uint64_t(v[0]) << 42) | (uint64_t(v[1]) << 21) | v[2]);
            key[K * dp1 + l] = k;
            idx[K * dp1 + l] = uint32_t(K * dp1 + l);
        }
    }
    radix_sort_pairs(key, idx, 64);

    cr_mesh* m = new cr_mesh();
    m->d = d;
    m->ne = ne;
    m->nv = nv;
    m->k0 = k0;
    std::vector<int32_t> elem_face(ninc, -1);
    std::vector<uint8_t> elem_side(ninc, 0);
    int64_t nf = 0, next = 0;
    for (int64_t t = 0; t < ninc;) {
        int64_t u = t + 1;
        while (u < ninc && key[u] == key[t]) ++u;
        const int64_t run = u - t;
        if (run > 2) {
            delete m;
            return fail(CR_ERR_MESH, "cr_mesh_load: a face belongs to more than two simplices");
        }
        if (run == 2) {
            const uint32_t a = idx[t], b = idx[t + 1];   // stable sort: a belongs to the lower simplex
            const int64_t Ka = a / dp1, Kb = b / dp1;
            if (Ka == Kb) {
                delete m;
                return fail(CR_ERR_MESH, "cr_mesh_load: a simplex repeats a face");
            }
            elem_face[a] = int32_t(nf);
            elem_face[b] = int32_t(nf);
            elem_side[a] = 0;
            elem_side[b] = 1;
            m->h_face_elems.push_back(int32_t(Ka));
            m->h_face_elems.push_back(int32_t(Kb));
            m->h_face_local.push_back(int32_t(a % dp1));
            m->h_face_local.push_back(int32_t(b % dp1));
            const uint64_t k = key[t];
            if (d == 2) {
                m->h_face_vertices.push_back(int32_t(k >> 32));
                m->h_face_vertices.push_back(int32_t(k & 0xFFFFFFFFu));
            } else {
                m->h_face_vertices.push_back(int32_t(k >> 42));
                m->h_face_vertices.push_back(int32_t((k >> 21) & 0x1FFFFF));
                m->h_face_vertices.push_back(int32_t(k & 0x1FFFFF));
            }
            ++nf;
        } else {
            ++next;
        }
        t = u;
    }
    m->nf = nf;
    m->nf_ext = next;
    if (nf == 0) {
        delete m;
        return fail(CR_ERR_MESH, "cr_mesh_load: the mesh has no interior face");
    }

    // ---- ELL columns (slots 1..2d), sliced ----
    const int64_t nfp = (nf + kSlice - 1) / kSlice * kSlice;
    m->nfp = nfp;
    std::vector<int32_t> cols(size_t(2 * d) * nfp, 0);
    for (int64_t f = 0; f < nf; ++f) {
        for (int s = 0; s < 2; ++s) {
            const int64_t E = m->h_face_elems[2 * f + s];
            const int l = m->h_face_local[2 * f + s];
            for (int r = 0; r < d; ++r) {
                const int mm = r < l ? r : r + 1;
                const int32_t c = elem_face[E * dp1 + mm];
                cols[sell(f, s * d + r, 2 * d)] = c < 0 ? int32_t(f) : c;
            }
        }
    }

    // ---- maximal independent set (greedy, increasing simplex index) ----
    if (opts && opts->need_mis) {
        m->h_mis.assign(ne, 0);
        for (int64_t K = 0; K < ne; ++K) {
            bool free_ = true;
            for (int l = 0; l < dp1 && free_; ++l) {
                const int32_t f = elem_face[K * dp1 + l];
                if (f < 0) continue;
                const int64_t L = m->h_face_elems[2 * f + (1 - elem_side[K * dp1 + l])];
                if (m->h_mis[L]) free_ = false;
            }
            if (free_) m->h_mis[K] = 1;
        }
        m->has_mis = true;
    }

    // ---- device copies ----
    m->user_stream = static_cast<cudaStream_t>(stream);
    auto cleanup = [&](int rc) { cr_destroy_mesh(m); return rc; };
    cudaError_t e = cudaGetDevice(&m->device);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaGetDevice"));
    e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaStreamCreateWithFlags"));
    if ((e = cudaEventCreateWithFlags(&m->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaEventCreate"));
    int rc;
    if ((rc = m->arena.alloc_n(&m->coords, size_t(nv) * d)) ||
        (rc = m->arena.alloc_n(&m->elems, size_t(ninc))) ||
        (rc = m->arena.alloc_n(&m->elem_face, size_t(ninc))) ||
        (rc = m->arena.alloc_n(&m->elem_side, size_t(ninc))) ||
        (rc = m->arena.alloc_n(&m->face_elems, size_t(2 * nf))) ||
        (rc = m->arena.alloc_n(&m->face_local, size_t(2 * nf))) ||
        (rc = m->arena.alloc_n(&m->cols, size_t(2 * d) * nfp)))
        return cleanup(rc);
    if (m->has_mis && (rc = m->arena.alloc_n(&m->mis, size_t(ne)))) return cleanup(rc);
    struct Cp { void* dst; const void* src; size_t bytes; };
    const size_t ni = size_t(ninc), nvd = size_t(nv) * d, nf2 = size_t(2 * nf);
    const Cp cps[] = {
        {m->coords, coords, sizeof(double) * nvd},
        {m->elems, elems, sizeof(int32_t) * ni},
        {m->elem_face, elem_face.data(), sizeof(int32_t) * ni},
        {m->elem_side, elem_side.data(), ni},
        {m->face_elems, m->h_face_elems.data(), sizeof(int32_t) * nf2},
        {m->face_local, m->h_face_local.data(), sizeof(int32_t) * nf2},
        {m->cols, cols.data(), sizeof(int32_t) * cols.size()},
        {m->mis, m->h_mis.data(), m->h_mis.size()},
    };
    for (auto& c : cps) {
        if (!c.dst || !c.bytes) continue;
        e = cudaMemcpy(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMemcpy (mesh upload)"));
    }
    *out = m;
    return CR_OK;
}

extern "C" int cr_mesh_info(const cr_mesh* m, int32_t* dim, int64_t* ne, int64_t* nf_int, int64_t* nf_ext) {
    if (!m) return crhyb::fail(CR_ERR_ARG, "cr_mesh_info: NULL mesh");
    if (dim) *dim = m->d;
    if (ne) *ne = m->ne;
    if (nf_int) *nf_int = m->nf;
    if (nf_ext) *nf_ext = m->nf_ext;
    return CR_OK;
}

static int copy_out(void* dst, const void* src, size_t bytes) {
    if (!bytes) return CR_OK;
    cudaError_t e = cudaMemcpy(dst, src, bytes, crhyb::is_device_pointer(dst) ? cudaMemcpyHostToDevice
                                                                             : cudaMemcpyHostToHost);
    if (e != cudaSuccess) return crhyb::cuda_fail(e, "cudaMemcpy (export)");
    return CR_OK;
}

extern "C" int cr_mesh_faces(const cr_mesh* m, int32_t* fv) {
    if (!m || !fv) return crhyb::fail(CR_ERR_ARG, "cr_mesh_faces: NULL argument");
    CR_TRY(crhyb::check_call(m, "cr_mesh_faces", {fv}));
    return copy_out(fv, m->h_face_vertices.data(), sizeof(int32_t) * m->h_face_vertices.size());
}

extern "C" int cr_mesh_face_elements(const cr_mesh* m, int32_t* fe, int32_t* fl) {
    if (!m) return crhyb::fail(CR_ERR_ARG, "cr_mesh_face_elements: NULL mesh");
    CR_TRY(crhyb::check_call(m, "cr_mesh_face_elements", {fe, fl}));
    if (fe) CR_TRY(copy_out(fe, m->h_face_elems.data(), sizeof(int32_t) * m->h_face_elems.size()));
    if (fl) CR_TRY(copy_out(fl, m->h_face_local.data(), sizeof(int32_t) * m->h_face_local.size()));
    return CR_OK;
}

extern "C" int cr_mesh_mis(const cr_mesh* m, uint8_t* in_m1) {
    if (!m || !in_m1) return crhyb::fail(CR_ERR_ARG, "cr_mesh_mis: NULL argument");
    if (!m->has_mis) return crhyb::fail(CR_ERR_ARG, "cr_mesh_mis: mesh loaded without need_mis");
    CR_TRY(crhyb::check_call(m, "cr_mesh_mis", {in_m1}));
    return copy_out(in_m1, m->h_mis.data(), m->h_mis.size());
}

extern "C" void cr_destroy_mesh(cr_mesh* m) {
    if (!m) return;
    m->arena.release();
    if (m->ev_in) cudaEventDestroy(m->ev_in);
    if (m->ev_out) cudaEventDestroy(m->ev_out);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}
