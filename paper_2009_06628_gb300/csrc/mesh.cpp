// Host-side mesh construction (Section 4): validation of a Morton-sorted leaf list,
// independent-node enumeration, element-to-node map with hanging-node constraints,
// boundary nodes, and the upload to the current CUDA device.
#include <algorithm>
#include <cmath>
#include <parallel/algorithm>
#include <cstring>
#include <new>
#include <utility>

#include "chns_internal.h"
#include "morton.h"

namespace {

struct Leaves {
    int dim, L;
    std::vector<uint64_t> key;
    std::vector<int32_t> level;
    // index of the leaf containing point p (p inside the domain)
    int64_t containing(const int64_t* p) const {
        uint64_t k = morton(dim, p);
        auto it = std::upper_bound(key.begin(), key.end(), k);
        return (int64_t)(it - key.begin()) - 1;
    }
    bool is_leaf(const int64_t* anchor, int lev) const {
        int64_t j = containing(anchor);
        return j >= 0 && key[j] == morton(dim, anchor) && level[j] == lev;
    }
};

template <class T>
chns_status dev_upload(T** dst, const std::vector<T>& src) {
    size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)dst, bytes);
    if (e != cudaSuccess) return chns_cuda_status(e, "cudaMalloc(mesh)");
    if (!src.empty()) {
        e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return chns_cuda_status(e, "cudaMemcpy(mesh)");
    }
    return CHNS_OK;
}

}  // namespace

extern "C" chns_status chns_mesh_create(int32_t dim, int32_t max_level, int64_t n_leaves,
                                        const chns_leaf* leaves, double lo, double hi,
                                        chns_mesh** out) {
    chns_set_error("");
    if (!out || !leaves) { chns_set_error("null argument"); return CHNS_EINVAL; }
    *out = nullptr;
    if (dim != 2 && dim != 3) { chns_set_error("dim must be 2 or 3"); return CHNS_EINVAL; }
    if (max_level < 1 || max_level > 20) { chns_set_error("max_level must be in [1, 20]"); return CHNS_EINVAL; }
    if (n_leaves <= 0 || n_leaves > ((int64_t)1 << 31) / 8) { chns_set_error("bad n_leaves"); return CHNS_EINVAL; }
    if (!(hi > lo)) { chns_set_error("domain must satisfy hi > lo"); return CHNS_EINVAL; }
    const int d = dim, nc = 1 << dim, L = max_level;
    const int64_t n_side = (int64_t)1 << L;
    const int64_t E = n_leaves;

    Leaves lv;
    lv.dim = d;
    lv.L = L;
    lv.key.resize(E);
    lv.level.resize(E);
    std::vector<int64_t> anchor((size_t)E * d);
    for (int64_t e = 0; e < E; ++e) {
        const chns_leaf& f = leaves[e];
        int64_t a[3] = {f.x, f.y, f.z};
        if (f.level < 0 || f.level > L) { chns_set_error("leaf level out of range"); return CHNS_EINVAL; }
        if (d == 2 && f.z != 0) { chns_set_error("2D leaves need z == 0"); return CHNS_EINVAL; }
        int64_t s = (int64_t)1 << (L - f.level);
        for (int k = 0; k < d; ++k) {
            if (a[k] < 0 || a[k] + s > n_side) { chns_set_error("leaf outside the domain"); return CHNS_ENOTCOMPLETE; }
            if (a[k] % s) { chns_set_error("leaf anchor not aligned to its size"); return CHNS_ENOTCOMPLETE; }
            anchor[(size_t)e * d + k] = a[k];
        }
        lv.key[e] = morton(d, a);
        lv.level[e] = f.level;
    }
    for (int64_t e = 0; e + 1 < E; ++e)
        if (lv.key[e + 1] <= lv.key[e]) { chns_set_error("leaves are not sorted in Morton order"); return CHNS_ENOTSORTED; }
    // completeness: consecutive Morton ranges tile [0, 2^(L d))
    {
        uint64_t expect = 0;
        for (int64_t e = 0; e < E; ++e) {
            if (lv.key[e] != expect) { chns_set_error("leaves overlap or leave a gap"); return CHNS_ENOTCOMPLETE; }
            uint64_t s = (uint64_t)1 << (L - lv.level[e]);
            expect += (d == 2) ? s * s : s * s * s;
        }
        uint64_t total = (uint64_t)1 << (L * d);
        if (expect != total) { chns_set_error("leaves do not cover the domain"); return CHNS_ENOTCOMPLETE; }
    }
    // full 2:1 balance: the leaf holding a point just outside each face/edge/vertex
    // may be at most one level coarser
    int unbalanced = 0;
#pragma omp parallel for schedule(static) reduction(| : unbalanced)
    for (int64_t e = 0; e < E; ++e) {
        const int64_t* a = &anchor[(size_t)e * d];
        int64_t s = (int64_t)1 << (L - lv.level[e]);
        int ndir = (d == 2) ? 9 : 27;
        for (int t = 0; t < ndir; ++t) {
            int dv[3] = {t % 3 - 1, (t / 3) % 3 - 1, (t / 9) % 3 - 1};
            if (dv[0] == 0 && dv[1] == 0 && (d == 2 || dv[2] == 0)) continue;
            int64_t p[3] = {0, 0, 0};
            bool inside = true;
            for (int k = 0; k < d; ++k) {
                p[k] = dv[k] < 0 ? a[k] - 1 : (dv[k] > 0 ? a[k] + s : a[k]);
                if (p[k] < 0 || p[k] >= n_side) inside = false;
            }
            if (!inside) continue;
            int64_t j = lv.containing(p);
            if (lv.level[j] < lv.level[e] - 1) unbalanced = 1;
        }
    }
    if (unbalanced) { chns_set_error("octree is not 2:1 balanced"); return CHNS_ENOTBALANCED; }

    // corners: hanging test and keys (Morton with L + 1 bits per axis)
    const size_t ncorner = (size_t)E * nc;
    std::vector<uint64_t> ckey(ncorner);
    std::vector<uint8_t> chang(ncorner, 0);
    std::vector<uint64_t> node_keys;
    node_keys.reserve(ncorner / 2 + 16);
    std::vector<std::pair<uint64_t, int64_t>> hang_pts;  // (key, corner index)
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        const int64_t* a = &anchor[(size_t)e * d];
        int lev = lv.level[e];
        int64_t s = (int64_t)1 << (L - lev);
        for (int c = 0; c < nc; ++c) {
            int64_t p[3] = {0, 0, 0};
            for (int k = 0; k < d; ++k) p[k] = a[k] + (((c >> k) & 1) ? s : 0);
            size_t ci = (size_t)e * nc + c;
            ckey[ci] = morton(d, p);
            bool odd[3] = {false, false, false};
            int nodd = 0;
            for (int k = 0; k < d; ++k) {
                odd[k] = ((p[k] / s) & 1) != 0;
                nodd += odd[k];
            }
            bool hanging = false;
            if (lev > 0 && nodd >= 1 && nodd <= 2 && nodd < d) {
                int free_ax[3], nfree = 0;
                for (int k = 0; k < d; ++k)
                    if (!odd[k]) free_ax[nfree++] = k;
                for (int combo = 0; combo < (1 << nfree) && !hanging; ++combo) {
                    int64_t q[3] = {0, 0, 0};
                    bool ok = true;
                    for (int k = 0; k < d; ++k) q[k] = odd[k] ? p[k] - s : p[k];
                    for (int j = 0; j < nfree; ++j)
                        if ((combo >> j) & 1) q[free_ax[j]] = p[free_ax[j]] - 2 * s;
                    for (int k = 0; k < d; ++k)
                        if (q[k] < 0 || q[k] >= n_side) ok = false;
                    if (ok && lv.is_leaf(q, lev - 1)) hanging = true;
                }
            }
            chang[ci] = hanging ? 1 : 0;
        }
    }
    for (size_t ci = 0; ci < ncorner; ++ci) {
        if (chang[ci])
            hang_pts.push_back({ckey[ci], (int64_t)ci});
        else
            node_keys.push_back(ckey[ci]);
    }
    __gnu_parallel::sort(node_keys.begin(), node_keys.end());
    node_keys.erase(std::unique(node_keys.begin(), node_keys.end()), node_keys.end());
    __gnu_parallel::sort(hang_pts.begin(), hang_pts.end());
    std::vector<uint64_t> hang_keys;
    std::vector<int64_t> hang_corner;
    for (auto& hp : hang_pts)
        if (hang_keys.empty() || hang_keys.back() != hp.first) {
            hang_keys.push_back(hp.first);
            hang_corner.push_back(hp.second);
        }
    const int64_t N = (int64_t)node_keys.size();
    const int64_t H = (int64_t)hang_keys.size();
    auto node_of = [&](uint64_t k) -> int64_t {
        auto it = std::lower_bound(node_keys.begin(), node_keys.end(), k);
        if (it == node_keys.end() || *it != k) return -1;
        return (int64_t)(it - node_keys.begin());
    };

    std::vector<int32_t> e2n(ncorner);
#pragma omp parallel for schedule(static)
    for (int64_t cii = 0; cii < (int64_t)ncorner; ++cii) {
        const size_t ci = (size_t)cii;
        if (!chang[ci]) {
            e2n[ci] = (int32_t)node_of(ckey[ci]);
        } else {
            auto it = std::lower_bound(hang_keys.begin(), hang_keys.end(), ckey[ci]);
            e2n[ci] = -(int32_t)(it - hang_keys.begin()) - 1;
        }
    }
    std::vector<int32_t> hang((size_t)std::max<int64_t>(H, 1) * 4, -1);
    for (int64_t h = 0; h < H; ++h) {
        int64_t ci = hang_corner[h];
        int64_t e = ci / nc;
        int c = (int)(ci % nc);
        const int64_t* a = &anchor[(size_t)e * d];
        int64_t s = (int64_t)1 << (L - lv.level[e]);
        int64_t p[3] = {0, 0, 0};
        int odd_ax[3], nodd = 0;
        for (int k = 0; k < d; ++k) {
            p[k] = a[k] + (((c >> k) & 1) ? s : 0);
            if ((p[k] / s) & 1) odd_ax[nodd++] = k;
        }
        for (int m = 0; m < (1 << nodd); ++m) {
            int64_t q[3] = {p[0], p[1], p[2]};
            for (int j = 0; j < nodd; ++j) q[odd_ax[j]] += ((m >> j) & 1) ? s : -s;
            int64_t n = node_of(morton(d, q));
            if (n < 0) { chns_set_error("a hanging node's parent is itself hanging (octree not 2:1 balanced)"); return CHNS_ENOTBALANCED; }
            hang[(size_t)h * 4 + m] = (int32_t)n;
        }
    }

    chns_mesh* m = new (std::nothrow) chns_mesh();
    if (!m) { chns_set_error("host allocation failed"); return CHNS_ENOMEM; }
    m->max_level = L;
    m->node_coords.resize((size_t)N * d);
    std::vector<uint8_t> nflag(N, 0);
    std::vector<int32_t> bnodes;
    for (int64_t n = 0; n < N; ++n) {
        uint64_t k = node_keys[n];
        bool bnd = false;
        for (int c = 0; c < d; ++c) {
            int64_t v = 0;
            for (int b = 0; b <= L; ++b) v |= (int64_t)((k >> (b * d + c)) & 1) << b;
            m->node_coords[(size_t)n * d + c] = (int32_t)v;
            if (v == 0 || v == n_side) bnd = true;
        }
        if (bnd) {
            nflag[n] = (uint8_t)((1u << d) - 1u);   // no-slip: every velocity component
            bnodes.push_back((int32_t)n);
        }
    }
    // integral of each independent node's Q1 basis function: a corner of element e
    // carries |e| / 2^d, shared among its parents with the constraint weights
    std::vector<double> nmass(N, 0.0);
    const double dom = hi - lo;
    for (int64_t e = 0; e < E; ++e) {
        const double h = std::ldexp(dom, -lv.level[e]);
        const double share = (d == 2 ? h * h : h * h * h) / nc;
        for (int c = 0; c < nc; ++c) {
            const int32_t ent = e2n[(size_t)e * nc + c];
            if (ent >= 0) {
                nmass[ent] += share;
            } else {
                const int32_t* hp = &hang[(size_t)(-ent - 1) * 4];
                const int np = hp[2] < 0 ? 2 : 4;
                for (int j = 0; j < np; ++j) nmass[hp[j]] += share / np;
            }
        }
    }
    std::vector<int32_t> anchor32((size_t)E * d);
    for (size_t i = 0; i < anchor32.size(); ++i) anchor32[i] = (int32_t)anchor[i];
    std::vector<int8_t> level8(E);
    for (int64_t e = 0; e < E; ++e) level8[e] = (int8_t)lv.level[e];

    {
        cudaError_t de = cudaGetDevice(&m->device);
        if (de != cudaSuccess) {
            chns_mesh_destroy(m);
            return chns_cuda_status(de, "cudaGetDevice");
        }
    }
    chns_status st;
    if ((st = dev_upload(&m->d_e2n, e2n)) != CHNS_OK ||
        (st = dev_upload(&m->d_hang, hang)) != CHNS_OK ||
        (st = dev_upload(&m->d_level, level8)) != CHNS_OK ||
        (st = dev_upload(&m->d_nflag, nflag)) != CHNS_OK ||
        (st = dev_upload(&m->d_bnodes, bnodes)) != CHNS_OK ||
        (st = dev_upload(&m->d_anchor, anchor32)) != CHNS_OK ||
        (st = dev_upload(&m->d_nmass, nmass)) != CHNS_OK) {
        chns_mesh_destroy(m);
        return st;
    }
    m->n_partials = 4096;
    cudaError_t ce = cudaMalloc((void**)&m->d_partials, (size_t)m->n_partials * 8 * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&m->d_flags, 64);
    if (ce == cudaSuccess) ce = cudaMemset(m->d_flags, 0, 64);
    if (ce == cudaSuccess) ce = cudaMallocHost((void**)&m->h_pinned, 64 * sizeof(double));
    if (ce != cudaSuccess) {
        chns_mesh_destroy(m);
        return chns_cuda_status(ce, "cudaMalloc(mesh workspace)");
    }
    DevMesh& dm = m->dm;
    dm.dim = d;
    dm.nc = nc;
    dm.nf = d + 3;
    dm.E = E;
    dm.N = N;
    dm.H = H;
    dm.NB = (int64_t)bnodes.size();
    dm.e2n = m->d_e2n;
    dm.hang = m->d_hang;
    dm.level = m->d_level;
    dm.nflag = m->d_nflag;
    dm.bnodes = m->d_bnodes;
    dm.bcval = nullptr;
    dm.anchor = m->d_anchor;
    dm.max_level = L;
    dm.lo = lo;
    dm.hi = hi;
    m->volume = (d == 2) ? dom * dom : dom * dom * dom;
    m->h_e2n = std::move(e2n);
    m->h_hang = std::move(hang);
    m->h_anchor = std::move(anchor32);
    m->h_level = std::move(level8);
    *out = m;
    return CHNS_OK;
}

void chns_solver_ws_free(SolverWS* ws);  // solver.cu
void chns_mg_free(MGHier* mg);           // multigrid.cu

extern "C" void chns_mesh_destroy(chns_mesh* m) {
    if (!m) return;
    if (m->ws) chns_solver_ws_free(m->ws);
    if (m->mg) chns_mg_free(m->mg);
    cudaFree(m->d_e2n);
    cudaFree(m->d_hang);
    cudaFree(m->d_level);
    cudaFree(m->d_nflag);
    cudaFree(m->d_bnodes);
    cudaFree(m->d_bcval);
    cudaFree(m->d_elist);
    cudaFree(m->d_anchor);
    cudaFree(m->d_nmass);
    cudaFree(m->d_partials);
    cudaFree(m->d_flags);
    if (m->h_pinned) cudaFreeHost(m->h_pinned);
    delete m;
}

extern "C" int64_t chns_mesh_num_nodes(const chns_mesh* m) { return m ? m->dm.N : -1; }
extern "C" int64_t chns_mesh_num_elements(const chns_mesh* m) { return m ? m->dm.E : -1; }
extern "C" int64_t chns_mesh_num_hanging(const chns_mesh* m) { return m ? m->dm.H : -1; }
extern "C" int32_t chns_mesh_dim(const chns_mesh* m) { return m ? m->dm.dim : -1; }

extern "C" chns_status chns_mesh_node_coords(const chns_mesh* m, int32_t* coords) {
    if (!m || !coords) { chns_set_error("null argument"); return CHNS_EINVAL; }
    std::memcpy(coords, m->node_coords.data(), m->node_coords.size() * sizeof(int32_t));
    return CHNS_OK;
}

extern "C" chns_status chns_mesh_set_velocity_bc(chns_mesh* m, const uint8_t* face_mask, const double* values) {
    if (!m || !face_mask) { chns_set_error("chns_mesh_set_velocity_bc: null argument"); return CHNS_EINVAL; }
    const int d = m->dm.dim;
    const int64_t N = m->dm.N;
    const int64_t side = (int64_t)1 << m->max_level;
    for (int f = 0; f < 2 * d; ++f)
        if (face_mask[f] >> d) { chns_set_error("chns_mesh_set_velocity_bc: a face mask has bits >= dim"); return CHNS_EINVAL; }
    std::vector<uint8_t> nflag((size_t)N, 0);
    std::vector<int32_t> bnodes;
    for (int64_t n = 0; n < N; ++n) {
        uint8_t fl = 0;
        for (int k = 0; k < d; ++k) {
            const int32_t c = m->node_coords[(size_t)n * d + k];
            if (c == 0) fl |= face_mask[2 * k];
            if (c == side) fl |= face_mask[2 * k + 1];
        }
        nflag[(size_t)n] = fl;
        if (fl) bnodes.push_back((int32_t)n);
    }
    int32_t* nb = nullptr;
    double* bv = nullptr;
    cudaError_t e = cudaMalloc((void**)&nb, std::max<size_t>(bnodes.size(), 1) * sizeof(int32_t));
    if (e == cudaSuccess && !bnodes.empty())
        e = cudaMemcpy(nb, bnodes.data(), bnodes.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_nflag, nflag.data(), (size_t)N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && values) {
        e = cudaMalloc((void**)&bv, (size_t)N * d * sizeof(double));
        if (e == cudaSuccess) e = cudaMemcpy(bv, values, (size_t)N * d * sizeof(double), cudaMemcpyDeviceToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(nb);
        cudaFree(bv);
        return chns_cuda_status(e, "chns_mesh_set_velocity_bc");
    }
    cudaFree(m->d_bnodes);
    cudaFree(m->d_bcval);
    m->d_bnodes = nb;
    m->d_bcval = bv;
    m->dm.bnodes = nb;
    m->dm.bcval = bv;
    m->dm.NB = (int64_t)bnodes.size();
    if (m->mg) {
        // coarse multigrid levels keep the pressure operator only; nothing to update
    }
    return CHNS_OK;
}

// Greedy element colouring for the deterministic scatter: two elements that share an
// independent node (a corner, or a constraint parent of a hanging corner) get different
// colours.  Elements are visited in Morton order and take the smallest colour not used by
// an already coloured element sharing one of their nodes; within a colour the Morton
// order is kept.
static chns_status build_colouring(chns_mesh* m) {
    const int64_t E = m->dm.E, N = m->dm.N;
    const int nc = m->dm.nc;
    auto nodes_of = [&](int64_t e, int32_t* out) -> int {
        int k = 0;
        for (int a = 0; a < nc; ++a) {
            const int32_t ent = m->h_e2n[(size_t)e * nc + a];
            if (ent >= 0) {
                out[k++] = ent;
            } else {
                const int32_t* hp = &m->h_hang[(size_t)(-ent - 1) * 4];
                const int np = hp[2] < 0 ? 2 : 4;
                for (int j = 0; j < np; ++j) out[k++] = hp[j];
            }
        }
        return k;
    };
    std::vector<int64_t> off((size_t)N + 1, 0);
    int32_t buf[32];
    for (int64_t e = 0; e < E; ++e) {
        const int k = nodes_of(e, buf);
        for (int i = 0; i < k; ++i) off[(size_t)buf[i] + 1]++;
    }
    for (int64_t n = 0; n < N; ++n) off[(size_t)n + 1] += off[(size_t)n];
    std::vector<int32_t> adj((size_t)off[(size_t)N]);
    {
        std::vector<int64_t> pos(off.begin(), off.end() - 1);
        for (int64_t e = 0; e < E; ++e) {
            const int k = nodes_of(e, buf);
            for (int i = 0; i < k; ++i) adj[(size_t)pos[(size_t)buf[i]]++] = (int32_t)e;
        }
    }
    std::vector<int8_t> colour((size_t)E, -1);
    int ncol = 0;
    for (int64_t e = 0; e < E; ++e) {
        uint64_t used = 0;
        const int k = nodes_of(e, buf);
        for (int i = 0; i < k; ++i)
            for (int64_t j = off[(size_t)buf[i]]; j < off[(size_t)buf[i] + 1]; ++j) {
                const int8_t c = colour[(size_t)adj[(size_t)j]];
                if (c >= 0) used |= 1ull << c;
            }
        int c = 0;
        while (c < 64 && ((used >> c) & 1ull)) ++c;
        if (c >= 64) { chns_set_error("element colouring needs more than 64 colours"); return CHNS_EINVAL; }
        colour[(size_t)e] = (int8_t)c;
        ncol = std::max(ncol, c + 1);
    }
    std::vector<int64_t> coff((size_t)ncol + 1, 0);
    for (int64_t e = 0; e < E; ++e) coff[(size_t)colour[(size_t)e] + 1]++;
    for (int c = 0; c < ncol; ++c) coff[(size_t)c + 1] += coff[(size_t)c];
    std::vector<int32_t> elist((size_t)E);
    {
        std::vector<int64_t> pos(coff.begin(), coff.end() - 1);
        for (int64_t e = 0; e < E; ++e) elist[(size_t)pos[(size_t)colour[(size_t)e]]++] = (int32_t)e;
    }
    int32_t* d = nullptr;
    chns_status st = dev_upload(&d, elist);
    if (st != CHNS_OK) return st;
    cudaFree(m->d_elist);
    m->d_elist = d;
    m->colour_off = coff;
    return CHNS_OK;
}

extern "C" chns_status chns_mesh_set_scatter(chns_mesh* m, int32_t mode) {
    if (!m || mode < 0 || mode > 2) {
        chns_set_error("chns_mesh_set_scatter: mode must be 0 (atomics), 1 (colouring) or 2 (warp-aggregated)");
        return CHNS_EINVAL;
    }
    if (mode != 0 && chns_require_q1(m, "scatter modes 1 and 2") != CHNS_OK) return CHNS_EINVAL;
    if (mode == 1 && m->colour_off.empty()) {
        chns_status st = build_colouring(m);
        if (st != CHNS_OK) return st;
    }
    m->scatter = mode;
    return CHNS_OK;
}

extern "C" int32_t chns_mesh_num_colours(const chns_mesh* m) {
    return (m && !m->colour_off.empty()) ? (int32_t)m->colour_off.size() - 1 : 0;
}

// Q2 mesh of a uniform octree at `level`: elements in Morton order of their anchors, 3^d
// nodes each on the lattice of half the element size, numbered in Morton order of their
// integer coordinates (units of 2^-(level + 1)); no hanging nodes.
extern "C" chns_status chns_mesh_create_q2(int32_t dim, int32_t level, double lo, double hi, chns_mesh** out) {
    chns_set_error("");
    if (!out) { chns_set_error("null argument"); return CHNS_EINVAL; }
    *out = nullptr;
    if (dim != 2 && dim != 3) { chns_set_error("dim must be 2 or 3"); return CHNS_EINVAL; }
    if (level < 1 || level > (dim == 3 ? 8 : 11)) {
        chns_set_error("Q2 level must be in [1, 8] (3D) or [1, 11] (2D)");
        return CHNS_EINVAL;
    }
    if (!(hi > lo)) { chns_set_error("domain must satisfy hi > lo"); return CHNS_EINVAL; }
    const int d = dim, L = level, NN = d == 2 ? 9 : 27;
    const int64_t n = (int64_t)1 << L, E = d == 2 ? n * n : n * n * n;
    const int64_t side = 2 * n;
    std::vector<std::pair<uint64_t, int64_t>> ek((size_t)E);
    for (int64_t i = 0; i < E; ++i) {
        int64_t a[3] = {i % n, (i / n) % n, d == 3 ? i / (n * n) : 0};
        ek[(size_t)i] = {morton(d, a), i};
    }
    std::sort(ek.begin(), ek.end());
    std::vector<int32_t> anchor((size_t)E * d);
    std::vector<uint64_t> nkeys;
    nkeys.reserve((size_t)E * NN);
    for (int64_t e = 0; e < E; ++e) {
        const int64_t i = ek[(size_t)e].second;
        const int64_t a[3] = {i % n, (i / n) % n, d == 3 ? i / (n * n) : 0};
        for (int k = 0; k < d; ++k) anchor[(size_t)e * d + k] = (int32_t)a[k];
        for (int c = 0; c < NN; ++c) {
            int64_t p[3] = {0, 0, 0};
            for (int k = 0, cc = c; k < d; ++k, cc /= 3) p[k] = 2 * a[k] + cc % 3;
            nkeys.push_back(morton(d, p));
        }
    }
    std::vector<uint64_t> keys(nkeys);
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    const int64_t N = (int64_t)keys.size();
    std::vector<int32_t> e2n((size_t)E * NN);
    for (size_t j = 0; j < nkeys.size(); ++j)
        e2n[j] = (int32_t)(std::lower_bound(keys.begin(), keys.end(), nkeys[j]) - keys.begin());
    chns_mesh* m = new (std::nothrow) chns_mesh();
    if (!m) { chns_set_error("host allocation failed"); return CHNS_ENOMEM; }
    m->order = 2;
    m->q2_level = L;
    m->max_level = L + 1;
    m->node_coords.resize((size_t)N * d);
    std::vector<uint8_t> nflag((size_t)N, 0);
    std::vector<int32_t> bnodes;
    for (int64_t i = 0; i < N; ++i) {
        bool bnd = false;
        for (int c = 0; c < d; ++c) {
            int64_t v = 0;
            for (int b = 0; b <= L + 1; ++b) v |= (int64_t)((keys[(size_t)i] >> (b * d + c)) & 1) << b;
            m->node_coords[(size_t)i * d + c] = (int32_t)v;
            if (v == 0 || v == side) bnd = true;
        }
        if (bnd) {
            nflag[(size_t)i] = (uint8_t)((1u << d) - 1u);
            bnodes.push_back((int32_t)i);
        }
    }
    // node masses: int N_a = (h/2)^d prod_k (1/3, 4/3, 1/3)[a_k]
    std::vector<double> nmass((size_t)N, 0.0);
    const double h = std::ldexp(hi - lo, -L), w1[3] = {1.0 / 3.0, 4.0 / 3.0, 1.0 / 3.0};
    const double jac = std::pow(0.5 * h, d);
    for (int64_t e = 0; e < E; ++e)
        for (int c = 0; c < NN; ++c) {
            double w = jac;
            for (int k = 0, cc = c; k < d; ++k, cc /= 3) w *= w1[cc % 3];
            nmass[(size_t)e2n[(size_t)e * NN + c]] += w;
        }
    std::vector<int8_t> level8((size_t)E, (int8_t)L);
    std::vector<int32_t> hang(4, -1);
    {
        cudaError_t de = cudaGetDevice(&m->device);
        if (de != cudaSuccess) { chns_mesh_destroy(m); return chns_cuda_status(de, "cudaGetDevice"); }
    }
    chns_status st;
    if ((st = dev_upload(&m->d_e2n, e2n)) != CHNS_OK || (st = dev_upload(&m->d_hang, hang)) != CHNS_OK ||
        (st = dev_upload(&m->d_level, level8)) != CHNS_OK || (st = dev_upload(&m->d_nflag, nflag)) != CHNS_OK ||
        (st = dev_upload(&m->d_bnodes, bnodes)) != CHNS_OK || (st = dev_upload(&m->d_anchor, anchor)) != CHNS_OK ||
        (st = dev_upload(&m->d_nmass, nmass)) != CHNS_OK) {
        chns_mesh_destroy(m);
        return st;
    }
    m->n_partials = 4096;
    cudaError_t ce = cudaMalloc((void**)&m->d_partials, (size_t)m->n_partials * 8 * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&m->d_flags, 64);
    if (ce == cudaSuccess) ce = cudaMemset(m->d_flags, 0, 64);
    if (ce == cudaSuccess) ce = cudaMallocHost((void**)&m->h_pinned, 64 * sizeof(double));
    if (ce != cudaSuccess) { chns_mesh_destroy(m); return chns_cuda_status(ce, "cudaMalloc(mesh workspace)"); }
    DevMesh& dm = m->dm;
    dm.dim = d;
    dm.nc = NN;
    dm.nf = d + 3;
    dm.E = E;
    dm.N = N;
    dm.H = 0;
    dm.NB = (int64_t)bnodes.size();
    dm.e2n = m->d_e2n;
    dm.hang = m->d_hang;
    dm.level = m->d_level;
    dm.nflag = m->d_nflag;
    dm.bnodes = m->d_bnodes;
    dm.bcval = nullptr;
    dm.anchor = m->d_anchor;
    dm.max_level = L + 1;
    dm.lo = lo;
    dm.hi = hi;
    m->volume = std::pow(hi - lo, d);
    m->h_e2n = std::move(e2n);
    m->h_hang = std::move(hang);
    m->h_anchor = std::move(anchor);
    m->h_level = std::move(level8);
    *out = m;
    return CHNS_OK;
}

extern "C" int32_t chns_mesh_order(const chns_mesh* m) { return m ? m->order : -1; }
