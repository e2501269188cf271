// Transfer operators between the Q1 spaces of two octree meshes of the same domain, and
// the geometric multigrid hierarchy built from them (Section 4: the octree's levels;
// Section 6 and the conclusions name the preconditioner as the cost to attack).
//
// Transfer P (source mesh S -> target mesh T): every independent node of T is located in
// the leaf of S that contains it (Morton search over S's sorted leaf keys), and P's row
// holds the Q1 weights of that leaf's corners at the node, each corner folded into its
// parents with the hanging-node weights (1/2, 1/4) of S.  When T refines S the result
// is the same Q1 function (no interpolation error); when T coarsens S it is injection at
// T's nodes.  Rows and the transposed rows are built on the host once and applied by
// gather kernels (no atomics, deterministic).
//
// Multigrid hierarchy: level l + 1 caps every leaf of level l at (deepest level) - 1,
// replacing a deeper leaf by its ancestor.  Two leaves that touch differ by at most one
// level, and capping cannot widen that gap, so every level stays complete and 2:1
// balanced; every coarse element is a union of fine elements, so the coarse Q1 space is
// a subspace of the fine one and P_{l+1 -> l} is exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "chns_internal.h"
#include "morton.h"

namespace {

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
    cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(src.size(), 1) * sizeof(T));
    if (e == cudaSuccess && !src.empty())
        e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

// y[row] (+)= sum_j w_j x[col_j] for every field f < nf of node-major vectors
template <class T, class W, bool ADD>
__global__ void csr_apply_kernel(int64_t rows, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const W* __restrict__ w, int nf, const T* __restrict__ x, T* __restrict__ y) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j0 = rp[r], j1 = rp[r + 1];
        for (int f = 0; f < nf; ++f) {
            T acc = T(0);
            for (int64_t j = j0; j < j1; ++j) acc += (T)w[j] * x[(size_t)col[j] * nf + f];
            if (ADD)
                y[(size_t)r * nf + f] += acc;
            else
                y[(size_t)r * nf + f] = acc;
        }
    }
}

int grid_rows(int64_t rows) {
    const int64_t b = (rows + 255) / 256;
    const int64_t cap = 16 * (int64_t)chns_num_sms();
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

chns_status transfer_build(const chns_mesh* S, const chns_mesh* D, TransferDev* T) {
    *T = TransferDev();
    if (!S || !D || S->dm.dim != D->dm.dim || S->dm.lo != D->dm.lo || S->dm.hi != D->dm.hi) {
        chns_set_error("transfer: the meshes must share dimension and domain");
        return CHNS_EINVAL;
    }
    const int d = S->dm.dim, nc = 1 << d;
    const int LS = S->max_level, LD = D->max_level, L = std::max(LS, LD);
    const int shS = L - LS, shD = L - LD;
    const int64_t ES = S->dm.E, ND = D->dm.N;
    const int64_t side = (int64_t)1 << L;
    std::vector<uint64_t> key((size_t)ES);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ES; ++e) {
        int64_t a[3] = {0, 0, 0};
        for (int k = 0; k < d; ++k) a[k] = (int64_t)S->h_anchor[(size_t)e * d + k] << shS;
        key[(size_t)e] = morton(d, a);
    }
    constexpr int CAP = 32;   // 2^d corners x up to 4 constraint parents
    // row n of P into (rc, rw), ascending columns; returns its length
    auto row = [&](int64_t n, int32_t* rc, double* rw) -> int {
        int64_t c[3] = {0, 0, 0}, q[3] = {0, 0, 0};
        for (int k = 0; k < d; ++k) {
            c[k] = (int64_t)D->node_coords[(size_t)n * d + k] << shD;
            q[k] = std::min<int64_t>(c[k], side - 1);   // a node on the upper face: the leaf below
        }
        const uint64_t kq = morton(d, q);
        const int64_t e = (int64_t)(std::upper_bound(key.begin(), key.end(), kq) - key.begin()) - 1;
        const int lev = S->h_level[(size_t)e];
        const double s = (double)((int64_t)1 << (L - lev));
        double t[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < d; ++k)
            t[k] = (double)(c[k] - ((int64_t)S->h_anchor[(size_t)e * d + k] << shS)) / s;
        int m = 0;
        auto add = [&](int32_t node, double wv) {
            for (int i = 0; i < m; ++i)
                if (rc[i] == node) { rw[i] += wv; return; }
            rc[m] = node;
            rw[m] = wv;
            ++m;
        };
        for (int a = 0; a < nc; ++a) {
            double wv = 1.0;
            for (int k = 0; k < d; ++k) wv *= ((a >> k) & 1) ? t[k] : 1.0 - t[k];
            if (wv == 0.0) continue;
            const int32_t ent = S->h_e2n[(size_t)e * nc + a];
            if (ent >= 0) {
                add(ent, wv);
            } else {
                const int32_t* hp = &S->h_hang[(size_t)(-ent - 1) * 4];
                const int np = hp[2] < 0 ? 2 : 4;
                for (int j = 0; j < np; ++j) add(hp[j], wv / np);
            }
        }
        for (int i = 1; i < m; ++i)   // ascending columns: a fixed summation order
            for (int j = i; j > 0 && rc[j - 1] > rc[j]; --j) {
                std::swap(rc[j - 1], rc[j]);
                std::swap(rw[j - 1], rw[j]);
            }
        return m;
    };
    // two passes (lengths, then entries) keep the host memory at the size of P
    std::vector<int64_t> rp((size_t)ND + 1, 0);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < ND; ++n) {
        int32_t rc[CAP];
        double rw[CAP];
        rp[(size_t)n + 1] = row(n, rc, rw);
    }
    for (int64_t n = 0; n < ND; ++n) rp[(size_t)n + 1] += rp[(size_t)n];
    const int64_t nnz = rp[(size_t)ND];
    std::vector<int32_t> col((size_t)nnz);
    std::vector<double> w((size_t)nnz);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < ND; ++n) {
        int32_t rc[CAP];
        double rw[CAP];
        const int m = row(n, rc, rw);
        for (int i = 0; i < m; ++i) {
            col[(size_t)(rp[(size_t)n] + i)] = rc[i];
            w[(size_t)(rp[(size_t)n] + i)] = rw[i];
        }
    }
    // transpose by counting sort over source nodes (rows of P^T keep ascending columns)
    const int64_t NS = S->dm.N;
    std::vector<int64_t> rpT((size_t)NS + 1, 0);
    for (int64_t j = 0; j < nnz; ++j) rpT[(size_t)col[(size_t)j] + 1]++;
    for (int64_t i = 0; i < NS; ++i) rpT[(size_t)i + 1] += rpT[(size_t)i];
    std::vector<int32_t> colT((size_t)nnz);
    std::vector<double> wT((size_t)nnz);
    {
        std::vector<int64_t> pos(rpT.begin(), rpT.end() - 1);
        for (int64_t n = 0; n < ND; ++n)
            for (int64_t j = rp[(size_t)n]; j < rp[(size_t)n + 1]; ++j) {
                const int64_t p = pos[(size_t)col[(size_t)j]]++;
                colT[(size_t)p] = (int32_t)n;
                wT[(size_t)p] = w[(size_t)j];
            }
    }
    std::vector<float> wf(w.begin(), w.end()), wTf(wT.begin(), wT.end());
    T->n_src = NS;
    T->n_dst = ND;
    T->nnz = nnz;
    cudaError_t e = upload(&T->rp, rp);
    if (e == cudaSuccess) e = upload(&T->col, col);
    if (e == cudaSuccess) e = upload(&T->w, w);
    if (e == cudaSuccess) e = upload(&T->wf, wf);
    if (e == cudaSuccess) e = upload(&T->rpT, rpT);
    if (e == cudaSuccess) e = upload(&T->colT, colT);
    if (e == cudaSuccess) e = upload(&T->wT, wT);
    if (e == cudaSuccess) e = upload(&T->wTf, wTf);
    if (e != cudaSuccess) {
        transfer_free(T);
        return chns_cuda_status(e, "cudaMalloc(transfer)");
    }
    return CHNS_OK;
}

void transfer_free(TransferDev* T) {
    cudaFree(T->rp);
    cudaFree(T->col);
    cudaFree(T->w);
    cudaFree(T->wf);
    cudaFree(T->rpT);
    cudaFree(T->colT);
    cudaFree(T->wT);
    cudaFree(T->wTf);
    *T = TransferDev();
}

cudaError_t transfer_apply_f64(const TransferDev& T, bool transpose, int nf, const double* in, double* out,
                               cudaStream_t s) {
    const int64_t rows = transpose ? T.n_src : T.n_dst;
    if (transpose)
        csr_apply_kernel<double, double, false><<<grid_rows(rows), 256, 0, s>>>(rows, T.rpT, T.colT, T.wT, nf, in, out);
    else
        csr_apply_kernel<double, double, false><<<grid_rows(rows), 256, 0, s>>>(rows, T.rp, T.col, T.w, nf, in, out);
    chns_count_launches(1);
    return cudaGetLastError();
}

cudaError_t transfer_apply_f32(const TransferDev& T, bool transpose, bool add, const float* in, float* out,
                               cudaStream_t s) {
    const int64_t rows = transpose ? T.n_src : T.n_dst;
    const int64_t* rp = transpose ? T.rpT : T.rp;
    const int32_t* col = transpose ? T.colT : T.col;
    const float* w = transpose ? T.wTf : T.wf;
    if (add)
        csr_apply_kernel<float, float, true><<<grid_rows(rows), 256, 0, s>>>(rows, rp, col, w, 1, in, out);
    else
        csr_apply_kernel<float, float, false><<<grid_rows(rows), 256, 0, s>>>(rows, rp, col, w, 1, in, out);
    chns_count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Capped leaf list: every leaf deeper than `cap` replaced by its ancestor at `cap`
// (consecutive duplicates merged; Morton order is kept).  Anchors of the input are in
// units of 2^-Lin, of the output in units of 2^-cap.  fmap[e] = output leaf of input e.
// ---------------------------------------------------------------------------------
static void cap_leaves(int d, int Lin, int64_t E, const int32_t* anchor, const int8_t* level, int cap,
                       std::vector<chns_leaf>& out, std::vector<int32_t>& fmap) {
    out.clear();
    fmap.resize((size_t)E);
    const int sh = Lin - cap;
    for (int64_t e = 0; e < E; ++e) {
        const int lev = std::min<int>(level[e], cap);
        const int64_t mask = ~(((int64_t)1 << (Lin - lev)) - 1);
        chns_leaf f;
        f.x = (int32_t)((anchor[(size_t)e * d] & mask) >> sh);
        f.y = (int32_t)((anchor[(size_t)e * d + 1] & mask) >> sh);
        f.z = d == 3 ? (int32_t)((anchor[(size_t)e * d + 2] & mask) >> sh) : 0;
        f.level = lev;
        if (out.empty() || out.back().x != f.x || out.back().y != f.y || out.back().z != f.z ||
            out.back().level != f.level)
            out.push_back(f);
        fmap[(size_t)e] = (int32_t)(out.size() - 1);
    }
}

extern "C" chns_status chns_coarsen_leaves(int32_t dim, int32_t max_level, int64_t n_leaves, const chns_leaf* leaves,
                                           int32_t cap, chns_leaf* out, int32_t* fmap, int64_t* n_out) {
    if ((dim != 2 && dim != 3) || max_level < 1 || max_level > 20 || n_leaves < 1 || !leaves || !out || !n_out ||
        cap < 0 || cap > max_level) {
        chns_set_error("chns_coarsen_leaves: bad argument");
        return CHNS_EINVAL;
    }
    std::vector<int32_t> anchor((size_t)n_leaves * dim);
    std::vector<int8_t> level((size_t)n_leaves);
    for (int64_t e = 0; e < n_leaves; ++e) {
        const int32_t a[3] = {leaves[e].x, leaves[e].y, leaves[e].z};
        for (int k = 0; k < dim; ++k) anchor[(size_t)e * dim + k] = a[k];
        if (leaves[e].level < 0 || leaves[e].level > max_level) {
            chns_set_error("chns_coarsen_leaves: leaf level out of range");
            return CHNS_EINVAL;
        }
        level[(size_t)e] = (int8_t)leaves[e].level;
    }
    std::vector<chns_leaf> o;
    std::vector<int32_t> fm;
    cap_leaves(dim, max_level, n_leaves, anchor.data(), level.data(), cap, o, fm);
    std::memcpy(out, o.data(), o.size() * sizeof(chns_leaf));
    if (fmap) std::memcpy(fmap, fm.data(), fm.size() * sizeof(int32_t));
    *n_out = (int64_t)o.size();
    return CHNS_OK;
}

static chns_status alloc_level(MGLevel& L) {
    cudaError_t e = cudaSuccess;
    for (float** p : {&L.dinv, &L.bnd, &L.b, &L.x, &L.t, &L.cr, &L.cx, &L.cd, &L.cy})
        if (e == cudaSuccess) e = cudaMalloc((void**)p, (size_t)std::max<int64_t>(L.N, 1) * sizeof(float));
    // level 0 reads the Schur coefficients of the solver workspace; coarse levels own theirs
    if (e == cudaSuccess && L.mesh) e = cudaMalloc((void**)&L.ce, (size_t)std::max<int64_t>(L.E, 1) * sizeof(float));
    return e == cudaSuccess ? CHNS_OK : chns_cuda_status(e, "cudaMalloc(multigrid level)");
}

chns_status mg_hier_build(chns_mesh* m) {
    if (m->mg) return CHNS_OK;
    MGHier* mg = new MGHier();
    const int d = m->dm.dim;
    {
        MGLevel L0;
        L0.dm = m->dm;
        L0.N = m->dm.N;
        L0.E = m->dm.E;
        mg->lv.push_back(L0);
    }
    // coarsen until the level is small (the coarsest is solved by a long Chebyshev sweep)
    const chns_mesh* cur = m;
    chns_status st = CHNS_OK;
    while (true) {
        int deepest = 0;
        for (int8_t l : cur->h_level) deepest = std::max<int>(deepest, l);
        if (deepest <= 1 || cur->dm.N <= 300) break;
        const int cap = deepest - 1;
        std::vector<chns_leaf> leaves;
        std::vector<int32_t> fmap;
        cap_leaves(d, cur->max_level, cur->dm.E, cur->h_anchor.data(), cur->h_level.data(), cap, leaves, fmap);
        chns_mesh* cm = nullptr;
        st = chns_mesh_create(d, cap, (int64_t)leaves.size(), leaves.data(), m->dm.lo, m->dm.hi, &cm);
        if (st != CHNS_OK) break;
        MGLevel L;
        L.mesh = cm;
        L.dm = cm->dm;
        L.N = cm->dm.N;
        L.E = cm->dm.E;
        st = transfer_build(cm, cur, &L.P);
        if (st != CHNS_OK) { chns_mesh_destroy(cm); break; }
        cudaError_t e = upload(&L.fmap, fmap);
        if (e != cudaSuccess) { st = chns_cuda_status(e, "cudaMalloc(multigrid map)"); transfer_free(&L.P); chns_mesh_destroy(cm); break; }
        mg->lv.push_back(L);
        cur = cm;
    }
    if (st == CHNS_OK)
        for (size_t l = 0; l < mg->lv.size() && st == CHNS_OK; ++l) st = alloc_level(mg->lv[l]);
    if (st == CHNS_OK) {
        cudaError_t e = cudaMalloc((void**)&mg->kmax, 64 * sizeof(unsigned int));
        if (e != cudaSuccess) st = chns_cuda_status(e, "cudaMalloc(multigrid bounds)");
    }
    if (st != CHNS_OK) {
        chns_mg_free(mg);
        return st;
    }
    m->mg = mg;
    return CHNS_OK;
}

void chns_mg_free(MGHier* mg) {
    if (!mg) return;
    for (auto& L : mg->lv) {
        transfer_free(&L.P);
        cudaFree(L.fmap);
        for (float* p : {L.ce, L.dinv, L.bnd, L.b, L.x, L.t, L.cr, L.cx, L.cd, L.cy}) cudaFree(p);
        if (L.mesh) chns_mesh_destroy(L.mesh);
    }
    cudaFree(mg->kmax);
    delete mg;
}

// ---------------------------------------------------------------------------------
// Public transfer entry points
// ---------------------------------------------------------------------------------
struct chns_transfer {
    TransferDev T;
};

extern "C" chns_status chns_transfer_create(const chns_mesh* src, const chns_mesh* dst, chns_transfer** out) {
    if (!src || !dst || !out) {
        chns_set_error("chns_transfer_create: null argument");
        return CHNS_EINVAL;
    }
    *out = nullptr;
    if (chns_require_q1(src, "chns_transfer_create") != CHNS_OK || chns_require_q1(dst, "chns_transfer_create") != CHNS_OK)
        return CHNS_EINVAL;
    chns_transfer* t = new (std::nothrow) chns_transfer();
    if (!t) {
        chns_set_error("host allocation failed");
        return CHNS_ENOMEM;
    }
    chns_status st = transfer_build(src, dst, &t->T);
    if (st != CHNS_OK) {
        delete t;
        return st;
    }
    *out = t;
    return CHNS_OK;
}

extern "C" void chns_transfer_destroy(chns_transfer* t) {
    if (!t) return;
    transfer_free(&t->T);
    delete t;
}

extern "C" int64_t chns_transfer_nnz(const chns_transfer* t) { return t ? t->T.nnz : -1; }

extern "C" chns_status chns_transfer_apply(const chns_transfer* t, int32_t nf, int32_t transpose, const double* in,
                                           double* out, void* stream) {
    if (!t || !in || !out || nf < 1 || nf > 16 || (transpose != 0 && transpose != 1)) {
        chns_set_error("chns_transfer_apply: bad argument (nf in [1, 16], transpose 0/1, non-null vectors)");
        return CHNS_EINVAL;
    }
    cudaError_t e = transfer_apply_f64(t->T, transpose == 1, nf, in, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return chns_cuda_status(e, "chns_transfer_apply");
    return CHNS_OK;
}
