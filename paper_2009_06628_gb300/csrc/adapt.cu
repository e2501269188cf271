// Remeshing (Section 4, "Re-meshing and interpolation"): the mesh follows the interface.
// One adaptation pass = refinement / coarsening flags from the current phase field on the
// GPU, a new leaf list on the host (flagged leaves split into their 2^d children, complete
// sibling families whose members are all flagged for coarsening merged into their parent,
// then 2:1 balance restored by refinement only), a new mesh, and the parent <-> child
// Q1 transfer of the fields (chns_transfer_*).  A pass moves each leaf by at most one
// level; repeated passes reach the target levels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "chns_internal.h"
#include "morton.h"

namespace {

// flag = +1 (refine) where some corner of the element has |phi| < thr and the element is
// shallower than max_level; -1 (coarsening candidate) where every corner has |phi| >= thr
// and the element is deeper than min_level; 0 otherwise.  Corner values of hanging
// corners are the constraint means of their parents (the Q1 field of the mesh).
__global__ void adapt_flags_kernel(DevMesh m, const double* __restrict__ U, double thr, int min_level,
                                   int max_level, int8_t* __restrict__ flags) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.E) return;
    const int NC = m.nc, NF = m.nf, f = m.dim + 1;
    bool near = false;
    for (int a = 0; a < NC; ++a) {
        const int ent = m.e2n[e * NC + a];
        double v;
        if (ent >= 0) {
            v = U[(size_t)ent * NF + f];
        } else {
            const int4 hp = reinterpret_cast<const int4*>(m.hang)[-ent - 1];
            if (hp.z < 0) {
                v = 0.5 * (U[(size_t)hp.x * NF + f] + U[(size_t)hp.y * NF + f]);
            } else {
                v = 0.25 * ((U[(size_t)hp.x * NF + f] + U[(size_t)hp.y * NF + f]) +
                            (U[(size_t)hp.z * NF + f] + U[(size_t)hp.w * NF + f]));
            }
        }
        if (fabs(v) < thr) near = true;
    }
    const int lev = m.level[e];
    int8_t fl = 0;
    if (near && lev < max_level) fl = 1;
    if (!near && lev > min_level) fl = -1;
    flags[e] = fl;
}

struct Box {
    int64_t a[3];
    int lev;
};

inline uint64_t box_key(int d, const Box& b) { return morton(d, b.a); }

}  // namespace

extern "C" chns_status chns_adapt_flags(const chns_mesh* m, const double* U, double phi_threshold, int32_t min_level,
                                        int32_t max_level, int8_t* flags, void* stream) {
    if (!m || !U || !flags || !(phi_threshold > 0.0) || min_level < 0 || max_level < min_level || max_level > 20) {
        chns_set_error("chns_adapt_flags: bad argument (threshold > 0, 0 <= min_level <= max_level <= 20)");
        return CHNS_EINVAL;
    }
    if (chns_require_q1(m, "chns_adapt_flags") != CHNS_OK) return CHNS_EINVAL;
    const int g = (int)((m->dm.E + 255) / 256);
    adapt_flags_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(m->dm, U, phi_threshold, min_level, max_level, flags);
    chns_count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return chns_cuda_status(e, "adapt_flags_kernel");
    return CHNS_OK;
}

extern "C" chns_status chns_adapt_leaves(int32_t dim, int32_t max_level, int64_t n_leaves, const chns_leaf* leaves,
                                         const int8_t* flags, int32_t min_level, int32_t max_level_new,
                                         chns_leaf* out, int64_t capacity, int64_t* n_out,
                                         int32_t* out_max_level) {
    if ((dim != 2 && dim != 3) || max_level < 1 || max_level > 20 || n_leaves < 1 || !leaves || !flags || !n_out ||
        !out_max_level || min_level < 0 || max_level_new < min_level || max_level_new > 20) {
        chns_set_error("chns_adapt_leaves: bad argument");
        return CHNS_EINVAL;
    }
    const int d = dim, nc = 1 << d;
    const int Lr = std::max(max_level, max_level_new);   // working resolution
    const int sh = Lr - max_level;
    const int64_t side = (int64_t)1 << Lr;
    std::vector<Box> cur;
    cur.reserve((size_t)n_leaves);
    for (int64_t i = 0; i < n_leaves; ++i) {
        Box b;
        b.a[0] = (int64_t)leaves[i].x << sh;
        b.a[1] = (int64_t)leaves[i].y << sh;
        b.a[2] = d == 3 ? (int64_t)leaves[i].z << sh : 0;
        b.lev = leaves[i].level;
        if (b.lev < 0 || b.lev > max_level) {
            chns_set_error("chns_adapt_leaves: leaf level out of range");
            return CHNS_EINVAL;
        }
        cur.push_back(b);
    }
    auto size_of = [&](int lev) { return (int64_t)1 << (Lr - lev); };
    // 1. coarsening: a complete family of 2^d siblings (consecutive in Morton order), all
    //    flagged -1 and deeper than min_level, becomes its parent
    std::vector<Box> nxt;
    std::vector<int8_t> nflag;   // carried refinement flags of the kept leaves
    nxt.reserve(cur.size());
    for (int64_t i = 0; i < (int64_t)cur.size();) {
        const Box& b = cur[(size_t)i];
        bool fam = false;
        if (b.lev > min_level && i + nc <= (int64_t)cur.size()) {
            const int64_t ps = size_of(b.lev - 1), s = size_of(b.lev);
            bool ok = true;
            for (int k = 0; k < d; ++k) ok = ok && (b.a[k] % ps) == 0;
            for (int c = 0; c < nc && ok; ++c) {
                const Box& q = cur[(size_t)(i + c)];
                ok = q.lev == b.lev && flags[i + c] == -1;
                for (int k = 0; k < d && ok; ++k) ok = q.a[k] == b.a[k] + (((c >> k) & 1) ? s : 0);
            }
            fam = ok;
        }
        if (fam) {
            Box p = b;
            p.lev = b.lev - 1;
            nxt.push_back(p);
            nflag.push_back(0);
            i += nc;
        } else {
            nxt.push_back(b);
            nflag.push_back(flags[i] == 1 && b.lev < max_level_new ? 1 : 0);
            ++i;
        }
    }
    // 2. refinement of the flagged leaves, children in Morton order (x fastest)
    auto refine_marked = [&](const std::vector<Box>& in, const std::vector<int8_t>& mark, std::vector<Box>& o) {
        o.clear();
        o.reserve(in.size() + 8 * std::count(mark.begin(), mark.end(), (int8_t)1));
        for (size_t i = 0; i < in.size(); ++i) {
            if (!mark[i]) {
                o.push_back(in[i]);
                continue;
            }
            const int64_t s = size_of(in[i].lev + 1);
            for (int c = 0; c < nc; ++c) {
                Box q = in[i];
                q.lev = in[i].lev + 1;
                for (int k = 0; k < d; ++k) q.a[k] += ((c >> k) & 1) ? s : 0;
                o.push_back(q);
            }
        }
    };
    refine_marked(nxt, nflag, cur);
    // 3. 2:1 balance by refinement: a leaf that touches (face, edge or vertex) a leaf more
    //    than one level deeper is split; repeated until no leaf is split
    for (int pass = 0; pass < 64; ++pass) {
        const int64_t E = (int64_t)cur.size();
        std::vector<uint64_t> key((size_t)E);
        for (int64_t i = 0; i < E; ++i) key[(size_t)i] = box_key(d, cur[(size_t)i]);
        std::vector<int8_t> mark((size_t)E, 0);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < E; ++i) {
            const Box& b = cur[(size_t)i];
            const int64_t s = size_of(b.lev);
            const int ndir = d == 2 ? 9 : 27;
            for (int t = 0; t < ndir; ++t) {
                const int dv[3] = {t % 3 - 1, (t / 3) % 3 - 1, (t / 9) % 3 - 1};
                if (dv[0] == 0 && dv[1] == 0 && (d == 2 || dv[2] == 0)) continue;
                int64_t p[3] = {0, 0, 0};
                bool inside = true;
                for (int k = 0; k < d; ++k) {
                    p[k] = dv[k] < 0 ? b.a[k] - 1 : (dv[k] > 0 ? b.a[k] + s : b.a[k]);
                    if (p[k] < 0 || p[k] >= side) inside = false;
                }
                if (!inside) continue;
                const int64_t j = (int64_t)(std::upper_bound(key.begin(), key.end(), morton(d, p)) - key.begin()) - 1;
                if (cur[(size_t)j].lev < b.lev - 1) {
#pragma omp atomic write
                    mark[(size_t)j] = 1;
                }
            }
        }
        if (std::find(mark.begin(), mark.end(), (int8_t)1) == mark.end()) break;
        refine_marked(cur, mark, nxt);
        std::swap(cur, nxt);
    }
    int deepest = 0;
    for (const Box& b : cur) deepest = std::max(deepest, b.lev);
    const int Lout = std::max(deepest, 1);
    *n_out = (int64_t)cur.size();
    *out_max_level = Lout;
    if ((int64_t)cur.size() > capacity || !out) {
        chns_set_error("chns_adapt_leaves: the output needs " + std::to_string(cur.size()) + " leaves");
        return CHNS_EINVAL;
    }
    for (size_t i = 0; i < cur.size(); ++i) {
        const int osh = Lr - Lout;
        out[i].x = (int32_t)(cur[i].a[0] >> osh);
        out[i].y = (int32_t)(cur[i].a[1] >> osh);
        out[i].z = (int32_t)(cur[i].a[2] >> osh);
        out[i].level = cur[i].lev;
    }
    return CHNS_OK;
}
