// mg_tree.cpp -- host side of the GB300 octree geometric multigrid: mesh and
// level construction (Sec. 2.5), device tables, the coarsest-level factors
// (dense inverse, block-tridiagonal form), and the C ABI declared in
// include/mg.h.
#include <algorithm>
#include <array>
#include <chrono>
#include <functional>
#include <unordered_map>
#include <atomic>
#include <thread>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include "mg_internal.h"

using namespace mg;

static thread_local std::string g_err;
void mg_set_error(const std::string &msg) { g_err = msg; }
extern "C" const char *mg_last_error(void) { return g_err.c_str(); }

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            mg_set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                 \
            return MG_ERR_CUDA;                                                               \
        }                                                                                     \
    } while (0)

static int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

static long long ipow(int n, int d) { return d == 2 ? (long long)n * n : (long long)n * n * n; }

// ------------------------------------------------------------ create ----

extern "C" int mg_tree_create(int dim, int block_size, int geometry, const mg_bc *bc, const int base_cells[3],
                              const double lo[3], const double hi[3], int coarse_max_cells, double helmholtz,
                              mg_tree **out) {
    if (!out || !bc || !base_cells || !lo || !hi) return fail(MG_ERR_ARG, "null argument");
    if (dim != 2 && dim != 3) return fail(MG_ERR_ARG, "dim must be 2 or 3");
    if (block_size < 2 || block_size % 2) return fail(MG_ERR_ARG, "block_size must be even and >= 2");
    if (geometry != MG_CART && !(geometry == MG_CYL && dim == 2)) return fail(MG_ERR_ARG, "bad geometry");
    if (helmholtz < 0) return fail(MG_ERR_ARG, "helmholtz must be >= 0");
    for (int d = 0; d < dim; d++) {
        if (base_cells[d] < block_size || base_cells[d] % block_size)
            return fail(MG_ERR_ARG, "base_cells must be positive multiples of block_size");
        if (!(hi[d] > lo[d])) return fail(MG_ERR_ARG, "hi must exceed lo");
        const bool p0 = bc->type[2 * d] == MG_BC_PERIODIC, p1 = bc->type[2 * d + 1] == MG_BC_PERIODIC;
        if (p0 != p1) return fail(MG_ERR_ARG, "periodic faces must come in pairs");
    }
    for (int f = 0; f < 2 * dim; f++)
        if (bc->type[f] < 0 || bc->type[f] > MG_BC_AXIS) return fail(MG_ERR_ARG, "bad boundary type");
    if (geometry == MG_CYL && bc->type[1] == MG_BC_AXIS) return fail(MG_ERR_ARG, "axis must be the -r face");
    mg_tree *t = new mg_tree();
    t->dim = dim;
    t->N = block_size;
    t->geom = geometry;
    t->bc = *bc;
    for (int d = 0; d < 3; d++) {
        t->base[d] = d < dim ? base_cells[d] : 1;
        t->lo[d] = lo[d];
        t->hi[d] = d < dim ? hi[d] : lo[d] + 1.0;
    }
    t->coarse_max = coarse_max_cells;
    t->helm = helmholtz;
    *out = t;
    return MG_OK;
}

extern "C" int mg_tree_refine(mg_tree *t, int n, const int32_t *e) {
    if (!t || n < 0 || (n > 0 && !e)) return fail(MG_ERR_ARG, "bad refine arguments");
    if (t->built) return fail(MG_ERR_STATE, "refine after the mesh was built");
    t->refine.insert(t->refine.end(), e, e + 4 * (size_t)n);
    return MG_OK;
}

// ------------------------------------------------------------- build ----
// Levels (Sec. 2.5): below the base grid the block count is halved while all
// counts are even, then the block size is halved while the level holds more
// than coarse_max cells; above it the refined levels.  Per level the
// covered blocks come first, then the leaves, each in Morton order.

// sweep variants of a tree made by adapt: the old tree's choice at the same
// level depth (-1, the default kernel, where the depth is new)
static bool apply_tune_hint(mg_tree *t, int prec) {
    if (t->tune_hint[prec].empty()) return false;
    t->sweep_choice[prec].assign(t->lev.size(), -1);
    for (size_t l = 0; l < t->lev.size(); l++) {
        auto it = t->tune_hint[prec].find(t->lev[l].depth);
        if (it != t->tune_hint[prec].end()) t->sweep_choice[prec][l] = it->second;
    }
    return true;
}

static double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Level skeleton: the coarse levels (block count halved while every count
// is even, then block size halved while the level holds more than
// coarse_max cells), the base grid, and maxdepth + 1 refined levels.
std::vector<LvSkel> mg::level_skeleton(const mg_tree *t, int maxdepth) {
    const int D = t->dim;
    std::vector<LvSkel> coarse;
    int nb0[3] = {1, 1, 1};
    for (int d = 0; d < D; d++) nb0[d] = t->base[d] / t->N;
    int n = t->N, b[3] = {nb0[0], nb0[1], nb0[2]};
    while (true) {
        long long cells = 1;
        bool even = true;
        for (int d = 0; d < D; d++) { cells *= (long long)n * b[d]; if (b[d] % 2) even = false; }
        if (even) for (int d = 0; d < D; d++) b[d] /= 2;
        else if (cells > t->coarse_max && n % 2 == 0) n /= 2;
        else break;
        LvSkel c;
        c.n = n; c.depth = -(int)coarse.size() - 1;
        for (int d = 0; d < 3; d++) c.nblk[d] = b[d];
        coarse.push_back(c);
        if (coarse.size() > 60) break;
    }
    std::reverse(coarse.begin(), coarse.end());
    std::vector<LvSkel> lv = coarse;
    LvSkel base;
    base.n = t->N; base.depth = 0;
    for (int d = 0; d < 3; d++) base.nblk[d] = nb0[d];
    lv.push_back(base);
    for (int r = 0; r <= maxdepth; r++) {
        LvSkel c;
        c.n = t->N; c.depth = r + 1;
        for (int d = 0; d < 3; d++) c.nblk[d] = d < D ? 2 * lv.back().nblk[d] : 1;
        lv.push_back(c);
    }
    return lv;
}

int mg::max_refine_depth(const mg_tree *t) {
    int maxdepth = -1;
    for (size_t e = 0; e < t->refine.size() / 4; e++) maxdepth = std::max(maxdepth, t->refine[4 * e]);
    return maxdepth;
}

// Level descriptors from the skeleton and the block counts: 32-element
// (128/256-byte) aligned cell and ghost ranges, global ids level by level.
void mg::fill_levels(mg_tree *t, const std::vector<LvSkel> &lv, const std::vector<int> &nb,
                 const std::vector<int> &nref) {
    const int D = t->dim, nl = (int)lv.size();
    t->lev.assign(nl, LevelHost());
    int g = 0;
    long long co = 0, go = 0, leaf = 0;
    for (int l = 0; l < nl; l++) {
        LevelHost &L = t->lev[l];
        L.n = lv[l].n; L.depth = lv[l].depth;
        for (int d = 0; d < 3; d++) {
            L.nblk[d] = lv[l].nblk[d];
            L.ncell[d] = d < D ? lv[l].nblk[d] * lv[l].n : 1;
            L.h[d] = d < D ? (t->hi[d] - t->lo[d]) / L.ncell[d] : 1.0;
        }
        L.first = g;
        L.nb = nb[l];
        L.nref = nref[l];
        co = (co + 31) / 32 * 32;
        go = (go + 31) / 32 * 32;
        L.cell_first = co;
        L.ghost_first = go;
        L.ncells = L.nb * ipow(L.n, D);
        L.nghost = L.nb * 2LL * D * (D == 2 ? L.n : (long long)L.n * L.n);
        leaf += (long long)(L.nb - L.nref) * ipow(L.n, D);
        g += L.nb;
        co += L.ncells;
        go += L.nghost;
    }
    t->ncells = co;
    t->nghost = go;
    t->nleaf_cells = leaf;
}

// Block tables on the host: per level, the blocks (the coarse levels and the
// base grid whole, refined levels from the refine entries), covered blocks
// first and Morton order within each group, then per block its offsets,
// parent and face neighbours (same level, physical, or one level coarser).
static int build_tables_host(mg_tree *t) {
    const int D = t->dim;
    const int maxdepth = max_refine_depth(t);
    const std::vector<LvSkel> sk = level_skeleton(t, maxdepth);
    const int nl = (int)sk.size(), ibase = nl - 1 - (maxdepth + 1);
    std::vector<std::vector<std::array<int, 3>>> lb(nl);
    for (int l = 0; l <= ibase; l++)
        for (int k = 0; k < sk[l].nblk[2]; k++)
            for (int j = 0; j < sk[l].nblk[1]; j++)
                for (int i = 0; i < sk[l].nblk[0]; i++) lb[l].push_back({i, j, k});
    for (int r = 0; r <= maxdepth; r++) {
        const LvSkel &P = sk[ibase + r];
        std::vector<char> exists((size_t)P.nblk[0] * P.nblk[1] * P.nblk[2], 0), done(exists.size(), 0);
        for (auto &q : lb[ibase + r]) exists[((size_t)q[2] * P.nblk[1] + q[1]) * P.nblk[0] + q[0]] = 1;
        std::vector<std::array<int, 3>> &C = lb[ibase + r + 1];
        for (size_t e = 0; e < t->refine.size() / 4; e++) {
            if (t->refine[4 * e] != r) continue;
            int q[3] = {t->refine[4 * e + 1], t->refine[4 * e + 2], D == 3 ? t->refine[4 * e + 3] : 0};
            bool ok = true;
            for (int d = 0; d < 3; d++) ok = ok && q[d] >= 0 && q[d] < P.nblk[d];
            size_t m = ok ? ((size_t)q[2] * P.nblk[1] + q[1]) * P.nblk[0] + q[0] : 0;
            if (!ok || !exists[m]) return fail(MG_ERR_ARG, "refined block does not exist");
            if (done[m]) continue;
            done[m] = 1;
            for (int c = 0; c < (1 << D); c++)
                C.push_back({2 * q[0] + (c & 1), 2 * q[1] + ((c >> 1) & 1), D == 3 ? 2 * q[2] + ((c >> 2) & 1) : 0});
        }
        if (C.empty()) return fail(MG_ERR_ARG, "refinement depths must be contiguous");
    }
    // dense coordinate maps and "has children" flags
    std::vector<std::vector<int>> map(nl);
    std::vector<std::vector<char>> haschild(nl);
    auto key = [&](int l, int i, int j, int k) { return ((size_t)k * sk[l].nblk[1] + j) * sk[l].nblk[0] + i; };
    for (int l = 0; l < nl; l++) {
        map[l].assign((size_t)sk[l].nblk[0] * sk[l].nblk[1] * sk[l].nblk[2], -1);
        haschild[l].assign(lb[l].size(), 0);
        for (size_t b = 0; b < lb[l].size(); b++) map[l][key(l, lb[l][b][0], lb[l][b][1], lb[l][b][2])] = (int)b;
    }
    auto parent_of = [&](int l, const std::array<int, 3> &q, int *pq, int *poff) {
        const bool same = sk[l - 1].n == sk[l].n;
        for (int d = 0; d < 3; d++) {
            pq[d] = d < D ? (same ? q[d] / 2 : q[d]) : 0;
            poff[d] = d < D ? (same ? (q[d] % 2) * (sk[l].n / 2) : 0) : 0;
        }
    };
    for (int l = 1; l < nl; l++)
        for (auto &q : lb[l]) {
            int pq[3], po[3];
            parent_of(l, q, pq, po);
            haschild[l - 1][map[l - 1][key(l - 1, pq[0], pq[1], pq[2])]] = 1;
        }
    // order: covered blocks, then leaves, Morton within each group (one
    // 64-bit key per block: the leaf flag above the 63-bit Morton code)
    std::vector<std::vector<int>> order(nl);
    std::vector<int> nb(nl), nref(nl, 0);
    for (int l = 0; l < nl; l++) {
        std::vector<std::pair<uint64_t, int>> kv(lb[l].size());
        for (size_t b = 0; b < kv.size(); b++) {
            nref[l] += haschild[l][b];
            kv[b] = {((uint64_t)(haschild[l][b] ? 0 : 1) << 63) | morton3(lb[l][b][0], lb[l][b][1], lb[l][b][2]),
                     (int)b};
        }
        std::sort(kv.begin(), kv.end());
        order[l].resize(kv.size());
        for (size_t r = 0; r < kv.size(); r++) order[l][r] = kv[r].second;
        nb[l] = (int)kv.size();
    }
    fill_levels(t, sk, nb, nref);
    std::vector<std::vector<int>> gid(nl);
    for (int l = 0; l < nl; l++) {
        gid[l].assign(nb[l], -1);
        for (int r = 0; r < nb[l]; r++) gid[l][order[l][r]] = t->lev[l].first + r;
    }
    int g = 0;
    for (int l = 0; l < nl; l++) g += nb[l];
    t->blocks.assign(g, BlockDesc());
    for (int l = 0; l < nl; l++) {
        const LevelHost &L = t->lev[l];
        const long long C = ipow(L.n, D), F = 2LL * D * (D == 2 ? L.n : (long long)L.n * L.n);
        for (int r = 0; r < L.nb; r++) {
            const int b = order[l][r];
            BlockDesc &B = t->blocks[L.first + r];
            const auto &q = lb[l][b];
            B.cell_off = L.cell_first + r * C;
            B.ghost_off = L.ghost_first + r * F;
            B.n = L.n;
            B.lev = l;
            B.flags = haschild[l][b] ? 1 : 0;
            for (int d = 0; d < 3; d++) B.ijk[d] = q[d];
            B.parent = -1;
            for (int d = 0; d < 3; d++) B.poff[d] = 0;
            if (l > 0) {
                int pq[3];
                parent_of(l, q, pq, B.poff);
                B.parent = gid[l - 1][map[l - 1][key(l - 1, pq[0], pq[1], pq[2])]];
            }
            for (int f = 0; f < 6; f++) { B.nbr[f] = -1; B.push[f] = -1; }
            for (int d = 0; d < D; d++)
                for (int s = 0; s < 2; s++) {
                    int nq[3] = {q[0], q[1], q[2]};
                    nq[d] += s ? 1 : -1;
                    if (nq[d] < 0 || nq[d] >= L.nblk[d]) {
                        if (t->bc.type[2 * d + s] != MG_BC_PERIODIC) continue;  // physical face
                        nq[d] = (nq[d] + L.nblk[d]) % L.nblk[d];
                    }
                    const int m = map[l][key(l, nq[0], nq[1], nq[2])];
                    if (m >= 0) {
                        B.nbr[2 * d + s] = gid[l][m];
                        const long long Fd = D == 2 ? L.n : (long long)L.n * L.n;
                        const int rn = gid[l][m] - L.first;  // neighbour's rank in the level
                        B.push[2 * d + s] = L.ghost_first + rn * 2LL * D * Fd + ((2 * d + s) ^ 1) * Fd;
                        continue;
                    }
                    // no same-level neighbour: the region one level coarser must exist (2:1)
                    if (l == 0 || sk[l - 1].n != L.n) return fail(MG_ERR_BALANCE, "incomplete coarse level");
                    int cq[3] = {0, 0, 0};
                    for (int e = 0; e < D; e++) cq[e] = nq[e] / 2;
                    const int cm = map[l - 1][key(l - 1, cq[0], cq[1], cq[2])];
                    if (cm < 0) return fail(MG_ERR_BALANCE, "mesh is not 2:1 balanced across faces");
                    B.nbr[2 * d + s] = -2 - gid[l - 1][cm];
                }
        }
    }
    return MG_OK;
}

// Device build where a CUDA device is present and the tree has not asked
// for the host build (mg_tree_build_on); the two give identical tables.
static bool use_device_build(const mg_tree *t) {
    if (t->build_where == 1) return false;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return false;
    }
    return true;
}

static int build(mg_tree *t) {
    if (t->built) return MG_OK;
    const auto t0 = std::chrono::steady_clock::now();
    const int D = t->dim;
    const bool dev = use_device_build(t);
    int rc = dev ? build_tables_device(t) : build_tables_host(t);
    if (rc) return rc;
    t->built_on_device = dev;
    const int nl = (int)t->lev.size();
    // red and black must alternate across periodic faces on every smoothed
    // level (the fused sweep relies on it); the coarsest level is solved directly
    for (int l = 1; l < nl; l++)
        for (int d = 0; d < D; d++)
            if (t->bc.type[2 * d] == MG_BC_PERIODIC && t->lev[l].ncell[d] % 2)
                return fail(MG_ERR_UNSUPPORTED, "odd periodic extent on a smoothed level");
    t->singular = t->helm <= 0;
    for (int f = 0; f < 2 * D; f++)
        if (t->bc.type[f] == MG_BC_DIRICHLET) t->singular = false;
    t->nc = (int)(t->lev[0].nb * ipow(t->lev[0].n, D));
    t->ns = t->nc + (t->singular ? 1 : 0);
    t->groups.assign(nl, {});
    for (int l = 0; l < nl; l++) {
        t->lev[l].group = l;
        t->lev[l].coarsest = l == 0;
        t->lev[l].parent_same_n = l > 0 && t->lev[l - 1].n == t->lev[l].n;
        t->groups[l] = {l};
    }
    TreeCoarse tc{};
    tc.first = t->lev[0].first; tc.nb = t->lev[0].nb; tc.n = t->lev[0].n;
    tc.nc = t->nc; tc.ns = t->ns; tc.singular = t->singular ? 1 : 0; tc.group = 0; tc.lvl = 0;
    tc.cell0 = t->lev[0].cell_first; tc.minv_off = 0; tc.cvec_off = 0;
    t->tcoarse = {tc};
    t->minv_total = (long long)t->ns * t->ns;
    t->cvec_total = t->ns;
    t->max_nc = t->nc;
    t->built = true;
    t->build_s[0] = seconds_since(t0);
    return MG_OK;
}

extern "C" int mg_tree_build_on(mg_tree *t, int where) {
    if (!t || where < 0 || where > 2) return fail(MG_ERR_ARG, "bad arguments");
    if (t->built) return fail(MG_ERR_STATE, "the mesh is already built");
    if (where == 2) {
        int n = 0;
        if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
            cudaGetLastError();
            return fail(MG_ERR_UNSUPPORTED, "no CUDA device for the device mesh build");
        }
    }
    t->build_where = where;
    return MG_OK;
}

extern "C" int mg_tree_built_on(mg_tree *t, int *where) {
    if (!t || !where) return fail(MG_ERR_ARG, "null argument");
    int rc = build(t);
    if (rc) return rc;
    *where = t->built_on_device ? 2 : 1;
    return MG_OK;
}

extern "C" int mg_tree_block_table(mg_tree *t, int64_t *nblocks, int64_t *out) {
    if (!t || !nblocks) return fail(MG_ERR_ARG, "null argument");
    int rc = build(t);
    if (rc) return rc;
    *nblocks = (int64_t)t->blocks.size();
    if (!out) return MG_OK;
    for (size_t g = 0; g < t->blocks.size(); g++) {
        const BlockDesc &B = t->blocks[g];
        int64_t *o = out + 24 * g;
        o[0] = B.cell_off; o[1] = B.ghost_off; o[2] = B.n; o[3] = B.lev; o[4] = B.flags; o[5] = B.parent;
        for (int d = 0; d < 3; d++) { o[6 + d] = B.ijk[d]; o[9 + d] = B.poff[d]; }
        for (int f = 0; f < 6; f++) { o[12 + f] = B.nbr[f]; o[18 + f] = B.push[f]; }
    }
    return MG_OK;
}

extern "C" int mg_tree_num_levels(mg_tree *t, int *nlev) {
    if (!t || !nlev) return fail(MG_ERR_ARG, "null argument");
    int rc = build(t);
    if (rc) return rc;
    *nlev = (int)t->lev.size();
    return MG_OK;
}

extern "C" int mg_tree_level_info(mg_tree *t, int level, int32_t info[9], double h[3]) {
    if (!t || !info || !h) return fail(MG_ERR_ARG, "null argument");
    int rc = build(t);
    if (rc) return rc;
    if (level < 0 || level >= (int)t->lev.size()) return fail(MG_ERR_ARG, "level out of range");
    const LevelHost &L = t->lev[level];
    info[0] = L.n; info[1] = L.depth; info[2] = L.nb;
    for (int d = 0; d < 3; d++) { info[3 + d] = L.nblk[d]; info[6 + d] = L.ncell[d]; h[d] = L.h[d]; }
    return MG_OK;
}

extern "C" int mg_tree_num_leaf_cells(mg_tree *t, int64_t *n) {
    if (!t || !n) return fail(MG_ERR_ARG, "null argument");
    int rc = build(t);
    if (rc) return rc;
    *n = t->nleaf_cells;
    return MG_OK;
}

extern "C" int mg_tree_leaf_blocks(mg_tree *t, int32_t *out) {
    if (!t || !out) return fail(MG_ERR_ARG, "null argument");
    int rc = build(t);
    if (rc) return rc;
    long long m = 0;
    for (const LevelHost &L : t->lev)
        for (int r = L.nref; r < L.nb; r++) {
            const BlockDesc &B = t->blocks[L.first + r];
            out[4 * m] = L.depth;
            out[4 * m + 1] = B.ijk[0];
            out[4 * m + 2] = B.ijk[1];
            out[4 * m + 3] = B.ijk[2];
            m++;
        }
    return MG_OK;
}

// ------------------------------------------------ device allocation ----

template <class T> static int dalloc(T **p, long long n) {
    if (*p) return MG_OK;
    CK(cudaMalloc((void **)p, sizeof(T) * (size_t)std::max(1LL, n)));
    CK(cudaMemset(*p, 0, sizeof(T) * (size_t)std::max(1LL, n)));
    return MG_OK;
}

template <class T> static int alloc_fields(mg_tree *t, Fields<T> &F, bool with_eps) {
    int rc;
    if ((rc = dalloc(&F.X, t->ncells)) || (rc = dalloc(&F.XG, t->nghost)) || (rc = dalloc(&F.F, t->ncells)) ||
        (rc = dalloc(&F.V, t->ncells)) || (rc = dalloc(&F.VG, t->nghost)))
        return rc;
    if (with_eps && ((rc = dalloc(&F.E, t->ncells)) || (rc = dalloc(&F.EG, t->nghost)))) return rc;
    return MG_OK;
}

template <class T> static void free_fields(Fields<T> &F, bool free_eps) {
    cudaFree(F.X); cudaFree(F.XG); cudaFree(F.F); cudaFree(F.V); cudaFree(F.VG);
    if (free_eps) { cudaFree(F.E); cudaFree(F.EG); }
    F = Fields<T>();
}

static void drop_graphs(mg_tree *t);

static int upload_bc(mg_tree *t) {
    drop_graphs(t);
    std::vector<double> all;
    const std::vector<LevelHost> &src = t->is_batch ? t->tl : t->lev;
    std::vector<LevelDesc> ld(src.size());
    for (size_t l = 0; l < src.size(); l++) {
        const LevelHost &L = src[l];
        LevelDesc &d = ld[l];
        for (int e = 0; e < 3; e++) {
            d.h[e] = L.h[e];
            d.inv_h2[e] = 1.0 / (L.h[e] * L.h[e]);
            d.ncell[e] = L.ncell[e];
        }
        d.n = L.n; d.first = L.first; d.nb = L.nb; d.nref = L.nref;
        {
            double sw = 0;
            for (int e = 0; e < t->dim; e++) sw += d.inv_h2[e];
            d.diag = 2.0 * sw + t->helm;
            d.inv_diag = 1.0 / d.diag;
            d.vol = L.h[0] * L.h[1] * (t->dim == 3 ? L.h[2] : 1.0);
            for (int e = 0; e < 3; e++) d.inv_h2f[e] = (float)d.inv_h2[e];
            d.inv_diagf = (float)d.inv_diag;
            d.h0f = (float)L.h[0];
            d.hvf = (float)(2.0 * M_PI * L.h[0] * L.h[1]);
        }
        for (int f = 0; f < 6; f++) {
            d.bc_off[f] = -1;
            if (!L.bc[f].empty()) {
                d.bc_off[f] = (long long)all.size();
                all.insert(all.end(), L.bc[f].begin(), L.bc[f].end());
            }
        }
    }
    if (!t->d_levels) CK(cudaMalloc((void **)&t->d_levels, sizeof(LevelDesc) * ld.size()));
    CK(cudaMemcpy(t->d_levels, ld.data(), sizeof(LevelDesc) * ld.size(), cudaMemcpyHostToDevice));
    if ((long long)all.size() > t->n_bcplanes) {
        cudaFree(t->d_bcplanes);
        t->d_bcplanes = nullptr;
        CK(cudaMalloc((void **)&t->d_bcplanes, sizeof(double) * all.size()));
        t->n_bcplanes = (long long)all.size();
    }
    if (!all.empty())
        CK(cudaMemcpy(t->d_bcplanes, all.data(), sizeof(double) * all.size(), cudaMemcpyHostToDevice));
    t->bc_dirty = false;
    return MG_OK;
}

// The coarsest-level operator with homogeneous boundary values, assembled
// from the 5/7-point stencil (bordered by sum V x = 0 when the problem has
// no Dirichlet face): emit(row, col, value) adds value to M[row][col];
// rows and columns are tree-local cells in block order (b C + c), col == nc
// is the border.
template <class Emit>
static void assemble_coarse(const mg_tree *t, const TreeCoarse &tc, const LevelHost &L, const double *eps,
                            Emit emit) {
    const int D = t->dim;
    const int n = L.n, C = (int)ipow(n, D), nc = tc.nc;
    std::vector<int> rowmap((size_t)L.ncell[0] * L.ncell[1] * L.ncell[2]);
    auto cellkey = [&](const int *G) { return ((size_t)G[2] * L.ncell[1] + G[1]) * L.ncell[0] + G[0]; };
    for (int b = 0; b < tc.nb; b++) {
        const BlockDesc &B = t->blocks[tc.first + b];
        for (int c = 0; c < C; c++) {
            int G[3] = {B.ijk[0] * n + c % n, B.ijk[1] * n + (c / n) % n, D == 3 ? B.ijk[2] * n + c / (n * n) : 0};
            rowmap[cellkey(G)] = b * C + c;
        }
    }
    for (int b = 0; b < tc.nb; b++) {
        const BlockDesc &B = t->blocks[tc.first + b];
        for (int c = 0; c < C; c++) {
            const int row = b * C + c;
            int G[3] = {B.ijk[0] * n + c % n, B.ijk[1] * n + (c / n) % n, D == 3 ? B.ijk[2] * n + c / (n * n) : 0};
            const double ri = t->lo[0] + (G[0] + 0.5) * L.h[0];
            for (int d = 0; d < D; d++)
                for (int s = 0; s < 2; s++) {
                    int Q[3] = {G[0], G[1], G[2]};
                    Q[d] += s ? 1 : -1;
                    bool phys = false;
                    if (Q[d] < 0 || Q[d] >= L.ncell[d]) {
                        if (t->bc.type[2 * d + s] == MG_BC_PERIODIC) Q[d] = (Q[d] + L.ncell[d]) % L.ncell[d];
                        else phys = true;
                    }
                    double w = 1.0 / (L.h[d] * L.h[d]);
                    const int col = phys ? -1 : rowmap[cellkey(Q)];
                    const double ec = eps ? eps[row] : 1.0, eo = phys ? ec : (eps ? eps[col] : 1.0);
                    w *= 2.0 * ec * eo / (ec + eo);
                    if (t->geom == MG_CYL && d == 0) w *= (t->lo[0] + (G[0] + s) * L.h[0]) / ri;
                    if (!phys) {
                        emit(row, col, w);
                        emit(row, row, -w);
                    } else if (t->bc.type[2 * d + s] == MG_BC_DIRICHLET) {
                        emit(row, row, -2.0 * w);
                    }
                }
            emit(row, row, -t->helm);
            if (tc.singular) {
                double V = 1.0;
                for (int d = 0; d < D; d++) V *= L.h[d];
                if (t->geom == MG_CYL) V = 2.0 * M_PI * ri * L.h[0] * L.h[1];
                emit(row, nc, 1.0);
                emit(nc, row, V);
            }
        }
    }
}

// In-place inverse of the m x m row-major matrix A by Gauss-Jordan
// elimination with partial pivoting; A is overwritten, Inv receives A^-1.
static bool gauss_jordan(std::vector<double> &A, double *Inv, int m) {
    for (size_t i = 0; i < (size_t)m * m; i++) Inv[i] = 0.0;
    for (int i = 0; i < m; i++) Inv[(size_t)i * m + i] = 1.0;
    for (int c = 0; c < m; c++) {
        int p = c;
        for (int r = c + 1; r < m; r++)
            if (std::fabs(A[(size_t)r * m + c]) > std::fabs(A[(size_t)p * m + c])) p = r;
        if (A[(size_t)p * m + c] == 0.0) return false;
        if (p != c)
            for (int e = 0; e < m; e++) {
                std::swap(A[(size_t)c * m + e], A[(size_t)p * m + e]);
                std::swap(Inv[(size_t)c * m + e], Inv[(size_t)p * m + e]);
            }
        const double piv = 1.0 / A[(size_t)c * m + c];
        for (int e = 0; e < m; e++) { A[(size_t)c * m + e] *= piv; Inv[(size_t)c * m + e] *= piv; }
        for (int r = 0; r < m; r++) {
            if (r == c) continue;
            const double f = A[(size_t)r * m + c];
            if (f == 0.0) continue;
            for (int e = 0; e < m; e++) {
                A[(size_t)r * m + e] -= f * A[(size_t)c * m + e];
                Inv[(size_t)r * m + e] -= f * Inv[(size_t)c * m + e];
            }
        }
    }
    return true;
}

// Dense inverse of one tree's coarsest-level operator (FP64, host).
static std::string coarse_inverse_one(const mg_tree *t, const TreeCoarse &tc, const LevelHost &L,
                                      const double *eps, double *Inv) {
    const int ns = tc.ns;
    std::vector<double> M((size_t)ns * ns, 0.0);
    assemble_coarse(t, tc, L, eps, [&](int r, int c, double v) { M[(size_t)r * ns + c] += v; });
    if (!gauss_jordan(M, Inv, ns)) return "coarsest-level matrix is singular";
    return "";
}

// Plane of cell `row` (block order) across dimension bt_dim, and its index
// within the plane (the other dimensions lexicographically, lowest first).
static void plane_of(const mg_tree *t, const TreeCoarse &tc, const LevelHost &L, int row, int &j, int &p) {
    const int D = t->dim, n = L.n, C = (int)ipow(n, D), c = row % C;
    const BlockDesc &B = t->blocks[tc.first + row / C];
    const int G[3] = {B.ijk[0] * n + c % n, B.ijk[1] * n + (c / n) % n, D == 3 ? B.ijk[2] * n + c / (n * n) : 0};
    j = G[tc.bt_dim];
    p = 0;
    for (int d = D - 1; d >= 0; d--)
        if (d != tc.bt_dim) p = p * L.ncell[d] + G[d];
}

// Block-tridiagonal factorisation of one tree's coarsest-level operator
// over the planes j = 0 .. NP-1 of dimension bt_dim: with A_j, C_j the
// (diagonal) couplings of plane j to planes j-1, j+1 and B_j the operator
// within plane j, S_0 = B_0, S_j = B_j - A_j S_{j-1}^-1 C_{j-1}, and the
// solve M x = r runs z_j = r_j - A_j S_{j-1}^-1 z_{j-1} forwards, then
// x_j = S_j^-1 (z_j - C_j x_{j+1}) backwards.  Writes the plane records
// (S_j^-1 column by column, then the diagonals of A_j and C_j) and the
// plane-order -> row map.
static std::string coarse_btri_one(const mg_tree *t, const TreeCoarse &tc, const LevelHost &L, const double *eps,
                                   double *rec, int *perm) {
    const int P = tc.bt_P, NP = tc.bt_n, nc = tc.nc, st = bt_stride(P);
    std::vector<int> pos(nc);
    for (int row = 0; row < nc; row++) {
        int j, p;
        plane_of(t, tc, L, row, j, p);
        if (j < 0 || j >= NP || p < 0 || p >= P) return "internal: plane index out of range";
        pos[row] = j * P + p;
        perm[j * P + p] = row;
    }
    std::vector<double> B((size_t)NP * P * P, 0.0), A((size_t)NP * P, 0.0), Cu((size_t)NP * P, 0.0);
    bool ok = true;
    assemble_coarse(t, tc, L, eps, [&](int r, int c, double v) {
        if (r >= nc || c >= nc) { ok = false; return; }  // bordered systems keep the dense form
        const int jr = pos[r] / P, pr = pos[r] % P, jc = pos[c] / P, pc = pos[c] % P;
        if (jc == jr) B[((size_t)jr * P + pr) * P + pc] += v;
        else if (jc == jr - 1 && pc == pr) A[(size_t)jr * P + pr] += v;
        else if (jc == jr + 1 && pc == pr) Cu[(size_t)jr * P + pr] += v;
        else ok = false;
    });
    if (!ok) return "internal: coarsest operator is not block tridiagonal across the planes";
    std::vector<double> S((size_t)P * P), Sinv((size_t)P * P), prev((size_t)P * P);
    for (int j = 0; j < NP; j++) {
        for (int p = 0; p < P; p++)
            for (int q = 0; q < P; q++) {
                double v = B[((size_t)j * P + p) * P + q];
                if (j > 0) v -= A[(size_t)j * P + p] * prev[(size_t)p * P + q] * Cu[(size_t)(j - 1) * P + q];
                S[(size_t)p * P + q] = v;
            }
        if (!gauss_jordan(S, Sinv.data(), P)) return "coarsest-level matrix is singular";
        double *R = rec + (size_t)j * st;
        for (int k = 0; k < P; k++)
            for (int p = 0; p < P; p++) R[(size_t)k * P + p] = Sinv[(size_t)p * P + k];
        for (int p = 0; p < P; p++) {
            R[P * P + p] = A[(size_t)j * P + p];       // zero on plane 0
            R[P * P + P + p] = Cu[(size_t)j * P + p];  // zero on the last plane
        }
        for (int e = P * P + 2 * P; e < st; e++) R[e] = 0.0;
        prev.swap(Sinv);
    }
    return "";
}

// Chooses the block-tridiagonal form for one tree of a pool of several
// trees: a non-singular coarsest level with a non-periodic dimension of at
// least 4 planes whose planes hold at most kBtriMaxPlane cells (the longest
// such dimension).  Its forward and backward sweeps cost 2 nc P FMAs and
// bytes against nc^2 for the dense inverse.  A single tree keeps the dense
// inverse, whose rows are applied by many CTAs at once.
static void coarse_plan(const mg_tree *src, TreeCoarse &tc, const LevelHost &L, bool pool) {
    tc.bt_n = tc.bt_P = tc.bt_dim = 0;
    if (!pool || tc.singular) return;
    int best = -1;
    for (int d = 0; d < src->dim; d++) {
        if (src->bc.type[2 * d] == MG_BC_PERIODIC) continue;
        const int np = L.ncell[d];
        if (np < 4 || tc.nc / np > kBtriMaxPlane) continue;
        if (best < 0 || np > L.ncell[best]) best = d;
    }
    if (best < 0) return;
    tc.bt_dim = best;
    tc.bt_n = L.ncell[best];
    tc.bt_P = tc.nc / tc.bt_n;
}

// Coarsest-level factors of every tree (trees in parallel host threads):
// dense inverses, and plane records of the block-tridiagonal trees.
int build_coarse_inverse(mg_tree *t) {
    std::vector<double> eps;
    if (t->var_eps) {
        CK(cudaStreamSynchronize(t->stream));
        eps.resize(t->ncells);
        CK(cudaMemcpy(eps.data(), t->f64.E, sizeof(double) * t->ncells, cudaMemcpyDeviceToHost));
    }
    std::vector<double> inv(t->minv_total), bt(t->bt_total);
    std::vector<float> bt32(t->bt_total32);
    std::vector<int> perm(t->btperm_total);
    std::vector<std::string> errs(t->tcoarse.size());
    const int nthr = (int)std::max<unsigned>(1, std::min<unsigned>(std::thread::hardware_concurrency(), 64));
    std::atomic<int> next(0);
    auto work = [&]() {
        for (int i = next++; i < (int)t->tcoarse.size(); i = next++) {
            const TreeCoarse &tc = t->tcoarse[i];
            const LevelHost &L = t->is_batch ? t->tl[tc.lvl] : t->lev[tc.lvl];
            const double *e = t->var_eps ? eps.data() + tc.cell0 : nullptr;
            if (!tc.bt_n) {
                errs[i] = coarse_inverse_one(t, tc, L, e, inv.data() + tc.minv_off);
                continue;
            }
            errs[i] = coarse_btri_one(t, tc, L, e, bt.data() + tc.bt_off, perm.data() + tc.perm_off);
            const int Pp = tc.bt_P, st = bt_stride(Pp), st32 = bt32_stride(Pp), row = bt32_row(Pp);
            const int r4 = bt_round4(Pp);
            for (int j = 0; j < tc.bt_n; j++) {  // FP32 records, padding zero
                const double *R = bt.data() + tc.bt_off + (size_t)j * st;
                float *Q = bt32.data() + tc.bt_off32 + (size_t)j * st32;
                for (int q = 0; q < st32; q++) Q[q] = 0.0f;
                for (int p = 0; p < Pp; p++) {
                    for (int k = 0; k < Pp; k++) Q[(size_t)p * row + k] = (float)R[(size_t)k * Pp + p];
                    if (j + 1 < tc.bt_n)  // A_{j+1}: the next plane's record holds it at P^2 + p
                        Q[(size_t)Pp * row + p] = (float)R[(size_t)st + (size_t)Pp * Pp + p];
                    if (j > 0)  // C_{j-1}: the previous plane's record holds it at P^2 + P + p
                        Q[(size_t)Pp * row + r4 + p] = (float)R[-(ptrdiff_t)st + (ptrdiff_t)Pp * Pp + Pp + p];
                }
            }
        }
    };
    std::vector<std::thread> pool;
    for (int k = 1; k < std::min<int>(nthr, (int)t->tcoarse.size()); k++) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
    for (auto &e : errs)
        if (!e.empty()) return fail(MG_ERR_ARG, e);
    if (!t->d_minv) CK(cudaMalloc((void **)&t->d_minv, sizeof(double) * (size_t)std::max(1LL, t->minv_total)));
    if (t->minv_total) CK(cudaMemcpy(t->d_minv, inv.data(), sizeof(double) * (size_t)t->minv_total, cudaMemcpyHostToDevice));
    if (t->bt_total) {
        if (!t->d_bt) CK(cudaMalloc((void **)&t->d_bt, sizeof(double) * (size_t)t->bt_total));
        if (!t->d_bt32) CK(cudaMalloc((void **)&t->d_bt32, sizeof(float) * (size_t)t->bt_total32));
        if (!t->d_btperm) CK(cudaMalloc((void **)&t->d_btperm, sizeof(int) * (size_t)t->btperm_total));
        CK(cudaMemcpy(t->d_bt, bt.data(), sizeof(double) * (size_t)t->bt_total, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(t->d_bt32, bt32.data(), sizeof(float) * (size_t)t->bt_total32, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(t->d_btperm, perm.data(), sizeof(int) * (size_t)t->btperm_total, cudaMemcpyHostToDevice));
    }
    t->minv_ok = true;
    return MG_OK;
}

// per segment: refinement faces present, and the segments of its parents
static void annotate_segments(mg_tree *t) {
    std::vector<int> seg(t->blocks.size(), 0);
    for (size_t l = 0; l < t->lev.size(); l++)
        for (int b = 0; b < t->lev[l].nb; b++) seg[t->lev[l].first + b] = (int)l;
    for (LevelHost &L : t->lev) {
        L.has_cf = 0;
        L.parents.clear();
        for (int b = L.first; b < L.first + L.nb; b++) {
            const BlockDesc &B = t->blocks[b];
            for (int f = 0; f < 2 * t->dim; f++)
                if (B.nbr[f] <= -2) L.has_cf = 1;
            if (B.parent >= 0 && std::find(L.parents.begin(), L.parents.end(), seg[B.parent]) == L.parents.end())
                L.parents.push_back(seg[B.parent]);
        }
    }
}

extern "C" int mg_tree_finalize(mg_tree *t, void *stream) {
    if (!t) return fail(MG_ERR_ARG, "null tree");
    if (t->finalized) return fail(MG_ERR_STATE, "already finalized");
    int rc = build(t);
    if (rc) return rc;
    const auto t1 = std::chrono::steady_clock::now();
    annotate_segments(t);
    CK(cudaGetDevice(&t->device));
    CK(cudaDeviceGetAttribute(&t->nsm, cudaDevAttrMultiProcessorCount, t->device));
    t->stream = (cudaStream_t)stream;
    if (t->d_blocks_built) {  // the device build's table (same entries as t->blocks)
        t->d_blocks = t->d_blocks_built;
        t->d_blocks_built = nullptr;
    } else {
        CK(cudaMalloc((void **)&t->d_blocks, sizeof(BlockDesc) * t->blocks.size()));
        CK(cudaMemcpy(t->d_blocks, t->blocks.data(), sizeof(BlockDesc) * t->blocks.size(), cudaMemcpyHostToDevice));
    }
    if ((rc = upload_bc(t))) return rc;
    if ((rc = alloc_fields(t, t->f64, false))) return rc;
    int maxleaf = 0;
    long long nleafb = 0;
    for (auto &L : t->lev) { maxleaf = std::max(maxleaf, L.nb - L.nref); nleafb += L.nb - L.nref; }
    t->n_partials = (int)nleafb;
    if ((rc = dalloc(&t->d_partials, 3 * nleafb))) return rc;
    if ((rc = dalloc(&t->d_red, 3))) return rc;
    if ((rc = dalloc(&t->d_status, kStatusWords))) return rc;
    if ((rc = dalloc(&t->d_cvec, t->cvec_total))) return rc;
    CK(cudaMalloc((void **)&t->d_tcoarse, sizeof(TreeCoarse) * t->tcoarse.size()));
    CK(cudaMemcpy(t->d_tcoarse, t->tcoarse.data(), sizeof(TreeCoarse) * t->tcoarse.size(), cudaMemcpyHostToDevice));
    {  // work lists of the coarse solve: kCoarseRows rows of one dense tree
       // per CTA; one CTA per block-tridiagonal tree
        std::vector<int2> ch;
        std::vector<int> bl;
        t->bt_pmax = t->bt_ncmax = 0;
        for (size_t i = 0; i < t->tcoarse.size(); i++) {
            const TreeCoarse &tc = t->tcoarse[i];
            if (tc.bt_n) {
                bl.push_back((int)i);
                t->bt_pmax = std::max(t->bt_pmax, tc.bt_P);
                t->bt_ncmax = std::max(t->bt_ncmax, tc.nc);
                continue;
            }
            for (int r = 0; r < tc.nc; r += kCoarseRows) ch.push_back(make_int2((int)i, r));
        }
        // largest first: CTAs start in list order, so the SMs each get a
        // share of the large trees
        std::stable_sort(bl.begin(), bl.end(), [&](int a, int b) {
            const TreeCoarse &A = t->tcoarse[a], &B = t->tcoarse[b];
            return (long long)A.nc * A.bt_P > (long long)B.nc * B.bt_P;
        });
        std::vector<int2> bc;  // block-form residual: kBtResidCells cells of one tree per CTA
        for (int i : bl)
            for (int r = 0; r < t->tcoarse[i].nc; r += kBtResidCells) bc.push_back(make_int2(i, r));
        t->n_bt_chunks = (int)bc.size();
        CK(cudaMalloc((void **)&t->d_bt_chunks, sizeof(int2) * std::max<size_t>(1, bc.size())));
        if (!bc.empty()) CK(cudaMemcpy(t->d_bt_chunks, bc.data(), sizeof(int2) * bc.size(), cudaMemcpyHostToDevice));
        t->n_coarse_chunks = (int)ch.size();
        t->n_btri = (int)bl.size();
        CK(cudaMalloc((void **)&t->d_coarse_chunks, sizeof(int2) * std::max<size_t>(1, ch.size())));
        if (!ch.empty()) CK(cudaMemcpy(t->d_coarse_chunks, ch.data(), sizeof(int2) * ch.size(), cudaMemcpyHostToDevice));
        CK(cudaMalloc((void **)&t->d_btlist, sizeof(int) * std::max<size_t>(1, bl.size())));
        if (!bl.empty()) CK(cudaMemcpy(t->d_btlist, bl.data(), sizeof(int) * bl.size(), cudaMemcpyHostToDevice));
    }
    CK(cudaMallocHost((void **)&t->h_red, 3 * sizeof(double)));
    CK(cudaStreamCreateWithFlags(&t->cap_stream, cudaStreamNonBlocking));
    t->finalized = true;
    if ((rc = build_coarse_inverse(t))) return rc;
    if (t->geom == MG_CYL) {  // r-face factors: precomputed FP64 face coefficients
        if ((rc = dalloc(&t->d_wface, t->ncells * wstride(t->dim)))) return rc;
        t->f64.W = t->d_wface;
        face_coef(t);
    }
    CK(cudaStreamSynchronize(t->stream));
    t->build_s[1] = seconds_since(t1);
    const auto t2 = std::chrono::steady_clock::now();
    if (!apply_tune_hint(t, 0)) tune_sweeps<double>(t, t->f64);  // fields and ghosts are still zero here
    CK(cudaMemsetAsync(t->f64.X, 0, sizeof(double) * t->ncells, t->stream));
    refresh<double>(t, t->f64, 0);
    rc = check_cuda("finalize");
    CK(cudaStreamSynchronize(t->stream));
    t->build_s[2] = seconds_since(t2);
    return rc;
}

#define NEED_FINAL(t)                                                            \
    do {                                                                         \
        if (!(t)) return fail(MG_ERR_ARG, "null tree");                           \
        if (!(t)->finalized) return fail(MG_ERR_STATE, "tree not finalized");     \
    } while (0)

extern "C" int mg_tree_build_times(mg_tree *t, double *out4) {
    if (!t || !out4) return fail(MG_ERR_ARG, "null argument");
    for (int i = 0; i < 4; i++) out4[i] = t->build_s[i];
    return MG_OK;
}

// ------------------------------------------------------------- adapt ----
// A new mesh from a finalized one (Sec. 2.5, "Adapting the grid structure"):
// the refinement list of t with the listed leaf blocks refined and the
// listed refinements (of blocks whose children are all leaves) undone;
// phi is carried over on the device (k_transfer).

static uint64_t block_key(int depth, int i, int j, int k) {
    return ((uint64_t)(depth + 128) << 56) | ((uint64_t)i << 36) | ((uint64_t)j << 18) | (uint64_t)k;
}

extern "C" int mg_tree_adapt(mg_tree *t, int n_add, const int32_t *add, int n_remove, const int32_t *remove,
                             mg_tree **out) {
    NEED_FINAL(t);
    if (!out || n_add < 0 || n_remove < 0 || (n_add > 0 && !add) || (n_remove > 0 && !remove))
        return fail(MG_ERR_ARG, "bad adapt arguments");
    if (t->is_batch) return fail(MG_ERR_ARG, "adapt takes a single tree");
    *out = nullptr;
    const int D = t->dim;
    // blocks of t by (depth, coordinates): global id, and whether a leaf
    std::unordered_map<uint64_t, int> old_id;
    old_id.reserve(t->blocks.size() * 2);
    for (const LevelHost &L : t->lev)
        for (int b = 0; b < L.nb; b++) {
            const BlockDesc &q = t->blocks[L.first + b];
            if (q.ijk[0] >= (1 << 18) || q.ijk[1] >= (1 << 18) || q.ijk[2] >= (1 << 18))
                return fail(MG_ERR_ARG, "mesh too large to adapt");
            old_id[block_key(L.depth, q.ijk[0], q.ijk[1], q.ijk[2])] = L.first + b;
        }
    auto is_leaf = [&](int g) { return !(t->blocks[g].flags & 1); };
    auto rec = [&](const int32_t *e) { return std::array<int, 4>{e[0], e[1], e[2], D == 3 ? e[3] : 0}; };
    auto find = [&](const std::array<int, 4> &r) -> int {
        if (r[1] < 0 || r[2] < 0 || r[3] < 0 || r[1] >= (1 << 18) || r[2] >= (1 << 18) || r[3] >= (1 << 18))
            return -1;
        auto it = old_id.find(block_key(r[0], r[1], r[2], r[3]));
        return it == old_id.end() ? -1 : it->second;
    };
    // refined blocks of t (depth >= 0), then the requested changes
    std::map<std::array<int, 4>, char> ref;
    for (size_t e = 0; e < t->refine.size() / 4; e++) ref[rec(&t->refine[4 * e])] = 1;
    for (int r = 0; r < n_remove; r++) {
        const auto q = rec(remove + 4 * r);
        auto it = ref.find(q);
        if (it == ref.end() || !it->second) return fail(MG_ERR_ARG, "removed refinement does not exist");
        for (int c = 0; c < (1 << D); c++) {
            const int g = find({q[0] + 1, 2 * q[1] + (c & 1), 2 * q[2] + ((c >> 1) & 1), D == 3 ? 2 * q[3] + ((c >> 2) & 1) : 0});
            if (g < 0 || !is_leaf(g)) return fail(MG_ERR_ARG, "a removed refinement has refined children");
        }
        it->second = 0;
    }
    for (int a = 0; a < n_add; a++) {
        const auto q = rec(add + 4 * a);
        const int g = q[0] >= 0 ? find(q) : -1;
        if (g < 0 || !is_leaf(g)) return fail(MG_ERR_ARG, "refined block is not a leaf of the mesh");
        auto it = ref.find(q);
        if (it != ref.end()) return fail(MG_ERR_ARG, "block both refined and coarsened");
        ref[q] = 1;
    }
    mg_tree *nt = nullptr;
    int rc = mg_tree_create(D, t->N, t->geom, &t->bc, t->base, t->lo, t->hi, t->coarse_max, t->helm, &nt);
    if (rc) return rc;
    for (const auto &kv : ref)
        if (kv.second) nt->refine.insert(nt->refine.end(), kv.first.begin(), kv.first.end());
    // boundary planes of the levels both meshes have (same depth, same size)
    if ((rc = build(nt))) {
        const std::string msg = mg_last_error();
        mg_tree_destroy(nt);
        return fail(rc, msg);
    }
    for (LevelHost &NL : nt->lev)
        for (const LevelHost &OL : t->lev)
            if (OL.depth == NL.depth && OL.n == NL.n)
                for (int f = 0; f < 6; f++) NL.bc[f] = OL.bc[f];
    // sweep kernels: the old tree's choices by depth, no second autotuning
    for (int prec = 0; prec < 2; prec++)
        for (size_t l = 0; l < t->sweep_choice[prec].size() && l < t->lev.size(); l++)
            nt->tune_hint[prec][t->lev[l].depth] = t->sweep_choice[prec][l];
    if ((rc = mg_tree_finalize(nt, t->stream))) {
        const std::string msg = mg_last_error();
        mg_tree_destroy(nt);
        return fail(rc, msg);
    }
    // source of every new leaf block: the same block of t, or its parent
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<int> nid, src;
    for (const LevelHost &L : nt->lev)
        for (int b = L.nref; b < L.nb; b++) {
            const BlockDesc &q = nt->blocks[L.first + b];
            int g = find({L.depth, q.ijk[0], q.ijk[1], q.ijk[2]});
            if (g < 0) {
                const int p = find({L.depth - 1, q.ijk[0] / 2, q.ijk[1] / 2, D == 3 ? q.ijk[2] / 2 : 0});
                if (p < 0 || !is_leaf(p)) {
                    mg_tree_destroy(nt);
                    return fail(MG_ERR_ARG, "adapted block without a source block");
                }
                g = -2 - p;
            }
            nid.push_back(L.first + b);
            src.push_back(g);
        }
    if ((rc = transfer_phi(t, nt, nid, src))) {
        mg_tree_destroy(nt);
        return rc;
    }
    nt->build_s[3] = seconds_since(t0);
    *out = nt;
    return MG_OK;
}

// device status word: a bounded wait inside a kernel gave up (reported once)
static int check_status(mg_tree *t) {
    int st = 0;
    CK(cudaStreamSynchronize(t->stream));
    CK(cudaMemcpy(&st, t->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
        CK(cudaMemset(t->d_status, 0, sizeof(int) * kStatusWords));
        return fail(MG_ERR_TIMEOUT, "a bounded wait in a kernel expired");
    }
    return MG_OK;
}

// Graphs of cycle sequences: captured once per key on the private capture
// stream, replayed on the user stream.  Pointers baked into the captured
// kernels (fields, tables, boundary planes) are stable until a call that
// reallocates or rebinds them, which drops every graph.
static void drop_graphs(mg_tree *t) {
    for (auto &kv : t->graphs) cudaGraphExecDestroy(kv.second.exec);
    t->graphs.clear();
}

template <class Fn> static int run_graph(mg_tree *t, const std::string &key, Fn &&enqueue) {
    if (!t->use_graphs) {
        enqueue();
        return check_cuda("enqueue");
    }
    auto it = t->graphs.find(key);
    if (it == t->graphs.end()) {
        cudaStream_t user = t->stream;
        const long long l0 = t->launches;
        CK(cudaStreamSynchronize(user));
        t->stream = t->cap_stream;
        cudaError_t e = cudaStreamBeginCapture(t->cap_stream, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) enqueue();
        const std::string le = take_launch_error();  // a launch refused during capture is missing from the graph
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(t->cap_stream, &g);
        t->stream = user;
        cudaGetLastError();
        if (!le.empty()) {
            if (g) cudaGraphDestroy(g);
            return fail(MG_ERR_CUDA, "kernel launch failed while capturing " + key + ": " + le);
        }
        if (e != cudaSuccess || e2 != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            t->use_graphs = false;  // capture unavailable: launch directly from now on
            t->launches = l0;
            enqueue();
            return check_cuda("enqueue");
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        it = t->graphs.emplace(key, mg_tree::Graph{exec, t->launches - l0}).first;
        t->launches = l0;
    }
    t->launches += it->second.launches;
    CK(cudaGraphLaunch(it->second.exec, t->stream));
    return MG_OK;
}

extern "C" int mg_set_bc_plane(mg_tree *t, int face, int level, const double *vals) {
    if (!t || !vals) return fail(MG_ERR_ARG, "null argument");
    int rc = build(t);
    if (rc) return rc;
    if (face < 0 || face >= 2 * t->dim || level < 0 || level >= (int)t->lev.size())
        return fail(MG_ERR_ARG, "face or level out of range");
    LevelHost &L = t->lev[level];
    const int d = face / 2;
    long long cnt = 1;
    for (int e = 0; e < t->dim; e++)
        if (e != d) cnt *= L.ncell[e];
    L.bc[face].assign(vals, vals + cnt);
    if (t->finalized) {
        if ((rc = upload_bc(t))) return rc;
        refresh<double>(t, t->f64, 0);
        return check_cuda("set_bc_plane");
    }
    return MG_OK;
}

// copy between a leaf-order vector and the leaf cells of a pool field
template <class T> static int leaf_copy(mg_tree *t, T *cells, const T *leaf, bool to_cells) {
    if (t->is_batch) {
        if constexpr (sizeof(T) == sizeof(double)) {
            leaf_runs_copy(t, cells, leaf, to_cells);
            return MG_OK;
        } else {
            return fail(MG_ERR_UNSUPPORTED, "batch leaf copies are FP64");
        }
    }
    long long off = 0;
    for (auto &L : t->lev) {
        const long long n = (long long)(L.nb - L.nref) * ipow(L.n, t->dim);
        if (n == 0) continue;
        const long long c0 = t->blocks[L.first + L.nref].cell_off;
        if (to_cells)
            CK(cudaMemcpyAsync(cells + c0, leaf + off, sizeof(T) * n, cudaMemcpyDeviceToDevice, t->stream));
        else
            CK(cudaMemcpyAsync((T *)leaf + off, cells + c0, sizeof(T) * n, cudaMemcpyDeviceToDevice, t->stream));
        off += n;
    }
    return MG_OK;
}

extern "C" int mg_set_rhs(mg_tree *t, const double *f) {
    NEED_FINAL(t);
    if (!f) return fail(MG_ERR_ARG, "null rhs");
    return leaf_copy(t, t->f64.F, f, true);
}

extern "C" int mg_set_phi(mg_tree *t, const double *x) {
    NEED_FINAL(t);
    if (!x) return fail(MG_ERR_ARG, "null phi");
    int rc = leaf_copy(t, t->f64.X, x, true);
    if (rc) return rc;
    refresh<double>(t, t->f64, 0);
    return check_cuda("set_phi");
}

extern "C" int mg_get_phi(mg_tree *t, double *x) {
    NEED_FINAL(t);
    if (!x) return fail(MG_ERR_ARG, "null phi");
    return leaf_copy(t, t->f64.X, (const double *)x, false);
}

extern "C" int mg_set_eps(mg_tree *t, const double *e) {
    NEED_FINAL(t);
    if (!e) return fail(MG_ERR_ARG, "null eps");
    int rc;
    if ((rc = dalloc(&t->f64.E, t->ncells)) || (rc = dalloc(&t->f64.EG, t->nghost))) return rc;
    if (!t->var_eps) drop_graphs(t);  // eps pointers enter the captured kernels
    t->var_eps = true;
    if ((rc = leaf_copy(t, t->f64.E, e, true))) return rc;
    refresh_eps<double>(t, t->f64);
    if ((rc = dalloc(&t->d_wface, t->ncells * wstride(t->dim)))) return rc;
    t->f64.W = t->d_wface;  // precomputed FP64 face coefficients for the residual
    face_coef(t);
    t->adj.E = t->f64.E;
    t->adj.W = t->f64.W;
    t->adj.EG = t->f64.EG;
    if (t->f32.X) {
        if ((rc = dalloc(&t->f32.E, t->ncells)) || (rc = dalloc(&t->f32.EG, t->nghost))) return rc;
        copy_eps_to_f32(t);
    }
    if ((rc = check_cuda("set_eps"))) return rc;
    return build_coarse_inverse(t);
}

static void params_or_default(const mg_params *p, mg_params *q) {
    if (p) *q = *p;
    else {
        *q = mg_params{};
        q->n_down = 2; q->n_up = 2; q->precision = MG_FP64; q->inner_cycles = 1; q->smoother = MG_SMOOTH_RBGS;
        q->coarse_mode = MG_COARSE_EXACT;
    }
    if (q->inner_cycles < 1) q->inner_cycles = 1;
    if (q->coarse_max_it <= 0) q->coarse_max_it = 1000;
    if (!(q->coarse_abs_tol > 0)) q->coarse_abs_tol = 1e-8;
    if (!(q->coarse_rel_tol > 0)) q->coarse_rel_tol = 1e-8;
}

// padded cells ((n_d + 2) per dimension) of the largest coarsest level
static int coarse_padded_cells(const mg_tree *t) {
    long long mx = 0;
    for (const TreeCoarse &tc : t->tcoarse) {
        const LevelHost &L = t->is_batch ? t->tl[tc.lvl] : t->lev[tc.lvl];
        long long c = 1;
        for (int d = 0; d < t->dim; d++) c *= L.ncell[d] + 2;
        mx = std::max(mx, c);
    }
    return (int)std::min<long long>(mx, 1 << 30);
}

// Parameters of one call: defaults, validation, the smoother and its Jacobi
// weight on the tree (read by the cycle driver), the Jacobi scratch of the
// precisions in use.  *key gets the graph-key suffix of these parameters.
static int use_params(mg_tree *t, const mg_params *p, mg_params *q, std::string *key) {
    params_or_default(p, q);
    if (q->smoother != MG_SMOOTH_RBGS && q->smoother != MG_SMOOTH_JACOBI) return fail(MG_ERR_ARG, "unknown smoother");
    double om = q->omega > 0 ? q->omega : (t->dim == 2 ? 0.8 : 6.0 / 7.0);
    if (q->smoother == MG_SMOOTH_JACOBI && !(om > 0 && om <= 1.0)) return fail(MG_ERR_ARG, "Jacobi weight must be in (0, 1]");
    q->omega = om;
    t->smoother = q->smoother;
    t->omega = om;
    if (q->coarse_mode != MG_COARSE_EXACT && q->coarse_mode != MG_COARSE_SMOOTH)
        return fail(MG_ERR_ARG, "unknown coarse_mode");
    if (q->coarse_mode == MG_COARSE_SMOOTH) {
        t->coarse_pad = coarse_padded_cells(t);
        if ((size_t)t->coarse_pad * sizeof(double) * (t->var_eps ? 3 : 2) > 200 * 1024)
            return fail(MG_ERR_UNSUPPORTED, "coarsest level too large for the smoothing coarse solve (one CTA)");
    }
    t->coarse_mode = q->coarse_mode;
    t->coarse_max_it = q->coarse_max_it;
    t->coarse_abs = q->coarse_abs_tol;
    t->coarse_rel = q->coarse_rel_tol;
    int rc;
    if (q->smoother == MG_SMOOTH_JACOBI) {
        if ((rc = dalloc(&t->d_jac64, t->ncells))) return rc;
        t->f64.J = t->adj.J = t->d_jac64;
        if (q->precision == MG_FP32_DC) {
            if ((rc = dalloc(&t->d_jac32, t->ncells))) return rc;
            t->f32.J = t->d_jac32;
        }
    }
    char buf[192];
    snprintf(buf, sizeof(buf), ":%d:%d:s%d:%a:c%d:%d:%a:%a", q->n_down, q->n_up, q->smoother,
             q->smoother == MG_SMOOTH_JACOBI ? om : 0.0, q->coarse_mode, q->coarse_max_it, q->coarse_abs_tol,
             q->coarse_rel_tol);
    if (key) *key = buf + t->sched_key;
    return MG_OK;
}

extern "C" int mg_vcycle(mg_tree *t, int n, const mg_params *p) {
    NEED_FINAL(t);
    mg_params q;
    std::string pk;
    int prc = use_params(t, p, &q, &pk);
    if (prc) return prc;
    const std::string key = "v64" + pk;
    for (int c = 0; c < n; c++) {
        int rc = run_graph(t, key, [&] { vcycle<double>(t, t->f64, (int)t->groups.size() - 1, q.n_down, q.n_up, 0); });
        if (rc) return rc;
    }
    return check_cuda("vcycle");
}

extern "C" int mg_fmg(mg_tree *t, const mg_params *p) {
    NEED_FINAL(t);
    mg_params q;
    std::string pk;
    int prc = use_params(t, p, &q, &pk);
    if (prc) return prc;
    const std::string key = "fmg64" + pk;
    int rc = run_graph(t, key, [&] { fmg<double>(t, t->f64, q.n_down, q.n_up, 0); });
    if (rc) return rc;
    return check_cuda("fmg");
}

extern "C" int mg_residual_norm(mg_tree *t, double *l2, double *linf, double *dev_r) {
    NEED_FINAL(t);
    if (!l2 || !linf) return fail(MG_ERR_ARG, "null output");
    double o[3];
    residual_norm(t, t->f64, 0, o, dev_r, nullptr);
    int rc = check_cuda("residual_norm");
    if (rc || (rc = check_status(t))) return rc;
    *l2 = std::sqrt(o[0] / o[1]);
    *linf = o[2];
    if (!std::isfinite(*l2) || !std::isfinite(*linf)) return fail(MG_ERR_NAN, "residual is not finite");
    return MG_OK;
}

static int ensure_f32(mg_tree *t) {
    int rc;
    const bool fresh = !t->f32.X;
    if (fresh) drop_graphs(t);
    if ((rc = alloc_fields(t, t->f32, t->var_eps))) return rc;
    if (t->var_eps) copy_eps_to_f32(t);
    if (fresh && !apply_tune_hint(t, 1)) {
        tune_sweeps<float>(t, t->f32);  // freshly zeroed fields: the sweeps leave them zero
        if ((rc = check_cuda("tune"))) return rc;
    }
    return MG_OK;
}

extern "C" int mg_solve(mg_tree *t, double rel_tol, int max_cycles, int fmg_first, const mg_params *p,
                        int *cycles_done, double *rel_out) {
    NEED_FINAL(t);
    mg_params q;
    std::string sfx;
    int rc;
    if ((rc = use_params(t, p, &q, &sfx))) return rc;
    const int top = (int)t->groups.size() - 1;
    double o[3];
    int cycles = 0;
    double rel = 1.0;
    if (t->singular && !t->is_batch) {
        // no Dirichlet face and lambda = 0: the weighted mean of the residual
        // does not change with phi, so its size bounds what cycles can reach
        if ((rc = dalloc(&t->d_r64, t->nleaf_cells))) return rc;
        residual_norm(t, t->f64, 0, o, t->d_r64, nullptr);
        const double l2 = std::sqrt(o[0] / o[1]), mean = std::fabs(leaf_mean(t, t->d_r64));
        if ((rc = check_cuda("compatibility")) != MG_OK) return rc;
        if (l2 > 0 && mean > rel_tol * l2)
            return fail(MG_ERR_INCOMPATIBLE_RHS,
                        "the residual's volume-weighted mean (" + std::to_string(mean / l2) +
                            " of its norm) cannot be removed on a problem without Dirichlet faces: "
                            "project f to a compatible right-hand side");
    }
    // each step is one graph: the cycle(s) and the FP64 composite residual,
    // whose norms arrive in pinned host memory; the host only waits
    if (q.precision == MG_FP64) {
        if ((rc = run_graph(t, "res64", [&] { residual_enqueue(t, t->f64, 0, nullptr, nullptr); }))) return rc;
        residual_wait(t, o);
        const double r0 = std::sqrt(o[0] / o[1]);
        rel = r0 > 0 ? 1.0 : 0.0;
        if (fmg_first && max_cycles > 0 && rel > 0) {
            rc = run_graph(t, "fmg64+res" + sfx, [&] {
                fmg<double>(t, t->f64, q.n_down, q.n_up, 0);
                residual_enqueue(t, t->f64, 0, nullptr, nullptr);
            });
            if (rc) return rc;
            residual_wait(t, o);
            cycles++;
            rel = std::sqrt(o[0] / o[1]) / r0;
        }
        while (rel > rel_tol && cycles < max_cycles) {
            rc = run_graph(t, "v64+res" + sfx, [&] {
                vcycle<double>(t, t->f64, top, q.n_down, q.n_up, 0);
                residual_enqueue(t, t->f64, 0, nullptr, nullptr);
            });
            if (rc) return rc;
            residual_wait(t, o);
            cycles++;
            rel = std::sqrt(o[0] / o[1]) / r0;
            if (!std::isfinite(rel)) break;
        }
    } else if (q.precision == MG_FP32_DC) {
        if ((rc = ensure_f32(t))) return rc;
        if ((rc = run_graph(t, "res64f32", [&] { residual_enqueue(t, t->f64, 0, nullptr, t->f32.F); }))) return rc;
        residual_wait(t, o);
        const double r0 = std::sqrt(o[0] / o[1]);
        rel = r0 > 0 ? 1.0 : 0.0;
        const std::string ki = sfx + ":" + std::to_string(q.inner_cycles);
        while (rel > rel_tol && cycles < max_cycles) {
            const bool first_fmg = fmg_first && cycles == 0;
            rc = run_graph(t, (first_fmg ? "dc-fmg" : "dc-v") + ki, [&] {
                cudaMemsetAsync(t->f32.X, 0, sizeof(float) * t->ncells, t->stream);
                cudaMemsetAsync(t->f32.XG, 0, sizeof(float) * t->nghost, t->stream);
                if (first_fmg) {
                    fmg<float>(t, t->f32, q.n_down, q.n_up, 1);
                    for (int c = 1; c < q.inner_cycles; c++) vcycle<float>(t, t->f32, top, q.n_down, q.n_up, 1);
                } else {
                    for (int c = 0; c < q.inner_cycles; c++) vcycle<float>(t, t->f32, top, q.n_down, q.n_up, 1);
                }
                residual_enqueue(t, t->f64, 0, nullptr, t->f32.F, false, t->f32.X);  // phi += e, refresh, residual
            });
            if (rc) return rc;
            residual_wait(t, o);
            cycles++;
            rel = std::sqrt(o[0] / o[1]) / r0;
            if (!std::isfinite(rel)) break;
        }
    } else {
        return fail(MG_ERR_ARG, "unknown precision");
    }
    if ((rc = check_cuda("solve")) || (rc = check_status(t))) return rc;
    if (t->singular && !t->is_batch && std::isfinite(rel)) {
        // no Dirichlet face: phi is fixed up to a constant; return the
        // solution with zero volume-weighted mean (covered cells and ghosts
        // shift with it)
        if ((rc = dalloc(&t->d_r64, t->nleaf_cells)) || (rc = leaf_copy(t, t->f64.X, (const double *)t->d_r64, false)))
            return rc;
        const double mean = leaf_mean(t, t->d_r64);
        sub_scalar(t, t->f64.X, mean, t->ncells);
        sub_scalar(t, t->f64.XG, mean, t->nghost);
        if ((rc = check_cuda("solve"))) return rc;
    }
    if (cycles_done) *cycles_done = cycles;
    if (rel_out) *rel_out = rel;
    if (!std::isfinite(rel)) return fail(MG_ERR_NAN, "residual is not finite");
    if (rel > rel_tol) return fail(MG_ERR_NOT_CONVERGED, "max_cycles reached");
    return MG_OK;
}

// The adjoint solve of mg_adjoint / mg_adjoint_solve (reading R16, see
// mg_adjoint.cu): lambda = A^-T g by defect correction with A's V-cycle on
// the volume-weighted form, then dL/deps through the transposed eps chain.
static bool has_refinement_faces(const mg_tree *t) {
    for (const BlockDesc &B : t->blocks)
        for (int f = 0; f < 2 * t->dim; f++)
            if (B.nbr[f] <= -2) return true;
    return false;
}

static int adjoint_setup(mg_tree *t, const mg_params *p, mg_params *q) {
    if (t->is_batch) return fail(MG_ERR_UNSUPPORTED, "the adjoint works on one tree, not a batch");
    // a singular problem's compatibility condition is sum V f = 0 only where
    // fluxes are conserved; with variable eps at refinement faces they are
    // not (Sec. 2.6 states the identity for constant eps)
    if (t->singular && t->var_eps && has_refinement_faces(t))
        return fail(MG_ERR_UNSUPPORTED, "adjoint of a problem without Dirichlet faces needs constant eps on a "
                                        "mesh with refinement faces");
    int rc;
    if ((rc = use_params(t, p, q, nullptr))) return rc;
    if (q->precision == MG_FP32_DC && (rc = ensure_f32(t))) return rc;
    if ((rc = alloc_fields(t, t->adj, false))) return rc;
    t->adj.E = t->f64.E;
    t->adj.W = t->f64.W;
    t->adj.EG = t->f64.EG;
    return adjoint_buffers(t);
}

static int adjoint_run(mg_tree *t, const double *g, double *dLdf, double *dLdeps, const mg_params *p, double rel_tol,
                       int max_cycles, int *cycles_done, double *rel_out) {
    NEED_FINAL(t);
    if (!g || !dLdf) return fail(MG_ERR_ARG, "null argument");
    if (max_cycles < 0) return fail(MG_ERR_ARG, "negative cycle count");
    mg_params q;
    int rc, it = 0;
    double rel = 0.0;
    if ((rc = adjoint_setup(t, p, &q))) return rc;
    if ((rc = adjoint_dc(t, g, dLdf, q.n_down, q.n_up, rel_tol, max_cycles, &it, &rel, q.precision == MG_FP32_DC)))
        return rc;
    if (dLdeps) eps_grad_transpose(t, dLdf, dLdeps);
    if ((rc = check_cuda("adjoint")) || (rc = check_status(t))) return rc;
    if (cycles_done) *cycles_done = it;
    if (rel_out) *rel_out = rel;
    if (!std::isfinite(rel)) return fail(MG_ERR_NAN, "adjoint residual is not finite");
    if (rel_tol > 0 && rel > rel_tol) return fail(MG_ERR_NOT_CONVERGED, "adjoint: max_cycles reached");
    return MG_OK;
}

extern "C" int mg_adjoint(mg_tree *t, const double *g, double *dLdf, double *dLdeps, const mg_params *p,
                          int n_cycles) {
    return adjoint_run(t, g, dLdf, dLdeps, p, 0.0, n_cycles, nullptr, nullptr);
}

extern "C" int mg_adjoint_solve(mg_tree *t, const double *g, double *dLdf, double *dLdeps, const mg_params *p,
                                double rel_tol, int max_cycles, int *cycles_done, double *rel_out) {
    if (!(rel_tol > 0)) return fail(MG_ERR_ARG, "rel_tol must be positive");
    return adjoint_run(t, g, dLdf, dLdeps, p, rel_tol, max_cycles, cycles_done, rel_out);
}

extern "C" int mg_apply_transpose(mg_tree *t, const double *y, double *out) {
    NEED_FINAL(t);
    if (!y || !out) return fail(MG_ERR_ARG, "null argument");
    if (t->is_batch) return fail(MG_ERR_UNSUPPORTED, "the transpose works on one tree, not a batch");
    int rc;
    if ((rc = adjoint_buffers(t))) return rc;
    apply_transpose(t, y, out);
    return check_cuda("apply_transpose");
}

extern "C" int mg_clean_adjoint(mg_tree *t, const double *gBnew, double *gB, const mg_params *p, double rel_tol,
                                int max_cycles, int *cycles_done, double *rel_out) {
    NEED_FINAL(t);
    if (!gBnew || !gB || gBnew == gB) return fail(MG_ERR_ARG, "null or aliased argument");
    if (t->geom != MG_CART) return fail(MG_ERR_UNSUPPORTED, "divergence cleaning: Cartesian meshes only");
    if (!(rel_tol > 0) || max_cycles < 0) return fail(MG_ERR_ARG, "rel_tol must be positive, max_cycles >= 0");
    mg_params q;
    int rc, it = 0;
    double rel = 0.0;
    if ((rc = adjoint_setup(t, p, &q))) return rc;
    if ((rc = clean_adjoint(t, gBnew, gB, q.n_down, q.n_up, rel_tol, max_cycles, &it, &rel,
                            q.precision == MG_FP32_DC)))
        return rc;
    if ((rc = check_status(t))) return rc;
    if (cycles_done) *cycles_done = it;
    if (rel_out) *rel_out = rel;
    if (!std::isfinite(rel)) return fail(MG_ERR_NAN, "adjoint residual is not finite");
    if (rel > rel_tol) return fail(MG_ERR_NOT_CONVERGED, "clean adjoint: max_cycles reached");
    return MG_OK;
}

extern "C" int mg_set_schedule(mg_tree *t, int n, const int *down, const int *up) {
    if (!t) return fail(MG_ERR_ARG, "null tree");
    if (n < 0 || (n > 0 && (!down || !up))) return fail(MG_ERR_ARG, "bad schedule arguments");
    if (!t->built) {
        int rc;
        if ((rc = build(t))) return rc;
    }
    if (n > (int)t->lev.size()) return fail(MG_ERR_ARG, "schedule longer than the level count");
    for (int l = 0; l < n; l++)
        if (down[l] < -1 || up[l] < -1 || down[l] > 16 || up[l] > 16)
            return fail(MG_ERR_ARG, "smoothing steps per level must lie in [-1, 16]");
    t->sched_down.assign(down, down + n);
    t->sched_up.assign(up, up + n);
    t->sched_key.clear();
    if (n) {
        t->sched_key = ":S";
        for (int l = 0; l < n; l++) t->sched_key += std::to_string(down[l]) + "," + std::to_string(up[l]) + ";";
    }
    return MG_OK;
}

extern "C" int mg_get_schedule(mg_tree *t, int n, int *down, int *up) {
    if (!t || n < 0 || (n > 0 && (!down || !up))) return fail(MG_ERR_ARG, "bad schedule arguments");
    for (int l = 0; l < n; l++) {
        down[l] = l < (int)t->sched_down.size() ? t->sched_down[l] : -1;
        up[l] = l < (int)t->sched_up.size() ? t->sched_up[l] : -1;
    }
    return MG_OK;
}

// Schedule autotuner: time full solves of the current problem (one tree,
// or the pool of a batch through its own solve) for a set of candidate
// schedules and keep the fastest that converges.  Levels (segments) from
// the lowest one holding leaves upwards take the candidate's leaf sweeps,
// those below its coarse sweeps.
using SolveFn = std::function<int(const mg_params *, int *, double *)>;
static int tune_schedule_impl(mg_tree *t, double rel_tol, int max_cycles, int precision, int *inner_out,
                              double *ms_out, const SolveFn &solve) {
    if (!(rel_tol > 0) || max_cycles < 1) return fail(MG_ERR_ARG, "rel_tol > 0 and max_cycles >= 1 required");
    if (precision != MG_FP64 && precision != MG_FP32_DC) return fail(MG_ERR_ARG, "unknown precision");
    const int nl = (int)t->lev.size();
    int lmin = nl;  // lowest level with leaves: the "leaf" levels are lmin..nl-1
    for (int l = 0; l < nl; l++)
        if (t->lev[l].nb > t->lev[l].nref) { lmin = l; break; }
    struct Cand { int dl, ul, dc, uc, inner; };
    std::vector<Cand> cands = {{2, 2, 2, 2, 1}, {1, 1, 1, 1, 1}, {1, 2, 1, 2, 1}, {2, 1, 2, 1, 1}, {3, 3, 3, 3, 1},
                               {1, 1, 2, 2, 1}, {2, 2, 1, 1, 1}, {1, 1, 3, 3, 1}, {1, 2, 2, 2, 1}};
    if (precision == MG_FP32_DC)  // more FP32 cycles per FP64 residual and update
        for (const Cand &c : {Cand{2, 2, 2, 2, 2}, Cand{1, 2, 1, 2, 2}, Cand{2, 1, 2, 1, 2}, Cand{1, 1, 1, 1, 2},
                              Cand{2, 2, 2, 2, 3}, Cand{2, 2, 2, 2, 4}})
            cands.push_back(c);
    // save phi (cells and ghosts) to restore it afterwards
    double *save = nullptr;
    CK(cudaMalloc((void **)&save, sizeof(double) * (size_t)(t->ncells + t->nghost)));
    CK(cudaMemcpyAsync(save, t->f64.X, sizeof(double) * t->ncells, cudaMemcpyDeviceToDevice, t->stream));
    CK(cudaMemcpyAsync(save + t->ncells, t->f64.XG, sizeof(double) * t->nghost, cudaMemcpyDeviceToDevice, t->stream));
    const std::vector<int> old_down = t->sched_down, old_up = t->sched_up;
    const std::string old_key = t->sched_key;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    int best_i = -1, rc = MG_OK;
    std::string report;  // every candidate's outcome, for the error message
    for (size_t i = 0; i < cands.size() && rc == MG_OK; i++) {
        const Cand &c = cands[i];
        std::vector<int> d(nl), u(nl);
        for (int l = 0; l < nl; l++) {
            d[l] = l >= lmin ? c.dl : c.dc;
            u[l] = l >= lmin ? c.ul : c.uc;
        }
        mg_set_schedule(t, nl, d.data(), u.data());
        mg_params q{2, 2, precision, c.inner, MG_SMOOTH_RBGS, 0.0, MG_COARSE_EXACT, 0, 0.0, 0.0};
        float fastest = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; rep++) {  // the first run captures the graphs
            cudaMemsetAsync(t->f64.X, 0, sizeof(double) * t->ncells, t->stream);
            refresh<double>(t, t->f64, 0);
            cudaEventRecord(e0, t->stream);
            int cyc = 0;
            double rel = 0;
            const int r = solve(&q, &cyc, &rel);
            cudaEventRecord(e1, t->stream);
            cudaEventSynchronize(e1);
            if (r == MG_ERR_NOT_CONVERGED || r == MG_ERR_NAN) ok = false;
            else if (r != MG_OK) rc = r;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep) fastest = std::min(fastest, ms);
            if (rep == 0 || r != MG_OK) {
                char buf[128];
                snprintf(buf, sizeof buf, " [%d,%d|%d,%d x%d: rc %d, %d cycles, rel %.2e]", c.dl, c.ul, c.dc, c.uc,
                         c.inner, r, cyc, rel);
                report += buf;
            }
        }
        if (ok && rc == MG_OK && fastest < best) { best = fastest; best_i = (int)i; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaMemcpyAsync(t->f64.X, save, sizeof(double) * t->ncells, cudaMemcpyDeviceToDevice, t->stream));
    CK(cudaMemcpyAsync(t->f64.XG, save + t->ncells, sizeof(double) * t->nghost, cudaMemcpyDeviceToDevice, t->stream));
    CK(cudaStreamSynchronize(t->stream));
    cudaFree(save);
    if (rc != MG_OK || best_i < 0) {
        t->sched_down = old_down;
        t->sched_up = old_up;
        t->sched_key = old_key;
        return rc != MG_OK ? rc : fail(MG_ERR_NOT_CONVERGED, "no candidate schedule reached rel_tol:" + report);
    }
    const Cand &c = cands[best_i];
    std::vector<int> d(nl), u(nl);
    for (int l = 0; l < nl; l++) {
        d[l] = l >= lmin ? c.dl : c.dc;
        u[l] = l >= lmin ? c.ul : c.uc;
    }
    mg_set_schedule(t, nl, d.data(), u.data());
    if (inner_out) *inner_out = c.inner;
    if (ms_out) *ms_out = best;
    return MG_OK;
}

extern "C" int mg_tune_schedule(mg_tree *t, double rel_tol, int max_cycles, int precision, int *inner_out,
                                double *ms_out) {
    NEED_FINAL(t);
    if (t->is_batch) return fail(MG_ERR_ARG, "a batch pool: use mg_batch_tune_schedule");
    return tune_schedule_impl(t, rel_tol, max_cycles, precision, inner_out, ms_out,
                              [&](const mg_params *q, int *cyc, double *rel) {
                                  return mg_solve(t, rel_tol, max_cycles, 1, q, cyc, rel);
                              });
}

extern "C" int mg_set_wait_limit(mg_tree *t, int64_t polls) {
    if (!t) return fail(MG_ERR_ARG, "null tree");
    if (polls > 0xFFFFFFFFll) return fail(MG_ERR_ARG, "wait limit above 2^32 - 1");
    t->wait_limit = polls < 0 ? kDefaultWaitLimit : (uint32_t)polls;
    drop_graphs(t);  // captured launches carry the old limit
    return MG_OK;
}

extern "C" int mg_set_tail(mg_tree *t, int64_t max_cells) {
    if (!t) return fail(MG_ERR_ARG, "null tree");
    t->tail_cells = max_cells < 0 ? 0 : max_cells;
    drop_graphs(t);  // captured cycles hold the previous split
    return MG_OK;
}

extern "C" int mg_launch_count(mg_tree *t, int64_t *n) {
    if (!t || !n) return fail(MG_ERR_ARG, "null argument");
    *n = t->launches;
    return MG_OK;
}

extern "C" int mg_sweep_variant(mg_tree *t, int precision, int level, int *variant) {
    NEED_FINAL(t);
    if (!variant || level < 0 || level >= (int)t->lev.size() || (precision != MG_FP64 && precision != MG_FP32_DC))
        return fail(MG_ERR_ARG, "bad arguments");
    *variant = sweep_variant(t, precision == MG_FP32_DC ? 1 : 0, level);
    return MG_OK;
}

static int ensure_f32(mg_tree *t);

extern "C" int mg_set_sweep_variant(mg_tree *t, int precision, int level, int variant) {
    NEED_FINAL(t);
    if ((precision != MG_FP64 && precision != MG_FP32_DC) || level < -1 || level >= (int)t->lev.size() ||
        variant < -1 || variant >= kNumSweepVariants)
        return fail(MG_ERR_ARG, "bad arguments");
    int rc;
    if (precision == MG_FP32_DC && (rc = ensure_f32(t))) return rc;
    const int prec = precision == MG_FP32_DC ? 1 : 0;
    std::vector<int> &ch = t->sweep_choice[prec];
    if (ch.size() != t->lev.size()) ch.assign(t->lev.size(), -1);
    if (level >= 0 && variant >= 0 && !sweep_variant_ok(t, prec, level, variant))
        return fail(MG_ERR_ARG, "sweep variant does not apply to this level");
    for (int l = 0; l < (int)t->lev.size(); l++) {
        if (level >= 0 && l != level) continue;
        if (variant < 0) ch[l] = -1;
        else if (sweep_variant_ok(t, prec, l, variant)) ch[l] = variant;
    }
    drop_graphs(t);  // captured cycles hold the previous choice
    return MG_OK;
}

extern "C" int mg_time_sweeps(mg_tree *t, int level, int n_sweeps, int precision, double out[4]) {
    NEED_FINAL(t);
    if (!out || n_sweeps < 1 || level < 0 || level >= (int)t->lev.size() ||
        (precision != MG_FP64 && precision != MG_FP32_DC))
        return fail(MG_ERR_ARG, "bad arguments");
    int rc;
    if (precision == MG_FP32_DC && (rc = ensure_f32(t))) return rc;
    rc = time_sweeps(t, level, n_sweeps, precision, out);
    if (rc) return rc;
    return check_cuda("time_sweeps");
}

extern "C" int mg_divergence_order(mg_tree *t, const double *B, double *divB, int order) {
    NEED_FINAL(t);
    if (!B || !divB) return fail(MG_ERR_ARG, "null argument");
    if (order != 2 && order != 4) return fail(MG_ERR_ARG, "divergence order must be 2 or 4");
    if (t->geom != MG_CART) return fail(MG_ERR_UNSUPPORTED, "divergence: Cartesian meshes only");
    int rc;
    if ((rc = alloc_fields(t, t->adj, false))) return rc;
    divergence(t, B, divB, order);
    return check_cuda("divergence");
}

extern "C" int mg_divergence(mg_tree *t, const double *B, double *divB) { return mg_divergence_order(t, B, divB, 2); }

extern "C" int mg_project(mg_tree *t, const double *B, double *Bnew) {
    NEED_FINAL(t);
    if (!B || !Bnew) return fail(MG_ERR_ARG, "null argument");
    if (t->geom != MG_CART) return fail(MG_ERR_UNSUPPORTED, "projection: Cartesian meshes only");
    project(t, B, Bnew);
    return check_cuda("project");
}


// One divergence-cleaning step (Sec. 4.1) on the device: f = div B (order 2
// or 4); on a problem without Dirichlet faces f loses its volume-weighted
// mean; phi = 0; solve Lap phi = f; Bnew = B - grad phi.
extern "C" int mg_clean(mg_tree *t, const double *B, double *Bnew, double *divB, int order, double rel_tol,
                        int max_cycles, const mg_params *p, int *cycles_done, double *rel_out) {
    NEED_FINAL(t);
    if (!B || !Bnew) return fail(MG_ERR_ARG, "null argument");
    int rc;
    if ((rc = dalloc(&t->d_r64, t->nleaf_cells))) return rc;
    if ((rc = mg_divergence_order(t, B, t->d_r64, order))) return rc;
    if (t->singular) sub_scalar(t, t->d_r64, leaf_mean(t, t->d_r64), t->nleaf_cells);
    if (divB) CK(cudaMemcpyAsync(divB, t->d_r64, sizeof(double) * t->nleaf_cells, cudaMemcpyDeviceToDevice, t->stream));
    if ((rc = leaf_copy(t, t->f64.F, (const double *)t->d_r64, true))) return rc;
    CK(cudaMemsetAsync(t->f64.X, 0, sizeof(double) * t->ncells, t->stream));
    refresh<double>(t, t->f64, 0);
    rc = mg_solve(t, rel_tol, max_cycles, 1, p, cycles_done, rel_out);
    if (rc != MG_OK && rc != MG_ERR_NOT_CONVERGED) return rc;
    const int rp = mg_project(t, B, Bnew);
    return rp ? rp : rc;
}

extern "C" int mg_tree_destroy(mg_tree *t) {
    if (!t) return MG_OK;
    if (t->d_blocks_built) cudaFree(t->d_blocks_built);
    if (t->finalized) {
        cudaStreamSynchronize(t->stream);
        free_fields(t->f64, true);
        free_fields(t->adj, false);
        free_fields(t->f32, true);
        cudaFree(t->d_blocks); cudaFree(t->d_levels); cudaFree(t->d_bcplanes);
        cudaFree(t->d_r64); cudaFree(t->d_wface); cudaFree(t->d_jac64); cudaFree(t->d_jac32); cudaFree(t->d_minv); cudaFree(t->d_cvec); cudaFree(t->d_partials); cudaFree(t->d_red); cudaFree(t->d_status); cudaFree(t->d_tcoarse); cudaFree(t->d_coarse_chunks);
        cudaFree(t->d_bt); cudaFree(t->d_bt32); cudaFree(t->d_btperm); cudaFree(t->d_btlist); cudaFree(t->d_bt_chunks);
        cudaFreeHost(t->h_red);
        cudaFree(t->d_runs); cudaFree(t->d_slot_off); cudaFree(t->d_slots); cudaFree(t->d_tree3);
        cudaFree(t->d_at); cudaFree(t->d_atg); cudaFree(t->d_lam); cudaFree(t->d_gh); cudaFree(t->d_lv);
        cudaFreeHost(t->h_tree3);
        drop_graphs(t);
        if (t->cap_stream) cudaStreamDestroy(t->cap_stream);
    }
    delete t;
    return MG_OK;
}

// ------------------------------------------------------------- batch ----
// A batch merges many independent trees into one pool so that every cycle
// step is one launch over the blocks of all trees.  Levels are aligned from
// the top: level l of a tree with L levels joins group G - L + l (G the
// largest level count), so the finest levels of all trees form the top
// group and each tree still sees its own V-cycle (Sec. 2.4) in its own
// order.  A group is split into segments, one per (block size, coarsest,
// parent block size); a segment holds the covered blocks of its trees
// first, then the leaves, tree by tree, Morton order within a tree.  A
// tree's coarsest level stays contiguous for its exact solve; the level
// descriptors are kept per (tree, level), since trees differ in spacing.

struct mg_batch {
    mg_tree *pool = nullptr;
    int ntrees = 0;
};

static int merge_trees(mg_tree *P, int n, mg_tree *const *trees) {
    const int D = trees[0]->dim;
    int G = 0;
    for (int i = 0; i < n; i++) G = std::max(G, (int)trees[i]->lev.size());
    struct Key {
        int group, coarsest, n, psn, solo;
        bool operator<(const Key &o) const {
            return std::tie(group, coarsest, n, psn, solo) < std::tie(o.group, o.coarsest, o.n, o.psn, o.solo);
        }
    };
    std::map<Key, std::vector<std::pair<int, int>>> segs;  // members (tree, level) in tree order
    std::vector<int> tl_off(n + 1, 0);
    for (int i = 0; i < n; i++) {
        const mg_tree *T = trees[i];
        const int nl = (int)T->lev.size();
        for (int l = 0; l < nl; l++) {
            const LevelHost &L = T->lev[l];
            // a coarsest level holding leaves gets a segment of its own, so
            // that both its covered prefix and its contiguity hold
            const int solo = (l == 0 && L.nref < L.nb) ? i : -1;
            segs[Key{G - nl + l, l == 0, L.n, L.parent_same_n, solo}].push_back({i, l});
        }
        tl_off[i + 1] = tl_off[i] + nl;
    }
    P->tl.clear();
    for (int i = 0; i < n; i++)
        for (const LevelHost &L : trees[i]->lev) P->tl.push_back(L);
    for (int i = 0; i < n; i++)
        for (int l = 0; l < (int)trees[i]->lev.size(); l++) P->tl[tl_off[i] + l].group = G - (int)trees[i]->lev.size() + l;
    // block ids and storage
    std::vector<std::vector<int>> nid(n);
    std::vector<int> btree;  // pool block -> tree
    for (int i = 0; i < n; i++) nid[i].assign(trees[i]->blocks.size(), -1);
    P->lev.clear();
    P->groups.assign(G, {});
    P->blocks.clear();
    long long co = 0, go = 0;
    int g = 0;
    for (auto &kv : segs) {
        const Key &k = kv.first;
        LevelHost S;
        S.n = k.n;
        S.group = k.group;
        S.coarsest = k.coarsest;
        S.parent_same_n = k.psn;
        S.first = g;
        co = (co + 31) / 32 * 32;
        go = (go + 31) / 32 * 32;
        S.cell_first = co;
        S.ghost_first = go;
        const long long C = ipow(k.n, D), F = 2LL * D * (D == 2 ? k.n : (long long)k.n * k.n);
        for (int part = 0; part < 2; part++)  // covered blocks, then leaves
            for (auto &m : kv.second) {
                const mg_tree *T = trees[m.first];
                const LevelHost &L = T->lev[m.second];
                const int r0 = part == 0 ? 0 : L.nref, r1 = part == 0 ? L.nref : L.nb;
                for (int r = r0; r < r1; r++) {
                    BlockDesc B = T->blocks[L.first + r];
                    const int id = (int)P->blocks.size();
                    nid[m.first][L.first + r] = id;
                    B.cell_off = co + (long long)(id - S.first) * C;
                    B.ghost_off = go + (long long)(id - S.first) * F;
                    B.lev = tl_off[m.first] + m.second;
                    P->blocks.push_back(B);
                    btree.push_back(m.first);
                }
                if (part == 0) S.nref += L.nref;
            }
        S.nb = (int)P->blocks.size() - S.first;
        S.ncells = S.nb * C;
        S.nghost = S.nb * F;
        co += S.ncells;
        go += S.nghost;
        g += S.nb;
        P->groups[k.group].push_back((int)P->lev.size());
        P->lev.push_back(S);
    }
    P->ncells = co;
    P->nghost = go;
    // links: parents, neighbours and ghost push slots in pool ids
    for (size_t b = 0; b < P->blocks.size(); b++) {
        BlockDesc &B = P->blocks[b];
        const std::vector<int> &m = nid[btree[b]];
        if (B.parent >= 0) B.parent = m[B.parent];
        for (int f = 0; f < 6; f++) {
            if (B.nbr[f] >= 0) B.nbr[f] = m[B.nbr[f]];
            else if (B.nbr[f] <= -2) B.nbr[f] = -2 - m[-2 - B.nbr[f]];
        }
    }
    for (auto &B : P->blocks)
        for (int f = 0; f < 6; f++) {
            B.push[f] = -1;
            if (B.nbr[f] >= 0) {
                const long long Fd = D == 2 ? B.n : (long long)B.n * B.n;
                B.push[f] = P->blocks[B.nbr[f]].ghost_off + (f ^ 1) * Fd;
            }
        }
    // coarsest level of every tree
    P->tcoarse.clear();
    P->minv_total = P->cvec_total = P->bt_total = P->bt_total32 = P->btperm_total = 0;
    P->max_nc = 0;
    for (int i = 0; i < n; i++) {
        const mg_tree *T = trees[i];
        const LevelHost &L0 = T->lev[0];
        TreeCoarse tc{};
        tc.first = nid[i][L0.first];
        for (int r = 0; r < L0.nb; r++)
            if (nid[i][L0.first + r] != tc.first + r) return fail(MG_ERR_ARG, "internal: coarsest level not contiguous");
        tc.nb = L0.nb;
        tc.n = L0.n;
        tc.nc = (int)(L0.nb * ipow(L0.n, D));
        tc.singular = T->singular ? 1 : 0;
        tc.ns = tc.nc + tc.singular;
        tc.group = G - (int)T->lev.size();
        tc.lvl = tl_off[i];
        tc.cell0 = P->blocks[tc.first].cell_off;
        tc.cvec_off = P->cvec_total;
        P->cvec_total += tc.ns;
        coarse_plan(T, tc, L0, n > 1);
        if (tc.bt_n) {
            tc.bt_off = P->bt_total;
            tc.bt_off32 = P->bt_total32;
            tc.perm_off = P->btperm_total;
            P->bt_total += (long long)tc.bt_n * bt_stride(tc.bt_P);
            P->bt_total32 += (long long)tc.bt_n * bt32_stride(tc.bt_P);
            P->btperm_total += tc.nc;
        } else {
            tc.minv_off = P->minv_total;
            P->minv_total += (long long)tc.ns * tc.ns;
        }
        P->max_nc = std::max(P->max_nc, tc.nc);
        P->tcoarse.push_back(tc);
    }
    // leaf runs: tree i's leaf order is its levels in order, leaf blocks in
    // order; in the pool each (tree, level) leaf range is one contiguous run
    P->run_cell.clear(); P->run_leaf.clear(); P->run_len.clear();
    P->tree_leaf_off.assign(n + 1, 0);
    long long leaf = 0;
    for (int i = 0; i < n; i++) {
        const mg_tree *T = trees[i];
        P->tree_leaf_off[i] = leaf;
        for (const LevelHost &L : T->lev) {
            const int nleaf = L.nb - L.nref;
            if (nleaf <= 0) continue;
            const int b0 = nid[i][L.first + L.nref];
            for (int r = 1; r < nleaf; r++)
                if (nid[i][L.first + L.nref + r] != b0 + r) return fail(MG_ERR_ARG, "internal: leaf run not contiguous");
            const long long len = nleaf * ipow(L.n, D);
            P->run_cell.push_back(P->blocks[b0].cell_off);
            P->run_leaf.push_back(leaf);
            P->run_len.push_back(len);
            leaf += len;
        }
    }
    P->tree_leaf_off[n] = leaf;
    P->nleaf_cells = leaf;
    P->singular = trees[0]->singular;
    P->nc = P->max_nc;
    P->ns = P->max_nc + (P->singular ? 1 : 0);
    return MG_OK;
}

static int batch_device_tables(mg_tree *P, int n) {
    // run chunks of at most 8192 values, one CTA each
    std::vector<long long> runs;
    for (size_t r = 0; r < P->run_len.size(); r++)
        for (long long o = 0; o < P->run_len[r]; o += 8192) {
            runs.push_back(P->run_cell[r] + o);
            runs.push_back(P->run_leaf[r] + o);
            runs.push_back(std::min<long long>(8192, P->run_len[r] - o));
        }
    P->n_runs = (int)(runs.size() / 3);
    CK(cudaMalloc((void **)&P->d_runs, sizeof(long long) * std::max<size_t>(3, runs.size())));
    if (!runs.empty()) CK(cudaMemcpy(P->d_runs, runs.data(), sizeof(long long) * runs.size(), cudaMemcpyHostToDevice));
    // residual slots: one per leaf block, in the order the residual pass
    // visits them (segments in order, leaf blocks in order), listed per tree
    std::vector<std::vector<int>> per(n);
    std::vector<int> tree_of(P->blocks.size(), 0);
    {
        // the tree of a block is the tree of its level descriptor
        std::vector<int> tl_tree(P->tl.size(), 0);
        for (int i = 0; i < n; i++) {
            const int lo_ = P->tcoarse[i].lvl, hi_ = i + 1 < n ? P->tcoarse[i + 1].lvl : (int)P->tl.size();
            for (int l = lo_; l < hi_; l++) tl_tree[l] = i;
        }
        for (size_t b = 0; b < P->blocks.size(); b++) tree_of[b] = tl_tree[P->blocks[b].lev];
    }
    int slot = 0;
    for (const LevelHost &L : P->lev)
        for (int r = L.nref; r < L.nb; r++) per[tree_of[L.first + r]].push_back(slot++);
    std::vector<int> off(n + 1, 0), slots;
    for (int i = 0; i < n; i++) {
        off[i + 1] = off[i] + (int)per[i].size();
        slots.insert(slots.end(), per[i].begin(), per[i].end());
    }
    CK(cudaMalloc((void **)&P->d_slot_off, sizeof(int) * (n + 1)));
    CK(cudaMemcpy(P->d_slot_off, off.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
    CK(cudaMalloc((void **)&P->d_slots, sizeof(int) * std::max<size_t>(1, slots.size())));
    if (!slots.empty()) CK(cudaMemcpy(P->d_slots, slots.data(), sizeof(int) * slots.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc((void **)&P->d_tree3, sizeof(double) * 3 * n));
    CK(cudaMallocHost((void **)&P->h_tree3, sizeof(double) * 3 * n));
    return MG_OK;
}

extern "C" int mg_batch_create(int n, mg_tree *const *trees, void *stream, mg_batch **out) {
    if (!out || !trees || n < 1) return fail(MG_ERR_ARG, "need at least one tree");
    *out = nullptr;
    for (int i = 0; i < n; i++) {
        if (!trees[i]) return fail(MG_ERR_ARG, "null tree");
        int rc = build(trees[i]);
        if (rc) return rc;
    }
    const mg_tree *A = trees[0];
    for (int i = 1; i < n; i++) {
        const mg_tree *T = trees[i];
        bool same = T->dim == A->dim && T->geom == A->geom && T->helm == A->helm;
        for (int f = 0; f < 6; f++)
            same = same && T->bc.type[f] == A->bc.type[f] && T->bc.value[f] == A->bc.value[f];
        for (int d = 0; d < 3; d++) same = same && T->lo[d] == A->lo[d];
        if (!same) return fail(MG_ERR_ARG, "batch trees differ in dimension, geometry, boundary conditions, lambda or lo");
    }
    mg_tree *P = new mg_tree();
    P->dim = A->dim; P->N = A->N; P->geom = A->geom; P->bc = A->bc; P->helm = A->helm;
    for (int d = 0; d < 3; d++) { P->lo[d] = A->lo[d]; P->hi[d] = A->hi[d]; }
    P->is_batch = true;
    int rc = merge_trees(P, n, trees);
    if (rc) { delete P; return rc; }
    P->built = true;
    if ((rc = mg_tree_finalize(P, stream)) || (rc = batch_device_tables(P, n))) {
        mg_tree_destroy(P);
        return rc;
    }
    mg_batch *b = new mg_batch();
    b->pool = P;
    b->ntrees = n;
    *out = b;
    return MG_OK;
}

#define NEED_BATCH(b)                                                     \
    do {                                                                  \
        if (!(b) || !(b)->pool) return fail(MG_ERR_ARG, "null batch");    \
    } while (0)

extern "C" int mg_batch_leaf_offsets(mg_batch *b, int64_t *off) {
    NEED_BATCH(b);
    if (!off) return fail(MG_ERR_ARG, "null output");
    for (int i = 0; i <= b->ntrees; i++) off[i] = b->pool->tree_leaf_off[i];
    return MG_OK;
}

extern "C" int mg_batch_set_rhs(mg_batch *b, const double *f) { NEED_BATCH(b); return mg_set_rhs(b->pool, f); }
extern "C" int mg_batch_set_phi(mg_batch *b, const double *x) { NEED_BATCH(b); return mg_set_phi(b->pool, x); }
extern "C" int mg_batch_get_phi(mg_batch *b, double *x) { NEED_BATCH(b); return mg_get_phi(b->pool, x); }
extern "C" int mg_batch_set_eps(mg_batch *b, const double *e) { NEED_BATCH(b); return mg_set_eps(b->pool, e); }
extern "C" int mg_batch_vcycle(mg_batch *b, int n, const mg_params *p) { NEED_BATCH(b); return mg_vcycle(b->pool, n, p); }
extern "C" int mg_batch_fmg(mg_batch *b, const mg_params *p) { NEED_BATCH(b); return mg_fmg(b->pool, p); }

static int batch_norms_wait(mg_tree *P, int n, double *l2, double *linf) {
    CK(cudaStreamSynchronize(P->stream));
    for (int i = 0; i < n; i++) {
        const double *o = P->h_tree3 + 3 * i;
        l2[i] = o[1] > 0 ? std::sqrt(o[0] / o[1]) : 0.0;
        if (linf) linf[i] = o[2];
    }
    return MG_OK;
}

extern "C" int mg_batch_residual_norms(mg_batch *b, double *l2, double *linf) {
    NEED_BATCH(b);
    if (!l2 || !linf) return fail(MG_ERR_ARG, "null output");
    mg_tree *P = b->pool;
    residual_enqueue_trees(P, P->f64, nullptr, true);
    int rc = check_cuda("batch residual");
    if (rc || (rc = batch_norms_wait(P, b->ntrees, l2, linf)) || (rc = check_status(P))) return rc;
    for (int i = 0; i < b->ntrees; i++)
        if (!std::isfinite(l2[i]) || !std::isfinite(linf[i])) return fail(MG_ERR_NAN, "residual is not finite");
    return MG_OK;
}

// Cycles until every tree's composite residual is below rel_tol times its
// initial one (all trees cycle together; a converged tree keeps cycling).
extern "C" int mg_batch_solve(mg_batch *b, double rel_tol, int max_cycles, int fmg_first, const mg_params *p,
                              int *cycles_done, double *rel_out) {
    NEED_BATCH(b);
    mg_tree *t = b->pool;
    const int n = b->ntrees;
    mg_params q;
    std::string sfx;
    int rc;
    if ((rc = use_params(t, p, &q, &sfx))) return rc;
    const int top = (int)t->groups.size() - 1;
    std::vector<double> r0(n), l2(n), rel(n, 1.0);
    int cycles = 0;
    auto update = [&](bool first) -> double {
        batch_norms_wait(t, n, l2.data(), nullptr);
        double worst = 0;
        for (int i = 0; i < n; i++) {
            if (first) { r0[i] = l2[i]; rel[i] = r0[i] > 0 ? 1.0 : 0.0; }
            else rel[i] = r0[i] > 0 ? l2[i] / r0[i] : 0.0;
            worst = std::isfinite(rel[i]) ? std::max(worst, rel[i]) : rel[i];
        }
        return worst;
    };
    double worst;
    if (q.precision == MG_FP64) {
        if ((rc = run_graph(t, "b-res64", [&] { residual_enqueue_trees(t, t->f64, nullptr, false); }))) return rc;
        worst = update(true);
        if (fmg_first && max_cycles > 0 && worst > 0) {
            rc = run_graph(t, "b-fmg64+res" + sfx, [&] {
                fmg<double>(t, t->f64, q.n_down, q.n_up, 0);
                residual_enqueue_trees(t, t->f64, nullptr, false);
            });
            if (rc) return rc;
            cycles++;
            worst = update(false);
        }
        while (worst > rel_tol && cycles < max_cycles) {
            rc = run_graph(t, "b-v64+res" + sfx, [&] {
                vcycle<double>(t, t->f64, top, q.n_down, q.n_up, 0);
                residual_enqueue_trees(t, t->f64, nullptr, false);
            });
            if (rc) return rc;
            cycles++;
            worst = update(false);
            if (!std::isfinite(worst)) break;
        }
    } else if (q.precision == MG_FP32_DC) {
        if ((rc = ensure_f32(t))) return rc;
        if ((rc = run_graph(t, "b-res64f32", [&] { residual_enqueue_trees(t, t->f64, t->f32.F, false); }))) return rc;
        worst = update(true);
        const std::string ki = sfx + ":" + std::to_string(q.inner_cycles);
        while (worst > rel_tol && cycles < max_cycles) {
            const bool first_fmg = fmg_first && cycles == 0;
            rc = run_graph(t, (first_fmg ? "b-dc-fmg" : "b-dc-v") + ki, [&] {
                cudaMemsetAsync(t->f32.X, 0, sizeof(float) * t->ncells, t->stream);
                cudaMemsetAsync(t->f32.XG, 0, sizeof(float) * t->nghost, t->stream);
                if (first_fmg) {
                    fmg<float>(t, t->f32, q.n_down, q.n_up, 1);
                    for (int c = 1; c < q.inner_cycles; c++) vcycle<float>(t, t->f32, top, q.n_down, q.n_up, 1);
                } else {
                    for (int c = 0; c < q.inner_cycles; c++) vcycle<float>(t, t->f32, top, q.n_down, q.n_up, 1);
                }
                residual_enqueue_trees(t, t->f64, t->f32.F, false, t->f32.X);  // phi += e, refresh, residual
            });
            if (rc) return rc;
            cycles++;
            worst = update(false);
            if (!std::isfinite(worst)) break;
        }
    } else {
        return fail(MG_ERR_ARG, "unknown precision");
    }
    if ((rc = check_cuda("batch solve")) || (rc = check_status(t))) return rc;
    if (cycles_done) *cycles_done = cycles;
    if (rel_out)
        for (int i = 0; i < n; i++) rel_out[i] = rel[i];
    if (!std::isfinite(worst)) return fail(MG_ERR_NAN, "residual is not finite");
    if (worst > rel_tol) return fail(MG_ERR_NOT_CONVERGED, "max_cycles reached");
    return MG_OK;
}

extern "C" int mg_batch_tune_schedule(mg_batch *b, double rel_tol, int max_cycles, int precision, int *inner_out,
                                      double *ms_out) {
    NEED_BATCH(b);
    std::vector<double> rel(b->ntrees);
    return tune_schedule_impl(b->pool, rel_tol, max_cycles, precision, inner_out, ms_out,
                              [&](const mg_params *q, int *cyc, double *worst) {
                                  const int r = mg_batch_solve(b, rel_tol, max_cycles, 1, q, cyc, rel.data());
                                  *worst = rel.empty() ? 0.0 : *std::max_element(rel.begin(), rel.end());
                                  return r;
                              });
}

extern "C" int mg_batch_launch_count(mg_batch *b, int64_t *n) {
    NEED_BATCH(b);
    return mg_launch_count(b->pool, n);
}

extern "C" int mg_batch_set_tail(mg_batch *b, int64_t max_cells) {
    NEED_BATCH(b);
    return mg_set_tail(b->pool, max_cells);
}

extern "C" int mg_batch_time_sweeps(mg_batch *b, int level, int n_sweeps, int precision, double out[4]) {
    NEED_BATCH(b);
    return mg_time_sweeps(b->pool, level, n_sweeps, precision, out);
}

extern "C" int mg_batch_coarse_info(mg_batch *b, int64_t out[4]) {
    NEED_BATCH(b);
    if (!out) return fail(MG_ERR_ARG, "null output");
    const mg_tree *P = b->pool;
    out[0] = (int64_t)P->tcoarse.size() - P->n_btri;
    out[1] = P->n_btri;
    out[2] = (int64_t)sizeof(double) * P->minv_total;
    out[3] = (int64_t)sizeof(double) * P->bt_total;
    return MG_OK;
}

extern "C" int mg_batch_num_segments(mg_batch *b, int *nseg, int *ngroups) {
    NEED_BATCH(b);
    if (!nseg || !ngroups) return fail(MG_ERR_ARG, "null output");
    *nseg = (int)b->pool->lev.size();
    *ngroups = (int)b->pool->groups.size();
    return MG_OK;
}

extern "C" int mg_batch_segment_info(mg_batch *b, int seg, int32_t info[6]) {
    NEED_BATCH(b);
    if (!info || seg < 0 || seg >= (int)b->pool->lev.size()) return fail(MG_ERR_ARG, "bad arguments");
    const LevelHost &L = b->pool->lev[seg];
    info[0] = L.n; info[1] = L.group; info[2] = L.nb; info[3] = L.nref; info[4] = L.coarsest; info[5] = L.parent_same_n;
    return MG_OK;
}

extern "C" int mg_batch_destroy(mg_batch *b) {
    if (!b) return MG_OK;
    mg_tree_destroy(b->pool);
    delete b;
    return MG_OK;
}
