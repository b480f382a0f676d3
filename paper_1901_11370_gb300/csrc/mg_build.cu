// mg_build.cu -- mesh construction on the device (Sec. 2.5, "creating the
// grid" and "adapting the grid"): the block tables of an octree/quadtree of
// fixed-size blocks from its refinement list.
//
// The result equals the host construction in mg_tree.cpp entry for entry:
// per level the blocks (coarse levels and the base grid whole; a refined
// level is the 2^D children of the refined blocks one level down), covered
// blocks first and Morton order within each group, then per block its cell
// and ghost offsets, parent, and face neighbours (same level with periodic
// wrap, physical, or the block one level coarser under 2:1 balance).
//
// Steps, all on one stream: full grids for the coarse levels and the base;
// children of the refine entries of each depth (duplicates dropped by an
// atomic flag per parent, sizes read back once per level); a dense
// coordinate map per level; "has children" flags through the parents;
// one radix sort per level on the 64-bit key (leaf flag, 63-bit Morton
// code); ranks and global ids; the descriptor of every block.  The block
// table stays on the device for the tree's finalize and is copied to the
// host for the host-side setup (segments, coarsest-level factors).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include <cub/device/device_radix_sort.cuh>

#include "mg_internal.h"

namespace mg {
namespace {

struct I3b {
    int x, y, z;
};

// device error codes, first one wins
enum { BE_OK = 0, BE_NO_BLOCK = 1, BE_INCOMPLETE = 2, BE_UNBALANCED = 3 };

__device__ __forceinline__ void set_err(int *err, int code) { atomicCAS(err, BE_OK, code); }

__device__ __forceinline__ long long gkey(const I3b q, int nx, int ny) {
    return ((long long)q.z * ny + q.y) * nx + q.x;
}

// every block of an nx x ny x nz grid, lexicographic; map[key] = index
__global__ void k_grid(I3b *coords, int *map, int nx, int ny, int nz) {
    const long long total = (long long)nx * ny * nz;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < total;
         b += (long long)gridDim.x * blockDim.x) {
        coords[b] = I3b{(int)(b % nx), (int)((b / nx) % ny), (int)(b / ((long long)nx * ny))};
        map[b] = (int)b;
    }
}

// children of the refine entries of one depth (entries: i, j, k per entry)
__global__ void k_children(const int *entries, int n_entries, int D, const int *pmap, int pnx, int pny, int pnz,
                           int *done, I3b *child, int *count, int *err) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_entries) return;
    const I3b q{entries[3 * e], entries[3 * e + 1], D == 3 ? entries[3 * e + 2] : 0};
    if (q.x < 0 || q.y < 0 || q.z < 0 || q.x >= pnx || q.y >= pny || q.z >= pnz) {
        set_err(err, BE_NO_BLOCK);
        return;
    }
    const long long m = gkey(q, pnx, pny);
    if (pmap[m] < 0) {
        set_err(err, BE_NO_BLOCK);
        return;
    }
    if (atomicExch(done + m, 1)) return;  // a duplicate entry
    const int nc = 1 << D, base = atomicAdd(count, nc);
    for (int c = 0; c < nc; c++)
        child[base + c] = I3b{2 * q.x + (c & 1), 2 * q.y + ((c >> 1) & 1), D == 3 ? 2 * q.z + ((c >> 2) & 1) : 0};
}

// map[key(coords[b])] = b
__global__ void k_map(const I3b *coords, int nb, int *map, int nx, int ny) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) map[gkey(coords[b], nx, ny)] = b;
}

// parent coordinates of a block (the same rule as the host construction)
__device__ __forceinline__ I3b parent_coord(const I3b q, bool same, int D) {
    if (!same) return q;
    return I3b{q.x / 2, q.y / 2, D == 3 ? q.z / 2 : 0};
}

// has-children flags of level l-1 through the blocks of level l
__global__ void k_haschild(const I3b *coords, int nb, bool same, int D, const int *pmap, int pnx, int pny,
                           unsigned char *phas) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int pi = pmap[gkey(parent_coord(coords[b], same, D), pnx, pny)];
    if (pi >= 0) phas[pi] = 1;  // every parent exists; the guard keeps a bad table in bounds
}

// sort keys: leaf flag above the Morton code; values: the block index;
// covered blocks counted
__global__ void k_keys(const I3b *coords, const unsigned char *has, int nb, unsigned long long *keys, int *vals,
                       int *nref) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const I3b q = coords[b];
    keys[b] = ((unsigned long long)(has[b] ? 0 : 1) << 63) | (unsigned long long)morton3(q.x, q.y, q.z);
    vals[b] = b;
    if (has[b]) atomicAdd(nref, 1);
}

// gid of every block from its rank; the map from block index to gid
__global__ void k_rank(const int *sorted_vals, int nb, int first, int *gid_of) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nb) gid_of[sorted_vals[r]] = first + r;
}
__global__ void k_remap(int *map, long long size, const int *gid_of) {
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < size;
         m += (long long)gridDim.x * blockDim.x)
        if (map[m] >= 0) map[m] = gid_of[map[m]];
}

struct LevelArgs {
    int l, D, n, first, nb, same_parent, coarser_same_n;
    int nblk[3], pnblk[3];
    long long cell_first, ghost_first;
    int periodic[3];
};

// the descriptor of every block of one level (maps hold global ids)
__global__ void k_desc(LevelArgs A, const I3b *coords, const unsigned char *has, const int *sorted_vals,
                       const int *map, const int *pmap, BlockDesc *blocks, int *err) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.nb) return;
    const int D = A.D, n = A.n, b = sorted_vals[r];
    const I3b q = coords[b];
    const long long C = D == 2 ? (long long)n * n : (long long)n * n * n;
    const long long Fd = D == 2 ? n : (long long)n * n, F = 2LL * D * Fd;
    BlockDesc B;
    B.cell_off = A.cell_first + r * C;
    B.ghost_off = A.ghost_first + r * F;
    B.n = n;
    B.lev = A.l;
    B.flags = has[b] ? 1 : 0;
    B.ijk[0] = q.x; B.ijk[1] = q.y; B.ijk[2] = q.z;
    B.parent = -1;
    B.poff[0] = B.poff[1] = B.poff[2] = 0;
    if (A.l > 0) {
        const I3b pq = parent_coord(q, A.same_parent, D);
        B.parent = pmap[gkey(pq, A.pnblk[0], A.pnblk[1])];
        if (A.same_parent) {
            B.poff[0] = (q.x % 2) * (n / 2);
            B.poff[1] = (q.y % 2) * (n / 2);
            B.poff[2] = D == 3 ? (q.z % 2) * (n / 2) : 0;
        }
    }
    for (int f = 0; f < 6; f++) { B.nbr[f] = -1; B.push[f] = -1; }
    for (int d = 0; d < D; d++)
        for (int s = 0; s < 2; s++) {
            int nq[3] = {q.x, q.y, q.z};
            nq[d] += s ? 1 : -1;
            if (nq[d] < 0 || nq[d] >= A.nblk[d]) {
                if (!A.periodic[d]) continue;  // physical face
                nq[d] = (nq[d] + A.nblk[d]) % A.nblk[d];
            }
            const int m = map[gkey(I3b{nq[0], nq[1], nq[2]}, A.nblk[0], A.nblk[1])];
            if (m >= 0) {
                B.nbr[2 * d + s] = m;
                B.push[2 * d + s] = A.ghost_first + (long long)(m - A.first) * F + ((2 * d + s) ^ 1) * Fd;
                continue;
            }
            // no same-level neighbour: the region one level coarser must exist (2:1)
            if (A.l == 0 || !A.coarser_same_n) {
                set_err(err, BE_INCOMPLETE);
                continue;
            }
            const I3b cq{nq[0] / 2, nq[1] / 2, D == 3 ? nq[2] / 2 : 0};
            const int cm = pmap[gkey(cq, A.pnblk[0], A.pnblk[1])];
            if (cm < 0) {
                set_err(err, BE_UNBALANCED);
                continue;
            }
            B.nbr[2 * d + s] = -2 - cm;
        }
    blocks[A.first + r] = B;
}

#define BK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            mg_set_error(std::string("device mesh build: ") + #call + ": " + cudaGetErrorString(e_)); \
            rc = MG_ERR_CUDA;                                                                 \
            goto done;                                                                        \
        }                                                                                     \
    } while (0)

int fail_code(int code, const std::string &msg) {
    mg_set_error(msg);
    return code;
}

inline int grid_for(long long n, int t = 256) { return (int)std::max<long long>(1, std::min<long long>((n + t - 1) / t, 1 << 20)); }

}  // namespace

int build_tables_device(mg_tree *t) {
    const int D = t->dim;
    const int maxdepth = max_refine_depth(t);
    const std::vector<LvSkel> sk = level_skeleton(t, maxdepth);
    const int nl = (int)sk.size(), ibase = nl - 1 - (maxdepth + 1);
    int rc = MG_OK;
    cudaStream_t s = nullptr;
    std::vector<I3b *> coords(nl, nullptr);
    std::vector<int *> map(nl, nullptr);
    std::vector<unsigned char *> has(nl, nullptr);
    std::vector<long long> msize(nl);
    std::vector<int> nb(nl, 0), nref(nl, 0);
    int *d_entries = nullptr, *d_done = nullptr, *d_cnt = nullptr, *d_err = nullptr;
    unsigned long long *keys = nullptr, *keys2 = nullptr;
    int *vals = nullptr, *vals2 = nullptr, *gid_of = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    BlockDesc *d_blocks = nullptr;
    std::vector<int> ecount(maxdepth + 2, 0), eoff(maxdepth + 2, 0), ent;
    int maxnb = 0;
    int h_cnt[2 + 64] = {0};
    int h_err = 0;
    int total = 0;
    if (nl > 64) return fail_code(MG_ERR_UNSUPPORTED, "device mesh build: too many levels");
    BK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    // refine entries by depth (i, j, k), the host order kept within a depth
    for (size_t e = 0; e < t->refine.size() / 4; e++)
        if (t->refine[4 * e] >= 0) ecount[t->refine[4 * e]]++;
    for (int r = 1; r <= maxdepth + 1; r++) eoff[r] = eoff[r - 1] + ecount[r - 1];
    ent.resize(3 * (size_t)std::max(1, eoff[maxdepth + 1]));
    {
        std::vector<int> fillp(eoff.begin(), eoff.end());
        for (size_t e = 0; e < t->refine.size() / 4; e++) {
            const int r = t->refine[4 * e];
            if (r < 0) continue;
            const int q = fillp[r]++;
            ent[3 * (size_t)q] = t->refine[4 * e + 1];
            ent[3 * (size_t)q + 1] = t->refine[4 * e + 2];
            ent[3 * (size_t)q + 2] = t->refine[4 * e + 3];
        }
    }
    BK(cudaMalloc((void **)&d_entries, sizeof(int) * ent.size()));
    BK(cudaMemcpyAsync(d_entries, ent.data(), sizeof(int) * ent.size(), cudaMemcpyHostToDevice, s));
    BK(cudaMalloc((void **)&d_cnt, sizeof(int) * (2 + 64)));
    BK(cudaMemsetAsync(d_cnt, 0, sizeof(int) * (2 + 64), s));
    d_err = d_cnt;  // d_cnt[0]: error code, d_cnt[1]: children counter, d_cnt[2 + l]: covered blocks of level l
    for (int l = 0; l < nl; l++) {
        msize[l] = (long long)sk[l].nblk[0] * sk[l].nblk[1] * sk[l].nblk[2];
        BK(cudaMalloc((void **)&map[l], sizeof(int) * msize[l]));
        BK(cudaMemsetAsync(map[l], 0xFF, sizeof(int) * msize[l], s));  // -1: no block
    }
    // coarse levels and the base grid: whole grids
    for (int l = 0; l <= ibase; l++) {
        nb[l] = (int)msize[l];
        BK(cudaMalloc((void **)&coords[l], sizeof(I3b) * std::max(1, nb[l])));
        k_grid<<<grid_for(msize[l]), 256, 0, s>>>(coords[l], map[l], sk[l].nblk[0], sk[l].nblk[1], sk[l].nblk[2]);
    }
    // refined levels: the children of the entries of each depth
    for (int r = 0; r <= maxdepth; r++) {
        const int lp = ibase + r, lc = lp + 1, ne = ecount[r];
        const long long cap = (long long)ne << D;
        BK(cudaMalloc((void **)&coords[lc], sizeof(I3b) * std::max<long long>(1, cap)));
        BK(cudaMalloc((void **)&d_done, sizeof(int) * msize[lp]));
        BK(cudaMemsetAsync(d_done, 0, sizeof(int) * msize[lp], s));
        BK(cudaMemsetAsync(d_cnt + 1, 0, sizeof(int), s));
        if (ne > 0)
            k_children<<<grid_for(ne), 256, 0, s>>>(d_entries + 3LL * eoff[r], ne, D, map[lp], sk[lp].nblk[0],
                                                    sk[lp].nblk[1], sk[lp].nblk[2], d_done, coords[lc], d_cnt + 1,
                                                    d_err);
        BK(cudaMemcpyAsync(h_cnt, d_cnt, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        BK(cudaStreamSynchronize(s));
        BK(cudaFree(d_done));
        d_done = nullptr;
        if (h_cnt[0] == BE_NO_BLOCK) { rc = fail_code(MG_ERR_ARG, "refined block does not exist"); goto done; }
        nb[lc] = h_cnt[1];
        if (nb[lc] == 0) { rc = fail_code(MG_ERR_ARG, "refinement depths must be contiguous"); goto done; }
        k_map<<<grid_for(nb[lc]), 256, 0, s>>>(coords[lc], nb[lc], map[lc], sk[lc].nblk[0], sk[lc].nblk[1]);
    }
    // has-children flags, sort keys, covered counts
    for (int l = 0; l < nl; l++) {
        BK(cudaMalloc((void **)&has[l], std::max(1, nb[l])));
        BK(cudaMemsetAsync(has[l], 0, std::max(1, nb[l]), s));
        maxnb = std::max(maxnb, nb[l]);
        total += nb[l];
    }
    for (int l = 1; l < nl; l++)
        k_haschild<<<grid_for(nb[l]), 256, 0, s>>>(coords[l], nb[l], sk[l - 1].n == sk[l].n, D, map[l - 1],
                                                    sk[l - 1].nblk[0], sk[l - 1].nblk[1], has[l - 1]);
    BK(cudaMalloc((void **)&keys, sizeof(unsigned long long) * maxnb));
    BK(cudaMalloc((void **)&keys2, sizeof(unsigned long long) * maxnb));
    BK(cudaMalloc((void **)&vals, sizeof(int) * maxnb));
    BK(cudaMalloc((void **)&gid_of, sizeof(int) * maxnb));
    BK(cudaMalloc((void **)&vals2, sizeof(int) * (size_t)total));  // sorted block indices, all levels
    BK(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys, keys2, vals, vals2, maxnb, 0, 64, s));
    BK(cudaMalloc(&tmp, std::max<size_t>(tmp_bytes, 1)));
    {
        int off = 0;
        for (int l = 0; l < nl; l++) {
            k_keys<<<grid_for(nb[l]), 256, 0, s>>>(coords[l], has[l], nb[l], keys, vals, d_cnt + 2 + l);
            size_t tb = tmp_bytes;
            BK(cub::DeviceRadixSort::SortPairs(tmp, tb, keys, keys2, vals, vals2 + off, nb[l], 0, 64, s));
            off += nb[l];
        }
    }
    BK(cudaMemcpyAsync(h_cnt, d_cnt, sizeof(int) * (2 + nl), cudaMemcpyDeviceToHost, s));
    BK(cudaStreamSynchronize(s));
    for (int l = 0; l < nl; l++) nref[l] = h_cnt[2 + l];
    fill_levels(t, sk, nb, nref);
    // global ids into the maps, then the descriptors
    {
        int off = 0;
        for (int l = 0; l < nl; l++) {
            k_rank<<<grid_for(nb[l]), 256, 0, s>>>(vals2 + off, nb[l], t->lev[l].first, gid_of);
            k_remap<<<grid_for(msize[l]), 256, 0, s>>>(map[l], msize[l], gid_of);
            off += nb[l];
        }
    }
    BK(cudaMalloc((void **)&d_blocks, sizeof(BlockDesc) * std::max(1, total)));
    {
        int off = 0;
        for (int l = 0; l < nl; l++) {
            const LevelHost &L = t->lev[l];
            LevelArgs A{};
            A.l = l; A.D = D; A.n = L.n; A.first = L.first; A.nb = L.nb;
            A.same_parent = l > 0 && sk[l - 1].n == sk[l].n;
            A.coarser_same_n = A.same_parent;
            for (int d = 0; d < 3; d++) {
                A.nblk[d] = sk[l].nblk[d];
                A.pnblk[d] = l > 0 ? sk[l - 1].nblk[d] : 1;
                A.periodic[d] = d < D && t->bc.type[2 * d] == MG_BC_PERIODIC;
            }
            A.cell_first = L.cell_first;
            A.ghost_first = L.ghost_first;
            k_desc<<<grid_for(L.nb), 256, 0, s>>>(A, coords[l], has[l], vals2 + off, map[l], l > 0 ? map[l - 1] : nullptr,
                                                  d_blocks, d_err);
            off += L.nb;
        }
    }
    BK(cudaGetLastError());
    t->blocks.assign(total, BlockDesc());
    BK(cudaMemcpyAsync(t->blocks.data(), d_blocks, sizeof(BlockDesc) * total, cudaMemcpyDeviceToHost, s));
    BK(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BK(cudaStreamSynchronize(s));
    if (h_err == BE_INCOMPLETE) { rc = fail_code(MG_ERR_BALANCE, "incomplete coarse level"); goto done; }
    if (h_err == BE_UNBALANCED) { rc = fail_code(MG_ERR_BALANCE, "mesh is not 2:1 balanced across faces"); goto done; }
    if (h_err != BE_OK) { rc = fail_code(MG_ERR_ARG, "refined block does not exist"); goto done; }
    cudaFree(t->d_blocks_built);
    t->d_blocks_built = d_blocks;  // handed to finalize
    d_blocks = nullptr;
done:
    if (s) cudaStreamSynchronize(s);
    for (int l = 0; l < nl; l++) { cudaFree(coords[l]); cudaFree(map[l]); cudaFree(has[l]); }
    cudaFree(d_entries); cudaFree(d_done); cudaFree(d_cnt);
    cudaFree(keys); cudaFree(keys2); cudaFree(vals); cudaFree(vals2); cudaFree(gid_of); cudaFree(tmp);
    cudaFree(d_blocks);
    if (s) cudaStreamDestroy(s);
    return rc;
}

}  // namespace mg
