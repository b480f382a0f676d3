// mg_adjoint.cu -- transposed operators and the adjoint solve of the octree
// geometric multigrid (Teunissen & Keppens, arXiv:1901.11370).
//
// On a mesh with refinement faces the composite operator A is not symmetric
// (Sec. 2.6): a fine row reads the coarse cell B through its refinement
// ghost with weight 1/2, while the row of B reads the fine cells through the
// mean of the covered cell D, 1/2^D each.  The adjoint of a loss through the
// solve therefore needs A^T.  Every forward operator is a stencil over
// interior values and face ghosts after a refresh (restriction of covered
// cells bottom-up, then ghost fills coarsest level first).  Its transpose
// runs those steps in reverse with transposed coefficients, accumulating
// into an adjoint array with the pool's layout (interior cells + face
// ghosts):
//   1. k_stencil_T on the leaf blocks: every leaf row hands its weights to
//      the values it reads.  Within a block this is a gather (each cell sums
//      the rows that read it); a value read across a block face is a ghost
//      slot, written by the one row beside it.  No atomics.
//   2. k_ghost_T level by level, finest first: every ghost slot's adjoint
//      goes to the values the ghost was formed from -- the same-level
//      neighbour's cell, the block's own cell (physical faces), or
//      B'/2 + 3c/4 - d/4 with B' = B + sum_t s_t (C_t - A_t)/8 at a
//      refinement face.  Several slots feed one value, so these are FP64
//      atomic adds.
//   3. k_restrict_T level by level, coarsest first: every cell takes 1/2^D
//      of its parent cell's adjoint (the mean restriction of Sec. 2.3).
// The leaf cells then hold the result.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "mg_internal.h"
#include "mg_device.cuh"

namespace mg {

enum { T_OPERATOR = 0, T_EPS = 1, T_DIV = 2, T_GRAD = 3 };        // stencil transposes
enum { G_PHI = 0, G_EPS = 1, G_VEC = 2 };                          // ghost rules
enum { V_INIT = 0, V_RESID = 1, V_SET = 2, V_ADD = 3, V_SUM = 4, V_PROJ = 5, V_SUB = 6 };  // leaf vector ops

// Weight of face (d, s) in the row of cell (i, j, k) of block b (Sec. 2.2):
// (1/h_d^2) times the harmonic mean of the two cells' coefficients (the
// neighbour may be a ghost), times r_face / r_cell on r-faces of the
// cylindrical form.
template <int D>
__device__ __forceinline__ double face_w(const KParams &P, const LevelDesc &L, const BlockDesc &b,
                                         const double *__restrict__ E, const double *__restrict__ EG, int i, int j,
                                         int k, int d, int s) {
    double w = L.inv_h2[d];
    if (E) {
        const int o = s ? 1 : -1;
        const double ec = E[b.cell_off + cidx<D>(b.n, i, j, k)];
        const double en = load<double, D>(E, EG, b, i + (d == 0 ? o : 0), j + (d == 1 ? o : 0), k + (d == 2 ? o : 0));
        w *= 2.0 * ec * en / (ec + en);
    }
    if (P.geom == MG_CYL && d == 0) {
        const int I = b.ijk[0] * b.n + i;
        w *= (P.lo[0] + (I + s) * L.h[0]) / (P.lo[0] + (I + 0.5) * L.h[0]);
    }
    return w;
}

// r_face / r_cell of face (0, s) of the cell at global radial index I
// (1 outside the cylindrical form or on other dimensions)
__device__ __forceinline__ double kappa(const KParams &P, const LevelDesc &L, int d, int I, int s) {
    if (P.geom != MG_CYL || d != 0) return 1.0;
    return (P.lo[0] + (I + s) * L.h[0]) / (P.lo[0] + (I + 0.5) * L.h[0]);
}

// Address of the value at (i, j, k) of block b, at most one coordinate one
// cell outside the block (then a ghost slot): the pointer form of load().
template <int D>
__device__ __forceinline__ double *addr(double *A, double *AG, const BlockDesc &b, int i, int j, int k) {
    const int n = b.n, F = face_of<D>(n);
    const long long go = b.ghost_off;
    if (i < 0) return AG + go + 0 * F + tidx<D>(n, 0, i, j, k);
    if (i >= n) return AG + go + 1 * F + tidx<D>(n, 0, i, j, k);
    if (j < 0) return AG + go + 2 * F + tidx<D>(n, 1, i, j, k);
    if (j >= n) return AG + go + 3 * F + tidx<D>(n, 1, i, j, k);
    if (D == 3) {
        if (k < 0) return AG + go + 4 * F + tidx<D>(n, 2, i, j, k);
        if (k >= n) return AG + go + 5 * F + tidx<D>(n, 2, i, j, k);
    }
    return A + b.cell_off + cidx<D>(n, i, j, k);
}

// Step 1 on the leaf blocks [first, first + gridDim.x) of one level.  Y is
// the leaf-order input (kind T_GRAD: dim arrays of nleaf values).  Writes
// the adjoint of every interior cell (A) and of every ghost slot a row of
// this block reads (AG); the caller zeroes AG first.
//   T_OPERATOR: rows sum_f w_f (x_nb - x_c) - lambda x_c of A (Sec. 2.2);
//   T_EPS:      y = lambda, the rows' derivative -y d(w_f)/d eps with the
//               harmonic mean w_f ~ 2 e_c e_o / (e_c + e_o) and phi = X;
//   T_DIV:      component dc of (B(c+e) - B(c-e)) / (2 h) (Sec. 4.1);
//   T_GRAD:     all components of the central gradient of phi.
template <int D>
__global__ void __launch_bounds__(kMaxThreads) k_stencil_T(KParams P, int first, int kind, int dc,
                                                           const double *__restrict__ Y, long long leaf_base,
                                                           long long nleaf, const double *__restrict__ X,
                                                           const double *__restrict__ XG,
                                                           const double *__restrict__ E,
                                                           const double *__restrict__ EG, double *__restrict__ A,
                                                           double *__restrict__ AG) {
    pdl_entry();
    __shared__ BlockDesc sb;
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, C = cells_of<D>(n), F = face_of<D>(n);
    const double *y = Y + leaf_base + (long long)blockIdx.x * C;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        const I3 p{i, j, k};
        double acc = 0.0;
        if (kind == T_OPERATOR) {
            double sw = 0.0;
            const double yc = y[c];
#pragma unroll
            for (int d = 0; d < D; d++)
#pragma unroll
                for (int s = 0; s < 2; s++) {
                    const double w = face_w<D>(P, L, b, E, EG, i, j, k, d, s);
                    sw += w;
                    I3 q = p;
                    put(q, d, get(p, d) + (s ? 1 : -1));
                    const int qd = get(q, d);
                    if (qd >= 0 && qd < n)  // the neighbour's row reads this cell across its face (d, 1 - s)
                        acc += face_w<D>(P, L, b, E, EG, q.x, q.y, q.z, d, 1 - s) * y[cidx<D>(n, q.x, q.y, q.z)];
                    else
                        AG[b.ghost_off + (2 * d + s) * F + tidx<D>(n, d, i, j, k)] = w * yc;
                }
            acc -= (sw + P.helm) * yc;
        } else if (kind == T_EPS) {
            const double xc = X[b.cell_off + c], ec = E ? E[b.cell_off + c] : 1.0, yc = y[c];
            const int I = b.ijk[0] * n + i;
#pragma unroll
            for (int d = 0; d < D; d++)
#pragma unroll
                for (int s = 0; s < 2; s++) {
                    I3 q = p;
                    put(q, d, get(p, d) + (s ? 1 : -1));
                    const double xo = load<double, D>(X, XG, b, q.x, q.y, q.z);
                    const double eo = E ? load<double, D>(E, EG, b, q.x, q.y, q.z) : 1.0;
                    const double sm = ec + eo, hm = 2.0 * L.inv_h2[d] / (sm * sm);
                    // this row's term: -y_c kappa_c w' (x_o - x_c)
                    const double dwc = -yc * kappa(P, L, d, I, s) * hm * (xo - xc);
                    acc += dwc * eo * eo;
                    const int qd = get(q, d);
                    if (qd >= 0 && qd < n) {
                        // the neighbour's row reads e_c through the same face
                        const int Io = I + (d == 0 ? (s ? 1 : -1) : 0);
                        const double dwo = -y[cidx<D>(n, q.x, q.y, q.z)] * kappa(P, L, d, Io, 1 - s) * hm * (xc - xo);
                        acc += dwo * eo * eo;
                    } else {
                        AG[b.ghost_off + (2 * d + s) * F + tidx<D>(n, d, i, j, k)] = dwc * ec * ec;
                    }
                }
        } else {
#pragma unroll
            for (int d = 0; d < D; d++) {
                if (kind == T_DIV && d != dc) continue;
                const double *yd = kind == T_GRAD ? Y + (long long)d * nleaf + leaf_base + (long long)blockIdx.x * C : y;
                const double s2h = 0.5 / L.h[d];
                const int pd = get(p, d);
                I3 q = p;
                if (pd >= 1) {  // row c - e_d reads this cell as its + neighbour
                    put(q, d, pd - 1);
                    acc += yd[cidx<D>(n, q.x, q.y, q.z)] * s2h;
                } else {
                    AG[b.ghost_off + (2 * d) * F + tidx<D>(n, d, i, j, k)] = -yd[c] * s2h;
                }
                if (pd <= n - 2) {  // row c + e_d reads this cell as its - neighbour
                    put(q, d, pd + 1);
                    acc -= yd[cidx<D>(n, q.x, q.y, q.z)] * s2h;
                } else {
                    AG[b.ghost_off + (2 * d + 1) * F + tidx<D>(n, d, i, j, k)] = yd[c] * s2h;
                }
            }
        }
        A[b.cell_off + c] = acc;
    }
}

// Step 2 on all blocks [first, first + gridDim.x) of one level: the
// transpose of the ghost fill (k_ghost).  mode G_PHI: physical ghosts
// -x_i (Dirichlet) / x_i (Neumann, axis), refinement ghosts
// B'/2 + 3c/4 - d/4; G_EPS: physical ghosts x_i, refinement ghosts B;
// G_VEC: physical ghosts x_i, refinement ghosts as G_PHI.
template <int D>
__global__ void __launch_bounds__(kMaxThreads) k_ghost_T(KParams P, int first, int mode, double *__restrict__ A,
                                                         double *__restrict__ AG) {
    pdl_entry();
    __shared__ BlockDesc sb;
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, F = face_of<D>(n);
    for (int t = threadIdx.x; t < 2 * D * F; t += blockDim.x) {
        const double gb = AG[b.ghost_off + t];
        if (gb == 0.0) continue;
        const int face = t / F, u = t - face * F, d = face >> 1, s = face & 1;
        const I3 ii = face_cell<D>(n, face, u, false);
        const int nb = b.nbr[face];
        if (nb >= 0) {
            const BlockDesc &q = P.B[nb];
            I3 jj = ii;
            put(jj, d, s ? 0 : n - 1);
            atomicAdd(A + q.cell_off + cidx<D>(n, jj.x, jj.y, jj.z), gb);
        } else if (nb == -1) {
            const double coef = (mode == G_PHI && P.bct[face] == MG_BC_DIRICHLET) ? -1.0 : 1.0;
            atomicAdd(A + b.cell_off + cidx<D>(n, ii.x, ii.y, ii.z), coef * gb);
        } else {
            const BlockDesc &q = P.B[-2 - nb];
            const int qn = q.n;
            I3 G{b.ijk[0] * n + ii.x, b.ijk[1] * n + ii.y, b.ijk[2] * n + ii.z};
            int gd = b.ijk[d] * n + (s ? n : -1);
            const int nd = L.ncell[d];
            gd = gd < 0 ? gd + nd : (gd >= nd ? gd - nd : gd);
            put(G, d, gd);
            const I3 lc{(G.x >> 1) - q.ijk[0] * qn, (G.y >> 1) - q.ijk[1] * qn,
                        D == 3 ? (G.z >> 1) - q.ijk[2] * qn : 0};
            atomicAdd(A + q.cell_off + cidx<D>(qn, lc.x, lc.y, lc.z), mode == G_EPS ? gb : 0.5 * gb);
            if (mode == G_EPS) continue;
#pragma unroll
            for (int e = 0; e < D; e++) {
                if (e == d) continue;
                const double w = ((get(G, e) & 1) ? 1.0 : -1.0) * gb / 16.0;
                const int ox = e == 0, oy = e == 1, oz = e == 2;
                atomicAdd(addr<D>(A, AG, q, lc.x + ox, lc.y + oy, lc.z + oz), w);
                atomicAdd(addr<D>(A, AG, q, lc.x - ox, lc.y - oy, lc.z - oz), -w);
            }
            I3 dd = ii;
            put(dd, d, s ? n - 2 : 1);
            atomicAdd(A + b.cell_off + cidx<D>(n, ii.x, ii.y, ii.z), 0.75 * gb);
            atomicAdd(A + b.cell_off + cidx<D>(n, dd.x, dd.y, dd.z), -0.25 * gb);
        }
    }
}

// Step 3 on all blocks [first, first + gridDim.x) of one level above the
// coarsest: every cell adds 1/2^D of its parent cell's adjoint.
template <int D>
__global__ void __launch_bounds__(kMaxThreads) k_restrict_T(KParams P, int first, double *__restrict__ A) {
    pdl_entry();
    __shared__ BlockDesc sb;
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
    const BlockDesc &p = P.B[b.parent];
    const int n = b.n, C = cells_of<D>(n);
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        const double pv = A[p.cell_off + cidx<D>(p.n, b.poff[0] + i / 2, b.poff[1] + j / 2,
                                                 D == 3 ? b.poff[2] + k / 2 : 0)];
        A[b.cell_off + c] += pv * (1.0 / (1 << D));
    }
}

// Leaf-vector steps of the adjoint iteration, one CTA per leaf block of one
// level; V is the cell volume.  la, lb, lo are leaf-order vectors, ca / co
// pool cells.  Per-CTA partial sums (3 doubles) where an op reduces.
//   V_INIT:  co = la / V;              partials sum V (la/V)^2, sum V
//   V_RESID: co = (la - lb) / V;       partials sum V ((la-lb)/V)^2, sum V
//   V_SET:   lo = V ca                 V_ADD: lo += V ca
//   V_SUM:   partials sum la, sum V    V_PROJ: lo = la - scal V
//   V_SUB:   lo = la - lb
template <int D>
__global__ void __launch_bounds__(256) k_adj_vec(KParams P, int first, long long leaf_base, int op,
                                                 const double *__restrict__ la, const double *__restrict__ lb,
                                                 double *__restrict__ lo, const double *__restrict__ ca,
                                                 double *__restrict__ co, double scal,
                                                 double *__restrict__ partials) {
    pdl_entry();
    const BlockDesc &b = P.B[first + blockIdx.x];
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, C = cells_of<D>(n);
    const long long m0 = leaf_base + (long long)blockIdx.x * C;
    double s0 = 0.0, s1 = 0.0;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        double V = L.vol;
        if (P.geom == MG_CYL) V = 2.0 * M_PI * (P.lo[0] + (b.ijk[0] * n + c % n + 0.5) * L.h[0]) * L.h[0] * L.h[1];
        const long long m = m0 + c;
        switch (op) {
        case V_INIT:
        case V_RESID: {
            const double r = (op == V_INIT ? la[m] : la[m] - lb[m]) / V;
            co[b.cell_off + c] = r;
            s0 = fma(V * r, r, s0);
            s1 += V;
            break;
        }
        case V_SET: lo[m] = V * ca[b.cell_off + c]; break;
        case V_ADD: lo[m] = fma(V, ca[b.cell_off + c], lo[m]); break;
        case V_SUM: s0 += la[m]; s1 += V; break;
        case V_PROJ: lo[m] = la[m] - scal * V; break;
        default: lo[m] = la[m] - lb[m]; break;
        }
    }
    if (op != V_INIT && op != V_RESID && op != V_SUM) return;
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
    }
    __shared__ double sh[2][8];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][w] = s0; sh[1][w] = s1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, z = 0;
        for (int e = 0; e < (int)(blockDim.x >> 5); e++) { x += sh[0][e]; z += sh[1][e]; }
        partials[3 * blockIdx.x] = x;
        partials[3 * blockIdx.x + 1] = z;
        partials[3 * blockIdx.x + 2] = 0.0;
    }
}

// Sum of n partial pairs (one CTA, fixed order: deterministic).
__global__ void __launch_bounds__(1024) k_sum_partials(const double *__restrict__ partials, int n,
                                                       double *__restrict__ out) {
    pdl_entry();
    double a = 0, z = 0;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        a += partials[3 * e];
        z += partials[3 * e + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        z += __shfl_down_sync(0xffffffffu, z, o);
    }
    __shared__ double sh[2][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][w] = a; sh[1][w] = z; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int e = 0; e < (int)(blockDim.x >> 5); e++) { x += sh[0][e]; y += sh[1][e]; }
        out[0] = x;
        out[1] = y;
    }
}

// ------------------------------------------------------------ host side ---

static int threads_of(int cells) {
    const int t = ((cells + 31) / 32) * 32;
    return t < 32 ? 32 : (t > kMaxThreads ? kMaxThreads : t);
}

static int dmalloc(double **p, long long n) {
    if (*p) return MG_OK;
    if (cudaMalloc((void **)p, sizeof(double) * (size_t)std::max(1LL, n)) != cudaSuccess) {
        cudaGetLastError();
        mg_set_error("adjoint: device allocation failed");
        return MG_ERR_CUDA;
    }
    return MG_OK;
}

int adjoint_buffers(mg_tree *t) {
    int rc;
    if ((rc = dmalloc(&t->d_at, t->ncells)) || (rc = dmalloc(&t->d_atg, t->nghost)) ||
        (rc = dmalloc(&t->d_lam, t->nleaf_cells)) || (rc = dmalloc(&t->d_gh, t->nleaf_cells)) ||
        (rc = dmalloc(&t->d_lv, t->nleaf_cells)))
        return rc;
    return MG_OK;
}

// leaf cells of a pool array into a leaf-order vector (levels ascending)
static void cells_to_leaf(mg_tree *t, const double *cells, double *leaf) {
    long long off = 0;
    for (const LevelHost &L : t->lev) {
        const long long m = (long long)(L.nb - L.nref) * (t->dim == 2 ? (long long)L.n * L.n : (long long)L.n * L.n * L.n);
        if (m == 0) continue;
        cudaMemcpyAsync(leaf + off, cells + t->blocks[L.first + L.nref].cell_off, sizeof(double) * m,
                        cudaMemcpyDeviceToDevice, t->stream);
        off += m;
    }
}

template <int D> struct Adj {
    // steps 1-3 (and the leaf read-out) for one transposed operator
    static void stencil(mg_tree *t, const KParams &P, int kind, int dc, const double *Y, const double *X,
                        const double *XG, const double *E, const double *EG) {
        cudaMemsetAsync(t->d_atg, 0, sizeof(double) * (size_t)t->nghost, t->stream);
        cudaMemsetAsync(t->d_at, 0, sizeof(double) * (size_t)t->ncells, t->stream);
        long long leaf_base = 0;
        for (const LevelHost &L : t->lev) {
            const int nleaf = L.nb - L.nref;
            if (nleaf <= 0) continue;
            ++t->launches;
            launch_k(k_stencil_T<D>, nleaf, threads_of(cells_of<D>(L.n)), 0, t->stream, P, L.first + L.nref, kind,
                     dc, Y, leaf_base, (long long)t->nleaf_cells, X, XG, E, EG, t->d_at, t->d_atg);
            leaf_base += (long long)nleaf * cells_of<D>(L.n);
        }
    }
    static void refresh_T(mg_tree *t, const KParams &P, int mode) {
        const int nl = (int)t->lev.size();
        for (int l = nl - 1; l >= 0; l--) {
            const LevelHost &L = t->lev[l];
            ++t->launches;
            launch_k(k_ghost_T<D>, L.nb, threads_of(2 * D * face_of<D>(L.n)), 0, t->stream, P, L.first, mode,
                     t->d_at, t->d_atg);
        }
        for (int l = 1; l < nl; l++) {
            const LevelHost &L = t->lev[l];
            ++t->launches;
            launch_k(k_restrict_T<D>, L.nb, threads_of(cells_of<D>(L.n)), 0, t->stream, P, L.first, t->d_at);
        }
    }
    // leaf-vector op over all leaf blocks; with a reduction, the two sums
    // arrive on the host (synchronises the stream)
    static void vec(mg_tree *t, const KParams &P, int op, const double *la, const double *lb, double *lo,
                    const double *ca, double *co, double scal, double *sums) {
        long long leaf_base = 0;
        int slot = 0;
        for (const LevelHost &L : t->lev) {
            const int nleaf = L.nb - L.nref;
            if (nleaf <= 0) continue;
            ++t->launches;
            launch_k(k_adj_vec<D>, nleaf, 256, 0, t->stream, P, L.first + L.nref, leaf_base, op, la, lb, lo, ca,
                     co, scal, t->d_partials + 3LL * slot);
            slot += nleaf;
            leaf_base += (long long)nleaf * cells_of<D>(L.n);
        }
        if (!sums) return;
        ++t->launches;
        launch_k(k_sum_partials, 1, 1024, 0, t->stream, (const double *)t->d_partials, slot, t->d_red);
        cudaMemcpyAsync(t->h_red, t->d_red, 2 * sizeof(double), cudaMemcpyDeviceToHost, t->stream);
        cudaStreamSynchronize(t->stream);
        sums[0] = t->h_red[0];
        sums[1] = t->h_red[1];
    }
};

template <int D> static void apply_T_d(mg_tree *t, const double *y, double *out) {
    const KParams P = kparams(t, 1);
    Adj<D>::stencil(t, P, T_OPERATOR, 0, y, nullptr, nullptr, t->var_eps ? t->f64.E : nullptr,
                    t->var_eps ? t->f64.EG : nullptr);
    Adj<D>::refresh_T(t, P, G_PHI);
    cells_to_leaf(t, t->d_at, out);
}

void apply_transpose(mg_tree *t, const double *y, double *out) {
    if (t->dim == 2) apply_T_d<2>(t, y, out);
    else apply_T_d<3>(t, y, out);
}

template <int D> static void eps_grad_T_d(mg_tree *t, const double *lam, double *out) {
    refresh<double>(t, t->f64, 0);  // phi: covered cells and the ghosts the leaf rows read
    const KParams P = kparams(t, 0);
    Adj<D>::stencil(t, P, T_EPS, 0, lam, t->f64.X, t->f64.XG, t->var_eps ? t->f64.E : nullptr,
                    t->var_eps ? t->f64.EG : nullptr);
    Adj<D>::refresh_T(t, P, G_EPS);
    cells_to_leaf(t, t->d_at, out);
}

void eps_grad_transpose(mg_tree *t, const double *lam, double *out) {
    if (t->dim == 2) eps_grad_T_d<2>(t, lam, out);
    else eps_grad_T_d<3>(t, lam, out);
}

// The adjoint solve (reading R16).  With W the cell volumes, A* = W^-1 A^T W
// equals A where W A is symmetric and stays close to it at refinement faces,
// so A's V-cycle M approximates its inverse:
//   mu_0 = FMG(W^-1 g), lambda_0 = W mu_0,
//   lambda += W M W^-1 (g - A^T lambda)   (homogeneous boundary values)
// until the volume-weighted norm of W^-1 (g - A^T lambda) is at most rel_tol
// times that of W^-1 g, or max_it iterations.  Singular problems: g is made
// compatible (sum g = 0) and lambda returned as lambda - W sum(lambda) / sum W.
template <int D>
static int adjoint_dc_d(mg_tree *t, const double *g, double *lam, int nd, int nu, double rel_tol, int max_it,
                        int *it_out, double *rel_out, bool fp32) {
    const KParams P = kparams(t, 1);
    double s[2];
    cudaMemcpyAsync(t->d_gh, g, sizeof(double) * (size_t)t->nleaf_cells, cudaMemcpyDeviceToDevice, t->stream);
    if (t->singular) {
        Adj<D>::vec(t, P, V_SUM, t->d_gh, nullptr, nullptr, nullptr, nullptr, 0.0, s);
        Adj<D>::vec(t, P, V_PROJ, t->d_gh, nullptr, t->d_gh, nullptr, nullptr, s[1] > 0 ? s[0] / s[1] : 0.0, nullptr);
    }
    Adj<D>::vec(t, P, V_INIT, t->d_gh, nullptr, nullptr, nullptr, t->adj.F, 0.0, s);
    const double r0 = s[1] > 0 ? std::sqrt(s[0] / s[1]) : 0.0;
    cudaMemsetAsync(t->adj.X, 0, sizeof(double) * (size_t)t->ncells, t->stream);
    cudaMemsetAsync(t->adj.XG, 0, sizeof(double) * (size_t)t->nghost, t->stream);
    fmg<double>(t, t->adj, nd, nu, 1);
    Adj<D>::vec(t, P, V_SET, nullptr, nullptr, lam, t->adj.X, nullptr, 0.0, nullptr);
    const int top = (int)t->groups.size() - 1;
    int it = 0;
    double rel = 0.0;
    for (;;) {
        apply_T_d<D>(t, lam, t->d_lv);
        Adj<D>::vec(t, P, V_RESID, t->d_gh, t->d_lv, nullptr, nullptr, t->adj.F, 0.0, s);
        rel = r0 > 0 ? std::sqrt(s[0] / s[1]) / r0 : 0.0;
        if (it >= max_it || rel <= rel_tol || !std::isfinite(rel)) break;
        if (fp32) {  // the FP32 V-cycle on the residual's FP32 copy, as in the forward solve's defect correction
            narrow_f32(t, t->adj.F, t->f32.F, t->ncells);
            cudaMemsetAsync(t->f32.X, 0, sizeof(float) * (size_t)t->ncells, t->stream);
            cudaMemsetAsync(t->f32.XG, 0, sizeof(float) * (size_t)t->nghost, t->stream);
            vcycle<float>(t, t->f32, top, nd, nu, 1);
            widen_f64(t, t->f32.X, t->adj.X, t->ncells);
        } else {
            cudaMemsetAsync(t->adj.X, 0, sizeof(double) * (size_t)t->ncells, t->stream);
            cudaMemsetAsync(t->adj.XG, 0, sizeof(double) * (size_t)t->nghost, t->stream);
            vcycle<double>(t, t->adj, top, nd, nu, 1);
        }
        Adj<D>::vec(t, P, V_ADD, nullptr, nullptr, lam, t->adj.X, nullptr, 0.0, nullptr);
        it++;
    }
    if (t->singular) {
        Adj<D>::vec(t, P, V_SUM, lam, nullptr, nullptr, nullptr, nullptr, 0.0, s);
        Adj<D>::vec(t, P, V_PROJ, lam, nullptr, lam, nullptr, nullptr, s[1] > 0 ? s[0] / s[1] : 0.0, nullptr);
    }
    if (it_out) *it_out = it;
    if (rel_out) *rel_out = rel;
    return check_cuda("adjoint");
}

int adjoint_dc(mg_tree *t, const double *g, double *lam, int nd, int nu, double rel_tol, int max_it, int *it_out,
               double *rel_out, bool fp32) {
    return t->dim == 2 ? adjoint_dc_d<2>(t, g, lam, nd, nu, rel_tol, max_it, it_out, rel_out, fp32)
                       : adjoint_dc_d<3>(t, g, lam, nd, nu, rel_tol, max_it, it_out, rel_out, fp32);
}

// Vector-Jacobian product of the cleaning map B -> B - G phi, phi the
// solution of A phi = P D B (second-order central divergence and gradient,
// Sec. 4.1): gB = gBn - D^T P^T A^-T Q^T G^T gBn, the projections P, Q of a
// singular problem applied inside adjoint_dc.
template <int D>
static int clean_adjoint_d(mg_tree *t, const double *gBn, double *gB, int nd, int nu, double rel_tol, int max_it,
                           int *it_out, double *rel_out, bool fp32) {
    const KParams P = kparams(t, 1);
    const long long nl = t->nleaf_cells;
    // u = G^T gBn into gB's first component (free until the end)
    Adj<D>::stencil(t, P, T_GRAD, 0, gBn, nullptr, nullptr, nullptr, nullptr);
    Adj<D>::refresh_T(t, P, G_PHI);
    double *u = gB;
    cells_to_leaf(t, t->d_at, u);
    int rc = adjoint_dc_d<D>(t, u, t->d_lam, nd, nu, rel_tol, max_it, it_out, rel_out, fp32);
    if (rc) return rc;
    for (int d = 0; d < D; d++) {
        Adj<D>::stencil(t, P, T_DIV, d, t->d_lam, nullptr, nullptr, nullptr, nullptr);
        Adj<D>::refresh_T(t, P, G_VEC);
        cells_to_leaf(t, t->d_at, t->d_lv);
        Adj<D>::vec(t, P, V_SUB, gBn + d * nl, t->d_lv, gB + d * nl, nullptr, nullptr, 0.0, nullptr);
    }
    return check_cuda("clean adjoint");
}

int clean_adjoint(mg_tree *t, const double *gBn, double *gB, int nd, int nu, double rel_tol, int max_it, int *it_out,
                  double *rel_out, bool fp32) {
    return t->dim == 2 ? clean_adjoint_d<2>(t, gBn, gB, nd, nu, rel_tol, max_it, it_out, rel_out, fp32)
                       : clean_adjoint_d<3>(t, gBn, gB, nd, nu, rel_tol, max_it, it_out, rel_out, fp32);
}

}  // namespace mg
