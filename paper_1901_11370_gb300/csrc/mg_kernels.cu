// mg_kernels.cu -- sm_103a kernels and the cycle driver of the octree
// geometric multigrid (Teunissen & Keppens, arXiv:1901.11370).
//
// Every kernel works on a contiguous range of global block ids (one level,
// or its covered / leaf part) with one CTA per block.  Fields are stored
// interior-only, block-major (x fastest), plus a face-ghost array (see
// BlockDesc).  The 5/7-point stencil is memory-bound, so nothing here uses
// tensor cores: the kernels are written for coalesced HBM access of whole
// blocks, with neighbour faces served by L1/L2.
#include <cmath>
#include <cstdio>
#include <vector>

#include "mg_internal.h"

namespace mg {

static constexpr int kMaxThreads = 256;

template <int D> __host__ __device__ __forceinline__ int cells_of(int n) { return D == 2 ? n * n : n * n * n; }
template <int D> __host__ __device__ __forceinline__ int face_of(int n) { return D == 2 ? n : n * n; }
template <int D> __device__ __forceinline__ int cidx(int n, int i, int j, int k) {
    return D == 2 ? j * n + i : (k * n + j) * n + i;
}
// index of cell (i,j,k) on the face of dimension d: t1 + n*t2, t1 < t2 the
// two other dimensions
template <int D> __device__ __forceinline__ int tidx(int n, int d, int i, int j, int k) {
    if (D == 2) return d == 0 ? j : i;
    return d == 0 ? j + n * k : (d == 1 ? i + n * k : i + n * j);
}

// Value at (i,j,k) of block b, where at most one coordinate lies one cell
// outside the block (a face ghost).
template <class T, int D>
__device__ __forceinline__ T load(const T *__restrict__ X, const T *__restrict__ XG, const BlockDesc &b,
                                  int i, int j, int k) {
    const int n = b.n, F = face_of<D>(n);
    const long long go = b.ghost_off;
    if (i < 0) return XG[go + 0 * F + tidx<D>(n, 0, i, j, k)];
    if (i >= n) return XG[go + 1 * F + tidx<D>(n, 0, i, j, k)];
    if (j < 0) return XG[go + 2 * F + tidx<D>(n, 1, i, j, k)];
    if (j >= n) return XG[go + 3 * F + tidx<D>(n, 1, i, j, k)];
    if (D == 3) {
        if (k < 0) return XG[go + 4 * F + tidx<D>(n, 2, i, j, k)];
        if (k >= n) return XG[go + 5 * F + tidx<D>(n, 2, i, j, k)];
    }
    return X[b.cell_off + cidx<D>(n, i, j, k)];
}

// 5/7-point row at a cell (Sec. 2.2): for every face the weight
// w = eps_f * kappa_f / h_d^2 (eps_f harmonic mean of the two cells, kappa
// r_f/r_i on r-faces of the cylindrical form), giving
//   lap = sum w (x_nb - x_c),  num = sum w x_nb,  den = sum w.
template <class A, class T, int D>
__device__ __forceinline__ void stencil(const KParams &P, const LevelDesc &L, const BlockDesc &b,
                                        const T *__restrict__ X, const T *__restrict__ XG,
                                        const T *__restrict__ E, const T *__restrict__ EG,
                                        int i, int j, int k, A &lap, A &num, A &den, A &xc) {
    const int n = b.n;
    xc = (A)X[b.cell_off + cidx<D>(n, i, j, k)];
    A ec = 1;
    if (E) ec = (A)E[b.cell_off + cidx<D>(n, i, j, k)];
    lap = 0; num = 0; den = 0;
    A ri = 0;
    if (P.geom == MG_CYL) ri = (A)(P.lo[0] + (b.ijk[0] * n + i + 0.5) * L.h[0]);
#pragma unroll
    for (int d = 0; d < D; d++) {
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int o = s ? 1 : -1;
            const int ii = i + (d == 0 ? o : 0), jj = j + (d == 1 ? o : 0), kk = k + (d == 2 ? o : 0);
            const A xn = (A)load<T, D>(X, XG, b, ii, jj, kk);
            A w = (A)L.inv_h2[d];
            if (E) {
                const A en = (A)load<T, D>(E, EG, b, ii, jj, kk);
                w *= (A)2 * ec * en / (ec + en);
            }
            if (P.geom == MG_CYL && d == 0) {
                const A rf = (A)(P.lo[0] + (b.ijk[0] * n + i + s) * L.h[0]);
                w *= rf / ri;
            }
            lap += w * (xn - xc);
            num += w * xn;
            den += w;
        }
    }
}

__device__ __forceinline__ void cell_of(int c, int n, int D, int &i, int &j, int &k) {
    i = c % n;
    j = (c / n) % n;
    k = D == 3 ? c / (n * n) : 0;
}

// ------------------------------------------------------------- ghosts ----
// Face ghosts of every block in [first, first + gridDim.x) (Sec. 2.6):
// same-level or periodic copy; physical boundary (Dirichlet 2a - x_i,
// Neumann x_i -/+ h b, axis x_i); refinement boundary
// g = B'/2 + 3c/4 - d/4 with B' = B + sum_t s_t (C_t - A_t)/8 read from the
// coarser block and its own ghosts.  mode 1 (coefficient): physical ghosts
// copy the interior value, refinement ghosts take B.
template <class T, int D>
__global__ void __launch_bounds__(kMaxThreads) k_ghost(KParams P, int first, T *__restrict__ X,
                                                       T *__restrict__ XG, int mode) {
    const BlockDesc b = P.B[first + blockIdx.x];
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, F = face_of<D>(n);
    for (int t = threadIdx.x; t < 2 * D * F; t += blockDim.x) {
        const int face = t / F, u = t - face * F, d = face >> 1, s = face & 1;
        int ii[3] = {0, 0, 0};
        {
            int t1 = u % n, t2 = u / n, a = 0;
            for (int e = 0; e < D; e++)
                if (e != d) ii[e] = (a++ == 0) ? t1 : t2;
        }
        ii[d] = s ? n - 1 : 0;
        const int nb = b.nbr[face];
        T val;
        if (nb >= 0) {
            const BlockDesc &q = P.B[nb];
            int jj[3] = {ii[0], ii[1], ii[2]};
            jj[d] = s ? 0 : n - 1;
            val = X[q.cell_off + cidx<D>(n, jj[0], jj[1], jj[2])];
        } else if (nb == -1) {
            const T xi = X[b.cell_off + cidx<D>(n, ii[0], ii[1], ii[2])];
            if (mode == 1) {
                val = xi;
            } else {
                double a = 0.0;
                if (!P.homog) {
                    if (L.bc_off[face] >= 0) {
                        int G[3], t1 = -1, t2 = -1;
                        for (int e = 0; e < 3; e++) G[e] = b.ijk[e] * n + ii[e];
                        for (int e = 0; e < D; e++)
                            if (e != d) { if (t1 < 0) t1 = e; else t2 = e; }
                        long long idx = G[t1];
                        if (t2 >= 0) idx += (long long)L.ncell[t1] * G[t2];
                        a = P.bcplanes[L.bc_off[face] + idx];
                    } else {
                        a = P.bcv[face];
                    }
                }
                switch (P.bct[face]) {
                case MG_BC_DIRICHLET: val = (T)(2.0 * a) - xi; break;
                case MG_BC_NEUMANN: val = s ? xi + (T)(L.h[d] * a) : xi - (T)(L.h[d] * a); break;
                default: val = xi; break;
                }
            }
        } else {
            const BlockDesc &q = P.B[-2 - nb];
            const int qn = q.n;
            int G[3];
            for (int e = 0; e < 3; e++) G[e] = b.ijk[e] * n + ii[e];
            G[d] = b.ijk[d] * n + (s ? n : -1);
            if (G[d] < 0) G[d] += L.ncell[d];
            if (G[d] >= L.ncell[d]) G[d] -= L.ncell[d];
            int lc[3] = {0, 0, 0};
            for (int e = 0; e < D; e++) lc[e] = (G[e] >> 1) - q.ijk[e] * qn;
            const T B = X[q.cell_off + cidx<D>(qn, lc[0], lc[1], lc[2])];
            if (mode == 1) {
                val = B;
            } else {
                T Bp = B;
                for (int e = 0; e < D; e++) {
                    if (e == d) continue;
                    const T sg = (G[e] & 1) ? (T)1 : (T)-1;
                    int la[3] = {lc[0], lc[1], lc[2]}, lb[3] = {lc[0], lc[1], lc[2]};
                    la[e] -= 1;
                    lb[e] += 1;
                    const T Av = load<T, D>(X, XG, q, la[0], la[1], la[2]);
                    const T Cv = load<T, D>(X, XG, q, lb[0], lb[1], lb[2]);
                    Bp += sg * (Cv - Av) / (T)8;
                }
                int dd[3] = {ii[0], ii[1], ii[2]};
                dd[d] = s ? n - 2 : 1;
                const T c = X[b.cell_off + cidx<D>(n, ii[0], ii[1], ii[2])];
                const T dv = X[b.cell_off + cidx<D>(n, dd[0], dd[1], dd[2])];
                val = (T)0.5 * Bp + (T)0.75 * c - (T)0.25 * dv;
            }
        }
        XG[b.ghost_off + face * F + u] = val;
    }
}

// --------------------------------------------------------- smoother -----
// One colour of red-black Gauss-Seidel (Sec. 2.2): cells with
// (I+J+K) % 2 == colour (global level indices) take the local solution
// (sum w x_nb - f) / (sum w + lambda).  Cells of the other colour and all
// ghosts are only read, so the update is order-independent.
template <class T, int D>
__global__ void __launch_bounds__(kMaxThreads) k_smooth(KParams P, int first, Fields<T> F, int colour) {
    const BlockDesc b = P.B[first + blockIdx.x];
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, C = cells_of<D>(n);
    const int par0 = (b.ijk[0] + b.ijk[1] + b.ijk[2]) * n;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        if (((par0 + i + j + k) & 1) != colour) continue;
        T lap, num, den, xc;
        stencil<T, T, D>(P, L, b, F.X, F.XG, F.E, F.EG, i, j, k, lap, num, den, xc);
        F.X[b.cell_off + c] = (num - F.F[b.cell_off + c]) / (den + (T)P.helm);
    }
}

// ------------------------------------------------------- transfers ------
// Restriction (Sec. 2.3): the parent cells under fine block b receive the
// mean of their 2^D children; with_res also stores the mean of the child
// residuals f - L x into the parent's right-hand side (first half of the
// coarse right-hand side of Sec. 2.4).
template <class T, int D>
__global__ void __launch_bounds__(kMaxThreads) k_restrict(KParams P, int first, T *__restrict__ X,
                                                          const T *__restrict__ XG, const T *__restrict__ Fr,
                                                          const T *__restrict__ E, const T *__restrict__ EG,
                                                          T *__restrict__ Fdst, int with_res) {
    const BlockDesc b = P.B[first + blockIdx.x];
    const LevelDesc &L = P.L[b.lev];
    const BlockDesc &p = P.B[b.parent];
    const int n = b.n, m = n / 2, M = cells_of<D>(m);
    for (int c = threadIdx.x; c < M; c += blockDim.x) {
        int ci, cj, ck;
        cell_of(c, m, D, ci, cj, ck);
        T sx = 0, sr = 0;
#pragma unroll 1
        for (int ch = 0; ch < (1 << D); ch++) {
            const int fi = 2 * ci + (ch & 1), fj = 2 * cj + ((ch >> 1) & 1), fk = D == 3 ? 2 * ck + ((ch >> 2) & 1) : 0;
            const int fc = cidx<D>(n, fi, fj, fk);
            sx += X[b.cell_off + fc];
            if (with_res) {
                T lap, num, den, xc;
                stencil<T, T, D>(P, L, b, X, XG, E, EG, fi, fj, fk, lap, num, den, xc);
                sr += Fr[b.cell_off + fc] - (lap - (T)P.helm * xc);
            }
        }
        const int pc = cidx<D>(p.n, b.poff[0] + ci, b.poff[1] + cj, b.poff[2] + ck);
        X[p.cell_off + pc] = sx / (T)(1 << D);
        if (with_res) Fdst[p.cell_off + pc] = sr / (T)(1 << D);
    }
}

// Covered cells: f^H = R(r^h) + L^H v^H (eq. for the coarse right-hand side).
template <class T, int D>
__global__ void __launch_bounds__(kMaxThreads) k_fas_rhs(KParams P, int first, Fields<T> F) {
    const BlockDesc b = P.B[first + blockIdx.x];
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, C = cells_of<D>(n);
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        T lap, num, den, xc;
        stencil<T, T, D>(P, L, b, F.X, F.XG, F.E, F.EG, i, j, k, lap, num, den, xc);
        F.F[b.cell_off + c] += lap - (T)P.helm * xc;
    }
}

// Coarse-grid correction (Sec. 2.4, Sec. 2.3): x^h += P(x^H - x^H_old), P the
// nearest-neighbour linear interpolation, 2D (2 c0 + c_x + c_y)/4, 3D
// (c0 + c_x + c_y + c_z)/4, neighbours on the fine cell's side (coarse
// ghosts included).
template <class T, int D>
__global__ void __launch_bounds__(kMaxThreads) k_prolong(KParams P, int first, Fields<T> F) {
    const BlockDesc b = P.B[first + blockIdx.x];
    const BlockDesc &p = P.B[b.parent];
    const int n = b.n, C = cells_of<D>(n);
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        const int I[3] = {b.ijk[0] * n + i, b.ijk[1] * n + j, b.ijk[2] * n + k};
        const int cc[3] = {b.poff[0] + i / 2, b.poff[1] + j / 2, D == 3 ? b.poff[2] + k / 2 : 0};
        const T c0 = load<T, D>(F.X, F.XG, p, cc[0], cc[1], cc[2]) - load<T, D>(F.V, F.VG, p, cc[0], cc[1], cc[2]);
        T nbs = 0;
#pragma unroll
        for (int d = 0; d < D; d++) {
            int q[3] = {cc[0], cc[1], cc[2]};
            q[d] += (I[d] & 1) ? 1 : -1;
            nbs += load<T, D>(F.X, F.XG, p, q[0], q[1], q[2]) - load<T, D>(F.V, F.VG, p, q[0], q[1], q[2]);
        }
        const T val = D == 2 ? ((T)2 * c0 + nbs) / (T)4 : (c0 + nbs) / (T)4;
        F.X[b.cell_off + c] += val;
    }
}

// ------------------------------------------------------ residual norm ---
// Composite residual on leaf blocks [first, first + gridDim.x): per-CTA
// partial sums of V r^2 and V and the max |r| (warp shuffles, then shared
// memory); optional r in leaf order and (float) r into FP32 cells.
template <int D>
__global__ void __launch_bounds__(kMaxThreads) k_resnorm(KParams P, int first, Fields<double> F,
                                                         double *__restrict__ partials,
                                                         double *__restrict__ rleaf, long long leaf_base,
                                                         long long cell_base, float *__restrict__ f32) {
    const BlockDesc b = P.B[first + blockIdx.x];
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, C = cells_of<D>(n);
    double s2 = 0, sv = 0, mx = 0;
    double vol = 1.0;
    for (int d = 0; d < D; d++) vol *= L.h[d];
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        double lap, num, den, xc;
        stencil<double, double, D>(P, L, b, F.X, F.XG, F.E, F.EG, i, j, k, lap, num, den, xc);
        const double r = F.F[b.cell_off + c] - (lap - P.helm * xc);
        double V = vol;
        if (P.geom == MG_CYL) V = 2.0 * M_PI * (P.lo[0] + (b.ijk[0] * n + i + 0.5) * L.h[0]) * L.h[0] * L.h[1];
        s2 += V * r * r;
        sv += V;
        mx = fmax(mx, fabs(r));
        if (rleaf) rleaf[leaf_base + (b.cell_off - cell_base) + c] = r;
        if (f32) f32[b.cell_off + c] = (float)r;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
        sv += __shfl_down_sync(0xffffffffu, sv, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    __shared__ double sh[3][kMaxThreads / 32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) { sh[0][w] = s2; sh[1][w] = sv; sh[2][w] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, bb = 0, m = 0;
        for (int e = 0; e < nw; e++) { a += sh[0][e]; bb += sh[1][e]; m = fmax(m, sh[2][e]); }
        partials[3 * blockIdx.x] = a;
        partials[3 * blockIdx.x + 1] = bb;
        partials[3 * blockIdx.x + 2] = m;
    }
}

__global__ void __launch_bounds__(1024) k_reduce3(const double *__restrict__ partials, int n, double *out) {
    double a = 0, b = 0, m = 0;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        a += partials[3 * e];
        b += partials[3 * e + 1];
        m = fmax(m, partials[3 * e + 2]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    __shared__ double sh[3][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][w] = a; sh[1][w] = b; sh[2][w] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0, z = 0;
        for (int e = 0; e < (int)((blockDim.x + 31) >> 5); e++) { x += sh[0][e]; y += sh[1][e]; z = fmax(z, sh[2][e]); }
        out[0] = x; out[1] = y; out[2] = z;
    }
}

// ------------------------------------------------------ coarsest level --
// Exact coarsest solve: r = f - L x in FP64 for every cell of level 0 (one
// CTA), with -sum V x appended for the zero-mean constraint; then
// dx = Minv r, one warp per row.
template <class T, int D>
__global__ void __launch_bounds__(1024) k_coarse_resid(KParams P, int nb, Fields<T> F, double *cvec, int singular) {
    const BlockDesc b0 = P.B[0];
    const LevelDesc &L = P.L[0];
    const int n = b0.n, C = cells_of<D>(n), nc = nb * C;
    double wx = 0;
    for (int row = threadIdx.x; row < nc; row += blockDim.x) {
        const BlockDesc &b = P.B[row / C];
        int i, j, k;
        cell_of(row % C, n, D, i, j, k);
        double lap, num, den, xc;
        stencil<double, T, D>(P, L, b, F.X, F.XG, F.E, F.EG, i, j, k, lap, num, den, xc);
        cvec[row] = (double)F.F[b.cell_off + row % C] - (lap - P.helm * xc);
        double V = 1.0;
        for (int d = 0; d < D; d++) V *= L.h[d];
        if (P.geom == MG_CYL) V = 2.0 * M_PI * (P.lo[0] + (b.ijk[0] * n + i + 0.5) * L.h[0]) * L.h[0] * L.h[1];
        wx += V * xc;
    }
    if (!singular) return;
    for (int o = 16; o > 0; o >>= 1) wx += __shfl_down_sync(0xffffffffu, wx, o);
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = wx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int e = 0; e < (int)((blockDim.x + 31) >> 5); e++) s += sh[e];
        cvec[nc] = -s;
    }
}

template <class T>
__global__ void k_coarse_apply(const double *__restrict__ minv, int ns, int nc, const double *__restrict__ cvec,
                               T *__restrict__ X) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= nc) return;
    double s = 0;
    for (int c = lane; c < ns; c += 32) s += minv[(long long)row * ns + c] * cvec[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) X[row] = (T)((double)X[row] + s);  // level-0 cells come first in the pool
}

// --------------------------------------------------- elementwise ops ----
__global__ void k_add_e(const float *__restrict__ e, double *__restrict__ x, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += (double)e[i];
}
__global__ void k_cast_f32(const double *__restrict__ a, float *__restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}
// leaf-order vector times (divide: 1/) r_i of its cell; leaf blocks of one level
template <int D>
__global__ void k_scale_r(KParams P, int first, const double *__restrict__ in, double *__restrict__ out,
                          long long leaf_base, int divide) {
    const BlockDesc b = P.B[first + blockIdx.x];
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, C = cells_of<D>(n);
    const long long base = leaf_base + (long long)blockIdx.x * C;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        const int i = c % n;
        const double r = P.lo[0] + (b.ijk[0] * n + i + 0.5) * L.h[0];
        out[base + c] = divide ? in[base + c] / r : in[base + c] * r;
    }
}

// dL/d eps_c = -sum over faces of lambda^T d(A phi + b)/d eps_f * d eps_f/d eps_c
// (harmonic face coefficient of Sec. 2.2); uniform meshes (no refinement faces).
template <int D>
__global__ void __launch_bounds__(kMaxThreads) k_eps_grad(KParams P, int first, const double *__restrict__ X,
                                                          const double *__restrict__ XG,
                                                          const double *__restrict__ Y, const double *__restrict__ YG,
                                                          const double *__restrict__ E, const double *__restrict__ EG,
                                                          double *__restrict__ out, long long leaf_base) {
    const BlockDesc b = P.B[first + blockIdx.x];
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, C = cells_of<D>(n);
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        const int I0 = b.ijk[0] * n + i;
        const double xc = X[b.cell_off + c], yc = Y[b.cell_off + c];
        const double ec = E ? E[b.cell_off + c] : 1.0;
        double g = 0;
        for (int d = 0; d < D; d++)
            for (int s = 0; s < 2; s++) {
                const int o = s ? 1 : -1;
                const int ii = i + (d == 0 ? o : 0), jj = j + (d == 1 ? o : 0), kk = k + (d == 2 ? o : 0);
                const double xo = load<double, D>(X, XG, b, ii, jj, kk);
                const bool outside = (d == 0 ? ii : d == 1 ? jj : kk) < 0 || (d == 0 ? ii : d == 1 ? jj : kk) >= n;
                const bool phys = outside && b.nbr[2 * d + s] == -1;
                double kc = 1.0, ko = 1.0;
                if (P.geom == MG_CYL && d == 0) {
                    const double rf = P.lo[0] + (I0 + s) * L.h[0];
                    const double rc = P.lo[0] + (I0 + 0.5) * L.h[0];
                    const double ro = P.lo[0] + (I0 + (s ? 1.5 : -0.5)) * L.h[0];
                    kc = rf / rc;
                    ko = rf / ro;
                }
                const double ih2 = L.inv_h2[d];
                double dA = yc * kc * ih2 * (xo - xc), de;
                if (phys) {
                    de = 1.0;
                } else {
                    const double yo = load<double, D>(Y, YG, b, ii, jj, kk);
                    const double eo = E ? load<double, D>(E, EG, b, ii, jj, kk) : 1.0;
                    dA += yo * ko * ih2 * (xc - xo);
                    const double sm = ec + eo;
                    de = 2.0 * eo * eo / (sm * sm);
                }
                g += -dA * de;
            }
        out[leaf_base + (long long)blockIdx.x * C + c] = g;
    }
}

// ------------------------------------------------------------ driver ----

KParams kparams(mg_tree *t, int homog) {
    KParams P;
    P.B = t->d_blocks;
    P.L = t->d_levels;
    P.bcplanes = t->d_bcplanes;
    for (int d = 0; d < 3; d++) P.lo[d] = t->lo[d];
    for (int f = 0; f < 6; f++) { P.bcv[f] = t->bc.value[f]; P.bct[f] = t->bc.type[f]; }
    P.helm = t->helm;
    P.geom = t->geom;
    P.var_eps = t->var_eps ? 1 : 0;
    P.homog = homog;
    return P;
}

static int threads_for(int cells) {
    int t = ((cells + 31) / 32) * 32;
    return t < 32 ? 32 : (t > kMaxThreads ? kMaxThreads : t);
}

template <class T, int D> struct Launch {
    static void ghost(mg_tree *t, const KParams &P, int l, T *X, T *XG, int mode) {
        const LevelHost &L = t->lev[l];
        if (L.nb == 0) return;
        ++t->launches;
        k_ghost<T, D><<<L.nb, threads_for(2 * D * face_of<D>(L.n)), 0, t->stream>>>(P, L.first, X, XG, mode);
    }
    static void smooth(mg_tree *t, const KParams &P, int l, Fields<T> &F, int sweeps) {
        const LevelHost &L = t->lev[l];
        const int th = threads_for(cells_of<D>(L.n));
        for (int s = 0; s < sweeps; s++)
            for (int colour = 0; colour < 2; colour++) {
                ++t->launches;
                k_smooth<T, D><<<L.nb, th, 0, t->stream>>>(P, L.first, F, colour);
                ghost(t, P, l, F.X, F.XG, 0);
            }
    }
    // downward FAS step from level l to l-1 (Sec. 2.4)
    static void restrict_fas(mg_tree *t, const KParams &P, int l, Fields<T> &F) {
        const LevelHost &L = t->lev[l], &C = t->lev[l - 1];
        ++t->launches;
        k_restrict<T, D><<<L.nb, threads_for(cells_of<D>(L.n / 2)), 0, t->stream>>>(P, L.first, F.X, F.XG, F.F,
                                                                                     F.E, F.EG, F.F, 1);
        ghost(t, P, l - 1, F.X, F.XG, 0);
        cudaMemcpyAsync(F.V + C.cell_first, F.X + C.cell_first, sizeof(T) * C.ncells, cudaMemcpyDeviceToDevice, t->stream);
        cudaMemcpyAsync(F.VG + C.ghost_first, F.XG + C.ghost_first, sizeof(T) * C.nghost, cudaMemcpyDeviceToDevice,
                        t->stream);
        if (C.nref > 0) {
            ++t->launches;
            k_fas_rhs<T, D><<<C.nref, threads_for(cells_of<D>(C.n)), 0, t->stream>>>(P, C.first, F);
        }
    }
    static void prolong(mg_tree *t, const KParams &P, int l, Fields<T> &F) {
        const LevelHost &L = t->lev[l];
        ++t->launches;
        k_prolong<T, D><<<L.nb, threads_for(cells_of<D>(L.n)), 0, t->stream>>>(P, L.first, F);
        ghost(t, P, l, F.X, F.XG, 0);
    }
    static void coarse(mg_tree *t, const KParams &P, Fields<T> &F) {
        const LevelHost &L = t->lev[0];
        ++t->launches;
        k_coarse_resid<T, D><<<1, 1024, 0, t->stream>>>(P, L.nb, F, t->d_cvec, t->singular ? 1 : 0);
        const int rows_per_cta = 8;
        ++t->launches;
        k_coarse_apply<T><<<(t->nc + rows_per_cta - 1) / rows_per_cta, 32 * rows_per_cta, 0, t->stream>>>(
            t->d_minv, t->ns, t->nc, t->d_cvec, F.X);
        ghost(t, P, 0, F.X, F.XG, 0);
    }
    static void vcycle(mg_tree *t, Fields<T> &F, int top, int nd, int nu, int homog) {
        const KParams P = kparams(t, homog);
        for (int l = top; l >= 1; l--) {
            smooth(t, P, l, F, nd);
            restrict_fas(t, P, l, F);
        }
        coarse(t, P, F);
        for (int l = 1; l <= top; l++) {
            prolong(t, P, l, F);
            smooth(t, P, l, F, nu);
        }
    }
    static void fmg(mg_tree *t, Fields<T> &F, int nd, int nu, int homog) {
        const KParams P = kparams(t, homog);
        const int top = (int)t->lev.size() - 1;
        for (int l = top; l >= 1; l--) restrict_fas(t, P, l, F);
        coarse(t, P, F);
        for (int l = 1; l <= top; l++) {
            prolong(t, P, l, F);
            vcycle(t, F, l, nd, nu, homog);
        }
    }
    // covered cells <- mean of children (finest first), then all ghosts
    static void refresh(mg_tree *t, Fields<T> &F, int homog) {
        const KParams P = kparams(t, homog);
        const int top = (int)t->lev.size() - 1;
        for (int l = top; l >= 1; l--) {
            const LevelHost &L = t->lev[l];
            ++t->launches;
            k_restrict<T, D><<<L.nb, threads_for(cells_of<D>(L.n / 2)), 0, t->stream>>>(P, L.first, F.X, F.XG, F.F,
                                                                                         F.E, F.EG, F.F, 0);
        }
        for (int l = 0; l <= top; l++) ghost(t, P, l, F.X, F.XG, 0);
    }
    static void refresh_eps(mg_tree *t, Fields<T> &F) {
        const KParams P = kparams(t, 0);
        const int top = (int)t->lev.size() - 1;
        for (int l = top; l >= 1; l--) {
            const LevelHost &L = t->lev[l];
            ++t->launches;
            k_restrict<T, D><<<L.nb, threads_for(cells_of<D>(L.n / 2)), 0, t->stream>>>(P, L.first, F.E, F.EG,
                                                                                         nullptr, nullptr, nullptr,
                                                                                         nullptr, 0);
        }
        for (int l = 0; l <= top; l++) ghost(t, P, l, F.E, F.EG, 1);
    }
};

template <class T> void vcycle(mg_tree *t, Fields<T> &F, int top, int nd, int nu, int homog) {
    if (t->dim == 2) Launch<T, 2>::vcycle(t, F, top, nd, nu, homog);
    else Launch<T, 3>::vcycle(t, F, top, nd, nu, homog);
}
template <class T> void fmg(mg_tree *t, Fields<T> &F, int nd, int nu, int homog) {
    if (t->dim == 2) Launch<T, 2>::fmg(t, F, nd, nu, homog);
    else Launch<T, 3>::fmg(t, F, nd, nu, homog);
}
template <class T> void refresh(mg_tree *t, Fields<T> &F, int homog) {
    if (t->dim == 2) Launch<T, 2>::refresh(t, F, homog);
    else Launch<T, 3>::refresh(t, F, homog);
}
template <class T> void refresh_eps(mg_tree *t, Fields<T> &F) {
    if (t->dim == 2) Launch<T, 2>::refresh_eps(t, F);
    else Launch<T, 3>::refresh_eps(t, F);
}
template void vcycle<double>(mg_tree *, Fields<double> &, int, int, int, int);
template void vcycle<float>(mg_tree *, Fields<float> &, int, int, int, int);
template void fmg<double>(mg_tree *, Fields<double> &, int, int, int);
template void fmg<float>(mg_tree *, Fields<float> &, int, int, int);
template void refresh<double>(mg_tree *, Fields<double> &, int);
template void refresh<float>(mg_tree *, Fields<float> &, int);
template void refresh_eps<double>(mg_tree *, Fields<double> &);
template void refresh_eps<float>(mg_tree *, Fields<float> &);

template <int D>
static void residual_norm_d(mg_tree *t, Fields<double> &F, int homog, double *out3, double *r64_leaf,
                            float *f32_cells) {
    Launch<double, D>::refresh(t, F, homog);
    const KParams P = kparams(t, homog);
    int slot = 0;
    long long leaf_base = 0;
    for (size_t l = 0; l < t->lev.size(); l++) {
        const LevelHost &L = t->lev[l];
        const int nleaf = L.nb - L.nref;
        if (nleaf <= 0) continue;
        const long long cell_base = t->blocks[L.first + L.nref].cell_off;
        ++t->launches;
        k_resnorm<D><<<nleaf, threads_for(cells_of<D>(L.n)), 0, t->stream>>>(
            P, L.first + L.nref, F, t->d_partials + 3 * slot, r64_leaf, leaf_base, cell_base, f32_cells);
        slot += nleaf;
        leaf_base += (long long)nleaf * cells_of<D>(L.n);
    }
    ++t->launches;
    k_reduce3<<<1, 1024, 0, t->stream>>>(t->d_partials, slot, t->d_red);
    cudaMemcpyAsync(t->h_red, t->d_red, 3 * sizeof(double), cudaMemcpyDeviceToHost, t->stream);
    cudaStreamSynchronize(t->stream);
    out3[0] = t->h_red[0];
    out3[1] = t->h_red[1];
    out3[2] = t->h_red[2];
}

void residual_norm(mg_tree *t, Fields<double> &F, int homog, double *out3, double *r64_leaf, float *f32_cells) {
    if (t->dim == 2) residual_norm_d<2>(t, F, homog, out3, r64_leaf, f32_cells);
    else residual_norm_d<3>(t, F, homog, out3, r64_leaf, f32_cells);
}

void add_e_to_phi(mg_tree *t, const float *e, double *phi) {
    ++t->launches;
    k_add_e<<<1216, 256, 0, t->stream>>>(e, phi, t->ncells);
}

void copy_eps_to_f32(mg_tree *t) {
    if (!t->f64.E || !t->f32.E) return;
    ++t->launches;
    k_cast_f32<<<1216, 256, 0, t->stream>>>(t->f64.E, t->f32.E, t->ncells);
    ++t->launches;
    k_cast_f32<<<1216, 256, 0, t->stream>>>(t->f64.EG, t->f32.EG, t->nghost);
}

void scale_by_radius(mg_tree *t, const double *in_leaf, double *out_leaf, int divide) {
    const KParams P = kparams(t, 0);
    long long leaf_base = 0;
    for (size_t l = 0; l < t->lev.size(); l++) {
        const LevelHost &L = t->lev[l];
        const int nleaf = L.nb - L.nref;
        if (nleaf <= 0) continue;
        ++t->launches;
        k_scale_r<2><<<nleaf, threads_for(L.n * L.n), 0, t->stream>>>(P, L.first + L.nref, in_leaf, out_leaf,
                                                                       leaf_base, divide);
        leaf_base += (long long)nleaf * L.n * L.n;
    }
}

void eps_grad(mg_tree *t, const double *lam_cells, const double *phi_cells, double *out_leaf) {
    (void)phi_cells;
    const KParams P = kparams(t, 0);
    const LevelHost &L = t->lev.back();
    const int nleaf = L.nb - L.nref;
    ++t->launches;
    if (t->dim == 2)
        k_eps_grad<2><<<nleaf, threads_for(cells_of<2>(L.n)), 0, t->stream>>>(
            P, L.first + L.nref, t->f64.X, t->f64.XG, lam_cells, t->adj.XG, t->f64.E, t->f64.EG, out_leaf, 0);
    else
        k_eps_grad<3><<<nleaf, threads_for(cells_of<3>(L.n)), 0, t->stream>>>(
            P, L.first + L.nref, t->f64.X, t->f64.XG, lam_cells, t->adj.XG, t->f64.E, t->f64.EG, out_leaf, 0);
}

template <int D>
static int time_sweeps_d(mg_tree *t, int level, int n_sweeps, double *out) {
    const KParams P = kparams(t, 0);
    const LevelHost &L = t->lev[level];
    const int th = threads_for(cells_of<D>(L.n));
    std::vector<cudaEvent_t> ev(8 * n_sweeps);
    for (auto &e : ev) cudaEventCreate(&e);
    int m = 0;
    for (int s = 0; s < n_sweeps; s++)
        for (int colour = 0; colour < 2; colour++) {
            cudaEventRecord(ev[m++], t->stream);
            ++t->launches;
            k_smooth<double, D><<<L.nb, th, 0, t->stream>>>(P, L.first, t->f64, colour);
            cudaEventRecord(ev[m++], t->stream);
            cudaEventRecord(ev[m++], t->stream);
            Launch<double, D>::ghost(t, P, level, t->f64.X, t->f64.XG, 0);
            cudaEventRecord(ev[m++], t->stream);
        }
    cudaStreamSynchronize(t->stream);
    double ts = 0, tg = 0;
    for (int i = 0; i < m; i += 4) {
        float a = 0, b = 0;
        cudaEventElapsedTime(&a, ev[i], ev[i + 1]);
        cudaEventElapsedTime(&b, ev[i + 2], ev[i + 3]);
        ts += a;
        tg += b;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    const int nl = 2 * n_sweeps;
    const double cells = (double)L.nb * cells_of<D>(L.n), ghosts = (double)L.nb * 2 * D * face_of<D>(L.n);
    const double per = t->var_eps ? 32.0 : 24.0;
    out[0] = ts / nl;
    out[1] = tg / nl;
    out[2] = cells * per + ghosts * (t->var_eps ? 16.0 : 8.0);
    out[3] = ghosts * 16.0;
    return MG_OK;
}

int time_sweeps(mg_tree *t, int level, int n_sweeps, double *out4) {
    return t->dim == 2 ? time_sweeps_d<2>(t, level, n_sweeps, out4) : time_sweeps_d<3>(t, level, n_sweeps, out4);
}

int check_cuda(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        mg_set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    return MG_OK;
}

}  // namespace mg
