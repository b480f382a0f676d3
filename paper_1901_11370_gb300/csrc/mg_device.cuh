// mg_device.cuh -- device helpers shared by the kernel translation units
// (mg_kernels.cu: cycles and solver kernels; mg_adjoint.cu: the transposed
// operators).  Block and level descriptors, indexing of cells and face
// ghosts, the 5/7-point row, the ghost rules of Sec. 2.6 and the launch
// helper.  Not part of the public ABI.
#pragma once
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>

#include "mg_internal.h"

namespace mg {

static constexpr int kMaxThreads = 256;

template <int D> __host__ __device__ constexpr int cells_of(int n) { return D == 2 ? n * n : n * n * n; }
template <int D> __host__ __device__ constexpr int face_of(int n) { return D == 2 ? n : n * n; }
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

// Programmatic dependent launch: every kernel first waits for the grid it
// depends on to complete (stream order is kept exactly), then lets the next
// grid start launching, so launch latency overlaps the tail of this one.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Every launch goes through launch_k: plainly, or with the
// programmatic-serialization attribute when MG_PDL=1 (the kernel's pdl_entry
// keeps the stream order).  Off by default: inside CUDA graphs it measured
// slower on GB300 (20.0 vs 19.7 ms mixed, 44 vs 39 ms FP64 on the 20M-unknown
// tree) -- the early dependent CTAs compete with the tail of the running grid.
static int pdl_mode() {
    static int mode = [] {
        const char *e = std::getenv("MG_PDL");
        return (e && e[0] == '1') ? 1 : 0;
    }();
    return mode;
}
static bool g_pdl_ok = true;
// first failed kernel launch since the last check_cuda (0: none), with the
// kernel and configuration it was launched with
inline std::atomic<int> g_launch_error{0};
struct LaunchFail {
    const void *kern;
    unsigned grid, block;
    size_t smem;
};
inline LaunchFail g_launch_fail{};
template <class... KArgs, class... Args>
static void launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (pdl_mode() && g_pdl_ok) ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
    if (e != cudaSuccess && cfg.numAttrs) {
        cudaGetLastError();  // attribute refused: plain launches from now on
        g_pdl_ok = false;
        cfg.numAttrs = 0;
        e = cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
    }
    if (e != cudaSuccess) {  // kept until check_cuda reports it (a capture would otherwise drop it)
        int none = 0;
        if (g_launch_error.compare_exchange_strong(none, (int)e))
            g_launch_fail = {(const void *)kern, grid.x, block.x, smem};
    }
}

// A cooperative launch (every CTA resident at once, as a grid barrier
// needs); a refused launch is kept for check_cuda like launch_k's.
template <class... KArgs, class... Args>
static void launch_coop(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
    if (e != cudaSuccess) {
        int none = 0;
        if (g_launch_error.compare_exchange_strong(none, (int)e))
            g_launch_fail = {(const void *)kern, grid.x, block.x, 0};
    }
}

// Quotient for the operator's coefficients and the Gauss-Seidel update: the
// FP32 smoother (an inner solver under FP64 defect correction) takes the
// fast reciprocal-based intrinsic; FP64 keeps the correctly rounded division.
template <class T> __device__ __forceinline__ T qdiv(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float qdiv<float>(float a, float b) { return __fdividef(a, b); }

// Level and launch scalars in the kernel precision (FP32 copies are stored,
// so FP32 kernels never convert from double).
template <class T> __device__ __forceinline__ T lv_ih(const LevelDesc &L, int d) { return (T)L.inv_h2[d]; }
template <> __device__ __forceinline__ float lv_ih<float>(const LevelDesc &L, int d) { return L.inv_h2f[d]; }
template <class T> __device__ __forceinline__ T lv_idiag(const LevelDesc &L) { return (T)L.inv_diag; }
template <> __device__ __forceinline__ float lv_idiag<float>(const LevelDesc &L) { return L.inv_diagf; }
template <class T> __device__ __forceinline__ T lv_h0(const LevelDesc &L) { return (T)L.h[0]; }
template <> __device__ __forceinline__ float lv_h0<float>(const LevelDesc &L) { return L.h0f; }
template <class T> __device__ __forceinline__ T kp_lo0(const KParams &P) { return (T)P.lo[0]; }
template <> __device__ __forceinline__ float kp_lo0<float>(const KParams &P) { return P.lo0f; }
template <class T> __device__ __forceinline__ T kp_helm(const KParams &P) { return (T)P.helm; }
template <> __device__ __forceinline__ float kp_helm<float>(const KParams &P) { return P.helmf; }

// threads per CTA of the TMA sweep for NCOL colour cells per block
// Largest CTA of the staged transfer kernels (restriction, prolongation,
// FAS right-hand side, ghost fill): 3D 16^3 blocks run one 512-thread CTA
// per SM, every other block size at most kMaxThreads.
__host__ __device__ constexpr int transfer_bound(int D, int NT) {
    return (D == 3 && NT == 16) ? 2 * kMaxThreads : kMaxThreads;
}

// Threads of the staged sweep for a block of 2 ncol cells: one per colour
// cell up to kMaxThreads; 3D 16^3 blocks (2048 colour cells), whose
// double-buffered stage leaves room for one CTA per SM, take twice that.
__host__ __device__ constexpr int sweep_tma_threads(int ncol, bool half) {
    const int cap = ncol >= 2048 ? 2 * kMaxThreads : kMaxThreads;
    const int full = ncol < 32 ? 32 : (ncol > cap ? cap : ncol);
    return half ? (full / 2 < 32 ? 32 : full / 2) : full;
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
    const A lo0 = kp_lo0<A>(P), h0 = lv_h0<A>(L);
    if (P.geom == MG_CYL) ri = lo0 + ((A)(b.ijk[0] * n + i) + (A)0.5) * h0;
#pragma unroll
    for (int d = 0; d < D; d++) {
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int o = s ? 1 : -1;
            const int ii = i + (d == 0 ? o : 0), jj = j + (d == 1 ? o : 0), kk = k + (d == 2 ? o : 0);
            const A xn = (A)load<T, D>(X, XG, b, ii, jj, kk);
            A w = lv_ih<A>(L, d);
            if (E) {
                const A en = (A)load<T, D>(E, EG, b, ii, jj, kk);
                w *= qdiv<A>((A)2 * ec * en, ec + en);
            }
            if (P.geom == MG_CYL && d == 0) {
                const A rf = lo0 + (A)(b.ijk[0] * n + i + s) * h0;
                w *= qdiv<A>(rf, ri);
            }
            lap += w * (xn - xc);
            num += w * xn;
            den += w;
        }
    }
}

// The FP64 operator from the precomputed face coefficients W (variable eps
// or the cylindrical form; wstride(D) slots per cell, [slot][cell] within
// a block: the 2D face weights in face order, the diagonal -- the weights'
// sum plus lambda -- and its reciprocal), in the difference form of
// `stencil`: lap = sum_f w_f (x_f - x_c), the same terms in the same order
// as the on-the-fly form (whose weights W holds), so the result is the
// same and its rounding stays at eps |w| |x_f - x_c|.  No division: GB300
// spends about ten FP64 instructions on one, and the on-the-fly harmonic
// means take six per cell.
template <int D>
__device__ __forceinline__ double lap_w(const BlockDesc &b, const double *X, const double *XG, const double *W,
                                        int i, int j, int k, double xc) {
    const int n = b.n, C = cells_of<D>(n);
    const double *ws = W + b.cell_off * wstride(D) + cidx<D>(n, i, j, k);
    double lap = 0;
    lap += ws[0] * (load<double, D>(X, XG, b, i - 1, j, k) - xc);
    lap += ws[C] * (load<double, D>(X, XG, b, i + 1, j, k) - xc);
    lap += ws[2 * C] * (load<double, D>(X, XG, b, i, j - 1, k) - xc);
    lap += ws[3 * C] * (load<double, D>(X, XG, b, i, j + 1, k) - xc);
    if (D == 3) {
        lap += ws[4 * C] * (load<double, D>(X, XG, b, i, j, k - 1) - xc);
        lap += ws[5 * C] * (load<double, D>(X, XG, b, i, j, k + 1) - xc);
    }
    return lap;
}

__device__ __forceinline__ void cell_of(int c, int n, int D, int &i, int &j, int &k) {
    i = c % n;
    j = (c / n) % n;
    k = D == 3 ? c / (n * n) : 0;
}

// Small integer triple handled with selects (no dynamically indexed arrays,
// which would live in local memory).
struct I3 {
    int x, y, z;
};
__device__ __forceinline__ int get(const I3 &v, int d) { return d == 0 ? v.x : (d == 1 ? v.y : v.z); }
__device__ __forceinline__ void put(I3 &v, int d, int val) {
    v.x = d == 0 ? val : v.x;
    v.y = d == 1 ? val : v.y;
    v.z = d == 2 ? val : v.z;
}
// interior cell beside face cell u of face `face` (ghost side when ghost)
template <int D> __device__ __forceinline__ I3 face_cell(int n, int face, int u, bool ghost) {
    const int d = face >> 1, s = face & 1, a = u % n, c = u / n;
    const int e = ghost ? (s ? n : -1) : (s ? n - 1 : 0);
    if (D == 2) return d == 0 ? I3{e, a, 0} : I3{a, e, 0};
    return d == 0 ? I3{e, a, c} : (d == 1 ? I3{a, e, c} : I3{a, c, e});
}

// Copy of the CTA's block descriptor in shared memory.
__device__ __forceinline__ void stage_desc(const KParams &P, int g, BlockDesc &sb) {
    static_assert(sizeof(BlockDesc) % 4 == 0, "descriptor copied as words");
    if (threadIdx.x < sizeof(BlockDesc) / 4)
        reinterpret_cast<int *>(&sb)[threadIdx.x] = reinterpret_cast<const int *>(P.B + g)[threadIdx.x];
    __syncthreads();
}

// Boundary value a (Dirichlet) or b (Neumann) of physical face `face` at
// the face cell beside interior cell ii of block b.
__device__ __forceinline__ double bc_value(const KParams &P, const LevelDesc &L, const BlockDesc &b, int D,
                                           int face, I3 ii) {
    if (P.homog) return 0.0;
    if (L.bc_off[face] < 0) return P.bcv[face];
    const int d = face >> 1, n = b.n;
    const int t1 = d == 0 ? 1 : 0, t2 = D == 2 ? -1 : (d == 2 ? 1 : 2);
    long long idx = b.ijk[t1] * n + get(ii, t1);
    if (t2 >= 0) idx += (long long)L.ncell[t1] * (b.ijk[t2] * n + get(ii, t2));
    return P.bcplanes[L.bc_off[face] + idx];
}

// Physical-boundary ghost (Sec. 2.6): Dirichlet 2a - x_i, Neumann
// x_i -/+ h b on the low/high face, axis x_i.
template <class T>
__device__ __forceinline__ T phys_ghost(const KParams &P, const LevelDesc &L, int face, T xi, double a) {
    const int d = face >> 1, s = face & 1;
    switch (P.bct[face]) {  // homogeneous values (correction cycles): no FP64 work
    case MG_BC_DIRICHLET: return P.homog ? -xi : (T)(2.0 * a) - xi;
    case MG_BC_NEUMANN: return P.homog ? xi : (s ? xi + (T)(L.h[d] * a) : xi - (T)(L.h[d] * a));
    default: return xi;
    }
}

// Refinement-boundary ghost of fine block b on face `face` beside interior
// cell ii (Sec. 2.6): B' = B + sum_t s_t (C_t - A_t)/8 from the coarser
// neighbour q (its own ghosts supply A_t / C_t outside q), then
// g = B'/2 + 3c/4 - d/4 with c = x(ii) and d the next cell inwards.  With
// coef set, the coefficient ghost is B itself.
template <class T, int D>
__device__ __forceinline__ T cf_ghost(const KParams &P, const LevelDesc &L, const BlockDesc &b, int face, I3 ii,
                                      T c, T dv, const T *__restrict__ X, const T *__restrict__ XG, int nbcode,
                                      bool coef) {
    const BlockDesc &q = P.B[-2 - nbcode];
    const int n = b.n, qn = q.n, d = face >> 1, s = face & 1;
    I3 G{b.ijk[0] * n + ii.x, b.ijk[1] * n + ii.y, b.ijk[2] * n + ii.z};
    int gd = b.ijk[d] * n + (s ? n : -1);
    const int nd = L.ncell[d];
    gd = gd < 0 ? gd + nd : (gd >= nd ? gd - nd : gd);
    put(G, d, gd);
    const I3 lc{(G.x >> 1) - q.ijk[0] * qn, (G.y >> 1) - q.ijk[1] * qn, D == 3 ? (G.z >> 1) - q.ijk[2] * qn : 0};
    const T B = X[q.cell_off + cidx<D>(qn, lc.x, lc.y, lc.z)];
    if (coef) return B;
    T Bp = B;
#pragma unroll
    for (int e = 0; e < D; e++) {
        if (e == d) continue;
        const T sg = (get(G, e) & 1) ? (T)1 : (T)-1;
        const int ox = e == 0, oy = e == 1, oz = e == 2;
        const T Av = load<T, D>(X, XG, q, lc.x - ox, lc.y - oy, lc.z - oz);
        const T Cv = load<T, D>(X, XG, q, lc.x + ox, lc.y + oy, lc.z + oz);
        Bp += sg * (Cv - Av) / (T)8;
    }
    return (T)0.5 * Bp + (T)0.75 * c - (T)0.25 * dv;
}


}  // namespace mg
