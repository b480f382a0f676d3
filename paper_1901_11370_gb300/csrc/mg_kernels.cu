// mg_kernels.cu -- sm_103a kernels and the cycle driver of the octree
// geometric multigrid (Teunissen & Keppens, arXiv:1901.11370).
//
// Every kernel works on a contiguous range of global block ids (one level,
// or its covered / leaf part) with one CTA per block.  Fields are stored
// interior-only, block-major (x fastest), plus a face-ghost array (see
// BlockDesc).  The 5/7-point stencil is memory-bound, so nothing here uses
// tensor cores: the kernels are written for coalesced HBM access of whole
// blocks, with neighbour faces served by L1/L2.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <mutex>
#include <string>
#include <cstdio>
#include <vector>

#include "mg_internal.h"
#include "mg_device.cuh"
#include "mg_exact.h"

namespace mg {

// A sweep changes neither the coarse level nor, before its ghost pushes, the
// interior values that the current coarse-fine ghost g = B'/2 + 3c/4 - d/4
// was formed with.  It therefore recovers B'/2 from g and the old (c, d)
// and forms the new ghost from B'/2 and the new (c, d), with no reads of the
// coarser block.  The two agree with cf_ghost up to rounding.
template <class T> __device__ __forceinline__ T cf_half_base(T g, T c, T dv) {
    return g - (T)0.75 * c + (T)0.25 * dv;
}
template <class T> __device__ __forceinline__ T cf_from_half_base(T bh, T c, T dv) {
    return bh + (T)0.75 * c - (T)0.25 * dv;
}
// bit f set: face f of the block borders a coarser block
__device__ __forceinline__ int cf_faces(const BlockDesc &b, int D) {
    int m = 0;
    for (int f = 0; f < 2 * D; f++) m |= (b.nbr[f] <= -2) << f;
    return m;
}

// ------------------------------------------------------------- ghosts ----
// Face ghosts of every block in [first, first + gridDim.x) (Sec. 2.6):
// same-level or periodic copy; physical boundary (Dirichlet 2a - x_i,
// Neumann x_i -/+ h b, axis x_i); refinement boundary
// g = B'/2 + 3c/4 - d/4 with B' = B + sum_t s_t (C_t - A_t)/8 read from the
// coarser block and its own ghosts.  mode 1 (coefficient): physical ghosts
// copy the interior value, refinement ghosts take B.  mode 2 (a vector
// component): physical ghosts copy the interior value, refinement ghosts
// are interpolated as for phi.
template <class T, int D>
__global__ void __launch_bounds__(kMaxThreads) k_ghost(KParams P, int first, T *__restrict__ X,
                                                       T *__restrict__ XG, int mode) {
    pdl_entry();
    __shared__ BlockDesc sb;
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, F = face_of<D>(n);
    for (int t = threadIdx.x; t < 2 * D * F; t += blockDim.x) {
        const int face = t / F, u = t - face * F, d = face >> 1, s = face & 1;
        const I3 ii = face_cell<D>(n, face, u, false);
        const int nb = b.nbr[face];
        T val;
        if (nb >= 0) {
            const BlockDesc &q = P.B[nb];
            I3 jj = ii;
            put(jj, d, s ? 0 : n - 1);
            val = X[q.cell_off + cidx<D>(n, jj.x, jj.y, jj.z)];
        } else if (nb == -1) {
            const T xi = X[b.cell_off + cidx<D>(n, ii.x, ii.y, ii.z)];
            val = mode >= 1 ? xi : phys_ghost<T>(P, L, face, xi, bc_value(P, L, b, D, face, ii));
        } else {
            I3 dd = ii;
            put(dd, d, s ? n - 2 : 1);
            const T c = X[b.cell_off + cidx<D>(n, ii.x, ii.y, ii.z)];
            const T dv = X[b.cell_off + cidx<D>(n, dd.x, dd.y, dd.z)];
            val = cf_ghost<T, D>(P, L, b, face, ii, c, dv, X, XG, nb, mode == 1);
        }
        XG[b.ghost_off + face * F + u] = val;
    }
}

// --------------------------------------------------------- smoother -----
// Fused red-black half-sweep: one CTA per block.
//  1. the block and its face ghosts (and eps) are staged in shared memory,
//     padded to (n+2)^D;
//  2. every cell of the colour (one thread per colour cell) takes the local
//     solution from its neighbours in shared memory; the block is written
//     back whole with coalesced stores;
//  3. the ghosts that depend on the updated cells are pushed: a same-level
//     neighbour's ghost slot opposite an updated boundary cell, the block's
//     own physical ghosts beside updated cells, and all its refinement-face
//     ghosts (c or d changed).
// The ghost state after the launch equals a full ghost fill of the level
// after the colour (reading R1 of the oracle).  A CTA reads only ghost
// slots beside cells of the updated colour, i.e. slots fed by the other
// colour of its neighbours, so reads and pushes of concurrent CTAs never
// touch the same slot.
template <class T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

// 16-byte vector <-> VW consecutive shared-memory elements
template <class T> __device__ __forceinline__ void vscatter(T *dst, const typename Vec16<T>::type &v) {
    if constexpr (sizeof(T) == 4) { dst[0] = v.x; dst[1] = v.y; dst[2] = v.z; dst[3] = v.w; }
    else { dst[0] = v.x; dst[1] = v.y; }
}
template <class T> __device__ __forceinline__ typename Vec16<T>::type vgather(const T *src) {
    if constexpr (sizeof(T) == 4) return make_float4(src[0], src[1], src[2], src[3]);
    else return make_double2(src[0], src[1]);
}

template <class T, int D, int NT>
__global__ void __launch_bounds__(kMaxThreads) k_sweep(KParams P, int first, Fields<T> F, int colour) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockDesc sb;
    __shared__ long long s_ngo[6];
    const int tid = threadIdx.x, nth = blockDim.x;
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
    if (tid < 2 * D) {
        const int nb = b.nbr[tid];
        s_ngo[tid] = nb >= 0 ? P.B[nb].ghost_off : -1;
    }
    const LevelDesc &L = P.L[b.lev];
    const T lo0 = kp_lo0<T>(P), h0 = lv_h0<T>(L);  // operator scalars in the kernel precision
    const T ih0 = lv_ih<T>(L, 0), ih1 = lv_ih<T>(L, 1), ih2 = lv_ih<T>(L, 2);
    const int n = NT ? NT : b.n;
    const int C = cells_of<D>(n), Fc = face_of<D>(n), S = n + 2;
    const int PAD = D == 2 ? S * S : S * S * S;
    T *sx = reinterpret_cast<T *>(smem_raw);
    T *se = sx + PAD;
    const bool var = F.E != nullptr;
    const int sy = S, sz = D == 3 ? S * S : 0;
    auto sid = [&](int i, int j, int k) { return (D == 3 ? (k + 1) * sz : 0) + (j + 1) * sy + (i + 1); };
    const int par0 = (b.ijk[0] + b.ijk[1] + b.ijk[2]) * n;
    const int ncol = (n & 1) ? C : C / 2;
    constexpr int VW = 16 / sizeof(T);
    constexpr int CPT = NT ? ((cells_of<D>(NT) / 2 + kMaxThreads - 1) / kMaxThreads) : 1;

    // 1. stage block + ghosts (+ eps), prefetch f of this thread's colour cells
    if (NT) {
        using V = typename Vec16<T>::type;
        const V *src = reinterpret_cast<const V *>(F.X + b.cell_off);
        for (int v = tid; v < C / VW; v += nth) {
            const int c = v * VW, i = c % n, j = (c / n) % n, k = D == 3 ? c / (n * n) : 0;
            vscatter<T>(sx + sid(i, j, k), src[v]);
        }
        const V *gsrc = reinterpret_cast<const V *>(F.XG + b.ghost_off);
        for (int v = tid; v < 2 * D * Fc / VW; v += nth) {
            const V val = gsrc[v];
            const int t0 = v * VW, face = t0 / Fc, u0 = t0 - face * Fc;
            const int step = (face >> 1) == 0 ? sy : 1;  // consecutive u: next t1 cell
            const I3 q = face_cell<D>(n, face, u0, true);
            T *dst = sx + sid(q.x, q.y, q.z);
            if constexpr (sizeof(T) == 4) { dst[0] = val.x; dst[step] = val.y; dst[2 * step] = val.z; dst[3 * step] = val.w; }
            else { dst[0] = val.x; dst[step] = val.y; }
        }
    } else {
        for (int c = tid; c < C; c += nth) {
            const int i = c % n, j = (c / n) % n, k = D == 3 ? c / (n * n) : 0;
            sx[sid(i, j, k)] = F.X[b.cell_off + c];
        }
        for (int t = tid; t < 2 * D * Fc; t += nth) {
            const I3 q = face_cell<D>(n, t / Fc, t % Fc, true);
            sx[sid(q.x, q.y, q.z)] = F.XG[b.ghost_off + t];
        }
    }
    if (var && !F.W) {
        for (int c = tid; c < C; c += nth) {
            const int i = c % n, j = (c / n) % n, k = D == 3 ? c / (n * n) : 0;
            se[sid(i, j, k)] = F.E[b.cell_off + c];
        }
        for (int t = tid; t < 2 * D * Fc; t += nth) {
            const I3 q = face_cell<D>(n, t / Fc, t % Fc, true);
            se[sid(q.x, q.y, q.z)] = F.EG[b.ghost_off + t];
        }
    }
    // colour cell qi -> (i, j, k)
    auto colour_cell = [&](int qi, int &i, int &j, int &k) -> bool {
        if (n & 1) {
            i = qi % n; j = (qi / n) % n; k = D == 3 ? qi / (n * n) : 0;
            return ((par0 + i + j + k) & 1) == colour;
        }
        const int h = n >> 1, rr = qi / h, m = qi - rr * h;
        j = rr % n;
        k = D == 3 ? rr / n : 0;
        i = 2 * m + ((colour + par0 + j + k) & 1);
        return true;
    };
    int ci[CPT], cj[CPT], ck[CPT];
    T fpre[CPT];
    if (NT) {
#pragma unroll
        for (int r = 0; r < CPT; r++) {
            const int qi = tid + r * nth;
            ci[r] = -1;
            if (qi >= ncol) continue;
            int i, j, k;
            if (!colour_cell(qi, i, j, k)) continue;
            ci[r] = i; cj[r] = j; ck[r] = k;
            fpre[r] = F.F[b.cell_off + cidx<D>(n, i, j, k)];
        }
    }
    __syncthreads();

    // 2. red-black update of this colour (Sec. 2.2)
    const bool cyl = P.geom == MG_CYL;
    const T helm = kp_helm<T>(P);
    const T w0 = lv_ih<T>(L, 0), w1 = lv_ih<T>(L, 1), w2 = lv_ih<T>(L, 2);
    const T inv_den = (T)1 / ((T)2 * (w0 + w1 + (D == 3 ? w2 : (T)0)) + helm);
    const T *W = F.W;  // FP64 face coefficients (variable eps or cylindrical form), else null
    auto update = [&](int i, int j, int k, T fc) {
        const int c0 = sid(i, j, k);
        T xnew;
        if (W) {  // the coefficients and 1 / diagonal precomputed: no division
            const T *ws = W + b.cell_off * wstride(D) + cidx<D>(n, i, j, k);
            T num = ws[0] * sx[c0 - 1];
            num += ws[C] * sx[c0 + 1];
            num += ws[2 * C] * sx[c0 - sy];
            num += ws[3 * C] * sx[c0 + sy];
            if (D == 3) {
                num += ws[4 * C] * sx[c0 - sz];
                num += ws[5 * C] * sx[c0 + sz];
            }
            xnew = (num - fc) * ws[(2 * D + 1) * C];
        } else if (!var && !cyl) {
            T num = w0 * (sx[c0 - 1] + sx[c0 + 1]) + w1 * (sx[c0 - sy] + sx[c0 + sy]);
            if (D == 3) num += w2 * (sx[c0 - sz] + sx[c0 + sz]);
            xnew = (num - fc) * inv_den;
        } else {
            const T ec = var ? se[c0] : (T)1;
            T num = 0, den = 0, ri = 0;
            if (cyl) ri = lo0 + ((T)(b.ijk[0] * n + i) + (T)0.5) * h0;
#pragma unroll
            for (int d = 0; d < D; d++)
#pragma unroll
                for (int s = 0; s < 2; s++) {
                    const int o = (s ? 1 : -1) * (d == 0 ? 1 : d == 1 ? sy : sz);
                    T w = d == 0 ? ih0 : (d == 1 ? ih1 : ih2);
                    if (var) {
                        const T en = se[c0 + o];
                        w *= qdiv<T>((T)2 * ec * en, ec + en);
                    }
                    if (cyl && d == 0) w *= qdiv<T>(lo0 + (T)(b.ijk[0] * n + i + s) * h0, ri);
                    num += w * sx[c0 + o];
                    den += w;
                }
            xnew = qdiv<T>(num - fc, den + helm);
        }
        sx[c0] = xnew;
    };
    if (NT) {
#pragma unroll
        for (int r = 0; r < CPT; r++)
            if (ci[r] >= 0) update(ci[r], cj[r], ck[r], fpre[r]);
    } else {
        for (int qi = tid; qi < ncol; qi += nth) {
            int i, j, k;
            if (colour_cell(qi, i, j, k)) update(i, j, k, F.F[b.cell_off + cidx<D>(n, i, j, k)]);
        }
    }
    __syncthreads();

    // 3. write the block back, push the ghosts that depend on updated cells
    if (NT) {
        using V = typename Vec16<T>::type;
        V *dst = reinterpret_cast<V *>(F.X + b.cell_off);
        for (int v = tid; v < C / VW; v += nth) {
            const int c = v * VW, i = c % n, j = (c / n) % n, k = D == 3 ? c / (n * n) : 0;
            dst[v] = vgather<T>(sx + sid(i, j, k));
        }
    } else {
        for (int c = tid; c < C; c += nth) {
            const int i = c % n, j = (c / n) % n, k = D == 3 ? c / (n * n) : 0;
            F.X[b.cell_off + c] = sx[sid(i, j, k)];
        }
    }
    for (int t = tid; t < 2 * D * Fc; t += nth) {
        const int face = t / Fc, u = t - face * Fc, d = face >> 1, s = face & 1;
        const I3 ii = face_cell<D>(n, face, u, false);
        const bool updated = ((par0 + ii.x + ii.y + ii.z) & 1) == colour;
        const int nb = b.nbr[face];
        const T xi = sx[sid(ii.x, ii.y, ii.z)];
        if (nb >= 0) {
            if (updated) F.XG[s_ngo[face] + (face ^ 1) * Fc + u] = xi;
        } else if (nb == -1) {
            if (updated) F.XG[b.ghost_off + t] = phys_ghost<T>(P, L, face, xi, bc_value(P, L, b, D, face, ii));
        } else {
            I3 dd = ii;
            put(dd, d, s ? n - 2 : 1);
            F.XG[b.ghost_off + t] = cf_ghost<T, D>(P, L, b, face, ii, xi, sx[sid(dd.x, dd.y, dd.z)], F.X, F.XG, nb,
                                                   false);
        }
    }
}

// ------------------------------------------------ TMA bulk-copy sweep ---
// Persistent variant of the fused sweep for 8- and 16-cell blocks.  Each
// CTA walks blocks g = blockIdx.x, + gridDim.x, ...; the interior, the face
// ghosts, f (and eps) of the next block arrive by cp.async.bulk into the
// other half of a double buffer while the current block is updated; the
// updated interior leaves by a bulk store.  Every mbarrier wait is bounded:
// on expiry the kernel raises P.status and the CTA stops.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Right-hand sides and coefficients (eps and its ghosts) of the FP32 cycles
// are read-only during smoothing and read once per colour launch: they are
// the largest arrays a sweep streams.  Their lines are marked evict-first
// in L2, so that on a level whose fields together exceed L2 the level's x
// and ghost slots stay resident between the launches of a smoothing phase
// instead of being streamed out by f and eps.  FP64 fields are left at the
// default policy.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
template <class T> __device__ __forceinline__ void bulk_g2s_f(void *dst, const T *src, uint32_t bytes, uint64_t *bar) {
    if constexpr (sizeof(T) == 4) {
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
                smem_u32(dst)),
            "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(l2_evict_first())
            : "memory");
    } else {
        bulk_g2s(dst, src, bytes, bar);
    }
}
__device__ __forceinline__ float4 ldg_f_ef(const float4 *p, uint64_t pol) {
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

static constexpr uint32_t kWaitLimit = kDefaultWaitLimit;

// Bounded wait on an mbarrier phase: true once it completed, false after
// `limit` polls (limit 0 gives up at once; a test setting of the tree).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t tries = 0; tries < limit; tries++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// HALF: half as many threads per CTA (two colour cells each), which wastes
// less at the CTA barriers on levels with few blocks per SM.
template <class T, int D, int NT, bool HALF = false>
__global__ void __launch_bounds__(sweep_tma_threads(cells_of<D>(NT) / 2, HALF), (D == 3 && NT == 16) ? 1 : 5) k_sweep_tma(KParams P, int first, int nblocks, Fields<T> F,
                                                           int colour) {
    pdl_entry();
    constexpr int n = NT, C = cells_of<D>(NT), FC = face_of<D>(NT), GH = 2 * D * FC;
    constexpr int NCOL = C / 2, TPB = sweep_tma_threads(NCOL, HALF), CPT = (NCOL + TPB - 1) / TPB;
    constexpr int GPT = (GH + TPB - 1) / TPB;  // ghost slots per thread (launched with TPB threads)
    constexpr int DESC = (int)((sizeof(BlockDesc) + sizeof(LevelDesc)) / sizeof(T));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ __align__(16) LevelDesc sL;
    __shared__ int s_abort;
    const bool var = F.E != nullptr, wc = F.W != nullptr;  // wc: precomputed face coefficients (FP64)
    // per stage: descriptor, x[C], ghosts[GH], f[C] (, eps[C], eps ghosts[GH] | coefficients[(2D+1) C])
    const int stage_elems = DESC + 2 * C + GH + (wc ? (2 * D + 1) * C : (var ? C + GH : 0));
    T *stage0 = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const uint32_t tx_bytes = (uint32_t)(sizeof(T) * stage_elems);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    if (tid < (int)(sizeof(LevelDesc) / 4))
        reinterpret_cast<int *>(&sL)[tid] = reinterpret_cast<const int *>(P.L + P.B[first].lev)[tid];
    __syncthreads();
    // co, go, lev: the block's cell and ghost offsets and level (thread 0
    // reads them one iteration ahead, so that a refill does not wait on them)
    auto issue = [&](int it, int g, long long co, long long go, int lev) {  // thread 0 only
        T *st = stage0 + (it & 1) * stage_elems;
        uint64_t *bar = &bars[it & 1];
        fence_async_smem();
        mbar_expect_tx(bar, tx_bytes);
        bulk_g2s(st, P.B + g, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st) + sizeof(BlockDesc), P.L + lev, sizeof(LevelDesc), bar);
        bulk_g2s(st + DESC, F.X + co, sizeof(T) * C, bar);
        bulk_g2s(st + DESC + C, F.XG + go, sizeof(T) * GH, bar);
        bulk_g2s_f<T>(st + DESC + C + GH, F.F + co, sizeof(T) * C, bar);
        if (wc) {
            // face weights, then 1 / diagonal (slot 2D + 1) in the place of the diagonal
            bulk_g2s(st + DESC + 2 * C + GH, F.W + co * wstride(D), sizeof(T) * 2 * D * C, bar);
            bulk_g2s(st + DESC + 2 * C + GH + 2 * D * C, F.W + co * wstride(D) + (2 * D + 1) * C, sizeof(T) * C, bar);
        } else if (var) {
            bulk_g2s_f<T>(st + DESC + 2 * C + GH, F.E + co, sizeof(T) * C, bar);
            bulk_g2s_f<T>(st + DESC + 3 * C + GH, F.EG + go, sizeof(T) * GH, bar);
        }
    };
    int g = blockIdx.x;
    long long rco = 0, rgo = 0;
    int rlev = 0;
    auto fetch = [&](int gn) {
        if (gn < nblocks) {
            rco = P.B[first + gn].cell_off;
            rgo = P.B[first + gn].ghost_off;
            rlev = P.B[first + gn].lev;
        }
    };
    if (tid == 0) {
        if (g < nblocks) {
            fetch(g);
            issue(0, first + g, rco, rgo, rlev);
        }
        fetch(g + (int)gridDim.x);
    }
    // level descriptor: CTA-wide copy when every block shares it, else per block
    const bool cyl = P.geom == MG_CYL;
    const T helm = kp_helm<T>(P);
    for (int it = 0; g < nblocks; it++, g += gridDim.x) {
        if (!mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, P.wait_limit)) {
            atomicExch(P.status, 1);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) {
            // the copy this wait was for may still be landing in shared
            // memory: let it arrive (normal bound) before the CTA exits
            if (tid == 0) mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, kWaitLimit);
            break;
        }
        // every thread is past the previous block: its stage may be refilled
        // once its bulk store has read it
        if (tid == 0) {
            if (g + (int)gridDim.x < nblocks) {
                bulk_wait_read0();
                issue(it + 1, first + g + gridDim.x, rco, rgo, rlev);
            }
            fetch(g + 2 * (int)gridDim.x);
        }
        T *st = stage0 + (it & 1) * stage_elems;
        const BlockDesc &b = *reinterpret_cast<const BlockDesc *>(st);
        const LevelDesc &L = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st) + sizeof(BlockDesc));
        const T lo0 = kp_lo0<T>(P), h0 = lv_h0<T>(L);  // operator scalars in the kernel precision
        const T ih0 = lv_ih<T>(L, 0), ih1 = lv_ih<T>(L, 1), ih2 = lv_ih<T>(L, 2);
        const T w0 = lv_ih<T>(L, 0), w1 = lv_ih<T>(L, 1), w2 = lv_ih<T>(L, 2);
        const T inv_den = lv_idiag<T>(L);
        T *xs = st + DESC, *gs = xs + C, *fs = gs + GH, *es = fs + C, *egs = es + C;
        const int bi = b.ijk[0], bj = b.ijk[1], bk = b.ijk[2];
        const int par0 = (bi + bj + bk) * n;
        // neighbour (d, side) of cell (i,j,k): interior or the face ghost
        auto nbv = [&](const T *xi, const T *gi, int i, int j, int k, int d, int s) -> T {
            const int o = s ? 1 : -1;
            if (d == 0) {
                const int ii = i + o;
                if (ii < 0 || ii >= n) return gi[(s ? 1 : 0) * FC + (D == 2 ? j : j + n * k)];
                return xi[cidx<D>(n, ii, j, k)];
            }
            if (d == 1) {
                const int jj = j + o;
                if (jj < 0 || jj >= n) return gi[(s ? 3 : 2) * FC + (D == 2 ? i : i + n * k)];
                return xi[cidx<D>(n, i, jj, k)];
            }
            const int kk = k + o;
            if (kk < 0 || kk >= n) return gi[(s ? 5 : 4) * FC + i + n * j];
            return xi[cidx<D>(n, i, j, kk)];
        };
        // coarse-fine faces: B'/2 of this thread's ghost slots from the old
        // interior values (see cf_half_base), before the update overwrites them
        const int cfm = cf_faces(b, D);
        T bh[GPT];
        if (cfm) {
#pragma unroll
            for (int r = 0; r < GPT; r++) {
                const int t = tid + r * TPB, face = t / FC;
                if (t >= GH || !((cfm >> face) & 1)) continue;
                const int u = t - face * FC, d = face >> 1, s = face & 1;
                const I3 ii = face_cell<D>(n, face, u, false);
                I3 dd = ii;
                put(dd, d, s ? n - 2 : 1);
                bh[r] = cf_half_base(gs[t], xs[cidx<D>(n, ii.x, ii.y, ii.z)], xs[cidx<D>(n, dd.x, dd.y, dd.z)]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < CPT; r++) {
            const int qi = tid + r * nth;
            if (qi >= NCOL) continue;
            const int h = n >> 1, rr = qi / h, m = qi - rr * h;
            const int j = rr % n, k = D == 3 ? rr / n : 0;
            const int i = 2 * m + ((colour + par0 + j + k) & 1);
            const int c = cidx<D>(n, i, j, k);
            T xnew;
            if (!var && !cyl) {
                T num = w0 * (nbv(xs, gs, i, j, k, 0, 0) + nbv(xs, gs, i, j, k, 0, 1)) +
                        w1 * (nbv(xs, gs, i, j, k, 1, 0) + nbv(xs, gs, i, j, k, 1, 1));
                if (D == 3) num += w2 * (nbv(xs, gs, i, j, k, 2, 0) + nbv(xs, gs, i, j, k, 2, 1));
                xnew = (num - fs[c]) * inv_den;
            } else if (wc) {  // same terms and order as below, coefficients read, 1 / diagonal precomputed
                const T *ws = es + c;
                T num = ws[0] * nbv(xs, gs, i, j, k, 0, 0);
#pragma unroll
                for (int f = 1; f < 2 * D; f++) num += ws[f * C] * nbv(xs, gs, i, j, k, f >> 1, f & 1);
                xnew = (num - fs[c]) * ws[2 * D * C];
            } else {
                const T ec = var ? es[c] : (T)1;
                T num = 0, den = 0, ri = 0;
                if (cyl) ri = lo0 + ((T)(bi * n + i) + (T)0.5) * h0;
#pragma unroll
                for (int d = 0; d < D; d++)
#pragma unroll
                    for (int s = 0; s < 2; s++) {
                        T w = d == 0 ? ih0 : (d == 1 ? ih1 : ih2);
                        if (var) {
                            const T en = nbv(es, egs, i, j, k, d, s);
                            w *= qdiv<T>((T)2 * ec * en, ec + en);
                        }
                        if (cyl && d == 0) w *= qdiv<T>(lo0 + (T)(bi * n + i + s) * h0, ri);
                        num += w * nbv(xs, gs, i, j, k, d, s);
                        den += w;
                    }
                xnew = qdiv<T>(num - fs[c], den + helm);
            }
            xs[c] = xnew;  // cells of the other colour are not read by this colour
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            bulk_s2g(F.X + b.cell_off, xs, sizeof(T) * C);
            bulk_commit();
        }
        // ghost pushes beside updated cells (see k_sweep)
#pragma unroll
        for (int r = 0; r < GPT; r++) {
            const int t = tid + r * TPB;
            if (t >= GH) continue;
            const int face = t / FC, u = t - face * FC, d = face >> 1, s = face & 1;
            const I3 ii = face_cell<D>(n, face, u, false);
            const bool updated = ((par0 + ii.x + ii.y + ii.z) & 1) == colour;
            const int nb = b.nbr[face];
            if (nb >= 0) {
                if (updated) F.XG[b.push[face] + u] = xs[cidx<D>(n, ii.x, ii.y, ii.z)];
            } else if (nb == -1) {
                if (updated)
                    F.XG[b.ghost_off + t] = phys_ghost<T>(P, L, face, xs[cidx<D>(n, ii.x, ii.y, ii.z)],
                                                          bc_value(P, L, b, D, face, ii));
            } else {
                I3 dd = ii;
                put(dd, d, s ? n - 2 : 1);
                F.XG[b.ghost_off + t] = cf_from_half_base(bh[r], xs[cidx<D>(n, ii.x, ii.y, ii.z)],
                                                          xs[cidx<D>(n, dd.x, dd.y, dd.z)]);
            }
        }
    }
    if (tid == 0) bulk_wait0();
}

// Warp-per-block variant of the TMA sweep for 8-cell blocks: each warp owns
// a double-buffered stage and two mbarriers and walks its own blocks
// (g = warp id, + all warps, ...), so the only synchronisation is within a
// warp.  Same arithmetic and ghost pushes as k_sweep_tma.
template <class T, int D, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) k_sweep_warp(KParams P, int first, int nblocks, Fields<T> F,
                                                           int colour) {
    pdl_entry();
    constexpr int n = 8, C = cells_of<D>(8), FC = face_of<D>(8), GH = 2 * D * FC;
    constexpr int NCOL = C / 2, PER = NCOL / 32;
    constexpr int DESC = (int)((sizeof(BlockDesc) + sizeof(LevelDesc)) / sizeof(T));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[WARPS][2];
    __shared__ __align__(16) LevelDesc sL;
    const bool var = F.E != nullptr;
    const int stage_elems = DESC + 2 * C + GH + (var ? C + GH : 0);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    T *wst = reinterpret_cast<T *>(smem_raw) + warp * 2 * stage_elems;
    const uint32_t tx_bytes = (uint32_t)(sizeof(T) * stage_elems);
    if (lane == 0) {
        mbar_init(&bars[warp][0], 1);
        mbar_init(&bars[warp][1], 1);
        fence_mbar_init();
    }
    if (tid < (int)(sizeof(LevelDesc) / 4))
        reinterpret_cast<int *>(&sL)[tid] = reinterpret_cast<const int *>(P.L + P.B[first].lev)[tid];
    __syncthreads();
    auto issue = [&](int it, int g) {  // lane 0 only
        T *st = wst + (it & 1) * stage_elems;
        const long long co = P.B[g].cell_off, go = P.B[g].ghost_off;
        uint64_t *bar = &bars[warp][it & 1];
        fence_async_smem();
        mbar_expect_tx(bar, tx_bytes);
        bulk_g2s(st, P.B + g, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st) + sizeof(BlockDesc), P.L + P.B[g].lev, sizeof(LevelDesc), bar);
        bulk_g2s(st + DESC, F.X + co, sizeof(T) * C, bar);
        bulk_g2s(st + DESC + C, F.XG + go, sizeof(T) * GH, bar);
        bulk_g2s_f<T>(st + DESC + C + GH, F.F + co, sizeof(T) * C, bar);
        if (var) {
            bulk_g2s_f<T>(st + DESC + 2 * C + GH, F.E + co, sizeof(T) * C, bar);
            bulk_g2s_f<T>(st + DESC + 3 * C + GH, F.EG + go, sizeof(T) * GH, bar);
        }
    };
    const int stride = gridDim.x * WARPS;
    int g = blockIdx.x * WARPS + warp;
    if (lane == 0 && g < nblocks) issue(0, first + g);
    // level descriptor: CTA-wide copy when every block shares it, else per block
    const bool cyl = P.geom == MG_CYL;
    const T helm = kp_helm<T>(P);
    for (int it = 0; g < nblocks; it++, g += stride) {
        const bool timed_out = !mbar_wait_bounded(&bars[warp][it & 1], (it >> 1) & 1, P.wait_limit);
        if (__any_sync(0xffffffffu, timed_out)) {
            if (lane == 0) {  // let this warp's copy in flight land before it leaves
                atomicExch(P.status, 1);
                mbar_wait_bounded(&bars[warp][it & 1], (it >> 1) & 1, kWaitLimit);
            }
            break;
        }
        __syncwarp();
        if (lane == 0 && g + stride < nblocks) {
            bulk_wait_read0();
            issue(it + 1, first + g + stride);
        }
        T *st = wst + (it & 1) * stage_elems;
        const BlockDesc &b = *reinterpret_cast<const BlockDesc *>(st);
        const LevelDesc &L = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st) + sizeof(BlockDesc));
        const T lo0 = kp_lo0<T>(P), h0 = lv_h0<T>(L);  // operator scalars in the kernel precision
        const T ih0 = lv_ih<T>(L, 0), ih1 = lv_ih<T>(L, 1), ih2 = lv_ih<T>(L, 2);
        const T w0 = lv_ih<T>(L, 0), w1 = lv_ih<T>(L, 1), w2 = lv_ih<T>(L, 2);
        const T inv_den = lv_idiag<T>(L);
        T *xs = st + DESC, *gs = xs + C, *fs = gs + GH, *es = fs + C, *egs = es + C;
        const int bi = b.ijk[0], bj = b.ijk[1], bk = b.ijk[2];
        const int par0 = (bi + bj + bk) * n;
        auto nbv = [&](const T *xi, const T *gi, int i, int j, int k, int d, int s) -> T {
            const int o = s ? 1 : -1;
            if (d == 0) {
                const int ii = i + o;
                if (ii < 0 || ii >= n) return gi[(s ? 1 : 0) * FC + (D == 2 ? j : j + n * k)];
                return xi[cidx<D>(n, ii, j, k)];
            }
            if (d == 1) {
                const int jj = j + o;
                if (jj < 0 || jj >= n) return gi[(s ? 3 : 2) * FC + (D == 2 ? i : i + n * k)];
                return xi[cidx<D>(n, i, jj, k)];
            }
            const int kk = k + o;
            if (kk < 0 || kk >= n) return gi[(s ? 5 : 4) * FC + i + n * j];
            return xi[cidx<D>(n, i, j, kk)];
        };
#pragma unroll
        for (int r = 0; r < PER; r++) {
            const int qi = lane + 32 * r;
            const int rr = qi >> 2, m = qi & 3;
            const int j = rr % n, k = D == 3 ? rr / n : 0;
            const int i = 2 * m + ((colour + par0 + j + k) & 1);
            const int c = cidx<D>(n, i, j, k);
            T xnew;
            if (!var && !cyl) {
                T num = w0 * (nbv(xs, gs, i, j, k, 0, 0) + nbv(xs, gs, i, j, k, 0, 1)) +
                        w1 * (nbv(xs, gs, i, j, k, 1, 0) + nbv(xs, gs, i, j, k, 1, 1));
                if (D == 3) num += w2 * (nbv(xs, gs, i, j, k, 2, 0) + nbv(xs, gs, i, j, k, 2, 1));
                xnew = (num - fs[c]) * inv_den;
            } else {
                const T ec = var ? es[c] : (T)1;
                T num = 0, den = 0, ri = 0;
                if (cyl) ri = lo0 + ((T)(bi * n + i) + (T)0.5) * h0;
#pragma unroll
                for (int d = 0; d < D; d++)
#pragma unroll
                    for (int s = 0; s < 2; s++) {
                        T w = d == 0 ? ih0 : (d == 1 ? ih1 : ih2);
                        if (var) {
                            const T en = nbv(es, egs, i, j, k, d, s);
                            w *= qdiv<T>((T)2 * ec * en, ec + en);
                        }
                        if (cyl && d == 0) w *= qdiv<T>(lo0 + (T)(bi * n + i + s) * h0, ri);
                        num += w * nbv(xs, gs, i, j, k, d, s);
                        den += w;
                    }
                xnew = qdiv<T>(num - fs[c], den + helm);
            }
            xs[c] = xnew;
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
            bulk_s2g(F.X + b.cell_off, xs, sizeof(T) * C);
            bulk_commit();
        }
        for (int t = lane; t < GH; t += 32) {
            const int face = t / FC, u = t - face * FC, d = face >> 1, s = face & 1;
            const I3 ii = face_cell<D>(n, face, u, false);
            const bool updated = ((par0 + ii.x + ii.y + ii.z) & 1) == colour;
            const int nb = b.nbr[face];
            if (nb >= 0) {
                if (updated) F.XG[b.push[face] + u] = xs[cidx<D>(n, ii.x, ii.y, ii.z)];
            } else if (nb == -1) {
                if (updated)
                    F.XG[b.ghost_off + t] = phys_ghost<T>(P, L, face, xs[cidx<D>(n, ii.x, ii.y, ii.z)],
                                                          bc_value(P, L, b, D, face, ii));
            } else {
                I3 dd = ii;
                put(dd, d, s ? n - 2 : 1);
                F.XG[b.ghost_off + t] = cf_ghost<T, D>(P, L, b, face, ii, xs[cidx<D>(n, ii.x, ii.y, ii.z)],
                                                       xs[cidx<D>(n, dd.x, dd.y, dd.z)], F.X, F.XG, nb, false);
            }
        }
    }
    if (lane == 0) bulk_wait0();
}

// Row-wise variant of the warp-per-block sweep for 8^3 blocks with a
// constant coefficient (Cartesian): lane l updates x-rows l and l + 32 of
// the block.  A row, its four neighbour rows (or the matching contiguous
// ghost rows on the block faces) and its right-hand side come in with
// 16-byte shared-memory loads; the colour cells of the row are chosen by
// register selects.  Ghost pushes go face by face, one updated face cell
// per lane.  Same arithmetic as k_sweep_tma.
// Rows of 8 values.  FP32 rows are 32 B apart, so the lanes of a
// quarter-warp reading the same half of their rows would meet twice on
// every bank; with sw = 1 a lane takes the halves in the other order, and
// its registers then hold the row rotated by 4 (r[e] = element e ^ 4).
template <class T> __device__ __forceinline__ void ld8(const T *p, T *r, int sw = 0) {
    using V = typename Vec16<T>::type;
    if constexpr (sizeof(T) == 4) {
        const V a = reinterpret_cast<const V *>(p)[sw], b = reinterpret_cast<const V *>(p)[sw ^ 1];
        r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
        r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
    } else {
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const V x = reinterpret_cast<const V *>(p)[v];
            r[2 * v] = x.x; r[2 * v + 1] = x.y;
        }
    }
}
template <class T> __device__ __forceinline__ void st8(T *p, const T *r, int sw = 0) {
    using V = typename Vec16<T>::type;
    if constexpr (sizeof(T) == 4) {
        reinterpret_cast<V *>(p)[sw] = make_float4(r[0], r[1], r[2], r[3]);
        reinterpret_cast<V *>(p)[sw ^ 1] = make_float4(r[4], r[5], r[6], r[7]);
    } else {
#pragma unroll
        for (int v = 0; v < 4; v++) reinterpret_cast<V *>(p)[v] = make_double2(r[2 * v], r[2 * v + 1]);
    }
}

// FG: f is not staged; each lane loads the right-hand side of its two rows
// straight into registers one block ahead (smaller stages, more in flight).
template <class T, int WARPS, int STAGES, bool FG = false>
__global__ void __launch_bounds__(32 * WARPS, WARPS == 8 ? ((FG && STAGES == 2) ? 3 : 2) : 3) k_sweep_rows(KParams P, int first, int nblocks, Fields<T> F,
                                                           int colour) {
    pdl_entry();
    constexpr int n = 8, C = 512, FC = 64, GH = 384;
    constexpr int DESC = (int)((sizeof(BlockDesc) + sizeof(LevelDesc)) / sizeof(T));
    constexpr int STAGE = DESC + C + GH + (FG ? 0 : C);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[WARPS][STAGES];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    T *wst = reinterpret_cast<T *>(smem_raw) + warp * STAGES * STAGE;
    if (lane == 0) {
        for (int q = 0; q < STAGES; q++) mbar_init(&bars[warp][q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // co, go, lev: the block's cell and ghost offsets and level
    auto issue = [&](int it, int g, long long co, long long go, int lev) {  // lane 0 only
        T *st = wst + (it % STAGES) * STAGE;
        uint64_t *bar = &bars[warp][it % STAGES];
        fence_async_smem();
        mbar_expect_tx(bar, (uint32_t)(sizeof(T) * STAGE));
        bulk_g2s(st, P.B + g, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st) + sizeof(BlockDesc), P.L + lev, sizeof(LevelDesc), bar);
        bulk_g2s(st + DESC, F.X + co, sizeof(T) * C, bar);
        bulk_g2s(st + DESC + C, F.XG + go, sizeof(T) * GH, bar);
        if (!FG) bulk_g2s_f<T>(st + DESC + C + GH, F.F + co, sizeof(T) * C, bar);
    };
    const int stride = gridDim.x * WARPS;
    int g = blockIdx.x * WARPS + warp;
    const int sw = sizeof(T) == 4 ? (lane >> 2) & 1 : 0;  // row half order of this lane (see ld8)
    T fnx[16], fcur[16];
    // The offsets of the blocks that the next iteration's stage refill
    // (block g + STAGES stride) and right-hand-side load (g + 2 stride)
    // need are read one iteration ahead, so that neither waits on the
    // descriptor table.
    long long rco = 0, rgo = 0, fco = 0;
    int rlev = 0;
    auto fetch_desc = [&](int gr, int gf) {
        if (gr < nblocks) {
            rco = P.B[first + gr].cell_off;
            rgo = P.B[first + gr].ghost_off;
            rlev = P.B[first + gr].lev;
        }
        if (FG && gf < nblocks) fco = P.B[first + gf].cell_off;
    };
    const uint64_t fpol = l2_evict_first();
    auto loadf = [&](long long cell_off) {  // rows lane and lane + 32 of the block at cell_off
        const T *fp = F.F + cell_off;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            using V = typename Vec16<T>::type;
            constexpr int VW = 16 / sizeof(T);
            const V *vp = reinterpret_cast<const V *>(fp + 8 * (lane + 32 * h));
#pragma unroll
            for (int v = 0; v < 8 / VW; v++) {
                V x;
                if constexpr (sizeof(T) == 4) x = ldg_f_ef(vp + (v ^ sw), fpol);
                else x = __ldg(vp + v);
                if constexpr (sizeof(T) == 4) {
                    fnx[8 * h + 4 * v] = x.x; fnx[8 * h + 4 * v + 1] = x.y;
                    fnx[8 * h + 4 * v + 2] = x.z; fnx[8 * h + 4 * v + 3] = x.w;
                } else {
                    fnx[8 * h + 2 * v] = x.x; fnx[8 * h + 2 * v + 1] = x.y;
                }
            }
        }
    };
    if (FG && g < nblocks) loadf(P.B[first + g].cell_off);
    if (lane == 0)
        for (int q = 0; q < STAGES - 1; q++)
            if (g + q * stride < nblocks) {
                const BlockDesc &bq = P.B[first + g + q * stride];
                issue(q, first + g + q * stride, bq.cell_off, bq.ghost_off, bq.lev);
            }
    fetch_desc(g + (STAGES - 1) * stride, g + stride);
    const T helm = kp_helm<T>(P);
    for (int it = 0; g < nblocks; it++, g += stride) {
        const bool timed_out = !mbar_wait_bounded(&bars[warp][it % STAGES], (it / STAGES) & 1, P.wait_limit);
        if (__any_sync(0xffffffffu, timed_out)) {
            if (lane == 0) {
                // copies in flight: the blocks of iterations it .. it + STAGES - 2
                // that exist; let them land (normal bound) before the warp leaves
                atomicExch(P.status, 1);
                for (int q = 0; q < STAGES - 1; q++)
                    if (g + q * stride < nblocks)
                        mbar_wait_bounded(&bars[warp][(it + q) % STAGES], ((it + q) / STAGES) & 1, kWaitLimit);
            }
            break;
        }
        __syncwarp();
        // refill the stage of block it-1 (every lane is past it) with block it+STAGES-1
        if (lane == 0 && g + (STAGES - 1) * stride < nblocks) {
            bulk_wait_read0();
            issue(it + STAGES - 1, first + g + (STAGES - 1) * stride, rco, rgo, rlev);
        }
        if (FG) {
#pragma unroll
            for (int e = 0; e < 16; e++) fcur[e] = fnx[e];
            if (g + stride < nblocks) loadf(fco);
        }
        fetch_desc(g + STAGES * stride, g + 2 * stride);
        T *st = wst + (it % STAGES) * STAGE;
        const BlockDesc &b = *reinterpret_cast<const BlockDesc *>(st);
        const LevelDesc &L = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st) + sizeof(BlockDesc));
        const T w0 = lv_ih<T>(L, 0), w1 = lv_ih<T>(L, 1), w2 = lv_ih<T>(L, 2);
        const T inv_den = lv_idiag<T>(L);
        T *xs = st + DESC, *gs = xs + C, *fs = gs + GH;
        const int par0 = (b.ijk[0] + b.ijk[1] + b.ijk[2]) * n;
        T newrow[2][8];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int q = lane + 32 * h, j = q & 7, k = q >> 3;
            T r[8], dn[8], up[8], bk[8], fw[8], fr[8];
            ld8(xs + 8 * q, r, sw);
            ld8(j > 0 ? xs + 8 * (q - 1) : gs + 2 * FC + 8 * k, dn, sw);
            ld8(j < 7 ? xs + 8 * (q + 1) : gs + 3 * FC + 8 * k, up, sw);
            ld8(k > 0 ? xs + 8 * (q - 8) : gs + 4 * FC + 8 * j, bk, sw);
            ld8(k < 7 ? xs + 8 * (q + 8) : gs + 5 * FC + 8 * j, fw, sw);
            if (FG) {
#pragma unroll
                for (int e = 0; e < 8; e++) fr[e] = fcur[8 * h + e];
            } else {
                ld8(fs + 8 * q, fr, sw);
            }
            const T xl = gs[0 * FC + j + 8 * k], xr = gs[1 * FC + j + 8 * k];
            const bool p = ((colour + par0 + j + k) & 1) != 0;  // colour cells at i = 2m + p
            // register e holds element e ^ 4 sw (same parity); the x
            // neighbours that cross a row half come from the other end
#pragma unroll
            for (int m = 0; m < 4; m++) {
                const int e = 2 * m, o = 2 * m + 1;
                T lft = m > 0 ? r[e - 1] : xl, rgt = m < 3 ? r[o + 1] : xr;
                if (m == 0) lft = sw ? r[7] : xl;
                if (m == 2) lft = sw ? xl : r[3];
                if (m == 1) rgt = sw ? xr : r[4];
                if (m == 3) rgt = sw ? r[0] : xr;
                const T xm = p ? r[e] : lft;
                const T xp = p ? rgt : r[o];
                const T sy = p ? dn[o] + up[o] : dn[e] + up[e];
                const T sz = p ? bk[o] + fw[o] : bk[e] + fw[e];
                const T fv = p ? fr[o] : fr[e];
                const T num = w0 * (xm + xp) + w1 * sy + w2 * sz;
                const T xnew = (num - fv) * inv_den;
                newrow[h][e] = p ? r[e] : xnew;
                newrow[h][o] = p ? xnew : r[o];
            }
        }
        // every lane has read its neighbour rows: write the rows back
        __syncwarp();
        // coarse-fine faces: B'/2 into the stage ghost slots while the rows
        // still hold the old values (see cf_half_base)
        const int cfm = cf_faces(b, 3);
        if (cfm) {
#pragma unroll 1
            for (int face = 0; face < 6; face++) {
                if (!((cfm >> face) & 1)) continue;
                const int d = face >> 1, s = face & 1, edge = s ? n - 1 : 0;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int u = 2 * lane + h, t1 = u & 7, t2 = u >> 3;
                    const I3 ii = d == 0 ? I3{edge, t1, t2} : (d == 1 ? I3{t1, edge, t2} : I3{t1, t2, edge});
                    I3 dd = ii;
                    put(dd, d, s ? n - 2 : 1);
                    gs[face * FC + u] = cf_half_base(gs[face * FC + u], xs[cidx<3>(n, ii.x, ii.y, ii.z)],
                                                     xs[cidx<3>(n, dd.x, dd.y, dd.z)]);
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int h = 0; h < 2; h++) st8(xs + 8 * (lane + 32 * h), newrow[h], sw);
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
            bulk_s2g(F.X + b.cell_off, xs, sizeof(T) * C);
            bulk_commit();
        }
        // ghost pushes, one face at a time (warp-uniform face type)
#pragma unroll 1
        for (int face = 0; face < 6; face++) {
            const int d = face >> 1, s = face & 1, nb = b.nbr[face];
            const int edge = s ? n - 1 : 0;
            if (nb <= -2) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int u = 2 * lane + h, t1 = u & 7, t2 = u >> 3;
                    const I3 ii = d == 0 ? I3{edge, t1, t2} : (d == 1 ? I3{t1, edge, t2} : I3{t1, t2, edge});
                    I3 dd = ii;
                    put(dd, d, s ? n - 2 : 1);
                    F.XG[b.ghost_off + face * FC + u] =
                        cf_from_half_base(gs[face * FC + u], xs[cidx<3>(n, ii.x, ii.y, ii.z)],
                                          xs[cidx<3>(n, dd.x, dd.y, dd.z)]);
                }
                continue;
            }
            // the lane's updated face cell: tangential row t2 = lane / 4, 4 per row
            const int t2 = lane >> 2;
            const int po = (colour + par0 + edge + t2) & 1;
            const int t1 = 2 * (lane & 3) + po;
            const I3 ii = d == 0 ? I3{edge, t1, t2} : (d == 1 ? I3{t1, edge, t2} : I3{t1, t2, edge});
            const int u = t1 + 8 * t2;
            const T xi = xs[cidx<3>(n, ii.x, ii.y, ii.z)];
            if (nb >= 0) F.XG[b.push[face] + u] = xi;
            else F.XG[b.ghost_off + face * FC + u] = phys_ghost<T>(P, L, face, xi, bc_value(P, L, b, 3, face, ii));
        }
    }
    if (lane == 0) bulk_wait0();
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
    pdl_entry();
    __shared__ BlockDesc sb;
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
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
                sr += Fr[b.cell_off + fc] - (lap - kp_helm<T>(P) * xc);
            }
        }
        const int pc = cidx<D>(p.n, b.poff[0] + ci, b.poff[1] + cj, b.poff[2] + ck);
        X[p.cell_off + pc] = sx * (T)(1.0 / (1 << D));
        if (with_res) Fdst[p.cell_off + pc] = sr * (T)(1.0 / (1 << D));
    }
}

// The defect-correction update fused into the covered-cell refresh: for one
// block of a level (one CTA each; the level's first nref blocks are
// covered), a leaf block first takes phi += e (e the FP32 correction,
// widened exactly with integer operations) and writes phi back; then every
// block restricts its values into the parent cells under it (mean of the
// 2^D children, summed in the same order as k_restrict, so the result is
// the one of the update followed by the plain refresh).  Fine cells are
// read and written coalesced, kUpdCells per thread with every load issued
// before the first use (bytes in flight against DRAM latency), and staged
// in shared memory for the parent means.
constexpr int kUpdCells = 4;
template <int D>
__global__ void __launch_bounds__(256) k_update_restrict(KParams P, int first, int nref, double *__restrict__ X,
                                                         const float *__restrict__ e) {
    pdl_entry();
    __shared__ BlockDesc sb;
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
    const BlockDesc &p = P.B[b.parent];
    const int n = b.n, m = n / 2, C = cells_of<D>(n), M = cells_of<D>(m);
    const bool leaf = (int)blockIdx.x >= nref;
    extern __shared__ double xs[];
    double *xb = X + b.cell_off;
    const float *eb = e + b.cell_off;
    for (int c0 = threadIdx.x; c0 < C; c0 += kUpdCells * blockDim.x) {
        double xv[kUpdCells];
        float ev[kUpdCells];
#pragma unroll
        for (int k = 0; k < kUpdCells; k++) {
            const int c = c0 + k * blockDim.x;
            if (c < C) {
                xv[k] = xb[c];
                ev[k] = leaf ? eb[c] : 0.0f;
            }
        }
#pragma unroll
        for (int k = 0; k < kUpdCells; k++) {
            const int c = c0 + k * blockDim.x;
            if (c < C) {
                double x = xv[k];
                if (leaf) {
                    x += mg_from_float(ev[k]);
                    xb[c] = x;
                }
                xs[c] = x;
            }
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < M; c += blockDim.x) {
        int ci, cj, ck;
        cell_of(c, m, D, ci, cj, ck);
        double sx = 0;
#pragma unroll
        for (int ch = 0; ch < (1 << D); ch++)
            sx += xs[cidx<D>(n, 2 * ci + (ch & 1), 2 * cj + ((ch >> 1) & 1), D == 3 ? 2 * ck + ((ch >> 2) & 1) : 0)];
        X[p.cell_off + cidx<D>(p.n, b.poff[0] + ci, b.poff[1] + cj, b.poff[2] + ck)] = sx * (1.0 / (1 << D));
    }
}

// ------------------------------------------- transfers with ghost pushes ---
// Push the ghosts that depend on the cells of one face of block b after those
// cells changed: the same-level neighbour's slot opposite each cell, or the
// block's own physical or refinement ghost.  `val(ii)` returns the new value
// of interior cell ii of b (an in-range cell index triple).
template <class T, int D, class ValFn>
__device__ __forceinline__ void push_face_cell(const KParams &P, const LevelDesc &L, const BlockDesc &b, int face,
                                               int u, I3 ii, T *__restrict__ X, T *__restrict__ XG, ValFn val) {
    const int n = b.n, Fc = face_of<D>(n), d = face >> 1, s = face & 1;
    const int nb = b.nbr[face];
    const T c = val(ii);
    if (nb >= 0) {
        XG[b.push[face] + u] = c;
    } else if (nb == -1) {
        XG[b.ghost_off + face * Fc + u] = phys_ghost<T>(P, L, face, c, bc_value(P, L, b, D, face, ii));
    } else {
        I3 dd = ii;
        put(dd, d, s ? n - 2 : 1);
        XG[b.ghost_off + face * Fc + u] = cf_ghost<T, D>(P, L, b, face, ii, c, val(dd), X, XG, nb, false);
    }
}

// Restriction with the FAS residual (Sec. 2.3, 2.4) for fine block b, fused
// with the ghost update of the parent level: the parent cells under b receive
// the mean of their children (and the mean child residual goes to the
// parent's right-hand side); then every parent ghost that depends on those
// cells is pushed.  Each parent face cell belongs to exactly one child, so
// every ghost slot has one writer.  Needs n >= 4 (a child octant then holds
// the two parent layers c and d of a refinement ghost).
template <class T, int D>
__global__ void __launch_bounds__(kMaxThreads) k_restrict_push(KParams P, int first, Fields<T> F) {
    pdl_entry();
    __shared__ BlockDesc sb, sp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *oct = reinterpret_cast<T *>(smem_raw);
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
    stage_desc(P, b.parent, sp);
    const BlockDesc &p = sp;
    const LevelDesc &L = P.L[b.lev];
    const LevelDesc &PL = P.L[p.lev];
    const int n = b.n, m = n / 2, M = cells_of<D>(m), pn = p.n;
    for (int c = threadIdx.x; c < M; c += blockDim.x) {
        int ci, cj, ck;
        cell_of(c, m, D, ci, cj, ck);
        T sx = 0, sr = 0;
#pragma unroll 1
        for (int ch = 0; ch < (1 << D); ch++) {
            const int fi = 2 * ci + (ch & 1), fj = 2 * cj + ((ch >> 1) & 1), fk = D == 3 ? 2 * ck + ((ch >> 2) & 1) : 0;
            const int fc = cidx<D>(n, fi, fj, fk);
            if constexpr (sizeof(T) == 8) {
                if (F.W) {  // precomputed face coefficients (no FP64 division)
                    const double xc = F.X[b.cell_off + fc];
                    sx += xc;
                    sr += F.F[b.cell_off + fc] - (lap_w<D>(b, F.X, F.XG, F.W, fi, fj, fk, xc) - P.helm * xc);
                    continue;
                }
            }
            T lap, num, den, xc;
            stencil<T, T, D>(P, L, b, F.X, F.XG, F.E, F.EG, fi, fj, fk, lap, num, den, xc);
            sx += xc;
            sr += F.F[b.cell_off + fc] - (lap - kp_helm<T>(P) * xc);
        }
        const T xv = sx * (T)(1.0 / (1 << D));
        const int pc = cidx<D>(pn, b.poff[0] + ci, b.poff[1] + cj, b.poff[2] + ck);
        F.X[p.cell_off + pc] = xv;
        F.F[p.cell_off + pc] = sr * (T)(1.0 / (1 << D));
        oct[c] = xv;
    }
    __syncthreads();
    const int Fm = face_of<D>(m);
    auto val = [&](I3 q) {  // parent cell q, inside this child's octant
        return oct[cidx<D>(m, q.x - b.poff[0], q.y - b.poff[1], q.z - b.poff[2])];
    };
    for (int t = threadIdx.x; t < 2 * D * Fm; t += blockDim.x) {
        const int face = t / Fm, v = t - face * Fm, d = face >> 1, s = face & 1;
        const int off = d == 0 ? b.poff[0] : d == 1 ? b.poff[1] : b.poff[2];
        if (s ? (off + m != pn) : (off != 0)) continue;  // octant not on this parent face
        I3 ii = face_cell<D>(m, face, v, false);       // octant-local cell on the face
        ii.x += b.poff[0];
        ii.y += b.poff[1];
        ii.z += D == 3 ? b.poff[2] : 0;
        put(ii, d, s ? pn - 1 : 0);
        int u;  // parent face index t1 + pn t2
        if (D == 2) u = d == 0 ? ii.y : ii.x;
        else u = d == 0 ? ii.y + pn * ii.z : (d == 1 ? ii.x + pn * ii.z : ii.x + pn * ii.y);
        push_face_cell<T, D>(P, PL, p, face, u, ii, F.X, F.XG, val);
    }
}

// Covered cells: f^H = R(r^h) + L^H v^H (eq. for the coarse right-hand side),
// and the FAS copy v_old = v^H with its ghosts (only covered blocks are read
// by the prolongation).
template <class T, int D>
__global__ void __launch_bounds__(kMaxThreads) k_fas_rhs_vold(KParams P, int first, Fields<T> F) {
    pdl_entry();
    __shared__ BlockDesc sb;
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, C = cells_of<D>(n), G = 2 * D * face_of<D>(n);
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        if constexpr (sizeof(T) == 8) {
            if (F.W) {  // precomputed face coefficients (no FP64 division)
                const double xc = F.X[b.cell_off + c];
                F.F[b.cell_off + c] += lap_w<D>(b, F.X, F.XG, F.W, i, j, k, xc) - P.helm * xc;
                F.V[b.cell_off + c] = xc;
                continue;
            }
        }
        T lap, num, den, xc;
        stencil<T, T, D>(P, L, b, F.X, F.XG, F.E, F.EG, i, j, k, lap, num, den, xc);
        F.F[b.cell_off + c] += lap - kp_helm<T>(P) * xc;
        F.V[b.cell_off + c] = xc;
    }
    for (int t = threadIdx.x; t < G; t += blockDim.x) F.VG[b.ghost_off + t] = F.XG[b.ghost_off + t];
}

// Coarse-grid correction (Sec. 2.4, 2.3): x^h += P(x^H - x^H_old), P the
// nearest-neighbour linear interpolation -- 2D (2 c0 + c_x + c_y)/4, 3D
// (c0 + c_x + c_y + c_z)/4 with the neighbours on the fine cell's side
// (coarse ghosts included).  Fused with the fine-level ghost update: every
// cell of block b changes, so after the correction all its face ghosts that
// depend on its cells are pushed (the kernel reads only the coarser level's
// fields and its own interior, never this level's ghosts).
template <class T, int D>
__global__ void __launch_bounds__(kMaxThreads) k_prolong_push(KParams P, int first, Fields<T> F) {
    pdl_entry();
    __shared__ BlockDesc sb, sp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
    stage_desc(P, b.parent, sp);
    const BlockDesc &p = sp;
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, C = cells_of<D>(n);
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        const int I0 = b.ijk[0] * n + i, I1 = b.ijk[1] * n + j, I2 = b.ijk[2] * n + k;
        const int c0 = b.poff[0] + i / 2, c1 = b.poff[1] + j / 2, c2 = D == 3 ? b.poff[2] + k / 2 : 0;
        const T v0 = load<T, D>(F.X, F.XG, p, c0, c1, c2) - load<T, D>(F.V, F.VG, p, c0, c1, c2);
        const int sx = (I0 & 1) ? 1 : -1, sy = (I1 & 1) ? 1 : -1, sz = (I2 & 1) ? 1 : -1;
        T nbs = load<T, D>(F.X, F.XG, p, c0 + sx, c1, c2) - load<T, D>(F.V, F.VG, p, c0 + sx, c1, c2);
        nbs += load<T, D>(F.X, F.XG, p, c0, c1 + sy, c2) - load<T, D>(F.V, F.VG, p, c0, c1 + sy, c2);
        if (D == 3) nbs += load<T, D>(F.X, F.XG, p, c0, c1, c2 + sz) - load<T, D>(F.V, F.VG, p, c0, c1, c2 + sz);
        const T val = D == 2 ? ((T)2 * v0 + nbs) / (T)4 : (v0 + nbs) / (T)4;
        const T xn = F.X[b.cell_off + c] + val;
        F.X[b.cell_off + c] = xn;
        xs[c] = xn;
    }
    __syncthreads();
    const int Fc = face_of<D>(n);
    auto val = [&](I3 q) { return xs[cidx<D>(n, q.x, q.y, q.z)]; };
    for (int t = threadIdx.x; t < 2 * D * Fc; t += blockDim.x) {
        const int face = t / Fc, u = t - face * Fc;
        push_face_cell<T, D>(P, L, b, face, u, face_cell<D>(n, face, u, false), F.X, F.XG, val);
    }
}

// Ghost fill by pushing (8- and 16-cell blocks), persistent and
// TMA-staged: each block stages its own interior and writes every ghost slot
// its cells feed -- the opposite slot of each same-level neighbour, its own
// physical ghosts and its own refinement ghosts (Sec. 2.6) -- so all reads
// of the level are contiguous.  Every slot of a launch has exactly one
// writer; refinement ghosts read only the coarser level.  mode as k_ghost.
template <class T, int D, int NT>
__global__ void __launch_bounds__(transfer_bound(D, NT)) k_ghost_tma(KParams P, int first, int nblocks, T *__restrict__ X,
                                                           T *__restrict__ XG, int mode) {
    pdl_entry();
    constexpr int n = NT, C = cells_of<D>(NT), FC = face_of<D>(NT), GH = 2 * D * FC;
    constexpr int DESC = (int)((sizeof(BlockDesc) + sizeof(LevelDesc)) / sizeof(T));
    constexpr int STAGE = DESC + C;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    T *stage0 = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    // co, lev: the block's cell offset and level (thread 0 reads them one
    // iteration ahead, so that a refill does not wait on them)
    auto issue = [&](int it, int g, long long co, int lev) {  // thread 0 only
        T *st = stage0 + (it & 1) * STAGE;
        uint64_t *bar = &bars[it & 1];
        fence_async_smem();
        mbar_expect_tx(bar, (uint32_t)(sizeof(T) * STAGE));
        bulk_g2s(st, P.B + g, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st) + sizeof(BlockDesc), P.L + lev, sizeof(LevelDesc), bar);
        bulk_g2s(st + DESC, X + co, sizeof(T) * C, bar);
    };
    int g = blockIdx.x;
    long long rco = 0;
    int rlev = 0;
    auto fetch = [&](int gn) {
        if (gn < nblocks) { rco = P.B[first + gn].cell_off; rlev = P.B[first + gn].lev; }
    };
    if (tid == 0) {
        if (g < nblocks) {
            fetch(g);
            issue(0, first + g, rco, rlev);
        }
        fetch(g + (int)gridDim.x);
    }
    for (int it = 0; g < nblocks; it++, g += gridDim.x) {
        if (!mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, P.wait_limit)) {
            atomicExch(P.status, 1);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) {
            // the copy this wait was for may still be landing in shared
            // memory: let it arrive (normal bound) before the CTA exits
            if (tid == 0) mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, kWaitLimit);
            break;
        }
        if (tid == 0) {
            if (g + (int)gridDim.x < nblocks) issue(it + 1, first + g + gridDim.x, rco, rlev);
            fetch(g + 2 * (int)gridDim.x);
        }
        const T *st = stage0 + (it & 1) * STAGE;
        const BlockDesc &b = *reinterpret_cast<const BlockDesc *>(st);
        const LevelDesc &L = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st) + sizeof(BlockDesc));
        const T *xs = st + DESC;
        for (int t = tid; t < GH; t += nth) {
            const int face = t / FC, u = t - face * FC, d = face >> 1, s = face & 1;
            const I3 ii = face_cell<D>(n, face, u, false);
            const T xi = xs[cidx<D>(n, ii.x, ii.y, ii.z)];
            const int nb = b.nbr[face];
            if (nb >= 0) {
                XG[b.push[face] + u] = xi;
            } else if (nb == -1) {
                XG[b.ghost_off + t] = mode >= 1 ? xi : phys_ghost<T>(P, L, face, xi, bc_value(P, L, b, D, face, ii));
            } else {
                I3 dd = ii;
                put(dd, d, s ? n - 2 : 1);
                XG[b.ghost_off + t] = cf_ghost<T, D>(P, L, b, face, ii, xi, xs[cidx<D>(n, dd.x, dd.y, dd.z)], X, XG, nb,
                                                     mode == 1);
            }
        }
        __syncthreads();  // stage reads done before it is refilled
    }
}

// FAS right-hand side of covered blocks (Sec. 2.4), persistent and
// TMA-staged (8- and 16-cell blocks): f^H += L^H x^H - lambda x^H from the
// staged block, its ghosts (and eps); f^H, v_old = x^H and its ghosts leave
// by bulk stores.  Same arithmetic as the stencil helper.
template <class T, int D, int NT>
__global__ void __launch_bounds__(transfer_bound(D, NT)) k_fas_tma(KParams P, int first, int nblocks, Fields<T> F) {
    pdl_entry();
    constexpr int n = NT, C = cells_of<D>(NT), FC = face_of<D>(NT), GH = 2 * D * FC;
    constexpr int DESC = (int)((sizeof(BlockDesc) + sizeof(LevelDesc)) / sizeof(T));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    const bool var = F.E != nullptr, wc = F.W != nullptr;
    const int stage_elems = DESC + 2 * C + GH + (wc ? 2 * D * C : (var ? C + GH : 0));
    T *stage0 = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const uint32_t tx_bytes = (uint32_t)(sizeof(T) * stage_elems);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    // co, go, lev: the block's cell and ghost offsets and level (thread 0
    // reads them one iteration ahead, so that a refill does not wait on them)
    auto issue = [&](int it, int g, long long co, long long go, int lev) {  // thread 0 only
        T *st = stage0 + (it & 1) * stage_elems;
        uint64_t *bar = &bars[it & 1];
        fence_async_smem();
        mbar_expect_tx(bar, tx_bytes);
        bulk_g2s(st, P.B + g, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st) + sizeof(BlockDesc), P.L + lev, sizeof(LevelDesc), bar);
        bulk_g2s(st + DESC, F.X + co, sizeof(T) * C, bar);
        bulk_g2s(st + DESC + C, F.XG + go, sizeof(T) * GH, bar);
        bulk_g2s(st + DESC + C + GH, F.F + co, sizeof(T) * C, bar);
        if (wc) {
            bulk_g2s(st + DESC + 2 * C + GH, F.W + co * wstride(D), sizeof(T) * 2 * D * C, bar);
        } else if (var) {
            bulk_g2s(st + DESC + 2 * C + GH, F.E + co, sizeof(T) * C, bar);
            bulk_g2s(st + DESC + 3 * C + GH, F.EG + go, sizeof(T) * GH, bar);
        }
    };
    const bool cyl = P.geom == MG_CYL;
    int g = blockIdx.x;
    long long rco = 0, rgo = 0;
    int rlev = 0;
    auto fetch = [&](int gn) {
        if (gn < nblocks) {
            rco = P.B[first + gn].cell_off;
            rgo = P.B[first + gn].ghost_off;
            rlev = P.B[first + gn].lev;
        }
    };
    if (tid == 0) {
        if (g < nblocks) {
            fetch(g);
            issue(0, first + g, rco, rgo, rlev);
        }
        fetch(g + (int)gridDim.x);
    }
    for (int it = 0; g < nblocks; it++, g += gridDim.x) {
        if (!mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, P.wait_limit)) {
            atomicExch(P.status, 1);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) {
            // the copy this wait was for may still be landing in shared
            // memory: let it arrive (normal bound) before the CTA exits
            if (tid == 0) mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, kWaitLimit);
            break;
        }
        if (tid == 0) {
            if (g + (int)gridDim.x < nblocks) {
                bulk_wait_read0();  // the other stage's stores have left shared memory
                issue(it + 1, first + g + gridDim.x, rco, rgo, rlev);
            }
            fetch(g + 2 * (int)gridDim.x);
        }
        T *st = stage0 + (it & 1) * stage_elems;
        const BlockDesc &b = *reinterpret_cast<const BlockDesc *>(st);
        const LevelDesc &L = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st) + sizeof(BlockDesc));
        const T lo0 = kp_lo0<T>(P), h0 = lv_h0<T>(L);  // operator scalars in the kernel precision
        const T ih0 = lv_ih<T>(L, 0), ih1 = lv_ih<T>(L, 1), ih2 = lv_ih<T>(L, 2);
        const T *xs = st + DESC, *gs = xs + C, *es = gs + C + GH, *egs = es + C;
        T *fs = st + DESC + C + GH;
        auto nbv = [&](const T *xi, const T *gi, int i, int j, int k, int d, int s) -> T {
            const int o = s ? 1 : -1;
            if (d == 0) {
                const int ii = i + o;
                if (ii < 0 || ii >= n) return gi[(s ? 1 : 0) * FC + (D == 2 ? j : j + n * k)];
                return xi[cidx<D>(n, ii, j, k)];
            }
            if (d == 1) {
                const int jj = j + o;
                if (jj < 0 || jj >= n) return gi[(s ? 3 : 2) * FC + (D == 2 ? i : i + n * k)];
                return xi[cidx<D>(n, i, jj, k)];
            }
            const int kk = k + o;
            if (kk < 0 || kk >= n) return gi[(s ? 5 : 4) * FC + i + n * j];
            return xi[cidx<D>(n, i, j, kk)];
        };
        for (int c = tid; c < C; c += nth) {
            const int i = c % n, j = (c / n) % n, k = D == 3 ? c / (n * n) : 0;
            const T xc = xs[c];
            if (wc) {  // same terms and order as below, coefficients read
                T lap = 0;
#pragma unroll
                for (int f = 0; f < 2 * D; f++) lap += es[f * C + c] * (nbv(xs, gs, i, j, k, f >> 1, f & 1) - xc);
                fs[c] += lap - kp_helm<T>(P) * xc;
                continue;
            }
            const T ec = var ? es[c] : (T)1;
            T lap = 0, ri = 0;
            if (cyl) ri = lo0 + ((T)(b.ijk[0] * n + i) + (T)0.5) * h0;
#pragma unroll
            for (int d = 0; d < D; d++)
#pragma unroll
                for (int s = 0; s < 2; s++) {
                    T w = d == 0 ? ih0 : (d == 1 ? ih1 : ih2);
                    if (var) {
                        const T en = nbv(es, egs, i, j, k, d, s);
                        w *= qdiv<T>((T)2 * ec * en, ec + en);
                    }
                    if (cyl && d == 0) w *= qdiv<T>(lo0 + (T)(b.ijk[0] * n + i + s) * h0, ri);
                    lap += w * (nbv(xs, gs, i, j, k, d, s) - xc);
                }
            fs[c] += lap - kp_helm<T>(P) * xc;
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            bulk_s2g(F.F + b.cell_off, fs, sizeof(T) * C);
            bulk_s2g(F.V + b.cell_off, xs, sizeof(T) * C);
            bulk_s2g(F.VG + b.ghost_off, gs, sizeof(T) * GH);
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait0();
}

// Coarse-grid correction, persistent and TMA-staged (8- and 16-cell
// blocks): per child block the descriptors, the child interior and the
// parent's x, x_old and their ghosts arrive by cp.async.bulk into one stage
// of a double buffer; x^H - x^H_old on the octant under the child and its
// face halo goes to a small box, every fine cell takes
// (2 c0 + cx + cy)/4 (2D) or (c0 + cx + cy + cz)/4 (3D) of it (Sec. 2.3),
// the child leaves by a bulk store and its face ghosts are pushed as in
// k_prolong_push.  pn is the parent block size (NT or NT/2, uniform per
// launch).  Bounded waits as in the sweeps.
template <class T, int D, int NT>
__global__ void __launch_bounds__(transfer_bound(D, NT)) k_prolong_tma(KParams P, int first, int nblocks, Fields<T> F, int pn) {
    pdl_entry();
    constexpr int n = NT, m = NT / 2, C = cells_of<D>(NT), FC = face_of<D>(NT), B = m + 2;
    constexpr int BOX = D == 2 ? B * B : B * B * B;
    constexpr int DESC = (int)((sizeof(BlockDesc) + sizeof(LevelDesc)) / sizeof(T));
    constexpr int PD = (int)(sizeof(BlockDesc) / sizeof(T));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    __shared__ __align__(16) T box[BOX];
    const int Cp = D == 2 ? pn * pn : pn * pn * pn, FCp = D == 2 ? pn : pn * pn, GHp = 2 * D * FCp;
    const int stage_elems = DESC + PD + C + 2 * (Cp + GHp);
    T *stage0 = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const uint32_t tx_bytes = (uint32_t)(sizeof(T) * stage_elems);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    auto issue = [&](int it, int g) {  // thread 0 only
        T *st = stage0 + (it & 1) * stage_elems;
        const BlockDesc *bd = P.B + g;
        const int par = bd->parent;
        const long long co = bd->cell_off, pco = P.B[par].cell_off, pgo = P.B[par].ghost_off;
        uint64_t *bar = &bars[it & 1];
        fence_async_smem();
        mbar_expect_tx(bar, tx_bytes);
        bulk_g2s(st, bd, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st) + sizeof(BlockDesc), P.L + bd->lev, sizeof(LevelDesc), bar);
        bulk_g2s(st + DESC, P.B + par, sizeof(BlockDesc), bar);
        T *d = st + DESC + PD;
        bulk_g2s(d, F.X + co, sizeof(T) * C, bar);
        bulk_g2s(d + C, F.X + pco, sizeof(T) * Cp, bar);
        bulk_g2s(d + C + Cp, F.XG + pgo, sizeof(T) * GHp, bar);
        bulk_g2s(d + C + Cp + GHp, F.V + pco, sizeof(T) * Cp, bar);
        bulk_g2s(d + C + 2 * Cp + GHp, F.VG + pgo, sizeof(T) * GHp, bar);
    };
    int g = blockIdx.x;
    if (tid == 0 && g < nblocks) issue(0, first + g);
    auto bid = [](int a, int c, int e) { return D == 2 ? c * B + a : (e * B + c) * B + a; };
    for (int it = 0; g < nblocks; it++, g += gridDim.x) {
        if (!mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, P.wait_limit)) {
            atomicExch(P.status, 1);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) {
            // the copy this wait was for may still be landing in shared
            // memory: let it arrive (normal bound) before the CTA exits
            if (tid == 0) mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, kWaitLimit);
            break;
        }
        if (tid == 0 && g + (int)gridDim.x < nblocks) {
            bulk_wait_read0();  // the other stage's store has left shared memory
            issue(it + 1, first + g + gridDim.x);
        }
        T *st = stage0 + (it & 1) * stage_elems;
        const BlockDesc &b = *reinterpret_cast<const BlockDesc *>(st);
        const LevelDesc &L = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st) + sizeof(BlockDesc));
        T *xs = st + DESC + PD;
        const T *px = xs + C, *pg = px + Cp, *pv = pg + GHp, *pvg = pv + Cp;
        // parent value at (i, j, k), at most one coordinate outside the parent
        auto pval = [&](const T *xi, const T *gi, int i, int j, int k) -> T {
            if (i < 0) return gi[0 * FCp + (D == 2 ? j : j + pn * k)];
            if (i >= pn) return gi[1 * FCp + (D == 2 ? j : j + pn * k)];
            if (j < 0) return gi[2 * FCp + (D == 2 ? i : i + pn * k)];
            if (j >= pn) return gi[3 * FCp + (D == 2 ? i : i + pn * k)];
            if (D == 3) {
                if (k < 0) return gi[4 * FCp + i + pn * j];
                if (k >= pn) return gi[5 * FCp + i + pn * j];
            }
            return xi[cidx<D>(pn, i, j, k)];
        };
        for (int q = tid; q < BOX; q += nth) {
            const int a = q % B, c = (q / B) % B, e = D == 3 ? q / (B * B) : 1;
            const int out = (a == 0 || a == B - 1) + (c == 0 || c == B - 1) + (D == 3 && (e == 0 || e == B - 1));
            if (out > 1) continue;  // edge / corner of the box: never read
            const int pi = b.poff[0] + a - 1, pj = b.poff[1] + c - 1, pk = D == 3 ? b.poff[2] + e - 1 : 0;
            box[bid(a, c, e)] = pval(px, pg, pi, pj, pk) - pval(pv, pvg, pi, pj, pk);
        }
        __syncthreads();
        const int ox = (b.ijk[0] * n) & 1, oy = (b.ijk[1] * n) & 1, oz = (b.ijk[2] * n) & 1;
        for (int c = tid; c < C; c += nth) {
            const int i = c % n, j = (c / n) % n, k = D == 3 ? c / (n * n) : 0;
            const int a = i / 2 + 1, cc = j / 2 + 1, e = D == 3 ? k / 2 + 1 : 1;
            const int sx = ((ox + i) & 1) ? 1 : -1, sy = ((oy + j) & 1) ? 1 : -1, sz = ((oz + k) & 1) ? 1 : -1;
            const T v0 = box[bid(a, cc, e)];
            T nbs = box[bid(a + sx, cc, e)];
            nbs += box[bid(a, cc + sy, e)];
            if (D == 3) nbs += box[bid(a, cc, e + sz)];
            const T val = D == 2 ? ((T)2 * v0 + nbs) / (T)4 : (v0 + nbs) / (T)4;
            xs[c] = xs[c] + val;
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            bulk_s2g(F.X + b.cell_off, xs, sizeof(T) * C);
            bulk_commit();
        }
        auto val = [&](I3 q) { return xs[cidx<D>(n, q.x, q.y, q.z)]; };
        for (int t = tid; t < 2 * D * FC; t += nth) {
            const int face = t / FC, u = t - face * FC;
            push_face_cell<T, D>(P, L, b, face, u, face_cell<D>(n, face, u, false), F.X, F.XG, val);
        }
        __syncthreads();  // box and stage reads done before the next block
    }
    if (tid == 0) bulk_wait0();
}

// Row-wise form of k_prolong_tma for 3D 8^3 blocks with 8^3 parents (128
// threads).  Same staging and arithmetic; what changes is the work split,
// because k_prolong_tma is bound by its per-cell index work and barriers:
//  - each thread corrects half a fine row (4 cells) with one vector load and
//    store, reading the 8 parent values x^H - x^H_old it needs straight from
//    the staged parent (no shared correction box, no barrier for it);
//  - it pushes the same-level and physical ghosts of its cells from
//    registers: x faces take its row's end cell, y and z faces its 4 cells,
//    which are contiguous in the ghost face;
//  - it stores its corrected cells to global memory itself, so a block
//    without refinement faces takes no barrier beyond the stage wait;
//  - refinement ghosts also need the inward cell of another row; on blocks
//    that have them they are formed after a barrier from shared memory.
template <class T>
__global__ void __launch_bounds__(128) k_prolong_rows(KParams P, int first, int nblocks, Fields<T> F) {
    pdl_entry();
    constexpr int n = 8, C = 512, FC = 64, GH = 384;
    constexpr int DESC = (int)((sizeof(BlockDesc) + sizeof(LevelDesc)) / sizeof(T));
    constexpr int PD = (int)(sizeof(BlockDesc) / sizeof(T));
    constexpr int STAGE = DESC + PD + C + 2 * (C + GH);
    using V = typename Vec16<T>::type;
    constexpr int VW = 16 / sizeof(T);  // elements per 16-byte vector
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    T *stage0 = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x;
    constexpr int ISSUER = 127;  // stage copies and stores
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    // offsets of a block and its parent for the stage copies; the issuer
    // reads them two iterations ahead (the block's own fields one iteration
    // before its parent's), so that a refill never waits on the table
    struct Src { long long co, pco, pgo; int par, lev; };
    auto own = [&](int g, Src &r) {
        if (g < nblocks) {
            const BlockDesc &q = P.B[first + g];
            r.co = q.cell_off; r.par = q.parent; r.lev = q.lev;
        }
    };
    auto parent = [&](int g, Src &r) {
        if (g < nblocks) { r.pco = P.B[r.par].cell_off; r.pgo = P.B[r.par].ghost_off; }
    };
    auto issue = [&](int it, int g, const Src &r) {  // thread ISSUER only
        T *st = stage0 + (it & 1) * STAGE;
        uint64_t *bar = &bars[it & 1];
        fence_async_smem();
        mbar_expect_tx(bar, (uint32_t)(sizeof(T) * STAGE));
        bulk_g2s(st, P.B + first + g, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st) + sizeof(BlockDesc), P.L + r.lev, sizeof(LevelDesc), bar);
        bulk_g2s(st + DESC, P.B + r.par, sizeof(BlockDesc), bar);
        T *d = st + DESC + PD;
        bulk_g2s(d, F.X + r.co, sizeof(T) * C, bar);
        bulk_g2s(d + C, F.X + r.pco, sizeof(T) * C, bar);
        bulk_g2s(d + 2 * C, F.XG + r.pgo, sizeof(T) * GH, bar);
        bulk_g2s(d + 2 * C + GH, F.V + r.pco, sizeof(T) * C, bar);
        bulk_g2s(d + 3 * C + GH, F.VG + r.pgo, sizeof(T) * GH, bar);
    };
    int g = blockIdx.x;
    Src n1{}, n2{};
    if (tid == ISSUER) {
        if (g < nblocks) {
            Src r0{};
            own(g, r0);
            parent(g, r0);
            issue(0, g, r0);
        }
        own(g + (int)gridDim.x, n1);
        parent(g + (int)gridDim.x, n1);
        own(g + 2 * (int)gridDim.x, n2);
    }
    // fine half-row of this thread: row r = (j, k), cells i = 4h .. 4h + 3
    const int r = tid >> 1, h = tid & 1, j = r & 7, k = r >> 3;
    const int sy = (j & 1) ? 1 : -1, sz = (k & 1) ? 1 : -1;
    for (int it = 0; g < nblocks; it++, g += gridDim.x) {
        if (!mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, P.wait_limit)) {
            atomicExch(P.status, 1);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) {
            // the copy this wait was for may still be landing in shared
            // memory: let it arrive (normal bound) before the CTA exits
            if (tid == 0) mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, kWaitLimit);
            break;
        }
        if (tid == ISSUER) {
            if (g + (int)gridDim.x < nblocks) {
                bulk_wait_read0();  // the other stage's store has left shared memory
                issue(it + 1, g + gridDim.x, n1);
            }
            n1 = n2;
            parent(g + 2 * (int)gridDim.x, n1);
            own(g + 3 * (int)gridDim.x, n2);
        }
        T *st = stage0 + (it & 1) * STAGE;
        const BlockDesc &b = *reinterpret_cast<const BlockDesc *>(st);
        const LevelDesc &L = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st) + sizeof(BlockDesc));
        T *xs = st + DESC + PD;
        const T *px = xs + C, *pg = px + C, *pv = pg + GH, *pvg = pv + C;
        // correct this thread's 4 cells, (c0 + c_x + c_y + c_z)/4 of x^H - x^H_old
        // (Sec. 2.3): parent cells p0, p0 + 1 of row (pj, pk), their x
        // neighbours p0 - 1, p0 + 2 and the two cells of the neighbour rows on
        // the cells' y and z sides, parent ghosts where these leave the parent
        T v[4];
        const int cfm = cf_faces(b, 3);
        {
            const int p0 = b.poff[0] + 2 * h, pj = b.poff[1] + (j >> 1), pk = b.poff[2] + (k >> 1);
            auto dx = [&](const T *x, const T *o, int idx) { return x[idx] - o[idx]; };
            const int row = 8 * (pj + 8 * pk);
            const T xm = p0 > 0 ? dx(px, pv, row + p0 - 1) : dx(pg, pvg, pj + 8 * pk);
            const T x0 = dx(px, pv, row + p0), x1 = dx(px, pv, row + p0 + 1);
            const T xp = p0 + 2 < n ? dx(px, pv, row + p0 + 2) : dx(pg, pvg, FC + pj + 8 * pk);
            const int qj = pj + sy, qk = pk + sz;
            const int ry = qj >= 0 && qj < n ? 8 * (qj + 8 * pk) : -1, rz = qk >= 0 && qk < n ? 8 * (pj + 8 * qk) : -1;
            const int gy = (qj < 0 ? 2 : 3) * FC + 8 * pk, gz = (qk < 0 ? 4 : 5) * FC + 8 * pj;
            const T y0 = ry >= 0 ? dx(px, pv, ry + p0) : dx(pg, pvg, gy + p0);
            const T y1 = ry >= 0 ? dx(px, pv, ry + p0 + 1) : dx(pg, pvg, gy + p0 + 1);
            const T z0 = rz >= 0 ? dx(px, pv, rz + p0) : dx(pg, pvg, gz + p0);
            const T z1 = rz >= 0 ? dx(px, pv, rz + p0 + 1) : dx(pg, pvg, gz + p0 + 1);
            const T c0[4] = {x0, x0, x1, x1}, cx[4] = {xm, x1, x0, xp};
            const T cy[4] = {y0, y0, y1, y1}, cz[4] = {z0, z0, z1, z1};
            T *xr = xs + 8 * r + 4 * h;
#pragma unroll
            for (int q = 0; q < 4; q += VW) vscatter(v + q, *reinterpret_cast<const V *>(xr + q));
#pragma unroll
            for (int q = 0; q < 4; q++) {
                T nbs = cx[q];
                nbs += cy[q];
                nbs += cz[q];
                v[q] = v[q] + (c0[q] + nbs) / (T)4;
            }
            // the corrected cells go straight to global memory (16-byte
            // stores, a warp's rows contiguous); the stage keeps them only
            // where refinement ghosts read other rows below
            V *xg = reinterpret_cast<V *>(F.X + b.cell_off + 8 * r + 4 * h);
#pragma unroll
            for (int q = 0; q < 4; q += VW) {
                V w;
                if constexpr (sizeof(T) == 4) w = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                else w = make_double2(v[q], v[q + 1]);
                xg[q / VW] = w;
                if (cfm) *reinterpret_cast<V *>(xr + q) = w;
            }
        }
        // same-level and physical ghosts of these cells, from registers
        {
            const int fx = h ? 1 : 0, nbx = b.nbr[fx];  // x face: the row's end cell
            const T ve = h ? v[3] : v[0];
            if (nbx >= 0) F.XG[b.push[fx] + j + 8 * k] = ve;
            else if (nbx == -1)
                F.XG[b.ghost_off + fx * FC + j + 8 * k] =
                    phys_ghost<T>(P, L, fx, ve, bc_value(P, L, b, 3, fx, I3{h ? n - 1 : 0, j, k}));
            auto face4 = [&](int face, int u0, int t1) {  // 4 cells at u0.. on face, t1: their second coordinate
                const int nb = b.nbr[face];
                if (nb >= 0) {
                    T *dst = F.XG + b.push[face] + u0;
#pragma unroll
                    for (int q = 0; q < 4; q += VW) {
                        V w;
                        if constexpr (sizeof(T) == 4) w = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                        else w = make_double2(v[q], v[q + 1]);
                        *reinterpret_cast<V *>(dst + q) = w;
                    }
                } else if (nb == -1) {
                    const int d = face >> 1, edge = (face & 1) ? n - 1 : 0;
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const I3 ii = d == 1 ? I3{4 * h + q, edge, t1} : I3{4 * h + q, t1, edge};
                        F.XG[b.ghost_off + face * FC + u0 + q] =
                            phys_ghost<T>(P, L, face, v[q], bc_value(P, L, b, 3, face, ii));
                    }
                }
            };
            if (j == 0 || j == n - 1) face4(j ? 3 : 2, 4 * h + 8 * k, k);  // y face: u = i + 8 k
            if (k == 0 || k == n - 1) face4(k ? 5 : 4, 4 * h + 8 * j, j);  // z face: u = i + 8 j
        }
        if (cfm) {
            __syncthreads();  // the updated rows in the stage
            for (int t = tid; t < GH; t += 128) {
                const int face = t / FC, u = t - face * FC;
                if (!((cfm >> face) & 1)) continue;
                const I3 ii = face_cell<3>(n, face, u, false);
                I3 dd = ii;
                put(dd, face >> 1, (face & 1) ? n - 2 : 1);
                F.XG[b.ghost_off + t] = cf_ghost<T, 3>(P, L, b, face, ii, xs[cidx<3>(n, ii.x, ii.y, ii.z)],
                                                       xs[cidx<3>(n, dd.x, dd.y, dd.z)], F.X, F.XG, b.nbr[face], false);
            }
        }
        // no barrier here: the next iteration's wait barrier already orders
        // this block's stage reads before the refill of this stage
    }
    if (tid == ISSUER) bulk_wait0();
}

// k_prolong_rows for 2D 16^2 blocks with 16^2 parents (64 threads): thread
// (j, q) corrects cells 4q .. 4q + 3 of fine row j, (2 c0 + c_x + c_y)/4 of
// x^H - x^H_old from parent cells p0, p0 + 1 of row pj, their x neighbours
// and the two cells of row pj +- 1 on the cells' y side.  Same staging and
// arithmetic as k_prolong_tma<T, 2, 16>.
template <class T>
__global__ void __launch_bounds__(64) k_prolong_rows2(KParams P, int first, int nblocks, Fields<T> F) {
    pdl_entry();
    constexpr int n = 16, C = 256, FC = 16, GH = 64;
    constexpr int DESC = (int)((sizeof(BlockDesc) + sizeof(LevelDesc)) / sizeof(T));
    constexpr int PD = (int)(sizeof(BlockDesc) / sizeof(T));
    constexpr int STAGE = DESC + PD + C + 2 * (C + GH);
    using V = typename Vec16<T>::type;
    constexpr int VW = 16 / sizeof(T);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    T *stage0 = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x;
    constexpr int ISSUER = 63;  // stage copies and stores
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    auto issue = [&](int it, int g) {  // thread ISSUER only
        T *st = stage0 + (it & 1) * STAGE;
        const BlockDesc *bd = P.B + g;
        const int par = bd->parent;
        const long long co = bd->cell_off, pco = P.B[par].cell_off, pgo = P.B[par].ghost_off;
        uint64_t *bar = &bars[it & 1];
        fence_async_smem();
        mbar_expect_tx(bar, (uint32_t)(sizeof(T) * STAGE));
        bulk_g2s(st, bd, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st) + sizeof(BlockDesc), P.L + bd->lev, sizeof(LevelDesc), bar);
        bulk_g2s(st + DESC, P.B + par, sizeof(BlockDesc), bar);
        T *d = st + DESC + PD;
        bulk_g2s(d, F.X + co, sizeof(T) * C, bar);
        bulk_g2s(d + C, F.X + pco, sizeof(T) * C, bar);
        bulk_g2s(d + 2 * C, F.XG + pgo, sizeof(T) * GH, bar);
        bulk_g2s(d + 2 * C + GH, F.V + pco, sizeof(T) * C, bar);
        bulk_g2s(d + 3 * C + GH, F.VG + pgo, sizeof(T) * GH, bar);
    };
    int g = blockIdx.x;
    if (tid == ISSUER && g < nblocks) issue(0, first + g);
    const int j = tid >> 2, qd = tid & 3, sy = (j & 1) ? 1 : -1;
    for (int it = 0; g < nblocks; it++, g += gridDim.x) {
        if (!mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, P.wait_limit)) {
            atomicExch(P.status, 1);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) {
            // the copy this wait was for may still be landing in shared
            // memory: let it arrive (normal bound) before the CTA exits
            if (tid == 0) mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, kWaitLimit);
            break;
        }
        if (tid == ISSUER && g + (int)gridDim.x < nblocks) {
            bulk_wait_read0();  // the other stage's store has left shared memory
            issue(it + 1, first + g + gridDim.x);
        }
        T *st = stage0 + (it & 1) * STAGE;
        const BlockDesc &b = *reinterpret_cast<const BlockDesc *>(st);
        const LevelDesc &L = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st) + sizeof(BlockDesc));
        T *xs = st + DESC + PD;
        const T *px = xs + C, *pg = px + C, *pv = pg + GH, *pvg = pv + C;
        T v[4];
        {
            const int p0 = b.poff[0] + 2 * qd, pj = b.poff[1] + (j >> 1), qj = pj + sy;
            auto dx = [&](const T *x, const T *o, int idx) { return x[idx] - o[idx]; };
            const int row = n * pj;
            const T xm = p0 > 0 ? dx(px, pv, row + p0 - 1) : dx(pg, pvg, pj);
            const T x0 = dx(px, pv, row + p0), x1 = dx(px, pv, row + p0 + 1);
            const T xp = p0 + 2 < n ? dx(px, pv, row + p0 + 2) : dx(pg, pvg, FC + pj);
            const int ry = qj >= 0 && qj < n ? n * qj : -1, gy = (qj < 0 ? 2 : 3) * FC;
            const T y0 = ry >= 0 ? dx(px, pv, ry + p0) : dx(pg, pvg, gy + p0);
            const T y1 = ry >= 0 ? dx(px, pv, ry + p0 + 1) : dx(pg, pvg, gy + p0 + 1);
            const T c0[4] = {x0, x0, x1, x1}, cx[4] = {xm, x1, x0, xp}, cy[4] = {y0, y0, y1, y1};
            T *xr = xs + n * j + 4 * qd;
#pragma unroll
            for (int q = 0; q < 4; q += VW) vscatter(v + q, *reinterpret_cast<const V *>(xr + q));
#pragma unroll
            for (int q = 0; q < 4; q++) {
                T nbs = cx[q];
                nbs += cy[q];
                v[q] = v[q] + ((T)2 * c0[q] + nbs) / (T)4;
            }
#pragma unroll
            for (int q = 0; q < 4; q += VW) {
                V w;
                if constexpr (sizeof(T) == 4) w = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                else w = make_double2(v[q], v[q + 1]);
                *reinterpret_cast<V *>(xr + q) = w;
            }
        }
        // same-level and physical ghosts of these cells, from registers
        if (qd == 0 || qd == 3) {  // x faces: the row's end cells
            const int fx = qd ? 1 : 0, nbx = b.nbr[fx];
            const T ve = qd ? v[3] : v[0];
            if (nbx >= 0) F.XG[b.push[fx] + j] = ve;
            else if (nbx == -1)
                F.XG[b.ghost_off + fx * FC + j] = phys_ghost<T>(P, L, fx, ve, bc_value(P, L, b, 2, fx, I3{qd ? n - 1 : 0, j, 0}));
        }
        if (j == 0 || j == n - 1) {  // y faces: 4 cells, contiguous in the ghost face (u = i)
            const int face = j ? 3 : 2, nb = b.nbr[face];
            if (nb >= 0) {
                T *dst = F.XG + b.push[face] + 4 * qd;
#pragma unroll
                for (int q = 0; q < 4; q += VW) {
                    V w;
                    if constexpr (sizeof(T) == 4) w = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                    else w = make_double2(v[q], v[q + 1]);
                    *reinterpret_cast<V *>(dst + q) = w;
                }
            } else if (nb == -1) {
#pragma unroll
                for (int q = 0; q < 4; q++)
                    F.XG[b.ghost_off + face * FC + 4 * qd + q] =
                        phys_ghost<T>(P, L, face, v[q], bc_value(P, L, b, 2, face, I3{4 * qd + q, j, 0}));
            }
        }
        fence_async_smem();
        __syncthreads();
        if (tid == ISSUER) {
            bulk_s2g(F.X + b.cell_off, xs, sizeof(T) * C);
            bulk_commit();
        }
        const int cfm = cf_faces(b, 2);
        if (cfm)
            for (int t = tid; t < GH; t += 64) {
                const int face = t / FC, u = t - face * FC;
                if (!((cfm >> face) & 1)) continue;
                const I3 ii = face_cell<2>(n, face, u, false);
                I3 dd = ii;
                put(dd, face >> 1, (face & 1) ? n - 2 : 1);
                F.XG[b.ghost_off + t] = cf_ghost<T, 2>(P, L, b, face, ii, xs[cidx<2>(n, ii.x, ii.y, ii.z)],
                                                       xs[cidx<2>(n, dd.x, dd.y, dd.z)], F.X, F.XG, b.nbr[face], false);
            }
        __syncthreads();  // stage reads done before the next block
    }
    if (tid == ISSUER) bulk_wait0();
}

// Restriction with the FAS residual for 8- and 16-cell blocks, persistent
// and TMA-staged like the sweep: the child block (descriptor, x, ghosts, f,
// eps) and its parent's descriptor arrive by cp.async.bulk; child residuals
// are formed from shared memory, then each parent cell under the child gets
// the mean of its children and the parent-level ghosts are pushed (see
// k_restrict_push).
template <class T, int D, int NT>
__global__ void __launch_bounds__(transfer_bound(D, NT), (D == 3 && NT == 16) ? 1 : 4) k_restrict_tma(KParams P, int first, int nblocks, Fields<T> F) {
    pdl_entry();
    constexpr int n = NT, m = NT / 2, C = cells_of<D>(NT), FC = face_of<D>(NT), GH = 2 * D * FC;
    constexpr int M = cells_of<D>(m);
    constexpr int DESC = (int)((sizeof(BlockDesc) + sizeof(LevelDesc)) / sizeof(T));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ __align__(16) LevelDesc sL, sPL;
    __shared__ int s_abort;
    __shared__ __align__(16) T rs[C];
    const bool var = F.E != nullptr, wc = F.W != nullptr;
    const int stage_elems = 2 * DESC + 2 * C + GH + (wc ? 2 * D * C : (var ? C + GH : 0));
    T *stage0 = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const uint32_t tx_bytes = (uint32_t)(sizeof(T) * stage_elems);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    if (tid < (int)(sizeof(LevelDesc) / 4)) {
        const BlockDesc &b0 = P.B[first];
        reinterpret_cast<int *>(&sL)[tid] = reinterpret_cast<const int *>(P.L + b0.lev)[tid];
        reinterpret_cast<int *>(&sPL)[tid] = reinterpret_cast<const int *>(P.L + P.B[b0.parent].lev)[tid];
    }
    __syncthreads();
    auto issue = [&](int it, int g) {
        T *st = stage0 + (it & 1) * stage_elems;
        const long long co = P.B[g].cell_off, go = P.B[g].ghost_off;
        const int par = P.B[g].parent;
        uint64_t *bar = &bars[it & 1];
        fence_async_smem();
        mbar_expect_tx(bar, tx_bytes);
        bulk_g2s(st, P.B + g, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st) + sizeof(BlockDesc), P.L + P.B[g].lev, sizeof(LevelDesc), bar);
        bulk_g2s(st + DESC, P.B + par, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st + DESC) + sizeof(BlockDesc), P.L + P.B[par].lev, sizeof(LevelDesc), bar);
        bulk_g2s(st + 2 * DESC, F.X + co, sizeof(T) * C, bar);
        bulk_g2s(st + 2 * DESC + C, F.XG + go, sizeof(T) * GH, bar);
        bulk_g2s_f<T>(st + 2 * DESC + C + GH, F.F + co, sizeof(T) * C, bar);
        if (wc) {
            bulk_g2s(st + 2 * DESC + 2 * C + GH, F.W + co * wstride(D), sizeof(T) * 2 * D * C, bar);
        } else if (var) {
            bulk_g2s_f<T>(st + 2 * DESC + 2 * C + GH, F.E + co, sizeof(T) * C, bar);
            bulk_g2s_f<T>(st + 2 * DESC + 3 * C + GH, F.EG + go, sizeof(T) * GH, bar);
        }
    };
    int g = blockIdx.x;
    if (tid == 0 && g < nblocks) issue(0, first + g);
    // level descriptor: CTA-wide copy when every block shares it, else per block
    const bool cyl = P.geom == MG_CYL;
    for (int it = 0; g < nblocks; it++, g += gridDim.x) {
        if (!mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, P.wait_limit)) {
            atomicExch(P.status, 1);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) {
            // the copy this wait was for may still be landing in shared
            // memory: let it arrive (normal bound) before the CTA exits
            if (tid == 0) mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, kWaitLimit);
            break;
        }
        if (tid == 0 && g + (int)gridDim.x < nblocks) issue(it + 1, first + g + gridDim.x);
        const T *st = stage0 + (it & 1) * stage_elems;
        const BlockDesc &b = *reinterpret_cast<const BlockDesc *>(st);
        const BlockDesc &p = *reinterpret_cast<const BlockDesc *>(st + DESC);
        const LevelDesc &L = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st) + sizeof(BlockDesc));
        const T lo0 = kp_lo0<T>(P), h0 = lv_h0<T>(L);  // operator scalars in the kernel precision
        const T ih0 = lv_ih<T>(L, 0), ih1 = lv_ih<T>(L, 1), ih2 = lv_ih<T>(L, 2);
        const LevelDesc &PL = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st + DESC) + sizeof(BlockDesc));
        const T *xs = st + 2 * DESC, *gs = xs + C, *fs = gs + GH, *es = fs + C, *egs = es + C;
        auto nbv = [&](const T *xi, const T *gi, int i, int j, int k, int d, int s) -> T {
            const int o = s ? 1 : -1;
            if (d == 0) {
                const int ii = i + o;
                if (ii < 0 || ii >= n) return gi[(s ? 1 : 0) * FC + (D == 2 ? j : j + n * k)];
                return xi[cidx<D>(n, ii, j, k)];
            }
            if (d == 1) {
                const int jj = j + o;
                if (jj < 0 || jj >= n) return gi[(s ? 3 : 2) * FC + (D == 2 ? i : i + n * k)];
                return xi[cidx<D>(n, i, jj, k)];
            }
            const int kk = k + o;
            if (kk < 0 || kk >= n) return gi[(s ? 5 : 4) * FC + i + n * j];
            return xi[cidx<D>(n, i, j, kk)];
        };
        // child residuals (same arithmetic as the stencil helper)
        for (int c = tid; c < C; c += nth) {
            const int i = c % n, j = (c / n) % n, k = D == 3 ? c / (n * n) : 0;
            const T xc = xs[c];
            if (wc) {  // same terms and order as below, coefficients read
                T lap = 0;
#pragma unroll
                for (int f = 0; f < 2 * D; f++) lap += es[f * C + c] * (nbv(xs, gs, i, j, k, f >> 1, f & 1) - xc);
                rs[c] = fs[c] - (lap - kp_helm<T>(P) * xc);
                continue;
            }
            const T ec = var ? es[c] : (T)1;
            T lap = 0, ri = 0;
            if (cyl) ri = lo0 + ((T)(b.ijk[0] * n + i) + (T)0.5) * h0;
#pragma unroll
            for (int d = 0; d < D; d++)
#pragma unroll
                for (int s = 0; s < 2; s++) {
                    T w = d == 0 ? ih0 : (d == 1 ? ih1 : ih2);
                    if (var) {
                        const T en = nbv(es, egs, i, j, k, d, s);
                        w *= qdiv<T>((T)2 * ec * en, ec + en);
                    }
                    if (cyl && d == 0) w *= qdiv<T>(lo0 + (T)(b.ijk[0] * n + i + s) * h0, ri);
                    lap += w * (nbv(xs, gs, i, j, k, d, s) - xc);
                }
            rs[c] = fs[c] - (lap - kp_helm<T>(P) * xc);
        }
        __syncthreads();
        const int pn = p.n;
        for (int c = tid; c < M; c += nth) {
            const int ci = c % m, cj = (c / m) % m, ck = D == 3 ? c / (m * m) : 0;
            T sx = 0, sr = 0;
#pragma unroll
            for (int ch = 0; ch < (1 << D); ch++) {
                const int fc = cidx<D>(n, 2 * ci + (ch & 1), 2 * cj + ((ch >> 1) & 1), D == 3 ? 2 * ck + ((ch >> 2) & 1) : 0);
                sx += xs[fc];
                sr += rs[fc];
            }
            const int pc = cidx<D>(pn, b.poff[0] + ci, b.poff[1] + cj, b.poff[2] + ck);
            F.X[p.cell_off + pc] = sx * (T)(1.0 / (1 << D));
            F.F[p.cell_off + pc] = sr * (T)(1.0 / (1 << D));
        }
        __syncthreads();  // rs is reused below for the octant values
        for (int c = tid; c < M; c += nth) {
            const int ci = c % m, cj = (c / m) % m, ck = D == 3 ? c / (m * m) : 0;
            T sx = 0;
#pragma unroll
            for (int ch = 0; ch < (1 << D); ch++)
                sx += xs[cidx<D>(n, 2 * ci + (ch & 1), 2 * cj + ((ch >> 1) & 1), D == 3 ? 2 * ck + ((ch >> 2) & 1) : 0)];
            rs[c] = sx * (T)(1.0 / (1 << D));
        }
        __syncthreads();
        const int Fm = face_of<D>(m);
        auto val = [&](I3 q) { return rs[cidx<D>(m, q.x - b.poff[0], q.y - b.poff[1], q.z - b.poff[2])]; };
        for (int t = tid; t < 2 * D * Fm; t += nth) {
            const int face = t / Fm, v = t - face * Fm, d = face >> 1, s = face & 1;
            const int off = d == 0 ? b.poff[0] : d == 1 ? b.poff[1] : b.poff[2];
            if (s ? (off + m != pn) : (off != 0)) continue;
            I3 ii = face_cell<D>(m, face, v, false);
            ii.x += b.poff[0];
            ii.y += b.poff[1];
            ii.z += D == 3 ? b.poff[2] : 0;
            put(ii, d, s ? pn - 1 : 0);
            int u;
            if (D == 2) u = d == 0 ? ii.y : ii.x;
            else u = d == 0 ? ii.y + pn * ii.z : (d == 1 ? ii.x + pn * ii.z : ii.x + pn * ii.y);
            push_face_cell<T, D>(P, PL, p, face, u, ii, F.X, F.XG, val);
        }
    }
}

// Row-wise form of k_restrict_tma for 3D 8^3 blocks with 8^3 parents and
// the constant-coefficient Cartesian operator (128 threads).  Each thread
// takes half a fine row (4 cells): its rows and ghost rows come in with
// vector loads, it forms the 4 child residuals (same terms and order as
// k_restrict_tma), sums x and the residual over the cell pairs under each
// parent cell, and two warp shuffles add the other three rows of the 2x2x2
// children (j +- 1: lane ^ 2, k +- 1: lane ^ 16).  One thread per parent cell
// pair then stores the means; the parent ghosts beside the octant are pushed
// from a small shared copy, as in k_restrict_tma.
template <class T>
__global__ void __launch_bounds__(128) k_restrict_rows(KParams P, int first, int nblocks, Fields<T> F) {
    pdl_entry();
    constexpr int n = 8, C = 512, FC = 64, GH = 384;
    constexpr int DESC = (int)((sizeof(BlockDesc) + sizeof(LevelDesc)) / sizeof(T));
    constexpr int STAGE = 2 * DESC + 2 * C + GH;
    using V = typename Vec16<T>::type;
    constexpr int VW = 16 / sizeof(T);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    __shared__ T oct[64];  // parent cells under the block, [ck][cj][ci]
    T *stage0 = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x;
    constexpr int ISSUER = 127;  // stage copies
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    // offsets of a block and its parent for the stage copies; the issuer
    // reads them two iterations ahead (the block's own fields one iteration
    // before its parent's), so that a refill never waits on the table
    struct Src { long long co, go; int par, lev, plev; };
    auto own = [&](int g, Src &r) {
        if (g < nblocks) {
            const BlockDesc &q = P.B[first + g];
            r.co = q.cell_off; r.go = q.ghost_off; r.par = q.parent; r.lev = q.lev;
        }
    };
    auto parent = [&](int g, Src &r) {
        if (g < nblocks) r.plev = P.B[r.par].lev;
    };
    auto issue = [&](int it, int g, const Src &r) {  // thread ISSUER only
        T *st = stage0 + (it & 1) * STAGE;
        uint64_t *bar = &bars[it & 1];
        fence_async_smem();
        mbar_expect_tx(bar, (uint32_t)(sizeof(T) * STAGE));
        bulk_g2s(st, P.B + first + g, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st) + sizeof(BlockDesc), P.L + r.lev, sizeof(LevelDesc), bar);
        bulk_g2s(st + DESC, P.B + r.par, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st + DESC) + sizeof(BlockDesc), P.L + r.plev, sizeof(LevelDesc), bar);
        bulk_g2s(st + 2 * DESC, F.X + r.co, sizeof(T) * C, bar);
        bulk_g2s(st + 2 * DESC + C, F.XG + r.go, sizeof(T) * GH, bar);
        bulk_g2s_f<T>(st + 2 * DESC + C + GH, F.F + r.co, sizeof(T) * C, bar);
    };
    int g = blockIdx.x;
    Src n1{}, n2{};
    if (tid == ISSUER) {
        if (g < nblocks) {
            Src r0{};
            own(g, r0);
            parent(g, r0);
            issue(0, g, r0);
        }
        own(g + (int)gridDim.x, n1);
        parent(g + (int)gridDim.x, n1);
        own(g + 2 * (int)gridDim.x, n2);
    }
    const int r = tid >> 1, h = tid & 1, j = r & 7, k = r >> 3;
    auto ld4 = [&](const T *src, T *dst) {
#pragma unroll
        for (int q = 0; q < 4; q += VW) vscatter(dst + q, *reinterpret_cast<const V *>(src + q));
    };
    for (int it = 0; g < nblocks; it++, g += gridDim.x) {
        if (!mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, P.wait_limit)) {
            atomicExch(P.status, 1);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) {
            // the copy this wait was for may still be landing in shared
            // memory: let it arrive (normal bound) before the CTA exits
            if (tid == 0) mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, kWaitLimit);
            break;
        }
        if (tid == ISSUER) {
            if (g + (int)gridDim.x < nblocks) issue(it + 1, g + gridDim.x, n1);
            n1 = n2;
            parent(g + 2 * (int)gridDim.x, n1);
            own(g + 3 * (int)gridDim.x, n2);
        }
        const T *st = stage0 + (it & 1) * STAGE;
        const BlockDesc &b = *reinterpret_cast<const BlockDesc *>(st);
        const BlockDesc &p = *reinterpret_cast<const BlockDesc *>(st + DESC);
        const LevelDesc &L = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st) + sizeof(BlockDesc));
        const LevelDesc &PL = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st + DESC) + sizeof(BlockDesc));
        const T *xs = st + 2 * DESC, *gs = xs + C, *fs = gs + GH;
        const T w0 = lv_ih<T>(L, 0), w1 = lv_ih<T>(L, 1), w2 = lv_ih<T>(L, 2), helm = kp_helm<T>(P);
        // x of cells 4h - 1 .. 4h + 4 of row (j, k) and the 4 cells of the
        // neighbour rows (face ghost rows outside the block)
        T xr[6], dn[4], up[4], bk[4], fw[4], f4[4];
        ld4(xs + 8 * r + 4 * h, xr + 1);
        xr[0] = h ? xs[8 * r + 3] : gs[j + 8 * k];
        xr[5] = h ? gs[FC + j + 8 * k] : xs[8 * r + 4];
        ld4(j > 0 ? xs + 8 * (r - 1) + 4 * h : gs + 2 * FC + 4 * h + 8 * k, dn);
        ld4(j < n - 1 ? xs + 8 * (r + 1) + 4 * h : gs + 3 * FC + 4 * h + 8 * k, up);
        ld4(k > 0 ? xs + 8 * (r - 8) + 4 * h : gs + 4 * FC + 4 * h + 8 * j, bk);
        ld4(k < n - 1 ? xs + 8 * (r + 8) + 4 * h : gs + 5 * FC + 4 * h + 8 * j, fw);
        ld4(fs + 8 * r + 4 * h, f4);
        T res[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const T xc = xr[1 + q];
            T lap = 0;
            lap += w0 * (xr[q] - xc);
            lap += w0 * (xr[q + 2] - xc);
            lap += w1 * (dn[q] - xc);
            lap += w1 * (up[q] - xc);
            lap += w2 * (bk[q] - xc);
            lap += w2 * (fw[q] - xc);
            res[q] = f4[q] - (lap - helm * xc);
        }
        // sums under parent cells 2h, 2h + 1: this row's pairs, then rows j ^ 1, k ^ 1
        T s4[4] = {xr[1] + xr[2], xr[3] + xr[4], res[0] + res[1], res[2] + res[3]};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            s4[q] += __shfl_xor_sync(0xffffffffu, s4[q], 2);
            s4[q] += __shfl_xor_sync(0xffffffffu, s4[q], 16);
        }
        if (!(j & 1) && !(k & 1)) {
            const int ci = 2 * h, cj = j >> 1, ck = k >> 1;
            const T inv = (T)(1.0 / 8);
            const int pc = cidx<3>(n, b.poff[0] + ci, b.poff[1] + cj, b.poff[2] + ck);
            F.X[p.cell_off + pc] = s4[0] * inv;
            F.X[p.cell_off + pc + 1] = s4[1] * inv;
            F.F[p.cell_off + pc] = s4[2] * inv;
            F.F[p.cell_off + pc + 1] = s4[3] * inv;
            oct[(ck * 4 + cj) * 4 + ci] = s4[0] * inv;
            oct[(ck * 4 + cj) * 4 + ci + 1] = s4[1] * inv;
        }
        __syncthreads();
        // parent ghosts beside the octant: faces where it meets the parent's boundary
        if (tid < 96) {
            const int face = tid >> 4, v = tid & 15, d = face >> 1, s = face & 1;
            const int off = d == 0 ? b.poff[0] : d == 1 ? b.poff[1] : b.poff[2];
            if (s ? (off + 4 == n) : (off == 0)) {
                const int a = v & 3, c = v >> 2, e = s ? 3 : 0, e2 = s ? 2 : 1;  // octant-local
                const I3 lo = d == 0 ? I3{e, a, c} : (d == 1 ? I3{a, e, c} : I3{a, c, e});
                const I3 li = d == 0 ? I3{e2, a, c} : (d == 1 ? I3{a, e2, c} : I3{a, c, e2});
                const I3 ii{b.poff[0] + lo.x, b.poff[1] + lo.y, b.poff[2] + lo.z};
                const int u = d == 0 ? ii.y + n * ii.z : (d == 1 ? ii.x + n * ii.z : ii.x + n * ii.y);
                const T cv = oct[(lo.z * 4 + lo.y) * 4 + lo.x];
                const int nb = p.nbr[face];
                if (nb >= 0) {
                    F.XG[p.push[face] + u] = cv;
                } else if (nb == -1) {
                    F.XG[p.ghost_off + face * FC + u] = phys_ghost<T>(P, PL, face, cv, bc_value(P, PL, p, 3, face, ii));
                } else {
                    F.XG[p.ghost_off + face * FC + u] =
                        cf_ghost<T, 3>(P, PL, p, face, ii, cv, oct[(li.z * 4 + li.y) * 4 + li.x], F.X, F.XG, nb, false);
                }
            }
        }
        __syncthreads();  // oct and stage reads done before the next block
    }
}

// ---------------------------------------------- divergence cleaning -----
// Second-order central differences on leaf blocks (Sec. 4.1): component d of
// a vector field X (with ghosts) adds (X(c+e_d) - X(c-e_d)) / (2 h_d) to the
// divergence; the projection writes B_d - (phi(c+e_d) - phi(c-e_d)) / (2 h_d).
template <int D>
__global__ void __launch_bounds__(kMaxThreads) k_div_comp(KParams P, int first, const double *__restrict__ X,
                                                          const double *__restrict__ XG, int d,
                                                          double *__restrict__ out, long long leaf_base, int add,
                                                          int order) {
    pdl_entry();
    __shared__ BlockDesc sb;
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, C = cells_of<D>(n);
    const double s2h = 0.5 / L.h[d];
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        const int ox = d == 0, oy = d == 1, oz = d == 2;
        const double bp = load<double, D>(X, XG, b, i + ox, j + oy, k + oz);
        const double bm = load<double, D>(X, XG, b, i - ox, j - oy, k - oz);
        double v = (bp - bm) * s2h;
        if (order == 4) {
            // cells two away: in this block or the same-level neighbour block
            // across the face (fourth order only where both exist, reading R14)
            bool okp, okm;
            auto far = [&](int off, bool &ok) -> double {
                I3 q{i, j, k};
                const int qd = get(q, d) + off;
                if (qd >= 0 && qd < n) {
                    put(q, d, qd);
                    ok = true;
                    return X[b.cell_off + cidx<D>(n, q.x, q.y, q.z)];
                }
                const int nb = b.nbr[2 * d + (off > 0 ? 1 : 0)];
                if (nb < 0) {
                    ok = false;
                    return 0.0;
                }
                put(q, d, qd - (off > 0 ? n : -n));
                ok = true;
                return X[P.B[nb].cell_off + cidx<D>(n, q.x, q.y, q.z)];
            };
            const double bpp = far(2, okp), bmm = far(-2, okm);
            if (okp && okm) v = (-bpp + 8.0 * bp - 8.0 * bm + bmm) / (12.0 * L.h[d]);
        }
        const long long m = leaf_base + (long long)blockIdx.x * C + c;
        out[m] = add ? out[m] + v : v;
    }
}

template <int D>
__global__ void __launch_bounds__(kMaxThreads) k_grad_sub(KParams P, int first, const double *__restrict__ X,
                                                          const double *__restrict__ XG, int d,
                                                          const double *__restrict__ Bin, double *__restrict__ Bout,
                                                          long long leaf_base) {
    pdl_entry();
    __shared__ BlockDesc sb;
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, C = cells_of<D>(n);
    const double s2h = 0.5 / L.h[d];
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        const int ox = d == 0, oy = d == 1, oz = d == 2;
        const double gd = (load<double, D>(X, XG, b, i + ox, j + oy, k + oz) -
                           load<double, D>(X, XG, b, i - ox, j - oy, k - oz)) * s2h;
        const long long m = leaf_base + (long long)blockIdx.x * C + c;
        Bout[m] = Bin[m] - gd;
    }
}

// ------------------------------------------------------ residual norm ---
// Composite residual on leaf blocks [first, first + gridDim.x): per-CTA
// partial sums of V r^2 and V and the max |r| (warp shuffles, then shared
// memory); optional r in leaf order and (float) r into FP32 cells.  MX off
// (the solve loops, which read only the L2 norm): r^2 accumulated in FP32
// from the FP32-rounded residual and scaled by the block's cell volume once,
// no max -- the FP64 work per cell is then the operator alone.  NT > 0: the
// block size at compile time and kMaxThreads threads, so that a thread's
// cells form a fixed loop the compiler unrolls (the loads of several cells
// are in flight before their FP64 arithmetic, which on GB300 holds a warp
// for many cycles per instruction).
template <int D, bool MX = true, int NT = 0>
__global__ void __launch_bounds__(kMaxThreads, NT ? 3 : 2) k_resnorm(KParams P, int first, Fields<double> F,
                                                         double *__restrict__ partials,
                                                         double *__restrict__ rleaf, long long leaf_base,
                                                         long long cell_base, float *__restrict__ f32) {
    pdl_entry();
    __shared__ BlockDesc sb;
    stage_desc(P, first + blockIdx.x, sb);
    const BlockDesc &b = sb;
    const LevelDesc &L = P.L[b.lev];
    const int n = NT ? NT : b.n, C = cells_of<D>(n);
    const bool cyl = P.geom == MG_CYL, helm0 = P.helm == 0.0;
    double s2 = 0, sv = 0, mx = 0;
    float acc_r = 0.f, acc_v = 0.f;
    double vol = 1.0;
    for (int d = 0; d < D; d++) vol *= L.h[d];
    constexpr int PER = NT ? (cells_of<D>(NT) + kMaxThreads - 1) / kMaxThreads : 1;
    const int stride = NT ? kMaxThreads : (int)blockDim.x;
#pragma unroll 2
    for (int q = 0; q < (NT ? PER : (C + stride - 1) / stride); q++) {
        const int c = threadIdx.x + q * stride;
        if (c >= C) break;
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        double r;
        if (F.W) {  // precomputed face coefficients (the weights of the form below)
            const double xc = F.X[b.cell_off + c];
            const double lap = lap_w<D>(b, F.X, F.XG, F.W, i, j, k, xc);
            r = helm0 ? F.F[b.cell_off + c] - lap : F.F[b.cell_off + c] - (lap - P.helm * xc);
        } else {
            double lap, num, den, xc;
            stencil<double, double, D>(P, L, b, F.X, F.XG, F.E, F.EG, i, j, k, lap, num, den, xc);
            r = F.F[b.cell_off + c] - (lap - P.helm * xc);
        }
        const float rf = mg_to_float(r);  // integer rounding: no FP64-pipe conversion
        if (MX) {
            double V = vol;
            if (cyl) V = 2.0 * M_PI * (P.lo[0] + (b.ijk[0] * n + i + 0.5) * L.h[0]) * L.h[0] * L.h[1];
            s2 += V * r * r;
            sv += V;
            mx = fmax(mx, fabs(r));
        } else if (cyl) {
            const float Vf = (P.lo0f + ((float)(b.ijk[0] * n + i) + 0.5f) * L.h0f) * L.hvf;
            acc_r = fmaf(Vf * rf, rf, acc_r);
            acc_v += Vf;
        } else {
            acc_r = fmaf(rf, rf, acc_r);
        }
        if (rleaf) rleaf[leaf_base + (b.cell_off - cell_base) + c] = r;
        if (f32) f32[b.cell_off + c] = rf;
    }
    if (!MX) {
        for (int o = 16; o > 0; o >>= 1) {
            acc_r += __shfl_down_sync(0xffffffffu, acc_r, o);
            acc_v += __shfl_down_sync(0xffffffffu, acc_v, o);
        }
        __shared__ float shf[2][kMaxThreads / 32];
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
        if (lane == 0) { shf[0][w] = acc_r; shf[1][w] = acc_v; }
        __syncthreads();
        if (threadIdx.x == 0) {
            float a = 0.f, v = 0.f;
            for (int e = 0; e < nw; e++) { a += shf[0][e]; v += shf[1][e]; }
            partials[3 * blockIdx.x] = cyl ? (double)a : vol * (double)a;
            partials[3 * blockIdx.x + 1] = cyl ? (double)v : vol * C;
            partials[3 * blockIdx.x + 2] = 0.0;
        }
        return;
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

// Composite residual on the leaf blocks of one level, TMA-staged like the
// sweep: x, the face ghosts and f (and eps) of the next block arrive by
// cp.async.bulk while the current block is evaluated.  r = f - (L x - lambda x)
// is formed in FP64 with the difference form sum_d w_d ((x_- - x_c) +
// (x_+ - x_c)) (rounding error ~ eps |grad x| h rather than eps |x|).  Writes per-CTA partials (sum V r^2, sum V,
// max |r|) and optionally r (leaf order) and (float) r into FP32 cells.
// FP64 form of the constant-coefficient residual f - (sum_d w_d (x_d- + x_d+)
// - diag x_c), for the cells the integer sum declines (non-cubic cells, or
// inputs outside the normal range).  Not inlined: a short branch inlined into
// the cell loop is evaluated under a predicate for every cell, spending the
// FP64 pipe even where the integer sum was taken.
__device__ __noinline__ double resid_const_fp64(double xc, double a0, double a1, double b0, double b1, double c0,
                                                double c1, double f, double w0, double w1, double w2, double dg) {
    double sx = w0 * (a0 + a1);
    sx = fma(w1, b0 + b1, sx);
    sx = fma(w2, c0 + c1, sx);
    return f - fma(-dg, xc, sx);
}

// S 2^(emax - 1080) in FP64 arithmetic, for a result outside the normal range
// (not inlined, for the reason above).
__device__ __noinline__ double unfix_wide(int64_t S, int emax) { return ldexp((double)S, emax - 1080); }

template <int D, int NT, bool MX = true>
__global__ void __launch_bounds__(kMaxThreads, (NT == 8 || D == 2) ? 4 : 3) k_resid_tma(KParams P, int first, int nblocks, Fields<double> F,
                                                              double *__restrict__ partials,
                                                              double *__restrict__ rleaf, long long leaf_base,
                                                              float *__restrict__ f32, int per_block = 0) {
    pdl_entry();
    using T = double;
    constexpr int n = NT, C = cells_of<D>(NT), FC = face_of<D>(NT), GH = 2 * D * FC;
    constexpr int DESC = (int)((sizeof(BlockDesc) + sizeof(LevelDesc)) / sizeof(T));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ __align__(16) LevelDesc sL;
    __shared__ int s_abort;
    __shared__ double sred[3][kMaxThreads / 32];
    __shared__ float sredf[2][kMaxThreads / 32];
    __shared__ int semax[kMaxThreads / 32];
    const bool var = F.E != nullptr, wc = F.W != nullptr;  // wc: precomputed face coefficients
    const int stage_elems = DESC + 2 * C + GH + (wc ? (2 * D + 1) * C : (var ? C + GH : 0));
    T *stage0 = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const uint32_t tx_bytes = (uint32_t)(sizeof(T) * stage_elems);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    auto issue = [&](int it, int g) {
        T *st = stage0 + (it & 1) * stage_elems;
        const long long co = P.B[g].cell_off, go = P.B[g].ghost_off;
        uint64_t *bar = &bars[it & 1];
        fence_async_smem();
        mbar_expect_tx(bar, tx_bytes);
        bulk_g2s(st, P.B + g, sizeof(BlockDesc), bar);
        bulk_g2s(reinterpret_cast<char *>(st) + sizeof(BlockDesc), P.L + P.B[g].lev, sizeof(LevelDesc), bar);
        bulk_g2s(st + DESC, F.X + co, sizeof(T) * C, bar);
        bulk_g2s(st + DESC + C, F.XG + go, sizeof(T) * GH, bar);
        bulk_g2s(st + DESC + C + GH, F.F + co, sizeof(T) * C, bar);
        if (wc) {
            bulk_g2s(st + DESC + 2 * C + GH, F.W + co * wstride(D), sizeof(T) * (2 * D + 1) * C, bar);
        } else if (var) {
            bulk_g2s(st + DESC + 2 * C + GH, F.E + co, sizeof(T) * C, bar);
            bulk_g2s(st + DESC + 3 * C + GH, F.EG + go, sizeof(T) * GH, bar);
        }
    };
    int g = blockIdx.x;
    if (tid == 0 && g < nblocks) issue(0, first + g);
    const bool helm0 = P.helm == 0.0;  // Poisson: no lambda term
    const bool cyl = P.geom == MG_CYL;
    double s2 = 0, sv = 0;
    double mx = 0.0;
    // solve-loop norms (MX off) in FP32 across all blocks of the thread: no
    // FP64 work per block (every launch is one level of one tree, so the
    // Cartesian cell volume is uniform; the batch's per-block slots are
    // reduced in FP32 and scaled by thread 0)
    float acc_r = 0.f, acc_v = 0.f;
    double vol_u = 0;
    for (int it = 0; g < nblocks; it++, g += gridDim.x) {
        if (!mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, P.wait_limit)) {
            atomicExch(P.status, 1);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) {
            // the copy this wait was for may still be landing in shared
            // memory: let it arrive (normal bound) before the CTA exits
            if (tid == 0) mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, kWaitLimit);
            break;
        }
        if (tid == 0 && g + (int)gridDim.x < nblocks) issue(it + 1, first + g + gridDim.x);
        T *st = stage0 + (it & 1) * stage_elems;
        const BlockDesc &b = *reinterpret_cast<const BlockDesc *>(st);
        const LevelDesc &L = *reinterpret_cast<const LevelDesc *>(reinterpret_cast<const char *>(st) + sizeof(BlockDesc));
        const double w0 = L.inv_h2[0], w1 = L.inv_h2[1], w2 = L.inv_h2[2];
        const double vol = L.vol;
        T *xs = st + DESC;
        const T *gs = xs + C, *fs = gs + GH, *es = fs + C, *egs = es + C;
        auto nbv = [&](const T *xi, const T *gi, int i, int j, int k, int d, int s) -> T {
            const int o = s ? 1 : -1;
            if (d == 0) {
                const int ii = i + o;
                if (ii < 0 || ii >= n) return gi[(s ? 1 : 0) * FC + (D == 2 ? j : j + n * k)];
                return xi[cidx<D>(n, ii, j, k)];
            }
            if (d == 1) {
                const int jj = j + o;
                if (jj < 0 || jj >= n) return gi[(s ? 3 : 2) * FC + (D == 2 ? i : i + n * k)];
                return xi[cidx<D>(n, i, jj, k)];
            }
            const int kk = k + o;
            if (kk < 0 || kk >= n) return gi[(s ? 5 : 4) * FC + i + n * j];
            return xi[cidx<D>(n, i, j, kk)];
        };
        // A x as (sum_f w_f x_f) - (sum_f w_f + lambda) x_c: FP64 operations
        // are GB300's scarcest resource here; the rounding stays at
        // eps * sum_f w_f |x|, far below any tolerance the solves use
        const double dg = L.diag;
        // Cubic cells, constant coefficient, no Helmholtz term: the stencil
        // sum in exact integer arithmetic (mg_exact.h).  The block's values
        // and ghosts are aligned once to their largest exponent, in place in
        // the stage; per cell that leaves integer adds, one FP64 FMA and an
        // integer rounding to FP32 (GB300's FP64 pipe is 1/64 of FP32).
        // The aligned values go to a padded (n+2)^D array (interior at
        // (i+1, j+1, k+1), each face ghost at its outside position), so that
        // a cell's six neighbours are fixed offsets with no branch.
        const bool iso = !var && !cyl && helm0 && w0 == w1 && (D == 2 || w0 == w2);
        constexpr int W = n + 2, W2 = D == 3 ? W * W : 0;
        int64_t *xp = reinterpret_cast<int64_t *>(stage0 + 2 * stage_elems);  // allocated when !var && !wc
        int em = 0x7FF;
        if (iso) {
            int e = 1;
            for (int q = tid; q < C + GH; q += nth) e = max(e, mg_expo(xs[q]));
            e = __reduce_max_sync(0xffffffffu, e);
            if ((tid & 31) == 0) semax[tid >> 5] = e;
            __syncthreads();
            em = 1;
            for (int w = 0; w < (nth >> 5); w++) em = max(em, semax[w]);
            if (em != 0x7FF) {  // a non-finite value anywhere: the FP64 form below
                for (int q = tid; q < C + GH; q += nth) {
                    I3 p3;
                    if (q < C) p3 = I3{q % n, (q / n) % n, D == 3 ? q / (n * n) : 0};
                    else p3 = face_cell<D>(n, (q - C) / FC, (q - C) % FC, true);
                    xp[(D == 3 ? (p3.z + 1) * W2 : 0) + (p3.y + 1) * W + p3.x + 1] = mg_fix(xs[q], em);
                }
            }
            __syncthreads();
        }
        double bs2 = 0;
        const float lo0f = P.lo0f, h0f = L.h0f, hvf = L.hvf;
        vol_u = vol;
        for (int c = tid; c < C; c += nth) {
            const int i = c % n, j = (c / n) % n, k = D == 3 ? c / (n * n) : 0;
            double lap;  // A x + lambda x (the residual below subtracts lambda x)
            double r;
            if (iso && em != 0x7FF) {
                const int64_t *xc = xp + (D == 3 ? (k + 1) * W2 : 0) + (j + 1) * W + i + 1;
                int64_t S = (xc[-1] + xc[1]) + (xc[-W] + xc[W]) - (int64_t)(2 * D) * xc[0];
                if (D == 3) S += xc[-W2] + xc[W2];
                double sd;
                if (!mg_unfix(S, em, sd)) sd = unfix_wide(S, em);  // outside the normal range
                r = fma(-w0, sd, fs[c]);
                lap = 0;
            } else if (!var && !cyl) {
                const double xc = xs[c];
                r = resid_const_fp64(xc, nbv(xs, gs, i, j, k, 0, 0), nbv(xs, gs, i, j, k, 0, 1),
                                     nbv(xs, gs, i, j, k, 1, 0), nbv(xs, gs, i, j, k, 1, 1),
                                     D == 3 ? nbv(xs, gs, i, j, k, 2, 0) : 0.0, D == 3 ? nbv(xs, gs, i, j, k, 2, 1) : 0.0,
                                     fs[c], w0, w1, D == 3 ? w2 : 0.0, dg);
                lap = 0;
            } else if (wc) {
                // r = f + w_diag x_c - sum_f w_f x_f: 2D + 1 FMAs, the FP64
                // issue cost of the variable-coefficient residual
                const double xc = xs[c];
                const double *ws = es + c;  // coefficients [face][cell], the diagonal last
                r = fma(ws[2 * D * C], xc, fs[c]);
#pragma unroll
                for (int f = 0; f < 2 * D; f++) r = fma(-ws[f * C], nbv(xs, gs, i, j, k, f >> 1, f & 1), r);
                lap = 0;
            } else {
                const double xc = xs[c];
                const double ec = var ? es[c] : 1.0;
                double ri = 0;
                if (cyl) ri = P.lo[0] + (b.ijk[0] * n + i + 0.5) * L.h[0];
                lap = 0;
#pragma unroll
                for (int d = 0; d < D; d++)
#pragma unroll
                    for (int s = 0; s < 2; s++) {
                        double w = L.inv_h2[d];
                        if (var) {
                            const double en = nbv(es, egs, i, j, k, d, s);
                            w *= 2.0 * ec * en / (ec + en);
                        }
                        if (cyl && d == 0) w *= (P.lo[0] + (b.ijk[0] * n + i + s) * L.h[0]) / ri;
                        lap += w * (nbv(xs, gs, i, j, k, d, s) - xc);
                    }
                r = helm0 ? fs[c] - lap : fs[c] - (lap - P.helm * xc);
            }
            const float rf = mg_to_float(r);  // integer rounding: no FP64-pipe conversion
            if (MX) {
                if (cyl) {
                    const double V = 2.0 * M_PI * (P.lo[0] + (b.ijk[0] * n + i + 0.5) * L.h[0]) * L.h[0] * L.h[1];
                    s2 = fma(V * r, r, s2);
                    sv += V;
                } else {
                    bs2 = fma(r, r, bs2);
                }
                mx = fmax(mx, fabs(r));
            } else if (cyl) {
                const float Vf = (lo0f + ((float)(b.ijk[0] * n + i) + 0.5f) * h0f) * hvf;
                acc_r = fmaf(Vf * rf, rf, acc_r);
                acc_v += Vf;
            } else {
                acc_r = fmaf(rf, rf, acc_r);
            }
            if (f32) f32[b.cell_off + c] = rf;
            if (rleaf) rleaf[leaf_base + (long long)g * C + c] = r;
        }
        if (MX && !cyl) s2 = fma(vol, bs2, s2);
        if (!cyl && tid == 0) sv += vol * C;
        if (per_block && !MX) {  // this block's FP32 sums into its slot, scaled once by thread 0
            float a = acc_r, v = acc_v;
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_down_sync(0xffffffffu, a, o);
                v += __shfl_down_sync(0xffffffffu, v, o);
            }
            const int w = tid >> 5, lane = tid & 31, nw = (nth + 31) >> 5;
            if (lane == 0) { sredf[0][w] = a; sredf[1][w] = v; }
            __syncthreads();
            if (tid == 0) {
                float x = 0.f, y = 0.f;
                for (int e = 0; e < nw; e++) { x += sredf[0][e]; y += sredf[1][e]; }
                partials[3LL * g] = cyl ? (double)x : vol * (double)x;
                partials[3LL * g + 1] = cyl ? (double)y : vol * C;
                partials[3LL * g + 2] = 0.0;
            }
            __syncthreads();  // sredf is reused by the next block
            acc_r = 0.f; acc_v = 0.f; sv = 0;
        } else if (per_block) {  // this block's sums into its own slot (per-tree norms of a batch)
            double a = s2, bb = sv, mm = mx;
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_down_sync(0xffffffffu, a, o);
                bb += __shfl_down_sync(0xffffffffu, bb, o);
                mm = fmax(mm, __shfl_down_sync(0xffffffffu, mm, o));
            }
            const int w = tid >> 5, lane = tid & 31, nw = (nth + 31) >> 5;
            if (lane == 0) { sred[0][w] = a; sred[1][w] = bb; sred[2][w] = mm; }
            __syncthreads();
            if (tid == 0) {
                double x = 0, y = 0, z = 0;
                for (int e = 0; e < nw; e++) { x += sred[0][e]; y += sred[1][e]; z = fmax(z, sred[2][e]); }
                partials[3LL * g] = x;
                partials[3LL * g + 1] = y;
                partials[3LL * g + 2] = z;
            }
            s2 = 0; sv = 0; mx = 0;
        }
    }
    if (per_block) {
        if (tid == 0) bulk_wait0();
        return;
    }
    if (tid == 0) bulk_wait0();
    if (!MX) {
        s2 = cyl ? (double)acc_r : vol_u * (double)acc_r;
        if (cyl) sv = (double)acc_v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
        sv += __shfl_down_sync(0xffffffffu, sv, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    const int w = tid >> 5, lane = tid & 31, nw = (nth + 31) >> 5;
    if (lane == 0) { sred[0][w] = s2; sred[1][w] = sv; sred[2][w] = mx; }
    __syncthreads();
    if (tid == 0) {
        double a = 0, bb = 0, m = 0;
        for (int e = 0; e < nw; e++) { a += sred[0][e]; bb += sred[1][e]; m = fmax(m, sred[2][e]); }
        partials[3 * blockIdx.x] = a;
        partials[3 * blockIdx.x + 1] = bb;
        partials[3 * blockIdx.x + 2] = m;
    }
}

// Per-tree sums of per-block residual partials (slots listed per tree).
__global__ void __launch_bounds__(256) k_reduce_trees(const double *__restrict__ partials,
                                                      const int *__restrict__ slot_off,
                                                      const int *__restrict__ slots, double *__restrict__ out) {
    pdl_entry();
    const int tr = blockIdx.x;
    double a = 0, b = 0, m = 0;
    for (int e = slot_off[tr] + threadIdx.x; e < slot_off[tr + 1]; e += blockDim.x) {
        const long long q = 3LL * slots[e];
        a += partials[q];
        b += partials[q + 1];
        m = fmax(m, partials[q + 2]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    __shared__ double sh[3][8];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][w] = a; sh[1][w] = b; sh[2][w] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0, z = 0;
        for (int e = 0; e < (int)(blockDim.x >> 5); e++) { x += sh[0][e]; y += sh[1][e]; z = fmax(z, sh[2][e]); }
        out[3 * tr] = x;
        out[3 * tr + 1] = y;
        out[3 * tr + 2] = z;
    }
}

__global__ void __launch_bounds__(1024) k_reduce3(const double *__restrict__ partials, int n, double *out) {
    pdl_entry();
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

// Exact coarsest solves of several trees at once (one CTA per tree): r = f -
// L x in FP64 for every cell of the tree's coarsest level, with -sum V x
// appended for the zero-mean constraint; then dx = Minv r, one warp per row.
// Trees whose coarsest group is not selected (group > top, or >= top when
// strict) are skipped.
template <class T, int D>
__global__ void __launch_bounds__(1024) k_coarse_resid_b(KParams P, const TreeCoarse *__restrict__ TC, int top,
                                                          int strict, Fields<T> F, double *__restrict__ cvec) {
    pdl_entry();
    const TreeCoarse tc = TC[blockIdx.x];
    if (tc.bt_n || (strict ? tc.group >= top : tc.group > top)) return;  // block form: k_coarse_btri
    const int n = tc.n, C = cells_of<D>(n);
    double wx = 0;
    for (int row = threadIdx.x; row < tc.nc; row += blockDim.x) {
        const BlockDesc &b = P.B[tc.first + row / C];
        const LevelDesc &L = P.L[b.lev];
        int i, j, k;
        cell_of(row % C, n, D, i, j, k);
        double lap, num, den, xc;
        stencil<double, T, D>(P, L, b, F.X, F.XG, F.E, F.EG, i, j, k, lap, num, den, xc);
        cvec[tc.cvec_off + row] = (double)F.F[b.cell_off + row % C] - (lap - P.helm * xc);
        double V = 1.0;
        for (int d = 0; d < D; d++) V *= L.h[d];
        if (P.geom == MG_CYL) V = 2.0 * M_PI * (P.lo[0] + (b.ijk[0] * n + i + 0.5) * L.h[0]) * L.h[0] * L.h[1];
        wx += V * xc;
    }
    if (!tc.singular) return;
    for (int o = 16; o > 0; o >>= 1) wx += __shfl_down_sync(0xffffffffu, wx, o);
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = wx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0;
        for (int e = 0; e < (int)((blockDim.x + 31) >> 5); e++) sum += sh[e];
        cvec[tc.cvec_off + tc.nc] = -sum;
    }
}

// The coarse-grid solve of the paper (Sec. 2.4): red-black Gauss-Seidel on
// the coarsest level until max |f - L x| is at most abs_tol, or at most
// rel_tol times its value before the first sweep, or max_it sweeps.  One CTA
// per tree: the tree's coarsest level is a complete grid, held in shared
// memory (FP64, as the coarsest solve always is) with one layer of padding
// that takes the ghost rules of Sec. 2.6 (periodic wrap, Dirichlet
// 2a - x_i, Neumann x_i -/+ h b, axis x_i; the coefficient copies x_i).
// Without Dirichlet faces f is first projected to zero volume-weighted mean
// and x returned with zero mean.
struct CoarseSmooth {
    double abs_tol, rel_tol;
    int max_it;
};
template <class T, int D>
__global__ void __launch_bounds__(1024) k_coarse_gs(KParams P, const TreeCoarse *__restrict__ TC, int top, int strict,
                                                    Fields<T> F, CoarseSmooth cs) {
    pdl_entry();
    const TreeCoarse tc = TC[blockIdx.x];
    if (strict ? tc.group >= top : tc.group > top) return;
    const LevelDesc &L = P.L[tc.lvl];
    const int n = tc.n, C = cells_of<D>(n);
    const int nx = L.ncell[0], ny = L.ncell[1], nz = D == 3 ? L.ncell[2] : 1;
    const int px = nx + 2, py = ny + 2, pz = D == 3 ? nz + 2 : 1;
    const int npad = px * py * pz;
    extern __shared__ __align__(16) double sm[];
    double *sx = sm, *sf = sx + npad, *se = sf + npad;  // se only with variable eps
    const bool var = F.E != nullptr, cyl = P.geom == MG_CYL;
    __shared__ double red[32];
    auto pad = [&](int I, int J, int K) { return ((D == 3 ? (K + 1) : 0) * py + (J + 1)) * px + (I + 1); };
    auto vol = [&](int I) {
        double V = 1.0;
        for (int d = 0; d < D; d++) V *= L.h[d];
        if (cyl) V = 2.0 * M_PI * (P.lo[0] + (I + 0.5) * L.h[0]) * L.h[0] * L.h[1];
        return V;
    };
    // block-wide reductions (sum or max) of one value per thread
    auto reduce = [&](double v, bool mx) {
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, v, o);
            v = mx ? fmax(v, w) : v + w;
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        double a = mx ? 0.0 : 0.0;
        for (int e = 0; e < (int)(blockDim.x >> 5); e++) a = mx ? fmax(a, red[e]) : a + red[e];
        return a;
    };
    for (int row = threadIdx.x; row < tc.nc; row += blockDim.x) {
        const BlockDesc &b = P.B[tc.first + row / C];
        int i, j, k;
        cell_of(row % C, n, D, i, j, k);
        const int q = pad(b.ijk[0] * n + i, b.ijk[1] * n + j, D == 3 ? b.ijk[2] * n + k : 0);
        sx[q] = (double)F.X[b.cell_off + row % C];
        sf[q] = (double)F.F[b.cell_off + row % C];
        if (var) se[q] = (double)F.E[b.cell_off + row % C];
    }
    __syncthreads();
    // the padding layer of x (and once of eps) from the interior
    auto fill = [&](double *A, bool coef) {
        const int nface = 2 * (ny * nz) + 2 * (nx * nz) + (D == 3 ? 2 * nx * ny : 0);
        for (int t = threadIdx.x; t < nface; t += blockDim.x) {
            int face, u = t, a, c;
            if (u < 2 * ny * nz) { face = u / (ny * nz); u %= ny * nz; a = u % ny; c = u / ny; }
            else if ((u -= 2 * ny * nz) < 2 * nx * nz) { face = 2 + u / (nx * nz); u %= nx * nz; a = u % nx; c = u / nx; }
            else { u -= 2 * nx * nz; face = 4 + u / (nx * ny); u %= nx * ny; a = u % nx; c = u / nx; }
            const int d = face >> 1, s = face & 1, N = d == 0 ? nx : (d == 1 ? ny : nz);
            int I, J, K;  // interior cell beside the padding cell
            if (d == 0) { I = s ? nx - 1 : 0; J = a; K = c; }
            else if (d == 1) { I = a; J = s ? ny - 1 : 0; K = c; }
            else { I = a; J = c; K = s ? nz - 1 : 0; }
            int gI = I + (d == 0 ? (s ? 1 : -1) : 0), gJ = J + (d == 1 ? (s ? 1 : -1) : 0),
                gK = K + (d == 2 ? (s ? 1 : -1) : 0);
            const double xi = A[pad(I, J, K)];
            double g;
            if (P.bct[face] == MG_BC_PERIODIC) {
                int wI = I, wJ = J, wK = K;  // the cell on the other side of the domain
                if (d == 0) wI = s ? 0 : nx - 1;
                else if (d == 1) wJ = s ? 0 : ny - 1;
                else wK = s ? 0 : nz - 1;
                g = A[pad(wI, wJ, wK)];
            } else if (coef) {
                g = xi;
            } else {
                double a0 = 0.0;
                if (!P.homog) {
                    const int t1 = d == 0 ? 1 : 0, t2 = D == 2 ? -1 : (d == 2 ? 1 : 2);
                    const int G1 = t1 == 0 ? I : J, G2 = t2 < 0 ? 0 : (t2 == 1 ? J : K);
                    a0 = L.bc_off[face] < 0 ? P.bcv[face]
                                            : P.bcplanes[L.bc_off[face] + G1 + (t2 >= 0 ? (long long)L.ncell[t1] * G2 : 0)];
                }
                switch (P.bct[face]) {
                case MG_BC_DIRICHLET: g = 2.0 * a0 - xi; break;
                case MG_BC_NEUMANN: g = s ? xi + L.h[d] * a0 : xi - L.h[d] * a0; break;
                default: g = xi; break;
                }
            }
            (void)N;
            A[pad(gI, gJ, gK)] = g;
        }
    };
    if (var) fill(se, true);
    fill(sx, false);
    __syncthreads();
    // row weights of cell (I,J,K) (Sec. 2.2): sum w x_nb and sum w
    auto row_terms = [&](int I, int J, int K, double &num, double &den) {
        const int q = pad(I, J, K);
        num = 0.0;
        den = 0.0;
        const double ec = var ? se[q] : 1.0;
        const double ri = P.lo[0] + (I + 0.5) * L.h[0];
#pragma unroll
        for (int d = 0; d < D; d++)
#pragma unroll
            for (int s = 0; s < 2; s++) {
                const int o = s ? 1 : -1;
                const int qn = pad(I + (d == 0 ? o : 0), J + (d == 1 ? o : 0), K + (d == 2 ? o : 0));
                double w = L.inv_h2[d];
                if (var) w *= 2.0 * ec * se[qn] / (ec + se[qn]);
                if (cyl && d == 0) w *= (P.lo[0] + (I + s) * L.h[0]) / ri;
                num += w * sx[qn];
                den += w;
            }
    };
    const int ncell = nx * ny * nz;
    auto max_res = [&]() {
        double m = 0.0;
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int I = c % nx, J = (c / nx) % ny, K = D == 3 ? c / (nx * ny) : 0;
            double num, den;
            row_terms(I, J, K, num, den);
            const double xc = sx[pad(I, J, K)];
            m = fmax(m, fabs(sf[pad(I, J, K)] - (num - den * xc - P.helm * xc)));
        }
        return reduce(m, true);
    };
    auto mean = [&](const double *A) {
        double a = 0.0, v = 0.0;
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int I = c % nx, J = (c / nx) % ny, K = D == 3 ? c / (nx * ny) : 0;
            const double V = vol(I);
            a += V * A[pad(I, J, K)];
            v += V;
        }
        const double sa = reduce(a, false);
        const double sv = reduce(v, false);
        return sa / sv;
    };
    if (tc.singular) {
        const double mf = mean(sf);
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int I = c % nx, J = (c / nx) % ny, K = D == 3 ? c / (nx * ny) : 0;
            sf[pad(I, J, K)] -= mf;
        }
        __syncthreads();
    }
    const double r0 = max_res();
    for (int it = 0; it < cs.max_it && r0 > cs.abs_tol; it++) {
        for (int colour = 0; colour < 2; colour++) {
            for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
                const int I = c % nx, J = (c / nx) % ny, K = D == 3 ? c / (nx * ny) : 0;
                if (((I + J + K) & 1) != colour) continue;
                double num, den;
                row_terms(I, J, K, num, den);
                sx[pad(I, J, K)] = (num - sf[pad(I, J, K)]) / (den + P.helm);
            }
            __syncthreads();
            fill(sx, false);
            __syncthreads();
        }
        const double r = max_res();
        if (r <= cs.abs_tol || r <= cs.rel_tol * r0) break;
    }
    if (tc.singular) {
        const double mx = mean(sx);
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int I = c % nx, J = (c / nx) % ny, K = D == 3 ? c / (nx * ny) : 0;
            sx[pad(I, J, K)] -= mx;
        }
        __syncthreads();
    }
    for (int row = threadIdx.x; row < tc.nc; row += blockDim.x) {
        const BlockDesc &b = P.B[tc.first + row / C];
        int i, j, k;
        cell_of(row % C, n, D, i, j, k);
        F.X[b.cell_off + row % C] = (T)sx[pad(b.ijk[0] * n + i, b.ijk[1] * n + j, D == 3 ? b.ijk[2] * n + k : 0)];
    }
}

// One CTA per chunk of kCoarseRows rows of one tree (chunk list built on
// the host), one warp per row.
template <class T>
__global__ void k_coarse_apply_b(const TreeCoarse *__restrict__ TC, const int2 *__restrict__ chunks, int top,
                                 int strict, const double *__restrict__ minv, const double *__restrict__ cvec,
                                 T *__restrict__ X) {
    pdl_entry();
    const int2 ch = chunks[blockIdx.x];  // (tree, first row)
    const TreeCoarse tc = TC[ch.x];
    if (strict ? tc.group >= top : tc.group > top) return;
    const int row = ch.y + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= tc.nc) return;
    double sacc = 0;
    const double *mr = minv + tc.minv_off + (long long)row * tc.ns;
    for (int c = lane; c < tc.ns; c += 32) sacc += mr[c] * cvec[tc.cvec_off + c];
    for (int o = 16; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o);
    if (lane == 0) X[tc.cell0 + row] = (T)((double)X[tc.cell0 + row] + sacc);
}

// Block-tridiagonal coarsest solves (one CTA per tree, trees listed on the
// host, largest first), residual included: r = f - (L x - lambda x) on the
// tree's coarsest cells, then dx = M^-1 r by the plane recursion
//   forwards   w_j = S_j^-1 (r_j - A_j w_{j-1}),
//   backwards  x_j = w_j - S_j^-1 (C_j x_{j+1}),   x_{NP-1} = w_{NP-1},
// and x + dx written back.  Arithmetic and plane records are of the cycle's
// type T: FP64 cycles use the FP64 factors and the precomputed FP64 face
// coefficients (or 1/h^2); FP32 cycles the factors rounded to FP32 and the
// FP32 stencil the rest of their cycle uses.  GB300's FP64 unit holds a warp
// for about 64 cycles per instruction (FP32 FMAs take under 5), so the
// layout keeps the instructions besides the P^2 FMAs of each plane few:
// warp q of the CTA owns columns [k0, k1) of every plane (lane = row for the
// products); the input u of a plane is formed by the owner of each column
// from the previous plane's partial sums (one add per extra warp and one
// coupling FMA) and reaches the other lanes by shuffles, so each plane
// costs one barrier.  The plane records (S_j^-1 column by column, then
// A_j, C_j) are staged into a ring of `ring` shared-memory slots, one bulk
// copy (cp.async.bulk, mbarrier completion) per record issued ring - 1
// planes ahead by thread 0; the visit order is planes 0 .. NP-1, then
// NP-2 .. 0.  Every mbarrier wait is bounded: on expiry the kernel raises
// P.status, lets the copies in flight land and the CTA stops.
constexpr int kBtriMaxRing = 7;
constexpr int kBtriThreads = 128;  // at most four warps (one per SM sub-partition)
__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }
template <class T> __device__ __forceinline__ const T *bt_records(const double *b64, const float *b32);
template <> __device__ __forceinline__ const double *bt_records<double>(const double *b64, const float *) { return b64; }
template <> __device__ __forceinline__ const float *bt_records<float>(const double *, const float *b32) { return b32; }

// r = f - (L x - lambda x) at one coarsest cell, in T
template <class T, int D>
__device__ __forceinline__ T coarse_resid(const KParams &P, const BlockDesc &b, int c, const Fields<T> &F,
                                          const double *__restrict__ W64) {
    const int n = b.n, C = cells_of<D>(n);
    int ci, cj, ck;
    cell_of(c, n, D, ci, cj, ck);
    const LevelDesc &L = P.L[b.lev];
    if constexpr (sizeof(T) == 8) {
        const double *wc = W64 ? W64 + b.cell_off * wstride(D) + c : nullptr;
        double acc = 0, wsum = 0;
#pragma unroll
        for (int d = 0; d < D; d++)
#pragma unroll
            for (int s = 0; s < 2; s++) {
                const int o = s ? 1 : -1;
                const double xn = load<T, D>(F.X, F.XG, b, ci + (d == 0 ? o : 0), cj + (d == 1 ? o : 0),
                                             ck + (d == 2 ? o : 0));
                const double wf = wc ? wc[(2 * d + s) * C] : L.inv_h2[d];
                acc = fma(wf, xn, acc);
                wsum += wf;
            }
        const double diag = wc ? wc[2 * D * C] : wsum + P.helm;
        return F.F[b.cell_off + c] - fma(-diag, (double)F.X[b.cell_off + c], acc);
    } else {
        float lap, num, den, xc;
        stencil<float, T, D>(P, L, b, F.X, F.XG, F.E, F.EG, ci, cj, ck, lap, num, den, xc);
        return F.F[b.cell_off + c] - (lap - P.helmf * xc);
    }
}

// Residual of the block-form trees' coarsest cells in plane order, one
// thread per cell: r (of the cycle's type T) into the tree's coarsest
// vector (viewed as T).
template <class T, int D>
__global__ void __launch_bounds__(kBtResidCells) k_coarse_resid_bt(KParams P, const TreeCoarse *__restrict__ TC,
                                                                   const int2 *__restrict__ chunks, int top,
                                                                   int strict, Fields<T> F,
                                                                   const double *__restrict__ W64,
                                                                   const int *__restrict__ perm,
                                                                   double *__restrict__ cvec) {
    pdl_entry();
    const int2 ch = chunks[blockIdx.x];  // (tree, first cell)
    const TreeCoarse tc = TC[ch.x];
    if (strict ? tc.group >= top : tc.group > top) return;
    const int i = ch.y + threadIdx.x;
    if (i >= tc.nc) return;
    const int row = perm[tc.perm_off + i], C = cells_of<D>(tc.n);
    T *rb = reinterpret_cast<T *>(cvec) + (sizeof(double) / sizeof(T)) * tc.cvec_off;
    rb[i] = coarse_resid<T, D>(P, P.B[tc.first + row / C], row % C, F, W64);
}

// FP32 form of the plane recursion, one warp per tree: lane p owns row p
// (and p + 32) of every plane, so w_j[p], x_j[p] and the couplings that
// act on them stay in the lane; only the input u of each plane is shared
// (two buffers, zero padded).  Products read 4 coefficients of the row
// and 4 inputs per 128-bit shared load; the ring of plane records is
// filled by bulk copies as in k_coarse_btri.
template <int D>
__global__ void __launch_bounds__(32) k_coarse_btri_f32(KParams P, const TreeCoarse *__restrict__ TC,
                                                        const int *__restrict__ list, int top, int strict,
                                                        float *__restrict__ X, const double *__restrict__ cvec,
                                                        const float *__restrict__ bt32,
                                                        const int *__restrict__ perm, int ring, int slot) {
    pdl_entry();
    const TreeCoarse tc = TC[list[blockIdx.x]];
    if (strict ? tc.group >= top : tc.group > top) return;
    const int Pp = tc.bt_P, NP = tc.bt_n, nc = tc.nc, NV = 2 * NP - 1;
    const int st = bt32_stride(Pp), row = bt32_row(Pp), r4 = bt_round4(Pp), lane = threadIdx.x;
    extern __shared__ __align__(16) unsigned char bt_smem[];
    __shared__ __align__(8) uint64_t bars[kBtriMaxRing];
    float *sm = reinterpret_cast<float *>(bt_smem);
    float *us = sm + (size_t)ring * slot;  // plane inputs: 2 buffers of kBtriMaxPlane
    float *r = us + 2 * kBtriMaxPlane;     // residual, plane order
    float *w = r + nc;                     // w_j, then x_j
    const float *rec = bt32 + tc.bt_off32;
    const int *pm = perm + tc.perm_off;
    const float *rb = reinterpret_cast<const float *>(cvec) + 2 * tc.cvec_off;
    const uint32_t bytes = (uint32_t)(sizeof(float) * st);
    if (lane == 0) {
        for (int s = 0; s < ring; s++) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    for (int q = lane; q < 2 * kBtriMaxPlane; q += 32) us[q] = 0.0f;
    __syncwarp();
    auto issue = [&](int v, int s) {  // lane 0: the record of visit v into slot s
        const int j = v < NP ? v : 2 * NP - 2 - v;
        mbar_expect_tx(&bars[s], bytes);
        bulk_g2s(sm + (size_t)s * slot, rec + (size_t)j * st, bytes, &bars[s]);
    };
    if (lane == 0)
        for (int v = 0; v < ring - 1 && v < NV; v++) issue(v, v);
    for (int i = lane; i < nc; i += 32) r[i] = rb[i];
    __syncwarp();
    for (int p = lane; p < Pp; p += 32) us[p] = r[p];  // u of plane 0 = r_0
    __syncwarp();
    int sv = 0;       // ring slot of visit v
    uint32_t ph = 0;  // phase parity of that slot
    for (int v = 0; v < NV; v++) {
        const bool ok = mbar_wait_bounded(&bars[sv], ph, P.wait_limit);
        if (!__all_sync(0xffffffffu, ok)) {
            // copies issued for visits v .. v + ring - 2 may still be landing:
            // let them arrive (normal bound) before the CTA exits
            if (lane == 0) {
                atomicExch(P.status, 1);
                int s = sv;
                uint32_t q = ph;
                for (int u = v; u < NV && u <= v + ring - 2; u++) {
                    mbar_wait_bounded(&bars[s], q, kWaitLimit);
                    if (++s == ring) { s = 0; q ^= 1; }
                }
            }
            return;
        }
        if (lane == 0 && v + ring - 1 < NV) issue(v + ring - 1, sv == 0 ? ring - 1 : sv - 1);  // slot of visit v-1
        const float *R = sm + (size_t)sv * slot;
        const float *lo = R + (size_t)Pp * row, *up = lo + r4;  // A_{j+1}, C_{j-1}
        const int j = v < NP ? v : 2 * NP - 2 - v;
        const float *ub = us + (v & 1) * kBtriMaxPlane;
        float *un = us + ((v + 1) & 1) * kBtriMaxPlane;
        for (int pb = 0; pb < Pp; pb += 32) {
            const int p = pb + lane;
            const float *Rr = R + (size_t)(p < Pp ? p : 0) * row;  // idle lanes read row 0
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            for (int q = 0; q < Pp; q += 4) {
                const float4 rv = *reinterpret_cast<const float4 *>(Rr + q);
                const float4 uv = *reinterpret_cast<const float4 *>(ub + q);
                a0 = fmaf(rv.x, uv.x, a0);
                a1 = fmaf(rv.y, uv.y, a1);
                a2 = fmaf(rv.z, uv.z, a2);
                a3 = fmaf(rv.w, uv.w, a3);
            }
            const float acc = (a0 + a1) + (a2 + a3);
            if (p < Pp) {
                if (v < NP) {  // w_j = S_j^-1 u_j
                    w[j * Pp + p] = acc;
                    un[p] = j + 1 < NP ? fmaf(-lo[p], acc, r[(j + 1) * Pp + p])  // u_{j+1} = r_{j+1} - A_{j+1} w_j
                                       : up[p] * acc;                           // x_{NP-1} = w_{NP-1}
                } else {  // x_j = w_j - S_j^-1 C_j x_{j+1}
                    const float x = w[j * Pp + p] - acc;
                    w[j * Pp + p] = x;
                    if (j > 0) un[p] = up[p] * x;
                }
            }
        }
        __syncwarp();
        if (++sv == ring) { sv = 0; ph ^= 1; }
    }
    for (int i = lane; i < nc; i += 32) X[tc.cell0 + pm[i]] += w[i];
}

template <class T, int D>
__global__ void __launch_bounds__(kBtriThreads) k_coarse_btri(KParams P, const TreeCoarse *__restrict__ TC,
                                                              const int *__restrict__ list, int top, int strict,
                                                              Fields<T> F, const double *__restrict__ cvec,
                                                              const double *__restrict__ bt64,
                                                              const float *__restrict__ bt32,
                                                              const int *__restrict__ perm, int ring, int slot) {
    pdl_entry();
    const TreeCoarse tc = TC[list[blockIdx.x]];
    if (strict ? tc.group >= top : tc.group > top) return;
    const int Pp = tc.bt_P, NP = tc.bt_n, nc = tc.nc, st = bt_stride(Pp), NV = 2 * NP - 1;
    const int tid = threadIdx.x, lane = tid & 31, nw = blockDim.x >> 5, wq = tid >> 5;
    const int k0 = wq * Pp / nw, k1 = (wq + 1) * Pp / nw, m = k1 - k0;  // this warp's columns (m <= 32)
    extern __shared__ __align__(16) unsigned char bt_smem[];
    __shared__ __align__(8) uint64_t bars[kBtriMaxRing];
    __shared__ int s_abort;
    T *sm = reinterpret_cast<T *>(bt_smem);
    T *r = sm + (size_t)ring * slot;  // residual, plane order
    T *w = r + nc;                    // w_j, then x_j
    T *part = w + nc;                 // partial sums: 2 buffers of nw x Pp
    const T *rec = bt_records<T>(bt64, bt32) + (sizeof(T) == 8 ? tc.bt_off : tc.bt_off32);
    const int *pm = perm + tc.perm_off;
    const uint32_t bytes = (uint32_t)(sizeof(T) * st);
    if (tid == 0) {
        for (int s = 0; s < ring; s++) mbar_init(&bars[s], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    auto issue = [&](int v, int s) {  // thread 0: the record of visit v into slot s
        const int j = v < NP ? v : 2 * NP - 2 - v;
        mbar_expect_tx(&bars[s], bytes);
        bulk_g2s(sm + (size_t)s * slot, rec + (size_t)j * st, bytes, &bars[s]);
    };
    if (tid == 0)
        for (int v = 0; v < ring - 1 && v < NV; v++) issue(v, v);
    {  // residual of the coarsest cells, plane order (k_coarse_resid_bt)
        const T *rb = reinterpret_cast<const T *>(cvec) + (sizeof(double) / sizeof(T)) * tc.cvec_off;
        for (int i = tid; i < nc; i += blockDim.x) r[i] = rb[i];
    }
    int sv = 0;       // ring slot of visit v
    uint32_t ph = 0;  // phase parity of that slot
    for (int v = 0; v < NV; v++) {
        if (!mbar_wait_bounded(&bars[sv], ph, P.wait_limit)) {
            atomicExch(P.status, 1);
            s_abort = 1;
        }
        __syncthreads();  // the record is in; every thread is past visit v-1
        if (s_abort) {
            // copies issued for visits v .. v + ring - 2 may still be landing:
            // let them arrive (normal bound) before the CTA exits
            if (tid == 0) {
                int s = sv;
                uint32_t q = ph;
                for (int u = v; u < NV && u <= v + ring - 2; u++) {
                    mbar_wait_bounded(&bars[s], q, kWaitLimit);
                    if (++s == ring) { s = 0; q ^= 1; }
                }
            }
            return;
        }
        if (tid == 0 && v + ring - 1 < NV) issue(v + ring - 1, sv == 0 ? ring - 1 : sv - 1);  // slot of visit v-1
        const T *R = sm + (size_t)sv * slot;
        const int j = v < NP ? v : 2 * NP - 2 - v;
        const T *pprev = part + (size_t)((v - 1) & 1) * nw * Pp;
        T u = 0;
        const int k = k0 + lane;
        if (lane < m) {
            if (v < NP) {  // u = r_j - A_j w_{j-1}; w_{j-1} is complete now
                u = r[j * Pp + k];
                if (j > 0) {
                    T sum = pprev[k];
                    for (int q = 1; q < nw; q++) sum += pprev[q * Pp + k];
                    w[(j - 1) * Pp + k] = sum;
                    u = tfma(-R[Pp * Pp + k], sum, u);
                }
            } else {  // u = C_j x_{j+1}; x_{j+1} is complete now
                T sum = pprev[k];
                for (int q = 1; q < nw; q++) sum += pprev[q * Pp + k];
                const T x = j + 1 == NP - 1 ? sum : w[(j + 1) * Pp + k] - sum;
                w[(j + 1) * Pp + k] = x;
                u = R[Pp * Pp + Pp + k] * x;
            }
        }
        T *pcur = part + (size_t)(v & 1) * nw * Pp;
        for (int pb = 0; pb < Pp; pb += 32) {  // all lanes take part in the shuffles
            const int p = pb + lane;
            const T *Rp = R + k0 * Pp + (p < Pp ? p : 0);  // idle lanes read row 0
            T acc;
            if constexpr (sizeof(T) == 8) {  // one chain: FP64 FMAs do not overlap within a warp
                T a0 = 0;
                for (int q = 0; q < m; q++) a0 = tfma(Rp[q * Pp], __shfl_sync(0xffffffffu, u, q), a0);
                acc = a0;
            } else {
                T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
                int q = 0;
                for (; q + 4 <= m; q += 4) {
                    const T u0 = __shfl_sync(0xffffffffu, u, q), u1 = __shfl_sync(0xffffffffu, u, q + 1);
                    const T u2 = __shfl_sync(0xffffffffu, u, q + 2), u3 = __shfl_sync(0xffffffffu, u, q + 3);
                    a0 = tfma(Rp[q * Pp], u0, a0);
                    a1 = tfma(Rp[(q + 1) * Pp], u1, a1);
                    a2 = tfma(Rp[(q + 2) * Pp], u2, a2);
                    a3 = tfma(Rp[(q + 3) * Pp], u3, a3);
                }
                for (; q < m; q++) a0 = tfma(Rp[q * Pp], __shfl_sync(0xffffffffu, u, q), a0);
                acc = (a0 + a1) + (a2 + a3);
            }
            if (p < Pp) pcur[wq * Pp + p] = acc;
        }
        if (++sv == ring) { sv = 0; ph ^= 1; }
    }
    __syncthreads();
    {  // x_0 = w_0 - S_0^-1 C_0 x_1
        const T *pl = part + (size_t)((NV - 1) & 1) * nw * Pp;
        const int k = k0 + lane;
        if (lane < m) {
            T sum = pl[k];
            for (int q = 1; q < nw; q++) sum += pl[q * Pp + k];
            w[k] -= sum;
        }
    }
    __syncthreads();
    for (int i = tid; i < nc; i += blockDim.x) F.X[tc.cell0 + pm[i]] += w[i];
}

// --------------------------------------------------- elementwise ops ----
// phi64 += e32 (the defect-correction update) on leaf cells (one contiguous
// range per level or segment) of the segments that k_update_restrict does
// not cover; covered cells are restored from their children before the
// next residual, and the levels below the leaves are rebuilt by every
// cycle.  The widening of e is exact and done with integer operations
// (mg_from_float; GB300 runs the conversion instruction on its FP64 pipe),
// leaving one FP64 add per cell.
constexpr int kMaxLeafRanges = 96;
struct LeafRanges {
    int n;
    long long start[kMaxLeafRanges], len[kMaxLeafRanges];
};
__global__ void k_add_e_leaf(LeafRanges R, const float *__restrict__ e, double *__restrict__ x) {
    pdl_entry();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < R.n; r++) {
        double *xr = x + R.start[r];
        const float *er = e + R.start[r];
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < R.len[r]; i += stride)
            xr[i] += mg_from_float(er[i]);
    }
}
// phi += e on the leaf cells of the listed segments (chunks of
// kMaxLeafRanges ranges per launch; covered cells are never touched)
static void enqueue_add_leaf(mg_tree *t, const std::vector<int> &segs, const float *e, double *phi) {
    LeafRanges R;
    R.n = 0;
    auto flush = [&]() {
        if (!R.n) return;
        ++t->launches;
        launch_k(k_add_e_leaf, 1216, 256, 0, t->stream, R, e, phi);
        R.n = 0;
    };
    for (int l : segs) {
        const LevelHost &L = t->lev[l];
        if (L.nb <= L.nref) continue;
        if (R.n == kMaxLeafRanges) flush();
        R.start[R.n] = t->blocks[L.first + L.nref].cell_off;
        R.len[R.n] = (long long)(L.nb - L.nref) * (t->dim == 2 ? L.n * L.n : L.n * L.n * L.n);
        R.n++;
    }
    flush();
}
__global__ void k_cast_f32(const double *__restrict__ a, float *__restrict__ b, long long n) {
    pdl_entry();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}
// Whole-field copies between the FP64 and FP32 sets, rounded to nearest /
// widened exactly with integer operations (GB300 runs the conversion
// instructions on its FP64 pipe)
__global__ void k_narrow(const double *__restrict__ a, float *__restrict__ b, long long n) {
    pdl_entry();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = mg_to_float(a[i]);
}
__global__ void k_widen(const float *__restrict__ a, double *__restrict__ b, long long n) {
    pdl_entry();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = mg_from_float(a[i]);
}
void narrow_f32(mg_tree *t, const double *a, float *b, long long n) {
    ++t->launches;
    launch_k(k_narrow, 8 * t->nsm, 256, 0, t->stream, a, b, n);
}
void widen_f64(mg_tree *t, const float *a, double *b, long long n) {
    ++t->launches;
    launch_k(k_widen, 8 * t->nsm, 256, 0, t->stream, a, b, n);
}
// ------------------------------------------------------------ driver ----

// Face coefficients of the FP64 operator (Sec. 2.2), one thread per cell:
// w = (1/h_d^2) * 2 eps_c eps_n / (eps_c + eps_n) * (r_face / r_cell), and
// the row's diagonal sum w + lambda.  Stored per block as [face][cell],
// 2D + 1 "faces" (the last the diagonal), after cell_off * (2D + 1).
template <int D>
__global__ void __launch_bounds__(256) k_face_coef(KParams P, int first, int nblocks, int n,
                                                   const double *__restrict__ E, const double *__restrict__ EG,
                                                   double *__restrict__ W) {
    pdl_entry();
    const int C = cells_of<D>(n);
    const long long total = (long long)nblocks * C;
    const bool cyl = P.geom == MG_CYL;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const BlockDesc &b = P.B[first + (int)(idx / C)];
        const LevelDesc &L = P.L[b.lev];
        const int c = (int)(idx % C);
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        const double ec = E ? E[b.cell_off + c] : 1.0;
        double ri = 0;
        if (cyl) ri = P.lo[0] + (b.ijk[0] * n + i + 0.5) * L.h[0];
        double *w_out = W + b.cell_off * wstride(D) + c;
        double wsum = 0;
#pragma unroll
        for (int d = 0; d < D; d++)
#pragma unroll
            for (int s = 0; s < 2; s++) {
                double w = L.inv_h2[d];
                if (E) {
                    const int o = s ? 1 : -1;
                    const double en = load<double, D>(E, EG, b, i + (d == 0 ? o : 0), j + (d == 1 ? o : 0),
                                                      k + (d == 2 ? o : 0));
                    w *= 2.0 * ec * en / (ec + en);
                }
                if (cyl && d == 0) w *= (P.lo[0] + (b.ijk[0] * n + i + s) * L.h[0]) / ri;
                w_out[(2 * d + s) * C] = w;
                wsum += w;
            }
        w_out[2 * D * C] = wsum + P.helm;  // diagonal of the row
        w_out[(2 * D + 1) * C] = 1.0 / (wsum + P.helm);  // its reciprocal
    }
}

void face_coef(mg_tree *t) {
    const KParams P = kparams(t, 0);
    for (const LevelHost &L : t->lev) {
        if (L.nb == 0) continue;
        ++t->launches;
        const long long items = (long long)L.nb * (t->dim == 2 ? L.n * L.n : L.n * L.n * L.n);
        const int grid = (int)std::max<long long>(1, std::min<long long>((items + 255) / 256, 8LL * t->nsm));
        if (t->dim == 2)
            launch_k(k_face_coef<2>, grid, 256, 0, t->stream, P, L.first, L.nb, L.n, t->f64.E, t->f64.EG, t->d_wface);
        else
            launch_k(k_face_coef<3>, grid, 256, 0, t->stream, P, L.first, L.nb, L.n, t->f64.E, t->f64.EG, t->d_wface);
    }
}

// ----------------------------------------------- flat small-block path ---
// Segments of tiny blocks (at most kFlatCells cells, the halved block sizes
// of the levels below the base grid) run one thread per work item across
// all blocks of the segment instead of one CTA per block.  Same arithmetic
// as the CTA kernels, read straight from global memory.
// One launch covers several such segments of a group (FlatSegs: per
// segment its first block, block count, block size and first work item).
constexpr int kFlatCells = 16;
constexpr int kMaxFlatSegs = 16;
struct FlatSegs {
    int nseg;
    int first[kMaxFlatSegs], nb[kMaxFlatSegs], n[kMaxFlatSegs];
    long long off[kMaxFlatSegs + 1];  // work items of segments 0..s-1
};
__device__ __forceinline__ int flat_seg(const FlatSegs &S, long long gi) {
    int s = 0;
    while (s + 1 < S.nseg && gi >= S.off[s + 1]) s++;
    return s;
}

// Each flat kernel is a grid-stride loop over the work items of its
// segments; the work of one item is a device function, which the tail
// kernel (k_tail) runs the same way.  These functions take plain pointers:
// in the tail kernel the arrays they read are written by its earlier phases.

// ghost slot t of every block: as k_ghost
template <class T, int D>
__device__ __forceinline__ void ghost_flat_item(const KParams &P, const FlatSegs &S, T *X, T *XG, int mode,
                                                long long gi) {
    {
        const int sg = flat_seg(S, gi), n = S.n[sg], F = face_of<D>(n), G = 2 * D * F;
        const long long idx = gi - S.off[sg];
        const int g = S.first[sg] + (int)(idx / G), t = (int)(idx % G);
        const BlockDesc &b = P.B[g];
        const LevelDesc &L = P.L[b.lev];
        const int face = t / F, u = t - face * F, d = face >> 1, s = face & 1;
        const I3 ii = face_cell<D>(n, face, u, false);
        const int nb = b.nbr[face];
        T val;
        if (nb >= 0) {
            const BlockDesc &q = P.B[nb];
            I3 jj = ii;
            put(jj, d, s ? 0 : n - 1);
            val = X[q.cell_off + cidx<D>(n, jj.x, jj.y, jj.z)];
        } else if (nb == -1) {
            const T xi = X[b.cell_off + cidx<D>(n, ii.x, ii.y, ii.z)];
            val = mode >= 1 ? xi : phys_ghost<T>(P, L, face, xi, bc_value(P, L, b, D, face, ii));
        } else {
            I3 dd = ii;
            put(dd, d, s ? n - 2 : 1);
            const T c = X[b.cell_off + cidx<D>(n, ii.x, ii.y, ii.z)];
            const T dv = X[b.cell_off + cidx<D>(n, dd.x, dd.y, dd.z)];
            val = cf_ghost<T, D>(P, L, b, face, ii, c, dv, X, XG, nb, mode == 1);
        }
        XG[b.ghost_off + t] = val;
    }
}
template <class T, int D>
__global__ void __launch_bounds__(256) k_ghost_flat(KParams P, FlatSegs S, T *__restrict__ X, T *__restrict__ XG,
                                                    int mode) {
    pdl_entry();
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < S.off[S.nseg];
         gi += (long long)gridDim.x * blockDim.x)
        ghost_flat_item<T, D>(P, S, X, XG, mode, gi);
}

// red-black half-sweep, one thread per cell of the colour, pushing the
// same-level and physical ghosts fed by its cell (segments without
// refinement faces; reads touch only slots of the other colour, as in the
// CTA sweep)
template <class T, int D>
__device__ __forceinline__ void sweep_flat_item(const KParams &P, const FlatSegs &S, const Fields<T> &F, int colour,
                                                long long gi) {
    {
        const int sg = flat_seg(S, gi), n = S.n[sg];
        const int C = cells_of<D>(n), Fc = face_of<D>(n), ncol = (n & 1) ? C : C / 2;
        const long long idx = gi - S.off[sg];
        const int g = S.first[sg] + (int)(idx / ncol), qi = (int)(idx % ncol);
        const BlockDesc &b = P.B[g];
        const LevelDesc &L = P.L[b.lev];
        const int par0 = (b.ijk[0] + b.ijk[1] + b.ijk[2]) * n;
        int i, j, k;
        if (n & 1) {
            i = qi % n; j = (qi / n) % n; k = D == 3 ? qi / (n * n) : 0;
            if (((par0 + i + j + k) & 1) != colour) return;
        } else {
            const int h = n >> 1, rr = qi / h, m = qi - rr * h;
            j = rr % n;
            k = D == 3 ? rr / n : 0;
            i = 2 * m + ((colour + par0 + j + k) & 1);
        }
        const int c = cidx<D>(n, i, j, k);
        T lap, num, den, xc;
        stencil<T, T, D>(P, L, b, F.X, F.XG, F.E, F.EG, i, j, k, lap, num, den, xc);
        const T xnew = qdiv<T>(num - F.F[b.cell_off + c], den + kp_helm<T>(P));
        F.X[b.cell_off + c] = xnew;
        const I3 ii{i, j, k};
#pragma unroll
        for (int face = 0; face < 2 * D; face++) {
            const int d = face >> 1, s = face & 1;
            if (get(ii, d) != (s ? n - 1 : 0)) continue;
            int u;
            if (D == 2) u = d == 0 ? j : i;
            else u = d == 0 ? j + n * k : (d == 1 ? i + n * k : i + n * j);
            const int nb = b.nbr[face];
            if (nb >= 0) F.XG[b.push[face] + u] = xnew;
            else if (nb == -1) F.XG[b.ghost_off + face * Fc + u] = phys_ghost<T>(P, L, face, xnew, bc_value(P, L, b, D, face, ii));
        }
    }
}
template <class T, int D>
__global__ void __launch_bounds__(256) k_sweep_flat(KParams P, FlatSegs S, Fields<T> F, int colour) {
    pdl_entry();
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < S.off[S.nseg];
         gi += (long long)gridDim.x * blockDim.x)
        sweep_flat_item<T, D>(P, S, F, colour, gi);
}

// covered cells <- mean of their children, one thread per parent cell
// (with_res: mean child residual into Fdst); as k_restrict, no ghost push
template <class T, int D>
__device__ __forceinline__ void restrict_flat_item(const KParams &P, const FlatSegs &S, T *X, const T *XG,
                                                   const T *Fr, const T *E, const T *EG, T *Fdst, int with_res,
                                                   long long gi) {
    {
        const int sg = flat_seg(S, gi), n = S.n[sg], m = n / 2, M = cells_of<D>(m);
        const long long idx = gi - S.off[sg];
        const int g = S.first[sg] + (int)(idx / M), c = (int)(idx % M);
        const BlockDesc &b = P.B[g];
        const LevelDesc &L = P.L[b.lev];
        const BlockDesc &p = P.B[b.parent];
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
                sr += Fr[b.cell_off + fc] - (lap - kp_helm<T>(P) * xc);
            }
        }
        const int pc = cidx<D>(p.n, b.poff[0] + ci, b.poff[1] + cj, b.poff[2] + ck);
        X[p.cell_off + pc] = sx * (T)(1.0 / (1 << D));
        if (with_res) Fdst[p.cell_off + pc] = sr * (T)(1.0 / (1 << D));
    }
}
template <class T, int D>
__global__ void __launch_bounds__(256) k_restrict_flat(KParams P, FlatSegs S, T *__restrict__ X,
                                                       const T *__restrict__ XG, const T *__restrict__ Fr,
                                                       const T *__restrict__ E, const T *__restrict__ EG,
                                                       T *__restrict__ Fdst, int with_res) {
    pdl_entry();
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < S.off[S.nseg];
         gi += (long long)gridDim.x * blockDim.x)
        restrict_flat_item<T, D>(P, S, X, XG, Fr, E, EG, Fdst, with_res, gi);
}

// covered cells: f^H += L^H v^H (Sec. 2.4); vold also keeps v_old = v^H and
// its ghosts (items past the cells copy the ghost slots)
template <class T, int D>
__device__ __forceinline__ void fas_flat_item(const KParams &P, const FlatSegs &S, const Fields<T> &F, int vold,
                                              long long gi) {
    {
        const int sg = flat_seg(S, gi), n = S.n[sg], first = S.first[sg];
        const int C = cells_of<D>(n), G = 2 * D * face_of<D>(n);
        const long long ncells = (long long)S.nb[sg] * C, idx = gi - S.off[sg];
        if (idx < ncells) {
            const int g = first + (int)(idx / C), c = (int)(idx % C);
            const BlockDesc &b = P.B[g];
            const LevelDesc &L = P.L[b.lev];
            int i, j, k;
            cell_of(c, n, D, i, j, k);
            T lap, num, den, xc;
            stencil<T, T, D>(P, L, b, F.X, F.XG, F.E, F.EG, i, j, k, lap, num, den, xc);
            F.F[b.cell_off + c] += lap - kp_helm<T>(P) * xc;
            if (vold) F.V[b.cell_off + c] = xc;
        } else {
            const long long e = idx - ncells;
            const BlockDesc &b = P.B[first + (int)(e / G)];
            const long long o = b.ghost_off + e % G;
            F.VG[o] = F.XG[o];
        }
    }
}
template <class T, int D>
__global__ void __launch_bounds__(256) k_fas_flat(KParams P, FlatSegs S, Fields<T> F, int vold) {
    pdl_entry();
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < S.off[S.nseg];
         gi += (long long)gridDim.x * blockDim.x)
        fas_flat_item<T, D>(P, S, F, vold, gi);
}

// One weighted-Jacobi step of a segment (reading R13), one thread per cell:
// J = x + omega (x_GS - x), x_GS the local solution from the values before
// the step (the caller copies J back and refreshes the ghosts).
template <class T, int D>
__global__ void __launch_bounds__(256) k_jacobi_flat(KParams P, int first, int nblocks, int n, Fields<T> F, T omega) {
    pdl_entry();
    const int C = cells_of<D>(n);
    const long long total = (long long)nblocks * C;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const BlockDesc &b = P.B[first + (int)(idx / C)];
        const LevelDesc &L = P.L[b.lev];
        const int c = (int)(idx % C);
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        T lap, num, den, xc;
        stencil<T, T, D>(P, L, b, F.X, F.XG, F.E, F.EG, i, j, k, lap, num, den, xc);
        const T xgs = qdiv<T>(num - F.F[b.cell_off + c], den + kp_helm<T>(P));
        F.J[b.cell_off + c] = xc + omega * (xgs - xc);
    }
}

// coarse-grid correction x^h += P(x^H - x^H_old) (as k_prolong), one
// thread per fine cell, no ghost push (a ghost fill follows)
template <class T, int D>
__device__ __forceinline__ void prolong_flat_item(const KParams &P, const FlatSegs &S, const Fields<T> &F,
                                                  long long gi) {
    {
        const int sg = flat_seg(S, gi), n = S.n[sg], C = cells_of<D>(n);
        const long long idx = gi - S.off[sg];
        const int g = S.first[sg] + (int)(idx / C), c = (int)(idx % C);
        const BlockDesc &b = P.B[g];
        const BlockDesc &p = P.B[b.parent];
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        const int I0 = b.ijk[0] * n + i, I1 = b.ijk[1] * n + j, I2 = b.ijk[2] * n + k;
        const int c0x = b.poff[0] + i / 2, c0y = b.poff[1] + j / 2, c0z = D == 3 ? b.poff[2] + k / 2 : 0;
        const T c0 = load<T, D>(F.X, F.XG, p, c0x, c0y, c0z) - load<T, D>(F.V, F.VG, p, c0x, c0y, c0z);
        T nbs = 0;
#pragma unroll
        for (int d = 0; d < D; d++) {
            const int o = ((d == 0 ? I0 : d == 1 ? I1 : I2) & 1) ? 1 : -1;
            const int qx = c0x + (d == 0 ? o : 0), qy = c0y + (d == 1 ? o : 0), qz = c0z + (d == 2 ? o : 0);
            nbs += load<T, D>(F.X, F.XG, p, qx, qy, qz) - load<T, D>(F.V, F.VG, p, qx, qy, qz);
        }
        const T val = D == 2 ? ((T)2 * c0 + nbs) / (T)4 : (c0 + nbs) / (T)4;
        F.X[b.cell_off + c] += val;
    }
}
template <class T, int D>
__global__ void __launch_bounds__(256) k_prolong_flat(KParams P, FlatSegs S, Fields<T> F) {
    pdl_entry();
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < S.off[S.nseg];
         gi += (long long)gridDim.x * blockDim.x)
        prolong_flat_item<T, D>(P, S, F, gi);
}

// ------------------------------------------------------ tail kernel ---
// The small levels at the bottom of a V-cycle (below a cell bound, without
// refinement faces) are a chain of launches whose work is a few
// microseconds each.  With a bound set (mg_set_tail; off by default) the
// cycle steps there (colour sweeps, restriction, parent ghost fills, FAS
// right-hand sides, prolongation, ghost fills) are recorded as a program of
// flat phases instead of being launched, and one cooperative launch runs
// the program: every CTA takes the work items of a phase in grid-stride
// order, then all CTAs meet at a grid barrier before the next phase.  On
// GB300, inside the solve's CUDA graphs, a phase plus a barrier costs more
// than the launch it replaces (the benchmark solve: 11.3 ms without, 11.8
// ms with only the 8-block level in the tail, 14.1 ms up to 64^3 cells), so
// the split stays an option.  Phases split only because a launch holds at most
// kMaxFlatSegs segments need no barrier between them (independent
// segments).  The barrier's counter and generation live beside the tree's
// status word; its wait is bounded like every other: on expiry the CTA
// sets the status word and returns, and the host reports MG_ERR_TIMEOUT
// and clears the three words.
enum { TK_GHOST, TK_SWEEP, TK_RESTRICT, TK_FAS, TK_PROLONG };
constexpr int kTailMaxOps = 40;
constexpr int kTailThreads = 256;
struct TailOp {
    int kind, arg, bar;  // bar: grid barrier after this phase
    FlatSegs S;
};
struct TailProg {
    int nops;
    TailOp op[kTailMaxOps];
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Grid barrier of a cooperative launch (every CTA resident): thread 0 of
// each CTA arrives on the counter after the CTA's writes; the last arrival
// resets the counter and advances the generation, the others poll it (at
// most `limit` polls).  Returns false when the wait gave up.
__device__ __forceinline__ bool tail_grid_sync(unsigned *cnt, unsigned *gen, uint32_t limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g0 = ld_acquire_u32(gen);
        __threadfence();
        if (atomicAdd(cnt, 1u) == gridDim.x - 1) {
            atomicExch(cnt, 0u);
            __threadfence();
            st_release_u32(gen, g0 + 1);
        } else {
            uint32_t tries = 0;
            while (ld_acquire_u32(gen) == g0) {
                if (++tries > limit) { ok = 0; break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class T, int D>
__global__ void __launch_bounds__(kTailThreads) k_tail(KParams P, Fields<T> F, const __grid_constant__ TailProg prog) {
    unsigned *cnt = reinterpret_cast<unsigned *>(P.status + 1), *gen = reinterpret_cast<unsigned *>(P.status + 2);
    const long long stride = (long long)gridDim.x * blockDim.x, g0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (int o = 0; o < prog.nops; o++) {
        const TailOp &op = prog.op[o];
        const long long items = op.S.off[op.S.nseg];
        switch (op.kind) {
        case TK_GHOST:
            for (long long gi = g0; gi < items; gi += stride) ghost_flat_item<T, D>(P, op.S, F.X, F.XG, op.arg, gi);
            break;
        case TK_SWEEP:
            for (long long gi = g0; gi < items; gi += stride) sweep_flat_item<T, D>(P, op.S, F, op.arg, gi);
            break;
        case TK_RESTRICT:
            for (long long gi = g0; gi < items; gi += stride)
                restrict_flat_item<T, D>(P, op.S, F.X, F.XG, F.F, F.E, F.EG, F.F, op.arg, gi);
            break;
        case TK_FAS:
            for (long long gi = g0; gi < items; gi += stride) fas_flat_item<T, D>(P, op.S, F, op.arg, gi);
            break;
        default:
            for (long long gi = g0; gi < items; gi += stride) prolong_flat_item<T, D>(P, op.S, F, gi);
            break;
        }
        if (op.bar && o + 1 < prog.nops && !tail_grid_sync(cnt, gen, P.wait_limit)) {
            atomicExch(P.status, 1);
            return;
        }
    }
}

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
    P.status = t->d_status;
    P.uniform = t->is_batch ? 0 : 1;
    P.lo0f = (float)t->lo[0];
    P.helmf = (float)t->helm;
    P.wait_limit = t->wait_limit;
    return P;
}

// The dynamic shared-memory ceiling of a kernel is a property of the kernel,
// shared by every tree and launch site: it only ever rises, so a launch
// asking for less never lowers it under another launch that needs more.  It
// is raised for any request, not only above 48 KB: the kernel's static
// shared memory counts against the same default limit.
template <class K> static void set_smem(K kernel, size_t bytes) {
    if (bytes == 0) return;
    static std::mutex mu;
    static std::vector<std::pair<const void *, size_t>> ceil;
    std::lock_guard<std::mutex> lock(mu);
    for (auto &c : ceil)
        if (c.first == (const void *)kernel) {
            if (c.second >= bytes) return;
            c.second = bytes;
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
            return;
        }
    ceil.push_back({(const void *)kernel, bytes});
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// resident CTAs per SM of a kernel at (threads, dynamic smem), queried once
// per distinct request (host launch overhead stays off the hot path)
template <class K> static int resident_ctas(K kernel, int threads, size_t smem) {
    struct Entry { const void *k; int th; size_t sm; int per; };
    static std::vector<Entry> cache;
    for (const Entry &e : cache)
        if (e.k == (const void *)kernel && e.th == threads && e.sm == smem) return e.per;
    set_smem(kernel, smem);
    int per = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    per = std::max(1, per);
    cache.push_back({(const void *)kernel, threads, smem, per});
    return per;
}

static int threads_for(int cells) {
    int t = ((cells + 31) / 32) * 32;
    return t < 32 ? 32 : (t > kMaxThreads ? kMaxThreads : t);
}

// CTA size of the TMA transfer kernels (restriction, prolongation, FAS
// right-hand side, ghost fill): their phases are uneven (all cells, then a
// parent octant, then face cells), so small CTAs waste less at barriers.
// 128 threads measured best on GB300 (mixed solve of the 20M-unknown tree:
// 19.8 ms at 256, 18.8 at 128, 19.1 at 64); MG_TRANSFER_THREADS overrides.
// Threads per CTA of the staged transfer kernels: 128, where several CTAs
// share an SM (their phases are uneven, and 256-thread CTAs lost more at
// the barriers); blocks of 16^3 cells, whose double-buffered stages leave
// room for one CTA per SM, take transfer_bound (512).
static int transfer_threads(int want, int cells) {
    static int cap = [] {
        const char *e = std::getenv("MG_TRANSFER_THREADS");
        const int v = e ? std::atoi(e) : 128;
        return (v >= 32 && v <= kMaxThreads && v % 32 == 0) ? v : 128;
    }();
    return cells >= 4096 ? 2 * kMaxThreads : std::min(want, cap);
}

template <class T, int D> struct Launch {
    static bool is_flat(const LevelHost &L) { return cells_of<D>(L.n) <= kFlatCells; }
    // ---- tail recording (see k_tail).  While a cycle records, the flat
    // helpers append phases instead of launching, and the group steps take
    // the flat path on every segment.
    struct TailRec {
        std::vector<TailOp> ops;
        int seq = 0;  // first phase of the flat step being recorded
        KParams P;
        Fields<T> F;
    };
    static TailRec *rec(mg_tree *t) { return static_cast<TailRec *>(t->tail_rec); }
    static bool flat_mode(mg_tree *t, const LevelHost &L) { return is_flat(L) || t->tail_rec != nullptr; }
    static int tail_capacity(mg_tree *t) {
        static int per = 0;
        if (!per) {
            per = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tail<T, D>, kTailThreads, 0);
            per = std::max(1, per);
        }
        return per * t->nsm;
    }
    static void tail_launch(mg_tree *t, TailRec &r) {
        if (r.ops.empty()) return;
        static TailProg prog;  // 14 KB: kept off the stack
        prog.nops = (int)r.ops.size();
        long long items = 1;
        for (int o = 0; o < prog.nops; o++) {
            prog.op[o] = r.ops[o];
            items = std::max(items, r.ops[o].S.off[r.ops[o].S.nseg]);
        }
        // at most two CTAs per SM: fewer arrivals per grid barrier
        const long long need = (items + kTailThreads - 1) / kTailThreads;
        const int grid = (int)std::max(1LL, std::min<long long>(need, std::min(tail_capacity(t), 2 * t->nsm)));
        ++t->launches;
        launch_coop(k_tail<T, D>, grid, kTailThreads, t->stream, r.P, r.F, prog);
        r.ops.clear();
        r.seq = 0;
    }
    // a flat step's phase, when recording; false: launch it
    static bool tail_add(mg_tree *t, int kind, int arg, const FlatSegs &S) {
        TailRec *r = rec(t);
        if (!r) return false;
        if ((int)r->ops.size() == kTailMaxOps) tail_launch(t, *r);
        if ((int)r->ops.size() > r->seq) r->ops.back().bar = 0;  // same step: independent segments
        TailOp op;
        op.kind = kind;
        op.arg = arg;
        op.bar = 1;
        op.S = S;
        r->ops.push_back(op);
        return true;
    }
    static void tail_begin(mg_tree *t, TailRec &r) { t->tail_rec = &r; }
    static void tail_end(mg_tree *t, TailRec &r) {
        if (t->tail_rec != &r) return;
        t->tail_rec = nullptr;
        tail_launch(t, r);
    }
    // Groups 1..cut of a cycle topped at `top` run in the tail kernel: every
    // non-coarsest segment of them without refinement faces, each group
    // holding at most tail_cells cells; red-black smoothing only.
    static int tail_cut(mg_tree *t, int top) {
        if (tail_state() != 1 || t->smoother == MG_SMOOTH_JACOBI || t->tail_cells <= 0) return 0;
        const long long lim = t->tail_cells;
        int cut = 0;
        for (int g = 1; g <= top; g++) {
            long long cells = 0;
            bool ok = true;
            for (int l : t->groups[g]) {
                const LevelHost &L = t->lev[l];
                if (L.coarsest) continue;
                if (L.has_cf) ok = false;
                cells += L.ncells;
            }
            if (!ok || cells > lim) break;
            cut = g;
        }
        return cut;
    }
    static int flat_grid(mg_tree *t, long long items) {
        return (int)std::max<long long>(1, std::min<long long>((items + 255) / 256, 8LL * t->nsm));
    }
    // work items per block of the flat kernels
    enum { FK_GHOST, FK_SWEEP, FK_RESTRICT, FK_FAS_VOLD, FK_PROLONG };
    static long long flat_items(int kind, int n) {
        const int C = cells_of<D>(n), G = 2 * D * face_of<D>(n);
        switch (kind) {
        case FK_GHOST: return G;
        case FK_SWEEP: return (n & 1) ? C : C / 2;
        case FK_RESTRICT: return cells_of<D>(n / 2);
        case FK_FAS_VOLD: return C + G;
        default: return C;
        }
    }
    // flat launches over the segments ls (their covered blocks only when
    // nref_only), at most kMaxFlatSegs segments per launch; launch(S, items)
    // enqueues one kernel
    template <class Fn>
    static void flat_launches(mg_tree *t, const std::vector<int> &ls, int kind, bool nref_only, Fn launch,
                              int nb_cap = -1) {
        FlatSegs S;
        S.nseg = 0;
        S.off[0] = 0;
        if (TailRec *r = rec(t)) r->seq = (int)r->ops.size();
        auto flush = [&]() {
            if (!S.nseg) return;
            if (!t->tail_rec) ++t->launches;
            launch(S, S.off[S.nseg]);
            S.nseg = 0;
        };
        for (int l : ls) {
            const LevelHost &L = t->lev[l];
            int nb = nref_only ? L.nref : L.nb;
            if (nb_cap >= 0) nb = std::min(nb, nb_cap);
            if (nb <= 0) continue;
            if (S.nseg == kMaxFlatSegs) flush();
            S.first[S.nseg] = L.first;
            S.nb[S.nseg] = nb;
            S.n[S.nseg] = L.n;
            S.off[S.nseg + 1] = S.off[S.nseg] + (long long)nb * flat_items(kind, L.n);
            S.nseg++;
        }
        flush();
    }
    // one segment (nb blocks from its first), for the per-segment call sites
    static FlatSegs one_seg(const LevelHost &L, int nb, int kind) {
        FlatSegs S;
        S.nseg = 1;
        S.first[0] = L.first;
        S.nb[0] = nb;
        S.n[0] = L.n;
        S.off[0] = 0;
        S.off[1] = (long long)nb * flat_items(kind, L.n);
        return S;
    }
    static void ghost_flat(mg_tree *t, const KParams &P, const std::vector<int> &ls, T *X, T *XG, int mode) {
        flat_launches(t, ls, FK_GHOST, false, [&](const FlatSegs &S, long long items) {
            if (tail_add(t, TK_GHOST, mode, S)) return;
            launch_k(k_ghost_flat<T, D>, flat_grid(t, items), 256, 0, t->stream, P, S, X, XG, mode);
        });
    }
    static void sweep_flat(mg_tree *t, const KParams &P, const std::vector<int> &ls, Fields<T> &F, int colour,
                           int nb_cap = -1) {
        flat_launches(t, ls, FK_SWEEP, false, [&](const FlatSegs &S, long long items) {
            if (tail_add(t, TK_SWEEP, colour, S)) return;
            launch_k(k_sweep_flat<T, D>, flat_grid(t, items), 256, 0, t->stream, P, S, F, colour);
        }, nb_cap);
    }
    static void restrict_flat(mg_tree *t, const KParams &P, const std::vector<int> &ls, T *X, const T *XG,
                              const T *Fr, const T *E, const T *EG, T *Fdst, int with_res) {
        flat_launches(t, ls, FK_RESTRICT, false, [&](const FlatSegs &S, long long items) {
            if (tail_add(t, TK_RESTRICT, with_res, S)) return;  // recorded only with the cycle's own fields
            launch_k(k_restrict_flat<T, D>, flat_grid(t, items), 256, 0, t->stream, P, S, X, XG, Fr, E, EG, Fdst,
                     with_res);
        });
    }
    static void fas_flat(mg_tree *t, const KParams &P, const std::vector<int> &ls, Fields<T> &F) {
        flat_launches(t, ls, FK_FAS_VOLD, true, [&](const FlatSegs &S, long long items) {
            if (tail_add(t, TK_FAS, 1, S)) return;
            launch_k(k_fas_flat<T, D>, flat_grid(t, items), 256, 0, t->stream, P, S, F, 1);
        });
    }
    static void prolong_flat(mg_tree *t, const KParams &P, const std::vector<int> &ls, Fields<T> &F) {
        flat_launches(t, ls, FK_PROLONG, false, [&](const FlatSegs &S, long long items) {
            if (tail_add(t, TK_PROLONG, 0, S)) return;
            launch_k(k_prolong_flat<T, D>, flat_grid(t, items), 256, 0, t->stream, P, S, F);
        });
    }
    static void ghost(mg_tree *t, const KParams &P, int l, T *X, T *XG, int mode) {
        const LevelHost &L = t->lev[l];
        if (L.nb == 0) return;
        ++t->launches;
        if (L.n == 8 || L.n == 16) {
            const size_t smt = 2 * (sizeof(BlockDesc) + sizeof(LevelDesc) + sizeof(T) * cells_of<D>(L.n));
            if (smt <= 200 * 1024) {
                auto kern = L.n == 8 ? k_ghost_tma<T, D, 8> : k_ghost_tma<T, D, 16>;
                set_smem(kern, smt);
                const int thr = transfer_threads(threads_for(2 * D * face_of<D>(L.n)), cells_of<D>(L.n));
                const int grid = std::min(L.nb, resident_ctas(kern, thr, smt) * t->nsm);
                launch_k(kern, grid, thr, smt, t->stream, P, L.first, L.nb, X, XG, mode);
                return;
            }
        }
        if (is_flat(L)) {
            const FlatSegs S = one_seg(L, L.nb, FK_GHOST);
            launch_k(k_ghost_flat<T, D>, flat_grid(t, S.off[1]), 256, 0, t->stream, P, S, X, XG, mode);
            return;
        }
        launch_k(k_ghost<T, D>, L.nb, threads_for(2 * D * face_of<D>(L.n)), 0, t->stream, P, L.first, X, XG, mode);
    }
    // Sweep variants (candidate ids for the autotuner):
    //  0 persistent CTA-per-block TMA sweep (8- and 16-cell blocks)
    //  1 CTA-per-block sweep with plain loads (any block size)
    //  2 / 3 warp-per-block TMA sweep, 8 / 4 warps per CTA (8-cell blocks)
    //  4 / 5 row-wise warp sweep, 8 warps x 2 stages / 4 warps x 3 stages
    //        (8^3 blocks, constant coefficient, Cartesian)
    //  6 flat sweep, one thread per colour cell (tiny blocks, no refinement faces)
    //  7 / 8 / 9 row-wise warp sweep with f in registers (FP32): 8 warps x 3
    //        stages / 4 warps x 4 stages / 8 warps x 2 stages
    // 10 candidate 0 with half the threads per CTA (two colour cells each)
    static size_t cand_smem(mg_tree *t, int l, Fields<T> &F, int cand) {
        const int n = t->lev[l].n, C = cells_of<D>(n), GH = 2 * D * face_of<D>(n);
        // stage of the kernels that read eps (k_sweep_warp, k_sweep_rows) and
        // of k_sweep_tma, which reads the face coefficients when present
        const size_t stage = sizeof(BlockDesc) + sizeof(LevelDesc) + sizeof(T) * (2 * C + GH + (F.E ? C + GH : 0));
        const size_t stage_tma = F.W ? sizeof(BlockDesc) + sizeof(LevelDesc) + sizeof(T) * (2 * C + GH + (2 * D + 1) * C)
                                     : stage;
        switch (cand) {
        case 0: return (n == 8 || n == 16) ? 2 * stage_tma : 0;
        case 10:  // half-width TMA sweep: only where it differs from candidate 0
            return ((n == 8 || n == 16) &&
                    sweep_tma_threads(cells_of<D>(n) / 2, true) != sweep_tma_threads(cells_of<D>(n) / 2, false))
                       ? 2 * stage_tma : 0;
        case 1: return 1;
        case 2: return n == 8 ? 16 * stage : 0;
        case 3: return n == 8 ? 8 * stage : 0;
        case 4: return (D == 3 && n == 8 && !F.E && t->geom == MG_CART) ? 16 * stage : 0;
        case 5: return (D == 3 && n == 8 && !F.E && t->geom == MG_CART) ? 12 * stage : 0;
        case 6: return (is_flat(t->lev[l]) && !t->lev[l].has_cf) ? 1 : 0;
        case 7: case 8: case 9: {
            if (!(D == 3 && n == 8 && !F.E && t->geom == MG_CART && sizeof(T) == 4)) return 0;
            const size_t sfg = sizeof(BlockDesc) + sizeof(LevelDesc) + sizeof(T) * (C + GH);
            return (cand == 7 ? 24 : 16) * sfg;
        }
        }
        return 0;
    }
    static bool cand_ok(mg_tree *t, int l, Fields<T> &F, int cand) {
        const size_t sm = cand_smem(t, l, F, cand);
        return sm > 0 && sm <= 200 * 1024;
    }
    static int default_cand(mg_tree *t, int l, Fields<T> &F) {
        for (int c : {6, 4, 0}) if (cand_ok(t, l, F, c)) return c;
        return 1;
    }
    static void sweep(mg_tree *t, const KParams &P, int l, Fields<T> &F, int colour) {
        const LevelHost &L = t->lev[l];
        const int prec = sizeof(T) == 4 ? 1 : 0;
        int cand = (int)t->sweep_choice[prec].size() > l ? t->sweep_choice[prec][l] : -1;
        if (cand < 0 || !cand_ok(t, l, F, cand)) cand = default_cand(t, l, F);
        sweep_cand(t, P, l, F, colour, cand);
        (void)L;
    }
    // nbx: the first nbx blocks of the level only (the autotuner's timed
    // subset of a very large level); -1 for the whole level
    static void sweep_cand(mg_tree *t, const KParams &P, int l, Fields<T> &F, int colour, int cand, int nbx = -1) {
        const LevelHost &L = t->lev[l];
        const int nb = nbx >= 0 ? std::min(L.nb, nbx) : L.nb;
        const int n = L.n;
        ++t->launches;
        const size_t sm = cand_smem(t, l, F, cand);
        switch (cand) {
        case 0: case 10: {
            const bool half = cand == 10;
            auto kern = n == 8 ? (half ? k_sweep_tma<T, D, 8, true> : k_sweep_tma<T, D, 8>)
                               : (half ? k_sweep_tma<T, D, 16, true> : k_sweep_tma<T, D, 16>);
            const int thr = sweep_tma_threads(cells_of<D>(n) / 2, half);
            const int grid = std::min(nb, resident_ctas(kern, thr, sm) * t->nsm);
            launch_k(kern, grid, thr, sm, t->stream, P, L.first, nb, F, colour);
            return;
        }
        case 2: case 3: {
            const int W = cand == 2 ? 8 : 4;
            auto kern = cand == 2 ? k_sweep_warp<T, D, 8> : k_sweep_warp<T, D, 4>;
            const int grid = std::min((nb + W - 1) / W, resident_ctas(kern, 32 * W, sm) * t->nsm);
            launch_k(kern, grid, 32 * W, sm, t->stream, P, L.first, nb, F, colour);
            return;
        }
        case 4: case 5: case 7: case 8: case 9: {
            if constexpr (D == 3) {
                const int W = (cand == 5 || cand == 8) ? 4 : 8;
                auto kern = cand == 4 ? k_sweep_rows<T, 8, 2> : cand == 5 ? k_sweep_rows<T, 4, 3>
                          : cand == 7 ? k_sweep_rows<T, 8, 3, true> : cand == 8 ? k_sweep_rows<T, 4, 4, true>
                                      : k_sweep_rows<T, 8, 2, true>;
                set_smem(kern, sm);
                const int grid = std::min((nb + W - 1) / W, resident_ctas(kern, 32 * W, sm) * t->nsm);
                launch_k(kern, grid, 32 * W, sm, t->stream, P, L.first, nb, F, colour);
            }
            return;
        }
        case 6: {
            const int ncol = (n & 1) ? cells_of<D>(n) : cells_of<D>(n) / 2;
            const FlatSegs S = one_seg(L, nb, FK_SWEEP);
            launch_k(k_sweep_flat<T, D>, flat_grid(t, (long long)nb * ncol), 256, 0, t->stream, P, S, F, colour);
            return;
        }
        default: {
            const int pad = D == 2 ? (n + 2) * (n + 2) : (n + 2) * (n + 2) * (n + 2);
            const size_t smp = sizeof(T) * pad * (F.E ? 2 : 1);
            const int th = threads_for((n & 1) ? cells_of<D>(n) : cells_of<D>(n) / 2);
            if (n == 8) {
                launch_k(k_sweep<T, D, 8>, nb, th, smp, t->stream, P, L.first, F, colour);
            } else if (n == 16) {
                set_smem(k_sweep<T, D, 16>, smp);
                launch_k(k_sweep<T, D, 16>, nb, th, smp, t->stream, P, L.first, F, colour);
            } else {
                set_smem(k_sweep<T, D, 0>, smp);
                launch_k(k_sweep<T, D, 0>, nb, th, smp, t->stream, P, L.first, F, colour);
            }
        }
        }
    }
    // Autotuner: per level, time every applicable sweep variant on the
    // given fields (all zero at the call sites, so sweeps leave them
    // unchanged) and keep the fastest.  Small levels keep the default.
    // Whether a cooperative launch of the tail kernel can be captured into a
    // graph and replayed here (once per process and kernel instance, when
    // the first tree tunes its sweeps): an empty program, captured on a
    // private stream.  Until it has passed, cycles run without the tail
    // kernel.
    static int &tail_state() {  // 0: not probed, 1: works, -1: refused
        static int state = 0;
        return state;
    }
    static void tail_probe(mg_tree *t) {
        int &state = tail_state();
        if (!state) {
            static TailProg empty;
            empty.nops = 0;
            cudaStream_t s = nullptr;
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            bool ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
            ok = ok && cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)std::min(tail_capacity(t), 2 * t->nsm));
                cfg.blockDim = dim3(kTailThreads);
                cfg.stream = s;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeCooperative;
                at[0].val.cooperative = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                const bool launched =
                    cudaLaunchKernelEx(&cfg, k_tail<T, D>, kparams(t, 1), Fields<T>{}, (const TailProg)empty) ==
                    cudaSuccess;
                ok = (cudaStreamEndCapture(s, &g) == cudaSuccess) && launched && g;
            }
            ok = ok && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
            ok = ok && cudaGraphLaunch(ge, s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
            if (ge) cudaGraphExecDestroy(ge);
            if (g) cudaGraphDestroy(g);
            if (s) cudaStreamDestroy(s);
            cudaGetLastError();
            state = ok ? 1 : -1;
        }
    }
    static void tune(mg_tree *t, Fields<T> &F) {
        const int prec = sizeof(T) == 4 ? 1 : 0;
        const KParams P = kparams(t, 1);
        tail_probe(t);
        t->sweep_choice[prec].assign(t->lev.size(), -1);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (size_t l = 1; l < t->lev.size(); l++) {
            if (t->lev[l].nb < 256) continue;
            std::vector<int> cands;
            for (int cand = 0; cand < kNumSweepVariants; cand++)
                if (cand_ok(t, (int)l, F, cand)) cands.push_back(cand);
            // warm-up (clocks, caches, first-launch costs), then the median
            // of five interleaved rounds of four launches per candidate; of
            // the candidates within 3 % of the fastest median the lowest
            // variant number wins, so near-ties resolve the same way in
            // every process
            // a level above kTuneCells cells is timed on its first blocks
            // (per-block costs do not change with the count beyond that)
            constexpr long long kTuneCells = 32LL << 20;
            const int nbx = (int)std::min<long long>(t->lev[l].nb, std::max<long long>(1, kTuneCells / cells_of<D>(t->lev[l].n)));
            for (int cand : cands)
                for (int w = 0; w < 4; w++) sweep_cand(t, P, (int)l, F, w & 1, cand, nbx);
            constexpr int kRounds = 5;
            std::vector<std::vector<float>> times(cands.size());
            for (int round = 0; round < kRounds; round++)
                for (size_t ci = 0; ci < cands.size(); ci++) {
                    cudaEventRecord(e0, t->stream);
                    for (int w = 0; w < 4; w++) sweep_cand(t, P, (int)l, F, w & 1, cands[ci], nbx);
                    cudaEventRecord(e1, t->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    times[ci].push_back(ms);
                }
            std::vector<float> med(cands.size());
            float bmin = 1e30f;
            for (size_t ci = 0; ci < cands.size(); ci++) {
                std::sort(times[ci].begin(), times[ci].end());
                med[ci] = times[ci][kRounds / 2];
                bmin = std::min(bmin, med[ci]);
            }
            for (size_t ci = 0; ci < cands.size(); ci++)
                if (med[ci] <= 1.03f * bmin) { t->sweep_choice[prec][l] = cands[ci]; break; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaGetLastError();
    }
    static void jacobi(mg_tree *t, const KParams &P, int l, Fields<T> &F) {
        const LevelHost &L = t->lev[l];
        ++t->launches;
        launch_k(k_jacobi_flat<T, D>, flat_grid(t, L.ncells), 256, 0, t->stream, P, L.first, L.nb, L.n, F,
                 (T)t->omega);
        cudaMemcpyAsync(F.X + L.cell_first, F.J + L.cell_first, sizeof(T) * L.ncells, cudaMemcpyDeviceToDevice,
                        t->stream);
        ghost(t, P, l, F.X, F.XG, 0);
    }
    static void smooth(mg_tree *t, const KParams &P, int l, Fields<T> &F, int sweeps) {
        for (int s = 0; s < sweeps; s++) {
            if (t->smoother == MG_SMOOTH_JACOBI && F.J) {
                jacobi(t, P, l, F);
                continue;
            }
            for (int colour = 0; colour < 2; colour++) sweep(t, P, l, F, colour);
        }
    }
    // Downward FAS step from group g to g-1 (Sec. 2.4): every non-coarsest
    // segment of g restricts into its parents (pushing the parent-level
    // ghosts), then f^H and v_old are formed on the covered blocks of g-1.
    static void restrict_group(mg_tree *t, const KParams &P, int g, Fields<T> &F) {
        // parent segments fed by a restriction without ghost push get a
        // ghost fill before their FAS right-hand side
        std::vector<char> plain(t->lev.size(), 0);
        std::vector<int> flat;  // flat segments: shared launches below
        for (int l : t->groups[g]) {
            const LevelHost &L = t->lev[l];
            if (L.coarsest) continue;
            if (flat_mode(t, L)) {
                flat.push_back(l);
                for (int q : L.parents) plain[q] = 1;
                continue;
            }
            ++t->launches;
            const int C8 = cells_of<D>(L.n), GH8 = 2 * D * face_of<D>(L.n);
            const size_t smt = 2 * (2 * (sizeof(BlockDesc) + sizeof(LevelDesc)) +
                                    sizeof(T) * (2 * C8 + GH8 + (F.W ? 2 * D * C8 : (F.E ? C8 + GH8 : 0))));
            if (D == 3 && L.n == 8 && L.parent_same_n && !F.W && !F.E && t->geom == MG_CART) {
                const size_t sr = 2 * sizeof(T) * (2 * C8 + GH8) + 4 * (sizeof(BlockDesc) + sizeof(LevelDesc));
                set_smem(k_restrict_rows<T>, sr);
                const int grid = std::min(L.nb, resident_ctas(k_restrict_rows<T>, 128, sr) * t->nsm);
                launch_k(k_restrict_rows<T>, grid, 128, sr, t->stream, P, L.first, L.nb, F);
            } else if ((L.n == 8 || L.n == 16) && smt + sizeof(T) * C8 <= 200 * 1024) {
                auto kern = L.n == 8 ? k_restrict_tma<T, D, 8> : k_restrict_tma<T, D, 16>;
                const int thr = transfer_threads(threads_for(C8), C8);
                const int grid = std::min(L.nb, resident_ctas(kern, thr, smt) * t->nsm);
                launch_k(kern, grid, thr, smt, t->stream, P, L.first, L.nb, F);
            } else if (L.n >= 4) {
                launch_k(k_restrict_push<T, D>, L.nb, threads_for(cells_of<D>(L.n / 2)), sizeof(T) * cells_of<D>(L.n / 2), t->stream, P, L.first, F);
            } else {
                launch_k(k_restrict<T, D>, L.nb, threads_for(cells_of<D>(L.n / 2)), 0, t->stream, P, L.first, F.X, F.XG,
                                                                                             F.F, F.E, F.EG, F.F, 1);
                for (int q : L.parents) plain[q] = 1;
            }
        }
        if (!flat.empty()) restrict_flat(t, P, flat, F.X, F.XG, F.F, F.E, F.EG, F.F, 1);
        std::vector<int> flat_ghost, flat_fas;
        for (int c : t->groups[g - 1])
            if (plain[c]) {
                if (flat_mode(t, t->lev[c])) flat_ghost.push_back(c);
                else ghost(t, P, c, F.X, F.XG, 0);
            }
        if (!flat_ghost.empty()) ghost_flat(t, P, flat_ghost, F.X, F.XG, 0);
        for (int c : t->groups[g - 1]) {
            const LevelHost &C = t->lev[c];
            if (C.nref <= 0) continue;
            if (flat_mode(t, C)) {
                flat_fas.push_back(c);
                continue;
            }
            ++t->launches;
            const int Cc = cells_of<D>(C.n), Gc = 2 * D * face_of<D>(C.n);
            const size_t smf = 2 * (sizeof(BlockDesc) + sizeof(LevelDesc) +
                                    sizeof(T) * (2 * Cc + Gc + (F.W ? 2 * D * Cc : (F.E ? Cc + Gc : 0))));
            if ((C.n == 8 || C.n == 16) && smf <= 200 * 1024) {
                auto kern = C.n == 8 ? k_fas_tma<T, D, 8> : k_fas_tma<T, D, 16>;
                set_smem(kern, smf);
                const int thr = transfer_threads(threads_for(cells_of<D>(C.n)), cells_of<D>(C.n));
                const int grid = std::min(C.nref, resident_ctas(kern, thr, smf) * t->nsm);
                launch_k(kern, grid, thr, smf, t->stream, P, C.first, C.nref, F);
            } else {
                launch_k(k_fas_rhs_vold<T, D>, C.nref, threads_for(cells_of<D>(C.n)), 0, t->stream, P, C.first, F);
            }
        }
        if (!flat_fas.empty()) fas_flat(t, P, flat_fas, F);
    }
    static size_t prolong_tma_smem(const LevelHost &L) {
        const int n = L.n, pn = L.parent_same_n ? n : n / 2;
        const size_t Cp = cells_of<D>(pn), GHp = 2 * D * face_of<D>(pn);
        return 2 * (sizeof(BlockDesc) + sizeof(LevelDesc) + sizeof(BlockDesc) +
                    sizeof(T) * (cells_of<D>(n) + 2 * (Cp + GHp)));
    }
    static void prolong(mg_tree *t, const KParams &P, int l, Fields<T> &F) {
        const LevelHost &L = t->lev[l];
        ++t->launches;
        if (D == 3 && L.n == 8 && L.parent_same_n) {
            const size_t smt = prolong_tma_smem(L);
            set_smem(k_prolong_rows<T>, smt);
            const int grid = std::min(L.nb, resident_ctas(k_prolong_rows<T>, 128, smt) * t->nsm);
            launch_k(k_prolong_rows<T>, grid, 128, smt, t->stream, P, L.first, L.nb, F);
            return;
        }
        if (D == 2 && L.n == 16 && L.parent_same_n && sizeof(T) == 4) {  // FP64: the CTA-per-cell form timed faster
            const size_t smt = prolong_tma_smem(L);
            set_smem(k_prolong_rows2<T>, smt);
            const int grid = std::min(L.nb, resident_ctas(k_prolong_rows2<T>, 64, smt) * t->nsm);
            launch_k(k_prolong_rows2<T>, grid, 64, smt, t->stream, P, L.first, L.nb, F);
            return;
        }
        if ((L.n == 8 || L.n == 16) && prolong_tma_smem(L) <= 200 * 1024) {
            const size_t smt = prolong_tma_smem(L);
            auto kern = L.n == 8 ? k_prolong_tma<T, D, 8> : k_prolong_tma<T, D, 16>;
            set_smem(kern, smt);
            const int thr = transfer_threads(threads_for(cells_of<D>(L.n) / 2), cells_of<D>(L.n));
            const int grid = std::min(L.nb, resident_ctas(kern, thr, smt) * t->nsm);
            launch_k(kern, grid, thr, smt, t->stream, P, L.first, L.nb, F, L.parent_same_n ? L.n : L.n / 2);
            return;
        }
        if (is_flat(L)) {
            const FlatSegs S = one_seg(L, L.nb, FK_PROLONG);
            launch_k(k_prolong_flat<T, D>, flat_grid(t, S.off[1]), 256, 0, t->stream, P, S, F);
            ghost(t, P, l, F.X, F.XG, 0);
            return;
        }
        const size_t sm = sizeof(T) * cells_of<D>(L.n);
        set_smem(k_prolong_push<T, D>, sm);
        launch_k(k_prolong_push<T, D>, L.nb, threads_for(cells_of<D>(L.n)), sm, t->stream, P, L.first, F);
    }
    // exact coarsest solves of the trees whose coarsest group is below `top`
    // (strict) or at most `top`; then ghost fills of the coarsest segments
    static void coarse(mg_tree *t, const KParams &P, Fields<T> &F, int top, int strict) {
        coarse_solve(t, P, F, top, strict);
        coarse_ghosts(t, P, F, top);
    }
    static void coarse_solve(mg_tree *t, const KParams &P, Fields<T> &F, int top, int strict) {
        const int ntr = (int)t->tcoarse.size();
        if (t->coarse_mode == 1) {  // the paper's smoothing of the coarsest level
            const size_t sm = sizeof(double) * (size_t)t->coarse_pad * (F.E ? 3 : 2);
            set_smem(k_coarse_gs<T, D>, sm);
            ++t->launches;
            launch_k(k_coarse_gs<T, D>, ntr, 1024, sm, t->stream, P, t->d_tcoarse, top, strict, F,
                     CoarseSmooth{t->coarse_abs, t->coarse_rel, t->coarse_max_it});
            return;
        }
        if (t->n_coarse_chunks) {  // trees with a dense inverse
            ++t->launches;
            launch_k(k_coarse_resid_b<T, D>, ntr, 1024, 0, t->stream, P, t->d_tcoarse, top, strict, F, t->d_cvec);
            ++t->launches;
            launch_k(k_coarse_apply_b<T>, t->n_coarse_chunks, 32 * kCoarseRows, 0, t->stream, t->d_tcoarse,
                     t->d_coarse_chunks, top, strict, t->d_minv, t->d_cvec, F.X);
        }
        if (t->n_btri) {
            ++t->launches;
            launch_k(k_coarse_resid_bt<T, D>, t->n_bt_chunks, kBtResidCells, 0, t->stream, P, t->d_tcoarse,
                     t->d_bt_chunks, top, strict, F, (const double *)t->d_wface, (const int *)t->d_btperm,
                     t->d_cvec);
            ++t->launches;
            if constexpr (sizeof(T) == 4) {  // one warp per tree; ring of about 40 KB
                const int slot = bt32_stride(t->bt_pmax);
                const int ring = std::max(2, std::min(kBtriMaxRing, (int)(40960 / (sizeof(float) * slot))));
                const size_t sm = sizeof(float) * ((size_t)ring * slot + 2 * kBtriMaxPlane + 2 * (size_t)t->bt_ncmax);
                set_smem(k_coarse_btri_f32<D>, sm);
                launch_k(k_coarse_btri_f32<D>, t->n_btri, 32, sm, t->stream, P, t->d_tcoarse, t->d_btlist, top,
                         strict, F.X, (const double *)t->d_cvec, (const float *)t->d_bt32,
                         (const int *)t->d_btperm, ring, slot);
            } else {
                // two warps per tree with two or more trees per SM (the FP64
                // units are then busy with other trees), else four; ring of
                // about 40 KB
                const int slot = bt_stride(t->bt_pmax);
                const int ring = std::max(2, std::min(kBtriMaxRing, (int)(40960 / (sizeof(double) * slot))));
                const int threads = t->n_btri >= 2 * t->nsm ? 64 : kBtriThreads;
                const size_t sm = sizeof(double) * ((size_t)ring * slot + 2 * (size_t)t->bt_ncmax +
                                                    2 * (threads / 32) * (size_t)t->bt_pmax);
                set_smem(k_coarse_btri<T, D>, sm);
                launch_k(k_coarse_btri<T, D>, t->n_btri, threads, sm, t->stream, P, t->d_tcoarse, t->d_btlist,
                         top, strict, F, (const double *)t->d_cvec, (const double *)t->d_bt,
                         (const float *)t->d_bt32, (const int *)t->d_btperm, ring, slot);
            }
        }
    }
    // smoothing steps on level l: the per-level schedule where one is set
    // (mg_set_schedule), else the cycle's n_down / n_up
    static int steps(const mg_tree *t, int l, int n, bool down) {
        const std::vector<int> &s = down ? t->sched_down : t->sched_up;
        return (l < (int)s.size() && s[l] >= 0) ? s[l] : n;
    }
    // the sweep variant segment l runs (the autotuner's pick, else the default)
    static int chosen_cand(mg_tree *t, int l, Fields<T> &F) {
        const int prec = sizeof(T) == 4 ? 1 : 0;
        int cand = (int)t->sweep_choice[prec].size() > l ? t->sweep_choice[prec][l] : -1;
        if (cand < 0 || !cand_ok(t, l, F, cand)) cand = default_cand(t, l, F);
        return cand;
    }
    // smoothing of every non-coarsest segment of group g; segments on the
    // flat sweep with the same step count share each colour launch (the
    // segments of a group are independent trees' levels)
    static void smooth_group(mg_tree *t, const KParams &P, int g, Fields<T> &F, int n, bool down) {
        std::map<int, std::vector<int>> flat;  // step count -> segments
        const bool jac = t->smoother == MG_SMOOTH_JACOBI && F.J;
        for (int l : t->groups[g]) {
            if (t->lev[l].coarsest) continue;
            const int st = steps(t, l, n, down);
            if (!jac && (t->tail_rec || chosen_cand(t, l, F) == 6)) flat[st].push_back(l);
            else smooth(t, P, l, F, st);
        }
        for (auto &kv : flat)
            for (int s = 0; s < kv.first; s++)
                for (int colour = 0; colour < 2; colour++) sweep_flat(t, P, kv.second, F, colour);
    }
    // prolongation into every non-coarsest segment of group g (flat
    // segments in shared launches, then their ghosts)
    static void prolong_group(mg_tree *t, const KParams &P, int g, Fields<T> &F) {
        std::vector<int> flat;
        for (int l : t->groups[g]) {
            if (t->lev[l].coarsest) continue;
            if (flat_mode(t, t->lev[l])) flat.push_back(l);
            else prolong(t, P, l, F);
        }
        if (flat.empty()) return;
        prolong_flat(t, P, flat, F);
        ghost_flat(t, P, flat, F.X, F.XG, 0);
    }
    // The groups up to tail_cut run in the tail kernel: the downward steps
    // below the cut in one launch, the coarsest solve, then the coarsest
    // ghosts and the upward steps up to the cut in another.
    static void vcycle(mg_tree *t, Fields<T> &F, int top, int nd, int nu, int homog, int strict = 0) {
        const KParams P = kparams(t, homog);
        const int cut = tail_cut(t, top);
        TailRec tr;
        tr.P = P;
        tr.F = F;
        for (int g = top; g >= 1; g--) {
            if (g == cut) tail_begin(t, tr);
            smooth_group(t, P, g, F, nd, true);
            restrict_group(t, P, g, F);
        }
        tail_end(t, tr);
        coarse_solve(t, P, F, top, strict);
        if (cut) tail_begin(t, tr);
        coarse_ghosts(t, P, F, top);
        for (int g = 1; g <= top; g++) {
            prolong_group(t, P, g, F);
            smooth_group(t, P, g, F, nu, false);
            if (g == cut) tail_end(t, tr);
        }
        tail_end(t, tr);
    }
    static void fmg(mg_tree *t, Fields<T> &F, int nd, int nu, int homog) {
        const KParams P = kparams(t, homog);
        const int top = (int)t->groups.size() - 1;
        const int cut = tail_cut(t, top);
        TailRec tr;
        tr.P = P;
        tr.F = F;
        for (int g = top; g >= 1; g--) {
            if (g == cut) tail_begin(t, tr);
            restrict_group(t, P, g, F);
        }
        tail_end(t, tr);
        coarse(t, P, F, top, 0);
        for (int g = 1; g <= top; g++) {
            prolong_group(t, P, g, F);
            vcycle(t, F, g, nd, nu, homog, 1);
        }
    }
    // ghosts of the coarsest segments of groups up to top (after their
    // solve); flat segments in shared launches
    static void coarse_ghosts(mg_tree *t, const KParams &P, Fields<T> &F, int top) {
        std::vector<int> flat;
        for (size_t l = 0; l < t->lev.size(); l++) {
            if (!t->lev[l].coarsest || t->lev[l].group > top || t->lev[l].nb == 0) continue;
            if (flat_mode(t, t->lev[l])) flat.push_back((int)l);
            else ghost(t, P, (int)l, F.X, F.XG, 0);
        }
        if (!flat.empty()) ghost_flat(t, P, flat, F.X, F.XG, 0);
    }
    // covered cells <- mean of children (finest first), then all ghosts
    // Lowest group whose values a leaf stencil can reach: groups with leaves,
    // the group below a level with refinement faces (the coarser cells of its
    // ghosts) and, where that group has refinement faces too, the one below
    // it (a refinement ghost reads the coarser block's own ghosts).  Every
    // refresh consumer reads leaf stencils only; a V-cycle restricts into
    // the groups below itself.
    static int refresh_gmin(const mg_tree *t) {
        const int ng = (int)t->groups.size();
        std::vector<char> cf(ng, 0);
        for (int g = 0; g < ng; g++)
            for (int l : t->groups[g]) cf[g] |= t->lev[l].has_cf ? 1 : 0;
        int gmin = ng;
        for (int g = 0; g < ng; g++)
            for (int l : t->groups[g]) {
                const LevelHost &L = t->lev[l];
                if (L.nb > L.nref) gmin = std::min(gmin, g);
                if (L.has_cf && g >= 1) gmin = std::min(gmin, cf[g - 1] && g >= 2 ? g - 2 : g - 1);
            }
        return gmin;
    }
    // full: every group, for readers of covered cells other than leaf
    // stencils (the transfer of phi to an adapted mesh copies a coarsened
    // block's covered cells, which may lie below every leaf stencil)
    // e_add (FP64 fields only): the defect-correction update phi += e on
    // the leaf cells, fused into the restriction of the segments it passes
    // (k_update_restrict) and done first elsewhere
    static void refresh(mg_tree *t, Fields<T> &F, int homog, int mode = 0, bool full = false,
                        const float *e_add = nullptr) {
        const KParams P = kparams(t, homog);
        const int top = (int)t->groups.size() - 1;
        const int gmin = full ? 0 : refresh_gmin(t);
        std::vector<char> updated(t->lev.size(), 0);
        for (int g = top; g >= 1 && g - 1 >= gmin; g--)
            for (int l : t->groups[g]) {
                const LevelHost &L = t->lev[l];
                if (L.coarsest) continue;
                if constexpr (sizeof(T) == 8) {
                    if (e_add && L.nb > L.nref) {
                        updated[l] = 1;
                        if (L.n >= 4) {
                            const int C = cells_of<D>(L.n);
                            ++t->launches;
                            const int thr = std::max(32, std::min(256, (C / kUpdCells + 31) / 32 * 32));
                            launch_k(k_update_restrict<D>, L.nb, thr, sizeof(double) * C, t->stream, P, L.first, L.nref, F.X,
                                     e_add);
                            continue;
                        }
                        enqueue_add_leaf(t, {l}, e_add, F.X);  // before this segment's restriction reads it
                    }
                }
                ++t->launches;
                if (is_flat(L))
                    launch_k(k_restrict_flat<T, D>, flat_grid(t, (long long)L.nb * cells_of<D>(L.n / 2)), 256, 0,
                             t->stream, P, one_seg(L, L.nb, FK_RESTRICT), F.X, F.XG, F.F, F.E, F.EG, F.F, 0);
                else
                    launch_k(k_restrict<T, D>, L.nb, threads_for(cells_of<D>(L.n / 2)), 0, t->stream, P, L.first, F.X, F.XG,
                                                                                                 F.F, F.E, F.EG, F.F, 0);
            }
        if constexpr (sizeof(T) == 8) {
            if (e_add) {  // leaf segments no restriction above passed
                std::vector<int> rest;
                for (size_t l = 0; l < t->lev.size(); l++)
                    if (!updated[l] && t->lev[l].nb > t->lev[l].nref) rest.push_back((int)l);
                enqueue_add_leaf(t, rest, e_add, F.X);
            }
        }
        for (int g = gmin; g <= top; g++)
            for (int l : t->groups[g]) ghost(t, P, l, F.X, F.XG, mode);
    }
    static void refresh_eps(mg_tree *t, Fields<T> &F) {
        const KParams P = kparams(t, 0);
        const int top = (int)t->groups.size() - 1;
        for (int g = top; g >= 1; g--)
            for (int l : t->groups[g]) {
                const LevelHost &L = t->lev[l];
                if (L.coarsest) continue;
                ++t->launches;
                if (is_flat(L))
                    launch_k(k_restrict_flat<T, D>, flat_grid(t, (long long)L.nb * cells_of<D>(L.n / 2)), 256, 0,
                             t->stream, P, one_seg(L, L.nb, FK_RESTRICT), F.E, F.EG, nullptr, nullptr, nullptr,
                             nullptr, 0);
                else
                    launch_k(k_restrict<T, D>, L.nb, threads_for(cells_of<D>(L.n / 2)), 0, t->stream, P, L.first, F.E, F.EG, nullptr, nullptr, nullptr, nullptr, 0);
            }
        for (int g = 0; g <= top; g++)
            for (int l : t->groups[g]) ghost(t, P, l, F.E, F.EG, 1);
    }
};

template <class T> void tune_sweeps(mg_tree *t, Fields<T> &F) {
    if (t->dim == 2) Launch<T, 2>::tune(t, F);
    else Launch<T, 3>::tune(t, F);
}
template void tune_sweeps<double>(mg_tree *, Fields<double> &);
int sweep_variant(mg_tree *t, int prec, int level) {
    if (prec == 1 && !t->f32.X) return -1;
    if (t->dim == 2) {
        int c = (int)t->sweep_choice[prec].size() > level ? t->sweep_choice[prec][level] : -1;
        if (prec == 1) return c >= 0 && Launch<float, 2>::cand_ok(t, level, t->f32, c) ? c : Launch<float, 2>::default_cand(t, level, t->f32);
        return c >= 0 && Launch<double, 2>::cand_ok(t, level, t->f64, c) ? c : Launch<double, 2>::default_cand(t, level, t->f64);
    }
    int c = (int)t->sweep_choice[prec].size() > level ? t->sweep_choice[prec][level] : -1;
    if (prec == 1) return c >= 0 && Launch<float, 3>::cand_ok(t, level, t->f32, c) ? c : Launch<float, 3>::default_cand(t, level, t->f32);
    return c >= 0 && Launch<double, 3>::cand_ok(t, level, t->f64, c) ? c : Launch<double, 3>::default_cand(t, level, t->f64);
}
template void tune_sweeps<float>(mg_tree *, Fields<float> &);
bool sweep_variant_ok(mg_tree *t, int prec, int level, int variant) {
    if (variant < 0 || variant >= kNumSweepVariants) return false;
    if (prec == 1) {
        if (!t->f32.X) return false;
        return t->dim == 2 ? Launch<float, 2>::cand_ok(t, level, t->f32, variant)
                           : Launch<float, 3>::cand_ok(t, level, t->f32, variant);
    }
    return t->dim == 2 ? Launch<double, 2>::cand_ok(t, level, t->f64, variant)
                       : Launch<double, 3>::cand_ok(t, level, t->f64, variant);
}
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

// bytes of the two stages of k_resid_tma for n-cell blocks
template <int D> static size_t resid_smem(int n, const Fields<double> &F) {
    const int C = cells_of<D>(n), GH = 2 * D * face_of<D>(n);
    const size_t padded = (!F.W && !F.E) ? sizeof(int64_t) * cells_of<D>(n + 2) : 0;  // exact-sum stencil array
    return 2 * (sizeof(BlockDesc) + sizeof(LevelDesc) +
                sizeof(double) * (2 * C + GH + (F.W ? (2 * D + 1) * C : (F.E ? C + GH : 0)))) + padded;
}

template <int D>
static void residual_norm_d(mg_tree *t, Fields<double> &F, int homog, double *out3, double *r64_leaf,
                            float *f32_cells, bool want_max = true, const float *e_add = nullptr) {
    Launch<double, D>::refresh(t, F, homog, 0, false, e_add);
    const KParams P = kparams(t, homog);
    int slot = 0;
    long long leaf_base = 0;
    for (size_t l = 0; l < t->lev.size(); l++) {
        const LevelHost &L = t->lev[l];
        const int nleaf = L.nb - L.nref;
        if (nleaf <= 0) continue;
        const long long cell_base = t->blocks[L.first + L.nref].cell_off;
        ++t->launches;
        const int C = cells_of<D>(L.n), GH = 2 * D * face_of<D>(L.n);
        const size_t smt = resid_smem<D>(L.n, F);
        if ((L.n == 8 || L.n == 16) && smt <= 200 * 1024) {
            auto kern = want_max ? (L.n == 8 ? k_resid_tma<D, 8, true> : k_resid_tma<D, 16, true>)
                                 : (L.n == 8 ? k_resid_tma<D, 8, false> : k_resid_tma<D, 16, false>);
            const int thr = threads_for(C);
            const int grid = std::min(nleaf, resident_ctas(kern, thr, smt) * t->nsm);
            launch_k(kern, grid, thr, smt, t->stream, P, L.first + L.nref, nleaf, F, t->d_partials + 3 * slot, r64_leaf,
                                               leaf_base, f32_cells, 0);
            slot += grid;
        } else {
            if (D == 3 && L.n == 16)
                launch_k(want_max ? k_resnorm<D, true, 16> : k_resnorm<D, false, 16>, nleaf, kMaxThreads, 0,
                         t->stream, P, L.first + L.nref, F, t->d_partials + 3 * slot, r64_leaf, leaf_base, cell_base,
                         f32_cells);
            else
                launch_k(want_max ? k_resnorm<D, true> : k_resnorm<D, false>, nleaf, threads_for(C), 0, t->stream, P,
                         L.first + L.nref, F, t->d_partials + 3 * slot, r64_leaf, leaf_base, cell_base, f32_cells);
            slot += nleaf;
        }
        leaf_base += (long long)nleaf * cells_of<D>(L.n);
    }
    ++t->launches;
    launch_k(k_reduce3, 1, 1024, 0, t->stream, t->d_partials, slot, t->d_red);
    cudaMemcpyAsync(t->h_red, t->d_red, 3 * sizeof(double), cudaMemcpyDeviceToHost, t->stream);
    (void)out3;
}

// enqueue only (no synchronisation: usable inside a stream capture); the
// reduced values land in the pinned t->h_red
void residual_enqueue(mg_tree *t, Fields<double> &F, int homog, double *r64_leaf, float *f32_cells, bool want_max,
                      const float *e_add) {
    if (t->dim == 2) residual_norm_d<2>(t, F, homog, nullptr, r64_leaf, f32_cells, want_max, e_add);
    else residual_norm_d<3>(t, F, homog, nullptr, r64_leaf, f32_cells, want_max, e_add);
}

// Batch: composite residual with one partial per leaf block, reduced per
// tree into d_tree3 (3 values per tree), copied to the pinned t->h_tree3.
template <int D> static void residual_trees_d(mg_tree *t, Fields<double> &F, float *f32, bool want_max,
                                             const float *e_add) {
    Launch<double, D>::refresh(t, F, 0, 0, false, e_add);
    const KParams P = kparams(t, 0);
    int slot = 0;
    for (size_t l = 0; l < t->lev.size(); l++) {
        const LevelHost &L = t->lev[l];
        const int nleaf = L.nb - L.nref;
        if (nleaf <= 0) continue;
        const long long cell_base = t->blocks[L.first + L.nref].cell_off;
        ++t->launches;
        const int C = cells_of<D>(L.n), GH = 2 * D * face_of<D>(L.n);
        const size_t smt = resid_smem<D>(L.n, F);
        if ((L.n == 8 || L.n == 16) && smt <= 200 * 1024) {
            auto kern = want_max ? (L.n == 8 ? k_resid_tma<D, 8, true> : k_resid_tma<D, 16, true>)
                                 : (L.n == 8 ? k_resid_tma<D, 8, false> : k_resid_tma<D, 16, false>);
            const int thr = threads_for(C);
            const int grid = std::min(nleaf, resident_ctas(kern, thr, smt) * t->nsm);
            launch_k(kern, grid, thr, smt, t->stream, P, L.first + L.nref, nleaf, F, t->d_partials + 3LL * slot, nullptr, 0,
                                               f32, 1);
        } else {
            launch_k(k_resnorm<D>, nleaf, threads_for(C), 0, t->stream, P, L.first + L.nref, F, t->d_partials + 3LL * slot,
                                                                  nullptr, 0, cell_base, f32);
        }
        slot += nleaf;
    }
    ++t->launches;
    launch_k(k_reduce_trees, (int)t->tcoarse.size(), 256, 0, t->stream, t->d_partials, t->d_slot_off, t->d_slots,
                                                                   t->d_tree3);
    cudaMemcpyAsync(t->h_tree3, t->d_tree3, 3 * sizeof(double) * t->tcoarse.size(), cudaMemcpyDeviceToHost,
                    t->stream);
}

// Batch leaf I/O: one CTA per run chunk (pool cell, leaf index, length),
// copying between the concatenated per-tree leaf arrays and the pool.
__global__ void __launch_bounds__(256) k_runs_copy(const long long *__restrict__ runs, double *cells, double *leaf,
                                                   int to_cells) {
    pdl_entry();
    const long long c0 = runs[3LL * blockIdx.x], l0 = runs[3LL * blockIdx.x + 1], len = runs[3LL * blockIdx.x + 2];
    if (to_cells)
        for (long long i = threadIdx.x; i < len; i += blockDim.x) cells[c0 + i] = leaf[l0 + i];
    else
        for (long long i = threadIdx.x; i < len; i += blockDim.x) leaf[l0 + i] = cells[c0 + i];
}

void leaf_runs_copy(mg_tree *t, double *cells, const double *leaf, bool to_cells) {
    if (t->n_runs == 0) return;
    ++t->launches;
    launch_k(k_runs_copy, t->n_runs, 256, 0, t->stream, t->d_runs, cells, const_cast<double *>(leaf), to_cells ? 1 : 0);
}

void residual_enqueue_trees(mg_tree *t, Fields<double> &F, float *f32_cells, bool want_max, const float *e_add) {
    if (t->dim == 2) residual_trees_d<2>(t, F, f32_cells, want_max, e_add);
    else residual_trees_d<3>(t, F, f32_cells, want_max, e_add);
}

void residual_wait(mg_tree *t, double *out3) {
    cudaStreamSynchronize(t->stream);
    out3[0] = t->h_red[0];
    out3[1] = t->h_red[1];
    out3[2] = t->h_red[2];
}

// Volume-weighted sum of a leaf-order field (one CTA per leaf block):
// partials (sum V r, sum V, 0).  For singular problems sum V r of the
// residual does not depend on phi (the operator maps into zero weighted mean).
template <int D>
__global__ void __launch_bounds__(256) k_leaf_vsum(KParams P, int first, const double *__restrict__ rleaf,
                                                   long long leaf_base, double *__restrict__ partials) {
    pdl_entry();
    const BlockDesc &b = P.B[first + blockIdx.x];
    const LevelDesc &L = P.L[b.lev];
    const int n = b.n, C = cells_of<D>(n);
    double a = 0, v = 0;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        double V = L.vol;
        if (P.geom == MG_CYL) V = 2.0 * M_PI * (P.lo[0] + (b.ijk[0] * n + c % n + 0.5) * L.h[0]) * L.h[0] * L.h[1];
        a = fma(V, rleaf[leaf_base + (long long)blockIdx.x * C + c], a);
        v += V;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __shared__ double sh[2][8];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][w] = a; sh[1][w] = v; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int e = 0; e < (int)(blockDim.x >> 5); e++) { x += sh[0][e]; y += sh[1][e]; }
        partials[3 * blockIdx.x] = x;
        partials[3 * blockIdx.x + 1] = y;
        partials[3 * blockIdx.x + 2] = 0;
    }
}

// sum V r / sum V over the leaves of r (leaf order); synchronises the stream
double leaf_mean(mg_tree *t, const double *rleaf) {
    const KParams P = kparams(t, 0);
    int slot = 0;
    long long leaf_base = 0;
    for (const LevelHost &L : t->lev) {
        const int nleaf = L.nb - L.nref;
        if (nleaf <= 0) continue;
        ++t->launches;
        if (t->dim == 2)
            launch_k(k_leaf_vsum<2>, nleaf, 256, 0, t->stream, P, L.first + L.nref, rleaf, leaf_base, t->d_partials + 3LL * slot);
        else
            launch_k(k_leaf_vsum<3>, nleaf, 256, 0, t->stream, P, L.first + L.nref, rleaf, leaf_base, t->d_partials + 3LL * slot);
        slot += nleaf;
        leaf_base += (long long)nleaf * (t->dim == 2 ? L.n * L.n : L.n * L.n * L.n);
    }
    ++t->launches;
    launch_k(k_reduce3, 1, 1024, 0, t->stream, t->d_partials, slot, t->d_red);
    double o[3];
    cudaMemcpyAsync(t->h_red, t->d_red, 3 * sizeof(double), cudaMemcpyDeviceToHost, t->stream);
    cudaStreamSynchronize(t->stream);
    for (int e = 0; e < 3; e++) o[e] = t->h_red[e];
    return o[1] > 0 ? o[0] / o[1] : 0.0;
}

void residual_norm(mg_tree *t, Fields<double> &F, int homog, double *out3, double *r64_leaf, float *f32_cells) {
    residual_enqueue(t, F, homog, r64_leaf, f32_cells, true);
    residual_wait(t, out3);
}

// ---------------------------------------------------- mesh adaptation ---
// Carry phi to an adapted mesh (Sec. 2.5, "Adapting the grid structure").
// New leaf block nid[q] takes, for src[q] >= 0, the cells of old block
// src[q] (a leaf, or a block whose refinement was removed: its covered
// cells hold the mean of its former children after a refresh); for
// src[q] <= -2 it is a new child of old leaf block -2 - src[q] and takes
// that block's prolongation (Sec. 2.3): (2 c0 + c_x + c_y)/4 in 2D,
// (c0 + c_x + c_y + c_z)/4 in 3D, c_d the parent neighbour on the fine
// cell's side, parent ghosts included.  One CTA per new leaf block.
template <int D>
__global__ void __launch_bounds__(256) k_transfer(const BlockDesc *__restrict__ OB, const double *__restrict__ OX,
                                                  const double *__restrict__ OXG, const BlockDesc *__restrict__ NB,
                                                  const int *__restrict__ nid, const int *__restrict__ src,
                                                  double *__restrict__ NX) {
    const BlockDesc &b = NB[nid[blockIdx.x]];
    const int s = src[blockIdx.x], n = b.n, C = cells_of<D>(n);
    if (s >= 0) {
        const BlockDesc &o = OB[s];
        for (int c = threadIdx.x; c < C; c += blockDim.x) NX[b.cell_off + c] = OX[o.cell_off + c];
        return;
    }
    const BlockDesc &p = OB[-2 - s];
    const int pn = p.n, FCp = face_of<D>(pn);
    // parent value at (i, j, k), at most one coordinate outside the parent
    auto pval = [&](int i, int j, int k) -> double {
        if (i < 0) return OXG[p.ghost_off + 0 * FCp + (D == 2 ? j : j + pn * k)];
        if (i >= pn) return OXG[p.ghost_off + 1 * FCp + (D == 2 ? j : j + pn * k)];
        if (j < 0) return OXG[p.ghost_off + 2 * FCp + (D == 2 ? i : i + pn * k)];
        if (j >= pn) return OXG[p.ghost_off + 3 * FCp + (D == 2 ? i : i + pn * k)];
        if (D == 3) {
            if (k < 0) return OXG[p.ghost_off + 4 * FCp + i + pn * j];
            if (k >= pn) return OXG[p.ghost_off + 5 * FCp + i + pn * j];
        }
        return OX[p.cell_off + cidx<D>(pn, i, j, k)];
    };
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int i, j, k;
        cell_of(c, n, D, i, j, k);
        const int a = b.poff[0] + i / 2, e = b.poff[1] + j / 2, f = D == 3 ? b.poff[2] + k / 2 : 0;
        const int sx = ((b.ijk[0] * n + i) & 1) ? 1 : -1, sy = ((b.ijk[1] * n + j) & 1) ? 1 : -1,
                  sz = ((b.ijk[2] * n + k) & 1) ? 1 : -1;
        const double v0 = pval(a, e, f);
        double nbs = pval(a + sx, e, f);
        nbs += pval(a, e + sy, f);
        if (D == 3) nbs += pval(a, e, f + sz);
        NX[b.cell_off + c] = D == 2 ? (2.0 * v0 + nbs) / 4.0 : (v0 + nbs) / 4.0;
    }
}

int transfer_phi(mg_tree *old, mg_tree *nt, const std::vector<int> &nid, const std::vector<int> &src) {
    // covered cells of every level and all ghosts of the old mesh: a block
    // whose refinement is removed copies its covered cells, and its group
    // may lie below every leaf stencil of the old mesh
    if (old->dim == 2) Launch<double, 2>::refresh(old, old->f64, 0, 0, true);
    else Launch<double, 3>::refresh(old, old->f64, 0, 0, true);
    if (!nid.empty()) {
        int *d = nullptr;
        if (cudaMalloc((void **)&d, sizeof(int) * 2 * nid.size()) != cudaSuccess) return check_cuda("transfer alloc");
        cudaMemcpyAsync(d, nid.data(), sizeof(int) * nid.size(), cudaMemcpyHostToDevice, nt->stream);
        cudaMemcpyAsync(d + nid.size(), src.data(), sizeof(int) * src.size(), cudaMemcpyHostToDevice, nt->stream);
        ++nt->launches;
        if (nt->dim == 2)
            launch_k(k_transfer<2>, (int)nid.size(), 128, 0, nt->stream, (const BlockDesc *)old->d_blocks,
                     (const double *)old->f64.X, (const double *)old->f64.XG, (const BlockDesc *)nt->d_blocks,
                     (const int *)d, (const int *)(d + nid.size()), nt->f64.X);
        else
            launch_k(k_transfer<3>, (int)nid.size(), 256, 0, nt->stream, (const BlockDesc *)old->d_blocks,
                     (const double *)old->f64.X, (const double *)old->f64.XG, (const BlockDesc *)nt->d_blocks,
                     (const int *)d, (const int *)(d + nid.size()), nt->f64.X);
        cudaStreamSynchronize(nt->stream);
        cudaFree(d);
    }
    refresh<double>(nt, nt->f64, 0);
    return check_cuda("transfer");
}

__global__ void k_sub_scalar(double *__restrict__ x, double c, long long n) {
    pdl_entry();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] -= c;
}

void sub_scalar(mg_tree *t, double *x, double c, long long n) {
    ++t->launches;
    launch_k(k_sub_scalar, 1216, 256, 0, t->stream, x, c, n);
}

void copy_eps_to_f32(mg_tree *t) {
    if (!t->f64.E || !t->f32.E) return;
    ++t->launches;
    launch_k(k_cast_f32, 1216, 256, 0, t->stream, t->f64.E, t->f32.E, t->ncells);
    ++t->launches;
    launch_k(k_cast_f32, 1216, 256, 0, t->stream, t->f64.EG, t->f32.EG, t->nghost);
}

template <int D>
static int time_sweeps_d(mg_tree *t, int level, int n_sweeps, int prec, double *out) {
    const KParams P = kparams(t, 0);
    const LevelHost &L = t->lev[level];
    std::vector<cudaEvent_t> ev(8 * n_sweeps);
    for (auto &e : ev) cudaEventCreate(&e);
    int m = 0;
    for (int s = 0; s < n_sweeps; s++)
        for (int colour = 0; colour < 2; colour++) {
            cudaEventRecord(ev[m++], t->stream);
            if (prec == 1) Launch<float, D>::sweep(t, P, level, t->f32, colour);
            else Launch<double, D>::sweep(t, P, level, t->f64, colour);
            cudaEventRecord(ev[m++], t->stream);
            cudaEventRecord(ev[m++], t->stream);
            if (prec == 1) Launch<float, D>::ghost(t, P, level, t->f32.X, t->f32.XG, 0);
            else Launch<double, D>::ghost(t, P, level, t->f64.X, t->f64.XG, 0);
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
    const double w = prec == 1 ? 4.0 : 8.0;
    out[0] = ts / nl;
    out[1] = tg / nl;
    out[2] = cells * w * (t->var_eps ? 4.0 : 3.0) + ghosts * w * (t->var_eps ? 2.0 : 1.0);
    out[3] = ghosts * w * 2.0;
    return MG_OK;
}

int time_sweeps(mg_tree *t, int level, int n_sweeps, int prec, double *out4) {
    return t->dim == 2 ? time_sweeps_d<2>(t, level, n_sweeps, prec, out4)
                       : time_sweeps_d<3>(t, level, n_sweeps, prec, out4);
}

// ------------------------------------------- residual norm, no allocation ---
// Scratch for mg_residual_norm_noalloc: per-CTA partial sums (3 doubles per
// CTA of the residual launches) followed by the 3 reduced values.  Every
// GPU that loads this library holds it until the process exits.  All calls
// share it and it keeps the last call's contents; each call overwrites every
// slot it reads, so nothing needs clearing, but calls that overlap on the GPU
// (two streams, two threads) race on it.
static constexpr int kNoAllocSlots = 16384;  // 384 KiB of partials
static __device__ __align__(256) double g_noalloc_scratch[3 * kNoAllocSlots + 4];

// Device address of the scratch array, looked up once per device with that
// device current (the host-side name of the array is only a stand-in).  The
// cached address belongs to the device's primary context: it is never
// looked up again, so it goes stale if that context is reset
// (cudaDeviceReset) while this library stays loaded.
static int noalloc_scratch(int device, double **out) {
    static std::mutex mu;
    static double *addr[64] = {nullptr};
    if (device < 0 || device >= 64) {
        mg_set_error("mg_residual_norm_noalloc: device ordinal out of range");
        return MG_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            mg_set_error(std::string("mg_residual_norm_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return MG_ERR_CUDA;
        }
        addr[device] = static_cast<double *>(p);
    }
    *out = addr[device];
    return MG_OK;
}

template <int D>
static int residual_norm_noalloc_d(mg_tree *t, double *scratch, double *out3) {
    // partial slots the residual launches will use, checked before any work
    long long need = 0;
    for (size_t l = 0; l < t->lev.size(); l++) {
        const LevelHost &L = t->lev[l];
        const int nleaf = L.nb - L.nref;
        if (nleaf <= 0) continue;
        const int C = cells_of<D>(L.n), GH = 2 * D * face_of<D>(L.n);
        const size_t smt = resid_smem<D>(L.n, t->f64);
        (void)GH;
        if ((L.n == 8 || L.n == 16) && smt <= 200 * 1024) {
            auto kern = L.n == 8 ? k_resid_tma<D, 8> : k_resid_tma<D, 16>;
            need += std::min(nleaf, resident_ctas(kern, threads_for(C), smt) * t->nsm);
        } else {
            need += nleaf;
        }
    }
    if (need > kNoAllocSlots) {
        mg_set_error("mg_residual_norm_noalloc: the residual needs " + std::to_string(need) +
                     " CTA partial sums, more than the static scratch holds (" + std::to_string(kNoAllocSlots) + ")");
        return MG_ERR_ARG;
    }
    Fields<double> &F = t->f64;
    Launch<double, D>::refresh(t, F, 0);
    const KParams P = kparams(t, 0);
    int slot = 0;
    for (size_t l = 0; l < t->lev.size(); l++) {
        const LevelHost &L = t->lev[l];
        const int nleaf = L.nb - L.nref;
        if (nleaf <= 0) continue;
        const long long cell_base = t->blocks[L.first + L.nref].cell_off;
        const int C = cells_of<D>(L.n), GH = 2 * D * face_of<D>(L.n);
        const size_t smt = resid_smem<D>(L.n, F);
        ++t->launches;
        if ((L.n == 8 || L.n == 16) && smt <= 200 * 1024) {
            auto kern = L.n == 8 ? k_resid_tma<D, 8> : k_resid_tma<D, 16>;
            const int grid = std::min(nleaf, resident_ctas(kern, threads_for(C), smt) * t->nsm);
            launch_k(kern, grid, threads_for(C), smt, t->stream, P, L.first + L.nref, nleaf, F, scratch + 3 * slot,
                                                           nullptr, 0, nullptr, 0);
            slot += grid;
        } else {
            launch_k(k_resnorm<D>, nleaf, threads_for(C), 0, t->stream, P, L.first + L.nref, F, scratch + 3 * slot,
                                                                  nullptr, 0, cell_base, nullptr);
            slot += nleaf;
        }
    }
    ++t->launches;
    launch_k(k_reduce3, 1, 1024, 0, t->stream, scratch, slot, scratch + 3 * kNoAllocSlots);
    cudaError_t e = cudaMemcpyAsync(out3, scratch + 3 * kNoAllocSlots, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                                    t->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
    if (e != cudaSuccess) {
        mg_set_error(std::string("mg_residual_norm_noalloc: ") + cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    return check_cuda("mg_residual_norm_noalloc");
}

}  // namespace mg

// The paper has no counterpart: this is an allocation-free variant of
// mg_residual_norm (see include/mg.h).
extern "C" int mg_residual_norm_noalloc(mg_tree *t, double *l2, double *linf) {
    using namespace mg;
    if (!t) {
        mg_set_error("mg_residual_norm_noalloc: null tree");
        return MG_ERR_ARG;
    }
    if (!t->finalized) {
        mg_set_error("mg_residual_norm_noalloc: tree not finalized");
        return MG_ERR_STATE;
    }
    if (!l2 || !linf) {
        mg_set_error("mg_residual_norm_noalloc: null output");
        return MG_ERR_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != t->device) {
        mg_set_error("mg_residual_norm_noalloc: the tree's device must be current");
        return MG_ERR_ARG;
    }
    double *scratch = nullptr;
    int rc = noalloc_scratch(dev, &scratch);
    if (rc) return rc;
    double o[3];
    rc = t->dim == 2 ? residual_norm_noalloc_d<2>(t, scratch, o) : residual_norm_noalloc_d<3>(t, scratch, o);
    if (rc) return rc;
    int st = 0;
    if (cudaMemcpy(&st, t->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        mg_set_error("mg_residual_norm_noalloc: status read failed");
        return MG_ERR_CUDA;
    }
    if (st) {
        cudaMemset(t->d_status, 0, sizeof(int) * kStatusWords);
        mg_set_error("a bounded wait in a residual kernel expired");
        return MG_ERR_TIMEOUT;
    }
    *l2 = std::sqrt(o[0] / o[1]);
    *linf = o[2];
    if (!std::isfinite(*l2) || !std::isfinite(*linf)) {
        mg_set_error("residual is not finite");
        return MG_ERR_NAN;
    }
    return MG_OK;
}

namespace mg {

template <int D> static void divergence_d(mg_tree *t, const double *B, double *out, int order) {
    const KParams P = kparams(t, 1);
    for (int d = 0; d < D; d++) {
        // component d into the scratch field, covered cells and ghosts refreshed
        long long off = 0;
        for (auto &L : t->lev) {
            const long long n = (long long)(L.nb - L.nref) * cells_of<D>(L.n);
            if (n == 0) continue;
            cudaMemcpyAsync(t->adj.X + t->blocks[L.first + L.nref].cell_off, B + (long long)d * t->nleaf_cells + off,
                            sizeof(double) * n, cudaMemcpyDeviceToDevice, t->stream);
            off += n;
        }
        Launch<double, D>::refresh(t, t->adj, 1, 2);
        long long leaf_base = 0;
        for (auto &L : t->lev) {
            const int nleaf = L.nb - L.nref;
            if (nleaf <= 0) continue;
            ++t->launches;
            launch_k(k_div_comp<D>, nleaf, threads_for(cells_of<D>(L.n)), 0, t->stream, P, L.first + L.nref,
                     t->adj.X, t->adj.XG, d, out, leaf_base, d > 0, order);
            leaf_base += (long long)nleaf * cells_of<D>(L.n);
        }
    }
}

template <int D> static void project_d(mg_tree *t, const double *B, double *Bout) {
    Launch<double, D>::refresh(t, t->f64, 0);
    const KParams P = kparams(t, 0);
    for (int d = 0; d < D; d++) {
        long long leaf_base = 0;
        for (auto &L : t->lev) {
            const int nleaf = L.nb - L.nref;
            if (nleaf <= 0) continue;
            ++t->launches;
            launch_k(k_grad_sub<D>, nleaf, threads_for(cells_of<D>(L.n)), 0, t->stream, P, L.first + L.nref, t->f64.X, t->f64.XG, d, B + (long long)d * t->nleaf_cells,
                Bout + (long long)d * t->nleaf_cells, leaf_base);
            leaf_base += (long long)nleaf * cells_of<D>(L.n);
        }
    }
}

void divergence(mg_tree *t, const double *B, double *out, int order) {
    if (t->dim == 2) divergence_d<2>(t, B, out, order);
    else divergence_d<3>(t, B, out, order);
}
void project(mg_tree *t, const double *B, double *Bout) {
    if (t->dim == 2) project_d<2>(t, B, Bout);
    else project_d<3>(t, B, Bout);
}

// "kernel name <<<grid, block, smem>>>" of the recorded failed launch
static std::string launch_fail_text() {
    const char *name = nullptr;
    if (cudaFuncGetName(&name, g_launch_fail.kern) != cudaSuccess || !name) name = "?";
    cudaGetLastError();
    return std::string(name) + " <<<" + std::to_string(g_launch_fail.grid) + ", " +
           std::to_string(g_launch_fail.block) + ", " + std::to_string(g_launch_fail.smem) + " B>>>";
}

int check_cuda(const char *what) {
    cudaError_t e = cudaGetLastError();
    const int le = g_launch_error.exchange(0);
    std::string where;
    if (le) {
        where = " (launch of " + launch_fail_text() + ")";
        if (e == cudaSuccess) e = (cudaError_t)le;
    }
    if (e != cudaSuccess) {
        mg_set_error(std::string(what) + ": " + cudaGetErrorString(e) + where);
        return MG_ERR_CUDA;
    }
    return MG_OK;
}

std::string take_launch_error() {
    const int le = g_launch_error.exchange(0);
    if (!le) return std::string();
    return std::string(cudaGetErrorString((cudaError_t)le)) + " in " + launch_fail_text();
}

}  // namespace mg
