// mg_internal.h -- shared between the host tree builder (mg_tree.cpp) and the
// CUDA kernels and cycle driver (mg_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mg.h"

namespace mg {

// polls of a bounded mbarrier wait before a kernel gives up, sets the status
// word and returns (a few milliseconds)
constexpr uint32_t kDefaultWaitLimit = 1u << 20;
// device words per tree: the status word and the tail kernel's grid barrier
constexpr int kStatusWords = 4;

// Per-block descriptor, one per block of every level (device table).
// Storage is interior-only, block-major, x fastest; face ghosts live in a
// separate array: block g owns 2*D faces of n^(D-1) values each at
// ghost_off, face f = 2*d + side, tangential index t1 + n*t2 (t1 < t2 the
// two dimensions other than d).
struct BlockDesc {
    long long cell_off;   // first interior cell in the field arrays
    long long ghost_off;  // first ghost value in the ghost arrays
    int n;                // cells per edge
    int lev;              // level index (0 = coarsest)
    int flags;            // bit 0: covered by children
    int parent;           // global id of the parent block, -1 on level 0
    int ijk[3];           // block coordinates on its level
    int poff[3];          // offset of this block inside its parent, in parent cells
    int nbr[6];           // >= 0 same-level neighbour id; -1 physical face;
                          // <= -2: coarser neighbour, id = -2 - nbr
    long long push[6];    // same-level neighbour across face f: first ghost slot
                          // of its face f^1 (ghost_off + (f^1) * face size), else -1
};
static_assert(sizeof(BlockDesc) % 16 == 0, "BlockDesc is copied with 16-byte bulk copies");

struct LevelDesc {
    double h[3];
    double inv_h2[3];
    int ncell[3];
    int n;
    int first;            // global id of the first block
    int nb;               // blocks on the level
    int nref;             // of which the first nref are covered by children
    long long bc_off[6];  // offset of the boundary plane of each face, -1: constant
    double inv_diag;      // 1 / (2 sum_d 1/h_d^2 + lambda): constant-coefficient Gauss-Seidel divisor
    double diag;          // 2 sum_d 1/h_d^2 + lambda: the constant-coefficient row diagonal
    double vol;           // cell volume (Cartesian)
    // FP32 copies, so that FP32 kernels do no FP64 arithmetic or conversion
    float inv_h2f[3];
    float inv_diagf, h0f, hvf;  // 1/diag, h_0, 2 pi h_0 h_1 (cylindrical volume per unit r)
};
static_assert(sizeof(LevelDesc) % 16 == 0, "LevelDesc is copied with 16-byte bulk copies");

// Scalars every kernel needs, passed by value.
struct KParams {
    const BlockDesc *B;
    const LevelDesc *L;
    const double *bcplanes;
    double lo[3];
    double bcv[6];
    int bct[6];
    double helm;
    int geom;
    int var_eps;
    int homog;            // 1: boundary values read as zero
    int *status;          // device status word: 1 = a bounded wait gave up
    int uniform;          // 1: every block of a launch shares one level descriptor
    float lo0f;           // lo[0] in FP32 (cylindrical radius in FP32 kernels)
    float helmf;          // lambda in FP32
    uint32_t wait_limit;  // polls of a bounded wait before it gives up (0: at once)
};

// Coarsest level of one tree of a pool (one tree, or a batch of trees):
// a contiguous range of blocks solved exactly, by its dense inverse or, in
// a pool of several trees, by the block-tridiagonal factorisation over the
// planes of one non-periodic dimension (bt_n > 0).
struct TreeCoarse {
    int first, nb, n;     // blocks of the coarsest level
    int nc, ns;           // cells, system size (nc + 1 when bordered)
    int singular;         // bordered by sum V x = 0
    int group;            // group index of the coarsest level
    int lvl;              // index of its level descriptor
    long long cell0;      // first cell of the level
    long long minv_off;   // offset of the ns x ns inverse (row-major), dense form
    long long cvec_off;   // offset of the residual vector (ns)
    int bt_n, bt_P;       // planes and cells per plane (0: dense form)
    int bt_dim;           // dimension across the planes
    int bt_pad;
    long long bt_off;     // offset of the bt_n FP64 plane records (bt_stride(bt_P) doubles each)
    long long bt_off32;   // offset of the bt_n FP32 plane records (bt32_stride(bt_P) floats each)
    long long perm_off;   // offset of the plane-order -> row map (nc ints)
};

// Plane records of the block-tridiagonal coarsest solve (16-byte aligned).
// FP64 (FP64 cycles): S_j^-1 stored column by column (element (p, k) at
// k P + p), then the coupling of plane j to plane j-1 (diagonal of A_j, P
// values), then that of plane j to plane j+1 (diagonal of C_j, P values).
// FP32 (FP32 cycles, whose whole cycle runs in FP32 inside the FP64 defect
// correction): S_j^-1 rounded to FP32 row by row with the padded row
// stride bt32_row(P) (zero padding), then A_{j+1} (P values, padded to 4),
// then C_{j-1} (the same), each coupling stored on the plane whose solve
// produces the value it multiplies.
constexpr int kBtriMaxPlane = 64;  // largest plane (cells) in the block form
__host__ __device__ inline int bt_stride(int P) { return (P * P + 2 * P + 1) & ~1; }
__host__ __device__ inline int bt_round4(int P) { return (P + 3) & ~3; }
// a multiple of 4 floats that is 4 mod 8: 128-bit row reads of 8
// consecutive lanes fall into distinct bank groups
__host__ __device__ inline int bt32_row(int P) {
    const int r = bt_round4(P);
    return (r % 8) ? r : r + 4;
}
__host__ __device__ inline int bt32_stride(int P) { return P * bt32_row(P) + 2 * bt_round4(P); }

// Morton code of block coordinates (21 bits each: i at bit 3b, j at 3b+1,
// k at 3b+2), the order of blocks within a level.
__host__ __device__ inline uint64_t morton3(int i, int j, int k) {
    uint64_t c = 0;
    for (int b = 0; b < 21; b++) {
        c |= (uint64_t)((i >> b) & 1) << (3 * b);
        c |= (uint64_t)((j >> b) & 1) << (3 * b + 1);
        c |= (uint64_t)((k >> b) & 1) << (3 * b + 2);
    }
    return c;
}

// Level skeleton of the mesh construction: block size, depth and block grid.
struct LvSkel {
    int n = 0, depth = 0;
    int nblk[3] = {1, 1, 1};
};

// Precomputed FP64 operator coefficients per cell (variable eps or the
// cylindrical form): the 2D face weights, the row diagonal (sum of the
// weights + lambda) and its reciprocal (the Gauss-Seidel divisor, so that
// an FP64 sweep multiplies instead of dividing).
__host__ __device__ constexpr int wstride(int D) { return 2 * D + 2; }

template <class T>
struct Fields {
    T *X = nullptr, *XG = nullptr;   // solution: interior + ghosts
    T *F = nullptr;                  // right-hand side (interior)
    T *E = nullptr, *EG = nullptr;   // coefficient: interior + ghosts (nullptr: eps = 1)
    T *V = nullptr, *VG = nullptr;   // FAS copy v_old: interior + ghosts
    T *W = nullptr;                  // face coefficients, diagonal, 1 / diagonal: wstride(D) per cell ([slot][cell] per block)
    T *J = nullptr;                  // Jacobi scratch (cells), owned by the tree
};

// A level of one tree; in a pool of several trees (a batch), a segment:
// a contiguous block range of one block size at one depth from the top
// ("group"), covered blocks first.
struct LevelHost {
    int n = 0, depth = 0;
    int nblk[3] = {1, 1, 1}, ncell[3] = {1, 1, 1};
    double h[3] = {1, 1, 1};
    int first = 0, nb = 0, nref = 0;
    long long cell_first = 0, ghost_first = 0, ncells = 0, nghost = 0;
    std::vector<double> bc[6];
    int group = 0;      // cycle group (0 = coarsest)
    int coarsest = 0;   // 1: coarsest level of its tree(s), solved exactly
    int parent_same_n = 0;  // 1: every block's parent has the same block size
    int has_cf = 0;         // 1: some block has a refinement face (coarser neighbour)
    std::vector<int> parents;  // segments holding the parents of its blocks
};

}  // namespace mg

struct mg_tree {
    int dim = 3, N = 8, geom = MG_CART, coarse_max = 512;
    mg_bc bc{};
    int base[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    double helm = 0.0;
    std::vector<int32_t> refine;  // 4 per entry
    // wall seconds of the mesh build: mesh tables, device setup, sweep
    // autotuning (FP64, at finalize), phi transfer (a tree made by adapt)
    double build_s[4] = {0, 0, 0, 0};
    bool built = false, finalized = false, singular = false, bc_dirty = false;
    bool var_eps = false;
    std::vector<mg::LevelHost> lev;           // levels (one tree) or segments (batch)
    std::vector<mg::LevelHost> tl;            // batch only: level descriptors per (tree, level)
    std::vector<std::vector<int>> groups;     // segments of each group, coarsest group first
    std::vector<mg::TreeCoarse> tcoarse;      // coarsest level of each tree
    mg::TreeCoarse *d_tcoarse = nullptr;
    int2 *d_coarse_chunks = nullptr;          // (tree, first row) per chunk of the coarse apply
    int n_coarse_chunks = 0;
    int2 *d_bt_chunks = nullptr;              // (tree, first cell) per chunk of the block-form residual
    int n_bt_chunks = 0;
    bool is_batch = false;
    int max_nc = 0;                           // largest coarsest-level system
    // batch only: leaf runs (pool cell, concatenated leaf index, count) for
    // I/O, first leaf of each tree, and the residual slots of each tree
    std::vector<long long> run_cell, run_leaf, run_len, tree_leaf_off;
    long long *d_runs = nullptr;              // run chunks (cell, leaf, length), 3 per chunk
    int n_runs = 0;
    int *d_slot_off = nullptr, *d_slots = nullptr;
    double *d_tree3 = nullptr, *h_tree3 = nullptr;
    std::vector<mg::BlockDesc> blocks;
    long long ncells = 0, nghost = 0, nleaf_cells = 0;

    // device state
    int device = 0;
    cudaStream_t stream = nullptr;
    mg::BlockDesc *d_blocks = nullptr;
    mg::LevelDesc *d_levels = nullptr;
    double *d_bcplanes = nullptr;
    long long n_bcplanes = 0;
    mg::Fields<double> f64, adj;   // solve and adjoint solve (adj shares E/EG)
    mg::Fields<float> f32;         // inner defect-correction cycles
    double *d_r64 = nullptr;       // leaf residual scratch (FP64)
    double *d_wface = nullptr;     // FP64 face coefficients (variable eps or cylindrical form)
    double *d_jac64 = nullptr;     // Jacobi scratch, FP64 and FP32 cycles
    float *d_jac32 = nullptr;
    int smoother = MG_SMOOTH_RBGS; // of the current call (mg_params)
    int coarse_mode = MG_COARSE_EXACT;  // coarsest-level solve of the current call
    int coarse_max_it = 1000;
    double coarse_abs = 1e-8, coarse_rel = 1e-8;
    int coarse_pad = 0;            // padded cells of the largest coarsest level (smoothing mode)
    double omega = 0.8;            // Jacobi weight of the current call
    double *d_minv = nullptr;      // coarsest-level inverses, row-major ns x ns per tree
    long long minv_total = 0, cvec_total = 0;
    int build_where = 0;           // mesh tables: 0 device when present, 1 host, 2 device (mg_tree_build_on)
    bool built_on_device = false;
    mg::BlockDesc *d_blocks_built = nullptr;  // block table left on the device by the device build
    double *d_bt = nullptr;        // plane records of the block-tridiagonal trees (FP64)
    float *d_bt32 = nullptr;       // the same rounded to FP32 (FP32 cycles)
    int *d_btperm = nullptr;       // their plane-order -> row maps
    int *d_btlist = nullptr;       // indices of the block-tridiagonal trees
    long long bt_total = 0, bt_total32 = 0, btperm_total = 0;
    int n_btri = 0, bt_pmax = 0, bt_ncmax = 0;
    int nc = 0, ns = 0;            // coarsest cells, system size (nc + singular) -- one tree
    bool minv_ok = false;
    double *d_cvec = nullptr;      // coarsest residual vector (ns)
    double *d_partials = nullptr;  // per-CTA norm partials (3 per CTA)
    int n_partials = 0;
    double *d_red = nullptr;       // reduced norms (3)
    double *h_red = nullptr;       // pinned host copy
    long long launches = 0;        // kernels launched so far
    int *d_status = nullptr;       // device status word (0 = ok), then the tail kernel's grid-barrier
                                   // counter and generation (kStatusWords ints, cleared together)
    uint32_t wait_limit = mg::kDefaultWaitLimit;  // bounded-wait polls (mg_set_wait_limit)
    // adjoint (mg_adjoint.cu): adjoint of every pool value (cells, ghosts),
    // lambda, the compatible right-hand side and a leaf-order scratch
    double *d_at = nullptr, *d_atg = nullptr, *d_lam = nullptr, *d_gh = nullptr, *d_lv = nullptr;
    int nsm = 0;                   // multiprocessors of the device
    // CUDA graphs of whole cycle sequences, keyed by what they enqueue; a
    // private non-blocking stream is used for capture (the user stream may
    // be the legacy default stream, which cannot be captured)
    struct Graph {
        cudaGraphExec_t exec;
        long long launches;
    };
    std::map<std::string, Graph> graphs;
    cudaStream_t cap_stream = nullptr;
    bool use_graphs = true;
    std::vector<int> sweep_choice[2];  // autotuned sweep variant per level (FP64, FP32); -1 default
    // the tail kernel (mg_kernels.cu): cell bound of the groups it runs
    // (0: off, the default; mg_set_tail) and the program being recorded (a
    // Launch<T, D>::TailRec while a cycle records, else null)
    long long tail_cells = 0;
    void *tail_rec = nullptr;
    // smoothing steps per level (mg_set_schedule / mg_tune_schedule); an
    // entry < 0, or no entry, takes the cycle's n_down / n_up
    std::vector<int> sched_down, sched_up;
    std::string sched_key;             // graph-key suffix of the schedule
    // a tree made by adapt: sweep variants by level depth taken over from the
    // old tree instead of autotuning (per precision; empty: tune)
    std::map<int, int> tune_hint[2];
};

namespace mg {
// mesh construction (mg_tree.cpp, mg_build.cu)
std::vector<LvSkel> level_skeleton(const mg_tree *t, int maxdepth);
int max_refine_depth(const mg_tree *t);
void fill_levels(mg_tree *t, const std::vector<LvSkel> &lv, const std::vector<int> &nb, const std::vector<int> &nref);
int build_tables_device(mg_tree *t);
// cycle driver and kernels (mg_kernels.cu); all enqueue on t->stream
template <class T> void vcycle(mg_tree *t, Fields<T> &F, int top, int nd, int nu, int homog);
template <class T> void fmg(mg_tree *t, Fields<T> &F, int nd, int nu, int homog);
template <class T> void refresh(mg_tree *t, Fields<T> &F, int homog);
template <class T> void refresh_eps(mg_tree *t, Fields<T> &F);
template <class T> void tune_sweeps(mg_tree *t, Fields<T> &F);
int sweep_variant(mg_tree *t, int prec, int level);
constexpr int kNumSweepVariants = 11;
constexpr int kCoarseRows = 8;  // rows of one tree per CTA of the coarse apply
constexpr int kBtResidCells = 256;  // cells per CTA of the block-form coarsest residual
bool sweep_variant_ok(mg_tree *t, int prec, int level, int variant);
void divergence(mg_tree *t, const double *B, double *out, int order);
void project(mg_tree *t, const double *B, double *Bout);
// composite residual of FP64 fields on the leaves; optional outputs:
// r64 (FP64 leaf order), f32 (FP32 into the leaf cells of an FP32 field)
void residual_norm(mg_tree *t, Fields<double> &F, int homog, double *out3, double *r64_leaf,
                   float *f32_cells);
// want_max: also the max norm (solve loops read only the L2 norm); e_add:
// first apply the defect-correction update phi += e on the leaves (fused
// into the refresh before the residual)
void residual_enqueue(mg_tree *t, Fields<double> &F, int homog, double *r64_leaf, float *f32_cells,
                      bool want_max = false, const float *e_add = nullptr);
void residual_wait(mg_tree *t, double *out3);
// volume-weighted mean of a leaf-order FP64 field (synchronises the stream)
double leaf_mean(mg_tree *t, const double *rleaf);
void sub_scalar(mg_tree *t, double *x, double c, long long n);  // x[0..n) -= c
// phi of old carried to the leaf blocks nid of the adapted mesh nt (see k_transfer)
int transfer_phi(mg_tree *old, mg_tree *nt, const std::vector<int> &nid, const std::vector<int> &src);
void copy_eps_to_f32(mg_tree *t);
// whole-field copies FP64 -> FP32 (rounded to nearest) and FP32 -> FP64 (exact)
void narrow_f32(mg_tree *t, const double *a, float *b, long long n);
void widen_f64(mg_tree *t, const float *a, double *b, long long n);
// FP64 face coefficients of every cell into t->d_wface (eps ghosts current)
void face_coef(mg_tree *t);
KParams kparams(mg_tree *t, int homog);
int time_sweeps(mg_tree *t, int level, int n_sweeps, int prec, double *out4);
// batch: per-tree composite residual sums (3 per tree, on the host after wait)
void residual_enqueue_trees(mg_tree *t, Fields<double> &F, float *f32_cells, bool want_max,
                            const float *e_add = nullptr);
// copies between a concatenated per-tree leaf array and the pool cells
void leaf_runs_copy(mg_tree *t, double *cells, const double *leaf, bool to_cells);
int check_cuda(const char *what);
std::string take_launch_error();  // first failed kernel launch since the last check ("" if none), cleared
// transposed operators and the adjoint solve (mg_adjoint.cu); leaf-order
// device vectors
int adjoint_buffers(mg_tree *t);
void apply_transpose(mg_tree *t, const double *y, double *out);
void eps_grad_transpose(mg_tree *t, const double *lam, double *out);
// fp32: FP32 V-cycles (the tree's FP32 set, allocated) as the approximate
// inverse inside the FP64 defect correction, else FP64 V-cycles
int adjoint_dc(mg_tree *t, const double *g, double *lam, int nd, int nu, double rel_tol, int max_it, int *it_out,
               double *rel_out, bool fp32 = false);
int clean_adjoint(mg_tree *t, const double *gBn, double *gB, int nd, int nu, double rel_tol, int max_it,
                  int *it_out, double *rel_out, bool fp32 = false);
}  // namespace mg

void mg_set_error(const std::string &msg);
