/*
 * mg_oracle.c -- plain, slow FP64 reference of the quadtree/octree geometric
 * multigrid of Teunissen & Keppens, "A geometric multigrid library for
 * quadtree/octree AMR grids coupled to MPI-AMRVAC" (arXiv:1901.11370).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The CUDA product
 * path neither links nor calls it, and this file shares no code with it.
 *
 * Layout (the paper's own, Sec. 2.6): every block stores its N^D cells plus
 * one ghost layer, padded to (N+2)^D, face ghosts only (edge and corner
 * ghosts are never written or read).  Everything is FP64 and written as
 * plain loops in the order the paper states the algorithm.
 *
 * Readings where the paper is silent or ambiguous (each one is listed in the
 * design notes):
 *  R1  ghost cells are refreshed after every colour of a red-black sweep,
 *      physical-boundary ghosts included (lagged, not folded into the
 *      diagonal) -- Sec. 2.4 last paragraph, Sec. 2.6 last paragraph;
 *  R2  red/black parity uses global level indices (I+J+K) -- Sec. 2.2;
 *  R3  refinement-boundary ghost g = (B' + c')/2 with
 *      B' = B + sum_t s_t (C_t - A_t)/8 and c' = (3c - d)/2 -- Sec. 2.6;
 *  R4  eps on coarse levels is the mean of the children; eps ghosts are
 *      copied across same-level faces, equal the interior value at physical
 *      faces and the coarse value B at refinement faces;
 *  R5  cylindrical (r,z) finite-volume form with r-face weights r_f/r_i and
 *      zero flux through the axis; restriction stays the plain mean;
 *  R6  coarse levels follow the construction rule of Sec. 2.5: halve the
 *      block count while every count is even; after that halve the block
 *      size while the level holds more than `coarse_max` cells; that level is
 *      solved exactly by dense LU (bordered by a zero-mean constraint when
 *      the problem has no Dirichlet face);
 *  R7  FMG: restrict solution and FAS right-hand side to the coarsest level,
 *      solve, then for each finer level prolong the correction and run one
 *      V-cycle topped at that level -- Sec. 2.4 and its figure caption;
 *  R8  residual norm: composite residual on leaf cells after restricting
 *      covered cells bottom-up, volume-weighted L2 and max norm;
 *  R14 the fourth-order divergence (Sec. 4.1) uses the fourth-order
 *      difference along a dimension only where both cells two away are
 *      same-level cells; elsewhere (beside physical and refinement faces,
 *      the grid having one ghost layer) the second-order difference;
 *  R13 the optional Jacobi smoother (the one the paper's scaling runs use,
 *      Sec. 3.3; its weight is not stated) is weighted Jacobi over every
 *      cell of the level, x <- x + omega (x_GS - x) with x_GS the local
 *      solution from the old values, then a ghost refresh; omega defaults
 *      to the standard smoothing weight of the 5/7-point Laplacian, 4/5 in
 *      2D and 6/7 in 3D;
 *  R16 the adjoint on refined meshes uses the exact transpose of the
 *      composite operator: the forward steps (restriction of covered cells,
 *      ghost fills, stencil) undone in reverse order with transposed
 *      coefficients; A is not symmetric at refinement faces (Sec. 2.6);
 *  R20 the paper's coarse-grid solve (Sec. 2.4) is red-black smoothing of
 *      the coarsest level until max |r| meets an absolute or relative
 *      threshold or N_max sweeps; the max norm is this oracle's reading;
 *  R15 phi carried to an adapted mesh (Sec. 2.5 leaves the data to the
 *      caller): a leaf block that is also a block of the old mesh keeps its
 *      values (the restriction of its former children where a refinement
 *      was removed), a new child takes the prolongation of Sec. 2.3 of its
 *      old parent leaf, parent ghost layer included.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { GEOM_CART = 0, GEOM_CYL = 1 };
enum { BC_DIR = 0, BC_NEU = 1, BC_PER = 2, BC_AXIS = 3 };
enum { F_PHI = 0, F_EPS = 1, F_LAM = 2, F_VEC = 3 };

typedef struct {
    int n;        /* cells per block edge */
    int depth;    /* 0 = base grid, < 0 added coarse levels, > 0 refined */
    int nblk[3];  /* blocks per dimension over the whole domain */
    int ncell[3]; /* cells per dimension over the whole domain */
    double h[3];
    int nb;
    int *ijk;     /* [nb][3] block coordinates */
    int *map;     /* dense block-coordinate -> block index (or -1) */
    int *parent;  /* [nb] block index at the next coarser level */
    int *poff;    /* [nb][3] offset of this block inside its parent, parent cells */
    int *haschild;/* [nb] 1 if covered by finer blocks */
    double *phi, *f, *eps, *vold, *tmp, *lam;
    double *adj;  /* adjoint of every padded value (transposed operators) */
    double *bc[6];
} Lev;

typedef struct {
    int dim, N, geom, bct[6];
    double bcv[6];
    int base[3];
    double lo[3], hi[3];
    double helm;
    int nlev;
    Lev *L;
    int homog; /* 1: physical boundary values treated as zero */
    int n_down, n_up;
    int *sched;     /* optional per-level steps: sched[2l] down, sched[2l+1] up (< 0: n_down / n_up) */
    int smoother;   /* 0 red-black Gauss-Seidel, 1 weighted Jacobi (R13) */
    double omega;   /* Jacobi weight */
    /* coarsest-level dense factorisation */
    int nc, nsys, singular, lu_ok;
    /* coarsest-level solve: 0 exact (dense LU), 1 smoothing as in Sec. 2.4
     * (reading R20): up to coarse_max_it sweeps until max |r| is at most
     * coarse_abs or coarse_rel times its value before the first sweep */
    int coarse_mode, coarse_max_it;
    double coarse_abs, coarse_rel;
    double *lu;
    int *piv;
} Tree;

static char g_err[512];
const char *or_last_error(void) { return g_err; }

/* ------------------------------------------------------------ indexing -- */

static int P(const Tree *T, int n) { return T->dim == 2 ? (n + 2) * (n + 2) : (n + 2) * (n + 2) * (n + 2); }
static int C(const Tree *T, int n) { return T->dim == 2 ? n * n : n * n * n; }
static int pidx(const Tree *T, int n, int i, int j, int k) {
    if (T->dim == 2) return (j + 1) * (n + 2) + (i + 1);
    return ((k + 1) * (n + 2) + (j + 1)) * (n + 2) + (i + 1);
}
static double *fld(Lev *lv, int which) {
    return which == F_PHI ? lv->phi : which == F_EPS ? lv->eps : lv->lam;  /* F_VEC uses lam storage */
}
static int mapidx(const Lev *lv, const int *q) {
    return (q[2] * lv->nblk[1] + q[1]) * lv->nblk[0] + q[0];
}
static int lookup(const Lev *lv, const int *q) {
    for (int d = 0; d < 3; d++)
        if (q[d] < 0 || q[d] >= lv->nblk[d]) return -1;
    return lv->map[mapidx(lv, q)];
}
static uint64_t morton(const int *q) {
    uint64_t c = 0;
    for (int b = 0; b < 21; b++) {
        c |= (uint64_t)((q[0] >> b) & 1) << (3 * b);
        c |= (uint64_t)((q[1] >> b) & 1) << (3 * b + 1);
        c |= (uint64_t)((q[2] >> b) & 1) << (3 * b + 2);
    }
    return c;
}

/* ---------------------------------------------------- mesh construction -- */

typedef struct { uint64_t key; int idx; } keyed;
static int cmp_keyed(const void *a, const void *b) {
    uint64_t x = ((const keyed *)a)->key, y = ((const keyed *)b)->key;
    return x < y ? -1 : x > y ? 1 : 0;
}

static int alloc_level(Tree *T, Lev *lv, int nb, const int *ijk) {
    lv->nb = nb;
    size_t nmap = (size_t)lv->nblk[0] * lv->nblk[1] * lv->nblk[2];
    lv->ijk = malloc(sizeof(int) * 3 * (nb ? nb : 1));
    lv->map = malloc(sizeof(int) * nmap);
    lv->parent = malloc(sizeof(int) * (nb ? nb : 1));
    lv->poff = calloc(3 * (nb ? nb : 1), sizeof(int));
    lv->haschild = calloc(nb ? nb : 1, sizeof(int));
    /* Morton-sort the blocks: leaf I/O order is depth, then Morton code */
    keyed *ks = malloc(sizeof(keyed) * (nb ? nb : 1));
    for (int b = 0; b < nb; b++) { ks[b].key = morton(ijk + 3 * b); ks[b].idx = b; }
    qsort(ks, nb, sizeof(keyed), cmp_keyed); /* codes are distinct */
    for (size_t m = 0; m < nmap; m++) lv->map[m] = -1;
    for (int b = 0; b < nb; b++) {
        memcpy(lv->ijk + 3 * b, ijk + 3 * ks[b].idx, sizeof(int) * 3);
        lv->map[mapidx(lv, lv->ijk + 3 * b)] = b;
    }
    free(ks);
    size_t np = (size_t)nb * P(T, lv->n);
    lv->phi = calloc(np ? np : 1, sizeof(double));
    lv->f = calloc(np ? np : 1, sizeof(double));
    lv->eps = calloc(np ? np : 1, sizeof(double));
    lv->vold = calloc(np ? np : 1, sizeof(double));
    lv->tmp = calloc(np ? np : 1, sizeof(double));
    lv->lam = calloc(np ? np : 1, sizeof(double));
    lv->adj = calloc(np ? np : 1, sizeof(double));
    for (size_t m = 0; m < np; m++) lv->eps[m] = 1.0;
    for (int s = 0; s < 6; s++) lv->bc[s] = NULL;
    return 0;
}

static void free_level(Lev *lv) {
    free(lv->ijk); free(lv->map); free(lv->parent); free(lv->poff); free(lv->haschild);
    free(lv->phi); free(lv->f); free(lv->eps); free(lv->vold); free(lv->tmp); free(lv->lam); free(lv->adj);
    for (int s = 0; s < 6; s++) free(lv->bc[s]);
}

void or_destroy(void *h) {
    Tree *T = h;
    if (!T) return;
    for (int l = 0; l < T->nlev; l++) free_level(&T->L[l]);
    free(T->L); free(T->lu); free(T->piv); free(T->sched); free(T);
}

static void ghost_fill(Tree *T, int l, int which);
static void refresh(Tree *T);

/*
 * Builds the level hierarchy: the base grid (depth 0), the added coarse
 * levels (Sec. 2.5, "Construction of additional coarse grids" and its table)
 * and the refined levels listed in `refine` (entries depth,i,j,k; each
 * covers that block by 2^D children, Sec. 2.5).  2:1 balance across faces is
 * checked, not imposed (Sec. 2.7: the library assumes it).
 */
void *or_create(int dim, int N, int geom, const int *bct, const double *bcv,
                const int *base, const double *lo, const double *hi, int coarse_max,
                double helm, int n_refine, const int *refine) {
    g_err[0] = 0;
    if ((dim != 2 && dim != 3) || N < 1 || (geom == GEOM_CYL && dim != 2)) {
        snprintf(g_err, sizeof g_err, "bad dim/N/geometry"); return NULL;
    }
    int nb0[3] = {1, 1, 1};
    for (int d = 0; d < dim; d++) {
        if (base[d] % N) { snprintf(g_err, sizeof g_err, "base not divisible by N"); return NULL; }
        nb0[d] = base[d] / N;
    }
    for (int d = 0; d < dim; d++) {
        int per0 = bct[2 * d] == BC_PER, per1 = bct[2 * d + 1] == BC_PER;
        if (per0 != per1) { snprintf(g_err, sizeof g_err, "periodic faces must pair"); return NULL; }
    }
    Tree *T = calloc(1, sizeof(Tree));
    T->dim = dim; T->N = N; T->geom = geom; T->helm = helm;
    memcpy(T->bct, bct, sizeof(int) * 6); memcpy(T->bcv, bcv, sizeof(double) * 6);
    for (int d = 0; d < 3; d++) { T->base[d] = d < dim ? base[d] : 1; T->lo[d] = lo[d]; T->hi[d] = hi[d]; }
    T->n_down = 2; T->n_up = 2;
    T->smoother = 0; T->omega = dim == 2 ? 0.8 : 6.0 / 7.0;

    /* coarse levels: list of (n, nblk) from the base downwards */
    int cn[64], cb[64][3], nco = 0;
    {
        int n = N, b[3] = {nb0[0], nb0[1], nb0[2]};
        for (;;) {
            long cells = 1;
            for (int d = 0; d < dim; d++) cells *= (long)n * b[d];
            int alleven = 1;
            for (int d = 0; d < dim; d++) if (b[d] % 2) alleven = 0;
            if (alleven) { for (int d = 0; d < dim; d++) b[d] /= 2; }
            else if (cells > coarse_max && n % 2 == 0) n /= 2;
            else break;
            cn[nco] = n; memcpy(cb[nco], b, sizeof b); nco++;
            if (nco >= 60) break;
        }
    }
    int maxdepth = -1;
    for (int e = 0; e < n_refine; e++) if (refine[4 * e] > maxdepth) maxdepth = refine[4 * e];
    T->nlev = nco + 1 + (maxdepth + 1);
    T->L = calloc(T->nlev, sizeof(Lev));
    int ibase = nco;
    /* coarse levels (index 0 = coarsest) */
    for (int c = 0; c < nco; c++) {
        Lev *lv = &T->L[ibase - 1 - c];
        lv->n = cn[c]; lv->depth = -(c + 1);
        for (int d = 0; d < 3; d++) lv->nblk[d] = d < dim ? cb[c][d] : 1;
    }
    for (int l = 0; l <= ibase; l++) {
        Lev *lv = &T->L[l];
        if (l == ibase) { lv->n = N; lv->depth = 0; for (int d = 0; d < 3; d++) lv->nblk[d] = nb0[d]; }
        int nb = lv->nblk[0] * lv->nblk[1] * lv->nblk[2];
        int *ijk = malloc(sizeof(int) * 3 * nb);
        int m = 0;
        for (int k = 0; k < lv->nblk[2]; k++)
            for (int j = 0; j < lv->nblk[1]; j++)
                for (int i = 0; i < lv->nblk[0]; i++) { ijk[3 * m] = i; ijk[3 * m + 1] = j; ijk[3 * m + 2] = k; m++; }
        alloc_level(T, lv, nb, ijk);
        free(ijk);
    }
    /* refined levels */
    for (int r = 0; r <= maxdepth; r++) {
        Lev *pl = &T->L[ibase + r], *lv = &T->L[ibase + r + 1];
        lv->n = N; lv->depth = r + 1;
        for (int d = 0; d < 3; d++) lv->nblk[d] = d < dim ? 2 * pl->nblk[d] : 1;
        int cap = 16, nb = 0;
        int *ijk = malloc(sizeof(int) * 3 * cap);
        for (int e = 0; e < n_refine; e++) {
            if (refine[4 * e] != r) continue;
            int q[3] = {refine[4 * e + 1], refine[4 * e + 2], dim == 3 ? refine[4 * e + 3] : 0};
            int pb = lookup(pl, q);
            if (pb < 0) { snprintf(g_err, sizeof g_err, "refined block does not exist"); free(ijk); or_destroy(T); return NULL; }
            if (pl->haschild[pb]) continue;
            pl->haschild[pb] = 1;
            for (int c = 0; c < (1 << dim); c++) {
                if (nb == cap) { cap *= 2; ijk = realloc(ijk, sizeof(int) * 3 * cap); }
                ijk[3 * nb] = 2 * q[0] + (c & 1);
                ijk[3 * nb + 1] = 2 * q[1] + ((c >> 1) & 1);
                ijk[3 * nb + 2] = dim == 3 ? 2 * q[2] + ((c >> 2) & 1) : 0;
                nb++;
            }
        }
        alloc_level(T, lv, nb, ijk);
        free(ijk);
    }
    /* cell counts and sizes */
    for (int l = 0; l < T->nlev; l++) {
        Lev *lv = &T->L[l];
        for (int d = 0; d < 3; d++) {
            lv->ncell[d] = d < dim ? lv->n * lv->nblk[d] : 1;
            lv->h[d] = d < dim ? (hi[d] - lo[d]) / lv->ncell[d] : 1.0;
        }
    }
    /* parents: same block size => parent coords are halved and the block
     * fills one 2^-D part of the parent; halved block size => one child
     * covers its parent entirely */
    for (int l = 0; l < T->nlev; l++) {
        Lev *lv = &T->L[l];
        for (int b = 0; b < lv->nb; b++) lv->parent[b] = -1;
        if (l == 0) continue;
        Lev *pl = &T->L[l - 1];
        int same = pl->n == lv->n;
        for (int b = 0; b < lv->nb; b++) {
            int q[3], *bi = lv->ijk + 3 * b;
            for (int d = 0; d < 3; d++) {
                q[d] = d < dim ? (same ? bi[d] / 2 : bi[d]) : 0;
                lv->poff[3 * b + d] = d < dim ? (same ? (bi[d] % 2) * (lv->n / 2) : 0) : 0;
            }
            int pb = lookup(pl, q);
            if (pb < 0) { snprintf(g_err, sizeof g_err, "missing parent"); or_destroy(T); return NULL; }
            lv->parent[b] = pb;
            pl->haschild[pb] = 1;
        }
    }
    /* face 2:1 balance: the region beside every refined block must exist one
     * level coarser */
    for (int l = ibase + 1; l < T->nlev; l++) {
        Lev *lv = &T->L[l], *pl = &T->L[l - 1];
        for (int b = 0; b < lv->nb; b++)
            for (int d = 0; d < dim; d++)
                for (int s = 0; s < 2; s++) {
                    int q[3] = {lv->ijk[3 * b], lv->ijk[3 * b + 1], lv->ijk[3 * b + 2]};
                    q[d] += s ? 1 : -1;
                    if (q[d] < 0 || q[d] >= lv->nblk[d]) {
                        if (T->bct[2 * d + s] != BC_PER) continue;
                        q[d] = (q[d] + lv->nblk[d]) % lv->nblk[d];
                    }
                    if (lookup(lv, q) >= 0) continue;
                    int pq[3];
                    for (int e = 0; e < 3; e++) pq[e] = e < dim ? q[e] / 2 : 0;
                    if (lookup(pl, pq) < 0) {
                        snprintf(g_err, sizeof g_err, "mesh is not 2:1 balanced");
                        or_destroy(T); return NULL;
                    }
                }
    }
    T->singular = 1;
    for (int s = 0; s < 2 * dim; s++) if (bct[s] == BC_DIR) T->singular = 0;
    if (helm > 0) T->singular = 0;
    refresh(T);
    return T;
}

int or_num_levels(void *h) { return ((Tree *)h)->nlev; }
int or_level_info(void *h, int l, int *out /* n, depth, nb, nblk[3], ncell[3] */, double *hh) {
    Tree *T = h; Lev *lv = &T->L[l];
    out[0] = lv->n; out[1] = lv->depth; out[2] = lv->nb;
    for (int d = 0; d < 3; d++) { out[3 + d] = lv->nblk[d]; out[6 + d] = lv->ncell[d]; hh[d] = lv->h[d]; }
    return 0;
}
void or_set_cycle(void *h, int n_down, int n_up) { Tree *T = h; T->n_down = n_down; T->n_up = n_up; }
/* N_down / N_up of Sec. 2.4 chosen per level: down[l], up[l] for levels
 * 0..n-1 (values < 0 keep or_set_cycle's); n = 0 clears the schedule */
void or_set_schedule(void *h, int n, const int *down, const int *up) {
    Tree *T = h;
    free(T->sched);
    T->sched = NULL;
    if (n <= 0) return;
    T->sched = malloc(sizeof(int) * 2 * T->nlev);
    for (int l = 0; l < T->nlev; l++) {
        T->sched[2 * l] = l < n ? down[l] : -1;
        T->sched[2 * l + 1] = l < n ? up[l] : -1;
    }
}
static int steps(const Tree *T, int l, int up) {
    int v = T->sched ? T->sched[2 * l + up] : -1;
    return v >= 0 ? v : (up ? T->n_up : T->n_down);
}
/* smoother 0: red-black Gauss-Seidel; 1: weighted Jacobi with weight omega
 * (omega <= 0: 4/5 in 2D, 6/7 in 3D) -- reading R13 */
void or_set_smoother(void *h, int smoother, double omega) {
    Tree *T = h;
    T->smoother = smoother;
    T->omega = omega > 0 ? omega : (T->dim == 2 ? 0.8 : 6.0 / 7.0);
}
void or_set_homogeneous(void *h, int on) { ((Tree *)h)->homog = on; }

/* --------------------------------------------------------- geometry ----- */

static void cell_global(const Lev *lv, int b, int i, int j, int k, int *G) {
    G[0] = lv->ijk[3 * b] * lv->n + i;
    G[1] = lv->ijk[3 * b + 1] * lv->n + j;
    G[2] = lv->ijk[3 * b + 2] * lv->n + k;
}
static double cell_volume(const Tree *T, const Lev *lv, const int *G) {
    if (T->geom == GEOM_CYL) {
        double r = T->lo[0] + (G[0] + 0.5) * lv->h[0];
        return 2.0 * M_PI * r * lv->h[0] * lv->h[1];
    }
    double v = 1.0;
    for (int d = 0; d < T->dim; d++) v *= lv->h[d];
    return v;
}

/* ----------------------------------------------------- ghost cells ------ */

/* boundary value a (Dirichlet) or b (Neumann) at a face cell */
static double bc_value(const Tree *T, const Lev *lv, int face, const int *G) {
    if (T->homog) return 0.0;
    if (!lv->bc[face]) return T->bcv[face];
    int d = face / 2, t1 = -1, t2 = -1;
    for (int t = 0; t < T->dim; t++) if (t != d) { if (t1 < 0) t1 = t; else t2 = t; }
    int idx = G[t1];
    if (t2 >= 0) idx += lv->ncell[t1] * G[t2];
    return lv->bc[face][idx];
}

/*
 * Fill the face ghost cells of every block of level l for one field
 * (Sec. 2.6): a copy from a same-level (or periodic) neighbour; the
 * physical-boundary formulas phi_g = 2a - phi_i (Dirichlet) and
 * phi_g = phi_i -/+ h b (Neumann, low/high face); or, beside a coarser
 * block, the refinement-boundary scheme of reading R3.  Level l-1 must
 * have current ghosts.
 */
static void ghost_fill(Tree *T, int l, int which) {
    Lev *lv = &T->L[l];
    int n = lv->n, dim = T->dim, ps = P(T, n);
    double *X = fld(lv, which);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < lv->nb; b++) {
        double *xb = X + (size_t)b * ps;
        for (int d = 0; d < dim; d++)
            for (int s = 0; s < 2; s++) {
                int face = 2 * d + s;
                int q[3] = {lv->ijk[3 * b], lv->ijk[3 * b + 1], lv->ijk[3 * b + 2]};
                q[d] += s ? 1 : -1;
                int phys = 0;
                if (q[d] < 0 || q[d] >= lv->nblk[d]) {
                    if (T->bct[face] == BC_PER) q[d] = (q[d] + lv->nblk[d]) % lv->nblk[d];
                    else phys = 1;
                }
                int nbk = phys ? -1 : lookup(lv, q);
                /* loop over the tangential cells of the face */
                int tdim[2] = {-1, -1}, nt = 0;
                for (int t = 0; t < dim; t++) if (t != d) tdim[nt++] = t;
                int n1 = n, n2 = nt > 1 ? n : 1;
                for (int u2 = 0; u2 < n2; u2++)
                    for (int u1 = 0; u1 < n1; u1++) {
                        int gi[3] = {0, 0, 0}, ii[3] = {0, 0, 0};
                        gi[tdim[0]] = u1; if (nt > 1) gi[tdim[1]] = u2;
                        memcpy(ii, gi, sizeof ii);
                        gi[d] = s ? n : -1;       /* ghost cell */
                        ii[d] = s ? n - 1 : 0;    /* adjacent interior cell */
                        double *g = xb + pidx(T, n, gi[0], gi[1], gi[2]);
                        double xi = xb[pidx(T, n, ii[0], ii[1], ii[2])];
                        if (phys) {
                            int G[3]; cell_global(lv, b, ii[0], ii[1], ii[2], G);
                            if (which == F_EPS || which == F_VEC) { *g = xi; continue; }
                            int hom = T->homog || which == F_LAM;
                            double v = hom ? 0.0 : bc_value(T, lv, face, G);
                            switch (T->bct[face]) {
                            case BC_DIR: *g = 2.0 * v - xi; break;
                            case BC_NEU: *g = s ? xi + lv->h[d] * v : xi - lv->h[d] * v; break;
                            default: *g = xi; break; /* axis: zero flux, value mirrored */
                            }
                        } else if (nbk >= 0) {
                            int jj[3]; memcpy(jj, gi, sizeof jj);
                            jj[d] = s ? 0 : n - 1;
                            *g = X[(size_t)nbk * ps + pidx(T, n, jj[0], jj[1], jj[2])];
                        } else {
                            /* refinement boundary: coarse neighbour one level down */
                            Lev *cl = &T->L[l - 1];
                            double *CX = fld(cl, which);
                            int G[3]; cell_global(lv, b, gi[0], gi[1], gi[2], G);
                            if (G[d] < 0) G[d] += lv->ncell[d];
                            if (G[d] >= lv->ncell[d]) G[d] -= lv->ncell[d];
                            int Gc[3] = {G[0] / 2, G[1] / 2, G[2] / 2};
                            int cq[3], nc = cl->n;
                            for (int e = 0; e < 3; e++) cq[e] = e < dim ? Gc[e] / nc : 0;
                            int cb = lookup(cl, cq);
                            double *cx = CX + (size_t)cb * P(T, nc);
                            int lc[3];
                            for (int e = 0; e < 3; e++) lc[e] = e < dim ? Gc[e] - cq[e] * nc : 0;
                            double B = cx[pidx(T, nc, lc[0], lc[1], lc[2])];
                            if (which == F_EPS) { *g = B; continue; }
                            double Bp = B;
                            for (int a = 0; a < nt; a++) {
                                int t = tdim[a];
                                double sg = (G[t] & 1) ? 1.0 : -1.0;
                                int la[3], lcc[3];
                                memcpy(la, lc, sizeof la); memcpy(lcc, lc, sizeof lcc);
                                la[t] -= 1; lcc[t] += 1;
                                double A = cx[pidx(T, nc, la[0], la[1], la[2])];
                                double Cc = cx[pidx(T, nc, lcc[0], lcc[1], lcc[2])];
                                Bp += sg * (Cc - A) / 8.0;
                            }
                            int dd[3]; memcpy(dd, ii, sizeof dd);
                            dd[d] = s ? n - 2 : 1;
                            double c = xi, dv = xb[pidx(T, n, dd[0], dd[1], dd[2])];
                            *g = 0.5 * Bp + 0.75 * c - 0.25 * dv;
                        }
                    }
            }
    }
}

/* ---------------------------------------------------------- operator ---- */

/*
 * Row weights of the 5/7-point operator at a cell (Sec. 2.2, eqs. for the
 * constant- and variable-coefficient Poisson operator): for every face the
 * weight w_f = eps_f * kappa_f / h_d^2 multiplying (phi_nb - phi_i), with
 * eps_f the harmonic mean of the two cell coefficients and kappa_f = r_f/r_i
 * for the r-faces of the cylindrical form (reading R5), else 1.
 */
static void face_weights(const Tree *T, const Lev *lv, int b, int i, int j, int k, double *w) {
    int n = lv->n, ps = P(T, n);
    const double *E = lv->eps + (size_t)b * ps;
    int c = pidx(T, n, i, j, k);
    int G[3]; cell_global(lv, b, i, j, k, G);
    for (int d = 0; d < T->dim; d++)
        for (int s = 0; s < 2; s++) {
            int q[3] = {i, j, k};
            q[d] += s ? 1 : -1;
            double e0 = E[c], e1 = E[pidx(T, n, q[0], q[1], q[2])];
            double ef = 2.0 * e0 * e1 / (e0 + e1);
            double kap = 1.0;
            if (T->geom == GEOM_CYL && d == 0) {
                double ri = T->lo[0] + (G[0] + 0.5) * lv->h[0];
                double rf = T->lo[0] + (G[0] + s) * lv->h[0];
                kap = rf / ri;
            }
            w[2 * d + s] = ef * kap / (lv->h[d] * lv->h[d]);
        }
}

static double apply_L(const Tree *T, const Lev *lv, const double *X, int b, int i, int j, int k) {
    int n = lv->n, ps = P(T, n);
    const double *x = X + (size_t)b * ps;
    double w[6], sum = 0.0;
    face_weights(T, lv, b, i, j, k, w);
    double xc = x[pidx(T, n, i, j, k)];
    for (int d = 0; d < T->dim; d++)
        for (int s = 0; s < 2; s++) {
            int q[3] = {i, j, k};
            q[d] += s ? 1 : -1;
            sum += w[2 * d + s] * (x[pidx(T, n, q[0], q[1], q[2])] - xc);
        }
    return sum - T->helm * xc;
}

/* ----------------------------------------------------------- smoother --- */

/*
 * One colour of a red-black Gauss-Seidel sweep (Sec. 2.2): every cell with
 * (I+J+K) % 2 == colour is replaced by the local solution with its
 * neighbours held fixed; ghosts are refreshed afterwards (reading R1).
 */
static void smooth_colour(Tree *T, int l, int colour) {
    Lev *lv = &T->L[l];
    int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
#pragma omp parallel for schedule(static)
    for (int b = 0; b < lv->nb; b++) {
        double *x = lv->phi + (size_t)b * ps, *f = lv->f + (size_t)b * ps;
        for (int k = 0; k < nk; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    int G[3]; cell_global(lv, b, i, j, k, G);
                    if (((G[0] + G[1] + G[2]) & 1) != colour) continue;
                    double w[6], num = 0.0, den = 0.0;
                    face_weights(T, lv, b, i, j, k, w);
                    for (int d = 0; d < T->dim; d++)
                        for (int s = 0; s < 2; s++) {
                            int q[3] = {i, j, k};
                            q[d] += s ? 1 : -1;
                            num += w[2 * d + s] * x[pidx(T, n, q[0], q[1], q[2])];
                            den += w[2 * d + s];
                        }
                    int c = pidx(T, n, i, j, k);
                    x[c] = (num - f[c]) / (den + T->helm);
                }
    }
    ghost_fill(T, l, F_PHI);
}

/*
 * One weighted-Jacobi step (reading R13): every cell of the level takes
 * x + omega (x_GS - x), x_GS the local solution computed from the values
 * before the step (ghosts included); ghosts are refreshed afterwards.
 */
static void smooth_jacobi(Tree *T, int l) {
    Lev *lv = &T->L[l];
    int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
    double *old = malloc(sizeof(double) * (size_t)lv->nb * ps);
    memcpy(old, lv->phi, sizeof(double) * (size_t)lv->nb * ps);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < lv->nb; b++) {
        const double *xo = old + (size_t)b * ps;
        double *x = lv->phi + (size_t)b * ps, *f = lv->f + (size_t)b * ps;
        for (int k = 0; k < nk; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    double w[6], num = 0.0, den = 0.0;
                    face_weights(T, lv, b, i, j, k, w);
                    for (int d = 0; d < T->dim; d++)
                        for (int s = 0; s < 2; s++) {
                            int q[3] = {i, j, k};
                            q[d] += s ? 1 : -1;
                            num += w[2 * d + s] * xo[pidx(T, n, q[0], q[1], q[2])];
                            den += w[2 * d + s];
                        }
                    int c = pidx(T, n, i, j, k);
                    double xgs = (num - f[c]) / (den + T->helm);
                    x[c] = xo[c] + T->omega * (xgs - xo[c]);
                }
    }
    free(old);
    ghost_fill(T, l, F_PHI);
}

static void smooth(Tree *T, int l, int nsweeps) {
    for (int s = 0; s < nsweeps; s++) {
        if (T->smoother == 1) {
            smooth_jacobi(T, l);
        } else {
            smooth_colour(T, l, 0);
            smooth_colour(T, l, 1);
        }
    }
}

/* ------------------------------------------------ transfers and cycles -- */

/* fine block b of level l covers parent cells poff .. poff + n/2 - 1 */
static void restrict_block(Tree *T, int l, int b, const double *Xf, double *Xc, int what_res) {
    Lev *lv = &T->L[l], *pl = &T->L[l - 1];
    int n = lv->n, ps = P(T, n), pn = pl->n, pps = P(T, pn), dim = T->dim;
    int pb = lv->parent[b], m = n / 2, mk = dim == 3 ? m : 1;
    const int *po = lv->poff + 3 * b;
    for (int k = 0; k < mk; k++)
        for (int j = 0; j < m; j++)
            for (int i = 0; i < m; i++) {
                double sum = 0.0;
                for (int c = 0; c < (1 << dim); c++) {
                    int fi = 2 * i + (c & 1), fj = 2 * j + ((c >> 1) & 1), fk = dim == 3 ? 2 * k + ((c >> 2) & 1) : 0;
                    if (what_res) {
                        int ci = pidx(T, n, fi, fj, fk);
                        sum += lv->f[(size_t)b * ps + ci] - apply_L(T, lv, lv->phi, b, fi, fj, fk);
                    } else {
                        sum += Xf[(size_t)b * ps + pidx(T, n, fi, fj, fk)];
                    }
                }
                Xc[(size_t)pb * pps + pidx(T, pn, po[0] + i, po[1] + j, po[2] + k)] = sum / (1 << dim);
            }
}

/*
 * Downward FAS step from level l to l-1 (Sec. 2.4): r = f - L v on level l,
 * v^H = R v^h, ghost update, v^H_old = v^H, and on the covered coarse cells
 * f^H = R r^h + L^H v^H (eq. for the coarse right-hand side).  R is the mean
 * of the 2^D children (Sec. 2.3).
 */
static void restrict_fas(Tree *T, int l) {
    Lev *lv = &T->L[l], *pl = &T->L[l - 1];
#pragma omp parallel for schedule(static)
    for (int b = 0; b < lv->nb; b++) {
        restrict_block(T, l, b, NULL, pl->tmp, 1);
        restrict_block(T, l, b, lv->phi, pl->phi, 0);
    }
    ghost_fill(T, l - 1, F_PHI);
    size_t np = (size_t)pl->nb * P(T, pl->n);
    memcpy(pl->vold, pl->phi, np * sizeof(double));
    int pn = pl->n, pps = P(T, pn), nk = T->dim == 3 ? pn : 1;
#pragma omp parallel for schedule(static)
    for (int b = 0; b < pl->nb; b++) {
        if (!pl->haschild[b]) continue;
        for (int k = 0; k < nk; k++)
            for (int j = 0; j < pn; j++)
                for (int i = 0; i < pn; i++) {
                    int c = pidx(T, pn, i, j, k);
                    pl->f[(size_t)b * pps + c] = pl->tmp[(size_t)b * pps + c] + apply_L(T, pl, pl->phi, b, i, j, k);
                }
    }
}

/*
 * Upward correction on level l (Sec. 2.4, eq. for the coarse-grid
 * correction): v^h += P(v^H - v^H_old), with P the nearest-neighbour linear
 * interpolation of Sec. 2.3 -- in 2D (2 c0 + c_x + c_y)/4, in 3D
 * (c0 + c_x + c_y + c_z)/4, where c_x etc. are the coarse neighbours on the
 * fine cell's side (coarse ghosts included, no diagonal ones).
 */
static void prolong_correct(Tree *T, int l) {
    Lev *lv = &T->L[l], *pl = &T->L[l - 1];
    int n = lv->n, ps = P(T, n), pn = pl->n, pps = P(T, pn), dim = T->dim, nk = dim == 3 ? n : 1;
#pragma omp parallel for schedule(static)
    for (int b = 0; b < lv->nb; b++) {
        int pb = lv->parent[b];
        const int *po = lv->poff + 3 * b;
        const double *cv = pl->phi + (size_t)pb * pps, *co = pl->vold + (size_t)pb * pps;
        for (int k = 0; k < nk; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    int G[3]; cell_global(lv, b, i, j, k, G);
                    int cc[3] = {po[0] + i / 2, po[1] + j / 2, po[2] + (dim == 3 ? k / 2 : 0)};
                    int c0 = pidx(T, pn, cc[0], cc[1], cc[2]);
                    double corr0 = cv[c0] - co[c0], val;
                    double nbs = 0.0;
                    for (int d = 0; d < dim; d++) {
                        int q[3] = {cc[0], cc[1], cc[2]};
                        q[d] += (G[d] & 1) ? 1 : -1;
                        int cq = pidx(T, pn, q[0], q[1], q[2]);
                        nbs += cv[cq] - co[cq];
                    }
                    if (dim == 2) val = (2.0 * corr0 + nbs) / 4.0;
                    else val = (corr0 + nbs) / 4.0;
                    lv->phi[(size_t)b * ps + pidx(T, n, i, j, k)] += val;
                }
    }
    ghost_fill(T, l, F_PHI);
}

/* ------------------------------------------------ coarsest-level solve -- */

static int factor_coarse(Tree *T) {
    Lev *lv = &T->L[0];
    int n = lv->n, ps = P(T, n), cpb = C(T, n), nk = T->dim == 3 ? n : 1;
    int nc = lv->nb * cpb, ns = nc + (T->singular ? 1 : 0);
    free(T->lu); free(T->piv);
    T->nc = nc; T->nsys = ns;
    T->lu = calloc((size_t)ns * ns, sizeof(double));
    T->piv = malloc(sizeof(int) * ns);
    double *save = malloc(sizeof(double) * (size_t)lv->nb * ps);
    memcpy(save, lv->lam, sizeof(double) * (size_t)lv->nb * ps);
    /* column j = L_hom e_j, with homogeneous boundary ghosts */
    for (int col = 0; col < nc; col++) {
        memset(lv->lam, 0, sizeof(double) * (size_t)lv->nb * ps);
        int cb = col / cpb, cl = col % cpb;
        int ci = cl % n, cj = (cl / n) % n, ck = T->dim == 3 ? cl / (n * n) : 0;
        lv->lam[(size_t)cb * ps + pidx(T, n, ci, cj, ck)] = 1.0;
        ghost_fill(T, 0, F_LAM);
        for (int b = 0; b < lv->nb; b++)
            for (int k = 0; k < nk; k++)
                for (int j = 0; j < n; j++)
                    for (int i = 0; i < n; i++) {
                        int row = b * cpb + (k * n + j) * n + i;
                        T->lu[(size_t)row * ns + col] = apply_L(T, lv, lv->lam, b, i, j, k);
                    }
    }
    if (T->singular) {
        for (int b = 0; b < lv->nb; b++)
            for (int k = 0; k < nk; k++)
                for (int j = 0; j < n; j++)
                    for (int i = 0; i < n; i++) {
                        int row = b * cpb + (k * n + j) * n + i, G[3];
                        cell_global(lv, b, i, j, k, G);
                        T->lu[(size_t)row * ns + nc] = 1.0;
                        T->lu[(size_t)nc * ns + row] = cell_volume(T, lv, G);
                    }
    }
    memcpy(lv->lam, save, sizeof(double) * (size_t)lv->nb * ps);
    free(save);
    /* LU with partial pivoting (Doolittle, row exchanges) */
    double *A = T->lu;
    for (int c = 0; c < ns; c++) {
        int p = c;
        for (int r = c + 1; r < ns; r++) if (fabs(A[(size_t)r * ns + c]) > fabs(A[(size_t)p * ns + c])) p = r;
        T->piv[c] = p;
        if (A[(size_t)p * ns + c] == 0.0) { snprintf(g_err, sizeof g_err, "singular coarse matrix"); return -1; }
        if (p != c)
            for (int e = 0; e < ns; e++) { double t = A[(size_t)c * ns + e]; A[(size_t)c * ns + e] = A[(size_t)p * ns + e]; A[(size_t)p * ns + e] = t; }
        for (int r = c + 1; r < ns; r++) {
            double m = A[(size_t)r * ns + c] / A[(size_t)c * ns + c];
            A[(size_t)r * ns + c] = m;
            for (int e = c + 1; e < ns; e++) A[(size_t)r * ns + e] -= m * A[(size_t)c * ns + e];
        }
    }
    T->lu_ok = 1;
    return 0;
}

static void lu_solve(const Tree *T, double *x) {
    int ns = T->nsys;
    const double *A = T->lu;
    for (int c = 0; c < ns; c++) { int p = T->piv[c]; if (p != c) { double t = x[c]; x[c] = x[p]; x[p] = t; } }
    for (int r = 0; r < ns; r++) for (int c = 0; c < r; c++) x[r] -= A[(size_t)r * ns + c] * x[c];
    for (int r = ns - 1; r >= 0; r--) {
        for (int c = r + 1; c < ns; c++) x[r] -= A[(size_t)r * ns + c] * x[c];
        x[r] /= A[(size_t)r * ns + r];
    }
}

/*
 * Exact solve on the coarsest level (reading R6; the paper smooths there and
 * notes that a direct solver was not yet implemented, Sec. 2.4): with
 * r = f - L v, solve M dv = r (M the linear part of L) and set v += dv; for a
 * problem without Dirichlet faces the bordered system also imposes
 * sum V (v + dv) = 0.
 */
/* max |f - L v| over the coarsest level (ghosts current) */
static double coarse_max_res(Tree *T) {
    Lev *lv = &T->L[0];
    int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
    double mx = 0.0;
    for (int b = 0; b < lv->nb; b++)
        for (int k = 0; k < nk; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    double r = lv->f[(size_t)b * ps + pidx(T, n, i, j, k)] - apply_L(T, lv, lv->phi, b, i, j, k);
                    if (fabs(r) > mx) mx = fabs(r);
                }
    return mx;
}

/* volume-weighted mean of a field over the coarsest level */
static double coarse_mean(Tree *T, const double *X) {
    Lev *lv = &T->L[0];
    int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
    double sv = 0.0, s = 0.0;
    for (int b = 0; b < lv->nb; b++)
        for (int k = 0; k < nk; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    int G[3]; cell_global(lv, b, i, j, k, G);
                    double V = cell_volume(T, lv, G);
                    s += V * X[(size_t)b * ps + pidx(T, n, i, j, k)];
                    sv += V;
                }
    return s / sv;
}

static void coarse_add(Tree *T, double *X, double c) {
    Lev *lv = &T->L[0];
    int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
    for (int b = 0; b < lv->nb; b++)
        for (int k = 0; k < nk; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) X[(size_t)b * ps + pidx(T, n, i, j, k)] += c;
}

/*
 * The coarse-grid solve the paper describes (Sec. 2.4, reading R20):
 * red-black Gauss-Seidel sweeps on the coarsest level, up to coarse_max_it,
 * until max |f - L v| is at most coarse_abs or at most coarse_rel times its
 * value before the first sweep.  On a problem without Dirichlet faces the
 * level's right-hand side is first projected to zero volume-weighted mean
 * (the constants are in the null space, so smoothing cannot remove that
 * part of the residual), and v is returned with zero mean, as the bordered
 * exact solve returns it.
 */
static void coarse_smooth(Tree *T) {
    Lev *lv = &T->L[0];
    if (T->singular) coarse_add(T, lv->f, -coarse_mean(T, lv->f));
    ghost_fill(T, 0, F_PHI);
    double r0 = coarse_max_res(T);
    for (int it = 0; it < T->coarse_max_it; it++) {
        if (r0 <= T->coarse_abs) break;
        smooth_colour(T, 0, 0);
        smooth_colour(T, 0, 1);
        double r = coarse_max_res(T);
        if (r <= T->coarse_abs || r <= T->coarse_rel * r0) break;
    }
    if (T->singular) {
        coarse_add(T, lv->phi, -coarse_mean(T, lv->phi));
        ghost_fill(T, 0, F_PHI);
    }
}

void or_set_coarse_mode(void *h, int mode, double abs_tol, double rel_tol, int max_it) {
    Tree *T = h;
    T->coarse_mode = mode;
    T->coarse_abs = abs_tol;
    T->coarse_rel = rel_tol;
    T->coarse_max_it = max_it;
}

static void coarse_solve(Tree *T) {
    Lev *lv = &T->L[0];
    if (T->coarse_mode == 1) {
        coarse_smooth(T);
        return;
    }
    if (!T->lu_ok) factor_coarse(T);
    int n = lv->n, ps = P(T, n), cpb = C(T, n), nk = T->dim == 3 ? n : 1;
    double *x = calloc(T->nsys, sizeof(double));
    double wv = 0.0;
    for (int b = 0; b < lv->nb; b++)
        for (int k = 0; k < nk; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    int c = pidx(T, n, i, j, k), row = b * cpb + (k * n + j) * n + i, G[3];
                    x[row] = lv->f[(size_t)b * ps + c] - apply_L(T, lv, lv->phi, b, i, j, k);
                    cell_global(lv, b, i, j, k, G);
                    wv += cell_volume(T, lv, G) * lv->phi[(size_t)b * ps + c];
                }
    if (T->singular) x[T->nc] = -wv;
    lu_solve(T, x);
    for (int b = 0; b < lv->nb; b++)
        for (int k = 0; k < nk; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++)
                    lv->phi[(size_t)b * ps + pidx(T, n, i, j, k)] += x[b * cpb + (k * n + j) * n + i];
    free(x);
    ghost_fill(T, 0, F_PHI);
}

/* V-cycle topped at level `top` (Sec. 2.4). */
static void vcycle_top(Tree *T, int top) {
    for (int l = top; l >= 1; l--) {
        smooth(T, l, steps(T, l, 0));
        restrict_fas(T, l);
    }
    coarse_solve(T);
    for (int l = 1; l <= top; l++) {
        prolong_correct(T, l);
        smooth(T, l, steps(T, l, 1));
    }
}

int or_vcycle(void *h, int ncycles) {
    Tree *T = h;
    for (int c = 0; c < ncycles; c++) vcycle_top(T, T->nlev - 1);
    return 0;
}

/* FMG cycle (reading R7). */
int or_fmg(void *h) {
    Tree *T = h;
    int top = T->nlev - 1;
    for (int l = top; l >= 1; l--) restrict_fas(T, l);
    coarse_solve(T);
    for (int l = 1; l <= top; l++) {
        prolong_correct(T, l);
        vcycle_top(T, l);
    }
    return 0;
}

/* covered cells <- mean of children, finest to coarsest; then all ghosts */
static void refresh_field(Tree *T, int which) {
    for (int l = T->nlev - 1; l >= 1; l--) {
        Lev *lv = &T->L[l];
#pragma omp parallel for schedule(static)
        for (int b = 0; b < lv->nb; b++) restrict_block(T, l, b, fld(lv, which), fld(&T->L[l - 1], which), 0);
    }
    for (int l = 0; l < T->nlev; l++) ghost_fill(T, l, which);
}
static void refresh(Tree *T) { refresh_field(T, F_PHI); }

/* ------------------------------------------------------------ leaf I/O -- */

static int64_t leaf_loop(Tree *T, double *io, int which, int dir) {
    int64_t m = 0;
    for (int l = 0; l < T->nlev; l++) {
        Lev *lv = &T->L[l];
        int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
        double *X = which == 0 ? lv->phi : which == 1 ? lv->f : which == 2 ? lv->eps : which == 3 ? lv->lam : lv->adj;
        for (int b = 0; b < lv->nb; b++) {
            if (lv->haschild[b]) continue;
            for (int k = 0; k < nk; k++)
                for (int j = 0; j < n; j++)
                    for (int i = 0; i < n; i++) {
                        double *p = X + (size_t)b * ps + pidx(T, n, i, j, k);
                        if (io) { if (dir) io[m] = *p; else *p = io[m]; }
                        m++;
                    }
        }
    }
    return m;
}
int64_t or_num_leaf_cells(void *h) { return leaf_loop(h, NULL, 0, 0); }
int64_t or_leaf_blocks(void *h, int *out) {
    Tree *T = h; int64_t m = 0;
    for (int l = 0; l < T->nlev; l++) {
        Lev *lv = &T->L[l];
        for (int b = 0; b < lv->nb; b++) {
            if (lv->haschild[b]) continue;
            if (out) { out[4 * m] = lv->depth; memcpy(out + 4 * m + 1, lv->ijk + 3 * b, 3 * sizeof(int)); }
            m++;
        }
    }
    return m;
}

void or_set_rhs(void *h, const double *v) { leaf_loop(h, (double *)v, 1, 0); }
void or_set_phi(void *h, const double *v) { leaf_loop(h, (double *)v, 0, 0); refresh(h); }
void or_get_phi(void *h, double *v) { leaf_loop(h, v, 0, 1); }
void or_get_lam(void *h, double *v) { leaf_loop(h, v, 3, 1); }
int or_set_bc_plane(void *h, int face, int l, const double *v) {
    Tree *T = h; Lev *lv = &T->L[l];
    int d = face / 2, cnt = 1;
    for (int t = 0; t < T->dim; t++) if (t != d) cnt *= lv->ncell[t];
    free(lv->bc[face]);
    lv->bc[face] = malloc(sizeof(double) * cnt);
    memcpy(lv->bc[face], v, sizeof(double) * cnt);
    return 0;
}
void or_refresh(void *h) { refresh(h); }

/* eps on leaves; covered cells take the mean of their children (R4) */
void or_set_eps(void *h, const double *v) {
    Tree *T = h;
    leaf_loop(T, (double *)v, 2, 0);
    refresh_field(T, F_EPS);
    T->lu_ok = 0;
}

/* ------------------------------------------------------ residual norms -- */

/*
 * Composite residual r = f - L phi on all leaf cells (reading R8) after the
 * covered cells are reset to the mean of their children.  Returns the
 * volume-weighted L2 norm sqrt(sum V r^2 / sum V) (the norm of Sec. 4.2)
 * and the max norm; `res` (optional) receives r in leaf order.
 */
void or_residual_norm(void *h, double *l2, double *linf, double *res) {
    Tree *T = h;
    refresh(T);
    double s2 = 0.0, sv = 0.0, mx = 0.0;
    int64_t m0 = 0;
    for (int l = 0; l < T->nlev; l++) {
        Lev *lv = &T->L[l];
        int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1, cpb = C(T, n);
        /* leaf-order offset of every leaf block, then the blocks in parallel
         * with per-block sums added in block order (independent of threads) */
        int64_t *off = malloc(sizeof(int64_t) * (lv->nb ? lv->nb : 1));
        double *bs = calloc(3 * (size_t)(lv->nb ? lv->nb : 1), sizeof(double));
        int64_t m = m0;
        for (int b = 0; b < lv->nb; b++) { off[b] = m; if (!lv->haschild[b]) m += cpb; }
#pragma omp parallel for schedule(static)
        for (int b = 0; b < lv->nb; b++) {
            if (lv->haschild[b]) continue;
            int64_t q = off[b];
            for (int k = 0; k < nk; k++)
                for (int j = 0; j < n; j++)
                    for (int i = 0; i < n; i++) {
                        int G[3]; cell_global(lv, b, i, j, k, G);
                        double r = lv->f[(size_t)b * ps + pidx(T, n, i, j, k)] - apply_L(T, lv, lv->phi, b, i, j, k);
                        double V = cell_volume(T, lv, G);
                        bs[3 * b] += V * r * r; bs[3 * b + 1] += V;
                        if (fabs(r) > bs[3 * b + 2]) bs[3 * b + 2] = fabs(r);
                        if (res) res[q] = r;
                        q++;
                    }
        }
        for (int b = 0; b < lv->nb; b++) {
            s2 += bs[3 * b]; sv += bs[3 * b + 1];
            if (bs[3 * b + 2] > mx) mx = bs[3 * b + 2];
        }
        free(off); free(bs);
        m0 = m;
    }
    *l2 = sqrt(s2 / sv);
    *linf = mx;
}

/* Number of threads for the block loops (OpenMP over the blocks of a
 * level; within a colour the updates are order-independent, so every
 * result is the same for any thread count).  n <= 0 keeps the current
 * setting.  Returns the count in use (1 without OpenMP). */
int or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* composite operator on a leaf vector: out = L x (x clobbers phi) */
void or_apply(void *h, const double *x, double *out) {
    Tree *T = h;
    or_set_phi(T, x);
    int64_t m = 0;
    for (int l = 0; l < T->nlev; l++) {
        Lev *lv = &T->L[l];
        int n = lv->n, nk = T->dim == 3 ? n : 1;
        for (int b = 0; b < lv->nb; b++) {
            if (lv->haschild[b]) continue;
            for (int k = 0; k < nk; k++)
                for (int j = 0; j < n; j++)
                    for (int i = 0; i < n; i++) out[m++] = apply_L(T, lv, lv->phi, b, i, j, k);
        }
    }
}

/* cell volumes and r_i per leaf cell (for weighting in tests) */
void or_leaf_geometry(void *h, double *vol, double *rad) {
    Tree *T = h; int64_t m = 0;
    for (int l = 0; l < T->nlev; l++) {
        Lev *lv = &T->L[l];
        int n = lv->n, nk = T->dim == 3 ? n : 1;
        for (int b = 0; b < lv->nb; b++) {
            if (lv->haschild[b]) continue;
            for (int k = 0; k < nk; k++)
                for (int j = 0; j < n; j++)
                    for (int i = 0; i < n; i++) {
                        int G[3]; cell_global(lv, b, i, j, k, G);
                        vol[m] = cell_volume(T, lv, G);
                        rad[m] = T->lo[0] + (G[0] + 0.5) * lv->h[0];
                        m++;
                    }
        }
    }
}

/* ---------------------------------------------------------- adjoint ----- */

/*
 * Sensitivity of a loss to the cell coefficients, given the converged phi
 * (tree state) and lambda = A^-T dL/dphi (leaf order).  From A phi + b = f:
 * dL/d(eps_f) = -lambda^T d(A phi + b)/d(eps_f) for every face coefficient
 * eps_f (the harmonic mean of Sec. 2.2), chained to the two cells by
 * d eps_f / d eps_c = 2 eps_o^2 / (eps_c + eps_o)^2.  Uniform (single leaf
 * level) meshes only.
 */
int or_eps_grad(void *h, const double *lam, double *out) {
    Tree *T = h;
    int top = T->nlev - 1;
    for (int l = 0; l < T->nlev; l++)
        for (int b = 0; b < T->L[l].nb; b++)
            if (!T->L[l].haschild[b] && l != top) { snprintf(g_err, sizeof g_err, "eps gradient needs a uniform mesh"); return -1; }
    Lev *lv = &T->L[top];
    leaf_loop(T, (double *)lam, 3, 0);
    ghost_fill(T, top, F_LAM);
    int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
    int64_t m = 0;
    for (int b = 0; b < lv->nb; b++) {
        const double *x = lv->phi + (size_t)b * ps, *y = lv->lam + (size_t)b * ps, *E = lv->eps + (size_t)b * ps;
        for (int k = 0; k < nk; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    int c = pidx(T, n, i, j, k), G[3];
                    cell_global(lv, b, i, j, k, G);
                    double g = 0.0;
                    for (int d = 0; d < T->dim; d++)
                        for (int s = 0; s < 2; s++) {
                            int q[3] = {i, j, k};
                            q[d] += s ? 1 : -1;
                            int o = pidx(T, n, q[0], q[1], q[2]);
                            int boundary = (q[d] < 0 || q[d] >= n);
                            int phys = 0;
                            if (boundary) {
                                int qb[3] = {lv->ijk[3 * b], lv->ijk[3 * b + 1], lv->ijk[3 * b + 2]};
                                qb[d] += s ? 1 : -1;
                                phys = (qb[d] < 0 || qb[d] >= lv->nblk[d]) && T->bct[2 * d + s] != BC_PER;
                            }
                            /* row weights without eps: kappa / h^2 for this cell and the other */
                            double kc = 1.0, ko = 1.0;
                            if (T->geom == GEOM_CYL && d == 0) {
                                double rf = T->lo[0] + (G[0] + s) * lv->h[0];
                                double ri = T->lo[0] + (G[0] + 0.5) * lv->h[0];
                                double ro = T->lo[0] + (G[0] + (s ? 1.5 : -0.5)) * lv->h[0];
                                kc = rf / ri; ko = rf / ro;
                            }
                            double h2 = lv->h[d] * lv->h[d];
                            double dA = lam[m] * kc / h2 * (x[o] - x[c]);
                            double de;
                            if (phys) {
                                de = 1.0; /* eps ghost = eps_c => eps_f = eps_c */
                            } else {
                                dA += y[o] * ko / h2 * (x[c] - x[o]);
                                double s2 = E[c] + E[o];
                                de = 2.0 * E[o] * E[o] / (s2 * s2);
                            }
                            g += -dA * de;
                        }
                    out[m++] = g;
                }
    }
    return 0;
}

/* ------------------------------------------------------- test hooks ----- */

/* which: 0 phi, 1 f, 2 eps, 3 vold, 4 lam.  Padded arrays of a whole level,
 * block order of that level (Morton); dir 1 = read, 0 = write. */
int64_t or_level_io(void *h, int l, int which, double *io, int dir) {
    Tree *T = h; Lev *lv = &T->L[l];
    double *X = which == 0 ? lv->phi : which == 1 ? lv->f : which == 2 ? lv->eps : which == 3 ? lv->vold : lv->lam;
    size_t np = (size_t)lv->nb * P(T, lv->n);
    if (io) { if (dir) memcpy(io, X, np * sizeof(double)); else memcpy(X, io, np * sizeof(double)); }
    return (int64_t)np;
}
int or_level_blocks(void *h, int l, int *ijk, int *parent, int *haschild) {
    Tree *T = h; Lev *lv = &T->L[l];
    memcpy(ijk, lv->ijk, sizeof(int) * 3 * lv->nb);
    memcpy(parent, lv->parent, sizeof(int) * lv->nb);
    memcpy(haschild, lv->haschild, sizeof(int) * lv->nb);
    return lv->nb;
}
/* op: 0 ghost_fill(phi), 1 smooth one colour (arg), 2 restrict_fas, 3 prolong_correct, 4 coarse solve */
int or_step(void *h, int op, int l, int arg) {
    Tree *T = h;
    switch (op) {
    case 0: ghost_fill(T, l, F_PHI); break;
    case 1: smooth_colour(T, l, arg); break;
    case 2: restrict_fas(T, l); break;
    case 3: prolong_correct(T, l); break;
    case 4: coarse_solve(T); break;
    case 5: smooth_jacobi(T, l); break;
    default: return -1;
    }
    return 0;
}

/* ------------------------------------------------ divergence cleaning --- */

/*
 * Value of the vector component held in lam at the cell `off` cells away
 * from cell (i,j,k) of block b along dimension d, when that cell lies in
 * this block or in the same-level neighbour block (periodic wrap included);
 * *ok = 0 when the neighbour across that face is not at this level (a
 * physical or refinement face).
 */
static double same_level_value(const Tree *T, const Lev *lv, int b, int i, int j, int k, int d, int off, int *ok) {
    int n = lv->n, ps = P(T, n);
    int q[3] = {i, j, k};
    q[d] += off;
    if (q[d] >= 0 && q[d] < n) { *ok = 1; return lv->lam[(size_t)b * ps + pidx(T, n, q[0], q[1], q[2])]; }
    int bq[3] = {lv->ijk[3 * b], lv->ijk[3 * b + 1], lv->ijk[3 * b + 2]};
    int step = q[d] < 0 ? -1 : 1;
    bq[d] += step;
    if (bq[d] < 0 || bq[d] >= lv->nblk[d]) {
        if (T->bct[2 * d] != BC_PER) { *ok = 0; return 0.0; }
        bq[d] = (bq[d] + lv->nblk[d]) % lv->nblk[d];
    }
    int nb = lookup(lv, bq);
    if (nb < 0) { *ok = 0; return 0.0; }
    q[d] -= step * n;
    *ok = 1;
    return lv->lam[(size_t)nb * ps + pidx(T, n, q[0], q[1], q[2])];
}

/*
 * Cell-centred divergence of a vector field given on the leaf cells
 * (Sec. 4.1).  order 2: sum_d (B_d(c + e_d) - B_d(c - e_d)) / (2 h_d); order
 * 4: sum_d (-B_d(c + 2e_d) + 8 B_d(c + e_d) - 8 B_d(c - e_d) + B_d(c - 2e_d))
 * / (12 h_d) where both cells two away are same-level cells (this block or
 * a same-level neighbour), the second-order form otherwise (reading R14:
 * the grid carries one ghost layer).  Each component is restricted to
 * covered cells and ghost-filled with the rules of Sec. 2.6 (refinement
 * ghosts interpolated like phi; physical faces copy the interior value).
 * B holds dim leaf arrays back to back.  Cartesian meshes only.
 */
int or_divergence_order(void *h, const double *B, double *out, int order) {
    Tree *T = h;
    if (T->geom != GEOM_CART) { snprintf(g_err, sizeof g_err, "divergence: Cartesian meshes only"); return -1; }
    if (order != 2 && order != 4) { snprintf(g_err, sizeof g_err, "divergence: order 2 or 4"); return -1; }
    int64_t nl = or_num_leaf_cells(h);
    for (int64_t m = 0; m < nl; m++) out[m] = 0.0;
    for (int d = 0; d < T->dim; d++) {
        leaf_loop(T, (double *)(B + (size_t)d * nl), 3, 0);
        refresh_field(T, F_VEC);
        int64_t m = 0;
        for (int l = 0; l < T->nlev; l++) {
            Lev *lv = &T->L[l];
            int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
            for (int b = 0; b < lv->nb; b++) {
                if (lv->haschild[b]) continue;
                const double *x = lv->lam + (size_t)b * ps;
                for (int k = 0; k < nk; k++)
                    for (int j = 0; j < n; j++)
                        for (int i = 0; i < n; i++) {
                            int qm[3] = {i, j, k}, qp[3] = {i, j, k};
                            qm[d] -= 1; qp[d] += 1;
                            double bp = x[pidx(T, n, qp[0], qp[1], qp[2])], bm = x[pidx(T, n, qm[0], qm[1], qm[2])];
                            double v = (bp - bm) / (2.0 * lv->h[d]);
                            if (order == 4) {
                                int okp, okm;
                                double bpp = same_level_value(T, lv, b, i, j, k, d, 2, &okp);
                                double bmm = same_level_value(T, lv, b, i, j, k, d, -2, &okm);
                                if (okp && okm) v = (-bpp + 8.0 * bp - 8.0 * bm + bmm) / (12.0 * lv->h[d]);
                            }
                            out[m++] += v;
                        }
            }
        }
    }
    return 0;
}

int or_divergence(void *h, const double *B, double *out) { return or_divergence_order(h, B, out, 2); }

/*
 * Projection step B_new = B - grad phi (Sec. 4.1, eq. for the cleaned field),
 * grad phi by second-order central differences of the current phi (ghosts
 * from the refresh of phi).  Cartesian meshes only.
 */
int or_project(void *h, const double *B, double *out) {
    Tree *T = h;
    if (T->geom != GEOM_CART) { snprintf(g_err, sizeof g_err, "projection: Cartesian meshes only"); return -1; }
    refresh(T);
    int64_t nl = or_num_leaf_cells(h);
    for (int d = 0; d < T->dim; d++) {
        int64_t m = 0;
        for (int l = 0; l < T->nlev; l++) {
            Lev *lv = &T->L[l];
            int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
            for (int b = 0; b < lv->nb; b++) {
                if (lv->haschild[b]) continue;
                const double *x = lv->phi + (size_t)b * ps;
                for (int k = 0; k < nk; k++)
                    for (int j = 0; j < n; j++)
                        for (int i = 0; i < n; i++) {
                            int qm[3] = {i, j, k}, qp[3] = {i, j, k};
                            qm[d] -= 1; qp[d] += 1;
                            double gd = (x[pidx(T, n, qp[0], qp[1], qp[2])] - x[pidx(T, n, qm[0], qm[1], qm[2])]) /
                                        (2.0 * lv->h[d]);
                            out[(size_t)d * nl + m] = B[(size_t)d * nl + m] - gd;
                            m++;
                        }
            }
        }
    }
    return 0;
}

/* ----------------------------------------------------- mesh adaptation -- */

static Lev *level_at_depth(Tree *T, int depth) {
    for (int l = 0; l < T->nlev; l++)
        if (T->L[l].depth == depth) return &T->L[l];
    return NULL;
}

/*
 * Phi carried from the mesh `hold` to the adapted mesh `hnew` (reading R15).
 * The old mesh is refreshed first, so its covered cells hold the mean of
 * their children and every ghost layer is filled.  Then each leaf block of
 * the new mesh
 *   - that is a block of the old mesh (same depth and block coordinates)
 *     copies that block's cells;
 *   - otherwise is a child of an old leaf block and takes, for every cell,
 *     the prolongation of Sec. 2.3 from the parent cell c0 under it and the
 *     parent neighbours c_d on the cell's side in each dimension d:
 *     (2 c0 + c_x + c_y)/4 in 2D, (c0 + c_x + c_y + c_z)/4 in 3D.
 * The new mesh is then refreshed.  Returns 0, or -1 when a new leaf block
 * has neither source.
 */
int or_transfer(void *hold, void *hnew) {
    Tree *O = hold, *T = hnew;
    refresh(O);
    for (int l = 0; l < T->nlev; l++) {
        Lev *lv = &T->L[l];
        Lev *same = level_at_depth(O, lv->depth), *up = level_at_depth(O, lv->depth - 1);
        int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
        for (int b = 0; b < lv->nb; b++) {
            if (lv->haschild[b]) continue;
            const int *q = lv->ijk + 3 * b;
            double *dst = lv->phi + (size_t)b * ps;
            int ob = same ? lookup(same, q) : -1;
            if (ob >= 0) {
                const double *src = same->phi + (size_t)ob * P(O, same->n);
                for (int k = 0; k < nk; k++)
                    for (int j = 0; j < n; j++)
                        for (int i = 0; i < n; i++) dst[pidx(T, n, i, j, k)] = src[pidx(O, n, i, j, k)];
                continue;
            }
            int pq[3] = {q[0] / 2, q[1] / 2, T->dim == 3 ? q[2] / 2 : 0};
            int pb = up ? lookup(up, pq) : -1;
            if (pb < 0 || up->haschild[pb]) {
                snprintf(g_err, sizeof g_err, "transfer: a new leaf block has no source block");
                return -1;
            }
            int pn = up->n;
            const double *par = up->phi + (size_t)pb * P(O, pn);
            for (int k = 0; k < nk; k++)
                for (int j = 0; j < n; j++)
                    for (int i = 0; i < n; i++) {
                        int f[3] = {i, j, k}, cc[3];
                        for (int d = 0; d < 3; d++) cc[d] = d < T->dim ? (q[d] % 2) * (pn / 2) + f[d] / 2 : 0;
                        double c0 = par[pidx(O, pn, cc[0], cc[1], cc[2])], nbs = 0.0;
                        for (int d = 0; d < T->dim; d++) {
                            int e[3] = {cc[0], cc[1], cc[2]};
                            e[d] += ((q[d] * n + f[d]) & 1) ? 1 : -1;
                            nbs += par[pidx(O, pn, e[0], e[1], e[2])];
                        }
                        dst[pidx(T, n, i, j, k)] = T->dim == 2 ? (2.0 * c0 + nbs) / 4.0 : (c0 + nbs) / 4.0;
                    }
        }
    }
    refresh(T);
    return 0;
}

/* ------------------------------------------------ transposed operators -- */

/*
 * The adjoint of a loss through the solve needs A^T, and for divergence
 * cleaning the transposes of the central divergence and gradient (Sec. 4.1).
 * On refined meshes A is not symmetric (reading R16): a fine row reads the
 * coarse cell B through its refinement ghost with weight 1/2 (Sec. 2.6),
 * while the row of B reads the fine cells through the mean of the covered
 * cell D, 1/2^D each.  Every forward operator here is a stencil over padded
 * arrays after refresh_field (restriction of covered cells bottom-up, then
 * ghost fills coarsest level first).  Its transpose runs the steps in the
 * reverse order with transposed coefficients, accumulating into lv->adj, the
 * adjoint of every padded value (interior and ghosts).  Only the linear part
 * counts: boundary values and other constants have no adjoint.
 */

static void zero_adj(Tree *T) {
    for (int l = 0; l < T->nlev; l++)
        memset(T->L[l].adj, 0, sizeof(double) * (size_t)T->L[l].nb * P(T, T->L[l].n));
}

/*
 * Transpose of ghost_fill(T, l, which): every ghost value's adjoint is handed
 * to the values it was formed from and then cleared.  Same-level and periodic
 * ghosts copy a neighbour cell (coefficient 1); physical ghosts depend on the
 * adjacent cell with -1 (Dirichlet, 2a - x_i) or +1 (Neumann, axis; eps and
 * vector components copy x_i); a refinement ghost g = B'/2 + 3c/4 - d/4 with
 * B' = B + sum_t s_t (C_t - A_t)/8 (reading R3) gives 1/2 to B,
 * +-s_t/16 to C_t and A_t (level l-1, interior or ghost), 3/4 to c and -1/4
 * to d (eps ghosts take B alone, reading R4).
 */
static void ghost_fill_T(Tree *T, int l, int which) {
    Lev *lv = &T->L[l];
    int n = lv->n, dim = T->dim, ps = P(T, n);
    for (int b = 0; b < lv->nb; b++) {
        double *ab = lv->adj + (size_t)b * ps;
        for (int d = 0; d < dim; d++)
            for (int s = 0; s < 2; s++) {
                int face = 2 * d + s;
                int q[3] = {lv->ijk[3 * b], lv->ijk[3 * b + 1], lv->ijk[3 * b + 2]};
                q[d] += s ? 1 : -1;
                int phys = 0;
                if (q[d] < 0 || q[d] >= lv->nblk[d]) {
                    if (T->bct[face] == BC_PER) q[d] = (q[d] + lv->nblk[d]) % lv->nblk[d];
                    else phys = 1;
                }
                int nbk = phys ? -1 : lookup(lv, q);
                int tdim[2] = {-1, -1}, nt = 0;
                for (int t = 0; t < dim; t++) if (t != d) tdim[nt++] = t;
                int n1 = n, n2 = nt > 1 ? n : 1;
                for (int u2 = 0; u2 < n2; u2++)
                    for (int u1 = 0; u1 < n1; u1++) {
                        int gi[3] = {0, 0, 0}, ii[3] = {0, 0, 0};
                        gi[tdim[0]] = u1; if (nt > 1) gi[tdim[1]] = u2;
                        memcpy(ii, gi, sizeof ii);
                        gi[d] = s ? n : -1;
                        ii[d] = s ? n - 1 : 0;
                        double *g = ab + pidx(T, n, gi[0], gi[1], gi[2]);
                        double gb = *g;
                        *g = 0.0;
                        double *ai = ab + pidx(T, n, ii[0], ii[1], ii[2]);
                        if (phys) {
                            if (which == F_EPS || which == F_VEC) *ai += gb;
                            else *ai += T->bct[face] == BC_DIR ? -gb : gb;
                        } else if (nbk >= 0) {
                            int jj[3]; memcpy(jj, gi, sizeof jj);
                            jj[d] = s ? 0 : n - 1;
                            lv->adj[(size_t)nbk * ps + pidx(T, n, jj[0], jj[1], jj[2])] += gb;
                        } else {
                            Lev *cl = &T->L[l - 1];
                            int G[3]; cell_global(lv, b, gi[0], gi[1], gi[2], G);
                            if (G[d] < 0) G[d] += lv->ncell[d];
                            if (G[d] >= lv->ncell[d]) G[d] -= lv->ncell[d];
                            int Gc[3] = {G[0] / 2, G[1] / 2, G[2] / 2};
                            int cq[3], nc = cl->n;
                            for (int e = 0; e < 3; e++) cq[e] = e < dim ? Gc[e] / nc : 0;
                            int cb = lookup(cl, cq);
                            double *ca = cl->adj + (size_t)cb * P(T, nc);
                            int lc[3];
                            for (int e = 0; e < 3; e++) lc[e] = e < dim ? Gc[e] - cq[e] * nc : 0;
                            if (which == F_EPS) { ca[pidx(T, nc, lc[0], lc[1], lc[2])] += gb; continue; }
                            ca[pidx(T, nc, lc[0], lc[1], lc[2])] += 0.5 * gb;
                            for (int a = 0; a < nt; a++) {
                                int t = tdim[a];
                                double sg = (G[t] & 1) ? 1.0 : -1.0;
                                int la[3], lcc[3];
                                memcpy(la, lc, sizeof la); memcpy(lcc, lc, sizeof lcc);
                                la[t] -= 1; lcc[t] += 1;
                                ca[pidx(T, nc, lcc[0], lcc[1], lcc[2])] += 0.5 * sg / 8.0 * gb;
                                ca[pidx(T, nc, la[0], la[1], la[2])] -= 0.5 * sg / 8.0 * gb;
                            }
                            int dd[3]; memcpy(dd, ii, sizeof dd);
                            dd[d] = s ? n - 2 : 1;
                            *ai += 0.75 * gb;
                            ab[pidx(T, n, dd[0], dd[1], dd[2])] -= 0.25 * gb;
                        }
                    }
            }
    }
}

/* Transpose of restrict_block for every block of level l: each child cell
 * receives 1/2^D of its parent cell's adjoint (the mean of Sec. 2.3). */
static void restrict_T(Tree *T, int l) {
    Lev *lv = &T->L[l], *pl = &T->L[l - 1];
    int n = lv->n, ps = P(T, n), pn = pl->n, pps = P(T, pn), dim = T->dim;
    int m = n / 2, mk = dim == 3 ? m : 1;
    for (int b = 0; b < lv->nb; b++) {
        int pb = lv->parent[b];
        const int *po = lv->poff + 3 * b;
        for (int k = 0; k < mk; k++)
            for (int j = 0; j < m; j++)
                for (int i = 0; i < m; i++) {
                    double v = pl->adj[(size_t)pb * pps + pidx(T, pn, po[0] + i, po[1] + j, po[2] + k)] / (1 << dim);
                    for (int c = 0; c < (1 << dim); c++) {
                        int fi = 2 * i + (c & 1), fj = 2 * j + ((c >> 1) & 1), fk = dim == 3 ? 2 * k + ((c >> 2) & 1) : 0;
                        lv->adj[(size_t)b * ps + pidx(T, n, fi, fj, fk)] += v;
                    }
                }
    }
}

/* Reverse of refresh_field: ghost fills undone finest level first, then the
 * covered cells' adjoints handed to their children, coarsest level first.
 * Afterwards the leaf cells of lv->adj hold the adjoint of the leaf values. */
static void refresh_T(Tree *T, int which) {
    for (int l = T->nlev - 1; l >= 0; l--) ghost_fill_T(T, l, which);
    for (int l = 1; l < T->nlev; l++) restrict_T(T, l);
}

/* neighbour of cell (i,j,k) across face 2d+s in padded indexing */
static int nbr_pidx(const Tree *T, int n, int i, int j, int k, int d, int s) {
    int q[3] = {i, j, k};
    q[d] += s ? 1 : -1;
    return pidx(T, n, q[0], q[1], q[2]);
}

/*
 * out = A^T y on the leaf cells, A the linear part of the composite
 * operator (homogeneous boundary values): every leaf row
 * sum_f w_f (x_nb - x_c) - lambda x_c (Sec. 2.2) hands w_f y to its
 * neighbour value (interior or ghost) and -(sum_f w_f + lambda) y to its
 * own cell; refresh_T then carries the ghost and covered-cell adjoints to
 * the leaves.
 */
int or_apply_T(void *h, const double *y, double *out) {
    Tree *T = h;
    zero_adj(T);
    int64_t m = 0;
    for (int l = 0; l < T->nlev; l++) {
        Lev *lv = &T->L[l];
        int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
        for (int b = 0; b < lv->nb; b++) {
            if (lv->haschild[b]) continue;
            double *ab = lv->adj + (size_t)b * ps;
            for (int k = 0; k < nk; k++)
                for (int j = 0; j < n; j++)
                    for (int i = 0; i < n; i++) {
                        double w[6], sw = 0.0, yi = y[m++];
                        face_weights(T, lv, b, i, j, k, w);
                        for (int d = 0; d < T->dim; d++)
                            for (int s = 0; s < 2; s++) {
                                ab[nbr_pidx(T, n, i, j, k, d, s)] += w[2 * d + s] * yi;
                                sw += w[2 * d + s];
                            }
                        ab[pidx(T, n, i, j, k)] -= (sw + T->helm) * yi;
                    }
        }
    }
    refresh_T(T, F_PHI);
    leaf_loop(T, out, 4, 1);
    return 0;
}

/*
 * dL/d eps on the leaf cells of any mesh, given the current phi and
 * lambda = A^-T dL/dphi: -lambda^T d(A phi)/d eps.  The row of cell c has
 * the terms w_f (x_nb - x_c), w_f = kappa_f eps_f / h_d^2 with eps_f the
 * harmonic mean 2 e_c e_o / (e_c + e_o) of the cell's and the neighbour's
 * (or ghost's) coefficient (Sec. 2.2); d eps_f / d e_c = 2 e_o^2 / (e_c +
 * e_o)^2.  The eps ghosts and covered cells (reading R4) are undone by
 * refresh_T.  On a mesh without refinement faces this equals or_eps_grad.
 */
int or_eps_grad_T(void *h, const double *lam, double *out) {
    Tree *T = h;
    refresh(T);
    zero_adj(T);
    int64_t m = 0;
    for (int l = 0; l < T->nlev; l++) {
        Lev *lv = &T->L[l];
        int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
        for (int b = 0; b < lv->nb; b++) {
            if (lv->haschild[b]) continue;
            const double *x = lv->phi + (size_t)b * ps, *E = lv->eps + (size_t)b * ps;
            double *ab = lv->adj + (size_t)b * ps;
            for (int k = 0; k < nk; k++)
                for (int j = 0; j < n; j++)
                    for (int i = 0; i < n; i++) {
                        int c = pidx(T, n, i, j, k), G[3];
                        cell_global(lv, b, i, j, k, G);
                        double li = lam[m++];
                        for (int d = 0; d < T->dim; d++)
                            for (int s = 0; s < 2; s++) {
                                int o = nbr_pidx(T, n, i, j, k, d, s);
                                double kap = 1.0;
                                if (T->geom == GEOM_CYL && d == 0) {
                                    double ri = T->lo[0] + (G[0] + 0.5) * lv->h[0];
                                    double rf = T->lo[0] + (G[0] + s) * lv->h[0];
                                    kap = rf / ri;
                                }
                                double e0 = E[c], e1 = E[o], s2 = e0 + e1;
                                double dw = -li * kap / (lv->h[d] * lv->h[d]) * (x[o] - x[c]) * 2.0 / (s2 * s2);
                                ab[c] += dw * e1 * e1;
                                ab[o] += dw * e0 * e0;
                            }
                    }
        }
    }
    refresh_T(T, F_EPS);
    leaf_loop(T, out, 4, 1);
    return 0;
}

/*
 * Transpose of the second-order central divergence of or_divergence
 * (order 2): out (dim leaf arrays) = D^T v.  Each leaf row
 * sum_d (B_d(c+e_d) - B_d(c-e_d)) / (2 h_d) hands +-v/(2 h_d) to the two
 * values of component d; refresh_T with the vector-component ghost rules
 * (physical faces copy the interior value) carries them to the leaves.
 */
int or_divergence_T(void *h, const double *v, double *out) {
    Tree *T = h;
    if (T->geom != GEOM_CART) { snprintf(g_err, sizeof g_err, "divergence: Cartesian meshes only"); return -1; }
    int64_t nl = or_num_leaf_cells(h);
    for (int d = 0; d < T->dim; d++) {
        zero_adj(T);
        int64_t m = 0;
        for (int l = 0; l < T->nlev; l++) {
            Lev *lv = &T->L[l];
            int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
            for (int b = 0; b < lv->nb; b++) {
                if (lv->haschild[b]) continue;
                double *ab = lv->adj + (size_t)b * ps;
                for (int k = 0; k < nk; k++)
                    for (int j = 0; j < n; j++)
                        for (int i = 0; i < n; i++) {
                            double q = v[m++] / (2.0 * lv->h[d]);
                            ab[nbr_pidx(T, n, i, j, k, d, 1)] += q;
                            ab[nbr_pidx(T, n, i, j, k, d, 0)] -= q;
                        }
            }
        }
        refresh_T(T, F_VEC);
        leaf_loop(T, out + (size_t)d * nl, 4, 1);
    }
    return 0;
}

/*
 * Transpose of the central gradient of or_project, grad phi (dim leaf arrays
 * u): out = G^T u on the leaf cells, the ghosts of phi taken with their
 * linear part (homogeneous boundary values).
 */
int or_gradient_T(void *h, const double *u, double *out) {
    Tree *T = h;
    if (T->geom != GEOM_CART) { snprintf(g_err, sizeof g_err, "gradient: Cartesian meshes only"); return -1; }
    int64_t nl = or_num_leaf_cells(h);
    zero_adj(T);
    for (int d = 0; d < T->dim; d++) {
        int64_t m = 0;
        for (int l = 0; l < T->nlev; l++) {
            Lev *lv = &T->L[l];
            int n = lv->n, ps = P(T, n), nk = T->dim == 3 ? n : 1;
            for (int b = 0; b < lv->nb; b++) {
                if (lv->haschild[b]) continue;
                double *ab = lv->adj + (size_t)b * ps;
                for (int k = 0; k < nk; k++)
                    for (int j = 0; j < n; j++)
                        for (int i = 0; i < n; i++) {
                            double q = u[(size_t)d * nl + m++] / (2.0 * lv->h[d]);
                            ab[nbr_pidx(T, n, i, j, k, d, 1)] += q;
                            ab[nbr_pidx(T, n, i, j, k, d, 0)] -= q;
                        }
            }
        }
    }
    refresh_T(T, F_PHI);
    leaf_loop(T, out, 4, 1);
    return 0;
}
