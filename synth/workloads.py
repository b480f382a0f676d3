"""Problem descriptions and seeded input fields.

Interface conventions shared by every solver that consumes these inputs:

* Dimensions are x, y, z (x fastest).  2D problems use x, y (cylindrical:
  x = r, y = z).  Faces are numbered 0:-x 1:+x 2:-y 3:+y 4:-z 5:+z.
* Depth 0 is the unrefined base grid of ``base`` cells cut into blocks of
  ``N`` cells per edge; depth r > 0 are refined levels (cell size halves per
  depth).  A refinement entry ``(r, i, j, k)`` covers the depth-r block with
  block coordinates (i, j, k) by 2**dim children at depth r + 1.
* Leaf data (one value per leaf cell) are ordered by leaf block -- depth
  ascending, then the Morton code of the block coordinates (bit b of i, j, k
  goes to bit 3b, 3b+1, 3b+2) -- and within a block by cell, x fastest.

Nothing here implements any part of the multigrid method itself.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

GEOM_CART = 0
GEOM_CYL = 1
BC_DIRICHLET = 0
BC_NEUMANN = 1
BC_PERIODIC = 2
BC_AXIS = 3


@dataclasses.dataclass
class Problem:
    name: str
    dim: int
    N: int
    geom: int
    base: tuple  # cells per dimension at depth 0 (z = 1 in 2D)
    lo: tuple
    hi: tuple
    bc_type: tuple  # 6 entries
    bc_val: tuple  # 6 entries (used where no plane is given)
    refine: np.ndarray  # int32 [k, 4]  (depth, i, j, k)
    coarse_max: int = 512
    rhs: Optional[Callable] = None  # f(X, Y, Z) -> array
    eps: Optional[Callable] = None  # eps(X, Y, Z) -> array (None => 1)
    bc: Optional[Callable] = None  # value(face, X, Y, Z) -> array (None => bc_val)
    exact: Optional[Callable] = None  # closed-form solution, if any
    rhs_leaf: Optional[Callable] = None  # leaf-array generator (overrides rhs)
    eps_leaf: Optional[Callable] = None

    @property
    def nblk0(self):
        return tuple(max(1, b // self.N) if d < self.dim else 1
                     for d, b in enumerate(self.base))

    def h(self, depth):
        return tuple((self.hi[d] - self.lo[d]) / (self.base[d] * 2.0 ** depth)
                     if d < self.dim else 1.0 for d in range(3))


# ---------------------------------------------------------------- ordering --

def morton(i, j, k):
    """Interleave the bits of block coordinates (x lowest)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    k = np.asarray(k, dtype=np.int64)
    code = np.zeros(np.broadcast(i, j, k).shape, dtype=np.int64)
    for b in range(20):
        code |= ((i >> b) & 1) << (3 * b)
        code |= ((j >> b) & 1) << (3 * b + 1)
        code |= ((k >> b) & 1) << (3 * b + 2)
    return code


def _refine_sets(p: Problem):
    sets = {}
    for r, i, j, k in np.asarray(p.refine, dtype=np.int64).reshape(-1, 4):
        sets.setdefault(int(r), set()).add((int(i), int(j), int(k)))
    return sets


def blocks_by_depth(p: Problem):
    """Return {depth: sorted array [nb, 3] of block coords} (Morton order)."""
    sets = _refine_sets(p)
    n0 = p.nblk0
    cur = [(i, j, k) for k in range(n0[2]) for j in range(n0[1]) for i in range(n0[0])]
    out = {}
    depth = 0
    while cur:
        arr = np.array(cur, dtype=np.int64).reshape(-1, 3)
        order = np.argsort(morton(arr[:, 0], arr[:, 1], arr[:, 2]), kind="stable")
        out[depth] = arr[order]
        ref = sets.get(depth, set())
        nxt = []
        for (i, j, k) in ref:
            for c in range(1 << p.dim):
                ci, cj, ck = 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + ((c >> 2) & 1)
                if p.dim == 2:
                    ck = 0
                    if c >= 4:
                        continue
                nxt.append((ci, cj, ck))
        cur = nxt
        depth += 1
    return out


def leaf_blocks(p: Problem):
    """Canonical leaf block list: int64 [n, 4] (depth, i, j, k)."""
    sets = _refine_sets(p)
    rows = []
    for depth, arr in blocks_by_depth(p).items():
        ref = sets.get(depth, set())
        for (i, j, k) in arr.tolist():
            if (i, j, k) not in ref:
                rows.append((depth, i, j, k))
    return np.array(rows, dtype=np.int64).reshape(-1, 4)


def leaf_cell_centres(p: Problem):
    """Cell centres (X, Y, Z) and cell sizes of all leaf cells, canonical order."""
    N, D = p.N, p.dim
    lb = leaf_blocks(p)
    nc = N ** D
    a = np.arange(N)
    if D == 2:
        lj, li = np.meshgrid(a, a, indexing="ij")
        lk = np.zeros_like(li)
    else:
        lk, lj, li = np.meshgrid(a, a, a, indexing="ij")
    li, lj, lk = li.ravel(), lj.ravel(), lk.ravel()
    X = np.empty(len(lb) * nc)
    Y = np.empty_like(X)
    Z = np.zeros_like(X)
    H = np.empty((len(lb) * nc, 3))
    for depth in np.unique(lb[:, 0]):
        sel = np.nonzero(lb[:, 0] == depth)[0]
        h = p.h(int(depth))
        bi, bj, bk = lb[sel, 1][:, None], lb[sel, 2][:, None], lb[sel, 3][:, None]
        idx = (sel[:, None] * nc + np.arange(nc)[None, :]).ravel()
        X[idx] = (p.lo[0] + (bi * N + li[None, :] + 0.5) * h[0]).ravel()
        Y[idx] = (p.lo[1] + (bj * N + lj[None, :] + 0.5) * h[1]).ravel()
        if D == 3:
            Z[idx] = (p.lo[2] + (bk * N + lk[None, :] + 0.5) * h[2]).ravel()
        H[idx] = h
    return X, Y, Z, H


def leaf_cell_index(p: Problem):
    """Global cell indices (I, J, K) and depth of every leaf cell, canonical order."""
    N, D = p.N, p.dim
    lb = leaf_blocks(p)
    nc = N ** D
    a = np.arange(N)
    if D == 2:
        lj, li = np.meshgrid(a, a, indexing="ij")
        lk = np.zeros_like(li)
    else:
        lk, lj, li = np.meshgrid(a, a, a, indexing="ij")
    I = (lb[:, 1:2] * N + li.ravel()[None, :]).ravel()
    J = (lb[:, 2:3] * N + lj.ravel()[None, :]).ravel()
    K = (lb[:, 3:4] * N + lk.ravel()[None, :]).ravel() if D == 3 else np.zeros(len(lb) * nc, np.int64)
    dep = np.repeat(lb[:, 0], nc)
    return I, J, K, dep


def n_leaf_cells(p: Problem):
    return len(leaf_blocks(p)) * p.N ** p.dim


def leaf_field(p: Problem, which: str):
    """Evaluate 'rhs' or 'eps' at leaf cell centres (canonical order)."""
    gen = p.rhs_leaf if which == "rhs" else p.eps_leaf
    if gen is not None:
        return np.ascontiguousarray(gen(p), dtype=np.float64)
    fn = p.rhs if which == "rhs" else p.eps
    if fn is None:
        n = n_leaf_cells(p)
        return np.zeros(n) if which == "rhs" else np.ones(n)
    X, Y, Z, _ = leaf_cell_centres(p)
    return np.ascontiguousarray(np.broadcast_to(fn(X, Y, Z), X.shape), dtype=np.float64)


def bc_plane(p: Problem, face: int, ncell, h, lo=None):
    """Boundary values at the face centres of one level's boundary plane.

    ``ncell``/``h``: cells per dimension and cell size of that level.  The
    plane is indexed [t2][t1] with t1 < t2 the two tangential dimensions
    (2D: [t1] only).  Returns None when the face uses a constant value.
    """
    if p.bc is None or p.bc_type[face] in (BC_PERIODIC, BC_AXIS):
        return None
    d, side = face // 2, face % 2
    lo = p.lo if lo is None else lo
    tang = [t for t in range(p.dim) if t != d]
    coords = [None, None, None]
    coords[d] = np.array(p.lo[d] if side == 0 else p.hi[d])
    grids = [lo[t] + (np.arange(ncell[t]) + 0.5) * h[t] for t in tang]
    if len(tang) == 1:
        coords[tang[0]] = grids[0]
    else:
        G2, G1 = np.meshgrid(grids[1], grids[0], indexing="ij")
        coords[tang[0]] = G1
        coords[tang[1]] = G2
    shape = np.broadcast(*[c for c in coords if c is not None]).shape
    for t in range(3):
        if coords[t] is None:
            coords[t] = np.zeros(shape)
    vals = p.bc(face, coords[0], coords[1], coords[2])
    return np.ascontiguousarray(np.broadcast_to(vals, shape), dtype=np.float64).ravel()


# --------------------------------------------------------------- balancing --

def balance(dim, nblk0, periodic, sets):
    """Close refinement sets under face 2:1 balance.

    For every refined block at depth r >= 1, each face neighbour (at depth r)
    must exist, i.e. its parent must be refined at depth r - 1.
    """
    sets = {r: set(s) for r, s in sets.items()}
    maxd = max(sets) if sets else -1
    for r in range(maxd, 0, -1):
        nb = [nblk0[d] << r if d < dim else 1 for d in range(3)]
        for (i, j, k) in list(sets.get(r, ())):
            for d in range(dim):
                for s in (-1, 1):
                    q = [i, j, k]
                    q[d] += s
                    if q[d] < 0 or q[d] >= nb[d]:
                        if not periodic[d]:
                            continue
                        q[d] %= nb[d]
                    par = tuple(c >> 1 if dd < dim else 0 for dd, c in enumerate(q))
                    sets.setdefault(r - 1, set()).add(par)
    return sets


def sets_to_refine(sets):
    rows = [(r, i, j, k) for r in sorted(sets) for (i, j, k) in sorted(sets[r])]
    return np.array(rows, dtype=np.int32).reshape(-1, 4)


def refine_spheres(dim, N, base, lo, hi, centre, radii, periodic=(False,) * 3):
    """Refine every depth-r block whose centre lies within radii[r] of centre."""
    nblk0 = [max(1, base[d] // N) if d < dim else 1 for d in range(3)]
    sets = {}
    cur = {(i, j, k) for k in range(nblk0[2]) for j in range(nblk0[1]) for i in range(nblk0[0])}
    for r, R in enumerate(radii):
        bs = [(hi[d] - lo[d]) / (nblk0[d] << r) if d < dim else 0.0 for d in range(3)]
        chosen = set()
        for (i, j, k) in cur:
            c = [lo[0] + (i + 0.5) * bs[0], lo[1] + (j + 0.5) * bs[1],
                 lo[2] + (k + 0.5) * bs[2] if dim == 3 else 0.0]
            dist2 = sum((c[d] - centre[d]) ** 2 for d in range(dim))
            if dist2 <= R * R:
                chosen.add((i, j, k))
        sets[r] = chosen
        nxt = set()
        for (i, j, k) in chosen:
            for c in range(1 << dim):
                nxt.add((2 * i + (c & 1), 2 * j + ((c >> 1) & 1),
                         2 * k + ((c >> 2) & 1) if dim == 3 else 0))
        cur = nxt
    sets = balance(dim, nblk0, periodic, sets)
    return sets_to_refine(sets)


# ------------------------------------------------------------------ fields --

def gaussian_source(centre, sigma):
    """Right-hand side of a 3D Gaussian charge: f = -exp(-r^2/s^2)/(s^3 pi^1.5)."""
    c = centre

    def f(X, Y, Z):
        r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
        return -np.exp(-r2 / sigma ** 2) / (sigma ** 3 * math.pi ** 1.5)
    return f


def gaussian_potential(centre, sigma):
    """Closed-form potential of the Gaussian charge: erf(r/s)/(4 pi r)."""
    from scipy.special import erf
    c = centre

    def phi(X, Y, Z):
        r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
        r = np.maximum(r, 1e-300)
        small = r < 1e-8 * sigma
        val = erf(r / sigma) / (4 * math.pi * r)
        return np.where(small, 1.0 / (2 * math.pi ** 1.5 * sigma), val)
    return phi


# ---------------------------------------------------------------- problems --

def cfg1_poisson2d(n=64, N=8):
    """2D Poisson, unit square, uniform n^2 in N^2 blocks, zero Dirichlet,
    rhs from phi_m = exp(-|x-c|^2/s), s = 0.01, c = (0.5, 0.5)."""
    s = 0.01

    def phi(X, Y, Z):
        return np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / s)

    def rhs(X, Y, Z):
        r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2
        return phi(X, Y, Z) * (4 * r2 / s ** 2 - 4 / s)
    return Problem("poisson2d_%d_b%d" % (n, N), 2, N, GEOM_CART, (n, n, 1), (0.0, 0.0, 0.0),
                   (1.0, 1.0, 1.0), (BC_DIRICHLET,) * 6, (0.0,) * 6,
                   np.zeros((0, 4), np.int32), 512, rhs=rhs, exact=phi)


def cfg2_gauss3d(base=128, N=8, seed=0, radii=(0.3, 0.22, 0.14), sigma=0.02, coarse_max=512):
    """3D Poisson, octree of N^3 blocks, base^3 cells plus len(radii) levels in
    nested spheres around a seeded Gaussian source; Dirichlet from the
    closed-form potential."""
    rng = np.random.default_rng(seed)
    c = tuple(rng.uniform(0.3, 0.7, size=3))
    ref = refine_spheres(3, N, (base,) * 3, (0, 0, 0), (1, 1, 1), c, radii)
    pot = gaussian_potential(c, sigma)
    return Problem("gauss3d_%d_b%d_l%d" % (base, N, len(radii)), 3, N, GEOM_CART,
                   (base,) * 3, (0.0,) * 3, (1.0,) * 3, (BC_DIRICHLET,) * 6, (0.0,) * 6,
                   ref, coarse_max, rhs=gaussian_source(c, sigma),
                   bc=lambda face, X, Y, Z: pot(X, Y, Z), exact=pot)


def conv3d_problem(n=64, N=8, refine="none"):
    """Manufactured 3D convergence problem on the unit cube centred at the
    origin: phi = cos(pi n.x) + 10 exp(-100|x|^2), n = (1, 2, 3) (Sec. 3.1)."""
    nv = (1.0, 2.0, 3.0)

    def phi(X, Y, Z):
        return np.cos(math.pi * (nv[0] * X + nv[1] * Y + nv[2] * Z)) + \
            10 * np.exp(-100 * (X * X + Y * Y + Z * Z))

    def rhs(X, Y, Z):
        r2 = X * X + Y * Y + Z * Z
        lap_cos = -(math.pi ** 2) * sum(v * v for v in nv) * \
            np.cos(math.pi * (nv[0] * X + nv[1] * Y + nv[2] * Z))
        lap_g = 10 * np.exp(-100 * r2) * (4e4 * r2 - 600.0)
        return lap_cos + lap_g
    lo, hi = (-0.5,) * 3, (0.5,) * 3
    if refine == "none":
        ref = np.zeros((0, 4), np.int32)
    else:
        ctr = (0.0, 0.0, 0.0) if refine == "center" else (-0.25, -0.25, -0.25)
        nb = n // N
        sets = {0: set(), 1: set()}
        # depth 1 covers a 0.5^3 box, depth 2 a 0.25^3 box around ctr
        for dep, half in ((0, 0.25), (1, 0.125)):
            nbd = nb << dep
            bs = 1.0 / nbd
            for k in range(nbd):
                for j in range(nbd):
                    for i in range(nbd):
                        cc = [lo[0] + (i + 0.5) * bs, lo[1] + (j + 0.5) * bs, lo[2] + (k + 0.5) * bs]
                        if all(abs(cc[d] - ctr[d]) < half for d in range(3)):
                            sets[dep].add((i, j, k))
        ref = sets_to_refine(balance(3, (nb,) * 3, (False,) * 3, sets))
    return Problem("conv3d_%d_%s" % (n, refine), 3, N, GEOM_CART, (n,) * 3, lo, hi,
                   (BC_DIRICHLET,) * 6, (0.0,) * 6, ref, 512, rhs=rhs,
                   bc=lambda face, X, Y, Z: phi(X, Y, Z), exact=phi)


def random_field(n, corr_len, seed, dim=3):
    """Zero-mean, unit-variance Gaussian random field on a periodic n^dim grid,
    white noise filtered with the spectrum exp(-k^2 l^2 / 2)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n,) * dim)
    k = 2 * math.pi * np.fft.fftfreq(n, d=1.0 / n)
    ks = np.meshgrid(*([k] * dim), indexing="ij")
    k2 = sum(kk * kk for kk in ks)
    g = np.real(np.fft.ifftn(np.fft.fftn(w) * np.exp(-k2 * corr_len ** 2 / 2)))
    g -= g.mean()
    g /= g.std()
    return g  # indexed [x, y, z]


def cfg3_varcoef3d(n=256, N=16, seed=0, contrast=100.0, radius=0.25, corr_len=0.05):
    """3D variable-coefficient Poisson, uniform n^3 in N^3 blocks, eps = contrast
    inside a seeded sphere, Neumann (b = 0) on x faces, periodic in y and z,
    rhs a zero-mean Gaussian random field."""
    rng = np.random.default_rng(seed)
    xs = tuple(rng.uniform(0.25, 0.75, size=3))

    def eps(X, Y, Z):
        r2 = (X - xs[0]) ** 2 + (Y - xs[1]) ** 2 + (Z - xs[2]) ** 2
        return np.where(r2 < radius ** 2, contrast, 1.0)

    def rhs_leaf(p):
        g = random_field(n, corr_len, seed + 1000, 3)
        I, J, K, _ = leaf_cell_index(p)
        return g[I, J, K]
    bct = (BC_NEUMANN, BC_NEUMANN, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)
    return Problem("varcoef3d_%d_b%d" % (n, N), 3, N, GEOM_CART, (n,) * 3, (0.0,) * 3,
                   (1.0,) * 3, bct, (0.0,) * 6, np.zeros((0, 4), np.int32), 512,
                   eps=eps, rhs_leaf=rhs_leaf)


def cyl_ring_tree(seed, N=16, kmin=2, kmax=32, force_k=None):
    """One 2D cylindrical (r, z) tree: side N*k cells on [0,1]^2, 0-2 AMR
    levels around a seeded ring point, eps = 1 + 0.5 sin(2 pi z), Dirichlet 0
    at r = 1, z = 0, z = 1 and the symmetry axis at r = 0."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(kmin, kmax + 1)) if force_k is None else force_k
    nlev = int(rng.integers(0, 3))
    r0, z0 = rng.uniform(0.2, 0.8, size=2)
    n = N * k
    radii = (0.1, 0.05)[:nlev]
    ref = refine_spheres(2, N, (n, n, 1), (0, 0, 0), (1, 1, 1), (r0, z0, 0.0), radii)
    w = 0.03

    def rhs(X, Y, Z):
        return -np.exp(-((X - r0) ** 2 + (Y - z0) ** 2) / w ** 2) / (math.pi * w * w)

    def eps(X, Y, Z):
        return 1.0 + 0.5 * np.sin(2 * math.pi * Y)
    bct = (BC_AXIS, BC_DIRICHLET, BC_DIRICHLET, BC_DIRICHLET, BC_PERIODIC, BC_PERIODIC)
    return Problem("cyl_%d_k%d_l%d" % (seed, k, nlev), 2, N, GEOM_CYL, (n, n, 1),
                   (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), bct, (0.0,) * 6, ref, 1024,
                   rhs=rhs, eps=eps)


def kolmogorov_field(n, seed, dim=3):
    """dim-component periodic Gaussian field on n^dim cells whose component
    spectra fall as |B_k|^2 ~ k^(-11/3) (shell spectrum E(k) ~ k^(-5/3)) for
    integer wavenumbers 1 <= |k| <= n/2, zero elsewhere, random phases (the
    FFT of white noise), not projected; scaled so that mean |B|^2 = 1.
    Returns float64 [dim, n, ..., n] indexed [component, x, y, z]."""
    rng = np.random.default_rng(seed)
    k = np.fft.fftfreq(n, d=1.0 / n)
    kr = np.fft.rfftfreq(n, d=1.0 / n)
    ks = np.meshgrid(*([k] * (dim - 1) + [kr]), indexing="ij")
    kk = np.sqrt(sum(q * q for q in ks))
    amp = np.zeros_like(kk)
    band = (kk >= 1.0) & (kk <= n / 2)
    amp[band] = kk[band] ** (-11.0 / 6.0)
    del ks, kk, band
    import scipy.fft as sfft
    out = np.empty((dim,) + (n,) * dim)
    for c in range(dim):
        w = rng.standard_normal((n,) * dim)
        out[c] = sfft.irfftn(sfft.rfftn(w, workers=-1) * amp, s=(n,) * dim, workers=-1)
    out /= math.sqrt(np.mean(np.sum(out * out, axis=0)))
    return out


def _parallel_chunks(fn, n, chunk):
    """fn(lo, hi) over [0, n) in chunks on a thread pool (numpy releases the
    GIL in its array kernels); results in chunk order."""
    from concurrent.futures import ThreadPoolExecutor
    import os
    spans = [(a, min(a + chunk, n)) for a in range(0, n, chunk)]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        return list(ex.map(lambda ab: fn(*ab), spans))


class CleanInputs:
    """Config 5 inputs: a periodic 3D field B = B_turb + B_blob on an octree
    refined where |B| is large, and the target field B_t of the loss.

    B_turb is kolmogorov_field on the base grid (seed); on refined cells it
    takes the value of the base cell that contains them (the prolongation of
    the input is piecewise constant, an input definition).  The blob is the
    non-solenoidal field grad(A exp(-|x - x_b|^2 / w^2)), evaluated at every
    leaf cell centre, with x_b drawn from U[0.25, 0.75]^3 and A scaled so
    that its peak magnitude is `peak` times the rms of B_turb.  Refinement:
    depth 1 covers the base blocks whose max |B| is in the top `frac` of
    all base blocks, depth 2 likewise among the depth-1 blocks, then 2:1
    balance (periodic)."""

    def __init__(self, n=512, N=16, seed=0, levels=2, frac=0.1, w=0.05, peak=3.0, target_seed=3):
        self.n, self.N, self.seed, self.w, self.target_seed = n, N, seed, w, target_seed
        rng = np.random.default_rng(seed + 7919)
        self.xb = tuple(rng.uniform(0.25, 0.75, size=3))
        # peak of |grad(A exp(-r^2/w^2))| = A sqrt(2) exp(-1/2) / w at r = w / sqrt(2)
        self.A = peak * w / (math.sqrt(2.0) * math.exp(-0.5))
        self.turb = kolmogorov_field(n, seed)
        nb0 = n // N
        h0 = 1.0 / n
        # depth 0: max |B| per base block, B = turb + blob at the base cell centres
        a = (np.arange(n) + 0.5) * h0
        mag = self._magnitude(self.turb, a)
        bmax = mag.reshape(nb0, N, nb0, N, nb0, N).max(axis=(1, 3, 5))
        del mag
        sets = {}
        cur = np.argwhere(bmax >= np.quantile(bmax, 1.0 - frac))
        for depth in range(levels):
            sets[depth] = {tuple(int(x) for x in q) for q in cur}
            if depth + 1 == levels:
                break
            # children of the refined blocks, max |B| of each over its cells
            kids = np.array([(2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + (c >> 2))
                             for (i, j, k) in sorted(sets[depth]) for c in range(8)], np.int64)
            hd = h0 / 2 ** (depth + 1)
            li = np.arange(N)
            sh = depth + 1

            def kid_max(lo, hi, kids=kids, hd=hd, sh=sh):
                m = np.empty(hi - lo)
                for q in range(lo, hi):
                    i, j, k = kids[q]
                    gi, gj, gk = i * N + li, j * N + li, k * N + li
                    bt = self.turb[:, (gi >> sh)[:, None, None], (gj >> sh)[None, :, None], (gk >> sh)[None, None, :]]
                    bb = self._blob(((gi + 0.5) * hd)[:, None, None], ((gj + 0.5) * hd)[None, :, None],
                                    ((gk + 0.5) * hd)[None, None, :])
                    m[q - lo] = np.sqrt(((bt + bb) ** 2).sum(axis=0)).max()
                return m
            m = np.concatenate(_parallel_chunks(kid_max, len(kids), 512))
            cur = kids[m >= np.quantile(m, 1.0 - frac)]
        self.refine = sets_to_refine(balance(3, (nb0,) * 3, (True,) * 3, sets))
        self.problem = Problem("clean3d_%d_b%d_l%d" % (n, N, levels), 3, N, GEOM_CART, (n,) * 3, (0.0,) * 3,
                               (1.0,) * 3, (BC_PERIODIC,) * 6, (0.0,) * 6, self.refine, 512)

    def _blob(self, X, Y, Z):
        dx, dy, dz = X - self.xb[0], Y - self.xb[1], Z - self.xb[2]
        e = self.A * np.exp(-(dx * dx + dy * dy + dz * dz) / self.w ** 2) * (-2.0 / self.w ** 2)
        return np.stack(np.broadcast_arrays(e * dx, e * dy, e * dz))

    def _magnitude(self, turb, a):
        out = np.empty(turb.shape[1:])

        def slab(lo, hi):
            for k in range(lo, hi):
                bb = self._blob(a[:, None], a[None, :], a[k])
                out[:, :, k] = np.sqrt(((turb[:, :, :, k] + bb) ** 2).sum(axis=0))
        _parallel_chunks(slab, len(a), 8)
        return out

    def leaf_fields(self, with_blob=True, field=None):
        """B on the leaf cells, [3, n_leaf] in leaf order: the base-grid field
        at the base cell containing each leaf cell, plus the blob at the leaf
        cell centre (with_blob)."""
        p = self.problem
        lb = leaf_blocks(p)
        N, nc = self.N, self.N ** 3
        turb = self.turb if field is None else field
        out = np.empty((3, len(lb) * nc))
        li = np.arange(N)
        ck, cj, ci = np.meshgrid(li, li, li, indexing="ij")
        ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
        def fill(lo, hi):
            # leaf blocks [lo, hi) are one contiguous range of leaf cells
            part = np.arange(lo, hi)
            d = lb[part, 0][:, None]
            I = lb[part, 1][:, None] * N + ci[None, :]
            J = lb[part, 2][:, None] * N + cj[None, :]
            K = lb[part, 3][:, None] * N + ck[None, :]
            v = turb[:, I >> d, J >> d, K >> d].reshape(3, -1)
            if with_blob:
                h = 1.0 / (self.n * 2.0 ** d)
                v += self._blob((I + 0.5) * h, (J + 0.5) * h, (K + 0.5) * h).reshape(3, -1)
            out[:, lo * nc:hi * nc] = v
        _parallel_chunks(fill, len(lb), 256)
        return out

    def target(self):
        """B_t: the seeded turbulent field alone (target_seed), on the leaves."""
        return self.leaf_fields(with_blob=False, field=kolmogorov_field(self.n, self.target_seed))
