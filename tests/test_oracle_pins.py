"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test states what it pins.  None of them re-derives the oracle's own
formula: they check closed forms, invariants, a printed table, identities
derived independently, brute-force dense solves and convergence orders.
"""
import math
import os

import numpy as np
import pytest

from oracle import Oracle
from synth import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
DIR, NEU, PER, AXIS = W.BC_DIRICHLET, W.BC_NEUMANN, W.BC_PERIODIC, W.BC_AXIS


def lin_problem(dim, refine, coef, bct=None, N=4, base=16, geom=0):
    """Mesh with boundary planes taken from the linear function coef.x + 1."""
    def phi(X, Y, Z):
        return coef[0] * X + coef[1] * Y + (coef[2] * Z if dim == 3 else 0) + 1.0

    def bc(face, X, Y, Z):
        d, side = face // 2, face % 2
        if (bct or (DIR,) * 6)[face] == NEU:
            return np.full(np.shape(X), float(coef[d]))
        return phi(X, Y, Z)
    p = W.Problem("lin", dim, N, geom, (base, base, base if dim == 3 else 1),
                  (0.0,) * 3, (1.0,) * 3, bct or (DIR,) * 6, (0.0,) * 6, refine, 512,
                  rhs=None, bc=bc, exact=phi)
    return p


def amr_refine(dim, N, base, centre, radii, periodic=(False,) * 3):
    return W.refine_spheres(dim, N, (base, base, base if dim == 3 else 1), (0, 0, 0),
                            (1, 1, 1), centre, radii, periodic)


# ---------------------------------------------------------------- levels --

def test_coarse_levels_match_paper_table():
    """Level construction (Sec. 2.5, table of added coarse grids)."""
    rows = [list(map(int, ln.split())) for ln in open(os.path.join(GOLD, "coarse_levels_192x96.txt"))
            if ln.strip() and not ln.startswith("#")]
    o = Oracle(2, 8, 0, (DIR,) * 6, (0.0,) * 6, (192, 96), (0, 0), (2, 1), coarse_max=0)
    lv = o.levels()[::-1]  # finest first
    assert len(lv) == len(rows)
    for info, (level, cx, cy, bs, bx, by) in zip(lv, rows):
        assert info["depth"] == level - 1
        assert info["ncell"][:2] == (cx, cy)
        assert info["n"] == bs
        assert info["nblk"][:2] == (bx, by)


def test_coarsest_levels_of_the_workloads():
    """cfg1 keeps 4 levels down to one 8^2 block; a 16^3-block grid stops at 8^3."""
    o = Oracle(2, 8, 0, (DIR,) * 6, (0.0,) * 6, (64, 64), (0, 0), (1, 1))
    assert [(l["n"], l["nblk"][:2]) for l in o.levels()] == [(8, (1, 1)), (8, (2, 2)), (8, (4, 4)), (8, (8, 8))]
    o = Oracle(3, 16, 0, (DIR,) * 6, (0.0,) * 6, (64, 64, 64), (0,) * 3, (1,) * 3)
    assert [(l["n"], l["nblk"]) for l in o.levels()] == [(8, (1, 1, 1)), (16, (1, 1, 1)), (16, (2, 2, 2)), (16, (4, 4, 4))]


def test_unbalanced_mesh_rejected():
    """2:1 balance is a precondition (Sec. 2.5, Sec. 2.7)."""
    ref = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [2, 1, 1, 0]], np.int32)
    with pytest.raises(ValueError):
        Oracle(2, 4, 0, (DIR,) * 6, (0.0,) * 6, (16, 16), (0, 0), (1, 1), ref)


# -------------------------------------------------------------- operator --

@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("bcname", ["dirichlet", "neumann_x"])
def test_operator_exact_on_linear_with_refinement(dim, bcname):
    """Every ghost rule of Sec. 2.6 (same level, physical, refinement boundary)
    and the mean restriction are exact on linear functions, so the composite
    operator of a linear function vanishes on every leaf cell."""
    N, base = 4, (16 if dim == 2 else 8)
    ref = amr_refine(dim, N, base, (0.3, 0.6, 0.45), (0.35, 0.2))
    assert len(ref) > 0
    bct = None if bcname == "dirichlet" else (NEU, NEU, DIR, DIR, DIR, DIR)
    coef = (0.7, -1.3, 0.4)
    p = lin_problem(dim, ref, coef, bct, N=N, base=base)
    o = Oracle.from_problem(p, set_fields=False)
    o.set_bc_from_problem(p)
    X, Y, Z, H = W.leaf_cell_centres(p)
    Lx = o.apply(p.exact(X, Y, Z))
    assert np.abs(Lx).max() < 1e-9 * (1.0 / H[:, 0].min() ** 2)


def test_operator_quadratic_cartesian():
    """Sec. 2.2 discretisation: exact on quadratics away from the boundary."""
    p = lin_problem(3, np.zeros((0, 4), np.int32), (0, 0, 0), N=4, base=8)
    o = Oracle.from_problem(p, set_fields=False)
    X, Y, Z, H = W.leaf_cell_centres(p)
    Lx = o.apply(X * X + 2 * Y * Y - 0.5 * Z * Z)
    h = H[0, 0]
    inner = (X > h) & (X < 1 - h) & (Y > h) & (Y < 1 - h) & (Z > h) & (Z < 1 - h)
    np.testing.assert_allclose(Lx[inner], 2 + 4 - 1, rtol=0, atol=1e-9)


def test_operator_quadratic_cylindrical():
    """Cylindrical form: (1/r) d/dr (r d/dr r^2) = 4 and d^2/dz^2 z^2 = 2,
    including the cells on the axis."""
    p = lin_problem(2, np.zeros((0, 4), np.int32), (0, 0, 0),
                    bct=(AXIS, DIR, DIR, DIR, PER, PER), N=4, base=16, geom=W.GEOM_CYL)
    o = Oracle.from_problem(p, set_fields=False)
    X, Y, Z, H = W.leaf_cell_centres(p)
    h = H[0, 0]
    inner = (X < 1 - h) & (Y > h) & (Y < 1 - h)
    np.testing.assert_allclose(o.apply(X * X)[inner], 4.0, atol=1e-9)
    np.testing.assert_allclose(o.apply(Y * Y)[inner], 2.0, atol=1e-9)
    np.testing.assert_allclose(o.apply(np.full_like(X, 3.0))[inner], 0.0, atol=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_harmonic_face_coefficient_exact_for_layers(dim):
    """Sec. 2.2: with the harmonic mean of the two cell coefficients the
    discrete flux across a material interface lying on a cell face is exact
    for a layered medium, so the piecewise-linear solution with continuous
    flux eps dphi/dx = q satisfies the discrete equation on every cell."""
    base, N = 16, 4
    e1, e2, q = 1.0, 10.0, 0.8

    def phi(X, Y, Z):
        return np.where(X < 0.5, q * X / e1, q * 0.5 / e1 + q * (X - 0.5) / e2) + 0.3

    p = W.Problem("layers", dim, N, 0, (base, base, base if dim == 3 else 1), (0.0,) * 3,
                  (1.0,) * 3, (DIR, DIR, NEU, NEU, NEU, NEU), (0.0,) * 6,
                  np.zeros((0, 4), np.int32), 512, bc=lambda face, X, Y, Z: phi(X, Y, Z) if face < 2 else 0 * X)
    o = Oracle.from_problem(p, set_fields=False)
    o.set_bc_from_problem(p)
    X, Y, Z, H = W.leaf_cell_centres(p)
    o.set_eps(np.where(X < 0.5, e1, e2))
    np.testing.assert_allclose(o.apply(phi(X, Y, Z)), 0.0, atol=1e-10)


@pytest.mark.parametrize("case", ["2d_dir_eps", "3d_neu_per_eps", "cyl_eps"])
def test_operator_symmetric_on_uniform_mesh(case):
    """With homogeneous boundary values the uniform-mesh operator is symmetric
    (r-weighted in the cylindrical form): <u, A v> = <A u, v>."""
    rng = np.random.default_rng(3)
    if case == "2d_dir_eps":
        o = Oracle(2, 4, 0, (DIR, NEU, DIR, DIR, 0, 0), (0.0,) * 6, (16, 16), (0, 0), (1, 1))
    elif case == "3d_neu_per_eps":
        o = Oracle(3, 4, 0, (NEU, NEU, PER, PER, PER, PER), (0.0,) * 6, (8, 8, 8), (0,) * 3, (1,) * 3)
    else:
        o = Oracle(2, 4, 1, (AXIS, DIR, DIR, DIR, PER, PER), (0.0,) * 6, (16, 16), (0, 0), (1, 1))
    o.set_eps(np.exp(rng.uniform(-1, 1, o.n_leaf)))
    o.set_homogeneous(True)
    _, rad = o.leaf_geometry()
    w = rad if case == "cyl_eps" else np.ones(o.n_leaf)
    u, v = rng.standard_normal(o.n_leaf), rng.standard_normal(o.n_leaf)
    Au, Av = o.apply(u), o.apply(v)
    a, b = np.dot(w * u, Av), np.dot(w * Au, v)
    assert abs(a - b) <= 1e-12 * (abs(a) + np.linalg.norm(w * u) * np.linalg.norm(Av))


# ---------------------------------------------------- refinement ghosts --

def _flux_identity_residuals(dim):
    N, base = 4, (16 if dim == 2 else 8)
    ref = amr_refine(dim, N, base, (0.55, 0.4, 0.5), (0.3 if dim == 2 else 0.45,))
    o = Oracle(dim, N, 0, (DIR,) * 6, (0.0,) * 6, (base,) * dim, (0,) * dim, (1,) * dim, ref)
    rng = np.random.default_rng(7)
    o.set_phi(rng.standard_normal(o.n_leaf))  # restricts covered cells, fills ghosts
    levels = o.levels()
    lf = len(levels) - 1
    fine = o.level_get(lf, "phi")
    coarse = o.level_get(lf - 1, "phi")
    fijk, _, _ = o.level_blocks(lf)
    cijk, _, _ = o.level_blocks(lf - 1)
    fset = {tuple(x): b for b, x in enumerate(fijk.tolist())}
    cset = {tuple(x): b for b, x in enumerate(cijk.tolist())}
    nblk = levels[lf]["nblk"]
    out = []
    for b, q in enumerate(fijk.tolist()):
        for d in range(dim):
            for s in (0, 1):
                nq = list(q)
                nq[d] += 1 if s else -1
                if nq[d] < 0 or nq[d] >= nblk[d] or tuple(nq) in fset:
                    continue
                # coarse neighbour block and the cells along this face
                Fb = fine[b]
                tang = [t for t in range(dim) if t != d]
                for m in np.ndindex(*([N // 2] * (dim - 1))):
                    ci = [0] * 3
                    gsum, csum = 0.0, 0.0
                    allc = []
                    for sub in np.ndindex(*([2] * (dim - 1))):
                        idx = [0] * dim
                        for a, t in enumerate(tang):
                            idx[t] = 2 * m[a] + sub[a]
                        gidx, c_idx, d_idx = list(idx), list(idx), list(idx)
                        gidx[d] = N if s else -1
                        c_idx[d] = N - 1 if s else 0
                        d_idx[d] = N - 2 if s else 1
                        g = Fb[tuple(x + 1 for x in gidx[::-1])]
                        c = Fb[tuple(x + 1 for x in c_idx[::-1])]
                        dd = Fb[tuple(x + 1 for x in d_idx[::-1])]
                        gsum += g
                        csum += c
                        allc += [c, dd]
                    D = np.mean(allc)  # restriction of the 2^D fine cells
                    # B: the coarse cell across the face
                    G = [q[t] * N + (2 * m[tang.index(t)] if t != d else (N if s else -1)) for t in range(dim)]
                    Gc = [x // 2 for x in G]
                    cb = tuple(x // N for x in Gc) + (0,) * (3 - dim)
                    lc = [Gc[t] - cb[t] * N for t in range(dim)]
                    B = coarse[cset[cb]][tuple(x + 1 for x in lc[::-1])]
                    # face flux equality: (2^(dim-1) fine faces of size h^(dim-1)) vs coarse face
                    out.append((2 ** (dim - 2)) * (D - B) - (csum - gsum))
                    del ci
    return np.array(out)


@pytest.mark.parametrize("dim", [2, 3])
def test_refinement_ghosts_conserve_flux(dim):
    """Sec. 2.6: the refinement-boundary ghosts give the same coarse and summed
    fine flux through a coarse face.  With H = 2h this reads
    D - B = (c - g) + (a - h) in 2D and 2 (D - B) = sum_k (c_k - g_k) in 3D;
    the printed 2D form with halves is off by a factor two (checked with
    phi = x: D - B = 2h, c - g = a - h = h)."""
    res = _flux_identity_residuals(dim)
    assert len(res) > 0
    assert np.abs(res).max() < 1e-12


# ------------------------------------------------------------ transfers --

def _set_level_linear(o, l, coef):
    info = o.levels()[l]
    n, dim = info["n"], o.dim
    ijk, _, _ = o.level_blocks(l)
    arr = np.zeros((info["nb"],) + (n + 2,) * dim)
    idx = np.arange(-1, n + 1)
    for b, q in enumerate(ijk):
        grids = [(q[d] * n + idx + 0.5) * info["h"][d] for d in range(dim)]
        mesh = np.meshgrid(*grids[::-1], indexing="ij")  # z, y, x order
        val = np.ones_like(mesh[0])
        for d in range(dim):
            val = val + coef[d] * mesh[dim - 1 - d]
        arr[b] = val
    o.level_set(l, "phi", arr)


@pytest.mark.parametrize("dim", [2, 3])
def test_prolongation_exact_on_linear(dim):
    """Sec. 2.3, eqs. for 2D/3D interpolation: exact on linear functions."""
    base = 32 if dim == 2 else 16
    o = Oracle(dim, 4, 0, (DIR,) * 6, (0.0,) * 6, (base,) * dim, (0,) * dim, (1,) * dim)
    lf = len(o.levels()) - 1
    coef = (0.3, -0.8, 1.7)
    _set_level_linear(o, lf - 1, coef)
    o.level_set(lf - 1, "vold", np.zeros_like(o.level_get(lf - 1, "vold")))
    o.level_set(lf, "phi", np.zeros_like(o.level_get(lf, "phi")))
    o.step("prolong", lf)
    info = o.levels()[lf]
    fine = o.level_get(lf, "phi")
    ijk, _, _ = o.level_blocks(lf)
    n = info["n"]
    idx = np.arange(n)
    for b, q in enumerate(ijk):
        grids = [(q[d] * n + idx + 0.5) * info["h"][d] for d in range(dim)]
        mesh = np.meshgrid(*grids[::-1], indexing="ij")
        want = 1.0 + sum(coef[d] * mesh[dim - 1 - d] for d in range(dim))
        got = fine[b][(slice(1, n + 1),) * dim]
        np.testing.assert_allclose(got, want, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_restriction_of_prolongation(dim):
    """R P u = u + (H^2/8) Lap_H u (derived from the interpolation weights of
    Sec. 2.3 and the mean restriction): in 2D the four children sum to
    (8 u0 + 2 sum nb)/4, in 3D the eight to 2 u0 + sum nb."""
    base = 32 if dim == 2 else 16
    o = Oracle(dim, 4, 0, (DIR,) * 6, (0.0,) * 6, (base,) * dim, (0,) * dim, (1,) * dim)
    lf = len(o.levels()) - 1
    rng = np.random.default_rng(11)
    u = rng.standard_normal(o.level_get(lf - 1, "phi").shape)
    o.level_set(lf - 1, "phi", u)
    o.level_set(lf - 1, "vold", np.zeros_like(u))
    o.level_set(lf, "phi", np.zeros_like(o.level_get(lf, "phi")))
    o.step("prolong", lf)
    fine = o.level_get(lf, "phi")
    fijk, fpar, _ = o.level_blocks(lf)
    cinfo, finfo = o.levels()[lf - 1], o.levels()[lf]
    n, cn = finfo["n"], cinfo["n"]
    for b, q in enumerate(fijk):
        pb = fpar[b]
        F = fine[b][(slice(1, n + 1),) * dim]
        # mean over children
        if dim == 2:
            R = 0.25 * (F[0::2, 0::2] + F[0::2, 1::2] + F[1::2, 0::2] + F[1::2, 1::2])
        else:
            R = sum(F[a::2, c::2, e::2] for a in (0, 1) for c in (0, 1) for e in (0, 1)) / 8.0
        off = [(q[d] % 2) * (n // 2) if cn == n else 0 for d in range(dim)]
        U = u[pb]
        sl = tuple(slice(1 + off[d], 1 + off[d] + n // 2) for d in range(dim))[::-1]
        u0 = U[sl]
        nbsum = 0
        for d in range(dim):
            for s in (-1, 1):
                sl2 = list(sl)
                ax = dim - 1 - d
                sl2[ax] = slice(sl[ax].start + s, sl[ax].stop + s)
                nbsum = nbsum + U[tuple(sl2)]
        np.testing.assert_allclose(R, u0 + (nbsum - 2 * dim * u0) / 8.0, atol=1e-13)


def test_restriction_is_the_mean_and_conserves_volume_integral():
    """Sec. 2.3: a covered cell holds the mean of its children, so sum V x is
    the same on a refined patch and under it."""
    dim, N, base = 2, 4, 16
    ref = amr_refine(dim, N, base, (0.4, 0.4, 0), (0.3,))
    o = Oracle(dim, N, 0, (DIR,) * 6, (0.0,) * 6, (base,) * dim, (0,) * dim, (1,) * dim, ref)
    rng = np.random.default_rng(5)
    o.set_phi(rng.standard_normal(o.n_leaf))
    lv = o.levels()
    lf = len(lv) - 1
    fine, coarse = o.level_get(lf, "phi"), o.level_get(lf - 1, "phi")
    fijk, fpar, _ = o.level_blocks(lf)
    Vf, Vc = np.prod(lv[lf]["h"][:2]), np.prod(lv[lf - 1]["h"][:2])
    for b, q in enumerate(fijk):
        Fi = fine[b][1:N + 1, 1:N + 1]
        off = [(q[d] % 2) * (N // 2) for d in range(2)]
        Ci = coarse[fpar[b]][1 + off[1]:1 + off[1] + N // 2, 1 + off[0]:1 + off[0] + N // 2]
        assert abs(Vf * Fi.sum() - Vc * Ci.sum()) < 1e-14 * Vc * (1 + np.abs(Ci).sum())


# ------------------------------------------------------------- smoother --

@pytest.mark.parametrize("dim", [2, 3])
def test_red_black_sweeps_independent_of_block_size(dim):
    """With ghosts refreshed after each colour and global parity, red-black
    Gauss-Seidel on a uniform level does not depend on how the level is cut
    into blocks."""
    base = 32 if dim == 2 else 16
    rng = np.random.default_rng(2)
    res = []
    for N in (4, 8):
        o = Oracle(dim, N, 0, (DIR, NEU, DIR, DIR, DIR, DIR), (0.3, -0.2, 0, 0, 0, 0),
                   (base,) * dim, (0,) * dim, (1,) * dim)
        p = W.Problem("u", dim, N, 0, (base, base, base if dim == 3 else 1), (0,) * 3, (1,) * 3,
                      (DIR,) * 6, (0,) * 6, np.zeros((0, 4), np.int32))
        I, J, K, _ = W.leaf_cell_index(p)
        key = (K * base + J) * base + I
        vals = rng.standard_normal(base ** dim) if N == 4 else vals0
        fvals = np.sin(np.arange(base ** dim)) if N == 4 else fvals0
        vals0, fvals0 = vals, fvals
        o.set_phi(vals[key])
        o.set_rhs(fvals[key])
        lf = len(o.levels()) - 1
        for _ in range(3):
            o.step("smooth", lf, 0)
            o.step("smooth", lf, 1)
        out = np.empty(base ** dim)
        out[key] = o.get_phi()
        res.append(out)
    np.testing.assert_array_equal(res[0], res[1])


# ------------------------------------------------- composite dense solve --

def _dense(o):
    n = o.n_leaf
    b = o.apply(np.zeros(n))
    A = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = o.apply(e) - b
    return A, b


DENSE_CASES = {
    "2d_amr_dir_eps": dict(dim=2, N=4, base=8, bct=(DIR, DIR, NEU, DIR, 0, 0), radii=(0.3,), eps=True),
    "3d_amr_dir": dict(dim=3, N=2, base=4, bct=(DIR,) * 6, radii=(0.4,), eps=False),
    "3d_amr_dir_eps": dict(dim=3, N=4, base=8, bct=(DIR, NEU, DIR, DIR, DIR, DIR), radii=(0.3,), eps=True),
    "cyl_amr_eps": dict(dim=2, N=4, base=8, bct=(AXIS, DIR, DIR, DIR, 0, 0), radii=(0.3,), eps=True, geom=1),
    "2d_amr_periodic": dict(dim=2, N=4, base=8, bct=(PER, PER, PER, PER, 0, 0), radii=(0.3,), eps=False),
}


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_composite_operator_is_conservative(dim):
    """Constant coefficient, periodic, refined mesh: A 1 = 0 and, by the
    flux-matching ghosts of Sec. 2.6, sum_i V_i (A x)_i = 0 for every x."""
    N, base = 4, (8 if dim == 2 else 8)
    per = (True, True, True)
    ref = amr_refine(dim, N, base, (0.35, 0.6, 0.5), (0.3 if dim == 2 else 0.45,), per)
    assert len(ref) > 0
    o = Oracle(dim, N, 0, (PER,) * 6, (0.0,) * 6, (base,) * dim, (0,) * dim, (1,) * dim, ref)
    vol, _ = o.leaf_geometry()
    assert np.abs(o.apply(np.ones(o.n_leaf))).max() < 1e-10
    x = np.random.default_rng(4).standard_normal(o.n_leaf)
    Ax = o.apply(x)
    assert abs(np.dot(vol, Ax)) < 1e-12 * np.dot(vol, np.abs(Ax))


@pytest.mark.parametrize("case", sorted(DENSE_CASES))
def test_vcycles_converge_to_dense_composite_solution(case):
    """The V-cycle fixed point is the solution of the composite system
    assembled column by column and solved by dense LU (numpy)."""
    c = DENSE_CASES[case]
    dim, N, base = c["dim"], c["N"], c["base"]
    per = tuple(c["bct"][2 * d] == PER for d in range(3))
    ref = amr_refine(dim, N, base, (0.35, 0.6, 0.5), c["radii"], per)
    rng = np.random.default_rng(17)
    o = Oracle(dim, N, c.get("geom", 0), c["bct"], (0.5, -0.25, 1.0, 0.0, 0.3, 0.0),
               (base,) * dim, (0,) * dim, (1,) * dim, ref)
    if c["eps"]:
        o.set_eps(np.exp(0.5 * rng.standard_normal(o.n_leaf)))
    f = rng.standard_normal(o.n_leaf)
    A, b = _dense(o)
    vol, _ = o.leaf_geometry()
    if case.endswith("periodic"):
        # singular: project f to the range, pick the zero-mean solution
        f = f - np.dot(vol, f) / vol.sum()
        M = np.block([[A, np.ones((o.n_leaf, 1))], [vol[None, :], np.zeros((1, 1))]])
        x_ref = np.linalg.solve(M, np.concatenate([f - b, [0.0]]))[:-1]
    else:
        x_ref = np.linalg.solve(A, f - b)
    o.set_rhs(f)
    o.set_phi(np.zeros(o.n_leaf))
    o.fmg()
    o.vcycle(40)
    x = o.get_phi()
    if case.endswith("periodic"):
        x = x - np.dot(vol, x) / vol.sum()
    np.testing.assert_allclose(x, x_ref, rtol=0, atol=1e-11 * np.abs(x_ref).max())


@pytest.mark.parametrize("dim,omega", [(2, 0.8), (3, 2.0 / 3.0)])
def test_jacobi_damps_the_checkerboard_by_one_minus_two_omega(dim, omega):
    """Weighted Jacobi (reading R13) computes every cell from the values
    before the step: on a uniform periodic grid the checkerboard
    (-1)^(I+J+K) is an eigenvector of one step with factor 1 - 2 omega for
    any spacing (each neighbour is -x_c, so the local solution is -x_c).
    A Gauss-Seidel update or a missing weight gives another factor."""
    N, base = 4, 8
    h = (1.0, 0.5, 2.0)[:dim]  # anisotropic cells
    o = Oracle(dim, N, 0, (PER,) * 6, (0.0,) * 6, (base,) * dim, (0,) * dim, h, np.zeros((0, 4), np.int32))
    o.set_smoother(jacobi=True, omega=omega)
    top = len(o.levels()) - 1
    n = o.levels()[top]["n"]
    ijk, _, _ = o.level_blocks(top)
    x = np.zeros_like(o.level_get(top, "phi"))
    for b in range(x.shape[0]):
        idx = np.indices((n,) * dim)
        par = sum(ijk[b, d] * n + idx[::-1][d] for d in range(dim)) % 2
        x[b][(slice(1, n + 1),) * dim] = 1.0 - 2.0 * par
    o.level_set(top, "phi", x)
    o.level_set(top, "f", np.zeros_like(x))
    o.step("ghost", top)
    before = o.level_get(top, "phi")
    o.step("jacobi", top)
    after = o.level_get(top, "phi")
    inner = (slice(None),) + (slice(1, n + 1),) * dim
    np.testing.assert_allclose(after[inner], (1.0 - 2.0 * omega) * before[inner], rtol=0, atol=1e-14)


@pytest.mark.parametrize("case", ["2d_amr_dir_eps", "3d_amr_dir_eps", "cyl_amr_eps"])
def test_jacobi_vcycles_converge_to_dense_composite_solution(case):
    """V-cycles with the Jacobi smoother reach the same composite solution
    (dense LU of the system assembled column by column)."""
    c = DENSE_CASES[case]
    dim, N, base = c["dim"], c["N"], c["base"]
    ref = amr_refine(dim, N, base, (0.35, 0.6, 0.5), c["radii"])
    rng = np.random.default_rng(23)
    o = Oracle(dim, N, c.get("geom", 0), c["bct"], (0.5, -0.25, 1.0, 0.0, 0.3, 0.0),
               (base,) * dim, (0,) * dim, (1,) * dim, ref)
    o.set_eps(np.exp(0.5 * rng.standard_normal(o.n_leaf)))
    f = rng.standard_normal(o.n_leaf)
    A, b = _dense(o)
    x_ref = np.linalg.solve(A, f - b)
    o.set_smoother(jacobi=True)
    o.set_rhs(f)
    o.set_phi(np.zeros(o.n_leaf))
    o.fmg()
    o.vcycle(60)
    np.testing.assert_allclose(o.get_phi(), x_ref, rtol=0, atol=1e-10 * np.abs(x_ref).max())


# --------------------------------------------------------- convergence ----

def test_second_order_convergence_2d():
    """Second-order discretisation (Sec. 2.2): the error of the converged
    solution falls about 4x per halving of h (cfg-1 manufactured problem)."""
    errs = []
    for n in (32, 64, 128):
        p = W.cfg1_poisson2d(n=n, N=8)
        o = Oracle.from_problem(p)
        o.solve(1e-11)
        X, Y, Z, _ = W.leaf_cell_centres(p)
        errs.append(np.abs(o.get_phi() - p.exact(X, Y, Z)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.5 and 3.5 < r2 < 4.6, errs


@pytest.mark.slow
def test_paper_convergence_problem_3d():
    """Sec. 3.1 (E1) at 32^3: the residual reaches machine precision after
    about ten FMG cycles, the discretisation error after one or two, and a
    centred two-level refinement lowers the max error by about 16-20x."""
    p = W.conv3d_problem(n=32, N=8, refine="none")
    o = Oracle.from_problem(p)
    X, Y, Z, _ = W.leaf_cell_centres(p)
    r0 = o.residual_norm()[0]
    errs, res = [], []
    for _ in range(10):
        o.fmg()
        res.append(o.residual_norm()[0] / r0)
        errs.append(np.abs(o.get_phi() - p.exact(X, Y, Z)).max())
    assert res[-1] < 1e-12, res
    assert abs(errs[1] - errs[-1]) < 0.05 * errs[-1]
    pc = W.conv3d_problem(n=32, N=8, refine="center")
    oc = Oracle.from_problem(pc)
    for _ in range(6):
        oc.fmg()
    Xc, Yc, Zc, _ = W.leaf_cell_centres(pc)
    err_c = np.abs(oc.get_phi() - pc.exact(Xc, Yc, Zc)).max()
    assert errs[-1] / err_c > 10.0, (errs[-1], err_c)


def test_gaussian_closed_form_second_order():
    """Sec. 3.2 closed form erf(r/s)/(4 pi r) as a Dirichlet problem: second
    order convergence of the max error."""
    errs = []
    for n in (16, 32):
        p = W.cfg2_gauss3d(base=n, N=8, radii=(), sigma=0.1)
        o = Oracle.from_problem(p)
        o.solve(1e-10)
        X, Y, Z, _ = W.leaf_cell_centres(p)
        errs.append(np.abs(o.get_phi() - p.exact(X, Y, Z)).max())
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_cylindrical_second_order():
    """Cylindrical (r, z) form: phi = (1 - r^2) sin(pi z) with the axis at r = 0
    converges at second order."""
    def phi(X, Y, Z):
        return (1 - X * X) * np.sin(math.pi * Y)

    def rhs(X, Y, Z):
        return -4 * np.sin(math.pi * Y) - (1 - X * X) * math.pi ** 2 * np.sin(math.pi * Y)
    errs = []
    for n in (32, 64):
        p = W.Problem("cyl", 2, 8, W.GEOM_CYL, (n, n, 1), (0, 0, 0), (1, 1, 1),
                      (AXIS, DIR, DIR, DIR, PER, PER), (0.0,) * 6, np.zeros((0, 4), np.int32),
                      512, rhs=rhs, exact=phi)
        o = Oracle.from_problem(p)
        o.solve(1e-11)
        X, Y, Z, _ = W.leaf_cell_centres(p)
        errs.append(np.abs(o.get_phi() - phi(X, Y, Z)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


# -------------------------------------------------------------- adjoint ----

def _adjoint_case(case):
    rng = np.random.default_rng(23)
    if case == "2d":
        o = Oracle(2, 4, 0, (DIR, NEU, DIR, DIR, 0, 0), (0.2, 0.1, -0.3, 0.0, 0, 0), (8, 8), (0, 0), (1, 1))
    elif case == "3d":
        o = Oracle(3, 4, 0, (NEU, NEU, PER, PER, DIR, DIR), (0.1, 0.0, 0, 0, 0.5, 0.0), (8, 8, 8), (0,) * 3, (1,) * 3)
    else:
        o = Oracle(2, 4, 1, (AXIS, DIR, DIR, DIR, 0, 0), (0, 0.4, 0, 0.1, 0, 0), (8, 8), (0, 0), (1, 1))
    eps = np.exp(0.4 * rng.standard_normal(o.n_leaf))
    f = rng.standard_normal(o.n_leaf)
    t = rng.standard_normal(o.n_leaf)
    return o, eps, f, t


def _solve_exact(o, eps, f):
    o.set_eps(eps)
    o.set_rhs(f)
    o.set_phi(np.zeros(o.n_leaf))
    o.fmg()
    o.vcycle(30)
    return o.get_phi()


@pytest.mark.parametrize("case", ["2d", "3d", "cyl"])
def test_adjoint_matches_finite_differences(case):
    """dL/df = lambda = A^-T dL/dphi and dL/deps from the face coefficients,
    for L = 0.5 sum (phi - t)^2: central differences (exact for f since L is
    quadratic in f; O(delta^2) for eps)."""
    o, eps, f, t = _adjoint_case(case)
    phi = _solve_exact(o, eps, f)
    lam, geps = o.adjoint(phi - t, n_vcycles=30)

    def loss(e, ff):
        x = _solve_exact(o, e, ff)
        return 0.5 * np.sum((x - t) ** 2)
    rng = np.random.default_rng(1)
    for c in rng.choice(o.n_leaf, 6, replace=False):
        df = np.zeros(o.n_leaf)
        df[c] = 1e-3
        fd = (loss(eps, f + df) - loss(eps, f - df)) / 2e-3
        assert abs(fd - lam[c]) < 1e-7 * (abs(lam[c]) + np.abs(lam).max() * 1e-3)
        de = np.zeros(o.n_leaf)
        de[c] = 1e-4 * eps[c]
        fe = (loss(eps + de, f) - loss(eps - de, f)) / (2e-4 * eps[c])
        assert abs(fe - geps[c]) < 1e-6 * (abs(geps[c]) + np.abs(geps).max() * 1e-2), (c, fe, geps[c])


# ---------------------------------------------------- divergence cleaning --

def test_divergence_and_gradient_exact_on_linear_fields():
    """Sec. 4.1 central differences with the Sec. 2.6 ghosts: exact for linear
    fields on every cell not beside a physical face (refinement faces
    included, since the ghosts are exact on linear functions)."""
    dim, N, base = 3, 4, 16
    ref = amr_refine(dim, N, base, (0.45, 0.5, 0.55), (0.3, 0.15))
    o = Oracle(dim, N, 0, (0, 1, 0, 0, 1, 0), (0.0,) * 6, (base,) * 3, (0,) * 3, (1,) * 3, ref)
    p = W.Problem("lin", dim, N, 0, (base,) * 3, (0,) * 3, (1,) * 3, (0,) * 6, (0,) * 6, ref)
    X, Y, Z, H = W.leaf_cell_centres(p)
    B = np.stack([0.3 * X - Y + 2 * Z, 1.5 * Y + X, -0.7 * Z + 0.2 * X * 0 + Y])
    d = o.divergence(B)
    h = H[:, 0]
    inner = (X > h) & (X < 1 - h) & (Y > h) & (Y < 1 - h) & (Z > h) & (Z < 1 - h)
    np.testing.assert_allclose(d[inner], 0.3 + 1.5 - 0.7, atol=1e-11)
    o.set_phi(2 * X - 3 * Y + 0.5 * Z)
    Bn = o.project(np.zeros((3, o.n_leaf)))
    for comp, want in zip(Bn, (-2.0, 3.0, -0.5)):
        np.testing.assert_allclose(comp[inner], want, atol=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
def test_fourth_order_divergence_on_cubics(dim):
    """The fourth-order difference of Sec. 4.1 is exact on cubics; where a
    cell two away lies beyond a physical face the second-order difference is
    used (reading R14), whose error on x^3 is exactly h^2 (one cell from the
    face; the boundary cell itself depends on the ghost rule)."""
    N, base = 4, 16
    o = Oracle(dim, N, 0, (0,) * 6, (0.0,) * 6, (base,) * dim, (0,) * dim, (1,) * dim, np.zeros((0, 4), np.int32))
    p = W.Problem("cub", dim, N, 0, (base,) * dim + (1,) * (3 - dim), (0,) * 3, (1,) * 3, (0,) * 6, (0,) * 6,
                  np.zeros((0, 4), np.int32))
    X, Y, Z, H = W.leaf_cell_centres(p)
    coords = [X, Y, Z][:dim]
    B = np.stack([c ** 3 for c in coords])
    div = o.divergence(B, order=4)
    h = 1.0 / base
    idx = [np.rint(c / h - 0.5).astype(int) for c in coords]
    interior = np.all([(I >= 1) & (I <= base - 2) for I in idx], axis=0)
    want = np.zeros(o.n_leaf)
    for c, I in zip(coords, idx):
        near = (I == 1) | (I == base - 2)
        want += 3 * c ** 2 + np.where(near, h * h, 0.0)
    np.testing.assert_allclose(div[interior], want[interior], rtol=0, atol=1e-10)
    assert (np.abs(div[interior] - sum(3 * c ** 2 for c in coords)[interior]) > 0.5 * h * h).any()


def test_fourth_order_divergence_converges_at_fourth_order():
    """Smooth field on a uniform periodic mesh (every cell takes the
    fourth-order form): the error falls ~16x when h halves."""
    errs = []
    for base in (16, 32):
        dim, N = 2, 4
        o = Oracle(dim, N, 0, (PER,) * 6, (0.0,) * 6, (base, base), (0, 0), (1, 1), np.zeros((0, 4), np.int32))
        p = W.Problem("s", dim, N, 0, (base, base, 1), (0,) * 3, (1,) * 3, (PER,) * 6, (0,) * 6,
                      np.zeros((0, 4), np.int32))
        X, Y, Z, H = W.leaf_cell_centres(p)
        k = 2 * math.pi
        B = np.stack([np.sin(k * X) * np.cos(k * Y), np.cos(k * X + 0.3) * np.sin(k * Y)])
        exact = k * np.cos(k * X) * np.cos(k * Y) + k * np.cos(k * X + 0.3) * np.cos(k * Y)
        errs.append(np.abs(o.divergence(B, order=4) - exact).max())
    assert errs[0] / errs[1] > 12, errs


def test_central_divergence_is_minus_adjoint_of_gradient_periodic():
    """On a uniform periodic mesh the central divergence and gradient satisfy
    <u, D B> = -<G u, B> (summation by parts)."""
    rng = np.random.default_rng(9)
    o = Oracle(3, 4, 0, (2,) * 6, (0.0,) * 6, (8, 8, 8), (0,) * 3, (1,) * 3)
    u = rng.standard_normal(o.n_leaf)
    B = rng.standard_normal((3, o.n_leaf))
    o.set_phi(u)
    Gu = -o.project(np.zeros((3, o.n_leaf)))
    a, b = np.dot(u, o.divergence(B)), -np.sum(Gu * B)
    assert abs(a - b) < 1e-12 * (abs(a) + np.abs(u).sum())


def test_divergence_second_order_periodic():
    """Second-order convergence of the central divergence on a smooth field."""
    errs = []
    for n in (16, 32):
        o = Oracle(3, 8, 0, (2,) * 6, (0.0,) * 6, (n,) * 3, (0,) * 3, (1,) * 3)
        p = W.Problem("u", 3, 8, 0, (n,) * 3, (0,) * 3, (1,) * 3, (2,) * 6, (0,) * 6, np.zeros((0, 4), np.int32))
        X, Y, Z, _ = W.leaf_cell_centres(p)
        B = np.stack([np.sin(2 * np.pi * X), np.cos(2 * np.pi * Y), np.sin(2 * np.pi * Z)])
        ex = 2 * np.pi * (np.cos(2 * np.pi * X) - np.sin(2 * np.pi * Y) + np.cos(2 * np.pi * Z))
        errs.append(np.abs(o.divergence(B) - ex).max())
    assert 3.6 < errs[0] / errs[1] < 4.4, errs


def test_cleaning_adjoint_is_the_cleaning_of_g_periodic():
    """On a uniform periodic mesh B_new = B - G A^+ P D B is a self-adjoint
    map (G^T = -D, A^+ and the mean projection P symmetric), so for
    L = 0.5 sum |B_new - B_t|^2 the gradient is clean(B_new - B_t); central
    differences of L agree (L is quadratic in B)."""
    rng = np.random.default_rng(12)
    o = Oracle(3, 4, 0, (2,) * 6, (0.0,) * 6, (8, 8, 8), (0,) * 3, (1,) * 3)
    B = rng.standard_normal((3, o.n_leaf))
    Bt = rng.standard_normal((3, o.n_leaf))

    def loss(Bx):
        Bn, _, _ = o.clean(Bx, rel_tol=1e-14, max_cycles=80)
        return 0.5 * np.sum((Bn - Bt) ** 2), Bn
    L0, Bn = loss(B)
    grad, _, _ = o.clean(Bn - Bt, rel_tol=1e-14, max_cycles=80)
    for comp, c in ((0, 5), (1, 77), (2, 300), (0, 411)):
        dB = np.zeros_like(B)
        dB[comp, c] = 1e-3
        fd = (loss(B + dB)[0] - loss(B - dB)[0]) / 2e-3
        assert abs(fd - grad[comp, c]) < 1e-7 * (abs(grad[comp, c]) + np.abs(grad).max() * 1e-3), (fd, grad[comp, c])


@pytest.mark.parametrize("dim", [2, 3])
def test_helmholtz_term_is_minus_lambda_phi(dim):
    """The Helmholtz form of Sec. 2.2, div(eps grad phi) - lambda phi: on the
    same refined mesh the operators with lambda and without differ by
    exactly -lambda x on every leaf cell (boundary and refinement ghosts do
    not involve lambda)."""
    N, base, lam = 4, 8, 2.5
    ref = amr_refine(dim, N, base, (0.35, 0.6, 0.5), (0.3 if dim == 2 else 0.45,), (False,) * 3)
    assert len(ref) > 0
    bct = (DIR, NEU, DIR, DIR, NEU, DIR)
    args = (dim, N, 0, bct, (0.5, -0.25, 1.0, 0.0, 0.3, 0.0), (base,) * dim, (0,) * dim, (1,) * dim, ref)
    o0, o1 = Oracle(*args), Oracle(*args, helm=lam)
    x = np.random.default_rng(8).standard_normal(o0.n_leaf)
    d = o1.apply(x) - o0.apply(x)
    np.testing.assert_allclose(d, -lam * x, rtol=0, atol=1e-12 * np.abs(o0.apply(x)).max())


@pytest.mark.parametrize("bct", [(DIR, DIR, NEU, DIR, 0, 0), (NEU, NEU, NEU, NEU, 0, 0)])
def test_helmholtz_vcycles_converge_to_dense_solution(bct):
    """With lambda > 0 the V-cycle fixed point is the dense composite
    solution, also for an all-Neumann mesh, which lambda makes regular."""
    dim, N, base, lam = 2, 4, 8, 3.0
    ref = amr_refine(dim, N, base, (0.35, 0.6, 0.5), (0.3,), (False,) * 3)
    o = Oracle(dim, N, 0, bct, (0.5, -0.25, 1.0, 0.0, 0.0, 0.0), (base,) * dim, (0,) * dim, (1,) * dim, ref,
               helm=lam)
    f = np.random.default_rng(19).standard_normal(o.n_leaf)
    A, b = _dense(o)
    x_ref = np.linalg.solve(A, f - b)
    o.set_rhs(f)
    o.set_phi(np.zeros(o.n_leaf))
    o.fmg()
    o.vcycle(40)
    np.testing.assert_allclose(o.get_phi(), x_ref, rtol=0, atol=1e-11 * np.abs(x_ref).max())


def test_per_level_schedule():
    """N_down / N_up per level (Sec. 2.4 fixes one pair for all levels): a
    schedule repeating set_cycle's pair is the same cycle bit for bit, a
    uniform (1, 3) schedule equals set_cycle(1, 3), and a mixed schedule
    still converges to the composite solution of the dense LU."""
    p = W.cfg2_gauss3d(base=16, N=4, radii=(0.3,), sigma=0.1)

    def run(setup):
        o = Oracle.from_problem(p)
        setup(o)
        o.fmg()
        o.vcycle(2)
        return o.get_phi()

    nl = len(Oracle.from_problem(p).levels())
    base = run(lambda o: None)
    assert np.array_equal(base, run(lambda o: o.set_schedule([2] * nl, [2] * nl)))
    a = run(lambda o: o.set_cycle(1, 3))
    b = run(lambda o: o.set_schedule([1] * nl, [3] * nl))
    assert np.array_equal(a, b) and not np.array_equal(a, base)
    mixed = ([-1] + [1, 3, 2, 1][: nl - 1] + [2] * max(0, nl - 5), [-1] + [3, 1, 2, 2][: nl - 1] + [1] * max(0, nl - 5))
    o = Oracle.from_problem(p)
    o.set_schedule(*mixed)
    cyc, hist = o.solve(1e-12, 60)
    assert hist[-1] <= 1e-12 * hist[0]


def test_paper_coarse_solve_reaches_the_composite_solution():
    """The paper's coarse-grid solve (Sec. 2.4: smoothing sweeps on the
    coarsest level to an absolute or relative threshold, reading R20) in
    place of the exact one: the V-cycles still converge to the dense
    composite solution (2D Dirichlet, 3D refined, a singular variable-eps
    problem with its zero-mean solution); with max_it = 0 the coarsest
    level is left as it was, so the cycles stall."""
    cases = [W.cfg1_poisson2d(n=32, N=8), W.cfg2_gauss3d(base=16, N=4, radii=(0.3,), sigma=0.1),
             W.cfg3_varcoef3d(n=16, N=4, contrast=10.0)]
    for p in cases:
        exact = Oracle.from_problem(p)
        exact.solve(1e-13, 80)
        o = Oracle.from_problem(p)
        o.set_coarse_mode(True)
        cyc, hist = o.solve(1e-12, 80)
        assert hist[-1] <= 1e-12 * hist[0], (p.name, cyc)
        x, xr = o.get_phi(), exact.get_phi()
        assert np.abs(x - xr).max() <= 1e-9 * np.abs(xr).max(), p.name
    o = Oracle.from_problem(cases[0])
    o.set_coarse_mode(True, max_it=0)
    o.fmg()
    o.vcycle(6)
    r, _ = o.residual_norm()
    r0 = Oracle.from_problem(cases[0]).residual_norm()[0]
    assert r > 1e-4 * r0
