"""Batches of independent trees (one launch per segment over all trees)
against the FP64 oracle run tree by tree.  A batch runs every tree's own
cycle (Sec. 2.4) side by side, so after the same cycles each tree's slice of
the batch matches the oracle's single-tree result to rounding:
max |phi_batch - phi_oracle| <= 1e-12 max |phi_oracle| per tree."""
import numpy as np
import pytest

from oracle import Oracle
from synth import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def mg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_11370_gb300 import build as B
    B.build()
    import paper_1901_11370_gb300 as m
    return m


def _cart2d(name, n, N, hi=(1.0, 1.0), refine=None, c=(0.3, 0.6)):
    """2D Cartesian Dirichlet problem, boundary values x + 2y - xy."""
    ref = np.zeros((0, 4), np.int32) if refine is None else \
        W.refine_spheres(2, N, n + (1,), (0, 0, 0), hi + (1.0,), c + (0.0,), refine)
    return W.Problem(name, 2, N, W.GEOM_CART, n + (1,), (0.0, 0.0, 0.0), hi + (1.0,), (W.BC_DIRICHLET,) * 6,
                     (0.0,) * 6, ref, 512,
                     rhs=lambda X, Y, Z: np.exp(-20 * ((X - c[0]) ** 2 + (Y - c[1]) ** 2)) - 0.3,
                     eps=lambda X, Y, Z: 1.0 + 0.4 * np.cos(3 * X + Y),
                     bc=lambda face, X, Y, Z: X + 2 * Y - X * Y)


def forests():
    return {
        # cylindrical (r, z) ring trees of different sizes and depths
        "cyl": [W.cyl_ring_tree(s, force_k=k) for s, k in ((21, 2), (22, 3), (23, 4), (24, 5), (25, 6), (26, 3))],
        # mixed block sizes, spacings, single-level and refined trees
        "cart2d": [_cart2d("u64", (64, 64), 8), _cart2d("b16", (32, 32), 16, refine=(0.25,)),
                   _cart2d("amr", (32, 32), 8, refine=(0.3, 0.15)),
                   _cart2d("wide", (64, 32), 8, hi=(2.0, 1.0), refine=(0.2,), c=(1.3, 0.4)),
                   _cart2d("single", (8, 8), 8), _cart2d("one_ref", (8, 8), 8, refine=(0.9,)),
                   _cart2d("strip", (32, 16), 8)],
        "gauss3d": [W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15), sigma=0.05),
                    W.cfg2_gauss3d(base=16, N=8, seed=1, radii=(0.3,), sigma=0.08),
                    W.cfg2_gauss3d(base=16, N=4, seed=2, radii=(0.25,), sigma=0.06)],
        "periodic3d": [W.cfg3_varcoef3d(n=32, N=8, contrast=10.0), W.cfg3_varcoef3d(n=16, N=8, seed=1, contrast=5.0),
                       W.cfg3_varcoef3d(n=32, N=16, seed=2, contrast=10.0)],
    }


FORESTS = forests()


def make_batch(mg, probs):
    import torch
    trees = [mg.Tree.from_problem(p, finalize=False) for p in probs]
    b = mg.Batch(trees)
    if any(p.eps is not None or p.eps_leaf is not None for p in probs):
        b.set_eps(torch.from_numpy(np.concatenate([W.leaf_field(p, "eps") for p in probs])).cuda())
    b.set_rhs(torch.from_numpy(np.concatenate([W.leaf_field(p, "rhs") for p in probs])).cuda())
    return b


def rel_diff(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name", sorted(FORESTS))
def test_batch_fmg_and_vcycles_match_oracle_per_tree(mg, name):
    probs = FORESTS[name]
    b = make_batch(mg, probs)
    assert list(np.diff(b.offsets)) == [W.n_leaf_cells(p) for p in probs]
    b.fmg()
    phi1 = b.get_phi().cpu().numpy()
    b.vcycle(3)
    phi2 = b.get_phi().cpu().numpy()
    l2, li = b.residual_norms()
    for i, p in enumerate(probs):
        o = Oracle.from_problem(p)
        s = slice(b.offsets[i], b.offsets[i + 1])
        o.fmg()
        d1 = rel_diff(phi1[s], o.get_phi())
        o.vcycle(3)
        d2 = rel_diff(phi2[s], o.get_phi())
        assert d1 < TOL and d2 < TOL, (p.name, d1, d2)
        # per-tree norms: the batch's phi differs by dphi, so its residual by
        # at most |A| dphi (|A| <= 4 D eps_max / h_min^2) plus rounding of f - A phi
        l2o, lio = o.residual_norm()
        X, Y, Z, H = W.leaf_cell_centres(p)
        emax = np.abs(W.leaf_field(p, "eps")).max()
        dphi = np.abs(phi2[s] - o.get_phi()).max()
        bound = 2 * (4 * p.dim * emax / H[:, :p.dim].min() ** 2) * (dphi + 1e-15 * np.abs(o.get_phi()).max()) \
            + 1e-13 * (np.abs(W.leaf_field(p, "rhs")).max() + 1.0)
        assert abs(l2[i] - l2o) <= bound + 1e-12 * l2o and abs(li[i] - lio) <= bound + 1e-12 * lio, (p.name,)


def test_batch_segments_cover_every_tree(mg):
    """Segments: one block size each, grouped from the top; blocks of all
    trees accounted for, and fewer launch units than trees x levels."""
    probs = FORESTS["cart2d"]
    b = make_batch(mg, probs)
    seg = b.segments()
    n_blocks = sum(s["nb"] for s in seg)
    want = 0
    levels = 0
    for p in probs:
        o = Oracle.from_problem(p, set_fields=False)
        want += sum(l["nb"] for l in o.levels())
        levels += len(o.levels())
    assert n_blocks == want
    assert len(seg) < levels
    top = max(s["group"] for s in seg)
    assert {s["group"] for s in seg} == set(range(top + 1))


@pytest.mark.parametrize("name", ["cyl", "gauss3d", "periodic3d"])
def test_batch_solve_fp64_matches_oracle_cycles(mg, name):
    """FP64 batch solve: every tree below rel_tol; each tree's phi equals the
    oracle's after the same number of cycles (FMG, then V-cycles)."""
    probs = FORESTS[name]
    b = make_batch(mg, probs)
    cyc, rel = b.solve(1e-10, 40)
    assert (rel <= 1e-10).all()
    phi = b.get_phi().cpu().numpy()
    for i, p in enumerate(probs):
        o = Oracle.from_problem(p)
        o.fmg()
        o.vcycle(cyc - 1)
        s = slice(b.offsets[i], b.offsets[i + 1])
        assert rel_diff(phi[s], o.get_phi()) < TOL, p.name


@pytest.mark.parametrize("name", ["cyl", "cart2d", "gauss3d"])
def test_batch_solve_mixed_precision_residual_by_oracle(mg, name):
    """FP32 smoothing with FP64 defect correction: the oracle's composite
    residual of each tree's returned phi is below the tolerance (relative to
    the oracle's residual of phi = 0)."""
    import torch  # noqa: F401
    probs = FORESTS[name]
    b = make_batch(mg, probs)
    cyc, rel = b.solve(1e-9, 40, precision=mg.MG_FP32_DC)
    assert (rel <= 1e-9).all()
    phi = b.get_phi().cpu().numpy()
    for i, p in enumerate(probs):
        o = Oracle.from_problem(p)
        r0, _ = o.residual_norm()
        o.set_phi(phi[b.offsets[i]:b.offsets[i + 1]])
        r, _ = o.residual_norm()
        assert r <= 1.05e-9 * r0, (p.name, r / r0)


def test_batch_of_one_equals_single_tree(mg):
    import torch
    p = FORESTS["gauss3d"][0]
    b = make_batch(mg, [p])
    t = mg.Tree.from_problem(p)
    b.fmg(); t.fmg()
    b.vcycle(2); t.vcycle(2)
    assert rel_diff(b.get_phi().cpu().numpy(), t.get_phi().cpu().numpy()) < TOL
    x = torch.from_numpy(np.random.default_rng(1).standard_normal(t.n_leaf)).cuda()
    b.set_phi(x)
    assert torch.equal(b.get_phi(), x)


def test_batch_launches_do_not_grow_with_trees(mg):
    """One V-cycle of 24 trees launches no more kernels than one of 6 trees
    with the same level structure (launches per segment, not per tree)."""
    few = [W.cyl_ring_tree(s, force_k=4) for s in (31, 32)]
    many = [W.cyl_ring_tree(s, force_k=4) for s in range(31, 55)]

    def per_cycle(probs):
        b = make_batch(mg, probs)
        b.vcycle(1)
        n0 = b.launch_count()
        b.vcycle(2)
        return (b.launch_count() - n0) / 2, len(b.segments())

    l_few, s_few = per_cycle(few)
    l_many, s_many = per_cycle(many)
    assert s_many == s_few or l_many <= l_few * s_many / s_few
    assert l_many < 24 * l_few / 2


def test_batch_rejects_mismatched_trees(mg):
    p1 = FORESTS["cart2d"][0]
    p2 = W.cyl_ring_tree(40, force_k=2)
    with pytest.raises(mg.MGError):
        mg.Batch([mg.Tree.from_problem(p1, finalize=False), mg.Tree.from_problem(p2, finalize=False)])


def test_batch_jacobi_matches_oracle_per_tree(mg):
    """The Jacobi smoother in a batch: every tree matches the oracle's
    Jacobi cycles."""
    probs = FORESTS["cyl"]
    b = make_batch(mg, probs)
    b.fmg(smoother=mg.MG_SMOOTH_JACOBI)
    b.vcycle(2, smoother=mg.MG_SMOOTH_JACOBI)
    phi = b.get_phi().cpu().numpy()
    for i, p in enumerate(probs):
        o = Oracle.from_problem(p)
        o.set_smoother(jacobi=True)
        o.fmg()
        o.vcycle(2)
        assert rel_diff(phi[b.offsets[i]:b.offsets[i + 1]], o.get_phi()) < TOL, p.name


@pytest.mark.parametrize("name", ["cyl", "cart2d", "gauss3d"])
def test_batch_mixed_precision_converges_like_fp64(mg, name):
    """The FP32 cycles (their own restriction and prolongation kernels) cut
    the residual per cycle as the FP64 cycles do: the defect-correction
    solve needs at most one cycle more than the FP64 solve.  A wrong weight
    or side in an FP32 transfer would slow it down well beyond that."""
    probs = FORESTS[name]
    b = make_batch(mg, probs)
    c64, _ = b.solve(1e-10, 40)
    import torch
    b.set_phi(torch.zeros(b.n_leaf, dtype=torch.float64, device="cuda"))
    c32, rel = b.solve(1e-10, 40, precision=mg.MG_FP32_DC)
    assert (rel <= 1e-10).all() and c32 <= c64 + 1, (c32, c64)


@pytest.mark.parametrize("name", ["cyl", "periodic3d"])
def test_batch_paper_coarse_solve_matches_oracle_per_tree(mg, name):
    """The paper's coarse-grid smoothing (one CTA per tree's coarsest level)
    in a batch: every tree matches the oracle run with the same coarse solve."""
    probs = FORESTS[name]
    b = make_batch(mg, probs)
    b.fmg(coarse_mode=mg.MG_COARSE_SMOOTH)
    b.vcycle(2, coarse_mode=mg.MG_COARSE_SMOOTH)
    phi = b.get_phi().cpu().numpy()
    for i, p in enumerate(probs):
        o = Oracle.from_problem(p)
        o.set_coarse_mode(True)
        o.fmg()
        o.vcycle(2)
        d = rel_diff(phi[b.offsets[i]:b.offsets[i + 1]], o.get_phi())
        assert d < TOL, (p.name, d)


def test_batch_coarse_forms(mg):
    """Dirichlet trees of a batch take the block-tridiagonal coarsest solve
    (2 nc P values against nc^2 for the dense inverse); the periodic,
    singular trees keep the dense inverse; a batch of one keeps it too.
    Parity of both forms is the per-tree oracle comparison above."""
    cyl = make_batch(mg, FORESTS["cyl"]).coarse_info()
    assert cyl["dense"] == 0 and cyl["block"] == len(FORESTS["cyl"]) and cyl["dense_bytes"] == 0
    per = make_batch(mg, FORESTS["periodic3d"]).coarse_info()
    assert per["block"] == 0 and per["dense"] == len(FORESTS["periodic3d"])
    one = make_batch(mg, FORESTS["cyl"][:1]).coarse_info()
    assert one["block"] == 0 and one["dense"] == 1
    # the 31 x 31 coarsest level of a k = 31 tree: 31 planes of 31 cells
    big = make_batch(mg, [W.cyl_ring_tree(7, force_k=31), W.cyl_ring_tree(8, force_k=31)]).coarse_info()
    nc, P = 31 * 31, 31
    stride = (P * P + 2 * P + 1) & ~1  # plane record: S_j^-1, two couplings, padded to even
    assert big["block"] == 2 and big["block_bytes"] == 2 * 31 * stride * 8
    assert 2 * nc * nc * 8 >= 10 * big["block_bytes"]


def test_batch_block_coarse_solve_matches_dense(mg):
    """The block-tridiagonal coarsest solve of a tree equals the dense one of
    the same tree run alone (a batch of one) after FMG and V-cycles, to
    rounding, for large and small coarsest levels."""
    probs = [W.cyl_ring_tree(7, force_k=31), W.cyl_ring_tree(9, force_k=5), W.cyl_ring_tree(10, force_k=17)]
    b = make_batch(mg, probs)
    assert b.coarse_info()["block"] == 3
    b.fmg()
    b.vcycle(2)
    phi = b.get_phi().cpu().numpy()
    for i, p in enumerate(probs):
        one = make_batch(mg, [p])
        one.fmg()
        one.vcycle(2)
        s = slice(b.offsets[i], b.offsets[i + 1])
        assert rel_diff(phi[s], one.get_phi().cpu().numpy()) < TOL, p.name


def test_batch_schedule_tuner(mg):
    """The batch schedule autotuner keeps a schedule with which every tree
    reaches the tolerance; the tuned solve's phi passes the oracle's
    residual check, and phi is left as it was."""
    import torch
    probs = FORESTS["cyl"]
    b = make_batch(mg, probs)
    x = torch.from_numpy(np.random.default_rng(3).standard_normal(b.n_leaf)).cuda()
    b.set_phi(x)
    inner, ms = b.tune_schedule(1e-9, 60, mg.MG_FP32_DC)
    assert inner in (1, 2, 3, 4) and ms > 0
    assert torch.equal(b.get_phi(), x)
    b.set_phi(torch.zeros_like(x))
    cyc, rel = b.solve(1e-9, 60, precision=mg.MG_FP32_DC, inner_cycles=inner)
    assert (rel <= 1e-9).all()
    phi = b.get_phi().cpu().numpy()
    for i, p in enumerate(probs):
        o = Oracle.from_problem(p)
        r0, _ = o.residual_norm()
        o.set_phi(phi[b.offsets[i]:b.offsets[i + 1]])
        assert o.residual_norm()[0] <= 1.05e-9 * r0, p.name
