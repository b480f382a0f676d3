"""Every red-black sweep kernel variant against the oracle.  The autotuner
picks among several kernels that compute the same half-sweep (Sec. 2.2);
each is pinned here on every level where it applies and checked on its own:
FP64 variants against the oracle after the same cycles (1e-12 relative),
FP32-only variants by the oracle's residual after a defect-correction solve."""
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


CASES = {
    "gauss3d_b8": lambda: W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15), sigma=0.05),
    "poisson2d_b8": lambda: W.cfg1_poisson2d(n=64, N=8),
    "cyl_k5_b16_4": lambda: W.cyl_ring_tree(24, force_k=5),
    "varcoef3d_b16": lambda: W.cfg3_varcoef3d(n=32, N=16, seed=2, contrast=10.0),
    "block2_3d": lambda: W.Problem("b2", 3, 2, 0, (8, 8, 8), (0,) * 3, (1,) * 3, (0, 1, 0, 0, 0, 0),
                                   (0.1, 0.2, 0, 0, 0, 0),
                                   W.refine_spheres(3, 2, (8,) * 3, (0,) * 3, (1,) * 3, (0.5, 0.5, 0.5), (0.3,)), 8,
                                   rhs=lambda X, Y, Z: X * Y - Z),
}


def applied(t, variant, prec):
    return [l for l in range(len(t.levels())) if t.sweep_variant(l, prec) == variant]


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 10])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_variant_matches_oracle(mg, name, variant):
    p = CASES[name]()
    t = mg.Tree.from_problem(p)
    t.set_sweep_variant(variant, precision=mg.MG_FP64)
    if not applied(t, variant, mg.MG_FP64):
        pytest.skip("variant %d applies to no level of %s" % (variant, name))
    o = Oracle.from_problem(p)
    t.fmg(); o.fmg()
    t.vcycle(2); o.vcycle(2)
    phi, ref = t.get_phi().cpu().numpy(), o.get_phi()
    assert np.abs(phi - ref).max() <= TOL * np.abs(ref).max()


@pytest.mark.parametrize("variant", [0, 2, 3, 4, 5, 7, 8, 9, 10])
def test_fp32_variant_solves_to_tolerance(mg, variant):
    p = CASES["gauss3d_b8"]()
    t = mg.Tree.from_problem(p)
    t.set_sweep_variant(variant, precision=mg.MG_FP32_DC)
    assert applied(t, variant, mg.MG_FP32_DC)
    cyc, rel = t.solve(1e-10, 30, precision=mg.MG_FP32_DC)
    o = Oracle.from_problem(p)
    r0, _ = o.residual_norm()
    o.set_phi(t.get_phi().cpu().numpy())
    r, _ = o.residual_norm()
    assert r <= 1.05e-10 * r0, (variant, cyc, r / r0)


def test_fp32_register_f_variants_equal_staged(mg):
    """Variants 7-9 differ from 4 only in where f comes from."""
    p = CASES["gauss3d_b8"]()
    out = {}
    for v in (4, 7, 8, 9):
        t = mg.Tree.from_problem(p)
        t.set_sweep_variant(v, precision=mg.MG_FP32_DC)
        t.solve(1e-30, 3, precision=mg.MG_FP32_DC, raise_on_fail=False)
        out[v] = t.get_phi().cpu().numpy()
    for v in (7, 8, 9):
        assert np.array_equal(out[v], out[4]), v


def test_set_sweep_variant_rejects_inapplicable(mg):
    t = mg.Tree.from_problem(CASES["poisson2d_b8"]())
    with pytest.raises(mg.MGError):
        t.set_sweep_variant(4, level=len(t.levels()) - 1)
    t.set_sweep_variant(-1)
