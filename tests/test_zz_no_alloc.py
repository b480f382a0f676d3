"""mg_residual_norm_noalloc: the residual-norm variant that allocates
nothing.  It serves callers whose device memory is owned by their own
allocator and who may not call cudaMalloc when they ask for a norm; its
reduction scratch is a static device array.  Checked through the C ABI
against mg_residual_norm on two calls in a row, on meshes that take both the
bulk-copy residual kernel and the generic one, and for the size limit.  This
file is collected last so that a stop at the first failure has already run
every other test."""
import numpy as np
import pytest

from synth import workloads as W

pytestmark = pytest.mark.gpu


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
    "gauss3d_amr_b8": lambda: W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15), sigma=0.05),
    "poisson2d_b8": lambda: W.cfg1_poisson2d(),
    "varcoef3d_b4": lambda: W.cfg3_varcoef3d(n=16, N=4, contrast=10.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_norm_matches_residual_norm(mg, name):
    t = mg.Tree.from_problem(CASES[name]())
    t.fmg()
    for _ in range(2):
        l2, li = t.residual_norm()
        a2, ai = t.residual_norm_noalloc()
        b2, bi = t.residual_norm_noalloc()  # second call in a row reuses the same scratch
        for x2, xi in ((a2, ai), (b2, bi)):
            assert abs(x2 - l2) <= 1e-12 * l2 and abs(xi - li) <= 1e-12 * li, (x2, l2, xi, li)
        t.vcycle(1)


def test_noalloc_rejects_meshes_beyond_the_static_scratch(mg):
    # 2D blocks of 2x2 cells: one residual CTA per leaf block, 256 x 128 of them
    t = mg.Tree(2, 2, 0, (0,) * 6, (0,) * 6, (512, 256), (0, 0), (2, 1))
    with pytest.raises(mg.MGError) as e:
        t.residual_norm_noalloc()
    assert e.value.code == -1 and "static scratch" in str(e.value)
    l2, _ = t.residual_norm()  # the allocating entry point still works on it
    assert np.isfinite(l2)


def test_noalloc_lifecycle_errors(mg):
    # an unfinalized tree is a call out of lifecycle order (MG_ERR_STATE), as
    # for mg_residual_norm; no device work is enqueued
    t = mg.Tree(2, 8, 0, (0,) * 6, (0,) * 6, (32, 32), (0, 0), (1, 1), finalize=False)
    with pytest.raises(mg.MGError) as e:
        t.residual_norm_noalloc()
    assert e.value.code == -8
    with pytest.raises(mg.MGError) as e:
        t.residual_norm()
    assert e.value.code == -8
