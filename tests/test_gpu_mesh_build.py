"""Mesh construction on the device (Sec. 2.5) against the host construction:
the same refinement lists give identical block tables (every offset,
parent, neighbour code and ghost push slot), identical levels and leaf
counts, and the same error codes for a refine entry naming no block and
for a mesh that is not 2:1 balanced.  A solve on the device-built tree
matches the one on the host-built tree."""
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


def _tree(mg, p, where, refine=None):
    return mg.Tree(p.dim, p.N, p.geom, p.bc_type, p.bc_val, p.base, p.lo, p.hi,
                   p.refine if refine is None else refine, p.coarse_max, finalize=False, build_on=where)


def problems():
    return [
        W.cfg1_poisson2d(n=64, N=8),                                     # coarse levels down to 1 block
        W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15), sigma=0.05),     # 3D, two refined levels
        W.cfg2_gauss3d(base=16, N=4, seed=2, radii=(0.25,), sigma=0.06),  # small blocks
        W.cyl_ring_tree(3, force_k=5),                                   # 2D cylindrical, axis face
        W.cyl_ring_tree(11, force_k=7),                                  # odd counts: block size halves below
        W.cfg3_varcoef3d(n=32, N=8, contrast=10.0),                      # periodic y, z
        W.CleanInputs(n=32, N=8).problem,                                # periodic octree, two levels
    ]


@pytest.mark.parametrize("k", range(7))
def test_device_tables_equal_host_tables(mg, k):
    p = problems()[k]
    th, td = _tree(mg, p, 1), _tree(mg, p, 2)
    assert th.built_on() == "host" and td.built_on() == "device"
    bh, bd = th.block_table(), td.block_table()
    assert bh.shape == bd.shape and bh.shape[0] > 0
    assert np.array_equal(bh, bd), np.argwhere(bh != bd)[:5]
    assert th.levels() == td.levels()
    assert th.n_leaf == td.n_leaf


def test_duplicate_and_unordered_refine_entries(mg):
    """Entries listed twice and out of depth order refine once (both builds)."""
    p = W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15), sigma=0.05)
    ref = np.asarray(p.refine).reshape(-1, 4)
    messy = np.concatenate([ref[::-1], ref[: len(ref) // 3]])
    bh = _tree(mg, p, 1, messy).block_table()
    bd = _tree(mg, p, 2, messy).block_table()
    assert np.array_equal(bh, bd)
    assert np.array_equal(bd, _tree(mg, p, 2).block_table())


def test_build_errors_match(mg):
    from paper_1901_11370_gb300._lib import MGError
    p = W.cfg1_poisson2d(n=64, N=8)
    cases = {
        "no block": np.array([[0, 8, 0, 0]], np.int32),            # base grid is 8 x 8 blocks
        "unbalanced": np.array([[0, 3, 3, 0], [1, 6, 6, 0], [2, 12, 12, 0]], np.int32),
    }
    for name, ref in cases.items():
        codes = []
        for where in (1, 2):
            with pytest.raises(MGError) as e:
                _tree(mg, p, where, ref)
            codes.append(e.value.code)
        assert codes[0] == codes[1], (name, codes)
        assert codes[0] == (-1 if name == "no block" else -2), (name, codes)


def test_solve_on_device_built_tree_matches_host_built(mg):
    import torch
    p = W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15), sigma=0.05)
    out = []
    for where in (1, 2):
        t = mg.Tree.from_problem(p, build_on=where)
        t.fmg()
        t.vcycle(2)
        out.append(t.get_phi().cpu().numpy())
        torch.cuda.synchronize()
    assert np.abs(out[0] - out[1]).max() <= 1e-12 * np.abs(out[0]).max()
