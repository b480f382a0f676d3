"""C ABI and host logic, no GPU: the library loads, exports every entry point
of include/mg.h, builds the same level hierarchy and leaf order as the
oracle and rejects invalid meshes."""
import os
import re

import numpy as np
import pytest

from oracle import Oracle
from synth import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1901_11370_gb300 import build as B
    B.build()
    from paper_1901_11370_gb300 import _lib
    return _lib.load()


def header_symbols():
    src = open(os.path.join(ROOT, "include", "mg.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(mg_\w+)\s*\(", src, re.M)))


def test_exports_every_declared_symbol(lib):
    from paper_1901_11370_gb300 import _lib
    syms = header_symbols()
    assert len(syms) >= 19
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(_lib.EXPORTS) == syms


MESHES = {
    "cfg1": lambda: W.cfg1_poisson2d(),
    "gauss3d_small": lambda: W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15)),
    "cyl_odd": lambda: W.cyl_ring_tree(3, force_k=3),
    "cyl_31": lambda: W.cyl_ring_tree(5, force_k=31),
    "varcoef_small": lambda: W.cfg3_varcoef3d(n=64, N=16),
    "periodic_amr": lambda: W.Problem("p", 2, 4, 0, (32, 32, 1), (0, 0, 0), (1, 1, 1), (2, 2, 0, 0, 0, 0), (0,) * 6,
                                      W.refine_spheres(2, 4, (32, 32, 1), (0, 0, 0), (1, 1, 1), (0.02, 0.5, 0),
                                                       (0.3, 0.15), (True, False, False))),
}


@pytest.mark.parametrize("name", sorted(MESHES))
def test_levels_and_leaf_order_match_oracle(lib, name):
    import paper_1901_11370_gb300 as mg
    p = MESHES[name]()
    t = mg.Tree(p.dim, p.N, p.geom, p.bc_type, p.bc_val, p.base, p.lo, p.hi, p.refine, p.coarse_max,
                finalize=False)
    o = Oracle.from_problem(p, set_fields=False)
    assert t.levels() == o.levels()
    assert np.array_equal(t.leaf_blocks(), o.leaf_blocks())
    assert np.array_equal(t.leaf_blocks(), W.leaf_blocks(p).astype(np.int32))
    assert t.n_leaf == o.n_leaf == W.n_leaf_cells(p)


def test_coarse_levels_match_paper_table(lib):
    import paper_1901_11370_gb300 as mg
    t = mg.Tree(2, 8, 0, (0,) * 6, (0,) * 6, (192, 96), (0, 0), (2, 1), coarse_max=0, finalize=False)
    got = [(l["ncell"][:2], l["n"], l["nblk"][:2]) for l in t.levels()]
    assert got == [((6, 3), 1, (6, 3)), ((12, 6), 2, (6, 3)), ((24, 12), 4, (6, 3)), ((48, 24), 8, (6, 3)),
                   ((96, 48), 8, (12, 6)), ((192, 96), 8, (24, 12))]


def test_invalid_meshes_are_rejected(lib):
    import paper_1901_11370_gb300 as mg
    from paper_1901_11370_gb300 import MGError
    ref = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [2, 1, 1, 0]], np.int32)  # depth-2 block beside depth 0
    with pytest.raises(MGError) as e:
        mg.Tree(2, 4, 0, (0,) * 6, (0,) * 6, (16, 16), (0, 0), (1, 1), ref, finalize=False)
    assert e.value.code == -2
    with pytest.raises(MGError):
        mg.Tree(2, 4, 0, (0,) * 6, (0,) * 6, (16, 16), (0, 0), (1, 1), np.array([[0, 9, 0, 0]]), finalize=False)
    with pytest.raises(MGError):
        mg.Tree(2, 3, 0, (0,) * 6, (0,) * 6, (12, 12), (0, 0), (1, 1), finalize=False)  # odd N
    with pytest.raises(MGError):
        mg.Tree(2, 4, 0, (2, 0, 0, 0, 0, 0), (0,) * 6, (16, 16), (0, 0), (1, 1), finalize=False)  # lone periodic
    with pytest.raises(MGError):
        mg.Tree(3, 4, 1, (0,) * 6, (0,) * 6, (16, 16, 16), (0,) * 3, (1,) * 3, finalize=False)  # 3D cylindrical


def test_python_layer_has_no_fallback():
    """The binding refuses to run without the compiled library (no CPU path)."""
    src = open(os.path.join(ROOT, "paper_1901_11370_gb300", "_lib.py")).read()
    assert "raise ImportError" in src
    for f in os.listdir(os.path.join(ROOT, "paper_1901_11370_gb300")):
        if f.endswith(".py"):
            assert "oracle" not in open(os.path.join(ROOT, "paper_1901_11370_gb300", f)).read().split("import")[0] or True
            body = open(os.path.join(ROOT, "paper_1901_11370_gb300", f)).read()
            assert "from oracle" not in body and "import oracle" not in body, f


def test_calls_out_of_order_return_state_error(lib):
    """Lifecycle errors (MG_ERR_STATE): refinement after the mesh was built,
    field calls before finalize (checked before any device pointer is used)."""
    import ctypes as C
    import paper_1901_11370_gb300 as mg
    t = mg.Tree(2, 8, 0, (0,) * 6, (0,) * 6, (32, 32), (0, 0), (1, 1), finalize=False)
    t.levels()  # builds the level tables
    ref = np.array([[0, 0, 0, 0]], np.int32)
    assert t.L.mg_tree_refine(t._h, 1, ref.ctypes.data_as(C.c_void_p)) == -8
    assert t.L.mg_set_rhs(t._h, None) == -8
    assert t.L.mg_vcycle(t._h, 1, None) == -8


def test_adapt_and_build_times_on_the_host(lib):
    """mg_tree_adapt needs a finalized tree (MG_ERR_STATE before that, and
    MG_ERR_ARG for null arguments); mg_tree_build_times reports the host
    table time as soon as the tables exist and nothing for device steps not
    taken yet."""
    import ctypes as C
    import paper_1901_11370_gb300 as mg
    t = mg.Tree(3, 8, 0, (0,) * 6, (0,) * 6, (64, 64, 64), (0, 0, 0), (1, 1, 1), finalize=False)
    out = (C.c_double * 4)()
    t.levels()  # host tables (the wrapper's leaf count has built them already)
    assert t.L.mg_tree_build_times(t._h, out) == 0
    assert out[0] > 0 and out[1] == out[2] == out[3] == 0
    h = C.c_void_p()
    add = np.array([[0, 1, 1, 1]], np.int32)
    assert t.L.mg_tree_adapt(t._h, 1, add.ctypes.data_as(C.c_void_p), 0, None, C.byref(h)) == -8
    assert not h.value
    assert t.L.mg_tree_adapt(None, 0, None, 0, None, C.byref(h)) == -1
    assert t.L.mg_tree_build_times(t._h, None) == -1
