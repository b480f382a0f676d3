"""The bounded-wait error path of the staged (bulk-copy) kernels, without a
fault: with the tree's wait limit at 0 every staged kernel gives up at its
first wait, sets the status word, lets its own copies in flight land and
returns; the call reports MG_ERR_TIMEOUT and clears the word.  With the
limit restored the same tree solves again, and a fresh tree matches the
oracle, so the context stayed usable.  Nothing here faults or hangs a GPU:
every wait, the one after giving up included, is bounded."""
import numpy as np
import pytest

from oracle import Oracle
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


@pytest.mark.parametrize("prec", ["fp64", "fp32_dc"])
def test_expired_waits_report_timeout_and_leave_the_context_usable(mg, prec):
    import torch
    p = W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15), sigma=0.05)
    precision = mg.MG_FP64 if prec == "fp64" else mg.MG_FP32_DC
    t = mg.Tree.from_problem(p)
    zeros = torch.zeros(t.n_leaf, dtype=torch.float64, device="cuda")
    t.set_wait_limit(0)
    with pytest.raises(mg.MGError) as e:
        t.solve(1e-10, 3, precision=precision)
    assert e.value.code == -6
    t.set_wait_limit(None)
    t.set_phi(zeros)
    cyc, rel = t.solve(1e-10, 40, precision=precision)
    assert rel <= 1e-10
    fresh = mg.Tree.from_problem(p)
    o = Oracle.from_problem(p)
    fresh.fmg(); o.fmg()
    fresh.vcycle(2); o.vcycle(2)
    x, ref = fresh.get_phi().cpu().numpy(), o.get_phi()
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()
