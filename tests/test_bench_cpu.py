"""Host logic of bench.py, no GPU: the traffic file parser finds every
committed entry, returns its bytes per cell only while the kernel's source
hash matches, and the kernel hashes cover one whole template each."""
import os
import re

import bench


def entries():
    path = os.path.join(bench.ROOT, "profiles", "sweep_f32_traffic.txt")
    text = "".join(ln for ln in open(path) if not ln.startswith("#"))
    return [dict((k.strip(), v.strip()) for k, v in (ln.split(":", 1) for ln in e.splitlines() if ":" in ln))
            for e in text.split("\n\n") if e.strip()]


def test_traffic_entries_parse_and_follow_the_source_hash():
    es = entries()
    kernels = {e["kernel"] for e in es}
    assert "k_sweep_rows" in kernels and kernels <= {"k_sweep_rows", "k_sweep_tma"}
    for e in es:
        got = bench.measured_traffic(e["kernel"], "sweep_f32_traffic.txt")
        if e["source_sha1"] == bench.kernel_sha1(e["kernel"]):
            assert got == float(e["dram_bytes_per_cell"])
            assert 12.0 < got < 15.0  # at most the algorithmic 15 B/cell of an 8^3 block
        else:
            assert got is None
    assert bench.measured_traffic("k_no_such_kernel", "sweep_f32_traffic.txt") is None


def test_kernel_hash_covers_one_template():
    src = open(os.path.join(bench.ROOT, "paper_1901_11370_gb300", "csrc", "mg_kernels.cu")).read()
    for name in ("k_sweep_rows", "k_sweep_tma", "k_resid_tma"):
        h = bench.kernel_sha1(name)
        assert re.fullmatch(r"[0-9a-f]{40}", h)
    assert bench.kernel_sha1("k_sweep_rows") != bench.kernel_sha1("k_sweep_tma")
    assert "k_sweep_rows(" in src


def test_benchmark_workloads_have_their_stated_sizes():
    """The two benchmark workloads the JSON line names: the 3D AMR tree has
    19,827,200 leaf cells and the 512-tree cylindrical forest 54,636,032
    (seeded generators, so these are fixed)."""
    from synth import workloads as W
    assert W.n_leaf_cells(bench.problem()) == 19827200
    assert sum(W.n_leaf_cells(W.cyl_ring_tree(i)) for i in range(512)) == 54636032


def test_solve_algorithmic_bytes():
    """Per-solve algorithmic bytes: per level cell 136 B (FP64 V(2,2), 3D) or
    68 B (FP32 cycle) -- 24 or 12 B per sweep plus 40 or 20 B of transfers;
    the directly solved coarsest level has no sweeps -- per leaf 16 B (FP64
    composite residual) or 40 B (FP64 residual and update of the defect
    correction), times the outer steps; a schedule changes the sweeps per
    level and inner cycles repeat the cycle part."""
    lv = [{"nb": 1, "n": 8}, {"nb": 8, "n": 8}]
    b64, cells = bench.solve_alg_bytes(lv, 4096, 3, "fp64")
    assert cells == 4608 and b64 == 3 * (40 * 512 + 136 * 4096 + 16 * 4096)
    b32, _ = bench.solve_alg_bytes(lv, 4096, 3, "fp32_dc")
    assert b32 == 3 * (20 * 512 + 68 * 4096 + 40 * 4096)
    b32s, _ = bench.solve_alg_bytes(lv, 4096, 3, "fp32_dc", down=[-1, 1], up=[-1, 2], inner=2)
    assert b32s == 3 * (2 * (20 * 512 + 56 * 4096) + 40 * 4096)
