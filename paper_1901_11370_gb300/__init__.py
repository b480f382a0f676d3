"""GB300-native octree geometric multigrid (Teunissen & Keppens, arXiv:1901.11370).

``Tree`` wraps one mesh of the CUDA library (include/mg.h).  Fields are
torch CUDA tensors in leaf order (see ``synth`` / include/mg.h); torch
provides device memory and the stream, the library does every step.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import MGError, check  # noqa: F401

MG_CART, MG_CYL = 0, 1
MG_FP64, MG_FP32_DC = 0, 1
MG_SMOOTH_RBGS, MG_SMOOTH_JACOBI = 0, 1
MG_COARSE_EXACT, MG_COARSE_SMOOTH = 0, 1


def _ptr(t: torch.Tensor):
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), "need a contiguous CUDA float64 tensor"
    return C.c_void_p(t.data_ptr())


def _params(n_down=2, n_up=2, precision=MG_FP64, inner_cycles=1, smoother=MG_SMOOTH_RBGS, omega=0.0,
            coarse_mode=MG_COARSE_EXACT, coarse_max_it=1000, coarse_abs_tol=1e-8, coarse_rel_tol=1e-8):
    return _lib.mg_params(n_down, n_up, precision, inner_cycles, smoother, float(omega), int(coarse_mode),
                          int(coarse_max_it), float(coarse_abs_tol), float(coarse_rel_tol))


class Tree:
    """One quadtree/octree mesh and its device fields."""

    def __init__(self, dim, N, geom, bc_type, bc_val, base, lo, hi, refine=None, coarse_max=512,
                 helm=0.0, finalize=True, build_on=0):
        L = _lib.load()
        self.L = L
        bc = _lib.mg_bc((C.c_int * 6)(*[int(x) for x in bc_type]), (C.c_double * 6)(*[float(x) for x in bc_val]))
        b3 = (C.c_int * 3)(*([int(x) for x in base] + [1] * (3 - len(base))))
        lo3 = (C.c_double * 3)(*([float(x) for x in lo] + [0.0] * (3 - len(lo))))
        hi3 = (C.c_double * 3)(*([float(x) for x in hi] + [1.0] * (3 - len(hi))))
        h = C.c_void_p()
        check(L.mg_tree_create(dim, N, geom, C.byref(bc), b3, lo3, hi3, int(coarse_max), float(helm), C.byref(h)))
        self._h = h
        self.dim = dim
        if refine is not None and len(refine):
            ref = np.ascontiguousarray(refine, dtype=np.int32).reshape(-1, 4)
            check(L.mg_tree_refine(self._h, len(ref), ref.ctypes.data_as(C.c_void_p)))
        if build_on:  # 1: host mesh tables, 2: device (default: device when present)
            check(L.mg_tree_build_on(self._h, int(build_on)))
        n = C.c_int64()
        check(L.mg_tree_num_leaf_cells(self._h, C.byref(n)))
        self.n_leaf = n.value
        self.finalized = False
        if finalize:
            self.finalize()

    @classmethod
    def from_problem(cls, p, set_fields=True, device="cuda", finalize=True, build_on=0):
        """Tree of a synthetic problem with its boundary planes; finalize=False
        leaves it on the host (e.g. as a member of a Batch, which copies it)."""
        from synth import workloads as W
        t = cls(p.dim, p.N, p.geom, p.bc_type, p.bc_val, p.base, p.lo, p.hi, p.refine, p.coarse_max,
                finalize=False, build_on=build_on)
        if p.bc is not None:
            for l, info in enumerate(t.levels()):
                for face in range(2 * p.dim):
                    v = W.bc_plane(p, face, info["ncell"], info["h"])
                    if v is not None:
                        t.set_bc_plane(face, l, v)
        if not finalize:
            return t
        t.finalize()
        if set_fields:
            if p.eps is not None or p.eps_leaf is not None:
                t.set_eps(torch.from_numpy(W.leaf_field(p, "eps")).to(device))
            t.set_rhs(torch.from_numpy(W.leaf_field(p, "rhs")).to(device))
        return t

    def built_on(self):
        """Where the mesh tables were built: "host" or "device"."""
        w = C.c_int()
        check(self.L.mg_tree_built_on(self._h, C.byref(w)))
        return "device" if w.value == 2 else "host"

    def block_table(self):
        """The block descriptors (mg_tree_block_table): int64 array of shape
        (blocks, 24)."""
        n = C.c_int64()
        check(self.L.mg_tree_block_table(self._h, C.byref(n), None))
        out = np.zeros((n.value, 24), np.int64)
        check(self.L.mg_tree_block_table(self._h, C.byref(n), out.ctypes.data_as(C.c_void_p)))
        return out

    def finalize(self):
        stream = torch.cuda.current_stream().cuda_stream
        check(self.L.mg_tree_finalize(self._h, C.c_void_p(stream)))
        self.finalized = True

    def adapt(self, add=(), remove=()):
        """A new Tree for the adapted mesh (mg_tree_adapt): add lists leaf
        blocks (depth, i, j, k) to refine, remove lists refined blocks whose
        children are all leaves to coarsen.  phi is carried over; set rhs
        and eps for the new mesh."""
        a = np.ascontiguousarray(np.asarray(add, dtype=np.int32).reshape(-1, 4))
        r = np.ascontiguousarray(np.asarray(remove, dtype=np.int32).reshape(-1, 4))
        h = C.c_void_p()
        check(self.L.mg_tree_adapt(self._h, len(a), a.ctypes.data_as(C.c_void_p), len(r),
                                   r.ctypes.data_as(C.c_void_p), C.byref(h)))
        t = Tree.__new__(Tree)
        t.L, t._h, t.dim, t.finalized = self.L, h, self.dim, True
        n = C.c_int64()
        check(self.L.mg_tree_num_leaf_cells(h, C.byref(n)))
        t.n_leaf = n.value
        return t

    def build_times(self):
        """Seconds: mesh tables (device or host), device setup, FP64 autotuning, adapt's phi
        transfer (mg_tree_build_times)."""
        out = (C.c_double * 4)()
        check(self.L.mg_tree_build_times(self._h, out))
        return tuple(out)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.L.mg_tree_destroy(h)
            self._h = None

    # --------------------------------------------------------------- mesh --
    def levels(self):
        n = C.c_int()
        check(self.L.mg_tree_num_levels(self._h, C.byref(n)))
        out = []
        for l in range(n.value):
            info = np.zeros(9, np.int32)
            h = (C.c_double * 3)()
            check(self.L.mg_tree_level_info(self._h, l, info.ctypes.data_as(C.c_void_p), h))
            out.append(dict(n=int(info[0]), depth=int(info[1]), nb=int(info[2]),
                            nblk=tuple(int(x) for x in info[3:6]), ncell=tuple(int(x) for x in info[6:9]),
                            h=tuple(h)))
        return out

    def leaf_blocks(self):
        nb = self.n_leaf // self.levels()[-1]["n"] ** self.dim  # leaf blocks all have N^D cells
        out = np.zeros((nb, 4), np.int32)
        check(self.L.mg_tree_leaf_blocks(self._h, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_bc_plane(self, face, level, vals):
        v = np.ascontiguousarray(vals, dtype=np.float64)
        check(self.L.mg_set_bc_plane(self._h, face, level, v.ctypes.data_as(C.c_void_p)))

    # ------------------------------------------------------------- fields --
    def _leaf(self, t):
        assert t.numel() == self.n_leaf, "leaf field has %d values, expected %d" % (t.numel(), self.n_leaf)
        return _ptr(t)

    def set_rhs(self, f):
        check(self.L.mg_set_rhs(self._h, self._leaf(f)))

    def set_eps(self, e):
        check(self.L.mg_set_eps(self._h, self._leaf(e)))

    def set_phi(self, x):
        check(self.L.mg_set_phi(self._h, self._leaf(x)))

    def get_phi(self, out=None):
        out = torch.empty(self.n_leaf, dtype=torch.float64, device="cuda") if out is None else out
        check(self.L.mg_get_phi(self._h, self._leaf(out)))
        return out

    # ------------------------------------------------------------- cycles --
    def vcycle(self, n=1, n_down=2, n_up=2, smoother=MG_SMOOTH_RBGS, omega=0.0, coarse_mode=MG_COARSE_EXACT):
        p = _params(n_down, n_up, smoother=smoother, omega=omega, coarse_mode=coarse_mode)
        check(self.L.mg_vcycle(self._h, n, C.byref(p)))

    def fmg(self, n_down=2, n_up=2, smoother=MG_SMOOTH_RBGS, omega=0.0, coarse_mode=MG_COARSE_EXACT):
        p = _params(n_down, n_up, smoother=smoother, omega=omega, coarse_mode=coarse_mode)
        check(self.L.mg_fmg(self._h, C.byref(p)))

    def residual_norm(self, want_res=False):
        l2, li = C.c_double(), C.c_double()
        r = torch.empty(self.n_leaf, dtype=torch.float64, device="cuda") if want_res else None
        check(self.L.mg_residual_norm(self._h, C.byref(l2), C.byref(li), _ptr(r) if want_res else None))
        return (l2.value, li.value, r) if want_res else (l2.value, li.value)

    def residual_norm_noalloc(self):
        """Composite residual norms (l2, linf) through the entry point that
        allocates nothing (its scratch is a static device array)."""
        l2, li = C.c_double(), C.c_double()
        check(self.L.mg_residual_norm_noalloc(self._h, C.byref(l2), C.byref(li)))
        return l2.value, li.value

    def solve(self, rel_tol=1e-10, max_cycles=50, fmg_first=True, precision=MG_FP64, inner_cycles=1,
              n_down=2, n_up=2, raise_on_fail=True, smoother=MG_SMOOTH_RBGS, omega=0.0, coarse_mode=MG_COARSE_EXACT):
        p = _params(n_down, n_up, precision, inner_cycles, smoother, omega, coarse_mode)
        cyc, rel = C.c_int(), C.c_double()
        rc = self.L.mg_solve(self._h, float(rel_tol), int(max_cycles), int(bool(fmg_first)), C.byref(p),
                             C.byref(cyc), C.byref(rel))
        check(rc, allow=() if raise_on_fail else (-4,))
        return cyc.value, rel.value

    # ------------------------------------------------ divergence cleaning --
    def divergence(self, B, order=2):
        """Central-difference divergence of a leaf vector field (dim, n_leaf):
        second order, or fourth order where both cells two away are
        same-level cells (second order beside physical and refinement faces)."""
        B = B.contiguous().view(-1)
        assert B.numel() == self.dim * self.n_leaf
        out = torch.empty(self.n_leaf, dtype=torch.float64, device="cuda")
        check(self.L.mg_divergence_order(self._h, _ptr(B), _ptr(out), int(order)))
        return out

    def project(self, B):
        """B - grad(phi) with the current phi."""
        B = B.contiguous().view(-1)
        assert B.numel() == self.dim * self.n_leaf
        out = torch.empty_like(B)
        check(self.L.mg_project(self._h, _ptr(B), _ptr(out)))
        return out.view(self.dim, self.n_leaf)

    def leaf_volumes(self):
        """Cell volume of every leaf cell (Cartesian), leaf order, on the GPU."""
        lv = {l["depth"]: np.prod(l["h"][:self.dim]) for l in self.levels()}
        lb = self.leaf_blocks()
        per = self.n_leaf // len(lb)
        return torch.from_numpy(np.repeat([lv[int(d)] for d in lb[:, 0]], per)).cuda()

    def clean(self, B, rel_tol=1e-10, max_cycles=60, precision=MG_FP64, order=2, smoother=MG_SMOOTH_RBGS):
        """Divergence cleaning (Sec. 4.1) on the device (mg_clean): f = div B
        (second- or fourth-order), minus its volume-weighted mean when no
        face is Dirichlet; Lap phi = f; B - grad phi (second order, as in the
        paper).  Returns (B_new, f, cycles, rel)."""
        B = B.contiguous().view(-1)
        assert B.numel() == self.dim * self.n_leaf
        Bn = torch.empty_like(B)
        f = torch.empty(self.n_leaf, dtype=torch.float64, device="cuda")
        p = _params(2, 2, precision, 1, smoother)
        cyc, rel = C.c_int(), C.c_double()
        rc = self.L.mg_clean(self._h, _ptr(B), _ptr(Bn), _ptr(f), int(order), float(rel_tol), int(max_cycles),
                             C.byref(p), C.byref(cyc), C.byref(rel))
        check(rc, allow=(-4,))
        return Bn.view(self.dim, self.n_leaf), f, cyc.value, rel.value

    def launch_count(self):
        n = C.c_int64()
        check(self.L.mg_launch_count(self._h, C.byref(n)))
        return n.value

    def set_tail(self, max_cells=None):
        """Cell bound of the V-cycle levels run by the tail kernel
        (mg_set_tail); None or 0 turns it off (the default)."""
        check(self.L.mg_set_tail(self._h, 0 if max_cells is None else int(max_cells)))

    def set_wait_limit(self, polls=None):
        """Polls of the kernels' bounded waits (mg_set_wait_limit); None
        restores the default, 0 makes every staged kernel give up at once."""
        check(self.L.mg_set_wait_limit(self._h, -1 if polls is None else int(polls)))

    def set_schedule(self, down=None, up=None):
        """Smoothing steps per level (mg_set_schedule); None clears it."""
        if down is None:
            check(self.L.mg_set_schedule(self._h, 0, None, None))
            return
        d = np.ascontiguousarray(down, np.int32)
        u = np.ascontiguousarray(up, np.int32)
        check(self.L.mg_set_schedule(self._h, len(d), d.ctypes.data_as(C.c_void_p), u.ctypes.data_as(C.c_void_p)))

    def schedule(self):
        n = len(self.levels())
        d, u = np.zeros(n, np.int32), np.zeros(n, np.int32)
        check(self.L.mg_get_schedule(self._h, n, d.ctypes.data_as(C.c_void_p), u.ctypes.data_as(C.c_void_p)))
        return d, u

    def tune_schedule(self, rel_tol=1e-10, max_cycles=60, precision=MG_FP32_DC):
        """Autotune the sweeps per level and the inner cycles by timed solves
        (mg_tune_schedule); returns (inner_cycles, ms per solve)."""
        inner, ms = C.c_int(), C.c_double()
        check(self.L.mg_tune_schedule(self._h, float(rel_tol), int(max_cycles), int(precision), C.byref(inner),
                                      C.byref(ms)))
        return inner.value, ms.value

    SWEEP_VARIANTS = {0: "k_sweep_tma (CTA per block)", 1: "k_sweep (plain loads)", 2: "k_sweep_warp<8 warps>",
                      3: "k_sweep_warp<4 warps>", 4: "k_sweep_rows<8 warps, 2 stages>",
                      5: "k_sweep_rows<4 warps, 3 stages>", 6: "k_sweep_flat (thread per colour cell)",
                      7: "k_sweep_rows<8 warps, 3 stages, f in registers>",
                      8: "k_sweep_rows<4 warps, 4 stages, f in registers>",
                      9: "k_sweep_rows<8 warps, 2 stages, f in registers>",
                      10: "k_sweep_tma (CTA per block, half-width CTAs)", -1: "untuned"}

    def sweep_variant(self, level, precision=MG_FP64):
        v = C.c_int()
        check(self.L.mg_sweep_variant(self._h, precision, level, C.byref(v)))
        return v.value

    def set_sweep_variant(self, variant, level=-1, precision=MG_FP64):
        """Pin the sweep kernel variant (see SWEEP_VARIANTS) on one level or on
        every level where it applies (level -1); variant -1 restores the
        autotuned choice."""
        check(self.L.mg_set_sweep_variant(self._h, precision, level, variant))

    def time_sweeps(self, level=-1, n_sweeps=4, precision=MG_FP64):
        """(ms per sweep launch, ms per full ghost fill, bytes per sweep
        launch, bytes per ghost fill) on one level (default: the largest)."""
        lv = self.levels()
        if level < 0:
            level = max(range(len(lv)), key=lambda l: lv[l]["nb"] * lv[l]["n"] ** self.dim)
        out = (C.c_double * 4)()
        check(self.L.mg_time_sweeps(self._h, level, n_sweeps, precision, out))
        return tuple(out), level

    def adjoint(self, g, n_cycles=12, want_eps=True, n_down=2, n_up=2, smoother=MG_SMOOTH_RBGS, omega=0.0,
                rel_tol=None, max_cycles=80, precision=MG_FP64):
        """(dL/df, dL/deps) for dL/dphi = g at the current phi (mg_adjoint:
        n_cycles defect-correction iterations; with rel_tol, mg_adjoint_solve
        until the adjoint residual is below rel_tol, raising MGError when
        max_cycles is reached).  With rel_tol, self.last_adjoint holds
        (iterations, final relative residual).  precision=MG_FP32_DC: FP32
        V-cycles inside the FP64 defect correction."""
        p = _params(n_down, n_up, precision, smoother=smoother, omega=omega)
        dLdf = torch.empty(self.n_leaf, dtype=torch.float64, device="cuda")
        dLde = torch.empty(self.n_leaf, dtype=torch.float64, device="cuda") if want_eps else None
        if rel_tol is None:
            check(self.L.mg_adjoint(self._h, self._leaf(g.contiguous()), _ptr(dLdf),
                                    _ptr(dLde) if want_eps else None, C.byref(p), int(n_cycles)))
        else:
            cyc, rel = C.c_int(), C.c_double()
            check(self.L.mg_adjoint_solve(self._h, self._leaf(g.contiguous()), _ptr(dLdf),
                                          _ptr(dLde) if want_eps else None, C.byref(p), float(rel_tol),
                                          int(max_cycles), C.byref(cyc), C.byref(rel)))
            self.last_adjoint = (cyc.value, rel.value)
        return dLdf, dLde

    def apply_transpose(self, y):
        """A^T y on the leaf cells (homogeneous boundary values)."""
        out = torch.empty(self.n_leaf, dtype=torch.float64, device="cuda")
        check(self.L.mg_apply_transpose(self._h, self._leaf(y.contiguous()), _ptr(out)))
        return out

    def clean_adjoint(self, gBn, rel_tol=1e-12, max_cycles=80, n_down=2, n_up=2, precision=MG_FP64):
        """dL/dB of the cleaning map B -> B - grad phi, Lap phi = div B
        (mg_clean_adjoint), for gBn = dL/dB_new (dim, n_leaf); precision as
        for adjoint."""
        gBn = gBn.contiguous().view(-1)
        assert gBn.numel() == self.dim * self.n_leaf
        out = torch.empty_like(gBn)
        p = _params(n_down, n_up, precision)
        cyc, rel = C.c_int(), C.c_double()
        check(self.L.mg_clean_adjoint(self._h, _ptr(gBn), _ptr(out), C.byref(p), float(rel_tol), int(max_cycles),
                                      C.byref(cyc), C.byref(rel)))
        self.last_adjoint = (cyc.value, rel.value)
        return out.view(self.dim, self.n_leaf)


class Batch:
    """Many independent trees solved together (one launch per segment over
    the blocks of all trees).  Leaf fields are the trees' leaf arrays
    concatenated in tree order; ``offsets[i]:offsets[i+1]`` is tree i."""

    def __init__(self, trees):
        L = _lib.load()
        self.L = L
        self.trees = list(trees)
        arr = (C.c_void_p * len(self.trees))(*[t._h.value for t in self.trees])
        h = C.c_void_p()
        stream = torch.cuda.current_stream().cuda_stream
        check(L.mg_batch_create(len(self.trees), arr, C.c_void_p(stream), C.byref(h)))
        self._h = h
        off = np.zeros(len(self.trees) + 1, np.int64)
        check(L.mg_batch_leaf_offsets(self._h, off.ctypes.data_as(C.c_void_p)))
        self.offsets = off
        self.n_leaf = int(off[-1])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.L.mg_batch_destroy(h)
            self._h = None

    def _leaf(self, t):
        assert t.numel() == self.n_leaf, "batch leaf field has %d values, expected %d" % (t.numel(), self.n_leaf)
        return _ptr(t)

    def set_rhs(self, f):
        check(self.L.mg_batch_set_rhs(self._h, self._leaf(f)))

    def set_eps(self, e):
        check(self.L.mg_batch_set_eps(self._h, self._leaf(e)))

    def set_phi(self, x):
        check(self.L.mg_batch_set_phi(self._h, self._leaf(x)))

    def get_phi(self, out=None):
        out = torch.empty(self.n_leaf, dtype=torch.float64, device="cuda") if out is None else out
        check(self.L.mg_batch_get_phi(self._h, self._leaf(out)))
        return out

    def vcycle(self, n=1, n_down=2, n_up=2, smoother=MG_SMOOTH_RBGS, omega=0.0, coarse_mode=MG_COARSE_EXACT):
        p = _params(n_down, n_up, smoother=smoother, omega=omega, coarse_mode=coarse_mode)
        check(self.L.mg_batch_vcycle(self._h, n, C.byref(p)))

    def fmg(self, n_down=2, n_up=2, smoother=MG_SMOOTH_RBGS, omega=0.0, coarse_mode=MG_COARSE_EXACT):
        p = _params(n_down, n_up, smoother=smoother, omega=omega, coarse_mode=coarse_mode)
        check(self.L.mg_batch_fmg(self._h, C.byref(p)))

    def residual_norms(self):
        n = len(self.trees)
        l2, li = np.zeros(n), np.zeros(n)
        check(self.L.mg_batch_residual_norms(self._h, l2.ctypes.data_as(C.c_void_p), li.ctypes.data_as(C.c_void_p)))
        return l2, li

    def solve(self, rel_tol=1e-10, max_cycles=50, fmg_first=True, precision=MG_FP64, inner_cycles=1,
              n_down=2, n_up=2, raise_on_fail=True, smoother=MG_SMOOTH_RBGS, omega=0.0, coarse_mode=MG_COARSE_EXACT):
        p = _params(n_down, n_up, precision, inner_cycles, smoother, omega, coarse_mode)
        cyc = C.c_int()
        rel = np.zeros(len(self.trees))
        rc = self.L.mg_batch_solve(self._h, float(rel_tol), int(max_cycles), int(bool(fmg_first)), C.byref(p),
                                   C.byref(cyc), rel.ctypes.data_as(C.c_void_p))
        check(rc, allow=() if raise_on_fail else (-4,))
        return cyc.value, rel

    def launch_count(self):
        n = C.c_int64()
        check(self.L.mg_batch_launch_count(self._h, C.byref(n)))
        return n.value

    def set_tail(self, max_cells=None):
        """Cell bound of the groups run by the tail kernel (mg_batch_set_tail);
        None or 0 turns it off (the default)."""
        check(self.L.mg_batch_set_tail(self._h, 0 if max_cells is None else int(max_cells)))

    def segments(self):
        ns, ng = C.c_int(), C.c_int()
        check(self.L.mg_batch_num_segments(self._h, C.byref(ns), C.byref(ng)))
        out = []
        for s in range(ns.value):
            info = np.zeros(6, np.int32)
            check(self.L.mg_batch_segment_info(self._h, s, info.ctypes.data_as(C.c_void_p)))
            out.append(dict(n=int(info[0]), group=int(info[1]), nb=int(info[2]), nref=int(info[3]),
                            coarsest=bool(info[4]), parent_same_n=bool(info[5])))
        return out

    def tune_schedule(self, rel_tol=1e-10, max_cycles=60, precision=MG_FP32_DC):
        """Autotune the sweeps per segment and the inner cycles by timed batch
        solves (mg_batch_tune_schedule); returns (inner_cycles, ms per solve)."""
        inner, ms = C.c_int(), C.c_double()
        check(self.L.mg_batch_tune_schedule(self._h, float(rel_tol), int(max_cycles), int(precision),
                                            C.byref(inner), C.byref(ms)))
        return inner.value, ms.value

    def coarse_info(self):
        """Coarsest-level solves: trees with a dense inverse, trees in
        block-tridiagonal form, and the bytes each form stores."""
        out = np.zeros(4, np.int64)
        check(self.L.mg_batch_coarse_info(self._h, out.ctypes.data_as(C.c_void_p)))
        return dict(dense=int(out[0]), block=int(out[1]), dense_bytes=int(out[2]), block_bytes=int(out[3]))

    def time_sweeps(self, segment=-1, n_sweeps=4, precision=MG_FP64):
        seg = self.segments()
        if segment < 0:
            segment = max((s for s in range(len(seg)) if not seg[s]["coarsest"]),
                          key=lambda s: seg[s]["nb"] * seg[s]["n"] ** self.trees[0].dim)
        out = (C.c_double * 4)()
        check(self.L.mg_batch_time_sweeps(self._h, segment, n_sweeps, precision, out))
        return tuple(out), segment


from .autograd import CleanB, MGSolve  # noqa: E402,F401
