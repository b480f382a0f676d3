"""Plain FP64 CPU oracle of the octree geometric multigrid (arXiv:1901.11370).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The CUDA library never links,
imports or calls anything here, and nothing here calls it.

``Oracle`` wraps ``mg_oracle.c`` (compiled with gcc on first use or by
``build()``) through ctypes; every method maps to one C routine that cites
the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIB = os.path.join(_HERE, "libmg_oracle.so")
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force=False):
    """Compile the oracle into a shared library beside its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        try:  # OpenMP over the blocks of a level where the compiler has it
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = C.CDLL(_LIB)
    L.or_create.restype = C.c_void_p
    L.or_create.argtypes = [C.c_int, C.c_int, C.c_int, _ip, _dp, _ip, _dp, _dp, C.c_int,
                            C.c_double, C.c_int, _ip]
    L.or_last_error.restype = C.c_char_p
    L.or_destroy.argtypes = [C.c_void_p]
    L.or_num_levels.argtypes = [C.c_void_p]
    L.or_level_info.argtypes = [C.c_void_p, C.c_int, _ip, _dp]
    L.or_set_cycle.argtypes = [C.c_void_p, C.c_int, C.c_int]
    L.or_set_schedule.argtypes = [C.c_void_p, C.c_int, _ip, _ip]
    L.or_set_coarse_mode.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int]
    L.or_set_smoother.argtypes = [C.c_void_p, C.c_int, C.c_double]
    L.or_set_homogeneous.argtypes = [C.c_void_p, C.c_int]
    L.or_num_leaf_cells.restype = C.c_int64
    L.or_num_leaf_cells.argtypes = [C.c_void_p]
    L.or_leaf_blocks.restype = C.c_int64
    L.or_leaf_blocks.argtypes = [C.c_void_p, C.c_void_p]
    for name in ("or_set_rhs", "or_set_phi", "or_get_phi", "or_get_lam", "or_set_eps"):
        getattr(L, name).argtypes = [C.c_void_p, _dp]
    L.or_set_bc_plane.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp]
    L.or_refresh.argtypes = [C.c_void_p]
    L.or_vcycle.argtypes = [C.c_void_p, C.c_int]
    L.or_fmg.argtypes = [C.c_void_p]
    L.or_residual_norm.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]
    L.or_apply.argtypes = [C.c_void_p, _dp, _dp]
    L.or_leaf_geometry.argtypes = [C.c_void_p, _dp, _dp]
    L.or_eps_grad.argtypes = [C.c_void_p, _dp, _dp]
    L.or_level_io.restype = C.c_int64
    L.or_level_io.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int]
    L.or_level_blocks.argtypes = [C.c_void_p, C.c_int, _ip, _ip, _ip]
    L.or_step.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
    L.or_divergence.argtypes = [C.c_void_p, _dp, _dp]
    L.or_divergence_order.argtypes = [C.c_void_p, _dp, _dp, C.c_int]
    L.or_project.argtypes = [C.c_void_p, _dp, _dp]
    L.or_transfer.argtypes = [C.c_void_p, C.c_void_p]
    L.or_set_threads.argtypes = [C.c_int]
    for name in ("or_apply_T", "or_eps_grad_T", "or_divergence_T", "or_gradient_T"):
        getattr(L, name).argtypes = [C.c_void_p, _dp, _dp]
    _lib = L
    return L


def set_threads(n=0):
    """Threads of the oracle's block loops (n <= 0: leave as is); returns
    the count in use.  Results do not depend on it."""
    return int(_load().or_set_threads(int(n)))


class Oracle:
    """One mesh and its fields in the FP64 oracle."""

    def __init__(self, dim, N, geom, bc_type, bc_val, base, lo, hi, refine=None,
                 coarse_max=512, helm=0.0):
        L = _load()
        ref = np.ascontiguousarray(np.zeros((0, 4), np.int32) if refine is None else refine,
                                   dtype=np.int32).reshape(-1, 4)
        base3 = [int(b) for b in base] + [1] * (3 - len(base))
        self._h = L.or_create(int(dim), int(N), int(geom), np.array(bc_type, np.int32),
                              np.array(bc_val, np.float64), np.array(base3, np.int32),
                              np.array(list(lo) + [0.0] * (3 - len(lo)), np.float64),
                              np.array(list(hi) + [1.0] * (3 - len(hi)), np.float64),
                              int(coarse_max), float(helm), len(ref), ref.ravel())
        if not self._h:
            raise ValueError("oracle: " + L.or_last_error().decode())
        self.L = L
        self.dim = dim
        self.cyl = geom == 1
        # no Dirichlet face and no Helmholtz term: A has the constants as
        # its null space (reading of the compatibility condition)
        self._singular = all(int(t) != 0 for t in list(bc_type)[:2 * dim]) and float(helm) <= 0.0
        self._rhs = np.zeros(int(L.or_num_leaf_cells(self._h)))
        self.n_leaf = int(L.or_num_leaf_cells(self._h))

    @classmethod
    def from_problem(cls, p, set_fields=True):
        o = cls(p.dim, p.N, p.geom, p.bc_type, p.bc_val, p.base, p.lo, p.hi, p.refine,
                p.coarse_max)
        if set_fields:
            from synth import workloads as W
            o.set_bc_from_problem(p)
            if p.eps is not None or p.eps_leaf is not None:
                o.set_eps(W.leaf_field(p, "eps"))
            o.set_rhs(W.leaf_field(p, "rhs"))
        return o

    def transfer_from(self, old):
        """phi of the oracle mesh `old` carried to this (adapted) mesh
        (reading R15); afterwards get_phi() gives the carried field."""
        if self.L.or_transfer(old._h, self._h) != 0:
            raise ValueError("oracle: " + self.L.or_last_error().decode())

    def __del__(self):
        if getattr(self, "_h", None):
            self.L.or_destroy(self._h)
            self._h = None

    # -------------------------------------------------------------- mesh --
    def levels(self):
        out = []
        for l in range(self.L.or_num_levels(self._h)):
            iv = np.zeros(9, np.int32)
            hv = np.zeros(3)
            self.L.or_level_info(self._h, l, iv, hv)
            out.append(dict(n=int(iv[0]), depth=int(iv[1]), nb=int(iv[2]),
                            nblk=tuple(int(x) for x in iv[3:6]),
                            ncell=tuple(int(x) for x in iv[6:9]), h=tuple(hv)))
        return out

    def leaf_blocks(self):
        n = self.L.or_leaf_blocks(self._h, None)
        out = np.zeros((n, 4), np.int32)
        self.L.or_leaf_blocks(self._h, out.ctypes.data)
        return out

    def leaf_geometry(self):
        v = np.zeros(self.n_leaf)
        r = np.zeros(self.n_leaf)
        self.L.or_leaf_geometry(self._h, v, r)
        return v, r

    # ------------------------------------------------------------ fields --
    def set_rhs(self, f):
        self._rhs = np.array(f, np.float64)
        self.L.or_set_rhs(self._h, np.ascontiguousarray(f, np.float64))

    def set_eps(self, e):
        self.L.or_set_eps(self._h, np.ascontiguousarray(e, np.float64))

    def set_phi(self, x):
        self.L.or_set_phi(self._h, np.ascontiguousarray(x, np.float64))

    def get_phi(self):
        x = np.zeros(self.n_leaf)
        self.L.or_get_phi(self._h, x)
        return x

    def set_bc_plane(self, face, level, vals):
        self.L.or_set_bc_plane(self._h, face, level, np.ascontiguousarray(vals, np.float64))

    def set_bc_from_problem(self, p):
        from synth import workloads as W
        if p.bc is None:
            return
        for l, info in enumerate(self.levels()):
            for face in range(2 * p.dim):
                v = W.bc_plane(p, face, info["ncell"], info["h"])
                if v is not None:
                    self.set_bc_plane(face, l, v)
        self.L.or_refresh(self._h)

    def set_homogeneous(self, on):
        self.L.or_set_homogeneous(self._h, 1 if on else 0)
        self.L.or_refresh(self._h)

    # ------------------------------------------------------------ cycles --
    def set_cycle(self, n_down=2, n_up=2):
        self.L.or_set_cycle(self._h, n_down, n_up)

    def set_schedule(self, down=None, up=None):
        """Smoothing steps per level (level 0 coarsest; entries < 0 keep
        set_cycle's); None clears the schedule."""
        if down is None:
            self.L.or_set_schedule(self._h, 0, np.zeros(1, np.int32), np.zeros(1, np.int32))
            return
        d = np.ascontiguousarray(down, np.int32)
        u = np.ascontiguousarray(up, np.int32)
        self.L.or_set_schedule(self._h, len(d), d, u)

    def set_coarse_mode(self, smooth=False, abs_tol=1e-8, rel_tol=1e-8, max_it=1000):
        """Coarsest-level solve: exact (default) or the paper's smoothing to
        an absolute / relative max-norm threshold (Sec. 2.4, reading R20)."""
        self.L.or_set_coarse_mode(self._h, 1 if smooth else 0, float(abs_tol), float(rel_tol), int(max_it))

    def set_smoother(self, jacobi=False, omega=0.0):
        """Red-black Gauss-Seidel (default) or weighted Jacobi (omega <= 0:
        4/5 in 2D, 6/7 in 3D); reading R13."""
        self.L.or_set_smoother(self._h, 1 if jacobi else 0, float(omega))

    def vcycle(self, n=1):
        self.L.or_vcycle(self._h, n)

    def fmg(self):
        self.L.or_fmg(self._h)

    def residual_norm(self, want_res=False):
        l2, li = C.c_double(), C.c_double()
        res = np.zeros(self.n_leaf) if want_res else None
        self.L.or_residual_norm(self._h, C.byref(l2), C.byref(li),
                                res.ctypes.data if want_res else None)
        return (l2.value, li.value, res) if want_res else (l2.value, li.value)

    def apply(self, x):
        out = np.zeros(self.n_leaf)
        self.L.or_apply(self._h, np.ascontiguousarray(x, np.float64), out)
        return out

    def apply_T(self, y):
        """A^T y on the leaf cells, A the linear part of the composite operator
        (the exact transpose of its forward steps, reading R16)."""
        out = np.zeros(self.n_leaf)
        self.L.or_apply_T(self._h, np.ascontiguousarray(y, np.float64), out)
        return out

    def eps_grad_T(self, lam):
        """dL/d eps of the leaf cells on any mesh: -lambda^T d(A phi)/d eps
        through the harmonic face coefficients, eps ghosts and covered cells."""
        out = np.zeros(self.n_leaf)
        self.L.or_eps_grad_T(self._h, np.ascontiguousarray(lam, np.float64), out)
        return out

    def divergence_T(self, v):
        """D^T v, D the second-order central divergence (dim leaf arrays out)."""
        out = np.zeros((self.dim, self.n_leaf))
        if self.L.or_divergence_T(self._h, np.ascontiguousarray(v, np.float64), out.ravel()) != 0:
            raise ValueError("oracle: " + self.L.or_last_error().decode())
        return out

    def gradient_T(self, u):
        """G^T u, G the central gradient of the projection (u: dim leaf arrays)."""
        u = np.ascontiguousarray(u, np.float64).reshape(self.dim, self.n_leaf)
        out = np.zeros(self.n_leaf)
        if self.L.or_gradient_T(self._h, u.ravel(), out) != 0:
            raise ValueError("oracle: " + self.L.or_last_error().decode())
        return out

    def eps_grad(self, lam):
        out = np.zeros(self.n_leaf)
        if self.L.or_eps_grad(self._h, np.ascontiguousarray(lam, np.float64), out) != 0:
            raise ValueError("oracle: " + self.L.or_last_error().decode())
        return out

    # ------------------------------------------------ divergence cleaning --
    def divergence(self, B, order=2):
        """Central divergence of a leaf vector field (dim, n_leaf): second
        order, or fourth order where the cells two away are same-level cells
        (reading R14)."""
        B = np.ascontiguousarray(B, np.float64).reshape(self.dim, self.n_leaf)
        out = np.zeros(self.n_leaf)
        if self.L.or_divergence_order(self._h, B.ravel(), out, int(order)) != 0:
            raise ValueError("oracle: " + self.L.or_last_error().decode())
        return out

    def project(self, B):
        """B - grad(phi) with the current phi (central differences)."""
        B = np.ascontiguousarray(B, np.float64).reshape(self.dim, self.n_leaf)
        out = np.zeros_like(B)
        if self.L.or_project(self._h, B.ravel(), out.ravel()) != 0:
            raise ValueError("oracle: " + self.L.or_last_error().decode())
        return out

    def clean(self, B, rel_tol=1e-12, max_cycles=60):
        """Divergence cleaning (Sec. 4.1): solve Lap phi = div B (right-hand side
        projected to zero volume-weighted mean when no face is Dirichlet), then
        B - grad phi.  Returns (B_new, div B, cycles)."""
        f = self.divergence(B)
        vol, _ = self.leaf_geometry()
        if self._singular:
            f = f - np.dot(vol, f) / vol.sum()
        self.set_rhs(f)
        cycles, _ = self.solve(rel_tol, max_cycles)
        return self.project(B), f, cycles

    # -------------------------------------------------------- test hooks --
    FIELDS = {"phi": 0, "f": 1, "eps": 2, "vold": 3, "lam": 4}

    def level_get(self, l, which):
        """Padded field of level l as [nb, (n+2)] * dim (ghost layer included)."""
        info = self.levels()[l]
        n = self.L.or_level_io(self._h, l, self.FIELDS[which], None, 1)
        out = np.zeros(n)
        self.L.or_level_io(self._h, l, self.FIELDS[which], out.ctypes.data, 1)
        return out.reshape((info["nb"],) + (info["n"] + 2,) * self.dim)

    def level_set(self, l, which, arr):
        a = np.ascontiguousarray(arr, np.float64).ravel()
        self.L.or_level_io(self._h, l, self.FIELDS[which], a.ctypes.data, 0)

    def level_blocks(self, l):
        nb = self.levels()[l]["nb"]
        ijk = np.zeros(3 * nb, np.int32)
        par = np.zeros(nb, np.int32)
        hc = np.zeros(nb, np.int32)
        self.L.or_level_blocks(self._h, l, ijk, par, hc)
        return ijk.reshape(nb, 3), par, hc

    def step(self, op, l=0, arg=0):
        ops = {"ghost": 0, "smooth": 1, "restrict": 2, "prolong": 3, "coarse": 4, "jacobi": 5}
        self.L.or_step(self._h, ops[op], l, arg)

    # ---------------------------------------------------- composite solve --
    def solve(self, rel_tol=1e-10, max_cycles=50, fmg_first=True):
        """phi = 0, then (optionally) one FMG cycle and V-cycles until the
        composite residual drops by rel_tol; a singular problem's phi is
        returned with zero volume-weighted mean.  Returns (cycles, history)."""
        self.set_phi(np.zeros(self.n_leaf))
        r0, _ = self.residual_norm()
        hist = [r0]
        cycles = 0
        if fmg_first:
            self.fmg()
            cycles += 1
            hist.append(self.residual_norm()[0])
        while hist[-1] > rel_tol * r0 and cycles < max_cycles:
            self.vcycle(1)
            cycles += 1
            hist.append(self.residual_norm()[0])
        if self._singular:  # the solution with zero volume-weighted mean (reading c10)
            vol, _ = self.leaf_geometry()
            x = self.get_phi()
            self.set_phi(x - np.dot(vol, x) / vol.sum())
        return cycles, hist

    def adjoint(self, g, n_vcycles=12, rel_tol=0.0):
        """lambda = A^-T g and dL/deps, given the converged phi in the tree.

        With W the cell volumes, A* = W^-1 A^T W equals A wherever W A is
        symmetric (uniform meshes, the cylindrical form included) and is
        close to it on refined meshes, so A's V-cycle M approximates its
        inverse.  The iteration (reading R16): mu_0 = FMG(W^-1 g),
        lambda_0 = W mu_0, then lambda += W M W^-1 (g - A^T lambda), with
        homogeneous boundary values, n_vcycles times or until the
        volume-weighted norm of W^-1 (g - A^T lambda) falls below rel_tol
        times that of W^-1 g.  Without Dirichlet faces (and lambda = 0) A
        has the constants as null space: g is made compatible (sum g = 0) and
        lambda is returned as P^T lambda = lambda - W sum(lambda) / sum(W),
        the adjoint of the zero-mean projection of f.  Returns (lambda,
        dL/deps); last_adjoint holds (iterations, final relative residual)."""
        phi = self.get_phi()
        rhs = self._rhs.copy()
        vol, _ = self.leaf_geometry()
        vs = vol.sum()
        gh = np.array(g, np.float64)
        if self._singular:
            gh = gh - vol * gh.sum() / vs

        def nrm(r):
            return math.sqrt(np.dot(vol, (r / vol) ** 2) / vs)

        self.set_homogeneous(True)
        self.set_rhs(gh / vol)
        self.set_phi(np.zeros(self.n_leaf))
        self.fmg()
        lam = vol * self.get_phi()
        r0 = nrm(gh)
        it = 0
        while True:
            r = gh - self.apply_T(lam)
            rel = nrm(r) / r0 if r0 > 0 else 0.0
            if it >= n_vcycles or rel <= rel_tol:
                break
            self.set_rhs(r / vol)
            self.set_phi(np.zeros(self.n_leaf))
            self.vcycle(1)
            lam = lam + vol * self.get_phi()
            it += 1
        if self._singular:
            lam = lam - vol * lam.sum() / vs
        self.set_homogeneous(False)
        self.set_rhs(rhs)
        self.set_phi(phi)
        self.last_adjoint = (it, rel)
        return lam, self.eps_grad_T(lam)

    def clean_adjoint(self, gBn, n_vcycles=40, rel_tol=1e-13):
        """Vector-Jacobian product of the cleaning map B -> B - G phi,
        phi = A^-1 P D B (second-order divergence, Sec. 4.1): given
        gBn = dL/dB_new (dim leaf arrays), dL/dB = gBn - D^T P^T A^-T Q^T G^T gBn
        (P, Q the zero-mean projections of f and phi on a singular mesh, the
        adjoint solve as in adjoint())."""
        gBn = np.ascontiguousarray(gBn, np.float64).reshape(self.dim, self.n_leaf)
        lam, _ = self.adjoint(self.gradient_T(gBn), n_vcycles, rel_tol)
        return gBn - self.divergence_T(lam)
