"""B300-native cut-cell VEM pressure projection (Fast VEM Fluid Simulation,
Zhang & Ren 2026): Python binding of the C ABI in include/fastvem.h.

This module only marshals arguments: every step of the projection runs in the
CUDA kernels of the in-tree library `_lib/libfastvem.so`.  PyTorch provides
device memory and the stream.  There is no CPU fallback: if the library is
missing, importing the solver raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

_I64 = ctypes.c_int64
_P = ctypes.c_void_p

STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "degenerate geometry",
          4: "no convergence", 5: "CG breakdown", 6: "NaN or Inf", 7: "CUDA error", 8: "no CUDA device",
          9: "timeout in a persistent kernel"}
PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}


class Params(ctypes.Structure):
    _fields_ = [("order_k", ctypes.c_int), ("levels", ctypes.c_int), ("cheb_degree", ctypes.c_int),
                ("coarse_degree", ctypes.c_int), ("precision", ctypes.c_int), ("rel_tol", ctypes.c_double),
                ("max_iters", ctypes.c_int), ("coarse_solver", ctypes.c_int), ("balance", ctypes.c_int),
                ("naive_prolongation", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("levels", ctypes.c_int), ("order_k", ctypes.c_int), ("n_cells", _I64 * 16),
                ("n_vertices", _I64 * 16), ("n_dofs", _I64 * 16), ("n_dofs_all", _I64 * 16), ("nnz", _I64 * 16),
                ("nnz_p", _I64 * 16),
                ("n_trees", _I64), ("lmax", ctypes.c_double * 16), ("coarse_mode", ctypes.c_int),
                ("coarse_ms", ctypes.c_double * 2), ("sell_cfg64", ctypes.c_int * 16),
                ("sell_cfg32", ctypes.c_int * 16), ("coarse_cfg", ctypes.c_int * 2),
                ("coarse_ms32", ctypes.c_double), ("coarse_mode32", ctypes.c_int),
                ("coarse_ms32_coop", ctypes.c_double), ("stencil_slices32", _I64 * 16),
                ("stencil_classes32", _I64 * 16), ("stencil_used32", ctypes.c_int * 16),
                ("coarse_ms_persist", ctypes.c_double * 2), ("persist_ctas", ctypes.c_int),
                ("setup_s", ctypes.c_double * 2)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_res", ctypes.c_double), ("r0_norm", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FastVEMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

EXPORTS = ["fvem_default_params", "fvem_create", "fvem_destroy", "fvem_build_topology", "fvem_build",
           "fvem_query", "fvem_export_level", "fvem_export_placement", "fvem_export_dofs", "fvem_export_dofs_k2",
           "fvem_export_pattern_k2", "fvem_export_prolongation_pattern_k2",
           "fvem_export_matrix", "fvem_export_cells", "fvem_project", "fvem_project_host", "fvem_project_batched",
           "fvem_vcycle", "fvem_spmv", "fvem_project_adjoint", "fvem_set_profiling", "fvem_get_profile",
           "fvem_launch_count", "fvem_set_graphs", "fvem_set_precision", "fvem_set_tolerance",
           "fvem_vcycle_static", "fvem_set_cheb_lmax", "fvem_set_stencil", "fvem_export_elements_k2",
           "fvem_arm_coarse_abort", "fvem_quality", "fvem_status_str", "fvem_last_error", "fvem_p2g", "fvem_locate", "fvem_g2p", "fvem_advect"]


def lib():
    """Load the in-tree CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"libfastvem.so is not built ({LIB}); run paper_2607_17725_b300/build.py")
        L = ctypes.CDLL(LIB)
        L.fvem_create.argtypes = [ctypes.POINTER(Params), _P, ctypes.POINTER(_P)]
        L.fvem_destroy.argtypes = [_P]
        L.fvem_build_topology.argtypes = [_P, ctypes.c_int, _P, ctypes.c_int]
        L.fvem_build.argtypes = [_P, ctypes.c_int, _P, ctypes.c_int]
        L.fvem_query.argtypes = [_P, ctypes.POINTER(Info)]
        L.fvem_export_level.argtypes = [_P, ctypes.c_int] + [_P] * 10
        L.fvem_export_placement.argtypes = [_P, ctypes.c_int] + [_P] * 4
        L.fvem_export_dofs.argtypes = [_P, ctypes.c_int, _P]
        L.fvem_export_dofs_k2.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P]
        L.fvem_export_pattern_k2.argtypes = [_P, ctypes.c_int, _P, _P, _P]
        L.fvem_export_prolongation_pattern_k2.argtypes = [_P, ctypes.c_int, _P, _P, _P]
        L.fvem_export_matrix.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]
        L.fvem_export_cells.argtypes = [_P] * 5
        L.fvem_project.argtypes = [_P, _P, ctypes.c_double, _P, _P, ctypes.POINTER(Stats)]
        L.fvem_project_host.argtypes = [_P, _P, ctypes.c_double, _P, _P, ctypes.POINTER(Stats)]
        L.fvem_project_batched.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P]
        L.fvem_vcycle.argtypes = [_P, _P, _P]
        L.fvem_spmv.argtypes = [_P, ctypes.c_int, _P, _P]
        L.fvem_project_adjoint.argtypes = [_P, _P, _P, _P, ctypes.POINTER(Stats)]
        L.fvem_set_profiling.argtypes = [_P, ctypes.c_int]
        L.fvem_get_profile.argtypes = [_P, _P, _P, _P]
        L.fvem_launch_count.argtypes = [_P, _P]
        L.fvem_set_graphs.argtypes = [_P, ctypes.c_int]
        L.fvem_set_precision.argtypes = [_P, ctypes.c_int]
        L.fvem_vcycle_static.argtypes = [_P, _P, _P]
        L.fvem_set_tolerance.argtypes = [_P, ctypes.c_double, ctypes.c_int]
        L.fvem_set_cheb_lmax.argtypes = [_P, ctypes.c_int, ctypes.c_double]
        L.fvem_set_stencil.argtypes = [_P, ctypes.c_int, ctypes.c_int]
        L.fvem_arm_coarse_abort.argtypes = [_P]
        L.fvem_quality.argtypes = [_P, ctypes.c_int, _P, _P, _P]
        L.fvem_p2g.argtypes = [_P, ctypes.c_int64, _P, _P, ctypes.c_int, _P, _P]
        L.fvem_locate.argtypes = [_P, ctypes.c_int64, _P, _P]
        L.fvem_g2p.argtypes = [_P, ctypes.c_int64, _P, _P, _P, _P, ctypes.c_double, _P]
        L.fvem_advect.argtypes = [_P, ctypes.c_int64, ctypes.c_double, _P, _P, _P]
        L.fvem_export_elements_k2.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P]
        L.fvem_status_str.restype = ctypes.c_char_p
        L.fvem_status_str.argtypes = [ctypes.c_int]
        L.fvem_last_error.restype = ctypes.c_char_p
        L.fvem_last_error.argtypes = [_P]
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())


class Solver:
    """One cut-cell scene: topology, hierarchy and device operators."""

    def __init__(self, levels=5, cheb_degree=5, coarse_iters=80, precision="fp64", rel_tol=1e-6,
                 max_iters=500, coarse_solver="cg", stream=None, balance=True, order_k=1, naive_prolongation=False):
        L = lib()
        self.params = Params(int(order_k), levels, cheb_degree, coarse_iters, PREC[precision], rel_tol, max_iters,
                             {"chebyshev": 0, "cg": 1}[coarse_solver], 1 if balance else 0,
                             1 if naive_prolongation else 0)
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
            except Exception:
                stream = None
        self.stream = stream
        h = _P()
        st = L.fvem_create(ctypes.byref(self.params), _P(stream) if stream else None, ctypes.byref(h))
        if st:
            raise FastVEMError(st, "fvem_create")
        self._h = h
        self.built = False

    def close(self):
        if getattr(self, "_h", None):
            lib().fvem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st:
            msg = lib().fvem_last_error(self._h).decode()
            raise FastVEMError(st, f"{what}: {msg}")

    # -------------------------------------------------------------- build
    def build_topology(self, N, tris):
        t = np.ascontiguousarray(tris, dtype=np.float64).reshape(-1, 9)
        self._check(lib().fvem_build_topology(self._h, int(N), _ptr(t), len(t)), "build_topology")

    def build(self, N, tris):
        t = np.ascontiguousarray(tris, dtype=np.float64).reshape(-1, 9)
        self._check(lib().fvem_build(self._h, int(N), _ptr(t), len(t)), "build")
        self.built = True
        self.info = self.query()

    def query(self):
        info = Info()
        self._check(lib().fvem_query(self._h, ctypes.byref(info)), "query")
        n = info.levels
        return {"N": info.N, "levels": n, "order_k": info.order_k, "n_trees": info.n_trees,
                "n_dofs_all": list(info.n_dofs_all[:n]),
                "n_cells": list(info.n_cells[:n]), "n_vertices": list(info.n_vertices[:n]),
                "n_dofs": list(info.n_dofs[:n]), "nnz": list(info.nnz[:n]), "nnz_p": list(info.nnz_p[:n]),
                "lmax": list(info.lmax[:n]),
                "coarse_mode": ["cooperative", "kernel sequence", "persistent"][info.coarse_mode],
                "coarse_ms": list(info.coarse_ms), "sell_cfg64": list(info.sell_cfg64[:n]),
                "sell_cfg32": list(info.sell_cfg32[:n]), "coarse_cfg": list(info.coarse_cfg),
                "coarse_ms32": info.coarse_ms32, "stencil_slices32": list(info.stencil_slices32[:n]),
                "coarse_mode32": {0: "cooperative", 1: "kernel sequence", 2: "persistent"}.get(info.coarse_mode32),
                "coarse_ms_persist": list(info.coarse_ms_persist), "persist_ctas": info.persist_ctas,
                "coarse_ms32_coop": info.coarse_ms32_coop,
                "stencil_classes32": list(info.stencil_classes32[:n]),
                "stencil_used32": list(info.stencil_used32[:n]),
                "setup_s": {"topology": info.setup_s[0], "device": info.setup_s[1]}}

    # -------------------------------------------------------------- exports
    def export_level(self, l):
        c = np.zeros(5, dtype=np.int64)
        self._check(lib().fvem_export_level(self._h, l, _ptr(c), *([None] * 9)), "export_level")
        nv, nc, ncv, nf, nfv = (int(x) for x in c)
        q = self.query()
        out = {"V": np.zeros((nv, 3)), "cell_vptr": np.zeros(nc + 1, np.int32), "cell_v": np.zeros(ncv, np.int32),
               "cell_fptr": np.zeros(nc + 1, np.int32), "face_vptr": np.zeros(nf + 1, np.int32),
               "face_v": np.zeros(nfv, np.int32), "face_pid": np.zeros(nf, np.int32),
               "face_sg": np.zeros(nf, np.int8),
               "parent": np.zeros(nc if l + 1 < q["levels"] else 0, np.int32)}
        self._check(lib().fvem_export_level(self._h, l, _ptr(c), _ptr(out["V"]), _ptr(out["cell_vptr"]),
                                            _ptr(out["cell_v"]), _ptr(out["cell_fptr"]), _ptr(out["face_vptr"]),
                                            _ptr(out["face_v"]), _ptr(out["face_pid"]), _ptr(out["face_sg"]),
                                            _ptr(out["parent"]) if len(out["parent"]) else None), "export_level")
        return out

    def export_placement(self, l):
        nv = self.query()["n_vertices"][l]
        t = np.zeros(nv, np.int8)
        c, a, b = (np.zeros(nv, np.int32) for _ in range(3))
        self._check(lib().fvem_export_placement(self._h, l, _ptr(t), _ptr(c), _ptr(a), _ptr(b)), "export_placement")
        return t, c, a, b

    def export_dofs(self, l):
        nv = self.query()["n_vertices"][l]
        d = np.zeros(nv, np.int32)
        self._check(lib().fvem_export_dofs(self._h, l, _ptr(d)), "export_dofs")
        return d

    def export_dofs_k2(self, l):
        """Second-order DOF numbering of level l (see fvem_export_dofs_k2)."""
        c = np.zeros(6, dtype=np.int64)
        self._check(lib().fvem_export_dofs_k2(self._h, l, _ptr(c), None, None, None), "export_dofs_k2")
        n, nv, ne, nf, nc, m = (int(x) for x in c)
        ptr = np.zeros(nc + 1, np.int64)
        dof = np.zeros(m, np.int64)
        dirichlet = np.zeros(n, np.uint8)
        self._check(lib().fvem_export_dofs_k2(self._h, l, _ptr(c), _ptr(ptr), _ptr(dof), _ptr(dirichlet)),
                    "export_dofs_k2")
        return {"n": n, "nv": nv, "ne": ne, "nf": nf, "nc": nc, "elem_ptr": ptr, "elem_dof": dof,
                "dirichlet": dirichlet.astype(bool)}

    def export_prolongation_pattern_k2(self, l):
        """(shape, rowptr, col) of the k = 2 prolongation pattern, level l+1 -> l."""
        c = np.zeros(3, dtype=np.int64)
        fn = lib().fvem_export_prolongation_pattern_k2
        self._check(fn(self._h, l, _ptr(c), None, None), "export_prolongation_pattern_k2")
        rp = np.zeros(int(c[0]) + 1, np.int64)
        col = np.zeros(int(c[2]), np.int64)
        self._check(fn(self._h, l, _ptr(c), _ptr(rp), _ptr(col)), "export_prolongation_pattern_k2")
        return (int(c[0]), int(c[1])), rp, col

    def export_pattern_k2(self, l):
        """(rowptr, col) of the k = 2 operator's pattern over free DOFs."""
        c = np.zeros(2, dtype=np.int64)
        self._check(lib().fvem_export_pattern_k2(self._h, l, _ptr(c), None, None), "export_pattern_k2")
        rp = np.zeros(int(c[0]) + 1, np.int64)
        col = np.zeros(int(c[1]), np.int64)
        self._check(lib().fvem_export_pattern_k2(self._h, l, _ptr(c), _ptr(rp), _ptr(col)), "export_pattern_k2")
        return rp, col

    def export_elements_k2(self, l):
        """Second-order element matrices, projectors and cell moments of level l
        (see fvem_export_elements_k2), as flat arrays."""
        c = np.zeros(3, dtype=np.int64)
        fn = lib().fvem_export_elements_k2
        self._check(fn(self._h, l, _ptr(c), None, None, None), "export_elements_k2")
        K, Pis, mom = np.zeros(int(c[0])), np.zeros(int(c[1])), np.zeros(int(c[2]))
        self._check(fn(self._h, l, _ptr(c), _ptr(K), _ptr(Pis), _ptr(mom)), "export_elements_k2")
        return K, Pis, mom

    def export_matrix(self, which, l, values=True):
        c = np.zeros(3, dtype=np.int64)
        self._check(lib().fvem_export_matrix(self._h, which, l, _ptr(c), None, None, None), "export_matrix")
        rows, cols, nnz = (int(x) for x in c)
        rp = np.zeros(rows + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        val = np.zeros(nnz) if values else None
        self._check(lib().fvem_export_matrix(self._h, which, l, _ptr(c), _ptr(rp), _ptr(col), _ptr(val)),
                    "export_matrix")
        return (rows, cols), rp, col, val

    def export_cells(self):
        q = self.query()
        nc = q["n_cells"][0]
        lvl = self.export_level(0)
        n = np.diff(lvl["cell_vptr"]).astype(np.int64)
        vol, cen, h = np.zeros(nc), np.zeros((nc, 3)), np.zeros(nc)
        K = np.zeros(int((n * n).sum()))
        self._check(lib().fvem_export_cells(self._h, _ptr(vol), _ptr(cen), _ptr(h), _ptr(K)), "export_cells")
        return vol, cen, h, K

    # -------------------------------------------------------------- projection
    def project(self, u, u_inflow=0.0, p=None, cellpoly=None):
        """u: CUDA float64 tensor (3, n_vertices) (SoA).  Returns (p, cellpoly, stats)."""
        import torch
        nv = self.info["n_vertices"][0]
        nc = self.info["n_cells"][0]
        assert u.is_cuda and u.dtype == torch.float64 and u.is_contiguous() and u.numel() == 3 * nv
        if p is None:
            p = torch.empty(self.info["n_dofs_all"][0], dtype=torch.float64, device=u.device)
        if cellpoly is None:
            cellpoly = torch.empty((nc, 3, 4), dtype=torch.float64, device=u.device)
        st = Stats()
        rc = lib().fvem_project(self._h, _ptr(u), float(u_inflow), _ptr(p), _ptr(cellpoly), ctypes.byref(st))
        self._check(rc, "project")
        return p, cellpoly, st.as_dict()

    def project_host(self, u, u_inflow=0.0, want_outputs=True):
        nv = self.info["n_vertices"][0]
        nc = self.info["n_cells"][0]
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.size == 3 * nv
        p = np.zeros(self.info["n_dofs_all"][0]) if want_outputs else None
        cp = np.zeros((nc, 3, 4)) if want_outputs else None
        st = Stats()
        self._check(lib().fvem_project_host(self._h, _ptr(u), float(u_inflow), _ptr(p), _ptr(cp),
                                            ctypes.byref(st)), "project_host")
        return p, cp, st.as_dict()

    def project_host_pinned(self, u, p, cp, u_inflow=0.0):
        """Like project_host with caller-provided (pinned) torch CPU tensors."""
        st = Stats()
        self._check(lib().fvem_project_host(self._h, _ptr(u), float(u_inflow), _ptr(p), _ptr(cp),
                                            ctypes.byref(st)), "project_host")
        return st.as_dict()

    def set_profiling(self, on):
        self._check(lib().fvem_set_profiling(self._h, 1 if on else 0), "set_profiling")

    def get_profile(self):
        n = ctypes.c_int64(0)
        ms = ctypes.c_double(0.0)
        by = ctypes.c_double(0.0)
        self._check(lib().fvem_get_profile(self._h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)),
                    "get_profile")
        return {"launches": n.value, "total_ms": ms.value, "bytes_per_launch": by.value}

    def set_precision(self, precision):
        self._check(lib().fvem_set_precision(self._h, PREC[precision]), "set_precision")

    def set_tolerance(self, rel_tol, max_iters=500):
        self._check(lib().fvem_set_tolerance(self._h, float(rel_tol), int(max_iters)), "set_tolerance")

    def set_cheb_lmax(self, level, lmax):
        self._check(lib().fvem_set_cheb_lmax(self._h, int(level), float(lmax)), "set_cheb_lmax")

    def set_stencil(self, level, on):
        self._check(lib().fvem_set_stencil(self._h, int(level), 1 if on else 0), "set_stencil")

    def quality(self, level=0):
        """Element quality indicator of the level's cells (Eq. 18, App. C):
        (rho per cell as a device tensor, rho(P) over the cut cells (Eq. 19),
        the number of cut cells)."""
        import torch
        ncs = self.query()["n_cells"]
        if not 0 <= level < len(ncs):  # the library reports the bad level
            self._check(lib().fvem_quality(self._h, int(level), None, None, None), "quality")
        nc = ncs[level]
        rho = torch.empty(max(1, nc), dtype=torch.float64, device="cuda")
        g = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        self._check(lib().fvem_quality(self._h, int(level), ctypes.c_void_p(rho.data_ptr()), ctypes.byref(g),
                                       ctypes.byref(n)), "quality")
        return rho[:nc], g.value, n.value

    # ---- particle transfers (Sec. 3.2-3.3); tensors on the context's device

    @staticmethod
    def _dev(t, dtype, name):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
            raise TypeError(f"{name}: a contiguous CUDA tensor of {dtype}")
        return ctypes.c_void_p(t.data_ptr())

    def p2g(self, xp, fp, cell=None):
        """Radial-kernel averages of the particles' values at the level-0
        vertices (Sec. 3.2).  xp: (3, n) float64; fp: (c, n) float64 with
        c in 1..4; cell: optional (n,) int32 (particles with -1 skipped).
        Returns (c, n_vertices(0)) float64."""
        import torch
        nv = self.query()["n_vertices"][0]
        n, c = int(xp.shape[1]), int(fp.shape[0])
        out = torch.empty((c, nv), dtype=torch.float64, device=xp.device)
        cp = None if cell is None else self._dev(cell, torch.int32, "cell")
        self._check(lib().fvem_p2g(self._h, n, self._dev(xp, torch.float64, "xp"), cp, c,
                                   self._dev(fp, torch.float64, "fp"), ctypes.c_void_p(out.data_ptr())), "p2g")
        return out

    def locate(self, xp):
        """Level-0 cell of each particle, -1 in an obstacle or outside the box."""
        import torch
        n = int(xp.shape[1])
        cell = torch.empty(max(1, n), dtype=torch.int32, device=xp.device)
        self._check(lib().fvem_locate(self._h, n, self._dev(xp, torch.float64, "xp"),
                                      ctypes.c_void_p(cell.data_ptr())), "locate")
        return cell[:n]

    def g2p(self, xp, cell, u_old, cellpoly, up, alpha):
        """FLIP/PIC update of the particle velocities up (3, n), in place
        (Sec. 3.3); u_old: (3, n_vertices(0)) the P2G velocity, cellpoly:
        the projection's (n_cells(0), 12) output."""
        import torch
        self._check(lib().fvem_g2p(self._h, int(xp.shape[1]), self._dev(xp, torch.float64, "xp"),
                                   self._dev(cell, torch.int32, "cell"), self._dev(u_old, torch.float64, "u_old"),
                                   self._dev(cellpoly, torch.float64, "cellpoly"), float(alpha),
                                   self._dev(up, torch.float64, "up")), "g2p")
        return up

    def advect(self, xp, cell, cellpoly, dt):
        """One midpoint RK2 step of the particles in the projected velocity,
        xp (3, n) and cell (n,) in place (Sec. 3.3)."""
        import torch
        self._check(lib().fvem_advect(self._h, int(xp.shape[1]), float(dt), self._dev(cellpoly, torch.float64, "cellpoly"),
                                      self._dev(xp, torch.float64, "xp"), self._dev(cell, torch.int32, "cell")), "advect")
        return xp, cell

    def arm_coarse_abort(self):
        """Failure-path hook: the next persistent coarsest-CG launch leaves
        through its timeout exit, so the call that issues it raises
        FastVEMError(FVEM_ETIMEOUT) and the context is reset."""
        self._check(lib().fvem_arm_coarse_abort(self._h), "arm_coarse_abort")

    def set_graphs(self, on):
        self._check(lib().fvem_set_graphs(self._h, 1 if on else 0), "set_graphs")

    def launch_count(self):
        n = ctypes.c_int64(0)
        self._check(lib().fvem_launch_count(self._h, ctypes.byref(n)), "launch_count")
        return n.value

    def vcycle(self, r, z):
        self._check(lib().fvem_vcycle(self._h, _ptr(r), _ptr(z)), "vcycle")

    def vcycle_static(self, r, z):
        """FP64 V-cycle that allocates nothing (static device scratch); see
        fvem_vcycle_static in include/fastvem.h for its size limit and the
        rule that concurrent calls race on the shared array."""
        self._check(lib().fvem_vcycle_static(self._h, _ptr(r), _ptr(z)), "vcycle_static")

    def spmv(self, l, x, y):
        self._check(lib().fvem_spmv(self._h, int(l), _ptr(x), _ptr(y)), "spmv")

    def adjoint(self, gcell, gu=None):
        import torch
        nv = self.info["n_vertices"][0]
        if gu is None:
            gu = torch.empty((3, nv), dtype=torch.float64, device=gcell.device)
        gin = ctypes.c_double(0.0)
        st = Stats()
        self._check(lib().fvem_project_adjoint(self._h, _ptr(gcell.contiguous()), _ptr(gu), ctypes.byref(gin),
                                               ctypes.byref(st)), "adjoint")
        return gu, gin.value, st.as_dict()


def project_batched(solvers, us, u_inflows=None, ps=None, cellpolys=None):
    """A15: project many scenes in lockstep (see fvem_project_batched).  Each
    solver should own a distinct CUDA stream for the scenes to overlap."""
    import torch
    n = len(solvers)
    if ps is None:
        ps = [torch.empty(S.info["n_dofs_all"][0], dtype=torch.float64, device=u.device) for S, u in zip(solvers, us)]
    if cellpolys is None:
        cellpolys = [torch.empty((S.info["n_cells"][0], 3, 4), dtype=torch.float64, device=u.device)
                     for S, u in zip(solvers, us)]
    H = (ctypes.c_void_p * n)(*[S._h.value for S in solvers])
    U = (ctypes.c_void_p * n)(*[u.data_ptr() for u in us])
    Pp = (ctypes.c_void_p * n)(*[p.data_ptr() for p in ps])
    Cp = (ctypes.c_void_p * n)(*[c.data_ptr() for c in cellpolys])
    uin = None if u_inflows is None else (ctypes.c_double * n)(*[float(v) for v in u_inflows])
    st = (Stats * n)()
    rc = lib().fvem_project_batched(H, n, U, uin, Pp, Cp, st)
    if rc:
        raise FastVEMError(rc, "project_batched: " + lib().fvem_last_error(solvers[0]._h).decode())
    return ps, cellpolys, [x.as_dict() for x in st]


def projection_function():
    """torch.autograd.Function: (u (3,nv), u_inflow scalar tensor) -> cellpoly,
    with the hand-written adjoint (same hierarchy, symmetric operator)."""
    import torch

    class Projection(torch.autograd.Function):
        @staticmethod
        def forward(ctx, solver, u, u_inflow):
            _, cp, _ = solver.project(u.contiguous(), float(u_inflow))
            ctx.solver = solver
            return cp

        @staticmethod
        def backward(ctx, g):
            gu, gin, _ = ctx.solver.adjoint(g.contiguous())
            return None, gu, torch.tensor(gin, dtype=torch.float64, device=gu.device)

    return Projection
