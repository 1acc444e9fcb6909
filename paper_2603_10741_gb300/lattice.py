"""ctypes binding of liblattice.so (include/lattice.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module passes torch tensors' device
pointers, the handle's stream and plain sizes.  If the library is missing the import fails
loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblattice.so")

LAT_FP64, LAT_MIXED_FP32, LAT_MIXED_BF16 = 0, 1, 2
STATUS = {0: "LAT_OK", 1: "LAT_EINVAL", 2: "LAT_ENOMEM", 3: "LAT_ECUDA", 4: "LAT_ENEG_JACOBIAN",
          5: "LAT_ENOT_CONVERGED", 6: "LAT_EINDEFINITE", 7: "LAT_ETIMEOUT"}
EXPORTS = ["lattice_setup", "lattice_destroy", "lattice_sizes", "lattice_last_error",
           "lattice_set_mu_scale", "lattice_predictor", "lattice_gather", "assemble_residual_tangent",
           "greedy_select", "select_principal_cells", "set_principal_cells", "apply_reduced_tangent",
           "lattice_set_snapshots",
           "lattice_default_opts",
           "newton_step", "adjoint_gradient", "feti_apply", "lattice_prepare_solver", "feti_to_global",
           "feti_from_global", "lattice_checkpoint_save", "lattice_checkpoint_load", "tangent_solve",
           "lattice_set_timing", "lattice_kernel_time", "lattice_launch_count", "greedy_select_static"]


class LatticeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_cells", C.c_int32), ("n_nodes_cell", C.c_int32),
                ("n_el_cell", C.c_int32), ("n_glob_nodes", C.c_int64),
                ("X_ref", C.c_void_p), ("elems", C.c_void_p), ("cell_nodes", C.c_void_p),
                ("dof_fixed", C.c_void_p), ("dirichlet_unit", C.c_void_p), ("affine_unit", C.c_void_p),
                ("mu_scale", C.c_void_p), ("mu", C.c_double), ("lam", C.c_double),
                ("cell_layer", C.c_void_p)]


class Sizes(C.Structure):
    _fields_ = [("n_dof", C.c_int64), ("n_cells", C.c_int32), ("n_loc", C.c_int32),
                ("n_blocks", C.c_int32), ("nnz", C.c_int64), ("n_r_local", C.c_int32),
                ("n_p_local", C.c_int32), ("n_primal", C.c_int64), ("n_lambda", C.c_int64),
                ("n_krylov", C.c_int64), ("n_q_full", C.c_int32), ("n_q_reduced", C.c_int32),
                ("n_i_local", C.c_int32), ("n_coarse_blocks", C.c_int32), ("coarse_block", C.c_int32),
                ("coarse_block_lu", C.c_int32)]


class NewtonOpts(C.Structure):
    _fields_ = [("eps", C.c_double), ("max_nr", C.c_int32), ("force_all", C.c_int32),
                ("newton_rtol", C.c_double), ("newton_max_it", C.c_int32), ("krylov_rtol", C.c_double),
                ("krylov_max_it", C.c_int32), ("krylov_restart", C.c_int32), ("pcg_iters", C.c_int32),
                ("armijo_max_m", C.c_int32), ("pcg_rtol", C.c_double), ("interface_precond", C.c_int32),
                ("max_enrich", C.c_int32), ("coarse_block_lu", C.c_int32), ("precond_tangent", C.c_int32),
                ("min_enrich", C.c_int32), ("inner_its", C.c_int32), ("inner_rtol", C.c_double),
                ("snapshot", C.c_int32), ("eps_refine", C.c_int32),
                ("eps_refine_rate", C.c_double)]


class NewtonReport(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("r0_norm", C.c_double),
                ("r_norm", C.c_double), ("n_r_last", C.c_int32), ("krylov_its_total", C.c_int32),
                ("armijo_m_max", C.c_int32), ("t_residual_ms", C.c_double), ("t_select_ms", C.c_double),
                ("t_setup_ms", C.c_double), ("t_krylov_ms", C.c_double), ("t_linesearch_ms", C.c_double),
                ("pcg_its_total", C.c_int32), ("enrich_level", C.c_int32), ("inner_its_total", C.c_int32),
                ("eps_refinements", C.c_int32), ("eps_last", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"liblattice.so not built at {path}: run __graft_entry__.build()")
    lib = C.CDLL(path)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "lattice_setup": [C.POINTER(MeshDesc), C.c_int, P, C.POINTER(P)],
        "lattice_destroy": [P],
        "lattice_sizes": [P, C.POINTER(Sizes)],
        "lattice_set_mu_scale": [P, P],
        "lattice_predictor": [P, D, P, P, P],
        "lattice_gather": [P, P, P],
        "assemble_residual_tangent": [P, P, I32, P, I32, P, P, P, P],
        "greedy_select": [P, P, I64, I32, D, I32, P, P, P, P, P, P],
        "select_principal_cells": [P, P, D, I32, I32, P, P, P, P],
        "lattice_set_snapshots": [P, I32],
        "set_principal_cells": [P, P, P, I32, P],
        "apply_reduced_tangent": [P, P, P, I32],
        "lattice_default_opts": [P, C.POINTER(NewtonOpts)],
        "newton_step": [P, P, I32, C.POINTER(NewtonOpts), C.POINTER(NewtonReport)],
        "adjoint_gradient": [P, P, C.POINTER(NewtonOpts), P, P, C.POINTER(NewtonReport)],
        "feti_apply": [P, I32, P, P],
        "tangent_solve": [P, P, P, C.POINTER(NewtonOpts), P, P],
        "lattice_prepare_solver": [P, P, C.POINTER(NewtonOpts)],
        "feti_to_global": [P, P, P],
        "feti_from_global": [P, P, P],
        "lattice_checkpoint_save": [P, C.c_char_p, I32, D, P, P],
        "lattice_checkpoint_load": [P, C.c_char_p, P, P, P, P],
        "lattice_set_timing": [P, I32],
        "lattice_kernel_time": [P, C.c_char_p, P, P],
        "lattice_launch_count": [P, P],
        "greedy_select_static": [P, I64, I32, D, I32, P, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.lattice_last_error.argtypes = [P]
    lib.lattice_last_error.restype = C.c_char_p
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_cuda:
            raise ValueError("device tensor expected")
        if not t.is_contiguous():
            raise ValueError("contiguous tensor expected")
        return C.c_void_p(t.data_ptr())
    return t


def case_arrays(case):
    """Plain arrays of lat_mesh_desc for a latgen.LoadCase (load parameter = top displacement)."""
    lat = case.lattice
    d = lat.dim
    n_dof = lat.n_nodes * d
    fixed = np.zeros(n_dof, dtype=np.uint8)
    dunit = np.zeros(n_dof)
    for n in (lat.bottom_nodes(), lat.top_nodes()):
        for i in range(d):
            fixed[n * d + i] = 1
    dunit[lat.top_nodes() * d + lat.load_axis] = 1.0
    aff = np.zeros(n_dof)
    aff[lat.load_axis::d] = lat.X[:, lat.load_axis] / lat.height
    return dict(dim=d, X_ref=np.ascontiguousarray(lat.X_ref, dtype=np.float64),
                elems=np.ascontiguousarray(lat.elems, dtype=np.int32),
                cell_nodes=np.ascontiguousarray(lat.cell_nodes, dtype=np.int32),
                dof_fixed=fixed, dirichlet_unit=dunit, affine_unit=aff,
                mu_scale=np.ascontiguousarray(case.mu_scale, dtype=np.float64),
                mu=float(case.mu), lam=float(case.lam), n_glob_nodes=lat.n_nodes,
                cell_layer=np.ascontiguousarray(np.round(lat.cell_origin[:, lat.load_axis]), dtype=np.int32))


def greedy_select_static(T, eps, max_nr, stream=None):
    """Algorithm 1 without any device allocation by the library (greedy_select_static).

    For callers that cannot allocate device memory; the workspace is the library's fixed 16 MiB
    device array, shared by every call (calls must not overlap on the GPU).  T is a device
    tensor [n_cols, n_rows] (column s contiguous); S and alpha are allocated here by torch, the
    caller's allocator, and passed in.  Returns (S [n_r] int32, alpha [n_r, n_cols]).
    """
    if T.dtype != torch.float64 or not T.is_cuda or T.dim() != 2 or not T.is_contiguous():
        raise ValueError("T must be a contiguous 2-D float64 CUDA tensor [n_cols, n_rows]")
    n_cols, n_rows = T.shape
    with torch.cuda.device(T.device):
        stream = torch.cuda.current_stream() if stream is None else stream
        S = torch.zeros(max_nr, dtype=torch.int32, device=T.device)
        alpha = torch.zeros((max_nr, n_cols), dtype=torch.float64, device=T.device)
        n_r = C.c_int32(0)
        st = lib().greedy_select_static(_ptr(T), n_rows, n_cols, float(eps), int(max_nr), _ptr(S), C.byref(n_r),
                                        _ptr(alpha), C.c_void_p(stream.cuda_stream))
    if st != 0:
        raise LatticeError(st, "greedy_select_static failed (sizes beyond the 16 MiB workspace give LAT_EINVAL)")
    k = n_r.value
    return S[:k], alpha[:k]


class Lattice:
    """One lattice on the current CUDA device; methods mirror the C entry points."""

    def __init__(self, arrays: dict, precision: int = LAT_FP64, stream=None):
        self._lib = lib()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        a = arrays
        self._keep = a
        desc = MeshDesc()
        desc.dim = a["dim"]
        desc.n_cells = a["cell_nodes"].shape[0]
        desc.n_nodes_cell = a["X_ref"].shape[0]
        desc.n_el_cell = a["elems"].shape[0]
        desc.n_glob_nodes = int(a["n_glob_nodes"])
        for f in ("X_ref", "elems", "cell_nodes", "dof_fixed", "dirichlet_unit", "affine_unit", "mu_scale",
                  "cell_layer"):
            setattr(desc, f, a[f].ctypes.data if a.get(f) is not None else None)
        desc.mu, desc.lam = a["mu"], a["lam"]
        h = C.c_void_p()
        st = self._lib.lattice_setup(C.byref(desc), precision, C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != 0:
            raise LatticeError(st, self._lib.lattice_last_error(None).decode())
        self.h = h
        self.precision = precision
        self.dim = a["dim"]

    @property
    def sizes(self):
        """Current sizes.  The FETI-DP sizes (n_p_local, n_r_local, n_primal, n_lambda, n_krylov)
        change when the solver enriches the primal set, so they are queried on every access."""
        s = Sizes()
        self._check(self._lib.lattice_sizes(self.h, C.byref(s)))
        return s

    @classmethod
    def from_case(cls, case, precision=LAT_FP64, stream=None):
        return cls(case_arrays(case), precision, stream)

    def _check(self, st):
        if st != 0:
            raise LatticeError(st, self._lib.lattice_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self._lib.lattice_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- allocation helpers (torch provides device memory) ------------------------------------
    def zeros(self, n, dtype=torch.float64):
        return torch.zeros(int(n), dtype=dtype, device=self.device)

    def dof_vector(self):
        return self.zeros(self.sizes.n_dof)

    def cell_vector(self, dtype=torch.float64):
        return torch.zeros((self.sizes.n_loc, self.sizes.n_cells), dtype=dtype, device=self.device)

    def krylov_vector(self):
        return self.zeros(self.sizes.n_krylov)

    # --- entry points --------------------------------------------------------------------------
    def lattice_set_snapshots(self, kind):
        """Snapshot kind of select_principal_cells: 0 reduced-rule tangent data, 1 D^ref."""
        self._check(self._lib.lattice_set_snapshots(self.h, int(kind)))

    def lattice_set_mu_scale(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        self._check(self._lib.lattice_set_mu_scale(self.h, th.ctypes.data))

    def lattice_predictor(self, load, u_prev=None, u_prev2=None, out=None):
        out = self.dof_vector() if out is None else out
        self._check(self._lib.lattice_predictor(self.h, float(load), _ptr(u_prev), _ptr(u_prev2), _ptr(out)))
        return out

    def lattice_gather(self, u):
        x = self.cell_vector()
        self._check(self._lib.lattice_gather(self.h, _ptr(u), _ptr(x)))
        return x

    def assemble_residual_tangent(self, u, quad=0, cells=None, residual=True, local_forces=False,
                                  tangent=False, K_out=None):
        s = self.sizes
        n_sel = s.n_cells if cells is None else int(cells.numel())
        r = self.dof_vector() if residual else None
        f = self.cell_vector() if local_forces else None
        K = K_out
        if K is None and tangent:
            K = torch.zeros((n_sel, s.nnz), dtype=torch.float64, device=self.device)
        if K is not None:
            assert K.shape == (n_sel, s.nnz) and K.dtype == torch.float64 and K.is_contiguous()
        mdf = C.c_double(0)
        self._check(self._lib.assemble_residual_tangent(self.h, _ptr(u), quad, _ptr(cells), n_sel, _ptr(r),
                                                        _ptr(f), _ptr(K), C.byref(mdf)))
        return dict(r=r, f=f, K=K, min_detF=mdf.value)

    def greedy_select(self, T, eps, max_nr):
        """Algorithm 1 on T given as [n_cols, n_rows] (column s contiguous)."""
        n_cols, n_rows = T.shape
        S = torch.zeros(max_nr, dtype=torch.int32, device=self.device)
        alpha = torch.zeros((max_nr, n_cols), dtype=torch.float64, device=self.device)
        beta = torch.zeros((max_nr, n_cols), dtype=torch.float64, device=self.device)
        Z = torch.zeros((max_nr, n_rows), dtype=torch.float64, device=self.device)
        mres = np.zeros(max_nr + 1)
        n_r = C.c_int32(0)
        self._check(self._lib.greedy_select(self.h, _ptr(T), n_rows, n_cols, float(eps), int(max_nr), _ptr(S),
                                            C.byref(n_r), _ptr(alpha), _ptr(beta), _ptr(Z),
                                            mres.ctypes.data))
        k = n_r.value
        return dict(S=S[:k], alpha=alpha[:k], beta=beta[:k], Z=Z[:k], max_res=mres[:k + 1])

    def select_principal_cells(self, u, eps, max_nr=256, force_all=False):
        s = self.sizes
        S = torch.zeros(s.n_cells, dtype=torch.int32, device=self.device)
        cap = s.n_cells if force_all else min(max_nr, s.n_cells)
        alpha = torch.zeros((cap, s.n_cells), dtype=torch.float64, device=self.device)
        Kp = torch.zeros((cap, s.nnz), dtype=torch.float64, device=self.device)
        n_r = C.c_int32(0)
        self._check(self._lib.select_principal_cells(self.h, _ptr(u), float(eps), int(max_nr), int(force_all),
                                                     _ptr(S), C.byref(n_r), _ptr(alpha), _ptr(Kp)))
        k = n_r.value
        return dict(S=S[:k], alpha=alpha[:k], Kp=Kp[:k], n_r=k)

    def set_principal_cells(self, u, S, alpha):
        """Caller-given principal cells S (int32 [n_r]) and coefficients alpha ([n_r, n_cells])
        for the reduced tangent action; K^r evaluated at u."""
        S = S.to(device=self.device, dtype=torch.int32).contiguous()
        alpha = alpha.to(device=self.device, dtype=torch.float64).contiguous()
        assert alpha.shape == (S.numel(), self.sizes.n_cells)
        self._check(self._lib.set_principal_cells(self.h, _ptr(u), _ptr(S), int(S.numel()), _ptr(alpha)))

    def apply_reduced_tangent(self, x, y=None):
        y = torch.empty_like(x) if y is None else y
        dtype = {torch.float64: 0, torch.float32: 1}[x.dtype]
        self._check(self._lib.apply_reduced_tangent(self.h, _ptr(x), _ptr(y), dtype))
        return y

    def lattice_default_opts(self, **kw):
        o = NewtonOpts()
        self._check(self._lib.lattice_default_opts(self.h, C.byref(o)))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        return o

    def newton_step(self, u, opts=None, max_iterations=0):
        opts = self.lattice_default_opts() if opts is None else opts
        rep = NewtonReport()
        st = self._lib.newton_step(self.h, _ptr(u), int(max_iterations), C.byref(opts), C.byref(rep))
        self._check(st)
        return rep

    def adjoint_gradient(self, u, opts=None):
        opts = self.lattice_default_opts() if opts is None else opts
        g = self.zeros(self.sizes.n_cells)
        J = C.c_double(0)
        rep = NewtonReport()
        self._check(self._lib.adjoint_gradient(self.h, _ptr(u), C.byref(opts), _ptr(g), C.byref(J), C.byref(rep)))
        return g, J.value, rep

    def lattice_prepare_solver(self, u, opts=None):
        opts = self.lattice_default_opts() if opts is None else opts
        self._check(self._lib.lattice_prepare_solver(self.h, _ptr(u), C.byref(opts)))

    def tangent_solve(self, rhs, opts=None):
        opts = self.lattice_default_opts() if opts is None else opts
        x = self.dof_vector()
        it, rel = C.c_int32(0), C.c_double(0)
        self._check(self._lib.tangent_solve(self.h, _ptr(rhs), _ptr(x), C.byref(opts), C.byref(it), C.byref(rel)))
        return x, it.value, rel.value

    def feti_apply(self, mode, v):
        w = self.krylov_vector()
        self._check(self._lib.feti_apply(self.h, int(mode), _ptr(v), _ptr(w)))
        return w

    def feti_to_global(self, v):
        u = self.dof_vector()
        self._check(self._lib.feti_to_global(self.h, _ptr(v), _ptr(u)))
        return u

    def feti_from_global(self, u):
        v = self.krylov_vector()
        self._check(self._lib.feti_from_global(self.h, _ptr(u), _ptr(v)))
        return v

    def lattice_set_timing(self, enable=True):
        self._check(self._lib.lattice_set_timing(self.h, int(enable)))

    def lattice_kernel_time(self, name):
        """(summed ms, launches) of a named kernel since lattice_set_timing."""
        t, n = C.c_double(0), C.c_int32(0)
        self._check(self._lib.lattice_kernel_time(self.h, name.encode(), C.byref(t), C.byref(n)))
        return t.value, n.value

    def lattice_launch_count(self):
        n = C.c_int64(0)
        self._check(self._lib.lattice_launch_count(self.h, C.byref(n)))
        return n.value

    def lattice_checkpoint_save(self, path, step, load, u, u_prev=None):
        self._check(self._lib.lattice_checkpoint_save(self.h, str(path).encode(), int(step), float(load),
                                                      _ptr(u), _ptr(u_prev)))

    def lattice_checkpoint_load(self, path):
        u, up = self.dof_vector(), self.dof_vector()
        step, load = C.c_int32(0), C.c_double(0)
        self._check(self._lib.lattice_checkpoint_load(self.h, str(path).encode(), C.byref(step), C.byref(load),
                                                      _ptr(u), _ptr(up)))
        return step.value, load.value, u, up
