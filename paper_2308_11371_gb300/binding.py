"""ctypes binding of the C ABI in ``include/fetidp.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libfetidp.so``; this module
only converts a :class:`~paper_2308_11371_gb300.workloads.LatticeProblem` into
the ``fetidp_problem`` struct and passes device pointers of torch tensors.
There is no fallback: if the library is missing or CUDA is unavailable the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build
from .workloads import LatticeProblem

FETIDP_FP64 = 0
FETIDP_MIXED_BF16 = 1

STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error",
          -4: "not converged", -5: "device wait timed out", -6: "singular", -7: "Krylov breakdown"}

SYMBOLS = ["fetidp_sizes", "fetidp_default_options", "fetidp_setup", "fetidp_apply_F",
           "fetidp_precond", "fetidp_solve", "fetidp_solve_host", "fetidp_grad", "fetidp_gather_BT",
           "fetidp_scatter_B", "fetidp_apply_K", "fetidp_coarse_solve", "fetidp_local_rom_solve",
           "fetidp_apply_A", "fetidp_apply_P", "fetidp_rom_data", "fetidp_destroy",
           "fetidp_status_string", "fetidp_last_error", "fetidp_profile_enable",
           "fetidp_profile_read", "fetidp_kernel_launches", "fetidp_tc_selfcheck",
           "fetidp_tc_comb_selfcheck", "fetidp_tc_selfcheck_static",
           "fetidp_compliance", "fetidp_batch_layout", "fetidp_wait_selfcheck",
           "fetidp_precond_rom", "fetidp_tc_time"]

KCLASS = {"grouped_gemm": 0, "apply_K": 1, "maps": 2, "coarse": 3, "cell_gemv": 4, "vector": 5,
          "gram": 6, "tc_gemm": 7, "setup": 8, "sweep": 9, "traces": 10, "greedy": 11, "multi_K": 12,
          "asm_op": 13}


class FetidpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)} ({status}): {msg}")
        self.status = status


class Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("cells", ctypes.c_int * 3), ("elems", ctypes.c_int),
        ("nu", ctypes.c_double), ("E_solid", ctypes.c_double), ("E_void", ctypes.c_double),
        ("mask_kind", ctypes.c_int), ("mask_width", ctypes.c_double),
        ("r_cell", ctypes.POINTER(ctypes.c_double)),
        ("map_kind", ctypes.c_int), ("map_params", ctypes.c_double * 8),
        ("clamp_axis", ctypes.c_int), ("clamp_side", ctypes.c_int),
        ("n_loads", ctypes.c_int),
        ("load_kind", ctypes.POINTER(ctypes.c_int)), ("load_axis", ctypes.POINTER(ctypes.c_int)),
        ("load_side", ctypes.POINTER(ctypes.c_int)), ("load_dir", ctypes.POINTER(ctypes.c_double)),
        ("n_rb", ctypes.c_int), ("tol_rb", ctypes.c_double),
    ]


class Options(ctypes.Structure):
    _fields_ = [("tol_outer", ctypes.c_double), ("tol_inner", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("max_inner", ctypes.c_int),
                ("precision", ctypes.c_int), ("fixed_outer", ctypes.c_int),
                ("fixed_inner", ctypes.c_int), ("tc_split", ctypes.c_int),
                ("tol_inner_mixed", ctypes.c_double), ("gram_drop_mixed", ctypes.c_double),
                ("profile_mask", ctypes.c_uint), ("restart", ctypes.c_int),
                ("wait_budget_ns", ctypes.c_longlong), ("check_inputs", ctypes.c_int),
                ("mixed_assembled", ctypes.c_int), ("interface", ctypes.c_int), ("method", ctypes.c_int),
                ("tc_bn", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("outer_its", ctypes.c_int), ("inner_its_total", ctypes.c_int),
                ("n_rb", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("t_setup_s", ctypes.c_double), ("t_solve_s", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("kernel_launches", ctypes.c_longlong),
                ("host_launches", ctypes.c_longlong), ("inner_graph", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB: Optional[ctypes.CDLL] = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load the CUDA library (raises if it is not built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built ({_build.LIB}); run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P, V, I = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int
    lib.fetidp_status_string.restype = ctypes.c_char_p
    lib.fetidp_status_string.argtypes = [I]
    lib.fetidp_last_error.restype = ctypes.c_char_p
    lib.fetidp_last_error.argtypes = []
    lib.fetidp_default_options.restype = None
    lib.fetidp_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.fetidp_setup.restype = I
    lib.fetidp_setup.argtypes = [ctypes.POINTER(Problem), I, ctypes.POINTER(Options), V,
                                 ctypes.POINTER(P)]
    lib.fetidp_sizes.restype = I
    lib.fetidp_sizes.argtypes = [P, ctypes.POINTER(ctypes.c_longlong)]
    for name in ("fetidp_apply_F", "fetidp_precond", "fetidp_precond_rom", "fetidp_gather_BT", "fetidp_scatter_B",
                 "fetidp_apply_K", "fetidp_coarse_solve", "fetidp_local_rom_solve",
                 "fetidp_apply_A", "fetidp_apply_P"):
        f = getattr(lib, name)
        f.restype = I
        f.argtypes = [P, V, V]
    lib.fetidp_solve.restype = I
    lib.fetidp_solve.argtypes = [P, V, V, ctypes.POINTER(Info)]
    lib.fetidp_solve_host.restype = I
    lib.fetidp_solve_host.argtypes = [P, V, V, ctypes.POINTER(Info)]
    lib.fetidp_grad.restype = I
    lib.fetidp_grad.argtypes = [P, V, V, V]
    lib.fetidp_compliance.restype = I
    lib.fetidp_compliance.argtypes = [P, V, V]
    lib.fetidp_batch_layout.restype = I
    lib.fetidp_batch_layout.argtypes = [P, V, V, V]
    lib.fetidp_rom_data.restype = I
    lib.fetidp_rom_data.argtypes = [P, V, V, V, V]
    lib.fetidp_destroy.restype = None
    lib.fetidp_destroy.argtypes = [P]
    lib.fetidp_profile_enable.restype = I
    lib.fetidp_profile_enable.argtypes = [P, ctypes.c_uint]
    lib.fetidp_profile_read.restype = I
    lib.fetidp_profile_read.argtypes = [P, V, V, V, V]
    lib.fetidp_tc_comb_selfcheck.restype = I
    lib.fetidp_tc_comb_selfcheck.argtypes = [I, I, I, I, I, ctypes.POINTER(ctypes.c_double)]
    lib.fetidp_tc_selfcheck.restype = I
    lib.fetidp_tc_selfcheck.argtypes = [I, I, I, ctypes.POINTER(ctypes.c_double)]
    lib.fetidp_tc_selfcheck_static.restype = I
    lib.fetidp_tc_selfcheck_static.argtypes = [I, I, I, ctypes.POINTER(ctypes.c_double), V]
    lib.fetidp_wait_selfcheck.restype = I
    lib.fetidp_wait_selfcheck.argtypes = [ctypes.c_longlong, V, ctypes.POINTER(ctypes.c_double)]
    lib.fetidp_tc_time.restype = I
    lib.fetidp_tc_time.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.fetidp_kernel_launches.restype = ctypes.c_longlong
    lib.fetidp_kernel_launches.argtypes = []
    _LIB = lib
    return lib


def _check(status: int):
    if status != 0:
        msg = load().fetidp_last_error().decode(errors="replace")
        raise FetidpError(status, msg)


def class_mask(names) -> int:
    """Bit mask of the kernel classes named (KCLASS keys; None = all)."""
    mask = 0
    for n in (list(KCLASS) if names is None else names):
        mask |= 1 << KCLASS[n]
    return mask


def default_options(**kw) -> Options:
    """Library defaults with the given fields replaced; ``profile=[classes]`` sets profile_mask."""
    if "profile" in kw:
        kw["profile_mask"] = class_mask(kw.pop("profile"))
    o = Options()
    load().fetidp_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def make_problem_struct(p: LatticeProblem):
    """fetidp_problem for ``p``; returns (struct, keep-alive arrays)."""
    d = p.dim
    r = np.ascontiguousarray(p.r_cell, dtype=np.float64)
    kind = np.array([ld.kind for ld in p.loads], dtype=np.int32)
    axis = np.array([ld.axis for ld in p.loads], dtype=np.int32)
    side = np.array([ld.side for ld in p.loads], dtype=np.int32)
    ldir = np.ascontiguousarray(np.array([ld.direction[:d] for ld in p.loads], dtype=np.float64).ravel())
    s = Problem()
    s.dim = d
    s.cells[:] = list(p.cells)
    s.elems = p.elems
    s.nu, s.E_solid, s.E_void = p.nu, p.E_solid, p.E_void
    s.mask_kind, s.mask_width = p.mask_kind, p.mask_width
    s.r_cell = r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    s.map_kind = p.map_kind
    s.map_params[:] = list(p.map_params_array())
    s.clamp_axis, s.clamp_side = p.clamp_axis, p.clamp_side
    s.n_loads = len(p.loads)
    s.load_kind = kind.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    s.load_axis = axis.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    s.load_side = side.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    s.load_dir = ldir.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    s.n_rb, s.tol_rb = p.n_rb, p.tol_rb
    return s, (r, kind, axis, side, ldir)


def _ptr(t) -> int:
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float64 tensor")
    return t.data_ptr()


class Solver:
    """One FETI-DP context on the current CUDA device and torch's current stream."""

    def __init__(self, problem, precision: int = FETIDP_FP64, stream=None, **opts):
        """``problem``: one LatticeProblem, or a list of them solved together as a batch."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available; the FETI-DP library has no CPU path")
        lib = load()
        probs = list(problem) if isinstance(problem, (list, tuple)) else [problem]
        self.problem = problem
        self.n_lattices = len(probs)
        if precision == FETIDP_MIXED_BF16 and "tc_bn" not in opts:
            from . import tune   # the measured tile width of this problem shape, if tabulated
            opts = dict(opts, tc_bn=tune.table_choice(probs))
        self.options = default_options(precision=precision, **opts)
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        arr = (Problem * len(probs))()
        self._keep = []
        for i, q in enumerate(probs):
            s, keep = make_problem_struct(q)
            arr[i] = s
            self._keep.append(keep)
        h = ctypes.c_void_p()
        _check(lib.fetidp_setup(arr, len(probs), ctypes.byref(self.options),
                                ctypes.c_void_p(st.cuda_stream), ctypes.byref(h)))
        self._h = h
        sz = (ctypes.c_longlong * 12)()
        _check(lib.fetidp_sizes(h, sz))
        (self.N, self.n_dof, self.n_i, self.n_d, self.n_p, self.n_r, self.L, self.n_P,
         self.n_rhs, self.n_rb, self.n_snap, self.n_tot) = [int(v) for v in sz]

    # ---- helpers
    def _empty(self, *shape):
        import torch
        return torch.empty(*shape, dtype=torch.float64, device="cuda")

    def _call2(self, name, x, out):
        _check(getattr(load(), name)(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(out))))
        return out

    # ---- entry points
    def apply_F(self, lam, out=None):
        return self._call2("fetidp_apply_F", lam, out if out is not None else self._empty(self.n_rhs, self.L))

    def precond(self, r, out=None):
        return self._call2("fetidp_precond", r, out if out is not None else self._empty(self.n_rhs, self.L))

    def tc_time(self, bn: int, reps: int = 3) -> float:
        """Mean device time (ms) of this context's Eq. 46a tensor-core GEMM at column-tile width bn."""
        ms = ctypes.c_double(0.0)
        _check(load().fetidp_tc_time(self._h, int(bn), int(reps), ctypes.byref(ms)))
        return ms.value

    def precond_rom(self, r, out=None):
        """M_D^{-ROM} r (Eq. 47); needs a context set up with interface=1."""
        return self._call2("fetidp_precond_rom", r, out if out is not None else self._empty(self.n_rhs, self.L))

    def gather_BT(self, lam, out=None):
        o = out if out is not None else self._empty(self.n_rhs, self.N, self.n_d)
        return self._call2("fetidp_gather_BT", lam, o)

    def scatter_B(self, yd, out=None):
        return self._call2("fetidp_scatter_B", yd, out if out is not None else self._empty(self.n_rhs, self.L))

    def apply_K(self, u, out=None):
        o = out if out is not None else self._empty(self.n_rhs, self.N, self.n_dof)
        return self._call2("fetidp_apply_K", u, o)

    def coarse_solve(self, b, out=None):
        return self._call2("fetidp_coarse_solve", b, out if out is not None else self._empty(self.n_rhs, self.n_P))

    def local_rom_solve(self, v, out=None):
        o = out if out is not None else self._empty(self.n_rhs, self.N, self.n_r)
        return self._call2("fetidp_local_rom_solve", v, o)

    def apply_A(self, x, out=None):
        return self._call2("fetidp_apply_A", x, out if out is not None else self._empty(self.n_rhs, self.n_tot))

    def apply_P(self, x, out=None):
        return self._call2("fetidp_apply_P", x, out if out is not None else self._empty(self.n_rhs, self.n_tot))

    def solve(self, u=None, lam=None, allow_notconv=False):
        """Returns (u [rhs][N][n_dof], lambda [rhs][L], info dict)."""
        u = u if u is not None else self._empty(self.n_rhs, self.N, self.n_dof)
        lam = lam if lam is not None else self._empty(self.n_rhs, self.L)
        info = Info()
        st = load().fetidp_solve(self._h, ctypes.c_void_p(_ptr(u)), ctypes.c_void_p(_ptr(lam)),
                                 ctypes.byref(info))
        if not (allow_notconv and st == -4):
            _check(st)
        d = info.as_dict()
        d["status"] = st
        return u, lam, d

    def solve_host(self, u_host: np.ndarray, lam_host: Optional[np.ndarray] = None):
        """Solve with HOST output buffers (copies inside the call)."""
        info = Info()
        assert u_host.dtype == np.float64 and u_host.flags.c_contiguous
        lp = lam_host.ctypes.data if lam_host is not None else None
        _check(load().fetidp_solve_host(self._h, ctypes.c_void_p(u_host.ctypes.data),
                                        ctypes.c_void_p(lp), ctypes.byref(info)))
        return info.as_dict()

    def grad(self, u, w=None, out=None):
        o = out if out is not None else self._empty(self.n_rhs, self.N)
        wp = ctypes.c_void_p(_ptr(w)) if w is not None else ctypes.c_void_p(None)
        _check(load().fetidp_grad(self._h, ctypes.c_void_p(_ptr(u)), wp, ctypes.c_void_p(_ptr(o))))
        return o

    def compliance(self, u):
        """c[l] = sum_s f_l^(s) . u_l^(s) per load case (host numpy array)."""
        c = np.zeros(self.n_rhs)
        _check(load().fetidp_compliance(self._h, ctypes.c_void_p(_ptr(u)), ctypes.c_void_p(c.ctypes.data)))
        return c

    def batch_layout(self):
        """(cell0, L0, P0): first cell, multiplier row and primal DOF of every lattice, then the
        totals (numpy arrays of n_lattices + 1 entries)."""
        B = self.n_lattices
        cell0, L0, P0 = (np.zeros(B + 1, np.int64) for _ in range(3))
        _check(load().fetidp_batch_layout(self._h, ctypes.c_void_p(cell0.ctypes.data),
                                          ctypes.c_void_p(L0.ctypes.data), ctypes.c_void_p(P0.ctypes.data)))
        return cell0, L0, P0

    def rom_data(self):
        k, N = self.n_rb, self.N
        sigma = np.zeros(k, np.int32)
        alpha, pi, delta = (np.zeros((N, k)) for _ in range(3))
        _check(load().fetidp_rom_data(self._h, ctypes.c_void_p(sigma.ctypes.data),
                                      ctypes.c_void_p(alpha.ctypes.data),
                                      ctypes.c_void_p(pi.ctypes.data),
                                      ctypes.c_void_p(delta.ctypes.data)))
        return sigma, alpha, pi, delta

    def profile_enable(self, classes=None):
        """Time the given kernel classes (names of KCLASS; None = all)."""
        _check(load().fetidp_profile_enable(self._h, class_mask(classes)))

    def profile_disable(self):
        _check(load().fetidp_profile_enable(self._h, 0))

    def profile_read(self):
        """{class: {ms, launches, flops, bytes}} since the last enable/read."""
        n = 16
        ms = np.zeros(n); fl = np.zeros(n); by = np.zeros(n)
        la = np.zeros(n, np.int64)
        _check(load().fetidp_profile_read(self._h, ctypes.c_void_p(ms.ctypes.data),
                                          ctypes.c_void_p(la.ctypes.data),
                                          ctypes.c_void_p(fl.ctypes.data),
                                          ctypes.c_void_p(by.ctypes.data)))
        return {k: {"ms": float(ms[i]), "launches": int(la[i]), "flops": float(fl[i]),
                    "bytes": float(by[i])} for k, i in KCLASS.items()}

    def close(self):
        if getattr(self, "_h", None):
            load().fetidp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load().fetidp_kernel_launches())


def tc_selfcheck(M: int, K: int, N: int) -> float:
    """Max relative error of the tcgen05 GEMM against FP64 on the same BF16 inputs."""
    err = ctypes.c_double()
    _check(load().fetidp_tc_selfcheck(M, K, N, ctypes.byref(err)))
    return err.value


def tc_comb_selfcheck(M0: int, M1: int, K: int, N: int, nops: int) -> float:
    """Max relative error of the fused combine kernel against FP64 on the same BF16 inputs."""
    err = ctypes.c_double()
    _check(load().fetidp_tc_comb_selfcheck(M0, M1, K, N, nops, ctypes.byref(err)))
    return err.value


# Size of the static device scratch of tc_selfcheck_static (FETIDP_TC_STATIC_SCRATCH_BYTES).
TC_STATIC_SCRATCH_BYTES = 4194304


def tc_selfcheck_static(M: int, K: int, N: int, stream: int = 0) -> float:
    """tc_selfcheck without any device allocation: all buffers live in the library's fixed
    4 MiB device scratch (shapes that do not fit raise EINVAL).  stream: raw cudaStream_t
    handle, 0 for the legacy default stream.  Calls that overlap in time race on the scratch."""
    err = ctypes.c_double()
    _check(load().fetidp_tc_selfcheck_static(M, K, N, ctypes.byref(err), ctypes.c_void_p(stream or None)))
    return err.value


def wait_selfcheck(wait_budget_ns: int, stream: int = 0):
    """Run the bounded-wait probe; returns (status, seconds waited).  The expected status is
    FETIDP_ETIMEOUT (-5): the probe waits on a barrier nothing completes."""
    waited = ctypes.c_double()
    st = load().fetidp_wait_selfcheck(int(wait_budget_ns), ctypes.c_void_p(stream or None), ctypes.byref(waited))
    return int(st), waited.value
