"""Thin Python binding of libmgdamg.so (the C ABI in include/mgdamg.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
PyTorch provides device memory (tensors whose data pointers are passed in)
and the CUDA stream.  There is no CPU fallback: if the shared library is
missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmgdamg.so")

AMG, PCTL, SCHUR1, SCHUR2, BD, BLT = 0, 1, 2, 3, 4, 5
KINDS = {"amg": AMG, "pctl": PCTL, "schur1": SCHUR1, "schur2": SCHUR2, "bd": BD, "blt": BLT}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOCONV", 3: "EBREAKDOWN", 4: "ESINGULAR", 5: "ENAN", 6: "ETIMEOUT",
          7: "ECUDA", 8: "ENOMEM", 9: "ESTATE"}

# every entry point declared in include/mgdamg.h
ENTRY_POINTS = ["mgd_opts_default", "mgd_create", "mgd_setup", "mgd_update_values", "mgd_solve", "mgd_solve_host",
                "mgd_solve_transpose", "mgd_grad_values", "mgd_precond_apply", "mgd_get_stats", "mgd_get_history",
                "mgd_op_info", "mgd_level_info", "mgd_level_export", "mgd_block_vector", "mgd_coupling_dropped",
                "mgd_profile_enable", "mgd_profile_read", "mgd_kernel_launches", "mgd_last_error", "mgd_destroy", "mgd_plan_info",
                "mgd_setup_phases", "mgd_op_cycles", "mgd_level_keys", "mgd_precond_bench",
                "mgd_relres_noalloc", "mgd_profile_read_fp64", "mgd_fp64_issue_rate", "mgd_setup_host",
                "mgd_check_conversions"]


class MgdOpts(C.Structure):
    _fields_ = [("theta_str", C.c_double), ("max_coarse", C.c_int), ("max_levels", C.c_int),
                ("theta_wd", C.c_double), ("theta_wc", C.c_double), ("sigma_wc", C.c_double),
                ("inner_tol", C.c_double), ("inner_maxit", C.c_int), ("nvcyc_group", C.c_int),
                ("nvcyc_E", C.c_int), ("nvcyc_I", C.c_int), ("nvcyc_other", C.c_int),
                ("jacobi_sweeps", C.c_int), ("adaptive", C.c_int), ("seed", C.c_ulonglong),
                ("restart", C.c_int), ("max_it", C.c_int), ("precision", C.c_int), ("batched", C.c_int),
                ("use_graph", C.c_int), ("autotune", C.c_int), ("keep_transpose", C.c_int),
                ("fuse_rows", C.c_int), ("interp_type", C.c_int), ("pdl", C.c_int), ("inner_mode", C.c_int),
                ("smoother", C.c_int), ("agg_levels", C.c_int), ("arnoldi_resident", C.c_int),
                ("opt4_steps", C.c_int)]


class MgdStats(C.Structure):
    _fields_ = [("kind", C.c_int), ("G", C.c_int), ("N", C.c_int), ("n", C.c_int), ("nnz", C.c_int),
                ("n_ops", C.c_int), ("max_levels_used", C.c_int), ("grid_complexity", C.c_double),
                ("op_complexity", C.c_double), ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("last_iters", C.c_int), ("last_relres", C.c_double), ("vcycle_bytes", C.c_double),
                ("precond_bytes", C.c_double), ("iter_bytes_base", C.c_double), ("n_dropped", C.c_int),
                ("n_jacobi_ops", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load the in-tree shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2002_04958_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        P, I, D = C.c_void_p, C.c_int, C.c_double
        pI, pD, pLL = C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_longlong)
        sig = {
            "mgd_opts_default": (I, [C.POINTER(MgdOpts)]),
            "mgd_create": (I, [C.POINTER(P), C.POINTER(MgdOpts), P]),
            "mgd_setup": (I, [P, I, I, I, I, P, P, P, I]),
            "mgd_update_values": (I, [P, P]),
            "mgd_solve": (I, [P, P, D, P, pI, pD]),
            "mgd_solve_host": (I, [P, P, D, P, pI, pD]),
            "mgd_solve_transpose": (I, [P, P, D, P, pI, pD]),
            "mgd_grad_values": (I, [P, P, P, P]),
            "mgd_precond_apply": (I, [P, P, P]),
            "mgd_get_stats": (I, [P, C.POINTER(MgdStats)]),
            "mgd_get_history": (I, [P, P, I, pI]),
            "mgd_op_info": (I, [P, I, pI, pI, pI, pI, pI]),
            "mgd_level_info": (I, [P, I, I, pI, pI, pI, pI]),
            "mgd_op_cycles": (I, [P, I, pLL]),
            "mgd_precond_bench": (I, [P, P, P, I, pD, pD]),
            "mgd_level_keys": (I, [P, I, I, pI, P]),
            "mgd_level_export": (I, [P, I, I, P, P, P, P, P, P, P]),
            "mgd_block_vector": (I, [P, I, I, I, P]),
            "mgd_coupling_dropped": (I, [P, I, I]),
            "mgd_profile_enable": (I, [P, I]),
            "mgd_profile_read": (I, [P, I, pLL, pD, pD]),
            "mgd_profile_read_fp64": (I, [P, I, pD]),
            "mgd_fp64_issue_rate": (I, [P, pD]),
            "mgd_check_conversions": (I, [P, pLL]),
            "mgd_kernel_launches": (C.c_longlong, []),
            "mgd_relres_noalloc": (I, [I, P, P, P, P, P, P, P]),
            "mgd_setup_host": (I, [P, I, I, I, I, P, P, P, I]),
            "mgd_plan_info": (I, [P, I, I, pI, pI, pI, pI, pI, pI, pI, pI]),
            "mgd_setup_phases": (I, [P, P, I]),
            "mgd_last_error": (C.c_char_p, [P]),
            "mgd_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class MgdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def default_opts(**kw):
    o = MgdOpts()
    lib().mgd_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


NOALLOC_MAX_N = 1 << 19


def relres_noalloc(rowptr, col, val, b, x, out, stream=None):
    """||b - A x||, ||b|| and their ratio into the device tensor out[3], with no
    device allocation inside the library (see mgd_relres_noalloc).

    The library reads these buffers through raw pointers without checking
    them on the device, so everything that would make it read out of bounds
    is checked here first: int32 rowptr (n+1) and col, float64 val, b (n),
    x (n) and out (>= 3), all contiguous and on one CUDA device, and nnz =
    rowptr[-1] entries in col and val.  The call runs with that device current
    and, unless `stream` is given, on that device's current stream."""
    import torch
    named = {"rowptr": rowptr, "col": col, "val": val, "b": b, "x": x, "out": out}
    for k, t in named.items():
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"relres_noalloc: {k} must be a torch.Tensor")
        want = torch.int32 if k in ("rowptr", "col") else torch.float64
        if t.dtype != want:
            raise TypeError(f"relres_noalloc: {k} must be {want}, got {t.dtype}")
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"relres_noalloc: {k} must be a contiguous 1-D tensor")
    n = rowptr.numel() - 1
    if n < 1 or n > NOALLOC_MAX_N:
        raise ValueError(f"relres_noalloc: n = {n} outside [1, {NOALLOC_MAX_N}]")
    if b.numel() != n or x.numel() != n:
        raise ValueError(f"relres_noalloc: b and x need n = {n} entries, got {b.numel()} and {x.numel()}")
    if out.numel() < 3:
        raise ValueError("relres_noalloc: out needs 3 entries")
    for k, t in named.items():
        if not t.is_cuda:
            raise ValueError(f"relres_noalloc: {k} must be a CUDA tensor")
    dev = rowptr.device
    for k, t in named.items():
        if t.device != dev:
            raise ValueError(f"relres_noalloc: {k} is on {t.device}, rowptr on {dev}")
    nnz = int(rowptr[-1].item())
    if int(rowptr[0].item()) != 0 or nnz > col.numel() or nnz > val.numel():
        raise ValueError(f"relres_noalloc: rowptr[0] must be 0 and rowptr[-1] = {nnz} <= len(col), len(val)")
    if nnz > 0 and (int(col.min().item()) < 0 or int(col.max().item()) >= n
                    or bool((rowptr[1:] < rowptr[:-1]).any().item())):
        raise ValueError("relres_noalloc: rowptr must be non-decreasing and columns in [0, n)")
    with torch.cuda.device(dev):
        st = stream or torch.cuda.current_stream(dev)
        return lib().mgd_relres_noalloc(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(b), _ptr(x), _ptr(out),
                                        C.c_void_p(st.cuda_stream))


def kernel_launches():
    return lib().mgd_kernel_launches()


def fp64_issue_rate(stream=None):
    """FP64 multiply-add lane operations per second of the current device (measured)."""
    import torch
    st = stream or torch.cuda.current_stream()
    r = C.c_double()
    rc = lib().mgd_fp64_issue_rate(C.c_void_p(st.cuda_stream), C.byref(r))
    if rc != 0:
        raise MgdError(rc, "mgd_fp64_issue_rate failed")
    return r.value


def check_conversions(stream=None):
    """Mismatches of the library's integer-pipe binary32 <-> binary64
    conversions against the hardware ones (expected 0)."""
    import torch
    st = stream or torch.cuda.current_stream()
    r = C.c_longlong()
    rc = lib().mgd_check_conversions(C.c_void_p(st.cuda_stream), C.byref(r))
    if rc != 0:
        raise MgdError(rc, "mgd_check_conversions failed")
    return r.value


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Solver:
    """One context of the CUDA library bound to a torch CUDA stream."""

    def __init__(self, stream=None, **opts):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the solver needs a CUDA device")
        self.torch = torch
        # a dedicated stream (graph capture cannot use the legacy default
        # stream); every call first orders it after torch's current stream
        self.stream = stream or torch.cuda.Stream()
        self.opts = default_opts(**opts)
        h = C.c_void_p()
        rc = lib().mgd_create(C.byref(h), C.byref(self.opts), C.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise MgdError(rc, "mgd_create failed")
        self.h = h
        self.n = 0
        self.nnz = 0
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._keep = []

    def _vec(self, a, length, name, dtype=None):
        """a as a contiguous CUDA tensor on the context's device with `length`
        entries (float64 unless dtype is given): the library reads and writes
        these buffers through raw pointers, so a short or misplaced one is
        refused here instead of being read out of bounds."""
        t = self.torch
        a = a if isinstance(a, t.Tensor) else t.as_tensor(a)
        a = a.to(device=self.device, dtype=dtype or t.float64).contiguous()
        if a.dim() != 1 or a.numel() != length:
            raise ValueError(f"{name}: expected {length} entries, got shape {tuple(a.shape)}")
        return a

    def _need_setup(self):
        if self.n <= 0:
            raise MgdError(9, "call setup first")

    def _order(self):
        self.stream.wait_stream(self.torch.cuda.current_stream())

    def _check(self, rc, allow=()):
        if rc != 0 and rc not in allow:
            raise MgdError(rc, lib().mgd_last_error(self.h).decode())
        return rc

    def setup(self, G, N, rowptr, col, val, kind):
        t = self.torch
        kind = KINDS[kind] if isinstance(kind, str) else kind
        rowptr = rowptr.to(device=self.device, dtype=t.int32).contiguous()
        col = col.to(device=self.device, dtype=t.int32).contiguous()
        val = self._vec(val, col.numel(), "val")
        n = rowptr.numel() - 1
        self._order()
        self._check(lib().mgd_setup(self.h, G, N, n, col.numel(), _ptr(rowptr), _ptr(col), _ptr(val), kind))
        self.G, self.N, self.n, self.nnz, self.kind = G, N, n, col.numel(), kind
        self.rowptr, self.col = rowptr, col
        return self

    def setup_host(self, G, N, rowptr, col, val, kind):
        """Setup from host arrays (numpy or CPU torch tensors: int32 rowptr/col,
        float64 val); the library copies them to the device."""
        t = self.torch
        kind = KINDS[kind] if isinstance(kind, str) else kind

        def host(a, dt, tdt):
            if isinstance(a, t.Tensor):
                if a.is_cuda or a.dtype != tdt or not a.is_contiguous():
                    raise ValueError("setup_host wants contiguous CPU tensors of dtype %s" % tdt)
                return a, a.data_ptr()
            a = np.ascontiguousarray(a, dt)
            return a, a.ctypes.data
        rp, prp = host(rowptr, np.int32, t.int32)
        ci, pci = host(col, np.int32, t.int32)
        va, pva = host(val, np.float64, t.float64)
        n = int(rp.shape[0]) - 1
        nnz = int(ci.shape[0])
        if int(va.shape[0]) != nnz:
            raise ValueError("setup_host: col and val lengths differ")
        self._order()
        self._check(lib().mgd_setup_host(self.h, G, N, n, nnz, C.c_void_p(prp), C.c_void_p(pci), C.c_void_p(pva),
                                         kind))
        self.G, self.N, self.n, self.nnz, self.kind = G, N, n, nnz, kind
        self.rowptr, self.col = None, None
        return self

    def setup_system(self, sysm, kind):
        t = self.torch
        return self.setup(sysm.G, sysm.N, t.from_numpy(sysm.rowptr), t.from_numpy(sysm.col),
                          t.from_numpy(sysm.val), kind)

    def update_values(self, val):
        self._need_setup()
        val = self._vec(val, self.nnz, "val")
        self._order()
        self._check(lib().mgd_update_values(self.h, _ptr(val)))

    def solve(self, b, tol=1e-8, x0=None, allow_noconv=False):
        t = self.torch
        self._need_setup()
        b = self._vec(b, self.n, "b")
        x = t.zeros_like(b) if x0 is None else self._vec(x0, self.n, "x0").clone()
        it, rr = C.c_int(), C.c_double()
        self._order()
        rc = self._check(lib().mgd_solve(self.h, _ptr(b), tol, _ptr(x), C.byref(it), C.byref(rr)),
                         allow=(2,) if allow_noconv else ())
        return x, it.value, rr.value, rc

    def solve_host(self, b, tol=1e-8, x0=None):
        """Host buffers in and out (numpy float64); copies inside the library."""
        self._need_setup()
        b = np.ascontiguousarray(b, np.float64).reshape(-1)
        x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64).reshape(-1)
        if b.size != self.n or x.size != self.n:
            raise ValueError(f"solve_host: b and x0 need {self.n} entries")
        it, rr = C.c_int(), C.c_double()
        self._order()
        self._check(lib().mgd_solve_host(self.h, b.ctypes.data_as(C.c_void_p), tol, x.ctypes.data_as(C.c_void_p),
                                          C.byref(it), C.byref(rr)))
        return x, it.value, rr.value

    def solve_host_ptr(self, b_ptr, x_ptr, tol=1e-8):
        """Raw host addresses of n float64 values each (b in; x: initial guess
        in, solution out), e.g. the data_ptr() of page-locked CPU tensors; the
        caller vouches for their size."""
        self._need_setup()
        it, rr = C.c_int(), C.c_double()
        self._order()
        self._check(lib().mgd_solve_host(self.h, C.c_void_p(b_ptr), tol, C.c_void_p(x_ptr), C.byref(it),
                                         C.byref(rr)))
        return it.value, rr.value

    def solve_transpose(self, g, tol=1e-8):
        t = self.torch
        self._need_setup()
        g = self._vec(g, self.n, "g")
        lam = t.zeros_like(g)
        it, rr = C.c_int(), C.c_double()
        self._order()
        self._check(lib().mgd_solve_transpose(self.h, _ptr(g), tol, _ptr(lam), C.byref(it), C.byref(rr)))
        return lam, it.value, rr.value

    def grad_values(self, x, lam):
        self._need_setup()
        x = self._vec(x, self.n, "x")
        lam = self._vec(lam, self.n, "lam")
        g = self.torch.empty(self.nnz, dtype=self.torch.float64, device=self.device)
        self._order()
        self._check(lib().mgd_grad_values(self.h, _ptr(x), _ptr(lam), _ptr(g)))
        return g

    def precond_apply(self, v):
        self._need_setup()
        v = self._vec(v, self.n, "v")
        z = self.torch.empty_like(v)
        self._order()
        self._check(lib().mgd_precond_apply(self.h, _ptr(v), _ptr(z)))
        return z

    def precond_bench(self, v, count=100):
        """(ms per apply, algorithmic bytes per apply) of `count` preconditioner applies back to back."""
        self._need_setup()
        v = self._vec(v, self.n, "v")
        z = self.torch.empty_like(v)
        ms, by = C.c_double(), C.c_double()
        self._order()
        self._check(lib().mgd_precond_bench(self.h, _ptr(v), _ptr(z), int(count), C.byref(ms), C.byref(by)))
        return ms.value, by.value

    def stats(self):
        s = MgdStats()
        self._check(lib().mgd_get_stats(self.h, C.byref(s)))
        return s.as_dict()

    def history(self):
        cnt = C.c_int()
        lib().mgd_get_history(self.h, None, 0, C.byref(cnt))
        h = np.zeros(max(cnt.value, 1))
        lib().mgd_get_history(self.h, h.ctypes.data_as(C.c_void_p), cnt.value, C.byref(cnt))
        return h[:cnt.value]

    def op_info(self, op):
        v = [C.c_int() for _ in range(5)]
        self._check(lib().mgd_op_info(self.h, op, *[C.byref(x) for x in v]))
        return dict(zip(["kind", "comp", "nlevels", "use_jacobi", "coarse_lu"], [x.value for x in v]))

    def op_cycles(self, op):
        """V-cycles applied by operator op's inverse since setup (forward and transposed applies)."""
        v = C.c_longlong()
        self._check(lib().mgd_op_cycles(self.h, op, C.byref(v)))
        return v.value

    def level_keys(self, op, l):
        """Gauss-Seidel sweep index per point of level l of operator op (None without GS there)."""
        nk = C.c_int()
        self._check(lib().mgd_level_keys(self.h, op, l, C.byref(nk), None))
        if nk.value == 0:
            return None, 0
        n = C.c_int()
        self._check(lib().mgd_level_info(self.h, op, l, C.byref(n), None, None, None))
        key = np.zeros(n.value, np.int32)
        self._check(lib().mgd_level_keys(self.h, op, l, C.byref(nk), key.ctypes.data_as(C.c_void_p)))
        return key, nk.value

    def total_cycles(self):
        """V-cycles applied by every inverse since setup."""
        return sum(self.op_cycles(k) for k in range(self.stats()["n_ops"]))

    def level_info(self, op, l):
        """Sizes of level l of operator op: rows, nonzeros, nonzeros of P, coarse rows."""
        n, nnz, nnzp, ncoarse = (C.c_int() for _ in range(4))
        self._check(lib().mgd_level_info(self.h, op, l, C.byref(n), C.byref(nnz), C.byref(nnzp), C.byref(ncoarse)))
        return dict(n=n.value, nnz=nnz.value, nnzp=nnzp.value, ncoarse=ncoarse.value)

    def level(self, op, l):
        """Host copies of level l of operator op: A (rp, ci, v), CF, P (rp, ci, v)."""
        n, nnz, nnzp, ncoarse = (C.c_int() for _ in range(4))
        self._check(lib().mgd_level_info(self.h, op, l, C.byref(n), C.byref(nnz), C.byref(nnzp),
                                         C.byref(ncoarse)))
        n, nnz, nnzp = n.value, nnz.value, nnzp.value
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(max(nnz, 1), np.int32)
        v = np.zeros(max(nnz, 1))
        cf = np.zeros(max(n, 1), np.int8)
        prp = np.zeros(n + 1, np.int32)
        pci = np.zeros(max(nnzp, 1), np.int32)
        pv = np.zeros(max(nnzp, 1))
        vp = lambda a: a.ctypes.data_as(C.c_void_p)
        self._check(lib().mgd_level_export(self.h, op, l, vp(rp), vp(ci), vp(v), vp(cf), vp(prp), vp(pci), vp(pv)))
        out = dict(n=n, rp=rp, ci=ci[:nnz], v=v[:nnz], nc=ncoarse.value)
        if nnzp:
            out.update(cf=cf[:n], prp=prp, pci=pci[:nnzp], pv=pv[:nnzp])
        return out

    SETUP_PHASES = ["strength", "pmis", "interp", "transpose", "AP", "RAP", "finalize", "coarse_inverse",
                    "validate", "blocks", "hierarchies_wall", "pctl", "program_autotune", "krylov_graph",
                    "gs_colouring", "h2d_copies", "release_previous"]

    def setup_phases(self):
        ms = np.zeros(len(self.SETUP_PHASES))
        self._check(lib().mgd_setup_phases(self.h, ms.ctypes.data_as(C.c_void_p), len(self.SETUP_PHASES)))
        return {k: round(float(v), 3) for k, v in zip(self.SETUP_PHASES, ms)}

    def plan(self):
        """Autotuned launch plan: one list of per-level dicts per V-cycle batch."""
        out = []
        nb = C.c_int()
        v = [C.c_int() for _ in range(7)]  # depth, nsub, maxrows, fmtA, fmtR, fmtP, tail
        if lib().mgd_plan_info(self.h, 0, 0, C.byref(nb), *[C.byref(x) for x in v]) != 0:
            return out
        for b in range(nb.value):
            lib().mgd_plan_info(self.h, b, 0, C.byref(nb), *[C.byref(x) for x in v])
            depth, tail = v[0].value, v[6].value
            levels = []
            for l in range(depth):
                lib().mgd_plan_info(self.h, b, l, C.byref(nb), *[C.byref(x) for x in v])
                levels.append(dict(nsub=v[1].value, maxrows=v[2].value, fmtA=v[3].value, fmtR=v[4].value,
                                   fmtP=v[5].value))
            out.append(dict(depth=depth, tail=tail, levels=levels))
        return out

    def block_vector(self, which, comp, comp2=0):
        out = np.zeros(self.N)
        rc = lib().mgd_block_vector(self.h, which, comp, comp2, out.ctypes.data_as(C.c_void_p))
        return out if rc == 0 else None

    def coupling_dropped(self, a, b):
        return bool(lib().mgd_coupling_dropped(self.h, a, b))

    def profile(self, mask=-1):
        """mask: bit k records kernel class k (0 off, -1 all)."""
        self._check(lib().mgd_profile_enable(self.h, int(mask)))

    def profile_read(self, cls):
        nl, ms, by = C.c_longlong(), C.c_double(), C.c_double()
        self._check(lib().mgd_profile_read(self.h, cls, C.byref(nl), C.byref(ms), C.byref(by)))
        return nl.value, ms.value, by.value

    def profile_read_fp64(self, cls):
        """Algorithmic FP64 lane operations of the launches class cls recorded."""
        f = C.c_double()
        self._check(lib().mgd_profile_read_fp64(self.h, cls, C.byref(f)))
        return f.value

    def close(self):
        if getattr(self, "h", None):
            lib().mgd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class MGDSolve(torch.autograd.Function):
        """x = A(vals)^{-1} b with the GPU solver; backward solves A^T lambda = dL/dx
        with the transposed preconditioner and returns dL/dvals = -lambda_row x_col,
        dL/db = lambda."""

        @staticmethod
        def forward(ctx, vals, b, solver, tol):
            solver.update_values(vals.detach())
            x, it, rr, _ = solver.solve(b.detach(), tol)
            ctx.solver = solver
            ctx.tol = tol
            ctx.save_for_backward(x)
            return x

        @staticmethod
        def backward(ctx, gx):
            (x,) = ctx.saved_tensors
            lam, it, rr = ctx.solver.solve_transpose(gx.contiguous(), ctx.tol)
            gvals = ctx.solver.grad_values(x, lam)
            return gvals, lam, None, None

    return MGDSolve


def mgd_solve(vals, b, solver, tol=1e-8):
    """Differentiable solve (see MGDSolve)."""
    return _autograd_function().apply(vals, b, solver, tol)
