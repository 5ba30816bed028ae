"""ctypes wrapper of the FP64 CPU oracle (liborsolve).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use it to produce expected values.  The product path never
imports this module.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mgd_oracle.c")
LIB = os.path.join(HERE, "libmgd_oracle.so")

AMG, PCTL, SCHUR1, SCHUR2, BD, BLT = 0, 1, 2, 3, 4, 5
KINDS = {"amg": AMG, "pctl": PCTL, "schur1": SCHUR1, "schur2": SCHUR2, "bd": BD, "blt": BLT}
OP_A, OP_CE, OP_CG, OP_SG, OP_SI, OP_AC, OP_MONO = range(7)


def build(force=False):
    """Compile the oracle with plain gcc: -O2 -ffp-contract=off (no FMA contraction)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "mgd_oracle.h"))):
        return LIB
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
           "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


class Opts(C.Structure):
    _fields_ = [("theta_str", C.c_double), ("max_coarse", C.c_int), ("max_levels", C.c_int),
                ("theta_wd", C.c_double), ("theta_wc", C.c_double), ("sigma_wc", C.c_double),
                ("inner_tol", C.c_double), ("inner_maxit", C.c_int),
                ("nvcyc_group", C.c_int), ("nvcyc_E", C.c_int), ("nvcyc_I", C.c_int),
                ("nvcyc_other", C.c_int), ("jacobi_sweeps", C.c_int), ("adaptive", C.c_int),
                ("seed", C.c_uint64), ("inner_mode", C.c_int), ("interp_type", C.c_int),
                ("smoother", C.c_int), ("agg_levels", C.c_int), ("opt4_steps", C.c_int)]


INV_CB = C.CFUNCTYPE(None, C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                     C.POINTER(C.c_double))

_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.c_void_p
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        u8 = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        i8 = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
        sig = {
            "or_default_opts": (None, [C.POINTER(Opts)]),
            "or_uniform": (C.c_double, [C.c_uint64, C.c_uint64, C.c_uint64]),
            "or_splitmix64": (C.c_uint64, [C.c_uint64, C.c_uint64]),
            "or_csr_new": (P, [C.c_int, C.c_int, C.c_int, ip, ip, dp]),
            "or_csr_info": (None, [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "or_csr_export": (None, [P, ip, ip, dp]),
            "or_csr_free": (None, [P]),
            "or_spmv": (None, [P, dp, dp]),
            "or_transpose": (P, [P]),
            "or_spgemm": (P, [P, P]),
            "or_strength": (None, [P, C.c_double, u8]),
            "or_pmis": (C.c_int, [P, u8, C.c_uint64, C.c_int, i8]),
            "or_pmis_weights": (C.c_int, [P, u8, dp, i8]),
            "or_colour": (C.c_int, [P, C.c_uint64, C.c_int, ip]),
            "or_amg_key": (C.POINTER(C.c_int), [P, C.c_int, C.POINTER(C.c_int)]),
            "or_interp": (P, [P, u8, i8]),
            "or_interp_exti": (P, [P, u8, i8]),
            "or_rap": (P, [P, P]),
            "or_amg_setup": (P, [P, C.POINTER(Opts)]),
            "or_amg_nlevels": (C.c_int, [P]),
            "or_amg_A": (P, [P, C.c_int]),
            "or_amg_P": (P, [P, C.c_int]),
            "or_amg_CF": (C.POINTER(C.c_int8), [P, C.c_int]),
            "or_amg_coarse_is_lu": (C.c_int, [P]),
            "or_vcycle": (None, [P, dp, dp]),
            "or_vcycle_T": (None, [P, dp, dp]),
            "or_amg_free": (None, [P]),
            "or_lu_factor": (C.c_int, [C.c_int, dp, ip]),
            "or_lu_solve": (None, [C.c_int, dp, ip, dp, dp]),
            "or_lu_solve_T": (None, [C.c_int, dp, ip, dp, dp]),
            "or_gamma_wd": (C.c_double, [P, C.c_double]),
            "or_gamma_wc": (C.c_double, [C.c_int, dp, dp, C.c_double]),
            "or_block_setup": (P, [P, C.c_int, C.c_int, C.c_int, C.POINTER(Opts)]),
            "or_block_apply": (None, [P, dp, dp, INV_CB, C.c_void_p]),
            "or_block_apply_T": (None, [P, dp, dp]),
            "or_block_ninv": (C.c_int, [P]),
            "or_block_nmatvec": (C.c_int, [P]),
            "or_block_dropped": (C.c_int, [P, C.c_int, C.c_int]),
            "or_block_use_jacobi": (C.c_int, [P, C.c_int, C.c_int]),
            "or_block_cycles": (C.c_long, [P, C.c_int, C.c_int]),
            "or_block_amg": (P, [P, C.c_int, C.c_int]),
            "or_block_vec": (C.POINTER(C.c_double), [P, C.c_int, C.c_int]),
            "or_block_Ac": (P, [P]),
            "or_block_free": (None, [P]),
            "or_fgmres": (C.c_int, [P, P, C.c_int, dp, dp, C.c_double, C.c_int, C.c_int,
                                    C.POINTER(C.c_int), C.POINTER(C.c_double), dp]),
            "or_grad_vals": (None, [P, dp, dp, dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def opts(**kw):
    o = Opts()
    lib().or_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Csr:
    """Owned oracle CSR handle."""

    def __init__(self, handle, owned=True):
        self.h = handle
        self.owned = owned

    @classmethod
    def from_arrays(cls, n, m, rowptr, col, val):
        rp = np.ascontiguousarray(rowptr, np.int32)
        ci = np.ascontiguousarray(col, np.int32)
        v = np.ascontiguousarray(val, np.float64)
        return cls(lib().or_csr_new(n, m, int(ci.shape[0]), rp, ci, v))

    @classmethod
    def from_scipy(cls, A):
        A = A.tocsr()
        A.sort_indices()
        return cls.from_arrays(A.shape[0], A.shape[1], A.indptr, A.indices, A.data)

    def info(self):
        n, m, z = C.c_int(), C.c_int(), C.c_int()
        lib().or_csr_info(self.h, C.byref(n), C.byref(m), C.byref(z))
        return n.value, m.value, z.value

    def arrays(self):
        n, m, z = self.info()
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(max(z, 1), np.int32)
        v = np.zeros(max(z, 1), np.float64)
        lib().or_csr_export(self.h, rp, ci, v)
        return rp, ci[:z], v[:z]

    def scipy(self):
        import scipy.sparse as sp
        n, m, _ = self.info()
        rp, ci, v = self.arrays()
        return sp.csr_matrix((v, ci, rp), shape=(n, m))

    def __del__(self):
        if self.owned and self.h and _lib is not None:
            _lib.or_csr_free(self.h)
            self.h = None


def csr_of_system(sysm):
    return Csr.from_arrays(sysm.n, sysm.n, sysm.rowptr, sysm.col, sysm.val)


def strength(A: Csr, theta=0.25):
    _, _, z = A.info()
    S = np.zeros(max(z, 1), np.uint8)
    lib().or_strength(A.h, theta, S)
    return S[:z]


def pmis(A: Csr, S, seed=0, level=0):
    n, _, z = A.info()
    CF = np.zeros(max(n, 1), np.int8)
    Sb = np.zeros(max(z, 1), np.uint8)
    Sb[:z] = S
    nc = lib().or_pmis(A.h, Sb, seed, level, CF)
    return nc, CF[:n]


def colour(A: Csr, seed=0, level=0):
    """Jones-Plassmann colouring of the symmetrised graph of A: (ncolours, colour[n])."""
    n = A.info()[0]
    col = np.zeros(max(n, 1), np.int32)
    nc = lib().or_colour(A.h, seed, level, col)
    return nc, col[:n]


def pmis_weights(A: Csr, S, w):
    n, _, z = A.info()
    CF = np.zeros(max(n, 1), np.int8)
    Sb = np.zeros(max(z, 1), np.uint8)
    Sb[:z] = S
    wb = np.zeros(max(n, 1))
    wb[:n] = w
    nc = lib().or_pmis_weights(A.h, Sb, wb, CF)
    return nc, CF[:n]


def interp(A: Csr, S, CF):
    n, _, z = A.info()
    Sb = np.zeros(max(z, 1), np.uint8)
    Sb[:z] = S
    CFb = np.zeros(max(n, 1), np.int8)
    CFb[:n] = CF
    return Csr(lib().or_interp(A.h, Sb, CFb))


def interp_exti(A: Csr, S, CF):
    n, _, z = A.info()
    Sb = np.zeros(max(z, 1), np.uint8)
    Sb[:z] = S
    CFb = np.zeros(max(n, 1), np.int8)
    CFb[:n] = CF
    return Csr(lib().or_interp_exti(A.h, Sb, CFb))


def rap(A: Csr, P: Csr):
    return Csr(lib().or_rap(A.h, P.h))


def transpose(A: Csr):
    return Csr(lib().or_transpose(A.h))


def spgemm(X: Csr, Y: Csr):
    return Csr(lib().or_spgemm(X.h, Y.h))


def spmv(A: Csr, x):
    n, _, _ = A.info()
    y = np.zeros(n)
    lib().or_spmv(A.h, np.ascontiguousarray(x, np.float64), y)
    return y


class Amg:
    def __init__(self, A: Csr, o=None, handle=None, owner=None):
        self._owner = owner
        if handle is not None:
            self.h = handle
            self.owned = False
        else:
            self.h = lib().or_amg_setup(A.h, C.byref(o or opts()))
            self.owned = True

    @property
    def nlevels(self):
        return lib().or_amg_nlevels(self.h)

    def A(self, l):
        return Csr(lib().or_amg_A(self.h, l), owned=False)

    def P(self, l):
        h = lib().or_amg_P(self.h, l)
        return Csr(h, owned=False) if h else None

    def CF(self, l):
        n = self.A(l).info()[0]
        p = lib().or_amg_CF(self.h, l)
        if not p:
            return None
        return np.ctypeslib.as_array(p, shape=(n,)).copy()

    @property
    def coarse_is_lu(self):
        return bool(lib().or_amg_coarse_is_lu(self.h))

    def key(self, l):
        """Gauss-Seidel sweep index per point of level l (smoother 1), and the number of sweeps."""
        nk = C.c_int()
        p = lib().or_amg_key(self.h, l, C.byref(nk))
        if not p:
            return None, 0
        n = self.A(l).info()[0]
        return np.ctypeslib.as_array(p, shape=(n,)).copy(), nk.value

    def vcycle(self, b, transpose=False):
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros_like(b)
        (lib().or_vcycle_T if transpose else lib().or_vcycle)(self.h, b, x)
        return x

    def __del__(self):
        if getattr(self, "owned", False) and self.h and _lib is not None:
            _lib.or_amg_free(self.h)
            self.h = None


class Block:
    def __init__(self, A: Csr, G, N, kind, o=None):
        self.A = A
        self.G, self.N = G, N
        self.kind = KINDS[kind] if isinstance(kind, str) else kind
        self.h = lib().or_block_setup(A.h, G, N, self.kind, C.byref(o or opts()))

    def apply(self, v, cb=None):
        v = np.ascontiguousarray(v, np.float64)
        z = np.zeros_like(v)
        if cb is None:
            lib().or_block_apply(self.h, v, z, INV_CB(), None)
        else:
            def _cb(ctx, op, comp, N, rhs, out):
                r = np.ctypeslib.as_array(rhs, shape=(N,))
                o = np.ctypeslib.as_array(out, shape=(N,))
                o[:] = cb(op, comp, r.copy())
            f = INV_CB(_cb)
            lib().or_block_apply(self.h, v, z, f, None)
        return z

    def apply_T(self, v):
        v = np.ascontiguousarray(v, np.float64)
        z = np.zeros_like(v)
        lib().or_block_apply_T(self.h, v, z)
        return z

    @property
    def ninv(self):
        return lib().or_block_ninv(self.h)

    @property
    def nmatvec(self):
        return lib().or_block_nmatvec(self.h)

    def dropped(self, a, b):
        return bool(lib().or_block_dropped(self.h, a, b))

    def use_jacobi(self, op, comp):
        return bool(lib().or_block_use_jacobi(self.h, op, comp))

    def cycles(self, op, comp):
        return lib().or_block_cycles(self.h, op, comp)

    def amg(self, op, comp):
        h = lib().or_block_amg(self.h, op, comp)
        return Amg(None, handle=h, owner=self) if h else None

    def vec(self, which, comp):
        p = lib().or_block_vec(self.h, which, comp)
        if not p:
            return None
        return np.ctypeslib.as_array(p, shape=(self.N,)).copy()

    def Ac(self):
        h = lib().or_block_Ac(self.h)
        return Csr(h, owned=False) if h else None

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_block_free(self.h)
            self.h = None


def fgmres(A: Csr, b, M: Block | None = None, tol=1e-8, restart=30, maxit=1000, x0=None,
           transpose=False):
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    it = C.c_int()
    rr = C.c_double()
    hist = np.zeros(max(maxit, 1))
    st = lib().or_fgmres(A.h, M.h if M is not None else None, int(transpose), b, x, tol, restart, maxit,
                         C.byref(it), C.byref(rr), hist)
    return x, it.value, rr.value, st, hist[:it.value]


def grad_vals(A: Csr, x, lam):
    _, _, z = A.info()
    g = np.zeros(z)
    lib().or_grad_vals(A.h, np.ascontiguousarray(x, np.float64), np.ascontiguousarray(lam, np.float64), g)
    return g


def gamma_wd(A: Csr, theta=0.9):
    return lib().or_gamma_wd(A.h, theta)


def gamma_wc(d_ab, diag_a, theta=1e-2):
    d = np.ascontiguousarray(d_ab, np.float64)
    return lib().or_gamma_wc(d.shape[0], d, np.ascontiguousarray(diag_a, np.float64), theta)


def lu_factor(a):
    a = np.ascontiguousarray(a, np.float64).copy()
    n = a.shape[0]
    piv = np.zeros(n, np.int32)
    st = lib().or_lu_factor(n, a.reshape(-1), piv)
    return st, a, piv


def lu_solve(lu, piv, b, transpose=False):
    n = lu.shape[0]
    x = np.zeros(n)
    (lib().or_lu_solve_T if transpose else lib().or_lu_solve)(
        n, np.ascontiguousarray(lu).reshape(-1), piv, np.ascontiguousarray(b, np.float64), x)
    return x


def uniform(seed, stream, i):
    return lib().or_uniform(seed, stream, i)
