"""Seeded synthetic inputs: (G+2)x(G+2)-block radiation-diffusion systems.

This module is the only code shared by the CUDA path and the CPU oracle.  It
holds none of the solver's arithmetic: it only draws coefficients and assembles
the matrix that both sides then consume.

Structure (Section 2, Eq. 2.2): unknowns are grouped by physical quantity
("block-major"): unknown (alpha, k) of component alpha in cell k sits at index
alpha*N + k.  Components 0..G-1 are the radiation groups, G is the electron
temperature E and G+1 the ion temperature I.  Diagonal blocks A_alpha are
cell-centred two-point-flux finite-volume stencils (5-point in 2D, 7-point in
3D); the coupling blocks D_alpha,beta are diagonal.  Couplings follow the
arrow structure of Eq. 2.2: group g <-> E and E <-> I only, with D_EI = D_IE
and D_gE != D_Eg.

Readings of the paper (it starts from capsule-implosion matrices that are not
available, so the coefficients below are synthetic):
  * E has no diffusion stencil unless ``diffuse_E`` (A_E is then diagonal).
  * Off-diagonal coupling entries are -c with c > 0; the row diagonal is
    sum(face transmissibilities) + sum(row couplings) + 1 (unit mass term),
    so every row is strictly diagonally dominant; the matrix is nonsymmetric.
  * Transmissibility between neighbours is the harmonic mean 2 k_i k_j /
    (k_i + k_j) (unit spacing); boundary faces are homogeneous Dirichlet with
    transmissibility 2 k_i.

Random numbers come from a counter-based splitmix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014):
    mix64(z)   = the splitmix64 finaliser,
    key(s, t)  = mix64(mix64(s + GOLDEN) + t * GOLDEN)        (mod 2^64),
    u(s, t, i) = (mix64(key(s, t) + (i + 1) * GOLDEN) >> 11) * 2^-53,
i.e. the i-th output of a splitmix64 stream seeded with key(s, t).
"""
from __future__ import annotations

import dataclasses
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids (the PMIS weight streams 1000+level are drawn by the solver sides)
STREAM_DIFF = 10        # + component index
STREAM_C_GE = 100       # + group index: row g, column E
STREAM_C_EG = 200       # + group index: row E, column g
STREAM_C_EI = 300       # D_EI = D_IE
STREAM_B = 400
STREAM_INCLUSION = 500
STREAM_PMIS = 1000      # + level (used by the AMG setup on both sides)


def _mix64(z):
    with np.errstate(over="ignore"):
        z = np.asarray(z, dtype=np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = _mix64(np.uint64(seed % 2**64) + GOLDEN)
        return _mix64(s + np.uint64(stream % 2**64) * GOLDEN)


def uniform(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """u(seed, stream, i) for i in [start, start+n), doubles in [0, 1)."""
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = _mix64(key + idx * GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def log_uniform(seed, stream, n, lo, hi):
    u = uniform(seed, stream, n)
    return 10.0 ** (lo + (hi - lo) * u)


@dataclasses.dataclass
class BlockSystem:
    name: str
    G: int
    dims: tuple           # (nx, ny) or (nx, ny, nz); x fastest
    N: int                # cells
    nc: int               # components = G + 2
    n: int                # unknowns = nc * N
    rowptr: np.ndarray    # int32 [n+1]
    col: np.ndarray       # int32 [nnz], sorted within each row
    val: np.ndarray       # float64 [nnz]
    b: np.ndarray         # float64 [n], uniform [0, 1)

    @property
    def nnz(self):
        return int(self.col.shape[0])

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def _diffusion_coeffs(seed, G, dims, multigroup, inclusion, diffuse_E):
    """Per-component cell coefficient arrays (None for non-diffusing)."""
    N = int(np.prod(dims))
    nc = G + 2
    k = [None] * nc
    for a in range(nc):
        if a < G:
            if multigroup:
                g = a + 1
                k[a] = log_uniform(seed, STREAM_DIFF + a, N, -4.0, 2.0) * 10.0 ** (-g / 5.0)
            else:
                k[a] = log_uniform(seed, STREAM_DIFF + a, N, -3.0, 3.0)
        elif a == G:
            if diffuse_E:
                k[a] = log_uniform(seed, STREAM_DIFF + a, N, -3.0, 3.0)
        else:
            k[a] = log_uniform(seed, STREAM_DIFF + a, N, -3.0, 3.0)
    if inclusion:
        L = float(dims[0])
        u = uniform(seed, STREAM_INCLUSION, 3)
        cx, cy = u[0] * L, u[1] * L
        r = (0.1 + 0.15 * u[2]) * L
        nx, ny = dims[0], dims[1]
        ix = np.arange(nx) + 0.5
        iy = np.arange(ny) + 0.5
        inside = ((ix[None, :] - cx) ** 2 + (iy[:, None] - cy) ** 2) <= r * r   # (ny, nx)
        if len(dims) == 3:
            inside = np.broadcast_to(inside[None, :, :], (dims[2], ny, nx))
        inside = inside.reshape(-1)
        for a in range(nc):
            if k[a] is not None:
                k[a] = np.where(inside, k[a] * 1e4, k[a])
    return k


def _stencil_block(kc, dims):
    """Two-point-flux stencil of one component.

    Returns (offsets, T, diagT): offsets in cell index for each slot in sorted
    column order (excluding the centre), T[slot] (N,) transmissibility of that
    face (0 where the neighbour is outside), diagT (N,) sum of all face
    transmissibilities including Dirichlet boundary faces.
    """
    nd = len(dims)
    shape = tuple(reversed(dims))          # (nz, ny, nx) / (ny, nx)
    kk = kc.reshape(shape)
    N = kc.shape[0]
    strides = []
    s = 1
    for d in dims:
        strides.append(s)
        s *= d
    diagT = np.zeros(shape)
    lower, upper = [], []
    for ax_x in range(nd):                 # ax_x = 0 is x (fastest)
        ax = nd - 1 - ax_x                 # numpy axis
        n_ax = shape[ax]
        sl_lo = [slice(None)] * nd
        sl_hi = [slice(None)] * nd
        sl_lo[ax] = slice(0, n_ax - 1)
        sl_hi[ax] = slice(1, n_ax)
        ka = kk[tuple(sl_lo)]
        kb = kk[tuple(sl_hi)]
        Tf = 2.0 * ka * kb / (ka + kb)
        Tminus = np.zeros(shape)           # face to the lower neighbour
        Tplus = np.zeros(shape)            # face to the upper neighbour
        Tminus[tuple(sl_hi)] = Tf
        Tplus[tuple(sl_lo)] = Tf
        bnd_lo = [slice(None)] * nd
        bnd_hi = [slice(None)] * nd
        bnd_lo[ax] = slice(0, 1)
        bnd_hi[ax] = slice(n_ax - 1, n_ax)
        diagT += Tminus + Tplus
        diagT[tuple(bnd_lo)] += 2.0 * kk[tuple(bnd_lo)]
        diagT[tuple(bnd_hi)] += 2.0 * kk[tuple(bnd_hi)]
        lower.append((-strides[ax_x], Tminus.reshape(N), ax_x, -1))
        upper.append((strides[ax_x], Tplus.reshape(N), ax_x, +1))
    # sorted column order: most negative offset first
    lower.sort(key=lambda t: t[0])
    upper.sort(key=lambda t: t[0])
    return lower, upper, diagT.reshape(N)


def _neighbour_valid(dims, ax_x, sign):
    shape = tuple(reversed(dims))
    nd = len(dims)
    ax = nd - 1 - ax_x
    idx = np.indices(shape)[ax]
    if sign < 0:
        v = idx > 0
    else:
        v = idx < shape[ax] - 1
    return v.reshape(-1)


def make_system(G, dims, seed=0, multigroup=False, inclusion=False, diffuse_E=False, name=None):
    """Assemble the block-major CSR matrix and right-hand side."""
    dims = tuple(int(d) for d in dims)
    N = int(np.prod(dims))
    nc = G + 2
    n = nc * N
    E, I = G, G + 1
    kdiff = _diffusion_coeffs(seed, G, dims, multigroup, inclusion, diffuse_E)
    # coupling coefficients (positive); matrix entries are -c
    cgE = [log_uniform(seed, STREAM_C_GE + g, N, -2.0, 2.0) for g in range(G)]
    cEg = [log_uniform(seed, STREAM_C_EG + g, N, -2.0, 2.0) for g in range(G)]
    cEI = log_uniform(seed, STREAM_C_EI, N, -2.0, 2.0)
    couplings = {a: [] for a in range(nc)}     # a -> list of (beta, c)
    for g in range(G):
        couplings[g].append((E, cgE[g]))
        couplings[E].append((g, cEg[g]))
    couplings[E].append((I, cEI))
    couplings[I].append((E, cEI))
    cell = np.arange(N, dtype=np.int64)
    row_cols, row_vals, row_mask = [], [], []
    for a in range(nc):
        cpl = sorted(couplings[a], key=lambda t: t[0])
        csum = np.zeros(N)
        for _, c in cpl:
            csum = csum + c
        cols, vals, mask = [], [], []
        for beta, c in cpl:
            if beta < a:
                cols.append(beta * N + cell)
                vals.append(-c)
                mask.append(np.ones(N, bool))
        if kdiff[a] is not None:
            lower, upper, diagT = _stencil_block(kdiff[a], dims)
            for off, T, ax_x, sgn in lower:
                valid = _neighbour_valid(dims, ax_x, sgn)
                cols.append(a * N + np.where(valid, cell + off, cell))
                vals.append(-T)
                mask.append(valid)
            cols.append(a * N + cell)
            vals.append(diagT + csum + 1.0)
            mask.append(np.ones(N, bool))
            for off, T, ax_x, sgn in upper:
                valid = _neighbour_valid(dims, ax_x, sgn)
                cols.append(a * N + np.where(valid, cell + off, cell))
                vals.append(-T)
                mask.append(valid)
        else:
            cols.append(a * N + cell)
            vals.append(csum + 1.0)
            mask.append(np.ones(N, bool))
        for beta, c in cpl:
            if beta > a:
                cols.append(beta * N + cell)
                vals.append(-c)
                mask.append(np.ones(N, bool))
        C = np.stack(cols, axis=1)
        V = np.stack(vals, axis=1)
        M = np.stack(mask, axis=1)
        row_cols.append(C[M])
        row_vals.append(V[M])
        row_mask.append(M.sum(axis=1))
    counts = np.concatenate(row_mask)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = np.concatenate(row_cols).astype(np.int32)
    val = np.concatenate(row_vals).astype(np.float64)
    b = uniform(seed, STREAM_B, n)
    return BlockSystem(name=name or f"G{G}_{'x'.join(map(str, dims))}", G=G, dims=dims, N=N, nc=nc,
                       n=n, rowptr=rowptr.astype(np.int32), col=col, val=val, b=b)


# The five workloads: (G, grid, multigroup law, inclusion, default preconditioner, precision)
PRESETS = {
    0: dict(G=1, dims=(32, 32), multigroup=False, inclusion=False),
    1: dict(G=1, dims=(1024, 1024), multigroup=False, inclusion=True),
    2: dict(G=20, dims=(256, 256), multigroup=True, inclusion=False),
    3: dict(G=20, dims=(96, 96, 96), multigroup=True, inclusion=False),
    4: dict(G=4, dims=(256, 256), multigroup=True, inclusion=False),
    # Eq. 2.1 as printed: the electron energy diffuses too (E gets a stencil)
    5: dict(G=1, dims=(1024, 1024), multigroup=False, inclusion=True, diffuse_E=True),
    6: dict(G=20, dims=(256, 256), multigroup=True, inclusion=False, diffuse_E=True),
}

PRESET_NAMES = {
    0: "G1_3T_32x32_monolithicAMG",
    1: "G1_3T_1024x1024_inclusion_Schur1",
    2: "G20_256x256_blockdiag_fp32vcycle",
    3: "G20_96x96x96_Schur2",
    4: "G4_256x256_adjoint",
    5: "G1_3T_1024x1024_inclusion_diffuseE_Schur1",
    6: "G20_256x256_diffuseE_Schur2_cycles311",
}


def preset(i, dims=None, seed=0):
    p = dict(PRESETS[i])
    if dims is not None:
        p["dims"] = tuple(dims)
    return make_system(p["G"], p["dims"], seed=seed, multigroup=p["multigroup"],
                       inclusion=p["inclusion"], diffuse_E=p.get("diffuse_E", False), name=PRESET_NAMES[i])
