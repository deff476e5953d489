"""FP64 CPU oracle of the RFA bioheat explicit scheme -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or runs it; the two share no code.

The numeric work is in ``oracle.c`` (plain C, FP64, OpenMP over z so the result
does not depend on the thread count); this module only marshals numpy arrays.
``brute.py`` holds an independent dense-matrix formulation used to pin it.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
from typing import Optional

import numpy as np

from . import build as _build

_lib = None

_P_D = ctypes.POINTER(ctypes.c_double)
_P_U8 = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _lib
    if _lib is None:
        _lib = bind(ctypes.CDLL(_build.build()))
    return _lib


def bind(L):
    """Declare the C entry points' argument types on a loaded oracle library."""
    i, d, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
    L.or_round_bf16.argtypes = [d]
    L.or_round_bf16.restype = d
    L.or_setup.argtypes = [i, i, i, d, d, i, d, i, _P_U8, i, _P_D,
                           _P_D, _P_D, _P_D, _P_D, _P_U8, _P_D]
    L.or_source.argtypes = [i, i, i, d, d, _P_D, _P_D, _P_U8, _P_D, _P_D, _P_D]
    L.or_run.argtypes = [i, i, i, i64, _P_D, _P_D, _P_D, _P_D, _P_U8, _P_D, _P_U8, d, d,
                         i, d, d, d, d, _P_D, _P_D, i, _P_D, i]
    L.or_adjoint.argtypes = [i, i, i, i64, d, d, _P_D, _P_D, _P_D, _P_D, _P_U8, _P_U8, i,
                             _P_D, _P_D, _P_D, _P_D, _P_D, _P_D, _P_D, i, _P_D, _P_D, _P_D]
    L.or_source_grad.argtypes = [i, i, i, d, d, _P_D, _P_D, _P_U8, _P_D, _P_D]
    for f in ("or_setup", "or_source", "or_run", "or_adjoint", "or_source_grad"):
        getattr(L, f).restype = ctypes.c_int
    return L


def _threads(nthreads: int) -> int:
    """The OpenMP thread count to pass: nthreads, or every core for 0.  The
    count is always passed explicitly because omp_set_num_threads is
    process-wide: a one-thread call would otherwise leave later calls on one
    thread.  Results do not depend on it (OpenMP over z only)."""
    return int(nthreads) if nthreads and nthreads > 0 else (os.cpu_count() or 1)


def _pd(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P_D)


def _pu8(a):
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(_P_U8)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def round_bf16(x: float) -> float:
    return lib().or_round_bf16(float(x))


def table_array(table) -> np.ndarray:
    return np.ascontiguousarray(np.array([t.as_tuple() for t in table], dtype=np.float64))


def needle_array(nd) -> np.ndarray:
    ax = list(nd.axis)
    return np.ascontiguousarray(np.array(
        [nd.kind, nd.tip[0], nd.tip[1], nd.tip[2], ax[0], ax[1], ax[2], nd.active_len,
         nd.tine_len, nd.tine_polar_deg, nd.n_tines, nd.tine_axial, nd.power, nd.r_clamp],
        dtype=np.float64))


PARAM_MODE = {"f64": 0, "f32": 1, "bf16": 2}


@dataclasses.dataclass
class Model:
    """Per-voxel coefficients of one problem (all [nz, ny, nx] float64)."""
    nx: int
    ny: int
    nz: int
    h: float
    dt: float
    a: np.ndarray
    b: np.ndarray
    qm: np.ndarray
    rhoc: np.ndarray
    isfixed: np.ndarray
    theta0: np.ndarray
    s: np.ndarray
    dist: np.ndarray
    W: float
    labels: np.ndarray
    tab: np.ndarray
    needle: np.ndarray
    T_a: float
    # conservative conduction (None: the centre form): face weights [6][nz][ny][nx]
    # for x-, x+, y-, y+, z-, z+ and their derivatives by the voxel's K (dwa) and
    # by the neighbour's K (dwb)
    wf: Optional[np.ndarray] = None
    dwa: Optional[np.ndarray] = None
    dwb: Optional[np.ndarray] = None
    # perfusion weighted by the tissue state alpha = 1 / max(1, Omega) (0: constant)
    alpha_perf: int = 0


def face_weights(case, param_mode: str):
    """Conservative conduction, div(K grad T) of Eq. 2675-eq1_Kath with the face
    conductance of two voxels the harmonic mean of their K:
        w(l, m) = dt / (rho_l c_l h^2) * 2 K_l K_m / (K_l + K_m)
    for a voxel of label l and its neighbour of label m, rounded to FP32 for the
    'bf16' and 'f32' parameter modes (the values the GPU's label-pair table
    holds), and the exact derivatives dw/dK_l, dw/dK_m.  Returns (wf, dwa, dwb),
    each [6][nz][ny][nx] for the directions x-, x+, y-, y+, z-, z+ (0 outside)."""
    L = len(case.table)
    W = np.zeros((L, L))
    DA = np.zeros((L, L))
    DB = np.zeros((L, L))
    for l, tl in enumerate(case.table):
        g = case.dt / (tl.rho * tl.c * case.h * case.h)
        for m, tm in enumerate(case.table):
            Ks = tl.k + tm.k
            if Ks > 0.0:
                W[l, m] = g * (2.0 * tl.k * tm.k / Ks)
                DA[l, m] = g * 2.0 * tm.k * tm.k / (Ks * Ks)
                DB[l, m] = g * 2.0 * tl.k * tl.k / (Ks * Ks)
    if param_mode in ("bf16", "f32"):
        W = W.astype(np.float32).astype(np.float64)
    lab = case.labels.astype(np.int64).reshape(case.nz, case.ny, case.nx)
    out = [np.zeros((6, case.nz, case.ny, case.nx)) for _ in range(3)]
    # (array axis, shift): x- reads x-1, i.e. the neighbour label at index - 1
    for d, (ax, sh) in enumerate(((2, -1), (2, 1), (1, -1), (1, 1), (0, -1), (0, 1))):
        n = lab.shape[ax]
        idx = np.arange(n) + sh
        ok = (idx >= 0) & (idx < n)
        nb = np.take(lab, np.clip(idx, 0, n - 1), axis=ax)
        okb = np.broadcast_to(ok.reshape([-1 if k == ax else 1 for k in range(3)]), lab.shape)
        for arr, T in zip(out, (W, DA, DB)):
            arr[d] = np.where(okb, T[lab, nb], 0.0)
    return tuple(np.ascontiguousarray(a) for a in out)


def setup(case, param_mode: str = "f64", conduction: Optional[str] = None) -> Model:
    """Coefficients, fixed set, initial state and RF source of ``case``;
    ``conduction`` = 'centre' (K at the voxel, the paper's form) or 'harmonic'
    (conservative form, see ``face_weights``); default: ``case.conduction``."""
    if conduction is None:
        conduction = getattr(case, "conduction", "centre")
    nx, ny, nz = case.nx, case.ny, case.nz
    shape = (nz, ny, nx)
    labels = np.ascontiguousarray(case.labels.astype(np.uint8).reshape(shape))
    tab = table_array(case.table)
    a, b, qm, rhoc, th0 = (np.zeros(shape) for _ in range(5))
    fx = np.zeros(shape, dtype=np.uint8)
    _check(lib().or_setup(nx, ny, nz, case.h, case.dt, case.face_bc, case.T_a_C,
                          PARAM_MODE[param_mode], _pu8(labels), len(case.table), _pd(tab),
                          _pd(a), _pd(b), _pd(qm), _pd(rhoc), _pu8(fx), _pd(th0)), "setup")
    nd = needle_array(case.needle)
    s, dist = np.zeros(shape), np.zeros(shape)
    W = ctypes.c_double(0.0)
    _check(lib().or_source(nx, ny, nz, case.h, case.dt, _pd(nd), _pd(rhoc), _pu8(fx), _pd(s),
                           _pd(dist), ctypes.byref(W)), "source")
    m = Model(nx, ny, nz, case.h, case.dt, a, b, qm, rhoc, fx, th0, s, dist, W.value,
              labels, tab, nd, case.T_a_C)
    if getattr(case, "source", "needle") == "potential":
        _, _, m.s = potential_source(case, m)
    m.alpha_perf = int(getattr(case, "perfusion", "constant") == "tissue_state")
    if conduction == "harmonic":
        m.wf, m.dwa, m.dwb = face_weights(case, param_mode)
    elif conduction != "centre":
        raise ValueError(conduction)
    return m


@dataclasses.dataclass
class State:
    theta: np.ndarray
    latch: np.ndarray
    omega: np.ndarray
    omega_c: np.ndarray
    steps: int = 0


def initial_state(m: Model) -> State:
    shape = m.a.shape
    return State(m.theta0.copy(), np.zeros(shape, dtype=np.uint8), np.zeros(shape),
                 np.zeros(shape), 0)


def run(m: Model, st: State, nsteps: int, damage=None, T_thr_C: float = 60.0,
        nthreads: int = 0) -> State:
    """Advance ``st`` in place by ``nsteps`` explicit steps."""
    dmg = damage
    en = int(bool(dmg is not None and dmg.enable))
    A = dmg.A if en else 0.0
    Ea = dmg.Ea if en else 0.0
    R = dmg.R if en else 1.0
    thr = dmg.T_thr_C if dmg is not None else T_thr_C
    _check(lib().or_run(m.nx, m.ny, m.nz, int(nsteps), _pd(m.a), _pd(m.b), _pd(m.s), _pd(m.qm),
                        _pu8(m.isfixed), _pd(st.theta), _pu8(st.latch), m.T_a, thr, en, m.dt,
                        A, Ea, R, _pd(st.omega), _pd(st.omega_c), _threads(nthreads),
                        None if m.wf is None else _pd(m.wf), int(m.alpha_perf)), "run")
    st.steps += int(nsteps)
    return st


def adjoint(m: Model, nsteps: int, lam_N: np.ndarray, nthreads: int = 0):
    """Discrete adjoint of ``nsteps`` steps from m.theta0.  Returns
    (lambda_0, Lambda, g_k[L], g_wb[L], g_P, g_tip[3])."""
    lam = np.ascontiguousarray(lam_N.astype(np.float64).reshape(m.a.shape)).copy()
    Lam = np.zeros(m.a.shape)
    nl = m.tab.shape[0]
    gk, gw = np.zeros(nl), np.zeros(nl)
    _check(lib().or_adjoint(m.nx, m.ny, m.nz, int(nsteps), m.h, m.dt, _pd(m.a), _pd(m.b),
                            _pd(m.s), _pd(m.qm), _pu8(m.isfixed), _pu8(m.labels), nl, _pd(m.tab),
                            _pd(m.rhoc), _pd(m.theta0), _pd(lam), _pd(Lam), _pd(gk), _pd(gw),
                            _threads(nthreads), None if m.wf is None else _pd(m.wf),
                            None if m.wf is None else _pd(m.dwa),
                            None if m.wf is None else _pd(m.dwb)), "adjoint")
    g = np.zeros(4)
    _check(lib().or_source_grad(m.nx, m.ny, m.nz, m.h, m.dt, _pd(m.needle), _pd(m.rhoc),
                                _pu8(m.isfixed), _pd(Lam), _pd(g)), "source_grad")
    return lam, Lam, gk, gw, float(g[0]), g[1:].copy()


def necrosis(m: Model, st: State, T_a: Optional[float] = None, width_K: float = 1.0,
             thr_C: float = 60.0):
    """Mask bits (bit0 thermal latch, bit1 Arrhenius Omega >= 1), counts,
    volumes h^3*count and the smoothed volume h^3 sum sigmoid((T - thr)/width)."""
    Ta = m.T_a if T_a is None else T_a
    mask = (st.latch != 0).astype(np.uint8) | ((st.omega >= 1.0).astype(np.uint8) << 1)
    h3 = m.h ** 3
    n_th = int(np.count_nonzero(mask & 1))
    n_ar = int(np.count_nonzero(mask & 2))
    T = st.theta + Ta
    vs = h3 * float(np.sum(1.0 / (1.0 + np.exp(-(T - thr_C) / width_K))))
    return mask, (n_th, n_ar), (h3 * n_th, h3 * n_ar), vs


def warp_temperature(theta: np.ndarray, u_inv: np.ndarray, h: float, T_a: float) -> np.ndarray:
    """Breathing motion (Sec. "Consideration of Breathing Motion", Eq. breathing):
    T(x) = T_ref(x + u_inv(x)), T_ref = T_a + theta sampled by trilinear
    interpolation, in FP64.  theta: [nz][ny][nx]; u_inv: [3][nz][ny][nx] (x, y, z
    components, metres).  Per axis, with voxel index c and displacement
    d = u / h in voxels: i = c + floor(d); i < 0 samples voxel 0, i >= n-1 samples
    voxel n-1, otherwise the segment [i, i+1] at weight f = d - floor(d)."""
    nz, ny, nx = theta.shape
    d = u_inv.astype(np.float64) / h
    cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def axis(c, dd, n):
        dd = np.clip(np.nan_to_num(dd, nan=-(n + 1.0)), -(n + 1.0), n + 1.0)
        fl = np.floor(dd)
        i = c + fl.astype(np.int64)
        low, high = i < 0, i >= n - 1
        i0 = np.where(low, 0, np.where(high, n - 1, i))
        i1 = np.where(low | high, i0, i + 1)
        f = np.where(low | high, 0.0, dd - fl)
        return i0, i1, f

    x0, x1, fx = axis(cx, d[0], nx)
    y0, y1, fy = axis(cy, d[1], ny)
    z0, z1, fz = axis(cz, d[2], nz)
    out = np.zeros(theta.shape)
    # sum over the 8 corners of the cell, each with its product of 1-D weights
    for zi, wz in ((z0, 1.0 - fz), (z1, fz)):
        for yi, wy in ((y0, 1.0 - fy), (y1, fy)):
            for xi, wx in ((x0, 1.0 - fx), (x1, fx)):
                out += wz * wy * wx * theta[zi, yi, xi]
    return out + T_a


# ------------------------------------------------------------ potential source
def harmonic_faces(vals: np.ndarray):
    """Face values 2 u v / (u + v) of a per-voxel field to each neighbour, [6][nz][ny][nx]
    for x-, x+, y-, y+, z-, z+ (0 outside the grid)."""
    out = np.zeros((6,) + vals.shape)
    for d, (ax, sh) in enumerate(((2, -1), (2, 1), (1, -1), (1, 1), (0, -1), (0, 1))):
        n = vals.shape[ax]
        idx = np.arange(n) + sh
        ok = (idx >= 0) & (idx < n)
        nb = np.take(vals, np.clip(idx, 0, n - 1), axis=ax)
        s = vals + nb
        hm = np.divide(2.0 * vals * nb, s, out=np.zeros_like(s), where=s > 0)
        okb = np.broadcast_to(ok.reshape([-1 if k == ax else 1 for k in range(3)]), vals.shape)
        out[d] = np.where(okb, hm, 0.0)
    return out


def _shift(v, d):
    """Neighbour values of v in direction d (x-, x+, y-, y+, z-, z+), 0 outside."""
    ax, sh = ((2, -1), (2, 1), (1, -1), (1, 1), (0, -1), (0, 1))[d]
    n = v.shape[ax]
    idx = np.arange(n) + sh
    ok = (idx >= 0) & (idx < n)
    nb = np.take(v, np.clip(idx, 0, n - 1), axis=ax)
    okb = np.broadcast_to(ok.reshape([-1 if k == ax else 1 for k in range(3)]), v.shape)
    return np.where(okb, nb, 0.0), okb


def potential_solve(sig_face: np.ndarray, electrode: np.ndarray, ground: np.ndarray) -> np.ndarray:
    """Electric potential of Eq. 2675-eq1_Linte's source term: div(sigma grad V) = 0
    on the free voxels (neither electrode nor ground), V = 1 on the electrode and
    V = 0 on the ground, discretised with the face conductances sig_face
    ([6][nz][ny][nx]): sum_nb sigma_f (V_nb - V_i) = 0.  Direct sparse solve."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import spsolve
    shape = electrode.shape
    free = ~(electrode | ground)
    Vfix = electrode.astype(np.float64)
    nfree = int(free.sum())
    V = Vfix.copy()
    if nfree == 0:
        return V
    idx = -np.ones(shape, np.int64)
    idx[free] = np.arange(nfree)
    rows, cols, vals = [], [], []
    diag = np.zeros(nfree)
    rhs = np.zeros(nfree)
    for d in range(6):
        nb_idx, ok = _shift(idx.astype(np.float64), d)
        nb_fix, _ = _shift(Vfix, d)
        m = free & ok
        sf = sig_face[d][m]
        i = idx[m]
        j = nb_idx[m].astype(np.int64)
        np.add.at(diag, i, sf)
        jf = j >= 0
        rows.append(i[jf]); cols.append(j[jf]); vals.append(-sf[jf])
        np.add.at(rhs, i[~jf], sf[~jf] * nb_fix[m][~jf])
    rows.append(np.arange(nfree)); cols.append(np.arange(nfree)); vals.append(diag)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nfree, nfree))
    V[free] = spsolve(A, rhs)
    return V


def joule(V: np.ndarray, sig_face: np.ndarray, h: float) -> np.ndarray:
    """Resistive heating sigma |grad V|^2 per voxel, evaluated per face and split
    evenly between its two voxels: q_i = sum_nb sigma_f (V_nb - V_i)^2 / (2 h^2)
    [W/m^3 per V^2]; sum_i q_i h^3 is then the network's dissipated power."""
    q = np.zeros(V.shape)
    for d in range(6):
        nb, ok = _shift(V, d)
        q += np.where(ok, sig_face[d] * (nb - V) ** 2, 0.0)
    return q / (2.0 * h * h)


def potential_source(case, m: Model):
    """Linte's RF source for ``case``: electrode = voxels within r0 of the
    needle's active segments (the geometry of or_source), ground = the outer
    faces, sigma per label (Tissue.sigma) with harmonic-mean faces; the Joule
    heating q is scaled so that sum_free q h^3 = P.  Returns (V, q, s) with
    s = P q / (h^3 W) dt / (rho c) on the free voxels, W = sum_free q."""
    nz, ny, nx = m.a.shape
    lab = m.labels.astype(np.int64)
    sig = np.array([t.sigma for t in case.table], dtype=np.float64)[lab]
    sf = harmonic_faces(sig)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ground = (x == 0) | (y == 0) | (z == 0) | (x == nx - 1) | (y == ny - 1) | (z == nz - 1)
    electrode = (m.dist <= case.needle.r_clamp) & ~ground
    V = potential_solve(sf, electrode, ground)
    q = joule(V, sf, case.h)
    free = m.isfixed == 0
    W = float(np.sum(q[free]))
    s = np.zeros(V.shape)
    if W > 0.0:
        s[free] = case.needle.power * q[free] / (case.h ** 3 * W) * case.dt / m.rhoc[free]
    return V, q, s
