"""Python binding of the B300 RFA bioheat library (``librfa.so``, C ABI in include/rfa.h).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of ``librfa.so``.  There is no CPU fallback -- importing a function
whose library is missing raises immediately.

The functions keep the C names (``rfa_create_grid`` ... ``rfa_backward``);
``Grid`` is a small owning wrapper around a grid handle.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# RFA_CHECKED_BUILD=1 loads the checked build (index checks in the kernels,
# built by build.py --checked) instead of the ordinary one
LIB_PATH = os.path.join(_HERE, "librfa_check.so" if os.environ.get("RFA_CHECKED_BUILD") == "1" else "librfa.so")

STATE_F32, STATE_F32C, STATE_F64 = 0, 1, 2
PARAM_BF16, PARAM_F32, PARAM_F64 = 0, 1, 2
FACE_DIRICHLET, FACE_INSULATED = 0, 1
NEEDLE_STRAIGHT, NEEDLE_UMBRELLA, NEEDLE_FIXED_TIP = 0, 1, 2
FIELD_THETA, FIELD_A, FIELD_B, FIELD_S, FIELD_LATCH, FIELD_OMEGA, FIELD_THETA_LO = range(7)

STATUS = {0: "RFA_OK", 1: "RFA_E_INVALID", 2: "RFA_E_OOM", 3: "RFA_E_CUDA", 4: "RFA_E_UNSTABLE",
          5: "RFA_E_STATE", 6: "RFA_E_NONFINITE", 7: "RFA_E_TIMEOUT", 8: "RFA_E_UNSUPPORTED",
          9: "RFA_E_INTERNAL"}

EXPORTED = ("rfa_create_grid", "rfa_destroy_grid", "rfa_set_tissue", "rfa_place_needle",
            "rfa_set_damage", "rfa_step", "rfa_get_temperature", "rfa_get_field",
            "rfa_necrosis_mask", "rfa_backward", "rfa_get_state", "rfa_set_state",
            "rfa_set_schedule", "rfa_get_schedule", "rfa_autotune", "rfa_batch_create",
            "rfa_batch_step", "rfa_batch_destroy", "rfa_synchronize", "rfa_steps_done",
            "rfa_last_error", "rfa_necrosis_reduce_noalloc", "rfa_batch_autotune",
            "rfa_batch_get_schedule", "rfa_selftest_wait_timeout", "rfa_warp_temperature",
            "rfa_set_conduction", "rfa_place_needle_potential", "rfa_set_perfusion_coupling",
            "rfa_set_potential_preconditioner", "rfa_set_wait_limits")


class RfaError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class rfa_tissue(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("rho", ctypes.c_double), ("c", ctypes.c_double),
                ("w_b", ctypes.c_double), ("rho_b", ctypes.c_double), ("c_b", ctypes.c_double),
                ("Q_m", ctypes.c_double), ("fixed", ctypes.c_int), ("T_fixed_C", ctypes.c_double)]


class rfa_needle(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("tip_m", ctypes.c_double * 3),
                ("axis", ctypes.c_double * 3), ("active_len_m", ctypes.c_double),
                ("tine_len_m", ctypes.c_double), ("tine_polar_deg", ctypes.c_double),
                ("n_tines", ctypes.c_int), ("tine_axial", ctypes.c_int),
                ("power_W", ctypes.c_double), ("r_clamp_m", ctypes.c_double),
                ("T_tip_C", ctypes.c_double)]


_lib = None


def lib():
    """Load librfa.so (built in-tree by ``build.py``); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); run "
                           "python paper_1907_05709_b300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "rfa_create_grid": [I, I, I, D, D, I, I, I, D, P, ctypes.POINTER(P)],
        "rfa_destroy_grid": [P],
        "rfa_set_tissue": [P, P, ctypes.POINTER(rfa_tissue), I],
        "rfa_place_needle": [P, ctypes.POINTER(rfa_needle)],
        "rfa_set_damage": [P, I, D, D, D, D],
        "rfa_step": [P, I64, I],
        "rfa_get_temperature": [P, P, I, I],
        "rfa_get_field": [P, I, P],
        "rfa_necrosis_mask": [P, P, P, P, P, D],
        "rfa_backward": [P, P, P],
        "rfa_get_state": [P, P, ctypes.POINTER(ctypes.c_size_t)],
        "rfa_set_state": [P, P, ctypes.c_size_t],
        "rfa_set_schedule": [P, I, I],
        "rfa_get_schedule": [P, ctypes.POINTER(I), ctypes.POINTER(I)],
        "rfa_autotune": [P, ctypes.c_char_p],
        "rfa_batch_create": [P, I, ctypes.POINTER(P)],
        "rfa_batch_step": [P, I64],
        "rfa_batch_destroy": [P],
        "rfa_synchronize": [P],
        "rfa_steps_done": [P],
        "rfa_last_error": [],
        "rfa_necrosis_reduce_noalloc": [P, D, P],
        "rfa_batch_autotune": [P, ctypes.c_char_p],
        "rfa_batch_get_schedule": [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)],
        "rfa_selftest_wait_timeout": [ctypes.c_longlong],
        "rfa_set_wait_limits": [ctypes.c_longlong, ctypes.c_longlong],
        "rfa_warp_temperature": [P, P, P, I],
        "rfa_set_conduction": [P, I],
        "rfa_set_perfusion_coupling": [P, I],
        "rfa_set_potential_preconditioner": [P, I],
        "rfa_place_needle_potential": [P, ctypes.POINTER(rfa_needle), ctypes.POINTER(D), I, I, D, ctypes.POINTER(I),
                                       ctypes.POINTER(D)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.rfa_steps_done.restype = ctypes.c_int64
    L.rfa_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(st: int, what: str):
    if st != 0:
        raise RfaError(st, what, lib().rfa_last_error().decode(errors="replace"))


def _ptr(x) -> int:
    """Address of a numpy array or a torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_handle(stream) -> Optional[int]:
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def make_tissue(t) -> rfa_tissue:
    return rfa_tissue(t.k, t.rho, t.c, t.w_b, t.rho_b, t.c_b, t.Q_m, int(t.fixed), t.T_fixed_C)


def make_needle(nd) -> rfa_needle:
    n = rfa_needle()
    n.kind = int(nd.kind)
    n.tip_m[:] = [float(v) for v in nd.tip]
    n.axis[:] = [float(v) for v in nd.axis]
    n.active_len_m = nd.active_len
    n.tine_len_m = nd.tine_len
    n.tine_polar_deg = nd.tine_polar_deg
    n.n_tines = int(nd.n_tines)
    n.tine_axial = int(nd.tine_axial)
    n.power_W = nd.power
    n.r_clamp_m = nd.r_clamp
    n.T_tip_C = float(getattr(nd, "T_tip_C", 90.0))
    return n


# --------------------------------------------------------------------- C names
def rfa_create_grid(nx, ny, nz, h_m, dt_s, state_prec=STATE_F32C, param_prec=PARAM_BF16,
                    face_bc=FACE_DIRICHLET, T_a_C=37.0, cuda_stream=None) -> int:
    out = ctypes.c_void_p()
    _check(lib().rfa_create_grid(int(nx), int(ny), int(nz), float(h_m), float(dt_s),
                                 int(state_prec), int(param_prec), int(face_bc), float(T_a_C),
                                 _stream_handle(cuda_stream), ctypes.byref(out)),
           "rfa_create_grid")
    return out.value


def rfa_destroy_grid(g):
    _check(lib().rfa_destroy_grid(g), "rfa_destroy_grid")


def rfa_set_tissue(g, labels, table: Sequence):
    """labels: uint8 numpy array (host) or uint8 torch tensor (host, pinned or device)."""
    if hasattr(labels, "data_ptr"):
        assert str(labels.dtype) == "torch.uint8" and labels.is_contiguous()
        addr, keep = labels.data_ptr(), labels
    else:
        keep = np.ascontiguousarray(labels, dtype=np.uint8)
        addr = keep.ctypes.data
    arr = (rfa_tissue * len(table))(*[make_tissue(t) for t in table])
    _check(lib().rfa_set_tissue(g, addr, arr, len(table)), "rfa_set_tissue")
    del keep


def rfa_place_needle(g, needle):
    n = needle if isinstance(needle, rfa_needle) else make_needle(needle)
    _check(lib().rfa_place_needle(g, ctypes.byref(n)), "rfa_place_needle")


def rfa_place_needle_potential(g, needle, sigma, max_iters: int = 20000, tol: float = 1e-12):
    """Returns (iterations, relative residual) of the potential solve."""
    n = needle if isinstance(needle, rfa_needle) else make_needle(needle)
    s = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64))
    it, res = ctypes.c_int(0), ctypes.c_double(0.0)
    _check(lib().rfa_place_needle_potential(g, ctypes.byref(n), s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            len(s), int(max_iters), float(tol), ctypes.byref(it),
                                            ctypes.byref(res)), "rfa_place_needle_potential")
    return it.value, res.value


PRECOND_MULTIGRID, PRECOND_JACOBI = 0, 1


def rfa_set_potential_preconditioner(g, mode: int):
    _check(lib().rfa_set_potential_preconditioner(g, int(mode)), "rfa_set_potential_preconditioner")


def rfa_set_damage(g, enable=1, A=7.39e39, Ea=2.577e5, R=8.31, T_thr_C=60.0):
    _check(lib().rfa_set_damage(g, int(enable), float(A), float(Ea), float(R), float(T_thr_C)),
           "rfa_set_damage")


def rfa_step(g, nsteps: int, record_for_backward: int = 0):
    _check(lib().rfa_step(g, int(nsteps), int(record_for_backward)), "rfa_step")


def rfa_get_temperature(g, dst, dst_is_device: bool, as_f64: bool = False):
    _check(lib().rfa_get_temperature(g, _ptr(dst), int(bool(dst_is_device)), int(bool(as_f64))),
           "rfa_get_temperature")


COND_CENTRE, COND_HARMONIC = 0, 1


PERF_CONSTANT, PERF_TISSUE_STATE = 0, 1


def rfa_set_perfusion_coupling(g, mode: int):
    _check(lib().rfa_set_perfusion_coupling(g, int(mode)), "rfa_set_perfusion_coupling")


def rfa_set_conduction(g, mode: int):
    _check(lib().rfa_set_conduction(g, int(mode)), "rfa_set_conduction")


def rfa_warp_temperature(g, u_inv_dev, dst_dev, as_f64: bool = False):
    """u_inv_dev: CUDA float32 tensor [3, nz, ny, nx] (metres); dst_dev: CUDA tensor [nz, ny, nx]."""
    _check(lib().rfa_warp_temperature(g, _ptr(u_inv_dev), _ptr(dst_dev), int(bool(as_f64))),
           "rfa_warp_temperature")


def rfa_get_field(g, field: int, dst: np.ndarray):
    assert dst.dtype == np.float64
    _check(lib().rfa_get_field(g, int(field), _ptr(dst)), "rfa_get_field")


def rfa_necrosis_mask(g, mask: Optional[np.ndarray] = None, smooth_width_K: float = 1.0):
    counts = np.zeros(2, np.int64)
    vols = np.zeros(2, np.float64)
    sv = np.zeros(1, np.float64)
    _check(lib().rfa_necrosis_mask(g, None if mask is None else _ptr(mask), counts.ctypes.data,
                                   vols.ctypes.data, sv.ctypes.data, float(smooth_width_K)),
           "rfa_necrosis_mask")
    return counts, vols, float(sv[0])


def rfa_necrosis_reduce_noalloc(g, result_dev, smooth_width_K: float = 1.0):
    """Necrosis counts and smoothed volume into a caller-owned 32-byte device
    buffer {int64 thermal, int64 Arrhenius, float64 smooth volume m^3, 0};
    allocates nothing and does not synchronise (see include/rfa.h)."""
    _check(lib().rfa_necrosis_reduce_noalloc(g, float(smooth_width_K), _ptr(result_dev)),
           "rfa_necrosis_reduce_noalloc")


def rfa_backward(g, dLdT_final_dev, grads: np.ndarray):
    assert grads.dtype == np.float64
    _check(lib().rfa_backward(g, _ptr(dLdT_final_dev), _ptr(grads)), "rfa_backward")


def rfa_get_state(g) -> bytes:
    n = ctypes.c_size_t(0)
    _check(lib().rfa_get_state(g, None, ctypes.byref(n)), "rfa_get_state")
    buf = np.zeros(n.value, np.uint8)
    _check(lib().rfa_get_state(g, buf.ctypes.data, ctypes.byref(n)), "rfa_get_state")
    return buf.tobytes()


def rfa_set_state(g, blob: bytes):
    buf = np.frombuffer(blob, np.uint8)
    _check(lib().rfa_set_state(g, buf.ctypes.data, buf.size), "rfa_set_state")


def rfa_set_schedule(g, tb_depth: int, tile_variant: int = 0):
    _check(lib().rfa_set_schedule(g, int(tb_depth), int(tile_variant)), "rfa_set_schedule")


def rfa_get_schedule(g):
    d, v = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().rfa_get_schedule(g, ctypes.byref(d), ctypes.byref(v)), "rfa_get_schedule")
    return d.value, v.value


def rfa_autotune(g, cache_path: Optional[str] = None):
    _check(lib().rfa_autotune(g, None if cache_path is None else cache_path.encode()),
           "rfa_autotune")


def rfa_batch_create(members: Sequence[int]) -> int:
    arr = (ctypes.c_void_p * len(members))(*members)
    out = ctypes.c_void_p()
    _check(lib().rfa_batch_create(arr, len(members), ctypes.byref(out)), "rfa_batch_create")
    return out.value


def rfa_batch_step(b, nsteps: int):
    _check(lib().rfa_batch_step(b, int(nsteps)), "rfa_batch_step")


def rfa_batch_destroy(b):
    _check(lib().rfa_batch_destroy(b), "rfa_batch_destroy")


def rfa_batch_autotune(b, cache_path: Optional[str] = None):
    _check(lib().rfa_batch_autotune(b, None if cache_path is None else cache_path.encode()),
           "rfa_batch_autotune")


def rfa_batch_get_schedule(b):
    d, v, gr = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().rfa_batch_get_schedule(b, ctypes.byref(d), ctypes.byref(v), ctypes.byref(gr)),
           "rfa_batch_get_schedule")
    return d.value, v.value, bool(gr.value)


def rfa_selftest_wait_timeout(spin_limit_cycles: int):
    _check(lib().rfa_selftest_wait_timeout(int(spin_limit_cycles)), "rfa_selftest_wait_timeout")


WAIT_LIMIT_DEFAULT = 1 << 32


def rfa_set_wait_limits(mbarrier_cycles: int = WAIT_LIMIT_DEFAULT, grid_barrier_cycles: int = WAIT_LIMIT_DEFAULT):
    _check(lib().rfa_set_wait_limits(int(mbarrier_cycles), int(grid_barrier_cycles)), "rfa_set_wait_limits")


def rfa_synchronize(g):
    _check(lib().rfa_synchronize(g), "rfa_synchronize")


def rfa_steps_done(g) -> int:
    return int(lib().rfa_steps_done(g))


def rfa_last_error() -> str:
    return lib().rfa_last_error().decode(errors="replace")


# --------------------------------------------------------------------- wrapper
class Grid:
    """Owning wrapper of one grid handle."""

    def __init__(self, nx, ny, nz, h, dt, state_prec=STATE_F32C, param_prec=PARAM_BF16,
                 face_bc=FACE_DIRICHLET, T_a_C=37.0, cuda_stream=None):
        self.shape = (nz, ny, nx)
        self.nx, self.ny, self.nz, self.h, self.dt = nx, ny, nz, h, dt
        self.T_a = T_a_C
        self.state_prec = state_prec
        self.handle = rfa_create_grid(nx, ny, nz, h, dt, state_prec, param_prec, face_bc, T_a_C,
                                      cuda_stream)

    @classmethod
    def from_case(cls, case, state_prec=STATE_F32C, param_prec=PARAM_BF16, cuda_stream=None,
                  damage=True):
        g = cls(case.nx, case.ny, case.nz, case.h, case.dt, state_prec, param_prec, case.face_bc,
                case.T_a_C, cuda_stream)
        if getattr(case, "conduction", "centre") == "harmonic":
            rfa_set_conduction(g.handle, COND_HARMONIC)
        if getattr(case, "perfusion", "constant") == "tissue_state":
            rfa_set_perfusion_coupling(g.handle, PERF_TISSUE_STATE)
        g.set_tissue(case.labels, case.table)
        if getattr(case, "source", "needle") == "potential":
            rfa_place_needle_potential(g.handle, case.needle, [t.sigma for t in case.table])
        else:
            g.place_needle(case.needle)
        d = case.damage
        g.set_damage(int(bool(d.enable and damage)), d.A, d.Ea, d.R, d.T_thr_C)
        return g

    def close(self):
        if self.handle:
            rfa_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tissue(self, labels, table):
        self.n_labels = len(table)
        rfa_set_tissue(self.handle, labels, table)

    def place_needle(self, needle):
        rfa_place_needle(self.handle, needle)

    def set_damage(self, enable=1, A=7.39e39, Ea=2.577e5, R=8.31, T_thr_C=60.0):
        rfa_set_damage(self.handle, enable, A, Ea, R, T_thr_C)

    def step(self, n, record=False):
        rfa_step(self.handle, n, int(record))

    def temperature(self, as_f64=True) -> np.ndarray:
        out = np.zeros(self.shape, np.float64 if as_f64 else np.float32)
        rfa_get_temperature(self.handle, out, False, as_f64)
        return out

    def field(self, fid) -> np.ndarray:
        out = np.zeros(self.shape, np.float64)
        rfa_get_field(self.handle, fid, out)
        return out

    def necrosis(self, want_mask=True, smooth_width_K=1.0):
        mask = np.zeros(self.shape, np.uint8) if want_mask else None
        counts, vols, sv = rfa_necrosis_mask(self.handle, mask, smooth_width_K)
        return mask, counts, vols, sv

    def backward(self, dLdT_dev) -> np.ndarray:
        grads = np.zeros(4 + 2 * self.n_labels, np.float64)
        rfa_backward(self.handle, dLdT_dev, grads)
        return grads

    def synchronize(self):
        rfa_synchronize(self.handle)

    def set_schedule(self, depth, variant=0):
        rfa_set_schedule(self.handle, depth, variant)

    @property
    def steps_done(self):
        return rfa_steps_done(self.handle)
