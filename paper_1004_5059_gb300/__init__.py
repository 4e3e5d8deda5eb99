"""Python binding of the GB300 TVLBM library (include/tvlbm.h).

Argument marshalling only: every step of the time loop runs in the library's CUDA kernels.
PyTorch supplies device memory (contexts are created inside a torch-allocated block through
tvlbm_create_in) and the stream (torch's current stream).  There is no CPU fallback: if the
compiled library is missing, importing this package raises.

The functions mirror the C names; `Simulation` bundles them for one context.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtvlbm.so")

TVLBM_OK = 0
TVLBM_EINVAL = -1
TVLBM_ENOMEM = -2
TVLBM_ECUDA = -3
TVLBM_ESTATE = -4
TVLBM_ETIMEOUT = -5
TVLBM_ENONFINITE = -6

TVLBM_D2Q9, TVLBM_D2Q16, TVLBM_D2Q36 = 9, 16, 36
TVLBM_FP64, TVLBM_FP32, TVLBM_BF16_DEV, TVLBM_FP16_DEV, TVLBM_FP32_DEV = 0, 1, 2, 3, 4
TVLBM_FORM_PLAIN, TVLBM_FORM_TILED, TVLBM_FORM_FLOW, TVLBM_FORM_STRIP = 0, 1, 2, 3
TVLBM_SCHEME_VOLUMETRIC, TVLBM_SCHEME_FVLB = 0, 1
TVLBM_MLP_IN, TVLBM_MLP_IN_PAD, TVLBM_MLP_HIDDEN = 54, 64, 128
TVLBM_MLP_OUT, TVLBM_MLP_OUT_PAD, TVLBM_MLP_PARAMS = 12, 16, 25100
TVLBM_BC_PERIODIC, TVLBM_BC_WALLS = 0, 1

VELSETS = {"D2Q9": TVLBM_D2Q9, "D2Q16": TVLBM_D2Q16, "D2Q36": TVLBM_D2Q36}
STORAGES = {"fp64": TVLBM_FP64, "fp32": TVLBM_FP32, "bf16_dev": TVLBM_BF16_DEV, "fp16_dev": TVLBM_FP16_DEV,
            "fp32_dev": TVLBM_FP32_DEV}
FORMS = {"plain": TVLBM_FORM_PLAIN, "tiled": TVLBM_FORM_TILED, "flow": TVLBM_FORM_FLOW, "strip": TVLBM_FORM_STRIP}
STORAGE_NUMPY = {TVLBM_FP64: np.float64, TVLBM_FP32: np.float32, TVLBM_FP32_DEV: np.float32,
                 TVLBM_BF16_DEV: np.uint16, TVLBM_FP16_DEV: np.float16}


class TvlbmError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__("tvlbm error %d: %s" % (code, message))
        self.code = code


class tvlbm_bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("u_lo", ctypes.c_double), ("T_lo", ctypes.c_double),
                ("u_hi", ctypes.c_double), ("T_hi", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
_SZ = ctypes.c_size_t
_FP = ctypes.POINTER(ctypes.c_float)


def _load_library() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError("libtvlbm.so is not built (run __graft_entry__.build() or "
                          "python paper_1004_5059_gb300/build.py); there is no fallback")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "tvlbm_memory_bytes": (_I, [_I, _I, _I, ctypes.POINTER(tvlbm_bc), _I, ctypes.POINTER(_SZ)]),
        "tvlbm_create": (_I, [_I, _I, _I, _D, _D, ctypes.POINTER(tvlbm_bc), _I, _D, ctypes.POINTER(_P)]),
        "tvlbm_create_in": (_I, [_I, _I, _I, _D, _D, ctypes.POINTER(tvlbm_bc), _I, _D, _P, _SZ, ctypes.POINTER(_P)]),
        "tvlbm_destroy": (_I, [_P]),
        "tvlbm_set_stream": (_I, [_P, _P]),
        "tvlbm_set_form": (_I, [_P, _I]),
        "tvlbm_set_graphs": (_I, [_P, _I]),
        "tvlbm_set_scheme": (_I, [_P, _I, _D]),
        "tvlbm_set_fv_walls": (_I, [_P, _I, _I, _DP]),
        "tvlbm_set_fv_pressure_scaling": (_I, [_P, _I]),
        "tvlbm_set_fv_fused": (_I, [_P, _I]),
        "tvlbm_set_y_faces": (_I, [_P, _DP]),
        "tvlbm_set_reference": (_I, [_P, _D, _D, _D]),
        "tvlbm_set_reference_rows": (_I, [_P, _P, _P, _P]),
        "tvlbm_set_reference_refresh": (_I, [_P, _I]),
        "tvlbm_set_reference_kind": (_I, [_P, _I]),
        "tvlbm_tile_count": (_I, [_P]),
        "tvlbm_tile_shape": (_I, [_P, _I, _IP, _IP, _IP]),
        "tvlbm_set_tile": (_I, [_P, _I]),
        "tvlbm_init_moments": (_I, [_P, _DP, _DP, _DP, _DP]),
        "tvlbm_step": (_I, [_P, _I]),
        "tvlbm_moments": (_I, [_P, _DP, _DP, _DP, _DP]),
        "tvlbm_conserved_sums": (_I, [_P, _DP]),
        "tvlbm_set_flow_wait": (_I, [_P, _D, _I]),
        "tvlbm_population_bytes": (_SZ, [_P]),
        "tvlbm_get_populations": (_I, [_P, _P, _SZ]),
        "tvlbm_set_populations": (_I, [_P, _P, _SZ]),
        "tvlbm_get_populations_f64": (_I, [_P, _DP]),
        "tvlbm_set_populations_f64": (_I, [_P, _DP]),
        "tvlbm_velocity_set": (_I, [_I, _DP, _DP, _DP, _IP]),
        "tvlbm_stream_table": (_I, [_I, _D, _IP, _IP, _DP, _DP]),
        "tvlbm_bytes_per_cell": (_D, [_P]),
        "tvlbm_batch_memory_bytes": (_I, [_I, _IP, _IP, _I, _I, ctypes.POINTER(_SZ)]),
        "tvlbm_batch_create_in": (_I, [_I, _IP, _IP, _DP, _I, _I, _D, _D, _P, _SZ, ctypes.POINTER(_P)]),
        "tvlbm_batch_destroy": (_I, [_P]),
        "tvlbm_batch_set_stream": (_I, [_P, _P]),
        "tvlbm_batch_set_form": (_I, [_P, _I]),
        "tvlbm_batch_set_graphs": (_I, [_P, _I]),
        "tvlbm_batch_tile_count": (_I, [_P]),
        "tvlbm_batch_tile_shape": (_I, [_P, _I, _IP, _IP, _IP]),
        "tvlbm_batch_set_tile": (_I, [_P, _I]),
        "tvlbm_batch_init_moments": (_I, [_P, _I, _DP, _DP, _DP, _DP]),
        "tvlbm_batch_step": (_I, [_P, _I]),
        "tvlbm_batch_moments": (_I, [_P, _I, _DP, _DP, _DP, _DP]),
        "tvlbm_batch_conserved_sums": (_I, [_P, _I, _DP]),
        "tvlbm_batch_get_populations_f64": (_I, [_P, _I, _DP]),
        "tvlbm_batch_cells": (ctypes.c_longlong, [_P]),
        "tvlbm_batch_bytes_per_cell": (_D, [_P]),
        "tvlbm_batch_last_error": (ctypes.c_char_p, [_P]),
        "tvlbm_last_error": (ctypes.c_char_p, [_P]),
        "tvlbm_strerror": (ctypes.c_char_p, [_I]),
        # learned closure (include/tvlbm_closure.h)
        "tvlbm_mlp_create": (_I, [_I, ctypes.POINTER(_P)]),
        "tvlbm_mlp_destroy": (_I, [_P]),
        "tvlbm_mlp_set_stream": (_I, [_P, _P]),
        "tvlbm_mlp_set_params": (_I, [_P, _FP]),
        "tvlbm_mlp_get_params": (_I, [_P, _FP]),
        "tvlbm_mlp_forward": (_I, [_P, _P, _I, _P]),
        "tvlbm_mlp_loss_grad": (_I, [_P, _P, _P, _I, _DP, _FP]),
        "tvlbm_mlp_adam": (_I, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
        "tvlbm_mlp_last_error": (ctypes.c_char_p, [_P]),
        "tvlbm_mlp_activation": (_I, [_P, _P, _P, _I, _P]),
        "tvlbm_closure_moments": (_I, [_P, _P]),
        "tvlbm_closure_features": (_I, [_P, _FP, _FP, _P]),
        "tvlbm_closure_project": (_I, [_P, _P, _FP, _P]),
        "tvlbm_closure_noneq": (_I, [_P, _FP, _P]),
        "tvlbm_downsample": (_I, [_P, _P]),
        "tvlbm_copy_state": (_I, [_P, _P]),
        "tvlbm_step_closure": (_I, [_P, _P, _FP, _FP, _FP, _I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load_library()
lib = _lib


def _dp(a: np.ndarray):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def _check(rc: int, ctx=None):
    if rc != TVLBM_OK:
        msg = _lib.tvlbm_last_error(ctx).decode() if ctx else ""
        raise TvlbmError(rc, msg or _lib.tvlbm_strerror(rc).decode())


def _bc(bc):
    if bc is None:
        return None
    if isinstance(bc, tvlbm_bc):
        return ctypes.byref(bc)
    u_lo, T_lo, u_hi, T_hi = bc
    return ctypes.byref(tvlbm_bc(TVLBM_BC_WALLS, u_lo, T_lo, u_hi, T_hi))


# ---- functions with the C names -----------------------------------------------------------

def tvlbm_memory_bytes(nx, ny, velset, bc, storage) -> int:
    out = _SZ(0)
    _check(_lib.tvlbm_memory_bytes(nx, ny, velset, _bc(bc), storage, ctypes.byref(out)))
    return out.value


def tvlbm_create(nx, ny, velset, tau, dt, bc, storage, rho0):
    h = _P()
    _check(_lib.tvlbm_create(nx, ny, velset, tau, dt, _bc(bc), storage, rho0, ctypes.byref(h)))
    return h


def tvlbm_create_in(nx, ny, velset, tau, dt, bc, storage, rho0, device_ptr: int, nbytes: int):
    h = _P()
    _check(_lib.tvlbm_create_in(nx, ny, velset, tau, dt, _bc(bc), storage, rho0, _P(device_ptr), nbytes,
                                ctypes.byref(h)))
    return h


def tvlbm_destroy(ctx):
    _check(_lib.tvlbm_destroy(ctx))


def tvlbm_set_stream(ctx, stream_handle: int):
    _check(_lib.tvlbm_set_stream(ctx, _P(stream_handle)), ctx)


def tvlbm_set_form(ctx, form: int):
    _check(_lib.tvlbm_set_form(ctx, form), ctx)


def tvlbm_set_graphs(ctx, enable: bool):
    _check(_lib.tvlbm_set_graphs(ctx, 1 if enable else 0), ctx)


def tvlbm_set_reference(ctx, ux: float, uy: float, T: float):
    _check(_lib.tvlbm_set_reference(ctx, float(ux), float(uy), float(T)), ctx)


def tvlbm_set_reference_rows(ctx, ny: int, ux, uy, T):
    arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (ny,))) for a in (ux, uy, T)]
    _check(_lib.tvlbm_set_reference_rows(ctx, *(_dp(a) for a in arrs)), ctx)


def tvlbm_set_reference_refresh(ctx, every: int):
    _check(_lib.tvlbm_set_reference_refresh(ctx, int(every)), ctx)


REFERENCE_KINDS = {"equilibrium": 0, "mean": 1}


def tvlbm_set_reference_kind(ctx, kind: int):
    _check(_lib.tvlbm_set_reference_kind(ctx, int(kind)), ctx)


def tvlbm_tile_count(ctx) -> int:
    return int(_lib.tvlbm_tile_count(ctx))


def tvlbm_tile_shape(ctx, config: int):
    tx, ty, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib.tvlbm_tile_shape(ctx, config, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(r)), ctx)
    return tx.value, ty.value, r.value


def tvlbm_set_tile(ctx, config: int):
    _check(_lib.tvlbm_set_tile(ctx, int(config)), ctx)


def tvlbm_init_moments(ctx, rho, ux, uy, T):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy, T)]
    _check(_lib.tvlbm_init_moments(ctx, *[_dp(a) for a in arrs]), ctx)


def tvlbm_step(ctx, n: int):
    _check(_lib.tvlbm_step(ctx, int(n)), ctx)


def tvlbm_moments(ctx, nx, ny, out=None):
    outs = out if out is not None else [np.empty((ny, nx)) for _ in range(4)]
    _check(_lib.tvlbm_moments(ctx, *[_dp(o) for o in outs]), ctx)
    return tuple(outs)


def tvlbm_conserved_sums(ctx, allow_nonfinite: bool = False) -> np.ndarray:
    """(M, P_x, P_y, E, non-finite count); raises TvlbmError (TVLBM_ENONFINITE) when the count
    is not zero, unless allow_nonfinite."""
    out = np.zeros(5)
    rc = _lib.tvlbm_conserved_sums(ctx, _dp(out))
    if not (allow_nonfinite and rc == TVLBM_ENONFINITE):
        _check(rc, ctx)
    return out


def tvlbm_set_flow_wait(ctx, limit_s: float, unmet: bool = False):
    _check(_lib.tvlbm_set_flow_wait(ctx, float(limit_s), 1 if unmet else 0), ctx)


def tvlbm_population_bytes(ctx) -> int:
    return int(_lib.tvlbm_population_bytes(ctx))


def tvlbm_get_populations(ctx, host: np.ndarray):
    _check(_lib.tvlbm_get_populations(ctx, host.ctypes.data_as(_P), host.nbytes), ctx)
    return host


def tvlbm_set_populations(ctx, host: np.ndarray):
    host = np.ascontiguousarray(host)
    _check(_lib.tvlbm_set_populations(ctx, host.ctypes.data_as(_P), host.nbytes), ctx)


def tvlbm_get_populations_f64(ctx, out: np.ndarray):
    _check(_lib.tvlbm_get_populations_f64(ctx, _dp(out)), ctx)
    return out


def tvlbm_set_populations_f64(ctx, f: np.ndarray):
    _check(_lib.tvlbm_set_populations_f64(ctx, _dp(np.ascontiguousarray(f, dtype=np.float64))), ctx)


def tvlbm_velocity_set(velset: int):
    cx, cy, w = np.zeros(36), np.zeros(36), np.zeros(36)
    N = ctypes.c_int(0)
    _check(_lib.tvlbm_velocity_set(velset, _dp(cx), _dp(cy), _dp(w), ctypes.byref(N)))
    Q = velset
    return cx[:Q].copy(), cy[:Q].copy(), w[:Q].copy(), N.value


def tvlbm_stream_table(velset: int, dt: float):
    sx, sy = np.zeros(36, dtype=np.int32), np.zeros(36, dtype=np.int32)
    ax, ay = np.zeros(36), np.zeros(36)
    _check(_lib.tvlbm_stream_table(velset, dt, sx.ctypes.data_as(_IP), sy.ctypes.data_as(_IP), _dp(ax), _dp(ay)))
    Q = velset
    return sx[:Q].copy(), sy[:Q].copy(), ax[:Q].copy(), ay[:Q].copy()


def tvlbm_bytes_per_cell(ctx) -> float:
    return float(_lib.tvlbm_bytes_per_cell(ctx))


def tvlbm_last_error(ctx) -> str:
    return _lib.tvlbm_last_error(ctx).decode()


# ---- one context, torch-owned device memory and stream -------------------------------------

class Simulation:
    """A TVLBM context on the current CUDA device.  Device memory is a torch uint8 tensor held
    by this object; work is queued on torch's current stream at construction (or `stream`)."""

    def __init__(self, nx, ny, velset="D2Q16", tau=0.8, dt=1.0, walls=None, storage="fp32", rho0=1.0,
                 form=None, stream=None, graphs=True):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("TVLBM needs a CUDA GPU")
        self.nx, self.ny = int(nx), int(ny)
        self.velset = VELSETS[velset] if isinstance(velset, str) else int(velset)
        self.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
        self.Q = self.velset
        bc = None if walls is None else tuple(float(v) for v in walls)
        nbytes = tvlbm_memory_bytes(self.nx, self.ny, self.velset, bc, self.storage)
        self._mem = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self._mem.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.ctx = tvlbm_create_in(self.nx, self.ny, self.velset, float(tau), float(dt), bc, self.storage,
                                   float(rho0), aligned, nbytes)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        tvlbm_set_stream(self.ctx, s.cuda_stream)
        if form is not None:
            tvlbm_set_form(self.ctx, FORMS[form] if isinstance(form, str) else int(form))
        tvlbm_set_graphs(self.ctx, graphs)

    def close(self):
        if getattr(self, "ctx", None):
            tvlbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scheme(self, scheme, tau_g=float("inf")):
        """"volumetric" (default) or "fvlb" (the paper's finite-volume update, Prandtl time tau_g)."""
        code = {"volumetric": TVLBM_SCHEME_VOLUMETRIC, "fvlb": TVLBM_SCHEME_FVLB}[scheme] if isinstance(scheme, str) \
            else int(scheme)
        _check(_lib.tvlbm_set_scheme(self.ctx, code, float(tau_g)), self.ctx)

    def set_fv_walls(self, exact=False, nr_iters=32, y_nodes=None):
        """Finite-volume channel walls: diffuse (exact=False) or Newton-Raphson (exact=True)
        imposition; y_nodes: the ny node positions (None: unit spacing)."""
        yn = None if y_nodes is None else np.ascontiguousarray(y_nodes, dtype=np.float64)
        if yn is not None and yn.shape != (self.ny,):
            raise ValueError("y_nodes must hold ny positions")
        _check(_lib.tvlbm_set_fv_walls(self.ctx, 1 if exact else 0, int(nr_iters), _dp(yn)), self.ctx)

    def set_y_faces(self, faces=None):
        """Volumetric scheme on a mesh non-uniform in y: cell y spans [faces[y], faces[y+1]]
        (ny + 1 increasing values; None: unit cells).  Plain form only."""
        if faces is None:
            _check(_lib.tvlbm_set_y_faces(self.ctx, None), self.ctx)
            return
        fa = np.ascontiguousarray(faces, dtype=np.float64)
        if fa.shape != (self.ny + 1,):
            raise ValueError("faces must hold ny + 1 values")
        _check(_lib.tvlbm_set_y_faces(self.ctx, _dp(fa)), self.ctx)

    def set_fv_fused(self, fused=True):
        """Finite-volume scheme: one fused kernel per step (default) or the two-kernel form."""
        _check(_lib.tvlbm_set_fv_fused(self.ctx, 1 if fused else 0), self.ctx)

    def set_fv_pressure_scaling(self, enable=True):
        """Finite-volume scheme: tau -> tau / p, tau_g -> tau_g / p with p = rho T."""
        _check(_lib.tvlbm_set_fv_pressure_scaling(self.ctx, 1 if enable else 0), self.ctx)

    def set_form(self, form):
        tvlbm_set_form(self.ctx, FORMS[form] if isinstance(form, str) else int(form))

    def set_tile(self, config: int):
        tvlbm_set_tile(self.ctx, config)

    def set_reference(self, ux: float, uy: float, T: float):
        tvlbm_set_reference(self.ctx, ux, uy, T)

    def set_reference_rows(self, ux, uy, T):
        """Per-row deviation reference of a channel: ux, uy, T hold ny values (or scalars)."""
        tvlbm_set_reference_rows(self.ctx, self.ny, ux, uy, T)

    def set_reference_refresh(self, every: int, kind=None):
        """Reset the per-row reference to the rows every `every` steps (0: off); kind
        "equilibrium" (the rows' average equilibria) or "mean" (the rows' average populations),
        None keeps the current kind."""
        if kind is not None:
            tvlbm_set_reference_kind(self.ctx, REFERENCE_KINDS[kind] if isinstance(kind, str) else int(kind))
        tvlbm_set_reference_refresh(self.ctx, every)

    def init_moments(self, rho, ux, uy, T):
        tvlbm_init_moments(self.ctx, rho, ux, uy, T)

    def step(self, n=1):
        tvlbm_step(self.ctx, n)

    def moments(self):
        return tvlbm_moments(self.ctx, self.nx, self.ny)

    def conserved_sums(self, allow_nonfinite: bool = False):
        return tvlbm_conserved_sums(self.ctx, allow_nonfinite)

    def populations_f64(self):
        out = np.empty((self.Q, self.ny, self.nx))
        return tvlbm_get_populations_f64(self.ctx, out)

    def set_populations_f64(self, f):
        tvlbm_set_populations_f64(self.ctx, f)

    def raw_populations(self):
        out = np.empty((self.Q, self.ny, self.nx), dtype=STORAGE_NUMPY[self.storage])
        return tvlbm_get_populations(self.ctx, out)

    def set_raw_populations(self, host):
        tvlbm_set_populations(self.ctx, host)

    def bytes_per_cell(self):
        return tvlbm_bytes_per_cell(self.ctx)


# ---- batched domains -----------------------------------------------------------------------

def _bcheck(rc: int, b=None):
    if rc != TVLBM_OK:
        msg = _lib.tvlbm_batch_last_error(b).decode() if b else ""
        raise TvlbmError(rc, msg or _lib.tvlbm_strerror(rc).decode())


def tvlbm_batch_memory_bytes(nx, ny, velset, storage) -> int:
    n = len(nx)
    ax, ay = (np.ascontiguousarray(a, dtype=np.int32) for a in (nx, ny))
    out = _SZ(0)
    _bcheck(_lib.tvlbm_batch_memory_bytes(n, ax.ctypes.data_as(_IP), ay.ctypes.data_as(_IP), velset, storage,
                                          ctypes.byref(out)))
    return out.value


class Batch:
    """Independent periodic domains of different sizes and relaxation times, advanced together
    (tvlbm_batch_*).  Device memory is a torch tensor held by this object."""

    def __init__(self, nx, ny, tau, velset="D2Q16", storage="fp32_dev", dt=1.0, rho0=1.0, stream=None,
                 graphs=True):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("TVLBM needs a CUDA GPU")
        self.nx = np.ascontiguousarray(nx, dtype=np.int32)
        self.ny = np.ascontiguousarray(ny, dtype=np.int32)
        self.tau = np.ascontiguousarray(tau, dtype=np.float64)
        self.count = len(self.nx)
        self.velset = VELSETS[velset] if isinstance(velset, str) else int(velset)
        self.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
        self.Q = self.velset
        nbytes = tvlbm_batch_memory_bytes(self.nx, self.ny, self.velset, self.storage)
        self._mem = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        aligned = (self._mem.data_ptr() + 255) // 256 * 256
        h = _P()
        _bcheck(_lib.tvlbm_batch_create_in(self.count, self.nx.ctypes.data_as(_IP), self.ny.ctypes.data_as(_IP),
                                           _dp(self.tau), self.velset, self.storage, float(dt), float(rho0),
                                           _P(aligned), nbytes, ctypes.byref(h)))
        self.handle = h
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        _bcheck(_lib.tvlbm_batch_set_stream(h, _P(s.cuda_stream)), h)
        _bcheck(_lib.tvlbm_batch_set_graphs(h, 1 if graphs else 0), h)

    def close(self):
        if getattr(self, "handle", None):
            _lib.tvlbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tile_count(self) -> int:
        return int(_lib.tvlbm_batch_tile_count(self.handle))

    def tile_shape(self, config: int):
        tx, ty, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _bcheck(_lib.tvlbm_batch_tile_shape(self.handle, config, ctypes.byref(tx), ctypes.byref(ty),
                                            ctypes.byref(r)), self.handle)
        return tx.value, ty.value, r.value

    def set_tile(self, config: int):
        _bcheck(_lib.tvlbm_batch_set_tile(self.handle, int(config)), self.handle)

    def set_form(self, form):
        """"tiled" (one launch per time step) or "flow" (n steps in one persistent launch)."""
        _bcheck(_lib.tvlbm_batch_set_form(self.handle, FORMS[form] if isinstance(form, str) else int(form)),
                self.handle)

    def init_moments(self, d, rho, ux, uy, T):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy, T)]
        _bcheck(_lib.tvlbm_batch_init_moments(self.handle, int(d), *[_dp(a) for a in arrs]), self.handle)

    def step(self, n=1):
        _bcheck(_lib.tvlbm_batch_step(self.handle, int(n)), self.handle)

    def moments(self, d):
        outs = [np.empty((int(self.ny[d]), int(self.nx[d]))) for _ in range(4)]
        _bcheck(_lib.tvlbm_batch_moments(self.handle, int(d), *[_dp(o) for o in outs]), self.handle)
        return tuple(outs)

    def conserved_sums(self, d, allow_nonfinite: bool = False):
        out = np.zeros(5)
        rc = _lib.tvlbm_batch_conserved_sums(self.handle, int(d), _dp(out))
        if not (allow_nonfinite and rc == TVLBM_ENONFINITE):
            _bcheck(rc, self.handle)
        return out

    def populations_f64(self, d):
        out = np.empty((self.Q, int(self.ny[d]), int(self.nx[d])))
        _bcheck(_lib.tvlbm_batch_get_populations_f64(self.handle, int(d), _dp(out)), self.handle)
        return out

    def cells(self) -> int:
        return int(_lib.tvlbm_batch_cells(self.handle))

    def bytes_per_cell(self) -> float:
        return float(_lib.tvlbm_batch_bytes_per_cell(self.handle))


# ----------------------------------------------------------------------------------------------
# Learned coarse-grid closure (include/tvlbm_closure.h)
# ----------------------------------------------------------------------------------------------

def _fp(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_FP)


def _f32(a, n):
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float32).ravel())
    assert out.size == n
    return out


def _mcheck(rc: int, m=None):
    if rc != TVLBM_OK:
        msg = _lib.tvlbm_mlp_last_error(m).decode() if m else ""
        raise TvlbmError(rc, msg or _lib.tvlbm_strerror(rc).decode())


def _dev_ptr(t, dtype=None, shape=None):
    """Device address of a contiguous CUDA tensor (checked dtype / shape)."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError("expected dtype %s, got %s" % (dtype, t.dtype))
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, tuple(t.shape)))
    return _P(t.data_ptr())


class Mlp:
    """The closure network (54 -> 128 -> 128 -> 12, GELU) on the library's tensor-core kernels.
    Inputs are BF16 torch tensors [rows][64]; outputs and targets FP32 [rows][16]."""

    def __init__(self, max_rows: int, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the closure network needs a CUDA GPU")
        h = _P()
        _mcheck(_lib.tvlbm_mlp_create(int(max_rows), ctypes.byref(h)))
        self.handle = h
        self.max_rows = int(max_rows)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        _mcheck(_lib.tvlbm_mlp_set_stream(h, _P(s.cuda_stream)), h)

    def close(self):
        if getattr(self, "handle", None):
            _lib.tvlbm_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        _mcheck(_lib.tvlbm_mlp_set_params(self.handle, _fp(_f32(theta, TVLBM_MLP_PARAMS))), self.handle)

    def get_params(self) -> np.ndarray:
        out = np.zeros(TVLBM_MLP_PARAMS, dtype=np.float32)
        _mcheck(_lib.tvlbm_mlp_get_params(self.handle, _fp(out)), self.handle)
        return out

    def forward(self, x, y):
        import torch
        rows = x.shape[0]
        _mcheck(_lib.tvlbm_mlp_forward(self.handle, _dev_ptr(x, torch.bfloat16, (rows, TVLBM_MLP_IN_PAD)), rows,
                                       _dev_ptr(y, torch.float32, (rows, TVLBM_MLP_OUT_PAD))), self.handle)

    def loss_grad(self, x, ystar, want_loss=True, want_grad=False):
        import torch
        rows = x.shape[0]
        loss = ctypes.c_double(0.0)
        grad = np.zeros(TVLBM_MLP_PARAMS, dtype=np.float32) if want_grad else None
        _mcheck(_lib.tvlbm_mlp_loss_grad(self.handle, _dev_ptr(x, torch.bfloat16, (rows, TVLBM_MLP_IN_PAD)),
                                         _dev_ptr(ystar, torch.float32, (rows, TVLBM_MLP_OUT_PAD)), rows,
                                         ctypes.byref(loss) if want_loss else None,
                                         _fp(grad) if want_grad else None), self.handle)
        return (loss.value if want_loss else None), grad

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _mcheck(_lib.tvlbm_mlp_adam(self.handle, float(lr), float(beta1), float(beta2), float(eps)), self.handle)


def closure_moments(sim, m6):
    import torch
    _check(_lib.tvlbm_closure_moments(sim.ctx, _dev_ptr(m6, torch.float32, (6, sim.ny, sim.nx))), sim.ctx)


def closure_features(sim, mu, inv_sigma, x):
    import torch
    _check(_lib.tvlbm_closure_features(sim.ctx, _fp(_f32(mu, 6)), _fp(_f32(inv_sigma, 6)),
                                       _dev_ptr(x, torch.bfloat16, (sim.nx * sim.ny, TVLBM_MLP_IN_PAD))), sim.ctx)


def closure_project(a, b, o, inv_scale=None):
    import torch
    isc = _fp(_f32(inv_scale, TVLBM_MLP_OUT)) if inv_scale is not None else None
    _check(_lib.tvlbm_closure_project(a.ctx, b.ctx, isc,
                                      _dev_ptr(o, torch.float32, (a.nx * a.ny, TVLBM_MLP_OUT_PAD))), a.ctx)


def closure_noneq(sim, o, inv_scale=None):
    import torch
    isc = _fp(_f32(inv_scale, TVLBM_MLP_OUT)) if inv_scale is not None else None
    _check(_lib.tvlbm_closure_noneq(sim.ctx, isc, _dev_ptr(o, torch.float32, (sim.nx * sim.ny, TVLBM_MLP_OUT_PAD))),
           sim.ctx)


def mlp_activation(z, stream=None):
    """The network's activation as its kernels evaluate it: (GELU(z), GELU'(z)) for a device FP32
    tensor z, as new device tensors."""
    import torch
    z = z.contiguous()
    if z.dtype != torch.float32 or not z.is_cuda:
        raise TypeError("z must be a CUDA float32 tensor")
    g, dg = torch.empty_like(z), torch.empty_like(z)
    s = stream if stream is not None else torch.cuda.current_stream(z.device).cuda_stream
    rc = _lib.tvlbm_mlp_activation(_P(z.data_ptr()), _P(g.data_ptr()), _P(dg.data_ptr()), int(z.numel()), _P(s))
    if rc != TVLBM_OK:
        raise TvlbmError(rc, _lib.tvlbm_strerror(rc).decode())
    return g, dg


def downsample(fine, coarse):
    _check(_lib.tvlbm_downsample(fine.ctx, coarse.ctx), coarse.ctx)


def copy_state(src, dst):
    _check(_lib.tvlbm_copy_state(src.ctx, dst.ctx), dst.ctx)


def step_closure(sim, mlp, mu, inv_sigma, out_scale, n=1):
    _check(_lib.tvlbm_step_closure(sim.ctx, mlp.handle, _fp(_f32(mu, 6)), _fp(_f32(inv_sigma, 6)),
                                   _fp(_f32(out_scale, TVLBM_MLP_OUT)), int(n)), sim.ctx)
