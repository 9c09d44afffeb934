"""Thin ctypes binding of libdsmc.so (include/dsmc.h).

Argument marshalling only: every step of the collision path runs in the
library's CUDA kernels.  Tensors are torch CUDA tensors (device memory and
streams come from PyTorch); functions take them, check dtype/contiguity and
pass raw device pointers and the current stream.  There is no CPU fallback:
if the library cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import torch

from . import _build

DSMC_OK, DSMC_ERR_ARG, DSMC_ERR_CUDA, DSMC_ERR_CAPACITY = 0, -1, -2, -3
DSMC_ERR_TIMEOUT, DSMC_ERR_NONFINITE, DSMC_ERR_UNSUPPORTED = -4, -5, -6
PATH_VHS, PATH_JAGER, PATH_NEURAL, PATH_TABLE = 0, 1, 2, 3
MAX_ROUNDS = 1024
ORDER_ROUNDS, ORDER_LEVELS = 0, 1   # bucket order of the pair list (DSMC_ORDER_*)
_ERRS = {-1: "DSMC_ERR_ARG", -2: "DSMC_ERR_CUDA", -3: "DSMC_ERR_CAPACITY", -4: "DSMC_ERR_TIMEOUT",
         -5: "DSMC_ERR_NONFINITE", -6: "DSMC_ERR_UNSUPPORTED"}


class DsmcError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{_ERRS.get(code, code)}: {msg}")
        self.code = code


class Gas(C.Structure):
    _fields_ = [("mass", C.c_double), ("d_ref", C.c_double), ("omega", C.c_double),
                ("T_ref", C.c_double), ("fn_over_vc", C.c_double), ("dt", C.c_double),
                ("seed", C.c_uint64), ("model", C.c_int32), ("pad_", C.c_int32),
                ("b_max", C.c_double)]


class Potential(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("A", C.c_double),
                ("a1", C.c_double), ("a2", C.c_double), ("am1", C.c_double),
                ("am2", C.c_double), ("beta", C.c_double), ("C", C.c_double * 6),
                ("R_eps", C.c_double), ("At", C.c_double), ("at", C.c_double),
                ("d_hs", C.c_double), ("kappa", C.c_double), ("p", C.c_double)]


class Mlp(C.Structure):
    _fields_ = [("d_in", C.c_int32), ("width", C.c_int32), ("n_hidden", C.c_int32),
                ("d_out", C.c_int32), ("act", C.c_int32), ("pad_", C.c_int32),
                ("sigma_v", C.c_double), ("T_ref", C.c_double), ("eps", C.c_double)]


class SelectInfo(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("n_candidates", C.c_int64), ("n_rounds", C.c_int32),
                ("pad_", C.c_int32)]


class StepBuffers(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_cells", C.c_int32), ("capacity", C.c_int64),
                ("cell_id", C.c_void_p), ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p),
                ("perm", C.c_void_p), ("cell_start", C.c_void_p), ("svx", C.c_void_p),
                ("svy", C.c_void_p), ("svz", C.c_void_p), ("mom", C.c_void_p),
                ("sigma_g_max", C.c_void_p), ("pairs", C.c_void_p), ("round_offsets", C.c_void_p),
                ("info", C.c_void_p), ("ws", C.c_void_p), ("ws_bytes", C.c_size_t), ("deps", C.c_void_p)]


class ChiTableDesc(C.Structure):
    _fields_ = [("chi", C.c_void_p), ("nb", C.c_int32), ("nE", C.c_int32), ("lnE_min", C.c_double),
                ("lnE_max", C.c_double)]


class ChiTable:
    """A chi table over (b/b_max, ln(E_r/k_B)) in device memory (dsmc_chi_table_t)."""

    def __init__(self, chi: torch.Tensor, lnE_min: float, lnE_max: float):
        if chi.dtype != torch.float32 or chi.dim() != 2 or not chi.is_cuda or not chi.is_contiguous():
            raise ValueError("chi table: contiguous float32 CUDA tensor [nE x nb]")
        self.chi = chi
        self.lnE_min, self.lnE_max = float(lnE_min), float(lnE_max)
        self.desc = ChiTableDesc(chi.data_ptr(), chi.shape[1], chi.shape[0], self.lnE_min, self.lnE_max)


class TuneEntry(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("threads", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("ms", C.c_float)]


# DSMC_TUNE_* kernel ids and their names in the autotune cache
TUNE_KERNELS = ("gather", "moments", "moment_match", "collide_vhs", "collide_jager", "jager_chi", "collide_table")


class Path(C.Structure):
    _fields_ = [("path", C.c_int32), ("n_nodes", C.c_int32), ("pot", C.POINTER(Potential)),
                ("mlp", C.POINTER(Mlp)), ("weights_bf16", C.c_void_p), ("biases", C.c_void_p),
                ("table", C.POINTER(ChiTableDesc))]


# ------------------------------------------------------------------ library
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load libdsmc.so (building it first when sources changed)."""
    global _lib
    if _lib is None:
        if build:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libdsmc.so not built ({_build.LIB})")
        L = C.CDLL(_build.LIB)
        vp, i32, i64, u64, sz, d = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_size_t, C.c_double
        P = C.POINTER
        sig = {
            "dsmc_abi_version": (C.c_int, []),
            "dsmc_ctx_create": (C.c_int, [P(vp), C.c_int]),
            "dsmc_ctx_destroy": (None, [vp]),
            "dsmc_ctx_sync_status": (C.c_int, [vp, vp]),
            "dsmc_last_error": (C.c_char_p, [vp]),
            "dsmc_ctx_launch_count": (i64, [vp]),
            "dsmc_sort_workspace_size": (sz, [i32, i32]),
            "dsmc_sort_cells": (C.c_int, [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
            "dsmc_sort_cells_static": (C.c_int, [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "dsmc_cell_moments": (C.c_int, [vp, i32, vp, vp, vp, vp, vp, vp]),
            "dsmc_sigma_g_max_init": (C.c_int, [vp, P(Gas), i32, vp, d, vp, vp]),
            "dsmc_select_workspace_size": (sz, [i32, i32, i64]),
            "dsmc_select_pairs": (C.c_int, [vp, P(Gas), i32, i32, vp, vp, vp, vp, vp, u64, i64, vp, vp, vp,
                                            vp, vp, sz, vp]),
            "dsmc_select_pairs_ordered": (C.c_int, [vp, P(Gas), i32, i32, vp, vp, vp, vp, vp, u64, i64, vp, vp,
                                                    vp, vp, i32, vp, sz, vp]),
            "dsmc_collide_workspace_size": (sz, [i32]),
            "dsmc_collide_vhs": (C.c_int, [vp, P(Gas), u64, i32, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
            "dsmc_jager_chi": (C.c_int, [vp, P(Gas), P(Potential), i32, i64, vp, vp, vp, vp]),
            "dsmc_collide_jager": (C.c_int, [vp, P(Gas), P(Potential), i32, u64, i32, vp, vp, vp, vp, vp,
                                             vp, vp, vp, vp, sz, vp]),
            "dsmc_chi_table_build": (C.c_int, [vp, P(Gas), P(Potential), i32, i32, i32, d, d, vp, vp]),
            "dsmc_transport_q2": (C.c_int, [vp, P(Potential), i32, i32, vp, d, i32, vp, vp]),
            "dsmc_chi_mlp_packed_size": (C.c_size_t, []),
            "dsmc_chi_mlp_pack": (C.c_int, [vp, vp, vp, vp]),
            "dsmc_chi_mlp_forward": (C.c_int, [vp, vp, vp, i64, vp, vp, vp, vp]),
            "dsmc_chi_mlp_table": (C.c_int, [vp, vp, vp, i32, i32, vp, vp]),
            "dsmc_transport_workspace_size": (C.c_size_t, [i32, i32]),
            "dsmc_transport_viscosity": (C.c_int, [vp, P(Gas), P(Potential), i32, i32, vp, d, i32, i32, vp, vp,
                                                   vp, C.c_size_t, vp]),
            "dsmc_collide_table": (C.c_int, [vp, P(Gas), P(ChiTableDesc), u64, i32, vp, vp, vp, vp, vp, vp, vp, vp,
                                             vp, sz, vp]),
            "dsmc_collide_neural": (C.c_int, [vp, P(Gas), P(Mlp), vp, vp, u64, vp, i32, vp, vp, vp, vp, vp,
                                              vp, vp, vp, vp, sz, vp]),
            "dsmc_mlp_forward": (C.c_int, [vp, P(Mlp), vp, vp, i64, vp, vp, vp]),
            "dsmc_tc_selftest": (C.c_int, [vp, i32, i32, i32, vp, vp, vp, vp]),
            "dsmc_selftest_timeout": (C.c_int, [vp, i32, u64, vp]),
            "dsmc_selftest_peak_ops": (i64, [i32, i32]),
            "dsmc_selftest_math": (C.c_int, [vp, i32, i64, vp, vp, vp]),
            "dsmc_selftest_peak": (C.c_int, [vp, i32, i32, i32, i32, vp, vp]),
            "dsmc_moment_match": (C.c_int, [vp, i32, vp, vp, vp, vp, vp, vp]),
            "dsmc_step_workspace_size": (sz, [i32, i32, i64]),
            "dsmc_step": (C.c_int, [vp, P(Gas), P(Path), P(StepBuffers), u64, vp]),
            "dsmc_step_fused": (C.c_int, [vp, P(Gas), P(Path), P(StepBuffers), u64, vp]),
            "dsmc_ctx_reserve": (C.c_int, [vp, i32, i32, i64]),
            "dsmc_step_graph_capture": (C.c_int, [vp, P(Gas), P(Path), P(StepBuffers), vp]),
            "dsmc_step_graph_launch": (C.c_int, [vp, u64, vp]),
            "dsmc_step_host": (C.c_int, [vp, P(Gas), P(Path), i32, vp, vp, vp, vp, vp, u64, vp, vp,
                                         vp, vp, P(i64), vp]),
            "dsmc_harvest_jager": (C.c_int, [vp, P(Gas), P(Potential), i32, i64, vp, vp, vp, vp, vp,
                                             vp, vp]),
            "dsmc_mlp_param_count": (i32, [P(Mlp)]),
            "dsmc_train_workspace_size": (sz, [vp]),
            "dsmc_neural_operator_forward": (C.c_int, [vp, P(Mlp), vp, u64, u64, i64, vp, vp, vp, vp, vp, vp]),
            "dsmc_neural_operator_backward": (C.c_int, [vp, P(Mlp), vp, u64, u64, i64, vp, vp, vp, vp, vp, vp,
                                                        vp, sz, vp]),
            "dsmc_train_loss_grad": (C.c_int, [vp, P(Mlp), vp, u64, u64, i64, vp, vp, vp, vp, vp, vp, vp, vp,
                                               sz, vp]),
            "dsmc_train_act_size": (sz, [i64]),
            "dsmc_train_loss_grad_stored": (C.c_int, [vp, P(Mlp), vp, u64, u64, i64, vp, vp, vp, vp, vp, vp, vp, vp,
                                                      sz, vp, sz, vp]),
            "dsmc_adam_step": (C.c_int, [vp, i32, i32, vp, vp, vp, vp, i64, C.c_float, C.c_float, C.c_float,
                                         C.c_float, vp, vp, vp]),
            "dsmc_tune_set": (C.c_int, [vp, i32, i32, i32]),
            "dsmc_tune_get": (C.c_int, [vp, i32, P(i32), P(i32)]),
            "dsmc_tune_candidates": (C.c_int, [vp, i32, P(TuneEntry), i32, P(i32)]),
            "dsmc_autotune_step": (C.c_int, [vp, P(Gas), P(Path), P(StepBuffers), u64, i32, P(TuneEntry), i32,
                                             P(i32), vp]),
            "dsmc_autotune_chi": (C.c_int, [vp, P(Gas), P(Potential), i32, i64, vp, vp, vp, i32, P(TuneEntry),
                                            i32, P(i32), vp]),
            "dsmc_train_step": (C.c_int, [vp, P(Mlp), vp, vp, vp, i64, C.c_float, u64, i64, vp, vp, vp, vp,
                                          vp, vp, vp, vp, vp, vp, sz, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ------------------------------------------------------------------ helpers

def _ptr(t: torch.Tensor | None, dtype=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_gas(d: dict) -> Gas:
    return Gas(d["mass"], d.get("d_ref", 0.0), d.get("omega", 0.5), d.get("T_ref", 273.0),
               d["fn_over_vc"], d["dt"], int(d.get("seed", 0)), int(d.get("model", 0)), 0,
               d.get("b_max", 0.0))


def make_potential(d: dict) -> Potential:
    P = Potential()
    P.kind = int(d.get("kind", 0))
    for k in ("A", "a1", "a2", "am1", "am2", "beta", "R_eps", "At", "at", "d_hs", "kappa", "p"):
        setattr(P, k, float(d.get(k, 0.0)))
    cs = d.get("C", [0.0] * 6)
    for q in range(6):
        P.C[q] = float(cs[q])
    return P


def make_mlp(d_in=8, width=128, n_hidden=3, d_out=3, act=0, sigma_v=1.0, T_ref=273.0, eps=1e-12) -> Mlp:
    return Mlp(d_in, width, n_hidden, d_out, act, 0, sigma_v, T_ref, eps)


class Context:
    """A library context on one device (status word, barrier words)."""

    def __init__(self, device: int = 0):
        L = load()
        self._lib = L
        h = C.c_void_p()
        rc = L.dsmc_ctx_create(C.byref(h), device)
        if rc != 0:
            raise DsmcError(rc, "dsmc_ctx_create")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self._lib.dsmc_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != 0:
            raise DsmcError(rc, f"{what}: {self._lib.dsmc_last_error(self.h).decode()}")

    def launch_count(self) -> int:
        return self._lib.dsmc_ctx_launch_count(self.h)

    def sync_status(self, stream=None) -> int:
        return self._lib.dsmc_ctx_sync_status(self.h, _stream(stream))

    def check_status(self, stream=None):
        rc = self.sync_status(stream)
        if rc != 0:
            raise DsmcError(rc, "device-side status")

    # -------------------------------------------------------------- step pieces
    def sort_cells(self, cell_id, vx, vy, vz, n_cells, out=None, ws=None, stream=None):
        n = cell_id.numel()
        dev = cell_id.device
        if out is None:
            out = dict(perm=torch.empty(n, dtype=torch.int32, device=dev),
                       cell_start=torch.empty(n_cells + 1, dtype=torch.int32, device=dev),
                       svx=torch.empty(n, dtype=torch.float64, device=dev),
                       svy=torch.empty(n, dtype=torch.float64, device=dev),
                       svz=torch.empty(n, dtype=torch.float64, device=dev))
        nbytes = self._lib.dsmc_sort_workspace_size(n, n_cells)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        f64 = torch.float64
        self._check(self._lib.dsmc_sort_cells(
            self.h, n, n_cells, _ptr(cell_id, torch.int32), _ptr(vx, f64), _ptr(vy, f64), _ptr(vz, f64),
            _ptr(out["perm"]), _ptr(out["cell_start"]), _ptr(out["svx"]), _ptr(out["svy"]),
            _ptr(out["svz"]), _ptr(ws), nbytes, _stream(stream)), "sort_cells")
        return out

    def cell_moments(self, cell_start, vx, vy, vz, mom=None, stream=None):
        nc = cell_start.numel() - 1
        if mom is None:
            mom = torch.empty((nc, 5), dtype=torch.float64, device=cell_start.device)
        self._check(self._lib.dsmc_cell_moments(self.h, nc, _ptr(cell_start, torch.int32), _ptr(vx),
                                                _ptr(vy), _ptr(vz), _ptr(mom, torch.float64),
                                                _stream(stream)), "cell_moments")
        return mom

    def sigma_g_max_init(self, gas: Gas, T_cell, factor=5.0, out=None, stream=None):
        if out is None:
            out = torch.empty_like(T_cell)
        self._check(self._lib.dsmc_sigma_g_max_init(self.h, C.byref(gas), T_cell.numel(),
                                                    _ptr(T_cell, torch.float64), factor, _ptr(out),
                                                    _stream(stream)), "sigma_g_max_init")
        return out

    def select_pairs(self, gas: Gas, cell_start, vx, vy, vz, sgmax, step, capacity, out=None,
                     ws=None, stream=None, order=ORDER_ROUNDS):
        nc = cell_start.numel() - 1
        n = vx.numel()
        dev = vx.device
        if out is None:
            out = dict(pairs=torch.empty((max(capacity, 1), 4), dtype=torch.int32, device=dev),
                       deps=torch.empty(max(capacity, 1), dtype=torch.int32, device=dev),
                       round_offsets=torch.empty(MAX_ROUNDS + 1, dtype=torch.int32, device=dev),
                       info=torch.zeros(3, dtype=torch.int64, device=dev))
        nbytes = self._lib.dsmc_select_workspace_size(n, nc, capacity)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self._check(self._lib.dsmc_select_pairs_ordered(
            self.h, C.byref(gas), n, nc, _ptr(cell_start, torch.int32), _ptr(vx, torch.float64),
            _ptr(vy, torch.float64), _ptr(vz, torch.float64), _ptr(sgmax, torch.float64), step,
            capacity, _ptr(out["pairs"]), _ptr(out["deps"]), _ptr(out["round_offsets"]), _ptr(out["info"]),
            order, _ptr(ws), nbytes, _stream(stream)), "select_pairs")
        return out

    def _collide_ws(self, n, device, ws=None):
        """Workspace of the collide calls (one done stamp per particle): the
        caller's, else one kept by this object per device."""
        nbytes = self._lib.dsmc_collide_workspace_size(n)
        if ws is not None:
            if ws.numel() < nbytes:
                raise ValueError("collide workspace too small")
            return ws, nbytes
        key = ("collide_ws", str(device))
        cur = getattr(self, "_ws_cache", {}).get(key)
        if cur is None or cur.numel() < nbytes:
            cur = torch.empty(nbytes, dtype=torch.uint8, device=device)
            self._ws_cache = getattr(self, "_ws_cache", {})
            self._ws_cache[key] = cur
        return cur, nbytes

    def collide_vhs(self, gas: Gas, step, sel, vx, vy, vz, ws=None, stream=None):
        w, nb = self._collide_ws(vx.numel(), vx.device, ws)
        self._check(self._lib.dsmc_collide_vhs(self.h, C.byref(gas), step, vx.numel(), _ptr(sel["pairs"]),
                                               _ptr(sel["deps"]), _ptr(sel["round_offsets"]), _ptr(sel["info"]),
                                               _ptr(vx, torch.float64), _ptr(vy, torch.float64),
                                               _ptr(vz, torch.float64), _ptr(w), nb, _stream(stream)), "collide_vhs")

    def jager_chi(self, gas: Gas, pot: Potential, b, g, n_nodes=32, chi=None, stream=None):
        if chi is None:
            chi = torch.empty_like(b)
        self._check(self._lib.dsmc_jager_chi(self.h, C.byref(gas), C.byref(pot), n_nodes, b.numel(),
                                             _ptr(b, torch.float32), _ptr(g, torch.float32), _ptr(chi),
                                             _stream(stream)), "jager_chi")
        return chi

    def collide_jager(self, gas: Gas, pot: Potential, step, sel, vx, vy, vz, n_nodes=32,
                      chi_out=None, ws=None, stream=None):
        w, nb = self._collide_ws(vx.numel(), vx.device, ws)
        self._check(self._lib.dsmc_collide_jager(
            self.h, C.byref(gas), C.byref(pot), n_nodes, step, vx.numel(), _ptr(sel["pairs"]), _ptr(sel["deps"]),
            _ptr(sel["round_offsets"]), _ptr(sel["info"]), _ptr(vx, torch.float64),
            _ptr(vy, torch.float64), _ptr(vz, torch.float64), _ptr(chi_out, torch.float32),
            _ptr(w), nb, _stream(stream)), "collide_jager")

    def chi_table_build(self, gas: Gas, pot: Potential, nb=512, nE=512, lnE_min=math.log(5.0),
                        lnE_max=math.log(6.0e4), n_nodes=32, stream=None) -> "ChiTable":
        """dsmc_chi_table_build: the exact chi on the (b/b_max, ln E) grid."""
        chi = torch.empty((nE, nb), dtype=torch.float32, device=torch.device("cuda", self.device))
        self._check(self._lib.dsmc_chi_table_build(self.h, C.byref(gas), C.byref(pot), n_nodes, nb, nE, lnE_min,
                                                   lnE_max, _ptr(chi), _stream(stream)), "chi_table_build")
        return ChiTable(chi, lnE_min, lnE_max)

    def transport_q2(self, pot: Potential, E_kelvin, b_max_A=12.0, b_panels=32, n_nodes=32, out=None,
                     stream=None):
        """dsmc_transport_q2: Q2(E) in m^2 at the energies E_kelvin (float64, device)."""
        if out is None:
            out = torch.empty_like(E_kelvin)
        self._check(self._lib.dsmc_transport_q2(self.h, C.byref(pot), n_nodes, E_kelvin.numel(),
                                                _ptr(E_kelvin, torch.float64), b_max_A, b_panels,
                                                _ptr(out, torch.float64), _stream(stream)), "transport_q2")
        return out

    def transport_viscosity(self, gas: Gas, pot: Potential, T_kelvin, b_max_A=12.0, b_panels=32, x_panels=8,
                            n_nodes=32, stream=None):
        """dsmc_transport_viscosity: (Omega22 in m^2, mu in Pa s) at the temperatures T_kelvin."""
        n = T_kelvin.numel()
        om = torch.empty_like(T_kelvin)
        mu = torch.empty_like(T_kelvin)
        nb = self._lib.dsmc_transport_workspace_size(n, x_panels)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=T_kelvin.device)
        self._check(self._lib.dsmc_transport_viscosity(self.h, C.byref(gas), C.byref(pot), n_nodes, n,
                                                       _ptr(T_kelvin, torch.float64), b_max_A, b_panels, x_panels,
                                                       _ptr(om, torch.float64), _ptr(mu, torch.float64), _ptr(ws),
                                                       nb, _stream(stream)), "transport_viscosity")
        return om, mu

    def chi_mlp_pack(self, w_bits, stream=None):
        """dsmc_chi_mlp_pack: the chi-MLP weights (bf16 bits, int16 tensor) in the
        kernel's streamed operand layout."""
        nb = self._lib.dsmc_chi_mlp_packed_size()
        packed = torch.empty(nb, dtype=torch.uint8, device=w_bits.device)
        self._check(self._lib.dsmc_chi_mlp_pack(self.h, _ptr(w_bits, torch.int16), _ptr(packed), _stream(stream)),
                    "chi_mlp_pack")
        return packed

    def chi_mlp_forward(self, packed, bias, x, y=None, chi=None, stream=None):
        """dsmc_chi_mlp_forward: x [n, 2] float32 -> (y, chi), float32 [n]."""
        n = x.shape[0]
        if y is None:
            y = torch.empty(n, dtype=torch.float32, device=x.device)
        if chi is None:
            chi = torch.empty(n, dtype=torch.float32, device=x.device)
        self._check(self._lib.dsmc_chi_mlp_forward(self.h, _ptr(packed), _ptr(bias, torch.float32), n,
                                                   _ptr(x, torch.float32), _ptr(y, torch.float32),
                                                   _ptr(chi, torch.float32), _stream(stream)), "chi_mlp_forward")
        return y, chi

    def chi_mlp_table(self, packed, bias, nb=512, nE=512, out=None, stream=None):
        """dsmc_chi_mlp_table: the nE x nb chi table synthesised by the chi-MLP."""
        if out is None:
            out = torch.empty((nE, nb), dtype=torch.float32, device=packed.device)
        self._check(self._lib.dsmc_chi_mlp_table(self.h, _ptr(packed), _ptr(bias, torch.float32), nb, nE,
                                                 _ptr(out, torch.float32), _stream(stream)), "chi_mlp_table")
        return out

    def collide_table(self, gas: Gas, table: "ChiTable", step, sel, vx, vy, vz, chi_out=None, ws=None,
                      stream=None):
        w, nb = self._collide_ws(vx.numel(), vx.device, ws)
        self._check(self._lib.dsmc_collide_table(
            self.h, C.byref(gas), C.byref(table.desc), step, vx.numel(), _ptr(sel["pairs"]), _ptr(sel["deps"]),
            _ptr(sel["round_offsets"]), _ptr(sel["info"]), _ptr(vx, torch.float64), _ptr(vy, torch.float64),
            _ptr(vz, torch.float64), _ptr(chi_out, torch.float32), _ptr(w), nb, _stream(stream)), "collide_table")

    def collide_neural(self, gas: Gas, mlp: Mlp, w_bits, bias, step, mom, sel, vx, vy, vz,
                       u_out=None, ws=None, stream=None):
        w, nb = self._collide_ws(vx.numel(), vx.device, ws)
        self._check(self._lib.dsmc_collide_neural(
            self.h, C.byref(gas), C.byref(mlp), _ptr(w_bits, torch.int16), _ptr(bias, torch.float32),
            step, _ptr(mom, torch.float64), vx.numel(), _ptr(sel["pairs"]), _ptr(sel["deps"]),
            _ptr(sel["round_offsets"]), _ptr(sel["info"]), _ptr(vx, torch.float64), _ptr(vy, torch.float64),
            _ptr(vz, torch.float64), _ptr(u_out, torch.float32), _ptr(w), nb, _stream(stream)), "collide_neural")

    def mlp_forward(self, mlp: Mlp, w_bits, bias, x, y=None, stream=None):
        n = x.shape[0]
        if y is None:
            y = torch.empty((n, 3), dtype=torch.float32, device=x.device)
        self._check(self._lib.dsmc_mlp_forward(self.h, C.byref(mlp), _ptr(w_bits, torch.int16),
                                               _ptr(bias, torch.float32), n, _ptr(x, torch.float32),
                                               _ptr(y, torch.float32), _stream(stream)), "mlp_forward")
        return y

    def tc_selftest(self, A_bits, B_bits, layout=0, stream=None):
        K = A_bits.shape[1]
        N = B_bits.shape[0]
        D = torch.empty((128, N), dtype=torch.float32, device=A_bits.device)
        self._check(self._lib.dsmc_tc_selftest(self.h, N, K, layout, _ptr(A_bits, torch.int16),
                                               _ptr(B_bits, torch.int16), _ptr(D), _stream(stream)),
                    "tc_selftest")
        return D

    def selftest_math(self, which: int, x, stream=None):
        """dsmc_selftest_math: f(x) elementwise (float64 device tensors)."""
        y = torch.empty_like(x)
        self._check(self._lib.dsmc_selftest_math(self.h, which, x.numel(), _ptr(x, torch.float64), _ptr(y),
                                                 _stream(stream)), "selftest_math")
        return y

    PEAK_KINDS = ("fp32_fma", "fp32x2_fma", "fp64_fma", "mufu_ex2")

    def selftest_peak(self, which: int, blocks: int, threads: int, iters: int, sink=None, stream=None):
        """dsmc_selftest_peak: launch one pipe-rate kernel; returns (sink, total
        operations of the launch).  Time it with CUDA events on `stream`."""
        if sink is None or sink.numel() < blocks * threads:
            sink = torch.empty(blocks * threads, dtype=torch.float32, device=torch.device("cuda", self.device))
        self._check(self._lib.dsmc_selftest_peak(self.h, which, blocks, threads, iters, _ptr(sink, torch.float32),
                                                 _stream(stream)), "selftest_peak")
        return sink, int(self._lib.dsmc_selftest_peak_ops(which, iters)) * blocks * threads

    def selftest_timeout(self, which: int, limit_ns: int = 10_000_000, stream=None):
        self._check(self._lib.dsmc_selftest_timeout(self.h, which, limit_ns, _stream(stream)),
                    "selftest_timeout")

    def moment_match(self, cell_start, mom_pre, vx, vy, vz, stream=None):
        self._check(self._lib.dsmc_moment_match(self.h, cell_start.numel() - 1,
                                                _ptr(cell_start, torch.int32),
                                                _ptr(mom_pre, torch.float64), _ptr(vx, torch.float64),
                                                _ptr(vy, torch.float64), _ptr(vz, torch.float64),
                                                _stream(stream)), "moment_match")

    def harvest_jager(self, gas: Gas, pot: Potential, vi, vj, b, eps, n_nodes=32, stream=None):
        vio, vjo = torch.empty_like(vi), torch.empty_like(vj)
        self._check(self._lib.dsmc_harvest_jager(
            self.h, C.byref(gas), C.byref(pot), n_nodes, b.numel(), _ptr(vi, torch.float64),
            _ptr(vj, torch.float64), _ptr(b, torch.float64), _ptr(eps, torch.float64), _ptr(vio),
            _ptr(vjo), _stream(stream)), "harvest_jager")
        return vio, vjo

    # -------------------------------------------------------------- training
    def param_count(self, mlp: Mlp) -> int:
        return self._lib.dsmc_mlp_param_count(C.byref(mlp))

    def train_workspace(self, device="cuda"):
        nb = self._lib.dsmc_train_workspace_size(self.h)
        return torch.empty(nb, dtype=torch.uint8, device=device)

    def neural_operator_forward(self, mlp: Mlp, theta, seed, t, vi, vj, T, stream=None):
        vin, vjn = torch.empty_like(vi), torch.empty_like(vj)
        f64 = torch.float64
        self._check(self._lib.dsmc_neural_operator_forward(
            self.h, C.byref(mlp), _ptr(theta, torch.float32), seed, t, vi.shape[0], _ptr(vi, f64),
            _ptr(vj, f64), _ptr(T, f64), _ptr(vin), _ptr(vjn), _stream(stream)), "neural_operator_forward")
        return vin, vjn

    def neural_operator_backward(self, mlp: Mlp, theta, seed, t, vi, vj, T, g_vi, g_vj, ws=None,
                                 stream=None):
        grad = torch.empty_like(theta)
        ws = ws if ws is not None else self.train_workspace(theta.device)
        f64 = torch.float64
        self._check(self._lib.dsmc_neural_operator_backward(
            self.h, C.byref(mlp), _ptr(theta, torch.float32), seed, t, vi.shape[0], _ptr(vi, f64),
            _ptr(vj, f64), _ptr(T, f64), _ptr(g_vi, f64), _ptr(g_vj, f64), _ptr(grad), _ptr(ws),
            ws.numel(), _stream(stream)), "neural_operator_backward")
        return grad

    def train_loss_grad(self, mlp: Mlp, theta, seed, t, vi, vj, T, vi_t, vj_t, ws=None, stream=None):
        grad = torch.empty_like(theta)
        loss = torch.zeros(1, dtype=torch.float64, device=theta.device)
        ws = ws if ws is not None else self.train_workspace(theta.device)
        f64 = torch.float64
        self._check(self._lib.dsmc_train_loss_grad(
            self.h, C.byref(mlp), _ptr(theta, torch.float32), seed, t, vi.shape[0], _ptr(vi, f64),
            _ptr(vj, f64), _ptr(T, f64), _ptr(vi_t, f64), _ptr(vj_t, f64), _ptr(grad), _ptr(loss),
            _ptr(ws), ws.numel(), _stream(stream)), "train_loss_grad")
        return grad, loss

    def train_loss_grad_stored(self, mlp: Mlp, theta, seed, t, vi, vj, T, vi_t, vj_t, ws=None, act=None,
                               stream=None):
        """dsmc_train_loss_grad_stored: the same loss and gradient with the
        hidden layers' pre-activations stored by the forward and read back by
        the backward (the check of the recomputation)."""
        grad = torch.empty_like(theta)
        loss = torch.zeros(1, dtype=torch.float64, device=theta.device)
        ws = ws if ws is not None else self.train_workspace(theta.device)
        nb = self._lib.dsmc_train_act_size(vi.shape[0])
        if act is None or act.numel() * 4 < nb:
            act = torch.empty(max(nb // 4, 1), dtype=torch.float32, device=theta.device)
        f64 = torch.float64
        self._check(self._lib.dsmc_train_loss_grad_stored(
            self.h, C.byref(mlp), _ptr(theta, torch.float32), seed, t, vi.shape[0], _ptr(vi, f64),
            _ptr(vj, f64), _ptr(T, f64), _ptr(vi_t, f64), _ptr(vj_t, f64), _ptr(grad), _ptr(loss),
            _ptr(ws), ws.numel(), _ptr(act, torch.float32), act.numel() * 4, _stream(stream)),
            "train_loss_grad_stored")
        return grad, loss

    def adam_step(self, n_weights, grad, theta, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                  w_bits=None, bias=None, stream=None):
        self._check(self._lib.dsmc_adam_step(
            self.h, theta.numel(), n_weights, _ptr(grad, torch.float32), _ptr(theta, torch.float32),
            _ptr(m, torch.float32), _ptr(v, torch.float32), step, lr, beta1, beta2, eps,
            _ptr(w_bits, torch.int16), _ptr(bias, torch.float32), _stream(stream)), "adam_step")

    def train_step(self, mlp: Mlp, theta, m, v, step, lr, seed, vi, vj, T, vi_t, vj_t, grad, loss,
                   ws, w_bits=None, bias=None, stream=None):
        f64 = torch.float64
        self._check(self._lib.dsmc_train_step(
            self.h, C.byref(mlp), _ptr(theta, torch.float32), _ptr(m), _ptr(v), step, lr, seed,
            vi.shape[0], _ptr(vi, f64), _ptr(vj, f64), _ptr(T, f64), _ptr(vi_t, f64), _ptr(vj_t, f64),
            _ptr(grad), _ptr(loss), _ptr(w_bits, torch.int16), _ptr(bias, torch.float32), _ptr(ws),
            ws.numel(), _stream(stream)), "train_step")

    # -------------------------------------------------------------- whole step
    def step_workspace_size(self, n, n_cells, capacity) -> int:
        return self._lib.dsmc_step_workspace_size(n, n_cells, capacity)

    def step(self, gas: Gas, path: Path, bufs: "StepState", step: int, stream=None):
        self._check(self._lib.dsmc_step(self.h, C.byref(gas), C.byref(path), C.byref(bufs.desc),
                                        step, _stream(stream)), "step")

    def step_fused(self, gas: Gas, path: Path, bufs: "StepState", step: int, stream=None):
        """The step fused into one pass over cell groups (VHS and look-up paths)."""
        self._check(self._lib.dsmc_step_fused(self.h, C.byref(gas), C.byref(path), C.byref(bufs.desc),
                                              step, _stream(stream)), "step_fused")

    def step_graph_capture(self, gas: Gas, path: Path, bufs: "StepState", stream):
        """Capture a whole step as a CUDA graph (stream: a non-default torch stream)."""
        self._graph_keep = (gas, path, bufs)
        self._check(self._lib.dsmc_step_graph_capture(self.h, C.byref(gas), C.byref(path),
                                                      C.byref(bufs.desc), _stream(stream)),
                    "step_graph_capture")

    def step_graph_launch(self, step: int, stream=None):
        self._check(self._lib.dsmc_step_graph_launch(self.h, step, _stream(stream)), "step_graph_launch")

    def reserve(self, n_max, n_cells, capacity):
        self._check(self._lib.dsmc_ctx_reserve(self.h, n_max, n_cells, capacity), "reserve")

    def step_host(self, gas: Gas, path: Path, cell_id, vx, vy, vz, T_cell, step, perm, svx, svy,
                  svz, stream=None) -> int:
        """Host-memory step: all array arguments are (pinned) CPU tensors."""
        npairs = C.c_int64(0)
        hp = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        self._check(self._lib.dsmc_step_host(
            self.h, C.byref(gas), C.byref(path), cell_id.numel(), hp(cell_id), hp(vx), hp(vy), hp(vz),
            hp(T_cell), step, hp(perm), hp(svx), hp(svy), hp(svz), C.byref(npairs), _stream(stream)),
            "step_host")
        return npairs.value


    # -------------------------------------------------------------- launch shapes
    def tune_set(self, kernel: int, threads: int = 0, blocks_per_sm: int = 0):
        self._check(self._lib.dsmc_tune_set(self.h, kernel, threads, blocks_per_sm), "tune_set")

    def tune_get(self, kernel: int) -> tuple[int, int]:
        t, b = C.c_int32(0), C.c_int32(0)
        self._check(self._lib.dsmc_tune_get(self.h, kernel, C.byref(t), C.byref(b)), "tune_get")
        return t.value, b.value

    def tune_candidates(self, kernel: int) -> list[tuple[int, int]]:
        buf, n = (TuneEntry * 64)(), C.c_int32(0)
        self._check(self._lib.dsmc_tune_candidates(self.h, kernel, buf, 64, C.byref(n)), "tune_candidates")
        return [(buf[q].threads, buf[q].blocks_per_sm) for q in range(min(n.value, 64))]

    @staticmethod
    def _trials(buf, n):
        return [dict(kernel=TUNE_KERNELS[buf[q].kernel], threads=buf[q].threads,
                     blocks_per_sm=buf[q].blocks_per_sm, ms=float(buf[q].ms)) for q in range(n)]

    def autotune_step(self, gas: Gas, path: Path, bufs: "StepState", step: int = 0, reps: int = 3,
                      stream=None) -> list[dict]:
        """dsmc_autotune_step: time the candidate shapes of the step's tunable
        kernels on these buffers (their contents are consumed) and keep the
        fastest in the context.  Returns every measured trial."""
        buf, n = (TuneEntry * 256)(), C.c_int32(0)
        self._check(self._lib.dsmc_autotune_step(self.h, C.byref(gas), C.byref(path), C.byref(bufs.desc), step,
                                                 reps, buf, 256, C.byref(n), _stream(stream)), "autotune_step")
        return self._trials(buf, min(n.value, 256))

    def autotune_chi(self, gas: Gas, pot: Potential, b, g, n_nodes=32, chi=None, reps=3, stream=None):
        chi = torch.empty_like(b) if chi is None else chi
        buf, n = (TuneEntry * 64)(), C.c_int32(0)
        self._check(self._lib.dsmc_autotune_chi(self.h, C.byref(gas), C.byref(pot), n_nodes, b.numel(),
                                                _ptr(b, torch.float32), _ptr(g, torch.float32),
                                                _ptr(chi, torch.float32), reps, buf, 64, C.byref(n),
                                                _stream(stream)), "autotune_chi")
        return self._trials(buf, min(n.value, 64))

    def tuned_shapes(self) -> dict:
        return {name: self.tune_get(k) for k, name in enumerate(TUNE_KERNELS)}


# ------------------------------------------------------------------ autotune cache
# JSON: {device name: {kernel name: {size bucket: {"threads": t, "blocks_per_sm": b, "ms": m}}}},
# the bucket being floor(log2(particles)) (pairs for the chi batch).

def size_bucket(n: int) -> str:
    return str(max(int(n), 1).bit_length() - 1)


def tune_cache_store(path: str, ctx: Context, n: int, trials: list[dict], device_name: str | None = None):
    """Record the fastest measured shape of each kernel in ``trials`` under
    (device, kernel, size bucket) in the JSON file at ``path``."""
    import json
    dev = device_name or torch.cuda.get_device_name(ctx.device)
    try:
        with open(path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    best = {}
    for t in trials:
        if t["kernel"] not in best or t["ms"] < best[t["kernel"]]["ms"]:
            best[t["kernel"]] = t
    for k, t in best.items():
        cache.setdefault(dev, {}).setdefault(k, {})[size_bucket(n)] = dict(
            threads=t["threads"], blocks_per_sm=t["blocks_per_sm"], ms=t["ms"])
    with open(path, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    return cache


def tune_cache_apply(path: str, ctx: Context, n: int, device_name: str | None = None) -> dict:
    """Set the context's shapes from the cache entries of this device and
    size bucket; returns what was applied."""
    import json
    dev = device_name or torch.cuda.get_device_name(ctx.device)
    try:
        with open(path) as f:
            cache = json.load(f).get(dev, {})
    except (OSError, ValueError):
        return {}
    applied = {}
    for k, name in enumerate(TUNE_KERNELS):
        e = cache.get(name, {}).get(size_bucket(n))
        if e:
            ctx.tune_set(k, int(e["threads"]), int(e["blocks_per_sm"]))
            applied[name] = (int(e["threads"]), int(e["blocks_per_sm"]))
    return applied


STATIC_SORT_MAX_N, STATIC_SORT_MAX_CELLS = 1 << 20, 1 << 18


def sort_cells_static(cell_id, vx, vy, vz, n_cells, out=None, status=None, stream=None):
    """Allocation-free cell sort (dsmc_sort_cells_static): no context, no
    workspace; at most STATIC_SORT_MAX_N particles and STATIC_SORT_MAX_CELLS
    cells.  Output tensors may be passed in ``out`` so that nothing is
    allocated around the call either.  Every tensor must live on the same
    GPU; the call runs with that GPU current (the library looks up its
    scratch array on the current device)."""
    L = load()
    n = cell_id.numel()
    dev = cell_id.device
    if out is None:
        out = dict(perm=torch.empty(n, dtype=torch.int32, device=dev),
                   cell_start=torch.empty(n_cells + 1, dtype=torch.int32, device=dev),
                   svx=torch.empty(n, dtype=torch.float64, device=dev),
                   svy=torch.empty(n, dtype=torch.float64, device=dev),
                   svz=torch.empty(n, dtype=torch.float64, device=dev))
    need = dict(perm=n, cell_start=n_cells + 1, svx=n, svy=n, svz=n)
    for k, m in need.items():
        if out[k].numel() < m:
            raise ValueError(f"sort_cells_static: out['{k}'] holds {out[k].numel()} entries, needs {m}")
    for name, t in [("vx", vx), ("vy", vy), ("vz", vz), ("status", status)] + list(out.items()):
        if t is not None and t.device != dev:
            raise ValueError(f"sort_cells_static: {name} is on {t.device}, cell_id on {dev}")
    if min(vx.numel(), vy.numel(), vz.numel()) < n:
        raise ValueError("sort_cells_static: velocity arrays shorter than cell_id")
    f64 = torch.float64
    with torch.cuda.device(dev):
        rc = L.dsmc_sort_cells_static(n, n_cells, _ptr(cell_id, torch.int32), _ptr(vx, f64), _ptr(vy, f64),
                                      _ptr(vz, f64), _ptr(out["perm"], torch.int32),
                                      _ptr(out["cell_start"], torch.int32), _ptr(out["svx"], f64),
                                      _ptr(out["svy"], f64), _ptr(out["svz"], f64),
                                      _ptr(status, torch.int32), _stream(stream))
    if rc != 0:
        raise DsmcError(rc, "dsmc_sort_cells_static")
    return out


class StepState:
    """Device buffers of one collision step (see dsmc_step_buffers_t)."""

    def __init__(self, ctx: Context, n, n_cells, capacity, device="cuda"):
        dev = torch.device(device)
        f64, i32 = torch.float64, torch.int32
        self.n, self.n_cells, self.capacity = n, n_cells, capacity
        self.cell_id = torch.empty(n, dtype=i32, device=dev)
        self.vx, self.vy, self.vz = (torch.empty(n, dtype=f64, device=dev) for _ in range(3))
        self.perm = torch.empty(n, dtype=i32, device=dev)
        self.cell_start = torch.empty(n_cells + 1, dtype=i32, device=dev)
        self.svx, self.svy, self.svz = (torch.empty(n, dtype=f64, device=dev) for _ in range(3))
        self.mom = torch.empty((n_cells, 5), dtype=f64, device=dev)
        self.sigma_g_max = torch.empty(n_cells, dtype=f64, device=dev)
        self.pairs = torch.empty((max(capacity, 1), 4), dtype=i32, device=dev)
        self.deps = torch.empty(max(capacity, 1), dtype=i32, device=dev)
        self.round_offsets = torch.empty(MAX_ROUNDS + 1, dtype=i32, device=dev)
        self.info = torch.zeros(3, dtype=torch.int64, device=dev)
        nb = ctx.step_workspace_size(n, n_cells, capacity)
        self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        p = lambda t: t.data_ptr()
        self.desc = StepBuffers(n, n_cells, capacity, p(self.cell_id), p(self.vx), p(self.vy),
                                p(self.vz), p(self.perm), p(self.cell_start), p(self.svx), p(self.svy),
                                p(self.svz), p(self.mom), p(self.sigma_g_max), p(self.pairs),
                                p(self.round_offsets), p(self.info), p(self.ws), nb, p(self.deps))

    @property
    def sel(self):
        return dict(pairs=self.pairs, deps=self.deps, round_offsets=self.round_offsets, info=self.info)

    def info_host(self):
        i = self.info.cpu()
        return dict(n_pairs=int(i[0]), n_candidates=int(i[1]), n_rounds=int(i[2] & 0xFFFFFFFF))


def make_path(kind: int, pot: Potential | None = None, n_nodes: int = 32, mlp: Mlp | None = None,
              w_bits: torch.Tensor | None = None, bias: torch.Tensor | None = None,
              table: "ChiTable | None" = None) -> Path:
    P = Path()
    P.path = kind
    P.n_nodes = n_nodes
    P.pot = C.pointer(pot) if pot is not None else C.POINTER(Potential)()
    P.mlp = C.pointer(mlp) if mlp is not None else C.POINTER(Mlp)()
    P.weights_bf16 = w_bits.data_ptr() if w_bits is not None else None
    P.biases = bias.data_ptr() if bias is not None else None
    P.table = C.pointer(table.desc) if table is not None else C.POINTER(ChiTableDesc)()
    P._keep = (pot, mlp, w_bits, bias, table)
    return P


class NeuralCollisionOperator(torch.autograd.Function):
    """The neural collision operator on a batch of pairs in pseudo-cells of 16
    (MLP, shell projection, centre-of-mass update, moment matching) as a
    differentiable function of the FP32 parameters theta.  Forward and the
    hand-written backward both run in the library (dsmc_neural_operator_*);
    this class only hands tensors across."""

    @staticmethod
    def forward(ctx, theta, vi, vj, T, context, mlp, seed, t):
        vin, vjn = context.neural_operator_forward(mlp, theta, seed, t, vi, vj, T)
        ctx.save_for_backward(theta, vi, vj, T)
        ctx.args = (context, mlp, seed, t)
        return vin, vjn

    @staticmethod
    def backward(ctx, g_vi, g_vj):
        theta, vi, vj, T = ctx.saved_tensors
        context, mlp, seed, t = ctx.args
        if g_vi is None:
            g_vi = torch.zeros_like(vi)
        if g_vj is None:
            g_vj = torch.zeros_like(vj)
        grad = context.neural_operator_backward(mlp, theta, seed, t, vi, vj, T,
                                                g_vi.contiguous().to(torch.float64),
                                                g_vj.contiguous().to(torch.float64))
        return grad, None, None, None, None, None, None, None
