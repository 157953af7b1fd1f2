"""Python binding of the SAFR C ABI (include/safr.h).

Argument marshalling only: every step of the reconstruction runs in the CUDA
kernels of libsafr.so.  The functions keep the C names; device buffers are
torch CUDA tensors (or raw integer device pointers), streams are torch
streams (or raw cudaStream_t integers).  There is no fallback: if the library
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SAFR_OK = 0
SAFR_ERR_INVALID_ARG = 1
SAFR_ERR_UNSUPPORTED_SIZE = 2
SAFR_ERR_MISALIGNED = 3
SAFR_ERR_NOT_PRECOMPUTED = 4
SAFR_ERR_OOM = 5
SAFR_ERR_CUDA = 6
SAFR_ERR_TIMEOUT = 7
SAFR_ERR_DEVICE = 8
SAFR_ERR_IO = 9

SAFR_NGS, SAFR_LGS = 0, 1
SAFR_FP32, SAFR_FP16_STORAGE, SAFR_FP64 = 0, 1, 2
SAFR_NATIVE, SAFR_METRIC = 0, 1
SAFR_WARN_CONTAINMENT = 1
SAFR_PATH_AUTO, SAFR_PATH_FUSED, SAFR_PATH_PASSES, SAFR_PATH_CLUSTER = 0, 1, 2, 3

_PRECISION = {"fp32": SAFR_FP32, "fp16": SAFR_FP16_STORAGE, "fp64": SAFR_FP64}
_EXPORTS = ["safr_plan_create", "safr_precompute", "safr_reconstruct", "safr_reconstruct_host",
            "safr_get_status", "safr_get_plan_info", "safr_copy_B", "safr_trace", "safr_trace_read",
            "safr_launches_per_frame", "safr_trace_phases", "safr_set_path", "safr_get_path", "safr_debug_skip_barrier",
            "safr_destroy", "safr_status_string", "safr_reconstruct_noalloc", "safr_autotune",
            "safr_batch_create", "safr_batch_reconstruct", "safr_batch_get_status", "safr_batch_launches",
            "safr_batch_destroy", "safr_batch_graph", "safr_filter_train", "safr_filter_apply",
            "safr_filter_reset", "safr_polc", "safr_integrate", "safr_loop_step", "safr_refresh",
            "safr_plan_save", "safr_plan_load", "safr_trace_stamps", "safr_set_grid", "safr_get_grid",
            "safr_batch_chains", "safr_set_tile_rows", "safr_batch_set_chains", "safr_reconstruct_frames"]
SAFR_NOALLOC_SCRATCH_BYTES = 8 << 20
SAFR_FILTER_PARAMS = 8705


class SafrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {safr_status_string(status)}")


class safr_geometry(C.Structure):
    _fields_ = [("M", C.c_int), ("P", C.c_int), ("pitch_m", C.c_double), ("diameter_m", C.c_double),
                ("obstruction", C.c_double), ("L", C.c_int), ("h_m", C.POINTER(C.c_double)),
                ("cn2", C.POINTER(C.c_double)), ("G", C.c_int), ("dir_x", C.POINTER(C.c_double)),
                ("dir_y", C.POINTER(C.c_double)), ("kind", C.POINTER(C.c_int)), ("h_lgs_m", C.c_double),
                ("alpha", C.c_double), ("alpha_tt", C.c_double), ("beta", C.c_double),
                ("precision", C.c_int), ("output_grid", C.c_int), ("remove_tt", C.c_int)]


class safr_plan_info(C.Structure):
    _fields_ = [("M", C.c_int), ("P", C.c_int), ("L", C.c_int), ("G", C.c_int), ("ngroups", C.c_int),
                ("group_kind", C.c_int * 2), ("group_G", C.c_int * 2), ("b_bytes", C.c_size_t),
                ("workspace_bytes", C.c_size_t), ("in_bytes", C.c_size_t), ("out_bytes", C.c_size_t),
                ("warnings", C.c_int), ("precomputed", C.c_int), ("path", C.c_int), ("tile_rows", C.c_int),
                ("autotuned", C.c_int)]


class safr_update(C.Structure):
    _fields_ = [("cn2", C.POINTER(C.c_double)), ("dir_x", C.POINTER(C.c_double)), ("dir_y", C.POINTER(C.c_double)),
                ("alpha", C.c_double), ("alpha_tt", C.c_double)]


class safr_filter_config(C.Structure):
    _fields_ = [("r0", C.c_double), ("L0", C.c_double), ("noise_level", C.c_double), ("train_frames", C.c_int),
                ("valid_frames", C.c_int), ("epochs", C.c_int), ("lr", C.c_double), ("seed", C.c_ulonglong)]


class safr_filter_result(C.Structure):
    _fields_ = [("train_loss_first", C.c_double), ("train_loss_last", C.c_double),
                ("valid_loss_learned", C.c_double), ("valid_loss_plain", C.c_double), ("steps", C.c_long),
                ("used_learned", C.c_int), ("nonfinite", C.c_int)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsafr.so (building it first if needed and possible)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build_library()
    if not os.path.exists(path):
        raise OSError(f"libsafr.so is not built ({path}); run paper_2510_19542_gb300/build.py")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.safr_plan_create.argtypes = [C.POINTER(safr_geometry), C.c_int, C.POINTER(vp)]
    lib.safr_precompute.argtypes = [vp, vp]
    lib.safr_reconstruct.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.safr_reconstruct_host.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.safr_reconstruct_frames.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp]
    lib.safr_get_status.argtypes = [vp]
    lib.safr_get_plan_info.argtypes = [vp, C.POINTER(safr_plan_info)]
    lib.safr_copy_B.argtypes = [vp, C.c_int, vp]
    lib.safr_trace.argtypes = [vp, C.c_int]
    lib.safr_trace_read.argtypes = [vp, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)]
    lib.safr_launches_per_frame.argtypes = [vp]
    lib.safr_trace_phases.argtypes = [vp, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int)]
    lib.safr_trace_stamps.argtypes = [vp, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int)]
    lib.safr_set_path.argtypes = [vp, C.c_int]
    lib.safr_get_path.argtypes = [vp]
    lib.safr_set_grid.argtypes = [vp, C.c_int]
    lib.safr_get_grid.argtypes = [vp]
    lib.safr_set_tile_rows.argtypes = [vp, C.c_int]
    lib.safr_debug_skip_barrier.argtypes = [vp, C.c_int, C.c_double]
    lib.safr_destroy.argtypes = [vp]
    lib.safr_reconstruct_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, vp]
    lib.safr_autotune.argtypes = [vp, vp]
    lib.safr_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp)]
    lib.safr_batch_reconstruct.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), vp]
    lib.safr_batch_get_status.argtypes = [vp]
    lib.safr_batch_launches.argtypes = [vp]
    lib.safr_batch_graph.argtypes = [vp]
    lib.safr_batch_chains.argtypes = [vp]
    lib.safr_batch_set_chains.argtypes = [vp, C.c_int]
    lib.safr_batch_destroy.argtypes = [vp]
    lib.safr_filter_train.argtypes = [vp, C.POINTER(safr_filter_config), C.POINTER(C.c_float),
                                      C.POINTER(safr_filter_result), vp]
    lib.safr_filter_apply.argtypes = [vp, C.POINTER(C.c_float), C.c_double, vp]
    lib.safr_filter_reset.argtypes = [vp, vp]
    lib.safr_refresh.argtypes = [vp, C.POINTER(safr_update), vp]
    lib.safr_plan_save.argtypes = [vp, C.c_char_p]
    lib.safr_plan_load.argtypes = [C.c_char_p, C.c_int, C.POINTER(vp)]
    lib.safr_polc.argtypes = [vp, vp, vp, vp, vp]
    lib.safr_integrate.argtypes = [vp, vp, vp, C.c_double, vp]
    lib.safr_loop_step.argtypes = [vp, vp, vp, C.c_double, vp]
    lib.safr_status_string.argtypes = [C.c_int]
    lib.safr_status_string.restype = C.c_char_p
    for name in _EXPORTS:
        if name not in ("safr_status_string",):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != SAFR_OK:
        raise SafrError(status, where)


def _ptr(x):
    """Device or host pointer of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s):
    if s is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:  # noqa: BLE001 - no torch / no CUDA: the legacy default stream
            return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def safr_status_string(status: int) -> str:
    return load().safr_status_string(int(status)).decode()


def make_geometry(geom: dict):
    """safr_geometry from a dict (keys of synth.config); returns (struct, keepalive)."""
    h = np.ascontiguousarray(geom["h"], np.float64)
    cn2 = np.ascontiguousarray(geom["cn2"], np.float64)
    dx = np.ascontiguousarray(geom["dir_x"], np.float64)
    dy = np.ascontiguousarray(geom["dir_y"], np.float64)
    kind = np.ascontiguousarray(geom["kind"], np.int32)
    prec = geom.get("precision", "fp32")
    prec = _PRECISION[prec] if isinstance(prec, str) else int(prec)
    dp = C.POINTER(C.c_double)
    g = safr_geometry(
        M=int(geom["M"]), P=int(geom["P"]), pitch_m=float(geom["pitch"]),
        diameter_m=float(geom.get("diameter", 0.0)), obstruction=float(geom.get("obstruction", 0.0)),
        L=len(h), h_m=h.ctypes.data_as(dp), cn2=cn2.ctypes.data_as(dp), G=len(dx),
        dir_x=dx.ctypes.data_as(dp), dir_y=dy.ctypes.data_as(dp),
        kind=kind.ctypes.data_as(C.POINTER(C.c_int)), h_lgs_m=float(geom.get("h_lgs", 90e3)),
        alpha=float(geom["alpha"]), alpha_tt=float(geom.get("alpha_tt", geom["alpha"])),
        beta=float(geom["beta"]), precision=prec,
        output_grid=SAFR_METRIC if int(geom.get("output_metric", 1)) else SAFR_NATIVE,
        remove_tt=int(geom.get("remove_tt", 1)))
    return g, (h, cn2, dx, dy, kind)


def safr_plan_create(geom: dict, cuda_device: int = 0) -> int:
    g, keep = make_geometry(geom)
    out = C.c_void_p()
    _check(load().safr_plan_create(C.byref(g), int(cuda_device), C.byref(out)), "safr_plan_create")
    del keep
    return out.value


def safr_precompute(plan: int, stream=None):
    _check(load().safr_precompute(plan, _stream(stream)), "safr_precompute")


def safr_reconstruct(plan: int, wavefronts, layers, in_scales=None, out_scales=None, stream=None):
    _check(load().safr_reconstruct(plan, _ptr(wavefronts), _ptr(in_scales), _ptr(layers), _ptr(out_scales),
                                   _stream(stream)), "safr_reconstruct")


def safr_reconstruct_frames(plan: int, n: int, wavefronts, layers, in_scales=None, out_scales=None, stream=None):
    """n frames of one plan; contiguous [n][G][P][P] wavefronts, [n][L][M][M] layers."""
    _check(load().safr_reconstruct_frames(plan, int(n), _ptr(wavefronts), _ptr(in_scales), _ptr(layers),
                                          _ptr(out_scales), _stream(stream)), "safr_reconstruct_frames")


def safr_reconstruct_host(plan: int, wavefronts, layers, in_scales=None, out_scales=None, stream=None):
    _check(load().safr_reconstruct_host(plan, _ptr(wavefronts), _ptr(in_scales), _ptr(layers),
                                        _ptr(out_scales), _stream(stream)), "safr_reconstruct_host")


def safr_get_status(plan: int) -> int:
    return load().safr_get_status(plan)


def safr_get_plan_info(plan: int) -> dict:
    info = safr_plan_info()
    _check(load().safr_get_plan_info(plan, C.byref(info)), "safr_get_plan_info")
    return {k: (list(getattr(info, k)) if k in ("group_kind", "group_G") else getattr(info, k))
            for k, _ in safr_plan_info._fields_}


def safr_copy_B(plan: int, group: int) -> np.ndarray:
    """B of one group as complex128 [M/2][L][G_group][M] (k, l, g, j)."""
    info = safr_get_plan_info(plan)
    M, L, Gg = info["M"], info["L"], info["group_G"][group]
    out = np.empty((M // 2, L, Gg, M, 2), np.float64)
    _check(load().safr_copy_B(plan, int(group), out.ctypes.data), "safr_copy_B")
    return out[..., 0] + 1j * out[..., 1]


def safr_trace(plan: int, enable: bool = True):
    _check(load().safr_trace(plan, int(bool(enable))), "safr_trace")


def safr_trace_read(plan: int):
    ms = (C.c_float * 8)()
    n = C.c_int(0)
    _check(load().safr_trace_read(plan, ms, 8, C.byref(n)), "safr_trace_read")
    return [ms[i] for i in range(n.value)]


def safr_trace_phases(plan: int):
    """Phase completion times (us) of the last traced persistent-kernel or one-cluster frame."""
    us = (C.c_double * 32)()
    n = C.c_int(0)
    _check(load().safr_trace_phases(plan, us, 32, C.byref(n)), "safr_trace_phases")
    if safr_get_path(plan) == SAFR_PATH_CLUSTER:
        keys = ["start", "prologue", "p1_data_in", "p1_done", "bar1_out", "p2_star_fft", "p2_B_landed",
                "p2_first_column", "p2_done", "bar2_out", "p3_first_round", "p3_done", "end", "copies_issued",
                "unused", "p3_first_stored"]
    else:
        keys = ["start", "prologue", "p1_data_in", "p1_B_issued", "p1_fft", "p1_done", "bar1_arrive", "bar1_out",
                "p2_star_fft", "p2_synced", "p2_B_landed", "p2_apply", "p2_inv_fft", "p2_stored", "p2_done",
                "bar2_arrive", "bar2_out", "p3_tables", "p3_staged", "p3_fft", "p3_synced", "p3_first_stored",
                "p3_done"]
    return dict(zip(keys, [us[i] for i in range(min(n.value, len(keys)))]))


def safr_set_grid(plan: int, ctas: int):
    """CTAs of the persistent kernel (0: one per SM)."""
    _check(load().safr_set_grid(plan, int(ctas)), "safr_set_grid")


def safr_get_grid(plan: int) -> int:
    return load().safr_get_grid(plan)


def safr_set_tile_rows(plan: int, rows: int):
    """Output rows per phase-3 item of the persistent kernel (0: the cost model's choice)."""
    _check(load().safr_set_tile_rows(plan, int(rows)), "safr_set_tile_rows")


def safr_trace_stamps(plan: int) -> np.ndarray:
    """Per-CTA phase marks (us) of the last traced persistent-kernel frame, [n_cta][23]."""
    cap = 4096 * 23
    us = np.zeros(cap, np.float64)
    n = C.c_int(0)
    _check(load().safr_trace_stamps(plan, us.ctypes.data_as(C.POINTER(C.c_double)), cap, C.byref(n)),
           "safr_trace_stamps")
    return us[:n.value * 23].reshape(n.value, 23)


def safr_launches_per_frame(plan: int) -> int:
    return load().safr_launches_per_frame(plan)


def safr_set_path(plan: int, path: int):
    _check(load().safr_set_path(plan, int(path)), "safr_set_path")


def safr_get_path(plan: int) -> int:
    return load().safr_get_path(plan)


def safr_debug_skip_barrier(plan: int, cta: int, timeout_s: float = 0.0):
    _check(load().safr_debug_skip_barrier(plan, int(cta), float(timeout_s)), "safr_debug_skip_barrier")


def safr_reconstruct_noalloc(cuda_device: int, M: int, P: int, L: int, G: int, B, wavefronts, layers, status,
                             stream=None):
    """Plan-free FP32 frame of one star group with caller-owned buffers and no
    device allocation (scratch in the library's static device array)."""
    _check(load().safr_reconstruct_noalloc(int(cuda_device), int(M), int(P), int(L), int(G), _ptr(B),
                                           _ptr(wavefronts), _ptr(layers), _ptr(status), _stream(stream)),
           "safr_reconstruct_noalloc")


def safr_autotune(plan: int, stream=None):
    _check(load().safr_autotune(plan, _stream(stream)), "safr_autotune")


def safr_filter_train(plan: int, r0: float, L0: float, noise_level: float, train_frames: int, valid_frames: int,
                      epochs: int, lr: float = 2e-3, seed: int = 5, stream=None):
    """Train the learned spectral filter on the GPU; returns (weights [SAFR_FILTER_PARAMS]
    float32, rounded to BF16, and the result fields as a dict)."""
    cfg = safr_filter_config(float(r0), float(L0), float(noise_level), int(train_frames), int(valid_frames),
                             int(epochs), float(lr), int(seed))
    w = np.zeros(SAFR_FILTER_PARAMS, np.float32)
    res = safr_filter_result()
    _check(load().safr_filter_train(plan, C.byref(cfg), w.ctypes.data_as(C.POINTER(C.c_float)), C.byref(res),
                                    _stream(stream)), "safr_filter_train")
    return w, {name: getattr(res, name) for name, _ in safr_filter_result._fields_}


def safr_filter_apply(plan: int, weights, noise_level: float, stream=None):
    """B from the given MLP parameters (host float32 array of SAFR_FILTER_PARAMS)."""
    w = np.ascontiguousarray(weights, np.float32)
    if w.size != SAFR_FILTER_PARAMS:
        raise ValueError(f"expected {SAFR_FILTER_PARAMS} parameters, got {w.size}")
    _check(load().safr_filter_apply(plan, w.ctypes.data_as(C.POINTER(C.c_float)), float(noise_level),
                                    _stream(stream)), "safr_filter_apply")


def safr_filter_reset(plan: int, stream=None):
    _check(load().safr_filter_reset(plan, _stream(stream)), "safr_filter_reset")


def safr_polc(plan: int, wavefronts, a, out, stream=None):
    """Pseudo open loop data: out = mask * (wavefronts + A(a)) (device buffers)."""
    _check(load().safr_polc(plan, _ptr(wavefronts), _ptr(a), _ptr(out), _stream(stream)), "safr_polc")


def safr_integrate(plan: int, layers, a, gain: float, stream=None):
    """Integrator: a <- (1 - gain) a + gain layers (device buffers, in place on a)."""
    _check(load().safr_integrate(plan, _ptr(layers), _ptr(a), float(gain), _stream(stream)), "safr_integrate")


def safr_loop_step(plan: int, wavefronts, a, gain: float, stream=None):
    """POLC, SAFR and the integrator in one call; a is updated in place."""
    _check(load().safr_loop_step(plan, _ptr(wavefronts), _ptr(a), float(gain), _stream(stream)), "safr_loop_step")


def safr_refresh(plan: int, cn2=None, dir_x=None, dir_y=None, alpha: float = 0.0, alpha_tt: float = 0.0,
                 stream=None):
    """New layer weights, star directions or alphas; B recomputed in place on the stream."""
    keep = []

    def arr(x):
        if x is None:
            return None
        a = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_double))

    u = safr_update(arr(cn2), arr(dir_x), arr(dir_y), float(alpha), float(alpha_tt))
    _check(load().safr_refresh(plan, C.byref(u), _stream(stream)), "safr_refresh")


def safr_plan_save(plan: int, path: str):
    _check(load().safr_plan_save(plan, os.fsencode(path)), "safr_plan_save")


def safr_plan_load(path: str, cuda_device: int = 0) -> int:
    out = C.c_void_p()
    _check(load().safr_plan_load(os.fsencode(path), int(cuda_device), C.byref(out)), "safr_plan_load")
    return out.value


def _ptr_array(xs):
    if xs is None:
        return None
    arr = (C.c_void_p * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = _ptr(x)
    return arr


def safr_batch_create(plans) -> int:
    """Batch over plan handles (ints); returns the batch handle."""
    arr = (C.c_void_p * len(plans))(*plans)
    out = C.c_void_p()
    _check(load().safr_batch_create(arr, len(plans), C.byref(out)), "safr_batch_create")
    return out.value


def safr_batch_reconstruct(batch: int, wavefronts, layers, in_scales=None, out_scales=None, stream=None):
    """Lists of per-frame device buffers (tensors or pointers)."""
    _check(load().safr_batch_reconstruct(batch, _ptr_array(wavefronts), _ptr_array(in_scales), _ptr_array(layers),
                                         _ptr_array(out_scales), _stream(stream)), "safr_batch_reconstruct")


def safr_batch_get_status(batch: int) -> int:
    return load().safr_batch_get_status(batch)


def safr_batch_chains(batch: int) -> int:
    return load().safr_batch_chains(batch)


def safr_batch_launches(batch: int) -> int:
    return load().safr_batch_launches(batch)


def safr_batch_graph(batch: int) -> int:
    return load().safr_batch_graph(batch)


def safr_batch_set_chains(batch: int, chains: int):
    """Force the batch graph's chain count (1, 2, 4, 8), or 0 to time it again."""
    _check(load().safr_batch_set_chains(batch, int(chains)), "safr_batch_set_chains")


def safr_batch_destroy(batch: int):
    _check(load().safr_batch_destroy(batch), "safr_batch_destroy")


def safr_destroy(plan: int):
    _check(load().safr_destroy(plan), "safr_destroy")


class Plan:
    """Owning wrapper: create, precompute, reconstruct with torch tensors."""

    def __init__(self, geom: dict, device: int = 0, precompute: bool = True, stream=None, path: int | None = None):
        self.geom = dict(geom)
        self.handle = safr_plan_create(geom, device)
        self.device = device
        self.info = safr_get_plan_info(self.handle)
        if path is not None:
            safr_set_path(self.handle, path)
        if precompute:
            safr_precompute(self.handle, stream)
            self.info["precomputed"] = 1

    @classmethod
    def load(cls, path: str, device: int = 0):
        """A plan from a file written by safr_plan_save (B uploaded, not recomputed)."""
        with open(path, "rb") as f:
            head = f.read(12 + 8 * 4)
        precision = int(np.frombuffer(head[12:], dtype="<i4")[4])
        self = cls.__new__(cls)
        self.handle = safr_plan_load(path, device)
        self.device = device
        self.info = safr_get_plan_info(self.handle)
        self.geom = {"precision": {SAFR_FP32: "fp32", SAFR_FP16_STORAGE: "fp16", SAFR_FP64: "fp64"}[precision]}
        return self

    def close(self):
        if getattr(self, "handle", None):
            safr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    @property
    def io_dtype(self):
        import torch
        return {"fp32": torch.float32, "fp16": torch.float16, "fp64": torch.float64}[
            self.geom.get("precision", "fp32")]

    def empty_layers(self):
        import torch
        return torch.empty((self.info["L"], self.info["M"], self.info["M"]), dtype=self.io_dtype,
                           device=f"cuda:{self.device}")

    def reconstruct(self, wavefronts, layers=None, in_scales=None, out_scales=None, stream=None):
        import torch
        if layers is None:
            layers = self.empty_layers()
        if self.geom.get("precision") == "fp16" and out_scales is None:
            out_scales = torch.empty(self.info["L"], dtype=torch.float32, device=layers.device)
        safr_reconstruct(self.handle, wavefronts, layers, in_scales, out_scales, stream)
        return (layers, out_scales) if out_scales is not None else layers
