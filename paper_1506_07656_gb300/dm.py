"""Python binding of the C ABI in ``include/dm.h`` (ctypes; argument marshalling only).

Every step of the method runs in the CUDA library ``libdm.so``; this module
only converts torch tensors to pointers and sizes.  PyTorch provides device
memory and streams.  If the library is missing or fails to load, every call
raises -- there is no CPU fallback.

Names follow the C ABI: dm_create, dm_descriptors, dm_correlate_pyramid,
dm_backtrack, dm_match, dm_match_host, ...; ``Context`` bundles them.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdm.so")

DM_OK, DM_EINVAL, DM_ENOMEM, DM_ECUDA, DM_ETIMEOUT, DM_EUNSUPPORTED, DM_EOVERFLOW = range(7)
DM_FP32, DM_BF16, DM_FP8_E4M3 = 0, 1, 2
DM_DEV_FRONTIER_OVERFLOW, DM_DEV_OUTPUT_OVERFLOW, DM_DEV_TIMEOUT = 1, 2, 4
STATUS_NAMES = {0: "DM_OK", 1: "DM_EINVAL", 2: "DM_ENOMEM", 3: "DM_ECUDA", 4: "DM_ETIMEOUT",
                5: "DM_EUNSUPPORTED", 6: "DM_EOVERFLOW"}
MAXL = 30


class DmConfig(C.Structure):
    _fields_ = [("nu1", C.c_float), ("nu2", C.c_float), ("nu3", C.c_float), ("slope", C.c_float),
                ("mu", C.c_float), ("lambda_", C.c_float), ("image_scale", C.c_float), ("precision", C.c_int),
                ("compensated", C.c_int)]


class DmMatch(C.Structure):
    _fields_ = [("x1", C.c_float), ("y1", C.c_float), ("x2", C.c_float), ("y2", C.c_float), ("score", C.c_float)]


MATCH_BYTES = C.sizeof(DmMatch)


class DmPair(C.Structure):
    _fields_ = [("d_img1", C.c_void_p), ("W1", C.c_int), ("H1", C.c_int), ("d_img2", C.c_void_p), ("W2", C.c_int),
                ("H2", C.c_int), ("d_out", C.c_void_p), ("capacity", C.c_int), ("d_count", C.c_void_p)]

class DmPairHost(C.Structure):
    _fields_ = [("h_img1", C.c_void_p), ("W1", C.c_int), ("H1", C.c_int), ("h_img2", C.c_void_p),
                ("W2", C.c_int), ("H2", C.c_int), ("h_out", C.c_void_p), ("capacity", C.c_int), ("h_count", C.c_void_p)]


class DmFlowParams(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("sigma", "eta", "gamma", "delta", "beta", "b", "kappa", "zeta", "eps",
                                          "sigma_m", "omega", "image_scale")] + \
               [(k, C.c_int) for k in ("n_fixed", "n_sor", "min_size")]


# Exported symbols and their signatures (restype dm_status = c_int unless noted).
_SIGS = {
    "dm_config_default": (None, [C.POINTER(DmConfig)]),
    "dm_create": (C.c_int, [C.POINTER(DmConfig), C.c_int, C.POINTER(C.c_void_p)]),
    "dm_destroy": (C.c_int, [C.c_void_p]),
    "dm_last_error": (C.c_char_p, [C.c_void_p]),
    "dm_geometry": (C.c_int, [C.c_int] * 4 + [C.POINTER(C.c_int)] * 3 + [C.c_void_p, C.c_void_p]),
    "dm_workspace_bytes": (C.c_int, [C.c_void_p] + [C.c_int] * 4 + [C.POINTER(C.c_size_t)] * 4),
    "dm_descriptors": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_size_t,
                                 C.c_void_p]),
    "dm_correlate_pyramid": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                       C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p), C.c_void_p]),
    "dm_pyramid_level": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_void_p), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "dm_pyramid_free": (C.c_int, [C.c_void_p]),
    "dm_backtrack": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_int, C.c_void_p,
                               C.c_void_p]),
    "dm_match": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                           C.c_size_t, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "dm_match_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                C.c_size_t, C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_void_p]),
    "dm_read_status": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.c_void_p, C.c_int, C.c_void_p]),
    "dm_inject_fault": (C.c_int, [C.c_void_p, C.c_int, C.c_longlong]),
    "dm_grad_workspace_bytes": (C.c_int, [C.c_void_p] + [C.c_int] * 4 + [C.POINTER(C.c_size_t)]),
    "dm_loss_grad": (C.c_int, [C.c_void_p] * 5 + [C.c_size_t] + [C.c_void_p] * 5),
    "dm_batch_workspace_bytes": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_size_t)]),
    "dm_match_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "dm_set_batch_lanes": (C.c_int, [C.c_void_p, C.c_int]),
    "dm_set_merge_keys": (C.c_int, [C.c_void_p, C.c_int]),
    "dm_set_batch_wave": (C.c_int, [C.c_void_p, C.c_int]),
    "dm_autotune_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_int),
                                    C.c_void_p]),
    "dm_batch_host_workspace_bytes": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_size_t)]),
    "dm_match_batch_host": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "dm_backtrack_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "dm_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                              C.c_size_t, C.POINTER(C.c_int), C.c_void_p]),
    "dm_tuned_config": (C.c_int, [C.c_void_p] + [C.c_int] * 4 + [C.POINTER(C.c_int)]),
    "dm_set_tuned_config": (C.c_int, [C.c_void_p] + [C.c_int] * 4 + [C.POINTER(C.c_int)]),
    "dm_timing_start": (C.c_int, [C.c_void_p, C.c_int]),
    "dm_timing_read": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    "dm_prototypes_workspace_bytes": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "dm_prototypes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "dm_correlate_pyramid_approx": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                              C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t,
                                              C.POINTER(C.c_void_p), C.c_void_p]),
    "dm_flow_params_default": (None, [C.POINTER(DmFlowParams)]),
    "dm_deepflow_workspace_bytes": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(DmFlowParams),
                                              C.POINTER(C.c_size_t)]),
    "dm_deepflow": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                              C.POINTER(DmFlowParams), C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "dm_star_workspace_bytes": (C.c_int, [C.c_void_p] + [C.c_int] * 4 + [C.POINTER(C.c_size_t)] * 2),
    "dm_backtrack_star": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_int, C.c_void_p,
                                    C.c_void_p]),
    "dm_match_star": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                C.c_size_t, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "dm_invariant_workspace_bytes": (C.c_int, [C.c_void_p] + [C.c_int] * 4 + [C.POINTER(C.c_size_t)]),
    "dm_match_invariant": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                     C.c_void_p, C.c_size_t, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
}
NSTAGES = 4
STAGES = ("descriptors", "level0_correlation", "levels", "backtracking")

_LIB = None


def load(build_if_missing: bool = True):
    """Load libdm.so (building it with nvcc first if absent); raise if impossible."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing; run paper_1506_07656_gb300.build.build()")
        from . import build as _b
        _b.build()
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class DmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(ctx, st: int, what: str):
    if st != DM_OK:
        msg = load().dm_last_error(ctx).decode() if ctx else ""
        raise DmError(st, f"{what}: {msg}")


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _dptr(t) -> int:
    return int(t.data_ptr())


# ------------------------------------------------------------------------- #
# Thin wrappers with the C names                                             #
# ------------------------------------------------------------------------- #
def dm_config_default() -> DmConfig:
    cfg = DmConfig()
    load().dm_config_default(C.byref(cfg))
    return cfg


def dm_create(cfg: DmConfig | None = None, device: int = 0) -> int:
    h = C.c_void_p()
    st = load().dm_create(C.byref(cfg) if cfg is not None else None, device, C.byref(h))
    if st != DM_OK:
        raise DmError(st, "dm_create")
    return h.value


def dm_destroy(ctx: int) -> None:
    load().dm_destroy(ctx)


def dm_geometry(W1, H1, W2, H2):
    L, n0, n = C.c_int(), C.c_int(), C.c_int()
    dw = (C.c_int * (MAXL + 2))()
    dh = (C.c_int * (MAXL + 2))()
    st = load().dm_geometry(W1, H1, W2, H2, C.byref(L), C.byref(n0), C.byref(n), dw, dh)
    if st != DM_OK:
        raise DmError(st, f"dm_geometry {W1}x{H1}/{W2}x{H2}")
    return dict(L=L.value, n_patch0=n0.value, n_patch=n.value, dw=list(dw[:L.value + 2]), dh=list(dh[:L.value + 2]))


def dm_workspace_bytes(ctx, W1, H1, W2, H2):
    a, b, c, d = C.c_size_t(), C.c_size_t(), C.c_size_t(), C.c_size_t()
    st = load().dm_workspace_bytes(ctx, W1, H1, W2, H2, C.byref(a), C.byref(b), C.byref(c), C.byref(d))
    _check(ctx, st, "dm_workspace_bytes")
    return dict(desc=a.value, pyramid=b.value, backtrack=c.value, match=d.value)


def dm_descriptors(ctx, d_img, d_desc, d_tmp, stream=None):
    H, W = d_img.shape
    st = load().dm_descriptors(ctx, _dptr(d_img), W, H, _dptr(d_desc), _dptr(d_tmp), d_tmp.numel() * d_tmp.element_size(),
                               _stream_ptr(stream))
    _check(ctx, st, "dm_descriptors")


def dm_correlate_pyramid(ctx, d_desc1, d_desc2, d_ws, stream=None) -> int:
    H1, W1, _ = d_desc1.shape
    H2, W2, _ = d_desc2.shape
    h = C.c_void_p()
    st = load().dm_correlate_pyramid(ctx, _dptr(d_desc1), W1, H1, _dptr(d_desc2), W2, H2, _dptr(d_ws),
                                     d_ws.numel() * d_ws.element_size(), C.byref(h), _stream_ptr(stream))
    _check(ctx, st, "dm_correlate_pyramid")
    return h.value


def dm_prototypes_workspace_bytes(ctx, W1, H1, D) -> int:
    n = C.c_size_t()
    _check(ctx, load().dm_prototypes_workspace_bytes(ctx, W1, H1, D, C.byref(n)), "dm_prototypes_workspace_bytes")
    return n.value


def dm_prototypes(ctx, d_desc1, D, iters, d_protos, d_assign, d_ws, init=None, stream=None):
    """Approximate form (Sec. 4.1): the D-prototype dictionary of image 1's
    atomic patches (spherical k-means) into d_protos [D][144] and the
    prototype of every atomic patch into d_assign [P0] (int32).  `init`: D
    patch indices (a host sequence) or None for evenly spaced patches."""
    H1, W1, _ = d_desc1.shape
    h_init = None
    if init is not None:
        arr = (C.c_int * D)(*[int(v) for v in init])
        h_init = C.cast(arr, C.c_void_p)
    st = load().dm_prototypes(ctx, _dptr(d_desc1), W1, H1, D, iters, h_init, _dptr(d_protos), _dptr(d_assign),
                              _dptr(d_ws), d_ws.numel() * d_ws.element_size(), _stream_ptr(stream))
    _check(ctx, st, "dm_prototypes")


def dm_correlate_pyramid_approx(ctx, d_protos, d_assign, W1, H1, d_desc2, d_ws, stream=None) -> int:
    """Approximate form (Sec. 4.1): the pyramid with every atomic patch of
    image 1 replaced by its prototype (level 0 computed once per prototype)."""
    D = d_protos.shape[0]
    H2, W2, _ = d_desc2.shape
    h = C.c_void_p()
    st = load().dm_correlate_pyramid_approx(ctx, _dptr(d_protos), D, _dptr(d_assign), W1, H1, _dptr(d_desc2), W2, H2,
                                            _dptr(d_ws), d_ws.numel() * d_ws.element_size(), C.byref(h),
                                            _stream_ptr(stream))
    _check(ctx, st, "dm_correlate_pyramid_approx")
    return h.value


def dm_pyramid_level(pyr: int, level: int):
    vals, am, valid = C.c_void_p(), C.c_void_p(), C.c_void_p()
    n, mw, mh, pitch = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    st = load().dm_pyramid_level(pyr, level, C.byref(vals), C.byref(am), C.byref(valid), C.byref(n), C.byref(mw),
                                 C.byref(mh), C.byref(pitch))
    if st != DM_OK:
        raise DmError(st, "dm_pyramid_level")
    return dict(vals=vals.value, argmax=am.value, valid=valid.value, n=n.value, mw=mw.value, mh=mh.value,
                pitch=pitch.value)


def read_level(ws, info, patches=None):
    """Copy one pyramid level (values, argmax or None, valid) to host numpy arrays,
    padding dropped; `patches` (optional index list) selects patches on the device
    first, for levels too large to copy whole."""
    import torch
    n, mw, mh, pitch = info["n"], info["mw"], info["mh"], info["pitch"]
    base = ws.data_ptr()
    sel = None if patches is None else torch.as_tensor(patches, dtype=torch.long, device=ws.device)
    ov = info["vals"] - base
    v = ws[ov:ov + n * mh * pitch * 4].view(torch.float32).reshape(n, mh, pitch)
    vals = (v if sel is None else v[sel])[:, :, :mw].cpu().numpy()
    am = None
    if info["argmax"]:
        oa = info["argmax"] - base
        a = ws[oa:oa + n * mh * pitch].reshape(n, mh, pitch)
        am = (a if sel is None else a[sel])[:, :, :mw].cpu().numpy()
    ovl = info["valid"] - base
    vv = ws[ovl:ovl + n]
    valid = (vv if sel is None else vv[sel]).cpu().numpy()
    return vals, am, valid


def dm_pyramid_free(pyr: int) -> None:
    load().dm_pyramid_free(pyr)


def dm_backtrack(ctx, pyr, d_ws, d_out, d_count, stream=None):
    cap = d_out.numel() * d_out.element_size() // MATCH_BYTES
    st = load().dm_backtrack(ctx, pyr, _dptr(d_ws), d_ws.numel() * d_ws.element_size(), _dptr(d_out), cap,
                             _dptr(d_count), _stream_ptr(stream))
    _check(ctx, st, "dm_backtrack")


def dm_match(ctx, d_img1, d_img2, d_ws, d_out, d_count, stream=None):
    H1, W1 = d_img1.shape
    H2, W2 = d_img2.shape
    cap = d_out.numel() * d_out.element_size() // MATCH_BYTES
    st = load().dm_match(ctx, _dptr(d_img1), W1, H1, _dptr(d_img2), W2, H2, _dptr(d_ws),
                         d_ws.numel() * d_ws.element_size(), _dptr(d_out), cap, _dptr(d_count), _stream_ptr(stream))
    _check(ctx, st, "dm_match")


def dm_flow_params(**kw) -> DmFlowParams:
    """DeepFlow parameters: the library defaults (the paper's values) with the
    given fields replaced."""
    p = DmFlowParams()
    load().dm_flow_params_default(C.byref(p))
    for k, v in kw.items():
        if k not in dict(DmFlowParams._fields_):
            raise KeyError(f"unknown DeepFlow parameter {k}")
        setattr(p, k, v)
    return p


def dm_deepflow_workspace_bytes(ctx, W, H, capacity, prm: DmFlowParams | None = None) -> int:
    b = C.c_size_t()
    st = load().dm_deepflow_workspace_bytes(ctx, W, H, capacity, C.byref(prm) if prm is not None else None, C.byref(b))
    _check(ctx, st, "dm_deepflow_workspace_bytes")
    return b.value


def dm_deepflow(ctx, d_img1, d_img2, d_matches, d_count, d_u, d_v, d_ws, prm: DmFlowParams | None = None,
                stream=None):
    """d_matches: device float32 tensor [capacity][5] (or None), d_count: device
    int32 [1] (or None); d_u, d_v: device float32 [H][W] outputs."""
    H, W = d_img1.shape
    cap = 0 if d_matches is None else d_matches.numel() * d_matches.element_size() // MATCH_BYTES
    st = load().dm_deepflow(ctx, _dptr(d_img1), _dptr(d_img2), W, H, None if d_matches is None else _dptr(d_matches),
                            None if d_count is None else _dptr(d_count), cap,
                            C.byref(prm) if prm is not None else None, _dptr(d_u), _dptr(d_v), _dptr(d_ws),
                            d_ws.numel() * d_ws.element_size(), _stream_ptr(stream))
    _check(ctx, st, "dm_deepflow")


def dm_star_workspace_bytes(ctx, W1, H1, W2, H2) -> dict:
    b, m = C.c_size_t(), C.c_size_t()
    _check(ctx, load().dm_star_workspace_bytes(ctx, W1, H1, W2, H2, C.byref(b), C.byref(m)), "dm_star_workspace_bytes")
    return {"backtrack": b.value, "match": m.value}


def dm_backtrack_star(ctx, pyr, d_ws, d_out, d_count, stream=None):
    cap = d_out.numel() * d_out.element_size() // MATCH_BYTES
    st = load().dm_backtrack_star(ctx, pyr, _dptr(d_ws), d_ws.numel() * d_ws.element_size(), _dptr(d_out), cap,
                                  _dptr(d_count), _stream_ptr(stream))
    _check(ctx, st, "dm_backtrack_star")


def dm_match_star(ctx, d_img1, d_img2, d_ws, d_out, d_count, stream=None):
    H1, W1 = d_img1.shape
    H2, W2 = d_img2.shape
    cap = d_out.numel() * d_out.element_size() // MATCH_BYTES
    st = load().dm_match_star(ctx, _dptr(d_img1), W1, H1, _dptr(d_img2), W2, H2, _dptr(d_ws),
                              d_ws.numel() * d_ws.element_size(), _dptr(d_out), cap, _dptr(d_count), _stream_ptr(stream))
    _check(ctx, st, "dm_match_star")


def dm_invariant_workspace_bytes(ctx, W1, H1, W2, H2) -> int:
    b = C.c_size_t()
    _check(ctx, load().dm_invariant_workspace_bytes(ctx, W1, H1, W2, H2, C.byref(b)), "dm_invariant_workspace_bytes")
    return b.value


def dm_match_invariant(ctx, d_img1, d_img2, d_ws, d_out, d_count, stream=None):
    H1, W1 = d_img1.shape
    H2, W2 = d_img2.shape
    cap = d_out.numel() * d_out.element_size() // MATCH_BYTES
    st = load().dm_match_invariant(ctx, _dptr(d_img1), W1, H1, _dptr(d_img2), W2, H2, _dptr(d_ws),
                                   d_ws.numel() * d_ws.element_size(), _dptr(d_out), cap, _dptr(d_count),
                                   _stream_ptr(stream))
    _check(ctx, st, "dm_match_invariant")


def dm_match_host(ctx, h_img1, h_img2, d_ws, h_out, stream=None) -> int:
    """h_img*: pinned (or pageable) float32 CPU tensors; h_out: CPU tensor of capacity*5 float32."""
    H1, W1 = h_img1.shape
    H2, W2 = h_img2.shape
    cap = h_out.numel() * h_out.element_size() // MATCH_BYTES
    cnt = C.c_int()
    st = load().dm_match_host(ctx, _dptr(h_img1), W1, H1, _dptr(h_img2), W2, H2, _dptr(d_ws),
                              d_ws.numel() * d_ws.element_size(), _dptr(h_out), cap, C.byref(cnt),
                              _stream_ptr(stream))
    _check(ctx, st, "dm_match_host")
    return cnt.value


def dm_read_status(ctx, d_ws, n_levels: int, stream=None):
    status = C.c_int()
    reached = (C.c_longlong * n_levels)()
    st = load().dm_read_status(ctx, _dptr(d_ws), C.byref(status), reached, n_levels, _stream_ptr(stream))
    _check(ctx, st, "dm_read_status")
    return status.value, list(reached)


DM_FAULT_NONE, DM_FAULT_LAUNCH, DM_FAULT_CAPACITY, DM_FAULT_WAIT, DM_FAULT_ALLOC = 0, 1, 2, 3, 4


def dm_inject_fault(ctx, kind: int, arg: int = 0) -> None:
    """Arm a fault-injection hook (test use): see dm_inject_fault in dm.h.
    ctx may be None for DM_FAULT_ALLOC."""
    _check(ctx, load().dm_inject_fault(ctx, int(kind), int(arg)), "dm_inject_fault")


def dm_grad_workspace_bytes(ctx, W1, H1, W2, H2) -> int:
    b = C.c_size_t()
    _check(ctx, load().dm_grad_workspace_bytes(ctx, W1, H1, W2, H2, C.byref(b)), "dm_grad_workspace_bytes")
    return b.value


def dm_loss_grad(ctx, pyr, d_desc1, d_desc2, d_ws, d_loss, d_parts=None, d_g1=None, d_g2=None, stream=None):
    st = load().dm_loss_grad(ctx, pyr, _dptr(d_desc1), _dptr(d_desc2), _dptr(d_ws), d_ws.numel() * d_ws.element_size(),
                             _dptr(d_loss), _dptr(d_parts) if d_parts is not None else None,
                             _dptr(d_g1) if d_g1 is not None else None, _dptr(d_g2) if d_g2 is not None else None,
                             _stream_ptr(stream))
    _check(ctx, st, "dm_loss_grad")


def make_pairs(items):
    """items: list of (d_img1, d_img2, d_out, d_count) torch tensors -> ctypes array of DmPair."""
    arr = (DmPair * len(items))()
    for k, (i1, i2, out, cnt) in enumerate(items):
        H1, W1 = i1.shape
        H2, W2 = i2.shape
        arr[k] = DmPair(_dptr(i1), W1, H1, _dptr(i2), W2, H2, _dptr(out),
                        out.numel() * out.element_size() // MATCH_BYTES, _dptr(cnt))
    return arr


def dm_batch_workspace_bytes(ctx, pairs) -> int:
    b = C.c_size_t()
    _check(ctx, load().dm_batch_workspace_bytes(ctx, len(pairs), pairs, C.byref(b)), "dm_batch_workspace_bytes")
    return b.value


def dm_match_batch(ctx, pairs, d_ws, stream=None):
    st = load().dm_match_batch(ctx, len(pairs), pairs, _dptr(d_ws), d_ws.numel() * d_ws.element_size(),
                               _stream_ptr(stream))
    _check(ctx, st, "dm_match_batch")


def make_pairs_host(items):
    """items: list of (h_img1, h_img2, h_out, h_count) CPU tensors (page-locked for
    asynchronous, capturable copies) -> ctypes array of DmPairHost."""
    arr = (DmPairHost * len(items))()
    for k, (i1, i2, out, cnt) in enumerate(items):
        H1, W1 = i1.shape
        H2, W2 = i2.shape
        arr[k] = DmPairHost(i1.data_ptr(), W1, H1, i2.data_ptr(), W2, H2, out.data_ptr(),
                            out.numel() * out.element_size() // MATCH_BYTES, cnt.data_ptr())
    return arr


def dm_batch_host_workspace_bytes(ctx, pairs) -> int:
    b = C.c_size_t()
    _check(ctx, load().dm_batch_host_workspace_bytes(ctx, len(pairs), pairs, C.byref(b)),
           "dm_batch_host_workspace_bytes")
    return b.value


def dm_match_batch_host(ctx, pairs, d_ws, stream=None):
    st = load().dm_match_batch_host(ctx, len(pairs), pairs, _dptr(d_ws), d_ws.numel() * d_ws.element_size(),
                                    _stream_ptr(stream))
    _check(ctx, st, "dm_match_batch_host")


def dm_set_batch_lanes(ctx, lanes: int) -> None:
    _check(ctx, load().dm_set_batch_lanes(ctx, int(lanes)), "dm_set_batch_lanes")


def dm_set_batch_wave(ctx, pairs: int) -> None:
    """Pairs per cross-pair wave of the batched form (1: each pair its own launches)."""
    _check(ctx, load().dm_set_batch_wave(ctx, int(pairs)), "dm_set_batch_wave")


def dm_autotune_batch(ctx, pairs, d_ws, stream=None) -> dict:
    """Pick the batch shape (wave width, lanes) for these pairs within d_ws; returns it."""
    ch = (C.c_int * 2)()
    _check(ctx, load().dm_autotune_batch(ctx, len(pairs), pairs, _dptr(d_ws), d_ws.numel() * d_ws.element_size(), ch,
                                         _stream_ptr(stream)), "dm_autotune_batch")
    return {"wave": ch[0], "lanes": ch[1]}


def dm_set_merge_keys(ctx, bits: int) -> None:
    """0: 32-bit merge keys where they fit (else 64); 64: 64-bit keys at every size."""
    _check(ctx, load().dm_set_merge_keys(ctx, int(bits)), "dm_set_merge_keys")


def dm_backtrack_noalloc(ctx, pyr, d_out, d_count, stream=None):
    """Backtracking with the library's fixed internal scratch (no workspace argument)."""
    cap = d_out.numel() * d_out.element_size() // MATCH_BYTES
    st = load().dm_backtrack_noalloc(ctx, pyr, _dptr(d_out), cap, _dptr(d_count), _stream_ptr(stream))
    _check(ctx, st, "dm_backtrack_noalloc")


NOALLOC_SCRATCH_BYTES = 32 << 20

TUNE_KEYS = ("m_chunk", "level_tile_rows", "bt_ctas_per_sm", "level_ring")


def dm_autotune(ctx, d_img1, d_img2, d_ws, stream=None) -> dict:
    """Time the launch-shape candidates on this pair; keep the fastest for its sizes."""
    H1, W1 = d_img1.shape
    H2, W2 = d_img2.shape
    out = (C.c_int * 4)()
    st = load().dm_autotune(ctx, _dptr(d_img1), W1, H1, _dptr(d_img2), W2, H2, _dptr(d_ws),
                            d_ws.numel() * d_ws.element_size(), out, _stream_ptr(stream))
    _check(ctx, st, "dm_autotune")
    return dict(zip(TUNE_KEYS, list(out)))


def dm_tuned_config(ctx, W1, H1, W2, H2) -> dict:
    out = (C.c_int * 4)()
    _check(ctx, load().dm_tuned_config(ctx, W1, H1, W2, H2, out), "dm_tuned_config")
    return dict(zip(TUNE_KEYS, list(out)))


def dm_set_tuned_config(ctx, W1, H1, W2, H2, cfg: dict) -> None:
    arr = (C.c_int * 4)(*[int(cfg[k]) for k in TUNE_KEYS])
    _check(ctx, load().dm_set_tuned_config(ctx, W1, H1, W2, H2, arr), "dm_set_tuned_config")


def dm_timing_start(ctx, max_calls: int) -> None:
    _check(ctx, load().dm_timing_start(ctx, max_calls), "dm_timing_start")


def dm_timing_read(ctx):
    ms = (C.c_double * NSTAGES)()
    n = C.c_int()
    launches = C.c_longlong()
    _check(ctx, load().dm_timing_read(ctx, ms, C.byref(n), C.byref(launches)), "dm_timing_read")
    return dict(zip(STAGES, list(ms))), n.value, launches.value


# ------------------------------------------------------------------------- #
# Convenience                                                                #
# ------------------------------------------------------------------------- #
class Context:
    """A library context plus cached device workspaces (allocated by torch)."""

    def __init__(self, precision: int = DM_FP32, device: int = 0, **params):
        import torch
        self.torch = torch
        cfg = dm_config_default()
        for k, v in params.items():
            if k == "compensated":
                cfg.compensated = int(bool(v))
            else:
                setattr(cfg, "lambda_" if k in ("lam", "lambda") else k, float(v))
        cfg.precision = precision
        self.cfg = cfg
        self.device = device
        self.ctx = dm_create(cfg, device)
        self._ws = {}

    def close(self):
        if self.ctx:
            dm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_merge_keys(self, bits: int):
        """dm_set_merge_keys; drops the cached workspaces (their sizes depend on it)."""
        dm_set_merge_keys(self.ctx, bits)
        self._ws.clear()

    def workspace(self, kind: str, W1, H1, W2, H2):
        key = (kind, W1, H1, W2, H2)
        if key not in self._ws:
            nbytes = dm_workspace_bytes(self.ctx, W1, H1, W2, H2)[kind]
            self._ws[key] = self.torch.empty(max(nbytes, 256), dtype=self.torch.uint8, device=f"cuda:{self.device}")
        return self._ws[key]

    def match(self, img1, img2, stream=None):
        """Matches as a float32 tensor [n][5] (x1, y1, x2, y2, score) on the device."""
        torch = self.torch
        dev = f"cuda:{self.device}"
        i1 = torch.as_tensor(img1, dtype=torch.float32, device=dev).contiguous()
        i2 = torch.as_tensor(img2, dtype=torch.float32, device=dev).contiguous()
        H1, W1 = i1.shape
        H2, W2 = i2.shape
        ws = self.workspace("match", W1, H1, W2, H2)
        n0 = dm_geometry(W1, H1, W2, H2)["n_patch0"]
        out = torch.empty((max(n0, 1), 5), dtype=torch.float32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        dm_match(self.ctx, i1, i2, ws, out, cnt, stream)
        n = int(cnt.item())
        return out[:n]

    def deepflow(self, img1, img2, matches=None, stream=None, **params):
        """DeepFlow (Sec. 4.3) of two same-size images with optional matches
        (rows x1, y1, x2, y2, score); returns device tensors (u, v)."""
        torch = self.torch
        dev = f"cuda:{self.device}"
        i1 = torch.as_tensor(img1, dtype=torch.float32, device=dev).contiguous()
        i2 = torch.as_tensor(img2, dtype=torch.float32, device=dev).contiguous()
        H, W = i1.shape
        prm = dm_flow_params(**params)
        dm_m = cnt = None
        cap = 0
        if matches is not None:
            dm_m = torch.as_tensor(matches, dtype=torch.float32, device=dev).reshape(-1, 5).contiguous()
            cap = dm_m.shape[0]
            cnt = torch.full((1,), cap, dtype=torch.int32, device=dev)
            if cap == 0:
                dm_m = torch.zeros((1, 5), dtype=torch.float32, device=dev)
        ws = torch.empty(max(dm_deepflow_workspace_bytes(self.ctx, W, H, max(cap, 1) if dm_m is not None else 0, prm), 256),
                         dtype=torch.uint8, device=dev)
        u = torch.empty((H, W), dtype=torch.float32, device=dev)
        v = torch.empty((H, W), dtype=torch.float32, device=dev)
        dm_deepflow(self.ctx, i1, i2, dm_m, cnt, u, v, ws, prm, stream)
        return u, v

    def match_star(self, img1, img2, stream=None):
        """DM* matches (local-maximum entry points, start + end scores) as a
        float32 tensor [n][5] on the device."""
        torch = self.torch
        dev = f"cuda:{self.device}"
        i1 = torch.as_tensor(img1, dtype=torch.float32, device=dev).contiguous()
        i2 = torch.as_tensor(img2, dtype=torch.float32, device=dev).contiguous()
        H1, W1 = i1.shape
        H2, W2 = i2.shape
        key = ("star", W1, H1, W2, H2)
        if key not in self._ws:
            nbytes = dm_star_workspace_bytes(self.ctx, W1, H1, W2, H2)["match"]
            self._ws[key] = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        n0 = dm_geometry(W1, H1, W2, H2)["n_patch0"]
        out = torch.empty((max(n0, 1), 5), dtype=torch.float32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        dm_match_star(self.ctx, i1, i2, self._ws[key], out, cnt, stream)
        n = int(cnt.item())
        return out[:n]

    def match_invariant(self, img1, img2, stream=None):
        """Scale and rotation invariant matches (Algorithm 2) as a float32
        tensor [n][5] (x1, y1, x2, y2, score) on the device."""
        torch = self.torch
        dev = f"cuda:{self.device}"
        i1 = torch.as_tensor(img1, dtype=torch.float32, device=dev).contiguous()
        i2 = torch.as_tensor(img2, dtype=torch.float32, device=dev).contiguous()
        H1, W1 = i1.shape
        H2, W2 = i2.shape
        key = ("invariant", W1, H1, W2, H2)
        if key not in self._ws:
            nbytes = dm_invariant_workspace_bytes(self.ctx, W1, H1, W2, H2)
            self._ws[key] = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        n0 = dm_geometry(W1, H1, W2, H2)["n_patch0"]
        out = torch.empty((max(n0, 1), 5), dtype=torch.float32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        dm_match_invariant(self.ctx, i1, i2, self._ws[key], out, cnt, stream)
        n = int(cnt.item())
        return out[:n]

    def autotune(self, img1, img2, stream=None) -> dict:
        """Autotune the launch shapes for pairs of these images' sizes."""
        torch = self.torch
        dev = f"cuda:{self.device}"
        i1 = torch.as_tensor(img1, dtype=torch.float32, device=dev).contiguous()
        i2 = torch.as_tensor(img2, dtype=torch.float32, device=dev).contiguous()
        H1, W1 = i1.shape
        H2, W2 = i2.shape
        return dm_autotune(self.ctx, i1, i2, self.workspace("match", W1, H1, W2, H2), stream)

    def status(self, W1, H1, W2, H2, kind="match"):
        L = dm_geometry(W1, H1, W2, H2)["L"]
        return dm_read_status(self.ctx, self.workspace(kind, W1, H1, W2, H2), L + 1)


def exported_symbols() -> list:
    return list(_SIGS.keys())


def to_numpy_matches(t) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.float64)
