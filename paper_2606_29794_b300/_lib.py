"""ctypes binding of libhpxgs.so (argument marshalling only).

Every call lands in the CUDA library; there is no CPU fallback. Importing this
module does not touch the GPU; loading the library fails loudly if the in-tree
``libhpxgs.so`` is missing (build it with ``python -m paper_2606_29794_b300.build``
or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhpxgs.so")

OK = 0
E_INVALID_ARG, E_CAPACITY, E_TIMEOUT, E_CUDA, E_UNIMPLEMENTED, E_WORKSPACE, E_CAPTURE = -1, -2, -3, -4, -5, -6, -7
F_CAPACITY, F_TIMEOUT = 1, 2
CAM_FULL, CAM_PINHOLE, CAM_FISHEYE = 0, 1, 2
MAX_VIEWS = 64
NACC = 9
STAGES = ("mask", "preprocess", "depth_sort", "tile_count", "scan", "tile_emit", "pair_sort", "ranges",
          "blend_fwd", "blend_bwd", "preprocess_bwd", "hssim_fwd", "hssim_bwd")


class Gaussians(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("scales", ctypes.c_void_p), ("rotations", ctypes.c_void_p),
                ("opacities", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("P", ctypes.c_int32),
                ("sh_degree", ctypes.c_int32)]


class Camera(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("fov_x_deg", ctypes.c_float), ("fov_y_deg", ctypes.c_float),
                ("ppx", ctypes.c_float), ("ppy", ctypes.c_float)]


class View(ctypes.Structure):
    _fields_ = [("W", ctypes.c_float * 9), ("b", ctypes.c_float * 3), ("nside_log2", ctypes.c_int32),
                ("cam", Camera)]


class LossView(ctypes.Structure):
    _fields_ = [("maps", ctypes.c_void_p), ("targets", ctypes.c_void_p), ("table", ctypes.c_void_p),
                ("hssim_ws", ctypes.c_void_p), ("dloss", ctypes.c_void_p)]


class Config(ctypes.Structure):
    _fields_ = [("tile_level", ctypes.c_int32), ("eps_T", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("cutoff_m", ctypes.c_float), ("blur_rad2", ctypes.c_float), ("near_plane", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("lambda_ssim", ctypes.c_float), ("write_outside", ctypes.c_int32),
                ("fwd_ppt", ctypes.c_int32), ("bwd_ppt", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("query", ctypes.c_int32), ("query_log2f", ctypes.c_int32), ("blend_cull", ctypes.c_int32),
                ("blend_split", ctypes.c_int32)]


class WorkspaceView(ctypes.Structure):
    _fields_ = [("records", ctypes.c_void_p), ("radii", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("pair_tiles", ctypes.c_void_p), ("pair_ids", ctypes.c_void_p), ("ranges", ctypes.c_void_p),
                ("n_pairs", ctypes.c_void_p), ("accum", ctypes.c_void_p), ("n_eval", ctypes.c_void_p),
                ("n_contrib", ctypes.c_void_p), ("total_tiles", ctypes.c_int64), ("cull_masks", ctypes.c_void_p)]


class HpxgsError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


_lib = None
_P = ctypes.POINTER
_vp, _i32, _i64, _sz, _f32, _f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_float, ctypes.c_double

# FP32 work per (pixel, entry) pair of the blend kernels (the HPXGS_FLOPS_* and
# HPXGS_MUFU_* values of include/hpxgs.h; a test checks they agree).
FLOPS_EVAL, FLOPS_FWD_CONTRIB, FLOPS_BWD_CONTRIB = 40, 13, 83
QUERY_RING, QUERY_NESTED = 0, 1
PLAN_SPHERE_TO_IMAGE, PLAN_IMAGE_TO_SPHERE = 0, 1
MUFU_FWD_CONTRIB, MUFU_BWD_CONTRIB = 1, 2

_SIGS = {
    "hpxgs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "hpxgs_status_error": (ctypes.c_int, [_i32]),
    "hpxgs_config_default": (None, [_P(Config)]),
    "hpxgs_nside_for_image": (ctypes.c_int, [ctypes.c_int, _f64, _f64, _f64, _f64, _P(_f64), _P(ctypes.c_int),
                                             _P(ctypes.c_int), _P(ctypes.c_int)]),
    "hpxgs_pixrad": (ctypes.c_int, [ctypes.c_int, _P(_f64), ctypes.c_void_p]),
    "hpxgs_tile_rho": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P(_f64), _vp]),
    "hpxgs_prepare": (ctypes.c_int, [_P(View), ctypes.c_int, _P(Config), _vp]),
    "hpxgs_mask_build": (ctypes.c_int, [_P(View), _P(Config), _vp, _vp]),
    "hpxgs_pix2vec_nest": (ctypes.c_int, [ctypes.c_int, _vp, _i64, _vp, _vp, _vp]),
    "hpxgs_vec2pix_nest": (ctypes.c_int, [ctypes.c_int, _vp, _i64, _vp, _vp]),
    "hpxgs_pix2ang_nest": (ctypes.c_int, [ctypes.c_int, _vp, _i64, _vp, _vp, _vp]),
    "hpxgs_ang2pix_nest": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _i64, _vp, _vp]),
    "hpxgs_nest2ring": (ctypes.c_int, [ctypes.c_int, _vp, _i64, _vp, _vp]),
    "hpxgs_ring2nest": (ctypes.c_int, [ctypes.c_int, _vp, _i64, _vp, _vp]),
    "hpxgs_neighbours_nest": (ctypes.c_int, [ctypes.c_int, _vp, _i64, _vp, _vp]),
    "hpxgs_forward_workspace_size": (ctypes.c_int, [_i32, _P(View), ctypes.c_int, _P(Config), _i64, _P(_sz)]),
    "hpxgs_forward": (ctypes.c_int, [_P(Gaussians), _P(View), ctypes.c_int, _P(Config), _vp, _sz, _i64, _vp, _vp, _vp,
                                     _vp, _vp, _vp, _vp, _vp]),
    "hpxgs_backward": (ctypes.c_int, [_P(Gaussians), _P(View), ctypes.c_int, _P(Config), _vp, _sz, _i64, _vp, _vp,
                                      _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hpxgs_backward_hssim": (ctypes.c_int, [_P(Gaussians), _P(View), ctypes.c_int, _P(Config), _vp, _sz, _i64,
                                            _P(LossView), _f32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hpxgs_count_pairs": (ctypes.c_int, [_P(Gaussians), _P(View), ctypes.c_int, _P(Config), _vp, _sz, _vp, _vp, _vp]),
    "hpxgs_density_stats": (ctypes.c_int, [_i32, _P(View), ctypes.c_int, _P(Config), _vp, _sz, _i64, _vp, _vp, _vp,
                                           _vp, _vp]),
    "hpxgs_workspace_inspect": (ctypes.c_int, [_i32, _P(View), ctypes.c_int, _P(Config), _i64, _vp,
                                               _P(WorkspaceView)]),
    "hpxgs_profile_arm": (ctypes.c_int, [ctypes.c_int, _vp, _vp]),
    "hpxgs_profile_armed": (ctypes.c_int, [ctypes.c_int]),
    "hpxgs_sphere_to_image": (ctypes.c_int, [_vp, ctypes.c_int, _P(Camera), ctypes.c_int, ctypes.c_int, _vp, _vp,
                                             _vp]),
    "hpxgs_sphere_to_image_backward": (ctypes.c_int, [_vp, ctypes.c_int, _P(Camera), ctypes.c_int, ctypes.c_int,
                                                      _vp, _vp]),
    "hpxgs_image_to_sphere": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _P(Camera), ctypes.c_int, _vp, _vp,
                                             _vp]),
    "hpxgs_image_to_sphere_u8": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _P(Camera), ctypes.c_int, _vp,
                                                _vp, _vp]),
    "hpxgs_resample_plan_size": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P(_sz)]),
    "hpxgs_resample_plan_build": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P(Camera), ctypes.c_int, ctypes.c_int,
                                                 _vp, _sz, _vp]),
    "hpxgs_sphere_to_image_planned": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _sz, _vp,
                                                     _vp, _vp]),
    "hpxgs_sphere_to_image_backward_planned": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp,
                                                              _sz, _vp, _vp]),
    "hpxgs_image_to_sphere_planned": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _sz, _vp,
                                                     _vp, _vp]),
    "hpxgs_image_to_sphere_u8_planned": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _sz,
                                                        _vp, _vp, _vp]),
    "hpxgs_launch_count": (ctypes.c_uint64, []),
    "hpxgs_probe_alu_peak": (ctypes.c_int, [_P(_f64), _P(_f64), ctypes.c_void_p]),
    "hpxgs_probe_grid_barrier": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _vp, _vp, _vp, _vp]),
    "hpxgs_hssim_table_size": (ctypes.c_int, [ctypes.c_int, _P(_sz)]),
    "hpxgs_hssim_table_build": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _sz, _vp]),
    "hpxgs_hssim_forward_table": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _f32, _vp, _vp, _sz, _vp, _vp]),
    "hpxgs_hssim_backward_table": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _f32, _vp, _vp, _sz, _vp, _vp, _vp]),
    "hpxgs_hssim_workspace_size": (ctypes.c_int, [ctypes.c_int, _P(_sz)]),
    "hpxgs_hssim_forward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _f32, _vp, _sz, _vp, _vp]),
    "hpxgs_hssim_backward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _f32, _vp, _sz, _vp, _vp, _vp]),
    "hpxgs_hssim_loss_noalloc": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _f32, _vp, _vp]),
}

EXPORTS = tuple(_SIGS)


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhpxgs.so not built at {LIB_PATH}; run paper_2606_29794_b300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().hpxgs_strerror(code).decode()


def check(code: int, what: str):
    if code != OK:
        raise HpxgsError(code, what)


def default_config(**kw) -> Config:
    c = Config()
    lib().hpxgs_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if k == "bg":
            for i in range(3):
                c.bg[i] = float(v[i])
        elif k == "blur" and v is None:
            c.blur_rad2 = -1.0
        elif k == "blur":
            c.blur_rad2 = float(v)
        elif k == "lam":
            c.lambda_ssim = float(v)
        else:
            setattr(c, k, v)
    return c


def make_views(views) -> ctypes.Array:
    arr = (View * len(views))()
    for i, v in enumerate(views):
        W = [float(x) for x in list(getattr(v["W"], "ravel", lambda: v["W"])())]
        b = [float(x) for x in list(getattr(v["b"], "ravel", lambda: v["b"])())]
        for j in range(9):
            arr[i].W[j] = W[j]
        for j in range(3):
            arr[i].b[j] = b[j]
        arr[i].nside_log2 = int(v["nside_log2"])
        arr[i].cam.kind = int(v.get("cam", CAM_FULL))
        arr[i].cam.fov_x_deg = float(v.get("fov_x", 360.0))
        arr[i].cam.fov_y_deg = float(v.get("fov_y", v.get("fov_x", 360.0)))
        arr[i].cam.ppx, arr[i].cam.ppy = (float(x) for x in v.get("pp", (0.0, 0.0)))
    return arr
