"""The C-ABI library loads and exports every symbol include/hpxgs.h declares, and
rejects bad arguments on the host (no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

import pytest
import torch

from paper_2606_29794_b300 import _lib as L
from paper_2606_29794_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hpxgs.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hpxgs_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.EXPORTS)


def test_strerror_and_status(lib):
    assert L.strerror(0) == "ok"
    assert "capacity" in L.strerror(L.E_CAPACITY)
    assert lib.hpxgs_status_error(L.F_CAPACITY) == L.E_CAPACITY
    assert lib.hpxgs_status_error(0) == 0


def test_profile_arm_and_armed(lib):
    # arming records the events at the stage's next run; a stage that never ran stays armed
    # (host-side bookkeeping only: no event is recorded without a launch)
    st = L.STAGES.index("hssim_bwd")
    assert lib.hpxgs_profile_armed(st) in (0, 1)
    assert lib.hpxgs_profile_arm(st, ctypes.c_void_p(0x10), ctypes.c_void_p(0x20)) == 0
    try:                                   # placeholder handles: never leave them armed
        assert lib.hpxgs_profile_armed(st) == 1
    finally:
        assert lib.hpxgs_profile_arm(st, None, None) == 0
    assert lib.hpxgs_profile_armed(st) == 0
    assert lib.hpxgs_profile_armed(len(L.STAGES)) == L.E_INVALID_ARG
    assert lib.hpxgs_profile_armed(-1) == L.E_INVALID_ARG


def test_adaptive_nside(lib):
    ns = ctypes.c_double(); k = ctypes.c_int(); kl = ctypes.c_int(); kh = ctypes.c_int()
    assert lib.hpxgs_nside_for_image(0, 6080, 3040, 360, 360, ctypes.byref(ns), ctypes.byref(k), ctypes.byref(kl),
                                     ctypes.byref(kh)) == 0
    assert (kl.value, kh.value) == (10, 11)
    assert lib.hpxgs_nside_for_image(0, -1, 3040, 360, 360, None, None, None, None) == L.E_INVALID_ARG


def test_host_argument_checks(lib):
    cfg = L.default_config()
    v = L.make_views([dict(W=[1, 0, 0, 0, 1, 0, 0, 0, 1], b=[0, 0, 0], nside_log2=6, cam=0)])
    n = ctypes.c_size_t()
    assert lib.hpxgs_forward_workspace_size(1000, v, 1, ctypes.byref(cfg), 10000, ctypes.byref(n)) == 0
    assert n.value > 0
    bad = L.default_config(tile_level=2)
    assert lib.hpxgs_forward_workspace_size(1000, v, 1, ctypes.byref(bad), 10000, ctypes.byref(n)) == L.E_INVALID_ARG
    vb = L.make_views([dict(W=[1, 0, 0, 0, 1, 0, 0, 0, 1], b=[0, 0, 0], nside_log2=2, cam=0)])
    assert lib.hpxgs_forward_workspace_size(1000, vb, 1, ctypes.byref(cfg), 10000, ctypes.byref(n)) == L.E_INVALID_ARG
    vp = L.make_views([dict(W=[1, 0, 0, 0, 1, 0, 0, 0, 1], b=[0, 0, 0], nside_log2=6, cam=1, fov_x=200.0)])
    assert lib.hpxgs_forward_workspace_size(1000, vp, 1, ctypes.byref(cfg), 10000, ctypes.byref(n)) == L.E_INVALID_ARG
    # principal point: inside the image for the pinhole, centred for the fisheye and the full sphere
    I3 = [1, 0, 0, 0, 1, 0, 0, 0, 1]
    for cam, pp, rc in [(1, (0.5, -0.9), 0), (1, (1.0, 0.0), L.E_INVALID_ARG), (1, (0.0, float("nan")), L.E_INVALID_ARG),
                        (2, (0.1, 0.0), L.E_INVALID_ARG), (0, (0.0, 0.2), L.E_INVALID_ARG), (2, (0.0, 0.0), 0)]:
        vv = L.make_views([dict(W=I3, b=[0, 0, 0], nside_log2=6, cam=cam, fov_x=90.0, pp=pp)])
        assert lib.hpxgs_forward_workspace_size(1000, vv, 1, ctypes.byref(cfg), 10000, ctypes.byref(n)) == rc, (cam, pp)
    assert lib.hpxgs_forward_workspace_size(1000, v, 1, ctypes.byref(cfg), -5, ctypes.byref(n)) == L.E_INVALID_ARG
    assert lib.hpxgs_forward_workspace_size(1000, v, 0, ctypes.byref(cfg), 10, ctypes.byref(n)) == L.E_INVALID_ARG
    # the fused loss backward checks its loss views and lambda before any launch
    g0 = L.Gaussians(); g0.P = 0; g0.sh_degree = 0
    lv = (L.LossView * 1)()
    args = lambda lvs, lam: (ctypes.byref(g0), v, 1, ctypes.byref(cfg), ctypes.c_void_p(8), 1 << 20, 100, lvs, lam,
                             ctypes.c_void_p(8), ctypes.c_void_p(8), None, None, None, None, None, None, None)
    assert lib.hpxgs_backward_hssim(*args(None, 0.2)) == L.E_INVALID_ARG
    assert lib.hpxgs_backward_hssim(*args(lv, 0.2)) == L.E_INVALID_ARG          # null maps / table / workspace
    assert lib.hpxgs_backward_hssim(*args(lv, 1.5)) == L.E_INVALID_ARG
    # null required pointers are rejected before any launch
    g = L.Gaussians(); g.P = 10; g.sh_degree = 0
    assert lib.hpxgs_forward(ctypes.byref(g), v, 1, ctypes.byref(cfg), None, 0, 0, None, None, None, None, None, None,
                             None, None) == L.E_INVALID_ARG
    assert lib.hpxgs_hssim_workspace_size(2, ctypes.byref(n)) == L.E_INVALID_ARG
    assert lib.hpxgs_pix2vec_nest(20, None, 1, None, None, None) == L.E_INVALID_ARG


def test_flop_counts_match_header():
    text = open(HEADER).read()
    vals = dict(re.findall(r"#define HPXGS_((?:FLOPS|MUFU)_[A-Z_]+)\s+(\d+)", text))
    assert {k: int(v) for k, v in vals.items()} == {
        "FLOPS_EVAL": L.FLOPS_EVAL, "FLOPS_FWD_CONTRIB": L.FLOPS_FWD_CONTRIB, "FLOPS_BWD_CONTRIB": L.FLOPS_BWD_CONTRIB,
        "MUFU_FWD_CONTRIB": L.MUFU_FWD_CONTRIB, "MUFU_BWD_CONTRIB": L.MUFU_BWD_CONTRIB}


def test_fused_backward_binding_wants_one_loss_view_per_view():
    # checked on the host before the library is called (the library reads nviews entries)
    from paper_2606_29794_b300 import raster as R
    rast = R.Rasterizer.__new__(R.Rasterizer)
    state = {"keep": [None] * 5, "nv": 2}
    with pytest.raises(ValueError):
        rast.backward_hssim_raw(state, [("I", "G", "tab", "ws", None)], 0.2)


def test_density_stats_binding_checks_buffers():
    from paper_2606_29794_b300 import raster as R
    rast = R.Rasterizer.__new__(R.Rasterizer)
    g = L.Gaussians()
    g.P = 4
    state = {"g": g, "nv": 2}
    cpu = torch.zeros(4)
    with pytest.raises(ValueError):
        rast.density_stats(state, cpu, cpu, cpu.int())          # host tensors are refused


def test_scene_tensors_are_validated_before_any_launch():
    from paper_2606_29794_b300 import raster as R
    P = 8
    t = lambda *s: torch.zeros(*s)
    with pytest.raises(ValueError):                              # host tensors
        R.gaussians_struct(t(P, 3), t(P, 3), t(P, 4), t(P), t(P, 16, 3), 3)
    with pytest.raises(ValueError):                              # SH rows do not match the degree
        R.gaussians_struct(t(P, 3), t(P, 3), t(P, 4), t(P), t(P, 9, 3), 3)
    with pytest.raises(ValueError):                              # degree out of range
        R.gaussians_struct(t(P, 3), t(P, 3), t(P, 4), t(P), t(P, 25, 3), 4)


def test_resample_plan_sizes_and_checks(lib):
    n = ctypes.c_size_t()
    assert lib.hpxgs_resample_plan_size(L.PLAN_SPHERE_TO_IMAGE, 7, 180, 120, ctypes.byref(n)) == 0
    al = lambda x: (x + 255) // 256 * 256
    assert n.value == al(16 * 180 * 120) + al(16 * 180 * 120) + al(180 * 120)
    assert lib.hpxgs_resample_plan_size(L.PLAN_IMAGE_TO_SPHERE, 7, 180, 120, ctypes.byref(n)) == 0
    npix = 12 * 4 ** 7
    assert n.value == al(16 * npix) + al(16 * npix) + al(4 * npix // 32)
    assert lib.hpxgs_resample_plan_size(2, 7, 180, 120, ctypes.byref(n)) == L.E_INVALID_ARG
    assert lib.hpxgs_resample_plan_size(L.PLAN_IMAGE_TO_SPHERE, 1, 180, 120, ctypes.byref(n)) == L.E_INVALID_ARG
    assert lib.hpxgs_resample_plan_size(L.PLAN_SPHERE_TO_IMAGE, 7, 65536, 65536, ctypes.byref(n)) == L.E_INVALID_ARG
    # an application with a plan smaller than its sizes is refused before any launch
    assert lib.hpxgs_sphere_to_image_planned(ctypes.c_void_p(16), 7, 180, 120, ctypes.c_void_p(16), 1024,
                                             ctypes.c_void_p(16), None, None) == L.E_WORKSPACE

