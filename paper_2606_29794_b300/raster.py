"""PyTorch front end of the HEALPix rasterizer: differentiable render and HSSIM loss.

PyTorch supplies device memory and the stream; every step of the path runs in
libhpxgs.so (see include/hpxgs.h). The autograd Function keeps the forward's
workspace (records, sorted tile lists, ranges, masks) together with the
per-pixel final transmittance and last-contributor count, and the backward
walks the same lists in reverse (Sec. 3.2), so no blend history is stored.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import torch

from . import _lib as L


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _f32(t):
    if not (t.is_cuda and t.dtype == torch.float32):
        raise TypeError("expected a float32 CUDA tensor")
    return t.contiguous()


def npix(k: int) -> int:
    return 12 * 4 ** k


def gaussians_struct(means, scales, rotations, opacities, sh, sh_degree) -> L.Gaussians:
    """The scene as the C ABI's struct of device pointers, after checking that every tensor is a
    contiguous float32 CUDA tensor on one device with the shapes the kernels index: means, scales
    [P, 3], rotations [P, 4], opacities [P] (or [P, 1]), sh [P, (sh_degree + 1)^2, 3]."""
    P = int(means.shape[0]) if means.dim() == 2 else -1
    K = (int(sh_degree) + 1) ** 2
    want = [(means, (P, 3)), (scales, (P, 3)), (rotations, (P, 4)), (sh, (P, K, 3))]
    ok = 0 <= int(sh_degree) <= 3 and P >= 0 and opacities.numel() == P and opacities.dim() in (1, 2)
    for t, shape in want + [(opacities, tuple(opacities.shape))]:
        ok = ok and tuple(t.shape) == shape and t.dtype == torch.float32 and t.is_cuda and t.is_contiguous() \
            and t.device == means.device
    if not ok:
        raise ValueError("gaussians: expected contiguous float32 CUDA tensors on one device: means, scales [P, 3], "
                         "rotations [P, 4], opacities [P], sh [P, (sh_degree + 1)^2, 3], 0 <= sh_degree <= 3")
    g = L.Gaussians()
    g.means, g.scales, g.rotations = means.data_ptr(), scales.data_ptr(), rotations.data_ptr()
    g.opacities, g.sh = opacities.data_ptr(), sh.data_ptr()
    g.P = int(means.shape[0])
    g.sh_degree = int(sh_degree)
    return g


@dataclass
class Layout:
    pix_base: list
    total_pix: int
    total_tiles: int


def view_layout(views, tile_level=4) -> Layout:
    base, tot, tiles = [], 0, 0
    for v in views:
        base.append(tot)
        tot += npix(v["nside_log2"])
        tiles += 12 * 4 ** (v["nside_log2"] - tile_level)
    return Layout(base, tot, tiles)


class Rasterizer:
    """Holds the config and the pair capacity; each forward gets its own workspace."""

    def __init__(self, tile_level=4, eps_T=1e-4, alpha_max=0.99, cutoff=9.0, blur=None, near=0.2,
                 bg=(0.0, 0.0, 0.0), lam=0.2, write_outside=1, capacity=None, headroom=1.15, fwd_ppt=0, bwd_ppt=0,
                 blocks_per_sm=0, query=0, query_log2f=0, blend_cull=1, blend_split=1):
        self.cfg = L.default_config(tile_level=tile_level, eps_T=eps_T, alpha_max=alpha_max, cutoff_m=cutoff,
                                    blur=blur, near_plane=near, bg=bg, lam=lam, write_outside=write_outside,
                                    fwd_ppt=fwd_ppt, bwd_ppt=bwd_ppt, blocks_per_sm=blocks_per_sm, query=query,
                                    query_log2f=query_log2f, blend_cull=blend_cull, blend_split=blend_split)
        self.capacity = capacity
        self.headroom = headroom

    @property
    def tile_level(self):
        return self.cfg.tile_level

    def workspace_bytes(self, P, cviews, nv, cap) -> int:
        n = ctypes.c_size_t()
        L.check(L.lib().hpxgs_forward_workspace_size(P, cviews, nv, ctypes.byref(self.cfg), int(cap), ctypes.byref(n)),
                "workspace size")
        return n.value

    def prepare(self, views):
        cv = L.make_views(views)
        L.check(L.lib().hpxgs_prepare(cv, len(views), ctypes.byref(self.cfg), ctypes.c_void_p(_stream())), "prepare")

    def count_pairs(self, g: L.Gaussians, cviews, nv, device) -> int:
        nb = self.workspace_bytes(g.P, cviews, nv, 0)
        ws = torch.empty(nb, dtype=torch.uint8, device=device)
        cnt = torch.zeros(1, dtype=torch.int64, device=device)
        st = torch.zeros(1, dtype=torch.int32, device=device)
        L.check(L.lib().hpxgs_count_pairs(ctypes.byref(g), cviews, nv, ctypes.byref(self.cfg), _ptr(ws), nb,
                                          _ptr(cnt), _ptr(st), ctypes.c_void_p(_stream())), "count_pairs")
        return int(cnt.item())

    def forward_raw(self, means, scales, rotations, opacities, sh, sh_degree, views, check_status=True, depth=False):
        """Runs hpxgs_forward; returns a dict of outputs and the state the backward needs.
        With depth=True the outputs also hold "depth", the inverse-depth channel."""
        means, scales, rotations, opacities, sh = map(_f32, (means, scales, rotations, opacities, sh))
        dev = means.device
        g = gaussians_struct(means, scales, rotations, opacities, sh, sh_degree)
        nv = len(views)
        cv = L.make_views(views)
        lay = view_layout(views, self.cfg.tile_level)
        if self.capacity is None:
            self.capacity = int(self.count_pairs(g, cv, nv, dev) * self.headroom) + 4096
        for _attempt in range(4):
            cap = int(self.capacity)
            nb = self.workspace_bytes(g.P, cv, nv, cap)
            ws = torch.empty(nb, dtype=torch.uint8, device=dev)
            maps = torch.empty((lay.total_pix, 3), dtype=torch.float32, device=dev)
            T = torch.empty(lay.total_pix, dtype=torch.float32, device=dev)
            last = torch.empty(lay.total_pix, dtype=torch.int32, device=dev)
            mask = torch.empty(lay.total_pix // 32, dtype=torch.int32, device=dev)
            radii = torch.empty((nv, g.P), dtype=torch.float32, device=dev)
            dmap = torch.empty(lay.total_pix, dtype=torch.float32, device=dev) if depth else None
            status = torch.zeros(1, dtype=torch.int32, device=dev)
            L.check(L.lib().hpxgs_forward(ctypes.byref(g), cv, nv, ctypes.byref(self.cfg), _ptr(ws), nb, cap, _ptr(maps),
                                          _ptr(T), _ptr(last), _ptr(mask), _ptr(radii),
                                          _ptr(dmap) if depth else None, _ptr(status),
                                          ctypes.c_void_p(_stream())), "forward")
            if not check_status:
                break
            flags = int(status.item())
            if not (flags & L.F_CAPACITY):
                L.check(L.lib().hpxgs_status_error(flags), "forward (device status)")
                break
            need = self.count_pairs(g, cv, nv, dev)
            self.capacity = int(need * self.headroom) + 4096
        else:
            raise L.HpxgsError(L.E_CAPACITY, "forward")
        state = dict(ws=ws, nb=nb, cap=cap, cviews=cv, nv=nv, g=g, T=T, last=last, status=status,
                     keep=(means, scales, rotations, opacities, sh), sh_degree=sh_degree)
        out = dict(maps=maps, T=T, last=last, mask=mask, radii=radii, status=status, layout=lay)
        if depth:
            out["depth"] = dmap
        return out, state

    def backward_raw(self, state, dmaps, ddepth=None):
        """Runs hpxgs_backward from dL/dmaps (and optionally dL/ddepth of the inverse-depth channel)."""
        means, scales, rotations, opacities, sh = state["keep"]
        dmaps = _f32(dmaps)
        ddepth = _f32(ddepth) if ddepth is not None else None
        npx = state["T"].numel()
        if dmaps.numel() != 3 * npx or (ddepth is not None and ddepth.numel() != npx):
            raise ValueError(f"backward: dL/dmaps needs {3 * npx} values and dL/ddepth {npx}")
        dm, ds, dq, do, dsh = (torch.empty_like(t) for t in (means, scales, rotations, opacities, sh))
        st = torch.zeros(1, dtype=torch.int32, device=means.device)
        L.check(L.lib().hpxgs_backward(ctypes.byref(state["g"]), state["cviews"], state["nv"], ctypes.byref(self.cfg),
                                       _ptr(state["ws"]), state["nb"], state["cap"], _ptr(dmaps), _ptr(state["T"]),
                                       _ptr(state["last"]), _ptr(ddepth) if ddepth is not None else None,
                                       _ptr(dm), _ptr(ds), _ptr(dq), _ptr(do), _ptr(dsh), _ptr(st),
                                       ctypes.c_void_p(_stream())), "backward")
        return dm, ds, dq, do, dsh

    def backward_hssim_raw(self, state, loss_views, lam):
        """Runs hpxgs_backward_hssim: the backward of the L1 + HSSIM loss of every view, with each
        pixel's dL/dI formed inside the backward blend. loss_views: one (maps, targets, table,
        hssim_ws, dloss or None) per view, after hpxgs_hssim_forward_table on the same stream."""
        means, scales, rotations, opacities, sh = state["keep"]
        if len(loss_views) != state["nv"]:
            raise ValueError(f"one loss view per rendered view: got {len(loss_views)} for {state['nv']}")
        lv = (L.LossView * len(loss_views))()
        for i, (I, G, tab, hws, dl) in enumerate(loss_views):
            lv[i].maps, lv[i].targets = I.data_ptr(), G.data_ptr()
            lv[i].table, lv[i].hssim_ws = tab.data_ptr(), hws.data_ptr()
            lv[i].dloss = dl.data_ptr() if dl is not None else None
        dm, ds, dq, do, dsh = (torch.empty_like(t) for t in (means, scales, rotations, opacities, sh))
        st = torch.zeros(1, dtype=torch.int32, device=means.device)
        L.check(L.lib().hpxgs_backward_hssim(ctypes.byref(state["g"]), state["cviews"], state["nv"],
                                             ctypes.byref(self.cfg), _ptr(state["ws"]), state["nb"], state["cap"], lv,
                                             float(lam), _ptr(state["T"]), _ptr(state["last"]), _ptr(dm), _ptr(ds),
                                             _ptr(dq), _ptr(do), _ptr(dsh), _ptr(st), ctypes.c_void_p(_stream())),
                "backward_hssim")
        return dm, ds, dq, do, dsh

    def density_stats(self, state, rs_max, grad_accum, vis_count, angular=None):
        """Radian-space density statistics (Sec. 4.2) after backward_raw on `state`: updates the
        per-Gaussian buffers rs_max (float32 [P]), grad_accum (float32 [P]) and vis_count (int32 [P])
        in place over the visible (view, Gaussian) pairs; angular (float32 [views, P, 2] or None)
        receives dL/domega, dL/dphi per pair."""
        P, nv = state["g"].P, state["nv"]
        for t, dt in ((rs_max, torch.float32), (grad_accum, torch.float32), (vis_count, torch.int32)):
            if not (t.is_cuda and t.is_contiguous() and t.dtype == dt and t.numel() == P):
                raise ValueError(f"density_stats: expected a contiguous CUDA {dt} tensor of {P} elements")
        if angular is not None and not (angular.is_cuda and angular.is_contiguous() and angular.dtype == torch.float32
                                        and angular.numel() == 2 * nv * P):
            raise ValueError(f"density_stats: angular must be a contiguous CUDA float32 tensor of {2 * nv * P} elements")
        L.check(L.lib().hpxgs_density_stats(state["g"].P, state["cviews"], state["nv"], ctypes.byref(self.cfg),
                                            _ptr(state["ws"]), state["nb"], state["cap"], _ptr(rs_max),
                                            _ptr(grad_accum), _ptr(vis_count),
                                            _ptr(angular) if angular is not None else None,
                                            ctypes.c_void_p(_stream())), "density_stats")


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, rotations, opacities, sh, rast, views, sh_degree, check_status):
        out, state = rast.forward_raw(means, scales, rotations, opacities, sh, sh_degree, views, check_status)
        ctx.rast = rast
        ctx.state = state
        ctx.mark_non_differentiable(out["T"], out["last"], out["mask"], out["radii"])
        return out["maps"], out["T"], out["last"], out["mask"], out["radii"]

    @staticmethod
    def backward(ctx, dmaps, dT, dlast, dmask, dradii):
        grads = ctx.rast.backward_raw(ctx.state, dmaps if dmaps is not None else torch.zeros_like(ctx.state["T"]).unsqueeze(1).expand(-1, 3).contiguous())
        ctx.state = None
        return (*grads, None, None, None, None)


class _RenderDepthFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, rotations, opacities, sh, rast, views, sh_degree, check_status):
        out, state = rast.forward_raw(means, scales, rotations, opacities, sh, sh_degree, views, check_status,
                                      depth=True)
        ctx.rast = rast
        ctx.state = state
        ctx.mark_non_differentiable(out["T"], out["last"], out["mask"], out["radii"])
        return out["maps"], out["depth"], out["T"], out["last"], out["mask"], out["radii"]

    @staticmethod
    def backward(ctx, dmaps, ddepth, dT, dlast, dmask, dradii):
        T = ctx.state["T"]
        if dmaps is None:
            dmaps = torch.zeros((T.shape[0], 3), dtype=torch.float32, device=T.device)
        if ddepth is None:
            ddepth = torch.zeros_like(T)
        grads = ctx.rast.backward_raw(ctx.state, dmaps.contiguous(), ddepth.contiguous())
        ctx.state = None
        return (*grads, None, None, None, None)


def render(means, scales, rotations, opacities, sh, views, rasterizer: Rasterizer | None = None, sh_degree=None,
           check_status=True, with_depth=False):
    """Differentiable render of `views`: returns (maps, T_final, last, mask_words, radii), packed over views;
    with with_depth, (maps, depth, T_final, last, mask_words, radii) where depth is the inverse-depth
    channel sum_i T_i alpha_i / r_i (Sec. 3.2), differentiable like maps."""
    rast = rasterizer or Rasterizer()
    if sh_degree is None:
        sh_degree = int(round(math.sqrt(sh.shape[1]))) - 1
    if with_depth:
        return _RenderDepthFn.apply(means, scales, rotations, opacities, sh, rast, views, sh_degree, check_status)
    return _RenderFn.apply(means, scales, rotations, opacities, sh, rast, views, sh_degree, check_status)


class _HSSIMFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, I, G, mask_words, k, lam):
        I, G = _f32(I), _f32(G)
        nb = ctypes.c_size_t()
        L.check(L.lib().hpxgs_hssim_workspace_size(k, ctypes.byref(nb)), "hssim workspace")
        ws = torch.empty(nb.value, dtype=torch.uint8, device=I.device)
        out = torch.empty(3, dtype=torch.float32, device=I.device)
        L.check(L.lib().hpxgs_hssim_forward(_ptr(I), _ptr(G), _ptr(mask_words), k, float(lam), _ptr(ws), nb.value,
                                            _ptr(out), ctypes.c_void_p(_stream())), "hssim forward")
        ctx.save_for_backward(I, G, mask_words, ws)
        ctx.k, ctx.lam, ctx.nb = k, lam, nb.value
        ctx.mark_non_differentiable(out)
        return out[0].clone(), out

    @staticmethod
    def backward(ctx, gloss, gout):
        I, G, mask_words, ws = ctx.saved_tensors
        gl = _f32(gloss.reshape(1)) if gloss is not None else torch.ones(1, device=I.device)
        dI = torch.empty_like(I)
        L.check(L.lib().hpxgs_hssim_backward(_ptr(I), _ptr(G), _ptr(mask_words), ctx.k, float(ctx.lam), _ptr(ws),
                                             ctx.nb, _ptr(gl), _ptr(dI), ctypes.c_void_p(_stream())), "hssim backward")
        return dI, None, None, None, None


def hssim_loss(I, G, mask_words, k, lam=0.2):
    """(1 - lam) L1 + lam (1 - HSSIM) over the in-mask pixels; returns (loss, [loss, HSSIM, L1])."""
    return _HSSIMFn.apply(I, G, mask_words, k, lam)


class _RenderLossFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, rotations, opacities, sh, targets, rast, views, sh_degree, lam):
        out, state = rast.forward_raw(means, scales, rotations, opacities, sh, sh_degree, views)
        lay = view_layout(views, rast.cfg.tile_level)
        G = _f32(targets)
        parts = torch.empty((len(views), 3), dtype=torch.float32, device=means.device)
        loss_views = []
        for vi, (v, base) in enumerate(zip(views, lay.pix_base)):
            k = v["nside_log2"]
            n = npix(k)
            I, Gv = out["maps"][base:base + n], G[base:base + n]
            m = out["mask"][base // 32:(base + n) // 32]
            tab = _window_table(rast, v, m)
            nb = ctypes.c_size_t()
            L.check(L.lib().hpxgs_hssim_workspace_size(k, ctypes.byref(nb)), "hssim workspace")
            ws = torch.empty(nb.value, dtype=torch.uint8, device=means.device)
            L.check(L.lib().hpxgs_hssim_forward_table(_ptr(I), _ptr(Gv), _ptr(m), k, float(lam), _ptr(tab), _ptr(ws),
                                                      nb.value, _ptr(parts[vi]), ctypes.c_void_p(_stream())),
                    "hssim forward")
            loss_views.append((I, Gv, tab, ws))
        ctx.rast, ctx.state, ctx.loss_views, ctx.lam = rast, state, loss_views, lam
        ctx.mark_non_differentiable(parts)
        return parts[:, 0].sum(), parts

    @staticmethod
    def backward(ctx, gloss, gparts):
        dev = ctx.state["T"].device
        dl = _f32(gloss.reshape(1)) if gloss is not None else torch.ones(1, device=dev)
        grads = ctx.rast.backward_hssim_raw(ctx.state, [(I, G, tab, ws, dl) for I, G, tab, ws in ctx.loss_views],
                                            ctx.lam)
        ctx.state, ctx.loss_views = None, None
        return (*grads, None, None, None, None, None)


def _window_table(rast: Rasterizer, view, mask_words):
    """HSSIM window table of a view's order and mask; a mask depends on the camera's
    intrinsics only, so tables are kept per (order, camera) on the rasterizer."""
    key = (int(view["nside_log2"]), int(view.get("cam", L.CAM_FULL)), float(view.get("fov_x", 360.0)),
           float(view.get("fov_y") or view.get("fov_x", 360.0)), tuple(float(x) for x in view.get("pp", (0.0, 0.0))))
    cache = rast.__dict__.setdefault("_tables", {})
    if key not in cache:
        cache[key] = hssim_table(mask_words, key[0])
    return cache[key]


def render_loss(means, scales, rotations, opacities, sh, views, targets, rasterizer: Rasterizer | None = None,
                sh_degree=None, lam=0.2):
    """The training loss of Sec. 4.1 summed over `views`: sum_v (1 - lam) L1_v + lam (1 - HSSIM_v)
    against `targets` (packed like the maps), with the render and loss backward in one pass
    (hpxgs_backward_hssim: each pixel's dL/dI is formed inside the backward blend). Returns
    (loss, per-view [loss, HSSIM, L1]); the same values and gradients as render + hssim_loss
    per view, up to the order of the atomic sums."""
    rast = rasterizer or Rasterizer()
    if sh_degree is None:
        sh_degree = int(round(math.sqrt(sh.shape[1]))) - 1
    return _RenderLossFn.apply(means, scales, rotations, opacities, sh, targets, rast, list(views), sh_degree, lam)


def workspace_view(rast: Rasterizer, state) -> L.WorkspaceView:
    out = L.WorkspaceView()
    L.check(L.lib().hpxgs_workspace_inspect(state["g"].P, state["cviews"], state["nv"], ctypes.byref(rast.cfg),
                                            state["cap"], _ptr(state["ws"]), ctypes.byref(out)), "inspect")
    return out


class _DevArray:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


_TYPESTR = {torch.float32: "<f4", torch.int32: "<i4", torch.int64: "<i8", torch.uint8: "|u1"}


def device_array(ptr, n, dtype, device=None):
    """Copy n elements at a device pointer into a new tensor (for inspection in tests)."""
    if n == 0:
        return torch.empty(0, dtype=dtype, device=device or "cuda")
    view = torch.as_tensor(_DevArray(ptr, n, _TYPESTR[dtype]), device=device or "cuda")
    return view.clone()


# ----------------------------------------------------------------------------
# Training step under a CUDA graph
# ----------------------------------------------------------------------------
class GraphStep:
    """One training step (forward render of `views`, L1 + HSSIM loss per view
    against `targets`, loss backward, render backward) captured once into a CUDA
    graph and replayed. Inputs live in static tensors: write new parameter values
    or targets into `params` / `targets` in place before `replay()`.

    The pair capacity is fixed at capture (from a count on the initial inputs
    with headroom); after a replay `status` holds the device flags, and a
    capacity overflow means the graph must be built again with more room.
    `before_capture` (optional) runs right before the capture, e.g. to arm
    stage events that the graph then records at every replay;
    `launches_per_replay` is the number of library kernels in the graph.
    With `host_targets` (a pinned host tensor shaped like `targets`) every
    replay first copies it into `targets`, on a forked stream that overlaps the
    forward render; the loss waits for the copy.
    With `host_images` (one pinned host uint8 camera image [H, W, 3] per view, the
    form a camera delivers) every replay copies each image in on a forked stream and
    resamples it onto the view's HEALPix grid as that view's target
    (hpxgs_image_to_sphere_u8, Eq. supp_image_to_healpix), overlapping the forward render.
    With `fused` (the default) the loss backward runs inside the render backward
    (hpxgs_backward_hssim): each pixel's dL/dI is formed where the backward blend reads
    it instead of going through a dL/dmaps buffer."""

    def __init__(self, params, sh_degree, views, targets, rasterizer: Rasterizer, lam=0.2, headroom=1.25,
                 before_capture=None, host_targets=None, fused=True, host_images=None):
        self.params = [p.contiguous() for p in params]
        self.views = list(views)
        self.targets = targets.contiguous()
        self.rast = rasterizer
        self.lam = lam
        self.fused = fused
        self.sh_degree = sh_degree
        dev = self.params[0].device
        rasterizer.prepare(self.views)
        g = gaussians_struct(*self.params, sh_degree)
        cv = L.make_views(self.views)
        need = rasterizer.count_pairs(g, cv, len(self.views), dev)
        rasterizer.capacity = max(rasterizer.capacity or 0, int(need * headroom) + 4096)
        self.lay = view_layout(self.views, rasterizer.cfg.tile_level)
        self.order = [v["nside_log2"] for v in self.views]
        # HSSIM workspaces per view (the loss is evaluated per view on its part of the packed maps)
        self.hws = []
        for k in self.order:
            nb = ctypes.c_size_t()
            L.check(L.lib().hpxgs_hssim_workspace_size(k, ctypes.byref(nb)), "hssim ws")
            self.hws.append((torch.empty(nb.value, dtype=torch.uint8, device=dev), nb.value))
        self.losses = torch.zeros((len(self.views), 3), dtype=torch.float32, device=dev)
        self.dmaps = torch.zeros((self.lay.total_pix, 3), dtype=torch.float32, device=dev)
        self.graph = None
        self.out = None
        self.grads = None
        self.host_targets = host_targets
        if host_targets is not None:
            if not host_targets.is_pinned() or host_targets.shape != self.targets.shape:
                raise ValueError("host_targets must be a pinned host tensor shaped like targets")
            self.side = torch.cuda.Stream(device=dev)
        self.host_images = host_images
        if host_images is not None:
            if host_targets is not None or len(host_images) != len(self.views):
                raise ValueError("host_images takes one image per view, without host_targets")
            for im in host_images:
                if not im.is_pinned() or im.dtype != torch.uint8 or im.dim() != 3 or im.shape[2] != 3:
                    raise ValueError("host_images must be pinned uint8 host tensors [H, W, 3]")
            self.dev_images = [torch.empty(im.shape, dtype=torch.uint8, device=dev) for im in host_images]
            self.side = torch.cuda.Stream(device=dev)
        # warm up eagerly once (allocator pools, rho cache); the HSSIM window tables come from
        # the masks of that step (one per distinct order and camera); then capture
        self.tables = None
        self._step()
        torch.cuda.synchronize()
        self.tables = self._build_tables()
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            self._step()
        torch.cuda.current_stream(dev).wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        if before_capture is not None:
            before_capture()
        n0 = L.lib().hpxgs_launch_count()
        with torch.cuda.graph(self.graph):
            self._step()
        torch.cuda.synchronize()
        self.launches_per_replay = int(L.lib().hpxgs_launch_count() - n0)

    def _step(self):
        cur = torch.cuda.current_stream(self.targets.device)
        if self.host_targets is not None:
            self.side.wait_stream(cur)
            with torch.cuda.stream(self.side):
                self.targets.copy_(self.host_targets, non_blocking=True)
        if self.host_images is not None:
            from . import resample
            self.side.wait_stream(cur)
            with torch.cuda.stream(self.side):
                for v, k, base, him, dim in zip(self.views, self.order, self.lay.pix_base, self.host_images,
                                                self.dev_images):
                    dim.copy_(him, non_blocking=True)
                    resample.image_to_sphere_into(dim, v, k, self.targets[base:base + npix(k)], stream=self.side)
        out, state = self.rast.forward_raw(*self.params, self.sh_degree, self.views, check_status=False)
        if self.host_targets is not None or self.host_images is not None:
            cur.wait_stream(self.side)
        st = _stream()
        fused = self.fused and self.tables is not None
        loss_views = []
        for vi, (k, base) in enumerate(zip(self.order, self.lay.pix_base)):
            n = npix(k)
            I = out["maps"][base:base + n]
            G = self.targets[base:base + n]
            m = out["mask"][base // 32:(base + n) // 32]
            ws, nb = self.hws[vi]
            tab = self.tables[vi] if self.tables else None
            if tab is not None:
                L.check(L.lib().hpxgs_hssim_forward_table(_ptr(I), _ptr(G), _ptr(m), k, float(self.lam), _ptr(tab),
                                                          _ptr(ws), nb, _ptr(self.losses[vi]), ctypes.c_void_p(st)),
                        "hssim fwd")
                if fused:
                    loss_views.append((I, G, tab, ws, None))
                    continue
                L.check(L.lib().hpxgs_hssim_backward_table(_ptr(I), _ptr(G), _ptr(m), k, float(self.lam), _ptr(tab),
                                                           _ptr(ws), nb, None, _ptr(self.dmaps[base:base + n]),
                                                           ctypes.c_void_p(st)), "hssim bwd")
            else:
                L.check(L.lib().hpxgs_hssim_forward(_ptr(I), _ptr(G), _ptr(m), k, float(self.lam), _ptr(ws), nb,
                                                    _ptr(self.losses[vi]), ctypes.c_void_p(st)), "hssim fwd")
                L.check(L.lib().hpxgs_hssim_backward(_ptr(I), _ptr(G), _ptr(m), k, float(self.lam), _ptr(ws), nb,
                                                     None, _ptr(self.dmaps[base:base + n]), ctypes.c_void_p(st)),
                        "hssim bwd")
        if fused:
            self.grads = self.rast.backward_hssim_raw(state, loss_views, self.lam)
        else:
            self.grads = self.rast.backward_raw(state, self.dmaps)
        self.out = out
        self.state = state

    def _build_tables(self):
        cache, per_view = {}, []
        for vi, (v, k, base) in enumerate(zip(self.views, self.order, self.lay.pix_base)):
            key = (k, int(v["cam"]), float(v.get("fov_x", 360.0)), float(v.get("fov_y") or v.get("fov_x", 360.0)),
                   tuple(float(x) for x in v.get("pp", (0.0, 0.0))))
            if key not in cache:
                m = self.out["mask"][base // 32:(base + npix(k)) // 32]
                cache[key] = hssim_table(m, k)
            per_view.append(cache[key])
        return per_view

    def replay(self):
        self.graph.replay()
        return self.losses, self.grads

    @property
    def status(self):
        return self.out["status"]


# ----------------------------------------------------------------------------
# Autotuner over the launch parameters that do not change results
# ----------------------------------------------------------------------------
def autotune(make_step, candidates, reps=5, warmup=2):
    """Times `make_step(cfg_kwargs)()` for each candidate dict and returns
    (best_kwargs, {repr(kwargs): ms}). make_step builds (and may capture) a step
    for one candidate and returns a callable that runs it once on the current stream."""
    timings = {}
    best, best_ms = None, float("inf")
    for kw in candidates:
        try:
            run = make_step(kw)
        except L.HpxgsError:
            continue
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            run()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        timings[repr(sorted(kw.items()))] = ms
        if ms < best_ms:
            best, best_ms = kw, ms
    return best, timings


def default_candidates():
    out = []
    for b in (3, 4, 5):
        for bps in (0, 2):
            out.append(dict(tile_level=b, blocks_per_sm=bps))
    out.append(dict(tile_level=4, fwd_ppt=2))
    out.append(dict(tile_level=4, bwd_ppt=2))
    return out


def hssim_table(mask_words, k):
    """HEALPix-SSIM window table of a mask (order k): neighbour ids, window weights and
    1 / window sum per pixel, for the *_table forward and backward calls."""
    nb = ctypes.c_size_t()
    L.check(L.lib().hpxgs_hssim_table_size(k, ctypes.byref(nb)), "hssim table size")
    tab = torch.empty(nb.value, dtype=torch.uint8, device=mask_words.device)
    L.check(L.lib().hpxgs_hssim_table_build(_ptr(mask_words), k, _ptr(tab), nb.value, ctypes.c_void_p(_stream())),
            "hssim table")
    return tab
