"""Continuous-batching render server over a resident Gaussian scene.

Requests (a camera view: pose, Nside, camera kind and FoV) arrive over time.
The server keeps the scene on the device and, as stream slots and memory free
up, admits the waiting requests in arrival order into a batch: up to
`max_views` views and `max_pixels` pixels, and only while the batch's memory
(workspace with its tile-list capacity, plus the output maps) fits in what is
left of `budget_bytes`. The tile-list capacity of a request is predicted from
the pair counts seen so far for its (Nside, camera kind), with headroom; the
forward reports the exact count on the device, and a batch whose lists did not
fit is rendered again with the exact capacity. Batches run on `slots` CUDA
streams, so later requests overlap with earlier ones on the device. A request's
latency runs from its arrival to the host seeing its batch's completion event.

`plain=True` serves one request at a time on one stream (no batching, no overlap)
for comparison. Every batch is one hpxgs_forward call; results do not depend on
how requests are grouped (a test checks a request alone against the same request
inside a mix).
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L
from . import raster as R


@dataclass
class Stats:
    latencies_ms: list = field(default_factory=list)
    served: int = 0
    batches: int = 0
    reruns: int = 0
    pixels: int = 0
    wall_s: float = 0.0
    peak_bytes: int = 0

    def summary(self):
        lat = np.asarray(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"served": self.served, "batches": self.batches, "reruns": self.reruns,
                "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "mean_ms": round(float(lat.mean()), 3), "throughput_rps": round(self.served / max(self.wall_s, 1e-9), 2),
                "mpix_per_s": round(self.pixels / max(self.wall_s, 1e-9) / 1e6, 2),
                "mean_batch": round(self.served / max(self.batches, 1), 2), "peak_budget_bytes": int(self.peak_bytes)}


class RenderServer:
    def __init__(self, params, sh_degree, budget_bytes=8 << 30, slots=3, max_views=8, max_pixels=64 << 20,
                 headroom=1.3, tile_level=0):
        self.params = [p.contiguous() for p in params]
        self.sh_degree = sh_degree
        self.budget = int(budget_bytes)
        self.slots = slots
        self.max_views = max_views
        self.max_pixels = max_pixels
        self.headroom = headroom
        self.tile_level = tile_level
        self.dev = self.params[0].device
        self.g = R.gaussians_struct(*self.params, sh_degree)
        self.cfg_by_level = {b: L.default_config(tile_level=b) for b in (3, 4, 5)}
        self.cfg = self.cfg_by_level[tile_level or 4]
        self.adaptive = tile_level is None or tile_level == 0
        self.pairs_per_pixel = {}          # (k, kind, tile level) -> running max of pairs per map pixel
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(slots)]

    def level_for(self, views):
        """Tile level of a batch: 5 (1024-pixel tiles) once a view reaches Nside 1024, else 4.
        Maps do not depend on it; it trades pair count against per-tile list length."""
        if not self.adaptive:
            return self.tile_level
        return 5 if max(v["nside_log2"] for v in views) >= 10 else 4

    # ---- memory model -------------------------------------------------------
    # Pair densities are kept per (Nside, camera kind, tile level): a batch's tile level
    # follows its largest view, so a view's list size is learned and predicted at the
    # level of the batch it runs in.
    def _estimate_pairs(self, v, level=None):
        level = self.level_for([v]) if level is None else level
        ppx = self.pairs_per_pixel.get((v["nside_log2"], v["cam"], level))
        if ppx is None:
            return None
        return int(ppx * R.npix(v["nside_log2"]) * self.headroom) + 4096

    def _learn(self, views, n_pairs):
        level = self.level_for(views)
        px = sum(R.npix(v["nside_log2"]) for v in views)
        ppx = n_pairs / max(px, 1)
        for v in views:
            key = (v["nside_log2"], v["cam"], level)
            self.pairs_per_pixel[key] = max(self.pairs_per_pixel.get(key, 0.0), ppx)

    def _ensure_known(self, v, levels):
        """Count the pairs of view v alone at each of `levels`, where not known yet."""
        for level in levels:
            if self._estimate_pairs(v, level) is None:
                self._count([v], level)

    def _batch_bytes(self, views, cap):
        cv = L.make_views(views)
        n = ctypes.c_size_t()
        cfg = self.cfg_by_level[self.level_for(views)]
        L.check(L.lib().hpxgs_forward_workspace_size(self.g.P, cv, len(views), ctypes.byref(cfg), int(cap),
                                                     ctypes.byref(n)), "workspace size")
        px = sum(R.npix(v["nside_log2"]) for v in views)
        return n.value + px * (12 + 4 + 4) + px // 8 + 64, cv

    def _count(self, views, level=None):
        """Exact pair count of a batch at a tile level (synchronises): used for a request kind
        never seen before."""
        level = self.level_for(views) if level is None else level
        cv = L.make_views(views)
        ws_n = ctypes.c_size_t()
        cfg = self.cfg_by_level[level]
        L.check(L.lib().hpxgs_forward_workspace_size(self.g.P, cv, len(views), ctypes.byref(cfg), 0,
                                                     ctypes.byref(ws_n)), "workspace size")
        ws = torch.empty(ws_n.value, dtype=torch.uint8, device=self.dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=self.dev)
        st = torch.zeros(1, dtype=torch.int32, device=self.dev)
        s = torch.cuda.current_stream(self.dev).cuda_stream
        L.check(L.lib().hpxgs_count_pairs(ctypes.byref(self.g), cv, len(views), ctypes.byref(cfg),
                                          ctypes.c_void_p(ws.data_ptr()), ws_n.value, ctypes.c_void_p(cnt.data_ptr()),
                                          ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(s)), "count")
        n = int(cnt.item())
        px = sum(R.npix(v["nside_log2"]) for v in views)
        for v in views:
            key = (v["nside_log2"], v["cam"], level)
            self.pairs_per_pixel[key] = max(self.pairs_per_pixel.get(key, 0.0), n / max(px, 1))
        return n

    # ---- one batch ------------------------------------------------------------
    def _launch(self, views, cap, stream):
        nbytes, cv = self._batch_bytes(views, cap)
        cfg = self.cfg_by_level[self.level_for(views)]
        lay = R.view_layout(views, cfg.tile_level)
        with torch.cuda.stream(stream):
            ws_n = ctypes.c_size_t()
            L.check(L.lib().hpxgs_forward_workspace_size(self.g.P, cv, len(views), ctypes.byref(cfg), int(cap),
                                                         ctypes.byref(ws_n)), "workspace size")
            ws = torch.empty(ws_n.value, dtype=torch.uint8, device=self.dev)
            maps = torch.empty((lay.total_pix, 3), dtype=torch.float32, device=self.dev)
            T = torch.empty(lay.total_pix, dtype=torch.float32, device=self.dev)
            last = torch.empty(lay.total_pix, dtype=torch.int32, device=self.dev)
            mask = torch.empty(lay.total_pix // 32, dtype=torch.int32, device=self.dev)
            status = torch.zeros(1, dtype=torch.int32, device=self.dev)
            p = lambda t: ctypes.c_void_p(t.data_ptr())
            L.check(L.lib().hpxgs_forward(ctypes.byref(self.g), cv, len(views), ctypes.byref(cfg), p(ws),
                                          ws_n.value, int(cap), p(maps), p(T), p(last), p(mask), None, None, p(status),
                                          ctypes.c_void_p(stream.cuda_stream)), "forward")
            ev = torch.cuda.Event()
            ev.record(stream)
        return dict(views=views, cap=cap, ws=ws, maps=maps, T=T, last=last, mask=mask, status=status, event=ev,
                    bytes=nbytes, layout=lay)

    def render_batch(self, views, stream=None):
        """Render a list of views now (synchronously) and return the packed outputs."""
        stream = stream or torch.cuda.current_stream(self.dev)
        cap = self._estimate_pairs_batch(views)
        job = self._launch(views, cap, stream)
        job["event"].synchronize()
        if int(job["status"].item()) & L.F_CAPACITY:
            n = self._workspace_pairs(job)
            self._learn(views, n)
            job = self._launch(views, int(n * self.headroom) + 4096, stream)
            job["event"].synchronize()
        return job

    def _estimate_pairs_batch(self, views):
        level = self.level_for(views)
        tot = 0
        for v in views:
            e = self._estimate_pairs(v, level)
            if e is None:
                self._count([v], level)
                e = self._estimate_pairs(v, level)
            tot += e
        return tot

    def _workspace_pairs(self, job):
        wv = L.WorkspaceView()
        L.check(L.lib().hpxgs_workspace_inspect(self.g.P, L.make_views(job["views"]), len(job["views"]),
                                                ctypes.byref(self.cfg_by_level[self.level_for(job["views"])]), job["cap"],
                                                ctypes.c_void_p(job["ws"].data_ptr()), ctypes.byref(wv)), "inspect")
        return int(R.device_array(wv.n_pairs, 1, torch.int32, self.dev).item()) & 0xffffffff

    # ---- the request loop ---------------------------------------------------------
    def run(self, requests, plain=False, keep_outputs=False, time_limit_s=120.0):
        """Serve `requests` (dicts with 'arrival' seconds and 'view') in real time."""
        # learn the pair density of every request kind up front, at its own tile level and, when
        # the stream holds a view that lifts a batch to level 5, at that level too
        top = self.level_for([r["view"] for r in requests]) if requests else None
        for r in requests:
            self._ensure_known(r["view"], {self.level_for([r["view"]]), top})
        torch.cuda.synchronize()
        pending = collections.deque(sorted(requests, key=lambda r: r["arrival"]))
        waiting = collections.deque()
        slots = 1 if plain else self.slots
        max_views = 1 if plain else self.max_views
        free = list(range(slots))
        inflight = []
        used = 0
        stats = Stats()
        results = {}
        t0 = time.perf_counter()
        while pending or waiting or inflight:
            now = time.perf_counter() - t0
            if now > time_limit_s:
                break
            while pending and pending[0]["arrival"] <= now:
                waiting.append(pending.popleft())
            # completions
            still = []
            for job in inflight:
                if job["event"].query():
                    if int(job["status"].item()) & L.F_CAPACITY:       # lists did not fit: learn and run again
                        n = self._workspace_pairs(job)
                        self._learn(job["views"], n)
                        stats.reruns += 1
                        used -= job["bytes"]
                        cap = int(n * self.headroom) + 4096
                        re = self._launch(job["views"], cap, self.streams[job["slot"]])
                        re.update(slot=job["slot"], reqs=job["reqs"])
                        used += re["bytes"]
                        still.append(re)
                        continue
                    tdone = time.perf_counter() - t0
                    for r in job["reqs"]:
                        stats.latencies_ms.append((tdone - r["arrival"]) * 1e3)
                        if keep_outputs:
                            results[r["id"]] = job
                    stats.served += len(job["reqs"])
                    stats.pixels += job["layout"].total_pix
                    stats.batches += 1
                    used -= job["bytes"]
                    free.append(job["slot"])
                else:
                    still.append(job)
            inflight = still
            # admission
            while free and waiting:
                batch, views, cap = [], [], 0
                px = 0
                while waiting and len(batch) < max_views:
                    v = waiting[0]["view"]
                    cand = views + [v]
                    level = self.level_for(cand)
                    cap_c = sum(self._estimate_pairs(x, level) for x in cand)   # at the batch's level
                    npx = R.npix(v["nside_log2"])
                    nb, _ = self._batch_bytes(cand, cap_c)
                    if batch and (px + npx > self.max_pixels or used + nb > self.budget):
                        break
                    if not batch and used + nb > self.budget and inflight:
                        break                                  # wait for memory to free up
                    batch.append(waiting.popleft()); views.append(v); cap = cap_c; px += npx
                if not batch:
                    break
                slot = free.pop()
                job = self._launch(views, cap, self.streams[slot])
                job.update(slot=slot, reqs=batch)
                used += job["bytes"]
                stats.peak_bytes = max(stats.peak_bytes, used)
                inflight.append(job)
            if not (pending and pending[0]["arrival"] <= time.perf_counter() - t0) and inflight and not free:
                time.sleep(5e-5)
            elif not waiting and not inflight and pending:
                time.sleep(max(0.0, min(1e-3, pending[0]["arrival"] - (time.perf_counter() - t0))))
        stats.wall_s = time.perf_counter() - t0
        return stats, results
