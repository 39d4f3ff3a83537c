"""Frame pipeline over libags with PyTorch-managed device memory.

``Renderer`` owns the device buffers of one batch of views and enqueues the
four stages (preprocess, pair emission, sort, blend) on the current CUDA
stream -- one launch sequence per stage for all views, no host
synchronisation, so a whole frame can be captured in a CUDA graph.  PyTorch
only provides memory, streams and graphs; every step runs in libags kernels.
``AgsRender`` wraps forward and backward as a ``torch.autograd.Function``.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B

SCENE_KEYS = ("mean", "log_scale", "quat", "opacity_logit", "sh")


def scene_to_device(scene: dict, device="cuda") -> dict:
    return {k: torch.as_tensor(np.ascontiguousarray(scene[k]), dtype=torch.float32).to(device).contiguous()
            for k in SCENE_KEYS}


def spatial_order(scene: dict) -> tuple:
    """The scene stored along a Morton curve of its means (a setup step, not in
    the paper): returns (permuted scene, perm) with new[k] = old[perm[k]].  The
    Gaussians of a warp then lie close together, so a view culls them together;
    the images are those of the original order (only Gaussians of exactly equal
    depth in one tile can swap places)."""
    n = int(scene["opacity_logit"].shape[0])
    dev = scene["mean"].device
    sh_degree = int(round(math.sqrt(scene["sh"].shape[0]))) - 1
    codes = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    ws = torch.empty(B.ags_morton_workspace_bytes(), dtype=torch.uint8, device=dev)
    B.ags_morton_codes(scene, codes, ws)
    codes_alt = torch.empty_like(codes)
    vals, vals_alt = torch.empty_like(codes), torch.empty_like(codes)
    count = torch.full((1,), n, dtype=torch.int64, device=dev)
    status = torch.zeros(4, dtype=torch.int64, device=dev)
    ws_sort = torch.empty(B.ags_sort_workspace_bytes(max(n, 1)), dtype=torch.uint8, device=dev)
    alt = B.ags_sort32(codes, vals, codes_alt, vals_alt, count, max(n, 1), 0, 30, 8, None, 0, status, ws_sort,
                       flags=B.AGS_SORT_IDENTITY_VALUES)
    perm = (vals_alt if alt else vals)[:n]
    out = {k: torch.empty_like(v) for k, v in scene.items()}
    B.ags_gather_gaussians(scene, perm, sh_degree, out)
    B.ags_check(status)
    return out, perm


def tiles_per_view(cam: dict) -> int:
    return ((cam["width"] + B.AGS_TILE - 1) // B.AGS_TILE) * ((cam["height"] + B.AGS_TILE - 1) // B.AGS_TILE)


def tile_key_bits(views: int, tiles: int) -> int:
    """Bits of the largest tile key view * tiles + tile."""
    return max(1, int(views * tiles - 1).bit_length())


def key_end_bit(views: int, tiles: int) -> int:
    """Highest bit + 1 of a 64-bit (tile | depth) key: 32 depth bits plus the tile key."""
    return 32 + tile_key_bits(views, tiles)


def view_major_default(views: int, tiles: int, digit_bits: int) -> bool:
    """View-major tile keys (view << tile_bits | tile, sorted by the tile bits
    alone) for batches of views wherever they add no pair-sort pass (narrower
    digits even at the same pass count: C2 sort 0.68 -> 0.61 ms for 0.05 ms
    more depth pre-sort)."""
    tb = max(1, (tiles - 1).bit_length())
    return views > 1 and digit_plan(tb, digit_bits)[0] <= digit_plan(tile_key_bits(views, tiles), digit_bits)[0]


def digit_plan(bits: int, max_digit: int = 9) -> tuple:
    """(passes, digit_bits) covering `bits` key bits with the fewest passes."""
    passes = max(1, -(-bits // max_digit))
    return passes, max(4, -(-bits // passes))


class Renderer:
    """Buffers and launch sequence for rendering `scene` into `cams` (one batch)."""

    def __init__(self, scene: dict, cams: list, scale_mode: int = B.AGS_SCALE_PLAIN, K: float = 0.0, lut=None,
                 sh_degree: int = 3, bg=(0.0, 0.0, 0.0), capacity: int | None = None, digit_bits: int = 9,
                 headroom: float = 1.25, want_backward: bool = False, want_stats: bool = False,
                 presort: bool = True, pair_rank_or: bool = True, emit_two_pass: bool = True,
                 keep_state: bool = True, tile_test: int = B.AGS_TILE_SQUARE, view_major: bool | None = None,
                 blend_flags: int = 0, sort_wide: bool = False, depth_rank_or: bool = True,
                 depth_persistent: bool = True):
        self.scene = scene
        self.cams = list(cams)
        self.V = len(self.cams)
        self.n = int(scene["opacity_logit"].shape[0])
        self.W, self.H = self.cams[0]["width"], self.cams[0]["height"]
        self.T = tiles_per_view(self.cams[0])
        self.device = scene["mean"].device
        self.digit_bits = digit_bits
        self.presort = presort
        self.pair_rank_or = pair_rank_or
        self.emit_two_pass = emit_two_pass
        self.tile_test = tile_test
        self.blend_flags = int(blend_flags)      # AGS_BLEND_*: launch shape of the blend
        self.sort_flags = B.AGS_SORT_WIDE_BLOCK if sort_wide else 0
        # depth keys: the low digits of the float bits are close to uniform, so a
        # warp's keys mostly carry distinct digits -- the case of the atomic-OR ranking
        self.depth_rank_flags = B.AGS_SORT_RANK_OR if depth_rank_or else 0
        # the depth keys' capacity is every Gaussian-view, the count only the
        # visible ones (a few to a few tens of percent): resident blocks can take
        # the partitions of the count instead of one block per partition of the capacity
        self.depth_pass_flags = B.AGS_SORT_PERSISTENT if depth_persistent else 0
        self.depth_rank_flags |= self.depth_pass_flags
        self.emit_flags = B.AGS_EMIT_ELLIPSE if tile_test == B.AGS_TILE_ELLIPSE else 0
        self.tile_bits = max(1, (self.T - 1).bit_length())
        if view_major is None:
            view_major = view_major_default(self.V, self.T, digit_bits)
        self.view_major = bool(view_major) and presort and (self.V << self.tile_bits) <= (1 << 32)
        self.keep_state = keep_state or want_backward   # final_T / n_contrib for the backward
        self.set_params(scale_mode, K, lut, sh_degree, bg)
        dev, V, n = self.device, self.V, self.n
        self.proj = dict(splat=torch.empty(V * n * 12, dtype=torch.float32, device=dev),
                         depth=torch.empty(V * n, dtype=torch.float32, device=dev),
                         rect=torch.empty(V * n * 4, dtype=torch.int16, device=dev),
                         tiles_touched=torch.empty(V * n, dtype=torch.int32, device=dev),
                         flags=torch.empty(V * n, dtype=torch.uint8, device=dev))
        if presort:
            # depth pre-sort of the Gaussian-views that have pairs (32-bit depth
            # keys, compacted first); pairs then carry 32-bit tile keys and the
            # pair sort needs only the tile digits
            self.dkey = torch.empty(V * n, dtype=torch.int32, device=dev)
            self.dkey_alt = torch.empty(V * n, dtype=torch.int32, device=dev)
            self.order = torch.empty(V * n, dtype=torch.int32, device=dev)
            self.order_alt = torch.empty(V * n, dtype=torch.int32, device=dev)
            self.n_visible = torch.zeros(1, dtype=torch.int64, device=dev)
            self.ws_vis = torch.empty(B.ags_compact_workspace_bytes(n, V), dtype=torch.uint8, device=dev)
            self.ws_dsort = torch.empty(B.ags_sort_workspace_bytes(V * n), dtype=torch.uint8, device=dev)
            self.dsort_end = 32
        self.status = torch.zeros(4, dtype=torch.int64, device=dev)
        self.num_pairs = torch.zeros(1, dtype=torch.int64, device=dev)
        ews = B.ags_emit_tile_workspace_bytes(n, V) if presort else B.ags_emit_workspace_bytes(n, V)
        self.ws_emit = torch.empty(max(ews, 16), dtype=torch.uint8, device=dev)
        self.ranges = torch.empty(V * self.T * 2, dtype=torch.int32, device=dev)
        self.image = torch.empty(V, 3, self.H, self.W, dtype=torch.float32, device=dev)
        self.final_T = torch.empty(V, self.H, self.W, dtype=torch.float32, device=dev) if self.keep_state else None
        self.n_contrib = torch.empty(V, self.H, self.W, dtype=torch.int32, device=dev) if self.keep_state else None
        self.stats = torch.zeros(3, dtype=torch.int64, device=dev) if want_stats else None
        if capacity is None:
            capacity = max(1024, int(math.ceil(self.count_pairs() * headroom)))
        self.alloc_pairs(capacity)
        self.ws_bwd = None
        if want_backward:
            self.ws_bwd = torch.empty(B.ags_backward_workspace_bytes(n, V), dtype=torch.uint8, device=dev)
        self.generation = 0          # forwards enqueued so far (the blend state belongs to the last one)
        self.headroom = headroom

    # -- configuration -------------------------------------------------------
    def set_params(self, scale_mode=None, K=None, lut=None, sh_degree=None, bg=None):
        prev = getattr(self, "_pargs", dict(scale_mode=B.AGS_SCALE_PLAIN, K=0.0, lut=None, sh_degree=3,
                                            bg=(0.0, 0.0, 0.0), tile_test=getattr(self, "tile_test", 0),
                                            blend_flags=getattr(self, "blend_flags", 0)))
        args = dict(scale_mode=prev["scale_mode"] if scale_mode is None else scale_mode,
                    K=prev["K"] if K is None else K, lut=prev["lut"] if lut is None else lut,
                    sh_degree=prev["sh_degree"] if sh_degree is None else sh_degree,
                    bg=prev["bg"] if bg is None else bg, tile_test=prev["tile_test"], blend_flags=prev["blend_flags"])
        self._pargs = args
        self.params = B.params(**args)

    def alloc_pairs(self, capacity: int):
        if capacity >= B.AGS_MAX_PAIRS:
            raise ValueError("more than %d pairs in one batch; render fewer views at once" % B.AGS_MAX_PAIRS)
        dev = self.device
        self.capacity = int(capacity)
        kt = torch.int32 if self.presort else torch.int64
        self.keys = torch.empty(self.capacity, dtype=kt, device=dev)
        self.vals = torch.empty(self.capacity, dtype=torch.int32, device=dev)
        self.keys_alt = torch.empty(self.capacity, dtype=kt, device=dev)
        self.vals_alt = torch.empty(self.capacity, dtype=torch.int32, device=dev)
        self.ws_sort = torch.empty(B.ags_sort_workspace_bytes(self.capacity), dtype=torch.uint8, device=dev)

    def count_pairs(self) -> int:
        """Preprocess + emission with zero capacity; returns the pair count (synchronises)."""
        B.ags_status_reset(self.status)
        B.ags_preprocess(self.scene, self.cams, self.params, self.proj, self.status)
        B.ags_emit_pairs(self.proj, self.n, self.cams, None, None, 0, self.num_pairs, self.status, self.ws_emit,
                         flags=self.emit_flags)
        B.ags_status_reset(self.status)
        return int(self.num_pairs.item())

    @property
    def end_bit(self) -> int:
        """Highest sorted key bit + 1: the tile key (32-bit keys; the tile alone with
        view-major keys) or tile | depth (64-bit keys)."""
        if self.presort:
            return self.tile_bits if self.view_major else tile_key_bits(self.V, self.T)
        return key_end_bit(self.V, self.T)

    def sort_plan(self) -> tuple:
        """(passes, digit_bits) of the pair sort."""
        if self.presort:
            return digit_plan(self.end_bit, self.digit_bits)
        return max(1, -(-self.end_bit // self.digit_bits)), self.digit_bits

    def launches_per_forward(self) -> int:
        """libags kernel launches of one forward (memsets are not kernels)."""
        ellipse = self.tile_test == B.AGS_TILE_ELLIPSE
        # preprocess (+ the ellipse test's tile count), blend
        n = 1 + (1 if ellipse else 0) + 1
        # pair sort: histogram, digit scan, passes, ranges initialisation and fix-up
        n += 2 + self.sort_plan()[0] + 2
        if self.presort:
            # emission: two passes (scan, pairs) or one fused pass
            n += 2 if self.emit_two_pass else 1
            # compaction (count, scan, write), then (histogram, digit scan, passes)
            n += 3 + 2 + digit_plan(self.dsort_end, self.digit_bits)[0]
            if self.view_major:   # view keys, then (histogram, digit scan, one pass)
                n += 1 + 3
        else:
            n += 1
        return n

    # -- stages ---------------------------------------------------------------
    def preprocess(self):
        B.ags_preprocess(self.scene, self.cams, self.params, self.proj, self.status)

    def depth_sort(self):
        """Stable sort of the Gaussian-views with pairs by depth: the emission
        order (each view's Gaussians in depth order, equal depths in index order)."""
        if self.presort:
            B.ags_compact_visible(self.proj, self.n, self.V, self.dkey, self.order, self.n_visible, self.status,
                                  self.ws_vis)
            passes, db = digit_plan(self.dsort_end, self.digit_bits)
            alt = B.ags_sort32(self.dkey, self.order, self.dkey_alt, self.order_alt, self.n_visible,
                               self.V * self.n, 0, self.dsort_end, db, None, 0, self.status, self.ws_dsort,
                               flags=B.AGS_SORT_DISCARD_KEYS | self.depth_rank_flags | self.sort_flags)
            self.emit_order = self.order_alt if alt else self.order
            if self.view_major:
                # then stably by view: the views one after the other, each in
                # depth order (the depth keys are spent; their buffers hold the views)
                other = self.order if alt else self.order_alt
                vb = max(1, (self.V - 1).bit_length())
                B.ags_view_keys(self.emit_order, self.n_visible, self.V * self.n, self.n, self.dkey)
                alt2 = B.ags_sort32(self.dkey, self.emit_order, self.dkey_alt, other, self.n_visible, self.V * self.n,
                                    0, vb, min(9, max(4, vb)), None, 0, self.status, self.ws_dsort,
                                    flags=B.AGS_SORT_DISCARD_KEYS | self.depth_rank_flags | self.sort_flags)
                self.emit_order = other if alt2 else self.emit_order

    def emit(self):
        if self.presort:
            B.ags_emit_tile_pairs(self.proj, self.n, self.cams, self.keys, self.vals, self.capacity,
                                  self.num_pairs, self.status, self.ws_emit, order=self.emit_order,
                                  order_count=self.n_visible,
                                  flags=self.emit_flags | (0 if self.emit_two_pass else B.AGS_EMIT_SINGLE_PASS)
                                  | (B.AGS_EMIT_VIEW_SHIFT if self.view_major else 0))
        else:
            B.ags_emit_pairs(self.proj, self.n, self.cams, self.keys, self.vals, self.capacity, self.num_pairs,
                             self.status, self.ws_emit, flags=self.emit_flags)

    def sort(self):
        """Stable sort of the pairs by tile (and depth); only the values and the
        per-tile ranges are kept."""
        _, db = self.sort_plan()
        flags = B.AGS_SORT_DISCARD_KEYS | (B.AGS_SORT_RANK_OR if self.pair_rank_or else 0) | self.sort_flags
        if self.view_major:
            alt = B.ags_sort_tiles(self.keys, self.vals, self.keys_alt, self.vals_alt, self.num_pairs, self.capacity,
                                   self.tile_bits, db, self.ranges, self.V, self.T, self.status, self.ws_sort,
                                   flags=flags)
        else:
            fn = B.ags_sort32 if self.presort else B.ags_sort
            alt = fn(self.keys, self.vals, self.keys_alt, self.vals_alt, self.num_pairs, self.capacity, 0,
                     self.end_bit, db, self.ranges, self.V * self.T, self.status, self.ws_sort, flags=flags)
        self.sorted_vals = self.vals_alt if alt else self.vals

    def rasterize(self, max_T=None):
        B.ags_rasterize(self.proj, self.n, self.sorted_vals, self.ranges, self.cams, self.params, self.image,
                        self.final_T, self.n_contrib, self.status, max_T=max_T, stats=self.stats)

    def forward(self, max_T=None):
        """Enqueue the whole frame on the current stream; returns the image tensor."""
        self.generation += 1
        self.preprocess()
        self.depth_sort()
        self.emit()
        self.sort()
        self.rasterize(max_T)
        return self.image

    def forward_fitted(self, max_T=None):
        """forward(), then synchronise and check the status block; when the
        pairs overflowed the capacity (the scene moved since the buffers were
        sized), grow the capacity to the needed count times the headroom and
        render again.  Raises on any other device-side error."""
        img = self.forward(max_T)
        code, detail = B.ags_check(self.status, raise_on_error=False)
        if code == B.AGS_ERR_CAPACITY:
            B.ags_status_reset(self.status)
            self.alloc_pairs(max(int(math.ceil(int(detail) * self.headroom)), self.capacity + 1))
            img = self.forward(max_T)
            code, detail = B.ags_check(self.status, raise_on_error=False)
        if code not in (B.AGS_OK, B.AGS_ERR_NUMERIC):
            raise B.AgsError(code, "render", detail)
        return img

    def capture(self) -> "torch.cuda.CUDAGraph":
        """Capture one whole forward (every stage, all views) in a CUDA graph.

        Replaying the graph re-renders from the current contents of the scene
        tensors and writes the same output buffers; the pair capacity must
        cover the pairs of every replay (an overflow is reported in the status
        block, as for an eager forward)."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):          # warm-up outside the capture
            self.forward()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.forward()
        return graph

    def backward(self, dL_dimage: torch.Tensor, grads: dict | None = None) -> dict:
        if not self.keep_state:
            raise RuntimeError("this renderer was built with keep_state=False: its forward keeps no blend state")
        if self.ws_bwd is None:
            self.ws_bwd = torch.empty(B.ags_backward_workspace_bytes(self.n, self.V), dtype=torch.uint8,
                                      device=self.device)
        if grads is None:
            grads = {k: torch.empty_like(self.scene[k]) for k in SCENE_KEYS}
        B.ags_rasterize_backward(self.scene, self.cams, self.params, self.proj, self.sorted_vals, self.ranges,
                                 self.final_T, self.n_contrib, dL_dimage.contiguous(), grads, self.status,
                                 self.ws_bwd)
        return grads

    def check(self):
        """Synchronise and raise on a device-side error (capacity, timeout)."""
        code, detail = B.ags_check(self.status, raise_on_error=False)
        if code not in (B.AGS_OK, B.AGS_ERR_NUMERIC):
            raise B.AgsError(code, "render", detail)
        return code, detail

    def pairs(self) -> int:
        return int(self.num_pairs.item())


class HostPipeline:
    """Frames from parameters in (pinned) host memory to images in host memory,
    double-buffered.  A frame uploads its parameters on an upload stream,
    renders them (a CUDA graph of the whole forward) on the caller's stream and
    downloads its images on a download stream.  With two sets of device
    buffers, the upload of the next frame and the download of the previous one
    run while a frame renders.  Every frame still copies all of its inputs and
    its whole result; nothing is kept from one frame to the next.  Takes the
    Renderer's arguments and twice its device memory."""

    def __init__(self, scene: dict, cams: list, *args, **kwargs):
        self.renderers = [Renderer({k: v.clone() for k, v in scene.items()}, cams, *args, **kwargs)
                          for _ in range(2)]
        self.graphs = [r.capture() for r in self.renderers]
        self.up, self.down = torch.cuda.Stream(), torch.cuda.Stream()
        cur = torch.cuda.current_stream()
        self.uploaded = [torch.cuda.Event() for _ in range(2)]
        self.rendered = [torch.cuda.Event() for _ in range(2)]
        self.downloaded = [torch.cuda.Event() for _ in range(2)]
        for e in self.rendered + self.downloaded:     # both slots free
            e.record(cur)
        self.frames = 0

    def submit(self, host_params: dict, host_image: torch.Tensor):
        """Enqueue one frame: upload `host_params` (pinned, the scene's keys and
        shapes), render, download into `host_image` (pinned, [views][3][H][W]).
        Returns at once; the host buffers must stay untouched until wait()."""
        slot = self.frames % 2
        self.frames += 1
        r = self.renderers[slot]
        cur = torch.cuda.current_stream()
        self.up.wait_event(self.rendered[slot])       # the slot's parameters are no longer read
        with torch.cuda.stream(self.up):
            for k, v in host_params.items():
                r.scene[k].copy_(v, non_blocking=True)
            self.uploaded[slot].record(self.up)
        cur.wait_event(self.uploaded[slot])
        cur.wait_event(self.downloaded[slot])         # the slot's previous images have left
        self.graphs[slot].replay()
        self.rendered[slot].record(cur)
        self.down.wait_event(self.rendered[slot])
        with torch.cuda.stream(self.down):
            host_image.copy_(r.image, non_blocking=True)
            self.downloaded[slot].record(self.down)

    def begin(self):
        """Order the frames submitted from now on after the work already queued
        on the caller's stream (e.g. an event that starts a timed region)."""
        cur = torch.cuda.current_stream()
        self.up.wait_stream(cur)
        self.down.wait_stream(cur)

    def wait(self):
        """Make the caller's stream wait for every submitted frame's download."""
        cur = torch.cuda.current_stream()
        for e in self.downloaded:
            cur.wait_event(e)

    def check(self):
        for r in self.renderers:
            r.check()


class AgsRender(torch.autograd.Function):
    """image = render(params) through libags; the backward runs the blend and
    preprocess adjoints with the pair lists of this forward held fixed (the
    AdaGScale selection is piecewise constant in the parameters).

    The forward synchronises once to check the status block (growing the
    pair capacity and rendering again if the pairs overflowed it).  The blend
    state the backward needs lives in the renderer, so the renderer must not
    run another forward between this forward and its backward: the backward
    raises if it did."""

    @staticmethod
    def forward(ctx, mean, log_scale, quat, opacity_logit, sh, renderer: Renderer):
        if not renderer.keep_state:
            raise RuntimeError("AgsRender needs a renderer built with keep_state=True (or want_backward=True)")
        renderer.scene = dict(mean=mean.detach().contiguous(), log_scale=log_scale.detach().contiguous(),
                              quat=quat.detach().contiguous(), opacity_logit=opacity_logit.detach().contiguous(),
                              sh=sh.detach().contiguous())
        img = renderer.forward_fitted()
        ctx.renderer = renderer
        ctx.generation = renderer.generation
        return img.clone()

    @staticmethod
    def backward(ctx, grad_image):
        r = ctx.renderer
        if r.generation != ctx.generation:
            raise RuntimeError("the renderer ran another forward after this one: its blend state belongs to that "
                               "frame now; render the frames to differentiate with separate renderers")
        g = r.backward(grad_image)
        r.check()
        return g["mean"], g["log_scale"], g["quat"], g["opacity_logit"], g["sh"], None
