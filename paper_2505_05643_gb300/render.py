"""Python front-end over the C ABI: a Renderer that owns the plan, the
workspace and the device plane table, and a torch.autograd.Function whose
forward and backward are the library's kernels.

Gaussian parameters live in one float32 device tensor of shape (rows, n):

  triangular front-end (11 rows):   mean[3], tri[6], logit, intensity
  scale/rotation front-end (12 rows): mean[3], log_scale[3], quat[4], logit, intensity
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import binding as B
from . import synth

ROWS = {B.UG_COV_TRI: 11, B.UG_COV_SCALE_ROT: 12}


def make_config(cov_param: int = B.UG_COV_TRI, cutoff: int = B.UG_CUTOFF_BOX, tile: int = 16,
                variant: int = 0, variant_bwd: int | None = None, **kw) -> B.ug_config:
    cfg = B.ug_config_default()
    cfg.cov_param = cov_param
    cfg.cutoff = cutoff
    cfg.tile = tile
    cfg.variant = variant
    cfg.variant_bwd = variant if variant_bwd is None else variant_bwd
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def pack_params(g: dict, cov_param: int) -> np.ndarray:
    """Gaussian dict (synth layout) -> (rows, n) float32 parameter matrix."""
    rows = [np.asarray(g["mean"], np.float32)]
    if cov_param == B.UG_COV_TRI:
        rows.append(np.asarray(g["tri"], np.float32))
    else:
        rows += [np.asarray(g["log_scale"], np.float32), np.asarray(g["quat"], np.float32)]
    rows += [np.asarray(g["logit"], np.float32)[None], np.asarray(g["intensity"], np.float32)[None]]
    return np.ascontiguousarray(np.concatenate(rows, axis=0))


def unpack_rows(mat, cov_param: int) -> dict:
    """(rows, n) matrix -> dict of row blocks (views)."""
    d = {"mean": mat[0:3]}
    if cov_param == B.UG_COV_TRI:
        d["tri"] = mat[3:9]
        k = 9
    else:
        d["log_scale"] = mat[3:6]
        d["quat"] = mat[6:10]
        k = 10
    d["logit"] = mat[k]
    d["intensity"] = mat[k + 1]
    return d


def _row_ptr(t: torch.Tensor, r: int) -> int:
    return t.data_ptr() + r * t.shape[1] * t.element_size()


def gaussians_struct(params: torch.Tensor, cov_param: int) -> B.ug_gaussians:
    g = B.ug_gaussians()
    g.mean = _row_ptr(params, 0)
    if cov_param == B.UG_COV_TRI:
        g.tri = _row_ptr(params, 3)
        k = 9
    else:
        g.log_scale = _row_ptr(params, 3)
        g.quat = _row_ptr(params, 6)
        k = 10
    g.opacity_logit = _row_ptr(params, k)
    g.intensity = _row_ptr(params, k + 1)
    return g


def grads_struct(grads: torch.Tensor, cov_param: int) -> B.ug_gaussian_grads:
    s = gaussians_struct(grads, cov_param)
    out = B.ug_gaussian_grads()
    for f, _ in B.ug_gaussians._fields_:
        setattr(out, f, getattr(s, f))
    return out


class Renderer:
    """One rendering problem: n Gaussians on a fixed set of plane sizes.

    Plane poses may change between calls (set_planes); sizes may not. The
    workspace grows automatically when a checked forward finds more records
    or instances than it holds.
    """

    def __init__(self, n: int, planes: dict, cfg: B.ug_config | None = None,
                 record_capacity: int | None = None, instance_capacity: int | None = None,
                 device: str | torch.device = "cuda"):
        B.load()
        self.cfg = cfg if cfg is not None else make_config()
        self.cov = int(self.cfg.cov_param)
        self.rows = ROWS[self.cov]
        self.n = int(n)
        self.device = torch.device(device)
        self.host_planes = synth.planes_to_struct(planes)
        self.P = len(self.host_planes)
        self.total_pixels = int((self.host_planes["pixel_offset"] +
                                 self.host_planes["width"].astype(np.int64) *
                                 self.host_planes["height"]).max())
        self.d_planes = torch.from_numpy(self.host_planes.view(np.uint8).copy()).to(self.device)
        pn = max(1, self.P * self.n)
        rec = record_capacity or int(min(pn, max(1 << 14, pn // 8)))
        inst = instance_capacity or int(min((1 << 31) - 1, max(1 << 18, 8 * rec)))
        self._alloc(rec, inst)
        self._status = torch.zeros(64, dtype=torch.uint8).pin_memory()

    # ------------------------------------------------------------- memory
    def _alloc(self, rec: int, inst: int):
        self.plan = B.ug_plan_init(self.cfg, self.n, self.host_planes, rec, inst)
        self.ws = torch.empty(int(self.plan.workspace_bytes), dtype=torch.uint8, device=self.device)
        assert self.ws.data_ptr() % 256 == 0

    def set_planes(self, planes):
        """Replace the plane poses (same sizes, same order) on the current stream."""
        arr = planes if isinstance(planes, np.ndarray) else synth.planes_to_struct(planes)
        if not (np.array_equal(arr["width"], self.host_planes["width"]) and
                np.array_equal(arr["height"], self.host_planes["height"]) and
                np.array_equal(arr["pixel_offset"], self.host_planes["pixel_offset"])):
            raise ValueError("plane sizes and offsets must not change")
        self.host_planes = arr.copy()
        self.d_planes.copy_(torch.from_numpy(arr.view(np.uint8).copy()), non_blocking=False)

    def new_image(self):
        return torch.empty(self.total_pixels, dtype=torch.float32, device=self.device)

    # ------------------------------------------------------------- calls
    def status(self, stream=None) -> dict:
        B.ug_read_status(self.plan, self.ws, self._status, stream)
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        st = B.ug_ws_status.from_buffer_copy(self._status.numpy().tobytes())
        return dict(status=st.status, detail=st.detail, records=st.records,
                    instances=st.instances, fp64_records=st.fp64_records,
                    box_pixels=st.box_pixels, evaluated_pairs=st.evaluated_pairs,
                    evaluated_pairs_bwd=st.evaluated_pairs_bwd)

    def preprocess(self, params: torch.Tensor, check: bool = True, stream=None):
        assert params.shape == (self.rows, self.n) and params.dtype == torch.float32
        g = gaussians_struct(params, self.cov)
        for _ in range(4):
            B.ug_preprocess(self.plan, g, self.d_planes, self.ws, stream)
            if not check:
                return
            st = self.status(stream)
            if st["status"] == B.UG_ERR_CAPACITY:
                rec = max(int(self.plan.record_capacity), int(st["records"] * 1.25) + 1024)
                inst = max(int(self.plan.instance_capacity), int(st["instances"] * 1.25) + 4096)
                if inst >= (1 << 31):
                    raise B.UgError(B.UG_ERR_CAPACITY, "more than 2^31 tile instances")
                self._alloc(min(rec, (1 << 31) - 1), inst)
                continue
            if st["status"] != B.UG_OK:
                raise B.UgError(st["status"], f"ug_preprocess (device, detail {st['detail']})")
            return st
        raise B.UgError(B.UG_ERR_CAPACITY, "ug_preprocess capacity")

    def forward(self, params: torch.Tensor, image=None, alpha=None, check: bool = True,
                stream=None):
        image = self.new_image() if image is None else image
        alpha = self.new_image() if alpha is None else alpha
        self.preprocess(params, check, stream)
        B.ug_bin_sort(self.plan, self.ws, stream)
        B.ug_render(self.plan, self.ws, image, alpha, stream)
        if check:
            st = self.status(stream)
            if st["status"] != B.UG_OK:
                raise B.UgError(st["status"], "ug_render (device)")
        return image, alpha

    def backward(self, params, image, alpha, grad_image, grads=None, check: bool = True,
                 stream=None):
        grads = torch.empty_like(params) if grads is None else grads
        B.ug_render_backward(self.plan, gaussians_struct(params, self.cov), self.d_planes, self.ws,
                             image, alpha, grad_image, grads_struct(grads, self.cov), stream)
        if check:
            st = self.status(stream)
            if st["status"] != B.UG_OK:
                raise B.UgError(st["status"], "ug_render_backward (device)")
        return grads

    def debug_views(self):
        """Host copies of the sorted keys (tile ids, with each instance's
        footprint-test byte apart), record ids, tile ranges, and the records'
        boxes, render data and planes of the last ug_bin_sort."""
        st = self.status()
        n_inst, n_rec = st["instances"], st["records"]
        kp, vp, rp, bp, ap, bbp, cp, pp = B.ug_debug_views(self.plan, self.ws)

        def grab(ptr, count, width=1):
            if count == 0:
                return np.zeros((0, width) if width > 1 else 0, np.uint32)
            base = self.ws.data_ptr()
            off = ptr - base
            t = self.ws[off:off + 4 * count * width].view(torch.int32).cpu().numpy().view(np.uint32)
            return t.reshape(-1, width) if width > 1 else t

        raw = grab(kp, n_inst)
        return dict(keys=raw & np.uint32(0x00FFFFFF), footprints=raw >> np.uint32(24),
                    records=grab(vp, n_inst),
                    ranges=grab(rp, int(self.plan.total_tiles), 2),
                    boxes=grab(bp, n_rec, 2), rec_a=grab(ap, n_rec, 4).view(np.float32),
                    rec_b=grab(bbp, n_rec, 4).view(np.float32),
                    rec_c=grab(cp, n_rec, 4).view(np.float32), rec_plane=grab(pp, n_rec),
                    status=st)


class UGRender(torch.autograd.Function):
    """image = UGRender.apply(params, renderer): forward = preprocess, sort,
    render; backward = the library's backward rasterizer and chain rule."""

    @staticmethod
    def forward(ctx, params, renderer: Renderer):
        image, alpha = renderer.forward(params.detach().contiguous())
        ctx.renderer = renderer
        ctx.save_for_backward(params, image, alpha)
        return image

    @staticmethod
    def backward(ctx, grad_image):
        params, image, alpha = ctx.saved_tensors
        grads = ctx.renderer.backward(params.detach().contiguous(), image, alpha,
                                      grad_image.contiguous())
        return grads, None
