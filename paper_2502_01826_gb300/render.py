"""PyTorch-facing wrapper of libgsrf.so.

PyTorch supplies device memory and the current stream; every computation runs in the
library's kernels through the C ABI (``_lib``).  Parameters are the raw learnable
tensors of Sec. 4.2: means [K,3], log_scales [K,3], quats [K,4] (w,x,y,z),
opacity_logit [K], coeffs [K,16,2], phase_b [K].
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logit", "coeffs", "phase_b")


def make_grid(n_az: int, n_el: int, az0_deg: float = 0.0, daz_deg: float | None = None,
              el0_deg: float = 0.0, del_deg: float | None = None, r_rx: float = 1.0,
              eps_T: float = 1e-4, alpha_max: float = 0.99, tile_w: int = 16, tile_h: int = 16) -> L.gsrf_grid:
    """Receiving-plane grid; defaults span azimuth [0, 360) and elevation [0, 90)."""
    if daz_deg is None:
        daz_deg = 360.0 / n_az
    if del_deg is None:
        del_deg = 90.0 / n_el
    return L.gsrf_grid(n_az, n_el, az0_deg, daz_deg, el0_deg, del_deg, r_rx, eps_T, alpha_max, tile_w, tile_h)


def grid_from_spec(spec: dict, **kw) -> L.gsrf_grid:
    args = dict(spec)
    args.update(kw)
    return make_grid(**args)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def gaussians_struct(p: dict) -> L.gsrf_gaussians:
    for k in PARAM_NAMES[:5]:
        t = p[k]
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("%s must be a contiguous float32 CUDA tensor" % k)
    pb = p.get("phase_b")
    n = p["means"].shape[0]
    return L.gsrf_gaussians(n, p["means"].data_ptr(), p["log_scales"].data_ptr(), p["quats"].data_ptr(),
                            p["opacity_logit"].data_ptr(), p["coeffs"].data_ptr(),
                            None if pb is None else pb.data_ptr())


def to_device(params: dict, device="cuda") -> dict:
    return {k: torch.as_tensor(params[k]).to(device=device, dtype=torch.float32).contiguous()
            for k in PARAM_NAMES if k in params and params[k] is not None}


class Renderer:
    """One render problem (one scene, n_rx receivers, one transmitter) with its workspace.

    The workspace holds every intermediate (records, sort buffers, pair lists); it is
    sized once and reused.  ``pair_capacity`` grows on demand when a bin reports that
    it needed more room (``ensure_capacity``)."""

    def __init__(self, n_gauss: int, n_rx: int, grid: L.gsrf_grid, f0_hz: float, df_hz: float = 0.0,
                 n_f: int = 1, pair_capacity: int | None = None, device="cuda", ray_block_w: int = 0,
                 stage: int = 0, ckpt_every: int = 0, ckpt_slots: int = 0, variant: int = 0, fle_degree: int = 0):
        self.device = torch.device(device)
        if pair_capacity is None:
            pair_capacity = max(1024, 8 * n_gauss * n_rx)
        self.plan = L.gsrf_plan(n_gauss, n_rx, n_f, f0_hz, df_hz, grid, int(pair_capacity), int(ray_block_w),
                                int(stage), int(ckpt_every), int(ckpt_slots), int(variant), int(fle_degree))
        self._alloc()

    def _alloc(self):
        nbytes = C.c_size_t()
        L.call("gsrf_workspace_size", C.byref(self.plan), C.byref(nbytes))
        self.ws_bytes = nbytes.value
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        assert self.ws.data_ptr() % 256 == 0

    @property
    def n_rx(self):
        return self.plan.n_rx

    def out_shape(self):
        g = self.plan.grid
        return (self.plan.n_rx, self.plan.n_f, g.n_el, g.n_az, 2)

    def ray_state(self):
        n = L.load().gsrf_ray_state_bytes(C.byref(self.plan))
        return torch.empty(n, dtype=torch.uint8, device=self.device)

    def project(self, params: dict, rx: torch.Tensor, tx: torch.Tensor, stream=None):
        gs = gaussians_struct(params)
        L.call("gsrf_project", C.byref(self.plan), C.byref(gs), _ptr(rx), _ptr(tx), _ptr(self.ws),
               self.ws_bytes, _stream(stream))

    def bin(self, stream=None):
        L.call("gsrf_bin", C.byref(self.plan), _ptr(self.ws), self.ws_bytes, _stream(stream))

    def render_fwd(self, params: dict, out: torch.Tensor | None = None, ray_state=None, stream=None):
        if out is None:
            out = torch.empty(self.out_shape(), dtype=torch.float32, device=self.device)
        gs = gaussians_struct(params)
        L.call("gsrf_render_fwd", C.byref(self.plan), C.byref(gs), _ptr(self.ws), self.ws_bytes,
               _ptr(out), _ptr(ray_state), _stream(stream))
        return out

    def forward(self, params: dict, rx: torch.Tensor, tx: torch.Tensor, out=None, ray_state=None,
                stream=None):
        if out is None:
            out = torch.empty(self.out_shape(), dtype=torch.float32, device=self.device)
        gs = gaussians_struct(params)
        L.call("gsrf_render", C.byref(self.plan), C.byref(gs), _ptr(rx), _ptr(tx), _ptr(self.ws),
               self.ws_bytes, _ptr(out), _ptr(ray_state), _stream(stream))
        return out

    def autotune(self, params: dict, rx: torch.Tensor, tx: torch.Tensor, reps: int = 3, stream=None,
                 training: bool = False):
        """Measure the work splits on this problem (gsrf_autotune) and adopt the fastest:
        the plan's tile shape, ray block and stage change and the workspace is re-allocated
        (and its pair capacity re-fitted) for them.  training=True times forward + backward
        renders (scratch upstream and gradient buffers).  Returns (best, every measurement)
        as dicts of tile_w, tile_h, ray_block_w, stage, project_bin_ms, render_ms."""
        nbytes = C.c_size_t()
        L.call("gsrf_autotune_workspace_size", C.byref(self.plan), C.byref(nbytes))
        ws = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        out = torch.empty(self.out_shape(), dtype=torch.float32, device=self.device)
        cap = 128
        results = (L.gsrf_tune_result * cap)()
        n = C.c_int32()
        best = L.gsrf_tune_result()
        gs = gaussians_struct(params)
        bwd, keep = None, []
        if training:
            state = self.ray_state()
            up = torch.randn(self.out_shape(), dtype=torch.float32, device=self.device)
            gr = {k: torch.zeros_like(v) for k, v in params.items() if v is not None}
            keep = [state, up, gr]
            bwd = L.gsrf_tune_backward(_ptr(state), _ptr(up), *[_ptr(gr.get(k)) for k in PARAM_NAMES])
        L.call("gsrf_autotune", C.byref(self.plan), C.byref(gs), _ptr(rx), _ptr(tx), _ptr(ws), nbytes.value,
               _ptr(out), C.byref(bwd) if bwd is not None else None, int(reps), results, cap, C.byref(n),
               C.byref(best), _stream(stream))
        as_dict = lambda r: {k: getattr(r, k) for k, _ in L.gsrf_tune_result._fields_}
        del ws, out, keep
        self.plan.grid.tile_w, self.plan.grid.tile_h = best.tile_w, best.tile_h
        self.plan.ray_block_w, self.plan.stage = best.ray_block_w, best.stage
        self._alloc()
        self.ensure_capacity(params, rx, tx)
        return as_dict(best), [as_dict(results[i]) for i in range(min(n.value, cap))]

    def render_bwd(self, params: dict, ray_state: torch.Tensor, grad_rays: torch.Tensor, grads: dict,
                   stream=None):
        """Add the gradients of sum Re(conj(grad_rays) S) to ``grads`` (same keys and
        shapes as the parameters; missing keys are skipped)."""
        gs = gaussians_struct(params)
        if not (grad_rays.is_cuda and grad_rays.dtype == torch.float32 and grad_rays.is_contiguous()):
            raise ValueError("grad_rays must be a contiguous float32 CUDA tensor")
        L.call("gsrf_render_bwd", C.byref(self.plan), C.byref(gs), _ptr(self.ws), self.ws_bytes,
               _ptr(ray_state), _ptr(grad_rays), *[_ptr(grads.get(k)) for k in PARAM_NAMES],
               _stream(stream))
        return grads

    def status(self, stream=None) -> L.gsrf_run_status:
        s = L.gsrf_run_status()
        L.call("gsrf_read_status", _ptr(self.ws), self.ws_bytes, C.byref(s), _stream(stream))
        return s

    def ensure_capacity(self, params: dict, rx: torch.Tensor, tx: torch.Tensor, slack: float = 1.05):
        """Run project + bin; if the pairs did not fit, grow the workspace and retry."""
        for _ in range(3):
            self.project(params, rx, tx)
            self.bin()
            s = self.status()
            if s.code == L.GSRF_ERR_CAPACITY:
                self.plan.pair_capacity = int(s.required_pairs * slack) + 1024
                self._alloc()
                continue
            L.check("gsrf_bin (device status)", s.code)
            return s.required_pairs
        raise L.GsrfError("ensure_capacity", L.GSRF_ERR_CAPACITY)

    def stage_times(self) -> dict:
        """Milliseconds of the last project, bin, forward and backward render on this
        workspace (gsrf_stage_times; a stage never run is absent).  Synchronises."""
        ms = (C.c_float * 8)()
        L.call("gsrf_stage_times", _ptr(self.ws), ms)
        names = ["project", "bin", "render_fwd", "render_bwd", "batch"]
        return {n: float(ms[i]) for i, n in enumerate(names) if ms[i] >= 0.0}

    def layout(self) -> L.gsrf_layout:
        lay = L.gsrf_layout()
        L.call("gsrf_workspace_layout", C.byref(self.plan), C.byref(lay))
        return lay

    def view_records(self) -> torch.Tensor:
        """View records after project: float32 [n_rx, n_gauss, 12] (see gsrf_layout.view)."""
        lay = self.layout()
        nr, n = self.plan.n_rx, self.plan.n_gauss
        return self.ws[lay.view: lay.view + 48 * nr * n].view(torch.float32).view(nr, n, 12)

    def pairs(self, stream=None):
        """Views into the workspace after bin: (keys uint64 [total], ids int32 [total],
        rx_base int64 [n_rx+1], tile_start int32 [n_rx, n_tiles+1]); the keys are formed
        here by gsrf_pair_keys (the bin itself writes only the ids and the ranges)."""
        L.call("gsrf_pair_keys", C.byref(self.plan), _ptr(self.ws), self.ws_bytes, _stream(stream))
        lay = self.layout()
        nt = lay.n_tiles_u * lay.n_tiles_v
        nr = self.plan.n_rx
        ws = self.ws
        rb = ws[lay.rx_pair_base: lay.rx_pair_base + 8 * (nr + 1)].view(torch.int64)
        total = int(rb[-1].item())
        keys = ws[lay.pair_keys: lay.pair_keys + 8 * total].view(torch.int64)
        ids = ws[lay.pair_ids: lay.pair_ids + 4 * total].view(torch.int32)
        ts = ws[lay.tile_start: lay.tile_start + 4 * nr * (nt + 1)].view(torch.int32).view(nr, nt + 1)
        return keys, ids, rb, ts


class BatchRender:
    """Many render problems (each a Renderer that has run project and bin) rendered by one
    persistent kernel launch, work items heaviest first (gsrf_render_batch).  ``outs``:
    optional output tensors, one per renderer (e.g. views of one buffer); ``stamps``: keep
    per-job completion times (``job_done_ns``, n_jobs + 1 int64 on the device);
    ``job_order``: take the jobs in the given order, heaviest first inside each, instead of
    heaviest first over all jobs."""

    def __init__(self, renderers: list, outs: list | None = None, stamps: bool = False, job_order: bool = False):
        if not 1 <= len(renderers) <= L.GSRF_MAX_BATCH_JOBS:
            raise ValueError("1..%d jobs per batch" % L.GSRF_MAX_BATCH_JOBS)
        self.renderers = list(renderers)
        n = len(self.renderers)
        self.plans = (L.gsrf_plan * n)(*[r.plan for r in self.renderers])
        nbytes = C.c_size_t()
        L.call("gsrf_batch_workspace_size", n, self.plans, C.byref(nbytes))
        self.ws_bytes = nbytes.value
        dev = self.renderers[0].device
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        self.outs = outs if outs is not None else [torch.empty(r.out_shape(), dtype=torch.float32, device=dev)
                                                   for r in self.renderers]
        self.job_done_ns = torch.zeros(n + 1, dtype=torch.int64, device=dev) if stamps else None
        self.flags = L.BATCH_JOB_ORDER if job_order else 0

    def render(self, stream=None):
        n = len(self.renderers)
        for i, r in enumerate(self.renderers):  # plans may have grown their capacity
            self.plans[i] = r.plan
        wss = (C.c_void_p * n)(*[r.ws.data_ptr() for r in self.renderers])
        wsb = (C.c_size_t * n)(*[r.ws_bytes for r in self.renderers])
        outs = (C.c_void_p * n)(*[o.data_ptr() for o in self.outs])
        L.call("gsrf_render_batch", n, self.plans, wss, wsb, outs, _ptr(self.ws), self.ws_bytes,
               _ptr(self.job_done_ns), self.flags, _stream(stream))
        return self.outs

    def completion_ms(self):
        """Each job's completion time (ms) after the start of the last launch (needs stamps)."""
        t = self.job_done_ns.cpu().numpy().view("uint64").astype("float64")
        return (t[:-1] - t[-1]) / 1e6


def received_signal(rays: torch.Tensor, mode: int = L.SIG_COMPLEX_SUM, stream=None) -> torch.Tensor:
    """rays [n_rx, n_f, n_el, n_az, 2] -> per mode (see include/gsrf.h)."""
    if not (rays.is_cuda and rays.dtype == torch.float32 and rays.is_contiguous() and rays.dim() == 5):
        raise ValueError("rays must be a contiguous float32 CUDA tensor [n_rx, n_f, n_el, n_az, 2]")
    n_rx, n_f, n_el, n_az, _ = rays.shape
    if mode == L.SIG_COMPLEX_SUM:
        out = torch.empty((n_rx, n_f, 2), dtype=torch.float32, device=rays.device)
    elif mode == L.SIG_SPECTRUM_MAG:
        out = torch.empty((n_rx, n_f, n_el, n_az), dtype=torch.float32, device=rays.device)
    else:
        out = torch.empty((n_rx, n_f), dtype=torch.float32, device=rays.device)
    L.call("gsrf_received_signal", _ptr(rays), n_rx, n_f, n_el, n_az, mode, _ptr(out), _stream(stream))
    return out


class RenderFunction(torch.autograd.Function):
    """S = render(theta) with the hand-written backward (App. D) as its gradient.

    forward(renderer, rx, tx, means, log_scales, quats, opacity_logit, coeffs, phase_b)
    returns the per-ray signal [n_rx, n_f, n_el, n_az, 2].  The renderer's workspace
    holds the forward's lists until backward runs, so one renderer serves one pending
    backward at a time."""

    @staticmethod
    def forward(ctx, renderer: Renderer, rx, tx, means, log_scales, quats, opacity_logit, coeffs, phase_b):
        params = dict(means=means.detach(), log_scales=log_scales.detach(), quats=quats.detach(),
                      opacity_logit=opacity_logit.detach(), coeffs=coeffs.detach(),
                      phase_b=None if phase_b is None else phase_b.detach())
        state = renderer.ray_state()
        out = renderer.forward(params, rx, tx, ray_state=state)
        ctx.renderer = renderer
        ctx.state = state
        ctx.params = params
        ctx.has_b = phase_b is not None
        return out

    @staticmethod
    def backward(ctx, grad_out):
        p = ctx.params
        grads = {k: torch.zeros_like(v) for k, v in p.items() if v is not None}
        ctx.renderer.render_bwd(p, ctx.state, grad_out.contiguous().float(), grads)
        return (None, None, None, grads["means"], grads["log_scales"], grads["quats"],
                grads["opacity_logit"], grads["coeffs"], grads.get("phase_b") if ctx.has_b else None)


def render(renderer: Renderer, params: dict, rx: torch.Tensor, tx: torch.Tensor) -> torch.Tensor:
    """Differentiable render: per-ray complex signal as [n_rx, n_f, n_el, n_az, 2]."""
    return RenderFunction.apply(renderer, rx, tx, params["means"], params["log_scales"], params["quats"],
                                params["opacity_logit"], params["coeffs"], params.get("phase_b"))
