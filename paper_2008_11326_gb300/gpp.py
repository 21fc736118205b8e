"""Python face of libgpp: the GPP self-energy summation on one GB300.

PyTorch supplies device memory and streams; every step of the sum runs in libgpp's CUDA
kernels through the C-ABI (``include/gpp.h``). Names follow the paper's kernel.
"""

from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import _native as N

PRECISIONS = {"fp64": N.GPP_FP64, "fp32_bulk": N.GPP_FP32_BULK}
OCC_MODES = {"all": N.GPP_OCC_ALL, "occupied": N.GPP_OCC_OCCUPIED}

_C128 = ("aqsmtemp", "aqsntemp", "I_eps_array", "wtilde_array")


@dataclasses.dataclass
class DeviceProblem:
    """Device tensors of one GPP instance (layouts as in include/gpp.h)."""

    number_bands: int
    nvband: int
    ncouls: int
    ngpown: int
    nw: int
    aqsmtemp: torch.Tensor      # complex128 [B][G]
    aqsntemp: torch.Tensor      # complex128 [B][G]
    I_eps_array: torch.Tensor   # complex128 [P][G]
    wtilde_array: torch.Tensor  # complex128 [P][G]
    vcoul: torch.Tensor         # float64 [G]
    inv_igp_index: torch.Tensor  # int32 [P]
    indinv: torch.Tensor        # int32 [G+1]
    wx_array: torch.Tensor      # float64 [B][W]
    aqsntemp_c64: torch.Tensor | None = None     # complex64 copy for fp32_bulk

    @classmethod
    def from_host(cls, prob, device="cuda", c64: bool = False, pin: bool = False):
        """Copy a host :class:`inputs.GppProblem` to ``device`` (or to pinned host memory
        when ``device == 'cpu'`` and ``pin``)."""
        def t(a, dt):
            x = torch.from_numpy(np.ascontiguousarray(a)).to(dt)
            if device == "cpu":
                return x.pin_memory() if pin else x
            return x.to(device)
        kw = dict(number_bands=prob.number_bands, nvband=prob.nvband, ncouls=prob.ncouls,
                  ngpown=prob.ngpown, nw=prob.nw)
        for f in _C128:
            kw[f] = t(getattr(prob, f), torch.complex128)
        kw["vcoul"] = t(prob.vcoul, torch.float64)
        kw["inv_igp_index"] = t(prob.inv_igp_index, torch.int32)
        kw["indinv"] = t(prob.indinv, torch.int32)
        kw["wx_array"] = t(prob.wx_array, torch.float64)
        dp = cls(**kw)
        if c64:
            dp.make_c64()
        return dp

    def make_c64(self, stream: torch.cuda.Stream | None = None):
        """The complex64 copy of aqsntemp that precision='fp32_bulk' reads per band, kept for
        later calls (without it, each fp32_bulk call converts into its workspace). On the
        device the library's conversion kernel makes it (enqueued on ``stream``); a host
        problem's copy is made on the host (pinned if aqsntemp is)."""
        src = self.aqsntemp
        if src.device.type == "cpu":
            c = src.to(torch.complex64)
            self.aqsntemp_c64 = c.pin_memory() if src.is_pinned() else c
            return self
        src = src.contiguous()
        c = torch.empty(src.shape, dtype=torch.complex64, device=src.device)
        N.check(N.lib().gpp_convert_c64(ctypes.c_void_p(src.data_ptr()),
                                        ctypes.c_void_p(c.data_ptr()), src.numel(),
                                        _stream_handle(stream, src.device)))
        _keep_for(stream, c)
        self.aqsntemp_c64 = c
        return self

    @property
    def device(self):
        return self.aqsmtemp.device

    def check(self, ach: torch.Tensor | None = None, asx: torch.Tensor | None = None):
        """Raise ValueError unless every array has the dtype, shape, device and layout that
        include/gpp.h requires for these sizes (the library reads exactly those extents, so
        a mismatch would read outside the tensors)."""
        B, G, P, W = self.number_bands, self.ncouls, self.ngpown, self.nw
        spec = [("aqsmtemp", torch.complex128, (B, G)), ("aqsntemp", torch.complex128, (B, G)),
                ("I_eps_array", torch.complex128, (P, G)),
                ("wtilde_array", torch.complex128, (P, G)), ("vcoul", torch.float64, (G,)),
                ("inv_igp_index", torch.int32, (P,)), ("indinv", torch.int32, (G + 1,)),
                ("wx_array", torch.float64, (B, W))]
        if self.aqsntemp_c64 is not None:
            spec.append(("aqsntemp_c64", torch.complex64, (B, G)))
        dev = self.aqsmtemp.device
        for name, dt, shape in spec:
            x = getattr(self, name)
            if (x.dtype != dt or tuple(x.shape) != shape or x.device != dev
                    or not x.is_contiguous()):
                raise ValueError(f"{name}: want a contiguous {dt} tensor of shape {shape} on "
                                 f"{dev}, got {x.dtype} {tuple(x.shape)} on {x.device}")
        for name, x in (("achtemp", ach), ("asxtemp", asx)):
            if x is not None and (x.dtype != torch.complex128 or x.numel() < W
                                  or x.device != dev or not x.is_contiguous()):
                raise ValueError(f"{name}: want a contiguous complex128 tensor of at least "
                                 f"{W} values on {dev}")

    def struct(self, ach: torch.Tensor, asx: torch.Tensor) -> N.GppProblem:
        def ptr(x):
            return None if x is None else x.data_ptr()
        self.check(ach, asx)
        return N.GppProblem(
            self.number_bands, self.nvband, self.ncouls, self.ngpown, self.nw,
            ptr(self.aqsmtemp), ptr(self.aqsntemp), ptr(self.I_eps_array),
            ptr(self.wtilde_array), ptr(self.vcoul), ptr(self.inv_igp_index), ptr(self.indinv),
            ptr(self.wx_array), ptr(self.aqsntemp_c64), ptr(ach), ptr(asx))


def _stream_handle(stream, device):
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _keep_for(stream, *tensors):
    """Tell torch's caching allocator that ``stream`` (when given) uses these tensors, which
    were allocated on the current stream: their memory is then not handed out again until
    the work enqueued on ``stream`` so far has finished, even once the tensors are freed."""
    if stream is None:
        return
    for t in tensors:
        if t is not None:
            t.record_stream(stream)


def make_options(precision="fp64", occ_mode="all", block_threads=0, blocks_per_sm=0,
                 debug_checks=False, stage_events=None, ig_per_thread=0, ch_half=False,
                 sexcut=0.0) -> N.GppOptions:
    """``stage_events``: four recorded ``torch.cuda.Event(enable_timing=True)`` (or raw
    cudaEvent_t handles) that the call re-records around its stages (see gpp_options).
    ``ch_half`` / ``sexcut`` (> 0 turns the cutoff on): the Sigma-code options."""
    if stage_events is not None:
        stage_events = [e.cuda_event if hasattr(e, "cuda_event") else int(e) for e in stage_events]
    return N.options(PRECISIONS[precision], OCC_MODES[occ_mode], block_threads, blocks_per_sm,
                     debug_checks, stage_events, ig_per_thread, ch_half, sexcut)


def workspace_size(dp: DeviceProblem, **opts) -> int:
    o = make_options(**opts)
    prob = dp.struct(None, None)
    n = N.lib().gpp_sigma_workspace_size(ctypes.byref(prob), ctypes.byref(o))
    err = N.lib().gpp_last_error().decode()
    if n == 0 and err:
        raise N.GppError(-2, err)
    return int(n)


def sigma(dp: DeviceProblem, *, out=None, workspace: torch.Tensor | None = None,
          stream: torch.cuda.Stream | None = None, **opts):
    """achtemp, asxtemp (complex128 [nw] device tensors) of one instance.

    Enqueued on ``stream`` (default: torch's current stream) without synchronising.
    ``opts``: precision ('fp64' | 'fp32_bulk'), occ_mode ('all' | 'occupied'),
    block_threads, blocks_per_sm, debug_checks, ig_per_thread, stage_events, and the
    Sigma-code options ch_half (achtemp halved) and sexcut (> 0: drop ssx where x < 0 and
    |ssx| > sexcut |I|).
    """
    dev = dp.device
    if out is None:
        ach = torch.empty(dp.nw, dtype=torch.complex128, device=dev)
        asx = torch.empty(dp.nw, dtype=torch.complex128, device=dev)
    else:
        ach, asx = out
    o = make_options(**opts)
    prob = dp.struct(ach, asx)
    lib = N.lib()
    need = lib.gpp_sigma_workspace_size(ctypes.byref(prob), ctypes.byref(o))
    if need == 0 and lib.gpp_last_error():
        raise N.GppError(-2, lib.gpp_last_error().decode())
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    N.check(lib.gpp_sigma(ctypes.byref(prob), ctypes.byref(o), ctypes.c_void_p(workspace.data_ptr()),
                          workspace.numel(), _stream_handle(stream, dev)))
    _keep_for(stream, workspace, ach, asx)
    return ach, asx


class BatchedPlan:
    """A prepared batch of instances (one persistent launch, optionally a CUDA graph).

    ``dps``: list of :class:`DeviceProblem` (same nw). Outputs are per-instance complex128
    [nw] device tensors in ``self.outputs``. ``run()`` enqueues the batch on the current
    stream (a graph replay when ``use_graph``).
    """

    def __init__(self, dps, *, use_graph=True, stream=None, **opts):
        self.dps = list(dps)
        dev = self.dps[0].device
        self.outputs = [(torch.empty(d.nw, dtype=torch.complex128, device=dev),
                         torch.empty(d.nw, dtype=torch.complex128, device=dev)) for d in self.dps]
        self._structs = (N.GppProblem * len(self.dps))(
            *[d.struct(a, s) for d, (a, s) in zip(self.dps, self.outputs)])
        self._opts = make_options(**opts)
        lib = N.lib()
        need = lib.gpp_batched_workspace_size(self._structs, len(self.dps), ctypes.byref(self._opts))
        if need == 0:
            raise N.GppError(-2, lib.gpp_last_error().decode())
        self.workspace = torch.empty(need, dtype=torch.uint8, device=dev)
        self._handle = ctypes.c_void_p()
        N.check(lib.gpp_batched_plan_create(ctypes.byref(self._handle), self._structs,
                                            len(self.dps), ctypes.byref(self._opts),
                                            ctypes.c_void_p(self.workspace.data_ptr()), need,
                                            1 if use_graph else 0, _stream_handle(stream, dev)))

    def run(self, stream=None):
        N.check(N.lib().gpp_batched_plan_run(self._handle, _stream_handle(stream, self.workspace.device)))
        return self.outputs

    def close(self):
        if self._handle:
            N.lib().gpp_batched_plan_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


GRAD_NAMES = ("wtilde", "I_eps", "aqsm", "aqsn")


def sigma_backward(dp: DeviceProblem, grad_achtemp: torch.Tensor, grad_asxtemp: torch.Tensor, *,
                   want=GRAD_NAMES, workspace: torch.Tensor | None = None,
                   stream: torch.cuda.Stream | None = None, **opts):
    """Gradients of a real loss through achtemp / asxtemp (PyTorch's complex convention).

    ``grad_achtemp`` / ``grad_asxtemp``: complex128 [nw] device tensors, dL/dRe + i dL/dIm of
    the outputs. Returns a dict with the requested complex128 gradients: 'wtilde' and
    'I_eps' [P][G], 'aqsm' and 'aqsn' [B][G].
    """
    dev = dp.device
    shapes = {"wtilde": (dp.ngpown, dp.ncouls), "I_eps": (dp.ngpown, dp.ncouls),
              "aqsm": (dp.number_bands, dp.ncouls), "aqsn": (dp.number_bands, dp.ncouls)}
    out = {k: torch.empty(shapes[k], dtype=torch.complex128, device=dev) for k in want}
    ga = grad_achtemp.to(device=dev, dtype=torch.complex128).contiguous()
    gs = grad_asxtemp.to(device=dev, dtype=torch.complex128).contiguous()
    o = make_options(**opts)
    prob = dp.struct(None, None)
    lib = N.lib()
    need = lib.gpp_sigma_backward_workspace_size(ctypes.byref(prob), ctypes.byref(o))
    if need == 0 and lib.gpp_last_error():
        raise N.GppError(-2, lib.gpp_last_error().decode())
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    grads = N.GppGrads(*[(out[k].data_ptr() if k in out else None) for k in GRAD_NAMES])
    N.check(lib.gpp_sigma_backward(ctypes.byref(prob), ctypes.byref(o),
                                   ctypes.c_void_p(ga.data_ptr()), ctypes.c_void_p(gs.data_ptr()),
                                   ctypes.byref(grads), ctypes.c_void_p(workspace.data_ptr()),
                                   workspace.numel(), _stream_handle(stream, dev)))
    _keep_for(stream, workspace, ga, gs, *out.values())
    return out


class GppSigma(torch.autograd.Function):
    """(achtemp, asxtemp) = GPP sum, differentiable in aqsmtemp, aqsntemp, I_eps_array and
    wtilde_array through libgpp's hand-written FP64 adjoint (terms recomputed in backward).

    apply(aqsmtemp, aqsntemp, I_eps_array, wtilde_array, vcoul, inv_igp_index, indinv,
          wx_array, nvband=0, occ_mode='all', ch_half=False, sexcut=0.0)
    """

    @staticmethod
    def forward(ctx, aqsmtemp, aqsntemp, I_eps_array, wtilde_array, vcoul, inv_igp_index,
                indinv, wx_array, nvband=0, occ_mode="all", ch_half=False, sexcut=0.0):
        dp = _problem_from(aqsmtemp, aqsntemp, I_eps_array, wtilde_array, vcoul, inv_igp_index,
                           indinv, wx_array, nvband)
        ctx.phys = dict(occ_mode=occ_mode, ch_half=ch_half, sexcut=sexcut)
        ach, asx = sigma(dp, **ctx.phys)
        ctx.save_for_backward(aqsmtemp, aqsntemp, I_eps_array, wtilde_array, vcoul,
                              inv_igp_index, indinv, wx_array)
        ctx.nvband = nvband
        return ach, asx

    @staticmethod
    def backward(ctx, g_ach, g_asx):
        t = ctx.saved_tensors
        dp = _problem_from(*t, ctx.nvband)
        W = dp.nw
        if g_ach is None:
            g_ach = torch.zeros(W, dtype=torch.complex128, device=dp.device)
        if g_asx is None:
            g_asx = torch.zeros(W, dtype=torch.complex128, device=dp.device)
        need = ctx.needs_input_grad
        want = [k for k, n in zip(("aqsm", "aqsn", "I_eps", "wtilde"), need[:4]) if n]
        if not want:
            return (None,) * 12
        g = sigma_backward(dp, g_ach, g_asx, want=want, **ctx.phys)
        return (g.get("aqsm"), g.get("aqsn"), g.get("I_eps"), g.get("wtilde"),
                None, None, None, None, None, None, None, None)


def _problem_from(aqsmtemp, aqsntemp, I_eps_array, wtilde_array, vcoul, inv_igp_index, indinv,
                  wx_array, nvband=0) -> DeviceProblem:
    B, G = aqsmtemp.shape
    P = wtilde_array.shape[0]
    W = wx_array.shape[1]
    c = lambda x, dt: x.detach().to(dt).contiguous()  # noqa: E731
    return DeviceProblem(B, int(nvband), G, P, W, c(aqsmtemp, torch.complex128),
                         c(aqsntemp, torch.complex128), c(I_eps_array, torch.complex128),
                         c(wtilde_array, torch.complex128), c(vcoul, torch.float64),
                         c(inv_igp_index, torch.int32), c(indinv, torch.int32),
                         c(wx_array, torch.float64))


def host_workspace_size(hp: DeviceProblem, **opts) -> int:
    o = make_options(**opts)
    prob = hp.struct(None, None)
    return int(N.lib().gpp_sigma_host_workspace_size(ctypes.byref(prob), ctypes.byref(o)))


def sigma_host(hp: DeviceProblem, *, workspace: torch.Tensor, out=None,
               stream: torch.cuda.Stream | None = None, **opts):
    """The sum on HOST tensors (ideally pinned): copies in, computes, copies the outputs
    back into host tensors and synchronises. ``workspace`` is a CUDA uint8 tensor of at
    least :func:`host_workspace_size` bytes."""
    if out is None:
        ach = torch.empty(hp.nw, dtype=torch.complex128).pin_memory()
        asx = torch.empty(hp.nw, dtype=torch.complex128).pin_memory()
    else:
        ach, asx = out
    o = make_options(**opts)
    prob = hp.struct(ach, asx)
    N.check(N.lib().gpp_sigma_host(ctypes.byref(prob), ctypes.byref(o),
                                   ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                   _stream_handle(stream, workspace.device)))
    return ach, asx


def peak_launch(kind: str, iters: int, blocks: int, threads: int, sink: torch.Tensor,
                stream=None) -> float:
    """Launch one throughput kernel; returns its operation count (see gpp_diag.h)."""
    N.check(N.lib().gpp_peak_launch(N.PEAK_KINDS[kind], iters, blocks, threads,
                                    ctypes.c_void_p(sink.data_ptr()),
                                    _stream_handle(stream, sink.device)))
    return float(blocks) * threads * N.PEAK_CHAINS * iters


def rcp(x: torch.Tensor) -> torch.Tensor:
    """The FP64 reciprocal the kernels use, applied elementwise (diagnostics)."""
    x = x.contiguous()
    out = torch.empty_like(x)
    N.check(N.lib().gpp_diag_rcp(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 x.numel(), _stream_handle(None, x.device)))
    return out
