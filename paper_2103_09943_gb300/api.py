"""Python binding of the F-BMP C-ABI on torch CUDA tensors.

Argument marshalling only: every step runs in the CUDA kernels of libps.so.
Tensors must be float32, contiguous and on the current CUDA device; the
current torch stream is passed to the library. Outputs and the workspace are
allocated with torch (the library itself allocates nothing).
"""
from __future__ import annotations

import ctypes
import json
import os
import tempfile
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import BandInfo, HrmsParams, KernelInfo, KernelParams, Scene, Tuning


class PsError(RuntimeError):
    pass


def _check(status: int) -> None:
    if status != 0:
        msg = _lib.load().ps_status_string(status).decode()
        raise PsError(f"libps status {status}: {msg}")


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _f32(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def default_kernel_params(**kw) -> KernelParams:
    p = KernelParams()
    _lib.load().ps_default_kernel_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def band_mask(bands) -> int:
    """The ps_kernel_params.band_mask of the LRMS channels X' (Eq. objective1)
    given as band indices; None or empty: all bands (0)."""
    m = 0
    for b in bands or ():
        if not 0 <= int(b) < 64:
            raise ValueError("band index out of range")
        m |= 1 << int(b)
    return m


def default_hrms_params(**kw) -> HrmsParams:
    p = HrmsParams()
    _lib.load().ps_default_hrms_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, "lambda_" if k == "lam" else k, v)
    return p


def workspace_size(N, H, W, ratio, R, hparams: HrmsParams | None = None) -> int:
    return int(_lib.load().ps_workspace_size(
        N, H, W, ratio, R, ctypes.byref(hparams) if hparams is not None else None))


def workspace(N, H, W, ratio, R, device=None, hparams: HrmsParams | None = None) -> torch.Tensor:
    n = workspace_size(N, H, W, ratio, R, hparams)
    if n == 0:
        raise PsError("invalid sizes for a workspace")
    return torch.empty(n, dtype=torch.uint8, device=device or "cuda")


TUNING_CHOICES = ("prec_rows", "llp_rows", "llp_pf", "split", "llp_bands", "prec_impl",
                  "db_impl", "llp_form")
TUNING_CACHE_VERSION = 1


def tuning_cache_key(gpu: str, N, H, W, ratio, R, r, with_scene: bool) -> str:
    """Key of one autotuner record in a tuning cache file: the GPU's name and
    the sizes the choices were timed on."""
    return f"{gpu}|N={N}|H={H}|W={W}|ratio={ratio}|R={R}|r={r}|scene={int(bool(with_scene))}"


def read_tuning_cache(path: str) -> dict:
    """The records of a tuning cache file (JSON), {} when it does not exist or
    was written by another format version."""
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        doc = json.load(fh)
    if not isinstance(doc, dict) or doc.get("version") != TUNING_CACHE_VERSION:
        return {}
    return dict(doc.get("entries", {}))


def write_tuning_cache(path: str, entries: dict) -> None:
    """Write the records atomically (a temporary file in the same folder,
    then a rename), so that a reader never sees a half-written file."""
    folder = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".tuning-", suffix=".json", dir=folder)
    try:
        with os.fdopen(fd, "w") as fh:
            json.dump({"version": TUNING_CACHE_VERSION, "entries": entries}, fh, indent=1,
                      sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def autotune(N, H, W, ratio, R, r=1, ws=None, device=None, lrms=None, pan=None,
             kernel=None, cache: str | None = None) -> dict:
    """Times the candidate launch shapes of the tunable kernels on these sizes
    and records the fastest for later solves (ps_autotune); with a scene
    (lrms, pan, kernel) also the number of parallel CG branches. With cache, a
    JSON file keyed by the GPU's name and the sizes: a record found there is
    applied (ps_set_tuning) instead of timing, and a new result is added."""
    key = None
    if cache is not None:
        dev = torch.device(device) if device is not None else torch.device("cuda")
        key = tuning_cache_key(torch.cuda.get_device_name(dev), N, H, W, ratio, R, r,
                               lrms is not None)
        rec = read_tuning_cache(cache).get(key)
        if rec is not None:
            choices = {k: int(rec["choices"][k]) for k in TUNING_CHOICES}
            set_tuning(N, H, W, ratio, r, **choices)
            return {**choices, "cached": True}
    ws = ws if ws is not None else workspace(N, H, W, ratio, R, device)
    t = Tuning()
    _check(_lib.load().ps_autotune(N, H, W, ratio, R, r, _ptr(lrms), _ptr(pan), _ptr(kernel),
                                   _ptr(ws), ws.numel(), _stream(), ctypes.byref(t)))
    out = {"prec_rows": t.prec_rows, "llp_rows": t.llp_rows,
            "prec_us": {str(k): round(v, 2) for k, v in zip((1, 2, 4, 8), t.prec_us) if v},
            "llp_pf": t.llp_pf,
            "llp_us": {f"{w}/{pf}": round(t.llp_us[3 * i + j], 2)
                       for i, w in enumerate(("long", "short")) for j, pf in enumerate((2, 3, 4))},
            "llp_bands": t.llp_bands,
            "llp2_us": {w: round(v, 2) for w, v in zip(("long/2", "short/2"), t.llp2_us) if v},
            "split": t.split,
            "split_us": {str(k): round(v, 2) for k, v in zip((1, 2, 4), t.split_us) if v},
            "prec_impl": t.prec_impl,
            "prec_impl_us": {n: round(v, 2) for n, v in zip(("smem", "reg"), t.prec_impl_us)
                             if v},
            "llp_ring_us": {w: round(v, 2) for w, v in zip(("long", "short"), t.llp_ring_us)
                            if v},
            "db_impl": t.db_impl,
            "db_impl_us": {n: round(v, 2) for n, v in zip(("site", "runs"), t.db_impl_us) if v},
            "llp_form": t.llp_form,
            "llp_lean_us": {f"form{f}/{w}/{pf}": round(t.llp_lean_us[4 * h + 2 * i + j], 2)
                            for h, f in enumerate((2, 4))
                            for i, w in enumerate(("long", "short"))
                            for j, pf in enumerate((2, 4)) if t.llp_lean_us[4 * h + 2 * i + j]}}
    if key is not None:
        entries = read_tuning_cache(cache)
        entries[key] = {"choices": {k: out[k] for k in TUNING_CHOICES}}
        write_tuning_cache(cache, entries)
    return out


def set_tuning(N, H, W, ratio, r=1, **choices) -> None:
    """Record launch choices for these sizes (ps_set_tuning): prec_rows,
    llp_rows, llp_pf, split, llp_bands, prec_impl, db_impl, llp_form; 0 or absent
    keeps a default."""
    t = Tuning()
    for k, v in choices.items():
        setattr(t, k, v)
    _check(_lib.load().ps_set_tuning(N, H, W, ratio, r, ctypes.byref(t)))


def get_tuning(N, H, W, ratio, r=1) -> dict:
    t = Tuning()
    _check(_lib.load().ps_get_tuning(N, H, W, ratio, r, ctypes.byref(t)))
    return {k: getattr(t, k) for k in ("prec_rows", "llp_rows", "llp_pf", "split", "llp_bands",
                                       "prec_impl", "db_impl", "llp_form")}


@dataclass
class SolveInfo:
    status: list
    iters: list
    rel_residual: list
    ms: list          # device time of each band's Z0 solve (ps_band_info.ms)


def _solve_info(bi):
    return SolveInfo([b.status for b in bi], [b.iters for b in bi],
                     [b.rel_residual for b in bi], [b.ms for b in bi])


def sync_status() -> int:
    """ps_sync_status on the current stream: waits for it, returns and clears
    the first device-detected status since the last read (0: none)."""
    return int(_lib.load().ps_sync_status(_stream()))


def estimate_kernel(lrms, pan, ratio: int, R: int, params: KernelParams | None = None,
                    omega=None, ws=None, info: bool = True):
    """Algorithm 1. Returns (kernel (n,n), omega (N,), KernelInfo or None)."""
    N, h, w = lrms.shape
    H, W = pan.shape
    _f32(lrms, "lrms"), _f32(pan, "pan")
    p = params or default_kernel_params()
    n = 2 * R + 1
    kern = torch.empty((n, n), dtype=torch.float32, device=lrms.device)
    om = torch.empty(N, dtype=torch.float32, device=lrms.device)
    ws = ws if ws is not None else workspace(N, H, W, ratio, R, lrms.device)
    ki = KernelInfo()
    _check(_lib.load().ps_estimate_kernel(
        _ptr(lrms), _ptr(pan), N, H, W, ratio, R, ctypes.byref(p),
        _ptr(None if omega is None else _f32(omega, "omega")), _ptr(kern), _ptr(om),
        ctypes.byref(ki) if info else None, _ptr(ws), ws.numel(), _stream()))
    return kern, om, (ki if info else None)


def solve_hrms(lrms, pan, kernel, ratio: int, params: HrmsParams | None = None,
               z_init=None, want_z0: bool = False, ws=None, info: bool = True, out=None):
    """Algorithm 2 on all bands. Returns (hrms, z0 or None, SolveInfo or None)."""
    N, h, w = lrms.shape
    H, W = pan.shape
    _f32(lrms, "lrms"), _f32(pan, "pan"), _f32(kernel, "kernel")
    R = kernel.shape[0] // 2
    p = params or default_hrms_params()
    hr = out if out is not None else torch.empty((N, H, W), dtype=torch.float32,
                                                 device=lrms.device)
    z0 = torch.empty_like(hr) if want_z0 else None
    ws = ws if ws is not None else workspace(N, H, W, ratio, R, lrms.device, p)
    bi = (BandInfo * N)()
    _check(_lib.load().ps_solve_hrms(
        _ptr(lrms), _ptr(pan), _ptr(kernel), N, H, W, ratio, R, ctypes.byref(p),
        _ptr(None if z_init is None else _f32(z_init, "z_init")), _ptr(hr), _ptr(z0),
        bi if info else None, _ptr(ws), ws.numel(), _stream()))
    si = None
    if info:
        si = _solve_info(bi)
    return hr, z0, si


def pansharpen(lrms, pan, ratio: int, R: int, kparams: KernelParams | None = None,
               hparams: HrmsParams | None = None, ws=None, info: bool = True, out=None,
               kernel_out=None):
    """The two-stage scheme: Algorithm 1 then Algorithm 2.
    Returns (hrms, kernel, KernelInfo or None, SolveInfo or None)."""
    N, h, w = lrms.shape
    H, W = pan.shape
    _f32(lrms, "lrms"), _f32(pan, "pan")
    kp = kparams or default_kernel_params()
    hp = hparams or default_hrms_params()
    n = 2 * R + 1
    hr = out if out is not None else torch.empty((N, H, W), dtype=torch.float32,
                                                 device=lrms.device)
    kern = kernel_out if kernel_out is not None else torch.empty(
        (n, n), dtype=torch.float32, device=lrms.device)
    ws = ws if ws is not None else workspace(N, H, W, ratio, R, lrms.device, hp)
    ki = KernelInfo()
    bi = (BandInfo * N)()
    _check(_lib.load().ps_pansharpen(
        _ptr(lrms), _ptr(pan), N, H, W, ratio, R, ctypes.byref(kp), ctypes.byref(hp),
        _ptr(hr), _ptr(kern), ctypes.byref(ki) if info else None, bi if info else None,
        _ptr(ws), ws.numel(), _stream()))
    si = None
    if info:
        si = _solve_info(bi)
    return hr, kern, (ki if info else None), si


class Batch:
    """Many scenes of uneven sizes in one graph launch (ps_pansharpen_batched).

    scenes: list of (lrms (N,h,w), pan (H,W), R) on the device, or
    (lrms, pan, R, band_mask) with the scene's own X' (see band_mask()). Outputs
    (hrms per scene, kernel per scene) and the workspace are allocated once;
    run() launches the whole batch, estimating every kernel when
    estimate=True, else using the kernels in self.kernels (fill them first).
    stage_host() makes every run copy the scenes' inputs from page-locked host
    tensors and their HRMS back to page-locked host tensors inside the graph.
    """

    def __init__(self, scenes, ratio: int, hparams: HrmsParams | None = None,
                 kparams: KernelParams | None = None, estimate: bool = True):
        self.hp = hparams or default_hrms_params()
        self.kp = (kparams or default_kernel_params()) if estimate else None
        self.inputs, self.hrms, self.kernels = [], [], []
        arr = (Scene * len(scenes))()
        for i, sc in enumerate(scenes):
            lrms, pan, R = sc[:3]
            mask = int(sc[3]) if len(sc) > 3 else 0
            _f32(lrms, "lrms"), _f32(pan, "pan")
            N = lrms.shape[0]
            H, W = pan.shape
            hr = torch.empty((N, H, W), dtype=torch.float32, device=lrms.device)
            kern = torch.zeros((2 * R + 1, 2 * R + 1), dtype=torch.float32, device=lrms.device)
            self.inputs.append((lrms, pan))
            self.hrms.append(hr)
            self.kernels.append(kern)
            arr[i] = Scene(lrms.data_ptr(), pan.data_ptr(), hr.data_ptr(), kern.data_ptr(),
                           N, H, W, ratio, R, mask)
        self.scenes = arr
        self.count = len(scenes)
        self.bands = sum(t.shape[0] for t in self.hrms)
        n = int(_lib.load().ps_batch_workspace_size(arr, self.count, ctypes.byref(self.hp)))
        if n == 0:
            raise PsError("invalid scene sizes for a batch")
        self.ws = torch.empty(n, dtype=torch.uint8, device=scenes[0][0].device)

    def run(self, info: bool = False):
        """Launch the batch. With info, block and return (list of KernelInfo
        or None, list of SolveInfo per scene)."""
        ki = (KernelInfo * self.count)() if info and self.kp is not None else None
        bi = (BandInfo * self.bands)() if info else None
        _check(_lib.load().ps_pansharpen_batched(
            self.scenes, self.count, ctypes.byref(self.kp) if self.kp is not None else None,
            ctypes.byref(self.hp), ki, bi, _ptr(self.ws), self.ws.numel(), _stream()))
        if not info:
            return None
        out, k = [], 0
        for hr in self.hrms:
            n = hr.shape[0]
            out.append(_solve_info(bi[k:k + n]))
            k += n
        return (list(ki) if ki is not None else None), out

    def stage_host(self, h_inputs, h_hrms=None):
        """From the next run on, copy each scene's (lrms, pan) from the
        page-locked host tensors h_inputs[i] into its device inputs, and its
        HRMS back into h_hrms[i] (allocated page-locked when None), as nodes of
        the batch's graph. Returns the host HRMS tensors."""
        if h_hrms is None:
            h_hrms = [torch.empty(t.shape, dtype=torch.float32).pin_memory() for t in self.hrms]
        for i, ((hx, hy), ho) in enumerate(zip(h_inputs, h_hrms)):
            dx, dy = self.inputs[i]
            for h, d in ((hx, dx), (hy, dy), (ho, self.hrms[i])):
                if (h.device.type != "cpu" or not h.is_pinned() or h.shape != d.shape
                        or h.dtype != torch.float32 or not h.is_contiguous()):
                    raise PsError("host staging needs page-locked contiguous float32 tensors "
                                  "of the scene's shapes")
            self.scenes[i].h_lrms, self.scenes[i].h_pan = hx.data_ptr(), hy.data_ptr()
            self.scenes[i].h_hrms = ho.data_ptr()
        self._host = (list(h_inputs), list(h_hrms))     # kept alive with the batch
        return self._host[1]

    def scene_ms(self) -> list:
        """Finish time of every scene of the last run, ms after it started."""
        ms = (ctypes.c_double * self.count)()
        _check(_lib.load().ps_batch_scene_ms(_ptr(self.ws), self.count, _stream(), ms))
        return list(ms)


class HostPipeline:
    """End-to-end path from HOST buffers: pinned host -> device copies of the
    LRMS and PAN, ps_pansharpen, device -> host copy of the HRMS, all on one
    stream. Buffers are allocated once for a given size."""

    def __init__(self, N, H, W, ratio, R, kparams=None, hparams=None, device="cuda"):
        self.N, self.H, self.W, self.ratio, self.R = N, H, W, ratio, R
        h, w = H // ratio, W // ratio
        self.kp = kparams or default_kernel_params()
        self.hp = hparams or default_hrms_params()
        self.d_lrms = torch.empty((N, h, w), dtype=torch.float32, device=device)
        self.d_pan = torch.empty((H, W), dtype=torch.float32, device=device)
        self.d_hrms = torch.empty((N, H, W), dtype=torch.float32, device=device)
        self.d_kern = torch.empty((2 * R + 1, 2 * R + 1), dtype=torch.float32, device=device)
        self.h_hrms = torch.empty((N, H, W), dtype=torch.float32).pin_memory()
        self.ws = workspace(N, H, W, ratio, R, device, self.hp)

    @property
    def h2d_bytes(self) -> int:
        return (self.d_lrms.numel() + self.d_pan.numel()) * 4

    @property
    def d2h_bytes(self) -> int:
        return self.d_hrms.numel() * 4

    def __call__(self, h_lrms: torch.Tensor, h_pan: torch.Tensor) -> torch.Tensor:
        self.d_lrms.copy_(h_lrms, non_blocking=True)
        self.d_pan.copy_(h_pan, non_blocking=True)
        pansharpen(self.d_lrms, self.d_pan, self.ratio, self.R, self.kp, self.hp, ws=self.ws,
                   info=False, out=self.d_hrms, kernel_out=self.d_kern)
        self.h_hrms.copy_(self.d_hrms, non_blocking=True)
        return self.h_hrms
