"""Thin Python binding of libsdfdock (ctypes): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module checks tensor
dtypes, devices and shapes, passes raw device pointers and the current torch
stream, and turns error codes into exceptions.  There is no CPU fallback: if the
library cannot be loaded, the calls raise.

Names follow the C ABI of include/sdfdock.h: sdf_build, score_rotations,
score_maps, top_k_poses, score_grad, score_pairs, refine, search_plan,
tune_export / tune_import, and the host-side adaptive sampling tree (Octree,
Context.sdf_build_octree).  Pose refinement comes three ways: Context.refine
(sd_refine: ascent, conjugate gradient or damped dynamics, all on the device),
Context.refine_poses (its ascent rule) and the module-level refine_poses, the
same ascent written as a PyTorch loop over the SdfScore autograd Function.
"""

from __future__ import annotations

import ctypes as ct
import math
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

SD_OK = 0
SD_ERR_ARG = -1
SD_ERR_OOM = -2
SD_ERR_CUDA = -3
SD_ERR_TIMEOUT = -4
SD_ERR_UNIMPLEMENTED = -5
SD_ERR_NONFINITE = -6
SD_F32, SD_F64 = 0, 1
SD_TOP_K_STATIC_MAX = 1 << 20

_ERRNAMES = {SD_ERR_ARG: "SD_ERR_ARG", SD_ERR_OOM: "SD_ERR_OOM", SD_ERR_CUDA: "SD_ERR_CUDA",
             SD_ERR_TIMEOUT: "SD_ERR_TIMEOUT", SD_ERR_UNIMPLEMENTED: "SD_ERR_UNIMPLEMENTED",
             SD_ERR_NONFINITE: "SD_ERR_NONFINITE"}


class SdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class sd_params(ct.Structure):
    _fields_ = [("dim", ct.c_int), ("precision", ct.c_int), ("lambda1", ct.c_double),
                ("lambda2", ct.c_double), ("sigma_t", ct.c_double), ("eps", ct.c_double),
                ("sigma_g", ct.c_double), ("w", ct.c_int), ("alpha", ct.c_int), ("beta", ct.c_double),
                ("phi", ct.c_int), ("phi_radius", ct.c_double)]


PHI_SDF, PHI_PROXIMAL, PHI_RADIAL, PHI_SKIN = 0, 1, 2, 3


class sd_grid(ct.Structure):
    _fields_ = [("N", ct.c_int), ("L", ct.c_double)]


class sd_pose(ct.Structure):
    _fields_ = [("score", ct.c_double), ("score_fp64", ct.c_double), ("score_fp64_im", ct.c_double),
                ("rot", ct.c_int32), ("idx", ct.c_int32), ("t", ct.c_double * 3)]


class sd_pair_job(ct.Structure):
    _fields_ = [("fixed", ct.c_void_p), ("moving", ct.c_void_p), ("quats", ct.c_void_p), ("n_r", ct.c_int64),
                ("grid", sd_grid), ("cand_out", ct.c_void_p)]


class sd_pair_stat(ct.Structure):
    _fields_ = [("ms", ct.c_double), ("batch", ct.c_int32), ("spread_bins", ct.c_int32), ("n", ct.c_int32),
                ("s", ct.c_int32), ("fft_plan", ct.c_int32)]


class sd_refine_params(ct.Structure):
    _fields_ = [("method", ct.c_int), ("lr_t", ct.c_double), ("lr_q", ct.c_double), ("mass", ct.c_double),
                ("inertia", ct.c_double), ("damping", ct.c_double), ("dt", ct.c_double)]


REFINE_ASCENT, REFINE_CG, REFINE_DYNAMICS = 0, 1, 2

CAND_BYTES = 16  # sd_cand: double score, int32 rot, int32 idx

_LIB = None

_SIGS = {
    "sd_default_params": (ct.c_int, [ct.POINTER(sd_params), ct.c_int, ct.c_int]),
    "sd_create": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int, ct.POINTER(sd_params)]),
    "sd_destroy": (ct.c_int, [ct.c_void_p]),
    "sd_last_error": (ct.c_char_p, [ct.c_void_p]),
    "sd_set_option": (ct.c_int, [ct.c_void_p, ct.c_char_p, ct.c_int64]),
    "sd_sdf_build": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_void_p,
                                ct.c_void_p, ct.c_int64, ct.c_void_p, ct.POINTER(ct.c_void_p), ct.c_void_p,
                                ct.c_void_p]),
    "sd_shape_from_samples": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int64,
                                         ct.POINTER(ct.c_void_p), ct.c_void_p]),
    "sd_shape_info": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_double)]),
    "sd_shape_free": (ct.c_int, [ct.c_void_p]),
    "sd_score_rotations": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int64,
                                      ct.POINTER(sd_grid), ct.c_int, ct.c_void_p, ct.c_void_p]),
    "sd_score_maps": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int64,
                                 ct.POINTER(sd_grid), ct.c_void_p, ct.c_void_p]),
    "sd_score_pairs": (ct.c_int, [ct.c_void_p, ct.POINTER(sd_pair_job), ct.c_int64, ct.POINTER(sd_pair_stat),
                                  ct.c_void_p]),
    "sd_search_plan": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.POINTER(sd_grid), ct.c_int64,
                                  ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32)]),
    "sd_tune_export": (ct.c_int, [ct.c_void_p, ct.c_char_p, ct.c_int64, ct.POINTER(ct.c_int64)]),
    "sd_tune_import": (ct.c_int, [ct.c_void_p, ct.c_char_p]),
    "sd_top_k_poses": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_int, ct.c_int, ct.c_void_p,
                                  ct.c_void_p, ct.c_void_p, ct.POINTER(sd_grid), ct.POINTER(sd_pose),
                                  ct.c_void_p]),
    "sd_score_grad": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.POINTER(sd_grid), ct.c_void_p,
                                 ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "sd_refine_poses": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.POINTER(sd_grid), ct.c_void_p,
                                   ct.c_void_p, ct.c_int64, ct.c_int, ct.c_double, ct.c_double, ct.c_void_p,
                                   ct.c_void_p]),
    "sd_refine": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.POINTER(sd_grid), ct.c_void_p, ct.c_void_p,
                             ct.c_int64, ct.c_int, ct.POINTER(sd_refine_params), ct.c_void_p, ct.c_void_p]),
    "sd_octree_create": (ct.c_int, [ct.c_int, ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_double, ct.c_int, ct.c_int,
                                    ct.c_double, ct.c_double, ct.c_double, ct.POINTER(ct.c_void_p)]),
    "sd_octree_pending": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int64), ct.c_void_p, ct.c_void_p]),
    "sd_octree_feed": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int64]),
    "sd_octree_leaves": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int64), ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "sd_octree_free": (ct.c_int, [ct.c_void_p]),
    "sd_host_line_fft": (ct.c_int, [ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p]),
    "sd_version": (ct.c_char_p, []),
    "sd_launch_count": (ct.c_int64, []),
    "sd_top_k_static": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_int, ct.c_void_p, ct.c_void_p]),
    "sd_pass_times": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_double)]),
    "sd_alu_peak": (ct.c_int, [ct.c_int, ct.c_int, ct.POINTER(ct.c_double)]),
}

PASS_NAMES = ["clear", "spread", "fwd_x", "fwd_y", "fused", "inv_y", "inv_x", "reduce", "graph", "spread_x", "inv_yx"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ct.CDLL:
    """Load libsdfdock.so (building it first if asked and absent); raise if impossible."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libsdfdock.so is not built ({path}); run paper_1712_00238_gb300.build.build()")
        path = _build.build()
    lib = ct.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


@dataclass
class Grid:
    N: int
    L: float

    def c(self) -> sd_grid:
        return sd_grid(self.N, float(self.L))


class Shape:
    """A shape's sampled SDF, owned by the library (freed with the context)."""

    def __init__(self, ctx: "Context", handle: ct.c_void_p):
        self.ctx = ctx
        self.handle = handle
        m = ct.c_int64()
        r = ct.c_double()
        ctx._check(ctx.lib.sd_shape_info(handle, ct.byref(m), ct.byref(r)))
        self.m = m.value
        self.radius = r.value

    def free(self):
        if self.handle:
            self.ctx.lib.sd_shape_free(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover - best effort
        try:
            if self.handle and self.ctx.handle:
                self.free()
        except Exception:
            pass


class Context:
    """A library context on one CUDA device with fixed SDF / kernel parameters."""

    def __init__(self, dim: int = 3, precision: str = "f32", device: int = 0, **params):
        self.lib = load()
        self.dim = dim
        self.precision = precision
        self.real = torch.float64 if precision == "f64" else torch.float32
        self.device = torch.device("cuda", device)
        p = sd_params()
        self._check_create(self.lib.sd_default_params(ct.byref(p), dim, SD_F64 if precision == "f64" else SD_F32))
        for k, v in params.items():
            if k == "eps" and v is None:
                v = math.inf
            setattr(p, k, v)
        self.params = p
        h = ct.c_void_p()
        rc = self.lib.sd_create(ct.byref(h), device, ct.byref(p))
        if rc != SD_OK:
            raise SdError(rc, self.lib.sd_last_error(None).decode())
        self.handle = h
        self.shapes = []

    def _check_create(self, rc):
        if rc != SD_OK:
            raise SdError(rc, "sd_default_params failed")

    def _check(self, rc):
        if rc != SD_OK:
            raise SdError(rc, self.lib.sd_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            for s in self.shapes:
                s.free()
            self.shapes = []
            self.lib.sd_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key: str, value: int):
        self._check(self.lib.sd_set_option(self.handle, key.encode(), int(value)))

    def pass_times(self, reset: bool = False) -> dict:
        """{pass name: (timed launches, summed device ms)} from CUDA events (option "timing")."""
        out = {}
        for k, name in enumerate(PASS_NAMES):
            n = ct.c_int64()
            ms = ct.c_double()
            self._check(self.lib.sd_pass_times(self.handle, k, ct.byref(n), ct.byref(ms)))
            out[name] = (n.value, ms.value)
        if reset:
            self._check(self.lib.sd_pass_times(self.handle, -1, None, None))
        return out

    # -- tensor helpers --------------------------------------------------------
    def _dev(self, x, dtype=None, cols=None) -> torch.Tensor:
        dtype = dtype or self.real
        t = torch.as_tensor(x)
        if cols is not None and t.shape[-1] != cols:
            pad = torch.zeros(t.shape[:-1] + (cols - t.shape[-1],), dtype=t.dtype)
            t = torch.cat([t, pad.to(t.device)], -1)
        return t.to(device=self.device, dtype=dtype).contiguous()

    def _need(self, t: torch.Tensor, dtype, name):
        if not (t.is_cuda and t.device == self.device and t.dtype == dtype and t.is_contiguous()):
            raise ValueError(f"{name}: expected a contiguous {dtype} tensor on {self.device}")

    # -- shapes ----------------------------------------------------------------
    def sdf_build(self, bnd, nrm, area, qry, vol, pmc=None, return_rho=False) -> Shape | tuple:
        """Sampled SDF of a solid (Eq. 10A-17t) from oriented boundary samples."""
        bnd = self._dev(bnd, cols=4)
        nrm = self._dev(nrm, cols=4)
        area = self._dev(area)
        qry = self._dev(qry, cols=4)
        vol = self._dev(vol)
        pm = None if pmc is None else self._dev(pmc, dtype=torch.int8)
        rho = torch.empty((qry.shape[0], 2), dtype=self.real, device=self.device) if return_rho else None
        h = ct.c_void_p()
        self._check(self.lib.sd_sdf_build(self.handle, _ptr(bnd), _ptr(nrm), _ptr(area), bnd.shape[0], _ptr(qry),
                                          _ptr(vol), qry.shape[0], _ptr(pm), ct.byref(h), _ptr(rho),
                                          _stream(self.device)))
        s = Shape(self, h)
        self.shapes.append(s)
        return (s, rho) if return_rho else s

    def sdf_build_octree(self, bnd, nrm, area, lo, size: float, depth_min: int, depth_max: int, tau: float,
                         clearance: float, return_leaves: bool = False, band: float = math.inf):
        """Sampled SDF on an adaptive tree (Section 5): sd_octree levels, rho by sd_sdf_build.

        Each level's pending centres are evaluated on the device and their rho
        fed back to the host tree; the leaves then become the shape's samples.
        With ``return_leaves`` also returns (centres, volumes, coords, rho) of
        the leaves (host arrays; rho as a device tensor)."""
        # the tree measures distances to the boundary samples as given, in FP64
        tree = Octree(self.dim, torch.as_tensor(bnd).double().cpu().numpy(), lo, size, depth_min, depth_max, tau,
                      clearance, band)
        bnd = self._dev(bnd, cols=4)
        nrm = self._dev(nrm, cols=4)
        area = self._dev(area)
        try:
            while True:
                cen, vol = tree.pending()
                if len(cen) == 0:
                    break
                part, rho = self.sdf_build(bnd, nrm, area, cen, vol, return_rho=True)
                part.free()
                self.shapes.remove(part)
                tree.feed(rho.double().cpu().numpy())
            cen, vol, crd = tree.leaves()
        finally:
            tree.close()
        shape, rho = self.sdf_build(bnd, nrm, area, cen, vol, return_rho=True)
        return (shape, (cen, vol, crd, rho)) if return_leaves else shape

    def shape_from_samples(self, pos, c) -> Shape:
        pos = self._dev(pos, cols=4)
        c = self._dev(c, cols=2)
        h = ct.c_void_p()
        self._check(self.lib.sd_shape_from_samples(self.handle, _ptr(pos), _ptr(c), pos.shape[0], ct.byref(h),
                                                   _stream(self.device)))
        s = Shape(self, h)
        self.shapes.append(s)
        return s

    # -- search ------------------------------------------------------------------
    def score_rotations(self, fixed: Shape, moving: Shape, quats: torch.Tensor, grid: Grid, k_r: int = 1,
                        out: torch.Tensor | None = None) -> torch.Tensor:
        """Per-rotation best translation; returns a uint8 (n_r, 16) candidate buffer."""
        self._need(quats, torch.float64, "quats")
        n_r = quats.shape[0]
        if out is None:
            out = torch.empty((n_r * k_r, CAND_BYTES), dtype=torch.uint8, device=self.device)
        g = grid.c()
        self._check(self.lib.sd_score_rotations(self.handle, fixed.handle, moving.handle, _ptr(quats), n_r,
                                                ct.byref(g), k_r, _ptr(out), _stream(self.device)))
        return out

    def score_maps(self, fixed: Shape, moving: Shape, quats: torch.Tensor, grid: Grid) -> torch.Tensor:
        """Complex score maps f_N, shape (n_r, N^dim) complex (flat translation order)."""
        self._need(quats, torch.float64, "quats")
        n_r = quats.shape[0]
        out = torch.empty((n_r, grid.N ** self.dim, 2), dtype=self.real, device=self.device)
        g = grid.c()
        self._check(self.lib.sd_score_maps(self.handle, fixed.handle, moving.handle, _ptr(quats), n_r,
                                           ct.byref(g), _ptr(out), _stream(self.device)))
        return torch.view_as_complex(out)

    def tune_export(self) -> str:
        """The autotuner's cached plans as JSON text (sd_tune_export)."""
        n = ct.c_int64()
        self._check(self.lib.sd_tune_export(self.handle, None, 0, ct.byref(n)))
        buf = ct.create_string_buffer(n.value)
        self._check(self.lib.sd_tune_export(self.handle, buf, n.value, ct.byref(n)))
        return buf.value.decode()

    def tune_import(self, text: str):
        """Add plans written by tune_export to this context's cache (sd_tune_import)."""
        self._check(self.lib.sd_tune_import(self.handle, text.encode()))

    def search_plan(self, moving: Shape, grid: Grid, n_r: int) -> dict:
        """The plan a search would use now: rotations per batch, the spreading variant
        (spread_bins, as sd_search_plan) and the forward-pass FFT plan (FFT_PLANS index)."""
        b, s, f = ct.c_int32(), ct.c_int32(), ct.c_int32()
        g = grid.c()
        self._check(self.lib.sd_search_plan(self.handle, moving.handle, ct.byref(g), n_r, ct.byref(b),
                                            ct.byref(s), ct.byref(f)))
        return {"batch": b.value, "spread_bins": s.value, "fft_plan": f.value}

    def score_pairs(self, jobs, outs: list | None = None, stats: bool = True):
        """Score many (fixed, moving, quats, grid) jobs in one launch sequence (a captured
        CUDA graph from the second call with the same job list on).  Returns the per-job
        candidate buffers (uint8 (n_r, 16)) and, if ``stats``, per-job dicts with the
        device time and the plan; the buffers must stay alive while the list is reused."""
        n = len(jobs)
        arr = (sd_pair_job * n)()
        if outs is None:
            outs = [torch.empty((q.shape[0], CAND_BYTES), dtype=torch.uint8, device=self.device)
                    for _, _, q, _ in jobs]
        for j, (fx, mv, q, grid) in enumerate(jobs):
            self._need(q, torch.float64, "quats")
            arr[j].fixed = fx.handle
            arr[j].moving = mv.handle
            arr[j].quats = _ptr(q)
            arr[j].n_r = q.shape[0]
            arr[j].grid = grid.c()
            arr[j].cand_out = _ptr(outs[j])
        st = (sd_pair_stat * n)() if stats else None
        self._check(self.lib.sd_score_pairs(self.handle, arr, n, st, _stream(self.device)))
        if not stats:
            return outs, None
        return outs, [dict(ms=x.ms, batch=x.batch, spread_bins=x.spread_bins, n=x.n, s=x.s,
                           fft_plan=x.fft_plan) for x in st]

    def top_k_poses(self, cand: torch.Tensor, k: int, fixed: Shape = None, moving: Shape = None,
                    quats: torch.Tensor = None, grid: Grid = None, rescore_fp64: bool = True) -> list[dict]:
        """Global top-k (score desc, rot asc, idx asc), optionally re-scored in FP64."""
        n = cand.numel() // CAND_BYTES
        out = (sd_pose * k)()
        g = grid.c()
        self._check(self.lib.sd_top_k_poses(self.handle, _ptr(cand), n, k, int(rescore_fp64),
                                            fixed.handle if fixed else None, moving.handle if moving else None,
                                            _ptr(quats), ct.byref(g), out, _stream(self.device)))
        return [dict(score=p.score, score_fp64=p.score_fp64, score_fp64_im=p.score_fp64_im, rot=p.rot,
                     idx=p.idx, t=list(p.t)[: self.dim]) for p in out]

    def score_grad(self, fixed: Shape, moving: Shape, grid: Grid, quats: torch.Tensor, trans: torch.Tensor):
        """Re f_N and its gradient w.r.t. raw quaternions and translations at P poses."""
        quats = quats.to(self.real).contiguous()
        trans = self._dev(trans, cols=3)
        self._need(quats, self.real, "quats")
        P = quats.shape[0]
        score = torch.empty(P, dtype=self.real, device=self.device)
        dq = torch.empty((P, 4), dtype=self.real, device=self.device)
        dt = torch.empty((P, 3), dtype=self.real, device=self.device)
        g = grid.c()
        self._check(self.lib.sd_score_grad(self.handle, fixed.handle, moving.handle, ct.byref(g), _ptr(quats),
                                           _ptr(trans), P, _ptr(score), _ptr(dq), _ptr(dt),
                                           _stream(self.device)))
        return score, dq, dt[:, : self.dim]


    def refine_poses(self, fixed: Shape, moving: Shape, grid: Grid, q0: torch.Tensor, t0: torch.Tensor,
                     steps: int = 50, lr_t: float = 0.05, lr_q: float = 0.02):
        """Gradient ascent on the device (sd_refine_poses): returns (q, t, score history (steps+1, P))."""
        q = q0.detach().to(device=self.device, dtype=self.real).contiguous().clone()
        t = self._dev(t0.detach(), cols=3).clone()
        P = q.shape[0]
        hist = torch.empty((steps + 1, P), dtype=self.real, device=self.device)
        g = grid.c()
        self._check(self.lib.sd_refine_poses(self.handle, fixed.handle, moving.handle, ct.byref(g), _ptr(q), _ptr(t),
                                             P, int(steps), float(lr_t), float(lr_q), _ptr(hist),
                                             _stream(self.device)))
        return q, t[:, : self.dim], hist


    def refine(self, fixed: Shape, moving: Shape, grid: Grid, q0: torch.Tensor, t0: torch.Tensor, steps: int,
               method: int = REFINE_CG, lr_t: float = 0.05, lr_q: float = 0.02, mass: float = 1.0,
               inertia: float = 1.0, damping: float = 0.1, dt: float = 0.1):
        """Maximise the score on the device from P poses with one of the sd_refine rules
        (REFINE_ASCENT, REFINE_CG, REFINE_DYNAMICS): returns (q, t, score history (steps+1, P))."""
        q = q0.detach().to(device=self.device, dtype=self.real).contiguous().clone()
        t = self._dev(t0.detach(), cols=3).clone()
        P = q.shape[0]
        hist = torch.empty((steps + 1, P), dtype=self.real, device=self.device)
        g = grid.c()
        rp = sd_refine_params(int(method), float(lr_t), float(lr_q), float(mass), float(inertia), float(damping),
                              float(dt))
        self._check(self.lib.sd_refine(self.handle, fixed.handle, moving.handle, ct.byref(g), _ptr(q), _ptr(t), P,
                                       int(steps), ct.byref(rp), _ptr(hist), _stream(self.device)))
        return q, t[:, : self.dim], hist


class Octree:
    """Host-side adaptive tree of SDF sample cells (sd_octree_*); needs no GPU."""

    def __init__(self, dim: int, bnd, lo, size: float, depth_min: int, depth_max: int, tau: float,
                 clearance: float, band: float = math.inf):
        self.lib = load()
        b = np.asarray(bnd, dtype=np.float64)
        if b.ndim != 2:
            raise ValueError("bnd: expected an (n_b, dim..4) array")
        if b.shape[1] < 4:
            b = np.concatenate([b, np.zeros((b.shape[0], 4 - b.shape[1]))], 1)
        b = np.ascontiguousarray(b[:, :4])
        lo = np.ascontiguousarray(np.asarray(lo, dtype=np.float64).reshape(-1))
        if lo.shape[0] < dim:
            raise ValueError("lo: expected dim values")
        self.dim = dim
        self.handle = ct.c_void_p()
        rc = self.lib.sd_octree_create(dim, b.ctypes.data if len(b) else None, b.shape[0], lo.ctypes.data,
                                       float(size), depth_min, depth_max, float(tau), float(clearance),
                                       float(band), ct.byref(self.handle))
        if rc != SD_OK:
            raise SdError(rc, "octree_create failed")

    def _check(self, rc, what):
        if rc != SD_OK:
            raise SdError(rc, f"octree_{what} failed")

    def pending(self):
        """Centres (n, 4) and volumes (n,) of the cells that need rho."""
        n = ct.c_int64()
        self._check(self.lib.sd_octree_pending(self.handle, ct.byref(n), None, None), "pending")
        cen = np.zeros((n.value, 4))
        vol = np.zeros(n.value)
        if n.value:
            self._check(self.lib.sd_octree_pending(self.handle, ct.byref(n), cen.ctypes.data, vol.ctypes.data),
                        "pending")
        return cen, vol

    def feed(self, rho):
        """rho at the pending centres: (n, 2) real pairs, (n,) complex or (n,) real."""
        r = np.asarray(rho)
        if np.iscomplexobj(r) or r.ndim == 1:
            r = np.stack([r.real, np.imag(r)], -1)
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 2)
        self._check(self.lib.sd_octree_feed(self.handle, r.ctypes.data if len(r) else None, r.shape[0]), "feed")

    def leaves(self):
        """Centres (m, 4), volumes (m,) and int32 coords (m, 4: k_x, k_y, k_z, depth) of the leaves."""
        m = ct.c_int64()
        self._check(self.lib.sd_octree_leaves(self.handle, ct.byref(m), None, None, None), "leaves")
        cen = np.zeros((m.value, 4))
        vol = np.zeros(m.value)
        crd = np.zeros((m.value, 4), np.int32)
        if m.value:
            self._check(self.lib.sd_octree_leaves(self.handle, ct.byref(m), cen.ctypes.data, vol.ctypes.data,
                                                  crd.ctypes.data), "leaves")
        return cen, vol, crd

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sd_octree_free(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass


PEAK_KINDS = {"fp32_fma": 0, "fp64_fma": 1, "sfu_ex2": 2, "sfu_rsqrt": 3, "shared_add32": 4, "shared_add64": 5}


def alu_peak(kind: str, device: int = 0) -> float:
    """Measured rate of one arithmetic class on a device (sd_alu_peak): FLOP/s for
    the FMA kinds, instructions/s for the special-function kinds."""
    lib = load()
    v = ct.c_double()
    rc = lib.sd_alu_peak(int(device), PEAK_KINDS[kind], ct.byref(v))
    if rc != 0:
        raise SdError(rc, f"sd_alu_peak({kind}) failed")
    return v.value


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().sd_launch_count())


def decode_cands(buf: torch.Tensor):
    """(score float64, rot int32, idx int32) views of a candidate buffer."""
    b = buf.reshape(-1, CAND_BYTES)
    score = b[:, :8].contiguous().view(torch.float64).reshape(-1)
    ri = b[:, 8:].contiguous().view(torch.int32).reshape(-1, 2)
    return score, ri[:, 0], ri[:, 1]


# ---------------------------------------------------------------------------
# autograd and refinement (Section 6: gradient-driven search of the score)
# ---------------------------------------------------------------------------

class SdfScore(torch.autograd.Function):
    """score = Re f_N(q, t); backward returns d score/dq and d score/dt from the type-2 gather."""

    @staticmethod
    def forward(fctx, quats, trans, ctx: Context, fixed: Shape, moving: Shape, grid: Grid):
        score, dq, dt = ctx.score_grad(fixed, moving, grid, quats.detach(), trans.detach())
        fctx.save_for_backward(dq, dt)
        fctx.tdim = trans.shape[-1]
        return score.to(quats.dtype)

    @staticmethod
    def backward(fctx, g):
        dq, dt = fctx.saved_tensors
        gq = g[:, None].to(dq.dtype) * dq
        gt = g[:, None].to(dt.dtype) * dt[:, : fctx.tdim]
        return gq, gt, None, None, None, None


def sdf_score(ctx: Context, fixed: Shape, moving: Shape, grid: Grid, quats: torch.Tensor, trans: torch.Tensor):
    return SdfScore.apply(quats, trans, ctx, fixed, moving, grid)


def refine_poses(ctx: Context, fixed: Shape, moving: Shape, grid: Grid, q0: torch.Tensor, t0: torch.Tensor,
                 steps: int = 50, lr_t: float = 0.05, lr_q: float = 0.02):
    """Gradient ascent on the score from P starting poses (all on the device).

    Each step normalises the step by the largest gradient entry so the sizes
    lr_t (length) and lr_q (quaternion units) are the largest moves per step.
    Returns (q, t, score history (steps+1, P)).
    """
    q = q0.detach().clone().to(ctx.real).requires_grad_(True)
    t = t0.detach().clone().to(ctx.real).requires_grad_(True)
    hist = []
    for _ in range(steps):
        s = sdf_score(ctx, fixed, moving, grid, q, t)
        hist.append(s.detach())
        gq, gt = torch.autograd.grad(s.sum(), (q, t))
        with torch.no_grad():
            st = gt.abs().amax(dim=1, keepdim=True).clamp_min(1e-30)
            sq = gq.abs().amax(dim=1, keepdim=True).clamp_min(1e-30)
            t += lr_t * gt / st
            q += lr_q * gq / sq
            q /= q.norm(dim=1, keepdim=True)
    with torch.no_grad():
        hist.append(ctx.score_grad(fixed, moving, grid, q, t)[0])
    return q.detach(), t.detach(), torch.stack(hist)


# ---------------------------------------------------------------------------
# rotation sharding across ranks (host logic)
# ---------------------------------------------------------------------------

def shard_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [lo, hi) share of n rotations for a rank."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def merge_top_k(parts, k: int):
    """Merge per-rank lists of (score, rot, idx) into the global top-k (score desc, rot asc, idx asc).

    Entries with rot < 0 are the padding a rank returns when it has fewer than k
    candidates; they are dropped, so they never rank ahead of a real candidate
    whose score is -inf or NaN (NaN ranks with -inf, last)."""
    allc = [c for p in parts for c in p if c[1] >= 0]
    allc.sort(key=lambda c: (-c[0] if c[0] == c[0] else math.inf, c[1], c[2]))
    return allc[:k]
