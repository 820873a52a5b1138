"""Python face of the C ABI: a Renderer owns one rt_ctx on one CUDA device.

Tensors are torch CUDA tensors (device memory from PyTorch's allocator); the
library enqueues on the torch stream given at construction.  Each method is a
single C-ABI call plus argument marshalling.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import _native


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _need(ok: bool, what: str):
    if not ok:
        raise ValueError(what)


def _check_device_out(t, n: int, dtype, device, what: str):
    """A caller-supplied device output: the library writes n elements of
    dtype through its pointer, so it must be a contiguous tensor of exactly
    n elements of that dtype on the renderer's device."""
    _need(hasattr(t, "data_ptr") and t.device == device and t.dtype == dtype and t.is_contiguous()
          and t.numel() == n, f"{what}: expected a contiguous {dtype} tensor of {n} elements on {device}")


def _check_host_out(a, n: int, np_dtype, what: str):
    """A caller-supplied host output: a C-contiguous numpy array or a
    contiguous CPU tensor of exactly n elements of the dtype."""
    if hasattr(a, "data_ptr"):
        ok = (a.device.type == "cpu" and a.is_contiguous() and a.numel() == n
              and str(a.dtype) == "torch." + np.dtype(np_dtype).name)
    else:
        ok = isinstance(a, np.ndarray) and a.dtype == np_dtype and a.flags.c_contiguous and a.size == n
    _need(ok, f"{what}: expected a contiguous host {np.dtype(np_dtype).name} buffer of {n} elements")


class Renderer:
    def __init__(self, device: int = 0, stream=None):
        import torch

        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("spectral_rt needs a CUDA device (no CPU fallback)")
        self.lib = _native.load()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        st = self.lib.rt_create(device, C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != 0:
            raise _native.RtError("rt_create", st, "device or allocation failure")
        self._h = h
        self.n_bands = 0
        self.n_mat = 0

    # -- plumbing ---------------------------------------------------------------
    def _check(self, fn: str, st: int):
        if st != 0:
            msg = self.lib.rt_last_error(self._h)
            raise _native.RtError(fn, st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            self.lib.rt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_counting(self, on: bool):
        self._check("rt_set_counting", self.lib.rt_set_counting(self._h, 1 if on else 0))

    def set_limits(self, queue_capacity: int = 0, traversal_steps: int = 0, fail_cuda_call: int = 0):
        """Diagnostic limits (rt_set_limits): small ray queues, capped
        traversal loops, an injected CUDA failure; zeros restore the defaults."""
        self._check("rt_set_limits", self.lib.rt_set_limits(self._h, queue_capacity, traversal_steps, fail_cuda_call))

    def set_timing(self, on: bool):
        self._check("rt_set_timing", self.lib.rt_set_timing(self._h, 1 if on else 0))

    def probe_l2(self, nbytes: int = 48 << 20, iters: int = 50) -> float:
        g = C.c_float()
        self._check("rt_probe_l2", self.lib.rt_probe_l2(self._h, nbytes, iters, C.byref(g)))
        return float(g.value)

    # -- scene and spectra ------------------------------------------------------
    def load_scene(self, scene, builder: int = 2):
        """builder 0: binned SAH on the host; 1: linear BVH on the device; 2 (default): SAH with
        spatial splits."""
        self._check("rt_set_bvh_builder", self.lib.rt_set_bvh_builder(self._h, int(builder)))
        v = np.ascontiguousarray(scene.verts, np.float32)
        t = np.ascontiguousarray(scene.tris, np.uint32)
        m = np.ascontiguousarray(scene.mat_id, np.uint32)
        mt = np.ascontiguousarray(scene.mat_type, np.int32)
        th = np.ascontiguousarray(scene.mat_thickness, np.float32)
        st = self.lib.rt_load_scene(self._h, v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0], m.ctypes.data,
                                    mt.ctypes.data, th.ctypes.data, mt.shape[0])
        self._check("rt_load_scene", st)
        self.n_mat = mt.shape[0]

    def set_spectra(self, sp):
        arrs = [np.ascontiguousarray(a, np.float32) for a in
                (sp.lambda_nm, sp.sun_L, sp.sun_dir, sp.n, sp.k, sp.rho, sp.le, sp.cmf_w)]
        lam, sun_L, sun_dir, n, k, rho, le, w = arrs
        st = self.lib.rt_set_spectra(self._h, lam.ctypes.data, lam.shape[0], sun_L.ctypes.data, sun_dir.ctypes.data,
                                     float(sp.sun_half_angle), n.ctypes.data, k.ctypes.data, rho.ctypes.data,
                                     le.ctypes.data, w.ctypes.data)
        self._check("rt_set_spectra", st)
        self.n_bands = lam.shape[0]

    def load(self, workload, builder: int = 2):
        self.load_scene(workload.scene, builder)
        self.set_spectra(workload.spectra)
        return self

    def scene_info(self) -> dict:
        info = _native.SceneInfo()
        self._check("rt_get_scene_info", self.lib.rt_get_scene_info(self._h, C.byref(info)))
        return {"n_tris": info.n_tris, "n_nodes4": info.n_nodes4,
                "builder": ("host_sah", "device_lbvh", "host_sbvh")[info.builder],
                "build_ms": info.build_ms}

    # -- render -----------------------------------------------------------------
    def render(self, cameras: Sequence, spp: int, depth: int, seed: int = 0, band_first: int = 0,
               band_count: Optional[int] = None, spectral: bool = True, xyz: bool = True,
               xyz_mode: int = _native.XYZ_BF16X3, wave_capacity: int = 0, probe_pixels=None,
               trace_block: int = 0, ctas_per_sm: int = 0, out_spectral=None, out_xyz=None, trace_variant: int = 0,
               trace_steps: int = 0, trace_refill: int = 0, shadow_steps: int = 0, shadow_refill: int = 0,
               guided: bool = False, guide_collect: int = 0, guide_train_steps: int = 0, guide_batch: int = 0,
               sample_first: int = 0, accumulate: bool = False, spp_total: int = 0, use_graph: bool = False,
               tuned: Optional[dict] = None, leaf_batch: int = 0, guide_order: int = 0, ray_order: int = 0,
               bands_per_path: int = 1, guide_records: bool = False):
        """Returns dict(spectral [P, band_count] f64 sums over samples,
        xyz [P, 3] f32, stats, probe_L / probe_sig [n_probe, spp, band_count]
        when probe_pixels is given, and with guide_records (guided,
        guide_collect = 1) the training records in path order,
        [guide_depth, spp * P * band_count, 2, 12])."""
        torch = self.torch
        if band_count is None:
            band_count = self.n_bands - band_first
        npix = sum(int(c.width) * int(c.height) for c in cameras)
        dev = self.device
        if out_spectral is not None:
            _check_device_out(out_spectral, npix * band_count, torch.float64, dev, "out_spectral")
        if out_xyz is not None:
            _check_device_out(out_xyz, npix * 3, torch.float32, dev, "out_xyz")
        sp = out_spectral if out_spectral is not None else (
            torch.empty((npix, band_count), dtype=torch.float64, device=dev) if spectral else None)
        xz = out_xyz if out_xyz is not None else (
            torch.empty((npix, 3), dtype=torch.float32, device=dev) if xyz else None)
        opts = _native.RenderOpts()
        opts.wave_capacity = wave_capacity
        opts.xyz_mode = xyz_mode
        opts.trace_block = trace_block
        opts.ctas_per_sm = ctas_per_sm
        opts.trace_variant = trace_variant
        opts.leaf_batch = leaf_batch
        opts.guide_order = guide_order
        opts.ray_order = ray_order
        opts.bands_per_path = bands_per_path
        opts.trace_steps, opts.trace_refill = trace_steps, trace_refill
        opts.shadow_steps, opts.shadow_refill = shadow_steps, shadow_refill
        opts.guided, opts.guide_collect = int(guided), guide_collect
        opts.guide_train_steps, opts.guide_batch = guide_train_steps, guide_batch
        opts.sample_first, opts.accumulate, opts.spp_total = sample_first, int(accumulate), spp_total
        opts.use_graph = int(use_graph)
        for k_, v_ in (tuned or {}).items():
            setattr(opts, k_, int(v_))
        out = {}
        if probe_pixels is not None:
            pp = torch.as_tensor(np.asarray(probe_pixels, np.int64), device=dev)
            pmap = torch.full((npix,), -1, dtype=torch.int64, device=dev)
            pmap[pp] = torch.arange(pp.shape[0], device=dev)
            pmap32 = pmap.to(torch.int32)
            pl = torch.zeros((pp.shape[0], spp, band_count), dtype=torch.float32, device=dev)
            ps = torch.zeros((pp.shape[0], spp, band_count), dtype=torch.int32, device=dev)
            opts.probe_map_dev = pmap32.data_ptr()
            opts.probe_L_dev = pl.data_ptr()
            opts.probe_sig_dev = ps.data_ptr()
            out["probe_L"] = pl
            out["probe_sig"] = ps
            out["_keep"] = pmap32
        if guide_records:
            _need(guided and guide_collect == 1, "guide_records needs guided=True and guide_collect=1")
            gd = min(self.guide_depth, depth)
            gr = torch.zeros((gd, spp * npix * band_count, 2, 12), dtype=torch.float32, device=dev)
            opts.guide_records_dev = gr.data_ptr()
            out["guide_records"] = gr
        cams = _native.cameras_struct(cameras)
        stats = _native.Stats()
        st = self.lib.rt_render(self._h, cams, len(cameras), band_first, band_count, spp, depth, seed,
                                C.byref(opts), _ptr(sp), _ptr(xz), C.byref(stats))
        self._check("rt_render", st)
        out.update(spectral=sp, xyz=xz, stats=stats.as_dict())
        return out

    def render_photons(self, cameras: Sequence, spp: int, depth: int, seed: int = 0, band_first: int = 0,
                       band_count: Optional[int] = None, n_photons: int = 0, photon_depth: int = 0,
                       r_caustic: float = 0.0, r_global: float = 0.0, log2_cells: int = 0,
                       xyz_mode: int = _native.XYZ_BF16X3, probe_pixels=None, out_spectral=None, emission: int = 0):
        """Photon-mapping render (rt_render_photons): dict(spectral [P, band_count]
        f64 sums over samples, xyz [P, 3], stats, probe_L / probe_sig)."""
        torch = self.torch
        if band_count is None:
            band_count = self.n_bands - band_first
        npix = sum(int(c.width) * int(c.height) for c in cameras)
        dev = self.device
        if out_spectral is not None:
            _check_device_out(out_spectral, npix * band_count, torch.float64, dev, "out_spectral")
        sp = out_spectral if out_spectral is not None else torch.empty((npix, band_count), dtype=torch.float64,
                                                                      device=dev)
        xz = torch.empty((npix, 3), dtype=torch.float32, device=dev)
        o = _native.PhotonOpts()
        o.n_photons, o.photon_depth, o.log2_cells, o.xyz_mode = n_photons, photon_depth, log2_cells, xyz_mode
        o.r_caustic, o.r_global, o.emission = r_caustic, r_global, emission
        out = {}
        if probe_pixels is not None:
            pp = torch.as_tensor(np.asarray(probe_pixels, np.int64), device=dev)
            pmap = torch.full((npix,), -1, dtype=torch.int64, device=dev)
            pmap[pp] = torch.arange(pp.shape[0], device=dev)
            pmap32 = pmap.to(torch.int32)
            pl = torch.zeros((pp.shape[0], spp, band_count), dtype=torch.float32, device=dev)
            ps = torch.zeros((pp.shape[0], spp, band_count), dtype=torch.int32, device=dev)
            o.probe_map_dev, o.probe_L_dev, o.probe_sig_dev = pmap32.data_ptr(), pl.data_ptr(), ps.data_ptr()
            out.update(probe_L=pl, probe_sig=ps, _keep=pmap32)
        stats = _native.Stats()
        st = self.lib.rt_render_photons(self._h, _native.cameras_struct(cameras), len(cameras), band_first,
                                        band_count, spp, depth, seed, C.byref(o), _ptr(sp), _ptr(xz),
                                        C.byref(stats))
        self._check("rt_render_photons", st)
        out.update(spectral=sp, xyz=xz, stats=stats.as_dict())
        return out

    def photon_records(self, n_photons: int, depth: int, seed: int = 0, band_first: int = 0,
                       band_count: Optional[int] = None, emission: int = 0):
        """Photon pass alone: (records [band_count, n_photons, depth, 4] float32
        {x, y, z, flux}, classes [band_count, n_photons, depth] uint8)."""
        torch = self.torch
        if band_count is None:
            band_count = self.n_bands - band_first
        rec = torch.zeros((band_count, n_photons, depth, 4), dtype=torch.float32, device=self.device)
        cls = torch.zeros((band_count, n_photons, depth), dtype=torch.uint8, device=self.device)
        st = self.lib.rt_photon_records(self._h, band_first, band_count, n_photons, depth, seed, emission,
                                        rec.data_ptr(), cls.data_ptr())
        self._check("rt_photon_records", st)
        return rec, cls

    HOST_OPTS = ("guided", "guide_collect", "guide_train_steps", "guide_batch", "sample_first", "accumulate",
                 "spp_total")

    def render_host(self, cameras, spp, depth, seed=0, band_first=0, band_count=None, spectral=False,
                    xyz_mode=_native.XYZ_BF16X3, wave_capacity=0, xyz_out=None, spectral_out=None, **opts_kw):
        """Host outputs (numpy; pinned torch tensors may be passed as outputs).
        opts_kw: further rt_render_opts fields among HOST_OPTS (guided
        rendering with online training, progressive sample ranges)."""
        for k_ in opts_kw:
            _need(k_ in self.HOST_OPTS, f"render_host: unknown option {k_}")
        if band_count is None:
            band_count = self.n_bands - band_first
        npix = sum(int(c.width) * int(c.height) for c in cameras)
        if xyz_out is not None:
            _check_host_out(xyz_out, npix * 3, np.float32, "xyz_out")
        if spectral_out is not None:
            _check_host_out(spectral_out, npix * band_count, np.float64, "spectral_out")
        xz = xyz_out if xyz_out is not None else np.empty((npix, 3), np.float32)
        sp = spectral_out if spectral_out is not None else (
            np.empty((npix, band_count), np.float64) if spectral else None)
        addr = lambda a: None if a is None else (a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)
        opts = _native.RenderOpts()
        opts.wave_capacity = wave_capacity
        opts.xyz_mode = xyz_mode
        for k_, v_ in opts_kw.items():
            setattr(opts, k_, int(v_))
        cams = _native.cameras_struct(cameras)
        stats = _native.Stats()
        st = self.lib.rt_render_host(self._h, cams, len(cameras), band_first, band_count, spp, depth, seed,
                                     C.byref(opts), addr(sp), addr(xz), C.byref(stats))
        self._check("rt_render_host", st)
        return {"xyz": xz, "spectral": sp, "stats": stats.as_dict()}

    # -- single steps -------------------------------------------------------------
    def philox(self, ctr, key0: int, key1: int):
        torch = self.torch
        ctr = ctr.to(self.device, torch.int32).contiguous()
        out = torch.empty_like(ctr)
        self._check("rt_philox", self.lib.rt_philox(self._h, ctr.data_ptr(), out.data_ptr(), ctr.shape[0], key0, key1))
        return out

    def trace_closest(self, o, d):
        torch = self.torch
        o = torch.as_tensor(o, dtype=torch.float32, device=self.device).contiguous()
        d = torch.as_tensor(d, dtype=torch.float32, device=self.device).contiguous()
        n = o.shape[0]
        t = torch.empty(n, dtype=torch.float32, device=self.device)
        p = torch.empty(n, dtype=torch.int32, device=self.device)
        self._check("rt_trace_closest", self.lib.rt_trace_closest(self._h, o.data_ptr(), d.data_ptr(), n,
                                                                   t.data_ptr(), p.data_ptr()))
        return t, p

    def trace_shadow(self, o, d, band):
        torch = self.torch
        o = torch.as_tensor(o, dtype=torch.float32, device=self.device).contiguous()
        d = torch.as_tensor(d, dtype=torch.float32, device=self.device).contiguous()
        n = o.shape[0]
        b = torch.as_tensor(np.broadcast_to(np.asarray(band, np.int32), (n,)).copy(), device=self.device)
        T = torch.empty(n, dtype=torch.float32, device=self.device)
        g = torch.empty(n, dtype=torch.int32, device=self.device)
        self._check("rt_trace_shadow", self.lib.rt_trace_shadow(self._h, o.data_ptr(), d.data_ptr(), b.data_ptr(), n,
                                                                 T.data_ptr(), g.data_ptr()))
        return T, g

    def optics(self, cos_i, n, k, lambda_nm=None, d=None):
        torch = self.torch
        f = lambda a: torch.as_tensor(np.asarray(a, np.float32), device=self.device).contiguous()
        c, nn, kk = f(cos_i), f(n), f(k)
        cnt = c.shape[0]
        R = torch.empty(cnt, dtype=torch.float32, device=self.device)
        lam = f(lambda_nm) if lambda_nm is not None else None
        dd = f(d) if d is not None else None
        Rs = torch.empty_like(R) if lam is not None else None
        Ts = torch.empty_like(R) if lam is not None else None
        st = self.lib.rt_optics_eval(self._h, c.data_ptr(), nn.data_ptr(), kk.data_ptr(), _ptr(lam), _ptr(dd), cnt,
                                     R.data_ptr(), _ptr(Rs), _ptr(Ts))
        self._check("rt_optics_eval", st)
        return R, Rs, Ts

    def xyz(self, spectral, band_first: int, spp: int, mode: int = _native.XYZ_BF16X3):
        torch = self.torch
        s = spectral.to(self.device, torch.float64).contiguous()
        out = torch.empty((s.shape[0], 3), dtype=torch.float32, device=self.device)
        st = self.lib.rt_xyz(self._h, s.data_ptr(), s.shape[0], band_first, s.shape[1], spp, mode, out.data_ptr())
        self._check("rt_xyz", st)
        return out

    # -- learned guide ------------------------------------------------------------
    def guide_init(self, seed: int = 0, **cfg):
        c = _native.GuideConfig()
        for k, v in cfg.items():
            setattr(c, k, v)
        self._check("rt_guide_init", self.lib.rt_guide_init(self._h, C.byref(c), seed))
        self.guide_log2_table = c.log2_table or 19
        self.guide_depth = c.guide_depth or 2
        self.guide_alpha = c.mis_alpha or 0.7

    def guide_set_params(self, grid=None, W=None):
        g = None if grid is None else np.ascontiguousarray(grid, np.float32).ravel()
        w = None if W is None else np.ascontiguousarray(W, np.float32).ravel()
        if hasattr(self, "guide_log2_table"):  # before guide_init the library refuses the call
            n_grid = _native.GUIDE_GRID_LEVELS * (1 << self.guide_log2_table) * _native.GUIDE_GRID_FEATURES
            _need(g is None or g.size == n_grid, f"grid: expected {n_grid} floats")
        _need(w is None or w.size == _native.GUIDE_W_SIZE, f"W: expected {_native.GUIDE_W_SIZE} floats")
        st = self.lib.rt_guide_set_params(self._h, None if g is None else g.ctypes.data,
                                          None if w is None else w.ctypes.data)
        self._check("rt_guide_set_params", st)

    def guide_get_params(self):
        g = np.zeros(_native.GUIDE_GRID_LEVELS * (1 << self.guide_log2_table) * _native.GUIDE_GRID_FEATURES, np.float32)
        w = np.zeros(_native.GUIDE_W_SIZE, np.float32)
        self._check("rt_guide_get_params", self.lib.rt_guide_get_params(self._h, g.ctypes.data, w.ctypes.data))
        return g, w

    def _records(self, rec):
        """Guide records [n][12] float32 on the device."""
        torch = self.torch
        if hasattr(rec, "data_ptr"):
            r = rec.to(self.device, torch.float32).contiguous()
        else:
            r = torch.as_tensor(np.ascontiguousarray(rec, np.float32), device=self.device).contiguous()
        _need(r.dim() == 2 and r.shape[1] == 12, "guide records: expected an [n, 12] array")
        return r

    def guide_eval(self, rec):
        torch = self.torch
        r = self._records(rec)
        n = r.shape[0]
        Y = torch.empty((n, 48), dtype=torch.float32, device=self.device)
        q = torch.empty(n, dtype=torch.float32, device=self.device)
        self._check("rt_guide_eval", self.lib.rt_guide_eval(self._h, r.data_ptr(), n, Y.data_ptr(), q.data_ptr()))
        return Y, q

    def guide_grad(self, rec):
        torch = self.torch
        r = self._records(rec)
        loss = C.c_float()
        dg = torch.empty(_native.GUIDE_GRID_LEVELS * (1 << self.guide_log2_table) * _native.GUIDE_GRID_FEATURES,
                         dtype=torch.float32, device=self.device)
        dw = torch.empty(_native.GUIDE_W_SIZE, dtype=torch.float32, device=self.device)
        st = self.lib.rt_guide_grad(self._h, r.data_ptr(), r.shape[0], C.byref(loss), dg.data_ptr(), dw.data_ptr())
        self._check("rt_guide_grad", st)
        return loss.value, dg, dw

    def guide_train_step(self, rec):
        if hasattr(rec, "data_ptr") and rec.device == self.device:
            r = rec
            _need(r.dtype == self.torch.float32 and r.is_contiguous() and r.dim() == 2 and r.shape[1] == 12,
                  "guide records: expected a contiguous float32 [n, 12] tensor")
        else:
            r = self._records(rec)
        loss = C.c_float()
        self._check("rt_guide_train_step", self.lib.rt_guide_train_step(self._h, r.data_ptr(), r.shape[0],
                                                                         C.byref(loss)))
        return loss.value

    STEP_FIELDS = ("omega_x", "omega_y", "omega_z", "pdf", "cos", "throughput", "nee_contrib", "esc_weight")

    def guide_sample_step(self, k, sample, band_first, band_count, seed, pos, normal, throughput, rho, sun_dir,
                          sun_contrib, has_sun):
        """rt_guide_sample_step on n vertices (vertex i: pixel i // band_count,
        band band_first + i % band_count): dict of float arrays named by
        STEP_FIELDS plus omega [n, 3] and continued [n] (bool)."""
        torch = self.torch
        pos = np.asarray(pos, np.float32).reshape(-1, 3)
        n = pos.shape[0]
        v = np.zeros((n, 16), np.float32)
        v[:, 0:3] = pos
        v[:, 3] = throughput
        v[:, 4:7] = np.asarray(normal, np.float32).reshape(-1, 3)
        v[:, 7] = rho
        v[:, 8:11] = np.asarray(sun_dir, np.float32).reshape(-1, 3)
        v[:, 11] = sun_contrib
        v.view(np.uint32)[:, 12] = np.asarray(has_sun, np.uint32)
        vd = torch.as_tensor(v, device=self.device).contiguous()
        od = torch.zeros((n, 12), dtype=torch.float32, device=self.device)
        st = self.lib.rt_guide_sample_step(self._h, vd.data_ptr(), n, k, sample, band_first, band_count, seed,
                                           od.data_ptr())
        self._check("rt_guide_sample_step", st)
        o = od.cpu().numpy()
        out = {f: o[:, i] for i, f in enumerate(self.STEP_FIELDS)}
        out["omega"] = o[:, 0:3]
        out["continued"] = o.view(np.uint32)[:, 8] == 1
        return out

    # -- autotuning ------------------------------------------------------------
    TUNED_FIELDS = ("wave_capacity", "trace_steps", "trace_refill", "shadow_steps", "shadow_refill", "trace_block",
                    "leaf_batch")

    def autotune(self, cameras, depth, band_first=0, band_count=None, spp_probe=1):
        """Native coordinate-descent autotuner (rt_autotune); returns
        (tuned option dict, report dict)."""
        if band_count is None:
            band_count = self.n_bands - band_first
        opts = _native.RenderOpts()
        rep = _native.AutotuneReport()
        cams = _native.cameras_struct(cameras)
        st = self.lib.rt_autotune(self._h, cams, len(cameras), band_first, band_count, spp_probe, depth,
                                  C.byref(opts), C.byref(rep))
        self._check("rt_autotune", st)
        return ({k: getattr(opts, k) for k in self.TUNED_FIELDS},
                {"trials": rep.trials, "best_ms": rep.best_ms, "default_ms": rep.default_ms})
