"""ctypes binding of libspectral_rt.so (argument marshalling only).

Every step of the path runs in the library's CUDA kernels.  There is no
fallback: if the library is missing or no CUDA device is present, loading
raises.  PyTorch supplies device memory (tensors) and the stream.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libspectral_rt.so")

RT_OK = 0
STATUS_NAMES = {0: "RT_OK", 1: "RT_ERR_ARG", 2: "RT_ERR_SCENE", 3: "RT_ERR_OOM", 4: "RT_ERR_CUDA",
                5: "RT_ERR_QUEUE_OVERFLOW", 6: "RT_ERR_TIMEOUT", 7: "RT_ERR_STATE", 8: "RT_ERR_STACK"}
XYZ_BF16X3, XYZ_BF16, XYZ_FP64 = 0, 1, 2

# every exported symbol of include/spectral_rt.h
EXPORTS = ["rt_create", "rt_destroy", "rt_last_error", "rt_set_stream", "rt_set_counting", "rt_set_timing",
           "rt_load_scene", "rt_set_spectra", "rt_render", "rt_render_host", "rt_philox", "rt_trace_closest",
           "rt_trace_shadow", "rt_optics_eval", "rt_xyz", "rt_probe_l2", "rt_render_static", "rt_guide_init",
           "rt_guide_set_params", "rt_guide_get_params", "rt_guide_eval", "rt_guide_grad", "rt_guide_train_step", "rt_guide_sample_step", "rt_autotune",
           "rt_set_bvh_builder", "rt_get_scene_info", "rt_set_limits", "rt_render_photons", "rt_photon_records"]


class RtError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} -> {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("look", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_uint32), ("height", C.c_uint32)]


class RenderOpts(C.Structure):
    _fields_ = [("wave_capacity", C.c_uint32), ("xyz_mode", C.c_uint32), ("trace_block", C.c_uint32),
                ("ctas_per_sm", C.c_uint32), ("probe_map_dev", C.c_void_p), ("probe_L_dev", C.c_void_p),
                ("probe_sig_dev", C.c_void_p), ("use_graph", C.c_uint32), ("trace_variant", C.c_uint32),
                ("trace_steps", C.c_uint32), ("trace_refill", C.c_uint32), ("shadow_steps", C.c_uint32),
                ("shadow_refill", C.c_uint32), ("guided", C.c_uint32), ("guide_collect", C.c_uint32),
                ("guide_train_steps", C.c_uint32), ("guide_batch", C.c_uint32), ("sample_first", C.c_uint32),
                ("accumulate", C.c_uint32), ("spp_total", C.c_uint32), ("leaf_batch", C.c_uint32),
                ("guide_order", C.c_uint32), ("ray_order", C.c_uint32), ("bands_per_path", C.c_uint32),
                ("guide_records_dev", C.c_void_p)]


class PhotonOpts(C.Structure):
    _fields_ = [("n_photons", C.c_uint32), ("photon_depth", C.c_uint32), ("r_caustic", C.c_float),
                ("r_global", C.c_float), ("log2_cells", C.c_uint32), ("xyz_mode", C.c_uint32),
                ("probe_map_dev", C.c_void_p), ("probe_L_dev", C.c_void_p), ("probe_sig_dev", C.c_void_p),
                ("emission", C.c_uint32), ("reserved", C.c_uint32 * 3)]


class SceneInfo(C.Structure):
    _fields_ = [("n_tris", C.c_uint32), ("n_nodes4", C.c_uint32), ("builder", C.c_uint32), ("build_ms", C.c_float)]


class AutotuneReport(C.Structure):
    _fields_ = [("trials", C.c_uint32), ("best_ms", C.c_float), ("default_ms", C.c_float)]


class GuideConfig(C.Structure):
    _fields_ = [("log2_table", C.c_uint32), ("n_min", C.c_float), ("n_max", C.c_float), ("lr_grid", C.c_float),
                ("lr_mlp", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("mis_alpha", C.c_float), ("guide_depth", C.c_uint32), ("reserved", C.c_uint32 * 6)]


GUIDE_W_SIZE = 64 * 64 * 3 + 64 * 48
GUIDE_GRID_LEVELS, GUIDE_GRID_FEATURES = 8, 4  # hash grid [levels][2^log2_table][features]


class Stats(C.Structure):
    _fields_ = [("paths", C.c_uint64), ("ext_rays", C.c_uint64), ("shadow_rays", C.c_uint64),
                ("nodes_visited", C.c_uint64), ("tris_tested", C.c_uint64),
                ("shadow_nodes_visited", C.c_uint64), ("shadow_tris_tested", C.c_uint64), ("waves", C.c_uint32),
                ("kernel_launches", C.c_uint32), ("ms_render", C.c_float), ("ms_xyz", C.c_float),
                ("ms_stage", C.c_float * 7), ("launches_stage", C.c_uint32 * 7)]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if k in ("ms_stage", "launches_stage") else v
        return d


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run paper_1912_04000_gb300.build.build())")
        L = C.CDLL(path)
        vp, u32, u64, i32, f32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32, C.c_float
        L.rt_create.argtypes = [C.c_int, vp, C.POINTER(vp)]
        L.rt_destroy.argtypes = [vp]
        L.rt_destroy.restype = None
        L.rt_last_error.argtypes = [vp]
        L.rt_last_error.restype = C.c_char_p
        L.rt_set_stream.argtypes = [vp, vp]
        L.rt_set_counting.argtypes = [vp, C.c_int]
        L.rt_set_timing.argtypes = [vp, C.c_int]
        L.rt_probe_l2.argtypes = [vp, u64, u32, C.POINTER(C.c_float)]
        L.rt_load_scene.argtypes = [vp, vp, u32, vp, u32, vp, vp, vp, u32]
        L.rt_set_bvh_builder.argtypes = [vp, u32]
        L.rt_set_limits.argtypes = [vp, u32, u32, u32]
        L.rt_get_scene_info.argtypes = [vp, C.POINTER(SceneInfo)]
        L.rt_set_spectra.argtypes = [vp, vp, u32, vp, vp, f32, vp, vp, vp, vp, vp]
        L.rt_render.argtypes = [vp, C.POINTER(Camera), u32, u32, u32, u32, u32, u64, C.POINTER(RenderOpts), vp, vp,
                                C.POINTER(Stats)]
        L.rt_render_host.argtypes = [vp, C.POINTER(Camera), u32, u32, u32, u32, u32, u64, C.POINTER(RenderOpts), vp,
                                     vp, C.POINTER(Stats)]
        L.rt_render_static.argtypes = [vp, C.POINTER(Camera), u32, u32, u32, u32, u32, u64, u32, vp, vp]
        L.rt_guide_init.argtypes = [vp, C.POINTER(GuideConfig), u64]
        L.rt_guide_set_params.argtypes = [vp, vp, vp]
        L.rt_guide_get_params.argtypes = [vp, vp, vp]
        L.rt_guide_eval.argtypes = [vp, vp, u64, vp, vp]
        L.rt_guide_grad.argtypes = [vp, vp, u64, C.POINTER(C.c_float), vp, vp]
        L.rt_guide_train_step.argtypes = [vp, vp, u64, C.POINTER(C.c_float)]
        L.rt_guide_sample_step.argtypes = [vp, vp, u32, u32, u32, u32, u32, u64, vp]
        L.rt_autotune.argtypes = [vp, C.POINTER(Camera), u32, u32, u32, u32, u32, C.POINTER(RenderOpts),
                                  C.POINTER(AutotuneReport)]
        L.rt_philox.argtypes = [vp, vp, vp, u64, u32, u32]
        L.rt_trace_closest.argtypes = [vp, vp, vp, u64, vp, vp]
        L.rt_trace_shadow.argtypes = [vp, vp, vp, vp, u64, vp, vp]
        L.rt_optics_eval.argtypes = [vp, vp, vp, vp, vp, vp, u64, vp, vp, vp]
        L.rt_xyz.argtypes = [vp, vp, u64, u32, u32, u32, u32, vp]
        L.rt_render_photons.argtypes = [vp, C.POINTER(Camera), u32, u32, u32, u32, u32, u64, C.POINTER(PhotonOpts),
                                        vp, vp, C.POINTER(Stats)]
        L.rt_photon_records.argtypes = [vp, u32, u32, u32, u32, u64, u32, vp, vp]
        for name in EXPORTS:
            if name not in ("rt_destroy", "rt_last_error"):
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


def cameras_struct(cameras):
    arr = (Camera * len(cameras))()
    for i, c in enumerate(cameras):
        arr[i].pos[:] = [float(x) for x in c.pos]
        arr[i].look[:] = [float(x) for x in c.look]
        arr[i].up[:] = [float(x) for x in c.up]
        arr[i].vfov_deg = float(c.vfov_deg)
        arr[i].width = int(c.width)
        arr[i].height = int(c.height)
    return arr
