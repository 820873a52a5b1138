#!/usr/bin/env python
"""Throughput of the GB300 spectral path tracer: spectral paths per second.

Headline workload: the largest single-GPU configuration, the 2M-triangle
stained-glass nave (40 leaded windows with per-pane Gaussian absorption
bands, brass fittings), 4 views at 2048 x 1536, 81 bands 380-780 nm, depth
12, guided (the learned guide, trained online on the tracer's own samples
in every pass) and batched (all 4 views and all bands in one render call).
One step = one full-frame sample pass of that job: 4 x 2048 x 1536 x 81 =
1,019,215,872 spectral paths, accumulated in FP64 into the job's spectral
image (64 passes make the configuration's 64 spp), scene, spectra and guide
resident on the device.

Sub-records on one GPU: the 200k-triangle nave (1024 x 768, 81 bands,
16 spp, depth 8; one step = one whole render) and the equal-time MSE of the
guided against the plain tracer on a 256 x 192 view of that nave against a
4096-spp plain reference (the configuration's full-size form:
--guided-mse --mse-width 1024 --mse-height 768).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU FP64 oracle
(guided estimator, same network architecture) on this machine's host cores on
a bounded pixel sample of the headline workload.  Under torchrun each rank
renders the whole job with its own Philox key (independent sample passes,
weak scaling); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("spectral paths/s on 1 GB300 (2M-triangle stained-glass nave, 4 views 2048x1536, 81 bands, depth 12, "
          "guided + batched)")
UNIT = "paths/s"
WORKLOAD = "large_nave_2M_4x2048x1536_b81_d12_guided_batched"
NAVE_WORKLOAD = "nave_200k_1024x768_b81_spp16_d8"
# guide settings of the headline job: every 8th path keeps training slots,
# 8 Adam steps after each wave
GUIDE_COLLECT, GUIDE_STEPS = 8, 8
PROFILE_TXT = os.path.join(ROOT, "profiles", "k_trace_closest_large_nave.txt")
KERNEL_SOURCES = ["paper_1912_04000_gb300/csrc/rt_kernels.cu", "paper_1912_04000_gb300/csrc/rt_device.cuh"]


BUILDERS = {"host": 0, "device": 1, "sbvh": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--builder", default="sbvh", choices=["host", "device", "sbvh"],
                    help="BVH builder: binned SAH, device linear BVH, or SAH with spatial splits")
    ap.add_argument("--partition", default="samples", choices=["samples", "bands"],
                    help="several GPUs: each rank renders whole sample passes with its own Philox key (weak "
                         "scaling), or its band sub-domain of every pass with the XYZ partials reduced to "
                         "rank 0 over NCCL (strong scaling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-subrecords", action="store_true",
                    help="skip the 200k-triangle nave sub-record and the equal-time MSE sub-record")
    ap.add_argument("--cpu-pixels", type=int, default=32768,
                    help="oracle sample size (pixels of one guided pass, all bands)")
    ap.add_argument("--guided-mse", action="store_true",
                    help="equal-time MSE of the guided vs the plain tracer against a high-spp plain reference")
    ap.add_argument("--bands-mse", action="store_true",
                    help="equal-time MSE, four bands per path vs one (nave or crystal nave)")
    ap.add_argument("--bands-workload", default="nave", choices=["nave", "crystal_nave"])
    ap.add_argument("--photon-mse", action="store_true",
                    help="equal-time MSE, photon mapping vs path tracing (nave or crystal nave)")
    ap.add_argument("--photons", type=int, default=1 << 16, help="photons per band")
    ap.add_argument("--photon-depth", type=int, default=4)
    ap.add_argument("--r-caustic", type=float, default=0.0)
    ap.add_argument("--r-global", type=float, default=0.0)
    ap.add_argument("--photon-emission", type=int, default=0, choices=[0, 1],
                    help="photon emission: 0 disk around the scene, 1 thin-glass portals")
    ap.add_argument("--mse-width", type=int, default=256)
    ap.add_argument("--mse-height", type=int, default=192)
    ap.add_argument("--mse-ref-spp", type=int, default=4096)
    ap.add_argument("--mse-spp", type=int, default=256)
    ap.add_argument("--mse-train-spp", type=int, default=32)
    ap.add_argument("--guide-depth", type=int, default=2)
    ap.add_argument("--guide-collect", type=int, default=4)
    ap.add_argument("--guide-steps", type=int, default=32)
    ap.add_argument("--mis-alpha", type=float, default=0.7)
    ap.add_argument("--mse-configs", default="",
                    help="extra guide settings depth:collect:steps:alpha[:train_spp[:order]] separated by ';' "
                         "(one shared reference; order 1 = guide queries sorted by position)")
    return ap.parse_args()


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def read_profile():
    """ncu summary of the closest-hit kernel: DRAM bytes per traced ray,
    valid only for the kernel sources it was captured from."""
    try:
        kv = {}
        for line in open(PROFILE_TXT):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        return kv
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_median": statistics.median(pw) if pw else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def oracle_guide_for(wl, seed=0, log2_table=19):
    """A seeded network of the guide's architecture for the oracle's guided
    estimator (its cost per query does not depend on the weights)."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(seed)
    grid = (rng.normal(size=oracle.GUIDE_LEVELS * (1 << log2_table) * oracle.GUIDE_FEATURES) * 1e-2).astype(np.float32)
    W = (rng.normal(size=oracle.GUIDE_W_SIZE) * 0.2).astype(np.float32)
    lo = wl.scene.verts.min(0).astype(np.float32)
    hi = wl.scene.verts.max(0).astype(np.float32)
    return oracle.OracleGuide(log2_table, lo, hi, grid, W)


def cpu_baseline(wl, n_pix: int, seed: int = 0, guided: bool = True, sc=None, guide=None):
    """The oracle as it stands, all host cores, on a seeded pixel sample of
    one sample pass (guided estimator with guide depth 2 when guided)."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(12345 + seed)
    pix = np.sort(rng.choice(wl.n_pixels, min(n_pix, wl.n_pixels), replace=False)).astype(np.uint32)
    sc = sc or oracle.OracleScene(wl.scene, wl.spectra)
    threads = oracle.hardware_threads()
    spp = 1 if guided else wl.spp
    t0 = time.perf_counter()
    if guided:
        guide = guide or oracle_guide_for(wl)
        sc.render_guided(guide, wl.cameras, 1, wl.depth, wl.seed + seed, alpha=0.7, guide_depth=2, pixels=pix,
                         n_threads=threads)
    else:
        sc.render(wl.cameras, spp, wl.depth, wl.seed + seed, pixels=pix, n_threads=threads)
    dt = time.perf_counter() - t0
    paths = len(pix) * spp * wl.band_count
    what = ("guided, one pass (1 spp) of the 4-view 2M-triangle nave" if guided
            else f"{spp} spp of the 1024x768 200k-triangle nave")
    return {"value": paths / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{len(pix)} seeded pixels x {wl.band_count} bands x depth {wl.depth}, {what} "
                      f"({paths} paths, {dt:.1f} s)"}


def run_reference(args):
    """--impl reference: the CPU FP64 oracle on the host cores, guided
    estimator on the headline workload, a bounded pixel sample per step."""
    import oracle
    from paper_1912_04000_gb300 import multigpu, scenes
    info = multigpu.DistInfo(int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
    if info.rank != 0:
        return 0
    wl = scenes.large_nave(spp=1)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    guide = oracle_guide_for(wl)
    per_step = max(16, args.cpu_pixels // 4)
    for i in range(args.warmup):
        cpu_baseline(wl, per_step, seed=100 + i, sc=sc, guide=guide)
    secs = []
    r = None
    for i in range(args.steps):
        r = cpu_baseline(wl, per_step, seed=i, sc=sc, guide=guide)
        secs.append(per_step * wl.band_count / r["value"])
    paths = per_step * wl.band_count
    value = paths * args.steps / sum(secs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_pixels_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                         "sample": f"{per_step} seeded pixels per step x 81 bands x depth 12, one guided pass"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_guided_mse(args):
    """Equal-time MSE, guided vs plain (prints the result line)."""
    print(json.dumps(guided_mse(args)), flush=True)
    return 0


def guided_mse(args, R=None):
    """Equal-time MSE, guided vs plain, on the nave view at a reduced
    resolution (the 4096-spp plain reference is rendered by the GPU plain
    tracer, itself parity-checked against the oracle)."""
    import numpy as np
    import torch

    from paper_1912_04000_gb300 import scenes
    from paper_1912_04000_gb300.renderer import Renderer

    wl = scenes.nave(width=args.mse_width, height=args.mse_height)
    R = (R or Renderer(0)).load(wl, builder=BUILDERS[args.builder])
    dev = R.device
    P, B = wl.n_pixels, wl.band_count

    def timed(fn):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize(dev)
        return out, time.perf_counter() - t0

    # reference: plain tracer, independent seed
    ref_sp = torch.zeros((P, B), dtype=torch.float64, device=dev)
    ref, t_ref = timed(lambda: R.render(wl.cameras, args.mse_ref_spp, wl.depth, 777, out_spectral=ref_sp))
    ref_xyz = ref["xyz"].cpu().numpy().astype(np.float64)

    def mse(x):
        return float(np.mean((x - ref_xyz) ** 2))

    def relmse(x):
        return float(np.mean((x - ref_xyz) ** 2 / (ref_xyz ** 2 + 1e-2 * np.mean(ref_xyz ** 2))))

    # plain tracer at equal spp, and its time per spp
    q_sp = torch.zeros((P, B), dtype=torch.float64, device=dev)
    q_out, t_q = timed(lambda: R.render(wl.cameras, args.mse_spp, wl.depth, 0, out_spectral=q_sp))
    q_xyz = q_out["xyz"].cpu().numpy().astype(np.float64)
    t_per_spp = t_q / args.mse_spp

    settings = [(args.guide_depth, args.guide_collect, args.guide_steps, args.mis_alpha, args.mse_train_spp, 0)]
    for item in filter(None, args.mse_configs.split(";")):
        f = item.split(":")
        settings.append((int(f[0]), int(f[1]), int(f[2]), float(f[3]), int(f[4]) if len(f) > 4 else args.mse_train_spp,
                         int(f[5]) if len(f) > 5 else 0))
    results = []
    for depth_g, collect, steps, alpha, train_spp, order in settings:
        # guided: online training over the first passes, then frozen
        R.guide_init(seed=11, guide_depth=depth_g, mis_alpha=alpha)
        g_sp = torch.zeros((P, B), dtype=torch.float64, device=dev)
        n_train = min(train_spp, args.mse_spp)
        stage = [0.0] * 7

        def guided_run():
            out = None
            for s_ in range(n_train):
                out = R.render(wl.cameras, 1, wl.depth, 0, out_spectral=g_sp, sample_first=s_, accumulate=s_ > 0,
                               spp_total=args.mse_spp, guided=True, guide_collect=collect, guide_train_steps=steps,
                               guide_order=order)
                for i_, v_ in enumerate(out["stats"]["ms_stage"]):
                    stage[i_] += v_
            if args.mse_spp > n_train:
                out = R.render(wl.cameras, args.mse_spp - n_train, wl.depth, 0, out_spectral=g_sp,
                               sample_first=n_train, accumulate=n_train > 0, spp_total=args.mse_spp, guided=True,
                               guide_order=order)
                for i_, v_ in enumerate(out["stats"]["ms_stage"]):
                    stage[i_] += v_
            return out

        R.set_timing(True)
        g_out, t_guided = timed(guided_run)
        R.set_timing(False)
        g_xyz = g_out["xyz"].cpu().numpy().astype(np.float64)
        # plain tracer with as many spp as fit in the guided time
        spp_eq = max(1, int(round(t_guided / t_per_spp)))
        p_sp = torch.zeros((P, B), dtype=torch.float64, device=dev)
        p_out, t_plain = timed(lambda: R.render(wl.cameras, spp_eq, wl.depth, 0, out_spectral=p_sp))
        p_xyz = p_out["xyz"].cpu().numpy().astype(np.float64)
        results.append({
            "guide_depth": depth_g, "guide_collect": collect, "guide_steps_per_wave": steps, "mis_alpha": alpha,
            "guide_order": "spatial" if order else "queue",
            "train_spp": n_train,
            "stage_ms": dict(zip(["camera", "closest_hit", "shade_nee", "sun_rays", "xyz", "guide", "train"],
                                 [round(v_, 1) for v_ in stage])),
            "guided": {"seconds": t_guided, "spp": args.mse_spp, "mse": mse(g_xyz), "relmse": relmse(g_xyz)},
            "plain_equal_time": {"seconds": t_plain, "spp": spp_eq, "mse": mse(p_xyz), "relmse": relmse(p_xyz)},
            "mse_ratio_equal_time": mse(p_xyz) / max(mse(g_xyz), 1e-300),
            "mse_ratio_equal_spp": mse(q_xyz) / max(mse(g_xyz), 1e-300),
            "relmse_ratio_equal_time": relmse(p_xyz) / max(relmse(g_xyz), 1e-300),
        })
    best = max(results, key=lambda r: r["mse_ratio_equal_time"])
    line = {
        "metric": "equal-time MSE, guided vs plain (nave, XYZ, vs 4096-spp plain reference)",
        "config": {"workload": f"nave_200k_{args.mse_width}x{args.mse_height}_b81_d8",
                   "reference_spp": args.mse_ref_spp, "guided_spp": args.mse_spp, "train_spp": args.mse_train_spp},
        "plain_equal_spp": {"spp": args.mse_spp, "seconds": t_q, "mse": mse(q_xyz), "relmse": relmse(q_xyz)},
        "runs": results,
        "mse_ratio_plain_over_guided_equal_time": best["mse_ratio_equal_time"],
        "reference_seconds": t_ref,
    }
    return line


def run_bands_mse(args):
    """Equal-time MSE of four bands per path against one band per path on a
    nave view at reduced resolution; the reference is the one-band tracer at
    --mse-ref-spp with an independent seed."""
    import numpy as np
    import torch

    from paper_1912_04000_gb300 import scenes
    from paper_1912_04000_gb300.renderer import Renderer

    make = scenes.crystal_nave if args.bands_workload == "crystal_nave" else scenes.nave
    wl = make(width=args.mse_width, height=args.mse_height)
    R = Renderer(0).load(wl, builder=BUILDERS[args.builder])
    dev = R.device
    P, B = wl.n_pixels, wl.band_count

    def timed(fn):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize(dev)
        return out, time.perf_counter() - t0

    def run(spp, seed, bpp):
        sp = torch.zeros((P, B), dtype=torch.float64, device=dev)
        out, t = timed(lambda: R.render(wl.cameras, spp, wl.depth, seed, out_spectral=sp, bands_per_path=bpp))
        return out["xyz"].cpu().numpy().astype(np.float64), sp.cpu().numpy() / spp, t, out["stats"]

    ref_xyz, ref_sp, t_ref, _ = run(args.mse_ref_spp, 777, 1)

    def errs(x, s):
        return {"mse_xyz": float(np.mean((x - ref_xyz) ** 2)), "mse_spectral": float(np.mean((s - ref_sp) ** 2))}

    run(8, 5, 4)  # warm both paths
    run(8, 5, 1)
    spp1 = args.mse_spp
    x1, s1, t1, st1 = run(spp1, 0, 1)
    _, _, t4probe, _ = run(spp1, 0, 4)
    spp4 = max(1, int(round(spp1 * t1 / t4probe)))
    x4, s4, t4, st4 = run(spp4, 0, 4)
    e1, e4 = errs(x1, s1), errs(x4, s4)
    line = {
        "metric": "equal-time MSE, four bands per path vs one (XYZ and spectral, vs a one-band reference)",
        "config": {"workload": f"{args.bands_workload}_{args.mse_width}x{args.mse_height}_b{B}_d{wl.depth}",
                   "reference_spp": args.mse_ref_spp},
        "one_band": {"spp": spp1, "seconds": t1, "estimates_per_s": st1["paths"] / t1, "ext_rays": st1["ext_rays"],
                     **e1},
        "four_bands": {"spp": spp4, "seconds": t4, "estimates_per_s": st4["paths"] / t4,
                       "ext_rays": st4["ext_rays"], **e4},
        "mse_xyz_ratio_one_over_four_equal_time": e1["mse_xyz"] / max(e4["mse_xyz"], 1e-300),
        "mse_spectral_ratio_one_over_four_equal_time": e1["mse_spectral"] / max(e4["mse_spectral"], 1e-300),
        "reference_seconds": t_ref,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_photon_mse(args):
    """Equal-time MSE of photon mapping (section 4's estimator) against path
    tracing on a nave view at reduced resolution; the reference is the path
    tracer at --mse-ref-spp with an independent seed.  Photon mapping is
    biased (gather radius), so its error does not fall to zero with time."""
    import numpy as np
    import torch

    from paper_1912_04000_gb300 import scenes
    from paper_1912_04000_gb300.renderer import Renderer

    make = scenes.crystal_nave if args.bands_workload == "crystal_nave" else scenes.nave
    wl = make(width=args.mse_width, height=args.mse_height)
    R = Renderer(0).load(wl, builder=BUILDERS[args.builder])
    dev = R.device
    P, B = wl.n_pixels, wl.band_count

    def timed(fn):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize(dev)
        return out, time.perf_counter() - t0

    ref, t_ref = timed(lambda: R.render(wl.cameras, args.mse_ref_spp, wl.depth, 777))
    ref_xyz = ref["xyz"].cpu().numpy().astype(np.float64)

    def mse(x):
        return float(np.mean((x - ref_xyz) ** 2))

    pkw = dict(n_photons=args.photons, photon_depth=args.photon_depth, r_caustic=args.r_caustic,
               r_global=args.r_global, emission=args.photon_emission)
    R.render_photons(wl.cameras, 1, wl.depth, 5, **pkw)  # warm
    R.render(wl.cameras, 4, wl.depth, 5)
    pt, t_pt = timed(lambda: R.render(wl.cameras, args.mse_spp, wl.depth, 0))
    p1, t1 = timed(lambda: R.render_photons(wl.cameras, 1, wl.depth, 0, **pkw))
    p4, t4 = timed(lambda: R.render_photons(wl.cameras, 4, wl.depth, 0, **pkw))
    per_spp = max((t4 - t1) / 3.0, 1e-6)
    fixed = max(t1 - per_spp, 0.0)
    spp_pm = max(1, int(round((t_pt - fixed) / per_spp)))
    pm, t_pm = timed(lambda: R.render_photons(wl.cameras, spp_pm, wl.depth, 0, **pkw))
    e_pt, e_pm = mse(pt["xyz"].cpu().numpy().astype(np.float64)), mse(pm["xyz"].cpu().numpy().astype(np.float64))
    line = {
        "metric": "equal-time MSE, photon mapping vs path tracing (XYZ, vs a path-traced reference)",
        "config": {"workload": f"{args.bands_workload}_{args.mse_width}x{args.mse_height}_b{B}_d{wl.depth}",
                   "reference_spp": args.mse_ref_spp, "photons_per_band": args.photons,
                   "photon_depth": args.photon_depth,
                   "photon_emission": ("disk", "portals")[args.photon_emission]},
        "path_tracing": {"spp": args.mse_spp, "seconds": t_pt, "mse_xyz": e_pt},
        "photon_mapping": {"spp": spp_pm, "seconds": t_pm, "mse_xyz": e_pm,
                           "photon_pass_ms": pm["stats"]["ms_stage"][0], "map_build_ms": pm["stats"]["ms_stage"][1],
                           "camera_pass_ms": pm["stats"]["ms_stage"][2]},
        "mse_ratio_pt_over_pm_equal_time": e_pt / max(e_pm, 1e-300),
        "reference_seconds": t_ref,
    }
    print(json.dumps(line), flush=True)
    return 0


STAGES = ["camera", "closest_hit", "shade_nee", "sun_rays", "xyz", "guide", "train"]


def trace_roofline(R, counts, ms_trace, n_trace, ext_rays, prof_ok_traffic=None):
    """Roofline of the closest-hit kernel: algorithmic bytes per ray (child
    slots and triangles tested, from a counting pass, plus the ray and its
    hit record) times rays per launch over the launch's device time."""
    ext_nodes = counts["nodes_visited"] / max(counts["ext_rays"], 1)
    ext_tris = counts["tris_tested"] / max(counts["ext_rays"], 1)
    l2_gbs = R.probe_l2()
    launch_ms = ms_trace / max(n_trace, 1)
    rays_per_launch = ext_rays / max(n_trace, 1)
    bytes_per_ray = ext_nodes * 32.0 + ext_tris * 48.0 + 32.0 + 8.0
    achieved = rays_per_launch * bytes_per_ray / (launch_ms * 1e-3) / 1e9
    traffic = prof_ok_traffic * rays_per_launch if prof_ok_traffic is not None else None
    return {
        "kernel": "k_trace (closest hit)", "bound": "l2", "achieved": achieved, "peak": l2_gbs, "unit": "GB/s",
        "frac": achieved / l2_gbs if l2_gbs > 0 else None, "traffic": traffic,
        "peak_source": "L2 streaming-read probe (rt_probe_l2, 48 MiB x 50) measured in this run",
        "hbm_peak_measured": HBM_PEAK, "frac_of_hbm": achieved / HBM_PEAK,
        "algorithmic_bytes_per_ray": bytes_per_ray, "nodes_per_ray": ext_nodes, "tris_per_ray": ext_tris,
        "sun_child_slots_per_ray": counts["shadow_nodes_visited"] / max(counts["shadow_rays"], 1),
        "sun_tris_per_ray": counts["shadow_tris_tested"] / max(counts["shadow_rays"], 1),
        "launch_ms": launch_ms, "rays_per_launch": rays_per_launch,
    }


def measured_hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6777.0


HBM_PEAK = measured_hbm_peak()


def nave_subrecord(R, dev, steps=3):
    """The 200k-triangle nave at its configuration (one step = one whole
    render of 1,019,215,872 paths), timed with CUDA events on the stream."""
    import torch

    from paper_1912_04000_gb300 import scenes
    wl = scenes.nave()
    R.load(wl)
    spectral = torch.empty((wl.n_pixels, wl.band_count), dtype=torch.float64, device=dev)
    xyz = torch.empty((wl.n_pixels, 3), dtype=torch.float32, device=dev)
    R.set_counting(True)
    counts = R.render(wl.cameras, 1, wl.depth, 1, xyz=False)["stats"]
    R.set_counting(False)
    R.render(wl.cameras, wl.spp, wl.depth, 0, out_spectral=spectral, out_xyz=xyz)
    R.set_timing(True)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(R.stream)
    ms_trace, n_trace, ext_rays = 0.0, 0, 0
    stage = [0.0] * 7
    for _ in range(steps):
        st = R.render(wl.cameras, wl.spp, wl.depth, 0, out_spectral=spectral, out_xyz=xyz)["stats"]
        ms_trace += st["ms_stage"][1]
        n_trace += st["launches_stage"][1]
        ext_rays += st["ext_rays"]
        stage = [a + b for a, b in zip(stage, st["ms_stage"])]
    e1.record(R.stream)
    torch.cuda.synchronize(dev)
    R.set_timing(False)
    ms = e0.elapsed_time(e1) / steps
    roof = trace_roofline(R, counts, ms_trace, n_trace, ext_rays)
    roof["stage_ms_per_step"] = dict(zip(STAGES, [m / steps for m in stage]))
    return {"workload": NAVE_WORKLOAD, "value": wl.n_paths / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "steps": steps, "paths_per_step": wl.n_paths, "triangles": int(wl.scene.n_tris), "roofline": roof}


def main():
    args = parse()
    if args.photon_mse:
        return run_photon_mse(args)
    if args.bands_mse:
        return run_bands_mse(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.guided_mse:
        return run_guided_mse(args)

    import numpy as np
    import torch

    from paper_1912_04000_gb300 import multigpu, scenes
    from paper_1912_04000_gb300.renderer import Renderer

    info = multigpu.init_from_env("nccl")
    dev = torch.device("cuda", info.local_rank)
    torch.cuda.set_device(dev)
    wl = scenes.large_nave(spp=1)
    t_load = time.perf_counter()
    R = Renderer(info.local_rank).load(wl, builder=BUILDERS[args.builder])
    t_load = time.perf_counter() - t_load
    bvh_info = R.scene_info()
    R.guide_init(seed=11)
    bands_split = args.partition == "bands" and info.world > 1
    seed = wl.seed if bands_split else multigpu.rank_seed(wl.seed, info.rank)
    band_first, band_count = multigpu.band_shard(wl.band_count, info.world, info.rank) if bands_split \
        else (0, wl.band_count)
    stream = R.stream
    P, B = wl.n_pixels, band_count
    spectral = torch.empty((P, B), dtype=torch.float64, device=dev)
    xyz = torch.empty((P, 3), dtype=torch.float32, device=dev)
    guide_kw = dict(guided=True, guide_collect=GUIDE_COLLECT, guide_train_steps=GUIDE_STEPS)
    passes = [0]

    def step():
        i = passes[0]
        passes[0] += 1
        out = R.render(wl.cameras, 1, wl.depth, seed, band_first=band_first, band_count=band_count,
                       out_spectral=spectral, out_xyz=xyz, sample_first=i, accumulate=i > 0, spp_total=i + 1,
                       **guide_kw)
        if bands_split:
            # the spectral decomposition's one exchange: XYZ partials summed on rank 0
            import torch.distributed as dist
            with torch.cuda.stream(stream):
                dist.reduce(xyz, dst=0, op=dist.ReduceOp.SUM)
        return out

    # traversal counts for the algorithmic bytes (outside the timed region;
    # one frozen guided pass into the library's own buffers)
    R.set_counting(True)
    counts = R.render(wl.cameras, 1, wl.depth, seed + 99, guided=True, xyz=False, spectral=False)["stats"]
    R.set_counting(False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    # timed region: K sample passes of the job, device time from CUDA events on the stream
    R.set_timing(True)
    clocks = ClockSampler(info.local_rank)
    clocks.start()
    multigpu.barrier(info, dev)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    ms_trace, n_trace, ext_rays, paths = 0.0, 0, 0, 0
    stage_ms = [0.0] * 7
    for _ in range(args.steps):
        st = step()["stats"]
        launches += st["kernel_launches"]
        ms_trace += st["ms_stage"][1]
        n_trace += st["launches_stage"][1]
        ext_rays += st["ext_rays"]
        paths += st["paths"]
        stage_ms = [a + b for a, b in zip(stage_ms, st["ms_stage"])]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    multigpu.barrier(info, dev)
    clk = clocks.stop()
    R.set_timing(False)
    ms = e0.elapsed_time(e1)
    ms_max = multigpu.max_over_ranks(info, ms, dev)
    paths_all = multigpu.sum_over_ranks(info, float(paths), dev)
    value = paths_all / (ms_max * 1e-3)
    assert paths == wl.n_pixels * B * args.steps

    # end to end through the C ABI with host buffers: camera upload, one
    # guided pass with training, the pass's XYZ image copied back into pinned
    # host memory
    xyz_host = torch.empty((P, 3), dtype=torch.float32, pin_memory=True)
    R.render_host(wl.cameras, 1, wl.depth, seed, band_first=band_first, band_count=band_count, xyz_out=xyz_host,
                  **guide_kw)  # allocates the library's buffers
    multigpu.barrier(info, dev)
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        R.render_host(wl.cameras, 1, wl.depth, seed, band_first=band_first, band_count=band_count, xyz_out=xyz_host,
                      sample_first=i, **guide_kw)
    t_e2e = multigpu.max_over_ranks(info, time.perf_counter() - t0, dev)
    e2e_value = multigpu.sum_over_ranks(info, float(P * B * e2e_steps), dev) / t_e2e

    prof = read_profile()
    traffic_per_ray = None
    if prof.get("kernel_sources_sha") == kernel_hash() and "dram_bytes_per_ray" in prof:
        traffic_per_ray = float(prof["dram_bytes_per_ray"])
    roof = trace_roofline(R, counts, ms_trace, n_trace, ext_rays, traffic_per_ray)
    roof["stage_ms_per_step"] = dict(zip(STAGES, [m / args.steps for m in stage_ms]))
    roof["sun_rays_per_step"] = counts["shadow_rays"]
    if traffic_per_ray is not None:
        roof["ncu"] = {k: float(prof[k]) for k in ("dram_bytes_per_ray", "l1_throughput_pct", "l1_hit_rate_pct",
                                                    "lts_throughput_pct", "warps_active_pct") if k in prof}
        roof["ncu"]["source"] = os.path.relpath(PROFILE_TXT, ROOT)

    sub = {}
    if info.world == 1 and not args.no_subrecords:
        sub["nave_200k"] = nave_subrecord(R, dev)
        mse = guided_mse(args, R)
        sub["equal_time_mse"] = {
            "workload": mse["config"]["workload"], "reference_spp": mse["config"]["reference_spp"],
            "mse_ratio_plain_over_guided_equal_time": mse["mse_ratio_plain_over_guided_equal_time"],
            "mse_ratio_equal_spp": mse["runs"][0]["mse_ratio_equal_spp"],
            "relmse_ratio_equal_time": mse["runs"][0]["relmse_ratio_equal_time"],
            "guided": mse["runs"][0]["guided"], "plain_equal_time": mse["runs"][0]["plain_equal_time"],
            "guide_stage_ms": mse["runs"][0]["stage_ms"],
            "full_size": "python bench.py --guided-mse --mse-width 1024 --mse-height 768",
        }

    if info.rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": info.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "strong" if bands_split else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": WORKLOAD, "triangles": int(wl.scene.n_tris), "views": len(wl.cameras),
                "width": wl.cameras[0].width, "height": wl.cameras[0].height, "bands": B, "depth": wl.depth,
                "step": "one full-frame sample pass of the 64-spp job (all views, all bands): "
                        f"{P * B} paths, accumulated in FP64",
                "paths_per_step_per_gpu": P * B, "accumulation": "f64",
                "guide": f"8-lobe vMF MLP guide, one-sample MIS alpha 0.7, guide depth 2, trained online in every "
                         f"pass (every {GUIDE_COLLECT}th path, {GUIDE_STEPS} Adam steps per wave)",
                "xyz": "bf16x3 tensor cores, f32 accumulate",
                "l2": "inputs larger than L2: 2M-triangle BVH and triangles (about 0.3 GB), 1.1 GB of wave queues "
                      "and an 8.2 GB FP64 spectral image per step",
                "partition": ("each rank renders its band sub-domain of every pass; XYZ partials reduced to rank 0 "
                              "over NCCL" if bands_split else
                              "each rank renders the whole job with its own Philox key"),
                "bvh": {"builder": bvh_info["builder"], "build_ms": round(bvh_info["build_ms"], 1),
                        "nodes4": bvh_info["n_nodes4"], "load_s": round(t_load, 2)},
            },
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 48 * len(wl.cameras),
                    "d2h_bytes_per_step": P * 3 * 4, "steps": e2e_steps},
            "gpu_launches": launches,
            "roofline": roof,
        }
        line.update(sub)
        if not args.no_cpu_baseline and info.world == 1:
            line["cpu_baseline"] = cpu_baseline(wl, args.cpu_pixels)
        print(json.dumps(line), flush=True)
    multigpu.finish(info)
    return 0


if __name__ == "__main__":
    sys.exit(main())
