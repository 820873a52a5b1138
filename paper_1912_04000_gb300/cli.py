"""Command line: render a synthetic workload on the GPU.

  python -m paper_1912_04000_gb300.cli render --workload nave --width 256 --height 192 --spp 1 [--out img.npy]

Prints the render statistics as one JSON line; --out writes the XYZ image.
"""
from __future__ import annotations

import argparse
import json
import sys
import time


def _workload(args):
    from . import scenes
    if args.workload == "tiny_box":
        return scenes.tiny_box(width=args.width or 128, height=args.height or 128, spp=args.spp or 4,
                               depth=args.depth or 4, seed=args.seed)
    if args.workload == "nave":
        return scenes.nave(width=args.width or 1024, height=args.height or 768, spp=args.spp or 16,
                           depth=args.depth or 8, seed=args.seed, n_bands=args.bands or 81)
    if args.workload == "crystal_nave":
        return scenes.crystal_nave(width=args.width or 1024, height=args.height or 768, spp=args.spp or 16,
                                   depth=args.depth or 8, seed=args.seed, n_bands=args.bands or 81)
    if args.workload == "nave_views":
        wl = scenes.nave_views(n_views=args.views or 32, spp=args.spp or 8, depth=args.depth or 8, seed=args.seed)
        return wl
    if args.workload == "large_nave":
        return scenes.large_nave(width=args.width or 2048, height=args.height or 1536, spp=args.spp or 64,
                                 depth=args.depth or 12, seed=args.seed, n_views=args.views or 4)
    raise SystemExit(f"unknown workload {args.workload}")


def main(argv=None):
    ap = argparse.ArgumentParser(prog="paper_1912_04000_gb300.cli")
    sub = ap.add_subparsers(dest="cmd", required=True)
    r = sub.add_parser("render")
    r.add_argument("--workload", default="nave", choices=["tiny_box", "nave", "crystal_nave", "nave_views", "large_nave"])
    r.add_argument("--width", type=int, default=0)
    r.add_argument("--height", type=int, default=0)
    r.add_argument("--spp", type=int, default=0)
    r.add_argument("--depth", type=int, default=0)
    r.add_argument("--bands", type=int, default=0)
    r.add_argument("--views", type=int, default=0)
    r.add_argument("--seed", type=int, default=0)
    r.add_argument("--xyz-mode", type=int, default=0)
    r.add_argument("--wave", type=int, default=0, help="wave capacity (paths in flight)")
    r.add_argument("--repeat", type=int, default=1)
    r.add_argument("--guided", action="store_true", help="learned guide at Lambertian vertices (freshly initialised)")
    r.add_argument("--guide-collect", type=int, default=0)
    r.add_argument("--guide-train-steps", type=int, default=0)
    r.add_argument("--graph", action="store_true", help="capture the render in a CUDA graph and replay it")
    r.add_argument("--tune", action="store_true", help="autotuned launch settings (cached per GPU and workload)")
    r.add_argument("--builder", default="sbvh", choices=["host", "device", "sbvh"],
                   help="BVH builder: binned SAH on the host, linear BVH on the device, or SAH with spatial splits")
    r.add_argument("--bands-per-path", type=int, default=1, choices=[1, 4],
                   help="4: every path carries four bands until its first refraction")
    r.add_argument("--estimator", default="path", choices=["path", "photon"],
                   help="path tracing, or photon mapping (caustic + indirect maps, density estimates)")
    r.add_argument("--photons", type=int, default=0, help="photon mapping: photons per band (0 = 65536)")
    r.add_argument("--out", default="")
    args = ap.parse_args(argv)

    from .renderer import Renderer
    wl = _workload(args)
    t0 = time.perf_counter()
    R = Renderer(0).load(wl, builder={"host": 0, "device": 1, "sbvh": 2}[args.builder])
    if args.guided:
        R.guide_init(seed=1)
    t_load = time.perf_counter() - t0
    tuned = None
    if args.tune:
        from .autotune import tuned_options
        tuned, _ = tuned_options(R, wl)
    out = None
    for _ in range(args.repeat):
        if args.estimator == "photon":
            out = R.render_photons(wl.cameras, wl.spp, wl.depth, wl.seed, n_photons=args.photons,
                                   xyz_mode=args.xyz_mode)
            continue
        out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=args.xyz_mode, wave_capacity=args.wave,
                       guided=args.guided, guide_collect=args.guide_collect,
                       guide_train_steps=args.guide_train_steps, use_graph=args.graph, tuned=tuned,
                       bands_per_path=args.bands_per_path)
    st = out["stats"]
    st.update(workload=wl.name, triangles=int(wl.scene.n_tris), load_s=t_load, tuned=tuned, bvh=R.scene_info(),
              paths_per_s=st["paths"] / (st["ms_render"] * 1e-3) if st["ms_render"] > 0 else None)
    print(json.dumps(st))
    if args.out:
        import numpy as np
        np.save(args.out, out["xyz"].cpu().numpy())
    return 0


if __name__ == "__main__":
    sys.exit(main())
