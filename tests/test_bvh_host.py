"""Host BVH builders (binned SAH, and SAH with spatial splits) checked on the
CPU by a small C++ program built from the library's builder source: every
triangle is reachable through a leaf whose box covers it, thin glass is never
split, boxes nest, and the four-wide trees reach every node once, tile the
leaf order with their leaves and cover every triangle."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from paper_1912_04000_gb300 import scenes

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1912_04000_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("bvh") / "bvh_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "bvh_check.cpp"),
                    os.path.join(CSRC, "rt_bvh.cpp"), "-o", out], check=True)
    return out


@pytest.mark.parametrize("name", ["tiny_box", "prism_room", "crystal_nave_small", "nave"])
def test_builders(checker, tmp_path, name):
    wl = {"tiny_box": scenes.tiny_box, "prism_room": scenes.prism_room,
          "crystal_nave_small": lambda: scenes.crystal_nave(width=8, height=8, col_seg=16, col_rings=8),
          "nave": lambda: scenes.nave(width=8, height=8)}[name]()
    sc = wl.scene
    split = (sc.mat_type[sc.mat_id] != scenes.THIN_GLASS).astype(np.uint8)
    path = str(tmp_path / "scene.bin")
    with open(path, "wb") as f:
        f.write(struct.pack("II", sc.verts.shape[0], sc.tris.shape[0]))
        f.write(np.ascontiguousarray(sc.verts, np.float32).tobytes())
        f.write(np.ascontiguousarray(sc.tris, np.uint32).tobytes())
        f.write(split.tobytes())
    r = subprocess.run([checker, path], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.split("\n")
    assert lines[0].startswith("sah ok") and lines[1].startswith("sbvh ok")
    refs = int(lines[1].split("refs=")[1].split()[0])
    assert sc.n_tris <= refs <= 2 * sc.n_tris
