"""Child process of tests/test_zz_no_alloc.py: a fresh process whose FIRST call into the library is
tgs_bin_sort_static. Prints one JSON line. Inputs come from the oracle's preprocess (host), are
uploaded with torch (the library is not involved), and the result is compared with the oracle's
bin sort here."""
import ctypes as C
import json
import os
import sys

import numpy as np

ROOT = sys.argv[1]
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import oracle  # noqa: E402
from paper_2605_17855_gb300 import build, scenes  # noqa: E402


class Projected(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("mean2d", "conic_opacity", "rgb", "depth", "radius", "rect")]


class Bins(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("keys", C.c_void_p), ("vals", C.c_void_p), ("masks", C.c_void_p),
                ("ranges", C.c_void_p), ("num_entries", C.c_void_p)]


class Tiling(C.Structure):
    _fields_ = [("group_w", C.c_int32), ("group_h", C.c_int32), ("flags", C.c_int32)]


def main():
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    scene, cams = scenes.box_2k_128()
    cam = cams[0]
    pr = oracle.preprocess(scene, cam)
    n = scene.n
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a, np.float32), device=dev)  # noqa: E731
    i32 = lambda a: torch.tensor(np.ascontiguousarray(a, np.int32), device=dev)  # noqa: E731
    co = np.concatenate([pr.conic, pr.opacity[:, None]], 1)
    arrs = dict(mean2d=f32(pr.mean2d), conic_opacity=f32(co), rgb=f32(pr.rgb), depth=f32(pr.depth),
                radius=i32(pr.radius), rect=i32(pr.rect))
    proj = Projected(**{k: v.data_ptr() for k, v in arrs.items()})
    lib = C.CDLL(build.LIB)
    lib.tgs_bin_sort_static.restype = C.c_int32
    lib.tgs_bin_sort_static.argtypes = [C.POINTER(Projected), C.c_int64, C.c_int32, C.c_int32,
                                        C.POINTER(Tiling), C.POINTER(Bins), C.POINTER(C.c_int64), C.c_void_p]
    lib.tgs_allocation_count.restype = C.c_int64
    lib.tgs_last_error_message.restype = C.c_char_p
    out = {"calls": []}
    frees = []
    torch.cuda.synchronize()
    frees.append(torch.cuda.mem_get_info(dev)[0])
    for (gw, gh) in ((2, 2), (2, 2), (4, 2)):  # the first one is the process's first library call
        ob = oracle.bin_sort(pr.mean2d, pr.radius, pr.depth, cam.width, cam.height, gw, gh,
                             conic=co[:, :3], opacity=co[:, 3])
        E = ob.num_entries
        GX = ((cam.width + 15) // 16 + gw - 1) // gw
        GY = ((cam.height + 15) // 16 + gh - 1) // gh
        bufs = dict(keys=torch.zeros(E, dtype=torch.int64, device=dev),
                    vals=torch.zeros(E, dtype=torch.int32, device=dev),
                    masks=torch.zeros(E, dtype=torch.int16, device=dev),
                    ranges=torch.zeros((GX * GY, 2), dtype=torch.int32, device=dev),
                    num_entries=torch.zeros(1, dtype=torch.int64, device=dev))
        torch.cuda.synchronize()
        before = torch.cuda.mem_get_info(dev)[0]
        b = Bins(E, *[bufs[k].data_ptr() for k in ("keys", "vals", "masks", "ranges", "num_entries")])
        host = C.c_int64(-7)
        st = lib.tgs_bin_sort_static(C.byref(proj), n, cam.width, cam.height, C.byref(Tiling(gw, gh)),
                                     C.byref(b), C.byref(host), None)
        torch.cuda.synchronize()
        after = torch.cuda.mem_get_info(dev)[0]
        npy = lambda t: t.cpu().numpy()  # noqa: E731
        out["calls"].append({
            "status": int(st), "message": lib.tgs_last_error_message().decode(),
            "entries": int(host.value), "oracle_entries": int(E),
            "equal": bool(np.array_equal(npy(bufs["keys"]).view(np.uint64), ob.keys)
                          and np.array_equal(npy(bufs["vals"]).view(np.uint32), ob.vals)
                          and np.array_equal(npy(bufs["masks"]).view(np.uint16), ob.masks)
                          and np.array_equal(npy(bufs["ranges"]).view(np.uint32), ob.ranges)),
            "free_before": int(before), "free_after": int(after)})
    out["allocation_count"] = int(lib.tgs_allocation_count())
    print(json.dumps(out))


if __name__ == "__main__":
    main()
