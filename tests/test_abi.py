"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every function that
include/*.h declares, validates arguments before touching the device, and the product package is
independent of the oracle."""
import ast
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(tgs_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_2605_17855_gb300 as tgs
    return tgs.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("tgs_preprocess", "tgs_bin_sort", "tgs_rasterize", "tgs_rasterize_backward",
                     "tgs_serve_create", "tgs_serve_add_scene", "tgs_serve_submit", "tgs_serve_poll",
                     "tgs_serve_wait", "tgs_serve_get_stats", "tgs_serve_destroy"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    import paper_2605_17855_gb300 as tgs
    names = _declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert names <= set(tgs.SIGNATURES), names - set(tgs.SIGNATURES)


def test_status_strings_and_version(lib):
    assert lib.tgs_abi_version() == 3
    assert lib.tgs_status_string(0) == b"TGS_OK"
    assert lib.tgs_status_string(3) == b"TGS_ERR_CAPACITY"
    assert lib.tgs_status_string(99) == b"TGS_ERR_UNKNOWN"


def test_argument_validation_is_host_side(lib):
    import ctypes as C

    import paper_2605_17855_gb300 as tgs
    out = C.c_size_t(0)
    bad = tgs._Tiling(0, 2)
    assert lib.tgs_bin_sort_workspace_size(10, 10, 64, 64, C.byref(bad), C.byref(out)) == 1
    good = tgs._Tiling(2, 2)
    assert lib.tgs_bin_sort_workspace_size(10, 10, 64, 64, C.byref(good), C.byref(out)) == 0
    assert out.value > 0
    assert lib.tgs_bin_sort_workspace_size(10, 10, 0, 64, C.byref(good), C.byref(out)) == 1
    # preprocess: bad SH degree and bad camera are rejected before any device work
    s = tgs._Scene(5, 7, None, None, None, None, None)
    cam = tgs._Camera()
    cam.width, cam.height, cam.fx, cam.fy = 64, 64, 50.0, 50.0
    proj = tgs._Projected()
    assert lib.tgs_preprocess(C.byref(s), C.byref(cam), C.byref(proj), None) == 1
    assert b"sh_degree" in lib.tgs_last_error_message()
    s = tgs._Scene(0, 0, None, None, None, None, None)
    assert lib.tgs_preprocess(C.byref(s), C.byref(cam), C.byref(proj), None) == 0  # empty scene: no-op
    cam.fx = -1.0
    assert lib.tgs_preprocess(C.byref(s), C.byref(cam), C.byref(proj), None) == 1
    # rasterize: null options
    b = tgs._Bins()
    assert lib.tgs_rasterize(C.byref(proj), 0, C.byref(b), 64, 64, C.byref(good), None, None, None, None,
                             None) == 1


def test_workspace_grows_with_capacity(lib):
    import paper_2605_17855_gb300 as tgs
    a = tgs.workspace_size(1000, 1000, 128, 128, (2, 2))
    b = tgs.workspace_size(1000, 100000, 128, 128, (2, 2))
    assert b > a


def _imports(path):
    tree = ast.parse(open(path).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module:
            mods.add(node.module.split(".")[0])
    return mods


def test_product_never_imports_the_oracle():
    for p in glob.glob(os.path.join(ROOT, "paper_2605_17855_gb300", "**", "*.py"), recursive=True):
        assert "oracle" not in _imports(p), p
    for p in glob.glob(os.path.join(ROOT, "paper_2605_17855_gb300", "csrc", "**", "*.*"), recursive=True):
        assert "oracle" not in open(p).read().lower(), p


def test_oracle_never_imports_the_product():
    for p in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert "paper_2605_17855_gb300" not in _imports(p), p
    for p in glob.glob(os.path.join(ROOT, "oracle", "*.[ch]")):
        assert "tgs_internal" not in open(p).read() and "tgs.h" not in open(p).read()


def test_serve_argument_validation_is_host_side(lib):
    import ctypes as C

    import paper_2605_17855_gb300 as tgs
    h = C.c_void_p()
    bad = tgs._ServeConfig(0, 4, 2, 0, 1, tgs._Tiling(2, 2), (C.c_float * 3)(0, 0, 0), 0)  # no budget
    assert lib.tgs_serve_create(C.byref(bad), C.byref(h)) == tgs.TGS_ERR_INVALID_ARGUMENT
    bad = tgs._ServeConfig(1 << 30, 0, 2, 0, 1, tgs._Tiling(2, 2), (C.c_float * 3)(0, 0, 0), 0)
    assert lib.tgs_serve_create(C.byref(bad), C.byref(h)) == tgs.TGS_ERR_INVALID_ARGUMENT
    bad = tgs._ServeConfig(1 << 30, 4, 17, 0, 1, tgs._Tiling(2, 2), (C.c_float * 3)(0, 0, 0), 0)
    assert lib.tgs_serve_create(C.byref(bad), C.byref(h)) == tgs.TGS_ERR_INVALID_ARGUMENT
    assert lib.tgs_serve_create(None, C.byref(h)) == tgs.TGS_ERR_INVALID_ARGUMENT

    def full(precision, gw, gh):  # complete apart from the grouping under test
        return tgs._ServeConfig(1 << 30, 4, 2, 0, precision, tgs._Tiling(gw, gh, 0),
                                (C.c_float * 3)(0, 0, 0), 0, 1000, 64, 64, 4096)

    # groupings the tensor-core rasterizer is not built for are refused before any device work
    for prec, gw, gh in ((1, 3, 1), (1, 1, 2), (2, 4, 1), (1, 5, 1), (0, 0, 1)):
        assert lib.tgs_serve_create(C.byref(full(prec, gw, gh)), C.byref(h)) == tgs.TGS_ERR_INVALID_ARGUMENT
        assert not h.value
    for prec, gw, gh in ((1, 2, 2), (2, 4, 4), (0, 3, 1)):  # accepted: fails later without a GPU
        s = lib.tgs_serve_create(C.byref(full(prec, gw, gh)), C.byref(h))
        assert s != tgs.TGS_ERR_INVALID_ARGUMENT
        if s == tgs.TGS_OK:
            assert lib.tgs_serve_destroy(h) == tgs.TGS_OK
    st = tgs._ServeStats()
    assert lib.tgs_serve_get_stats(None, C.byref(st)) == tgs.TGS_ERR_INVALID_ARGUMENT
    assert lib.tgs_serve_destroy(None) == tgs.TGS_ERR_INVALID_ARGUMENT


def test_frames_argument_validation_is_host_side(lib):
    import ctypes as C

    import paper_2605_17855_gb300 as tgs
    h = C.c_void_p()

    def cfg(**kw):
        f = dict(max_gaussians=1000, max_sh_degree=3, max_width=64, max_height=64, max_entries=4096,
                 tiling=tgs._Tiling(2, 2, 0), precision=1, bg=(C.c_float * 3)(0, 0, 0), sets=3,
                 device=0)
        f.update(kw)
        return tgs._FramesConfig(**f)

    assert lib.tgs_frames_create(None, C.byref(h)) == tgs.TGS_ERR_INVALID_ARGUMENT
    for bad in (cfg(sets=1), cfg(sets=9), cfg(max_gaussians=0), cfg(max_sh_degree=4),
                cfg(max_width=0), cfg(max_height=20000), cfg(max_entries=0), cfg(precision=7),
                cfg(tiling=tgs._Tiling(5, 1, 0)), cfg(tiling=tgs._Tiling(2, 2, 8)),
                # groupings the tensor-core rasterizer is not built for
                cfg(tiling=tgs._Tiling(3, 1, 0)), cfg(precision=2, tiling=tgs._Tiling(1, 2, 0))):
        assert lib.tgs_frames_create(C.byref(bad), C.byref(h)) == tgs.TGS_ERR_INVALID_ARGUMENT
        assert not h.value  # nothing was created
    for good in (cfg(), cfg(precision=0, tiling=tgs._Tiling(3, 1, 0))):  # fails later without a GPU
        s = lib.tgs_frames_create(C.byref(good), C.byref(h))
        assert s != tgs.TGS_ERR_INVALID_ARGUMENT
        if s == tgs.TGS_OK:
            assert lib.tgs_frames_destroy(h) == tgs.TGS_OK
    assert lib.tgs_frames_render(None, None, None, 0, None, None, None) == tgs.TGS_ERR_INVALID_ARGUMENT
    assert lib.tgs_frames_wait(None) == tgs.TGS_ERR_INVALID_ARGUMENT
    assert lib.tgs_frames_destroy(None) == tgs.TGS_ERR_INVALID_ARGUMENT
    assert lib.tgs_frames_device_bytes(None) == 0


def test_lookback_limit_setting(lib):
    # process-wide host setting: returns the previous limit, <= 0 restores the default of 1 s
    default = 1_000_000_000
    assert lib.tgs_set_lookback_limit(5000) == default
    assert lib.tgs_set_lookback_limit(0) == 5000
    assert lib.tgs_set_lookback_limit(-3) == default
    assert lib.tgs_set_lookback_limit(default) == default


def test_size_limits_are_checked_on_the_host(lib):
    import ctypes as C

    import paper_2605_17855_gb300 as tgs
    out = C.c_size_t(0)
    t = tgs._Tiling(2, 2)
    # counts and capacities are limited to < 2^30 (30-bit look-back counters in the bin sort)
    assert lib.tgs_bin_sort_workspace_size(1 << 30, 10, 64, 64, C.byref(t), C.byref(out)) == 1
    assert lib.tgs_bin_sort_workspace_size(10, 1 << 30, 64, 64, C.byref(t), C.byref(out)) == 1
    assert lib.tgs_bin_sort_workspace_size((1 << 30) - 1, (1 << 30) - 1, 64, 64, C.byref(t), C.byref(out)) == 0
    # image sizes up to 16384 per side
    assert lib.tgs_bin_sort_workspace_size(10, 10, 16385, 64, C.byref(t), C.byref(out)) == 1
    assert lib.tgs_bin_sort_workspace_size(10, 10, 16384, 16384, C.byref(t), C.byref(out)) == 0


def test_backward_rejects_a_tensor_core_forward(lib):
    # the backward replays the FP32 forward's decisions; a tensor-core forward's outputs would give
    # the gradient of a different image, so the ABI refuses any other precision before device work
    import ctypes as C

    import paper_2605_17855_gb300 as tgs
    proj = tgs._Projected()
    b = tgs._Bins()
    b.ranges = C.c_void_p(256)  # never dereferenced: the call stops at argument validation
    t = tgs._Tiling(2, 2)
    dummy = C.c_void_p(256)
    for prec in (tgs.PRECISION["fp16_tc"], tgs.PRECISION["bf16_tc"], 7):
        o = tgs._RasterOpts(prec, 0, (C.c_float * 3)(0, 0, 0), None)
        st = lib.tgs_rasterize_backward(C.byref(proj), 0, C.byref(b), 64, 64, C.byref(t), C.byref(o),
                                        dummy, dummy, dummy, None, None, None, None)
        assert st == tgs.TGS_ERR_INVALID_ARGUMENT
        assert b"FP32 forward" in lib.tgs_last_error_message()


def test_every_allocation_goes_through_the_counted_helpers():
    # tgs_allocation_count is only meaningful if no source allocates around it
    pat = re.compile(r"\bcuda(Malloc|MallocHost|MallocManaged|MallocAsync|HostAlloc|MallocPitch|"
                     r"Malloc3D|MallocArray)\s*\(")
    for p in glob.glob(os.path.join(ROOT, "paper_2605_17855_gb300", "csrc", "**", "*.*"), recursive=True):
        src = re.sub(r"//[^\n]*", "", re.sub(r"/\*.*?\*/", "", open(p).read(), flags=re.S))
        src = re.sub(r'"(?:[^"\\\n]|\\.)*"', '""', src)  # string literals (error messages)
        hits = pat.findall(src)
        if os.path.basename(p) == "abi.cu":
            assert sorted(hits) == ["Malloc", "MallocHost"], hits  # the two helpers themselves
        else:
            assert not hits, (p, hits)
