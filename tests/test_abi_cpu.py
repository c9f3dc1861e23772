"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol include/mhfd.h declares, validates parameters before touching a
device, and its host-only helpers (ladder, tile menu, kernel compilation)
work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2108_12050_gb300 import _build, _native
    _build.build_lib()
    return _native


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "mhfd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mhfd_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(native):
    lib = native.lib()
    declared = _declared_symbols()
    assert len(declared) >= 15
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(native.EXPORTS) == declared


def test_no_cpu_fallback_symbols(native):
    # the product path has no host implementation of the method: the only
    # host arithmetic is ladder/tap construction
    out = os.popen("nm -D --defined-only %s" % native.LIB_PATH).read()
    assert "oracle" not in out


def test_version_and_defaults(native):
    lib = native.lib()
    assert b"sm_103a" in lib.mhfd_version()
    p = native.Params()
    lib.mhfd_default_params(ctypes.byref(p))
    assert (p.n, p.t_min, p.t_max) == (10, 1.0, 10.0)
    assert abs(p.threshold - 0.1) < 1e-7 and abs(p.overlap - 0.5) < 1e-7
    assert p.truncate == 4.0 and p.clip_frac == 0.00175 and p.device == -1


@pytest.mark.parametrize("kw,code", [
    (dict(n=0), -1), (dict(n=64), -1), (dict(t_min=0.0), -1), (dict(t_min=3, t_max=2), -1),
    (dict(threshold=float("nan")), -1), (dict(overlap=-0.1), -1), (dict(clip_frac=0.5), -1),
    (dict(nms=7), -1), (dict(max_candidates=0), -1), (dict(truncate=0.0), -1),
    (dict(sigmas=[1.0, 3.0, 2.0] + [4.0] * 8), -1), (dict(t_min=1, t_max=200), -2),
])
def test_create_rejects_bad_parameters_before_any_device_work(native, kw, code):
    p = native.make_params(**kw)
    h = ctypes.c_void_p()
    rc = native.lib().mhfd_create_detector(ctypes.byref(p), ctypes.byref(h))
    assert rc == code, native.lib().mhfd_last_error()
    assert not h.value
    assert native.lib().mhfd_last_error()


def test_null_arguments(native):
    lib = native.lib()
    assert lib.mhfd_create_detector(None, None) == -1
    assert lib.mhfd_destroy_detector(None) == -1
    assert lib.mhfd_detect(None, None, 0, 1, 1, 1, None) == -1
    assert lib.mhfd_result_wait(None, None) == -1


def test_tile_menu_fits_shared_memory(native):
    for kw in (dict(n=10, t_min=1, t_max=10), dict(n=16, t_min=1, t_max=12),
               dict(n=16, t_min=1, t_max=12, nms=1)):
        kw["tensor_cores"] = False
        menu = native.tile_configs(**kw)
        assert len(menu) > 10
        for tx2, ty2, rb, nt, ng, item in menu:
            assert tx2 % 4 == 0 and ty2 >= 3 and rb >= 2 and nt % 32 == 0 and ng >= 1
            assert item in (1, 2, 3) and (item != 2 or rb % 2 == 0)
        chosen = native.chosen_tile(**kw)
        assert chosen in menu


def test_precompile_small_ladder_without_gpu(native, tmp_path, monkeypatch):
    monkeypatch.setenv("MHFD_JIT_CACHE", str(tmp_path))
    rc = native.precompile(n=2, t_min=1.0, t_max=1.5, nms=0, store=0)
    assert rc == 0
    files = os.listdir(tmp_path)
    assert any(f.endswith(".cubin") for f in files)


@pytest.mark.parametrize("store,width", [(0, 0), (1, 0), (0, 48)])
def test_precompile_two_pass_local26_without_gpu(native, tmp_path, monkeypatch, store, width):
    """The two-pass kernel with the 26-neighbour rule at the benchmark
    ladder (16 layers, the most its layer masks take) compiles with NVRTC,
    at the default 64-column strips and at 48; the kernel's own static
    checks hold its shared-memory layout to the host's estimate (the
    exchange buffers and masks included)."""
    monkeypatch.setenv("MHFD_JIT_CACHE", str(tmp_path))
    kw = dict(n=16, t_min=1.0, t_max=12.0, nms=1)
    if width:
        kw["tile_shape"] = (width, 0, 0, 0, 1)
    assert native.chosen_tile(tensor_cores=True, **kw)[:2] == (width or 64, 128)
    assert native.precompile(store=store, **kw) == 0
    assert any(f.endswith(".cubin") for f in os.listdir(tmp_path))


def test_two_pass_tile_choice(native):
    """The default for detection with the DoG response is the two-pass
    kernel: tiles of 128 computed rows, strips of 16-multiple width (64 by
    default), 288 threads; tile_shape[0] sets the strip width; the LoG
    response, and the 26-neighbour rule beyond 16 layers (its 16-bit layer
    masks), keep the vertical-pass kernel."""
    kw = dict(n=16, t_min=1.0, t_max=12.0)
    assert native.chosen_tile(tensor_cores=True, **kw) == (64, 128, 4, 288, 1, 1)
    assert native.chosen_tile(tensor_cores=True, tile_shape=(48, 0, 0, 0, 1), **kw)[:2] == (48, 128)
    for bad in ((72, 0, 0, 0, 1), (144, 0, 0, 0, 1)):  # not a multiple of 16; wider than 128
        with pytest.raises(native.MhfdError) as e:
            native.chosen_tile(tensor_cores=True, tile_shape=bad, **kw)
        assert e.value.code == -2, bad
    # a ladder whose halo leaves no 48-column strip in tensor memory (R up to
    # 64: V columns 48 + 128 + padding, twice, plus the L buffers) takes the
    # vertical-pass kernel; so does one beyond it
    for t_max in (16.0, 20.0):
        wide = dict(n=16, t_min=1.0, t_max=t_max)
        assert native.chosen_tile(tensor_cores=True, **wide) == native.chosen_tile(tensor_cores=2,
                                                                                 **wide)
    assert native.chosen_tile(tensor_cores=True, n=16, t_min=1.0, t_max=14.0)[:2] == (64, 128)
    assert native.chosen_tile(tensor_cores=True, response=1, **kw)[1] != 128
    assert native.chosen_tile(tensor_cores=True, nms=1, **kw) == (64, 128, 4, 288, 1, 1)
    l17 = dict(n=17, t_min=1.0, t_max=12.0, nms=1)
    assert native.chosen_tile(tensor_cores=True, **l17) == native.chosen_tile(tensor_cores=2, **l17)
    assert native.chosen_tile(tensor_cores=True, **l17)[1] != 128
    assert native.chosen_tile(tensor_cores=True, **kw) != native.chosen_tile(tensor_cores=2, **kw)


def test_tensor_core_tile_menu(native):
    """The vertical-pass tensor-core kernel's shapes (tensor_cores=2): four or eight rows per step, whole
    warps, at least one warpgroup, one or two horizontal items per thread
    (one-row items at four rows per step, two-row items at four or eight);
    the 26-neighbour rule (DoG response) has shapes of its own;
    the built-in choice (four rows) leaves exactly one warp free of
    horizontal items (the MMA issuer) and is on the menu."""
    for kw in (dict(n=10, t_min=1, t_max=10), dict(n=16, t_min=1, t_max=12)):
        menu = native.tile_configs(tensor_cores=True, **kw)
        assert len(menu) > 10
        for tx2, ty2, rb, nt, ng, item in menu:
            assert rb in (4, 8) and nt % 32 == 0 and nt >= 128 and item in (1, 2, 3)
            rows, cols = (2, 4) if item == 2 else (1, 2) if item == 3 else (1, 4)
            assert (rb // rows) * tx2 // cols <= 2 * nt and (item == 2 or rb == 4)
        assert any(s[5] == 2 and s[2] == 8 for s in menu)
        chosen = native.chosen_tile(tensor_cores=2, **kw)
        assert chosen in menu and chosen[0] == chosen[3] - 32
    # the LoG response and the 26-neighbour rule have tensor-core shapes of
    # their own; the 26-neighbour rule with the LoG response takes the FFMA
    # kernel (the flag changes nothing for it)
    assert native.tile_configs(tensor_cores=True, n=16, t_min=1, t_max=12, response=1)
    assert native.tile_configs(tensor_cores=True, n=16, t_min=1, t_max=12, nms=1)
    kw = dict(n=16, t_min=1, t_max=12, nms=1, response=1)
    assert not native.tile_configs(tensor_cores=True, **kw)
    assert native.chosen_tile(tensor_cores=True, **kw) == native.chosen_tile(
        tensor_cores=False, **kw)


def test_explicit_tensor_core_tile_shape(native):
    kw = dict(n=16, t_min=1.0, t_max=12.0, tensor_cores=2)
    assert native.chosen_tile(tile_shape=(352, 18, 4, 384, 3), **kw) == (352, 18, 4, 384, 3, 1)
    assert native.chosen_tile(tile_shape=(256, 18, 8, 288, 4, 2), **kw) == (256, 18, 8, 288, 4, 2)
    # rows per step other than 4 or 8, threads below a warpgroup, eight rows
    # of two-row items at a width whose accumulators exceed tensor memory:
    # unsupported
    for bad in ((352, 18, 6, 384, 3), (96, 18, 4, 96, 1), (352, 18, 8, 384, 3, 2)):
        with pytest.raises(native.MhfdError) as e:
            native.chosen_tile(tile_shape=bad, **kw)
        assert e.value.code == -2, bad
    # width not a multiple of 4, item kind not 1, 2 or 3
    for bad in ((350, 18, 4, 384, 3), (352, 18, 4, 384, 3, 4)):
        with pytest.raises(native.MhfdError) as e:
            native.chosen_tile(tile_shape=bad, **kw)
        assert e.value.code == -1, bad


def test_explicit_tile_shape(native):
    kw = dict(n=16, t_min=1.0, t_max=12.0, tensor_cores=False)
    assert native.chosen_tile(tile_shape=(320, 18, 4, 448, 3), **kw) == (320, 18, 4, 448, 3, 1)
    assert native.chosen_tile(tile_shape=(320, 18, 4, 448, 3, 2), **kw) == (320, 18, 4, 448, 3, 2)
    assert native.chosen_tile(tile_shape=(192, 18, 4, 384, 2, 3), **kw) == (192, 18, 4, 384, 2, 3)
    # out of range: width not a multiple of 4, threads not a multiple of 32,
    # too few rows per step, more groups than levels, more than two
    # horizontal items per thread, two-row items on an odd number of rows
    for bad in ((322, 18, 4, 448, 3), (320, 18, 4, 450, 3), (320, 18, 1, 448, 3),
                (320, 18, 4, 448, 18), (320, 18, 8, 128, 3), (320, 18, 5, 448, 3, 2)):
        with pytest.raises(native.MhfdError) as e:
            native.chosen_tile(tile_shape=bad, **kw)
        assert e.value.code == -1, bad
    # does not fit in shared memory for this ladder
    with pytest.raises(native.MhfdError) as e:
        native.chosen_tile(tile_shape=(1024, 18, 8, 1024, 1), **kw)
    assert e.value.code == -2


def test_heuristic_tile_is_one_vertical_round(native):
    import math
    for kw in (dict(n=16, t_min=1.0, t_max=12.0), dict(n=10, t_min=1.0, t_max=10.0),
               dict(n=4, t_min=1.0, t_max=4.0)):
        tx2, ty2, rb, nt, ng, hr = native.chosen_tile(tensor_cores=False, **kw)
        dt = (kw["t_max"] - kw["t_min"]) / kw["n"]
        rmax = max(math.ceil(4 * (kw["t_min"] + i * dt)) for i in range(kw["n"] + 1))
        assert nt >= tx2 + 2 * rmax and rb * tx2 // 4 <= nt


def test_tuned_shapes_are_valid_for_their_ladders(native):
    """Every shape the autotuner recorded is accepted for its ladder and
    response (fits shared memory, passes the range checks)."""
    import json
    import re
    path = os.path.join(os.path.dirname(native.__file__), "tuned_tiles.json")
    tab = json.load(open(path))
    assert tab
    for key, ent in tab.items():
        m = re.match(r"n(\d+)_t([0-9.e+-]+)-([0-9.e+-]+)_(paper|local26)_tr4(_log)?(_tc)?$", key)
        assert m, key
        kw = dict(n=int(m.group(1)), t_min=float(m.group(2)), t_max=float(m.group(3)),
                  nms=m.group(4), response="log" if m.group(5) else "dog",
                  tensor_cores=2 if m.group(6) else False)  # the vertical-pass kernel's shapes
        for best in ent.values():
            shape = tuple(best["shape"])
            assert native.chosen_tile(tile_shape=shape, **kw) == shape + (1,) * (6 - len(shape))


def test_kernel_layout_matches_host_shared_memory_estimate(native, tmp_path, monkeypatch):
    """The host sizes and chooses a tile by its shared-memory estimate; every
    generated kernel source asserts at compile time that its own layout
    (input window, V rows, ring, tap matrices, control block) takes exactly
    that many bytes.  Compiling (NVRTC, no GPU) a spread of variants and
    menu shapes therefore checks the two layouts against each other."""
    monkeypatch.setenv("MHFD_JIT_CACHE", str(tmp_path))
    small = dict(n=4, t_min=1.0, t_max=4.0)
    cases = [
        (dict(tensor_cores=True, **small), 0),                     # paper rule, two-pass kernel
        (dict(tensor_cores=True, **small), 1),                     # its stack-storing variant
        (dict(tensor_cores=2, **small), 0),                        # paper rule, vertical pass
        (dict(tensor_cores=True, response="log", **small), 0),     # LoG on tensor cores
        (dict(tensor_cores=False, nms="local26", **small), 0),     # 26-neighbour rule
        (dict(tensor_cores=False, boundary="periodic", **small), 1),  # stack-storing variant
        (dict(tensor_cores=False, **small), 2),                    # soft-score forward
        (dict(tensor_cores=False, **small), 3),                    # level blur of the adjoint
    ]
    # the two-pass kernel at strip widths 48 and 64 on the n = 16 ladder;
    # first and last shapes of the vertical-pass kernel's menu
    cases += [(dict(n=16, t_min=1.0, t_max=12.0, tensor_cores=True, tile_shape=(w, 0, 0, 0, 1)), 0)
              for w in (48, 64)]
    full = dict(n=16, t_min=1.0, t_max=12.0, tensor_cores=2)
    menu = native.tile_configs(**full)
    for shape in (menu[0], menu[-1]):
        cases.append((dict(tile_shape=shape, **full), 0))
    # two-row horizontal items: tensor-core and FFMA kernels, DoG and LoG,
    # the detection and the stack-storing variants
    cases += [(dict(tile_shape=(256, 18, 8, 288, 4, 2), **full), 0),
              (dict(tile_shape=(256, 18, 8, 288, 4, 2), **full), 1),
              (dict(tile_shape=(320, 18, 4, 448, 3, 2), n=16, t_min=1.0, t_max=12.0,
                    tensor_cores=False), 0),
              (dict(tile_shape=(96, 18, 4, 160, 1, 2), tensor_cores=2, response="log",
                    **small), 0),
              # one-row items of two outputs: 26-neighbour rule, LoG, stack-storing
              (dict(tile_shape=(192, 18, 4, 384, 2, 3), n=16, t_min=1.0, t_max=12.0,
                    nms="local26", tensor_cores=False), 0),
              (dict(tile_shape=(96, 18, 4, 224, 1, 3), response="log", tensor_cores=False,
                    **small), 1)]
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=min(len(cases), os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        rcs = list(ex.map(_precompile_case, cases))
    assert rcs == [0] * len(cases), list(zip(cases, rcs))


def _precompile_case(case):
    kw, store = case
    from paper_2108_12050_gb300 import _native
    try:
        return _native.precompile(store=store, **kw)
    except _native.MhfdError as e:
        return str(e)
