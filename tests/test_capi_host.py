"""CPU-side checks of the C ABI (no GPU): the library loads, exports every
symbol include/alb.h declares, the host sampler and shape logic agree with the
oracle, and argument errors are reported before any CUDA call."""
import ctypes as C
import os
import re

import pytest

import oracle as O
from helpers import EXTRA_CFGS, cfg_to_lib, same_params, suite_cfgs

from paper_1809_06839_gb300 import alb, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return alb.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "alb.h")).read()
    return sorted(set(re.findall(r"ALB_API\s+[\w\s\*]+?\b(alb_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("alb_sample_params", "alb_apply", "alb_apply_batch", "alb_apply_ragged", "alb_sample_params_batch",
                 "alb_warp_affine_f32_bwd", "alb_photometric_f32_bwd", "alb_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_version(L):
    assert alb.alb_version().startswith("alb ")


ALL = {**suite_cfgs(), **EXTRA_CFGS}


@pytest.mark.parametrize("name", sorted(ALL))
def test_host_sampler_matches_oracle(L, name):
    oc = ALL[name]
    lc = cfg_to_lib(oc, alb)
    for i in range(60):
        h, w = 333 + (i * 29) % 168, 333 + (i * 53) % 168
        op = O.sample_params(oc, 1809, oc.tid, i, h, w)
        lp = alb.alb_sample_params(lc, 1809, oc.tid, i, h, w)
        err = same_params(op, lp)
        assert err is None, (name, i, err)


def test_chain_sampler_matches_oracle(L):
    from helpers import CHAIN_CFG
    oc = O.make_cfg(O.CHAIN, **CHAIN_CFG)
    lc = cfg_to_lib(oc, alb)
    for i in range(200):
        h, w = 256 + (i * 37) % 769, 256 + (i * 91) % 769
        err = same_params(O.sample_params(oc, 7, 20, i, h, w), alb.alb_sample_params(lc, 7, 20, i, h, w))
        assert err is None, (i, err)


@pytest.mark.parametrize("name", sorted(ALL))
def test_output_shape_matches_oracle(L, name):
    oc = ALL[name]
    op = O.sample_params(oc, 3, 1, 0, 400, 450)
    from helpers import to_lib
    assert alb.alb_output_shape(to_lib(op, alb), 400, 450) == O.output_shape(op, 400, 450)


def test_sampler_rejects_crop_larger_than_image(L):
    with pytest.raises(alb.AlbError) as e:
        alb.alb_sample_params(alb.sample_cfg(alb.RANDOM_CROP, out_h=64, out_w=64), 1, 1, 0, 32, 100)
    assert e.value.code == alb.ALB_ESHAPE


def test_argument_errors_are_reported_without_cuda(L):
    assert L.alb_apply(None, None, None, None, None, None, 0, None, None, None, 0, None) == alb.ALB_EINVAL
    assert "required" in alb.alb_last_error()
    assert L.alb_apply_ragged(99, 1, None, None, None, None, None, None, None, 0, None, None, None, 0, None,
                              None) == alb.ALB_EINVAL
    assert L.alb_apply_ragged(alb.HFLIP, -1, None, None, None, None, None, None, None, 0, None, None, None, 0, None,
                              None) == alb.ALB_EINVAL
    assert L.alb_apply_batch(None, 1, None, None, None, 0, None, 0, None, None) == alb.ALB_EINVAL
    cfg = alb.chain_cfg()
    assert L.alb_apply_batch(C.byref(cfg), 4, None, None, None, 0, None, 0, None, None) == alb.ALB_EINVAL
    assert L.alb_warp_affine_f32_fwd(1, 0, 4, 4, None, None, None, None) == alb.ALB_ESHAPE
    # zero-sized batches are a no-op
    assert L.alb_apply_ragged(alb.HFLIP, 0, None, None, None, None, None, None, None, 0, None, None, None, 0, None,
                              None) == alb.ALB_OK


def test_schedule_fields_are_checked_without_cuda(L):
    """alb_apply_batch and alb_autotune_batch reject a bad schedule before any
    device work (the pointers below are never dereferenced)."""
    fake = C.c_void_p(16)
    for kw in (dict(tile_w=8), dict(tile_h=33), dict(tile_h=-1), dict(ctas_per_sm=-2)):
        cfg = alb.chain_cfg(**kw)
        assert L.alb_apply_batch(C.byref(cfg), 4, fake, fake, fake, 0, fake, 1 << 40, None, None) == alb.ALB_EINVAL, kw
        assert "tile_h" in alb.alb_last_error()
    cfg = alb.chain_cfg(jitter=2)
    assert L.alb_apply_batch(C.byref(cfg), 4, fake, fake, fake, 0, fake, 1 << 40, None, None) == alb.ALB_EINVAL
    assert "jitter" in alb.alb_last_error()
    best = alb.ChainCfg()
    cfg = alb.chain_cfg(tile_w=8)
    assert L.alb_autotune_batch(C.byref(cfg), 4, fake, fake, fake, fake, 1 << 40, 1, C.byref(best), None) == alb.ALB_EINVAL
    assert L.alb_autotune_batch(None, 4, fake, fake, fake, fake, 1 << 40, 1, C.byref(best), None) == alb.ALB_EINVAL
    assert L.alb_autotune_batch(C.byref(alb.chain_cfg()), 0, fake, fake, fake, fake, 1 << 40, 1, C.byref(best),
                                None) == alb.ALB_EINVAL
    assert L.alb_autotune_batch(C.byref(alb.chain_cfg()), 4, fake, fake, fake, fake, 0, 1, C.byref(best),
                                None) == alb.ALB_EWORKSPACE


def test_host_box_safe_sampler_matches_oracle(L):
    oc = O.make_cfg(O.CHAIN, out_h=224, out_w=224, lo=(0.08, 3 / 4, 0.6), hi=(1.0, 4 / 3, 1.4))
    lc = cfg_to_lib(oc, alb)
    from paper_1809_06839_gb300 import synth
    for i in range(80):
        h, w = 256 + (i * 37) % 700, 256 + (i * 91) % 700
        boxes = synth.random_boxes(h, w, i, 3)[: i % 7]
        op = O.sample_chain_box_safe(oc, 1809, 20, i, h, w, boxes)
        lp = alb.alb_sample_chain_box_safe(lc, 1809, 20, i, h, w, boxes)
        err = same_params(op, lp)
        assert err is None, (i, err)


def test_distortion_records_are_checked_without_cuda(L):
    """alb_apply rejects boxes with the elastic transform and out-of-range
    distortion records before any device work."""
    fake = C.c_void_p(16)
    img = alb.Image()
    img.data, img.h, img.w, img.c, img.row_stride = 16, 4, 4, 3, 12
    out = alb.Image()
    out.data, out.h, out.w, out.c, out.row_stride = 4096, 4, 4, 3, 12
    p = alb.Params()
    p.tid, p.apply, p.k, p.cw = alb.ELASTIC, 1, 32, 4
    box = (C.c_float * 4)(0, 0, 1, 1)
    nout = C.c_int32()
    assert L.alb_apply(C.byref(p), C.byref(img), C.byref(out), None, None, box, 1, box, C.byref(nout), fake,
                       1 << 30, None) == alb.ALB_EINVAL
    assert "elastic" in alb.alb_last_error()
    p.cw = 9
    assert L.alb_apply(C.byref(p), C.byref(img), None, None, None, None, 0, None, None, fake, 1 << 30,
                       None) == alb.ALB_EINVAL
    p.tid, p.k = alb.GRID_DISTORTION, 13
    assert L.alb_apply(C.byref(p), C.byref(img), None, None, None, None, 0, None, None, fake, 1 << 30,
                       None) == alb.ALB_EINVAL
    assert L.alb_apply_ragged(alb.ELASTIC, 2, fake, fake, fake, None, None, fake, fake, 4, fake, fake, fake,
                              1 << 30, None, None) == alb.ALB_EINVAL


def test_workspace_sizes(L):
    assert alb.alb_workspace_size(alb.EQUALIZE, 2000) > alb.alb_workspace_size(alb.BRIGHTNESS, 2000)
    assert alb.alb_workspace_size(alb.BRIGHTNESS, 2000) > alb.alb_workspace_size(alb.HFLIP, 2000)
    cfg = alb.chain_cfg()
    assert alb.alb_batch_workspace_size(cfg, 64, alb.MODE_PLAIN) > alb.alb_batch_workspace_size(cfg, 64,
                                                                                                alb.MODE_FUSED)


def test_float_path_shape_limits_without_cuda(L):
    """The float entry points reject a bad shape, a null pointer, a batch above
    the grid's y limit or an image whose per-image offsets leave int32 before
    any device work (the pointers below are never dereferenced)."""
    fake = C.c_void_p(16)
    fwd, bwd = L.alb_warp_affine_f32_fwd, L.alb_warp_affine_f32_bwd
    pfwd, pbwd = L.alb_photometric_f32_fwd, L.alb_photometric_f32_bwd
    assert fwd(2, 3, 0, 8, fake, fake, fake, None) == alb.ALB_ESHAPE
    assert fwd(2, 3, 8, 8, None, fake, fake, None) == alb.ALB_EINVAL
    assert fwd(70000, 3, 8, 8, fake, fake, fake, None) == alb.ALB_ESHAPE
    assert "65535" in alb.alb_last_error()
    assert fwd(1, 3, 1 << 15, 1 << 14, fake, fake, fake, None) == alb.ALB_ESHAPE
    assert "too large" in alb.alb_last_error()
    assert bwd(70000, 3, 8, 8, fake, fake, fake, fake, fake, fake, 1 << 40, None) == alb.ALB_ESHAPE
    assert bwd(1, 3, 8, 8, fake, fake, fake, None, fake, fake, 1 << 40, None) == alb.ALB_EINVAL
    assert bwd(1, 3, 1 << 15, 1 << 14, fake, fake, fake, fake, fake, fake, 1 << 40, None) == alb.ALB_ESHAPE
    assert pfwd(70000, 3, 8, 8, fake, fake, fake, None) == alb.ALB_ESHAPE
    assert pbwd(70000, 3, 8, 8, fake, fake, fake, fake, fake, fake, 1 << 40, None) == alb.ALB_ESHAPE
    # an empty batch is a no-op
    assert fwd(0, 3, 8, 8, None, None, None, None) == alb.ALB_OK
    assert bwd(0, 3, 8, 8, None, None, None, None, None, None, 0, None) == alb.ALB_OK


def test_selftest_bounded_wait_rejects_bad_arguments_before_any_launch(L):
    # refused on the host: no CUDA call is made (no GPU here)
    f = L.alb_selftest_bounded_wait
    for spins in (0, -3, (1 << 22) + 1):
        assert f(spins, C.c_void_p(16), C.c_void_p(64), C.c_void_p(128), None) == alb.ALB_EINVAL
    assert f(8, C.c_void_p(24), C.c_void_p(64), C.c_void_p(128), None) == alb.ALB_EALIGN
    assert f(8, None, C.c_void_p(64), C.c_void_p(128), None) == alb.ALB_EINVAL
    assert f(8, C.c_void_p(16), C.c_void_p(64), None, None) == alb.ALB_EINVAL


def test_autotune_load_rejects_bad_files_before_any_device_query(L, tmp_path):
    """A missing, malformed or out-of-range cache file is refused (ALB_EINVAL)
    after reading, before any CUDA call; a well-formed one reaches the
    device query (no GPU here: ALB_ECUDA)."""
    f = L.alb_autotune_load
    n = C.c_int32(-1)
    assert f(os.fsencode(str(tmp_path / "missing.json")), C.byref(n)) == alb.ALB_EINVAL
    good = ('{"format": "alb-autotune-1", "entries": [{"device": "NVIDIA GB300", "sms": 152, "out_h": 224, '
            '"out_w": 224, "jitter": 0, "bucket": 12, "rows_per_item": 32, "ctas_per_sm": 6}]}')
    bad = [
        "", "[]", '{"format": "alb-autotune-1"}', good.replace("alb-autotune-1", "other"),
        good.replace('"rows_per_item": 32', '"rows_per_item": 33'), good.replace('"jitter": 0', '"jitter": 2'),
        good.replace('"ctas_per_sm": 6', '"ctas_per_sm": 0'), good.replace('"sms": 152', '"sms": "x"'),
        good.replace('"bucket": 12', '"bucket": 12, "extra": 1'), good[:-3], good + "x",
    ]
    for k, text in enumerate(bad):
        p = tmp_path / f"bad{k}.json"
        p.write_text(text)
        assert f(os.fsencode(str(p)), C.byref(n)) == alb.ALB_EINVAL, text
        assert n.value == 0
    p = tmp_path / "good.json"
    p.write_text(good)
    assert f(os.fsencode(str(p)), C.byref(n)) == alb.ALB_ECUDA
    p.write_text('{"format": "alb-autotune-1", "entries": []}')
    assert f(os.fsencode(str(p)), C.byref(n)) in (alb.ALB_OK, alb.ALB_ECUDA)
