"""The C-ABI library on a machine without a GPU: it loads, exports every
function include/rt_stereo.h declares, and rejects bad arguments on the
host before any CUDA call."""
import ctypes

import numpy as np
import pytest

from paper_1702_01530_gb300 import build, capi, scenegen


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.lib()


def test_library_exports_every_header_function(lib):
    names = capi.header_functions()
    assert "rt_scene_create" in names and "rt_render_stereo" in names
    for n in names:
        assert hasattr(lib, n), n
    assert capi.rt_version().startswith("rt_stereo")


def _bad(**over):
    s = scenegen.config_small(1)
    sp, tr, mt, li = s.spheres.copy(), s.triangles.copy(), s.materials.copy(), s.lights.copy()
    for k, f in over.items():
        f({"sp": sp, "tr": tr, "mt": mt, "li": li})
    with pytest.raises(capi.RtError) as e:
        capi.rt_scene_create(sp, tr, mt, li, stream=0)
    return e.value


def _set(arr, field, idx, val):
    col = arr[field]
    col[idx] = val


@pytest.mark.parametrize("mut,frag", [
    (lambda a: _set(a["sp"], "radius", 0, 0.0), "sphere 0"),
    (lambda a: _set(a["sp"], "material", 3, 99), "material out of range"),
    (lambda a: _set(a["tr"], "v1", (1, 2), np.nan), "non-finite"),
    (lambda a: _set(a["mt"], "albedo", (2, 0), 1.5), "albedo"),
    (lambda a: _set(a["mt"], "reflectivity", 0, -0.1), "reflectivity"),
    (lambda a: _set(a["li"], "intensity", 0, np.inf), "light 0"),
])
def test_scene_create_rejects_bad_arguments(lib, mut, frag):
    err = _bad(m=mut)
    assert err.code == capi.RT_ERR_INVALID_ARG and frag in str(err)


def test_scene_create_rejects_empty_scene(lib):
    s = scenegen.config_small(1)
    with pytest.raises(capi.RtError) as e:
        capi.rt_scene_create(s.spheres[:0], s.triangles[:0], s.materials, s.lights, stream=0)
    assert e.value.code == capi.RT_ERR_INVALID_ARG
    with pytest.raises(capi.RtError) as e:
        capi.rt_scene_create(s.spheres, s.triangles, s.materials, s.lights[:0], stream=0)
    assert e.value.code == capi.RT_ERR_INVALID_ARG


def test_render_rejects_null_scene_and_bad_view(lib):
    cam = scenegen.config_small(1).camera
    with pytest.raises(capi.RtError) as e:
        capi.rt_render_stereo(None, cam, 0.065, 10.0, 32, 32, 3, 1, 1, stream=0)
    assert e.value.code == capi.RT_ERR_INVALID_ARG
    assert capi.rt_scene_num_prims(None) == 0
    with pytest.raises(capi.RtError):
        capi.rt_sync_status(None, stream=0)
    assert lib.rt_debug_set_node(None, 0, 0, 0, 0) == capi.RT_ERR_INVALID_ARG
    assert lib.rt_debug_set_pool_capacity(None, 0) == capi.RT_ERR_INVALID_ARG
    assert lib.rt_debug_get_sah_tree(None, None) == capi.RT_ERR_INVALID_ARG
    assert lib.rt_render_stereo_sequence(None, None, 1, 0.065, 10.0, 8, 8, 1, None, None,
                                         None) == capi.RT_ERR_INVALID_ARG
    assert "NULL" in capi.rt_last_error()


def test_struct_layouts_match_header():
    # the header states 20, 40, 16, 16, 40 bytes per record
    assert [d.itemsize for d in (scenegen.SPHERE_DT, scenegen.TRIANGLE_DT, scenegen.MATERIAL_DT,
                                 scenegen.LIGHT_DT, scenegen.CAMERA_DT)] == [20, 40, 16, 16, 40]
    src = open(capi.HEADER).read()
    for frag in ("float center[3]; float radius; uint32_t material;",
                 "float albedo[3]; float reflectivity;",
                 "float position[3]; float intensity;"):
        assert frag in src


def test_batch_create_rejects_empty_and_null_requests_before_any_device_work():
    import ctypes
    L = capi.lib()
    out = ctypes.c_void_p()
    assert L.rt_batch_create(None, 0, None, ctypes.byref(out)) == capi.RT_ERR_INVALID_ARG
    reqs = capi.make_requests([(None, scenegen.config_small(1).camera, 0.065, 10.0, 8, 8, 1, 16, 16)])
    assert L.rt_batch_create(reqs.ctypes.data, 1, None, ctypes.byref(out)) == capi.RT_ERR_INVALID_ARG
    assert "scene is NULL" in capi.rt_last_error()
    assert out.value is None
    reqs["scene"][0] = 0
    reqs["reserved"][0] = 0
    assert capi.REQUEST_DT.itemsize == 88 and capi.BATCH_CONFIG_DT.itemsize == 24
