"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/vr.h declares, and rejects invalid arguments on the host
before anything is enqueued (no CUDA work is issued by these calls)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1211_4896_gb300 import build
    build.build()
    from paper_1211_4896_gb300 import _lib
    return _lib


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(vr_\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(L):
    lib = L.load()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.EXPORTS)


def test_version(L):
    assert "sm_103a" in L.vr_version()


def _cam(**kw):
    d = dict(kind=1, eye=(0, 0, -5), forward=(0, 0, 1), up=(0, 1, 0), fov_y_deg=40.0, width=8, height=8)
    d.update(kw)
    return d


@pytest.mark.parametrize("cam_kw,msg", [
    (dict(kind=3), "camera.kind"),
    (dict(width=0), "width"),
    (dict(height=40000), "height"),
    (dict(fov_y_deg=0.0), "fov_y_deg"),
    (dict(fov_y_deg=180.0), "fov_y_deg"),
    (dict(up=(0, 0, 2)), "parallel"),
    (dict(forward=(0, 0, 0)), "non-zero"),
    (dict(eye=(float("nan"), 0, 0)), "finite"),
    (dict(kind=0, ortho_height=-1.0), "ortho_height"),
])
def test_camera_validation(L, cam_kw, msg):
    p = L.make_params(4096, 256, -3, 50, 0.5)
    with pytest.raises(L.VRError) as ei:
        L.vr_render(None, L.make_camera(_cam(**cam_kw)), p, 4096, None)
    assert ei.value.status == L.VR_ERR_INVALID_ARG and msg in str(ei.value)


@pytest.mark.parametrize("kw,msg", [
    (dict(tf_ptr=0), "tf_rgba is NULL"),
    (dict(tf_ptr=4100), "16-byte aligned"),
    (dict(K=1), "tf_size"),
    (dict(K=5000), "tf_size"),
    (dict(vmin=5.0, vmax=5.0), "vmax > vmin"),
    (dict(step=0.0), "step"),
    (dict(step=float("inf")), "step"),
    (dict(ert=0.0), "ert_threshold"),
    (dict(bg=(0, float("nan"), 0, 0)), "bg_rgba"),
    (dict(filter=7), "filter"),
])
def test_params_validation(L, kw, msg):
    a = dict(tf_ptr=4096, K=256, vmin=-3.0, vmax=50.0, step=0.5, ert=2.0, bg=(0, 0, 0, 0), filter=0)
    a.update(kw)
    p = L.make_params(a["tf_ptr"], a["K"], a["vmin"], a["vmax"], a["step"], a["ert"], a["bg"], a["filter"])
    with pytest.raises(L.VRError) as ei:
        L.vr_render(None, L.make_camera(_cam()), p, 4096, None)
    assert ei.value.status == L.VR_ERR_INVALID_ARG and msg in str(ei.value)


def test_output_and_volume_validation(L):
    p = L.make_params(4096, 256, -3, 50, 0.5)
    cam = L.make_camera(_cam())
    with pytest.raises(L.VRError, match="dev_rgba_out is NULL"):
        L.vr_render(None, cam, p, None, None)
    with pytest.raises(L.VRError, match="16-byte aligned"):
        L.vr_render(None, cam, p, 4104, None)
    with pytest.raises(L.VRError, match="volume handle is NULL"):
        L.vr_render(None, cam, p, 4096, None)
    with pytest.raises(L.VRError, match="texture|differentiable"):
        L.vr_render_backward(None, cam, L.make_params(4096, 256, -3, 50, 0.5, filter=1), 4096, 4096, 4096, 4096,
                             None)
    with pytest.raises(L.VRError, match="flags: unknown"):
        L.vr_render_backward(None, cam, L.make_params(4096, 256, -3, 50, 0.5), 4096, 4096, 4096, 4096, None, 8)
    with pytest.raises(L.VRError, match="exclude each other"):
        L.vr_render_backward(None, cam, L.make_params(4096, 256, -3, 50, 0.5), 4096, 4096, 4096, 4096, None,
                             L.VR_GRAD_DIRECT | L.VR_GRAD_SCRATCH)
    with pytest.raises(L.VRError) as ei:
        L.vr_render_backward(None, cam, L.make_params(4096, 256, -3, 50, 0.5, bg=(0, 0, 0, 1)), 4096, 4096, 4096,
                             4096, None)
    assert ei.value.status == L.VR_ERR_UNSUPPORTED
    p = L.make_params(4096, 256, -3, 50, 0.5)
    with pytest.raises(L.VRError, match="at least one view"):
        L.vr_render_backward_views(None, [], p, 4096, None)
    with pytest.raises(L.VRError, match="must not be NULL"):
        L.vr_render_backward_views(None, [L.vr_grad_view(cam, 4096, 4096, 4096), L.vr_grad_view(cam, 4096, None,
                                                                                                4096)], p, 4096, None)
    with pytest.raises(L.VRError, match="16-byte aligned"):
        L.vr_render_backward_views(None, [L.vr_grad_view(cam, 4104, 4096, 4096)], p, 4096, None)
    with pytest.raises(L.VRError, match="volume handle is NULL"):
        L.vr_render_backward_views(None, [L.vr_grad_view(cam, 4096, 4096, 4096)] * 3, p, 4096, None)
    with pytest.raises(L.VRError, match="volume handle is NULL"):
        L.vr_view_layout(None, cam)
    with pytest.raises(L.VRError, match="camera"):
        L.vr_view_layout(None, L.make_camera(dict(_cam(), width=0)))
    with pytest.raises(L.VRError, match="volume handle is NULL"):
        L.vr_render_subbox_of(None, (64, 64, 64), (0, 0, 0), cam, p, (0, 0, 0), (8, 8, 8), 4096, 4096, None)
    with pytest.raises(L.VRError, match="software filter"):
        L.vr_render_subbox_of(None, (64, 64, 64), (0, 0, 0), cam, L.make_params(4096, 256, -3, 50, 0.5, filter=1),
                              (0, 0, 0), (8, 8, 8), 4096, 4096, None)


def test_volume_create_validation(L):
    with pytest.raises(L.VRError, match="dev_cube is NULL"):
        L.vr_volume_create(None, L.VR_F32, L.VR_F32, (8, 8, 8))
    with pytest.raises(L.VRError, match="dims"):
        L.vr_volume_create(4096, L.VR_F32, L.VR_F32, (1, 8, 8))
    with pytest.raises(L.VRError, match="dtype"):
        L.vr_volume_create(4096, 7, L.VR_F32, (8, 8, 8))
    with pytest.raises(L.VRError, match="brick"):
        L.vr_volume_create(4096, L.VR_F32, L.VR_F32, (8, 8, 8), brick=24)
    with pytest.raises(L.VRError, match="spacing"):
        L.vr_volume_create(4096, L.VR_F32, L.VR_F32, (8, 8, 8), spacing=(1, 0, 1))
    assert L.vr_volume_destroy(None) is None


def test_batched_validation(L):
    with pytest.raises(L.VRError, match="n >= 1"):
        L.vr_render_batched([], L.vr_batch_opts(0, 0, 0, 0))
    job = L.vr_job(None, L.make_camera(_cam()), L.make_params(4096, 256, -3, 50, 0.5), 4096, None)
    with pytest.raises(L.VRError, match="tile_w"):
        L.vr_render_batched([job], L.vr_batch_opts(0, 5, 6, 0))
    with pytest.raises(L.VRError, match=r"jobs\[0\]"):
        L.vr_render_batched([job], L.vr_batch_opts(0, 8, 4, 0))
    for wpt in (3, 8, -1):
        with pytest.raises(L.VRError, match="warps_per_tile"):
            L.vr_render_batched([job], L.vr_batch_opts(0, 8, 4, 0, wpt))


def test_rebrick_validation(L):
    with pytest.raises(L.VRError, match="volume handle is NULL"):
        L.vr_volume_rebrick(None, 32)


def test_product_path_has_no_cpu_fallback(L):
    """Without a CUDA device the high-level API refuses CPU tensors."""
    torch = pytest.importorskip("torch")
    import paper_1211_4896_gb300 as P
    with pytest.raises(ValueError, match="CUDA"):
        P.Volume(torch.zeros((4, 4, 4)))
