"""GB300 direct volume rendering of radio spectral cubes (Hassan et al. 2012).

PyTorch supplies device memory and streams; every step of the rendering runs
in libvr.so's CUDA kernels (see include/vr.h).  High-level helpers:

    vol = Volume(cube_tensor, store_dtype="f32")        # bricked, resident
    img, nsamp = render(vol, cam, tf, vmin, vmax, step, ert)
    img = render_diff(cube, vol, tf, cam, ...)          # autograd-aware

There is no CPU path: without a CUDA device or the built library every call
raises.
"""
from __future__ import annotations

from . import _lib
from ._lib import (VR_BF16, VR_CAMERA_ORTHO, VR_CAMERA_PERSPECTIVE, VR_F16, VR_F32, VR_FILTER_SOFTWARE,
                   VR_FILTER_TEXTURE, VR_MODE_COMPOSITE, VR_MODE_MIP, VR_MODE_SIGMA, VRError, make_camera,
                   make_params, vr_autotune_batched, vr_batch_opts, vr_job, vr_minimap, vr_profile, vr_render,
                   vr_render_backward, vr_render_batched, vr_volume_create, vr_volume_destroy, vr_volume_info,
                   vr_volume_update)
from .api import (Volume, autotune_batched, autotune_batched_bricks, composite, histogram, median, minimap, moments, profile, render, render_backward,
                  render_backward_views, render_batched, render_diff, render_subbox, RenderFunction)

__all__ = ["Volume", "autotune_batched", "autotune_batched_bricks", "render", "render_backward", "render_backward_views", "render_batched", "render_diff", "RenderFunction", "minimap",
           "profile", "moments", "histogram", "median", "render_subbox", "composite", "vr_volume_create", "vr_volume_update", "vr_volume_destroy", "vr_volume_info", "vr_render",
           "vr_render_backward", "vr_render_batched", "vr_autotune_batched", "vr_minimap", "vr_profile", "vr_job",
           "vr_batch_opts", "make_camera", "make_params", "VRError", "VR_F32", "VR_F16", "VR_BF16",
           "VR_CAMERA_ORTHO", "VR_CAMERA_PERSPECTIVE", "VR_FILTER_SOFTWARE", "VR_FILTER_TEXTURE",
           "VR_MODE_COMPOSITE", "VR_MODE_MIP", "VR_MODE_SIGMA"]
