"""GB300-native probe-based irradiance field with visibility.

A C-ABI CUDA library (``include/ddgi.h``, sources in ``csrc/``) implements the
per-frame probe update and the shading-point query of Majercik, Marrs, Spjut
and McGuire, "Scaling Probe-Based Real-Time Dynamic Global Illumination for
Production" (JCGT 2021).  This package is its thin Python binding.
"""
from ._lib import (BLEND_BF16, BLEND_FP32, BLEND_TF32, BLEND_TF32X3, DIST_FP16, DIST_FP32, IRR_FP16,  # noqa: F401
                   IRR_FP32, IRR_RGB9E5, STATE_AWAKE, STATE_NEWLY_AWAKE, STATE_NEWLY_VIGILANT, STATE_OFF, STATE_SLEEPING,
                   STATE_UNINIT, STATE_VIGILANT, DDGIError, load)
from .api import (Cascade, IrradianceField, ProbeQuery, Scene, Volume, bvh_check, lights_struct, trace,  # noqa: F401
                  update_noalloc, update_noalloc_poll_status, measure_l2_read)
