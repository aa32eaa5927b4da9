"""Seeded synthetic pansharpening scenes (inputs only).

This package is shared by the tests, the benchmark and the oracle checks. It
holds none of the method's arithmetic: the degradation that turns a ground
truth HRMS cube into the observed LRMS (circular blur by a kernel, then
decimation, Sec. II-A, Eq. objective0) is simulated here with numpy's FFT, an
implementation independent of both the CUDA path and the oracle.
"""
from .scenes import (SceneConfig, CONFIGS, make_scene, make_kernel,
                     make_batch_configs, crop_scene, make_scenes_parallel)

__all__ = ["SceneConfig", "CONFIGS", "make_scene", "make_kernel",
           "make_batch_configs", "crop_scene", "make_scenes_parallel"]
