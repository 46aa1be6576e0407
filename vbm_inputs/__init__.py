"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds input generation only (volumes, orbit cameras, the
transfer-function knot table, random Gaussian sets and the workload table).
It contains none of the method's arithmetic: no wavelet transform, no
Gaussian mapping, no splatting and no ray marching.  Both the FP64 CPU oracle
and the CUDA path consume the arrays produced here, so that the two are
compared on identical bytes.
"""

from .volumes import blob_volume, spectral_noise, band_limited_blob_volume, \
    turbulence_volume, supernova_volume, volume_for_config
from .cameras import orbit_cameras, camera_array, CAMERA_FIELDS
from .tf_table import TF_KNOTS_X, TF_KNOTS_RGBA, TF_MODE_EDGES, tf_mode, tf_modes_union, transfer_function
from .configs import CONFIGS, config
from .gaussians import random_gaussians, gaussians_in_view

__all__ = [
    "blob_volume", "spectral_noise", "band_limited_blob_volume",
    "turbulence_volume", "supernova_volume", "volume_for_config",
    "orbit_cameras", "camera_array", "CAMERA_FIELDS",
    "TF_KNOTS_X", "TF_KNOTS_RGBA", "transfer_function", "TF_MODE_EDGES", "tf_mode", "tf_modes_union",
    "CONFIGS", "config", "random_gaussians", "gaussians_in_view",
]
