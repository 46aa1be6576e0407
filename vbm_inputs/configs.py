"""Workload table: the synthetic workloads the tests and benchmark use.

Each entry names the volume recipe, wavelet levels J, global coefficient
budget K_tot, number of views and image size.  K_tot is the budget handed to
the adaptive filter; because the MAD threshold leaves many subbands below
their share, the number of Gaussians kept is smaller, and each K_tot is set
so that the kept count lands at the workload's stated size (c0 keeps ~3.4k,
the cap of its MAD candidate set; c1 ~1.0e5; c2 ~5.0e5; c4 ~2.9e6).  Sizes follow the scale of the
paper's datasets (Sec. 5.1: 256^3 to 512^3 volumes; Sec. 5.3: ~1.8e5 Gaussians
for Supernova) while staying synthetic.
"""

import numpy as np

_C3_EDGE_CHOICES = (32, 48, 64, 96, 128)


def _c3_edges(seed=3, n=32):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(e) for e in rng.choice(_C3_EDGE_CHOICES, size=n)]


CONFIGS = {
    "c0": dict(key="c0", workload="tiny: 32^3 blobs, J=2, ~4k Gaussians, 1 view 128x128",
               volume="blobs", G=32, blobs=4, seed=0, levels=2, K_tot=10000,
               views=1, width=128, height=128),
    "c1": dict(key="c1", workload="128^3 blobs+k^-2 noise, J=3, ~100k Gaussians, 8 views 512x512",
               volume="blobs+bandnoise", G=128, blobs=32, seed=1, levels=3, K_tot=250000,
               views=8, width=512, height=512),
    "c2": dict(key="c2", workload="256^3 k^-5/3 turbulence, J=4, ~500k Gaussians, 16 views 800x800",
               volume="turbulence", G=256, seed=2, levels=4, K_tot=680000,
               views=16, width=800, height=800),
    "c3": dict(key="c3", workload="32 uneven blob volumes (edges 32..128), J=2, 4 views 256x256 each",
               volume="blobs", edges=_c3_edges(), seed=3, levels=2, K_tot_frac=0.07,
               views_per_volume=4, width=256, height=256),
    "c4": dict(key="c4", workload="512^3 supernova-like shells, J=5, ~3M Gaussians, 8 views 1024x1024",
               volume="supernova", G=512, seed=4, levels=5, K_tot=3000000,
               views=8, width=1024, height=1024, fwd_only=(1920, 1080), recompute=True),
    # Sec. 4.4's TF modes: the c1 volume under five transfer functions with
    # disjoint value intervals, one Gaussian set (scene) per mode, each
    # fine-tuned against its own DVR targets, all in one batch
    "c5": dict(key="c5", workload="c1 volume under 5 TF modes, one Gaussian set per mode, 8 views 512x512 per mode",
               volume="blobs+bandnoise", G=128, blobs=32, seed=1, levels=3, K_tot=250000,
               views=8, width=512, height=512, modes=5),
}


def config(key):
    """A copy of one workload entry."""
    return dict(CONFIGS[key])
