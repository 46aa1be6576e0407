"""Seeded synthetic scalar volumes standing in for the paper's datasets.

The paper evaluates on Supernova (432^3 float), Colon Prone (512x512x463,
16-bit) and Skull/Foot (256^3, 8-bit) (Sec. 5.1).  None of them is available
here, so these generators produce fields with comparable structure: smooth
anisotropic blobs plus noise, band-limited spectral noise, a turbulence-like
k^-5/3 field and a supernova-like set of perturbed radial shells.

Conventions: arrays are float32 with shape (nz, ny, nx) (x fastest); voxel
(i, j, k) covers [i, i+1) x [j, j+1) x [k, k+1) in world units, so its centre
sits at index + 0.5.  Every generator takes a numpy Generator (PCG64) so that
the same seed yields the same bytes on every machine.
"""

import numpy as np


def _random_rotation(rng):
    """Uniform random rotation matrix from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def _add_blobs(vol, n_blobs, rng, amp_range=(0.2, 1.0), sigma_range=(1.5, 5.0),
               centre_range=(0.2, 0.8)):
    """Add n_blobs anisotropic Gaussian blobs in place (float64 accumulation)."""
    nz, ny, nx = vol.shape
    dims = np.array([nx, ny, nz], dtype=np.float64)
    for _ in range(n_blobs):
        amp = rng.uniform(*amp_range)
        sig = rng.uniform(*sigma_range, size=3)
        rot = _random_rotation(rng)
        centre = rng.uniform(centre_range[0], centre_range[1], size=3) * dims
        prec = rot @ np.diag(1.0 / sig ** 2) @ rot.T
        half = 5.0 * sig.max()
        lo = np.maximum(np.floor(centre - half).astype(int), 0)
        hi = np.minimum(np.ceil(centre + half).astype(int) + 1, [nx, ny, nz])
        xs = np.arange(lo[0], hi[0]) + 0.5 - centre[0]
        ys = np.arange(lo[1], hi[1]) + 0.5 - centre[1]
        zs = np.arange(lo[2], hi[2]) + 0.5 - centre[2]
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        q = (prec[0, 0] * X * X + prec[1, 1] * Y * Y + prec[2, 2] * Z * Z
             + 2 * prec[0, 1] * X * Y + 2 * prec[0, 2] * X * Z + 2 * prec[1, 2] * Y * Z)
        vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += amp * np.exp(-0.5 * q)


def blob_volume(G, n_blobs, seed, noise_std=0.02):
    """Sum of n_blobs random anisotropic blobs + white noise, clamped to [0, 1].

    Amplitudes U[0.2, 1], per-axis sigmas U[1.5, 5] voxels under a uniform
    random rotation, centres U[0.2 G, 0.8 G] per axis.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    vol = np.zeros((G, G, G), dtype=np.float64)
    _add_blobs(vol, n_blobs, rng)
    vol += rng.normal(0.0, noise_std, size=vol.shape)
    return np.clip(vol, 0.0, 1.0).astype(np.float32)


def spectral_noise(G, amp_exponent, k_range, seed):
    """Random-phase Fourier field with per-mode amplitude |k|^-amp_exponent.

    Modes with integer wavenumber magnitude inside k_range = (k_lo, k_hi) get
    amplitude |k|^-p and a uniform random phase; all others are zero.  The
    result is real (inverse real FFT), zero mean and scaled to unit std.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    kx = np.fft.rfftfreq(G, d=1.0 / G)
    ky = np.fft.fftfreq(G, d=1.0 / G)
    kz = np.fft.fftfreq(G, d=1.0 / G)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    kmag = np.sqrt(KX * KX + KY * KY + KZ * KZ)
    band = (kmag >= k_range[0]) & (kmag <= k_range[1])
    amp = np.zeros_like(kmag)
    amp[band] = kmag[band] ** (-amp_exponent)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=kmag.shape)
    spec = amp * np.exp(1j * phase)
    field = np.fft.irfftn(spec, s=(G, G, G), axes=(0, 1, 2))
    field -= field.mean()
    std = field.std()
    if std > 0:
        field /= std
    return field


def band_limited_blob_volume(G, n_blobs, seed, noise_std=0.05):
    """Blobs plus band-limited noise with shell spectrum E(k) ~ k^-2 on [2, 16].

    E(k) ~ k^-2 integrated over a shell of area ~k^2 means a per-mode power
    ~k^-4, i.e. a per-mode amplitude ~k^-2.  The noise is scaled to
    noise_std and the sum clamped to [0, 1].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    vol = np.zeros((G, G, G), dtype=np.float64)
    _add_blobs(vol, n_blobs, rng)
    vol += noise_std * spectral_noise(G, 2.0, (2.0, 16.0), seed + 1000)
    return np.clip(vol, 0.0, 1.0).astype(np.float32)


def turbulence_volume(G, seed):
    """Turbulence-like field: E(k) ~ k^-5/3 on k in [1, G/2], min-max to [0, 1].

    A shell spectrum E(k) ~ k^-5/3 gives a per-mode amplitude ~k^-11/6.
    """
    f = spectral_noise(G, 11.0 / 6.0, (1.0, G / 2.0), seed)
    f = (f - f.min()) / (f.max() - f.min())
    return f.astype(np.float32)


def supernova_volume(G, seed):
    """Five noisy concentric radial shells plus a dense core, clamped to [0, 1].

    Shell s has radius R_s = f_s G/2 with f in {0.2, 0.35, 0.5, 0.65, 0.8},
    width w = 0.015 G and amplitude a_s in {0.4, 0.5, 0.6, 0.7, 0.8}; its
    radius is perturbed by 0.1 R_s n(x), n a unit-std k^-5/3 field.  The core
    is exp(-r^2 / (2 (0.05 G)^2)).
    """
    n = spectral_noise(G, 11.0 / 6.0, (1.0, G / 4.0), seed)
    c = np.arange(G, dtype=np.float64) + 0.5 - G / 2.0
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    vol = np.exp(-r * r / (2.0 * (0.05 * G) ** 2))
    w = 0.015 * G
    for f, a in zip((0.2, 0.35, 0.5, 0.65, 0.8), (0.4, 0.5, 0.6, 0.7, 0.8)):
        R = f * G / 2.0
        d = r - R * (1.0 + 0.1 * n)
        vol += a * np.exp(-d * d / (2.0 * w * w))
    return np.clip(vol, 0.0, 1.0).astype(np.float32)


def volume_for_config(cfg, index=0):
    """The volume a workload entry names (index picks one of several volumes)."""
    kind = cfg["volume"]
    seed = cfg["seed"] * 100 + index
    if kind == "blobs":
        G = cfg["edges"][index] if "edges" in cfg else cfg["G"]
        n_blobs = cfg.get("blobs", max(1, int(round(4 * (G / 32.0) ** 3))))
        return blob_volume(G, n_blobs, seed)
    if kind == "blobs+bandnoise":
        return band_limited_blob_volume(cfg["G"], cfg["blobs"], seed)
    if kind == "turbulence":
        return turbulence_volume(cfg["G"], seed)
    if kind == "supernova":
        return supernova_volume(cfg["G"], seed)
    raise ValueError(kind)
