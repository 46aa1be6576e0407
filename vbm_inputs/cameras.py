"""Orbit cameras around a volume (pinhole, world -> camera rigid transform).

Camera frame: x right, y down, z forward (view direction).  A world point p
maps to camera space as p_c = R p + t and to the image plane as
(fx x_c / z_c + cx, fy y_c / z_c + cy); pixel (i, j) covers [i, i+1) x [j, j+1)
so its centre is (i + 0.5, j + 0.5).

Orbit: radius 1.8 G about the volume centre, 60 degree vertical field of view,
fx = fy = (H/2) / tan(30 deg), principal point at the image centre, world up
+z.  View v of V sits at azimuth 2 pi v / V + pi / 7 and elevation +20 deg for
even v, -20 deg for odd v.
"""

import numpy as np

# Packed record layout shared with the C ABI's camera struct: 20 32-bit words.
CAMERA_FIELDS = [("R", np.float32, (9,)), ("t", np.float32, (3,)),
                 ("fx", np.float32), ("fy", np.float32), ("cx", np.float32),
                 ("cy", np.float32), ("znear", np.float32),
                 ("width", np.int32), ("height", np.int32), ("pad", np.int32)]
CAMERA_DTYPE = np.dtype(CAMERA_FIELDS)
assert CAMERA_DTYPE.itemsize == 80


def look_at(position, target, up=(0.0, 0.0, 1.0)):
    """World->camera rotation and translation for a camera at position."""
    position = np.asarray(position, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - position
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ position
    return R, t


def orbit_cameras(dims, n_views, width, height, fov_y_deg=60.0, radius_scale=1.8,
                  znear=0.2):
    """List of camera dicts (float64) for an orbit around a volume of dims (nx, ny, nz)."""
    dims = np.asarray(dims, dtype=np.float64)
    centre = dims / 2.0
    G = dims.max()
    focal = (height / 2.0) / np.tan(np.radians(fov_y_deg) / 2.0)
    cams = []
    for v in range(n_views):
        az = 2.0 * np.pi * v / n_views + np.pi / 7.0
        el = np.radians(20.0 if v % 2 == 0 else -20.0)
        pos = centre + radius_scale * G * np.array(
            [np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        R, t = look_at(pos, centre)
        cams.append(dict(R=R, t=t, fx=focal, fy=focal, cx=width / 2.0, cy=height / 2.0,
                         znear=znear, width=int(width), height=int(height)))
    return cams


def camera_array(cams):
    """Pack camera dicts into the 80-byte records the C ABI reads."""
    out = np.zeros(len(cams), dtype=CAMERA_DTYPE)
    for i, c in enumerate(cams):
        out[i]["R"] = np.asarray(c["R"], dtype=np.float64).reshape(9)
        out[i]["t"] = np.asarray(c["t"], dtype=np.float64)
        for k in ("fx", "fy", "cx", "cy", "znear"):
            out[i][k] = c[k]
        out[i]["width"] = c["width"]
        out[i]["height"] = c["height"]
    return out


def cameras_as_float32(cams):
    """The camera dicts rounded to the float32 values the GPU path sees."""
    packed = camera_array(cams)
    res = []
    for rec in packed:
        res.append(dict(R=rec["R"].astype(np.float64).reshape(3, 3),
                        t=rec["t"].astype(np.float64), fx=float(rec["fx"]),
                        fy=float(rec["fy"]), cx=float(rec["cx"]), cy=float(rec["cy"]),
                        znear=float(rec["znear"]), width=int(rec["width"]),
                        height=int(rec["height"])))
    return res
