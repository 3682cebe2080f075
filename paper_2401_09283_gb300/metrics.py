"""Evaluation of recovered motion: the reprojection error of Sec. IV-A.

RPE: project fixed 3D points with two geometries and average the distance
of their detector images, in detector mm (pixel distance times the pixel
pitch), over points and views.  Host-side numpy; not on the hot path."""
from __future__ import annotations

import numpy as np


def reprojection_error(Pa, Pb, points, du, dv):
    """Mean detector distance (mm) between the images of points (n,3) under
    the matrices Pa and Pb (V,3,4)."""
    Pa = np.asarray(Pa, dtype=np.float64)
    Pb = np.asarray(Pb, dtype=np.float64)
    X = np.concatenate([np.asarray(points, np.float64), np.ones((len(points), 1))], axis=1)
    a = np.einsum("vrk,nk->vnr", Pa, X)
    b = np.einsum("vrk,nk->vnr", Pb, X)
    du_mm = (a[..., 0] / a[..., 2] - b[..., 0] / b[..., 2]) * du
    dv_mm = (a[..., 1] / a[..., 2] - b[..., 1] / b[..., 2]) * dv
    return float(np.mean(np.sqrt(du_mm ** 2 + dv_mm ** 2)))
