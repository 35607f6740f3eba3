"""Contact angle of a sessile drop read off a concentration field (test helper).

The C = 1/2 contour of the drop is located by linear interpolation along rows
and columns, points closer than ``skip`` nodes to the wall plane are dropped
(the diffuse wall layer bends the contour there), a circle is fitted to the
rest by linear least squares (Kasa fit), and the angle through the drop
follows from the circle's centre height above the wall plane y_w:
cos theta = -(y_c - y_w) / R.
"""
import numpy as np


def drop_angle(C, y_wall: float, skip: float = 3.0, level: float = 0.5):
    """(theta in degrees through the drop, radius, centre height) for field C[y][x]."""
    ny, nx = C.shape
    pts = []
    for x in range(nx):
        col = C[:, x]
        s = np.nonzero((col[:-1] - level) * (col[1:] - level) < 0)[0]
        for y in s:
            yy = y + (level - col[y]) / (col[y + 1] - col[y])
            if yy > y_wall + skip:
                pts.append((x, yy))
    for y in range(int(np.ceil(y_wall + skip)), ny):
        row = C[y, :]
        s = np.nonzero((row[:-1] - level) * (row[1:] - level) < 0)[0]
        for x in s:
            pts.append((x + (level - row[x]) / (row[x + 1] - row[x]), y))
    P = np.asarray(pts, dtype=np.float64)
    if len(P) < 8:
        raise ValueError("no drop contour found")
    A = np.c_[2 * P[:, 0], 2 * P[:, 1], np.ones(len(P))]
    (xc, yc, c), *_ = np.linalg.lstsq(A, (P ** 2).sum(1), rcond=None)
    R = float(np.sqrt(c + xc ** 2 + yc ** 2))
    cos_t = np.clip(-(yc - y_wall) / R, -1.0, 1.0)
    return float(np.degrees(np.arccos(cos_t))), R, float(yc)
