"""Neumann angles of a liquid lens read off the concentration fields (test helper).

Geometry: a fluid-3 lens sitting on a horizontal fluid-1/fluid-2 interface,
fluid 1 below, fluid 2 above, in a periodic box (Sec. Liquid Lense).  The
C_3 = 1/2 contour is split at the 1/2 interface height into an upper arc
(lens against fluid 2) and a lower arc (lens against fluid 1); a circle is
fitted to each arc by linear least squares (points within ``skip`` nodes of the
triple points' height are dropped: the three diffuse interfaces overlap there).
The triple points are the circles' intersections; at them each cap meets the
horizontal at phi = arccos of (centre offset / radius), and the three angles
are theta_3 = phi_up + phi_low (inside the lens), theta_2 = 180 - phi_up (fluid
2), theta_1 = 180 - phi_low (fluid 1).
"""
import numpy as np


def _contour(C, level=0.5):
    ny, nx = C.shape
    pts = []
    for x in range(nx):
        col = C[:, x]
        for y in np.nonzero((col[:-1] > level) != (col[1:] > level))[0]:
            pts.append((x, y + (level - col[y]) / (col[y + 1] - col[y])))
    for y in range(ny):
        row = C[y, :]
        for x in np.nonzero((row[:-1] > level) != (row[1:] > level))[0]:
            pts.append((x + (level - row[x]) / (row[x + 1] - row[x]), y))
    return np.asarray(pts, dtype=np.float64)


def _circle(P):
    A = np.c_[2 * P[:, 0], 2 * P[:, 1], np.ones(len(P))]
    (xc, yc, c), *_ = np.linalg.lstsq(A, (P ** 2).sum(1), rcond=None)
    return xc, yc, float(np.sqrt(c + xc ** 2 + yc ** 2))


def interface_height(C1, C2, xs):
    """Mean height of the C_1 = C_2 crossing over the columns xs (far from the lens)."""
    ys = []
    for x in xs:
        d = C1[:, x] - C2[:, x]
        # the crossing with fluid 1 below and fluid 2 above
        for y in np.nonzero((d[:-1] > 0) & (d[1:] <= 0))[0]:
            ys.append(y + d[y] / (d[y] - d[y + 1]))
    return float(np.mean(ys))


def lens_angles(C1, C2, C3, far_columns, skip=4.0):
    """(theta_1, theta_2, theta_3) in degrees for fields [y][x] (one lens)."""
    y_if = interface_height(C1, C2, far_columns)
    P = _contour(C3)
    up = P[P[:, 1] > y_if + skip]
    low = P[P[:, 1] < y_if - skip]
    xu, yu, Ru = _circle(up)
    xl, yl, Rl = _circle(low)
    # intersection of the two circles (the triple points): their common chord
    d = np.hypot(xl - xu, yl - yu)
    a = (Ru ** 2 - Rl ** 2 + d ** 2) / (2 * d)
    yP = yu + a * (yl - yu) / d  # height of the chord's midpoint (the lens is symmetric in x)
    phi_up = np.degrees(np.arccos(np.clip((yP - yu) / Ru, -1, 1)))
    phi_low = np.degrees(np.arccos(np.clip((yl - yP) / Rl, -1, 1)))
    return 180.0 - phi_low, 180.0 - phi_up, phi_up + phi_low


def neumann_angles(g12, g13, g23):
    """(theta_1, theta_2, theta_3) from the force balance at the triple point:
    theta_m = 180 - (the angle of the tension triangle between the two sides that
    bound fluid m)."""
    def tri(a, b, opp):
        return np.degrees(np.arccos((a * a + b * b - opp * opp) / (2 * a * b)))
    t1 = 180.0 - tri(g12, g13, g23)
    t2 = 180.0 - tri(g12, g23, g13)
    t3 = 180.0 - tri(g13, g23, g12)
    return t1, t2, t3
