"""Contact angle of the fluid-3 meniscus in a square well (test helper).

Geometry (workloads.square_well with info=True): fluid columns x0..x1-1 between
side walls at x0 - 1/2 and x1 - 1/2 (halfway bounce-back), floor at y0 - 1/2,
top of the block at y1 - 1/2; fluid 3 below the meniscus, fluid 1 above.

The C_3 = 1/2 crossing is located in every column at least ``skip`` nodes from
the walls (linear interpolation along the column); an algebraic circle fit
(Pratt's normalisation, which also represents a straight line) is made to these
points.  At each wall the fitted curve's point and tangent give the angle
between the wall below the contact line (fluid 3's side) and the meniscus,
i.e. theta_31 through fluid 3.  The meniscus is "free" when, on both walls,
the C_3 = 1/2 crossing in the fluid column next to the wall (the contact line)
and the fitted curve at the wall lie at least ``margin`` nodes from the well's
floor and top, and its apex (the fitted curve at the well's centre) does too;
otherwise it is pinned at a corner or touches the floor and the angle is not a
contact angle.
"""
import numpy as np


def _pratt(P):
    """A (x^2 + y^2) + D x + E y + F = 0 with D^2 + E^2 - 4 A F = 1, least squares."""
    m = P.mean(0)
    Q = P - m
    Z = np.c_[(Q ** 2).sum(1), Q[:, 0], Q[:, 1], np.ones(len(Q))]
    M = Z.T @ Z
    B = np.array([[0, 0, 0, -2], [0, 1, 0, 0], [0, 0, 1, 0], [-2, 0, 0, 0]], dtype=float)
    w, V = np.linalg.eig(np.linalg.solve(M + 1e-300 * np.eye(4), B))
    # the sought solution maximises 1/eta: the largest real eigenvalue of M^-1 B
    k = int(np.argmax(np.real(w)))
    a = np.real(V[:, k])
    a /= np.sqrt(abs(a[1] ** 2 + a[2] ** 2 - 4 * a[0] * a[3]))
    A, D, E, F = a
    # back to the original coordinates: substitute x - mx, y - my
    mx, my = m
    D2 = D - 2 * A * mx
    E2 = E - 2 * A * my
    F2 = A * (mx * mx + my * my) - D * mx - E * my + F
    return A, D2, E2, F2


def meniscus_angle(C3, well, skip=3.0, margin=2.0, level=0.5):
    """(theta_31 in degrees, contact heights (left, right), free) for C3[y][x]."""
    x0, x1, y0, y1 = well["x0"], well["x1"], well["y0"], well["y1"]
    pts = []
    for x in range(x0, x1):
        if x - (x0 - 0.5) < skip or (x1 - 0.5) - x < skip:
            continue
        col = C3[y0:y1, x]
        s = np.nonzero((col[:-1] >= level) & (col[1:] < level))[0]
        if len(s) == 0:
            continue
        y = s[-1]
        pts.append((x, y0 + y + (col[y] - level) / (col[y] - col[y + 1])))
    if len(pts) < 5:
        return float("nan"), (float("nan"), float("nan")), False
    P = np.asarray(pts, dtype=np.float64)
    A, D, E, F = _pratt(P)
    ym = float(np.median(P[:, 1]))
    thetas, heights = [], []
    for xw, inward in ((x0 - 0.5, +1.0), (x1 - 0.5, -1.0)):
        c = A * xw * xw + D * xw + F
        if abs(A) < 1e-14:
            yw = -c / E
        else:
            disc = E * E - 4 * A * c
            if disc < 0:
                return float("nan"), (float("nan"), float("nan")), False
            r = np.sqrt(disc)
            roots = ((-E + r) / (2 * A), (-E - r) / (2 * A))
            yw = min(roots, key=lambda v: abs(v - ym))
        # tangent of the conic at the wall point, oriented into the well
        gx, gy = 2 * A * xw + D, 2 * A * yw + E
        t = np.array([-gy, gx])
        if t[0] * inward < 0:
            t = -t
        t /= np.hypot(*t)
        thetas.append(float(np.degrees(np.arccos(np.clip(-t[1], -1.0, 1.0)))))
        heights.append(float(yw))
    xm = 0.5 * (x0 + x1) - 0.5
    c = A * xm * xm + D * xm + F
    if abs(A) < 1e-14:
        apex = -c / E
    else:
        disc = E * E - 4 * A * c
        apex = min(((-E + np.sqrt(disc)) / (2 * A), (-E - np.sqrt(disc)) / (2 * A)),
                   key=lambda v: abs(v - ym)) if disc >= 0 else float("nan")
    lo, hi = y0 - 0.5 + margin, y1 - 0.5 - margin
    # contact line read directly in the fluid columns next to the walls
    walls = []
    for x in (x0, x1 - 1):
        col = C3[y0:y1, x]
        s = np.nonzero((col[:-1] >= level) & (col[1:] < level))[0]
        walls.append(y0 + s[-1] + (col[s[-1]] - level) / (col[s[-1]] - col[s[-1] + 1]) if len(s) else float("nan"))
    free = (all(lo <= h <= hi for h in heights) and all(lo <= h <= hi for h in walls)
            and lo <= apex <= hi)
    return float(np.mean(thetas)), tuple(heights), free
