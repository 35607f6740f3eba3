"""Seeded synthetic initial fields shaped like the paper's benchmarks.

This module holds no arithmetic of the lattice Boltzmann step: it only builds
initial concentration fields C_1, C_2, C_3 (and solid masks) and converts them
to the auxiliary fields rho = C_1 + C_2 + C_3, phi = C_1 - C_2, psi = C_3
(Sec. Auxiliary variables).  Both the GPU path's tests/benchmarks and the CPU
oracle receive the same float64 arrays from here.

Geometries follow the benchmark section: liquid lenses and double emulsions
(Sec. Liquid Lense and Double Emulsion), square wells (Sec. Contact Angles) and
spinodal decomposition from a noisy mixture (Sec. Ternary Phase Separation).
Interfaces are the flat-interface profile C = (1 + tanh(x / 2 alpha)) / 2 of
Eq. tanh, evaluated at integer node positions.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), mapped to [0, 1) by taking the
top 53 bits.  Layout: arrays are indexed [z][y][x] (x fastest), i.e. node
``x + nx*(y + ny*z)`` when flattened.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n consecutive SplitMix64 outputs for the given seed (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n doubles uniform in [lo, hi) from SplitMix64 (top 53 bits)."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def profile(d, alpha: float):
    """Equilibrium flat-interface profile (1 + tanh(d / 2 alpha)) / 2 (Eq. tanh)."""
    return 0.5 * (1.0 + np.tanh(np.asarray(d, dtype=np.float64) / (2.0 * alpha)))


def to_aux(C1, C2, C3):
    """(rho, phi, psi) from concentrations (Sec. Auxiliary variables)."""
    C1 = np.asarray(C1, dtype=np.float64)
    C2 = np.asarray(C2, dtype=np.float64)
    C3 = np.asarray(C3, dtype=np.float64)
    return C1 + C2 + C3, C1 - C2, C3.copy()


def _grid2(nx, ny):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                       indexing="ij")
    return x, y


def band(ny: int, nx: int, y_lo: float, y_hi: float, alpha: float):
    """Fluid band between two flat interfaces y_lo < y < y_hi, shape [ny][nx]."""
    _, y = _grid2(nx, ny)
    return 0.5 * (np.tanh((y - y_lo) / (2 * alpha)) - np.tanh((y - y_hi) / (2 * alpha)))


def lens(nx: int, ny: int, R: float, alpha: float = 1.0, y_lo=None, y_hi=None, centre=None):
    """Fluid-3 drop of radius R on a flat fluid-1 / fluid-2 interface (2-D).

    Fluid 1 fills the band y_lo < y < y_hi (default ny/4 .. 3ny/4), fluid 2 the
    rest; by periodicity there are two flat 1/2 interfaces.  The drop is centred
    on the upper interface, (nx/2, y_hi), unless ``centre`` is given.
    Returns C1, C2, C3 of shape [ny][nx].
    """
    y_lo = ny / 4 if y_lo is None else y_lo
    y_hi = 3 * ny / 4 if y_hi is None else y_hi
    cx, cy = (nx / 2, y_hi) if centre is None else centre
    x, y = _grid2(nx, ny)
    B = band(ny, nx, y_lo, y_hi, alpha)
    r = np.hypot(x - cx, y - cy)
    C3 = profile(-(r - R), alpha)
    return (1 - C3) * B, (1 - C3) * (1 - B), C3


def double_emulsion(nx: int, ny: int, r_core: float, r_shell: float, alpha: float = 1.0):
    """Concentric fluid-1 core (radius r_core) in a fluid-3 shell (outer radius
    r_shell) in fluid 2, centred at (nx/2, ny/2).  Returns C1, C2, C3."""
    x, y = _grid2(nx, ny)
    r = np.hypot(x - nx / 2, y - ny / 2)
    inner = profile(-(r - r_core), alpha)
    outer = profile(-(r - r_shell), alpha)
    C1 = inner
    C3 = outer - inner
    C2 = 1 - outer
    return C1, C2, C3


def drop(nx: int, ny: int, R: float, m: int, n: int, alpha: float = 1.0, nz: int = 1):
    """Drop of fluid m (radius R) in fluid n, centred in the box (0-based m, n).

    2-D if nz == 1 (shape [ny][nx]), else a sphere (shape [nz][ny][nx]).
    Returns the list [C1, C2, C3]."""
    if nz == 1:
        x, y = _grid2(nx, ny)
        r = np.hypot(x - nx / 2, y - ny / 2)
    else:
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        r = np.sqrt((x - nx / 2) ** 2 + (y - ny / 2) ** 2 + (z - nz / 2) ** 2)
    inside = profile(-(r - R), alpha)
    C = [np.zeros_like(inside) for _ in range(3)]
    C[m] = inside
    C[n] = 1 - inside
    return C


def flat_interfaces(nx: int, ny: int, m: int, n: int, alpha: float = 1.0, nz: int = 1):
    """Periodic slab: fluid m for nx/4 < x < 3nx/4, fluid n elsewhere.  The
    profile varies along x only.  Returns [C1, C2, C3] (shape [nz][ny][nx] or
    [ny][nx] when nz == 1)."""
    x = np.arange(nx, dtype=np.float64)
    s = 0.5 * (np.tanh((x - nx / 4) / (2 * alpha)) - np.tanh((x - 3 * nx / 4) / (2 * alpha)))
    shape = (ny, nx) if nz == 1 else (nz, ny, nx)
    inside = np.broadcast_to(s, shape).copy()
    C = [np.zeros(shape) for _ in range(3)]
    C[m] = inside
    C[n] = 1 - inside
    return C


def spinodal(shape, seed: int, C0=(1 / 3, 1 / 3, 1 / 3), amp: float = 0.01):
    """Homogeneous mixture C0 plus uniform noise in [-amp, amp) per node and
    component, renormalised so that C_1 + C_2 + C_3 = 1 (Sec. Ternary Phase
    Separation).  ``shape`` is (ny, nx) or (nz, ny, nx)."""
    n = int(np.prod(shape))
    C = []
    for m in range(3):
        noise = uniform(seed * 3 + m + 1, n, -amp, amp).reshape(shape)
        C.append(C0[m] + noise)
    s = C[0] + C[1] + C[2]
    return [c / s for c in C]


def walls_y(nx: int, ny: int, bottom: int = 1, top: int = 1):
    """Solid mask (uint8, [ny][nx]) with solid rows at the bottom and top."""
    s = np.zeros((ny, nx), dtype=np.uint8)
    if bottom:
        s[:bottom, :] = 1
    if top:
        s[ny - top:, :] = 1
    return s


def sessile_drop(nx: int, ny: int, R: float, m: int = 2, n: int = 0, alpha: float = 1.0,
                 wall: int = 1, lid: int = 1, theta0: float = 90.0):
    """Drop of fluid m resting on a bottom wall, in fluid n; solid rows at
    y < wall and y >= ny - lid.  The drop is a circular cap of radius R meeting
    the wall plane y = wall - 1/2 at the angle theta0 (degrees, through the
    drop; 90 = half disc).  Returns ([C1, C2, C3], solid)."""
    solid = walls_y(nx, ny, wall, lid)
    x, y = _grid2(nx, ny)
    r = np.hypot(x - nx / 2, y - (wall - 0.5 - R * np.cos(np.radians(theta0))))
    inside = profile(-(r - R), alpha)
    C = [np.zeros((ny, nx)) for _ in range(3)]
    C[m] = inside
    C[n] = 1 - inside
    for c in C:
        c[solid != 0] = 0.0
    return C, solid


def square_well(nx: int, ny: int, width: int, depth: int, floor: int = 8, alpha: float = 1.0,
                drop_radius=None, fill: float = 1.0, info: bool = False):
    """Square-well geometry of the contact-angle benchmark (Sec. Contact Angles).

    Solid: the bottom ``floor`` rows plus the top row, with a well of the given
    width and depth cut into a solid block that rises ``depth`` above the floor.
    The well is filled with fluid 3 up to ``fill`` of its depth (a flat surface
    with a tanh edge); fluid 1 fills the rest of the open region below a flat
    1/2 interface at mid-height of the region above the block, fluid 2 lies
    above it.  Returns ([C1, C2, C3], solid) with arrays of shape [ny][nx], and
    with info=True also the well's extent {x0, x1, y0, y1}: fluid columns
    x0..x1-1 between walls at x0 - 1/2 and x1 - 1/2, floor at y0 - 1/2, top of
    the block at y1 - 1/2.
    """
    solid = np.zeros((ny, nx), dtype=np.uint8)
    top_of_block = min(floor + depth, ny - 4)
    solid[:top_of_block, :] = 1
    x0 = max(1, (nx - width) // 2)
    x1 = min(nx - 1, x0 + width)
    solid[floor:top_of_block, x0:x1] = 0
    solid[ny - 1, :] = 1
    x, y = _grid2(nx, ny)
    # well filled with fluid 3 (a rectangle with diffuse top edge)
    level = floor - 0.5 + fill * (top_of_block - floor)
    inwell = (x >= x0) & (x < x1) & (y < top_of_block)
    C3 = np.where(inwell, profile(level - y, alpha), 0.0)
    if drop_radius is not None:
        r = np.hypot(x - nx / 2, y - top_of_block)
        C3 = np.maximum(C3, profile(-(r - drop_radius), alpha))
    y_if = top_of_block + (ny - 1 - top_of_block) / 2
    B = profile(y_if - y, alpha)
    C1 = (1 - C3) * B
    C2 = (1 - C3) * (1 - B)
    for c in (C1, C2, C3):
        c[solid != 0] = 0.0
    if info:
        return [C1, C2, C3], solid, dict(x0=x0, x1=x1, y0=floor, y1=top_of_block)
    return [C1, C2, C3], solid


# --------------------------------------------------------------- named configs

def lens_64_fp64():
    """64x64 periodic D2Q9 lens of the plain-FP64 parity run: fluid-1 band between
    y = 16 and y = 48, fluid-3 drop of radius 12 centred at (32, 48), alpha = 1,
    kappa = (0.01, 0.02, 0.03), tau_f = 1, M_phi = M_psi = 0.1."""
    C = lens(64, 64, 12.0, 1.0, 16.0, 48.0, (32.0, 48.0))
    return dict(Q=9, nx=64, ny=64, nz=1, kappa=(0.01, 0.02, 0.03), alpha=1.0, tau_f=1.0,
                M_phi=0.1, M_psi=0.1, h=(0.0, 0.0, 0.0), C=C, solid=None)


def kappa_draw(seed: int, lo: float = 0.005, hi: float = 0.05):
    """Three kappa values uniform in [lo, hi) from the given seed."""
    return tuple(float(v) for v in uniform(seed, 3, lo, hi))


def lens_512x256(seed: int = 2):
    """512x256 periodic D2Q9 liquid lens, radius 60 on a horizontal 1/2 interface
    at y = 128 (second interface at y = 0 by periodicity); kappa from seed."""
    C = lens(512, 256, 60.0, 1.0, 0.0, 128.0, (256.0, 128.0))
    return dict(Q=9, nx=512, ny=256, nz=1, kappa=kappa_draw(seed), alpha=1.0, tau_f=1.0,
                M_phi=0.1, M_psi=0.1, h=(0.0, 0.0, 0.0), C=C, solid=None)


def emulsion_512(seed: int = 2):
    """512x512 periodic D2Q9 double emulsion: fluid-1 core radius 60, fluid-3 shell
    to radius 100, in fluid 2; kappa from seed."""
    C = double_emulsion(512, 512, 60.0, 100.0, 1.0)
    return dict(Q=9, nx=512, ny=512, nz=1, kappa=kappa_draw(seed + 1), alpha=1.0, tau_f=1.0,
                M_phi=0.1, M_psi=0.1, h=(0.0, 0.0, 0.0), C=C, solid=None)


def spinodal_3d(n: int = 256, seed: int = 3):
    """n^3 periodic D3Q19 ternary spinodal decomposition: C_m = 1/3 + U[-0.01, 0.01)
    renormalised; kappa = 0.01 each, alpha = 1, tau_f = 0.8, M = 0.1."""
    C = spinodal((n, n, n), seed)
    return dict(Q=19, nx=n, ny=n, nz=n, kappa=(0.01, 0.01, 0.01), alpha=1.0, tau_f=0.8,
                M_phi=0.1, M_psi=0.1, h=(0.0, 0.0, 0.0), C=C, solid=None)


def probe_2d(n: int = 8192, seed: int = 5):
    """n^2 periodic D2Q9 spinodal mixture (an HBM-sized 2-D lattice)."""
    C = spinodal((n, n), seed)
    return dict(Q=9, nx=n, ny=n, nz=1, kappa=(0.01, 0.01, 0.01), alpha=1.0, tau_f=0.8,
                M_phi=0.1, M_psi=0.1, h=(0.0, 0.0, 0.0), C=C, solid=None)


def wells_2d(nx: int = 4096, ny: int = 2048, nwells: int = 32, seed: int = 4):
    """Wall-bounded D2Q9 lattice for timing the wetting path: solid floor
    (8 rows) and lid (1 row), ``nwells`` square wells of seeded width and depth
    cut into the floor block, each holding a fluid-3 drop; fluid 1 below a flat
    1/2 interface at mid-height, fluid 2 above.  Wetting h = (0.0004, -0.0004,
    0.0002) with kappa = (0.01, 0.01, 0.01)."""
    rng = uniform(seed, 2 * nwells)
    floor, block = 8, 40
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[:floor + block, :] = 1
    solid[ny - 1, :] = 1
    pitch = nx // nwells
    x, y = _grid2(nx, ny)
    C3 = np.zeros((ny, nx))
    for k in range(nwells):
        w = int(20 + 60 * rng[2 * k])
        dpt = int(10 + 30 * rng[2 * k + 1])
        x0 = k * pitch + (pitch - w) // 2
        y0 = floor + block - dpt
        solid[y0:floor + block, x0:x0 + w] = 0
        inwell = (x >= x0) & (x < x0 + w) & (y >= y0) & (y < floor + block)
        C3 = np.where(inwell, profile(floor + block - 0.5 - y, 1.0), C3)
    y_if = floor + block + (ny - 1 - floor - block) / 2
    B = profile(y_if - y, 1.0)
    C1 = (1 - C3) * B
    C2 = (1 - C3) * (1 - B)
    for c in (C1, C2, C3):
        c[solid != 0] = 0.0
    return dict(Q=9, nx=nx, ny=ny, nz=1, kappa=(0.01, 0.01, 0.01), alpha=1.0, tau_f=1.0,
                M_phi=0.1, M_psi=0.1, h=(0.0004, -0.0004, 0.0002), C=[C1, C2, C3], solid=solid)


def sweep_wells(count: int = 96, seed: int = 7, ncand: int = 16):
    """Contact-angle sweep of ``count`` independent D2Q9 square-well lattices of
    uneven size (Sec. Contact Angles, Fig. 2 settings: kappa = 0.01 each,
    alpha = 1, tau_f = 1, tau_phi = 1, tau_psi = 2/3 with Gamma = 1, i.e.
    M_phi = 1/2, M_psi = 1/6).

    Member k: nx = 128 + 32 j, j uniform in {0..20}, ny = nx / 2; floor 8 rows,
    a well of width uniform in [20, 120] (at most nx - 16) and depth uniform in
    [10, 60] (clipped to the lattice), its lower half filled with fluid 3 (the
    fluid-3/fluid-1 meniscus meets the well's side walls, away from its
    corners), fluid 1 above it and below a flat 1/2 interface, fluid 2 above.
    ``angles`` holds ``ncand`` candidate target pairs (theta_12, theta_13)
    uniform in [30, 150) degrees; the caller keeps the first pair its wetting
    inversion accepts and sets ``h`` from it.  ``well`` is the well's extent
    (square_well's info).
    """
    out = []
    for k in range(count):
        u = uniform(seed * 1000003 + k, 3 + 2 * ncand)
        nx = 128 + 32 * min(int(21 * u[0]), 20)
        ny = nx // 2
        width = min(int(20 + 100 * u[1]), nx - 16)
        depth = int(10 + 50 * u[2])
        C, solid, well = square_well(nx, ny, width, depth, floor=8, fill=0.5, info=True)
        angles = [(30 + 120 * u[3 + 2 * j], 30 + 120 * u[4 + 2 * j]) for j in range(ncand)]
        out.append(dict(Q=9, nx=nx, ny=ny, nz=1, kappa=(0.01, 0.01, 0.01), alpha=1.0, tau_f=1.0,
                        M_phi=0.5, M_psi=1.0 / 6.0, h=None, C=C, solid=solid, angles=angles, well=well))
    return out
