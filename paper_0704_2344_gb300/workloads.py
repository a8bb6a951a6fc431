"""Seeded synthetic inputs for the voxel H-field scattering solver.

This module only describes problems: voxel grids with a material per
hexahedron, material tables, frequencies and incident plane waves.  It holds
none of the finite-element arithmetic, so the CUDA path and the CPU oracle
both draw their inputs from here and from nowhere else.

Conventions (shared by every consumer):
  * element (i, j, k) has id  i + nx*(j + ny*k); ``material`` is a uint8 array
    of shape (nz, ny, nx) so that ``material.ravel()[id]`` is that element;
  * material byte m < len(eps_r) indexes the material table, 255 is a perfect
    electric conductor (the element is not meshed);
  * an incident plane wave is H_i(r) = p_hat * amplitude * exp(-j k0 k_hat . r)
    (e^{j omega t} time convention, SI units, r in metres from the world
    origin).

The workload shapes follow the paper's sizing example (a 3-wavelength cube at
3 GHz meshed with 10 first-order hexahedra per wavelength, Section 1), its PEC
airplane (Section 3.2) and its 10^6-node fighter estimate (Section 5.1); the
paper's own meshes are not available, so seeded voxel stand-ins replace them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

C0 = 299_792_458.0  # speed of light in vacuum, m/s (exact SI value)
AIR = 0
PEC = 255
SEED_BASE = 20070704


@dataclass
class VoxelProblem:
    nx: int
    ny: int
    nz: int
    h: tuple  # (hx, hy, hz) element edge lengths in metres
    origin: tuple  # world coordinates of node (0, 0, 0)
    material: np.ndarray  # uint8, shape (nz, ny, nx)
    eps_r: np.ndarray  # complex128 [n_materials]
    mu_r: np.ndarray  # complex128 [n_materials]
    freq_hz: float
    name: str = ""
    # kind of each box face (-x, +x, -y, +y, -z, +z): 0 absorbing boundary
    # (Eq. 3), 1 symmetry plane (n . H = 0, Eq. 6a), 2 antisymmetry plane
    # (n x H = 0, Eq. 6b)
    boundary: tuple = (0, 0, 0, 0, 0, 0)

    @property
    def n_elements(self) -> int:
        return self.nx * self.ny * self.nz


@dataclass
class PlaneWaves:
    k_hat: np.ndarray  # float64 [R, 3], unit propagation directions
    p_hat: np.ndarray  # float64 [R, 3], unit H polarisations, p_hat . k_hat = 0
    amplitude: np.ndarray = field(default=None)  # complex128 [R]

    def __post_init__(self):
        self.k_hat = np.ascontiguousarray(np.atleast_2d(self.k_hat), dtype=np.float64)
        self.p_hat = np.ascontiguousarray(np.atleast_2d(self.p_hat), dtype=np.float64)
        if self.amplitude is None:
            self.amplitude = np.ones(self.k_hat.shape[0], dtype=np.complex128)
        self.amplitude = np.ascontiguousarray(self.amplitude, dtype=np.complex128).reshape(-1)

    @property
    def count(self) -> int:
        return self.k_hat.shape[0]

    def column(self, r: int) -> "PlaneWaves":
        return PlaneWaves(self.k_hat[r:r + 1], self.p_hat[r:r + 1], self.amplitude[r:r + 1])


def wavelength(freq_hz: float) -> float:
    return C0 / freq_hz


def rng_for(config_index: int, extra: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + config_index + 1000 * extra)


def _air_table():
    return np.array([1.0 + 0j]), np.array([1.0 + 0j])


def empty_box(n, freq_hz=3e9, per_wavelength=10.0, name="empty") -> VoxelProblem:
    """Free-space box of n = (nx, ny, nz) cubic elements of edge lambda/per_wavelength."""
    if np.isscalar(n):
        n = (n, n, n)
    nx, ny, nz = (int(v) for v in n)
    hh = wavelength(freq_hz) / per_wavelength
    eps, mu = _air_table()
    return VoxelProblem(nx, ny, nz, (hh, hh, hh), (0.0, 0.0, 0.0),
                        np.zeros((nz, ny, nx), dtype=np.uint8), eps, mu, freq_hz, name)


def normal_incidence() -> PlaneWaves:
    """x-polarised H travelling along +z."""
    return PlaneWaves(np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))


def oblique_wave(theta: float, phi: float, pol: str = "theta") -> PlaneWaves:
    k, th, ph = _sph_frame(np.array([theta]), np.array([phi]))
    return PlaneWaves(k, th if pol == "theta" else ph)


def _sph_frame(theta, phi):
    st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    k = np.stack([st * cp, st * sp, ct], axis=-1)
    t = np.stack([ct * cp, ct * sp, -st], axis=-1)
    p = np.stack([-sp, cp, np.zeros_like(phi)], axis=-1)
    return k, t, p


def sphere_waves(n_dir: int = 32, seed: int = SEED_BASE + 3) -> PlaneWaves:
    """n_dir Fibonacci-sphere directions under a seeded random rotation, each
    with the two polarisations theta_hat and phi_hat of k_hat (2*n_dir waves,
    ordered direction-major)."""
    rng = np.random.default_rng(seed)
    i = np.arange(n_dir) + 0.5
    z = 1.0 - 2.0 * i / n_dir
    golden = np.pi * (3.0 - np.sqrt(5.0))
    phi0 = golden * np.arange(n_dir)
    r = np.sqrt(1.0 - z * z)
    pts = np.stack([r * np.cos(phi0), r * np.sin(phi0), z], axis=-1)
    q, rr = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(rr))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    pts = pts @ q.T
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    theta = np.arccos(np.clip(pts[:, 2], -1.0, 1.0))
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    k, t, p = _sph_frame(theta, phi)
    k_hat = np.repeat(k, 2, axis=0)
    p_hat = np.empty_like(k_hat)
    p_hat[0::2] = t
    p_hat[1::2] = p
    return PlaneWaves(k_hat, p_hat)


def random_waves(count: int, rng: np.random.Generator) -> PlaneWaves:
    v = rng.standard_normal((count, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    theta = np.arccos(np.clip(v[:, 2], -1.0, 1.0))
    phi = np.arctan2(v[:, 1], v[:, 0])
    k, t, p = _sph_frame(theta, phi)
    mix = rng.uniform(0.0, 2.0 * np.pi, count)
    pol = np.cos(mix)[:, None] * t + np.sin(mix)[:, None] * p
    return PlaneWaves(k, pol)


# --------------------------------------------------------------------------
# The five workloads.
# --------------------------------------------------------------------------

def config1() -> tuple[VoxelProblem, PlaneWaves]:
    """Empty free-space cube, 1 wavelength per side at 3 GHz, 10^3 elements."""
    return empty_box(10, 3e9, 10.0, name="cube1l_empty_10e3"), normal_incidence()


def config2_mesh(seed_index: int = 2) -> VoxelProblem:
    """3-wavelength cube (30^3 elements of lambda/10 at 3 GHz) with a centred
    6^3-element PEC cube and an eps_r = 4 slab (18 x 18 x 3 elements) at a
    seeded height, two or more elements from the outer box and the PEC cube."""
    rng = rng_for(seed_index)
    n = 30
    prob = empty_box(n, 3e9, 10.0, name="cube3l_pec_slab_30e3")
    mat = prob.material
    c0, c1 = 12, 18  # PEC cube occupies elements 12..17 on every axis
    mat[c0:c1, c0:c1, c0:c1] = PEC
    candidates = list(range(2, 8)) + list(range(20, 26))
    kz = int(rng.choice(candidates))
    mat[kz:kz + 3, 6:24, 6:24] = 1
    prob.eps_r = np.array([1.0 + 0j, 4.0 + 0j])
    prob.mu_r = np.array([1.0 + 0j, 1.0 + 0j])
    return prob


def config2() -> tuple[VoxelProblem, PlaneWaves]:
    return config2_mesh(2), normal_incidence()


def config3() -> tuple[VoxelProblem, PlaneWaves]:
    """The 3-wavelength mesh with 64 plane waves (32 directions x 2 pols)."""
    return config2_mesh(2), sphere_waves(32, SEED_BASE + 3)


def aircraft_mesh(n: int = 80, seed_index: int = 4, freq_hz: float = 3e9) -> VoxelProblem:
    """8-wavelength box around a voxel aircraft-like PEC body: a fuselage
    cylinder along x (5 wavelengths long, radius 0.4), a swept wing built from
    stepped boxes, a tail fin and a tailplane; dimensions seeded."""
    rng = rng_for(seed_index)
    prob = empty_box(n, freq_hz, 10.0, name=f"aircraft_{n}e3")
    mat = prob.material
    s = n / 80.0
    cy = cz = n // 2
    length = int(round(50 * s))
    radius = 4.0 * s
    x0 = (n - length) // 2
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    yc = j + 0.5 - cy
    zc = k + 0.5 - cz
    body = (i >= x0) & (i < x0 + length) & (yc * yc + zc * zc <= radius * radius)
    mat[body] = PEC
    span = int(round((36 + rng.integers(-4, 5)) * s))
    chord = int(round((10 + rng.integers(-2, 3)) * s))
    thick = int(rng.integers(1, 3))
    sweep = max(1, int(round(rng.uniform(1.0, 2.5) * s)))
    wx = x0 + int(round(length * 0.35))
    steps = 4
    half = span // 2
    for side in (-1, 1):
        for st in range(steps):
            ya = cy + side * (st * half // steps)
            yb = cy + side * ((st + 1) * half // steps)
            lo, hi = min(ya, yb), max(ya, yb)
            xa = wx + st * sweep
            mat[cz - 1:cz - 1 + thick, lo:hi + 1, xa:xa + max(2, chord - st)] = PEC
    tail_x = x0 + length - int(round(7 * s))
    fin_h = int(round((9 + rng.integers(-1, 2)) * s))
    mat[cz:cz + int(radius) + fin_h, cy:cy + thick, tail_x:tail_x + int(round(6 * s))] = PEC
    tp_span = int(round(14 * s))
    mat[cz:cz + 1, cy - tp_span // 2:cy + tp_span // 2 + 1, tail_x:tail_x + int(round(5 * s))] = PEC
    margin = 3
    inner = np.ones_like(mat, dtype=bool)
    inner[margin:-margin, margin:-margin, margin:-margin] = False
    if np.any(mat[inner] == PEC):
        raise ValueError("aircraft touches the outer margin")
    return prob


def config4() -> tuple[VoxelProblem, PlaneWaves]:
    rng = rng_for(4, extra=1)
    return aircraft_mesh(80, 4), random_waves(16, rng)


@dataclass
class Request:
    arrival_s: float
    problem: VoxelProblem
    waves: PlaneWaves


def pec_box_problem(n_elem: int, freq_hz: float, rng: np.random.Generator, name="req") -> VoxelProblem:
    """Cube of n_elem^3 elements of lambda/10 with a random PEC box two or more
    elements away from the outer faces."""
    prob = empty_box(n_elem, freq_hz, 10.0, name=name)
    room = n_elem - 4
    side_max = max(1, min(room, n_elem // 3))
    if room >= 1:
        side = [int(rng.integers(1, side_max + 1)) for _ in range(3)]
        lo = [int(rng.integers(2, n_elem - 2 - sd + 1)) for sd in side]
        prob.material[lo[2]:lo[2] + side[2], lo[1]:lo[1] + side[1], lo[0]:lo[0] + side[0]] = PEC
    return prob


def config5(n_requests: int = 512, mean_interarrival_s: float = 0.0,
            seed_index: int = 5) -> list[Request]:
    """Serving stream: cubes of 8^3..50^3 nodes (log-uniform), 1-6 GHz with
    h = lambda/10, a random PEC box, 1-16 plane waves, Poisson arrivals (all at
    t = 0 when mean_interarrival_s is 0)."""
    rng = rng_for(seed_index)
    out = []
    t = 0.0
    for q in range(n_requests):
        n_nodes = int(round(np.exp(rng.uniform(np.log(8), np.log(50)))))
        f = float(rng.uniform(1e9, 6e9))
        prob = pec_box_problem(n_nodes - 1, f, rng, name=f"req{q}")
        waves = random_waves(int(rng.integers(1, 17)), rng)
        if mean_interarrival_s > 0:
            t += float(rng.exponential(mean_interarrival_s))
        out.append(Request(t, prob, waves))
    return out


def mirror_part(prob: VoxelProblem, x_kind: int = 0, y_kind: int = 0) -> VoxelProblem:
    """The +x half (x_kind != 0) and/or +y half (y_kind != 0) of a problem
    that is mirror-symmetric about its mid planes, with those planes turned
    into symmetry (1) or antisymmetry (2) faces.  The element counts along the
    cut axes must be even, so that each plane passes through grid nodes."""
    mat = np.asarray(prob.material)
    nx, ny = prob.nx, prob.ny
    x0 = nx // 2 if x_kind else 0
    y0 = ny // 2 if y_kind else 0
    if (x_kind and nx % 2) or (y_kind and ny % 2):
        raise ValueError("the cut axes need an even element count")
    bnd = list(prob.boundary)
    if x_kind:
        bnd[0] = x_kind
    if y_kind:
        bnd[2] = y_kind
    origin = (prob.origin[0] + x0 * prob.h[0], prob.origin[1] + y0 * prob.h[1], prob.origin[2])
    return VoxelProblem(nx - x0, ny - y0, prob.nz, prob.h, origin,
                        np.ascontiguousarray(mat[:, y0:, x0:]), prob.eps_r, prob.mu_r, prob.freq_hz,
                        name=f"{prob.name}_part", boundary=tuple(bnd))


def config2_quarter() -> tuple[VoxelProblem, PlaneWaves]:
    """The +x, +y quarter of the 3-wavelength cube: with H along x at normal
    incidence the x = mid plane is an antisymmetry plane (n x H = 0) and the
    y = mid plane a symmetry plane (n . H = 0); the centred PEC cube and the
    centred slab keep the problem mirror-symmetric about both."""
    prob, waves = config2()
    return mirror_part(prob, x_kind=2, y_kind=1), waves


def random_small_grid(seed: int, n_max: int = 6, n_pec_boxes: int = 2,
                      freq_hz: float = 3e9, dielectric: bool = True) -> VoxelProblem:
    """Small box (2..n_max elements per axis, possibly anisotropic spacing) with
    random PEC boxes and an optional lossy dielectric; used for integer-map and
    value parity on tiny inputs."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = (int(v) for v in rng.integers(2, n_max + 1, 3))
    lam = wavelength(freq_hz)
    h = tuple(float(lam / 10 * rng.uniform(0.7, 1.3)) for _ in range(3))
    mat = np.zeros((nz, ny, nx), dtype=np.uint8)
    if dielectric and nx > 2 and ny > 2 and nz > 2:
        mat[1:-1, 1:-1, 1:-1][rng.random((nz - 2, ny - 2, nx - 2)) < 0.3] = 1
    for _ in range(n_pec_boxes):
        if min(nx, ny, nz) <= 2:
            break
        lo = [int(rng.integers(1, d - 1)) for d in (nx, ny, nz)]
        hi = [int(rng.integers(l + 1, d)) for l, d in zip(lo, (nx, ny, nz))]
        mat[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = PEC
    eps = np.array([1.0 + 0j, 2.5 - 0.4j])
    mu = np.array([1.0 + 0j, 1.2 - 0.1j])
    origin = tuple(float(v) for v in rng.uniform(-0.05, 0.05, 3))
    return VoxelProblem(nx, ny, nz, h, origin, mat, eps, mu, freq_hz, name=f"rand{seed}")


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4}
