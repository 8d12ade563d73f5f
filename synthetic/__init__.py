"""Seeded synthetic inputs for CTR-IBIM: signed-distance grids, charges, densities.

This module is shared by the oracle, the tests and the benchmark.  It holds
none of the method's arithmetic (no kernels, no quadrature, no weights): it
only produces the data a user of the method supplies, i.e. a signed distance
to the molecular surface sampled on a uniform Cartesian grid (Sec. 2.1, the
signed distance and closest-point projection), point charges (Eq. 1.1), the
dielectric constants and the screening parameter.

Conventions (shared with the C ABI):
  * grid node (i, j, k) sits at origin + h * (i, j, k); arrays are flat with
    x fastest, i.e. linear index i + nx * (j + ny * k);
  * the signed distance is positive OUTSIDE the molecule (the paper's Sec. 2.1
    uses the opposite sign; only the sign of d flips, P and the outward normal
    are unchanged).

Workloads (sizes and distributions follow the paper's test problems; the
paper's molecular data are not available, so seeded stand-ins are used):
  * sphere of radius 2 around one central unit charge (Sec. 2.6 sphere test,
    Kirkwood closed form);
  * ellipsoid with semi-axes (4, 3, 2) and three seeded charges;
  * a seeded random-walk molecule with a probe-1.4 solvent-excluded surface
    (Sec. 3.1 SES recipe: probe-accessible region, cavity removal, distance).
"""
from __future__ import annotations

import dataclasses
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

__all__ = [
    "Grid", "Problem", "sphere_problem", "ellipsoid_problem", "molecule_problem",
    "random_density", "sphere_sdist", "ellipsoid_sdist", "ellipsoid_area",
    "random_walk_molecule", "ses_sdist", "box_grid",
]

EPS_IN = 1.0        # dielectric constant inside (Sec. 2.6)
EPS_OUT = 80.0      # dielectric constant outside (Sec. 2.6)
KAPPA = 0.1257      # screening parameter, 1/Angstrom


@dataclasses.dataclass(frozen=True)
class Grid:
    n: tuple            # (nx, ny, nz)
    origin: tuple       # (x0, y0, z0)
    h: float

    @property
    def size(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    def axes(self):
        return [self.origin[c] + self.h * np.arange(self.n[c], dtype=np.float64) for c in range(3)]

    def points(self):
        """Node coordinates as three flat arrays (x fastest)."""
        x, y, z = self.axes()
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return X.ravel(), Y.ravel(), Z.ravel()


@dataclasses.dataclass
class Problem:
    name: str
    grid: Grid
    sdist: np.ndarray            # flat float64, size grid.size, d > 0 outside
    charge_xyz: np.ndarray       # (Nc, 3) float64
    charge_q: np.ndarray         # (Nc,) float64
    eps_in: float = EPS_IN
    eps_out: float = EPS_OUT
    kappa: float = KAPPA
    tube: float = 0.0            # tube half-width epsilon
    info: dict = dataclasses.field(default_factory=dict)


def box_grid(lo, hi, h, center_on_origin=True) -> Grid:
    """Smallest grid of spacing h covering [lo, hi] per axis.

    With center_on_origin the node set contains the origin and is symmetric.
    """
    n, origin = [], []
    for c in range(3):
        if center_on_origin:
            half = int(math.ceil(max(abs(lo[c]), abs(hi[c])) / h - 1e-12))
            n.append(2 * half + 1)
            origin.append(-half * h)
        else:
            i0 = int(math.floor(lo[c] / h))
            i1 = int(math.ceil(hi[c] / h))
            n.append(i1 - i0 + 1)
            origin.append(i0 * h)
    return Grid(tuple(n), tuple(origin), float(h))


# ---------------------------------------------------------------- sphere
def sphere_sdist(grid: Grid, R: float, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    X, Y, Z = grid.points()
    return np.sqrt((X - center[0]) ** 2 + (Y - center[1]) ** 2 + (Z - center[2]) ** 2) - R


def sphere_problem(h: float = 0.25, R: float = 2.0, half_box: float = 3.0, tube_mult: float = 2.0,
                   q: float = 1.0, kappa: float = KAPPA, eps_in: float = EPS_IN,
                   eps_out: float = EPS_OUT) -> Problem:
    """Sphere of radius R at the origin, one charge q at the centre (Sec. 2.6).

    Default: R = 2, grid [-3, 3]^3, h = 0.25 (25^3 nodes), tube 2h.
    """
    grid = box_grid((-half_box,) * 3, (half_box,) * 3, h)
    return Problem(
        name=f"sphere_R{R:g}_h{h:g}", grid=grid, sdist=sphere_sdist(grid, R),
        charge_xyz=np.zeros((1, 3)), charge_q=np.array([q], dtype=np.float64),
        eps_in=eps_in, eps_out=eps_out, kappa=kappa, tube=tube_mult * h,
        info={"R": R, "q": q})


def quadratic_sphere_problem(h: float = 0.1, R: float = 1.0, half_box: float = 1.9, tube: float = 0.65,
                             kappa: float = KAPPA) -> Problem:
    """Level-set function d = (|x|^2 - R^2) / (2R) (zero on the sphere of radius R, gradient |x|/R; not a
    distance).  Central differences are exact on a quadratic, so a node's finite-difference geometry is known
    in closed form: its level set is the sphere of radius r = |y|, curvature 1/r, and the surface curvature
    at its point P = y - d n is 1/(r - d).  The grid is offset by h/2 (an even node count per axis,
    symmetric about the origin), so no node sits at the centre, where the gradient vanishes.  One charge at
    (0.1, 0, 0)."""
    n = 2 * int(math.ceil(half_box / h))
    grid = Grid((n, n, n), (-(n - 1) * h / 2.0,) * 3, float(h))
    X, Y, Z = grid.points()
    sd = (X * X + Y * Y + Z * Z - R * R) / (2.0 * R)
    return Problem(name=f"quadsphere_R{R:g}_h{h:g}", grid=grid, sdist=sd, charge_xyz=np.array([[0.1, 0.0, 0.0]]),
                   charge_q=np.array([1.0]), kappa=kappa, tube=tube, info={"R": R})


def flat_cylinder_problem(h: float = 0.25, R: float = 1.5, c: float = 1.0, tube_mult: float = 2.0,
                          kappa: float = KAPPA) -> Problem:
    """A cylinder of radius R and height 2c with flat faces, d = max(|z| - c, rho - R) (rho = |(x, y)|): near
    the centre of a face the level sets are exact planes z = c + d.  One charge at the origin."""
    half = max(R, c) + tube_mult * h + 4 * h
    grid = box_grid((-half,) * 3, (half,) * 3, h)
    X, Y, Z = grid.points()
    sd = np.maximum(np.abs(Z) - c, np.sqrt(X * X + Y * Y) - R)
    return Problem(name=f"flatcyl_h{h:g}", grid=grid, sdist=sd, charge_xyz=np.zeros((1, 3)),
                   charge_q=np.array([1.0]), kappa=kappa, tube=tube_mult * h, info={"R": R, "c": c})


# ---------------------------------------------------------------- ellipsoid
def _ellipsoid_root(axes, y):
    """Closest point on an axis-aligned ellipsoid for points |y| (first octant).

    Solves sum_i (a_i y_i / (t + a_i^2))^2 = 1 for the Lagrange multiplier t by
    bisection (monotone in t on (-a_min^2, inf), a_min the smallest semi-axis
    with y_i != 0); exact up to rounding for points inside the reach.
    """
    a = np.asarray(axes, dtype=np.float64)
    a2 = a * a
    y = np.abs(y)
    nz = y > 0
    amin2 = np.min(np.where(nz, a2[None, :], np.inf), axis=1)
    amin2 = np.where(np.isfinite(amin2), amin2, a2.min())
    t_lo = -amin2
    t_hi = -amin2 + np.sqrt(np.sum(a2 * y * y, axis=1)) + 1e-300
    for _ in range(140):
        t = 0.5 * (t_lo + t_hi)
        with np.errstate(divide="ignore", invalid="ignore"):
            F = np.sum(np.where(nz, (a * y / (t[:, None] + a2)) ** 2, 0.0), axis=1) - 1.0
        pos = F > 0
        t_lo = np.where(pos, t, t_lo)
        t_hi = np.where(pos, t_hi, t)
    t = 0.5 * (t_lo + t_hi)
    x = a2 * y / (t[:, None] + a2)
    return x


def ellipsoid_sdist(grid: Grid, axes, band: float) -> np.ndarray:
    """Signed distance (positive outside) to the ellipsoid sum (x_i/a_i)^2 = 1.

    Exact (closest-point root solve) on nodes within `band` of the surface by
    a first-order estimate; elsewhere the first-order estimate, whose sign is
    exact (those nodes are never tube nodes nor in a tube node's stencil).
    """
    a = np.asarray(axes, dtype=np.float64)
    X, Y, Z = grid.points()
    P = np.stack([X, Y, Z], axis=1)
    F = np.sum((P / a) ** 2, axis=1) - 1.0
    gradn = 2.0 * np.sqrt(np.sum((P / (a * a)) ** 2, axis=1))
    est = np.where(gradn > 0, F / np.maximum(gradn, 1e-300), -a.min())
    out = est.copy()
    sel = np.abs(est) < band
    Ps = P[sel]
    # the root solve is elementwise: chunks on a thread pool (numpy releases the GIL) give the same bits
    chunk = 65536
    starts = range(0, Ps.shape[0], chunk)
    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        parts = list(ex.map(lambda i: _ellipsoid_root(a, Ps[i:i + chunk]), starts))
    xc = np.concatenate(parts) if parts else np.zeros((0, 3))
    dist = np.sqrt(np.sum((np.abs(Ps) - xc) ** 2, axis=1))
    sign = np.where(F[sel] > 0, 1.0, -1.0)
    out[sel] = sign * dist
    return out


def ellipsoid_area(axes, n: int = 4000) -> float:
    """Surface area by Gauss-Legendre quadrature of the exact parametric area element."""
    a, b, c = [float(v) for v in axes]
    u, wu = np.polynomial.legendre.leggauss(n)           # cos(theta) in [-1, 1]
    ph = (np.arange(2 * n) + 0.5) * (2 * np.pi / (2 * n))  # periodic: midpoint rule
    wp = 2 * np.pi / (2 * n)
    ct = u[:, None]
    st = np.sqrt(1 - ct * ct)
    cp, sp = np.cos(ph)[None, :], np.sin(ph)[None, :]
    # |r_theta x r_phi| / sin(theta), r = (a st cp, b st sp, c ct)
    nx = b * c * st * cp
    ny = a * c * st * sp
    nz = a * b * ct
    dA = np.sqrt(nx * nx + ny * ny + nz * nz)
    return float(np.sum(wu[:, None] * dA) * wp)


def ellipsoid_problem(h: float = 0.2, axes=(4.0, 3.0, 2.0), n_charges: int = 3, seed: int = 0,
                      tube_mult: float = 2.0, kappa: float = KAPPA) -> Problem:
    """Ellipsoid (4, 3, 2) with three seeded charges inside the 0.6-scaled ellipsoid.

    Charges: rejection sampling (numpy PCG64, `seed`), values uniform in [-1, 1].
    Grid: box [-(a_i + eps + 3h), a_i + eps + 3h] snapped to h, node at the origin.
    """
    eps = tube_mult * h
    a = np.asarray(axes, dtype=np.float64)
    ext = a + eps + 3 * h
    grid = box_grid(-ext, ext, h)
    sd = ellipsoid_sdist(grid, a, band=eps + 8 * h)
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = []
    while len(pts) < n_charges:
        p = rng.uniform(-1.0, 1.0, size=3) * a * 0.6
        if np.sum((p / (0.6 * a)) ** 2) <= 1.0:
            pts.append(p)
    q = rng.uniform(-1.0, 1.0, size=n_charges)
    return Problem(name=f"ellipsoid_{a[0]:g}x{a[1]:g}x{a[2]:g}_h{h:g}", grid=grid, sdist=sd,
                   charge_xyz=np.array(pts, dtype=np.float64), charge_q=q.astype(np.float64),
                   kappa=kappa, tube=eps, info={"axes": tuple(float(v) for v in a), "seed": seed})


# ---------------------------------------------------------------- molecule (SES)
_RADII = np.array([1.2, 1.5, 1.6, 1.7, 1.8])


def random_walk_molecule(n_atoms: int, seed: int, step: float = 1.5, min_sep: float = 2.0,
                         retries: int = 100):
    """Seeded self-avoiding random walk: atom centres, radii, partial charges.

    A step of length `step` in a uniformly random direction is rejected when it
    lands closer than `min_sep` to any non-adjacent atom; after `retries`
    rejections the walk backtracks one atom.  Radii are uniform over
    {1.2, 1.5, 1.6, 1.7, 1.8}; charges N(0, 0.4) shifted so the net charge is
    the nearest integer.  Centres are translated so their centroid is 0.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = [np.zeros(3)]
    fails = 0
    while len(pos) < n_atoms:
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        cand = pos[-1] + step * v
        P = np.array(pos[:-1]) if len(pos) > 1 else np.zeros((0, 3))
        ok = True
        if len(P):
            ok = np.min(np.sum((P - cand) ** 2, axis=1)) >= min_sep * min_sep
        if ok:
            pos.append(cand)
            fails = 0
        else:
            fails += 1
            if fails >= retries and len(pos) > 1:
                pos.pop()
                fails = 0
    xyz = np.array(pos, dtype=np.float64)
    xyz -= xyz.mean(axis=0)
    radii = _RADII[rng.integers(0, len(_RADII), size=n_atoms)].astype(np.float64)
    q = rng.normal(0.0, 0.4, size=n_atoms)
    q -= (q.sum() - np.round(q.sum())) / n_atoms
    return xyz, radii, q


def _flood_outside(mask_free: np.ndarray) -> np.ndarray:
    """Cells of `mask_free` (3-D bool) connected to the box boundary (6-connectivity)."""
    from scipy import ndimage
    lab, _ = ndimage.label(mask_free)
    border = np.unique(np.concatenate([
        lab[0].ravel(), lab[-1].ravel(), lab[:, 0].ravel(), lab[:, -1].ravel(),
        lab[:, :, 0].ravel(), lab[:, :, -1].ravel()]))
    border = border[border > 0]
    return np.isin(lab, border)


def ses_sdist(grid: Grid, xyz, radii, probe: float = 1.4, band: float = 3.0) -> np.ndarray:
    """Signed distance (positive outside) to the solvent-excluded surface.

    The probe-accessible region E is the complement of the union of balls
    B(z_k, r_k + probe), restricted to its component connected to the box
    boundary (cavity removal, Sec. 3.1 step 3).  Inside the molecule the SES
    distance is exactly dist(x, E) - probe; the distance to E is taken as the
    distance to the accessible part of the inflated spheres' union boundary,
    evaluated exactly against candidate spheres, circles and vertices near the
    node.  Outside, d = probe - dist(x, E) up to the probe radius and the
    distance to the van der Waals surface beyond (continuous, unit slope near
    the surface).  Nodes farther than `band` from the surface get a clamped
    value of the correct sign.
    """
    from synthetic._ses import ses_distance
    return ses_distance(grid, np.asarray(xyz, np.float64), np.asarray(radii, np.float64),
                        float(probe), float(band))


def molecule_problem(n_atoms: int = 500, seed: int = 0, h: float = 0.5, probe: float = 1.4,
                     tube_mult: float = 2.0, kappa: float = KAPPA) -> Problem:
    """Synthetic molecule: random-walk atoms, SES with probe 1.4, grid spacing h."""
    xyz, radii, q = random_walk_molecule(n_atoms, seed)
    eps = tube_mult * h
    pad = probe + eps + 4 * h
    lo = (xyz - radii[:, None]).min(axis=0) - pad
    hi = (xyz + radii[:, None]).max(axis=0) + pad
    grid = box_grid(lo, hi, h, center_on_origin=False)
    sd = ses_sdist(grid, xyz, radii, probe=probe, band=eps + 6 * h)
    return Problem(name=f"molecule_{n_atoms}_s{seed}_h{h:g}", grid=grid, sdist=sd,
                   charge_xyz=xyz, charge_q=q, kappa=kappa, tube=eps,
                   info={"n_atoms": n_atoms, "seed": seed, "probe": probe, "radii": radii})


# ---------------------------------------------------------------- convergence-study surfaces (Sec. 3.3.2)
TORUS_ANGLES = (1.99487, 2.54097947651017, 4.219760487439292)   # rotations about x, y, z (Sec. 3.3.2)


def torus_rotation(angles=TORUS_ANGLES) -> np.ndarray:
    """R = Rz(c) Ry(b) Rx(a): the body-frame torus (axis z) rotated about x, then y, then z."""
    a, b, c = angles
    Rx = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    Rz = np.array([[math.cos(c), -math.sin(c), 0], [math.sin(c), math.cos(c), 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def torus_sdist(grid: Grid, R1: float = 1.0, R2: float = 0.5, angles=TORUS_ANGLES) -> np.ndarray:
    """Exact signed distance to the rotated torus: sqrt((rho - R1)^2 + z^2) - R2 in the body frame."""
    X, Y, Z = grid.points()
    Rt = torus_rotation(angles).T
    xb = Rt[0, 0] * X + Rt[0, 1] * Y + Rt[0, 2] * Z
    yb = Rt[1, 0] * X + Rt[1, 1] * Y + Rt[1, 2] * Z
    zb = Rt[2, 0] * X + Rt[2, 1] * Y + Rt[2, 2] * Z
    return np.sqrt((np.sqrt(xb * xb + yb * yb) - R1) ** 2 + zb * zb) - R2


def torus_area(R1: float = 1.0, R2: float = 0.5) -> float:
    return 4.0 * math.pi ** 2 * R1 * R2


def torus_problem(h: float, R1: float = 1.0, R2: float = 0.5, q: float = 1.0, kappa: float = KAPPA,
                  tube_mult: float = 2.0) -> Problem:
    """The rotated torus of Sec. 3.3.2 (R1 = 1, R2 = 1/2), one charge q inside the tube at the body point
    (R1, 0, 0) (a charge at the origin, as printed, lies outside the torus), tube 2h."""
    eps = tube_mult * h
    half = R1 + R2 + eps + 3 * h
    grid = box_grid((-half,) * 3, (half,) * 3, h)
    z = torus_rotation() @ np.array([R1, 0.0, 0.0])
    return Problem(name=f"torus_h{h:g}", grid=grid, sdist=torus_sdist(grid, R1, R2),
                   charge_xyz=z.reshape(1, 3), charge_q=np.array([q]), kappa=kappa, tube=eps,
                   info={"R1": R1, "R2": R2, "area": torus_area(R1, R2)})


# ---------------------------------------------------------------- batches and request streams
def batch_specs(n: int, seed: int = 0, min_atoms: int = 20, max_atoms: int = 2000, spacings=(0.5, 0.35)):
    """Molecule specs of the batched workload: atom counts log-uniform in [min, max], h from `spacings`.

    Returns [(n_atoms, molecule seed, h)]; molecule k uses seed `seed + k`.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    atoms = np.rint(np.exp(rng.uniform(np.log(min_atoms), np.log(max_atoms), size=n))).astype(int)
    hs = rng.choice(np.asarray(spacings, dtype=np.float64), size=n)
    return [(int(a), int(seed + k), float(hh)) for k, (a, hh) in enumerate(zip(atoms, hs))]


def _molecule_from_spec(spec):
    n_atoms, seed, h = spec
    return molecule_problem(n_atoms=n_atoms, seed=seed, h=h)


def molecules_parallel(specs, workers: int | None = None):
    """Generate molecule problems in a spawn-started process pool (safe after CUDA initialisation)."""
    import multiprocessing as mp
    import os
    workers = workers or min(len(specs), os.cpu_count() or 1)
    if workers <= 1 or len(specs) <= 1:
        return [_molecule_from_spec(s) for s in specs]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_molecule_from_spec, specs, chunksize=1)


def request_stream(n: int, rate: float, seed: int = 0):
    """Poisson arrival times (seconds from 0) of n requests at `rate` per second, and pool indices."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    return np.cumsum(gaps) - gaps[0], rng


def sphere_with_nodes(target_M: int, h: float = 0.25, q: float = 1.0) -> Problem:
    """Sphere whose tube holds about target_M nodes (M ~ 4 pi R^2 * 2 eps / h^3 with eps = 2h)."""
    R = float(np.sqrt(target_M * h * h / (16.0 * np.pi)))
    return sphere_problem(h=h, R=R, half_box=R + 2 * h + 3 * h + h, q=q)


# ---------------------------------------------------------------- densities
def random_density(M: int, seed: int, smooth_points=None) -> np.ndarray:
    """Seeded test density p = (rho1, rho2), length 2M, values in [-1, 1].

    With `smooth_points` ((M, 3) node positions) the density is a smooth
    function of position plus noise, closer to a solution than white noise.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    p = rng.uniform(-1.0, 1.0, size=2 * M)
    if smooth_points is not None:
        X = np.asarray(smooth_points)
        k = rng.normal(size=(2, 3))
        p[:M] = 0.5 * np.cos(X @ k[0]) + 0.5 * p[:M]
        p[M:] = 0.5 * np.sin(X @ k[1]) + 0.5 * p[M:]
    return p
