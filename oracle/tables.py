"""Correction-weight tables by the paper's limit definition (Sec. 2.4.2).

For a function s_q(y) = |y|^{q-1} l(y/|y|) the correction weight is the limit
Eq. (2.29):

    omega[s_q; alpha, beta] = lim_{h->0} omega_h,
    omega_h = h^{-(q+1)} ( int_{R^2} s_q g  -  T0_h[ s_q(. - (alpha,beta)h) g(. - (alpha,beta)h) ] )
              / g(-(alpha,beta)h),

T0_h the trapezoidal rule on hZ^2 with the node 0 omitted, g radial, compactly
supported, C-infinity, g(0) = 1.  The limit is approximated as in the remark
after Eq. (2.29): omega_{2^-n} with n the first j >= 1 where
|omega_{2^-j} - omega_{2^-j-1}| <= Tol.

Tabulated functions (Sec. 2.4.2): |y|^{-1} cos(k psi) and |y|^{-1} sin(k psi)
for the Fourier modes k, on a stencil grid of shifts (alpha_m, beta_n).  The
constant function (q = 1, the s_1 term of K12) needs omega[1; alpha, beta],
which the limit gives exactly as 1 (see `omega_one`).

Readings where the paper leaves a choice open (all stated here and in the
design notes):
  * g: flat-top, g = 1 on |y| <= 0.3, C-infinity transition to 0 at |y| = 1
    (radial, compact support, g(0) = 1 as required).  Because g is constant
    near the singularity the limit converges spectrally; int s g is exact:
    2 pi (1 + r0)/2 for k = 0 (the transition integrates to 1/2 by symmetry)
    and 0 for k > 0.
  * Tol = 1e-12 (the paper used 1e-8 for its figures; parity with the GPU
    path needs table values to ~1e-12).
  * Only even k: every kernel's angular function l is even, l(-y) = l(y), so
    odd Fourier coefficients vanish identically.
  * N = 16 modes, stencil grid spacing 1/32 on [-19/32, 19/32]^2, tensor
    Lagrange interpolation of degree 5 (6 x 6 stencil) around (alpha, beta).

Test infrastructure only: see the package docstring.

Parity status: pinned (the square-lattice constant omega[1/r] = -4 zeta(1/2) beta(1/2), the limit
against an independent Ewald-split evaluation, the table symmetries, omega[1] = 1, and the plane rule's
second-order convergence for a smooth test function).
"""
from __future__ import annotations

import os
import threading

import numpy as np

from . import native

N_MODES = 16                  # highest Fourier mode kept
MODES = tuple(range(0, N_MODES + 1, 2))
SPACING = 1.0 / 32.0          # stencil grid spacing of (alpha_m, beta_n)
HALF = 19                     # grid indices -HALF..HALF per axis (alpha may round to just below -1/2)
R0 = 0.3                      # flat-top radius of g
TOL = 1e-12
JMAX = 12

_cache_lock = threading.Lock()
_cache = {}


def cutoff_g(r: float) -> float:
    return float(native.lib().oracle_cutoff_g(float(r), R0))


def integral_s_g(k: int) -> float:
    """int_{R^2} |y|^{-1} e^{i k psi} g(|y|) dy  (real; zero unless k = 0)."""
    if k != 0:
        return 0.0
    # 2 pi int_0^1 g(r) dr = 2 pi (r0 + (1 - r0)/2): S(t) + S(1 - t) = 1.
    return 2.0 * np.pi * (R0 + 0.5 * (1.0 - R0))


def omega_h(alpha: np.ndarray, beta: np.ndarray, h: float, kmax: int, kstep: int = 2):
    """omega_h of Eq. (2.29) for the harmonics k = 0, kstep, ..., kmax at many shifts.

    Returns complex array [n_pts, kmax/kstep+1]: real part = cos k psi weight,
    imaginary part = sin k psi weight.
    """
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    n = alpha.size
    nk = kmax // kstep + 1
    re = np.zeros((n, nk))
    im = np.zeros((n, nk))
    native.lib().oracle_punctured_lattice_many(n, native.dptr(alpha), native.dptr(beta), float(h), R0,
                                               int(kmax), int(kstep), native.dptr(re), native.dptr(im))
    T0 = re + 1j * im
    I = np.array([integral_s_g(q * kstep) for q in range(nk)])
    gnode = np.array([cutoff_g(h * np.hypot(a, b)) for a, b in zip(alpha, beta)])
    return (I[None, :] - T0) / h / gnode[:, None]


def omega_limit(alpha, beta, kmax: int = N_MODES, tol: float = TOL, jmax: int = JMAX, kstep: int = 2):
    """Limit of Eq. (2.29) by the stopping rule of the remark after it.

    Each (alpha, beta) point and each harmonic stops at its own n; returns
    (omega [n_pts, kmax/kstep+1] complex, n_used of the same shape), column q
    holding harmonic k = q * kstep.
    """
    alpha = np.atleast_1d(np.asarray(alpha, dtype=np.float64))
    beta = np.atleast_1d(np.asarray(beta, dtype=np.float64))
    prev = omega_h(alpha, beta, 0.5, kmax, kstep)
    result = np.full(prev.shape, np.nan + 0j)
    n_used = np.zeros(prev.shape, dtype=np.int64)
    done = np.zeros(prev.shape, dtype=bool)
    for j in range(1, jmax):
        cur = omega_h(alpha, beta, 2.0 ** (-(j + 1)), kmax, kstep)
        diff = np.abs(cur - prev)
        newly = (~done) & (diff <= tol)
        result[newly] = prev[newly]
        n_used[newly] = j
        done |= newly
        if done.all():
            break
        prev = cur
    if not done.all():
        raise RuntimeError("weight limit did not reach the tolerance")
    return result, n_used


def omega_one(alpha: float, beta: float, h: float) -> float:
    """omega_h[1; alpha, beta] of Eq. (2.29) with q = 1 (the s_1 term of K12).

    int g - h^2 sum_{n != 0} g(h n - h(alpha,beta)) = h^2 g(-h(alpha,beta)) up to
    the trapezoidal rule's spectral error for smooth compactly supported g,
    so omega[1; alpha, beta] = 1.  Computed here by the definition for tests.
    """
    R = int(np.ceil(1.0 / h)) + 2
    n = np.arange(-R, R + 1)
    X, Y = np.meshgrid(h * n - h * alpha, h * n - h * beta, indexing="ij")
    r = np.hypot(X, Y).ravel()
    mask = np.ones(r.shape, bool)
    mask[(R * (2 * R + 1)) + R] = False
    g = np.array([cutoff_g(v) for v in r[mask]])
    # int_{R^2} g = 2 pi int_0^1 g(r) r dr, by Gauss-Legendre on each smooth piece
    xg, wg = np.polynomial.legendre.leggauss(200)
    rr = 0.5 * R0 * (xg + 1)
    I = np.sum(0.5 * R0 * wg * rr)
    rr2 = R0 + 0.5 * (1 - R0) * (xg + 1)
    I += np.sum(0.5 * (1 - R0) * wg * rr2 * np.array([cutoff_g(v) for v in rr2]))
    I *= 2 * np.pi
    return float((I - h * h * np.sum(g)) / h ** 2 / cutoff_g(h * np.hypot(alpha, beta)))


def grid_points():
    idx = np.arange(-HALF, HALF + 1)
    return idx * SPACING


def build_tables(cache_dir: str | None = None):
    """Tables T[kind][mode_index, ia, ib] on the stencil grid, by the limit.

    kind 0: |y|^-1 cos(k psi), kind 1: |y|^-1 sin(k psi), k in MODES.
    Cached in memory and (optionally) in `cache_dir` as .npy.
    """
    key = (N_MODES, SPACING, HALF, R0, TOL)
    with _cache_lock:
        if key in _cache:
            return _cache[key]
    path = None
    if cache_dir:
        os.makedirs(cache_dir, exist_ok=True)
        path = os.path.join(cache_dir, f"ctr_tables_N{N_MODES}_h{HALF}_tol{TOL:g}.npy")
        if os.path.exists(path):
            T = np.load(path)
            with _cache_lock:
                _cache[key] = T
            return T
    g = grid_points()
    A, B = np.meshgrid(g, g, indexing="ij")
    om, _ = omega_limit(A.ravel(), B.ravel(), kmax=N_MODES, kstep=2)
    n = g.size
    T = np.zeros((2, len(MODES), n, n))
    for mi, k in enumerate(MODES):
        T[0, mi] = om[:, k // 2].real.reshape(n, n)
        T[1, mi] = om[:, k // 2].imag.reshape(n, n)
    if path:
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "wb") as f:
            np.save(f, T)
        os.replace(tmp, path)
    with _cache_lock:
        _cache[key] = T
    return T


def lagrange_weights(x: float):
    """Degree-5 Lagrange basis on the 6 stencil nodes around x (Sec. 2.4.2, c_{m,n}).

    Returns (first grid index, weights[6]); nodes are (i0 + m) * SPACING.
    """
    f = int(np.floor(x / SPACING))
    i0 = f - 2
    nodes = (i0 + np.arange(6)) * SPACING
    c = np.ones(6)
    for m in range(6):
        for l in range(6):
            if l != m:
                c[m] *= (x - nodes[l]) / (nodes[m] - nodes[l])
    return i0, c


def interpolate(T: np.ndarray, alpha: float, beta: float) -> np.ndarray:
    """omega at (alpha, beta) for every tabulated function: sum c_m(alpha) c_n(beta) T(alpha_m, beta_n).

    Returns [2, n_modes] (cos kind, sin kind).
    """
    ia, ca = lagrange_weights(alpha)
    ib, cb = lagrange_weights(beta)
    sa = slice(ia + HALF, ia + HALF + 6)
    sb = slice(ib + HALF, ib + HALF + 6)
    if ia + HALF < 0 or ib + HALF < 0 or ia + HALF + 6 > T.shape[2] or ib + HALF + 6 > T.shape[3]:
        raise ValueError("shift outside the tabulated range")
    blk = T[:, :, sa, sb]
    return np.einsum("kmab,a,b->km", blk, ca, cb)
