"""Correction nodes N_h(y_i) and weights omega^{(ij)} (Sec. 2.4).

For the target node y_i with surface point x* = P_i and unit normal n:
  * dominant axis a = argmax_j |n_j| (ties: lowest index; Sec. 2.4);
  * Q permutes the axes so that a comes last, the other two (b, c) first in
    ascending order; tilde coordinates are (x_b, x_c, x_a);
  * grid planes t_k = origin_a + h k along a; the singular line of Eq. (2.19)
    meets plane t_k at x* + eta_k n with eta_k = (t_k - x*_a)/n_a, and
    eta_k is the signed distance of that point (Sec. 2.4.1, eta(t));
  * in-plane: u0 = (x*_b + eta_k n_b, x*_c + eta_k n_c) = u_h + h(alpha, beta),
    u_h the nearest grid node, (alpha, beta) in [-1/2, 1/2)^2 (Sec. 2.4),
    computed as s = (u0 - origin)/h, k = floor(s + 1/2), alpha = s - k;
  * planes with |eta_k| <= eps + h are visited; the node (u_h, t_k) is a
    correction node when it is a tube node (other nodes carry no weight);
  * expansions, Eq. (2.28) of the theorem in Sec. 2.4.1, with
    D0 = (I - eta_k M)^{-1}, A the 2x2 block of the rows Q tau_1, Q tau_2
    (Eq. (2.26)), v(theta) = D0 A (cos theta, sin theta):
        l11 = (1 - eps_E/eps_I) v^T M v / (8 pi |v|^3)
        l22 = (1 - eps_I/eps_E) v^T M v / (8 pi |v|^3)
        l21 = kappa^2 / (8 pi |v|)          (reading: the printed s0^(21) lacks
                                              the factor kappa^2; K21 ~ kappa^2/(8 pi r))
        s1^(12) = kappa / (4 pi),  omega[1; alpha, beta] = 1  ->  omega12 = kappa/(4 pi)
  * omega[l; alpha, beta] = a_0 T^c_0 + sum_k (a_k T^c_k + b_k T^s_k) with the
    Fourier coefficients of l from an FFT of 4N equispaced samples, and the
    tabulated T interpolated on the (alpha_m, beta_n) stencil (Sec. 2.4.2).

K-reg rows (Sec. 2.3) for the targets the hybrid classification marks bad
(Sec. 3.2, HYB-IBIM): the kernel is replaced by the constant C in the
tangent-plane disc |x - y|_P < tau, tau = 2h, where |x - y|_P is the distance
between the projections of the grid node y and of x onto the tangent plane at
P(x): the correction set is every tube node in that cylinder, with
C11 = C21 = C22 = 0 and C12 = (e^{-kappa tau} - 1 + kappa tau) / (2 pi kappa tau^2)
(kappa -> 0: kappa/(4 pi)).  Membership: v = y - P, s = (v0 n0 + v1 n1) + v2 n2,
t_c = v_c - s n_c, (t0 t0 + t1 t1) + t2 t2 < tau^2, unfused FP64.  Entries in
ascending node order.

Parity status: pinned through the operator identities on the sphere
(double layer, consistency with the exact solution), the plane rule, and the
K-reg constant against a disc-average quadrature.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import tables as tb
from .geometry import TubeGeometry

N_SAMPLES = 4 * tb.N_MODES     # FFT samples of l(theta), 4N (Sec. 2.4.2)


@dataclasses.dataclass
class Correction:
    ptr: np.ndarray        # (M+1,) CSR row pointer by target
    node: np.ndarray       # (E,) correction node ids
    alpha: np.ndarray      # (E,)
    beta: np.ndarray       # (E,)
    eta: np.ndarray        # (E,)
    axis: np.ndarray       # (M,) dominant axis per target
    omega_A: np.ndarray    # (E,) omega[v^T M v / (8 pi |v|^3)]  (0 in K-reg rows)
    omega_B: np.ndarray    # (E,) omega[1 / (8 pi |v|)]          (0 in K-reg rows)
    kreg: np.ndarray       # (E,) bool: entry of a K-reg row

    def excl_csr(self):
        """Sorted correction node ids per target (the pairs the dense sum omits)."""
        M = self.ptr.size - 1
        idx = np.empty_like(self.node)
        for i in range(M):
            s, e = self.ptr[i], self.ptr[i + 1]
            idx[s:e] = np.sort(self.node[s:e])
        return self.ptr.copy(), idx


def dominant_axis(n: np.ndarray) -> np.ndarray:
    return np.argmax(np.abs(n), axis=1)


def kreg_constant(kappa: float, tau: float) -> float:
    """C12 of Sec. 2.3: the tangent-disc average of (G0 - Gk)."""
    if kappa == 0.0:
        return 0.0
    return (math.exp(-kappa * tau) - 1.0 + kappa * tau) / (2.0 * math.pi * kappa * tau * tau)


def kreg_nodes(geo: TubeGeometry, i: int, tau: float):
    """Tube nodes in the tangent-plane cylinder of radius tau around target i (ascending ids)."""
    h = geo.h
    nx, ny, nz = geo.grid_n
    K = int(math.ceil((geo.eps + tau) / h)) + 1
    r = np.arange(-K, K + 1)
    dk, dj, di = np.meshgrid(r, r, r, indexing="ij")          # k slowest: ascending grid index
    q = geo.ijk[i, 0] + di.ravel()
    j = geo.ijk[i, 1] + dj.ravel()
    k = geo.ijk[i, 2] + dk.ravel()
    ok = (q >= 0) & (q < nx) & (j >= 0) & (j < ny) & (k >= 0) & (k < nz)
    m = geo.node_of[(q + nx * (j + ny * k))[ok]]
    m = m[m >= 0]
    P = geo.P[i]
    n = geo.n[i]
    v0 = geo.y[m, 0] - P[0]
    v1 = geo.y[m, 1] - P[1]
    v2 = geo.y[m, 2] - P[2]
    s = (v0 * n[0] + v1 * n[1]) + v2 * n[2]
    t0 = v0 - s * n[0]
    t1 = v1 - s * n[1]
    t2 = v2 - s * n[2]
    inside = (t0 * t0 + t1 * t1) + t2 * t2 < tau * tau
    return [int(v) for v in m[inside]]


def correction_nodes(geo: TubeGeometry, targets=None):
    """(target, node, alpha, beta, eta, kreg) entries, targets ascending, planes ascending.

    `targets`: optional subset of target rows (default: all tube nodes).
    Bad targets get their K-reg cylinder instead (alpha = beta = eta = 0, kreg = 1).
    """
    h, eps = geo.h, geo.eps
    nx, ny, nz = geo.grid_n
    dims = (nx, ny, nz)
    origin = geo.origin
    K = int(math.ceil(2.0 * eps / h)) + 2
    ax = dominant_axis(geo.n)
    rows = []
    tau = 2.0 * h
    for i in (range(geo.M) if targets is None else sorted(int(t) for t in targets)):
        if geo.bad[i]:
            for m in kreg_nodes(geo, i, tau):
                rows.append((i, m, 0.0, 0.0, 0.0, 1.0))
            continue
        a = int(ax[i])
        b, c = [v for v in range(3) if v != a]
        Pa, Pb, Pc = geo.P[i, a], geo.P[i, b], geo.P[i, c]
        na, nb, nc = geo.n[i, a], geo.n[i, b], geo.n[i, c]
        ia = int(geo.ijk[i, a])
        for ka in range(ia - K, ia + K + 1):
            t = origin[a] + h * float(ka)
            eta = (t - Pa) / na
            if abs(eta) > eps + h:
                continue
            u0b = Pb + eta * nb
            u0c = Pc + eta * nc
            sb = (u0b - origin[b]) / h
            sc = (u0c - origin[c]) / h
            kb = math.floor(sb + 0.5)
            kc = math.floor(sc + 0.5)
            alpha = sb - kb
            beta = sc - kc
            idx = [0, 0, 0]
            idx[a], idx[b], idx[c] = ka, kb, kc
            if not (0 <= idx[0] < dims[0] and 0 <= idx[1] < dims[1] and 0 <= idx[2] < dims[2]):
                continue
            m = int(geo.node_of[idx[0] + nx * (idx[1] + ny * idx[2])])
            if m < 0:
                continue
            rows.append((i, m, alpha, beta, eta, 0.0))
    arr = np.array(rows, dtype=np.float64) if rows else np.zeros((0, 6))
    return arr, ax


def angular_functions(geo: TubeGeometry, tgt: np.ndarray, ax: np.ndarray, eta: np.ndarray):
    """Samples of v^T M v/(8 pi |v|^3) and 1/(8 pi |v|) at theta_j = 2 pi j / L."""
    L = N_SAMPLES
    theta = 2.0 * np.pi * np.arange(L) / L
    ct, st = np.cos(theta), np.sin(theta)
    perm = np.array([[1, 2, 0], [0, 2, 1], [0, 1, 2]])   # (b, c, a) for a = 0, 1, 2
    p = perm[ax[tgt]]                                       # (E, 3)
    tau = geo.tau[tgt]                                      # (E, 2, 3)
    Qt = np.take_along_axis(tau, p[:, None, :], axis=2)     # (E, 2, 3) rows Q tau_1, Q tau_2
    A = Qt[:, :, :2]                                        # (E, 2, 2)
    Mdiag = -geo.kappa_s[tgt]                               # (E, 2)
    D0 = 1.0 / (1.0 - eta[:, None] * Mdiag)                 # (I - eta M)^{-1}
    v1 = D0[:, 0:1] * (A[:, 0, 0:1] * ct[None, :] + A[:, 0, 1:2] * st[None, :])
    v2 = D0[:, 1:2] * (A[:, 1, 0:1] * ct[None, :] + A[:, 1, 1:2] * st[None, :])
    vMv = Mdiag[:, 0:1] * v1 * v1 + Mdiag[:, 1:2] * v2 * v2
    vn = np.sqrt(v1 * v1 + v2 * v2)
    lA = vMv / (8.0 * np.pi * vn ** 3)
    lB = 1.0 / (8.0 * np.pi * vn)
    return lA, lB


def fourier_coefficients(samples: np.ndarray):
    """a_k, b_k (k = 0..N) of l(theta) = a_0 + sum_k a_k cos k theta + b_k sin k theta, by FFT."""
    L = samples.shape[1]
    c = np.fft.rfft(samples, axis=1) / L
    N = tb.N_MODES
    a = np.empty((samples.shape[0], N + 1))
    b = np.zeros((samples.shape[0], N + 1))
    a[:, 0] = c[:, 0].real
    a[:, 1:] = 2.0 * c[:, 1:N + 1].real
    b[:, 1:] = -2.0 * c[:, 1:N + 1].imag
    return a, b


def interpolated_tables(T: np.ndarray, alpha: np.ndarray, beta: np.ndarray, chunk: int = 8192) -> np.ndarray:
    """Tabulated weights interpolated at every (alpha, beta): [E, 2, n_modes].

    Same arithmetic as tables.interpolate, for many shifts at once.
    """
    E = alpha.size
    out = np.empty((E, 2, len(tb.MODES)))
    six = np.arange(6)
    for s in range(0, E, chunk):
        a = alpha[s:s + chunk]
        b = beta[s:s + chunk]
        ia = np.floor(a / tb.SPACING).astype(np.int64) - 2
        ib = np.floor(b / tb.SPACING).astype(np.int64) - 2
        xa = (ia[:, None] + six[None, :]) * tb.SPACING
        xb = (ib[:, None] + six[None, :]) * tb.SPACING
        ca = np.ones((a.size, 6))
        cb = np.ones((a.size, 6))
        for m in range(6):
            for l in range(6):
                if l != m:
                    ca[:, m] *= (a - xa[:, l]) / (xa[:, m] - xa[:, l])
                    cb[:, m] *= (b - xb[:, l]) / (xb[:, m] - xb[:, l])
        IA = ia[:, None, None] + tb.HALF + six[None, :, None]
        IB = ib[:, None, None] + tb.HALF + six[None, None, :]
        blk = T[:, :, IA, IB]                                  # [2, modes, e, 6, 6]
        out[s:s + chunk] = np.einsum("kmeab,ea,eb->ekm", blk, ca, cb)
    return out


def weights_from_coefficients(a: np.ndarray, b: np.ndarray, Tint: np.ndarray) -> np.ndarray:
    """omega = a_0 T^c_0 + sum_{k in MODES, k>0} (a_k T^c_k + b_k T^s_k)  (Sec. 2.4.2)."""
    modes = np.array(tb.MODES)
    return np.sum(a[:, modes] * Tint[:, 0, :] + b[:, modes] * Tint[:, 1, :], axis=1)


def build_correction(geo: TubeGeometry, T: np.ndarray, targets=None) -> Correction:
    arr, ax = correction_nodes(geo, targets)
    tgt = arr[:, 0].astype(np.int64)
    node = arr[:, 1].astype(np.int64)
    alpha, beta, eta = arr[:, 2], arr[:, 3], arr[:, 4]
    kreg = arr[:, 5] != 0.0
    omA = np.zeros(tgt.size)
    omB = np.zeros(tgt.size)
    c = ~kreg
    if np.any(c):
        lA, lB = angular_functions(geo, tgt[c], ax, eta[c])
        aA, bA = fourier_coefficients(lA)
        aB, bB = fourier_coefficients(lB)
        Tint = interpolated_tables(T, alpha[c], beta[c])
        omA[c] = weights_from_coefficients(aA, bA, Tint)
        omB[c] = weights_from_coefficients(aB, bB, Tint)
    ptr = np.zeros(geo.M + 1, dtype=np.int64)
    np.add.at(ptr, tgt + 1, 1)
    ptr = np.cumsum(ptr)
    return Correction(ptr=ptr, node=node, alpha=alpha, beta=beta, eta=eta, axis=ax,
                      omega_A=omA, omega_B=omB, kreg=kreg)
