"""Signed distance to a solvent-excluded surface (SES) on a grid (input generator only).

Atoms z_k with radii r_k, probe radius p.  U = union of the balls
B(z_k, R_k), R_k = r_k + p (the solvent-accessible region's complement);
E = the component of the complement of U that reaches the box boundary
(probe-centre positions; other components are cavities and are removed,
Sec. 3.1 step 3).  The SES is {x : dist(x, E) = p}, the molecule is
{dist(x, E) > p}, and with d > 0 outside:

  * x in E:                d(x) = p + dist(x, U) = p + min_k (|x - z_k| - R_k);
  * x in U or a cavity:    d(x) = p - dist(x, E) = p - dist(x, dE).

dist(x, dE) is evaluated exactly against the pieces of the boundary of the
union of balls: spherical faces (the projection of x onto sphere k, if it is
covered by no other ball), circular edges of intersecting sphere pairs (the
nearest point of the full circle, if uncovered) and vertices of sphere
triples (if uncovered); the nearest boundary point is always one of these.
Pieces that bound a cavity instead of E are dropped (the grid cells one to
three steps beyond the piece along its own outward direction are looked up in
the flood-filled grid).
Nodes farther than `band` from the SES get a clamped value of the right sign.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage
from scipy.spatial import cKDTree


def _flood_outside(conn: np.ndarray) -> np.ndarray:
    """Components of `conn` (26-connected) that touch the box boundary."""
    lab, _ = ndimage.label(conn, structure=np.ones((3, 3, 3), dtype=bool))
    border = np.unique(np.concatenate([lab[0].ravel(), lab[-1].ravel(), lab[:, 0].ravel(), lab[:, -1].ravel(),
                                       lab[:, :, 0].ravel(), lab[:, :, -1].ravel()]))
    border = border[border > 0]
    return np.isin(lab, border)


def _covered(points, centers, radii, tree, exclude, rmax, tol=1e-9):
    """Whether each point lies strictly inside a ball other than those listed in `exclude` (per point)."""
    out = np.zeros(len(points), dtype=bool)
    neigh = tree.query_ball_point(points, r=rmax)
    for i, nb in enumerate(neigh):
        if not nb:
            continue
        nb = np.asarray(nb)
        nb = nb[~np.isin(nb, exclude[i])]
        if nb.size:
            d2 = np.sum((centers[nb] - points[i]) ** 2, axis=1)
            out[i] = np.any(d2 < (radii[nb] - tol) ** 2)
    return out


def _boundary_pieces(z, R):
    """Uncovered circles (center, normal, radius, pair) and vertices (point, triple) of the union of balls."""
    tree = cKDTree(z)
    rmax = R.max()
    pairs = np.array(sorted(tree.query_pairs(r=2 * rmax)), dtype=np.int64).reshape(-1, 2)
    circles = []
    if pairs.size:
        a, b = pairs[:, 0], pairs[:, 1]
        dvec = z[b] - z[a]
        dist = np.linalg.norm(dvec, axis=1)
        ok = (dist < R[a] + R[b]) & (dist > np.abs(R[a] - R[b])) & (dist > 0)
        a, b, dvec, dist = a[ok], b[ok], dvec[ok], dist[ok]
        u = dvec / dist[:, None]
        t = (dist ** 2 + R[a] ** 2 - R[b] ** 2) / (2 * dist)
        rho = np.sqrt(np.maximum(R[a] ** 2 - t ** 2, 0.0))
        cen = z[a] + t[:, None] * u
        circles = (cen, u, rho, np.stack([a, b], axis=1))
    # vertices: triples of mutually intersecting spheres
    verts, vtrip = [], []
    if len(circles):
        cen, u, rho, ab = circles
        neigh = tree.query_ball_point(z, r=2 * rmax)
        nbset = [set(n) for n in neigh]
        for c in range(len(ab)):
            i, j = ab[c]
            for k in nbset[i] & nbset[j]:
                if k <= j:
                    continue
                # intersection of circle c with sphere k: points on the circle at distance R_k from z_k
                w = z[k] - cen[c]
                wn = w - np.dot(w, u[c]) * u[c]
                h_ax = np.dot(w, u[c])
                L = np.linalg.norm(wn)
                if L < 1e-12:
                    continue
                # |cen + rho (cos e1 + sin e2) - z_k|^2 = R_k^2, with e1 = wn/L
                val = (rho[c] ** 2 + L ** 2 + h_ax ** 2 - R[k] ** 2) / (2 * rho[c] * L)
                if rho[c] <= 0 or abs(val) > 1:
                    continue
                e1 = wn / L
                e2 = np.cross(u[c], e1)
                ang = np.arccos(val)
                for sgn in (1.0, -1.0):
                    p = cen[c] + rho[c] * (np.cos(ang) * e1 + sgn * np.sin(ang) * e2)
                    verts.append(p)
                    vtrip.append((i, j, k))
    verts = np.array(verts).reshape(-1, 3)
    vtrip = np.array(vtrip, dtype=np.int64).reshape(-1, 3)
    if verts.size:
        cov = _covered(verts, z, R, tree, [tuple(t) for t in vtrip], rmax)
        verts, vtrip = verts[~cov], vtrip[~cov]
    return tree, circles, verts, vtrip


def ses_distance(grid, z, r, probe, band):
    h = grid.h
    R = r + probe
    X, Y, Zc = grid.points()
    P = np.stack([X, Y, Zc], axis=1)
    tree, circles, verts, vtrip = _boundary_pieces(z, R)
    # distance to U (outside) and membership
    dmin = np.full(P.shape[0], np.inf)
    for s in range(0, P.shape[0], 200_000):
        Q = P[s:s + 200_000]
        dd, idx = tree.query(Q, k=min(16, len(z)))
        dd = np.atleast_2d(dd)
        idx = np.atleast_2d(idx)
        dmin[s:s + 200_000] = np.min(dd - R[idx], axis=1)
    shape = (grid.n[2], grid.n[1], grid.n[0])
    # E on the grid: every point of E lies within half a cell diagonal of a node with dmin >= -sqrt(3) h / 2,
    # and a path in E visits 26-adjacent such nodes, so the components of that set that reach the box boundary
    # hold all of E (walls thinner than sqrt(3) h merge a cavity into E).
    outer = _flood_outside((dmin >= -0.5 * np.sqrt(3.0) * h).reshape(shape)).ravel() & (dmin >= 0)
    d = np.empty(P.shape[0])
    big = band + 4 * h
    # x in E
    d[outer] = probe + dmin[outer]
    # x in U or in a cavity (filled, Sec. 3.1): p - dist(x, dE), needed only within the band
    inside = ~outer
    need = inside & (dmin > -(probe + big))
    d[inside & ~need] = -big
    idxs = np.nonzero(need)[0]
    origin = np.array(grid.origin)
    dims = np.array(grid.n)

    free_flat = (dmin >= 0)
    corners = np.array([(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)], dtype=np.int64)

    def outer_side(pts, u):
        """Whether the free space just beyond boundary points `pts` (outward unit directions `u`) is E.

        Steps h, 2h, 3h outward; at each step the 8 grid nodes of the enclosing cell are looked up and the
        first step that reaches a free (probe-centre) node decides: outer if any free node there is in E.
        A piece with no free node within 3h is kept (cavities that small do not occur at these spacings).
        """
        res = np.ones(len(pts), dtype=bool)
        open_ = np.ones(len(pts), dtype=bool)
        for step in (1.0, 2.0, 3.0):
            q = pts + (step * h) * u
            base = np.clip(np.floor((q - origin) / h).astype(np.int64), 0, dims - 2)
            any_free = np.zeros(len(pts), dtype=bool)
            any_outer = np.zeros(len(pts), dtype=bool)
            for c in corners:
                ijk = base + c
                lin = ijk[:, 0] + dims[0] * (ijk[:, 1] + dims[1] * ijk[:, 2])
                any_free |= free_flat[lin]
                any_outer |= outer[lin]
            decide = open_ & any_free
            res[decide] = any_outer[decide]
            open_ &= ~any_free
        return res

    def unit(v):
        return v / np.maximum(np.linalg.norm(v, axis=1), 1e-12)[:, None]

    # which pieces bound E: decided once per piece from its own outward direction (radial for a face,
    # the sum of the two radial directions for an edge, of the three for a vertex)
    if len(verts):
        vdir = unit(sum((verts - z[vtrip[:, c]]) / R[vtrip[:, c], None] for c in range(3)))
        keepv = outer_side(verts, vdir)
        verts, vtrip = verts[keepv], vtrip[keepv]
    vtree = cKDTree(verts) if len(verts) else None
    if len(circles):
        ccen, cu, crho, cab = circles
        ctree = cKDTree(ccen)
        cr_max = crho.max() if crho.size else 0.0
    kz = min(16, len(z))

    def uncovered(pts, own):
        """Points covered by no ball except their own (own: [n, m] atom ids, -1 padded)."""
        dd, ii = tree.query(pts, k=kz)
        dd = np.atleast_2d(dd).reshape(len(pts), -1)
        ii = np.atleast_2d(ii).reshape(len(pts), -1)
        inside_ = dd < R[ii] - 1e-9
        for c in range(own.shape[1]):
            inside_ &= ii != own[:, c:c + 1]
        return ~inside_.any(axis=1)

    reach = probe + big + 2 * h
    for s in range(0, idxs.size, 50_000):
        ids = idxs[s:s + 50_000]
        Q = P[ids]
        n = ids.size
        best = np.full(n, np.inf)
        # vertices (already restricted to those that bound E): an upper bound that prunes the rest
        if vtree is not None:
            kv = min(16, len(verts))
            dv, _ = vtree.query(Q, k=kv)
            best = np.minimum(best, dv.reshape(n, -1).min(axis=1))
        # circular edges: the nearest point of each nearby intersection circle
        if len(circles):
            kc = min(48, len(ccen))
            dd, ii = ctree.query(Q, k=kc)
            dd = dd.reshape(n, -1)
            ii = ii.reshape(n, -1)
            t_idx = np.repeat(np.arange(n), dd.shape[1])
            c_idx = ii.ravel()
            keep = dd.ravel() < cr_max + reach
            t_idx, c_idx = t_idx[keep], c_idx[keep]
            w = Q[t_idx] - ccen[c_idx]
            ax = np.sum(w * cu[c_idx], axis=1)
            wp = w - ax[:, None] * cu[c_idx]
            Lp = np.linalg.norm(wp, axis=1)
            good = Lp > 1e-12
            t_idx, c_idx, wp, Lp = t_idx[good], c_idx[good], wp[good], Lp[good]
            cpts = ccen[c_idx] + (crho[c_idx] / Lp)[:, None] * wp
            dist = np.linalg.norm(cpts - Q[t_idx], axis=1)
            near = dist < best[t_idx]
            t_idx, c_idx, cpts, dist = t_idx[near], c_idx[near], cpts[near], dist[near]
            ok = uncovered(cpts, cab[c_idx])
            a, b = cab[c_idx, 0], cab[c_idx, 1]
            ok &= outer_side(cpts, unit((cpts - z[a]) / R[a, None] + (cpts - z[b]) / R[b, None]))
            np.minimum.at(best, t_idx[ok], dist[ok])
        # spherical faces: the projection of x onto each nearby sphere
        ka = min(32, len(z))
        dd, ii = tree.query(Q, k=ka)
        dd = dd.reshape(n, -1)
        ii = ii.reshape(n, -1)
        t_idx = np.repeat(np.arange(n), dd.shape[1])
        a_idx = ii.ravel()
        L = dd.ravel()
        dist = np.abs(L - R[a_idx])
        keep = (L > 1e-12) & (dist < reach) & (dist < best[t_idx])
        t_idx, a_idx, L, dist = t_idx[keep], a_idx[keep], L[keep], dist[keep]
        cpts = z[a_idx] + (R[a_idx] / L)[:, None] * (Q[t_idx] - z[a_idx])
        ok = uncovered(cpts, a_idx[:, None])
        ok &= outer_side(cpts, (cpts - z[a_idx]) / R[a_idx, None])
        np.minimum.at(best, t_idx[ok], dist[ok])
        d[ids] = np.where(np.isfinite(best), probe - best, -big)
    d = np.clip(d, -big, big)
    return d
