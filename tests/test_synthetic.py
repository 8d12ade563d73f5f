"""Input generators: the synthetic SES molecule field and the batch / request-stream helpers (CPU only)."""
import numpy as np
import pytest
from scipy import ndimage

import synthetic as syn
from synthetic import _ses


def _brute_ses(x, z, R, probe):
    """Signed SES distance at x by brute force over every atom, circle and vertex (no cavities assumed)."""
    dU = np.min(np.linalg.norm(z - x, axis=1) - R)
    if dU >= 0:
        return probe + dU
    cand = []

    def covered(p, own):
        others = [b for b in range(len(z)) if b not in own]
        return any(np.linalg.norm(z[b] - p) < R[b] - 1e-9 for b in others)

    for a in range(len(z)):
        L = np.linalg.norm(x - z[a])
        p = z[a] + R[a] / L * (x - z[a])
        if not covered(p, (a,)):
            cand.append(abs(L - R[a]))
    for a in range(len(z)):
        for b in range(a + 1, len(z)):
            dvec = z[b] - z[a]
            dist = np.linalg.norm(dvec)
            if not (abs(R[a] - R[b]) < dist < R[a] + R[b]):
                continue
            u = dvec / dist
            t = (dist ** 2 + R[a] ** 2 - R[b] ** 2) / (2 * dist)
            rho = np.sqrt(R[a] ** 2 - t ** 2)
            cen = z[a] + t * u
            w = x - cen
            wp = w - np.dot(w, u) * u
            p = cen + rho * wp / np.linalg.norm(wp)
            if not covered(p, (a, b)):
                cand.append(np.linalg.norm(p - x))
    _, _, verts, _ = _ses._boundary_pieces(z, R)
    for v in verts:
        cand.append(np.linalg.norm(v - x))
    return probe - min(cand)


def test_molecule_field_matches_brute_force():
    xyz, radii, _ = syn.random_walk_molecule(12, 3)
    prob = syn.molecule_problem(n_atoms=12, seed=3, h=0.5)
    g = prob.grid
    R = radii + 1.4
    X, Y, Z = g.points()
    P = np.stack([X, Y, Z], axis=1)
    dU = np.array([np.min(np.linalg.norm(xyz - p, axis=1) - R) for p in P])
    lab, nlab = ndimage.label((dU >= 0).reshape(g.n[2], g.n[1], g.n[0]))
    assert nlab == 1, "the test molecule must have no cavity"
    sd = np.asarray(prob.sdist)
    band = np.nonzero(np.abs(sd) < prob.tube + 2 * g.h)[0]
    rng = np.random.Generator(np.random.PCG64(0))
    for lin in rng.choice(band, size=60, replace=False):
        assert abs(sd[lin] - _brute_ses(P[lin], xyz, R, 1.4)) < 1e-9


@pytest.mark.parametrize("spec", [(120, 7, 0.5), (60, 11, 0.35)])
def test_molecule_field_is_a_distance(spec):
    """1-Lipschitz around the tube and a nonzero central-difference gradient at every tube node."""
    n_atoms, seed, h = spec
    prob = syn.molecule_problem(n_atoms=n_atoms, seed=seed, h=h)
    g = prob.grid
    D = np.asarray(prob.sdist).reshape(g.n[2], g.n[1], g.n[0])
    big = np.abs(D).max()
    for ax in range(3):
        a = np.take(D, range(0, D.shape[ax] - 1), axis=ax)
        b = np.take(D, range(1, D.shape[ax]), axis=ax)
        near = (np.abs(a) < prob.tube + 2 * h) | (np.abs(b) < prob.tube + 2 * h)
        assert not np.any(near & ((np.abs(a) >= big) | (np.abs(b) >= big)))
        assert np.max(np.abs(a - b)[near]) <= h * (1 + 1e-2)
    k, j, i = np.nonzero(np.abs(D) < prob.tube)
    gx = D[k, j, i + 1] - D[k, j, i - 1]
    gy = D[k, j + 1, i] - D[k, j - 1, i]
    gz = D[k + 1, j, i] - D[k - 1, j, i]
    gn = np.sqrt(gx * gx + gy * gy + gz * gz) / (2 * h)
    assert gn.min() > 0.2


def test_batch_specs_and_streams():
    a = syn.batch_specs(64, seed=0)
    assert a == syn.batch_specs(64, seed=0)
    atoms = np.array([s[0] for s in a])
    assert atoms.min() >= 20 and atoms.max() <= 2000
    assert {s[2] for s in a} <= {0.5, 0.35}
    assert len({s[1] for s in a}) == 64
    t, _ = syn.request_stream(4000, rate=8.0, seed=1)
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    assert abs(np.mean(np.diff(t)) * 8.0 - 1.0) < 0.06
    p = syn.sphere_with_nodes(20000)
    M = np.count_nonzero(np.abs(np.asarray(p.sdist)) < p.tube)
    assert abs(M / 20000 - 1) < 0.05
