"""Discrete direction sets and their isotropy tensors (oracle side).

Sec. 3.2.1 ("Velocity Discretization"): every direction is a unit vector, the
quadrature weights w_i sum to one, and a set has order p when it integrates
all harmonics up to degree p exactly (Eqs. sph-quad-cond, sph-quad-cond-2d).
The isotropy tensors are T^{a1..ak} = sum_i w_i n_i^{a1} ... n_i^{ak}
(Eq. iso-tensors).

Direction order is canonical so that populations can be compared index by
index with any other implementation: 2D rings keep k = 0..N-1; 3D sets are
sorted by the integer key (round(1e9 n_z), round(1e9 n_y), round(1e9 n_x)).
Components with |n| < 1e-15 are snapped to +0.0.
"""
import math

import numpy as np

SNAP = 1e-15


def _snap(n):
    n = np.array(n, dtype=np.float64)
    n[np.abs(n) < SNAP] = 0.0
    return n + 0.0  # turns -0.0 into +0.0


def ring2d(N, phi0=0.0):
    """N equally spaced directions on the unit circle, phi_k = phi0 + 2 pi k / N,
    equal weights 1/N (Sec. 3.2.1, 2D case).  Order p = N - 1 in the sense of
    Eq. (sph-quad-cond-2d); a rotation phi0 keeps the order."""
    k = np.arange(N, dtype=np.float64)
    phi = phi0 + 2.0 * math.pi * k / N
    n = np.stack([np.cos(phi), np.sin(phi), np.zeros(N)], axis=1)
    return _snap(n), np.full(N, 1.0 / N)


def _icosahedron():
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-g, g):
            v.append((0.0, a, b))
            v.append((a, b, 0.0))
            v.append((b, 0.0, a))
    v = np.array(v)
    # faces: triples of vertices that are pairwise at the edge length 2
    d2 = ((v[:, None, :] - v[None, :, :]) ** 2).sum(-1)
    adj = (d2 > 3.5) & (d2 < 4.5)
    faces = []
    for a in range(12):
        for b in range(a + 1, 12):
            if not adj[a, b]:
                continue
            for c in range(b + 1, 12):
                if adj[a, c] and adj[b, c]:
                    faces.append((a, b, c))
    assert len(faces) == 20
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    return v, faces


def icosphere(level):
    """Icosahedral geodesic set: the 12 vertices of the icosahedron, refined
    `level` times by splitting every triangle into four at its (renormalised)
    edge midpoints; 10 * 4**level + 2 points with equal weights.  The paper
    cites icosahedral-group quadratures among the rotation-invariant
    families (Sec. 3.2.1); this particular construction is the reading
    taken for the 42- and 162-direction sets."""
    verts, faces = _icosahedron()
    pts = [tuple(p) for p in verts]
    for _ in range(level):
        index = {}
        new_pts = list(pts)

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in index:
                m = (np.array(new_pts[a]) + np.array(new_pts[b])) / 2.0
                m = m / np.linalg.norm(m)
                index[key] = len(new_pts)
                new_pts.append(tuple(m))
            return index[key]

        new_faces = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        pts, faces = new_pts, new_faces
    n = _snap(np.array(pts))
    n = n[_canonical_order(n)]
    N = len(n)
    return n, np.full(N, 1.0 / N)


def gauss_legendre_product(n_theta, n_phi):
    """Product rule of Sec. 3.2.1: Gauss-Legendre in mu = cos(theta) times the
    trapezoid rule in phi.  Weights are (GL weight / 2) * (1 / n_phi)."""
    mu, wmu = np.polynomial.legendre.leggauss(n_theta)
    phi = 2.0 * math.pi * (np.arange(n_phi) + 0.5) / n_phi
    n, w = [], []
    for m, wm in zip(mu, wmu):
        s = math.sqrt(max(0.0, 1.0 - m * m))
        for p in phi:
            n.append((s * math.cos(p), s * math.sin(p), m))
            w.append(wm / 2.0 / n_phi)
    n, w = _snap(np.array(n)), np.array(w)
    order = _canonical_order(n)
    return n[order], w[order]


def _canonical_order(n):
    keys = np.rint(n * 1e9).astype(np.int64)
    return np.lexsort((keys[:, 0], keys[:, 1], keys[:, 2]))


def sgn(x):
    """Upwind sign of Eq. (interp): -1 for x < 0, else +1 (so sgn(0) = +1,
    paired with the interpolation weight 0)."""
    return np.where(np.asarray(x) < 0.0, -1, 1).astype(np.int64)


def isotropy_tensor(n, w, k, dims=3):
    """T^{a1..ak} = sum_i w_i n_i^{a1} ... n_i^{ak} (Eq. iso-tensors), as a
    dense array of shape (dims,)*k."""
    n = np.asarray(n)[:, :dims]
    T = np.array(w, dtype=np.float64)
    letters = "abcdefgh"
    out = np.einsum("i->", T) if k == 0 else None
    if k == 0:
        return out
    spec = ",".join("i" + letters[j] for j in range(k))
    return np.einsum("i," + spec + "->" + letters[:k], T, *([n] * k))
