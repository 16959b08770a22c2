"""Adaptive importance sampling of the generator's uniform variables: VEGAS
(G. P. Lepage, "A new algorithm for adaptive multidimensional integration",
J. Comput. Phys. 27 (1978) 192), the algorithm behind the BASES / gBASES
integrator the paper uses for its cross sections (Sect. 6).

Oracle module (test infrastructure only).

Grid: for each dimension d, bin edges 0 = x_{d,0} < x_{d,1} < ... < x_{d,N} = 1.
A uniform deviate y in (0, 1) lies in bin i = floor(N y) and maps to

    x = x_{d,i} + (N y - i) (x_{d,i+1} - x_{d,i}),

so that every bin receives the same number of points on average; the map's
Jacobian dx/dy = N (x_{d,i+1} - x_{d,i}) multiplies the weight.  For the
integrand f(x) the weight of a point is f(x) prod_d J_d.

Refinement, per dimension, from the sums d_i of the squared weights of the
points in bin i:
  1. smoothing: each d_i replaced by the mean of itself and its neighbours
     (two terms at the ends);
  2. normalisation r_i = d_i / sum_j d_j;
  3. damping m_i = ((1 - r_i) / ln(1 / r_i))^alpha (0 for r_i = 0, 1 for r_i = 1);
  4. new edges: with m_i spread uniformly over old bin i, the N new bins each
     take an equal share of sum_i m_i.
A dimension whose sums are all zero keeps its edges.
"""
import math

import numpy as np


def uniform_grid(n_dims, n_bins):
    """Equal bins in every dimension: edges [n_dims, n_bins + 1]."""
    return np.tile(np.linspace(0.0, 1.0, n_bins + 1), (n_dims, 1))


def vegas_map(edges, y):
    """Map uniforms y [..., D] through the grid: (x [..., D], jac [...], bins [..., D])."""
    edges = np.asarray(edges, dtype=np.float64)
    D, N = edges.shape[0], edges.shape[1] - 1
    y = np.asarray(y, dtype=np.float64)
    t = y * N
    i = np.minimum(np.floor(t).astype(np.int64), N - 1)
    lo = np.take_along_axis(np.broadcast_to(edges, y.shape[:-1] + edges.shape), i[..., None], axis=-1)[..., 0]
    hi = np.take_along_axis(np.broadcast_to(edges, y.shape[:-1] + edges.shape), (i + 1)[..., None], axis=-1)[..., 0]
    width = hi - lo
    x = lo + (t - i) * width
    jac = np.prod(N * width, axis=-1)
    return x, jac, i


def histogram(n_dims, n_bins, bins, w):
    """d[d, i] = sum of w^2 over the points whose dimension d lies in bin i."""
    bins = np.asarray(bins).reshape(-1, n_dims)
    w2 = np.asarray(w, dtype=np.float64).reshape(-1) ** 2
    out = np.zeros((n_dims, n_bins))
    for d in range(n_dims):
        out[d] = np.bincount(bins[:, d], weights=w2, minlength=n_bins)
    return out


def refine(edges, d, alpha=1.5):
    """New edges from the bin sums d [D, N] (steps 1-4 of the module docstring)."""
    edges = np.asarray(edges, dtype=np.float64)
    D, N = edges.shape[0], edges.shape[1] - 1
    new = edges.copy()
    for k in range(D):
        s = np.asarray(d[k], dtype=np.float64)
        if not np.any(s > 0):
            continue
        sm = np.empty(N)
        if N == 1:
            sm[:] = s
        else:
            sm[0] = (s[0] + s[1]) / 2.0
            sm[-1] = (s[-2] + s[-1]) / 2.0
            for i in range(1, N - 1):
                sm[i] = (s[i - 1] + s[i] + s[i + 1]) / 3.0
        r = sm / sm.sum()
        m = np.zeros(N)
        for i in range(N):
            if r[i] >= 1.0:
                m[i] = 1.0
            elif r[i] > 0.0:
                m[i] = ((1.0 - r[i]) / math.log(1.0 / r[i])) ** alpha
        total = m.sum()
        x = edges[k]
        cum = 0.0   # weight of the old bins before bin j
        j = 0
        for e in range(1, N):
            target = total * e / N
            while j < N - 1 and cum + m[j] < target:
                cum += m[j]
                j += 1
            frac = (target - cum) / m[j] if m[j] > 0 else 0.0
            new[k, e] = x[j] + min(max(frac, 0.0), 1.0) * (x[j + 1] - x[j])
        new[k, 0], new[k, N] = 0.0, 1.0
    return new
