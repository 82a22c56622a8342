"""Seeded synthetic inputs for the space-time heat solves.

This module names problem sizes and draws random numbers.  It holds none of the
discretisation or solver arithmetic (no finite-element integrals, no time
matrices, no Krylov steps), so the CPU oracle and the GPU library can both take
their inputs from it without sharing method code.

Workloads (unit domains, homogeneous initial and boundary data):

* ``heat1d``  -- 1D, 63 interior P1 nodes, 64 uniform time intervals, T = 1,
  manufactured forcing from u = sin(pi x) sin(pi t).
* ``heat2d``  -- 2D Q1 on a 255 x 255 interior grid (N_h = 65025), 256 time
  intervals, T = 1, manufactured forcing from u = sin(pi x) sin(pi y) sin(pi t).
* ``heat2d_gauss`` -- the same grid with a rank-2 Gaussian forcing (seed 2), so
  the Krylov loop has work to do.
* ``heat3d``  -- 3D Q1 on a 127^3 interior grid (N_h = 2,048,383), 512 time
  intervals, T = 1, rank-4 Gaussian forcing (seed 3, space factor drawn first).
* batched and served streams, drawn by :func:`batched_instances` and
  :func:`served_requests`.

The paper's own experiment (a 3D heat problem on unstructured P1 meshes of
(-1,1)^3, Section 5, Example 1) is not reproducible without its meshes; these
uniform-grid workloads stand in for it.
"""

from __future__ import annotations

import numpy as np

WORKLOADS = {
    "heat1d": dict(dim=1, n=63, n_t=64, T=1.0, kappa=1.0, rhs="manufactured"),
    "heat2d": dict(dim=2, n=255, n_t=256, T=1.0, kappa=1.0, rhs="manufactured"),
    "heat2d_gauss": dict(dim=2, n=255, n_t=256, T=1.0, kappa=1.0, rhs="gaussian", p=2, seed=2),
    "heat3d": dict(dim=3, n=127, n_t=512, T=1.0, kappa=1.0, rhs="gaussian", p=4, seed=3),
    # a smaller 3D case of the same kind (profiling captures)
    "heat3d_small": dict(dim=3, n=63, n_t=128, T=1.0, kappa=1.0, rhs="gaussian", p=4, seed=3),
    # many instances: drawn by batched_instances / served_requests
    "batched": dict(kind="batched", count=256, seed=4, p=2),
    # a smaller batch of the same kind (profiling captures that must fit a few GB)
    "batched_small": dict(kind="batched", count=24, seed=4, p=2),
    "served": dict(kind="served", count=2200, warmup=200, seed=5, mean_gap_s=2e-3, p=2),
}


def n_spatial(dim: int, n: int) -> int:
    """Number of interior nodes of a uniform grid with ``n`` nodes per side."""
    return int(n) ** int(dim)


def gaussian_factors(n_h: int, n_t: int, p: int, seed: int):
    """Return (F1, F2), F1 of shape (n_h, p) and F2 of shape (n_t, p), i.i.d. N(0,1).

    F1 is drawn first from ``numpy.random.default_rng(seed)``, then F2.  The load
    matrix of the space-time system is F = F1 @ F2.T.
    """
    rng = np.random.default_rng(seed)
    f1 = rng.standard_normal((n_h, p))
    f2 = rng.standard_normal((n_t, p))
    return f1, f2


def batched_instances(count: int = 256, seed: int = 4, sides=(63, 127, 255),
                      n_ts=(64, 128, 256, 512), p: int = 2):
    """Draw a batch of 2D heat instances.

    Each instance has a grid side drawn uniformly from ``sides``, a number of time
    intervals drawn uniformly from ``n_ts``, a diffusion coefficient
    kappa = 10**U(-1, 1) and a rank-``p`` Gaussian load factor pair.  The
    factors are drawn after all sizes, in instance order, from the same stream.
    """
    rng = np.random.default_rng(seed)
    side = rng.choice(np.asarray(sides), size=count)
    n_t = rng.choice(np.asarray(n_ts), size=count)
    kappa = 10.0 ** rng.uniform(-1.0, 1.0, size=count)
    out = []
    for i in range(count):
        n_h = int(side[i]) ** 2
        f1 = rng.standard_normal((n_h, p))
        f2 = rng.standard_normal((int(n_t[i]), p))
        out.append(dict(dim=2, n=int(side[i]), n_t=int(n_t[i]), T=1.0,
                        kappa=float(kappa[i]), F1=f1, F2=f2))
    return out


def served_requests(count: int = 2200, seed: int = 5, mean_gap_s: float = 2e-3,
                    p: int = 2, with_factors: bool = False):
    """Draw a Poisson request stream of heat and convection-diffusion solves.

    Kinds are uniform over {heat, convdiff} x {1D n=63/127, 2D n=63/127/255,
    3D n=31/63/127}; n_t is uniform over {64, 128, 256, 512}; eps = 10**U(-2, 0)
    (used as kappa for heat); beta = (1, 0.5, 0.25) truncated to the dimension.
    Arrival gaps are exponential with mean ``mean_gap_s``.  Factors are drawn
    per request from a child generator seeded by (seed, index) so that a request
    can be regenerated alone.
    """
    rng = np.random.default_rng(seed)
    shapes = [(1, 63), (1, 127), (2, 63), (2, 127), (2, 255), (3, 31), (3, 63), (3, 127)]
    ops = ["heat", "convdiff"]
    gaps = rng.exponential(mean_gap_s, size=count)
    arrival = np.cumsum(gaps)
    reqs = []
    for i in range(count):
        dim, n = shapes[int(rng.integers(len(shapes)))]
        op = ops[int(rng.integers(2))]
        n_t = int(rng.choice([64, 128, 256, 512]))
        eps = float(10.0 ** rng.uniform(-2.0, 0.0))
        beta = (1.0, 0.5, 0.25)[:dim]
        r = dict(index=i, arrival_s=float(arrival[i]), op=op, dim=dim, n=n, n_t=n_t,
                 T=1.0, eps=eps, beta=beta, p=p, seed=(seed, i))
        if with_factors:
            r["F1"], r["F2"] = request_factors(r)
        reqs.append(r)
    return reqs


def request_factors(req):
    """Gaussian load factors of one served request, reproducible from its seed."""
    rng = np.random.default_rng(list(req["seed"]))
    n_h = int(req["n"]) ** int(req["dim"])
    f1 = rng.standard_normal((n_h, req["p"]))
    f2 = rng.standard_normal((req["n_t"], req["p"]))
    return f1, f2


def simplex_mesh(dim: int, n: int, seed: int = 6, jitter: float = 0.25, flip: bool = True):
    """A seeded unstructured simplex mesh of the unit square (triangles) or cube (tetrahedra).

    Geometry only: a lattice of (n + 2)^dim nodes with spacing h = 1/(n + 1) (x fastest), every interior node
    moved by U(-jitter h, jitter h) in each coordinate; 2D cells split into two triangles along a diagonal
    drawn at random (``flip``; else always the diagonal from the lower-left corner), 3D cells into the six
    tetrahedra of the Kuhn subdivision along the main diagonal.  Returns dict(nodes (N x dim), elems (E x
    (dim + 1) node indices), interior (N bool: the nodes off the boundary)).
    """
    rng = np.random.default_rng(seed)
    m = n + 2
    h = 1.0 / (n + 1)
    axes = [np.arange(m) * h] * dim
    grid = np.meshgrid(*axes[::-1], indexing="ij")[::-1]   # x fastest in the flattened order
    nodes = np.stack([g.reshape(-1) for g in grid], axis=1)
    idx = np.stack(np.meshgrid(*[np.arange(m)] * dim, indexing="ij")[::-1], axis=-1).reshape(-1, dim)
    interior = np.all((idx >= 1) & (idx <= n), axis=1)
    nodes[interior] += rng.uniform(-jitter * h, jitter * h, size=(int(interior.sum()), dim))

    def nid(c):
        out = 0
        for d in range(dim - 1, -1, -1):
            out = out * m + c[d]
        return out

    elems = []
    if dim == 2:
        diag = rng.integers(0, 2, size=(n + 1, n + 1)) if flip else np.zeros((n + 1, n + 1), dtype=int)
        for j in range(n + 1):
            for i in range(n + 1):
                a, b, c, d = nid((i, j)), nid((i + 1, j)), nid((i, j + 1)), nid((i + 1, j + 1))
                if diag[j, i] == 0:
                    elems += [(a, b, d), (a, d, c)]
                else:
                    elems += [(a, b, c), (b, d, c)]
    elif dim == 3:
        perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
        for k in range(n + 1):
            for j in range(n + 1):
                for i in range(n + 1):
                    for p in perms:
                        c = [i, j, k]
                        path = [nid(tuple(c))]
                        for ax in p:
                            c[ax] += 1
                            path.append(nid(tuple(c)))
                        elems.append(tuple(path))
    else:
        raise ValueError("dim must be 2 or 3")
    return dict(nodes=nodes, elems=np.asarray(elems, dtype=np.int64), interior=interior)
