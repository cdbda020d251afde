"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds none of the method's arithmetic: it draws densities,
velocities and specific internal energies and assembles conserved variables
rho, rho v, rho (eps + |v|^2/2) from them.  No equation of state, flux,
operator or mesh quantity appears here.
"""
import numpy as np


def random_state(shape, seed, rho=(0.8, 1.2), vmax=0.5, eps=(1.8, 2.7), smooth=False):
    """Conserved state of shape [E, 5, n_z, n_y, n_x] (float64).

    rho ~ U(rho), v_c ~ U(-vmax, vmax), specific internal energy ~ U(eps).
    smooth=True replaces the independent draws by a few random low-order
    products of node indices within each element plus an element offset, so
    that neighbouring nodes differ little (closer to a resolved flow field).
    """
    rng = np.random.default_rng(seed)
    E, nv = shape[0], shape[1]
    dims = tuple(shape[2:])
    assert nv == 5 and len(dims) == 3

    def field(lo, hi):
        if not smooth:
            return rng.uniform(lo, hi, size=(E,) + dims)
        k, j, i = np.meshgrid(*(np.linspace(-1.0, 1.0, m) for m in dims), indexing="ij")
        base = rng.uniform(lo, hi, size=(E, 1, 1, 1))
        amp = 0.05 * (hi - lo)
        c = rng.uniform(-1, 1, size=(E, 4, 1, 1, 1))
        f = base + amp * (c[:, 0] * i + c[:, 1] * j + c[:, 2] * k + c[:, 3] * i * j)
        return np.clip(f, lo, hi)

    r = field(*rho)
    v = [field(-vmax, vmax) for _ in range(3)]
    e = field(*eps)
    u = np.empty(shape)
    u[:, 0] = r
    for c in range(3):
        u[:, 1 + c] = r * v[c]
    u[:, 4] = r * (e + 0.5 * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
    return u


def cube(ex, ey, ez, lo=-np.pi, hi=np.pi):
    """Box extents (lo, hi) for an ex*ey*ez mesh of a cube."""
    return (lo, lo, lo), (hi, hi, hi)


def random_degrees(E, seed, lo=1, hi=7):
    """Seeded per-element polynomial degrees, uniform in [lo, hi]."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=E).astype(np.int32)


def random_degree_triples(E, seed, lo=1, hi=7):
    """Seeded per-element, per-direction degrees (P_x, P_y, P_z), each
    uniform in [lo, hi]; shape (E, 3)."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=(E, 3)).astype(np.int32)


def random_state_blocks(degrees, seed, **kw):
    """Flat state of element blocks [5, n_z, n_y, n_x] in element order (the
    layout of a mesh whose elements carry their own degrees; `degrees` is
    (E,) or (E, 3)), each block drawn by random_state with a seed derived from
    `seed` and the element index."""
    out = []
    for e, N in enumerate(degrees):
        P = np.broadcast_to(np.asarray(N), (3,))
        dims = (int(P[2]) + 1, int(P[1]) + 1, int(P[0]) + 1)
        out.append(random_state((1, 5) + dims, seed * 100003 + e, **kw).reshape(-1))
    return np.concatenate(out)
