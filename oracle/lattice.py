"""Lattice geometry for unimproved staggered fermions (paper Sec. 2: "standard
(i.e. non-improved) staggered fermions" with even/odd preconditioning).

Directions mu = 0, 1, 2, 3 are x, y, z, t.  Arrays are indexed [t, z, y, x],
so array axis of direction mu is 3 - mu and the flattened order is the
lexicographic site = x + Lx*(y + Ly*(z + Lz*t)).

Staggered phases (the Kawamoto-Smit phases of the one-component staggered
field):  eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z).
Fermion boundary conditions: periodic in space, antiperiodic in time, carried
as an extra sign -1 on every t-link that leaves the last time slice.  The
paper does not spell out either convention; these are the standard ones.
"""
import numpy as np


def axis_of(mu):
    """Array axis (of a [t, z, y, x, ...] array) that direction mu runs along."""
    return 3 - mu


def coords(dims):
    """Integer coordinate arrays x, y, z, t of shape [Lt, Lz, Ly, Lx]."""
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly),
                             np.arange(Lx), indexing="ij")
    return x, y, z, t


def parity(dims):
    """(x + y + z + t) mod 2; 0 = even."""
    x, y, z, t = coords(dims)
    return (x + y + z + t) % 2


def eta(dims, antiperiodic_t=True):
    """Link sign eta_mu(x) including the temporal boundary sign.

    Returns float array [4, Lt, Lz, Ly, Lx].  The entry for (mu, x) multiplies
    both the forward hop through link (x, mu) and the backward hop through it.
    """
    x, y, z, t = coords(dims)
    e = np.empty((4,) + x.shape)
    e[0] = 1.0
    e[1] = (-1.0) ** x
    e[2] = (-1.0) ** (x + y)
    e[3] = (-1.0) ** (x + y + z)
    if antiperiodic_t:
        e[3] = np.where(t == dims[3] - 1, -e[3], e[3])
    return e


def shift_fwd(f, mu):
    """g(x) = f(x + mu_hat), periodic."""
    return np.roll(f, -1, axis=axis_of(mu))


def shift_bwd(f, mu):
    """g(x) = f(x - mu_hat), periodic."""
    return np.roll(f, +1, axis=axis_of(mu))


def volume(dims):
    return int(np.prod(dims))
