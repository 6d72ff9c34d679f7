"""Gauge and fermion actions and their forces (paper Sec. 2: "action divided
in gauge and fermion part"; Sec. 4: precision of each piece).

Force convention: F_a(x, mu) = dS / d omega_a  under
U_mu(x) -> exp(i omega_a T_a) U_mu(x);  the momenta obey dp_a/dt = -F_a.
Forces are arrays [4, t, z, y, x, 8] of su(3) coefficients.
"""
import numpy as np

from . import lattice as lat
from . import dirac
from .su3 import T, dag


def _mm(a, b):
    return np.einsum("...ij,...jk->...ik", a, b)


def plaquette_field(u, mu, nu):
    """U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag."""
    return _mm(_mm(u[mu], lat.shift_fwd(u[nu], mu)),
               _mm(dag(lat.shift_fwd(u[mu], nu)), dag(u[nu])))


def mean_plaquette(u):
    """<(1/3) Re tr U_P> over all sites and the six planes."""
    acc = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            acc += np.mean(np.real(np.trace(plaquette_field(u, mu, nu), axis1=-2, axis2=-1)))
    return acc / (6 * 3)


def wilson_action(u, beta):
    """S_g = beta sum_{x, mu<nu} (1 - (1/3) Re tr U_mu_nu(x)) (Wilson action)."""
    s = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            s += np.sum(1.0 - np.real(np.trace(plaquette_field(u, mu, nu), axis1=-2, axis2=-1)) / 3.0)
    return beta * s


def staple_sum(u, mu):
    """Sigma_mu(x) with sum over plaquettes through link (x, mu) of
    Re tr(U_mu(x) Sigma_mu(x)):  for each nu != mu the upper staple
    U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag and the lower staple
    U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)."""
    s = np.zeros_like(u[mu])
    for nu in range(4):
        if nu == mu:
            continue
        up = _mm(_mm(lat.shift_fwd(u[nu], mu), dag(lat.shift_fwd(u[mu], nu))), dag(u[nu]))
        u_nu_xmn = lat.shift_bwd(lat.shift_fwd(u[nu], mu), nu)       # U_nu(x+mu-nu)
        dn = _mm(_mm(dag(u_nu_xmn), dag(lat.shift_bwd(u[mu], nu))), lat.shift_bwd(u[nu], nu))
        s += up + dn
    return s


def _coeff_of_i_t(m):
    """Re tr(i T_a M) for every a: shape [..., 8]."""
    return np.real(1j * np.einsum("aij,...ji->...a", T, m))


def wilson_force(u, beta):
    """F_a = -(beta/3) Re tr(i T_a U_mu(x) Sigma_mu(x))."""
    return np.stack([-(beta / 3.0) * _coeff_of_i_t(_mm(u[mu], staple_sum(u, mu)))
                     for mu in range(4)])


def fermion_action(phi, xs, rat):
    """phi^dag r(A) phi = alpha_0 phi^dag phi + sum_i alpha_i phi^dag X_i."""
    s = rat.a0 * np.vdot(phi, phi)
    for a, x in zip(rat.alpha, xs):
        s += a * np.vdot(phi, x)
    return float(np.real(s))


def fermion_force(u, xs, alphas, eta, par):
    """Force of phi^dag r(A) phi given X_i = (A + beta_i)^(-1) phi (even fields).

    With A = m^2 - D_eo D_oe and D_oe = -D_eo^dag,
      d(phi^dag (A+beta)^(-1) phi) = X^dag (dD_eo) Y - Y^dag (dD_oe) X,  Y = D_oe X,
    and collecting the terms of each link (with Z = X on even, Y on odd sites,
    eps(x) = +1 / -1 on even / odd sites):
      F_a(x, mu) = sum_i alpha_i eps(x) eta_mu(x) Re tr[i T_a U_mu(x) Z_i(x+mu) Z_i(x)^dag].
    The paper gives no formula (Sec. 4 fixes only its precision); this is the
    derivation, and its sign is pinned by finite differences of the action.
    """
    epsx = np.where(par == 0, 1.0, -1.0)
    f = np.zeros(u.shape[:5] + (8,))
    for a_i, x in zip(alphas, xs):
        z = dirac.restrict(x, par, 0) + dirac.d_block(u, x, eta, par, 1)
        for mu in range(4):
            outer = lat.shift_fwd(z, mu)[..., :, None] * np.conj(z)[..., None, :]
            m = _mm(u[mu], outer)
            f[mu] += (a_i * epsx * eta[mu])[..., None] * _coeff_of_i_t(m)
    return f
