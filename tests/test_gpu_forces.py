"""GPU parity of the per-link kernels (paper Sec. 2-4): Wilson force, fermion
force from the multi-shift solutions, plaquette, and the Philox draws,
against the FP64 oracle through the C ABI."""
import json
import os

import numpy as np
import pytest

import synthetic as syn
from oracle import actions, dirac, lattice as lat, philox, solvers
from tests import layout as L
from tests.gpu_util import dev, host_complex, torch_cuda

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rationals.json")


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 2, 6, 8)])
def test_gauge_force_and_plaquette(torch, dims):
    from paper_1010_5433_gb300 import stag
    u = syn.haar_gauge(dims, 3) if dims[1] == 2 else syn.near_identity_gauge(dims, 3, width=0.6)
    beta = 5.5
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        f = torch.empty((4, 2, 8, int(np.prod(dims)) // 2), dtype=torch.float64, device="cuda")
        stag.stag_gauge_force(ctx, beta, f)
        got = L.mom_from_abi(f.cpu().numpy(), dims)
        assert _rel(got, actions.wilson_force(u, beta)) < 1e-12
        assert abs(stag.stag_plaquette(ctx) - actions.mean_plaquette(u)) < 1e-13
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 2e-5), (2, 2e-5)])
def test_fermion_force_matches_oracle(torch, prec, tol):
    from paper_1010_5433_gb300 import stag
    dims = (4, 4, 4, 6)
    u = syn.near_identity_gauge(dims, 11, width=0.5)
    eta, par = lat.eta(dims), lat.parity(dims)
    rat = json.load(open(GOLDEN))["c1_md"]
    mass = 0.1
    n_pf = 2
    phis = [syn.gaussian_fermion(dims, 20 + k, on_parity=0) for k in range(n_pf)]
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        r = stag.make_rational(rat["a0"], rat["alpha"], rat["beta"])
        d_phi = dev(torch, np.stack([L.to_half(p, dims, 0) for p in phis]))
        f = torch.empty((4, 2, 8, int(np.prod(dims)) // 2), dtype=torch.float64, device="cuda")
        stag.stag_fermion_force(ctx, mass, r, prec, n_pf, d_phi, f, 1e-12 if prec == 0 else 1e-8, 10000)
        got = L.mom_from_abi(f.cpu().numpy(), dims)
        want = np.zeros_like(got)
        s0 = min(rat["beta"])
        for p in phis:
            xs = solvers.multishift_cg(lambda v: dirac.a_op(u, v, mass, eta, par, s0), p, rat["beta"], 1e-13)[0]
            want += actions.fermion_force(u, xs, rat["alpha"], eta, par)
        assert _rel(got, want) < tol
    finally:
        stag.stag_destroy(ctx)


def test_philox_draws_match_oracle(torch):
    from paper_1010_5433_gb300 import stag
    dims = (2, 2, 4, 2)
    vh = int(np.prod(dims)) // 2
    ctx = stag.stag_create(dims, True)
    try:
        m = torch.empty((4, 2, 8, vh), dtype=torch.float64, device="cuda")
        stag.stag_draw_momenta(ctx, 0x5A0001, 7, m)
        got = L.mom_from_abi(m.cpu().numpy(), dims)
        np.testing.assert_allclose(got, philox.draw_momenta(dims, 0x5A0001, 7), rtol=0, atol=1e-13)
        xi = torch.empty((2, 3, 2 * vh), dtype=torch.float64, device="cuda")
        stag.stag_draw_sources(ctx, 99, 3, 16, 2, xi)
        g = host_complex(xi).reshape(2, 3, vh)
        for k in range(2):
            np.testing.assert_allclose(g[k], philox.draw_source_half(vh, 99, 3, 16 + k), rtol=0, atol=1e-13)
    finally:
        stag.stag_destroy(ctx)
