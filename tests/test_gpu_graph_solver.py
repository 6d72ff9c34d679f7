"""The three-kernel solver iteration (Dslash D_oe; D_eo with the A epilogue
and (p, Ap); the fused shift/residual update with (r, r)) driven by a
CUDA-graph WHILE loop whose condition the device sets, or the same kernels as
plain launches: the path STAG_PERSISTENT=0 selects instead of the persistent
solver.  Checked against the FP64 oracle at sizes the oracle solves in
seconds: the same bars as the persistent path (FP64 within 1e-10, mixed
within the 1e-6 true residual), and one whole trajectory."""
import numpy as np
import pytest

import synthetic as syn
from oracle import dirac, lattice as lat, solvers
from tests import layout as L
from tests.gpu_util import dev, host_complex, torch_cuda

pytestmark = pytest.mark.gpu

SHIFTS_8 = [0.0, 0.0009, 0.004, 0.02, 0.09, 0.4, 1.7, 9.0]


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.mark.parametrize("graphs", ["1", "0"])
@pytest.mark.parametrize("dims,nrhs", [((4, 4, 4, 4), 1), ((4, 6, 4, 8), 3)])
def test_fp64_three_kernel_solver_matches_oracle(torch, monkeypatch, dims, nrhs, graphs):
    from paper_1010_5433_gb300 import stag
    monkeypatch.setenv("STAG_PERSISTENT", "0")
    monkeypatch.setenv("STAG_GRAPHS", graphs)
    u = syn.haar_gauge(dims, 131)
    eta, par = lat.eta(dims), lat.parity(dims)
    mass = 0.1
    bs = [syn.gaussian_fermion(dims, 140 + k, on_parity=0) for k in range(nrhs)]
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        d_b = dev(torch, np.stack([L.to_half(b, dims, 0) for b in bs]))
        d_x = torch.empty((nrhs, len(SHIFTS_8)) + tuple(d_b.shape[1:]), dtype=torch.float64, device="cuda")
        info = stag.stag_multishift_solve(ctx, mass, SHIFTS_8, stag.STAG_FP64, nrhs, d_b, d_x, 1e-12, 5000)
        got = host_complex(d_x).reshape(nrhs, len(SHIFTS_8), 3, -1)
        for k, b in enumerate(bs):
            xs, its, _ = solvers.multishift_cg(lambda v: dirac.a_op(u, v, mass, eta, par, 0.0), b, SHIFTS_8, 1e-12)
            for s in range(len(SHIFTS_8)):
                assert L.rel_err(got[k, s], L.to_half(xs[s], dims, 0)) < 1e-10
            if nrhs == 1:
                assert abs(info.iterations - its) <= 1
        assert max(info.true_residual[s] for s in range(len(SHIFTS_8))) < 1e-11
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_mixed_three_kernel_solver_true_residual(torch, monkeypatch, prec):
    from paper_1010_5433_gb300 import stag
    monkeypatch.setenv("STAG_PERSISTENT", "0")
    dims = (8, 8, 8, 8)
    u = syn.haar_gauge(dims, 151)
    eta, par = lat.eta(dims), lat.parity(dims)
    mass, nrhs = 0.05, 2
    bs = [syn.gaussian_fermion(dims, 160 + k, on_parity=0) for k in range(nrhs)]
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        d_b = dev(torch, np.stack([L.to_half(b, dims, 0) for b in bs]))
        d_x = torch.empty((nrhs, len(SHIFTS_8)) + tuple(d_b.shape[1:]), dtype=torch.float64, device="cuda")
        info = stag.stag_multishift_solve(ctx, mass, SHIFTS_8, prec, nrhs, d_b, d_x, 1e-6, 20000)
        got = host_complex(d_x).reshape(nrhs, len(SHIFTS_8), 3, -1)
        for k, b in enumerate(bs):
            for s, sh in enumerate(SHIFTS_8):
                x = L.from_half(got[k, s], dims, 0)
                r = b - dirac.a_op(u, x, mass, eta, par, sh)
                assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-6 * 1.05, (k, s)
        assert info.reliable_updates >= 1
    finally:
        stag.stag_destroy(ctx)
