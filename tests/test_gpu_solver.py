"""GPU parity of the multi-shift CG (paper Sec. 6, Jegerlehner's recurrences)
against the FP64 oracle, through the C ABI: fp64 mode within 1e-10, mixed
modes (fp32 / bf16 Dslash, fp64 reliable updates) within a 1e-5 relative
true residual checked with the oracle's operator."""
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


def _setup(dims, seed, hot=True):
    u = syn.haar_gauge(dims, seed) if hot else syn.near_identity_gauge(dims, seed)
    return u, lat.eta(dims), lat.parity(dims)


@pytest.mark.parametrize("dims,nrhs", [((4, 4, 4, 4), 1), ((4, 4, 6, 4), 2), ((4, 6, 4, 8), 3), ((6, 4, 2, 4), 9)])
def test_fp64_multishift_matches_oracle(torch, dims, nrhs):
    from paper_1010_5433_gb300 import stag
    u, eta, par = _setup(dims, 31)
    mass = 0.1
    bs = [syn.gaussian_fermion(dims, 40 + k, on_parity=0) for k in range(nrhs)]
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        d_b = dev(torch, np.stack([L.to_half(b, dims, 0) for b in bs]))
        d_x = torch.empty((nrhs, len(SHIFTS_8)) + tuple(d_b.shape[1:]), dtype=torch.float64, device="cuda")
        info = stag.stag_multishift_solve(ctx, mass, SHIFTS_8, stag.STAG_FP64, nrhs, d_b, d_x, 1e-12, 5000)
        got = host_complex(d_x).reshape(nrhs, len(SHIFTS_8), 3, -1)
        for k, b in enumerate(bs):
            xs, its, per = solvers.multishift_cg(lambda v: dirac.a_op(u, v, mass, eta, par, 0.0), b, SHIFTS_8,
                                                 1e-12)
            for s in range(len(SHIFTS_8)):
                assert L.rel_err(got[k, s], L.to_half(xs[s], dims, 0)) < 1e-10
            if nrhs == 1:
                # the fp64 path iterates in float-float (about 48 bits): the iteration at
                # which a slowly converging shift crosses 1e-12 may move by a few
                assert abs(info.iterations - its) <= 1
                d = [abs(info.shift_iterations[s] - per[s]) for s in range(len(SHIFTS_8))]
                assert max(d) <= 3, (list(info.shift_iterations)[:len(SHIFTS_8)], list(per))
        assert max(info.true_residual[s] for s in range(len(SHIFTS_8))) < 1e-11
    finally:
        stag.stag_destroy(ctx)


def _oracle_true_residual(u, eta, par, mass, shift, x_half, b, dims):
    x = L.from_half(x_half, dims, 0)
    r = b - dirac.a_op(u, x, mass, eta, par, shift)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8)])
def test_mixed_multishift_true_residual(torch, prec, dims):
    from paper_1010_5433_gb300 import stag
    u, eta, par = _setup(dims, 51)
    mass = 0.05
    nrhs = 2
    bs = [syn.gaussian_fermion(dims, 60 + k, on_parity=0) for k in range(nrhs)]
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        d_b = dev(torch, np.stack([L.to_half(b, dims, 0) for b in bs]))
        d_x = torch.empty((nrhs, len(SHIFTS_8)) + tuple(d_b.shape[1:]), dtype=torch.float64, device="cuda")
        info = stag.stag_multishift_solve(ctx, mass, SHIFTS_8, prec, nrhs, d_b, d_x, 1e-6, 20000)
        got = host_complex(d_x).reshape(nrhs, len(SHIFTS_8), 3, -1)
        worst = np.zeros(len(SHIFTS_8))
        for k, b in enumerate(bs):
            for s, sh in enumerate(SHIFTS_8):
                res = _oracle_true_residual(u, eta, par, mass, sh, got[k, s], b, dims)
                assert res < 1e-6 * 1.05, (k, s, res)
                worst[s] = max(worst[s], res)
        # the library's own fp64 true residual (max over sources) agrees
        np.testing.assert_allclose(worst, [info.true_residual[s] for s in range(len(SHIFTS_8))], rtol=1e-6)
        assert info.reliable_updates >= 1
    finally:
        stag.stag_destroy(ctx)


def test_not_converged_is_reported(torch):
    from paper_1010_5433_gb300 import stag
    dims = (4, 4, 4, 4)
    u, eta, par = _setup(dims, 71)
    b = syn.gaussian_fermion(dims, 72, on_parity=0)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        d_b = dev(torch, L.to_half(b, dims, 0)[None])
        d_x = torch.empty((1, 2) + tuple(d_b.shape[1:]), dtype=torch.float64, device="cuda")
        st, info = stag.stag_multishift_solve(ctx, 0.01, [0.0, 0.5], 0, 1, d_b, d_x, 1e-12, 7, check=False)
        assert st == 4 and info.iterations == 7
        # partial results are the oracle's after 7 iterations
        xs, _, _ = solvers.multishift_cg(lambda v: dirac.a_op(u, v, 0.01, eta, par, 0.0), b, [0.0, 0.5], 0.0,
                                         max_iter=7)
        got = host_complex(d_x).reshape(2, 3, -1)
        assert L.rel_err(got[0], L.to_half(xs[0], dims, 0)) < 1e-10
    finally:
        stag.stag_destroy(ctx)


def test_zero_source_gives_zero(torch):
    from paper_1010_5433_gb300 import stag
    dims = (4, 4, 4, 4)
    u, _, _ = _setup(dims, 81)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        d_b = torch.zeros((1, 3, 2 * 128), dtype=torch.float64, device="cuda")
        d_x = torch.full((1, 2, 3, 2 * 128), 7.0, dtype=torch.float64, device="cuda")
        info = stag.stag_multishift_solve(ctx, 0.1, [0.0, 0.5], 0, 1, d_b, d_x, 1e-10, 100)
        assert info.iterations == 0 and float(d_x.abs().max()) == 0.0
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_16x4_twelve_shifts(torch, prec):
    """The 16^4, m = 0.02, 12-shift solve of the N_f = 2 workload, checked
    shift by shift with the oracle's operator (true residual)."""
    from paper_1010_5433_gb300 import stag
    dims = (16, 16, 16, 16)
    u, eta, par = _setup(dims, 0x5A0002)
    mass = 0.02
    shifts = list(np.geomspace(1e-5, 3.0, 11)) + [0.0]
    b = syn.gaussian_fermion(dims, 91, on_parity=0)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        d_b = dev(torch, L.to_half(b, dims, 0)[None])
        d_x = torch.empty((1, len(shifts)) + tuple(d_b.shape[1:]), dtype=torch.float64, device="cuda")
        tol = 1e-10 if prec == 0 else 1e-6
        info = stag.stag_multishift_solve(ctx, mass, shifts, prec, 1, d_b, d_x, tol, 20000)
        got = host_complex(d_x).reshape(len(shifts), 3, -1)
        for s in (0, 5, 11):
            res = _oracle_true_residual(u, eta, par, mass, shifts[s], got[s], b, dims)
            assert res < tol * 1.05, (s, res)
        print("16^4 prec", prec, "iterations", info.iterations, "reliable", info.reliable_updates)
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("nshift", [1, 32])
def test_shift_count_extremes_fp64(torch, nshift):
    """One shift (plain CG) and the maximum of 32 shifts, every solution
    against the oracle's multi-shift CG."""
    from paper_1010_5433_gb300 import stag
    dims = (4, 4, 4, 4)
    u, eta, par = _setup(dims, 95)
    mass = 0.1
    shifts = [0.0] if nshift == 1 else [0.0] + list(np.geomspace(1e-4, 20.0, 31))
    b = syn.gaussian_fermion(dims, 96, on_parity=0)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        d_b = dev(torch, L.to_half(b, dims, 0)[None])
        d_x = torch.empty((1, nshift) + tuple(d_b.shape[1:]), dtype=torch.float64, device="cuda")
        info = stag.stag_multishift_solve(ctx, mass, shifts, stag.STAG_FP64, 1, d_b, d_x, 1e-12, 5000)
        xs, its, _ = solvers.multishift_cg(lambda v: dirac.a_op(u, v, mass, eta, par, 0.0), b, shifts, 1e-12)
        got = host_complex(d_x).reshape(nshift, 3, -1)
        for s in range(nshift):
            assert L.rel_err(got[s], L.to_half(xs[s], dims, 0)) < 1e-10, s
        assert abs(info.iterations - its) <= 3
    finally:
        stag.stag_destroy(ctx)


def test_barrier_wait_gives_up_and_context_stays_usable(torch):
    """Failure detection without a fault: a grid barrier that one of its two
    blocks never reaches; the waiting block's bounded wait gives up, the
    library reports STAG_ERR_TIMEOUT, and the same context then solves as
    before (fp64, checked with the oracle)."""
    from paper_1010_5433_gb300 import stag
    dims = (4, 4, 4, 4)
    u, eta, par = _setup(dims, 91)
    b = syn.gaussian_fermion(dims, 92, on_parity=0)
    ctx = stag.stag_create(dims, True)
    try:
        assert stag.stag_selftest_barrier_timeout(ctx, 0) == 1           # bad limit: argument error
        assert stag.stag_selftest_barrier_timeout(ctx, 1 << 14) == 5     # the wait ran out
        assert stag.stag_selftest_barrier_timeout(ctx, 1 << 12) == 5     # and again, same context
        torch.cuda.synchronize()
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        d_b = dev(torch, L.to_half(b, dims, 0)[None])
        d_x = torch.empty((1, 2) + tuple(d_b.shape[1:]), dtype=torch.float64, device="cuda")
        stag.stag_multishift_solve(ctx, 0.1, [0.0, 0.5], 0, 1, d_b, d_x, 1e-12, 5000)
        xs, _, _ = solvers.multishift_cg(lambda v: dirac.a_op(u, v, 0.1, eta, par, 0.0), b, [0.0, 0.5], 1e-12)
        got = host_complex(d_x).reshape(2, 3, -1)
        for s in range(2):
            assert L.rel_err(got[s], L.to_half(xs[s], dims, 0)) < 1e-10
    finally:
        stag.stag_destroy(ctx)


def test_persistent_solve_is_reproducible_bit_for_bit(torch):
    """The same mixed solve with many in-launch reliable updates, three times
    on one context: the same iterations, residuals and solutions bit for bit
    (fixed reduction order, and no field that the launch rewrites is read
    through the non-coherent cache after a grid barrier)."""
    from paper_1010_5433_gb300 import stag
    dims = (16, 16, 16, 16)
    u, eta, par = _setup(dims, 0x5A0003)
    mass = 0.02
    shifts = list(np.geomspace(1e-5, 3.0, 11)) + [0.0]
    b = syn.gaussian_fermion(dims, 93, on_parity=0)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        d_b = dev(torch, L.to_half(b, dims, 0)[None])
        runs = []
        for _ in range(3):
            d_x = torch.empty((1, len(shifts)) + tuple(d_b.shape[1:]), dtype=torch.float64, device="cuda")
            info = stag.stag_multishift_solve(ctx, mass, shifts, 2, 1, d_b, d_x, 1e-8, 20000)
            runs.append((info.iterations, info.reliable_updates,
                         [info.true_residual[s] for s in range(len(shifts))], d_x.cpu().numpy()))
        assert runs[0][1] >= 3
        for it, rel, res, x in runs[1:]:
            assert (it, rel) == runs[0][:2]
            assert res == runs[0][2]
            assert np.array_equal(x, runs[0][3])
        got = host_complex(torch.from_numpy(runs[0][3])).reshape(len(shifts), 3, -1)
        for s in (0, 11):
            assert _oracle_true_residual(u, eta, par, mass, shifts[s], got[s], b, dims) < 1e-8 * 1.05
    finally:
        stag.stag_destroy(ctx)
