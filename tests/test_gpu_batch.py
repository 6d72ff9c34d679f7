"""GPU parity of the batched path: independent lattices of uneven sizes solved
(multi-shift CG, Sec. 6) and evolved (RHMC trajectories, Sec. 2) together,
one persistent launch per solve, against the FP64 oracle per lattice and
against the same lattices run one at a time."""
import json
import os

import numpy as np
import pytest

import synthetic as syn
from oracle import dirac, integrator, lattice as lat, solvers
from oracle.rational import Rational
from tests import layout as L
from tests.gpu_util import dev, host_complex, torch_cuda, wrap_device

pytestmark = pytest.mark.gpu

SHIFTS_8 = [0.0, 0.0009, 0.004, 0.02, 0.09, 0.4, 1.7, 9.0]
# uneven volumes: 128 .. 192 even sites, the x extent even everywhere
DIMS_SET = [(4, 4, 4, 4), (4, 4, 4, 6), (6, 4, 4, 4), (2, 4, 4, 4)]
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rationals.json")


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _contexts(stag, dims_set, seeds, hot=True):
    ctxs, us = [], []
    hots = hot if isinstance(hot, (list, tuple)) else [hot] * len(dims_set)
    for dims, seed, h in zip(dims_set, seeds, hots):
        u = syn.haar_gauge(dims, seed) if h else syn.near_identity_gauge(dims, seed)
        c = stag.stag_create(dims, True)
        stag.stag_load_gauge(c, L.gauge_host(u))
        ctxs.append(c)
        us.append(u)
    return ctxs, us


def _destroy(stag, ctxs):
    for c in ctxs:
        stag.stag_destroy(c)


def test_fp64_batched_multishift_matches_oracle(torch):
    """Every lattice's solutions within 1e-10 of the oracle's, and every
    lattice stops at its own iteration count (its convergence flag), not at
    the slowest lattice's: ordered and Haar-random fields converge at very
    different counts."""
    from paper_1010_5433_gb300 import stag
    mass = 0.1
    ctxs, us = _contexts(stag, DIMS_SET, [201, 202, 203, 204], hot=[True, False, True, False])
    try:
        bs = [syn.gaussian_fermion(d, 210 + k, on_parity=0) for k, d in enumerate(DIMS_SET)]
        d_b = [dev(torch, L.to_half(b, d, 0)) for b, d in zip(bs, DIMS_SET)]
        d_x = [torch.empty((len(SHIFTS_8),) + tuple(x.shape), dtype=torch.float64, device="cuda") for x in d_b]
        infos = stag.stag_multishift_solve_batch(ctxs, mass, SHIFTS_8, stag.STAG_FP64, d_b, d_x, 1e-12, 5000)
        its_all = []
        for k, (dims, u, b) in enumerate(zip(DIMS_SET, us, bs)):
            eta, par = lat.eta(dims), lat.parity(dims)
            xs, its, per = solvers.multishift_cg(lambda v: dirac.a_op(u, v, mass, eta, par, 0.0), b, SHIFTS_8, 1e-12)
            got = host_complex(d_x[k]).reshape(len(SHIFTS_8), 3, -1)
            for s in range(len(SHIFTS_8)):
                assert L.rel_err(got[s], L.to_half(xs[s], dims, 0)) < 1e-10
            # float-float iteration (about 48 bits): near 1e-12 the recursive
            # residual drifts from the fp64 one and the crossing moves by a few
            assert abs(infos[k].iterations - its) <= 5, (k, infos[k].iterations, its)
            assert max(infos[k].true_residual[s] for s in range(len(SHIFTS_8))) < 1e-11
            its_all.append(its)
        print("iterations per lattice:", [i.iterations for i in infos], "oracle:", its_all)
        assert max(its_all) - min(its_all) > 20      # the lattices really converge at different counts
    finally:
        _destroy(stag, ctxs)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_mixed_batched_multishift_true_residual(torch, prec):
    from paper_1010_5433_gb300 import stag
    mass = 0.05
    dims_set = [(4, 4, 4, 4), (8, 8, 8, 8), (6, 6, 6, 4)]
    ctxs, us = _contexts(stag, dims_set, [221, 222, 223])
    try:
        bs = [syn.gaussian_fermion(d, 230 + k, on_parity=0) for k, d in enumerate(dims_set)]
        d_b = [dev(torch, L.to_half(b, d, 0)) for b, d in zip(bs, dims_set)]
        d_x = [torch.empty((len(SHIFTS_8),) + tuple(x.shape), dtype=torch.float64, device="cuda") for x in d_b]
        infos = stag.stag_multishift_solve_batch(ctxs, mass, SHIFTS_8, prec, d_b, d_x, 1e-6, 20000)
        for k, (dims, u, b) in enumerate(zip(dims_set, us, bs)):
            eta, par = lat.eta(dims), lat.parity(dims)
            got = host_complex(d_x[k]).reshape(len(SHIFTS_8), 3, -1)
            for s, sh in enumerate(SHIFTS_8):
                r = b - dirac.a_op(u, L.from_half(got[s], dims, 0), mass, eta, par, sh)
                res = np.linalg.norm(r) / np.linalg.norm(b)
                assert res < 1e-6 * 1.05, (k, s, res)
            if prec != 3:
                assert infos[k].reliable_updates >= 1
    finally:
        _destroy(stag, ctxs)


def test_batched_solve_matches_one_at_a_time(torch):
    """FP32 with reliable updates: the batched solutions agree with the
    single-lattice solver's to the solve tolerance, and so do the counts."""
    from paper_1010_5433_gb300 import stag
    mass = 0.05
    dims_set = [(8, 8, 8, 8), (4, 4, 4, 8), (6, 6, 6, 6)]
    ctxs, us = _contexts(stag, dims_set, [241, 242, 243])
    try:
        bs = [dev(torch, L.to_half(syn.gaussian_fermion(d, 250 + k, on_parity=0), d, 0))
              for k, d in enumerate(dims_set)]
        xb = [torch.empty((len(SHIFTS_8),) + tuple(b.shape), dtype=torch.float64, device="cuda") for b in bs]
        infos = stag.stag_multishift_solve_batch(ctxs, mass, SHIFTS_8, stag.STAG_FP32, bs, xb, 1e-9, 20000)
        for k in range(len(dims_set)):
            xs = torch.empty_like(xb[k])
            one = stag.stag_multishift_solve(ctxs[k], mass, SHIFTS_8, stag.STAG_FP32, 1, bs[k], xs, 1e-9, 20000)
            rel = float((xs - xb[k]).norm() / xs.norm())
            assert rel < 1e-8, (k, rel)
            assert abs(infos[k].shift_iterations[0] - one.shift_iterations[0]) <= 3
    finally:
        _destroy(stag, ctxs)


def _rat(d):
    return Rational(d["s"], d["lo"], d["hi"], d["a0"], d["alpha"], d["beta"], d["err"])


def _hmc(stag, g, prec, **kw):
    p = stag.stag_hmc()
    p.beta, p.tau, p.n_outer, p.n_gauge, p.n_flavours = 5.5, 0.5, 4, 2, 1
    fl = p.flavour[0]
    fl.mass, fl.n_pf = 0.1, 1
    for k in ("hb", "md", "met"):
        setattr(fl, k, stag.make_rational(g["c1_" + k]["a0"], g["c1_" + k]["alpha"], g["c1_" + k]["beta"]))
    p.tol_md = 1e-12 if prec == 0 else 1e-8
    p.tol_met, p.max_iter, p.md_prec = 1e-12, 20000, prec
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("prec,tol_dh,tol_u", [(0, 1e-7, 1e-10), (1, 2e-3, 1e-5)])
def test_trajectory_batch_matches_oracle(torch, prec, tol_dh, tol_u):
    """Three chains of different volumes, supplied momenta and sources: each
    chain's dH and final field against the oracle's trajectory."""
    from paper_1010_5433_gb300 import stag
    g = json.load(open(GOLDEN))
    dims_set = DIMS_SET[:3]
    ctxs, us = _contexts(stag, dims_set, [261, 262, 263], hot=False)
    try:
        moms, xis, keep, hmcs, wants = [], [], [], [], []
        for k, dims in enumerate(dims_set):
            mom0 = syn.gaussian_momenta(dims, 270 + k)
            xi = syn.gaussian_fermion(dims, 280 + k, on_parity=0)
            fl = integrator.Flavour(mass=0.1, hb=_rat(g["c1_hb"]), md=_rat(g["c1_md"]), met=_rat(g["c1_met"]))
            prm = integrator.HMCParams(dims=dims, beta=5.5, tau=0.5, n_outer=4, n_gauge=2, flavours=[fl],
                                       tol_md=1e-13, tol_met=1e-13)
            wants.append(integrator.trajectory(integrator.Context(prm), us[k], mom0, [[xi]]))
            d_mom = torch.from_numpy(L.mom_to_abi(mom0, dims)).cuda()
            d_xi = dev(torch, L.to_half(xi, dims, 0)[None])
            keep += [d_mom, d_xi]
            hmcs.append(_hmc(stag, g, prec, ext_mom=d_mom.data_ptr(), ext_xi=d_xi.data_ptr(), no_metropolis=1))
        outs = stag.stag_md_trajectory_batch(ctxs, hmcs)
        for k, dims in enumerate(dims_set):
            buf = np.empty(4 * int(np.prod(dims)) * 18)
            stag.stag_store_gauge(ctxs[k], buf)
            du = np.abs(L.gauge_from_host(buf, dims) - wants[k]["u"]).max()
            print(f"chain {k} {dims}: dH gpu {outs[k].dH:.8f} oracle {wants[k]['dH']:.8f} max|dU| {du:.2e}")
            assert abs(outs[k].H0 - wants[k]["H0"]) < 1e-8 * abs(wants[k]["H0"])
            assert abs(outs[k].dH - wants[k]["dH"]) < tol_dh
            assert du < tol_u
    finally:
        _destroy(stag, ctxs)


@pytest.mark.parametrize("prec", [0, 1])
def test_trajectory_batch_matches_sequential_chains(torch, prec):
    """Drawn momenta and sources (own seed and counter per chain): the
    batched trajectories reproduce the one-at-a-time ones, including the
    Metropolis decisions, over two trajectories."""
    from paper_1010_5433_gb300 import stag
    g = json.load(open(GOLDEN))
    dims_set = [(4, 4, 4, 4), (8, 8, 8, 8), (6, 6, 6, 4), (4, 4, 4, 8)]
    seq, _ = _contexts(stag, dims_set, [291, 292, 293, 294], hot=False)
    bat, _ = _contexts(stag, dims_set, [291, 292, 293, 294], hot=False)
    try:
        for traj in range(2):
            hmcs = [_hmc(stag, g, prec, seed=0x5A0004 + k, counter=traj) for k in range(len(dims_set))]
            outs = stag.stag_md_trajectory_batch(bat, hmcs)
            for k in range(len(dims_set)):
                one = stag.stag_md_trajectory(seq[k], hmcs[k])
                tol = 1e-8 if prec == 0 else 5e-4
                print(f"traj {traj} chain {k}: dH batch {outs[k].dH:.9f} single {one.dH:.9f}")
                assert abs(outs[k].dH - one.dH) < tol * max(1.0, abs(one.dH))
                assert outs[k].accepted == one.accepted
                assert abs(outs[k].plaq - one.plaq) < (1e-12 if prec == 0 else 1e-6)
    finally:
        _destroy(stag, seq + bat)


def test_batch_rejects_bad_arguments(torch):
    from paper_1010_5433_gb300 import stag
    g = json.load(open(GOLDEN))
    ctxs, _ = _contexts(stag, DIMS_SET[:2], [301, 302])
    try:
        with pytest.raises(stag.StagError):
            stag.stag_md_trajectory_batch([ctxs[0], ctxs[0]], [_hmc(stag, g, 1), _hmc(stag, g, 1)])
        with pytest.raises(stag.StagError):
            stag.stag_md_trajectory_batch(ctxs, [_hmc(stag, g, 1), _hmc(stag, g, 1, n_outer=5)])
        # one chain: the single-chain trajectory
        out = stag.stag_md_trajectory_batch(ctxs[:1], [_hmc(stag, g, 1, counter=3)])
        assert np.isfinite(out[0].dH)
    finally:
        _destroy(stag, ctxs)


def test_full_size_eight_chains_match_sequential(torch):
    """The batched-chains workload at its full sizes (2 x 8^4, 2 x 12^4,
    2 x 16^4, 2 x 16^3 x 8; N_f = 2, m = 0.05, beta = 5.5, 12-pole MD rational,
    fp32 MD) in the launch configuration batch_bench.py times: one batched
    trajectory of every chain against the same chains one at a time."""
    from paper_1010_5433_gb300 import batch_bench, rational, stag
    chains = batch_bench.CHAINS
    rats = {k: rational.load("c4_" + k) for k in ("md", "met", "hb")}

    def hmc(k):
        p = stag.stag_hmc()
        p.beta, p.tau, p.n_outer, p.n_gauge, p.n_flavours = 5.5, 1.0, 10, 5, 1
        fl = p.flavour[0]
        fl.mass, fl.n_pf = 0.05, 1
        fl.hb, fl.md, fl.met = rats["hb"].to_abi(), rats["md"].to_abi(), rats["met"].to_abi()
        p.tol_md, p.tol_met, p.max_iter, p.md_prec = 1e-8, 1e-12, 20000, stag.STAG_FP32
        p.seed, p.counter = 0x5A0004 + k, 0
        return p

    seeds = [600 + k for k in range(len(chains))]
    seq, _ = _contexts(stag, chains, seeds, hot=False)
    bat, _ = _contexts(stag, chains, seeds, hot=False)
    try:
        outs = stag.stag_md_trajectory_batch(bat, [hmc(k) for k in range(len(chains))])
        for k in range(len(chains)):
            one = stag.stag_md_trajectory(seq[k], hmc(k))
            print(f"chain {k} {chains[k]}: dH batch {outs[k].dH:.6f} single {one.dH:.6f}")
            assert abs(outs[k].dH - one.dH) < 1e-3 * max(1.0, abs(one.dH))
            assert outs[k].accepted == one.accepted
            assert abs(outs[k].plaq - one.plaq) < 1e-6
    finally:
        _destroy(stag, seq + bat)
