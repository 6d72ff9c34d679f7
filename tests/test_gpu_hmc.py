"""GPU parity of the whole RHMC trajectory (paper Sec. 2 and Sec. 4) against
the FP64 oracle on the 4^4 workload (supplied momenta and sources), FP32
reversibility (Sec. 4 reports ~5e-6 per degree of freedom), Metropolis
rejection restoring the field."""
import json
import os

import numpy as np
import pytest

import synthetic as syn
from oracle import integrator, lattice as lat
from oracle.rational import Rational
from tests import layout as L
from tests.gpu_util import dev, host_complex, torch_cuda, wrap_device

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rationals.json")
DIMS = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _rat(d):
    return Rational(d["s"], d["lo"], d["hi"], d["a0"], d["alpha"], d["beta"], d["err"])


@pytest.fixture(scope="module")
def c1():
    g = json.load(open(GOLDEN))
    return {k: g["c1_" + k] for k in ("md", "met", "hb")}


def _hmc(stag, c1, prec, n_outer=10, n_gauge=1, tau=1.0, **kw):
    p = stag.stag_hmc()
    p.beta, p.tau, p.n_outer, p.n_gauge = 5.5, tau, n_outer, n_gauge
    p.n_flavours = 1
    fl = p.flavour[0]
    fl.mass, fl.n_pf = 0.1, 1
    fl.hb = stag.make_rational(c1["hb"]["a0"], c1["hb"]["alpha"], c1["hb"]["beta"])
    fl.md = stag.make_rational(c1["md"]["a0"], c1["md"]["alpha"], c1["md"]["beta"])
    fl.met = stag.make_rational(c1["met"]["a0"], c1["met"]["alpha"], c1["met"]["beta"])
    p.tol_md = 1e-12 if prec == 0 else 1e-8
    p.tol_met = 1e-12
    p.max_iter = 20000
    p.md_prec = prec
    p.seed, p.counter = 0x5A0001, 0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.fixture(scope="module")
def oracle_traj(c1):
    u0 = syn.near_identity_gauge(DIMS, 0x5A0001)
    mom0 = syn.gaussian_momenta(DIMS, 101)
    xi = syn.gaussian_fermion(DIMS, 102, on_parity=0)
    fl = integrator.Flavour(mass=0.1, hb=_rat(c1["hb"]), md=_rat(c1["md"]), met=_rat(c1["met"]))
    prm = integrator.HMCParams(dims=DIMS, beta=5.5, tau=1.0, n_outer=10, n_gauge=1, flavours=[fl],
                               tol_md=1e-13, tol_met=1e-13)
    out = integrator.trajectory(integrator.Context(prm), u0, mom0, [[xi]])
    return u0, mom0, xi, out


@pytest.mark.parametrize("prec,tol_dh,tol_u", [(0, 1e-7, 1e-10), (1, 2e-3, 1e-5), (2, 2e-3, 1e-5), (3, 2e-2, 1e-4)])
def test_trajectory_matches_oracle(torch, c1, oracle_traj, prec, tol_dh, tol_u):
    from paper_1010_5433_gb300 import stag
    u0, mom0, xi, want = oracle_traj
    ctx = stag.stag_create(DIMS, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u0))
        d_mom = torch.from_numpy(L.mom_to_abi(mom0, DIMS)).cuda()
        d_xi = dev(torch, L.to_half(xi, DIMS, 0)[None])
        p = _hmc(stag, c1, prec, ext_mom=d_mom.data_ptr(), ext_xi=d_xi.data_ptr(), ext_uniform=0.5,
                 no_metropolis=1)
        res = stag.stag_md_trajectory(ctx, p)
        buf = np.empty(4 * 256 * 18)
        stag.stag_store_gauge(ctx, buf)
        u1 = L.gauge_from_host(buf, DIMS)
        assert abs(res.H0 - want["H0"]) < 1e-8 * abs(want["H0"])
        assert abs(res.dH - want["dH"]) < tol_dh, (res.dH, want["dH"])
        assert np.abs(u1 - want["u"]).max() < tol_u
        print(f"prec {prec}: dH gpu {res.dH:.8f} oracle {want['dH']:.8f}  max|dU| {np.abs(u1 - want['u']).max():.2e}"
              f"  iters {res.cg_iterations}")
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec,bound", [(0, 1e-12), (1, 5e-5)])
def test_reversibility(torch, c1, prec, bound):
    """Forward trajectory, flip the momenta, integrate back with the same
    pseudo-fermion field; violation per degree of freedom (rms over the
    18 reals of every link)."""
    from paper_1010_5433_gb300 import stag
    u0 = syn.near_identity_gauge(DIMS, 0x5A0001)
    ctx = stag.stag_create(DIMS, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u0))
        d_mom = torch.from_numpy(L.mom_to_abi(syn.gaussian_momenta(DIMS, 7), DIMS)).cuda()
        d_phi = dev(torch, L.to_half(syn.gaussian_fermion(DIMS, 8, on_parity=0), DIMS, 0)[None])
        p = _hmc(stag, c1, prec, ext_mom=d_mom.data_ptr(), ext_phi=d_phi.data_ptr(), no_metropolis=1)
        r1 = stag.stag_md_trajectory(ctx, p)
        tmp = wrap_device(torch, stag.stag_momenta(ctx), d_mom.numel()).clone().view_as(d_mom)
        p2 = _hmc(stag, c1, prec, ext_mom=tmp.data_ptr(), ext_phi=d_phi.data_ptr(), no_metropolis=1, flip_momenta=1)
        r2 = stag.stag_md_trajectory(ctx, p2)
        buf = np.empty(4 * 256 * 18)
        stag.stag_store_gauge(ctx, buf)
        u2 = L.gauge_from_host(buf, DIMS)
        viol = np.sqrt(np.mean(np.abs(u2 - u0) ** 2 * 0.5))
        print(f"prec {prec}: reversibility violation per dof {viol:.3e}; dH fwd {r1.dH:.3e} back {r2.dH:.3e}")
        assert viol < bound
        assert abs(r1.dH + r2.dH) < (1e-9 if prec == 0 else 1e-2)
    finally:
        stag.stag_destroy(ctx)


def test_metropolis_reject_restores_field(torch, c1):
    from paper_1010_5433_gb300 import stag
    u0 = syn.near_identity_gauge(DIMS, 0x5A0001)
    ctx = stag.stag_create(DIMS, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u0))
        d_mom = torch.from_numpy(3.0 * L.mom_to_abi(syn.gaussian_momenta(DIMS, 9), DIMS)).cuda()
        d_xi = dev(torch, L.to_half(syn.gaussian_fermion(DIMS, 10, on_parity=0), DIMS, 0)[None])
        p = _hmc(stag, c1, 1, n_outer=2, ext_mom=d_mom.data_ptr(), ext_xi=d_xi.data_ptr(), ext_uniform=1.0 - 1e-16)
        res = stag.stag_md_trajectory(ctx, p)
        buf = np.empty(4 * 256 * 18)
        stag.stag_store_gauge(ctx, buf)
        if res.dH > 0:
            assert res.accepted == 0
            assert np.abs(L.gauge_from_host(buf, DIMS) - u0).max() < 1e-14
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_drawn_trajectory_runs_and_is_reproducible(torch, c1, prec):
    """Two runs from the same seed and counter give the same dH bit for bit."""
    from paper_1010_5433_gb300 import stag
    u0 = syn.near_identity_gauge(DIMS, 0x5A0001)
    out = []
    for _ in range(2):
        ctx = stag.stag_create(DIMS, True)
        try:
            stag.stag_load_gauge(ctx, L.gauge_host(u0))
            out.append(stag.stag_md_trajectory(ctx, _hmc(stag, c1, prec, counter=5)))
        finally:
            stag.stag_destroy(ctx)
    assert out[0].dH == out[1].dH and out[0].accepted == out[1].accepted
    assert abs(out[0].dH) < 1.0


@pytest.mark.parametrize("prec,tol_dh", [(0, 1e-7), (3, 5e-2)])
def test_two_flavours_two_pseudofermions_match_oracle(torch, prec, tol_dh):
    """The N_f = 2+1 structure of the 32^3x8 workload on 4^4: a light flavour
    (m = 0.01... here 0.1) and a strange one, two pseudo-fermions each, the
    exponents s = 1/4 and 1/8 per pseudo-fermion, supplied momenta/sources."""
    from paper_1010_5433_gb300 import stag
    g = json.load(open(GOLDEN))
    dims = DIMS
    u0 = syn.near_identity_gauge(dims, 0x5A0003)
    mom0 = syn.gaussian_momenta(dims, 301)
    xis = [[syn.gaussian_fermion(dims, 310 + 2 * f + k, on_parity=0) for k in range(2)] for f in range(2)]
    # light: x^(-1/4) (c1 tables, m = 0.1); strange: x^(-1/8) at m = 0.1 built from c3's strange degree
    rat = {"light": {k: g["c1_" + k] for k in ("md", "met", "hb")},
           "strange": {k: g["c3_strange_" + k] for k in ("md", "met", "hb")}}
    fls = [integrator.Flavour(mass=0.1, hb=_rat(rat["light"]["hb"]), md=_rat(rat["light"]["md"]),
                              met=_rat(rat["light"]["met"]), n_pf=2),
           integrator.Flavour(mass=0.1, hb=_rat(rat["strange"]["hb"]), md=_rat(rat["strange"]["md"]),
                              met=_rat(rat["strange"]["met"]), n_pf=2)]
    prm = integrator.HMCParams(dims=dims, beta=5.3, tau=0.5, n_outer=5, n_gauge=2, flavours=fls,
                               tol_md=1e-13, tol_met=1e-13)
    want = integrator.trajectory(integrator.Context(prm), u0, mom0, xis)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u0))
        d_mom = torch.from_numpy(L.mom_to_abi(mom0, dims)).cuda()
        d_xi = dev(torch, np.stack([L.to_half(x, dims, 0) for xl in xis for x in xl]))
        p = stag.stag_hmc()
        p.beta, p.tau, p.n_outer, p.n_gauge, p.n_flavours = 5.3, 0.5, 5, 2, 2
        for f, name in enumerate(("light", "strange")):
            fl = p.flavour[f]
            fl.mass, fl.n_pf = 0.1, 2
            for k in ("hb", "md", "met"):
                setattr(fl, k, stag.make_rational(rat[name][k]["a0"], rat[name][k]["alpha"], rat[name][k]["beta"]))
        p.tol_md = 1e-12 if prec == 0 else 1e-8
        p.tol_met, p.max_iter, p.md_prec = 1e-12, 20000, prec
        p.ext_mom, p.ext_xi, p.no_metropolis = d_mom.data_ptr(), d_xi.data_ptr(), 1
        res = stag.stag_md_trajectory(ctx, p)
        buf = np.empty(4 * 256 * 18)
        stag.stag_store_gauge(ctx, buf)
        assert abs(res.H0 - want["H0"]) < 1e-8 * abs(want["H0"])
        assert abs(res.dH - want["dH"]) < tol_dh, (res.dH, want["dH"])
        assert np.abs(L.gauge_from_host(buf, dims) - want["u"]).max() < (1e-10 if prec == 0 else 1e-4)
        print(f"2+1 flavours prec {prec}: dH gpu {res.dH:.8f} oracle {want['dH']:.8f}")
    finally:
        stag.stag_destroy(ctx)


def test_bench_configuration_trajectory_is_reversible(torch):
    """The 16^4, N_f = 2, m = 0.02, beta = 5.6 trajectory in the launch
    configuration bench.py times (12-pole MD rational of the product table,
    n_outer 20 x n_gauge 5, fp32 MD on 12-real links), from a thermalised
    start (hot start, quenched and dynamical trajectories, as the bench's
    recipe but shorter): forward with supplied momenta and pseudo-fermions,
    then back from the flipped final momenta.  The fp64 path returns dH to
    1e-8; the fp32 link updates and forces leave ~5e-7 per degree of freedom
    in the links (the paper quotes ~5e-6 for its fp32 update, Sec. 4) and,
    measured on GB300, 2e-3 .. 4e-3 in dH_forward + dH_backward at H ~ 2e6;
    the bound is 1e-2, below the equilibrium <|dH|> of ~0.06 at these
    settings.  (From an ordered near-identity start the same fp32 sum reaches
    0.13 with 5 gauge substeps, 5e-4 with one: that start is far from where
    the workload runs.)"""
    from paper_1010_5433_gb300 import rational, stag
    dims = (16, 16, 16, 16)
    V = int(np.prod(dims))
    rats = {k: rational.load("c2_" + k) for k in ("md", "met", "hb")}
    ctx = stag.stag_create(dims, True)

    def hmc(prec, **kw):
        p = stag.stag_hmc()
        p.beta, p.tau, p.n_outer, p.n_gauge, p.n_flavours = 5.6, 1.0, 20, 5, 1
        fl = p.flavour[0]
        fl.mass, fl.n_pf = 0.02, 1
        fl.hb, fl.md, fl.met = rats["hb"].to_abi(), rats["md"].to_abi(), rats["met"].to_abi()
        p.tol_md, p.tol_met, p.max_iter, p.md_prec = (1e-12 if prec == 0 else 1e-8), 1e-12, 20000, prec
        p.seed = 91
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    try:
        stag.stag_load_gauge(ctx, L.gauge_host(syn.haar_gauge(dims, 0x5A0013)))
        for k in range(20):
            stag.stag_md_trajectory(ctx, hmc(2, n_flavours=0, counter=100 + k))
        for k in range(10):
            stag.stag_md_trajectory(ctx, hmc(2, n_outer=10, counter=200 + k))
        u0 = np.empty(4 * V * 18)
        stag.stag_store_gauge(ctx, u0)
        d_mom = torch.from_numpy(L.mom_to_abi(syn.gaussian_momenta(dims, 17), dims)).cuda()
        d_phi = dev(torch, L.to_half(syn.gaussian_fermion(dims, 18, on_parity=0), dims, 0)[None])
        for prec, bound_h, bound_u in ((stag.STAG_FP32_12, 1e-2, 5e-6), (stag.STAG_FP64, 1e-8, 1e-13)):
            stag.stag_load_gauge(ctx, u0)
            r1 = stag.stag_md_trajectory(ctx, hmc(prec, ext_mom=d_mom.data_ptr(), ext_phi=d_phi.data_ptr(),
                                                  no_metropolis=1))
            back = wrap_device(torch, stag.stag_momenta(ctx), d_mom.numel()).clone().view_as(d_mom)
            r2 = stag.stag_md_trajectory(ctx, hmc(prec, ext_mom=back.data_ptr(), ext_phi=d_phi.data_ptr(),
                                                  no_metropolis=1, flip_momenta=1))
            buf = np.empty(4 * V * 18)
            stag.stag_store_gauge(ctx, buf)
            viol = np.sqrt(np.mean((buf - u0) ** 2))
            print(f"16^4 bench configuration, prec {prec}: H0 {r1.H0:.1f}, dH {r1.dH:.5f} back {r2.dH:.5f}, sum "
                  f"{r1.dH + r2.dH:.2e}, reversibility per dof {viol:.2e}, CG iterations {r1.cg_iterations}")
            assert viol < bound_u
            assert abs(r1.dH + r2.dH) < bound_h
    finally:
        stag.stag_destroy(ctx)


def test_full_size_two_plus_one_flavours_bf16_links(torch):
    """The 32^3 x 8, beta = 5.3, N_f = 2+1 (m_l = 0.01, m_s = 0.1) workload at
    full size: 2 pseudo-fermions per flavour, 15-pole MD rationals, bf16 12-real
    links in the MD inversions (iterated without residual replacement), one
    n-RHS force Dslash over flavours x pseudo-fermions x shifts (60 sources),
    float-float Metropolis.  Forward with supplied momenta and pseudo-fermions
    (tau shortened to 0.25), then back from the flipped final momenta."""
    from paper_1010_5433_gb300 import rational, stag
    dims = (32, 32, 32, 8)
    rl = {k: rational.load("c3_light_" + k) for k in ("md", "met", "hb")}
    rs = {k: rational.load("c3_strange_" + k) for k in ("md", "met", "hb")}
    u0 = syn.near_identity_gauge(dims, 0x5A0003)
    ctx = stag.stag_create(dims, True)

    def hmc(**kw):
        p = stag.stag_hmc()
        p.beta, p.tau, p.n_outer, p.n_gauge, p.n_flavours = 5.3, 0.25, 2, 4, 2
        for f, (m, r) in enumerate(((0.01, rl), (0.1, rs))):
            fl = p.flavour[f]
            fl.mass, fl.n_pf = m, 2
            fl.hb, fl.md, fl.met = r["hb"].to_abi(), r["md"].to_abi(), r["met"].to_abi()
        p.tol_md, p.tol_met, p.max_iter, p.md_prec = 1e-8, 1e-12, 40000, stag.STAG_BF16_12
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u0))
        d_mom = torch.from_numpy(L.mom_to_abi(syn.gaussian_momenta(dims, 31), dims)).cuda()
        phis = np.stack([L.to_half(syn.gaussian_fermion(dims, 40 + k, on_parity=0), dims, 0) for k in range(4)])
        d_phi = dev(torch, phis)
        r1 = stag.stag_md_trajectory(ctx, hmc(ext_mom=d_mom.data_ptr(), ext_phi=d_phi.data_ptr(), no_metropolis=1))
        back = wrap_device(torch, stag.stag_momenta(ctx), d_mom.numel()).clone().view_as(d_mom)
        r2 = stag.stag_md_trajectory(ctx, hmc(ext_mom=back.data_ptr(), ext_phi=d_phi.data_ptr(), no_metropolis=1,
                                             flip_momenta=1))
        buf = np.empty(4 * int(np.prod(dims)) * 18)
        stag.stag_store_gauge(ctx, buf)
        viol = np.sqrt(np.mean(np.abs(L.gauge_from_host(buf, dims) - u0) ** 2 * 0.5))
        print(f"32^3x8 2+1 bf16: H0 {r1.H0:.1f}, dH {r1.dH:.5f} back {r2.dH:.5f}, reversibility per dof "
              f"{viol:.2e}, CG iterations {r1.cg_iterations}, {r1.seconds:.2f} s")
        assert viol < 1e-4
        assert abs(r1.dH + r2.dH) < 1e-2
        assert np.isfinite(r1.dH) and abs(r1.dH) < 50.0
    finally:
        stag.stag_destroy(ctx)


def _c2_hmc(stag, rats, prec, **kw):
    """The integrator and rationals of the 16^4 N_f = 2 workload: m = 0.02,
    beta = 5.6, tau = 1, 20 outer x 5 gauge minimum-norm steps, 12-pole MD and
    24-pole heatbath / Metropolis rationals, MD tolerance 1e-8 (1e-12 on the
    FP64 path, which the oracle comparison holds to 1e-7 in dH)."""
    p = stag.stag_hmc()
    p.beta, p.tau, p.n_outer, p.n_gauge, p.n_flavours = 5.6, 1.0, 20, 5, 1
    fl = p.flavour[0]
    fl.mass, fl.n_pf = 0.02, 1
    for k in ("hb", "md", "met"):
        setattr(fl, k, stag.make_rational(rats[k]["a0"], rats[k]["alpha"], rats[k]["beta"]))
    p.tol_md = 1e-12 if prec == 0 else 1e-8
    p.tol_met, p.max_iter, p.md_prec = 1e-12, 20000, prec
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _golden_8x4():
    import importlib.util
    here = os.path.dirname(GOLDEN)
    spec = importlib.util.spec_from_file_location("make_traj_8x4_c2", os.path.join(here, "make_traj_8x4_c2.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    return mk, json.load(open(os.path.join(here, "traj_8x4_c2.json")))


@pytest.mark.parametrize("prec,tol_dh,tol_u", [(0, 1e-7, 1e-10), (2, 5e-3, 1e-5), (1, 5e-3, 1e-5)])
def test_trajectory_at_the_16x4_settings_matches_oracle_on_8x4(torch, prec, tol_dh, tol_u):
    """One trajectory on 8^4 with the 16^4 workload's rationals, mass and
    integrator (20 x 5 steps, tau = 1) against the oracle's, stored by
    tests/golden/make_traj_8x4_c2.py from the same seeded links, momenta and
    heatbath source.  FP64: dH to 1e-7, links to 1e-10.  Mixed (fp32 MD
    inversions with fp64 reliable updates, fp32 link updates): the fp32
    rounding of ~400 link updates and of the MD force (relative ~4e-6, the
    solver's fp32 operator) moves the links by a few 1e-6 and dH by ~1e-3 on
    this lattice; the bounds are 5e-3 and 1e-5."""
    from paper_1010_5433_gb300 import stag
    mk, gold = _golden_8x4()
    dims, u0, mom0, xi = mk.inputs(gold["setup"])
    rats = {k: json.load(open(GOLDEN))["c2_" + k] for k in ("md", "met", "hb")}
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u0))
        d_mom = torch.from_numpy(L.mom_to_abi(mom0, dims)).cuda()
        d_xi = dev(torch, L.to_half(xi, dims, 0)[None])
        res = stag.stag_md_trajectory(ctx, _c2_hmc(stag, rats, prec, ext_mom=d_mom.data_ptr(),
                                                   ext_xi=d_xi.data_ptr(), no_metropolis=1))
        buf = np.empty(4 * int(np.prod(dims)) * 18)
        stag.stag_store_gauge(ctx, buf)
        u1 = L.gauge_from_host(buf, dims)
        got = np.array([u1[tuple(q)].reshape(-1) for q in gold["u_sample_pos"]])
        want = np.array([[complex(*v) for v in row] for row in gold["u_sample"]])
        du = np.abs(got - want).max()
        print(f"8^4 c2 settings prec {prec}: dH gpu {res.dH:.9f} oracle {gold['dH']:.9f}, max|dU| {du:.2e}, "
              f"CG iterations {res.cg_iterations}")
        assert abs(res.H0 - gold["H0"]) < 1e-10 * abs(gold["H0"])
        assert abs(res.dH - gold["dH"]) < tol_dh
        assert du < tol_u
    finally:
        stag.stag_destroy(ctx)


def test_fp64_and_mixed_paths_integrate_alike_at_16x4(torch):
    """The two arms of the trajectories/hour comparison from identical links,
    momenta and heatbath source at the 16^4 workload's settings: the FP64 path
    and the mixed path (fp32 MD inversions on 12-real links with fp64
    reliable updates) end at the same links to 1e-4 and the same dH to 1e-2
    (measured on GB300: 4.5e-6 and 3.6e-3 at |dH| ~ 0.2, H ~ 2e6), so a
    difference in their |dH| statistics can only come from the random
    numbers or the start, not from the integration."""
    from paper_1010_5433_gb300 import rational, stag
    dims = (16, 16, 16, 16)
    V = int(np.prod(dims))
    rats = {k: rational.load("c2_" + k) for k in ("md", "met", "hb")}
    rj = {k: {"a0": r.a0, "alpha": list(r.alpha), "beta": list(r.beta)} for k, r in rats.items()}
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(syn.haar_gauge(dims, 0x5A0012)))
        for k in range(20):                       # quenched trajectories away from the hot start
            q = stag.stag_hmc()
            q.beta, q.tau, q.n_outer, q.n_gauge, q.n_flavours = 5.6, 1.0, 20, 5, 0
            q.tol_md, q.tol_met, q.max_iter, q.md_prec, q.seed, q.counter = 1e-8, 1e-12, 100, 2, 5, k
            stag.stag_md_trajectory(ctx, q)
        start = np.empty(4 * V * 18)
        stag.stag_store_gauge(ctx, start)
        d_mom = torch.from_numpy(L.mom_to_abi(syn.gaussian_momenta(dims, 1201), dims)).cuda()
        d_xi = dev(torch, L.to_half(syn.gaussian_fermion(dims, 1202, on_parity=0), dims, 0)[None])
        out = {}
        for prec in (0, 2):
            stag.stag_load_gauge(ctx, start)
            r = stag.stag_md_trajectory(ctx, _c2_hmc(stag, rj, prec, ext_mom=d_mom.data_ptr(),
                                                     ext_xi=d_xi.data_ptr(), no_metropolis=1, tol_md=1e-8))
            buf = np.empty(4 * V * 18)
            stag.stag_store_gauge(ctx, buf)
            out[prec] = (r, buf)
        (r64, u64), (r32, u32) = out[0], out[2]
        du = np.abs(u64 - u32).max()
        print(f"16^4 paired arms: H0 {r64.H0:.3f} / {r32.H0:.3f}, dH fp64 {r64.dH:.6f} mixed {r32.dH:.6f}, "
              f"max|dU| {du:.2e}")
        assert abs(r64.H0 - r32.H0) < 1e-9 * abs(r64.H0)
        assert abs(r64.dH - r32.dH) < 1e-2
        assert du < 1e-4
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec,tol_dh,tol_u", [(0, 1e-7, 1e-10), (2, 5e-3, 1e-5)])
def test_hasenbusch_split_trajectory_matches_oracle(torch, prec, tol_dh, tol_u):
    """A Hasenbusch mass split on 4^4: the ratio term ((x + delta) / x)^(1/2)
    at m = 0.1 on the outer level, the heavy term x^(-1/2) at m_h = 0.4 on
    a middle level of n_mid = 2 steps around the gauge level, against the
    oracle's three-level integrator (supplied momenta and sources).  FP64: dH
    to 1e-7, links to 1e-10; mixed (fp32 MD on 12-real links): the bounds of
    the other mixed-path trajectory tests."""
    from oracle import rational as orat
    from paper_1010_5433_gb300 import stag
    m, mh = 0.1, 0.4
    delta = mh * mh - m * m
    lo, hi, loh, hih = m * m, 16 + m * m, mh * mh, 16 + mh * mh
    # the ratio is smooth enough that 8 poles reach ~2e-13: at 12 poles the
    # levelled-error system of the oracle's Remez becomes singular at 40 digits
    ratio = {"md": orat.remez(0.5, lo, hi, 6, dps=40, delta=delta),
             "met": orat.remez(0.5, lo, hi, 8, dps=40, delta=delta),
             "hb": orat.remez(-0.25, lo, hi, 8, dps=40, delta=delta)}
    heavy = {"md": orat.remez(0.5, loh, hih, 6, dps=40),
             "met": orat.remez(0.5, loh, hih, 12, dps=40),
             "hb": orat.remez(-0.25, loh, hih, 12, dps=40)}
    dims = DIMS
    u0 = syn.near_identity_gauge(dims, 0x5A0004)
    mom0 = syn.gaussian_momenta(dims, 401)
    xis = [[syn.gaussian_fermion(dims, 402, on_parity=0)], [syn.gaussian_fermion(dims, 403, on_parity=0)]]
    fls = [integrator.Flavour(mass=m, hb=ratio["hb"], md=ratio["md"], met=ratio["met"], level=0),
           integrator.Flavour(mass=mh, hb=heavy["hb"], md=heavy["md"], met=heavy["met"], level=1)]
    prm = integrator.HMCParams(dims=dims, beta=5.5, tau=0.5, n_outer=3, n_gauge=2, flavours=fls,
                               tol_md=1e-13, tol_met=1e-13)
    want = integrator.trajectory(integrator.Context(prm), u0, mom0, xis, n_mid=2)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u0))
        d_mom = torch.from_numpy(L.mom_to_abi(mom0, dims)).cuda()
        d_xi = dev(torch, np.stack([L.to_half(x[0], dims, 0) for x in xis]))
        p = stag.stag_hmc()
        p.beta, p.tau, p.n_outer, p.n_gauge, p.n_flavours, p.n_mid = 5.5, 0.5, 3, 2, 2, 2
        for f, (mass, lev, r) in enumerate(((m, 0, ratio), (mh, 1, heavy))):
            fl = p.flavour[f]
            fl.mass, fl.n_pf, fl.level = mass, 1, lev
            for k in ("hb", "md", "met"):
                setattr(fl, k, stag.make_rational(r[k].a0, r[k].alpha, r[k].beta))
        p.tol_md = 1e-12 if prec == 0 else 1e-8
        p.tol_met, p.max_iter, p.md_prec = 1e-12, 20000, prec
        p.ext_mom, p.ext_xi, p.no_metropolis = d_mom.data_ptr(), d_xi.data_ptr(), 1
        res = stag.stag_md_trajectory(ctx, p)
        buf = np.empty(4 * 256 * 18)
        stag.stag_store_gauge(ctx, buf)
        du = np.abs(L.gauge_from_host(buf, dims) - want["u"]).max()
        print(f"Hasenbusch split prec {prec}: dH gpu {res.dH:.9f} oracle {want['dH']:.9f}, max|dU| {du:.2e}")
        assert abs(res.H0 - want["H0"]) < 1e-8 * abs(want["H0"])
        assert abs(res.dH - want["dH"]) < tol_dh
        assert du < tol_u
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_updated_links_are_special_unitary_to_double_precision(torch, c1, prec):
    """After a trajectory without Metropolis (so the field is the MD result),
    every link held in the two-float store (hi + lo) is special unitary to
    double precision: the fp64 path reunitarises in fp64, the fp32 paths in
    float-float (about 2^-46 from orthonormal), Sec. 4."""
    from paper_1010_5433_gb300 import stag
    u0 = syn.near_identity_gauge(DIMS, 0x5A0001)
    ctx = stag.stag_create(DIMS, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u0))
        stag.stag_md_trajectory(ctx, _hmc(stag, c1, prec, counter=7, no_metropolis=1))
        buf = np.empty(4 * 256 * 18)
        stag.stag_store_gauge(ctx, buf)
        u = L.gauge_from_host(buf, DIMS).reshape(-1, 3, 3)
        assert np.abs(u - u0.reshape(-1, 3, 3)).max() > 1e-3          # the links moved
        eye = np.eye(3)
        unit = np.abs(np.einsum("nij,nkj->nik", u, u.conj()) - eye).max()
        det = np.abs(np.linalg.det(u) - 1.0).max()
        print(f"prec {prec}: max |U U^dag - 1| {unit:.2e}, max |det U - 1| {det:.2e}")
        assert unit < 1e-12 and det < 1e-12
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 2])
def test_updated_field_survives_store_and_load_bit_for_bit(torch, c1, prec):
    """The links an MD evolution leaves in the two-float store are exactly
    the doubles a store returns: store, load, store gives the same doubles,
    and the fp32 and fp64 Dslash of the reloaded field equal those of the
    evolved one bit for bit (the end-to-end path reloads the field between
    trajectories)."""
    from paper_1010_5433_gb300 import stag
    u0 = syn.near_identity_gauge(DIMS, 0x5A0001)
    psi = L.to_half(syn.gaussian_fermion(DIMS, 104, on_parity=1), DIMS, 1)
    ctx = stag.stag_create(DIMS, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u0))
        stag.stag_md_trajectory(ctx, _hmc(stag, c1, prec, counter=9, no_metropolis=1))
        outs, stores = [], []
        for _ in range(2):
            for dprec, arr in ((0, psi), (1, psi.astype(np.complex64)), (2, psi.astype(np.complex64))):
                d_in = dev(torch, arr)
                d_out = torch.empty_like(d_in)
                stag.stag_dslash(ctx, 0, dprec, 1, d_in, d_out)
                outs.append(d_out.cpu().numpy())
            buf = np.empty(4 * 256 * 18)
            stag.stag_store_gauge(ctx, buf)
            stores.append(buf.copy())
            stag.stag_load_gauge(ctx, buf)
        assert np.array_equal(stores[0], stores[1])
        for a, b in zip(outs[:3], outs[3:]):
            assert np.array_equal(a, b)
    finally:
        stag.stag_destroy(ctx)
