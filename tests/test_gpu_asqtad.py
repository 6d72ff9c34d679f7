"""GPU parity of the improved (asqtad) staggered operator against the FP64
oracle (oracle/asqtad.py), through the C ABI: the fat and Naik links, the
Dslash on both parities and in both precisions, A and its no-allocation
form, the multi-shift solves, the fermion force through the fat-link paths,
and whole trajectories (FP64 parity, FP32 reversibility)."""
import json
import os

import numpy as np
import pytest

import synthetic as syn
from oracle import asqtad, integrator, lattice as lat, solvers
from oracle.rational import Rational
from tests import layout as L
from tests.gpu_util import dev, host_complex, torch_cuda, wrap_device

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rationals.json")
TOL = {0: 1e-10, 1: 2e-6}
# ragged volumes (Vh not a multiple of the block), a side of 2 (the third
# neighbour wraps onto the first), an odd-shaped lattice, and 8^4 / 16^4
CASES = [((4, 4, 4, 4), 1, 1.0), ((2, 4, 6, 8), 2, 0.9), ((6, 2, 4, 10), 3, 0.85), ((8, 8, 8, 8), 4, 1.0),
         ((16, 16, 16, 16), 5, 0.88)]


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _gauge(dims, seed):
    return syn.haar_gauge(dims, seed) if seed % 2 else syn.near_identity_gauge(dims, seed, width=0.5)


def _ctx(stag, dims, u, u0):
    ctx = stag.stag_create(dims, True)
    stag.stag_load_gauge(ctx, L.gauge_host(u))
    stag.stag_set_action(ctx, stag.STAG_ACTION_ASQTAD, u0)
    return ctx


def _round32(a):
    return a.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("dims,seed,u0", CASES[:4])
def test_fat_and_naik_links_match_oracle(torch, dims, seed, u0):
    from paper_1010_5433_gb300 import stag
    u = _gauge(dims, seed)
    ctx = _ctx(stag, dims, u, u0)
    try:
        vol = int(np.prod(dims))
        fat, naik = np.empty(4 * vol * 18), np.empty(4 * vol * 18)
        stag.stag_asqtad_links(ctx, fat, naik)
        v, w = asqtad.fat_long_links(u, u0, antiperiodic_t=False)    # the stores carry no boundary sign
        assert np.abs(L.gauge_from_host(fat, dims) - v).max() < 1e-13
        assert np.abs(L.gauge_from_host(naik, dims) - w).max() < 1e-14
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("dims,seed,u0", CASES)
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("out_par", [0, 1])
def test_dslash_matches_oracle(torch, dims, seed, u0, prec, out_par):
    from paper_1010_5433_gb300 import stag
    if dims[0] == 16 and out_par == 1:
        pytest.skip("16^4: one parity is enough")
    u = _gauge(dims, seed)
    psi = syn.gaussian_fermion(dims, seed + 100, on_parity=1 - out_par)
    ctx = _ctx(stag, dims, u, u0)
    try:
        h_in = L.to_half(psi, dims, 1 - out_par)
        d_in = dev(torch, h_in if prec == 0 else h_in.astype(np.complex64))
        d_out = torch.empty_like(d_in)
        stag.stag_dslash(ctx, out_par, prec, 1, d_in, d_out)
        torch.cuda.synchronize()
        got = host_complex(d_out).reshape(3, -1)
        v, w = asqtad.fat_long_links(u, u0, antiperiodic_t=True)
        psi_used = psi
        if prec == 1:      # the fp32 kernel reads the fat and Naik links' hi words and fp32 spinors
            v, w, psi_used = _round32(v), _round32(w), _round32(psi)
        # v, w carry the boundary signs here, so eta without them
        eta0, par = lat.eta(dims, antiperiodic_t=False), lat.parity(dims)
        want = L.to_half(asqtad.d_block(v, w, psi_used, eta0, par, out_par), dims, out_par)
        assert L.rel_err(got, want) < TOL[prec]
        assert np.abs(got - want).max() < 20 * TOL[prec] * np.abs(want).max()
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_multi_rhs_equals_single(torch, prec):
    """Five sources in one launch (each link load shared by four of them) give
    every source's single-source result bit for bit."""
    from paper_1010_5433_gb300 import stag
    dims = (4, 6, 4, 8)
    u = _gauge(dims, 7)
    ctx = _ctx(stag, dims, u, 0.9)
    try:
        srcs = np.stack([L.to_half(syn.gaussian_fermion(dims, 70 + k, on_parity=0), dims, 0) for k in range(5)])
        d_in = dev(torch, srcs if prec == 0 else srcs.astype(np.complex64))
        d_all = torch.empty_like(d_in)
        stag.stag_dslash(ctx, 1, prec, 5, d_in, d_all)
        for k in range(5):
            d_one = torch.empty_like(d_in[k:k + 1])
            stag.stag_dslash(ctx, 1, prec, 1, d_in[k:k + 1].contiguous(), d_one)
            assert torch.equal(d_one[0], d_all[k])
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_a_and_noalloc_match_oracle(torch, prec):
    from paper_1010_5433_gb300 import stag
    dims = (4, 4, 6, 4)
    u = _gauge(dims, 9)
    mass, shift = 0.15, 0.3
    psi = syn.gaussian_fermion(dims, 90, on_parity=0)
    ctx = _ctx(stag, dims, u, 0.92)
    try:
        h = L.to_half(psi, dims, 0)[None]
        d_in = dev(torch, h if prec == 0 else h.astype(np.complex64))
        d_a, d_n = torch.empty_like(d_in), torch.empty_like(d_in)
        stag.stag_apply_a(ctx, mass, shift, prec, 1, d_in, d_a)
        stag.stag_apply_a_noalloc(ctx, mass, shift, prec, 1, d_in, d_n)
        torch.cuda.synchronize()
        v, w = asqtad.fat_long_links(u, 0.92, antiperiodic_t=True)
        psi_used = psi
        if prec == 1:
            v, w, psi_used = _round32(v), _round32(w), _round32(psi)
        want = L.to_half(asqtad.a_op(v, w, psi_used, mass, lat.eta(dims, antiperiodic_t=False), lat.parity(dims),
                                     shift), dims, 0)
        for d in (d_a, d_n):
            assert L.rel_err(host_complex(d).reshape(3, -1), want) < TOL[prec]
    finally:
        stag.stag_destroy(ctx)


SHIFTS = [0.0, 0.002, 0.01, 0.05, 0.3, 1.4, 6.0, 30.0]


def _oracle_ops(u, u0, dims):
    v, w = asqtad.fat_long_links(u, u0, antiperiodic_t=True)
    return v, w, lat.eta(dims, antiperiodic_t=False), lat.parity(dims)


@pytest.mark.parametrize("dims,nrhs", [((4, 4, 4, 4), 1), ((4, 6, 4, 8), 2)])
def test_fp64_multishift_matches_oracle(torch, dims, nrhs):
    from paper_1010_5433_gb300 import stag
    u = _gauge(dims, 11)
    mass = 0.1
    bs = [syn.gaussian_fermion(dims, 110 + k, on_parity=0) for k in range(nrhs)]
    ctx = _ctx(stag, dims, u, 0.9)
    try:
        d_b = dev(torch, np.stack([L.to_half(b, dims, 0) for b in bs]))
        d_x = torch.empty((nrhs, len(SHIFTS)) + tuple(d_b.shape[1:]), dtype=torch.float64, device="cuda")
        info = stag.stag_multishift_solve(ctx, mass, SHIFTS, stag.STAG_FP64, nrhs, d_b, d_x, 1e-12, 5000)
        got = host_complex(d_x).reshape(nrhs, len(SHIFTS), 3, -1)
        v, w, eta0, par = _oracle_ops(u, 0.9, dims)
        for k, b in enumerate(bs):
            xs, _, _ = solvers.multishift_cg(lambda y: asqtad.a_op(v, w, y, mass, eta0, par), b, SHIFTS, 1e-13)
            for s in range(len(SHIFTS)):
                assert L.rel_err(got[k, s], L.to_half(xs[s], dims, 0)) < 1e-10
        assert max(info.true_residual[s] for s in range(len(SHIFTS))) < 1e-11
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8)])
def test_mixed_multishift_true_residual(torch, dims):
    """fp32 Dslash with fp64 reliable updates: every shift's true residual,
    recomputed with the oracle's operator, within 1e-5 relative of the FP64
    tolerance the solve was asked for (1e-6)."""
    from paper_1010_5433_gb300 import stag
    u = _gauge(dims, 13)
    mass = 0.05
    b = syn.gaussian_fermion(dims, 130, on_parity=0)
    ctx = _ctx(stag, dims, u, 1.0)
    try:
        d_b = dev(torch, L.to_half(b, dims, 0)[None])
        d_x = torch.empty((1, len(SHIFTS)) + tuple(d_b.shape[1:]), dtype=torch.float64, device="cuda")
        info = stag.stag_multishift_solve(ctx, mass, SHIFTS, stag.STAG_FP32, 1, d_b, d_x, 1e-6, 20000)
        got = host_complex(d_x).reshape(len(SHIFTS), 3, -1)
        v, w, eta0, par = _oracle_ops(u, 1.0, dims)
        for s, sh in enumerate(SHIFTS):
            x = L.from_half(got[s], dims, 0)
            r = b - asqtad.a_op(v, w, x, mass, eta0, par, sh)
            assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-5, (s, info.true_residual[s])
        assert info.reliable_updates >= 1
    finally:
        stag.stag_destroy(ctx)


def _rat(d):
    return Rational(d["s"], d["lo"], d["hi"], d["a0"], d["alpha"], d["beta"], d["err"])


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 2e-5)])
def test_fermion_force_matches_oracle(torch, prec, tol):
    from paper_1010_5433_gb300 import stag
    dims = (4, 4, 4, 6)
    u = _gauge(dims, 15)
    u0 = 0.9
    rat = json.load(open(GOLDEN))["c1_md"]
    mass = 0.1
    phis = [syn.gaussian_fermion(dims, 150 + k, on_parity=0) for k in range(2)]
    ctx = _ctx(stag, dims, u, u0)
    try:
        r = stag.make_rational(rat["a0"], rat["alpha"], rat["beta"])
        d_phi = dev(torch, np.stack([L.to_half(p, dims, 0) for p in phis]))
        f = torch.empty((4, 2, 8, int(np.prod(dims)) // 2), dtype=torch.float64, device="cuda")
        stag.stag_fermion_force(ctx, mass, r, prec, 2, d_phi, f, 1e-12 if prec == 0 else 1e-8, 10000)
        got = L.mom_from_abi(f.cpu().numpy(), dims)
        v, w, eta0, par = _oracle_ops(u, u0, dims)
        want = np.zeros_like(got)
        for p in phis:
            xs = solvers.multishift_cg(lambda y: asqtad.a_op(v, w, y, mass, eta0, par, min(rat["beta"])), p,
                                       rat["beta"], 1e-13)[0]
            want += asqtad.fermion_force(u, xs, rat["alpha"], par, u0, True)
        err = float(np.linalg.norm((got - want).ravel()) / np.linalg.norm(want.ravel()))
        assert err < tol, err
    finally:
        stag.stag_destroy(ctx)


DIMS = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def c1():
    g = json.load(open(GOLDEN))
    return {k: g["c1_" + k] for k in ("md", "met", "hb")}


def _hmc(stag, c1, prec, n_outer=4, **kw):
    p = stag.stag_hmc()
    p.beta, p.tau, p.n_outer, p.n_gauge = 5.5, 0.5, n_outer, 1
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
    for k, val in kw.items():
        setattr(p, k, val)
    return p


@pytest.fixture(scope="module")
def oracle_traj(c1):
    u0 = syn.near_identity_gauge(DIMS, 0x5A0001)
    mom0 = syn.gaussian_momenta(DIMS, 201)
    xi = syn.gaussian_fermion(DIMS, 202, on_parity=0)
    fl = integrator.Flavour(mass=0.1, hb=_rat(c1["hb"]), md=_rat(c1["md"]), met=_rat(c1["met"]))
    prm = integrator.HMCParams(dims=DIMS, beta=5.5, tau=0.5, n_outer=4, n_gauge=1, flavours=[fl],
                               tol_md=1e-13, tol_met=1e-13, action="asqtad", u0=0.9)
    out = integrator.trajectory(integrator.Context(prm), u0, mom0, [[xi]])
    return u0, mom0, xi, out


@pytest.mark.parametrize("prec,tol_dh,tol_u", [(0, 1e-7, 1e-10), (1, 2e-3, 1e-5)])
def test_trajectory_matches_oracle(torch, c1, oracle_traj, prec, tol_dh, tol_u):
    from paper_1010_5433_gb300 import stag
    u0, mom0, xi, want = oracle_traj
    ctx = _ctx(stag, DIMS, u0, 0.9)
    try:
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
        print(f"asqtad prec {prec}: dH gpu {res.dH:.8f} oracle {want['dH']:.8f}  "
              f"max|dU| {np.abs(u1 - want['u']).max():.2e}  iters {res.cg_iterations}")
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec,bound", [(0, 1e-12), (1, 5e-5)])
def test_reversibility(torch, c1, prec, bound):
    from paper_1010_5433_gb300 import stag
    u0 = syn.near_identity_gauge(DIMS, 0x5A0001)
    ctx = _ctx(stag, DIMS, u0, 1.0)
    try:
        d_mom = torch.from_numpy(L.mom_to_abi(syn.gaussian_momenta(DIMS, 17), DIMS)).cuda()
        d_phi = dev(torch, L.to_half(syn.gaussian_fermion(DIMS, 18, on_parity=0), DIMS, 0)[None])
        p = _hmc(stag, c1, prec, n_outer=5, ext_mom=d_mom.data_ptr(), ext_phi=d_phi.data_ptr(), no_metropolis=1)
        r1 = stag.stag_md_trajectory(ctx, p)
        tmp = wrap_device(torch, stag.stag_momenta(ctx), d_mom.numel()).clone().view_as(d_mom)
        p2 = _hmc(stag, c1, prec, n_outer=5, ext_mom=tmp.data_ptr(), ext_phi=d_phi.data_ptr(), no_metropolis=1,
                  flip_momenta=1)
        r2 = stag.stag_md_trajectory(ctx, p2)
        buf = np.empty(4 * 256 * 18)
        stag.stag_store_gauge(ctx, buf)
        viol = np.sqrt(np.mean(np.abs(L.gauge_from_host(buf, DIMS) - u0) ** 2 * 0.5))
        print(f"asqtad prec {prec}: reversibility per dof {viol:.3e}; dH fwd {r1.dH:.3e} back {r2.dH:.3e}")
        assert viol < bound
        assert abs(r1.dH + r2.dH) < (1e-9 if prec == 0 else 1e-2)
    finally:
        stag.stag_destroy(ctx)


def test_unsupported_combinations_are_refused(torch):
    """12-real and bf16 links (the fat links are not unitary) and the batched
    solver return STAG_ERR_ARG with the improved operator; switching back to
    the unimproved operator restores the paper's Dslash."""
    from paper_1010_5433_gb300 import stag
    dims = (4, 4, 4, 4)
    u = _gauge(dims, 19)
    ctx = _ctx(stag, dims, u, 1.0)
    try:
        d_in = dev(torch, L.to_half(syn.gaussian_fermion(dims, 190, on_parity=0), dims, 0).astype(np.complex64))
        d_out = torch.empty_like(d_in)
        for prec in (2, 3):
            with pytest.raises(stag.StagError) as e:
                stag.stag_dslash(ctx, 1, prec, 1, d_in, d_out)
            assert e.value.status == 1
        d_b = dev(torch, L.to_half(syn.gaussian_fermion(dims, 191, on_parity=0), dims, 0)[None])
        d_x = torch.empty((1, 2) + tuple(d_b.shape[1:]), dtype=torch.float64, device="cuda")
        st = stag.stag_multishift_solve_batch([ctx], 0.1, [0.0, 0.5], 0, [d_b], [d_x], 1e-10, 1000, check=False)
        assert (st[0] if isinstance(st, tuple) else st) == 1
        stag.stag_set_action(ctx, stag.STAG_ACTION_UNIMPROVED)
        stag.stag_dslash(ctx, 1, 1, 1, d_in, d_out)
        torch.cuda.synchronize()
        from oracle import dirac
        psi = L.from_half(host_complex(d_in).reshape(3, -1).astype(np.complex128), dims, 0)
        want = L.to_half(dirac.d_block(_round32(u), psi, lat.eta(dims), lat.parity(dims), 1), dims, 1)
        assert L.rel_err(host_complex(d_out).reshape(3, -1), want) < 2e-6
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_force_reverse_pass_equals_gather(torch, prec, tol):
    """The force as the reverse pass through the nested staples (the default)
    and as the per-link gather over the 508 path incidences of each direction
    (STAG_ASQ_FORCE=gather) are the same sum in two orders."""
    from paper_1010_5433_gb300 import stag
    dims = (4, 6, 4, 4)
    u = _gauge(dims, 21)
    rat = json.load(open(GOLDEN))["c1_md"]
    phi = syn.gaussian_fermion(dims, 210, on_parity=0)
    r = stag.make_rational(rat["a0"], rat["alpha"], rat["beta"])
    d_phi = dev(torch, L.to_half(phi, dims, 0)[None])
    forces = []
    for mode in ("", "gather"):
        os.environ["STAG_ASQ_FORCE"] = mode
        try:
            ctx = _ctx(stag, dims, u, 0.87)
        finally:
            os.environ.pop("STAG_ASQ_FORCE", None)
        try:
            f = torch.empty((4, 2, 8, int(np.prod(dims)) // 2), dtype=torch.float64, device="cuda")
            stag.stag_fermion_force(ctx, 0.1, r, prec, 1, d_phi, f, 1e-12 if prec == 0 else 1e-8, 10000)
            forces.append(f.cpu().numpy())
        finally:
            stag.stag_destroy(ctx)
    err = np.linalg.norm(forces[0] - forces[1]) / np.linalg.norm(forces[1])
    assert err < tol, err


def _golden_8x4_asqtad():
    import importlib.util
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_traj_8x4_asqtad",
                                                  os.path.join(here, "make_traj_8x4_asqtad.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    return mk, json.load(open(os.path.join(here, "traj_8x4_asqtad.json")))


@pytest.mark.parametrize("prec,tol_dh,tol_u", [(0, 1e-7, 1e-10), (1, 5e-3, 1e-5)])
def test_trajectory_at_the_workload_settings_matches_oracle_on_8x4(torch, prec, tol_dh, tol_u):
    """One improved-operator trajectory on 8^4 with the 16^4 workload's
    rationals (14-pole MD, 24-pole heatbath and Metropolis on [m^2, m^2 + 64]),
    mass 0.02 and integrator (10 x 5 minimum-norm steps, tau = 1) against the
    oracle's, stored by tests/golden/make_traj_8x4_asqtad.py from the same
    seeded links, momenta and heatbath source.  FP64: dH to 1e-7, links to
    1e-10; mixed (fp32 MD inversions with fp64 reliable updates on fp32-built
    fat links, fp32 link updates): 5e-3 and 1e-5."""
    from paper_1010_5433_gb300 import stag
    mk, gold = _golden_8x4_asqtad()
    s = gold["setup"]
    dims, u0, mom0, xi = mk.inputs(s)
    g = json.load(open(GOLDEN))
    rats = {k: g["asqtad_" + k] for k in ("md", "met", "hb")}
    ctx = _ctx(stag, dims, u0, s["u0"])
    try:
        d_mom = torch.from_numpy(L.mom_to_abi(mom0, dims)).cuda()
        d_xi = dev(torch, L.to_half(xi, dims, 0)[None])
        p = stag.stag_hmc()
        p.beta, p.tau, p.n_outer, p.n_gauge = s["beta"], s["tau"], s["n_outer"], s["n_gauge"]
        p.n_flavours = 1
        fl = p.flavour[0]
        fl.mass, fl.n_pf = s["mass"], 1
        for k in ("hb", "md", "met"):
            setattr(fl, k, stag.make_rational(rats[k]["a0"], rats[k]["alpha"], rats[k]["beta"]))
        p.tol_md = 1e-12 if prec == 0 else 1e-8
        p.tol_met = 1e-12
        p.max_iter = 40000
        p.md_prec = prec
        p.ext_mom, p.ext_xi, p.no_metropolis = d_mom.data_ptr(), d_xi.data_ptr(), 1
        res = stag.stag_md_trajectory(ctx, p)
        buf = np.empty(4 * int(np.prod(dims)) * 18)
        stag.stag_store_gauge(ctx, buf)
        u1 = L.gauge_from_host(buf, dims)
        got = np.array([u1[tuple(q)].reshape(-1) for q in gold["u_sample_pos"]])
        want = np.array([[complex(*v) for v in row] for row in gold["u_sample"]])
        du = np.abs(got - want).max()
        print(f"asqtad 8^4 at the workload settings, prec {prec}: dH gpu {res.dH:.9f} oracle {gold['dH']:.9f}, "
              f"max|dU| {du:.2e}, CG iterations {res.cg_iterations}")
        assert abs(res.H0 - gold["H0"]) < 1e-10 * abs(gold["H0"])
        assert abs(res.dH - gold["dH"]) < tol_dh
        assert du < tol_u
    finally:
        stag.stag_destroy(ctx)
