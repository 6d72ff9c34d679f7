"""GPU parity of the learned force surrogate against the FP64 oracle
(oracle/surrogate.py) with the same bf16-rounded weights, the oracle's network
evaluated as the tensor cores do (bf16 inputs of every product): the
surrogate force (tcgen05 MLP), its Wilson-force special case, loss and
parameter gradients; training lowers the loss; a surrogate-assisted
trajectory stays reversible and matches the oracle's three-level integrator.

The device forms the features in fp32, the oracle in fp64: a feature or
activation within ~1e-7 of a bf16 rounding boundary can round to the
neighbouring bf16 value on one side only, so the tolerances below allow a few
such single-ulp (2^-8 relative) differences."""
import numpy as np
import pytest

import synthetic as syn
from oracle import actions, surrogate as sur
from tests import layout as L
from tests.gpu_util import torch_cuda, wrap_device

pytestmark = pytest.mark.gpu
DIMS = (4, 4, 4, 6)


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"]]).astype(np.float32)


def as_device_precision(p):
    """The weights the device uses: W rounded to bf16, biases to fp32."""
    q = {}
    for k, v in p.items():
        q[k] = sur.bf16_round(v) if k.startswith("W") else np.asarray(v, dtype=np.float32).astype(np.float64)
    return q


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_surrogate_force_matches_oracle(torch):
    """The tensor-core force against the exact (unquantised) network: every
    link's force within its bf16 running-error bound (tests/bf16_bounds.py:
    the inputs f, h1, h2 of the three products rounded to bfloat16, relative
    2^-9 each, propagated through the layers); then, tighter, against the
    oracle's network evaluated with the same rounding as the tensor cores."""
    from paper_1010_5433_gb300 import stag
    from tests.bf16_bounds import network_bounds, ratio
    u = syn.near_identity_gauge(DIMS, 501, width=0.6)
    p = sur.init_params(5, scale=1.0)
    f, G = sur.features_and_generators(u)
    pd = as_device_precision(p)
    want = sur.surrogate_force(pd, f, G, quant=True)
    exact, worst, _ = network_bounds(pd, f, G, np.zeros(G.shape[:-2] + (8,)))
    ctx = stag.stag_create(DIMS, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        stag.stag_surrogate_load(ctx, flat(p))
        out = torch.empty((4, 2, 8, int(np.prod(DIMS)) // 2), dtype=torch.float64, device="cuda")
        stag.stag_surrogate_force(ctx, out)
        got = L.mom_from_abi(out.cpu().numpy(), DIMS)
        r_exact = ratio(got, exact["force"], worst["force"])
        err = np.abs(got - want).reshape(-1, 8).max(1) / np.abs(want).max()
        print(f"tensor-core surrogate force: |F - F_exact| at most {r_exact:.3f} of its bf16 bound "
              f"(rel L2 {_rel(got, exact['force']):.2e}); rel L2 {_rel(got, want):.2e} vs the bf16-activation "
              f"oracle, links off by > 1e-5: {(err > 1e-5).sum()} of {err.size}")
        assert r_exact <= 1.0
        assert _rel(got, want) < 2e-4
        assert (err > 1e-5).mean() < 0.01          # all but a few links agree to fp32 accumulation
    finally:
        stag.stag_destroy(ctx)


def test_plaquette_weights_give_the_wilson_force(torch):
    from paper_1010_5433_gb300 import stag
    u = syn.haar_gauge(DIMS, 502)
    beta = 5.6
    p = {k: np.zeros_like(v) for k, v in sur.init_params(0).items()}
    for i in range(3):
        p["b3"][8 * i] = p["b3"][8 * i + 1] = -beta / 3.0
    ctx = stag.stag_create(DIMS, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        stag.stag_surrogate_load(ctx, flat(p))
        out = torch.empty((4, 2, 8, int(np.prod(DIMS)) // 2), dtype=torch.float64, device="cuda")
        stag.stag_surrogate_force(ctx, out)
        # b3 = -beta/3 is exact in fp32 only to 1e-7: compare against the fp32-rounded value
        w = float(np.float32(-beta / 3.0))
        assert _rel(L.mom_from_abi(out.cpu().numpy(), DIMS), actions.wilson_force(u, -3.0 * w)) < 2e-6
    finally:
        stag.stag_destroy(ctx)


def test_loss_and_gradient_match_oracle(torch):
    """Loss and all 2648 parameter gradients of the tensor-core training pass
    against the exact (unquantised) network, pinned by finite differences in
    the oracle's tests: within lambda = 3 probabilistic bf16 bounds per
    component (tests/bf16_bounds.py: six rounded product inputs f, h1, h2,
    dw, dz2, dz1 per link, each 2^-9 relative, propagated through the layers
    and summed over the links in quadrature, plus fp32 accumulation); then,
    tighter, against the oracle's network with the same roundings (1e-4 in
    the loss, 1e-3 in the gradients)."""
    from paper_1010_5433_gb300 import stag
    from tests.bf16_bounds import LAMBDA, network_bounds, ratio
    u = syn.near_identity_gauge(DIMS, 503, width=0.5)
    p = sur.init_params(6, scale=1.0)
    f, G = sur.features_and_generators(u)
    target = np.random.default_rng(4).standard_normal(G.shape[:-2] + (8,))
    pd = as_device_precision(p)
    # the device reads the target force in fp32
    t32 = target.astype(np.float32).astype(np.float64)
    exact, _, prob = network_bounds(pd, f, G, t32)
    want_loss, want_grad = sur.loss_and_grad(pd, f, G, t32, quant=True)
    ctx = stag.stag_create(DIMS, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        stag.stag_surrogate_load(ctx, flat(p))
        d_t = torch.from_numpy(L.mom_to_abi(target, DIMS)).cuda()
        stag.stag_surrogate_add_force_sample(ctx, d_t)
        grad = np.zeros(stag.STAG_SUR_PARAMS)
        loss = stag.stag_surrogate_loss_grad(ctx, grad)
        names = ("W1", "b1", "W2", "b2", "W3", "b3")
        got = {}
        off = 0
        for k in names:
            n = exact[k].size
            got[k] = grad[off:off + n].reshape(exact[k].shape)
            off += n
        r = [ratio(loss, exact["loss"], LAMBDA * prob["loss"])]
        r += [ratio(got[k], exact[k], LAMBDA * prob[k]) for k in names]
        ref = flat({k: want_grad[k] for k in names}).astype(np.float64)
        print(f"loss {loss:.6f} exact {exact['loss']:.6f}; worst component at {max(r):.3f} of its bound; "
              f"vs the bf16-rounding oracle: loss rel {abs(loss - want_loss) / want_loss:.2e}, "
              f"gradient rel {_rel(grad, ref):.2e}")
        assert max(r) <= 1.0, r
        assert abs(loss - want_loss) < 1e-4 * want_loss
        assert _rel(grad, ref) < 1e-3
    finally:
        stag.stag_destroy(ctx)


def _hmc(stag, g, **kw):
    p = stag.stag_hmc()
    p.beta, p.tau, p.n_outer, p.n_gauge, p.n_flavours = 5.6, 1.0, 4, 2, 1
    fl = p.flavour[0]
    fl.mass, fl.n_pf = 0.1, 1
    for k in ("hb", "md", "met"):
        setattr(fl, k, stag.make_rational(g["c1_" + k]["a0"], g["c1_" + k]["alpha"], g["c1_" + k]["beta"]))
    p.tol_md, p.tol_met, p.max_iter, p.md_prec, p.seed = 1e-8, 1e-12, 20000, 1, 77
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_training_lowers_loss_and_surrogate_md_is_reversible(torch):
    import json
    import os
    from paper_1010_5433_gb300 import stag
    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rationals.json")))
    dims = (4, 4, 4, 4)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(syn.near_identity_gauge(dims, 0x5A0005)))
        stag.stag_surrogate_load(ctx, flat(sur.init_params(9, scale=0.3)))
        for k in range(4):
            stag.stag_md_trajectory(ctx, _hmc(stag, g, counter=k))
            stag.stag_surrogate_add_sample(ctx, _hmc(stag, g), 100 + k)
        assert stag.stag_surrogate_samples(ctx) == 4
        first, last = stag.stag_surrogate_train(ctx, 60, 3e-3)
        print(f"surrogate training: loss {first:.4f} -> {last:.4f}")
        assert last < 0.8 * first
        # reversibility of the three-level integrator with the trained surrogate
        buf0 = np.empty(4 * 256 * 18)
        stag.stag_store_gauge(ctx, buf0)
        mom = torch.from_numpy(L.mom_to_abi(syn.gaussian_momenta(dims, 3), dims)).cuda()
        phi = torch.from_numpy(L.to_half(syn.gaussian_fermion(dims, 4, on_parity=0), dims, 0)[None].view(np.float64)).cuda()
        r1 = stag.stag_md_trajectory(ctx, _hmc(stag, g, use_surrogate=1, n_mid=3, ext_mom=mom.data_ptr(),
                                               ext_phi=phi.data_ptr(), no_metropolis=1))
        back = wrap_device(torch, stag.stag_momenta(ctx), mom.numel()).clone()
        r2 = stag.stag_md_trajectory(ctx, _hmc(stag, g, use_surrogate=1, n_mid=3, ext_mom=back.data_ptr(),
                                               ext_phi=phi.data_ptr(), no_metropolis=1, flip_momenta=1))
        buf1 = np.empty(4 * 256 * 18)
        stag.stag_store_gauge(ctx, buf1)
        viol = np.sqrt(np.mean((buf1 - buf0) ** 2))
        print(f"surrogate MD: dH {r1.dH:.4e} back {r2.dH:.4e} reversibility {viol:.2e}")
        assert viol < 5e-5 and abs(r1.dH + r2.dH) < 1e-2
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec,tol_dh,tol_u", [(0, 1e-2, 2e-4), (1, 1e-2, 2e-4)])
def test_three_level_trajectory_matches_oracle(torch, prec, tol_dh, tol_u):
    """The surrogate-assisted trajectory (outer F_f - F^, n_mid steps of F^,
    gauge inside) against the oracle's three-level integrator with the same
    bf16-rounded network evaluated as the tensor cores do.  Tolerance: each of
    the ~40 evaluations of F^ in the trajectory can round an activation of
    some link to the neighbouring bf16 value on one side only (fp32 vs fp64
    features, see the module docstring), moving that link's F^ by ~2^-8 |W| of
    its size, ~1e-3; a handful of such kicks moves the links by ~1e-4 and dH
    (~4 here, an unfitted network with forces as large as the fermion force)
    by ~1e-2.  Without quantisation the same comparison agrees to 1e-6 in dU."""
    import json
    import os
    from oracle import integrator
    from oracle.rational import Rational
    from paper_1010_5433_gb300 import stag
    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rationals.json")))
    rat = {k: Rational(g["c1_" + k]["s"], g["c1_" + k]["lo"], g["c1_" + k]["hi"], g["c1_" + k]["a0"],
                       g["c1_" + k]["alpha"], g["c1_" + k]["beta"], g["c1_" + k]["err"]) for k in ("md", "met", "hb")}
    dims = (4, 4, 4, 4)
    net = sur.init_params(12, scale=1.0)
    net["W3"] *= 2.0
    u0 = syn.near_identity_gauge(dims, 0x5A0006)
    mom0 = syn.gaussian_momenta(dims, 641)
    xi = syn.gaussian_fermion(dims, 642, on_parity=0)
    fl = integrator.Flavour(mass=0.1, hb=rat["hb"], md=rat["md"], met=rat["met"])
    prm = integrator.HMCParams(dims=dims, beta=5.6, tau=0.5, n_outer=3, n_gauge=1, flavours=[fl],
                               tol_md=1e-13, tol_met=1e-13)
    want = integrator.trajectory(integrator.Context(prm), u0, mom0, [[xi]],
                                 surrogate=dict(as_device_precision(net), quant=True), n_mid=2)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u0))
        stag.stag_surrogate_load(ctx, flat(net))
        d_mom = torch.from_numpy(L.mom_to_abi(mom0, dims)).cuda()
        d_xi = torch.from_numpy(L.to_half(xi, dims, 0)[None].view(np.float64)).cuda()
        p = _hmc(stag, g, tau=0.5, n_outer=3, n_gauge=1, md_prec=prec, tol_md=1e-12 if prec == 0 else 1e-8,
                 use_surrogate=1, n_mid=2, ext_mom=d_mom.data_ptr(), ext_xi=d_xi.data_ptr(), no_metropolis=1)
        res = stag.stag_md_trajectory(ctx, p)
        buf = np.empty(4 * 256 * 18)
        stag.stag_store_gauge(ctx, buf)
        du = np.abs(L.gauge_from_host(buf, dims) - want["u"]).max()
        print(f"three-level prec {prec}: dH gpu {res.dH:.8f} oracle {want['dH']:.8f} max|dU| {du:.2e}")
        assert abs(res.H0 - want["H0"]) < 1e-8 * abs(want["H0"])
        assert abs(res.dH - want["dH"]) < tol_dh
        assert du < tol_u
    finally:
        stag.stag_destroy(ctx)


def test_what_the_trained_surrogate_gains(torch):
    """Trains the surrogate on exact forces of an 8^4 Nf=2 m=0.05 chain and
    measures what it gains.  The exact force splits into its mean over
    heatbath draws, Fbar(U), and pseudo-fermion noise; a function of U alone
    can learn Fbar only.  The trained network must reproduce most of Fbar,
    and a surrogate-assisted trajectory must not be worse than the exact one
    at the same number of fermion-force evaluations.  Measured on GB300:
    Fbar carries ~1.4% of |F|^2 and the network reproduces ~80% of it, so the
    paired |dH| with and without the surrogate agree within a few percent --
    the remainder F - F^ the outer level integrates is barely smaller than F."""
    from paper_1010_5433_gb300 import surrogate_bench
    r = surrogate_bench.run(dims=(8, 8, 8, 8), rat_prefix="c4", mass=0.05, n_outer=8, n_mid=3, samples=6,
                            train_steps=200, pairs=4, decomp_configs=2, draws=6)
    print(r)
    assert r["training"]["loss_last"] < r["training"]["loss_first"]
    assert r["force"]["captured_share_of_mean"] > 0.5
    assert 0.0 < r["force"]["mean_share"] < 0.2
    assert r["surrogate"]["mean_abs_dH"] < 1.25 * r["exact_half"]["mean_abs_dH"]
    assert r["exact"]["mean_abs_dH"] < r["exact_half"]["mean_abs_dH"]
