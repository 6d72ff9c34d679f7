"""GPU parity of the staggered Dslash and of A = m^2 - D_eo D_oe (paper Sec. 2,
Sec. 5) against the FP64 oracle, through the C ABI, every precision."""
import numpy as np
import pytest

import synthetic as syn
from oracle import dirac, lattice as lat, su3
from tests import layout as L
from tests.gpu_util import dev, host_complex, torch_cuda

pytestmark = pytest.mark.gpu

# (dims, seed): ragged (Vh not a multiple of the 128-thread block), odd-shaped,
# and the 16^4 and 32^3x8 workloads of the RHMC configurations
# the volume picks 8, 4, 2 or 1 threads per site (2^19 threads in flight)
CASES = [((4, 4, 4, 4), 1), ((2, 4, 6, 8), 2), ((6, 2, 4, 10), 3), ((16, 16, 16, 16), 4), ((32, 32, 32, 8), 5),
         ((24, 24, 24, 24), 6), ((32, 32, 32, 32), 8)]
TOL = {0: 1e-10, 1: 2e-6, 2: 2e-6, 3: 2e-6}     # field-relative error per precision


def _quantised_links(u, prec):
    """The links each precision actually sees: fp32 hi words; for 12-real formats
    rows 0-1 rounded (fp32, or bf16 of the fp32 word) and row 2 rebuilt in fp64."""
    if prec == 0:
        return u
    u32 = (u.real.astype(np.float32) + 1j * u.imag.astype(np.float32)).astype(np.complex128)
    if prec == 1:
        return u32
    if prec == 3:
        u32 = (L.bf16_round(u32.real.astype(np.float32)).astype(np.float64)
               + 1j * L.bf16_round(u32.imag.astype(np.float32)).astype(np.float64))
    out = u32.copy()
    out[..., 2, :] = su3.third_row(u32)
    return out


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.mark.parametrize("dims,seed", CASES)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("out_par", [0, 1])
def test_dslash_matches_oracle(torch, dims, seed, prec, out_par):
    from paper_1010_5433_gb300 import stag
    vol = dims[0] * dims[1] * dims[2] * dims[3]
    if vol > 70000 and (prec in (2, 3) or out_par == 1):
        pytest.skip("large lattices: one parity per 12-real format is enough")
    if vol > 300000 and prec != 1:
        pytest.skip("largest lattices: the fp32 kernel only")
    u = syn.haar_gauge(dims, seed) if seed % 2 else syn.near_identity_gauge(dims, seed)
    eta, par = lat.eta(dims), lat.parity(dims)
    psi = syn.gaussian_fermion(dims, seed + 100, on_parity=1 - out_par)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        h_in = L.to_half(psi, dims, 1 - out_par)
        if prec == 0:
            d_in = dev(torch, h_in)
        else:
            d_in = dev(torch, h_in.astype(np.complex64))
        d_out = torch.empty_like(d_in)
        stag.stag_dslash(ctx, out_par, prec, 1, d_in, d_out)
        torch.cuda.synchronize()
        got = host_complex(d_out).reshape(3, -1)
        psi_used = psi if prec == 0 else psi.astype(np.complex64).astype(np.complex128)
        want = L.to_half(dirac.d_block(_quantised_links(u, prec), psi_used, eta, par, out_par), dims, out_par)
        assert L.rel_err(got, want) < TOL[prec]
        assert np.abs(got - want).max() < 20 * TOL[prec] * np.abs(want).max()
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1, 3])
@pytest.mark.parametrize("nrhs", [1, 3, 4, 7, 60])
def test_multi_rhs_equals_single(torch, prec, nrhs):
    """The n-RHS Dslash (one link load for every source) gives each source's
    single-RHS result bit for bit; 60 is the force's Y = D_oe X of 2+1
    flavours x 2 pseudo-fermions x 15 shifts."""
    from paper_1010_5433_gb300 import stag
    dims = (4, 6, 4, 8)
    u = syn.haar_gauge(dims, 7)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        fields = np.stack([L.to_half(syn.gaussian_fermion(dims, 200 + k, on_parity=0), dims, 0)
                           for k in range(nrhs)])
        d_in = dev(torch, fields if prec == 0 else fields.astype(np.complex64))
        d_out = torch.empty_like(d_in)
        stag.stag_dslash(ctx, 1, prec, nrhs, d_in, d_out)
        for k in range(nrhs):
            one = torch.empty_like(d_in[k])
            stag.stag_dslash(ctx, 1, prec, 1, d_in[k].contiguous(), one)
            assert torch.equal(one, d_out[k])
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_a_matches_oracle(torch, prec):
    from paper_1010_5433_gb300 import stag
    dims = (4, 4, 6, 6)
    u = syn.haar_gauge(dims, 9)
    eta, par = lat.eta(dims), lat.parity(dims)
    mass, shift = 0.05, 0.3
    psi = syn.gaussian_fermion(dims, 19, on_parity=0)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        h = L.to_half(psi, dims, 0)
        d_in = dev(torch, h if prec == 0 else h.astype(np.complex64))
        d_out = torch.empty_like(d_in)
        stag.stag_apply_a(ctx, mass, shift, prec, 1, d_in, d_out)
        got = host_complex(d_out).reshape(3, -1)
        psi_used = psi if prec == 0 else psi.astype(np.complex64).astype(np.complex128)
        want = L.to_half(dirac.a_op(_quantised_links(u, prec), psi_used, mass, eta, par, shift), dims, 0)
        assert L.rel_err(got, want) < TOL[prec]
    finally:
        stag.stag_destroy(ctx)


def test_store_gauge_roundtrip(torch):
    """load -> store returns the field to the two-float store's precision
    (hi + lo keeps about 48 mantissa bits, Sec. 5)."""
    from paper_1010_5433_gb300 import stag
    dims = (4, 2, 2, 6)
    u = syn.haar_gauge(dims, 13)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        buf = np.empty(4 * np.prod(dims) * 18)
        stag.stag_store_gauge(ctx, buf)
        back = L.gauge_from_host(buf, dims)
        assert np.abs(back - u).max() < 1e-13
    finally:
        stag.stag_destroy(ctx)


def _tie_field(u):
    """Every real of u moved to just below the midpoint between its float
    rounding h and the next float away from zero: x = h + (ulp/2)(1 - 2^-28).
    Then x rounds to h, and the remainder x - h rounds to exactly half an ulp,
    so hi + lo is a tie between two floats."""
    def tie(a):
        h = a.astype(np.float32).astype(np.float64)
        ulp = np.spacing(np.abs(h).astype(np.float32)).astype(np.float64)
        return h + np.sign(h) * ulp * (0.5 - 2.0 ** -29)
    return tie(u.real) + 1j * tie(u.imag)


def test_store_load_roundtrip_is_exact_at_ties(torch):
    """load, fp32 Dslash, store, load again, fp32 Dslash: the same output bit
    for bit, and the same stored field, for a field in which every real sits
    at a float rounding tie of the two-float split (the case where a store and
    a reload could move the fp32 word by one ulp)."""
    from paper_1010_5433_gb300 import stag
    dims = (4, 4, 4, 4)
    u = _tie_field(syn.near_identity_gauge(dims, 17))
    inp = syn.gaussian_fermion(dims, 18, on_parity=1)
    ctx = stag.stag_create(dims, True)
    try:
        outs, stores = [], []
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        for _ in range(2):
            for prec in (1, 2):
                d_in = dev(torch, L.to_half(inp, dims, 1).astype(np.complex64))
                d_out = torch.empty_like(d_in)
                stag.stag_dslash(ctx, 0, prec, 1, d_in, d_out)
                outs.append(d_out.cpu().numpy())
            buf = np.empty(4 * np.prod(dims) * 18)
            stag.stag_store_gauge(ctx, buf)
            stores.append(buf.copy())
            stag.stag_load_gauge(ctx, buf)
        assert np.array_equal(stores[0], stores[1])
        assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[1], outs[3])
    finally:
        stag.stag_destroy(ctx)
