"""stag_apply_a_noalloc against stag_apply_a and against the oracle's A.

The no-allocation entry point serves callers that may not call cudaMalloc or
cudaFree (device memory owned by their own pool, or no room for the
synchronisation cudaFree implies).  It must give the same A = m^2 + shift -
D_eo D_oe as the allocating entry point, call after call, although every
call reuses the same fixed scratch array.  This file is collected last so
that a run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

import synthetic as syn
from oracle import dirac, lattice as lat
from tests import layout as L
from tests.gpu_util import dev, host_complex, torch_cuda

pytestmark = pytest.mark.gpu
TOL = {0: 1e-10, 1: 2e-6}     # the field-relative tolerances of the A-operator tests


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_apply_a_on_two_calls(prec):
    torch = torch_cuda()
    from paper_1010_5433_gb300 import stag
    dims = (4, 6, 4, 8)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(syn.haar_gauge(dims, 31)))
        for call, (seed, mass, shift, nrhs) in enumerate([(41, 0.05, 0.3, 2), (42, 0.1, 0.0, 3)]):
            fields = np.stack([L.to_half(syn.gaussian_fermion(dims, seed + k, on_parity=0), dims, 0)
                               for k in range(nrhs)])
            d_in = dev(torch, fields if prec == 0 else fields.astype(np.complex64))
            ref = torch.empty_like(d_in)
            got = torch.full_like(d_in, float("nan"))
            stag.stag_apply_a(ctx, mass, shift, prec, nrhs, d_in, ref)
            stag.stag_apply_a_noalloc(ctx, mass, shift, prec, nrhs, d_in, got)
            torch.cuda.synchronize()
            a, b = host_complex(got), host_complex(ref)
            assert np.isfinite(a).all(), f"call {call}"
            assert L.rel_err(a, b) < TOL[prec], f"call {call}"
    finally:
        stag.stag_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    torch = torch_cuda()
    from paper_1010_5433_gb300 import stag
    dims = (4, 4, 4, 4)
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(syn.haar_gauge(dims, 5)))
        buf = torch.zeros(16, dtype=torch.float64, device="cuda")
        # 6000 sources of 128 fp64 sites need 36.9 MB > 32 MiB: refused on the host, nothing launched
        with pytest.raises(stag.StagError) as e:
            stag.stag_apply_a_noalloc(ctx, 0.1, 0.0, 0, 6000, buf, buf)
        assert e.value.status == 1 and "scratch" in str(e.value)
    finally:
        stag.stag_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_first_call_on_a_fresh_context_matches_oracle(prec):
    """The path the entry point exists for: the very first call on a new
    context, on a ragged lattice no other test tunes, so no workspace and no
    Dslash tuning exist yet (the untuned Dslash runs one thread per site);
    compared directly with the oracle's A = m^2 + shift - D_eo D_oe."""
    torch = torch_cuda()
    from paper_1010_5433_gb300 import stag
    dims = (6, 2, 10, 4)
    u = syn.haar_gauge(dims, 57)
    eta, par = lat.eta(dims), lat.parity(dims)
    mass, shift, nrhs = 0.07, 0.21, 2
    psis = [syn.gaussian_fermion(dims, 58 + k, on_parity=0) for k in range(nrhs)]
    want = np.stack([L.to_half(dirac.a_op(u, p, mass, eta, par, shift), dims, 0) for p in psis])
    fields = np.stack([L.to_half(p, dims, 0) for p in psis])
    ctx = stag.stag_create(dims, True)
    try:
        stag.stag_load_gauge(ctx, L.gauge_host(u))
        d_in = dev(torch, fields if prec == 0 else fields.astype(np.complex64))
        got = torch.full_like(d_in, float("nan"))
        stag.stag_apply_a_noalloc(ctx, mass, shift, prec, nrhs, d_in, got)
        torch.cuda.synchronize()
        a = host_complex(got)
        # fp32: the oracle's A applied to the fp32-rounded input, as the device sees it
        ref = want if prec == 0 else np.stack([
            L.to_half(dirac.a_op(u, L.from_half(fields[k].astype(np.complex64).astype(complex), dims, 0), mass, eta,
                                 par, shift), dims, 0) for k in range(nrhs)])
        assert np.isfinite(a).all()
        assert L.rel_err(a, ref) < TOL[prec]
    finally:
        stag.stag_destroy(ctx)
