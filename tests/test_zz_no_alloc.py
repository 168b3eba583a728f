"""wilson_dslash_noalloc against wilson_dslash.

Callers that must not allocate device memory (code running under another
component's allocator, a memory pool that must not fragment, a loop that
cannot take cudaMalloc's implicit synchronisation) use the no-allocation
entry point; it must give the same operator application as the ordinary
one.  Two calls in a row with different inputs also show that nothing left
in the shared scratch array from one call leaks into the next.  This file is
collected last and passes on its own in a fresh process as well.
"""
import numpy as np
import pytest
import torch

from helpers import TOL, rel
from paper_1103_5103_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1103_5103_gb300 import api as A
    return A


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df"])
def test_noalloc_matches_dslash_twice(api, prec):
    dims = (8, 4, 6, 8)
    U = synth.gauge_field(dims, 0.5, seed=17)
    lat = api.Lattice(dims)
    g = api.Gauge(lat, torch.from_numpy(U).cuda(), precs=(prec,))
    for call in range(2):
        psi = torch.from_numpy(synth.gaussian_source(dims, seed=40 + call)).cuda()
        for op in (api.OP_HOP, api.OP_M, api.OP_MPREC):
            for dag in (False, True):
                want = torch.empty_like(psi)
                got = torch.full_like(psi, float("nan"))
                (api.wilson_dslash_dag if dag else api.wilson_dslash)(g, psi, want, 0.121, prec, op)
                api.wilson_dslash_noalloc(g, psi, got, 0.121, prec, op, dagger=dag)
                torch.cuda.synchronize()
                assert rel(got.cpu().numpy(), want.cpu().numpy()) <= TOL[prec], (call, op, dag)


def test_noalloc_rejects_oversized_lattice(api):
    dims = (24, 24, 24, 24)  # four FP64 half-lattice spinors need 127 MB > 64 MiB
    lat = api.Lattice(dims)
    g = api.Gauge(lat, torch.from_numpy(synth.unit_gauge_field(dims)).cuda(), precs=("f64",))
    psi = torch.zeros((lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
    out = torch.empty_like(psi)
    with pytest.raises(api.WilsonError) as e:
        api.wilson_dslash_noalloc(g, psi, out, 0.12, "f64", api.OP_M)
    assert e.value.status == api.WL_ERR_ARG and "64 MiB" in str(e.value)


def test_noalloc_allocates_nothing(api):
    """The property the entry point exists for: on a handle whose workspace
    is empty, the call leaves the device's free memory unchanged.  A first
    call on another handle comes before the measurement, because the first
    launch of a kernel may make the driver load its code.  The same
    measurement then sees wilson_dslash allocate the handle's workspace."""
    dims = (16, 16, 16, 16)  # four FP32 half-lattice spinors of 3.1 MB each
    U = torch.from_numpy(synth.gauge_field(dims, 0.5, seed=18)).cuda()
    lat = api.Lattice(dims)
    psi = torch.from_numpy(synth.gaussian_source(dims, seed=50)).cuda()
    got = torch.empty_like(psi)
    want = torch.empty_like(psi)
    warm = api.Gauge(lat, U, precs=("f32",))
    api.wilson_dslash_noalloc(warm, psi, got, 0.121, "f32", api.OP_MPREC)
    torch.cuda.synchronize()
    g = api.Gauge(lat, U, precs=("f32",))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        api.wilson_dslash_noalloc(g, psi, got, 0.121, "f32", api.OP_MPREC)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, free0 - free1
    api.wilson_dslash(g, psi, want, 0.121, "f32", api.OP_MPREC)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free1
    assert rel(got.cpu().numpy(), want.cpu().numpy()) <= TOL["f32"]
