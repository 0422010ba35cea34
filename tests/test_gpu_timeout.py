"""Time-out path of the bounded device waits of the streaming H~x kernel.

A test option (MCD_OPT_WAIT_TEST) makes the next cached product skip the
producer's arrival for one work item (one column) or work unit (many
columns) and poll each wait only 4096 times, so the consumer waits on it give
up: nothing is left waiting on a copy and no GPU fault is involved.  The library must report
MCD_E_TIMEOUT (from mcd_apply when it waits for its product, from
mcd_lanczos_ground at its next read-back, or from the next reading call when
mcd_apply runs asynchronously) instead of returning an incomplete y, and the
context must give the right product on the next call."""
import numpy as np
import pytest
import torch

import paper_2509_22975_gb300 as pkg
from workloads import configs as C

from gpu_common import device_ctx

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    pkg.build()
    c = device_ctx(C.tilted12_u8(), nf=1 << 16)
    c.mcd_set_option(pkg.MCD_OPT_HV_CACHE, pkg.CACHE_REQUIRED)
    yield c
    c.close()


def vectors(ctx, seed=0):
    n = ctx.mcd_basis_info(nnz=False)["n_states"]
    g = torch.Generator(device="cpu").manual_seed(seed)
    x = torch.randn(n, generator=g, dtype=torch.float32).to(DEV)
    return x, torch.empty_like(x)


def test_apply_reports_timeout_and_recovers(ctx):
    x, y = vectors(ctx)
    ctx.mcd_apply(x, y)
    ref = y.clone()
    assert ctx.mcd_hv_cache_info()["wait_errors"] == 0
    for item in (0, 5):
        ctx.mcd_set_option(pkg.MCD_OPT_WAIT_TEST, item)
        y.fill_(0.0)
        with pytest.raises(pkg.MCDError) as e:
            ctx.mcd_apply(x, y)
        assert e.value.status == pkg.MCD_E_TIMEOUT
        assert ctx.mcd_hv_cache_info()["wait_errors"] == 0     # reported once, then cleared
        y.fill_(0.0)
        ctx.mcd_apply(x, y)                                     # the option applied to one product
        assert torch.equal(y, ref)


def test_many_column_apply_reports_timeout_and_recovers(ctx):
    n = ctx.mcd_basis_info(nnz=False)["n_states"]
    g = torch.Generator(device="cpu").manual_seed(3)
    x = torch.randn(n, 8, generator=g, dtype=torch.float32).to(DEV)
    y = torch.empty_like(x)
    ctx.mcd_apply(x, y)
    ref = y.clone()
    ctx.mcd_set_option(pkg.MCD_OPT_WAIT_TEST, 1)
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_apply(x, y)
    assert e.value.status == pkg.MCD_E_TIMEOUT
    y.fill_(0.0)
    ctx.mcd_apply(x, y)
    assert torch.equal(y, ref)


def test_asynchronous_apply_reports_at_the_next_reading_call(ctx):
    x, y = vectors(ctx, 1)
    ctx.mcd_apply(x, y)
    ref = y.clone()
    ctx.mcd_set_option(pkg.MCD_OPT_APPLY_SYNC, 0)
    try:
        ctx.mcd_set_option(pkg.MCD_OPT_WAIT_TEST, 2)
        ctx.mcd_apply(x, y)                                     # returns after the launch
        torch.cuda.synchronize()
        assert ctx.mcd_hv_cache_info()["wait_errors"] == 1      # read, not cleared
        ctx.mcd_set_option(pkg.MCD_OPT_APPLY_SYNC, 1)
        with pytest.raises(pkg.MCDError) as e:                  # the next waiting call reports it
            ctx.mcd_apply(x, y)
        assert e.value.status == pkg.MCD_E_TIMEOUT
        ctx.mcd_apply(x, y)
        assert torch.equal(y, ref)
    finally:
        ctx.mcd_set_option(pkg.MCD_OPT_APPLY_SYNC, 1)


@pytest.mark.parametrize("dtype", [pkg.MCD_F32, pkg.MCD_F64])
def test_lanczos_reports_timeout_and_recovers(ctx, dtype):
    ref = ctx.mcd_lanczos_ground(40, 0.0, 0, dtype)
    ctx.mcd_set_option(pkg.MCD_OPT_WAIT_TEST, 3)                # the first step's product
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_lanczos_ground(40, 0.0, 0, dtype)
    assert e.value.status == pkg.MCD_E_TIMEOUT
    again = ctx.mcd_lanczos_ground(40, 0.0, 0, dtype)
    assert again["E0"] == ref["E0"] and again["iters"] == ref["iters"]
