"""Full-size H~ x parity on the 4x4 t-t' workload (1e7-state basis) and the
6x4 t-t' workload (5e7-state basis, hash-lookup kernels), in the launch
configurations the benchmark times: y for fp32 and fp64 vectors and one, 24
and 48 columns, checked on rows the oracle evaluates one by one."""
import numpy as np
import pytest
import torch

import paper_2509_22975_gb300 as pkg
from oracle import hamiltonian as H
from workloads import configs as C

from gpu_common import U32, U64, device_ctx, model, row_terms_bound

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = "cuda:0"


@pytest.fixture(scope="module")
def square16():
    pkg.build()
    w = C.square16_u8()
    ctx = device_ctx(w)
    B = ctx.mcd_get_basis()
    return w, ctx, B


@pytest.mark.parametrize("dtype,ncols", [(torch.float32, 1), (torch.float64, 1), (torch.float32, 24)])
def test_sampled_rows(square16, dtype, ncols):
    w, ctx, B = square16
    n = len(B)
    g = torch.Generator(device=DEV).manual_seed(ncols)
    x = torch.randn(n, ncols, dtype=dtype, device=DEV, generator=g)
    y = torch.empty_like(x)
    ctx.mcd_apply(x, y)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    ks = np.concatenate([[0, n - 1], rng.choice(n, 300, replace=False)])
    X = x.double().cpu().numpy()
    ref, absHx = H.apply_rows(model(w), B, X, ks)
    got = y.double().cpu().numpy()[ks]
    u = U64 if dtype == torch.float64 else U32
    nt = row_terms_bound(int(np.count_nonzero(np.triu(w.lat.t, 1))))
    assert np.all(np.abs(got - ref) <= nt * u * absHx + 4 * U64 * absHx)


@pytest.fixture(scope="module")
def rect24():
    pkg.build()
    w = C.rect24_u8()
    ctx = device_ctx(w)
    B = ctx.mcd_get_basis()
    return w, ctx, B


@pytest.mark.parametrize("dtype,ncols", [(torch.float32, 1), (torch.float64, 1), (torch.float32, 24),
                                         (torch.float32, 48)])
def test_rect24_sampled_rows(rect24, dtype, ncols):
    w, ctx, B = rect24
    n = len(B)
    assert n == w.n_f
    g = torch.Generator(device=DEV).manual_seed(100 + ncols)
    x = torch.randn(n, ncols, dtype=dtype, device=DEV, generator=g)
    y = torch.empty_like(x)
    ctx.mcd_apply(x, y)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    ks = np.concatenate([[0, n - 1], rng.choice(n, 200, replace=False)])
    Xs = x.double().cpu().numpy()
    ref, absHx = H.apply_rows(model(w), B, Xs, ks)
    got = y.double().cpu().numpy()[ks]
    u = U64 if dtype == torch.float64 else U32
    nt = row_terms_bound(int(np.count_nonzero(np.triu(w.lat.t, 1))))
    assert np.all(np.abs(got - ref) <= nt * u * absHx + 4 * U64 * absHx)
