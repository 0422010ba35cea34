"""GPU adjoint of H~v with respect to (t, eps, U) through the C ABI against
the oracle's derivative operators; torch.autograd through H~v; gradients of
E0 (Hellmann-Feynman) against finite differences of the device E0, including
the lattice-level (t, t', U) derivatives of the 4x4 t-t' cluster."""
import numpy as np
import pytest
import torch

import paper_2509_22975_gb300 as pkg
from paper_2509_22975_gb300 import autograd as AG
from oracle import hamiltonian as H
from workloads import configs as C, lattice as L

from gpu_common import device_ctx, model

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()


@pytest.mark.parametrize("dtype,ncols,tol", [(torch.float64, 1, 1e-11), (torch.float64, 3, 1e-11),
                                             (torch.float32, 2, 2e-5)])
def test_adjoint_matches_oracle(dtype, ncols, tol):
    w = C.tilted12_u8()
    w.mu = 1.7
    ctx = device_ctx(w, nf=30000)
    B = ctx.mcd_get_basis()
    g = torch.Generator(device=DEV).manual_seed(ncols)
    u = torch.randn(len(B), ncols, dtype=dtype, device=DEV, generator=g)
    v = torch.randn(len(B), ncols, dtype=dtype, device=DEV, generator=g)
    gt, ge, gu = ctx.mcd_hv_adjoint(u, v)
    rt, re, ru = H.parameter_derivatives(model(w), B, u.double().cpu().numpy(), v.double().cpu().numpy())
    for a, b in ((gt, rt), (ge, re), (gu, ru)):
        assert np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b)))
    assert np.all(gt[w.lat.t == 0] == 0)


def test_autograd_hv():
    w = C.ring8_u4()
    ctx = device_ctx(w)
    B = ctx.mcd_get_basis()
    t = torch.tensor(w.lat.t, dtype=torch.float64, requires_grad=True)
    eps = torch.tensor(w.eps, dtype=torch.float64, requires_grad=True)
    U = torch.tensor(w.U, dtype=torch.float64, requires_grad=True)
    x = torch.randn(len(B), dtype=torch.float64, device=DEV, requires_grad=True)
    gy = torch.randn(len(B), dtype=torch.float64, device=DEV)
    y = AG.hv(ctx, x, t, eps, U)
    (y * gy).sum().backward()
    P = H.build(model(w), B)
    assert torch.allclose(x.grad.cpu(), torch.from_numpy(P.sparse() @ gy.cpu().numpy()), atol=1e-12)
    rt, re, ru = H.parameter_derivatives(model(w), B, gy.cpu().numpy(), x.detach().cpu().numpy())
    assert np.max(np.abs(t.grad.numpy() - rt)) < 1e-10 * max(1, np.max(np.abs(rt)))
    assert np.max(np.abs(eps.grad.numpy() - re)) < 1e-10 * max(1, np.max(np.abs(re)))
    assert abs(U.grad.item() - ru.sum()) < 1e-10 * max(1, abs(ru.sum()))


def test_ground_energy_gradient_vs_finite_differences():
    # adjoint gradients agree with central finite differences to 1e-6
    w = C.ring8_u4()
    ctx = device_ctx(w)
    t = torch.tensor(w.lat.t, dtype=torch.float64, requires_grad=True)
    eps = torch.tensor(np.linspace(-0.3, 0.2, 8), dtype=torch.float64, requires_grad=True)
    U = torch.tensor(w.U, dtype=torch.float64, requires_grad=True)
    E = AG.ground_energy(ctx, t, eps, U, tol=1e-13)
    E.backward()
    assert U.dtype == torch.float64

    def E0(tt, ee, uu):
        f64 = torch.float64   # a Python float would become a float32 tensor
        return float(AG.ground_energy(ctx, torch.tensor(tt, dtype=f64), torch.tensor(ee, dtype=f64),
                                      torch.tensor(uu, dtype=f64), tol=1e-13))

    h = 1e-4
    tt = w.lat.t.copy()
    tp, tm = tt.copy(), tt.copy()
    tp[2, 3] += h; tp[3, 2] += h
    tm[2, 3] -= h; tm[3, 2] -= h
    e0 = eps.detach().numpy()
    fd_t = (E0(tp, e0, w.U) - E0(tm, e0, w.U)) / (2 * h)
    assert abs(fd_t - t.grad[2, 3].item()) < 1e-6
    d = np.zeros(8)
    d[5] = h
    fd_e = (E0(tt, e0 + d, w.U) - E0(tt, e0 - d, w.U)) / (2 * h)
    assert abs(fd_e - eps.grad[5].item()) < 1e-6
    fd_u = (E0(tt, e0, w.U + h) - E0(tt, e0, w.U - h)) / (2 * h)
    assert abs(fd_u - U.grad.item()) < 1e-6


def test_lattice_level_t_tprime_U_gradient():
    # 4x4 t-t' cluster (smaller MC basis): dE0/d(t, t', U) from the bond
    # gradients (t_ij = -t on nearest, -t' on next-nearest neighbours)
    w = C.square16_u8()
    ctx = device_ctx(w, nf=200000)

    def lattice_t(tv, tpv):
        return L.superlattice_cluster((4, 0), (0, 4), t=tv, tp=tpv).t

    t_nn = L.superlattice_cluster((4, 0), (0, 4), t=1.0, tp=0.0).t != 0
    t_nnn = L.superlattice_cluster((4, 0), (0, 4), t=0.0, tp=1.0).t != 0
    T = torch.tensor(lattice_t(1.0, -0.3), requires_grad=True)
    eps = torch.zeros(16, dtype=torch.float64, requires_grad=True)
    U = torch.tensor(8.0, dtype=torch.float64, requires_grad=True)
    E = AG.ground_energy(ctx, T, eps, U, max_iter=600, tol=1e-12)
    E.backward()
    g = T.grad.numpy()
    dE_dt = -0.5 * np.sum(g[t_nn])       # t_ij = -t, each bond stored twice
    dE_dtp = -0.5 * np.sum(g[t_nnn])

    def E0(tv, tpv, uv):
        f64 = torch.float64
        return float(AG.ground_energy(ctx, torch.tensor(lattice_t(tv, tpv), dtype=f64), torch.zeros(16, dtype=f64),
                                      torch.tensor(uv, dtype=f64), max_iter=600, tol=1e-12))

    h = 1e-4
    assert abs((E0(1 + h, -0.3, 8.0) - E0(1 - h, -0.3, 8.0)) / (2 * h) - dE_dt) < 1e-6
    assert abs((E0(1.0, -0.3 + h, 8.0) - E0(1.0, -0.3 - h, 8.0)) / (2 * h) - dE_dtp) < 1e-6
    assert abs((E0(1.0, -0.3, 8.0 + h) - E0(1.0, -0.3, 8.0 - h)) / (2 * h) - U.grad.item()) < 1e-6
