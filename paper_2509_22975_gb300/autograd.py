"""torch.autograd glue around the library's H~v, its parameter adjoint and the
Lanczos ground state (argument marshalling only; all arithmetic runs in the
library's kernels).

* ``hv(ctx, x, t, eps, U)``: y = H~(t, eps, U) x, differentiable in x and in
  the parameters (backward: H~ grad_y for x, ``mcd_hv_adjoint`` for t, eps, U).
* ``ground_energy(ctx, t, eps, U, ...)``: Lanczos E0, differentiable in the
  parameters by Hellmann-Feynman, dE0/dtheta = <Omega~| dH/dtheta |Omega~>,
  evaluated by the same adjoint kernel with u = v = |Omega~>.
* ``green(ctx, t, eps, U, orbitals, n_blocks, w_t, z)``: the band-Lanczos G(z)
  as [nz, L, L, 2] (real, imaginary), differentiable in the parameters
  (backward: ``mcd_green_gradient``).

t is the full symmetric [n, n] hopping matrix; its gradient is returned
symmetric with the bond derivative at [i, j] and [j, i] (0 where t_ij = 0).
U may be a scalar (uniform repulsion) or a per-site vector.
"""
from __future__ import annotations

import numpy as np
import torch

from . import MCD_F32, MCD_F64


def _set(ctx, t, eps, U):
    ctx.mcd_set_hamiltonian(t.detach().cpu().double().numpy(),
                            eps.detach().cpu().double().numpy(),
                            np.atleast_1d(U.detach().cpu().double().numpy()),
                            ctx.n_up, ctx.n_dn)


def _like(a, ref):
    return torch.as_tensor(a, dtype=ref.dtype, device=ref.device)


def _grad_U(gu, U):
    return _like(gu.sum() if U.dim() == 0 or U.numel() == 1 else gu, U).reshape(U.shape)


class _Hv(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, x, t, eps, U):
        _set(ctx, t, eps, U)
        y = torch.empty_like(x)
        ctx.mcd_apply(x.contiguous(), y)
        fctx.ctx = ctx
        fctx.save_for_backward(x, t, eps, U)
        return y

    @staticmethod
    def backward(fctx, gy):
        x, t, eps, U = fctx.saved_tensors
        ctx = fctx.ctx
        gy = gy.contiguous()
        gx = torch.empty_like(gy)
        ctx.mcd_apply(gy, gx)
        gt, ge, gu = ctx.mcd_hv_adjoint(gy, x.contiguous())
        return None, gx, _like(gt, t), _like(ge, eps), _grad_U(gu, U)


def hv(ctx, x, t, eps, U):
    """y = H~(t, eps, U) x (the context's basis), differentiable."""
    return _Hv.apply(ctx, x, t, eps, U)


class _E0(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, t, eps, U, max_iter, tol, seed, dtype):
        _set(ctx, t, eps, U)
        n = ctx.mcd_basis_info(nnz=False)["n_states"]
        psi = torch.empty(n, dtype=torch.float64 if dtype == MCD_F64 else torch.float32,
                          device=torch.device("cuda", ctx.device))
        r = ctx.mcd_lanczos_ground(max_iter, tol, seed, dtype, psi=psi, allow_not_converged=True)
        fctx.ctx = ctx
        fctx.save_for_backward(psi, t, eps, U)
        return torch.tensor(r["E0"], dtype=torch.float64)

    @staticmethod
    def backward(fctx, gE):
        psi, t, eps, U = fctx.saved_tensors
        gt, ge, gu = fctx.ctx.mcd_hv_adjoint(psi, psi)
        g = float(gE)
        return None, _like(g * gt, t), _like(g * ge, eps), _grad_U(g * gu, U), None, None, None, None


def ground_energy(ctx, t, eps, U, max_iter: int = 400, tol: float = 1e-12, seed: int = 0,
                  dtype: int = MCD_F64):
    """Lanczos E0 of H~(t, eps, U) on the context's basis; gradients by
    Hellmann-Feynman."""
    return _E0.apply(ctx, t, eps, U, max_iter, tol, seed, dtype)


class _Green(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, t, eps, U, orbitals, n_blocks, w_t, z, max_iter, tol):
        _set(ctx, t, eps, U)
        n = ctx.mcd_basis_info(nnz=False)["n_states"]
        psi = torch.empty(n, dtype=torch.float64, device=torch.device("cuda", ctx.device))
        ctx.mcd_lanczos_ground(max_iter, tol, 0, MCD_F64, psi=psi, allow_not_converged=True)
        G, _, _ = ctx.mcd_band_lanczos_green(orbitals, n_blocks, w_t, z)
        fctx.ctx = ctx
        fctx.args = (orbitals, n_blocks, w_t, z)
        fctx.save_for_backward(t, eps, U)
        return torch.stack([torch.from_numpy(G.real), torch.from_numpy(G.imag)], dim=-1)

    @staticmethod
    def backward(fctx, gG):
        t, eps, U = fctx.saved_tensors
        orbitals, n_blocks, w_t, z = fctx.args
        g = gG.detach().cpu().double().numpy()
        gt, ge, gu, _ = fctx.ctx.mcd_green_gradient(orbitals, n_blocks, w_t, z, g[..., 0] + 1j * g[..., 1])
        return None, _like(gt, t), _like(ge, eps), _grad_U(gu, U), None, None, None, None, None, None


def green(ctx, t, eps, U, orbitals, n_blocks: int, w_t: float, z, max_iter: int = 800, tol: float = 1e-13):
    """G(z) of H~(t, eps, U) on the context's basis (band Lanczos, fp64), as a real
    tensor [nz, L, L, 2] (real and imaginary parts); differentiable in the
    parameters through mcd_green_gradient."""
    z = np.ascontiguousarray(np.atleast_1d(z), dtype=np.complex128)
    return _Green.apply(ctx, t, eps, U, list(orbitals), n_blocks, w_t, z, max_iter, tol)


__all__ = ["hv", "ground_energy", "green", "MCD_F32", "MCD_F64"]
