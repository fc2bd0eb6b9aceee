"""torch.autograd.Function wrappers over the differentiation entry points.

Thin marshalling over the C-ABI: the forward passes call fft_homog_solve or
fft_homog_tangent, the backward passes fft_homog_tangent or
fft_homog_sensitivity (Section 3.3, Eq. 4; Section 4.4.2). All compute runs
in the CUDA library; the chain rule contracts the returned 9x9 tangent or
voxel field with the incoming gradient and nothing else.

``homogenized_stress(Fbar, ...)``   Pbar as a differentiable function of Fbar.
``homogenized_modulus(rho, ...)``   one entry Cbar_ijkl of a small-strain cell
                                    as a differentiable function of a voxel
                                    density rho (through the modulus scale
                                    s(rho) held in ``mat.scale``).
``homogenized_stress_of_density(rho, ...)``
                                    Pbar of a (finite-strain or linear) cell
                                    under a fixed Fbar as a differentiable
                                    function of the voxel density; backward
                                    contracts the incoming 9-gradient with
                                    fft_homog_stress_sensitivity's fields.
"""

from __future__ import annotations

import torch

from ._binding import Context, FhOptions, Material, default_options


class _HomogenizedStress(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Fbar, cell, mat, F, n_increments, options, tangent_options):
        fb = Fbar.detach().to("cpu", torch.float64).reshape(9).numpy()
        pbar, _, _ = cell.fft_homog_solve(mat, fb, F, n_increments=n_increments, options=options)
        ctx.cell, ctx.mat, ctx.F, ctx.topt = cell, mat, F, tangent_options
        return torch.as_tensor(pbar, dtype=torch.float64).reshape(Fbar.shape).to(Fbar.device)

    @staticmethod
    def backward(ctx, grad):
        C = ctx.cell.fft_homog_tangent(ctx.mat, ctx.F, ctx.topt)  # at the converged state of forward
        g = grad.detach().to("cpu", torch.float64).reshape(9).numpy()
        gF = torch.as_tensor(C.T @ g, dtype=torch.float64).reshape(grad.shape).to(grad.device)
        return gF, None, None, None, None, None, None


def homogenized_stress(Fbar: torch.Tensor, cell: Context, mat: Material, F: torch.Tensor, n_increments: int = 1,
                       options: FhOptions | None = None, tangent_options: FhOptions | None = None) -> torch.Tensor:
    """Homogenized stress Pbar(Fbar) (9 entries, the shape of Fbar) with dPbar/dFbar for backward.

    F is the caller's CUDA float64 field [9, nx, ny, nz]; forward leaves the
    converged state in it and backward evaluates the homogenized tangent
    there, so F must not change between the two.
    """
    return _HomogenizedStress.apply(Fbar, cell, mat, F, n_increments, options, tangent_options)


class _HomogenizedModulus(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, cell, mat, ijkl, dscale, options):
        shape = tuple(cell.shape)
        zero = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        C = cell.fft_homog_tangent(mat, zero, options)
        i, j, k, l = ijkl
        ctx.cell, ctx.mat, ctx.ijkl, ctx.dscale, ctx.opt = cell, mat, ijkl, dscale, options
        return torch.tensor(C[3 * i + j, 3 * k + l], dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, grad):
        out = torch.empty(tuple(ctx.cell.shape), dtype=torch.float64, device="cuda")
        ctx.cell.fft_homog_sensitivity(ctx.mat, ctx.ijkl, ctx.dscale, out, ctx.opt)
        return out * grad.to(out.device), None, None, None, None, None


def homogenized_modulus(rho: torch.Tensor, cell: Context, mat: Material, ijkl, dscale: torch.Tensor,
                        options: FhOptions | None = None) -> torch.Tensor:
    """Cbar_ijkl of a small-strain linear elastic cell, differentiable in rho.

    ``mat.scale`` must hold s(rho) and ``dscale`` ds/drho (CUDA float64 fields
    of the grid shape); the gradient with respect to rho is the voxel field of
    fft_homog_sensitivity times the incoming scalar gradient.
    """
    return _HomogenizedModulus.apply(rho, cell, mat, tuple(int(v) for v in ijkl), dscale,
                                     options if options is not None else default_options(cg_tol=1e-12))


class _HomogenizedStressOfDensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, cell, mat, Fbar, F, dscale, n_increments, options, adjoint_options):
        fb = Fbar.detach().to("cpu", torch.float64).reshape(9).numpy() if torch.is_tensor(Fbar) else Fbar
        pbar, _, _ = cell.fft_homog_solve(mat, fb, F, n_increments=n_increments, options=options)
        ctx.cell, ctx.mat, ctx.F, ctx.dscale, ctx.aopt = cell, mat, F, dscale, adjoint_options
        return torch.as_tensor(pbar, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, grad):
        # sum_ab g_ab dPbar_ab/drho: one adjoint (unit-response) solve per entry the gradient touches
        g = grad.detach().to("cpu", torch.float64).reshape(9).numpy()
        field = torch.empty(tuple(ctx.cell.shape), dtype=torch.float64, device="cuda")
        out = torch.zeros_like(field)
        for ab in range(9):
            if g[ab] == 0.0:
                continue
            ctx.cell.fft_homog_stress_sensitivity(ctx.mat, ctx.F, (ab // 3, ab % 3), ctx.dscale, field, ctx.aopt)
            out.add_(field, alpha=float(g[ab]))
        return out, None, None, None, None, None, None, None, None


def homogenized_stress_of_density(rho: torch.Tensor, cell: Context, mat: Material, Fbar, F: torch.Tensor,
                                  dscale: torch.Tensor, n_increments: int = 1, options: FhOptions | None = None,
                                  adjoint_options: FhOptions | None = None) -> torch.Tensor:
    """Pbar (9 entries) of the cell under Fbar, differentiable in the voxel density rho.

    ``mat.scale`` must hold s(rho) and ``dscale`` ds/drho (CUDA float64 fields of the grid shape); F is the
    caller's CUDA float64 field [9, nx, ny, nz], left at the converged state by forward and read there by
    backward (it must not change in between). The gradient is sum_ab g_ab dPbar_ab/drho, each term from
    fft_homog_stress_sensitivity (the adjoint of the linearised equilibrium is a unit response, since the
    tangent has major symmetry).
    """
    return _HomogenizedStressOfDensity.apply(rho, cell, mat, Fbar, F, dscale, n_increments, options,
                                             adjoint_options if adjoint_options is not None
                                             else default_options(cg_tol=1e-12))


__all__ = ["homogenized_stress", "homogenized_modulus", "homogenized_stress_of_density"]
