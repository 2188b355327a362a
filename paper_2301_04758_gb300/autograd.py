"""torch.autograd interface to the sweep and its adjoint.

`transport_phi(mesh, sigma_t, sigma_s, omega, weights, ...)` returns the scalar flux
phi = sum_d w_d psi_d of one transport inversion (Eq. transport with the scattering
source sigma_s phi_in / (4 pi) for a fixed phi_in), as nodal DG coefficients [E][n].
It is differentiable in sigma_t and sigma_s: the backward pass calls the library's
adjoint sweep (vef_adjoint_sweep) with g = dL/dphi and the forward psi as checkpoint,
so any loss built on phi in torch -- e.g. a region integral (g * phi).sum() with g from
Mesh.region_weights -- gets dL/dsigma_t and dL/dsigma_s per element.  All transport
work runs in the library's kernels; this module only wires them into autograd.
"""
import torch


class _TransportPhi(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_t, sigma_s, mesh, omega, weights, phi_in, source, inflow, ckpt):
        psi = mesh.sweep(sigma_t, sigma_s, omega, weights, phi_in=phi_in, source=source, inflow=inflow)
        phi = mesh.moments(psi, omega, weights, outputs=("phi",))["phi"]
        if ckpt == "fp32":   # the checkpoint at half the memory
            psi = psi.float()
        ctx.save_for_backward(sigma_t, sigma_s, psi)   # psi kept per direction as checkpoint
        ctx.mesh, ctx.omega, ctx.weights, ctx.phi_in = mesh, omega, weights, phi_in
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        sigma_t, sigma_s, psi = ctx.saved_tensors
        dst, dss, _ = ctx.mesh.adjoint(sigma_t, sigma_s, ctx.omega, ctx.weights, psi,
                                       grad_phi.contiguous(), phi_in=ctx.phi_in)
        if not ctx.needs_input_grad[0]:
            dst = None
        if not ctx.needs_input_grad[1]:
            dss = None
        return dst, dss, None, None, None, None, None, None, None


def transport_phi(mesh, sigma_t, sigma_s, omega, weights, phi_in=None, source=None, inflow=None,
                  ckpt="fp64"):
    """phi [E][n] of one transport inversion, differentiable in sigma_t and sigma_s.

    sigma_t, sigma_s: CUDA float64 [E] (leaf tensors may require grad); phi_in [E][n] or
    None (then dL/dsigma_s is zero: sigma_s has no effect); source [E][n] or [D][E][n];
    inflow [D][N_bf][nq] or None; omega [D][2] and weights [D] on the host.  ckpt: "fp64"
    keeps the forward psi for the backward pass as it is, "fp32" keeps an FP32 copy (half
    the memory; the gradients then carry its rounding, about 1e-7 relative)."""
    if ckpt not in ("fp64", "fp32"):
        raise ValueError("ckpt must be 'fp64' or 'fp32'")
    phi = _TransportPhi.apply(sigma_t, sigma_s, mesh, omega, weights, phi_in, source, inflow, ckpt)
    return phi
