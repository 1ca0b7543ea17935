"""The stirred run's kinetic-energy objective as a differentiable PyTorch function.

J(sigma, eta/s, F_body) is the time average over the states after steps 1 .. N of the
fluid-cell mean of |v|^2 / 2 (v = u^i / u^0); sigma_m multiplies the amplitude of
stirring mode m at every step (Sec. "The Driving Term").  The forward pass runs the
library's fused steps with checkpoints and its hand-written adjoint (rlbm_gradient):
the gradient comes out of the same call, and `backward` scales it by the incoming
gradient.  Memory: about 2 sqrt(N) lattice states (checkpoint segment sqrt(N)).
"""
import numpy as np
import torch

from . import rlbm


class StirredKineticEnergy(torch.autograd.Function):
    """J = StirredKineticEnergy.apply(sigma, eta_over_s, body_force, spec).

    sigma (nmodes,), eta_over_s (scalar) and body_force (2,) are float64 tensors; spec is
    a dict with the lattice keywords of rlbm.Lattice (nx, ny, precision, kmin, kmax,
    force_amp, seed, init fields, ...), `nsteps` and optionally `segment` and `state`
    (a (Q, ny, nx) start state with `step`, as from Lattice.get_state)."""

    @staticmethod
    def forward(ctx, sigma, eta_over_s, body_force, spec):
        kw = {k: v for k, v in spec.items() if k not in ("nx", "ny", "nsteps", "segment", "state", "step")}
        kw["eta_over_s"] = float(eta_over_s)
        kw["body_force"] = tuple(float(b) for b in body_force.detach().cpu().reshape(2))
        lat = rlbm.Lattice(spec["nx"], spec["ny"], **kw)
        try:
            if spec.get("state") is not None:
                lat.set_state(spec["state"], spec.get("step", 0))
            if lat.num_modes:
                lat.set_mode_scale(sigma.detach().cpu().numpy().astype(np.float64))
            J, gs, ge, gb = lat.gradient(spec["nsteps"], spec.get("segment", 0))
        finally:
            lat.close()
        dev = sigma.device
        ctx.save_for_backward(torch.as_tensor(gs, dtype=torch.float64, device=dev),
                              torch.tensor(ge, dtype=torch.float64, device=dev),
                              torch.as_tensor(gb, dtype=torch.float64, device=dev))
        return torch.tensor(J, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, gJ):
        gs, ge, gb = ctx.saved_tensors
        return gJ * gs, gJ * ge, gJ * gb, None


def kinetic_energy(sigma, eta_over_s, body_force, **spec):
    """Convenience wrapper: J as a differentiable scalar tensor."""
    return StirredKineticEnergy.apply(sigma, eta_over_s, body_force, spec)
