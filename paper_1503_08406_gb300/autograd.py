"""torch.autograd.Functions for objectives of a run, their gradients from the
CUDA adjoints (lbm_adjoint for the conduction step, lbm_adjoint_coupled with
the flow lattice on)."""
import torch


class MeltedFraction(torch.autograd.Function):
    """J = melted fraction after `nsteps` steps of `lattice` started from
    (T0, fl0) with the porosity field phi and the left wall profile
    wall_T_left; backward returns dJ/dphi and dJ/dwall_T_left from the adjoint.

    Usage: J = MeltedFraction.apply(phi, wall_T_left, lattice, K, T0, fl0, nsteps)
    """

    @staticmethod
    def forward(ctx, phi, wall_T_left, lattice, K, T0, fl0, nsteps, checkpoint_every=0):
        lattice.set_fields(phi.detach().cpu().numpy(), K, T0, fl0,
                           wall_T_left.detach().cpu().numpy())
        J, dphi, dtw = lattice.adjoint_melt(int(nsteps), int(checkpoint_every))
        ctx.save_for_backward(torch.as_tensor(dphi, device=phi.device),
                              torch.as_tensor(dtw, device=wall_T_left.device))
        return torch.tensor(J, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, grad_J):
        dphi, dtw = ctx.saved_tensors
        g = grad_J.to(dphi.dtype)
        return g * dphi, g * dtw, None, None, None, None, None, None


class HotWallNusselt(torch.autograd.Function):
    """J = the left-wall Nusselt number after each of `nsteps` steps of
    `lattice`, averaged over them, started from (T0, fl0) with the porosity
    field phi and the left wall profile wall_T_left; backward returns dJ/dphi
    and dJ/dwall_T_left from the adjoint.

    Usage: J = HotWallNusselt.apply(phi, wall_T_left, lattice, K, T0, fl0, nsteps)
    """

    @staticmethod
    def forward(ctx, phi, wall_T_left, lattice, K, T0, fl0, nsteps, checkpoint_every=0):
        lattice.set_fields(phi.detach().cpu().numpy(), K, T0, fl0,
                           wall_T_left.detach().cpu().numpy())
        J, dphi, dtw = lattice.adjoint(int(nsteps), "nusselt", int(checkpoint_every))
        ctx.save_for_backward(torch.as_tensor(dphi, device=phi.device),
                              torch.as_tensor(dtw, device=wall_T_left.device))
        return torch.tensor(J, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, grad_J):
        dphi, dtw = ctx.saved_tensors
        g = grad_J.to(dphi.dtype)
        return g * dphi, g * dtw, None, None, None, None, None, None


class CoupledObjective(torch.autograd.Function):
    """J = the melted fraction after `nsteps` steps (objective "melt") or the
    hot-wall Nusselt number averaged over them ("nusselt") of `lattice` with
    the flow lattice on, started from (T0, fl0) with the porosity field phi,
    the permeability field exp(lnK) and the left wall profile wall_T_left;
    backward returns dJ/dphi, dJ/dlnK and dJ/dwall_T_left from the adjoint
    of the coupled step (lbm_adjoint_coupled).

    Usage: J = CoupledObjective.apply(phi, lnK, wall_T_left, lattice, T0, fl0, nsteps, "melt")
    """

    @staticmethod
    def forward(ctx, phi, lnK, wall_T_left, lattice, T0, fl0, nsteps, objective="melt"):
        K = torch.exp(lnK.detach()).cpu().numpy()
        lattice.set_fields(phi.detach().cpu().numpy(), K, T0, fl0,
                           wall_T_left.detach().cpu().numpy())
        J, dphi, dlnK, dtw = lattice.adjoint_coupled(int(nsteps), objective)
        ctx.save_for_backward(torch.as_tensor(dphi, device=phi.device),
                              torch.as_tensor(dlnK, device=lnK.device),
                              torch.as_tensor(dtw, device=wall_T_left.device))
        return torch.tensor(J, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, grad_J):
        dphi, dlnK, dtw = ctx.saved_tensors
        g = grad_J.to(dphi.dtype)
        return g * dphi, g * dlnK, g * dtw, None, None, None, None, None
