"""torch.autograd.Functions for objectives of a run, their gradients from the
CUDA adjoints (lbm_adjoint for the conduction step, lbm_adjoint_coupled with
the flow lattice on).

Inputs that are CUDA tensors go to the library as device pointers, and the
gradients come back as CUDA tensors written by the library: nothing of the
run passes through host memory.  Host tensors take the host-pointer path.
"""
import torch


def _on_device(*ts):
    return all(isinstance(t, torch.Tensor) and t.is_cuda for t in ts)


def _field(t):
    """A field for Lattice.set_fields: the tensor itself when it lives on the
    GPU (the binding passes its device pointer), else a host array."""
    t = t.detach()
    return t if t.is_cuda else t.cpu().numpy()


def _as(t, like):
    return torch.as_tensor(t, device=like.device)


class MeltedFraction(torch.autograd.Function):
    """J = melted fraction after `nsteps` steps of `lattice` started from
    (T0, fl0) with the porosity field phi and the left wall profile
    wall_T_left; backward returns dJ/dphi and dJ/dwall_T_left from the adjoint.

    Usage: J = MeltedFraction.apply(phi, wall_T_left, lattice, K, T0, fl0, nsteps)
    """

    @staticmethod
    def forward(ctx, phi, wall_T_left, lattice, K, T0, fl0, nsteps, checkpoint_every=0):
        dev = _on_device(phi, wall_T_left)
        lattice.set_fields(_field(phi), K, T0, fl0, _field(wall_T_left))
        J, dphi, dtw = lattice.adjoint(int(nsteps), "melt", int(checkpoint_every), device=dev)
        ctx.save_for_backward(_as(dphi, phi), _as(dtw, wall_T_left))
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
        dev = _on_device(phi, wall_T_left)
        lattice.set_fields(_field(phi), K, T0, fl0, _field(wall_T_left))
        J, dphi, dtw = lattice.adjoint(int(nsteps), "nusselt", int(checkpoint_every), device=dev)
        ctx.save_for_backward(_as(dphi, phi), _as(dtw, wall_T_left))
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
    def forward(ctx, phi, lnK, wall_T_left, lattice, T0, fl0, nsteps, objective="melt",
                checkpoint_every=0):
        dev = _on_device(phi, lnK, wall_T_left)
        K = torch.exp(lnK.detach())   # the permeability the lattice takes
        lattice.set_fields(_field(phi), _field(K), T0, fl0, _field(wall_T_left))
        J, dphi, dlnK, dtw = lattice.adjoint_coupled(int(nsteps), objective,
                                                     int(checkpoint_every), device=dev)
        ctx.save_for_backward(_as(dphi, phi), _as(dlnK, lnK), _as(dtw, wall_T_left))
        return torch.tensor(J, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, grad_J):
        dphi, dlnK, dtw = ctx.saved_tensors
        g = grad_J.to(dphi.dtype)
        return g * dphi, g * dlnK, g * dtw, None, None, None, None, None, None
