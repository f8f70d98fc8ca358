"""The torch.autograd.Functions' plumbing on the host, with a stand-in for
the lattice (the CUDA adjoints themselves are checked in the GPU tests): the
fields reach set_fields, the objective and its gradients come back, and
backward scales them by the incoming gradient."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


class _FakeLattice:
    def __init__(self):
        self.fields = None

    def set_fields(self, phi, K, T0, fl0, wall_T_left=None):
        self.fields = (phi, K, T0, fl0, wall_T_left)

    def adjoint_coupled(self, nsteps, objective="melt", checkpoint_every=0, mu_sweeps=0,
                        device=False):
        assert not device   # host tensors in, host arrays out
        phi, K, _, _, tw = self.fields
        return (float(phi.sum() + np.log(K).sum() + tw.sum()), 2 * np.ones_like(phi),
                3 * np.ones_like(K), 4 * np.ones_like(tw))

    def adjoint(self, nsteps, objective="melt", checkpoint_every=0, mu_sweeps=0, device=False):
        assert not device
        phi, _, _, _, tw = self.fields
        return float(phi.sum() + tw.sum()), 5 * np.ones_like(phi), 6 * np.ones_like(tw)

    def adjoint_melt(self, nsteps, checkpoint_every=0, mu_sweeps=0):
        return self.adjoint(nsteps, "melt")


def test_coupled_objective_plumbing():
    from paper_1503_08406_gb300.autograd import CoupledObjective
    lat = _FakeLattice()
    phi = torch.full((3, 4), 0.5, dtype=torch.float32, requires_grad=True)
    lnK = torch.zeros((3, 4), dtype=torch.float32, requires_grad=True)
    tw = torch.ones(3, dtype=torch.float32, requires_grad=True)
    J = CoupledObjective.apply(phi, lnK, tw, lat, np.zeros((3, 4)), np.zeros((3, 4)), 7, "nusselt")
    assert abs(J.detach().item() - 9.0) < 1e-6   # phi 12 x 0.5, ln K 0, wall 3 x 1
    np.testing.assert_allclose(lat.fields[1], 1.0)   # K = exp(lnK)
    (0.5 * J).backward()
    np.testing.assert_allclose(phi.grad.numpy(), 1.0)
    np.testing.assert_allclose(lnK.grad.numpy(), 1.5)
    np.testing.assert_allclose(tw.grad.numpy(), 2.0)


@pytest.mark.parametrize("name", ["MeltedFraction", "HotWallNusselt"])
def test_conduction_objectives_plumbing(name):
    import paper_1503_08406_gb300.autograd as A
    fn = getattr(A, name)
    lat = _FakeLattice()
    phi = torch.full((2, 5), 0.5, dtype=torch.float32, requires_grad=True)
    tw = torch.ones(2, dtype=torch.float32, requires_grad=True)
    J = fn.apply(phi, tw, lat, np.ones((2, 5)), np.zeros((2, 5)), np.zeros((2, 5)), 3)
    (3.0 * J).backward()
    np.testing.assert_allclose(phi.grad.numpy(), 15.0)
    np.testing.assert_allclose(tw.grad.numpy(), 18.0)
