"""FP64 CPU reference for the adjoint of the conduction step (flow lattice off).

Test infrastructure: only tests/ may import this module.

It restates, in plain PyTorch CPU operations on float64 tensors, the thermal
step the C oracle runs when vartheta = 0 (Sec. 3.2 and 4): non-equilibrium
extrapolation on the wall columns before collision, the D2Q5 MRT collision of
Eq. (35) with u = 0 (n = N g, n+ = n - Theta (n - n^eq), g+ = N^-1 n+, Eq. (32),
(34), (37)), streaming (Eq. (36)), and the iterative enthalpy method of Eq.
(38), (40)-(42) with the latent source N^-1 S~ = S0 w~ streamed to the
neighbours (the superposition form the C oracle also offers, tested equal to
its literal form).  The gradient of an objective with respect to the
left-wall temperature profile and the porosity field is then the exact
derivative of this forward map, taken by torch.autograd through every step
and every inner iteration (clamp derivative 0 outside [0, 1], 1 inside).

Scope: lattices periodic in y with wall columns at x = 0 and x = nx - 1
(Dirichlet or adiabatic), no flow; tau_T the same in both phases.
"""
from __future__ import annotations

import numpy as np
import torch

# D2Q5 moments, Eq. (32): rows = (sum, x-flux, y-flux, energy, anisotropy)
N5 = torch.tensor([[1, 1, 1, 1, 1],
                   [0, 1, 0, -1, 0],
                   [0, 0, 1, 0, -1],
                   [-4, 1, 1, 1, 1],
                   [0, 1, -1, 1, -1]], dtype=torch.float64)
EX5 = (0, 1, 0, -1, 0)
EY5 = (0, 0, 1, 0, -1)


class ConductionRef:
    """The conduction step of the oracle for a given parameter set (the keys of
    oracle.DEFAULTS; tau_T must be given)."""

    def __init__(self, nx: int, ny: int, params: dict):
        bc = params["bc"]
        if not (bc[2] == "periodic" and bc[3] == "periodic"):
            raise ValueError("the reference covers lattices periodic in y")
        if bc[0] == "periodic" or bc[1] == "periodic":
            raise ValueError("the reference covers wall columns at x = 0 and nx - 1")
        if params.get("flow", 0):
            raise ValueError("the reference covers the conduction step (flow = 0)")
        self.nx, self.ny = nx, ny
        self.bc = bc
        self.T_bc = [float(t) for t in params["T_bc"]]
        varpi = float(params.get("varpi", -2.0))
        self.varpi = varpi
        self.w = torch.tensor([(1 - varpi) / 5] + [(4 + varpi) / 20] * 4, dtype=torch.float64)
        tau_T = float(params["tau_T"])
        ze = float(params.get("zeta_e", 0.0)) or 1.5
        zn = float(params.get("zeta_nu", 0.0)) or 1.5
        self.theta = torch.tensor([1.0, 1.0 / tau_T, 1.0 / tau_T, ze, zn], dtype=torch.float64)
        self.Ninv = N5.T @ torch.diag(1.0 / (N5 * N5).sum(dim=1))
        self.lat = float(params.get("dT", 1.0)) / (float(params.get("sigma", 1.0))
                                                    * float(params["St"]))
        self.T_s, self.T_l = float(params.get("T_s", 0.0)), float(params.get("T_l", 0.0))
        self.dT = float(params.get("dT", 1.0))
        self.H = float(params.get("H", 0.0)) or float(ny)   # the oracle's default
        self.tol = 1e-13
        wall = torch.zeros(ny, nx, dtype=torch.bool)
        wall[:, 0] = True
        wall[:, -1] = True
        self.wall = wall

    # one shift of a [ny, nx] field: out(y, x) = v(y - dy, x - dx), periodic in y,
    # zero where x - dx leaves the lattice
    @staticmethod
    def _shift(v, dx, dy):
        v = torch.roll(v, shifts=dy, dims=0)
        if dx == 0:
            return v
        z = torch.zeros_like(v[:, :1])
        if dx > 0:
            return torch.cat([z, v[:, :-1]], dim=1)
        return torch.cat([v[:, 1:], z], dim=1)

    def _walls(self, g, Tw_left):
        """Extrapolation before collision: g(x_b) = w~ T_w + g(x_f) - w~ T_f, u = 0."""
        cols = []
        for side, b, f in ((0, 0, 1), (1, self.nx - 1, self.nx - 2)):
            Tf = g[:, :, f].sum(dim=0)
            if self.bc[side] == "dirichlet":
                Tw = Tw_left if side == 0 else torch.full_like(Tf, self.T_bc[1])
            else:
                Tw = Tf
            cols.append((b, self.w[:, None] * Tw[None, :] + g[:, :, f] - self.w[:, None] * Tf[None, :]))
        out = g.clone()
        for b, v in cols:
            out[:, :, b] = v
        return out

    def _collide_stream(self, g):
        n = torch.einsum("ki,iyx->kyx", N5, g)
        T = n[0]
        zero = torch.zeros_like(T)
        neq = torch.stack([T, zero, zero, self.varpi * T, zero])
        npost = n - self.theta[:, None, None] * (n - neq)
        gpost = torch.einsum("ik,kyx->iyx", self.Ninv, npost)
        return torch.stack([self._shift(gpost[i], EX5[i], EY5[i]) for i in range(5)])

    def _source_streamed(self, src):
        return torch.stack([self.w[i] * self._shift(src, EX5[i], EY5[i]) for i in range(5)])

    def step(self, g, fl, a, Tw_left, max_inner: int = 1000):
        gstar = self._collide_stream(self._walls(g, Tw_left))
        base = gstar.sum(dim=0)
        fk = fl
        for _ in range(max_inner):
            src = torch.where(self.wall, torch.zeros_like(fl), -a * (fk - fl))
            Tk = base + self._source_streamed(src).sum(dim=0)
            h = Tk + a * fk
            fnext = torch.clamp((h - self.T_s) / (self.T_l - self.T_s + a), 0.0, 1.0)
            fnext = torch.where(self.wall, fl, fnext)
            diff = float((fnext - fk).detach().abs().max())
            fk = fnext
            if diff <= self.tol:
                break
        src = torch.where(self.wall, torch.zeros_like(fl), -a * (fk - fl))
        return gstar + self._source_streamed(src), fk

    def initial(self, T0):
        T0 = torch.as_tensor(np.asarray(T0, dtype=np.float64))
        return self.w[:, None, None] * T0[None]

    def run(self, steps, T0, fl0, phi, Tw_left):
        """(g, f_l) after `steps` steps; phi and Tw_left may require grad."""
        g = self.initial(T0)
        fl = torch.as_tensor(np.asarray(fl0, dtype=np.float64))
        a = phi * self.lat
        for _ in range(steps):
            g, fl = self.step(g, fl, a, Tw_left)
        return g, fl

    def melted_fraction(self, fl):
        return fl[~self.wall].mean()

    def nusselt_hot(self, g, Tw_left):
        """Left-wall Nusselt number of a state: -H/dT times the second-order
        one-sided gradient (-3 T_0 + 4 T_1 - T_2)/2, T_0 the wall's imposed
        temperature and T_1, T_2 the sums of g at x = 1, 2, averaged over the
        rows (the oracle's reduce, fourth output)."""
        T1 = g[:, :, 1].sum(dim=0)
        T2 = g[:, :, 2].sum(dim=0)
        return (-(-3.0 * Tw_left + 4.0 * T1 - T2) / 2.0 * self.H / self.dT).mean()

    def gradients(self, steps, T0, fl0, phi, Tw_left, objective: str = "melt"):
        """The objective and its gradient with respect to the porosity field
        and the left-wall temperature profile.  objective "melt": the melted
        fraction after `steps` steps; "nusselt": the left-wall Nusselt number
        after each of the `steps` steps, averaged over them."""
        if objective not in ("melt", "nusselt"):
            raise ValueError(objective)
        phi_t = torch.tensor(np.asarray(phi, dtype=np.float64), requires_grad=True)
        tw_t = torch.tensor(np.asarray(Tw_left, dtype=np.float64), requires_grad=True)
        g = self.initial(T0)
        fl = torch.as_tensor(np.asarray(fl0, dtype=np.float64))
        a = phi_t * self.lat
        nu = 0.0
        for _ in range(steps):
            g, fl = self.step(g, fl, a, tw_t)
            if objective == "nusselt":
                nu = nu + self.nusselt_hot(g, tw_t)
        J = self.melted_fraction(fl) if objective == "melt" else nu / steps
        d_phi, d_tw = torch.autograd.grad(J, (phi_t, tw_t))
        return float(J.detach()), d_phi.numpy(), d_tw.numpy()
