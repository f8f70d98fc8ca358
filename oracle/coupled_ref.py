"""FP64 CPU reference for the adjoint of the coupled step (flow lattice on).

Test infrastructure: only tests/ may import this module.

It restates, in plain PyTorch CPU operations on float64 tensors, the step the
C oracle runs with the flow lattice on (Sec. 3), so that torch.autograd gives
the exact derivative of that step's map with respect to the porosity field,
the logarithm of the permeability field and the left wall's temperature
profile:

- flow (Sec. 3.1): density and the velocity of Eq. (24)-(28) with the
  Darcy-Forchheimer force of Eq. (4)-(6) at varphi = phi f_l(n) and
  K_eff = K f_l^3 ((1 - phi) / (1 - phi f_l))^2, Boussinesq buoyancy of
  Eq. (5) from the temperature at the start of the step; the MRT collision
  m+ = m - Lambda (m - m^eq) + (I - Lambda / 2) S of Eq. (16)-(23); streaming
  of Eq. (21) with halfway bounce-back on links into nodes without flow (wall
  nodes and f_l < f_act), which keep their populations;
- thermal (Sec. 3.2, 4): non-equilibrium extrapolation on wall nodes before
  collision (inward neighbour; the diagonal one at corners), the D2Q5 MRT
  collision of Eq. (35) with n^eq of Eq. (34) at the new velocity, streaming
  of Eq. (36), and the iterative enthalpy method of Eq. (38), (40)-(42) with
  the latent source streamed to the neighbours (superposition form).

The flow nodes are chosen by f_l(n) >= f_act, a step function: its derivative
is 0 wherever it is defined, and finite differences that do not move a node
across f_act agree with it.  The clamp of Eq. (42) passes derivatives where
its output lies strictly inside (0, 1) (at a bound, the clamped side's
one-sided derivative, 0), as the CUDA adjoint takes it; a node held exactly
at T_s sits on the kink, where only one-sided derivatives exist.  Square
roots of speeds carry a 1e-300 floor so that a node at rest has a finite
derivative; the forward values are those of the oracle.  Scope: one sigma; one thermal diffusivity or, with
alpha_l != alpha_s (Sec. 4.1), the rate of the flux moments following f_l(n)
(a wall node's that of its inward node); the flow lattice on or off; any mix
of periodic axes and wall sides the oracle accepts (left and right walls
together, bottom and top together).
"""
from __future__ import annotations

import math

import numpy as np
import torch
from torch.utils.checkpoint import checkpoint

D = torch.float64

# D2Q9, Eq. (18)-(21)
EX9 = (0, 1, 0, -1, 0, 1, -1, -1, 1)
EY9 = (0, 0, 1, 0, -1, 1, 1, -1, -1)
OPP9 = (0, 3, 4, 1, 2, 7, 8, 5, 6)
W9 = torch.tensor([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=D)
M9 = torch.tensor([[1, 1, 1, 1, 1, 1, 1, 1, 1],
                   [-4, -1, -1, -1, -1, 2, 2, 2, 2],
                   [4, -2, -2, -2, -2, 1, 1, 1, 1],
                   [0, 1, 0, -1, 0, 1, -1, -1, 1],
                   [0, -2, 0, 2, 0, 1, -1, -1, 1],
                   [0, 0, 1, 0, -1, 1, 1, -1, -1],
                   [0, 0, -2, 0, 2, 1, 1, -1, -1],
                   [0, 1, -1, 1, -1, 0, 0, 0, 0],
                   [0, 0, 0, 0, 0, 1, -1, 1, -1]], dtype=D)
# D2Q5, Eq. (31)-(32)
EX5 = (0, 1, 0, -1, 0)
EY5 = (0, 0, 1, 0, -1)
N5 = torch.tensor([[1, 1, 1, 1, 1],
                   [0, 1, 0, -1, 0],
                   [0, 0, 1, 0, -1],
                   [-4, 1, 1, 1, 1],
                   [0, 1, -1, 1, -1]], dtype=D)
CS2 = 1.0 / 3.0
BC = {"periodic": 0, "dirichlet": 1, "adiabatic": 2}


class _Clamp01(torch.autograd.Function):
    """clamp(z, 0, 1) of Eq. (42), its derivative 1 where the result lies
    strictly inside (0, 1) and 0 elsewhere (torch.clamp's is 1 at the bounds
    themselves)."""

    @staticmethod
    def forward(ctx, z):
        out = torch.clamp(z, 0.0, 1.0)
        ctx.save_for_backward((out > 0.0) & (out < 1.0))
        return out

    @staticmethod
    def backward(ctx, grad):
        (open_,) = ctx.saved_tensors
        return grad * open_


def _inv_orthogonal_rows(M):
    """M^-1 = M^T (M M^T)^-1 for a matrix with orthogonal rows."""
    return M.T @ torch.diag(1.0 / (M * M).sum(dim=1))


class CoupledRef:
    """The oracle's step for a parameter set (the keys of oracle.DEFAULTS; with
    flow = 0 the flow populations stay as they are and u = 0)."""

    def __init__(self, nx: int, ny: int, params: dict):
        p = dict(params)
        self.nx, self.ny = nx, ny
        bc = [BC[b] if isinstance(b, str) else int(b) for b in p["bc"]]
        if (bc[0] == 0) != (bc[1] == 0) or (bc[2] == 0) != (bc[3] == 0):
            raise ValueError("left and right (bottom and top) are periodic together")
        self.flow = int(p.get("flow", 1))
        if float(p.get("sigma_solid", 0.0)):
            raise ValueError("one sigma")
        r = float(p.get("alpha_ratio", 0.0))
        self.alpha_ratio = r if (r > 0 and r != 1.0) else None
        self.bc = bc
        self.T_bc = [float(t) for t in p.get("T_bc", (1.0, 0.0, 0.0, 0.0))]
        self.per_x, self.per_y = bc[0] == 0, bc[2] == 0
        g = lambda k, d: float(p.get(k, d))
        self.rho0 = g("rho0", 1.0) or 1.0
        self.dT = g("dT", 1.0) or 1.0
        self.H = g("H", 0.0) or float(ny)
        self.sigma, self.St = g("sigma", 1.0), g("St", 1.0)
        self.varpi = g("varpi", -2.0)
        self.T_ref = g("T_ref", 0.0)
        self.T_s, self.T_l = g("T_s", 0.0), g("T_l", 0.0)
        self.f_act = g("f_act", 1e-3)
        self.tol = g("inner_tol", 1e-13)
        self.max_inner = int(p.get("max_inner_iters", 1000))
        csT2 = (4 + self.varpi) / 10.0
        self.csT2 = csT2
        # Sec. 4.3 relations for the relaxation times and the buoyancy
        J, Pr, Ra, Ma, lam = g("J", 1.0) or 1.0, g("Pr", 0.0), g("Ra", 0.0), g("Ma", 0.1), \
            g("lambda_", 1.0) or 1.0
        if self.flow:
            tau_nu = g("tau_nu", -1.0)
            if not tau_nu > 0:
                tau_nu = 0.5 + Ma * J * self.H * math.sqrt(3 * Pr) / math.sqrt(Ra)
            self.nu_l = CS2 * (tau_nu - 0.5) / J
            tau_T = g("tau_T", -1.0)
            if not tau_T > 0:
                tau_T = 0.5 + lam * CS2 * (tau_nu - 0.5) / (J * self.sigma * csT2 * Pr)
            g_beta = g("g_beta", -1.0)
            if not g_beta >= 0:
                alpha_l = self.nu_l / Pr
                g_beta = Ra * self.nu_l * alpha_l / (self.dT * self.H ** 3)
        else:   # conduction: tau_T given, no flow lattice
            tau_nu, self.nu_l, g_beta = 1.0, 0.0, 0.0
            tau_T = g("tau_T", -1.0)
        self.g_beta = g_beta
        self.tau_T = tau_T
        s_e, s_eps, s_q = (g("s_e", 0.0) or 1.1), (g("s_eps", 0.0) or 1.1), (g("s_q", 0.0) or 1.2)
        self.lam = torch.tensor([1, s_e, s_eps, 1, s_q, 1, s_q, 1 / tau_nu, 1 / tau_nu], dtype=D)
        ze, zn = (g("zeta_e", 0.0) or 1.5), (g("zeta_nu", 0.0) or 1.5)
        self.theta = torch.tensor([1, 1 / tau_T, 1 / tau_T, ze, zn], dtype=D)
        self.Minv = _inv_orthogonal_rows(M9)
        self.Ninv = _inv_orthogonal_rows(N5)
        self.w5 = torch.tensor([(1 - self.varpi) / 5] + [(4 + self.varpi) / 20] * 4, dtype=D)
        self.lat = self.dT / (self.sigma * self.St)
        self._walls()

    # ---- geometry ----------------------------------------------------------
    def _walls(self):
        nx, ny = self.nx, self.ny
        x = torch.arange(nx).expand(ny, nx)
        y = torch.arange(ny)[:, None].expand(ny, nx)
        vx = (~torch.tensor(self.per_x)) & ((x == 0) | (x == nx - 1))
        vy = (~torch.tensor(self.per_y)) & ((y == 0) | (y == ny - 1))
        self.wall = vx | vy
        corner = vx & vy
        # inward neighbour: the normal one on sides, the diagonal one at corners
        ix = torch.where(vx, torch.where(x == 0, 1, nx - 2), x)
        iy = torch.where(vy, torch.where(y == 0, 1, ny - 2), y)
        ix = torch.where(corner | vx, ix, x)
        iy = torch.where(corner | (vy & ~vx), iy, y)
        self.inward = (iy * nx + ix).reshape(-1)
        # side of each wall node (corners go to the vertical wall)
        side = torch.full((ny, nx), -1)
        side = torch.where(vy & (y == ny - 1), 3, side)
        side = torch.where(vy & (y == 0), 2, side)
        side = torch.where(vx & (x == nx - 1), 1, side)
        side = torch.where(vx & (x == 0), 0, side)
        self.side, self.corner = side, corner
        self.xg, self.yg = x, y

    def _shift(self, v, dx, dy, fill=0.0):
        """out(y, x) = v(y - dy, x - dx): wraps on periodic axes, `fill` where
        the source lies outside the lattice."""
        out = v
        if dy:
            out = torch.roll(out, shifts=dy, dims=-2)
            if not self.per_y:
                sl = [slice(None)] * out.dim()
                sl[-2] = slice(0, dy) if dy > 0 else slice(dy, None)
                out = out.clone()
                out[tuple(sl)] = fill
        if dx:
            out = torch.roll(out, shifts=dx, dims=-1)
            if not self.per_x:
                sl = [slice(None)] * out.dim()
                sl[-1] = slice(0, dx) if dx > 0 else slice(dx, None)
                out = out.clone()
                out[tuple(sl)] = fill
        return out

    def _inside(self, dx, dy):
        """(y, x) - (dx, dy) lies inside the lattice (or wraps)."""
        one = torch.ones(self.ny, self.nx, dtype=torch.bool)
        return self._shift(one, dx, dy, fill=False)

    # ---- flow --------------------------------------------------------------
    def _flow(self, f, T, fl, phi, K):
        """Collide and stream; returns f(n+1) and the velocity (0 off flow)."""
        active = (~self.wall) & (fl >= self.f_act)
        fls = torch.where(active, fl, torch.ones_like(fl))    # safe where unused
        fpost, ux, uy = self.collide_flow(f, T, fls, phi, K)
        fpost = torch.where(active[None], fpost, f)
        out = []
        for i in range(9):
            from_up = self._shift(fpost[i], EX9[i], EY9[i])
            up_active = self._shift(active, EX9[i], EY9[i], fill=False)
            v = torch.where(up_active, from_up, fpost[OPP9[i]])
            out.append(torch.where(active, v, f[i]))
        zero = torch.zeros_like(ux)
        return torch.stack(out), torch.where(active, ux, zero), torch.where(active, uy, zero)

    def collide_flow(self, f, T, fls, phi, K):
        """The flow collision of every node (f: [9, ...], the rest [...]):
        post-collision populations and the velocity of Eq. (26)."""
        rho0 = self.rho0
        rho = f.sum(dim=0)
        jx = sum(EX9[i] * f[i] for i in range(9))
        jy = sum(EY9[i] * f[i] for i in range(9))
        vphi = phi * fls
        G = self.g_beta * (T - self.T_ref)
        r = (1 - phi) / (1 - vphi)
        Keff = K * fls ** 3 * r * r
        CF = 1.75 / torch.sqrt(175 * vphi ** 3)
        vx = jx / rho0
        vy = jy / rho0 + 0.5 * vphi * G
        l0 = 0.5 * (1 + vphi * 0.5 * self.nu_l / Keff)
        l1 = vphi * 0.5 * CF / torch.sqrt(Keff)
        vmag = torch.sqrt(vx * vx + vy * vy + 1e-300)
        den = l0 + torch.sqrt(l0 * l0 + l1 * vmag)
        ux, uy = vx / den, vy / den
        umag = torch.sqrt(ux * ux + uy * uy + 1e-300)
        Fx = -vphi * self.nu_l / Keff * ux - vphi * CF / torch.sqrt(Keff) * umag * ux
        Fy = -vphi * self.nu_l / Keff * uy - vphi * CF / torch.sqrt(Keff) * umag * uy + vphi * G
        uu = ux * ux + uy * uy
        meq = torch.stack([rho, -2 * rho + 3 * rho0 * uu / vphi, rho - 3 * rho0 * uu / vphi,
                           rho0 * ux, -rho0 * ux, rho0 * uy, -rho0 * uy,
                           rho0 * (ux * ux - uy * uy) / vphi, rho0 * ux * uy / vphi])
        uF = ux * Fx + uy * Fy
        S = torch.stack([torch.zeros_like(rho), 6 * rho0 * uF / vphi, -6 * rho0 * uF / vphi,
                         rho0 * Fx, -rho0 * Fx, rho0 * Fy, -rho0 * Fy,
                         2 * rho0 * (ux * Fx - uy * Fy) / vphi,
                         rho0 * (ux * Fy + uy * Fx) / vphi])
        m = torch.einsum("ki,i...->k...", M9, f)
        lam = self.lam.reshape(9, *([1] * (f.dim() - 1)))
        mp = m - lam * (m - meq) + (1 - 0.5 * lam) * S
        fpost = torch.einsum("ik,k...->i...", self.Minv, mp)
        return fpost, ux, uy

    # ---- thermal -----------------------------------------------------------
    def _geq(self, T, ux, uy):
        return torch.stack([self.w5[i] * T * (1 + (EX5[i] * ux + EY5[i] * uy)
                                              / (self.sigma * self.csT2)) for i in range(5)])

    def _wall_T(self, Tf, Tw_left):
        """Imposed temperature per wall node given its inward neighbour's T."""
        bc = self.bc
        per_side = []
        for s in range(4):
            if bc[s] == 1:
                v = Tw_left[:, None].expand(self.ny, self.nx) if s == 0 else \
                    torch.full_like(Tf, self.T_bc[s])
            else:
                v = Tf
            per_side.append(v)
        T = Tf
        for s in range(4):
            T = torch.where(self.side == s, per_side[s], T)
        # a corner on an adiabatic vertical wall takes a Dirichlet horizontal value
        for s, yv in ((2, 0), (3, self.ny - 1)):
            vert_adiabatic = torch.tensor([bc[0] == 2, bc[1] == 2])[(self.xg != 0).long()]
            if bc[s] == 1:
                sel = self.corner & (self.yg == yv) & vert_adiabatic
                T = torch.where(sel, torch.full_like(Tf, self.T_bc[s]), T)
        return T

    def _thermal(self, g, fl, a, ux, uy, Tw_left):
        n = self.nx * self.ny
        flat = lambda v: v.reshape(*v.shape[:-2], n)
        # extrapolation on wall nodes, before collision
        gf = flat(g)[:, self.inward].reshape(5, self.ny, self.nx)
        Tf = gf.sum(dim=0)
        uxf = flat(ux)[self.inward].reshape(self.ny, self.nx)
        uyf = flat(uy)[self.inward].reshape(self.ny, self.nx)
        Tw = self._wall_T(Tf, Tw_left)
        zero = torch.zeros_like(Tf)
        gw = self._geq(Tw, zero, zero) + gf - self._geq(Tf, uxf, uyf)
        gpre = torch.where(self.wall[None], gw, g)
        # collision, Eq. (35), source-free part; with alpha_l != alpha_s the rate
        # follows f_l(n), a wall node's that of its inward node
        uxc = torch.where(self.wall, zero, ux)
        uyc = torch.where(self.wall, zero, uy)
        za = None
        if self.alpha_ratio is not None:
            flw = torch.where(self.wall, flat(fl)[self.inward].reshape(self.ny, self.nx), fl)
            za = self.theta_T(flw)
        gpost = self.collide_thermal(gpre, uxc, uyc, za)
        gstar = torch.stack([self._shift(gpost[i], EX5[i], EY5[i]) for i in range(5)])
        # the iterative enthalpy method with the streamed latent source
        base = gstar.sum(dim=0)
        dTt = self.T_l - self.T_s
        fk = fl
        for _ in range(self.max_inner):
            src = torch.where(self.wall, zero, -a * (fk - fl))
            Tk = base + sum(self.w5[i] * self._shift(src, EX5[i], EY5[i]) for i in range(5))
            fnext = _Clamp01.apply((Tk + a * fk - self.T_s) / (dTt + a))
            fnext = torch.where(self.wall, fl, fnext)
            diff = float((fnext - fk).detach().abs().max())
            fk = fnext
            if diff <= self.tol:
                break
        src = torch.where(self.wall, zero, -a * (fk - fl))
        gnew = torch.stack([gstar[i] + self.w5[i] * self._shift(src, EX5[i], EY5[i])
                            for i in range(5)])
        return gnew, fk

    def collide_thermal(self, g, ux, uy, za=None):
        """The source-free D2Q5 collision of Eq. (35) with n^eq of Eq. (34) of
        every node (g: [5, ...], u: [...]); za: the flux moments' rate per node
        (default 1/tau_T)."""
        nmom = torch.einsum("ki,i...->k...", N5, g)
        T = nmom[0]
        neq = torch.stack([T, ux * T / self.sigma, uy * T / self.sigma, self.varpi * T,
                           torch.zeros_like(T)])
        th = self.theta.reshape(5, *([1] * (g.dim() - 1))).expand_as(nmom)
        if za is not None:
            th = torch.stack([th[0], za.expand_as(T), za.expand_as(T), th[3], th[4]])
        npost = nmom - th * (nmom - neq)
        return torch.einsum("ik,k...->i...", self.Ninv, npost)

    def theta_T(self, fl):
        """The flux moments' rate with alpha_l != alpha_s (Sec. 4.1):
        1 / (1/2 + (tau_T - 1/2) (f_l + (1 - f_l) alpha_s / alpha_l))."""
        r = self.alpha_ratio
        return 1.0 / (0.5 + (self.tau_T - 0.5) * (fl + (1.0 - fl) / r))

    def extrapolate_wall(self, gf, Tw, uxf, uyf):
        """Populations a wall node takes before collision from its inward
        node's (gf: [5, ...]), the imposed temperature Tw and the inward node's
        velocity: g^eq(Tw, 0) + gf - g^eq(T_f, u_f)."""
        Tf = gf.sum(dim=0)
        zero = torch.zeros_like(Tf)
        return self._geq(Tw, zero, zero) + gf - self._geq(Tf, uxf, uyf)

    # ---- steps -------------------------------------------------------------
    def step(self, f, g, fl, phi, K, Tw_left):
        T = g.sum(dim=0)
        if self.flow:
            f1, ux, uy = self._flow(f, T, fl, phi, K)
        else:
            f1, ux, uy = f, torch.zeros_like(T), torch.zeros_like(T)
        g1, fl1 = self._thermal(g, fl, phi * self.lat, ux, uy, Tw_left)
        return f1, g1, fl1

    def initial(self, T0, fl0):
        T0 = torch.as_tensor(np.asarray(T0, dtype=np.float64))
        fl0 = torch.as_tensor(np.asarray(fl0, dtype=np.float64))
        f = (W9 * self.rho0)[:, None, None] * torch.ones(9, self.ny, self.nx, dtype=D)
        g = self.w5[:, None, None] * T0[None]
        return f, g, fl0

    def node_T(self, g, Tw_left):
        """Temperature per node as the oracle reports it (walls: imposed)."""
        n = self.nx * self.ny
        Tf = g.sum(dim=0).reshape(n)[self.inward].reshape(self.ny, self.nx)
        return torch.where(self.wall, self._wall_T(Tf, Tw_left), g.sum(dim=0))

    def nusselt_hot(self, g, Tw_left):
        T = self.node_T(g, Tw_left)
        rows = slice(1, self.ny - 1) if not self.per_y else slice(None)
        q = -(-3.0 * T[rows, 0] + 4.0 * T[rows, 1] - T[rows, 2]) / 2.0 * self.H / self.dT
        return q.mean()

    def melted_fraction(self, fl):
        return fl[~self.wall].mean()

    def run(self, steps, T0, fl0, phi, K, Tw_left, objective=None, ckpt=False):
        """State after `steps` steps, and the objective ("melt": melted
        fraction at the end; "nusselt": the hot-wall Nusselt number after each
        step, averaged), each step checkpointed for autograd when ckpt."""
        f, g, fl = self.initial(T0, fl0)
        nu = 0.0
        for _ in range(steps):
            if ckpt:
                f, g, fl = checkpoint(self.step, f, g, fl, phi, K, Tw_left, use_reentrant=False)
            else:
                f, g, fl = self.step(f, g, fl, phi, K, Tw_left)
            if objective == "nusselt":
                nu = nu + self.nusselt_hot(g, Tw_left)
        J = None
        if objective == "melt":
            J = self.melted_fraction(fl)
        elif objective == "nusselt":
            J = nu / steps
        return f, g, fl, J

    def gradients(self, steps, T0, fl0, phi, K, Tw_left, objective="melt", ckpt=True):
        """The objective and its gradients with respect to phi, ln K and the
        left wall profile."""
        phi_t = torch.tensor(np.asarray(phi, dtype=np.float64), requires_grad=True)
        lnK = torch.tensor(np.log(np.asarray(K, dtype=np.float64)), requires_grad=True)
        tw = torch.tensor(np.asarray(Tw_left, dtype=np.float64), requires_grad=True)
        _, _, _, J = self.run(steps, T0, fl0, phi_t, torch.exp(lnK), tw, objective, ckpt)
        grads = torch.autograd.grad(J, (phi_t, lnK, tw), allow_unused=True)
        d_phi, d_lnK, d_tw = (torch.zeros_like(x) if gr is None else gr
                              for gr, x in zip(grads, (phi_t, lnK, tw)))   # no wall: no T_w
        return float(J.detach()), d_phi.numpy(), d_lnK.numpy(), d_tw.numpy()
