"""Seeded synthetic inputs for the double-MRT phase-change LBM.

Both the FP64 oracle and the CUDA library are fed from here.  This module
holds none of the method's arithmetic: it only draws random fields, smooths
them, and writes down the dimensionless parameter sets of the workloads.  The
one formula it applies is the Kozeny-Carman form of Eq. (6) to turn a
porosity field into the *input* permeability field, as the workload recipe
asks; the lattice code evaluates Eq. (6) again, separately, at every step.

Every workload is a ``Workload``: lattice size, a parameter dict whose keys
are the parameter names shared by ``oracle.Oracle`` and
``paper_1503_08406_gb300.Lattice``, and float64 fields ``phi`` (porosity),
``K`` (fully liquid permeability, lattice units), ``T0`` (initial
temperature) and ``fl0`` (initial liquid fraction), row-major [ny][nx].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    params: dict
    phi: np.ndarray
    K: np.ndarray
    T0: np.ndarray
    fl0: np.ndarray
    wall_T_left: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny


def smoothed_gaussian(n: int, sigma_cells: float, seed: int, shape=None) -> np.ndarray:
    """Unit-variance, zero-mean Gaussian noise smoothed with a periodic Gaussian kernel.

    i.i.d. N(0,1) noise on an n x n (or ``shape``) grid, convolved (FFT,
    periodic) with a Gaussian of standard deviation ``sigma_cells`` cells and
    renormalised to zero mean and unit variance.
    """
    ny, nx = shape if shape is not None else (n, n)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((ny, nx))
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.fftfreq(nx)[None, :]
    kern = np.exp(-2.0 * np.pi ** 2 * sigma_cells ** 2 * (kx ** 2 + ky ** 2))
    s = np.real(np.fft.ifft2(np.fft.fft2(g) * kern))
    s -= s.mean()
    sd = s.std()
    return s / sd if sd > 0 else s


def kozeny_carman_K(phi: np.ndarray, mean_K: float) -> np.ndarray:
    """Input permeability K = phi^3 d^2 / (175 (1 - phi)^2), Eq. (6), with the
    particle diameter d chosen so that mean(K) = mean_K."""
    shape = phi ** 3 / (175.0 * (1.0 - phi) ** 2)
    d2 = mean_K / shape.mean()
    return shape * d2


def heterogeneous_porosity(n: int, seed: int, sigma_cells: float = 16.0) -> np.ndarray:
    """phi = clip(0.45 + 0.15 g, 0.3, 0.6), g unit-variance smoothed noise."""
    g = smoothed_gaussian(n, sigma_cells, seed)
    return np.clip(0.45 + 0.15 * g, 0.3, 0.6)


def block_average(a: np.ndarray, b: int) -> np.ndarray:
    ny, nx = a.shape
    return a.reshape(ny // b, b, nx // b, b).mean(axis=(1, 3))


def _cavity_fields(n: int, phi, K, hot_wall: bool = True):
    T0 = np.zeros((n, n))
    fl0 = np.zeros((n, n))
    if hot_wall:
        T0[:, 0] = 1.0
        fl0[:, 0] = 1.0
    phi = np.broadcast_to(np.asarray(phi, dtype=np.float64), (n, n)).copy()
    K = np.broadcast_to(np.asarray(K, dtype=np.float64), (n, n)).copy()
    return phi, K, T0, fl0


def conduction_slab(nx: int = 256, ny: int = 4, phi: float = 0.5, St: float = 1.0,
                    sigma: float = 1.0, alpha: float = 0.02, Da: float = 1e-2) -> Workload:
    """Conduction melting of a semi-infinite porous slab.

    256 x 4 lattice periodic in y, porosity 0.5, Ste = 1, sigma = 1, solid at
    T = T_m = 0, wall node x = 0 held at 1 and x = nx-1 at 0, no flow.
    alpha = 0.02 gives tau_T = 0.6 (Sec. 4.1 uses the same alpha_s).
    """
    csT2 = 0.2  # (4 + varpi)/10 with varpi = -2, Sec. 4 preamble
    params = dict(bc=("dirichlet", "dirichlet", "periodic", "periodic"),
                  T_bc=(1.0, 0.0, 0.0, 0.0), flow=0, St=St, sigma=sigma, dT=1.0,
                  T_s=0.0, T_l=0.0, tau_T=0.5 + alpha / (sigma * csT2), H=float(nx))
    T0 = np.zeros((ny, nx))
    fl0 = np.zeros((ny, nx))
    T0[:, 0] = 1.0
    fl0[:, 0] = 1.0
    return Workload("conduction_slab_%dx%d" % (nx, ny), nx, ny, params,
                    np.full((ny, nx), phi), np.full((ny, nx), Da * nx * nx), T0, fl0,
                    meta=dict(alpha=alpha))


def convection_cavity(n: int = 256, phi: float = 0.4, Da: float = 1e-4, Ra: float = 1e5,
                      Pr: float = 1.0, St: float = 1.0, sigma: float = 1.0) -> Workload:
    """Convection melting in a square porous cavity.

    Hot left wall T = 1, cold right wall T = 0 = T_m, adiabatic top and
    bottom, uniform porosity, K = Da H^2 with H = n, solid at T = 0 initially.
    """
    params = dict(bc=("dirichlet", "dirichlet", "adiabatic", "adiabatic"),
                  T_bc=(1.0, 0.0, 0.0, 0.0), flow=1, Ra=Ra, Pr=Pr, Ma=0.1, J=1.0,
                  lambda_=1.0, sigma=sigma, St=St, dT=1.0, H=float(n), T_ref=0.0,
                  T_s=0.0, T_l=0.0)
    phi_f, K, T0, fl0 = _cavity_fields(n, phi, Da * n * n)
    return Workload("convection_cavity_%d" % n, n, n, params, phi_f, K, T0, fl0)


def heterogeneous_cavity(n: int = 2048, seed: int = 3, Da: float = 1e-4, Ra: float = 1e6,
                         Pr: float = 1.0, St: float = 1.0, sigma: float = 1.0,
                         source_n: int | None = None) -> Workload:
    """Heterogeneous large cavity.

    Porosity phi = clip(0.45 + 0.15 g, 0.3, 0.6) with g seeded unit-variance
    noise smoothed by a 16-cell Gaussian; K from Kozeny-Carman with the
    particle diameter giving mean(K) = Da H^2.  With ``source_n`` > n the
    field is drawn at source_n^2 and block-averaged down to n^2 (the
    downsampled copy used for the precision study); Ra and Da are kept.
    """
    if source_n is not None and source_n != n:
        phi = block_average(heterogeneous_porosity(source_n, seed), source_n // n)
    else:
        phi = heterogeneous_porosity(n, seed)
    K = kozeny_carman_K(phi, Da * n * n)
    params = dict(bc=("dirichlet", "dirichlet", "adiabatic", "adiabatic"),
                  T_bc=(1.0, 0.0, 0.0, 0.0), flow=1, Ra=Ra, Pr=Pr, Ma=0.1, J=1.0,
                  lambda_=1.0, sigma=sigma, St=St, dT=1.0, H=float(n), T_ref=0.0,
                  T_s=0.0, T_l=0.0)
    phi_f, K_f, T0, fl0 = _cavity_fields(n, phi, K)
    return Workload("heterogeneous_cavity_%d_seed%d" % (n, seed), n, n, params,
                    phi_f, K_f, T0, fl0, meta=dict(seed=seed, Da=Da))


def parity_cavity(n: int = 256, seed: int = 1, Ra: float = 1e5) -> Workload:
    """The convection cavity with the heterogeneous porosity recipe (seed 1)."""
    w = heterogeneous_cavity(n=n, seed=seed, Ra=Ra)
    w.name = "parity_cavity_%d_seed%d" % (n, seed)
    return w


def melted_cavity(n: int = 64, seed: int = 7, Ra: float = 1e5, melted_cols: int | None = None,
                  Da: float = 1e-3) -> Workload:
    """Small cavity whose left part starts liquid and warm, so that flow, the
    moving front and the flow mask are all exercised within a few hundred steps."""
    w = heterogeneous_cavity(n=n, seed=seed, Ra=Ra, Da=Da)
    m = melted_cols if melted_cols is not None else n // 3
    x = np.arange(n)[None, :]
    w.fl0[:, :m] = 1.0
    w.T0[:, :] = np.where(x < m, 1.0 - x / (2.0 * m), 0.0)
    w.T0[:, 0] = 1.0
    w.name = "melted_cavity_%d_seed%d" % (n, seed)
    return w


def periodic_box(n: int = 32, seed: int = 11, flow: int = 1, Ra: float = 1e4,
                 St: float = 0.5, T_s: float = 0.0, T_l: float = 0.0,
                 ny: int | None = None) -> Workload:
    """Fully periodic n x ny box (no walls): a warm liquid blob, a solid block,
    random porosity.  Closed, so total mass and total enthalpy are invariants."""
    nx = n
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    phi = np.clip(0.45 + 0.1 * smoothed_gaussian(0, 3.0, seed, shape=(ny, nx)), 0.3, 0.6)
    K = kozeny_carman_K(phi, 1e-2 * ny * ny)
    yy, xx = np.mgrid[0:ny, 0:nx]
    r2 = (xx - nx / 3) ** 2 + (yy - ny / 2) ** 2
    T0 = np.where(r2 < (min(nx, ny) / 5) ** 2, 0.8, -0.2) + 0.05 * rng.standard_normal((ny, nx))
    fl0 = np.where(T0 > 0, 1.0, 0.0)
    fl0[(xx > 2 * nx // 3) & (yy > ny // 4) & (yy < 3 * ny // 4)] = 0.0
    params = dict(bc=("periodic",) * 4, T_bc=(0.0,) * 4, flow=flow, Ra=Ra, Pr=1.0,
                  Ma=0.1, J=1.0, lambda_=1.0, sigma=1.0, St=St, dT=1.0, H=float(ny),
                  T_ref=0.0, T_s=T_s, T_l=T_l)
    if not flow:
        params["tau_T"] = 0.8
    return Workload("periodic_box_%dx%d_seed%d" % (nx, ny, seed), nx, ny, params, phi, K, T0, fl0)


def corner_solidification(n: int = 100, St: float = 4.0, T_i: float = 0.3, T_c: float = -1.0,
                          T_s: float = -0.02, T_l: float = 0.02, alpha: float = 0.02) -> Workload:
    """Solidification in a semi-infinite corner (Sec. 4.2 parameters).

    Liquid at T_i, left and bottom walls lowered to T_c, phi = 1, sigma = 1,
    St = 4 with dT = T_m - T_c = 1, mushy band [T_s, T_l].  The far (right,
    top) walls are adiabatic so the far field is one-dimensional.  No flow.
    """
    csT2 = 0.2
    params = dict(bc=("dirichlet", "adiabatic", "dirichlet", "adiabatic"),
                  T_bc=(T_c, 0.0, T_c, 0.0), flow=0, St=St, sigma=1.0, dT=1.0,
                  T_s=T_s, T_l=T_l, tau_T=0.5 + alpha / csT2, H=n / 2.0)
    T0 = np.full((n, n), T_i)
    fl0 = np.ones((n, n))
    T0[0, :] = T_c
    T0[:, 0] = T_c
    fl0[0, :] = 0.0
    fl0[:, 0] = 0.0
    return Workload("corner_solidification_%d" % n, n, n, params, np.ones((n, n)),
                    np.full((n, n), 1e3), T0, fl0, meta=dict(alpha=alpha, T_i=T_i, T_c=T_c))


def bench_cavity(n: int = 2048, seed: int = 3, melted: float = 0.875, Ra: float = 1e6,
                 Da: float = 1e-4) -> Workload:
    """The heterogeneous cavity part-way through melting: the left ``melted``
    fraction of the columns is liquid with T falling linearly from the hot
    wall (1) to the front (0); the rest is solid at T_m = 0.  The flow lattice
    then runs on most nodes and a full-height front exercises the enthalpy
    solve."""
    w = heterogeneous_cavity(n=n, seed=seed, Ra=Ra, Da=Da)
    m = int(round(melted * n))
    x = np.arange(n)[None, :]
    w.fl0[:, :m] = 1.0
    w.T0[:, :] = np.where(x < m, 1.0 - x / float(m), 0.0)
    w.T0[:, 0] = 1.0
    w.name = "heterogeneous_cavity_%d_seed%d_melted%g" % (n, seed, melted)
    w.meta.update(melted=melted)
    return w


BATCH_SIDES = (64, 96, 128, 192, 256, 384, 512)


def batched_cavities(count: int = 64, seed: int = 4) -> list:
    """Uneven convection-melting cavities for the batched runs: side drawn
    uniformly from BATCH_SIDES, Ra log-uniform in [1e4, 1e7], Da log-uniform
    in [1e-5, 1e-2], porosity uniform in [0.3, 0.9], Pr = 1, St uniform in
    [0.1, 1] (one seeded generator, drawn in that order per cavity)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(BATCH_SIDES))
        Ra = float(10.0 ** rng.uniform(4.0, 7.0))
        Da = float(10.0 ** rng.uniform(-5.0, -2.0))
        eps = float(rng.uniform(0.3, 0.9))
        St = float(rng.uniform(0.1, 1.0))
        w = convection_cavity(n, phi=eps, Da=Da, Ra=Ra, St=St)
        w.name = "batched_%02d_n%d" % (i, n)
        w.meta.update(Ra=Ra, Da=Da, phi=eps, St=St, seed=seed)
        out.append(w)
    return out


def two_phase_slab(ratio: float = 10.0, nx: int = 200, ny: int = 6, alpha_s: float = 0.02,
                   St: float = 1.0) -> Workload:
    """Sec. 4.1 two-phase conduction melting: 200 x 6, periodic y, no flow,
    phi = sigma = 1, T_b = 1 at x = 0, T_m = 0 with the mushy band
    [-0.02, 0.02], solid initially at T_i = -1 (the right wall node held at
    T_i too), alpha_s = 0.02 and alpha_l = ratio alpha_s (tau_T from alpha_l,
    the solid value through alpha_ratio)."""
    csT2 = 0.2
    alpha_l = ratio * alpha_s
    params = dict(bc=("dirichlet", "dirichlet", "periodic", "periodic"),
                  T_bc=(1.0, -1.0, 0.0, 0.0), flow=0, St=St, sigma=1.0, dT=1.0,
                  T_s=-0.02, T_l=0.02, tau_T=0.5 + alpha_l / csT2, alpha_ratio=ratio,
                  H=float(nx))
    T0 = np.full((ny, nx), -1.0)
    T0[:, 0] = 1.0
    fl0 = np.zeros((ny, nx))
    fl0[:, 0] = 1.0
    return Workload("two_phase_slab_%dx%d_ratio%g" % (nx, ny, ratio), nx, ny, params,
                    np.ones((ny, nx)), np.full((ny, nx), 1e3), T0, fl0,
                    meta=dict(alpha_s=alpha_s, alpha_l=alpha_l, T_b=1.0, T_i=-1.0, T_m=0.0))


def adjoint_slab(nx: int = 2048, ny: int = 512, seed: int = 0) -> Workload:
    """The conduction slab of two_phase_slab (ratio 1) set up for gradients:
    a wide mushy band T_s / T_l = -/+0.3 (fronts stay off the clamps),
    porosity 0.6 + 0.2 U(0, 1) per node (seeded) and the left wall profile
    T_w(y) = 1 + 0.2 sin(2 pi y / ny) in `wall_T_left`."""
    w = two_phase_slab(1.0, nx=nx, ny=ny)
    params = dict(w.params)
    params.pop("alpha_ratio")
    params.update(T_s=-0.3, T_l=0.3)
    phi = 0.6 + 0.2 * np.random.default_rng(seed).random((ny, nx))
    tw = 1.0 + 0.2 * np.sin(2 * np.pi * np.arange(ny) / ny)
    return Workload("adjoint_slab_%dx%d_seed%d" % (nx, ny, seed), nx, ny, params, phi, w.K,
                    w.T0, w.fl0, wall_T_left=tw, meta=dict(w.meta))



def adjoint_cavity(n: int = 512, seed: int = 5, source_n: int = 512, melted: float = 0.0,
                   T_l: float = 0.05, Ra: float = 1e6, Da: float = 1e-4,
                   T_c: float = -0.05) -> Workload:
    """The inverse-problem cavity: Ra = 1e6, Pr = 1, Ste = 1, hot left wall
    (profile 1 in `wall_T_left`, one entry per row), cold right wall and
    initial solid at T_c = -0.05, below the melting range [T_s, T_l] = [0, T_l]
    by its width: a solid at T_s itself would sit on the clamp's kink of
    Eq. (42), where the objectives have only one-sided derivatives.

    Fields drawn at source_n^2 and block-averaged to n^2 when n < source_n
    (the small copies keep the large field's pattern):
    - ln K: seeded unit-variance noise smoothed to a Gaussian autocorrelation
      of 32 cells (kernel sigma 32 / sqrt 2), times 0.5, shifted so that
      mean(K) = Da H^2;
    - porosity: clip(0.45 + 0.15 g, 0.3, 0.6) as in the heterogeneous cavity
      (16-cell smoothing, seed + 1).
    Mushy band [T_s, T_l] = [0, T_l] above the melting point: 0 < f_l < 1
    holds across a few cells at the front.  ``melted`` > 0 starts the left
    fraction of the columns liquid with T falling linearly from 1 to 0 (short
    runs with the front already moving); the solid beyond is at T_c.
    """
    big = max(source_n, n)
    g = smoothed_gaussian(big, 32.0 / np.sqrt(2.0), seed)
    phi = heterogeneous_porosity(big, seed + 1)
    if big != n:
        g = block_average(g, big // n)
        phi = block_average(phi, big // n)
    lnK = 0.5 * g
    K = np.exp(lnK)
    K *= Da * n * n / K.mean()
    params = dict(bc=("dirichlet", "dirichlet", "adiabatic", "adiabatic"),
                  T_bc=(1.0, T_c, 0.0, 0.0), flow=1, Ra=Ra, Pr=1.0, Ma=0.1, J=1.0,
                  lambda_=1.0, sigma=1.0, St=1.0, dT=1.0, H=float(n), T_ref=0.0,
                  T_s=0.0, T_l=T_l)
    phi_f, K_f, T0, fl0 = _cavity_fields(n, phi, K)
    T0[:, 1:] = T_c
    if melted > 0:
        m = int(round(melted * n))
        x = np.arange(n)[None, :]
        fl0[:, :m] = 1.0
        T0[:, :] = np.where(x < m, 1.0 - x / float(m), T_c)
        T0[:, 0] = 1.0
    return Workload("adjoint_cavity_%d_seed%d%s" % (n, seed, "_melted%g" % melted if melted else ""),
                    n, n, params, phi_f, K_f, T0, fl0, wall_T_left=np.ones(n),
                    meta=dict(seed=seed, source_n=big, Da=Da))


def porous_gallium_cavity(n: int = 200, solid_sigma: bool = False) -> Workload:
    """Sec. 4.3: convection melting in a square cavity filled with porous
    media, with the paper's parameter set (the gallium / glass-bead
    experiment it compares with): Ra = 8.409e5, Da = 1.37e-5 (K = Da H^2),
    phi = 0.385, J = 1, Pr = 0.0208, lambda = alpha_e / alpha_l = 0.2719,
    alpha_l / alpha_s = 1, St = 0.1241, Ma = 0.1, H = n (200 in the paper).
    Temperatures scaled as (T - T_c) / (T_h - T_c) with T_h = 45, T_c = 20:
    hot wall 1, cold wall 0, T_m = (29.78 - 20) / 25 = 0.3912, initial solid
    at T_i = T_0 = 20 -> 0 (also the buoyancy reference).  The paper gives
    sigma = 0.8604 in the liquid and 0.8352 in the solid; by default the
    liquid value is used everywhere, with ``solid_sigma`` sigma follows f_l
    by Eq. (7) between the two (parameter sigma_solid).  The paper states no
    mushy band for this case: T_m -/+ 0.02 as in Sec. 4.1.  Adiabatic top and
    bottom."""
    T_m = (29.78 - 20.0) / 25.0
    params = dict(bc=("dirichlet", "dirichlet", "adiabatic", "adiabatic"),
                  T_bc=(1.0, 0.0, 0.0, 0.0), flow=1, Ra=8.409e5, Pr=0.0208, Ma=0.1, J=1.0,
                  lambda_=0.2719, sigma=0.8604, St=0.1241, dT=1.0, H=float(n), T_ref=0.0,
                  T_s=T_m - 0.02, T_l=T_m + 0.02)
    if solid_sigma:
        params["sigma_solid"] = 0.8352
    phi_f, K, T0, fl0 = _cavity_fields(n, 0.385, 1.37e-5 * n * n)
    return Workload("porous_gallium_cavity_%d%s" % (n, "_solid_sigma" if solid_sigma else ""),
                    n, n, params, phi_f, K, T0, fl0,
                    meta=dict(T_m=T_m, sigma_solid=0.8352))
