"""Seeded synthetic inputs for the axisymmetric Shan-Chen LBM workloads.

This module holds the input recipes only: initial density and velocity fields
(drops, threads, flat interfaces), per-instance parameter draws and the random
Legendre amplitudes of the differentiable drop.  It contains none of the
method's arithmetic (no equilibrium, pseudopotential, force or streaming), so
that both the CUDA path and the CPU oracle can consume exactly the same inputs.

Arrays are float64 with shape [Nr, Nz] (row j = radial index, r_j = j + 1/2,
or R_i + j for the flow between discs; column k = axial index, z_k = k).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Liquid/vapour densities at G = -5 used for the drop and thread workloads
# (the static-drop workload's stated values).
RHO_L_G5, RHO_V_G5 = 1.93, 0.16


def grid(Nz: int, Nr: int):
    z = np.arange(Nz, dtype=np.float64)[None, :]
    r = (np.arange(Nr, dtype=np.float64) + 0.5)[:, None]
    return z, r


def tanh_profile(d, R, w, rho_l, rho_v):
    """rho = rho_v + (rho_l - rho_v)/2 (1 - tanh((d - R)/w)): liquid where d < R."""
    return rho_v + 0.5 * (rho_l - rho_v) * (1.0 - np.tanh((d - R) / w))


def legendre(l: int, x):
    p0, p1 = np.ones_like(x), x
    if l == 0:
        return p0
    for m in range(1, l):
        p0, p1 = p1, ((2 * m + 1) * x * p1 - m * p0) / (m + 1)
    return p1


def drop(Nz, Nr, zc, R, rho_l=RHO_L_G5, rho_v=RHO_V_G5, w=2.0, amps=(), l0=2):
    """Axisymmetric drop centred on the axis at z = zc with surface
    r_s(theta) = R (1 + sum_m amps[m] P_{l0+m}(cos theta)); u = 0."""
    z, r = grid(Nz, Nr)
    dz = z - zc
    d = np.sqrt(dz * dz + r * r)
    ct = dz / d
    s = np.zeros_like(d)
    for m, a in enumerate(amps):
        s = s + a * legendre(l0 + m, ct)
    rho = tanh_profile(d, R * (1.0 + s), w, rho_l, rho_v)
    return rho, np.zeros_like(rho), np.zeros_like(rho)


def thread(Nz, Nr, R0=25.0, eps=0.1, rho_l=RHO_L_G5, rho_v=RHO_V_G5, w=2.0, eps_u=0.0):
    """Liquid thread along the axis, R(z) = R0 (1 + eps cos(2 pi z / Nz)), one
    wavelength per domain; optional axial velocity eps_u sin(2 pi z / Nz) in the liquid."""
    z, r = grid(Nz, Nr)
    Rz = R0 * (1.0 + eps * np.cos(2 * np.pi * z / Nz))
    rho = tanh_profile(r + 0 * z, Rz, w, rho_l, rho_v)
    uz = eps_u * np.sin(2 * np.pi * z / Nz) * (rho - rho_v) / (rho_l - rho_v)
    return rho, uz, np.zeros_like(rho)


def slab(Nz, Nr, r_int, rho_in, rho_out, w=2.0):
    """Flat interface at r = r_int: rho_in below it, rho_out above (z-independent)."""
    z, r = grid(Nz, Nr)
    rho = tanh_profile(r + 0 * z, r_int, w, rho_in, rho_out)
    return rho, np.zeros_like(rho), np.zeros_like(rho)


def noisy(Nz, Nr, seed, base=1.0, amp=0.05, uamp=0.01):
    """Smooth positive random field with random velocities (parity cases)."""
    rng = np.random.default_rng(seed)
    z, r = grid(Nz, Nr)
    rho = np.full((Nr, Nz), base)
    uz = np.zeros((Nr, Nz))
    ur = np.zeros((Nr, Nz))
    for _ in range(4):
        kz = rng.integers(1, 4) * 2 * np.pi / Nz
        kr = rng.uniform(0.05, 0.4)
        ph = rng.uniform(0, 2 * np.pi, size=3)
        rho = rho + amp * base * np.cos(kz * z + ph[0]) * np.cos(kr * r)
        uz = uz + uamp * np.sin(kz * z + ph[1]) * np.cos(kr * r)
        ur = ur + uamp * np.sin(kz * z + ph[2]) * np.sin(kr * r)
    rho = rho * (1.0 + amp * 0.2 * rng.standard_normal((Nr, Nz)))
    return rho, uz, ur


def coexistence(G: float):
    """Approximate liquid/vapour densities of the Shan-Chen fluid with
    psi = 1 - exp(-rho) at coupling G < -4 (initial guesses only): the
    mechanical-equilibrium condition of Shan & Chen (1993), equal values of
    p = rho/3 + G psi^2/6 on both sides and
    int_{rho_v}^{rho_l} (p0 - p) psi'/psi^2 drho = 0."""
    from scipy.integrate import quad
    from scipy.optimize import brentq

    def p(x):
        return x / 3.0 + G * (1 - np.exp(-x)) ** 2 / 6.0

    def dpsi(x):
        return np.exp(-x)

    def psi(x):
        return 1 - np.exp(-x)

    # spinodal points: dp/drho = 0
    xs = np.linspace(1e-3, 6, 6000)
    dp = np.gradient(p(xs), xs)
    sgn = np.where(np.diff(np.sign(dp)) != 0)[0]
    if len(sgn) < 2:
        raise ValueError("G above the critical coupling: no coexistence")
    a, b = xs[sgn[0]], xs[sgn[1]]
    pmin, pmax = p(b), p(a)

    def branches(p0):
        lo = brentq(lambda x: p(x) - p0, 1e-10, a)
        hi = brentq(lambda x: p(x) - p0, b, 20.0)
        return lo, hi

    def area(p0):
        lo, hi = branches(p0)
        return quad(lambda x: (p0 - p(x)) * dpsi(x) / psi(x) ** 2, lo, hi, limit=200)[0]

    eps = 1e-9 * (pmax - pmin)
    p0 = brentq(area, max(pmin, p(1e-9)) + eps, pmax - eps)
    lo, hi = branches(p0)
    return hi, lo


@dataclass
class DiscFlow:
    """The flow between two parallel discs of Sec. III.2: a lattice of H (z)
    x Nr (r) sites whose rows start at the inlet radius, r_j = R_i + j
    (r_off = R_i - 1/2), discs (no-slip walls) half a spacing beyond the first
    and last columns, so z = k + 1/2 is the distance from the lower disc.
    The inlet row carries Middleman's creeping-flow profile,
    u_r(z, r) = -U_2 (4 R_i / H^2) z (z - H) / r, with
    U_2 = u_r(H/2, R_i) = 3 Q / (4 pi R_i H) (Eq. sol-vel-test2)."""
    H: int
    R_i: float
    Nr: int
    U2: float

    @property
    def r_off(self) -> float:
        return self.R_i - 0.5

    @property
    def z(self):
        return np.arange(self.H, dtype=np.float64) + 0.5

    @property
    def r(self):
        return (np.arange(self.Nr, dtype=np.float64) + self.R_i)[:, None]

    @property
    def Q(self) -> float:
        """Volume flow rate, Q = 4 pi R_i H U_2 / 3."""
        return 4.0 * np.pi * self.R_i * self.H * self.U2 / 3.0

    def analytic(self):
        """u_r of Middleman's solution on every site, [Nr, H]."""
        z = self.z[None, :]
        return -self.U2 * (4.0 * self.R_i / self.H ** 2) * z * (z - self.H) / self.r

    @property
    def u_in(self):
        """Radial velocity imposed on the inlet row, [H]."""
        return self.analytic()[0].copy()

    def fields(self):
        """Initial state: fluid of density 1 at rest, the inlet row already moving."""
        rho = np.ones((self.Nr, self.H))
        uz = np.zeros((self.Nr, self.H))
        ur = np.zeros((self.Nr, self.H))
        ur[0] = self.u_in
        return rho, uz, ur


def disc_flow(H: int = 32, R_i: float = 9.5, Nr: int = 111, U2: float = 3.93e-4) -> DiscFlow:
    """The paper's case by default: 32 x 120 from the axis, R_i = 9.5, R = 119.5
    (111 rows from R_i to R), Q = 0.5, U_2 = 3.93e-4."""
    return DiscFlow(H, R_i, Nr, U2)


@dataclass
class Instance:
    """One lattice of a batch: grid, parameters and the drop that initialises it."""
    Nz: int
    Nr: int
    tau: float
    G: float
    R: float
    zc: float
    rho_l: float
    rho_v: float
    a2: float
    seed: int
    fields: tuple = field(default=None, repr=False)

    def make_fields(self):
        if self.fields is None:
            self.fields = drop(self.Nz, self.Nr, self.zc, self.R, self.rho_l, self.rho_v,
                               amps=(self.a2,) if self.a2 else ())
        return self.fields


def batch_sweep(n: int = 64, seed0: int = 1234, rmin: float = 10, rmax: float = 60):
    """The batched sweep: instance k uses numpy.random.default_rng(seed0 + k) to draw
    R ~ U[rmin, rmax] (grid 4R x 2R, R rounded to an integer), G ~ U[-5.5, -4.6],
    tau ~ U[0.6, 1.2] and an l = 2 amplitude ~ U[0, 0.08] for the oscillating half
    (even k: static drop, odd k: oscillating)."""
    out = []
    cache = {}
    for k in range(n):
        rng = np.random.default_rng(seed0 + k)
        R = int(round(rng.uniform(rmin, rmax)))
        G = float(rng.uniform(-5.5, -4.6))
        tau = float(rng.uniform(0.6, 1.2))
        a2 = float(rng.uniform(0.0, 0.08))
        if k % 2 == 0:
            a2 = 0.0
        key = round(G, 3)
        if key not in cache:
            cache[key] = coexistence(G)
        rl, rv = cache[key]
        out.append(Instance(Nz=4 * R, Nr=2 * R, tau=tau, G=G, R=float(R), zc=2.0 * R,
                            rho_l=rl, rho_v=rv, a2=a2, seed=seed0 + k))
    return out


def legendre_amplitudes(n: int = 16, sigma: float = 0.02, seed: int = 2024):
    """Amplitudes of P_2 .. P_{n+1} for the differentiable drop, N(0, sigma^2)."""
    return np.random.default_rng(seed).normal(0.0, sigma, size=n)
