"""Seeded synthetic workloads for the rational time stepper.

This module holds only workload definitions and seeded input generators:
grid sizes, PDE coefficients sampled at caller-given coordinates, and initial
conditions.  It contains none of the method's arithmetic (no rational fit, no
discretisation, no solve), so both the FP64 CPU oracle and the GPU path can use
it without sharing any computation.

The workloads follow the paper's two PDE families (rotating shallow water,
Section 4.1; variable-coefficient wave equation, Section 4.2), with the sizes,
coefficients and initial-condition recipes of the five benchmark
configurations.  Every random draw comes from ``numpy.random.default_rng`` with
a fixed seed (config index * 1000 + instance).
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

# ln(1/delta) based spectral cut-off of a Gaussian exp(-r^2 / (2 s^2)):
# its Fourier transform exp(-k^2 s^2 / 2) drops below delta at
# k = sqrt(2 ln(1/delta)) / s.


def gaussian_kmax(sigma: float, delta: float) -> float:
    """Wavenumber above which a Gaussian of std ``sigma`` has relative content < delta."""
    return math.sqrt(2.0 * math.log(1.0 / delta)) / sigma


@dataclass(frozen=True)
class Workload:
    name: str
    kind: str                 # "wave" (Dirichlet) or "sw" (no-normal-flow walls)
    nlx: int
    nly: int
    p: int
    delta: float
    n_poles: int = 0          # 2M+1 fixed by the workload (0: chosen from the band)
    tau: float = 0.0          # fixed step (0: chosen from the pole count and band)
    steps: int = 1
    n_rhs: int = 1
    seed: int = 0
    params: dict = field(default_factory=dict)

    @property
    def q(self) -> int:
        return self.p - 2


# Configuration 0: variable-coefficient wave equation, Dirichlet walls,
# 4x4 leaves, p = 12, 21 poles, Gaussian bump (sigma 0.05) at (0.4, 0.6).
WAVE_4X4_P12 = Workload(
    name="wave_dirichlet_4x4_p12_N21", kind="wave", nlx=4, nly=4, p=12,
    delta=1e-10, n_poles=21, steps=10, seed=0,
    params=dict(c_kind="sincos", ic="bump", bump_sigma=0.05, bump_centre=(0.4, 0.6),
                c_max=1.25),
)

# Configuration 1: linearised rotating shallow water, walls, gH = 1, f = 10,
# 16x16 leaves, p = 16, tau = 20 inertial periods, 3 seeded Gaussians.
SW_16X16_P16 = Workload(
    name="sw_walls_16x16_p16_tau20T", kind="sw", nlx=16, nly=16, p=16,
    delta=1e-10, tau=20.0 * 2.0 * math.pi / 10.0, steps=100, seed=1000,
    params=dict(f=10.0, g=1.0, H=1.0, n_gauss=3, sigma_range=(0.03, 0.08),
                amp_range=(0.1, 1.0), centre_range=(0.2, 0.8)),
)

# Configuration 2: wave equation with c = clip(exp(GRF), 0.5, 2), 32x32 leaves,
# p = 16, 61 poles, 256 initial conditions of 5 Gaussians each, 50 steps.
WAVE_32X32_P16 = Workload(
    name="wave_dirichlet_32x32_p16_N61", kind="wave", nlx=32, nly=32, p=16,
    delta=1e-10, n_poles=61, steps=50, n_rhs=256, seed=2000,
    params=dict(c_kind="grf", grf_corr=0.1, grf_std=0.3, c_clip=(0.5, 2.0), c_max=2.0,
                ic="gauss5", n_gauss=5, sigma_range=(0.03, 0.08),
                amp_range=(0.1, 1.0), centre_range=(0.2, 0.8)),
)

# Configuration 1 on a periodic square (the setting of the paper's shallow-water
# examples, Section 4.1): the same sizes, f, g, H, tau and Gaussian draws, summed over
# their periodic images so that the data are smooth across the seams; the consistent
# elimination of the velocities (its discrete step is stable on a periodic square).
SW_PERIODIC_16X16_P16 = dataclasses.replace(
    SW_16X16_P16, name="sw_periodic_16x16_p16_tau20T",
    params=dict(SW_16X16_P16.params, periodic=True, consistent=True),
)

# Configuration 4: the adjoint of configuration 1's problem on 32x32 leaves, p = 16,
# 61 poles (the step tau = X(61) / band follows from the pole count): a misfit of h at
# 512 seeded sensor nodes after each of 50 steps, data from a second seeded draw,
# checkpoints every 10 steps, 20 seeded central-difference directions.
SW_ADJOINT_32X32_P16 = dataclasses.replace(
    SW_16X16_P16, name="sw_walls_adjoint_32x32_p16_N61", nlx=32, nly=32, n_poles=61, tau=0.0, steps=50,
    seed=4000, params=dict(SW_16X16_P16.params, n_sensors=512, checkpoint_every=10, fd_directions=20),
)

WORKLOADS = {w.name: w for w in (WAVE_4X4_P12, SW_16X16_P16, WAVE_32X32_P16, SW_PERIODIC_16X16_P16)}

# Uneven batch (after configuration 3, scaled to fit the batch's operators in a
# few tens of GB): independent instances, alternately wave (variable c, per-box
# operators, 8x8 leaves) and shallow water (walls, shared operators, 8x8 or 16x16
# leaves), p in {8, 12, 16}, 2M+1 in [41, 201] (wave <= 101), 1-8 right-hand sides.
UNEVEN_BATCH = "uneven_batch_16"


def uneven_instances(n: int = 16, seed: int = 3000) -> list:
    """Seeded instance list of the uneven batch: Workload objects with sizes,
    pole counts and right-hand-side counts drawn per instance."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        p = int(rng.choice([8, 12, 16]))
        rhs = int(rng.integers(1, 9))
        if i % 2 == 0:
            npol = int(rng.integers(20, 51)) * 2 + 1
            out.append(dataclasses.replace(WAVE_32X32_P16, name=f"wave_8x8_p{p}_N{npol}_r{rhs}", nlx=8, nly=8, p=p,
                                           n_poles=npol, n_rhs=rhs, seed=seed + i))
        else:
            nl = int(rng.choice([8, 16]))
            npol = int(rng.integers(20, 101)) * 2 + 1
            out.append(dataclasses.replace(SW_16X16_P16, name=f"sw_{nl}x{nl}_p{p}_N{npol}_r{rhs}", nlx=nl, nly=nl,
                                           p=p, n_poles=npol, tau=0.0, n_rhs=rhs, seed=seed + i))
    return out

# Configuration 3 at its stated size: 64 seeded instances, alternately wave (variable c,
# per-box operators) and shallow water (walls, shared operators), leaves 8^2 .. 64^2,
# p in {8, 12, 16}, 2M+1 in [41, 201], 1-64 right-hand sides, admitted in draw order
# while their operators fit a 150 GB budget (an instance over the rest is rejected
# by the library with EO_ERR_BUDGET).
UNEVEN_BATCH_64 = "uneven_batch_64"
UNEVEN_64_BUDGET_GB = 150.0


def uneven_instances_64(n: int = 64, seed: int = 3000) -> list:
    """Seeded instance list of configuration 3 (see UNEVEN_BATCH_64)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nl = int(rng.choice([8, 16, 32, 64]))
        p = int(rng.choice([8, 12, 16]))
        npol = int(rng.integers(20, 101)) * 2 + 1
        rhs = int(rng.integers(1, 65))
        base = WAVE_32X32_P16 if i % 2 == 0 else SW_16X16_P16
        kind = "wave" if i % 2 == 0 else "sw"
        out.append(dataclasses.replace(base, name=f"{kind}_{nl}x{nl}_p{p}_N{npol}_r{rhs}", nlx=nl, nly=nl, p=p,
                                       n_poles=npol, tau=0.0, n_rhs=rhs, seed=seed + i))
    return out


# Band Lambda (largest resolved |eigenvalue|) per workload.  4x4/p12 wave: the
# content of the Gaussian bump above |lambda| = 320 of the discrete operator is
# below 1e-10 (dense eigendecomposition of that 4000-unknown operator); the
# others follow from the narrowest Gaussian the recipe can draw (sw_band,
# wave_band below).
BAND = {}


def _init_bands():
    BAND[WAVE_4X4_P12.name] = 320.0
    BAND[SW_16X16_P16.name] = sw_band(SW_16X16_P16)
    BAND[WAVE_32X32_P16.name] = wave_band(WAVE_32X32_P16)
    BAND[SW_PERIODIC_16X16_P16.name] = sw_band(SW_PERIODIC_16X16_P16)
    BAND[SW_ADJOINT_32X32_P16.name] = sw_band(SW_ADJOINT_32X32_P16)


def sw_band(w: Workload) -> float:
    """Band Lambda for the shallow-water workload: sqrt(f^2 + gH k_max^2),
    k_max from the narrowest Gaussian the recipe can draw."""
    pr = w.params
    k = gaussian_kmax(pr["sigma_range"][0], w.delta)
    return math.sqrt(pr["f"] ** 2 + pr["g"] * pr["H"] * k * k)


def wave_band(w: Workload) -> float:
    """Band Lambda for the wave workloads: c_max * k_max of the initial data."""
    pr = w.params
    s = pr.get("bump_sigma", pr.get("sigma_range", (0.05,))[0])
    return pr["c_max"] * gaussian_kmax(s, w.delta)


_init_bands()


# ---------------------------------------------------------------- coefficients

def wave_c_sincos(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """c(x, y) = 1 + 0.25 sin(2 pi x) cos(2 pi y)."""
    return 1.0 + 0.25 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)


def grf(x: np.ndarray, y: np.ndarray, seed: int, corr: float, std: float,
        period: float = 2.0) -> np.ndarray:
    """Smooth Gaussian random field with covariance std^2 exp(-r^2 / (2 corr^2)).

    Spectral synthesis on a periodic box of side ``period`` (larger than the
    unit square so no periodicity is imposed on [0,1]^2): random Fourier modes
    k = 2 pi n / period, |k| <= 7 / corr, amplitude sqrt(S(k) dk^2) with the
    Gaussian spectral density S(k) = std^2 corr^2 / (2 pi) exp(-k^2 corr^2 / 2).
    """
    rng = np.random.default_rng(seed)
    dk = 2 * np.pi / period
    nmax = int(math.ceil(7.0 / corr / dk))
    n = np.arange(-nmax, nmax + 1)
    kx, ky = np.meshgrid(n * dk, n * dk, indexing="ij")
    kx = kx.ravel(); ky = ky.ravel()
    kk = kx * kx + ky * ky
    sel = kk <= (7.0 / corr) ** 2
    kx, ky, kk = kx[sel], ky[sel], kk[sel]
    dens = std * std * corr * corr / (2 * np.pi) * np.exp(-0.5 * kk * corr * corr)
    amp = np.sqrt(dens * dk * dk)
    a = rng.standard_normal(kx.size) * amp
    b = rng.standard_normal(kx.size) * amp
    # sum_k a_k cos(k.x) + b_k sin(k.x) = Re sum_{n,m} (a - i b)_{nm} e^{i n dk x} e^{i m dk y}:
    # evaluated separably on the (n, m) lattice of the selected modes
    N = 2 * nmax + 1
    coef = np.zeros((N, N), dtype=np.complex128)
    ni = np.rint(kx / dk).astype(int) + nmax
    mi = np.rint(ky / dk).astype(int) + nmax
    coef[ni, mi] = a - 1j * b
    xf = np.asarray(x, dtype=np.float64).ravel()
    yf = np.asarray(y, dtype=np.float64).ravel()
    out = np.zeros(xf.size)
    for i in range(0, xf.size, 65536):
        ex = np.exp(1j * np.outer(xf[i:i + 65536], n * dk))
        ey = np.exp(1j * np.outer(yf[i:i + 65536], n * dk))
        out[i:i + 65536] = (ex * (ey @ coef.T)).sum(axis=1).real
    return out.reshape(np.shape(x))


def wave_c(w: Workload, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Wave speed c at the given coordinates for workload ``w``."""
    pr = w.params
    if pr["c_kind"] == "sincos":
        return wave_c_sincos(x, y)
    if pr["c_kind"] == "grf":
        g = grf(x, y, w.seed + 999, pr["grf_corr"], pr["grf_std"])
        lo, hi = pr["c_clip"]
        return np.clip(np.exp(g), lo, hi)
    if pr["c_kind"] == "const":
        return np.ones_like(np.asarray(x, dtype=np.float64))
    raise ValueError(pr["c_kind"])


# ---------------------------------------------------------- initial conditions

def draw_gaussians(seed: int, n: int, sigma_range, amp_range, centre_range):
    """Seeded parameters of ``n`` Gaussians: (centres [n,2], sigmas [n], amps [n])."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(centre_range[0], centre_range[1], size=(n, 2))
    s = rng.uniform(sigma_range[0], sigma_range[1], size=n)
    a = rng.uniform(amp_range[0], amp_range[1], size=n)
    return c, s, a


def gaussian_sum(x, y, centres, sigmas, amps, periodic: bool = False) -> np.ndarray:
    """Sum_j a_j exp(-|x - c_j|^2 / (2 s_j^2)); periodic=True sums each Gaussian over
    its images shifted by -1, 0, 1 in x and y (period 1), smooth across the seams of
    the periodic unit square."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out = np.zeros(np.broadcast(x, y).shape)
    shifts = (-1.0, 0.0, 1.0) if periodic else (0.0,)
    for (cx, cy), s, a in zip(centres, sigmas, amps):
        for sx in shifts:
            for sy in shifts:
                out += a * np.exp(-((x - cx - sx) ** 2 + (y - cy - sy) ** 2) / (2 * s * s))
    return out


def initial_fields(w: Workload, x: np.ndarray, y: np.ndarray, rhs: int = 0) -> list:
    """Initial fields at the given coordinates, as a list of arrays.

    wave: [u, v] with v = 0.  sw: [u, v, h] with u = v = 0.
    """
    pr = w.params
    if w.kind == "wave":
        if pr.get("ic") == "bump":
            cx, cy = pr["bump_centre"]
            u = gaussian_sum(x, y, [(cx, cy)], [pr["bump_sigma"]], [1.0])
        else:
            c, s, a = draw_gaussians(w.seed + rhs, pr["n_gauss"], pr["sigma_range"],
                                     pr["amp_range"], pr["centre_range"])
            u = gaussian_sum(x, y, c, s, a)
        return [u, np.zeros_like(u)]
    c, s, a = draw_gaussians(w.seed + rhs, pr["n_gauss"], pr["sigma_range"],
                             pr["amp_range"], pr["centre_range"])
    h = gaussian_sum(x, y, c, s, a, periodic=bool(pr.get("periodic", False)))
    return [np.zeros_like(h), np.zeros_like(h), h]
