"""Seeded synthetic reservoir cases.

This module only *describes inputs*: grid, rock, fluid tables, wells, initial
state, time-step schedule and solver options.  It holds none of the
simulator's arithmetic (no transmissibility, no property evaluation, no
residual), so both the CPU oracle and the CUDA path consume exactly the same
arrays from here and share nothing else.

Heterogeneity follows the kind of geology the paper simulates (SPE10-like
log-normal permeability spanning several decades, Sec. 4.1; an SPE1-like
black-oil deck, Sec. 4.4) without reproducing any dataset:

* noise: splitmix64 counter stream -> Box-Muller standard normals;
* correlation: white noise convolved with a separable Gaussian kernel
  exp(-2 r^2 / l^2) truncated at 3 l, reflective edges, then standardised;
* ln k = 4.6 + sigma * z (mD), kx = ky, kz = 0.1 kx;
* porosity = 0.15 + 0.10 * Phi(z) (standard normal CDF), i.e. 0.15..0.25.

Array layout everywhere: float64, cell index i + nx*(j + ny*k) (x fastest).
"""
from __future__ import annotations

import math
import numpy as np

MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)
GOLDEN = np.uint64(0x9E3779B97F4A7C15)

PRODUCER = 0
WATER_INJECTOR = 1

MODEL_OIL_WATER = 2
MODEL_BLACK_OIL = 3


# ----------------------------------------------------------------------------
# random numbers: splitmix64 (Steele, Lea, Flood 2014) used as a counter-based
# generator, Box-Muller for normals.
# ----------------------------------------------------------------------------
def splitmix64(counter: np.ndarray, seed: int) -> np.ndarray:
    """Output k of the splitmix64 stream seeded with ``seed`` (k = counter)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(n: int, seed: int, offset: int = 0) -> np.ndarray:
    """n doubles in (0, 1) from 53 random bits each."""
    k = np.arange(offset, offset + n, dtype=np.uint64)
    z = splitmix64(k, seed) >> np.uint64(11)
    return (z.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def std_normal(n: int, seed: int) -> np.ndarray:
    """n standard normals by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u1 = uniform01(m, seed, 0)
    u2 = uniform01(m, seed, m)
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
    return z[:n]


def correlated_field(nx: int, ny: int, nz: int, corr_len: float, seed: int) -> np.ndarray:
    """Standardised Gaussian random field with covariance ~ exp(-r^2/l^2)."""
    from scipy.ndimage import convolve1d

    z = std_normal(nx * ny * nz, seed).reshape(nz, ny, nx)
    if corr_len > 0:
        half = int(math.ceil(3.0 * corr_len))
        t = np.arange(-half, half + 1, dtype=np.float64)
        w = np.exp(-2.0 * t * t / (corr_len * corr_len))
        w /= w.sum()
        for axis in (0, 1, 2):
            z = convolve1d(z, w, axis=axis, mode="reflect")
    z = z - z.mean()
    s = z.std()
    if s > 0:
        z = z / s
    return np.ascontiguousarray(z.reshape(-1))


def normal_cdf(z: np.ndarray) -> np.ndarray:
    from scipy.special import ndtr

    return ndtr(z)


def lognormal_rock(nx, ny, nz, sigma, corr_len, seed, lnk_mean=4.6, kz_ratio=0.1):
    z = correlated_field(nx, ny, nz, corr_len, seed)
    kx = np.exp(lnk_mean + sigma * z)
    poro = 0.15 + 0.10 * normal_cdf(z)
    return kx, kx.copy(), kz_ratio * kx, poro


# ----------------------------------------------------------------------------
# fluids
# ----------------------------------------------------------------------------
def oil_water_fluid(mu_o=2.0, mu_w=0.5, c=1e-5, swc=0.1, sor=0.1):
    return dict(
        rho_w_ref=1000.0, rho_o_ref=800.0, c_w=c, c_o=c, mu_w=mu_w, mu_o=mu_o,
        swc=swc, sor=sor, sgc=0.0, sorg=0.0, nw=2.0, now=2.0, ng=2.0, nog=2.0,
    )


def black_oil_fluid():
    """Tabulated PVT over 50..400 bar (8 nodes), bubble point 200 bar."""
    p = np.arange(50.0, 401.0, 50.0)
    return dict(
        rho_ws=1000.0, rho_os=800.0, rho_gs=0.9,
        mu_w=0.5, bw_c=4e-5, bw_pref=200.0,
        bo_c_us=1e-4, muo_c_us=5e-4,
        pvt_p=p,
        pvt_bo=1.0 + 0.0015 * p,
        pvt_rs=0.5 * p,
        pvt_muo=1.5 - 0.0025 * (p - 50.0),
        pvt_bg=1.2 / p,
        pvt_mug=0.012 + 5e-5 * p,
        swc=0.1, sor=0.1, sgc=0.05, sorg=0.1, nw=2.0, now=2.0, ng=2.0, nog=2.0,
    )


def default_solver(**kw):
    s = dict(
        newton_tol=1e-10, newton_max=20, lin_tol=1e-8, gmres_m=30, gmres_max_restarts=20,
        precond=2, stage2=1, amg_theta=0.25, amg_rounds=4, amg_coarse_max=256,
        amg_max_levels=16, chop_ds=0.2, chop_dp=50.0, max_cuts=8, amg_cycles=1,
        decouple=0, cpr_stages=2, krylov=0, lin_max_iter=100, forcing=0, ew_gamma=0.9, ew_beta=2.0,
        theta_max=0.5, orth=0,
    )
    s.update(kw)
    return s


def paper_solver(**kw):
    """The settings of the paper's experiments (Sec. 4): BiCGSTAB with at most
    100 iterations, inexact Newton with an adaptive forcing term (Eq. 14,
    choice 2), CNV tolerance 1e-3, at most 20 Newton iterations."""
    s = default_solver(krylov=1, lin_max_iter=100, forcing=2, newton_tol=1e-3)
    s.update(kw)
    return s


def well(i, j, k0, k1, wtype, bhp, rw=0.1, skin=0.0, ctrl=0, rate=0.0):
    """A vertical well perforated in layers k0..k1.  ctrl 0: fixed BHP `bhp`;
    ctrl 1 / 2: fixed water / oil component mass rate `rate` (kg/day, positive
    into the reservoir), `bhp` then being the initial guess of its BHP."""
    return dict(i=int(i), j=int(j), k0=int(k0), k1=int(k1), type=int(wtype),
                bhp=float(bhp), rw=float(rw), skin=float(skin), ctrl=int(ctrl), rate=float(rate))


def _hydrostatic(nx, ny, nz, dz, top_depth, p_top, rho):
    """Initial pressure from a fixed reference density (an input, not an equilibrium)."""
    k = np.arange(nz, dtype=np.float64)
    depth = top_depth + (k + 0.5) * dz
    p = p_top + rho * 9.80665 * (depth - top_depth) / 1e5
    return np.repeat(p, nx * ny)


# ----------------------------------------------------------------------------
# cases
# ----------------------------------------------------------------------------
def oil_water_case(nx=20, ny=20, nz=5, dx=10.0, dy=10.0, dz=2.0, k=100.0, poro=0.2,
                   sigma=0.0, corr_len=10.0, seed=1000, nsteps=10, dt=1.0,
                   inj_bhp=300.0, prod_bhp=100.0, wells=None, fluid=None, gravity_top=2000.0,
                   p_top=200.0, **solver):
    """Two-phase oil-water quarter five-spot (homogeneous unless sigma > 0)."""
    N = nx * ny * nz
    if sigma > 0:
        kx, ky, kz, ph = lognormal_rock(nx, ny, nz, sigma, corr_len, seed)
    else:
        kx = np.full(N, float(k)); ky = kx.copy(); kz = kx.copy(); ph = np.full(N, float(poro))
    fl = fluid or oil_water_fluid()
    if wells is None:
        wells = [well(0, 0, 0, nz - 1, WATER_INJECTOR, inj_bhp),
                 well(nx - 1, ny - 1, 0, nz - 1, PRODUCER, prod_bhp)]
    p0 = _hydrostatic(nx, ny, nz, dz, gravity_top, p_top, fl["rho_o_ref"])
    return dict(
        name=f"oil-water {nx}x{ny}x{nz}", model=MODEL_OIL_WATER,
        nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, top_depth=gravity_top,
        kx=kx, ky=ky, kz=kz, poro=ph, c_rock=0.0, p_ref=200.0,
        fluid=fl, wells=wells,
        init=dict(p=p0, sw=np.full(N, fl["swc"]), x3=np.zeros(N), phase=np.ones(N, np.int8)),
        dt=[float(dt)] * nsteps, cnv_rho=[fl["rho_w_ref"], fl["rho_o_ref"], 1.0],
        solver=default_solver(**solver),
    )


def five_spot_wells(nx, ny, nz, inj_bhp=240.0, prod_bhp=180.0):
    return [well(nx // 2, ny // 2, 0, nz - 1, WATER_INJECTOR, inj_bhp),
            well(0, 0, 0, nz - 1, PRODUCER, prod_bhp),
            well(nx - 1, 0, 0, nz - 1, PRODUCER, prod_bhp),
            well(0, ny - 1, 0, nz - 1, PRODUCER, prod_bhp),
            well(nx - 1, ny - 1, 0, nz - 1, PRODUCER, prod_bhp)]


def pattern25_wells(nx, ny, nz, inj_bhp=240.0, prod_bhp=180.0):
    """25 vertical wells on a 5x5 pattern, checkerboard injector/producer."""
    ws = []
    for a in range(5):
        for b in range(5):
            i = min(nx - 1, int(round((a + 0.5) * nx / 5.0)))
            j = min(ny - 1, int(round((b + 0.5) * ny / 5.0)))
            t = WATER_INJECTOR if (a + b) % 2 == 0 else PRODUCER
            ws.append(well(i, j, 0, nz - 1, t, inj_bhp if t == WATER_INJECTOR else prod_bhp))
    return ws


def black_oil_case(nx=100, ny=100, nz=20, dx=10.0, dy=10.0, dz=2.0, sigma=1.0, corr_len=10.0,
                   seed=1001, nsteps=30, dt=10.0, wells="five_spot", top_depth=2000.0,
                   p_top=250.0, pb_init=200.0, **solver):
    """Three-phase black oil on log-normal rock, initially undersaturated."""
    N = nx * ny * nz
    kx, ky, kz, poro = lognormal_rock(nx, ny, nz, sigma, corr_len, seed)
    fl = black_oil_fluid()
    if wells == "five_spot":
        wl = five_spot_wells(nx, ny, nz)
    elif wells == "pattern25":
        wl = pattern25_wells(nx, ny, nz)
    else:
        wl = wells
    p0 = _hydrostatic(nx, ny, nz, dz, top_depth, p_top, 700.0)
    return dict(
        name=f"black-oil {nx}x{ny}x{nz}", model=MODEL_BLACK_OIL,
        nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, top_depth=top_depth,
        kx=kx, ky=ky, kz=kz, poro=poro, c_rock=5e-5, p_ref=200.0,
        fluid=fl, wells=wl,
        init=dict(p=p0, sw=np.full(N, fl["swc"]), x3=np.full(N, pb_init),
                  phase=np.zeros(N, np.int8)),
        dt=[float(dt)] * nsteps, cnv_rho=[1000.0, 800.0, 150.0],
        solver=default_solver(**solver),
    )


# the workloads, by what they are
def quarter_five_spot_20x20x5(**kw):
    """Oil-water 20x20x5, homogeneous 100 mD, 10 steps of 1 day."""
    return oil_water_case(**kw)


def black_oil_100x100x20(**kw):
    """Black oil 100x100x20 (200k cells), sigma 1, l = 10 cells, 30 steps of 10 days."""
    a = dict(nx=100, ny=100, nz=20, sigma=1.0, corr_len=10.0, seed=1001, nsteps=30, dt=10.0)
    a.update(kw)
    return black_oil_case(**a)


def black_oil_400cube(n=400, **kw):
    """Black oil n^3 (64M cells at n = 400), l = 20 cells, 25 wells, 5 steps of
    1 day (13 injectors feeding 2 m thick cells over a 2n m column: 10-day steps
    make Newton fail and halve the step repeatedly).  Two V-cycles per CPR
    pressure stage: on this field one cycle leaves a restarted FGMRES(30) solve
    of the first step stalled, two converge every solve in fewer iterations."""
    a = dict(nx=n, ny=n, nz=n, sigma=1.0, corr_len=20.0, seed=1002, nsteps=5, dt=1.0,
             wells="pattern25", amg_cycles=2)
    a.update(kw)
    return black_oil_case(**a)


def black_oil_128x128x32(**kw):
    """Black oil 128x128x32 (524k cells), sigma 1, l = 10 cells: the grid the
    learned pressure stage is trained on."""
    a = dict(nx=128, ny=128, nz=32, sigma=1.0, corr_len=10.0, seed=1004)
    a.update(kw)
    return black_oil_case(**a)


def black_oil_256x256x64_sigma2(**kw):
    """Black oil 256x256x64 (4.2M cells) with a heavier-tailed field (sigma 2,
    l = 20 cells): the grid the learned pressure stage is evaluated on."""
    a = dict(nx=256, ny=256, nz=64, sigma=2.0, corr_len=20.0, seed=1005)
    a.update(kw)
    return black_oil_case(**a)


def ensemble_members(n_members=64, seed=1003, nsteps=20, dt=1.0, scale=1.0):
    """Uneven oil-water realisations: nx, ny ~ U{32..128}, nz ~ U{8..32}, sigma ~ U[0.5, 2]."""
    u = uniform01(4 * n_members, seed)
    out = []
    for m in range(n_members):
        nx = 32 + int(u[4 * m] * 97)
        ny = 32 + int(u[4 * m + 1] * 97)
        nz = 8 + int(u[4 * m + 2] * 25)
        sig = 0.5 + 1.5 * u[4 * m + 3]
        if scale != 1.0:
            nx = max(4, int(nx * scale)); ny = max(4, int(ny * scale)); nz = max(2, int(nz * scale))
        out.append(oil_water_case(nx=nx, ny=ny, nz=nz, sigma=sig, corr_len=10.0,
                                  seed=seed + 1 + m, nsteps=nsteps, dt=dt))
    return out


def n_cells(case) -> int:
    return case["nx"] * case["ny"] * case["nz"]
