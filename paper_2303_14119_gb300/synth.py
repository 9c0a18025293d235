"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds no arithmetic of the method: it draws counter-based uniform
numbers and describes the workloads (grid sizes, velocity spans, fields, SEE
parameters, injection) as plain data.  Both sides of every parity test get
their initial distribution f0 from here and nowhere else.

Uniform numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  Output n of the generator
started in state ``seed`` is ``mix(seed + (n + 1) * GAMMA)``; its top 53 bits
scaled by 2**-53 give u in [0, 1).  The cell with linear index
``(k * nv1 + i) * nv2 + j`` takes output number equal to that index.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

QE = 1.602176634e-19  # elementary charge (C), CODATA 2018
ME = 9.1093837015e-31  # electron mass (kg), CODATA 2018


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """Outputs number ``index`` (uint64 array) of SplitMix64 seeded with ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (index.astype(np.uint64) + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, offset: int = 0, chunk: int = 1 << 24) -> np.ndarray:
    """u[m] in [0, 1) for m = offset .. offset + n - 1 (FP64)."""
    out = np.empty(n, dtype=np.float64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = np.arange(offset + s, offset + e, dtype=np.uint64)
        out[s:e] = (splitmix64(seed, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return out


def beam_scale(J: float, T_fe_eV: float) -> float:
    """Phase-space density scale (s^2 m^-5) of an injected beam: flux J/e
    divided by the cube of the thermal speed sqrt(T e / m_e).  A unit used
    to state noise amplitudes; not part of the method."""
    vth = (T_fe_eV * QE / ME) ** 0.5
    return (J / QE) / vth ** 3


def initial_f(shape, seed: int = 0, noise_rel: float = 1e-6, J: float = 1.0,
              T_fe_eV: float = 4.0, dtype=np.float64) -> np.ndarray:
    """f0 = noise_rel * beam_scale(J, T_fe) * u(seed, cell): zero plus seeded
    uniform noise relative to the injected beam's density scale."""
    n = int(np.prod(shape))
    return (noise_rel * beam_scale(J, T_fe_eV) * uniform(seed, n)).reshape(shape).astype(dtype)


def random_f(shape, seed: int, amplitude: float) -> np.ndarray:
    """A positive random distribution amplitude * u, for parity tests."""
    n = int(np.prod(shape))
    return (amplitude * uniform(seed, n)).reshape(shape)


# Workloads.  Velocity spans are symmetric; x spans [0, h_max] normal to the
# insulator; E_y < 0 (cathode on the left); J is the constant injected current
# density (A/m^2) on the band [10, 15] um; dt from CFL 0.4 on the x-Courant.
BASE = dict(h_max=20e-6, v1_span=6e7, v2_span=3e7, cfl=0.4,
            delta_max=3.0, A_max=400.0, k_s=1.0, T_se=2.0,
            J=1.0, x_lo=10e-6, x_hi=15e-6, T_fe=4.0, noise_rel=1e-6, seed=0)

WORKLOADS = {
    # single FP64 instance, 64 x 48 x 48, 2000 steps
    "small_64x48x48": dict(BASE, nx=64, nv1=48, nv2=48, Ey=-1e6, steps=2000),
    # full scale 1024 x 256 x 256, E_y swept
    "full_1024x256x256": dict(BASE, nx=1024, nv1=256, nv2=256, Ey=-1e6,
                              Ey_sweep=(-5e5, -1e6, -3e6), steps=20000),
    # mixed precision 2048 x 384 x 384 and its 4x-coarsened copy
    "large_2048x384x384": dict(BASE, nx=2048, nv1=384, nv2=384, Ey=-2e6, steps=10000),
    "coarse_512x96x96": dict(BASE, nx=512, nv1=96, nv2=96, Ey=-2e6, steps=10000),
    # parameter sweep: 256 independent instances of uneven size, each run
    # 5000 steps, every size and parameter drawn from one seed (sweep_instances)
    "sweep_256": dict(BASE, sweep=256, steps=5000, seed=2023),
    # a run to saturation (the convergence test of Sec. 2, window 1e4 steps,
    # tolerance 1e-3) on a grid that resolves the secondaries' hop height:
    # an 8 um gap in 64 cells (dx = 0.125 um), v1 in +-4e6 m/s (24 cells),
    # v2 in +-3e7 m/s (32 cells), the source band [5, 7] um at 1e5 A/m^2,
    # f0 = 0 and sigma0 = 0 (Sec. 2: no electron in the domain at first);
    # two applied fields above the SEEA threshold of this geometry
    "saturation_64x24x32": dict(BASE, nx=64, nv1=24, nv2=32, h_max=8e-6, v1_span=4e6,
                                v2_span=3e7, J=1e5, x_lo=5e-6, x_hi=7e-6, noise_rel=0.0,
                                Ey=-6e6, Ey_sweep=(-4e6, -6e6), sat_window=10000,
                                sat_tol=1e-3, steps=120000),
    # the surrogate's training data: 1536 runs of 64 x 48 x 48 (surrogate_runs)
    # stepped as one batch; 750 000 steps reach a 1.25 ns horizon at the
    # smallest gap (h_max = 16 um: dt = 0.4 (h_max / 64) / 6e7 m/s)
    "surrogate_1536": dict(BASE, runs=1536, steps=750000, seed=11),
}

# Offset of the sweep's draws in the SplitMix64 stream (far from the cell
# indices the distributions use).
_SWEEP_OFFSET = 1 << 60


def sweep_instances(n: int = 256, seed: int = 2023):
    """n parameter-sweep instances drawn from one seed: nx uniform in
    {128..512}, nv1 = nv2 uniform in {64..192}, applied field log-uniform in
    [3e5, 5e6] V/m (E_y = -|E|), delta_max uniform in [2, 4], A_max uniform in
    [250, 600] eV, emission temperature T_se uniform in [1, 5] eV; the rest
    (spans, CFL, injection, noise) as BASE, noise seed seed + 1 + index."""
    u = uniform(seed, 6 * n, offset=_SWEEP_OFFSET).reshape(n, 6)
    out = []
    for q in range(n):
        e = float(np.exp(np.log(3e5) + u[q, 2] * (np.log(5e6) - np.log(3e5))))
        nv = 64 + int(u[q, 1] * 129)
        out.append(dict(BASE, nx=128 + int(u[q, 0] * 385), nv1=nv, nv2=nv, Ey=-e,
                        delta_max=2.0 + 2.0 * float(u[q, 3]),
                        A_max=250.0 + 350.0 * float(u[q, 4]),
                        T_se=1.0 + 4.0 * float(u[q, 5]), seed=seed + 1 + q))
    return out


def batch_instances(w):
    """The instance list of a batched workload entry: a parameter sweep
    (key 'sweep') or the surrogate's training runs (key 'runs')."""
    if "sweep" in w:
        return sweep_instances(w["sweep"], w["seed"])
    return surrogate_runs(w["runs"], w["seed"])


# Surrogate training runs: the sweep's parameter draws plus the two inputs
# the surrogate also takes, the injected current J (log-uniform; strong
# enough that the surface charge moves within the runs' horizon) and the
# gap h_max (uniform), on the coarse grid of the small workload.
SURROGATE_J = (1e5, 1e7)        # A/m^2
SURROGATE_H = (16e-6, 24e-6)    # m
_SURROGATE_OFFSET = 1 << 61


def surrogate_runs(n: int, seed: int):
    """n run descriptions drawn from one seed: E_y log-uniform in
    [3e5, 5e6] V/m, delta_max in [2, 4], A_max in [250, 600] eV, T_se in
    [1, 5] eV (as sweep_instances), J log-uniform in SURROGATE_J, h_max
    uniform in SURROGATE_H; grid 64 x 48 x 48."""
    u = uniform(seed, 6 * n, offset=_SURROGATE_OFFSET).reshape(n, 6)
    out = []
    for q in range(n):
        e = float(np.exp(np.log(3e5) + u[q, 0] * (np.log(5e6) - np.log(3e5))))
        J = float(np.exp(np.log(SURROGATE_J[0]) + u[q, 4] * (np.log(SURROGATE_J[1]) - np.log(SURROGATE_J[0]))))
        out.append(dict(BASE, nx=64, nv1=48, nv2=48, Ey=-e,
                        delta_max=2.0 + 2.0 * float(u[q, 1]),
                        A_max=250.0 + 350.0 * float(u[q, 2]),
                        T_se=1.0 + 4.0 * float(u[q, 3]), J=J,
                        h_max=SURROGATE_H[0] + (SURROGATE_H[1] - SURROGATE_H[0]) * float(u[q, 5])))
    return out
