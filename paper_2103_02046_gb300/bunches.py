"""Seeded synthetic particle bunches.

This module only draws random numbers. It holds none of the P3M arithmetic, so the CUDA
path, the FP64 oracle, the tests and the benchmark can all take their inputs from it.

All lengths are in metres and all momenta in kg m/s. Every generator draws from
``numpy.random.default_rng(seed)`` in float64 and returns C-contiguous ``[N, 3]`` arrays.

The shapes follow the beam workloads of the P3M space-charge problem (macro-particles with
position and momentum, eq. (macroparticles) of Sec. 2.4.1):
  * a 3D Gaussian bunch, per-axis sigma;
  * a uniformly filled sphere (Coulomb-explosion test case);
  * a Gaussian core plus a uniform halo shell;
  * "cold" (zero) or thermal (Gaussian) momenta.
"""
from __future__ import annotations

import numpy as np

# CODATA 2018 values used to size the macro-particle mass in the momentum recipe.
ELECTRON_MASS = 9.1093837015e-31
ELEMENTARY_CHARGE = 1.602176634e-19
SPEED_OF_LIGHT = 299792458.0


def gaussian(n: int, sigma, seed: int) -> np.ndarray:
    """Positions ~ N(0, sigma_d) independently per axis."""
    rng = np.random.default_rng(seed)
    s = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (3,))
    return np.ascontiguousarray(rng.standard_normal((n, 3)) * s)


def _isotropic_dirs(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def uniform_sphere(n: int, radius: float, seed: int) -> np.ndarray:
    """Uniform density inside a sphere of the given radius, centred at the origin."""
    rng = np.random.default_rng(seed)
    d = _isotropic_dirs(rng, n)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    return np.ascontiguousarray(d * r[:, None])


def shell(n: int, r1: float, r2: float, seed: int) -> np.ndarray:
    """Uniform density in the spherical shell r1 <= r <= r2."""
    rng = np.random.default_rng(seed)
    d = _isotropic_dirs(rng, n)
    r = (r1 ** 3 + rng.random(n) * (r2 ** 3 - r1 ** 3)) ** (1.0 / 3.0)
    return np.ascontiguousarray(d * r[:, None])


def core_halo(n: int, sigma: float, halo_frac: float, r1_sig: float, r2_sig: float,
              seed: int) -> np.ndarray:
    """Gaussian core (isotropic sigma) plus a uniform halo shell [r1_sig, r2_sig] * sigma."""
    n_halo = int(round(n * halo_frac))
    core = gaussian(n - n_halo, sigma, seed)
    halo = shell(n_halo, r1_sig * sigma, r2_sig * sigma, seed + 1000003)
    x = np.concatenate([core, halo], axis=0)
    perm = np.random.default_rng(seed + 7).permutation(n)
    return np.ascontiguousarray(x[perm])


def thermal_momenta(n: int, rms: float, seed: int) -> np.ndarray:
    """Momenta ~ N(0, rms) per axis."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((n, 3)) * rms)


def lift_to_plane(x: np.ndarray, z_plane: float, gap: float) -> np.ndarray:
    """Translate along z so that the lowest particle sits `gap` above the plane z = z_plane."""
    y = np.array(x, dtype=np.float64, copy=True)
    y[:, 2] += (z_plane + gap) - y[:, 2].min()
    return y


def subsample(n_total: int, k: int, seed: int = 12345) -> np.ndarray:
    """Sorted indices of k distinct particles drawn from n_total."""
    idx = np.random.default_rng(seed).choice(n_total, size=k, replace=False)
    return np.sort(idx).astype(np.int64)


def macro_charge() -> float:
    """Macro-particle charge used by every workload here [C]."""
    return 1e-15


def macro_mass(q: float | None = None) -> float:
    """Mass of a macro-particle that carries q/e electrons [kg]."""
    q = macro_charge() if q is None else q
    return abs(q) / ELEMENTARY_CHARGE * ELECTRON_MASS


# The five workloads: inputs only (sizes, distributions, seeds).
WORKLOADS = {
    "gauss4k": dict(n=4096, kind="gaussian", sigma=(1e-3, 1e-3, 1e-3), seed=0, mesh=16,
                    rc_over_h=2.0, momenta="cold"),
    "gauss1m": dict(n=1_048_576, kind="gaussian", sigma=(1e-3, 1e-3, 3e-3), seed=2, mesh=64,
                    rc_over_h=2.0, momenta="thermal"),
    "sphere16m": dict(n=16_777_216, kind="sphere", radius=1e-3, seed=3, mesh=256,
                      rc_over_h=2.0, momenta="cold"),
    "gauss1m_grad": dict(n=1_048_576, kind="gaussian", sigma=(1e-3, 1e-3, 3e-3), seed=4,
                         mesh=64, rc_over_h=2.0, momenta="thermal"),
    "halo4m": dict(n=4_194_304, kind="core_halo", sigma=1e-3, halo_frac=0.05, r1=4.0, r2=6.0,
                   seed=5, mesh=128, rc_over_h=3.0, momenta="cold"),
}


def positions(spec: dict, n: int | None = None) -> np.ndarray:
    """Positions for a workload spec (optionally with a different particle count)."""
    n = spec["n"] if n is None else n
    kind = spec["kind"]
    if kind == "gaussian":
        return gaussian(n, spec["sigma"], spec["seed"])
    if kind == "sphere":
        return uniform_sphere(n, spec["radius"], spec["seed"])
    if kind == "core_halo":
        return core_halo(n, spec["sigma"], spec["halo_frac"], spec["r1"], spec["r2"], spec["seed"])
    raise ValueError(kind)


def momenta(spec: dict, n: int | None = None) -> np.ndarray:
    n = spec["n"] if n is None else n
    if spec["momenta"] == "cold":
        return np.zeros((n, 3))
    rms = 1e-4 * macro_mass() * SPEED_OF_LIGHT
    return thermal_momenta(n, rms, spec["seed"] + 100)
