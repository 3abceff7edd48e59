"""Seeded synthetic samples for the PLUGIN bandwidth selector.

This module is the one thing the GPU path and the CPU oracle share: it makes
input samples and nothing else.  It holds none of the method's arithmetic (no
moments, no kernel derivatives, no bandwidth formulas); it only turns a seed into
numbers with a stated distribution.

Random numbers come from SplitMix64 used as a counter-based generator: draw k of
stream s is ``mix(s + (k + 1) * GAMMA)`` with the published SplitMix64 finaliser
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators", 2014).
Uniforms are the top 53 bits, offset by half a step so they lie in the open
interval (0, 1).  Normals use the Box-Muller transform on consecutive uniform
pairs.  Student-t with 3 degrees of freedom is Z0 / sqrt((Z1^2 + Z2^2 + Z3^2)/3).

The paper's own experimental datasets (Section 4, Tables 2-4, n = 128 ... 1024)
are not published; the workloads below stand in for them with the sizes,
distributions and structure listed in the design notes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def derive_seed(seed: int, *keys: int) -> int:
    """Derive an independent stream seed from ``seed`` and integer keys:
    z <- mix((z xor key * 0xD1B54A32D192ED03) + GAMMA) for each key in turn."""
    z = seed & _MASK
    for k in keys:
        v = ((z ^ ((k * 0xD1B54A32D192ED03) & _MASK)) + int(GAMMA)) & _MASK
        z = int(_mix(np.array([v], dtype=np.uint64))[0])
    return z


def raw64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream ``seed``."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & _MASK) + k * GAMMA
    return _mix(state)


def uniform(seed: int, count: int) -> np.ndarray:
    """``count`` doubles, uniform on the open interval (0, 1)."""
    r = raw64(seed, count)
    return ((r >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int) -> np.ndarray:
    """``count`` standard normals by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * math.pi * u2
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(ang)
    z[1::2] = rad * np.sin(ang)
    return z[:count]


def student_t3(seed: int, count: int) -> np.ndarray:
    """Student-t with 3 degrees of freedom: Z0 / sqrt(mean of three squared normals)."""
    z = normal(seed, 4 * count).reshape(count, 4)
    return z[:, 0] / np.sqrt((z[:, 1] ** 2 + z[:, 2] ** 2 + z[:, 3] ** 2) / 3.0)


def lognormal(seed: int, count: int) -> np.ndarray:
    """exp(Z), Z standard normal."""
    return np.exp(normal(seed, count))


def normal_mixture(seed: int, count: int, weights, means, sds) -> np.ndarray:
    """Mixture of normals: component chosen by a uniform draw, then a normal draw."""
    w = np.asarray(weights, dtype=np.float64)
    cw = np.cumsum(w / w.sum())
    cw[-1] = 1.0
    comp = np.searchsorted(cw, uniform(derive_seed(seed, 1), count), side="right")
    comp = np.minimum(comp, len(w) - 1)
    z = normal(derive_seed(seed, 2), count)
    return np.asarray(means, dtype=np.float64)[comp] + np.asarray(sds, dtype=np.float64)[comp] * z


# ----------------------------------------------------------------------------
# Named workloads (sizes and structure of the paper's experiment, scaled up)
# ----------------------------------------------------------------------------

def single_normal(n: int = 1024, seed: int = 0) -> np.ndarray:
    """n iid N(0, 1) values: the small single-sample PLUGIN case."""
    return normal(seed, n)


def bimodal_offset(n: int = 65536, seed: int = 2, offset: float = 1.0e4) -> np.ndarray:
    """0.5 N(-1, 0.5^2) + 0.5 N(1, 0.5^2), shifted by +1e4 in FP64 (tests centring)."""
    return normal_mixture(seed, n, [0.5, 0.5], [-1.0, 1.0], [0.5, 0.5]) + offset


LARGE_FAMILIES = {"t3": 3, "lognormal": 4, "uniform": 5}


def large_sample(family: str, n: int = 1 << 20) -> np.ndarray:
    """n = 2^20 values from Student-t3 (seed 3), lognormal(0,1) (seed 4) or U[0,1] (seed 5)."""
    seed = LARGE_FAMILIES[family]
    if family == "t3":
        return student_t3(seed, n)
    if family == "lognormal":
        return lognormal(seed, n)
    if family == "uniform":
        return uniform(seed, n)
    raise ValueError(family)


@dataclass
class SampleSpec:
    index: int
    n: int
    family: str          # "normal" | "mixture" | "t3"
    params: dict
    seed: int


def _family_sample(spec: SampleSpec) -> np.ndarray:
    if spec.family == "normal":
        return spec.params["mu"] + spec.params["sigma"] * normal(spec.seed, spec.n)
    if spec.family == "mixture":
        p = spec.params
        return normal_mixture(spec.seed, spec.n, p["weights"], p["means"], p["sds"])
    if spec.family == "t3":
        return student_t3(spec.seed, spec.n)
    raise ValueError(spec.family)


def mixed_specs(count: int, seed: int, n_lo: int, n_hi: int) -> list[SampleSpec]:
    """Specs of ``count`` samples: n log-uniform in [n_lo, n_hi], family uniform among
    N(mu, sigma^2) (mu ~ U[-10, 10], sigma ~ logU[0.1, 10]), a k-component normal
    mixture (k ~ U{2..5}, weights = normalised Exp(1), mu_k ~ U[-5, 5],
    sigma_k ~ logU[0.2, 2]) and Student-t3."""
    specs = []
    for i in range(count):
        s = derive_seed(seed, i)
        u = uniform(derive_seed(s, 100), 32)
        n = int(math.floor(math.exp(math.log(n_lo) + u[0] * (math.log(n_hi) - math.log(n_lo)))))
        n = max(n_lo, min(n_hi, n))
        fam_idx = min(int(u[1] * 3), 2)
        family = ("normal", "mixture", "t3")[fam_idx]
        params: dict = {}
        if family == "normal":
            params = {"mu": -10.0 + 20.0 * u[2],
                      "sigma": math.exp(math.log(0.1) + u[3] * (math.log(10.0) - math.log(0.1)))}
        elif family == "mixture":
            k = 2 + min(int(u[4] * 4), 3)
            w = [-math.log(u[5 + c]) for c in range(k)]
            tot = sum(w)
            params = {
                "weights": [x / tot for x in w],
                "means": [-5.0 + 10.0 * u[10 + c] for c in range(k)],
                "sds": [math.exp(math.log(0.2) + u[15 + c] * (math.log(2.0) - math.log(0.2)))
                        for c in range(k)],
            }
        specs.append(SampleSpec(i, n, family, params, derive_seed(s, 200)))
    return specs


def sample_from_spec(spec: SampleSpec, dtype=np.float64) -> np.ndarray:
    return _family_sample(spec).astype(dtype)


def batch_specs(count: int = 512, seed: int = 6, n_lo: int = 256, n_hi: int = 262144):
    """The batched workload: 512 samples, n log-uniform in [256, 262144]."""
    return mixed_specs(count, seed, n_lo, n_hi)


def server_specs(count: int = 10000, seed: int = 7, n_lo: int = 1000, n_hi: int = 4194304):
    """The served workload: requests with n log-uniform in [1000, 4194304], FP32 samples."""
    return mixed_specs(count, seed, n_lo, n_hi)


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 7) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson stream with the given rate."""
    u = uniform(derive_seed(seed, 999), count)
    return np.cumsum(-np.log(u) / rate_per_s)
