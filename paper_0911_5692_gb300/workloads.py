"""Workload presets and seeded synthetic inputs.

This module holds parameter sets and seeded random-number generation only; it
contains none of the method's arithmetic. Both the CUDA path and the CPU oracle
take their inputs from here, so that they see identical states.

The presets follow the chaotic-inflation runs of Sainio (arXiv:0911.5692,
Sec. III) and the lambda phi^4 lineage it compares against:

* ``lphi4_32_fp64``   lambda phi^4/4 + g^2 phi^2 chi^2 / 2, lambda = 9e-14,
  g^2/lambda = 200, N = 32, L = 10, dt = dx/20, FP64, phi0 = 0.342 in
  non-reduced Planck units (8 pi G = 8 pi).
* ``m2phi2_256_fp32`` m^2 phi^2/2 + g^2 phi^2 chi^2/2, m = 1e-6, g^2 = 2.5e-7,
  N = 256, L = 10, dt = 2^-10, phi0 = 1.009343, phidot0 = -0.7137 m, reduced
  Planck units (8 pi G = 1), FP32 fields.
* ``lphi4_512_fp32``  the lambda phi^4 model at N = 512, FP32.
* ``ensemble_64``     64 lambda phi^4 lattices, N cycling over 32, 48, 64, 96,
  g^2/lambda log-uniform in [50, 500].
* ``lphi4_128_fp32``  the lambda phi^4 model at N = 128, FP32 (adjoint runs).

``split=1`` stores the inflaton as an FP64 homogeneous mode plus FP32
fluctuation arrays (lat_params.split); the FP32 evolution presets use it.
"""
from __future__ import annotations

import math

import numpy as np

LAMBDA = 9e-14


def lphi4(n: int, precision: int = 32, G: float = 200.0, seed: int = 0, expansion: int = 1,
          L: float = 10.0, dt_over_dx: float = 1.0 / 20.0, fluct: float = 1.0, split: int = 0) -> dict:
    dx = L / n
    return dict(n=n, precision=precision, model=0, expansion=expansion, L=L, dt=dx * dt_over_dx,
                lam=LAMBDA, m=0.0, g2=G * LAMBDA, phi0=(0.342, 0.0), dphi0=(0.0, 0.0),
                eight_pi_G=8.0 * math.pi, kcut=0.0, fluct=fluct, seed=seed, split=split)


def m2phi2(n: int, precision: int = 32, seed: int = 0, expansion: int = 1, L: float = 10.0,
           dt: float = 2.0 ** -10, fluct: float = 1.0, g2: float = 2.5e-7, m: float = 1e-6, split: int = 0) -> dict:
    return dict(n=n, precision=precision, model=1, expansion=expansion, L=L, dt=dt,
                lam=0.0, m=m, g2=g2, phi0=(1.009343, 0.0), dphi0=(-0.7137 * m, 0.0),
                eight_pi_G=1.0, kcut=0.0, fluct=fluct, seed=seed, split=split)


# FP32 evolution workloads store phi split (an FP64 homogeneous mode plus FP32
# fluctuation arrays); the derivative workload stores it whole (lat_adjoint
# does not take split lattices).
WORKLOADS = {
    "lphi4_32_fp64": dict(params=lphi4(32, precision=64), steps=1000),
    "m2phi2_256_fp32": dict(params=m2phi2(256, precision=32, split=1), steps=5000),
    "lphi4_512_fp32": dict(params=lphi4(512, precision=32, split=1), steps=2000),
    "lphi4_128_fp32": dict(params=lphi4(128, precision=32), steps=2000),
}


def ensemble_64(seed: int = 0, precision: int = 32, split: int = 0) -> list[dict]:
    """64 lattices: N cycles 32, 48, 64, 96; g^2/lambda = exp(U(ln 50, ln 500)) drawn
    from numpy's PCG64 seeded with ``seed``; lattice i uses init seed i; dt = dx_i/20."""
    rng = np.random.default_rng(seed)
    Gs = np.exp(rng.uniform(math.log(50.0), math.log(500.0), size=64))
    sizes = (32, 48, 64, 96)
    return [lphi4(sizes[i % 4], precision=precision, G=float(Gs[i]), seed=i, split=split) for i in range(64)]


def random_state(n: int, seed: int, precision: int = 32, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3),
                 pi_mean=(0.5, 0.0), pi_amp=(1e-3, 1e-3)):
    """Seeded synthetic lattice state (f0, f1, pi0, pi1), each float64 [z][y][x] whose
    values are exactly representable in the given precision (32 or 64). Shaped like
    the paper's runs: the inflaton near its homogeneous value in program units (1),
    the second field a small fluctuation around zero."""
    rng = np.random.default_rng(seed)
    out = []
    for mean, amp in zip(f_mean + pi_mean, f_amp + pi_amp):
        a = mean + amp * rng.standard_normal((n, n, n))
        if precision == 32:
            a = a.astype(np.float32).astype(np.float64)
        out.append(np.ascontiguousarray(a))
    return tuple(out)
