"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  Random numbers only: nothing here computes any part of the method.

* random_state: normalised complex Gaussian state vectors (kernel tests)
* sweep_specs: the batched lambda sweep (256 runs; lambda ~ U[0, 6), lattice
  uniform over 3x3, 4x3 and 2x2x2, T ~ U[5, 20], M ~ U{100..400}, symmetric)
* poisson_stream: a serving request stream (Poisson arrivals, lattices from
  2x2 to 5x3 plus 2x2x2, lambda ~ U[0, 6], M ~ U{50..500}, T = 0.04 M)
"""

from __future__ import annotations

import numpy as np

SWEEP_SEED = 20191018
SWEEP_LATTICES = [(2, (3, 3)), (2, (4, 3)), (3, (2, 2, 2))]
SERVE_LATTICES = [(2, (2, 2)), (2, (3, 2)), (2, (4, 2)), (2, (5, 2)), (2, (3, 3)), (2, (4, 3)), (2, (5, 3)),
                  (3, (2, 2, 2))]


def random_state(n, seed, dtype=np.complex128):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    v /= np.linalg.norm(v)
    return v.astype(dtype)


def sweep_specs(count=256, seed=SWEEP_SEED, lattices=SWEEP_LATTICES):
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        d, L = lattices[int(rng.integers(len(lattices)))]
        specs.append(dict(d=d, L=L, lam=float(rng.uniform(0.0, 6.0)), T=float(rng.uniform(5.0, 20.0)),
                          M=int(rng.integers(100, 401)), decomp=1))
    return specs


def poisson_stream(count=2000, rate=200.0, seed=SWEEP_SEED + 1, lattices=SERVE_LATTICES, m_range=(50, 500)):
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate))
        d, L = lattices[int(rng.integers(len(lattices)))]
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        reqs.append(dict(arrival=t, d=d, L=L, lam=float(rng.uniform(0.0, 6.0)), M=M, T=0.04 * M, decomp=1))
    return reqs
