"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  This module only draws random numbers; it contains none of the
discretisation's arithmetic (no B-splines, no quadrature, no matrices).

The paper (arXiv:1802.09277, Sec. 4) measures on a 21-patch spatial domain
that is not available here; unit interval/square/cube workloads with the
same degrees and time-dofs per slab stand in for it.
"""
import numpy as np


def normal_coeffs(seed, n):
    """i.i.d. N(0,1) B-spline coefficients (float64), numpy default_rng."""
    return np.random.default_rng(seed).standard_normal(int(n))


def uniform_vector(seed, n, lo=-1.0, hi=1.0):
    """i.i.d. U(lo, hi) float64 vector (operator-parity test inputs)."""
    return np.random.default_rng(seed).uniform(lo, hi, int(n))


def uniform_vectors_on_device(seed, n, count, device, lo=-1.0, hi=1.0):
    """`count` i.i.d. U(lo, hi) float64 vectors of length n drawn on `device`
    by one seeded torch generator, for sizes too large to draw on the host
    and copy (a test copies back only the parts an oracle checks)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return [torch.empty(int(n), dtype=torch.float64, device=device).uniform_(lo, hi, generator=g)
            for _ in range(count)]


def gaussian_bumps(seed, count=32, dim=3, wmin=0.05, wmax=0.2):
    """Space-time Gaussian bump parameters: centers U(0,1)^dim in
    (x, y, z, t) order, widths U(wmin, wmax), amplitudes N(0,1)."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0.0, 1.0, (count, dim))
    widths = rng.uniform(wmin, wmax, count)
    amps = rng.standard_normal(count)
    return centers, widths, amps


def poisson_arrivals(seed, count, rate_per_s):
    """Arrival times (seconds) of a Poisson process: exponential gaps."""
    gaps = np.random.default_rng(seed).exponential(1.0 / rate_per_s, int(count))
    return np.cumsum(gaps)


def serving_mix(seed, count, spans=(16, 32, 64, 128), degrees=(1, 2, 3),
                slabs=(8, 32, 128, 512)):
    """Per-request (spans, degree, slabs), each drawn uniformly."""
    rng = np.random.default_rng(seed)
    s = rng.choice(spans, count)
    p = rng.choice(degrees, count)
    n = rng.choice(slabs, count)
    return [(int(a), int(b), int(c)) for a, b, c in zip(s, p, n)]
