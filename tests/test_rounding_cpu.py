"""Floating-point identities that kernels rely on to reproduce other kernels' values bit for
bit (CPU, numpy FP64 / FP32 arithmetic, round to nearest even).

* The one-pass 5-point assembly forms a coupling as (a + b) * m with m = -(1/2)/h^2 formed
  exactly, where the separate assembly kernel forms (-(1/2) (a + b)) / h^2 as
  (-0.5 * (a + b)) * (1/h^2): halving is exact, so both are one rounding of the same real
  product.
* The even-row restriction sums (4 r(2I) + 2 (r(2I-1) + r(2I+1))) / 16, where the
  whole-residual kernel adds the odd-row terms, zero after an exact row solve: adding zeros
  changes no value (the sign of a zero result aside)."""
import numpy as np


def _spacings():
    # the workloads' spacings (annulus 8193^2 in x and theta, inclusion 1025^2, serving sides)
    # and random ones
    h = [0.8 / 8192, 2 * np.pi / 8192, 1.0 / 1024, 6.0 / 2048, 1.0 / 128]
    rng = np.random.default_rng(1)
    return np.concatenate([h, 10.0 ** rng.uniform(-5, 0, 200)])


def test_coupling_with_the_halved_constant_rounds_like_the_two_step_form():
    rng = np.random.default_rng(2)
    a = rng.uniform(1e-3, 1e3, 200_000)
    b = a * rng.uniform(0.5, 2.0, a.size)
    s = a + b
    for h in _spacings():
        ih2 = 1.0 / (h * h)
        m = -0.5 * ih2
        assert m == -(ih2 / 2)  # formed exactly
        two_step = (-0.5 * s) * ih2
        one_step = s * m
        assert np.array_equal(two_step.view(np.int64), one_step.view(np.int64)), h


def test_even_row_weights_equal_the_full_stencil_on_zero_odd_rows():
    rng = np.random.default_rng(3)
    for dt in (np.float64, np.float32):
        rc, rw, re = (rng.standard_normal(100_000).astype(dt) * dt(1e3) for _ in range(3))
        z = np.zeros_like(rc)
        edge = ((rw + re) + z) + z
        corner = ((z + z) + z) + z
        full = (dt(4) * rc + dt(2) * edge + corner) * dt(0.0625)
        even = (dt(4) * rc + dt(2) * (rw + re)) * dt(0.0625)
        assert full.dtype == even.dtype == dt
        assert np.array_equal(full, even)
