"""CPU checks of the numerical facts behind the FP32 closed-line design (the closure rows' end gain
and the cancellation of plain sums), computed from the oracle's bands with numpy.  They fix the
planner's threshold decision: the second derivative's closure makes the solve magnify an end row's
rounding by about 93 (above the threshold 16, so FP32 sweeps run those rows in FP64); the first
derivative's (about 5) and the filter's (about 2) stay below it."""
import numpy as np
import pytest

GAIN_THRESHOLD = 16.0


def end_gain(o, n, order, param):
    """Largest |entry| of A^{-1} and A^{-T} in the four columns at each end of a closed line."""
    a, b, c, _ = o.bands(n, order, "closed", param)
    A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    Ai = np.linalg.inv(A)
    cols = list(range(4)) + list(range(n - 4, n))
    return max(np.abs(Ai[:, cols]).max(), np.abs(Ai[cols, :]).max())


@pytest.mark.parametrize("n", [16, 64, 256])
def test_closure_end_gains(oracle_mod, n):
    h = oracle_mod.grid_spacing(n, "closed")
    g1 = end_gain(oracle_mod, n, 1, h)
    g2 = end_gain(oracle_mod, n, 2, h)
    gf = end_gain(oracle_mod, n, 3, 0.45)
    assert 4.0 < g1 < 6.0 and g1 < GAIN_THRESHOLD
    assert 90.0 < g2 < 95.0 and g2 > GAIN_THRESHOLD
    assert gf < 3.0


def test_plain_sum_cancellation_of_the_second_derivative(oracle_mod):
    """On a smooth line the plain FP32 sum of the second derivative's interior taps loses several
    bits to cancellation; the same taps on second differences (plus the zero tap sum) do not."""
    n = 512
    h = oracle_mod.grid_spacing(n, "periodic")
    _, _, _, B7 = oracle_mod.bands(n, 2, "periodic", h)
    t0, t1, t2 = B7[0, 3], B7[0, 4], B7[0, 5]
    x = np.arange(n) * h
    v = (np.cos(20 * x) + 0.5 * np.sin(7 * x)).astype(np.float32)
    exact = np.array([t0 * float(v[j]) + t1 * (float(v[(j + 1) % n]) + float(v[j - 1]))
                      + t2 * (float(v[(j + 2) % n]) + float(v[j - 2])) for j in range(n)])
    f32 = np.float32
    w = [np.roll(v, -k) for k in (-2, -1, 0, 1, 2)]
    plain = f32(t0) * w[2] + f32(t1) * (w[3] + w[1]) + f32(t2) * (w[4] + w[0])
    diffs = f32(t1) * ((w[3] - w[2]) - (w[2] - w[1])) + f32(t2) * ((w[4] - w[2]) - (w[2] - w[0]))
    scale = np.abs(exact).max()
    e_plain = np.abs(plain.astype(np.float64) - exact).max() / scale
    e_diffs = np.abs(diffs.astype(np.float64) - exact).max() / scale
    # measured: plain 4.1e-6, second differences 3.8e-7 (the rounding of the taps and of the sum)
    assert e_diffs < 1e-6
    assert e_plain > 5 * e_diffs
