"""The corrector's timestep criterion on the device (Aarseth's formula,
Section 2 step 6): wherever the FP32 screen decides, its value is the exact
power of two at or below the FP64 expression; elsewhere the FP64 expression
itself is returned, bit for bit.  Inputs span wide random ranges, single
time-scale derivatives (the physical case, including the very short steps
whose higher derivatives leave FP32's range before normalisation), and values
placed just beside a power-of-two boundary."""
import numpy as np
import pytest

hh = pytest.importorskip("paper_1602_02832_gb300")

pytestmark = pytest.mark.gpu

ETA = 0.02


def _fp64(A, J, S, T, eta):
    with np.errstate(all="ignore"):
        return np.sqrt(eta * (np.sqrt(A * S) + J) / (np.sqrt(J * T) + S))


def _pow2_floor(x):
    b = np.asarray(x, dtype=np.float64).view(np.int64) & np.int64(-(1 << 52))  # clear the mantissa
    return b.view(np.float64)


def _is_pow2(x):
    b = np.asarray(x, dtype=np.float64).view(np.int64)
    return (b & ((1 << 52) - 1)) == 0


def _check(A, J, S, T, eta=ETA):
    dev = hh.hh_selftest_aarseth(A, J, S, T, eta)
    ref = _fp64(A, J, S, T, eta)
    screened = _is_pow2(dev) & ~(dev == ref)
    # fallback values are the FP64 expression exactly (NaN where it is NaN)
    fb = ~screened
    same = (dev[fb] == ref[fb]) | (np.isnan(dev[fb]) & np.isnan(ref[fb]))
    assert same.all(), np.flatnonzero(fb)[~same][:5]
    # screened values are the power of two below the FP64 value
    assert np.array_equal(dev[screened], _pow2_floor(ref[screened]))
    return screened.mean()


def test_criterion_wide_random_ranges():
    rng = np.random.default_rng(1)
    n = 400_000
    A, J, S, T = (10.0 ** rng.uniform(-45, 45, n) for _ in range(4))
    _check(A, J, S, T)
    # zeros, subnormals, infinities
    A[:5] = [0.0, 5e-324, np.inf, 1.0, 1.0]
    S[5:8] = [0.0, np.inf, 1e-310]
    _check(A, J, S, T)


def test_criterion_single_timescale_is_screened():
    # a ~ |a|, tau a time scale: J ~ (a/tau)^2, S ~ (a/tau^2)^2, T ~ (a/tau^3)^2
    rng = np.random.default_rng(2)
    n = 400_000
    a = 10.0 ** rng.uniform(-3, 6, n)
    tau = 10.0 ** rng.uniform(-9, 0, n)
    r = [10.0 ** rng.uniform(-2, 2, n) for _ in range(3)]
    A, J, S, T = a * a, (a / tau) ** 2 * r[0], (a / tau ** 2) ** 2 * r[1], (a / tau ** 3) ** 2 * r[2]
    frac = _check(A, J, S, T)
    # the FP32 screen decides almost everywhere, including the shortest steps
    assert frac > 0.99
    short = tau < 1e-6
    assert short.sum() > 1000
    fs = _check(A[short], J[short], S[short], T[short])
    assert fs > 0.99


def test_criterion_next_to_power_of_two_boundaries():
    # a time-unit change c (A, J/c^2, S/c^4, T/c^6; the step scales by c)
    # puts the FP64 value within a relative delta of a power of two
    rng = np.random.default_rng(3)
    n = 200_000
    A = 10.0 ** rng.uniform(-2, 4, n)
    J = A * 10.0 ** rng.uniform(-1, 1, n)
    S = A * 10.0 ** rng.uniform(-1, 1, n)
    T = A * 10.0 ** rng.uniform(-1, 1, n)
    w = _fp64(A, J, S, T, ETA)
    k = rng.integers(-25, 0, n).astype(np.float64)
    delta = np.sign(rng.uniform(-1, 1, n)) * 10.0 ** rng.uniform(-9, -4, n)
    c = 2.0 ** k * (1.0 + delta) / w
    frac = _check(A, J / c ** 2, S / c ** 4, T / c ** 6)
    # both sides of the screen's margin (2^-18) are exercised
    assert 0.05 < frac < 0.95


def test_block_quantisation_matches_oracle():
    # the device's block quantisation (integer path and FP64 path) against the
    # oracle's, on block-rule inputs and on special values
    oracle = pytest.importorskip("oracle")
    rng = np.random.default_rng(4)
    n = 6000
    dt_min, dt_max = 2.0 ** -30, 2.0 ** -6
    lv = rng.integers(6, 31, n)
    dt_old = 2.0 ** -lv
    t_new = rng.integers(0, 2 ** 20, n) * dt_old           # multiples of dt_old
    t_new[::3] = rng.integers(0, 2 ** 30, n)[::3] * dt_min  # any multiple of dt_min
    want = dt_old * 10.0 ** rng.uniform(-3, 3, n)
    want[::7] = dt_old[::7] * 2.0 ** rng.integers(-3, 4, n)[::7]  # exact powers of two
    specials = [np.nan, -np.nan, np.inf, -np.inf, 0.0, -0.0, 5e-324, -3.0, 1e300, 2e300, 1e-310]
    want[: len(specials)] = specials
    t_new[20:30] = [0.0, 1e-320, np.inf, 2.0 ** -1000, 1.5, 3.0, 0.25, -0.5, 1e300, 2.0 ** -959]
    dt_old[40:45] = [1.0, 2.0, 0.75, 2.0 ** -1023, 3e-308]
    dev = hh.hh_selftest_block_dt(want, dt_old, t_new, dt_min, dt_max)
    ref = np.array([oracle.block_dt(w, d, t, dt_min, dt_max) for w, d, t in zip(want, dt_old, t_new)])
    same = (dev == ref) | (np.isnan(dev) & np.isnan(ref))
    assert same.all(), [(want[i], dt_old[i], t_new[i], dev[i], ref[i]) for i in np.flatnonzero(~same)[:5]]
