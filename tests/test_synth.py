"""The seeded input generators (`synth/`) against the distributions they
stand for: the SplitMix64 definition (Steele, Lea & Flood 2014), the Plummer
model in standard units (Section 3 inputs; Aarseth, Henon & Wielen 1974
sampling), the Salpeter mass spectrum, and the ensemble / request-stream
recipes (log-uniform N, Poisson arrivals).  No GPU, no oracle."""
import math

import numpy as np
import pytest

import synth

stats = pytest.importorskip("scipy.stats")

_M64 = 1 << 64


def test_splitmix64_published_outputs():
    # state 0: the generator's first outputs as published with its definition
    c1 = 0x2545F4914F6CDD1D  # (seed, stream) -> state mapping of synth
    seed = (-pow(c1, -1, _M64)) % _M64  # the seed whose state is 0
    z = [int(u) for u in synth.splitmix64(seed, 0, 3)]
    assert z == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # streams and seeds give different sequences; uniforms lie strictly in (0, 1)
    assert not np.array_equal(synth.splitmix64(1, 0, 8), synth.splitmix64(1, 1, 8))
    u = synth.uniform(3, 0, 200_000)
    assert u.min() > 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_plummer_mass_profile_and_velocities():
    # M(<r) = r^3 / (r^2 + a^2)^(3/2) with a = 3 pi / 16 in standard units,
    # truncated at the 0.999 mass fraction
    n = 40_000
    x, v, m = synth.plummer(n, 2)
    a = 3.0 * math.pi / 16.0
    r = np.linalg.norm(x, axis=1)
    cdf = lambda s: np.minimum(1.0, (s ** 3 / (s * s + a * a) ** 1.5) / 0.999)
    assert stats.kstest(r, cdf).pvalue > 1e-3
    assert np.allclose(m, 1.0 / n)
    # isotropic velocities, at rest on average, all bound to the cluster
    assert np.allclose((m[:, None] * v).sum(0), 0.0, atol=1e-15)
    s2 = (v * v).mean(0)
    assert np.all(np.abs(s2 / s2.mean() - 1.0) < 0.03)
    phi = -1.0 / np.sqrt(r * r + a * a)  # Plummer potential, standard units
    assert np.all(0.5 * (v * v).sum(1) + phi < 1e-12)


def test_salpeter_mass_spectrum():
    # dN/dm ~ m^-2.35 on [m_lo, 100 m_lo], total mass 1
    n = 100_000
    m = synth.salpeter_masses(n, 5)
    assert m.sum() == pytest.approx(1.0, rel=1e-12)
    lo = m.min()
    assert m.max() / lo <= 100.0 * (1 + 1e-12) and m.max() / lo > 50.0
    p = 1.0 - 2.35
    cdf = lambda y: np.clip((y ** p - 1.0) / (100.0 ** p - 1.0), 0.0, 1.0)
    assert stats.kstest(m / lo, cdf).pvalue > 1e-3
    # positions are the equal-mass model's (only the centre-of-mass shift
    # differs), so the masses are independent of them
    x0, _, _ = synth.plummer(1000, 7)
    x1, _, m1 = synth.plummer_salpeter(1000, 7)
    np.testing.assert_allclose(x1, x0 - (m1[:, None] * x0).sum(0), atol=1e-12)


def test_ensemble_and_request_stream_recipes():
    ens = synth.ensemble(4000, 1024, 32768, seed=1)
    n = np.array([e.n for e in ens])
    assert n.min() >= 1024 and n.max() <= 32768
    lu = (np.log(n) - math.log(1024)) / (math.log(32768) - math.log(1024))
    assert stats.kstest(lu, "uniform").pvalue > 1e-3
    assert {e.theta for e in ens} == {0.3, 0.5, 0.7}
    assert [e.seed for e in ens] == list(range(4000))
    req = synth.request_stream(4000, rate_per_s=20.0, seed=2)
    t = np.array([q.arrival_s for q in req])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert stats.kstest(gaps, "expon", args=(0, 1 / 20.0)).pvalue > 1e-3
    assert {q.t_end for q in req} == {0.125, 0.25, 0.5}
    nq = np.array([q.n for q in req])
    assert nq.min() >= 1 << 10 and nq.max() <= 1 << 18
