"""The seeded input generators: published SplitMix64 outputs, determinism,
and the stated ranges of the synthetic workloads."""
import numpy as np

import oracle
from paper_2001_06444_gb300 import inputs


def test_splitmix64_published_outputs():
    # first outputs of SplitMix64 from state 0 (reference implementation)
    got = [int(v) for v in inputs.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_normal_moments():
    z = inputs.normal(3, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_ricker_peak_and_zero_crossings():
    f, dt = 10.0, 1e-4
    w = inputs.ricker(f, dt, 4000)
    assert np.argmax(w) == round(0.1 / dt) and w.max() == 1.0
    # zeros at t0 +- 1/(pi f sqrt 2)
    tz = 0.1 + 1.0 / (np.pi * f * np.sqrt(2.0))
    assert abs(w[int(round(tz / dt))]) < 2e-3


def test_full_size_model_ranges():
    s = inputs.full_size(nshot=96, nt=10)
    assert s.vel.shape == (351, 1701)
    assert np.all(s.vel[:45] == 1500.0)
    assert s.vel.min() == 1500.0 and s.vel.max() == 4700.0
    assert np.any(s.vel == 4500.0)
    assert s.nshot == 96 and s.nrec == 1701
    assert np.all(np.diff(s.src_ix) == 17) and s.src_ix[0] == 43
    assert oracle.courant(s.vel.max(), s.dt, s.dx, s.dz) < 1.0
    again = inputs.full_size(nshot=96, nt=10)
    assert np.array_equal(s.vel, again.vel)


def test_ensemble_perturbation_statistics():
    s = inputs.scaled_survey(301, 121, 4, 10, 10.0, 5)
    ens = inputs.ensemble(s.vel, s.dx, s.dz, 3)
    assert ens.shape == (3, 121, 301)
    wet = np.arange(121) * s.dz < 450
    assert np.all(ens[:, wet] == s.vel[wet])
    rel = (ens[:, ~wet] / s.vel[~wet] - 1.0).reshape(3, -1)
    assert np.allclose(rel.std(axis=1), 0.04, rtol=0.05)
    assert ens.max() <= 5400.0
    assert not np.array_equal(ens[0], ens[1])


def test_request_stream_ranges():
    reqs = inputs.request_stream(256, rate_hz=2.0)
    assert len(reqs) == 256
    assert all(1 <= r["nshot"] <= 32 for r in reqs)
    assert all(2000 <= r["nt"] < 6000 for r in reqs)
    assert all(10.0 <= r["f"] <= 15.0 for r in reqs)
    assert {(r["nx"], r["nz"]) for r in reqs} == set(inputs.MIXED_GRIDS)
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.diff(t).mean() - 0.5) < 0.1
