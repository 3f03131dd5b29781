"""The seeded synthetic inputs match the distributions they state (the sweep
and serving workloads of the benchmark), and the same seed gives the same
workload on every machine."""
import numpy as np

from paper_1910_08020_gb300 import workloads as W


def test_random_state_is_normalised_and_seeded():
    a = W.random_state(10, 3)
    assert abs(np.linalg.norm(a) - 1) < 1e-12
    assert np.array_equal(a, W.random_state(10, 3)) and not np.array_equal(a, W.random_state(10, 4))


def test_sweep_specs_follow_their_distribution():
    specs = W.sweep_specs()
    assert len(specs) == 256 and specs == W.sweep_specs()
    lam = np.array([s["lam"] for s in specs])
    T = np.array([s["T"] for s in specs])
    M = np.array([s["M"] for s in specs])
    assert lam.min() >= 0 and lam.max() < 6 and T.min() >= 5 and T.max() <= 20
    assert M.min() >= 100 and M.max() <= 400 and all(s["decomp"] == 1 for s in specs)
    # uniform over the three lattices: each share within 4 sigma of 1/3
    counts = np.array([sum(1 for s in specs if (s["d"], s["L"]) == lt) for lt in W.SWEEP_LATTICES])
    assert counts.sum() == 256 and np.all(np.abs(counts - 256 / 3) < 4 * np.sqrt(256 * (1 / 3) * (2 / 3)))
    assert abs(lam.mean() - 3.0) < 4 * 6 / np.sqrt(12 * 256)


def test_poisson_stream_follows_its_distribution():
    reqs = W.poisson_stream()
    assert len(reqs) == 2000 and reqs == W.poisson_stream()
    t = np.array([r["arrival"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps at 200/s: mean 5 ms, within 4 standard errors
    assert abs(gaps.mean() - 1 / 200) < 4 * (1 / 200) / np.sqrt(len(gaps))
    assert all(50 <= r["M"] <= 500 and abs(r["T"] - 0.04 * r["M"]) < 1e-12 for r in reqs)
    assert {(r["d"], r["L"]) for r in reqs} == set(W.SERVE_LATTICES)
