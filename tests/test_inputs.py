"""The seeded input generators hold the recipe the design states: orthonormal
MO coefficients, an aufbau first determinant and distinct excitations within
the orbital set, c_0 = 1, walkers around their assigned nuclei with
alternating spins, the workload shapes of the measured configurations, the
serving stream's molecule and job ranges, and reproducibility from the seed.
These generators hold no arithmetic of the method; both the oracle and the
CUDA path take their inputs from them."""

import math

import numpy as np
import pytest

from paper_1909_08423_gb300 import synth

WORKLOADS = {"h2": (synth.h2, 2, 1, 32, 16, 2), "be": (synth.be, 4, 4, 64, 32, 3),
             "h10": (synth.h10, 10, 16, 64, 32, 3), "n2": (synth.n2, 14, 32, 128, 32, 4)}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_workload_shapes(name):
    make, N, n_det, D, K, L = WORKLOADS[name]
    s = make()
    assert s["n_up"] + s["n_dn"] == N and s["n_up"] - s["n_dn"] in (0, 1)
    assert int(round(s["Z"].sum())) == N  # neutral
    assert len(s["ci"]) == n_det and s["occ_up"].shape == (n_det, s["n_up"])
    assert (s["D"], s["K"], s["L"], s["Zd"]) == (D, K, L, D // 2)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_orbitals_and_determinants(name):
    s = WORKLOADS[name][0]()
    C = s["mo_coeffs"]
    np.testing.assert_allclose(C.T @ C, np.eye(C.shape[1]), atol=1e-12)
    n_orb = C.shape[1]
    assert s["ci"][0] == 1.0
    np.testing.assert_array_equal(s["occ_up"][0], np.arange(s["n_up"]))
    np.testing.assert_array_equal(s["occ_dn"][0], np.arange(s["n_dn"]))
    keys = set()
    for p in range(len(s["ci"])):
        u, d = s["occ_up"][p], s["occ_dn"][p]
        assert len(set(u)) == len(u) and len(set(d)) == len(d)  # no orbital twice in a spin block
        assert u.max(initial=-1) < n_orb and d.max(initial=-1) < n_orb
        # at most a double excitation from the aufbau determinant
        exc = len(set(u) - set(range(s["n_up"]))) + len(set(d) - set(range(s["n_dn"])))
        assert exc <= 2
        keys.add((tuple(u), tuple(d)))
    assert len(keys) == len(s["ci"])  # distinct determinants


def test_walkers_sit_around_their_nuclei_with_alternating_spins():
    s = synth.h10()
    nuc = synth.electron_nuclei(s)
    # ten protons: up electrons take entries 0, 2, 4, ... and down electrons 1, 3, 5, ...
    np.testing.assert_array_equal(nuc, [0, 2, 4, 6, 8, 1, 3, 5, 7, 9])
    r = synth.random_walkers(s, 20000, 3)
    d = r - s["R"][nuc][None]
    np.testing.assert_allclose(d.mean(axis=0), 0.0, atol=0.05)
    np.testing.assert_allclose(d.std(axis=0), 1.0, atol=0.05)
    np.testing.assert_array_equal(synth.random_walkers(s, 5, 3), synth.random_walkers(s, 5, 3))


def test_serving_molecules_follow_the_stream_recipe():
    for seed in range(40):
        s = synth.serving_system(seed)
        Z, R = s["Z"], s["R"]
        assert 1 <= len(Z) <= 6 and np.all((Z >= 1) & (Z <= 10))
        N = s["n_up"] + s["n_dn"]
        assert N == int(round(Z.sum())) and 2 <= N <= 30
        assert np.all(np.abs(R) <= 3.0)
        for a in range(len(Z)):
            for b in range(a + 1, len(Z)):
                assert np.linalg.norm(R[a] - R[b]) >= 1.0
        assert 1 <= len(s["ci"]) <= 32
    a, b = synth.serving_system(7), synth.serving_system(7)
    np.testing.assert_array_equal(a["R"], b["R"])
    np.testing.assert_array_equal(a["mo_coeffs"], b["mo_coeffs"])


def test_serving_stream_arrivals_and_job_mix():
    jobs = synth.serving_stream(n_jobs=4000, master_seed=2024, rate_per_s=50.0)
    t = np.array([j["arrival"] for j in jobs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 50.0) < 0.1 / 50.0  # Poisson arrivals at the set rate
    W = np.array([j["W"] for j in jobs])
    assert W.min() >= 256 and W.max() <= 16384
    lw = np.log(W)  # log-uniform walker counts
    assert abs(lw.mean() - 0.5 * (math.log(256) + math.log(16384))) < 0.1
    frac = np.mean([j["kind"] == "eloc" for j in jobs])
    assert abs(frac - 0.5) < 0.05
    assert all(j["kind"] == "eloc" or j["n_steps"] == 10 for j in jobs)
    assert synth.serving_stream(n_jobs=5) == synth.serving_stream(n_jobs=5)
