"""Serving loop: continuous batching of jobs for molecules of different
sizes, admission by device-memory footprint, bounded polling, cancellation,
host-injected failures, and results that are the same alone and in a mix."""

import numpy as np
import pytest
import torch

from paper_1909_08423_gb300 import synth

pytestmark = pytest.mark.gpu

GB = 1 << 30


def _systems(lib):
    mk = [synth.h2(), synth.be(), synth.h10(), synth.serving_system(3), synth.serving_system(11)]
    return [lib.System(s, precision=lib.PN_MIXED, max_walkers=1) for s in mk]


def _run(lib, server, jobs):
    ids = [server.submit(**j) for j in jobs]
    return [server.poll(i, timeout_us=-1) for i in ids]


def _job(system, kind, W, seed, out=True):
    e = torch.full((W,), np.nan, dtype=torch.float64, device="cuda") if out else None
    r = torch.full((W, system.N, 3), np.nan, dtype=torch.float64, device="cuda") if out else None
    return dict(system=system, kind=kind, W=W, n_steps=5 if kind == 1 else 0, sigma=0.2, seed=seed,
                eloc_out=e, r_out=r)


def test_eloc_job_matches_direct_call(lib):
    sysd = synth.be()
    s = lib.System(sysd, precision=lib.PN_MIXED, max_walkers=512)
    r = torch.as_tensor(synth.random_walkers(sysd, 700, 3), device="cuda")
    E = torch.empty(700, dtype=torch.float64, device="cuda")
    s.eval_local_energy(r, E)
    srv = lib.Server(4 * GB, n_slots=2, chunk_walkers=512)
    out = torch.empty_like(E)
    jid = srv.submit(s, lib.PN_JOB_ELOC, 700, r_init=r, eloc_out=out)
    res = srv.poll(jid, timeout_us=-1)
    torch.cuda.synchronize()
    assert res.status == 0 and res.W == 700
    np.testing.assert_array_equal(out.cpu().numpy(), E.cpu().numpy())
    En = E.cpu().numpy()
    assert abs(res.e_mean - En.mean()) < 1e-10 * abs(En.mean())
    assert abs(res.e_stderr - En.std(ddof=1) / np.sqrt(700)) < 1e-8
    srv.close()


def test_results_same_alone_and_in_a_mix(lib):
    """Twenty sampled jobs (five molecules, both kinds, 64-900 walkers) run
    alone, then again inside a mix of forty jobs on four slots: energies and
    final positions are bitwise equal (per-walker work does not depend on
    the batch, and the random stream is keyed by job seed, walker and step)."""
    systems = _systems(lib)
    srv = lib.Server(8 * GB, n_slots=4, chunk_walkers=1024)
    rng = np.random.default_rng(0)
    spec = [(k % len(systems), int(rng.integers(0, 2)), int(rng.integers(64, 900)), 500 + k) for k in range(20)]
    alone = []
    for si, kind, W, seed in spec:
        j = _job(systems[si], kind, W, seed)
        res = _run(lib, srv, [j])[0]
        torch.cuda.synchronize()
        assert res.status == 0
        alone.append((j["eloc_out"].cpu().numpy().copy(), j["r_out"].cpu().numpy().copy()))
    again = [_job(systems[si], kind, W, seed) for si, kind, W, seed in spec]
    filler = [_job(systems[k % len(systems)], int(rng.integers(0, 2)), int(rng.integers(64, 2048)), 100 + k)
              for k in range(20)]
    jobs = [x for pair in zip(filler, again) for x in pair]
    results = _run(lib, srv, jobs)
    torch.cuda.synchronize()
    assert all(r.status == 0 for r in results), [r.status for r in results]
    for (e_a, r_a), j in zip(alone, again):
        np.testing.assert_array_equal(j["eloc_out"].cpu().numpy(), e_a)
        np.testing.assert_array_equal(j["r_out"].cpu().numpy(), r_a)
    # the mix overlapped on the device: the device intervals of jobs on
    # different slots (CUDA events around each job's work) intersect
    iv = sorted((r.dev_start_ms, r.dev_end_ms) for r in results)
    assert all(b > a for a, b in iv)
    overlaps = sum(1 for k in range(1, len(iv)) if iv[k][0] < max(e for _, e in iv[:k]))
    assert overlaps >= 2, iv
    srv.close()


def test_one_slot_runs_jobs_one_after_another(lib):
    """With a single slot no two device intervals intersect."""
    systems = _systems(lib)
    srv = lib.Server(8 * GB, n_slots=1, chunk_walkers=1024)
    res = _run(lib, srv, [_job(systems[k % 3], lib.PN_JOB_ELOC, 256, 40 + k, out=False) for k in range(6)])
    assert all(r.status == 0 for r in res)
    iv = sorted((r.dev_start_ms, r.dev_end_ms) for r in res)
    assert all(iv[k][0] >= iv[k - 1][1] for k in range(1, len(iv)))
    srv.close()


def test_budget_rejects_and_serialises(lib):
    systems = _systems(lib)
    from paper_1909_08423_gb300 import binding
    s = systems[2]
    fp = binding.job_footprint(s, 4096, 1024)
    srv = lib.Server(int(fp * 1.5), n_slots=4, chunk_walkers=1024)
    with pytest.raises(binding.PNError) as e:
        srv.submit(s, lib.PN_JOB_ELOC, 50_000_000)
    assert e.value.code == 3  # PN_EBUDGET
    res = _run(lib, srv, [_job(s, lib.PN_JOB_ELOC, 4096, k) for k in range(3)])
    assert all(r.status == 0 for r in res)
    # only one job fits at a time: the later ones waited for admission
    assert sorted(r.queue_ms for r in res)[-1] > 0
    srv.close()


def test_cancel_timeout_and_injected_failure(lib):
    systems = _systems(lib)
    srv = lib.Server(8 * GB, n_slots=1, chunk_walkers=2048, debug_fail_nth=2)
    long_job = srv.submit(systems[2], lib.PN_JOB_SWEEP, 8192, n_steps=20, seed=1)
    failing = srv.submit(systems[0], lib.PN_JOB_ELOC, 128, seed=2)
    cancelled = srv.submit(systems[1], lib.PN_JOB_ELOC, 128, seed=3)
    assert srv.cancel(cancelled) == 0
    assert srv.poll(long_job, timeout_us=1) is None  # still running: bounded wait expires
    r0 = srv.poll(long_job, timeout_us=-1)
    r1 = srv.poll(failing, timeout_us=-1)
    r2 = srv.poll(cancelled, timeout_us=-1)
    assert r0.status == 0
    assert r1.status == 6  # PN_EDEVICE, injected on the host before any launch
    assert r2.status == 7  # PN_ECANCELLED
    # the server keeps serving after the failure
    r3 = _run(lib, srv, [_job(systems[0], lib.PN_JOB_ELOC, 64, 9)])[0]
    assert r3.status == 0
    srv.close()
