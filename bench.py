"""Benchmark: walker local energies per second on one GB300 (per rank).

One step = one pass of the whole hot path over the Be-atom workload (seeded
synthetic Be: Z=4, 2 up 2 down electrons, 4 determinants, 4s2p basis, D=64,
L=3, K=32; 4096 walkers): 100 Metropolis steps (Gaussian proposal sigma =
0.2 bohr), local energies of all walkers (forward Laplacian jet), clipping,
and the hand-written backward of ln|psi| for the VMC loss gradient.
value = walkers x ranks / step time.  The headline runs the mixed path; the
same step is also timed on the plain FP64 path.

--impl reference times the CPU oracle (the plain FP64 definition) on the
host cores on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "be"
W_PER_RANK = 4096
N_METROPOLIS = 100
SIGMA = 0.2
METRIC = "walker local energies/s"
UNIT = "walkers/s"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# Algorithmic floating-point work per launch class (multiply-add = 2), per
# walker, for the value pass (T = 1) and the jet pass (T = 3N + 2).
def tc_sampler_executed_flops(sysd, W, n_sms=152):
    """bf16 tensor-core FLOPs the tcgen05 sampler executes per Metropolis step
    over all CTAs: every stage is a 128-row tile with six piece products per
    float32 product (K x Np per product, Np padded to 16), the first layer's h
    excluded; CTAs hold WT walkers as the launcher sizes them."""
    N = sysd["n_up"] + sysd["n_dn"]
    M = len(sysd["Z"])
    D, Zd, K, L = sysd["D"], sysd["Zd"], sysd["K"], sysd["L"]
    Hw = max(K, Zd)
    no = sysd["mo_coeffs"].shape[1]
    pad = lambda x: (x + 15) // 16 * 16
    nup, ndn = sysd["n_up"], sysd["n_dn"]
    cnts = [nup * (nup - 1) // 2 + ndn * (ndn - 1) // 2, nup * ndn, N * M]
    live = sum(1 for c in cnts if c > 0)
    stages = [(D, Zd)] * (L - 1) + [(K, Hw), (Hw, Zd), (Zd, D)] * (L * live)
    stages += [(D, D), (D, D), (D, pad(no)), (D, D), (D, D), (D, 16)]
    macs_tile = sum(6 * k * n * 128 for k, n in stages)
    WT = min(128 // N, 128 // max(cnts), -(-W // n_sms))
    ctas = -(-W // WT)
    return 2 * macs_tile * ctas


def algorithmic_flops(sysd, kernel, mode):
    N = sysd["n_up"] + sysd["n_dn"]
    M = len(sysd["Z"])
    D, Zd, K, L = sysd["D"], sysd["Zd"], sysd["K"], sysd["L"]
    Hw = max(K, Zd)
    no = sysd["mo_coeffs"].shape[1]
    nd = len(sysd["ci"])
    P = N * (N - 1) // 2 + N * M
    T = 1 if mode == "value" else 3 * N + 2
    jc = 1 if mode == "value" else 3
    if kernel == "k_filter":
        return L * P * jc * 2 * (K * Hw + Hw * Zd)
    if kernel == "k_linear":
        per_layer = N * T * 2 * (D * Zd + 3 * Zd * D)
        heads = N * T * 2 * (D * D * 2 + D * no) + T * 2 * (2 * D * D + D)
        return L * per_layer + heads
    if kernel == "k_message":
        # value: 2 per partner; derivative rows 4; Laplacian row ~ 20
        per_row = 2 if T == 1 else (2 + 4 * (T - 2) + 20) / T
        return L * N * T * Zd * (N - 1 + M) * per_row
    if kernel in ("k_metropolis_warp", "k_metropolis_fused", "k_metropolis_tc"):
        # one value pass of the network per walker-step (float32 work):
        # filters, h and receiving maps, messages, both heads
        return sum(algorithmic_flops(sysd, k, "value") for k in ("k_filter", "k_linear", "k_message"))
    if kernel == "k_slater":
        nsig = [sysd["n_up"], sysd["n_dn"]]
        f = 0
        for ns in nsig:
            if ns == 0:
                continue
            f += 2 / 3 * ns ** 3 * 2
            if T > 1:
                f += 2 * ns ** 3 + 2 * ns ** 2 + 3 * N * (2 * ns ** 3 + 2 * ns ** 2 + 2 * ns ** 2)
        return nd * f
    return None


def _clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "20"],
                                stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except Exception:
        return None
    # start timing only once the sampler is writing, so that its samples fall
    # inside the timed region; the lines before it are dropped from the summary
    t0 = time.time()
    while time.time() - t0 < 10.0 and proc.poll() is None:
        try:
            if os.path.getsize(path) > 0:
                break
        except OSError:
            pass
        time.sleep(0.01)
    try:
        proc.skip = sum(1 for l in open(path) if l.strip())
    except OSError:
        proc.skip = 0
    return proc


def _clock_summary(path, dev_index, skip=0):
    try:
        rows = [l.strip().split(", ") for l in open(path) if l.strip()][skip:]
    except Exception:
        return None
    rows = [r for r in rows if len(r) >= 9 and r[0] == str(dev_index)]
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    reasons = set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        for k, nm in enumerate(names):
            if "Active" in r[5 + k] and "Not" not in r[5 + k]:
                reasons.add(nm)
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(rows)}


def run_reference(args):
    """The CPU oracle, as it stands, on a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    from oracle import clip as oclip
    from oracle import sampling
    from oracle.ansatz import Oracle
    from paper_1909_08423_gb300 import synth
    sysd = synth.WORKLOADS[WORKLOAD]["make"]()
    o = Oracle(sysd)
    Ws = args.ref_walkers
    r = sampling.init_walkers(sysd, Ws, 1)
    lp, _ = o.eval_logpsi(r)

    def step(k):
        nonlocal r, lp
        r, lp, _ = sampling.metropolis(o, r, lp, N_METROPOLIS, SIGMA, seed=1, step0=k * N_METROPOLIS)
        E, _, _ = o.local_energy(r)
        Ec = oclip.clip_local_energy(E)
        o.grad_logpsi(r, oclip.loss_cotangent(Ec))

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    dt = (time.perf_counter() - t0) / args.steps
    v = Ws / dt
    cores = torch.get_num_threads()
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"Be atom, {Ws} walkers sample of {W_PER_RANK}, {N_METROPOLIS} Metropolis steps "
                                   "+ E_loc + clip + grad per step", "walkers": Ws},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{Ws} walkers per step of the {W_PER_RANK}-walker Be workload"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(n_walkers=96):
    """Oracle timing on the host cores for the cpu_baseline key."""
    import torch
    from oracle import clip as oclip
    from oracle import sampling
    from oracle.ansatz import Oracle
    from paper_1909_08423_gb300 import synth
    sysd = synth.WORKLOADS[WORKLOAD]["make"]()
    o = Oracle(sysd)
    r = sampling.init_walkers(sysd, n_walkers, 1)
    lp, _ = o.eval_logpsi(r)
    t0 = time.perf_counter()
    r, lp, _ = sampling.metropolis(o, r, lp, N_METROPOLIS, SIGMA, seed=1, step0=0)
    E, _, _ = o.local_energy(r)
    Ec = oclip.clip_local_energy(E)
    o.grad_logpsi(r, oclip.loss_cotangent(Ec))
    dt = time.perf_counter() - t0
    cores = torch.get_num_threads()
    # the same step on one core, on a smaller sample of the same walkers
    n1 = max(2, n_walkers // 8)
    torch.set_num_threads(1)
    try:
        r1 = sampling.init_walkers(sysd, n1, 1)
        lp1, _ = o.eval_logpsi(r1)
        t1 = time.perf_counter()
        r1, lp1, _ = sampling.metropolis(o, r1, lp1, N_METROPOLIS, SIGMA, seed=1, step0=0)
        E1, _, _ = o.local_energy(r1)
        o.grad_logpsi(r1, oclip.loss_cotangent(oclip.clip_local_energy(E1)))
        dt1 = time.perf_counter() - t1
    finally:
        torch.set_num_threads(cores)
    return {"value": n_walkers / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_walkers} walkers: {N_METROPOLIS} Metropolis steps + E_loc + clip + grad (one step)",
            "seconds": dt, "value_1core": n1 / dt1, "sample_1core": f"{n1} walkers, same step, 1 thread"}


def run_langevin(sysd, W, target=0.57, steps=10):
    """The paper's Langevin sampler on the bench workload: tau bisected (on
    log tau, short runs) to the 57 % target acceptance, then `steps` steps
    timed with CUDA events (mixed path)."""
    import torch
    from paper_1909_08423_gb300 import binding
    s = binding.System(sysd, precision=binding.PN_MIXED, max_walkers=W)
    r = torch.empty(W, s.N, 3, dtype=torch.float64, device="cuda")
    s.init_walkers(r, 7)
    lp = torch.empty(W, dtype=torch.float64, device="cuda")
    g = torch.empty_like(r)
    s.eval_drift(r, g, lp)
    s.langevin_step(r, lp, g, 20, 0.05, 7, 0)  # leave the initial Gaussian cloud
    nacc = torch.zeros(1, dtype=torch.int64, device="cuda")
    lo, hi = np.log(1e-3), np.log(2.0)
    step0 = 100
    for _ in range(7):
        tau = float(np.exp(0.5 * (lo + hi)))
        s.langevin_step(r, lp, g, 5, tau, 7, step0, nacc)
        step0 += 5
        acc = int(nacc.item()) / (5 * W)
        if acc > target:
            lo = np.log(tau)
        else:
            hi = np.log(tau)
    tau = float(np.exp(0.5 * (lo + hi)))
    s.langevin_step(r, lp, g, 2, tau, 7, step0)
    step0 += 2
    torch.cuda.synchronize()

    def timed(k0):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.langevin_step(r, lp, g, steps, tau, 7, k0, nacc)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms = timed(step0)
    acc = int(nacc.item()) / (steps * W)
    # the same steps with the drift from the forward jet pass, for comparison
    s.set_option(binding.PN_OPT_DRIFT, 0)
    s.langevin_step(r, lp, g, 2, tau, 7, step0 + steps)
    ms_jet = timed(step0 + steps + 2)
    s.set_option(binding.PN_OPT_DRIFT, 1)
    out = {"tau": tau, "accept_rate": acc, "ms_per_step": ms,
           "walker_steps_per_s": W / (ms / 1e3), "walkers": W, "steps_timed": steps,
           "ms_per_step_jet_drift": ms_jet,
           "note": "all-electron drift-diffusion proposal with the drift clipped at the nearest nucleus; "
                   "tau bisected to the 57 % target acceptance; staged kernels, the drift at each proposal "
                   "by reverse mode (ms_per_step_jet_drift: the same steps with the forward jet pass)"}
    s.close()
    return out


def run_configs():
    """The H10 chain (8192 walkers: E_loc + clipping + grad ln|psi|) and the
    N2-shaped diatomic (16384 walkers in chunks of 4096: one Metropolis step
    + E_loc + clipping + grad ln|psi|) at full size, mixed path, CUDA events
    over two repetitions after one warm-up."""
    import torch
    from paper_1909_08423_gb300 import binding, synth

    def timed(fn, n=2):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    out = {}
    for name, make, W, chunk, sweep in (("h10", synth.h10, 8192, 8192, 0), ("n2", synth.n2, 16384, 4096, 1)):
        sysd = make()
        s = binding.System(sysd, precision=binding.PN_MIXED, max_walkers=chunk)
        r = torch.empty(W, s.N, 3, dtype=torch.float64, device="cuda")
        s.init_walkers(r, 3)
        lp = torch.empty(W, dtype=torch.float64, device="cuda")
        sg = torch.empty_like(lp)
        s.eval_logpsi(r, lp, sg)
        s.metropolis_step(r, lp, 20, SIGMA, 3, 0)
        E, Ec, cot = torch.empty_like(lp), torch.empty_like(lp), torch.empty_like(lp)
        g = torch.empty(s.n_params, dtype=torch.float64, device="cuda")
        k = [100]

        def step():
            if sweep:
                s.metropolis_step(r, lp, 1, SIGMA, 3, k[0])
                k[0] += 1
            s.eval_local_energy(r, E)
            binding.clip_local_energy(E, Ec, cot)
            s.grad_logpsi(r, cot, g)

        ms_step = timed(step)
        out[name] = {"walkers": W, "chunk": chunk, "ms_step": ms_step, "walker_eloc_per_s": W / (ms_step / 1e3),
                     "ms_eloc": timed(lambda: s.eval_local_energy(r, E)),
                     "ms_grad": timed(lambda: s.grad_logpsi(r, cot, g)),
                     "ms_metropolis_step": timed(lambda: s.metropolis_step(r, lp, 1, SIGMA, 5, 10 ** 6)) if sweep else None}
        s.close()
    return out


def run_line_scan(npts=4096):
    """E_loc along the LiH line scan through both nuclei and both fixed
    electrons (mixed path), timed with CUDA events."""
    import torch
    from paper_1909_08423_gb300 import binding, synth
    sysd = synth.lih()
    r0, e, d, t0, t1 = synth.lih_scan()
    s = binding.System(sysd, precision=binding.PN_MIXED, max_walkers=npts)
    r0d = torch.as_tensor(r0, device="cuda")
    E = torch.empty(npts, dtype=torch.float64, device="cuda")
    for _ in range(2):
        s.eval_line_scan(r0d, e, d, t0, t1, npts, E)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.eval_line_scan(r0d, e, d, t0, t1, npts, E)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    En = E.cpu().numpy()
    s.close()
    return {"points": npts, "ms": ms, "points_per_s": npts / (ms / 1e3), "system": "LiH-shaped, 4 e, 4 dets",
            "finite_fraction": float(np.isfinite(En).mean()),
            "note": "one electron moved along the molecular axis through both nuclei and both fixed electrons"}


def run_vmc_train(sysd, steps=10):
    """The paper's training configuration (batch 10000, 2000 walkers, pool
    refilled every 100 steps after 50 discarded steps) on the bench system:
    one optimisation step (clipped loss gradient on the batch, AdamW, new
    parameters uploaded) and one pool refill, timed separately."""
    import torch
    from paper_1909_08423_gb300 import binding, synth
    from paper_1909_08423_gb300.vmc import VMCTrainer
    s = binding.System(sysd, precision=binding.PN_MIXED, max_walkers=10000)
    tr = VMCTrainer(s, synth.flatten_params(sysd), walkers=2000, batch=10000, resample_period=100, n_discard=50,
                    n_decorr=1, seed=11)
    tr.step()  # first pool and one step
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = [tr.step() for _ in range(steps)]
    torch.cuda.synchronize()
    step_ms = (time.perf_counter() - t0) * 1e3 / steps
    t0 = time.perf_counter()
    tr.resample()
    torch.cuda.synchronize()
    refill_ms = (time.perf_counter() - t0) * 1e3
    s.close()
    return {"batch": 10000, "walkers": 2000, "train_step_ms": step_ms, "pool_refill_ms": refill_ms,
            "amortized_step_ms": step_ms + refill_ms / 100, "e_mean_last": hist[-1]["e_mean"],
            "note": "host-timed (the parameter upload synchronises); refill = 50 + 500 Metropolis steps of 2000 walkers"}


def run_ablation(W=4096, steps=3):
    """The paper's ablation variants on the bench atom (single or four
    determinants, with or without backflow, and both heads removed): the
    bench step (100 Metropolis steps + E_loc + clipping + backward) of W
    walkers per variant, mixed path, CUDA events."""
    import torch
    from paper_1909_08423_gb300 import binding, synth
    variants = {"SD-SJ": (1, 0, 1), "SD-BF": (1, 0, 0), "MD-SJ": (4, 0, 1), "MD-BF": (4, 0, 0), "MD-none": (4, 1, 1)}
    out = {}
    for name, (nd, nj, nb) in variants.items():
        sysd = synth.make_system([4.0], [[0, 0, 0]], lambda z: {0: 4, 1: 2}, n_det=nd, D=64, K=32, L=3, seed=0,
                                 no_jastrow=nj, no_backflow=nb)
        s = binding.System(sysd, precision=binding.PN_MIXED, max_walkers=W)
        r = torch.empty(W, s.N, 3, dtype=torch.float64, device="cuda")
        s.init_walkers(r, 5)
        lp = torch.empty(W, dtype=torch.float64, device="cuda")
        sg = torch.empty_like(lp)
        s.eval_logpsi(r, lp, sg)
        E, Ec, cot = torch.empty_like(lp), torch.empty_like(lp), torch.empty_like(lp)
        g = torch.empty(s.n_params, dtype=torch.float64, device="cuda")

        def step(k):
            s.metropolis_step(r, lp, N_METROPOLIS, SIGMA, 5, k * N_METROPOLIS)
            s.eval_local_energy(r, E)
            binding.clip_local_energy(E, Ec, cot)
            s.grad_logpsi(r, cot, g)

        step(0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(steps):
            step(1 + k)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"n_det": nd, "jastrow": not nj, "backflow": not nb, "ms_per_step": ms,
                     "walker_eloc_per_s": W / (ms / 1e3), "e_mean": float(Ec.mean())}
        s.close()
    return out


def run_serving(n_jobs, seed=2024, slots=4, chunk=2048, budget_gb=64, wmax=16384, load=0.7,
                precisions=("mixed", "fp64"), sweep=()):
    """Poisson stream of seeded molecules through the serving loop, mixed and
    plain FP64 servers.  The arrival rate is set to `load` times the mixed
    server's measured capacity (a closed-loop calibration burst first).
    `sweep` lists further loads at which the mixed server is measured again
    on the same stream (the latency-load curve)."""
    import torch
    from paper_1909_08423_gb300 import binding, synth
    stream = synth.serving_stream(n_jobs, seed, rate_per_s=1.0, wmax=wmax)
    out = {}
    rate = cap_mixed = None
    runs = [(p_, load) for p_ in precisions] + [("mixed", l_) for l_ in sweep]
    for prec_name, run_load in runs:
        prec = binding.PN_MIXED if prec_name == "mixed" else binding.PN_FP64
        systems = [binding.System(synth.serving_system(j["seed"]), precision=prec, max_walkers=1) for j in stream]
        srv = binding.Server(budget_gb << 30, n_slots=slots, chunk_walkers=chunk)
        # calibration: all jobs of a prefix at once -> walker-E_loc/s and jobs/s capacity
        ncal = min(len(stream), 24)
        t0 = time.perf_counter()
        ids = [srv.submit(systems[k], binding.PN_JOB_SWEEP if stream[k]["kind"] == "sweep" else binding.PN_JOB_ELOC,
                          stream[k]["W"], n_steps=stream[k]["n_steps"], sigma=0.2, seed=stream[k]["seed"])
               for k in range(ncal)]
        for i in ids:
            srv.poll(i, timeout_us=-1)
        cap_jobs = ncal / (time.perf_counter() - t0)
        if prec_name == "mixed" and cap_mixed is None:
            cap_mixed = cap_jobs
        if rate is None:  # every server sees the arrival rate set by the first calibration
            rate = load * cap_jobs
        this_rate = run_load * cap_mixed if (prec_name == "mixed" and run_load != load) else rate
        # open-loop Poisson arrivals at `rate`
        arr = np.cumsum(np.random.default_rng(seed).exponential(1.0 / this_rate, size=n_jobs))
        ids = []
        t0 = time.perf_counter()
        for k, j in enumerate(stream):
            while time.perf_counter() - t0 < arr[k]:
                time.sleep(min(0.0005, max(0.0, arr[k] - (time.perf_counter() - t0))))
            ids.append(srv.submit(systems[k], binding.PN_JOB_SWEEP if j["kind"] == "sweep" else binding.PN_JOB_ELOC,
                                  j["W"], n_steps=j["n_steps"], sigma=0.2, seed=j["seed"]))
        lat = []
        walkers = 0
        for k, i in enumerate(ids):
            res = srv.poll(i, timeout_us=-1)
            lat.append(res.queue_ms + res.run_ms)
            walkers += res.W
        span = time.perf_counter() - t0
        srv.close()
        lat = np.array(lat)
        rec = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
               "walker_eloc_per_s": walkers / span, "jobs_per_s": n_jobs / span,
               "calibrated_capacity_jobs_per_s": cap_jobs}
        if run_load == load and prec_name not in out:
            out[prec_name] = rec
        else:
            out.setdefault("load_sweep", []).append(dict(rec, load=run_load, arrival_rate_jobs_per_s=this_rate))
        for s_ in systems:
            s_.close()
    out["arrival_rate_jobs_per_s"] = rate
    out["jobs"] = n_jobs
    out["stream"] = (f"{n_jobs} Poisson jobs, seeded neutral molecules of 1-6 nuclei, Z 1-10, 2-30 electrons, "
                     f"1-32 determinants, 256-{wmax} walkers log-uniform, E_loc or 10-step sweep 50/50; "
                     f"{slots} slots, load {load} of calibrated mixed capacity")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-walkers", type=int, default=32)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-langevin", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=60)
    ap.add_argument("--serve-only", action="store_true")
    ap.add_argument("--serve-load", type=float, default=0.7, help="offered load, fraction of calibrated mixed capacity")
    ap.add_argument("--serve-precisions", default="mixed,fp64")
    ap.add_argument("--serve-sweep", default="", help="further loads for the mixed server, e.g. 0.5,0.9")
    ap.add_argument("--sampler", type=int, default=None,
                    help="PN_OPT_FUSED_SAMPLER for the timed mixed path (library default if absent)")
    ap.add_argument("--case", choices=["sampler", "jet_tc", "langevin", "drift_n2", "configs"], default=None,
                    help="run one small kernel case (for ncu captures) and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_1909_08423_gb300 import binding, synth

    if args.case == "configs":  # the H10 and N2-shaped configurations at full size
        torch.cuda.set_device(0)
        print(json.dumps(run_configs()), flush=True)
        return
    if args.case == "drift_n2":  # reverse-mode drift of 2048 N2-shaped walkers (inputs larger than L2)
        torch.cuda.set_device(0)
        sysd = synth.n2()
        W = 2048
        s = binding.System(sysd, precision=binding.PN_MIXED, max_walkers=W)
        r = torch.empty(W, s.N, 3, dtype=torch.float64, device="cuda")
        s.init_walkers(r, 1)
        lp = torch.empty(W, dtype=torch.float64, device="cuda")
        g = torch.empty_like(r)
        for _ in range(2):
            s.eval_drift(r, g, lp)
        s.device_status()
        print("case ok", flush=True)
        return
    if args.case:
        torch.cuda.set_device(0)
        sysd = synth.be()
        s = binding.System(sysd, precision=binding.PN_MIXED, max_walkers=W_PER_RANK)
        r = torch.empty(W_PER_RANK, s.N, 3, dtype=torch.float64, device="cuda")
        s.init_walkers(r, 1)
        if args.sampler is not None:
            s.set_option(binding.PN_OPT_FUSED_SAMPLER, args.sampler)
        if args.case == "sampler":  # 5 Metropolis steps of the Be workload
            lp = torch.empty(W_PER_RANK, dtype=torch.float64, device="cuda")
            sg = torch.empty_like(lp)
            s.eval_logpsi(r, lp, sg)
            s.metropolis_step(r, lp, 5, SIGMA, 3, 0)
        elif args.case == "langevin":  # initial drift + 3 Langevin steps of the Be workload
            lp = torch.empty(W_PER_RANK, dtype=torch.float64, device="cuda")
            g = torch.empty_like(r)
            s.eval_drift(r, g, lp)
            s.langevin_step(r, lp, g, 3, 0.1, 3, 0)
        else:  # one local-energy pass with every layer group on tcgen05
            s.set_option(binding.PN_OPT_TENSOR_CORES, 7)
            E = torch.empty(W_PER_RANK, dtype=torch.float64, device="cuda")
            s.eval_local_energy(r, E)
        s.device_status()
        print("case ok", flush=True)
        return

    if args.serve_only:
        torch.cuda.set_device(0)
        sweep = tuple(float(x) for x in args.serve_sweep.split(",") if x)
        print(json.dumps({"serve": run_serving(args.serve_jobs, load=args.serve_load,
                                               precisions=tuple(args.serve_precisions.split(",")), sweep=sweep)}),
              flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = binding.load()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sysd = synth.WORKLOADS[WORKLOAD]["make"]()
    W = W_PER_RANK
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def make_state(precision):
        s = binding.System(sysd, precision=precision, max_walkers=W)
        if args.sampler is not None and precision == binding.PN_MIXED:
            s.set_option(binding.PN_OPT_FUSED_SAMPLER, args.sampler)
        r = torch.empty(W, s.N, 3, dtype=torch.float64, device=dev)
        s.init_walkers(r, 1000 + rank)
        lp = torch.empty(W, dtype=torch.float64, device=dev)
        sg = torch.empty_like(lp)
        s.eval_logpsi(r, lp, sg)
        st = dict(s=s, r=r, lp=lp, E=torch.empty_like(lp), Ec=torch.empty_like(lp), cot=torch.empty_like(lp),
                  g=torch.empty(s.n_params, dtype=torch.float64, device=dev),
                  nacc=torch.zeros(1, dtype=torch.int64, device=dev), k=0)
        return st

    def step(st):
        s = st["s"]
        s.metropolis_step(st["r"], st["lp"], N_METROPOLIS, SIGMA, 7 + rank, st["k"] * N_METROPOLIS, st["nacc"])
        s.eval_local_energy(st["r"], st["E"])
        binding.clip_local_energy(st["E"], st["Ec"], st["cot"])
        s.grad_logpsi(st["r"], st["cot"], st["g"])
        st["k"] += 1

    def timed(st, steps, warmup, prof_kernel=None):
        for _ in range(warmup):
            step(st)
        barrier()
        if prof_kernel:
            lib.pn_profile_kernel(prof_kernel.encode())
        n0 = lib.pn_launch_count()
        times = []
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            step(st)
            b.record()
            times.append((a, b))
        barrier()
        launches = lib.pn_launch_count() - n0
        ms = sum(a.elapsed_time(b) for a, b in times) / steps
        kern = None
        if prof_kernel:
            cnt = C_int64()
            tot = C_double()
            binding.check(lib.pn_profile_read(ctypes.byref(cnt), ctypes.byref(tot)))
            lib.pn_profile_kernel(None)
            kern = (cnt.value, tot.value)
        return ms, launches, kern

    import ctypes
    C_int64, C_double = ctypes.c_int64, ctypes.c_double
    lib.pn_launch_count.restype = ctypes.c_ulonglong
    lib.pn_profile_kernel.argtypes = [ctypes.c_char_p]
    lib.pn_profile_read.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]

    mixed = make_state(binding.PN_MIXED)
    # find the dominant kernel class of the step (one profiled step each)
    for _ in range(max(1, args.warmup)):
        step(mixed)
    candidates = ["k_linear", "k_filter", "k_message", "k_slater", "k_orbitals", "k_combine", "k_features",
                  "k_ssp_jet", "k_wgrad", "k_slater_bwd", "k_propose", "k_accept", "k_geometry",
                  "k_metropolis_warp", "k_metropolis_fused", "k_metropolis_tc", "k_linear_tc"]
    share = {}
    for kname in candidates:
        lib.pn_profile_kernel(kname.encode())
        step(mixed)
        torch.cuda.synchronize()
        cnt, tot = C_int64(), C_double()
        binding.check(lib.pn_profile_read(ctypes.byref(cnt), ctypes.byref(tot)))
        share[kname] = (cnt.value, tot.value)
    lib.pn_profile_kernel(None)
    dom = max(share, key=lambda k: share[k][1])

    # nvidia-smi samples of the timed region: PN_CLOCK_LOG names the file to
    # keep them in (rank appended), else a temporary file
    clk_path = os.environ.get("PN_CLOCK_LOG")
    clk_path = f"{clk_path}.rank{rank}" if clk_path else os.path.join(tempfile.gettempdir(), f"pn_clocks_{rank}.csv")
    sampler = _clock_sampler(clk_path)
    ms, launches, kern = timed(mixed, args.steps, 0, prof_kernel=dom)
    if sampler:
        sampler.terminate()
        sampler.wait()
    clocks = _clock_summary(clk_path, local, getattr(sampler, "skip", 0))
    t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = W * world / (ms_max / 1e3)
    acc_rate = float(mixed["nacc"].item()) / (W * N_METROPOLIS)

    # FP64 path, same step (fewer steps: it is the slow comparator)
    f64 = make_state(binding.PN_FP64)
    ms64, _, _ = timed(f64, args.fp64_steps, 1)
    e64 = f64["E"].clone()

    # accuracy of the mixed path on the same sampled walkers
    mixed_err = None
    E_m = torch.empty_like(mixed["E"])
    E_d = torch.empty_like(mixed["E"])
    mixed["s"].eval_local_energy(mixed["r"], E_m)
    f64_check = binding.System(sysd, precision=binding.PN_FP64, max_walkers=W)
    f64_check.eval_local_energy(mixed["r"], E_d)
    torch.cuda.synchronize()
    err = (E_m - E_d).abs().cpu().numpy()
    mixed_err = {"max": float(err.max()), "p999": float(np.quantile(err, 0.999)), "mean": float(err.mean())}

    # end to end through the C ABI with host buffers in pinned (page-locked)
    # memory; every call copies its inputs in and its results out inside the
    # timed region
    e2e = None
    if not args.no_e2e:
        s = mixed["s"]

        def pinned(shape, dtype=torch.float64):
            return torch.zeros(shape, dtype=dtype).pin_memory().numpy()

        rh = pinned(tuple(mixed["r"].shape))
        rh[...] = mixed["r"].cpu().numpy()
        lph = pinned((W,))
        lph[...] = mixed["lp"].cpu().numpy()
        Eh = pinned((W,))
        Ech = pinned((W,))
        coth = pinned((W,))
        gh = pinned((s.n_params,))
        nah = pinned((1,), torch.int64)

        def host_step(k):
            s.metropolis_step(rh, lph, N_METROPOLIS, SIGMA, 11 + rank, k * N_METROPOLIS, nah)
            s.eval_local_energy(rh, Eh)
            binding.clip_local_energy(Eh, Ech, coth)
            s.grad_logpsi(rh, coth, gh)

        host_step(0)
        torch.cuda.synchronize()
        n_e2e = max(1, args.steps)
        t0 = time.perf_counter()
        for k in range(n_e2e):
            host_step(1 + k)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / n_e2e
        rb, lb = rh.nbytes, lph.nbytes
        h2d = rb + lb + rb + W * 8 + rb + W * 8
        d2h = rb + lb + 8 + W * 8 + 2 * W * 8 + gh.nbytes
        e2e = {"value": W * world / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": dt * 1e3}

    peaks, peak_src = _peaks()
    roof = None
    fl = algorithmic_flops(sysd, dom, "value")
    if kern and kern[0] > 0:
        # per step: value-pass launches dominate (Metropolis); count the
        # algorithmic work of all timed launches of this class in the step
        per_step_flops = None
        if dom in ("k_filter", "k_linear", "k_message", "k_slater"):
            per_step_flops = W * (N_METROPOLIS * algorithmic_flops(sysd, dom, "value") +
                                  algorithmic_flops(sysd, dom, "jet"))
        elif dom in ("k_metropolis_warp", "k_metropolis_fused", "k_metropolis_tc"):
            per_step_flops = W * N_METROPOLIS * algorithmic_flops(sysd, dom, "value")
        kern_ms_per_step = kern[1] / args.steps
        if per_step_flops:
            achieved = per_step_flops / (kern_ms_per_step / 1e3) / 1e12
            # FP32 CUDA-core peak: 152 SMs x 128 lanes x 2 flop x 2.07 GHz
            fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
            roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp32_peak, "traffic": None,
                    "launches_per_step": kern[0] / args.steps, "kernel_ms_per_step": kern_ms_per_step,
                    "peak_source": "fp32 CUDA-core nominal from unit counts and max clock",
                    "flops_per_step": per_step_flops,
                    "note": "algorithmic float32 network FLOPs of the launches timed; the sampler also "
                            "runs float64 determinants and log-sums"}
            if dom == "k_metropolis_tc":
                # DRAM bytes of one launch over these 4096 walkers, from an ncu
                # capture (dram__bytes_read.sum + dram__bytes_write.sum, 5-step
                # launch): positions, log-amplitudes and the first read of the
                # weights; it does not grow with the step count (the weights
                # stay in L2, the walker state in shared memory)
                roof["traffic"] = 1.13e6
                roof["traffic_note"] = ("ncu, one k_metropolis_tc launch on the same 4096 walkers (5 steps); "
                                        "independent of the step count")
                ex = tc_sampler_executed_flops(sysd, W) * N_METROPOLIS
                ex_tf = ex / (kern_ms_per_step / 1e3) / 1e12
                bf16 = peaks.get("bf16_tflops", 1900.0)
                roof["tensor_view"] = {
                    "executed_tflops": ex_tf, "peak": bf16, "frac": ex_tf / bf16, "unit": "TFLOP/s",
                    "note": "bf16 tcgen05 work actually issued (six piece products per float32 product, "
                            "128-row tiles incl. padding) against the bf16 peak (" + peak_src + ")"}
        else:
            roof = {"bound": "alu", "kernel": dom, "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None,
                    "traffic": None, "kernel_ms_per_step": kern_ms_per_step}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"Be atom (Z=4, 4 e, 4 dets, 4s2p, D=64 L=3 K=32), {W} walkers/GPU; step = "
                                   f"{N_METROPOLIS} Metropolis steps (sigma {SIGMA}) + E_loc + clip + grad ln|psi|",
                       "walkers_per_gpu": W, "precision": "mixed (float32 network, float64 orbitals/dets/sums)",
                       "l2": "flushed (256 MB write) between timed steps",
                       "parallelism": f"replicas x{world}"},
            "fp64": {"value": W * world / (ms64 / 1e3), "ms_per_step": ms64, "steps": args.fp64_steps},
            "mixed_vs_fp64_eloc_err_ha": mixed_err,
            "accept_rate": acc_rate,
            "kernel_share": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(share.items(), key=lambda x: -x[1][1])},
            "roofline": roof, "peaks_source": peak_src, "gpu_launches": int(launches),
            "clocks": clocks, "e2e": e2e}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    if rank == 0 and not args.no_langevin:
        line["langevin"] = run_langevin(sysd, W)
        line["line_scan"] = run_line_scan()
        line["vmc_train"] = run_vmc_train(sysd)
        line["ablation"] = run_ablation(W)
    if rank == 0 and args.serve_jobs > 0:
        line["serve"] = run_serving(args.serve_jobs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
