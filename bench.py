"""Benchmark: walker local energies per second on one GB300 (per rank).

One step = one pass of the whole hot path over the N2-shaped diatomic
(seeded synthetic: two Z=7 nuclei 2.068 bohr apart, 7 up 7 down electrons,
32 determinants, 4s4p2d Cartesian Gaussians per atom, D=128, Zd=64, K=32,
L=4; 16384 walkers in workspace chunks of 4096): one Metropolis step of all
walkers (Gaussian all-electron proposal, sigma = 0.2 bohr), local energies
of all walkers (forward Laplacian jet, with the mixed path's local-energy
guard), clipping, and the hand-written backward of ln|psi| for the VMC
loss gradient (value pass recomputed per memory-budgeted chunk).
value = walkers x ranks / step time.  The headline runs the mixed path; the
same step is also timed on the plain FP64 path, and the Be-atom step (4096
walkers, 100 Metropolis steps + E_loc + clip + grad) and the H10 chain
(8192 walkers, E_loc + clip + grad) are reported beside it.

--impl reference times the CPU oracle (the plain FP64 definition) on the
host cores on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "n2"
W_PER_RANK = 16384
CHUNK = 4096
N_METROPOLIS = 1
SIGMA = 0.2
METRIC = "walker local energies/s"
UNIT = "walkers/s"
WORKLOAD_DESC = ("N2-shaped diatomic (two Z=7 at 2.068 bohr, 14 e, 32 dets, 4s4p2d/atom, D=128 Zd=64 K=32 L=4), "
                 "{W} walkers/GPU in chunks of {C}; step = 1 Metropolis step (sigma 0.2) + E_loc + clip + grad ln|psi|")

# Kernel classes of the step and the unit that bounds each: "fp32" CUDA-core
# float32 FMA, "fp64" float64 FMA, "tensor" tcgen05 (bf16 pieces), "hbm"
# (the work the library reports for it is bytes).
KERNEL_UNIT = {
    "k_linear": "fp32", "k_linear_bt": "fp32", "k_filter": "fp32", "k_filter_tile": "fp32",
    "k_metropolis_warp": "fp32", "k_metropolis_fused": "fp32", "k_metropolis_tc": "tensor",
    "k_linear_tc": "tensor", "k_slater": "fp64", "k_message": "hbm", "k_linear_f64": "fp64",
    "k_filter_value": "fp32", "k_filter_f64": "fp64", "k_linear_f32x2": "fp32",
}
KERNEL_CLASSES = ["k_linear", "k_linear_f64", "k_linear_f32x2", "k_linear_bt", "k_linear_tc", "k_filter", "k_filter_value", "k_filter_f64",
                  "k_message", "k_message_f64", "k_slater", "k_orbitals", "k_perturb",
                  "k_combine", "k_features", "k_ssp_jet", "k_sum_electrons", "k_init_x", "k_geometry", "k_wgrad",
                  "k_slater_bwd", "k_filter_bwd", "k_filter_bwd_dist", "k_filter_tape", "k_msg_bwd_w",
                  "k_msg_bwd_h", "k_mul_sigmoid", "k_ssp_copy", "k_outer_row", "k_bcast_add", "k_message_value",
                  "k_metropolis_warp", "k_metropolis_fused", "k_metropolis_tc", "k_propose", "k_accept", "k_clip",
                  "k_guard_flag", "k_guard_gather", "k_guard_scatter", "k_filter_tile_jet", "k_filter_tile_value",
                  "k_filter_tile_bwd", "k_filter_tile_dist"]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _sha16(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def _traffic_per_work(kernel):
    """DRAM bytes per unit of algorithmic work of a kernel class, from the
    committed ncu capture summarised in profiles/traffic.json -- or None with
    the reason, also when the kernel's source file changed since the capture
    (its sha256 is recorded with the figures)."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None, "no committed ncu capture"
    rec = d.get(kernel)
    if not rec:
        return None, f"no committed ncu capture of {kernel}"
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src) or _sha16(src) != rec["source_sha16"]:
        return None, f"{rec['source']} changed since the capture"
    return rec["dram_bytes_per_work"], rec["note"]


def _roofline(kernel, count, ms, work, peaks, peak_src, fp32, fp64, nbytes=0.0):
    """Roofline record of one kernel class: achieved = algorithmic work of its
    launches / their summed CUDA-event time, against the peak of the unit
    that bounds it.  Where the launch sites also report the bytes the
    launches must move through HBM (the linear maps), both fractions are
    formed and the larger -- the binding constraint -- is the record's
    bound; the other is kept as `other_view`."""
    unit = KERNEL_UNIT.get(kernel)
    rec = {"kernel": kernel, "launches": count, "kernel_ms": ms, "work": work, "bytes": nbytes or None}
    if not unit or work <= 0 or ms <= 0:
        rec.update(bound=None, achieved=None, peak=None, frac=None, unit=None,
                   note="the library reports no algorithmic work for this class")
        return rec
    sec = ms / 1e3
    views = []
    if unit == "hbm":
        views.append(("hbm", work / sec / 1e9, peaks["hbm_gbs"], "GB/s",
                      f"hbm_gbs of MEASURED_PEAKS.json ({peak_src}); work = bytes that must cross HBM"))
    else:
        if unit == "tensor":
            views.append(("tensor", work / sec / 1e12, peaks["bf16_tflops"], "TFLOP/s",
                          f"bf16_tflops (burst) of MEASURED_PEAKS.json ({peak_src}); work counts each float32 product "
                          "once, the kernel issues six bf16 piece products for it"))
        else:
            views.append(("alu", work / sec / 1e12, fp32 if unit == "fp32" else fp64, "TFLOP/s",
                          f"{unit} FMA issue rate measured by pn_measure_peak on this GPU"))
        if nbytes > 0:
            views.append(("hbm", nbytes / sec / 1e9, peaks["hbm_gbs"], "GB/s",
                          f"hbm_gbs of MEASURED_PEAKS.json ({peak_src}); bytes = inputs read and outputs written once"))
    views.sort(key=lambda v: -v[1] / v[2])
    b, ach, peak, u, src = views[0]
    rec.update(bound=b, achieved=ach, peak=peak, unit=u, frac=ach / peak, peak_source=src,
               work_per_launch=(nbytes if b == "hbm" and unit != "hbm" else work) / max(count, 1))
    if len(views) > 1:
        b2, a2, p2, u2, s2 = views[1]
        rec["other_view"] = {"bound": b2, "achieved": a2, "peak": p2, "unit": u2, "frac": a2 / p2, "peak_source": s2}
    return rec


# ---------------------------------------------------------------- oracle
# The CPU oracle on a pool of processes, one per host core (spawned, so
# that no worker inherits a CUDA context), each on its own walkers with one
# torch thread.

_ORACLE = {}


def _oracle_of(name):
    if name not in _ORACLE:
        import torch
        torch.set_num_threads(1)
        from oracle.ansatz import Oracle
        from paper_1909_08423_gb300 import synth
        _ORACLE[name] = Oracle(synth.WORKLOADS[name]["make"]())
    return _ORACLE[name]


def _oracle_move_and_eloc(job):
    """One walker chunk: n_metro Metropolis steps, then E_loc."""
    from oracle import sampling
    name, r, walker0, n_metro, seed, step0 = job
    o = _oracle_of(name)
    lp, _ = o.eval_logpsi(r)
    if n_metro:
        r, lp, _ = sampling.metropolis(o, r, lp, n_metro, SIGMA, seed=seed, step0=step0, walker0=walker0)
    E, _, _ = o.local_energy(r)
    return r, E


def _oracle_grad(job):
    name, r, cot = job
    return _oracle_of(name).grad_logpsi(r, cot)


class OraclePool:
    """The oracle's VMC step on a sample of walkers over the host cores."""

    def __init__(self, name, cores=None):
        import multiprocessing as mp
        self.name = name
        self.cores = cores or len(os.sched_getaffinity(0))
        self.pool = mp.get_context("spawn").Pool(self.cores)

    def step(self, r, k, n_metro):
        from oracle import clip as oclip
        parts = np.array_split(np.arange(len(r)), min(self.cores, len(r)))
        jobs = [(self.name, r[p], int(p[0]), n_metro, 1, k * max(n_metro, 1)) for p in parts]
        res = self.pool.map(_oracle_move_and_eloc, jobs)
        r = np.concatenate([x[0] for x in res])
        E = np.concatenate([x[1] for x in res])
        cot = oclip.loss_cotangent(oclip.clip_local_energy(E))
        self.pool.map(_oracle_grad, [(self.name, r[p], cot[p]) for p in parts])
        return r

    def close(self):
        self.pool.close()
        self.pool.join()


def _oracle_walkers(name, W, seed=1):
    from oracle import sampling
    from paper_1909_08423_gb300 import synth
    return sampling.init_walkers(synth.WORKLOADS[name]["make"](), W, seed)


# walkers per host core in the oracle's timed samples (the oracle evaluates a
# process's walkers as one batch, so a few per core keep its fixed costs
# per call from dominating; the reference arm and cpu_baseline use the same)
ORACLE_PER_CORE = 8


def run_reference(args):
    """The CPU oracle, as it stands, on a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pool = OraclePool(WORKLOAD)
    Ws = args.ref_walkers or ORACLE_PER_CORE * pool.cores
    r = _oracle_walkers(WORKLOAD, Ws)
    for k in range(args.warmup):
        r = pool.step(r, k, N_METROPOLIS)
    t0 = time.perf_counter()
    for k in range(args.steps):
        r = pool.step(r, args.warmup + k, N_METROPOLIS)
    dt = (time.perf_counter() - t0) / args.steps
    pool.close()
    v = Ws / dt
    sample = (f"{Ws} walkers per step of the {W_PER_RANK}-walker N2-shaped workload (the same step: "
              f"{N_METROPOLIS} Metropolis step + E_loc + clip + grad), over {pool.cores} processes of one thread")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD_DESC.format(W=W_PER_RANK, C=CHUNK) + f"; sampled: {Ws} walkers per step",
                       "walkers": Ws},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(n_per_core=ORACLE_PER_CORE, cores=None):
    """Oracle timing on the host cores for the cpu_baseline key: one VMC step
    of the headline workload on a sample of walkers (n_per_core per core),
    after one untimed step of one walker per core (the workers' set-up)."""
    pool = OraclePool(WORKLOAD, cores)
    pool.step(_oracle_walkers(WORKLOAD, pool.cores), 0, N_METROPOLIS)
    Ws = n_per_core * pool.cores
    r = _oracle_walkers(WORKLOAD, Ws)
    t0 = time.perf_counter()
    pool.step(r, 1, N_METROPOLIS)
    dt = time.perf_counter() - t0
    pool.close()
    return {"value": Ws / dt, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"{Ws} walkers of the N2-shaped workload, one step ({N_METROPOLIS} Metropolis step + E_loc + "
                      f"clip + grad), {pool.cores} process{'es' if pool.cores > 1 else ''} of one thread, after one "
                      "untimed warm-up step",
            "seconds": dt}


def cpu_baseline_line(n_per_core=ORACLE_PER_CORE):
    """The cpu_baseline key: the oracle on all host cores, and the same
    per-core sample on one core (how far the pool scales over the cores)."""
    line = cpu_baseline_sample(n_per_core)
    one = cpu_baseline_sample(n_per_core, cores=1)
    line["one_core"] = {"value": one["value"], "unit": UNIT, "sample": one["sample"], "seconds": one["seconds"]}
    return line


def run_be_step(W=4096, steps=3, n_metro=100):
    """The Be-atom step: 100 Metropolis steps + E_loc + clip + grad, mixed."""
    import torch
    from paper_1909_08423_gb300 import binding, synth
    s = binding.System(synth.be(), precision=binding.PN_MIXED, max_walkers=W)
    r = torch.empty(W, s.N, 3, dtype=torch.float64, device="cuda")
    s.init_walkers(r, 5)
    lp = torch.empty(W, dtype=torch.float64, device="cuda")
    sg = torch.empty_like(lp)
    s.eval_logpsi(r, lp, sg)
    E, Ec, cot = torch.empty_like(lp), torch.empty_like(lp), torch.empty_like(lp)
    g = torch.empty(s.n_params, dtype=torch.float64, device="cuda")

    def step(k):
        s.metropolis_step(r, lp, n_metro, SIGMA, 5, k * n_metro)
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
    s.close()
    return {"walkers": W, "ms_per_step": ms, "walker_eloc_per_s": W / (ms / 1e3), "steps": steps,
            "step": f"{n_metro} Metropolis steps + E_loc + clip + grad, mixed, CUDA events"}


def run_h10_step(W=8192, steps=3):
    """The H10 chain: E_loc + clip + grad of 8192 walkers, mixed."""
    import torch
    from paper_1909_08423_gb300 import binding, synth
    s = binding.System(synth.h10(), precision=binding.PN_MIXED, max_walkers=W)
    r = torch.empty(W, s.N, 3, dtype=torch.float64, device="cuda")
    s.init_walkers(r, 3)
    lp = torch.empty(W, dtype=torch.float64, device="cuda")
    sg = torch.empty_like(lp)
    s.eval_logpsi(r, lp, sg)
    s.metropolis_step(r, lp, 50, SIGMA, 3, 0)
    E, Ec, cot = torch.empty_like(lp), torch.empty_like(lp), torch.empty_like(lp)
    g = torch.empty(s.n_params, dtype=torch.float64, device="cuda")

    def step():
        s.eval_local_energy(r, E)
        binding.clip_local_energy(E, Ec, cot)
        s.grad_logpsi(r, cot, g)

    step()
    s.guard_count()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ng = s.guard_count()
    s.close()
    return {"walkers": W, "ms_per_step": ms, "walker_eloc_per_s": W / (ms / 1e3), "steps": steps,
            "guard_reevaluated_per_step": ng / steps, "step": "E_loc + clip + grad, mixed, CUDA events"}


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



def run_serving(n_jobs, seed=2024, slots=4, chunk=2048, budget_gb=64, wmax=16384, load=0.6, fp64_jobs=100,
                sweep=(), guard=True, unguarded_jobs=0):
    """Poisson stream of seeded molecules through the serving loop.  The
    arrival rate is `load` times the mixed server's capacity, measured first
    by a closed-loop burst of the stream's first 48 jobs (also with one slot,
    to show what running jobs side by side gains).  A burst overstates the
    sustained capacity (about 1.4x on this stream), hence the default load.  The mixed server serves the
    whole stream; the plain FP64 server serves its first fp64_jobs jobs at the
    same arrival rate.  `sweep` lists further loads at which the mixed server
    is measured again (the latency-load curve)."""
    import torch
    from paper_1909_08423_gb300 import binding, synth
    stream = synth.serving_stream(n_jobs, seed, rate_per_s=1.0, wmax=wmax)
    kind = lambda j: binding.PN_JOB_SWEEP if j["kind"] == "sweep" else binding.PN_JOB_ELOC

    def burst(systems, idx, n_slots):
        srv = binding.Server(budget_gb << 30, n_slots=n_slots, chunk_walkers=chunk)
        t0 = time.perf_counter()
        ids = [srv.submit(systems[k], kind(stream[k]), stream[k]["W"], n_steps=stream[k]["n_steps"], sigma=0.2,
                          seed=stream[k]["seed"]) for k in idx]
        walkers = sum(srv.poll(i, timeout_us=-1).W for i in ids)
        dt = time.perf_counter() - t0
        srv.close()
        return len(idx) / dt, walkers / dt

    def spread(n_all, n):
        return [int(k) for k in np.unique(np.linspace(0, n_all - 1, min(n_all, n)).astype(int))]

    def open_loop(systems, n, rate):
        srv = binding.Server(budget_gb << 30, n_slots=slots, chunk_walkers=chunk)
        arr = np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, size=n))
        ids = []
        t0 = time.perf_counter()
        for k in range(n):
            while time.perf_counter() - t0 < arr[k]:
                time.sleep(min(0.0005, max(0.0, arr[k] - (time.perf_counter() - t0))))
            j = stream[k]
            ids.append(srv.submit(systems[k], kind(j), j["W"], n_steps=j["n_steps"], sigma=0.2, seed=j["seed"]))
        lat, walkers, over = [], 0, []
        for i in ids:
            res = srv.poll(i, timeout_us=-1)
            lat.append(res.queue_ms + res.run_ms)
            walkers += res.W
        span = time.perf_counter() - t0
        srv.close()
        lat = np.array(lat)
        return {"jobs": n, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "walker_eloc_per_s": walkers / span, "jobs_per_s": n / span, "arrival_rate_jobs_per_s": rate}

    out = {}
    cal = list(range(min(n_jobs, 48)))
    mixed_sys = [binding.System(synth.serving_system(j["seed"]), precision=binding.PN_MIXED, max_walkers=1)
                 for j in stream]
    if not guard:
        for s_ in mixed_sys:
            s_.set_option(binding.PN_OPT_GUARD, 0)
    cap_jobs, cap_walkers = burst(mixed_sys, cal, slots)
    cap1_jobs, cap1_walkers = burst(mixed_sys, cal, 1)
    rate = load * cap_jobs
    out["mixed"] = open_loop(mixed_sys, n_jobs, rate)
    out["mixed"].update(calibrated_capacity_jobs_per_s=cap_jobs, calibrated_walker_eloc_per_s=cap_walkers,
                        one_slot_capacity_jobs_per_s=cap1_jobs, one_slot_walker_eloc_per_s=cap1_walkers)
    for l_ in sweep:
        out.setdefault("load_sweep", []).append(dict(open_loop(mixed_sys, n_jobs, l_ * cap_jobs), load=l_))
    if guard and unguarded_jobs > 0:
        # the same mixed server without the local-energy guard, on a prefix
        nu = min(unguarded_jobs, n_jobs)
        for s_ in mixed_sys[:nu]:
            s_.set_option(binding.PN_OPT_GUARD, 0)
        cu, cuw = burst(mixed_sys, list(range(min(nu, 48))), slots)
        out["mixed_unguarded"] = open_loop(mixed_sys, nu, rate)
        out["mixed_unguarded"].update(calibrated_capacity_jobs_per_s=cu, calibrated_walker_eloc_per_s=cuw,
                                      note=f"the stream's first {nu} jobs without the local-energy guard, same rate")
    for s_ in mixed_sys:
        s_.close()
    if fp64_jobs > 0:
        nf = min(fp64_jobs, n_jobs)
        fcal = spread(n_jobs, 24)
        f64_sys = {k: binding.System(synth.serving_system(stream[k]["seed"]), precision=binding.PN_FP64, max_walkers=1)
                   for k in sorted(set(range(nf)) | set(fcal))}
        fcap, fcapw = burst(f64_sys, fcal, slots)
        out["fp64"] = open_loop(f64_sys, nf, rate)
        out["fp64"].update(calibrated_capacity_jobs_per_s=fcap, calibrated_walker_eloc_per_s=fcapw)
        out["fp64"]["note"] = (f"the stream's first {nf} jobs at the mixed server's arrival rate; capacity from "
                               f"a burst of {len(fcal)} jobs spread over the stream")
        for s_ in f64_sys.values():
            s_.close()
    out["arrival_rate_jobs_per_s"] = rate
    out["jobs"] = n_jobs
    out["stream"] = (f"{n_jobs} Poisson jobs, seeded neutral molecules of 1-6 nuclei, Z 1-10, 2-30 electrons, "
                     f"1-32 determinants, 256-{wmax} walkers log-uniform, E_loc or 10-step sweep 50/50; "
                     f"{slots} slots, load {load} of the mixed capacity measured on the first {len(cal)} jobs")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-walkers", type=int, default=0,
                    help="oracle walkers per step (default: ORACLE_PER_CORE per host core)")
    ap.add_argument("--walkers", type=int, default=W_PER_RANK)
    ap.add_argument("--chunk", type=int, default=CHUNK)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--burn", type=int, default=200, help="Metropolis steps before timing (walkers sampled from |psi|^2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the Be/H10 steps, Langevin, scan, training, ablation")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--serve-fp64-jobs", type=int, default=100)
    ap.add_argument("--serve-unguarded-jobs", type=int, default=0, help="also serve a prefix without the guard")
    ap.add_argument("--serve-no-guard", action="store_true")
    ap.add_argument("--serve-only", action="store_true")
    ap.add_argument("--serve-load", type=float, default=0.6, help="offered load, fraction of calibrated mixed capacity")
    ap.add_argument("--serve-sweep", default="", help="further loads for the mixed server, e.g. 0.5,0.9")
    ap.add_argument("--sampler", type=int, default=None,
                    help="PN_OPT_FUSED_SAMPLER for the timed mixed path (library default if absent)")
    ap.add_argument("--prof-kernel", default="k_linear", help="kernel class whose work --case n2_small reports")
    ap.add_argument("--case-quick", action="store_true", help="--case n2_small: only the ranged step")
    ap.add_argument("--case-walkers", type=int, default=2048,
                    help="--case n2_small: walkers (2048: one chunk whose jet filters take the pair-tile kernel)")
    ap.add_argument("--case", choices=["sampler", "jet_tc", "langevin", "drift_n2", "n2_small", "n2_step"], default=None,
                    help="run one small kernel case (for ncu captures) and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_1909_08423_gb300 import binding, synth

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
    if args.case == "n2_step":  # one headline step (16384 walkers) between cudaProfilerStart/Stop (and NVTX "pn_step")
        torch.cuda.set_device(0)
        sysd = synth.n2()
        s = binding.System(sysd, precision=binding.PN_MIXED, max_walkers=CHUNK)
        r = torch.empty(W_PER_RANK, s.N, 3, dtype=torch.float64, device="cuda")
        s.init_walkers(r, 1)
        lp = torch.empty(W_PER_RANK, dtype=torch.float64, device="cuda")
        sg = torch.empty_like(lp)
        s.eval_logpsi(r, lp, sg)
        s.metropolis_step(r, lp, args.burn, SIGMA, 999, 1 << 40)
        E, Ec, cot = torch.empty_like(lp), torch.empty_like(lp), torch.empty_like(lp)
        g = torch.empty(s.n_params, dtype=torch.float64, device="cuda")
        for k in range(2):
            if k == 1:
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_push("pn_step")
                torch.cuda.cudart().cudaProfilerStart()
            s.metropolis_step(r, lp, N_METROPOLIS, SIGMA, 7, k)
            s.eval_local_energy(r, E)
            binding.clip_local_energy(E, Ec, cot)
            s.grad_logpsi(r, cot, g)
            if k == 1:
                torch.cuda.synchronize()
                torch.cuda.cudart().cudaProfilerStop()
                torch.cuda.nvtx.range_pop()
        s.device_status()
        print("case ok", flush=True)
        return
    if args.case == "n2_small":
        # the headline step on --case-walkers N2-shaped walkers (one chunk): one step
        # between cudaProfilerStart/Stop (and in the NVTX range "pn_step")
        # with the algorithmic work of --prof-kernel's launches in it printed
        # (for an ncu capture limited to that step),
        # then every kernel class's work and time over one more step each
        torch.cuda.set_device(0)
        sysd = synth.n2()
        W = args.case_walkers
        s = binding.System(sysd, precision=binding.PN_MIXED, max_walkers=W)
        r = torch.empty(W, s.N, 3, dtype=torch.float64, device="cuda")
        s.init_walkers(r, 1)
        lp = torch.empty(W, dtype=torch.float64, device="cuda")
        sg = torch.empty_like(lp)
        s.eval_logpsi(r, lp, sg)
        s.metropolis_step(r, lp, args.burn, SIGMA, 999, 1 << 40)
        E, Ec, cot = torch.empty_like(lp), torch.empty_like(lp), torch.empty_like(lp)
        g = torch.empty(s.n_params, dtype=torch.float64, device="cuda")

        def step(k):
            s.metropolis_step(r, lp, N_METROPOLIS, SIGMA, 7, k)
            s.eval_local_energy(r, E)
            binding.clip_local_energy(E, Ec, cot)
            s.grad_logpsi(r, cot, g)

        step(0)
        torch.cuda.synchronize()
        binding.profile(args.prof_kernel)
        torch.cuda.nvtx.range_push("pn_step")
        torch.cuda.cudart().cudaProfilerStart()
        step(1)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        torch.cuda.nvtx.range_pop()
        n, ms, wk = binding.profile_read()
        binding.profile(None)
        ranged = {"kernel": args.prof_kernel, "launches": n, "ms": ms, "work": wk}
        work = {}
        if not args.case_quick:
            for kname in KERNEL_CLASSES:
                binding.profile(kname)
                step(2)
                torch.cuda.synchronize()
                n, ms, wk = binding.profile_read()
                if n:
                    work[kname] = {"launches": n, "ms": ms, "work": wk}
            binding.profile(None)
        s.device_status()
        print(json.dumps({"case": "n2_small", "walkers": W, "pn_step_range": ranged, "per_class_one_step": work}),
              flush=True)
        print("case ok", flush=True)
        return
    if args.case:
        torch.cuda.set_device(0)
        sysd = synth.be()
        s = binding.System(sysd, precision=binding.PN_MIXED, max_walkers=4096)
        r = torch.empty(4096, s.N, 3, dtype=torch.float64, device="cuda")
        s.init_walkers(r, 1)
        if args.sampler is not None:
            s.set_option(binding.PN_OPT_FUSED_SAMPLER, args.sampler)
        if args.case == "sampler":  # 5 Metropolis steps of the Be workload
            lp = torch.empty(4096, dtype=torch.float64, device="cuda")
            sg = torch.empty_like(lp)
            s.eval_logpsi(r, lp, sg)
            s.metropolis_step(r, lp, 5, SIGMA, 3, 0)
        elif args.case == "langevin":  # initial drift + 3 Langevin steps of the Be workload
            lp = torch.empty(4096, dtype=torch.float64, device="cuda")
            g = torch.empty_like(r)
            s.eval_drift(r, g, lp)
            s.langevin_step(r, lp, g, 3, 0.1, 3, 0)
        else:  # one local-energy pass with every layer group on tcgen05
            s.set_option(binding.PN_OPT_TENSOR_CORES, 7)
            E = torch.empty(4096, dtype=torch.float64, device="cuda")
            s.eval_local_energy(r, E)
        s.device_status()
        print("case ok", flush=True)
        return

    if args.serve_only:
        torch.cuda.set_device(0)
        sweep = tuple(float(x) for x in args.serve_sweep.split(",") if x)
        print(json.dumps({"serve": run_serving(args.serve_jobs, load=args.serve_load, fp64_jobs=args.serve_fp64_jobs,
                                               sweep=sweep, guard=not args.serve_no_guard,
                                               unguarded_jobs=args.serve_unguarded_jobs)}), flush=True)
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

    peaks, peak_src = _peaks()
    fp32_peak = binding.measure_peak(0)
    fp64_peak = binding.measure_peak(1)

    sysd = synth.WORKLOADS[WORKLOAD]["make"]()
    W, chunk = args.walkers, args.chunk
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def make_state(precision, burn=None):
        burn = args.burn if burn is None else burn
        s = binding.System(sysd, precision=precision, max_walkers=chunk)
        if args.sampler is not None and precision == binding.PN_MIXED:
            s.set_option(binding.PN_OPT_FUSED_SAMPLER, args.sampler)
        r = torch.empty(W, s.N, 3, dtype=torch.float64, device=dev)
        s.init_walkers(r, 1000 + rank)
        lp = torch.empty(W, dtype=torch.float64, device=dev)
        sg = torch.empty_like(lp)
        s.eval_logpsi(r, lp, sg)
        if burn:
            s.metropolis_step(r, lp, burn, SIGMA, 999 + rank, 1 << 40)  # leave the initial Gaussian cloud
        st = dict(s=s, r=r, lp=lp, E=torch.empty_like(lp), Ec=torch.empty_like(lp), cot=torch.empty_like(lp),
                  g=torch.empty(s.n_params, dtype=torch.float64, device=dev),
                  nacc=torch.zeros(1, dtype=torch.int64, device=dev), k=0)
        return st

    from paper_1909_08423_gb300 import distributed as pdist

    def step(st):
        s = st["s"]
        s.metropolis_step(st["r"], st["lp"], N_METROPOLIS, SIGMA, 7 + rank, st["k"] * N_METROPOLIS, st["nacc"])
        s.eval_local_energy(st["r"], st["E"])
        if world > 1:
            # the VMC step's exchange: the clipping window over every rank's
            # energies (all-gather), the gradient summed over ranks (all-reduce)
            Ec, cot, _ = pdist.global_clip(st["E"], binding.clip_local_energy)
            s.grad_logpsi(st["r"], cot, st["g"])
            pdist.allreduce_grad(st["g"])
        else:
            binding.clip_local_energy(st["E"], st["Ec"], st["cot"])
            s.grad_logpsi(st["r"], st["cot"], st["g"])
        st["k"] += 1

    def timed(st, steps, warmup, prof_kernel=None):
        for _ in range(warmup):
            step(st)
        barrier()
        if prof_kernel:
            binding.profile(prof_kernel)
        n0 = lib.pn_launch_count()
        times = []
        acc0 = 0
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
            kern = binding.profile_read(with_bytes=True)
            binding.profile(None)
        return ms, launches, kern

    mixed = make_state(binding.PN_MIXED)
    for _ in range(max(1, args.warmup)):
        step(mixed)
    # where the step's time goes: every kernel class timed over one step
    share = {}
    for kname in KERNEL_CLASSES:
        binding.profile(kname)
        step(mixed)
        torch.cuda.synchronize()
        n, ms_k, wk, by = binding.profile_read(with_bytes=True)
        if n:
            share[kname] = (n, ms_k, wk, by)
    binding.profile(None)
    dom = max(share, key=lambda k: share[k][1])
    mixed["s"].guard_count()

    # nvidia-smi samples of the timed region: PN_CLOCK_LOG names the file to
    # keep them in (rank appended), else a temporary file
    clk_path = os.environ.get("PN_CLOCK_LOG")
    clk_path = f"{clk_path}.rank{rank}" if clk_path else os.path.join(tempfile.gettempdir(), f"pn_clocks_{rank}.csv")
    sampler = _clock_sampler(clk_path)
    mixed["nacc"].zero_()
    ms, launches, kern = timed(mixed, args.steps, 0, prof_kernel=dom)
    if sampler:
        sampler.terminate()
        sampler.wait()
    clocks = _clock_summary(clk_path, local, getattr(sampler, "skip", 0))
    guard_n = mixed["s"].guard_count()
    t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = W * world / (ms_max / 1e3)
    acc_rate = float(mixed["nacc"].item()) / (W * N_METROPOLIS)

    roof = _roofline(dom, kern[0], kern[1], kern[2], peaks, peak_src, fp32_peak, fp64_peak, kern[3])
    roof["kernel_ms_per_step"] = kern[1] / args.steps
    tpw, tnote = _traffic_per_work(dom)
    # traffic per launch: the captured DRAM bytes per unit of the class's
    # algorithmic work, times this run's work per launch
    roof["traffic"] = tpw * kern[2] / max(kern[0], 1) if tpw is not None else None
    roof["traffic_note"] = tnote
    by_kernel = sorted((_roofline(k, v[0], v[1], v[2], peaks, peak_src, fp32_peak, fp64_peak, v[3])
                        for k, v in share.items()), key=lambda x: -x["kernel_ms"])[:8]

    # accuracy of the mixed path on the sampled walkers, against the FP64 path
    E_m = torch.empty_like(mixed["E"])
    E_d = torch.empty_like(mixed["E"])
    st_d = torch.empty(W, dtype=torch.int32, device=dev)
    mixed["s"].eval_local_energy(mixed["r"], E_m)
    g_err = mixed["s"].guard_count()
    f64_check = binding.System(sysd, precision=binding.PN_FP64, max_walkers=chunk)
    f64_check.eval_local_energy(mixed["r"], E_d, None, None, st_d)
    torch.cuda.synchronize()
    ok = (st_d == 0).cpu().numpy()
    err = (E_m - E_d).abs().cpu().numpy()[ok]
    mixed_err = {"max": float(err.max()), "p999": float(np.quantile(err, 0.999)), "mean": float(err.mean()),
                 "walkers": int(ok.sum()), "guard_reevaluated": int(g_err),
                 "note": "every walker of the timed state after the timed steps, mixed (guarded) vs float64 path"}
    f64_check.close()

    # FP64 path, same step (fewer steps: it is the slow comparator)
    f64 = make_state(binding.PN_FP64, burn=0)
    ms64, _, _ = timed(f64, args.fp64_steps, 1)
    f64["s"].close()
    del f64

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
        Eh, Ech, coth = pinned((W,)), pinned((W,)), pinned((W,))
        gh = pinned((s.n_params,))
        nah = pinned((1,), torch.int64)

        def host_step(k):
            s.metropolis_step(rh, lph, N_METROPOLIS, SIGMA, 11 + rank, k * N_METROPOLIS, nah)
            s.eval_local_energy(rh, Eh)
            if world > 1:  # the exchange runs on device copies (NCCL)
                _, cot_d, _ = pdist.global_clip(torch.from_numpy(Eh).to(dev), binding.clip_local_energy)
                coth[...] = cot_d.cpu().numpy()
                s.grad_logpsi(rh, coth, gh)
                gd = torch.from_numpy(gh).to(dev)
                pdist.allreduce_grad(gd)
                gh[...] = gd.cpu().numpy()
            else:
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
        # in: r and ln|psi| (sampler), r (E_loc), E (clip), r and cotangent (grad);
        # out: r, ln|psi|, accept count (sampler), E (E_loc), clipped E and
        # cotangent (clip), gradient
        h2d = rb + lb + rb + W * 8 + rb + W * 8
        d2h = rb + lb + 8 + W * 8 + 2 * W * 8 + gh.nbytes
        if world > 1:  # E and the gradient to the device for the exchange and back
            h2d += gh.nbytes
            d2h += gh.nbytes - W * 8
        e2e = {"value": W * world / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": dt * 1e3}

    cfg = {"workload": WORKLOAD_DESC.format(W=W, C=chunk), "walkers_per_gpu": W, "chunk": chunk,
           "precision": "mixed: float32 network (tcgen05 maps on three-piece bf16 operands), float64 "
                        "orbitals/determinants/sums/Coulomb; local-energy guard on (probe 2, tau 5e-5 Ha: flagged "
                        "walkers re-evaluated in float64 with float32-pair maps and filters)",
           "l2": "flushed (256 MB write) between timed steps; the per-chunk intermediates (~14 GB) exceed L2",
           "parallelism": (f"walkers sharded x{world}; clipping window all-gathered and gradient all-reduced "
                           "(NCCL) every step" if world > 1 else "1 GPU")}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": cfg,
            "roofline": roof, "roofline_by_kernel": by_kernel,
            "peaks": {"fp32_tflops": fp32_peak, "fp64_tflops": fp64_peak, "fp32_fp64_source": "pn_measure_peak",
                      "hbm_gbs": peaks["hbm_gbs"], "bf16_tflops": peaks["bf16_tflops"],
                      "hbm_bf16_source": f"MEASURED_PEAKS.json ({peak_src})"},
            "gpu_launches": int(launches), "clocks": clocks, "e2e": e2e,
            "fp64": {"value": W * world / (ms64 / 1e3), "ms_per_step": ms64, "steps": args.fp64_steps},
            "mixed_vs_fp64_eloc_err_ha": mixed_err,
            "guard_reevaluated_per_step": guard_n / max(args.steps, 1),
            "accept_rate": acc_rate,
            "kernel_share": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(share.items(), key=lambda x: -x[1][1])}}
    mixed["s"].close()
    del mixed
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line()
    # the single-GPU extras and the serving stream run in the one-GPU line
    # only: under torchrun they would hold every rank's GPU for one rank's work
    if rank == 0 and world == 1 and not args.no_extras:
        line["be"] = run_be_step()
        line["h10"] = run_h10_step()
        be = synth.be()
        line["langevin"] = run_langevin(be, 4096)
        line["line_scan"] = run_line_scan()
        line["vmc_train"] = run_vmc_train(be)
        line["ablation"] = run_ablation(4096)
    if rank == 0 and world == 1 and args.serve_jobs > 0:
        line["serve"] = run_serving(args.serve_jobs, load=args.serve_load, fp64_jobs=args.serve_fp64_jobs,
                                    guard=not args.serve_no_guard, unguarded_jobs=args.serve_unguarded_jobs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
