"""Thin ctypes binding to libpaulinet.so (argument marshalling only).

Every function takes torch tensors (CUDA tensors are passed as device
pointers on the current torch stream; CPU tensors and numpy arrays as host
pointers, which the library stages itself).  Nothing here computes any part
of the method.  Loading fails loudly if the compiled library is missing.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpaulinet.so")

PN_FP64, PN_MIXED = 0, 1
PN_JOB_ELOC, PN_JOB_SWEEP, PN_JOB_SCAN = 0, 1, 2
PN_OPT_FUSED_SAMPLER, PN_OPT_TENSOR_CORES, PN_OPT_DRIFT, PN_OPT_GUARD, PN_OPT_DET_TABLE = 1, 2, 3, 4, 5
PN_OPT_GUARD_PROBE = 6
ERRORS = {0: "PN_OK", 1: "PN_EINVAL", 2: "PN_ENOMEM", 3: "PN_EBUDGET", 4: "PN_ENOTREADY",
          5: "PN_ETIMEOUT", 6: "PN_EDEVICE", 7: "PN_ECANCELLED"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class SystemDesc(C.Structure):
    _fields_ = [
        ("M", C.c_int), ("Z", C.c_void_p), ("R", C.c_void_p),
        ("n_shells", C.c_int), ("shell_center", C.c_void_p), ("shell_l", C.c_void_p),
        ("shell_nprim", C.c_void_p), ("prim_exp", C.c_void_p), ("prim_coef", C.c_void_p),
        ("n_up", C.c_int), ("n_dn", C.c_int), ("n_orb", C.c_int),
        ("mo_coeffs", C.c_void_p),
        ("n_det", C.c_int), ("occ_up", C.c_void_p), ("occ_dn", C.c_void_p), ("ci", C.c_void_p),
        ("D", C.c_int), ("Zd", C.c_int), ("K", C.c_int), ("L", C.c_int), ("r_c", C.c_double),
        ("params", C.c_void_p), ("n_params", C.c_int64),
        ("cusp_phi0", C.c_void_p),
        ("use_cusp", C.c_int), ("use_gamma", C.c_int),
        ("precision", C.c_int), ("max_walkers", C.c_int),
        ("no_jastrow", C.c_int), ("no_backflow", C.c_int),
    ]


class ServerCfg(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("n_slots", C.c_int), ("chunk_walkers", C.c_int),
                ("debug_fail_nth", C.c_int)]


class Job(C.Structure):
    _fields_ = [("kind", C.c_int), ("W", C.c_int), ("n_steps", C.c_int), ("sigma", C.c_double),
                ("seed", C.c_uint64), ("r_init", C.c_void_p), ("eloc_out", C.c_void_p),
                ("r_out", C.c_void_p), ("scan_electron", C.c_int), ("scan_dir", C.c_double * 3),
                ("scan_t0", C.c_double), ("scan_t1", C.c_double)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("W", C.c_int), ("e_mean", C.c_double), ("e_stderr", C.c_double),
                ("accept_rate", C.c_double), ("n_nonfinite", C.c_int64), ("queue_ms", C.c_double),
                ("run_ms", C.c_double), ("dev_start_ms", C.c_double), ("dev_end_ms", C.c_double),
                ("n_guarded", C.c_int64)]


EXPORTS = {
    "pn_num_params_for": (C.c_int64, [C.c_int] * 6),
    "pn_init_system": (C.c_int, [C.POINTER(SystemDesc), C.POINTER(C.c_void_p)]),
    "pn_destroy_system": (C.c_int, [C.c_void_p]),
    "pn_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "pn_num_params": (C.c_int64, [C.c_void_p]),
    "pn_workspace_bytes": (C.c_size_t, [C.c_void_p]),
    "pn_eval_logpsi": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pn_eval_local_energy": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]),
    "pn_eval_components": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p]),
    "pn_metropolis_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double,
                                     C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p]),
    "pn_init_walkers": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_uint64, C.c_void_p]),
    "pn_adamw_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_double,
                                C.c_double, C.c_double, C.c_double, C.c_int64, C.c_void_p]),
    "pn_eval_drift": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pn_eval_line_scan": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.c_double, C.c_int,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pn_langevin_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double,
                                   C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p]),
    "pn_grad_logpsi": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_size_t,
                                 C.c_void_p]),
    "pn_clip_local_energy": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pn_server_create": (C.c_int, [C.POINTER(ServerCfg), C.POINTER(C.c_void_p)]),
    "pn_server_destroy": (C.c_int, [C.c_void_p]),
    "pn_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Job), C.POINTER(C.c_uint64)]),
    "pn_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(Result), C.c_int64]),
    "pn_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "pn_job_footprint": (C.c_size_t, [C.c_void_p, C.c_int, C.c_int]),
    "pn_set_option": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "pn_device_status": (C.c_int, [C.c_void_p]),
    "pn_guard_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "pn_test_linear_tc": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                    C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "pn_launch_count": (C.c_ulonglong, []),
    "pn_profile_kernel": (C.c_int, [C.c_char_p]),
    "pn_profile_read": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "pn_profile_work": (C.c_int, [C.POINTER(C.c_double)]),
    "pn_profile_bytes": (C.c_int, [C.POINTER(C.c_double)]),
    "pn_measure_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    "pn_last_error": (C.c_char_p, []),
}

_lib = None


def load(path=LIB_PATH):
    """Load the library once; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpaulinet.so not built at {path}; run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class PNError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def check(code):
    if code != 0:
        raise PNError(code, load().pn_last_error().decode())
    return code


# ------------------------------------------------------------------ helpers

def _ptr(x):
    """Device or host address of a torch tensor / numpy array, or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _stream(x=None):
    import torch
    if x is not None and hasattr(x, "is_cuda") and not x.is_cuda:
        return None
    if not torch.cuda.is_available():
        return None
    return torch.cuda.current_stream().cuda_stream


def _keep(arr, dtype):
    return np.ascontiguousarray(np.asarray(arr), dtype=dtype)


class System:
    """A system handle: owns the library's copy of the molecule, the network
    parameters and a workspace for max_walkers walkers."""

    def __init__(self, sysd, precision=PN_FP64, max_walkers=1024):
        lib = load()
        self.sysd = sysd
        self.N = sysd["n_up"] + sysd["n_dn"]
        self.n_orb = sysd["mo_coeffs"].shape[1]
        self.n_det = len(sysd["ci"])
        self.precision = precision
        k = {}
        k["Z"] = _keep(sysd["Z"], np.float64)
        k["R"] = _keep(sysd["R"], np.float64)
        k["sc"] = _keep(sysd["shell_center"], np.int32)
        k["sl"] = _keep(sysd["shell_l"], np.int32)
        k["sn"] = _keep(sysd["shell_nprim"], np.int32)
        k["pe"] = _keep(sysd["prim_exp"], np.float64)
        k["pc"] = _keep(sysd["prim_coef"], np.float64)
        k["mo"] = _keep(sysd["mo_coeffs"], np.float64)
        k["ou"] = _keep(sysd["occ_up"], np.int32)
        k["od"] = _keep(sysd["occ_dn"], np.int32)
        k["ci"] = _keep(sysd["ci"], np.float64)
        k["params"] = _keep(synth.flatten_params(sysd), np.float64)
        k["phi0"] = None if sysd.get("cusp_phi0") is None else _keep(sysd["cusp_phi0"], np.float64)
        self._keep = k
        d = SystemDesc()
        d.M = len(k["Z"])
        d.Z, d.R = k["Z"].ctypes.data, k["R"].ctypes.data
        d.n_shells = len(k["sc"])
        d.shell_center, d.shell_l, d.shell_nprim = k["sc"].ctypes.data, k["sl"].ctypes.data, k["sn"].ctypes.data
        d.prim_exp, d.prim_coef = k["pe"].ctypes.data, k["pc"].ctypes.data
        d.n_up, d.n_dn, d.n_orb = sysd["n_up"], sysd["n_dn"], self.n_orb
        d.mo_coeffs = k["mo"].ctypes.data
        d.n_det = self.n_det
        d.occ_up = k["ou"].ctypes.data if k["ou"].size else None
        d.occ_dn = k["od"].ctypes.data if k["od"].size else None
        d.ci = k["ci"].ctypes.data
        d.D, d.Zd, d.K, d.L, d.r_c = sysd["D"], sysd["Zd"], sysd["K"], sysd["L"], float(sysd["r_c"])
        d.params, d.n_params = k["params"].ctypes.data, len(k["params"])
        d.cusp_phi0 = None if k["phi0"] is None else k["phi0"].ctypes.data
        d.use_cusp, d.use_gamma = int(sysd["use_cusp"]), int(sysd["use_gamma"])
        d.no_jastrow, d.no_backflow = int(sysd.get("no_jastrow", 0)), int(sysd.get("no_backflow", 0))
        d.precision, d.max_walkers = precision, max_walkers
        self._desc = d
        h = C.c_void_p()
        check(lib.pn_init_system(C.byref(d), C.byref(h)))
        self.h = h
        self.n_params = lib.pn_num_params(h)

    def close(self):
        if getattr(self, "h", None):
            load().pn_destroy_system(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def workspace_bytes(self):
        return load().pn_workspace_bytes(self.h)

    def set_params(self, flat):
        check(load().pn_set_params(self.h, _ptr(flat), int(flat.numel() if hasattr(flat, "numel") else len(flat))))

    # -- evaluation ------------------------------------------------------
    def eval_logpsi(self, r, logabs, sign, status=None):
        W = r.shape[0]
        check(load().pn_eval_logpsi(self.h, _ptr(r), W, _ptr(logabs), _ptr(sign), _ptr(status), _stream(r)))

    def eval_local_energy(self, r, eloc, logabs=None, sign=None, status=None):
        W = r.shape[0]
        check(load().pn_eval_local_energy(self.h, _ptr(r), W, _ptr(eloc), _ptr(logabs), _ptr(sign),
                                          _ptr(status), _stream(r)))

    def eval_components(self, r, phi=None, J=None, f=None, ld=None):
        W = r.shape[0]
        check(load().pn_eval_components(self.h, _ptr(r), W, _ptr(phi), _ptr(J), _ptr(f), _ptr(ld), _stream(r)))

    def metropolis_step(self, r, logabs, n_steps, sigma, seed, step0, n_accept=None):
        W = r.shape[0]
        check(load().pn_metropolis_step(self.h, _ptr(r), _ptr(logabs), W, n_steps, float(sigma), int(seed),
                                        int(step0), _ptr(n_accept), _stream(r)))

    def eval_drift(self, r, drift, logabs=None):
        check(load().pn_eval_drift(self.h, _ptr(r), r.shape[0], _ptr(logabs), _ptr(drift), _stream(r)))

    def eval_line_scan(self, r0, electron, direction, t0, t1, npts, eloc, logabs=None, sign=None, status=None):
        d = np.ascontiguousarray(np.asarray(direction, dtype=np.float64).reshape(3))
        check(load().pn_eval_line_scan(self.h, _ptr(r0), int(electron), d.ctypes.data, float(t0), float(t1),
                                       int(npts), _ptr(eloc), _ptr(logabs), _ptr(sign), _ptr(status), _stream(eloc)))

    def langevin_step(self, r, logabs, drift, n_steps, tau, seed, step0, n_accept=None):
        check(load().pn_langevin_step(self.h, _ptr(r), _ptr(logabs), _ptr(drift), r.shape[0], n_steps, float(tau),
                                      int(seed), int(step0), _ptr(n_accept), _stream(r)))

    def device_status(self):
        check(load().pn_device_status(self.h))

    def set_option(self, option, value):
        check(load().pn_set_option(self.h, int(option), int(value)))

    def guard_count(self):
        """Walkers the local-energy guard re-evaluated in float64 since the
        last call (pn_guard_count)."""
        n = C.c_int64()
        check(load().pn_guard_count(self.h, C.byref(n)))
        return n.value

    def init_walkers(self, r, seed):
        check(load().pn_init_walkers(self.h, _ptr(r), r.shape[0], int(seed), _stream(r)))

    def grad_logpsi(self, r, cot, grad, mem_budget_bytes=0):
        check(load().pn_grad_logpsi(self.h, _ptr(r), r.shape[0], _ptr(cot), _ptr(grad), int(mem_budget_bytes),
                                    _stream(r)))


class Server:
    """The serving loop: submit jobs for any resident system, poll results."""

    def __init__(self, hbm_budget_bytes, n_slots=4, chunk_walkers=4096, debug_fail_nth=0):
        cfg = ServerCfg(int(hbm_budget_bytes), int(n_slots), int(chunk_walkers), int(debug_fail_nth))
        h = C.c_void_p()
        check(load().pn_server_create(C.byref(cfg), C.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, system, kind, W, n_steps=0, sigma=0.2, seed=0, r_init=None, eloc_out=None, r_out=None,
               scan_electron=0, scan_dir=(1.0, 0.0, 0.0), scan_t0=0.0, scan_t1=1.0):
        j = Job(kind, int(W), int(n_steps), float(sigma), int(seed), _ptr(r_init), _ptr(eloc_out), _ptr(r_out),
                int(scan_electron), (C.c_double * 3)(*[float(x) for x in scan_dir]), float(scan_t0), float(scan_t1))
        jid = C.c_uint64()
        check(load().pn_submit(self.h, system.h, C.byref(j), C.byref(jid)))
        self._keep[jid.value] = (r_init, eloc_out, r_out)
        return jid.value

    def poll(self, job_id, timeout_us=-1):
        """Returns a Result, or None when not ready / timed out."""
        res = Result()
        rc = load().pn_poll(self.h, C.c_uint64(job_id), C.byref(res), int(timeout_us))
        if rc in (4, 5):
            return None
        check(rc)
        self._keep.pop(job_id, None)
        return res

    def cancel(self, job_id):
        return load().pn_cancel(self.h, C.c_uint64(job_id))

    def close(self):
        if getattr(self, "h", None):
            load().pn_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def job_footprint(system, W, chunk_walkers):
    return load().pn_job_footprint(system.h, int(W), int(chunk_walkers))


def adamw_step(theta, grad, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01):
    """One AdamW step on device float64 tensors (pn_adamw_step)."""
    check(load().pn_adamw_step(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), int(theta.numel()), float(lr), float(beta1),
                               float(beta2), float(eps), float(weight_decay), int(t), _stream(theta)))


def clip_local_energy(eloc, out, cot=None, q=5.0):
    check(load().pn_clip_local_energy(_ptr(eloc), eloc.shape[0], float(q), _ptr(out), _ptr(cot), _stream(eloc)))


def measure_peak(kind):
    """TFLOP/s of the float32 (kind 0) or float64 (kind 1) FMA pipe, from the
    library's own microbenchmark kernel (pn_measure_peak)."""
    v = C.c_double()
    check(load().pn_measure_peak(int(kind), C.byref(v), _stream()))
    return v.value


def profile(name):
    """Start (name) or stop (None) CUDA-event timing of one kernel class."""
    check(load().pn_profile_kernel(name.encode() if name else None))


def profile_read(with_bytes=False):
    """(launches, total ms, algorithmic work[, algorithmic bytes]) of the
    timed kernel class."""
    n, ms, wk, by = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
    check(load().pn_profile_read(C.byref(n), C.byref(ms)))
    check(load().pn_profile_work(C.byref(wk)))
    check(load().pn_profile_bytes(C.byref(by)))
    return (n.value, ms.value, wk.value, by.value) if with_bytes else (n.value, ms.value, wk.value)


def num_params_for(D, Zd, K, L, M, n_orb):
    return load().pn_num_params_for(D, Zd, K, L, M, n_orb)
