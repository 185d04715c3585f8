"""The paper's hyperparameter table (Methods; `golden/hyperparameters.txt`)
against the defaults and the network structure the code uses: the VMC
trainer's optimisation and sampling schedule, the clipping window of the
library and of the oracle, the Langevin acceptance target of the bench, and
the number of layers of every network part in the parameter layout."""

import inspect
import os
import sys

from paper_1909_08423_gb300 import binding, synth
from paper_1909_08423_gb300.vmc import VMCTrainer
from oracle import clip as oclip

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "hyperparameters.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _defaults(fn):
    return {k: p.default for k, p in inspect.signature(fn).parameters.items() if p.default is not p.empty}


def test_training_schedule_defaults():
    g = _golden()
    d = _defaults(VMCTrainer.__init__)
    assert d["lr"] == g["learning_rate"]
    assert d["batch"] == g["batch_size"]
    assert d["walkers"] == g["walkers"]
    assert d["t0"] == g["lr_decay_t0"]
    assert d["q"] == g["clipping_window_q"]
    assert d["resample_period"] == g["resampling_period"]
    assert d["n_discard"] == g["discarded_sampling_steps"]
    assert d["n_decorr"] == g["decorrelation_sampling_steps"]


def test_clipping_window_defaults():
    q = _golden()["clipping_window_q"]
    assert _defaults(binding.clip_local_energy)["q"] == q
    assert _defaults(oclip.clip_local_energy)["q"] == q


def test_langevin_acceptance_target():
    sys.path.insert(0, os.path.dirname(HERE))
    import bench
    assert _defaults(bench.run_langevin)["target"] == _golden()["target_acceptance"]


def test_network_layer_counts():
    g = _golden()
    L = int(g["interaction_layers"])
    names = [n for n, _ in synth.param_shapes(128, 64, 32, L, 2, 8)]
    weights = lambda prefix: [n for n in names if n.startswith(prefix) and n.split(".")[-1].startswith("W")]
    assert len(weights("eta.")) == g["eta_layers"]
    assert len(weights("kappa.")) == g["kappa_layers"]
    for n in range(L):
        assert len(weights(f"h{n}.")) == g["h_layers"]
        for c in ("same", "anti", "nuc"):
            assert len(weights(f"w{n}.{c}.")) == g["w_layers"]
            assert len(weights(f"g{n}.{c}.")) == g["g_layers"]
    assert not any(n.startswith(f"h{L}.") for n in names)
    # the Be workload uses the paper's layer count and feature dimension
    be = synth.be()
    assert be["L"] == L and be["K"] == g["dim_e"]
