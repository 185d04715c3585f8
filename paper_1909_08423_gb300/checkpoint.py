"""Checkpoint and resume of sampling and training state.

The random numbers of every sampler step come from Philox4x32-10 keyed by
(seed, walker, step), so a Markov chain's whole random state is its seed
and the index of its next step.  A checkpoint therefore holds the walker
positions, ln|psi| (and the drift for the Langevin sampler), the seed and
the next step index -- plus, for training, the parameters, the AdamW
moments and counters and the pool of sampled configurations -- and a run
resumed from it continues bit for bit as the uninterrupted run would have.

Files are numpy .npz archives (arrays stored exactly, float64); the
metadata is a JSON string inside the archive.  Nothing here computes any
part of the method.
"""

from __future__ import annotations

import json

import numpy as np

FORMAT = "paulinet-gb300-checkpoint-1"


def _np(x):
    if x is None:
        return None
    if hasattr(x, "detach"):
        return x.detach().cpu().numpy()
    return np.asarray(x)


def save(path, arrays, meta):
    """Write tensors/arrays (dict name -> array or None) and JSON-able meta."""
    out = {k: _np(v) for k, v in arrays.items() if v is not None}
    out["__meta__"] = np.frombuffer(json.dumps(dict(meta, format=FORMAT)).encode(), dtype=np.uint8)
    with open(path, "wb") as f:
        np.savez(f, **out)


def load(path, device=None):
    """(arrays, meta); arrays become torch tensors on `device` if given."""
    with np.load(path, allow_pickle=False) as z:
        meta = json.loads(bytes(z["__meta__"]).decode())
        if meta.get("format") != FORMAT:
            raise ValueError(f"{path}: not a checkpoint of this library ({meta.get('format')})")
        arrays = {k: z[k].copy() for k in z.files if k != "__meta__"}
    if device is not None:
        import torch
        arrays = {k: torch.as_tensor(v, device=device) for k, v in arrays.items()}
    return arrays, meta


def save_chain(path, r, logabs, seed, next_step, drift=None, params=None):
    """A set of Markov chains: positions [W][N][3], ln|psi| [W], the seed
    and the index of the next step (and the Langevin drift, parameters)."""
    save(path, {"r": r, "logabs": logabs, "drift": drift, "params": params},
         {"kind": "chain", "seed": int(seed), "next_step": int(next_step)})


def load_chain(path, device="cuda"):
    a, m = load(path, device)
    if m.get("kind") != "chain":
        raise ValueError(f"{path}: holds {m.get('kind')}, not chains")
    return dict(r=a["r"].contiguous(), logabs=a["logabs"].contiguous(), drift=a.get("drift"),
                params=a.get("params"), seed=m["seed"], next_step=m["next_step"])
