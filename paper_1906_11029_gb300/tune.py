"""Autotuner: per GPU, dimension and degree, pick the fastest kernel configuration on a short
window of layers and cache the choice.

Two levels:

* launch configuration of a tents handle (`mtp_tents_autotune`, native): persistent DAG walk
  with the occupancy limit of CTAs per SM, DAG walk with one CTA per SM, or one launch per layer;
* contraction variant within an accuracy class (here): for FP32-level accuracy the SIMT FP32
  kernels or the tensor-core 3xTF32 split; for "tf32" accuracy additionally plain TF32 tensor
  cores;
* kernel shape of the SIMT FP32 kernels (here, `mtp_tents_set_variant`): stage items over pairs
  of patch elements (variant 0), single elements (variant 1) or single (element, row) pairs on
  512 threads (variant 2): more and shorter items, faster tents when the layers hold fewer
  tents than the GPU has CTA slots; variants 3 and 4 (3D, p = 2..4) take the item shapes of 1
  and 2 with the volume term on the tcgen05 tensor cores.
Candidates are timed on the same layer window of the caller's workload.

Choices are cached in a JSON file (default ``~/.cache/paper_1906_11029_gb300/tune.json``)
keyed by GPU name, dimension, degree, accuracy class, largest patch size and the workload's
shape: its element count and the power of two nearest its average number of tents per layer
(which decides between the DAG walk and per-layer launches), so a choice timed on a small mesh
is not reused for a large one.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import MTP_EUNSUPPORTED, MTP_FP32, MTP_TF32, MTP_TF32X3, Mesh, MtpError

CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1906_11029_gb300", "tune.json")
LAUNCH_NAMES = ["dag_walk", "dag_walk_1cta", "layer_launches"]


def _key(dim, p, accuracy, max_patch, n_elems, tents_per_layer):
    import math

    import torch
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    tpl = int(round(math.log2(max(1.0, tents_per_layer))))
    return f"{name}|dim{dim}|p{p}|{accuracy}|mp{max_patch}|ne{n_elems}|tpl2^{tpl}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(dim, p, accuracy):
    """(precision, kernel shape variant) pairs that the library compiles and that meet the
    accuracy class."""
    base = [(MTP_FP32, 0), (MTP_FP32, 1), (MTP_FP32, 2)]
    if dim == 3 and 2 <= p <= 4:
        base += [(MTP_FP32, 3), (MTP_FP32, 4)]   # volume term on tcgen05 (3xTF32, FP32 accuracy)
    if accuracy == "fp32":
        return base + ([(MTP_TF32X3, 0)] if dim == 3 and p <= 4 else [])
    if accuracy == "tf32":
        return base + ([(MTP_TF32X3, 0), (MTP_TF32, 0)] if dim == 3 and p <= 4 else [])
    raise ValueError("accuracy must be 'fp32' or 'tf32'")


def autotune(dim, vertices, elements, eps, mu, p, T, lattice_values, accuracy="fp32",
             causality_factor=0.5, window=(0.1, 0.02), cache=CACHE, force=False):
    """Return (precision, launch, record) for this workload; record["variant"] is the kernel shape
    variant to set on the evolving tents handle (Tents.set_variant).  ``lattice_values``: initial
    lattice values (as for Mesh.state_from_lattice) used as the scratch state; ``window``:
    (start, length) of the timed layer window as fractions of the layer count."""
    import torch
    data = _load(cache)
    probe = Mesh(dim, vertices, elements, eps, mu, p=p, precision=MTP_FP32)
    ptents = probe.pitch(T, causality_factor)
    key = _key(dim, p, accuracy, probe.info["max_patch"], len(elements),
               ptents.info["n_tents"] / max(1, ptents.info["n_layers"]))
    if key in data and not force:
        rec = data[key]
        return rec["precision"], rec["launch"], rec
    results = []
    vals = torch.as_tensor(np.ascontiguousarray(lattice_values), device="cuda")
    for prec, variant in candidates(dim, p, accuracy):
        m = Mesh(dim, vertices, elements, eps, mu, p=p, precision=prec, n_rhs=vals.shape[0])
        t = m.pitch(T, causality_factor)
        try:
            t.set_variant(variant)
        except MtpError as e:   # e.g. a patch too large for the tcgen05 variants
            if e.code != MTP_EUNSUPPORTED:
                raise
            continue
        nl = t.info["n_layers"]
        lb = min(nl - 1, int(window[0] * nl))
        le = min(nl, max(lb + 1, lb + int(window[1] * nl)))
        st = m.state_from_lattice(vals)
        best, ms = t.autotune(st, lb, le)
        results.append({"precision": prec, "variant": variant, "launch": best, "ms": ms[best], "launch_ms": ms})
    top = min(results, key=lambda r: r["ms"])
    rec = {"precision": top["precision"], "variant": top["variant"], "launch": top["launch"],
           "launch_name": LAUNCH_NAMES[top["launch"]], "candidates": results}
    data[key] = rec
    _save(cache, data)
    return rec["precision"], rec["launch"], rec
