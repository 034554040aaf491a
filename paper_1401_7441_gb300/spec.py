"""JSON system specification: the user parameters of a locreg system in one file.

A spec names the grid spacing h, the coarse grid N (or derives it from the atoms and
the largest radius), and per atom its position (bohr), locreg radius R_cut, fine-sphere
radius and number of support functions, plus the pair cutoff (or the r_a + r_b rule),
the L' margin, the fine-region mode, the precision and the seed of the synthetic
content.  Either the atoms are listed explicitly, or the spec names one of the seeded
generators with its arguments:

  {"h": 0.45, "atoms": [{"pos": [7.1, 8.0, 6.3], "r_loc": 6.0, "r_fine": 2.0,
                         "n_sf": 4}, ...],
   "pair_cutoff": 12.0, "lprime_margin": 8, "fine_mode": "union",
   "precision": "fp32", "seed": 7}

  {"generator": "scaled", "base": "atoms64", "n_atoms": 500, "seed": 77}

``load`` returns an ``inputs.Workload``; ``dump`` writes one back.
"""
from __future__ import annotations

import json
import math

import numpy as np

from . import inputs as I

PRECISIONS = ("fp64", "fp32", "bf16x")


class SpecError(ValueError):
    pass


def _require(d, key, kind):
    if key not in d:
        raise SpecError("spec: missing '%s'" % key)
    v = d[key]
    if kind is float and isinstance(v, (int, float)) and not isinstance(v, bool):
        return float(v)
    if kind is int and isinstance(v, int) and not isinstance(v, bool):
        return v
    if kind is str and isinstance(v, str):
        return v
    raise SpecError("spec: '%s' must be %s" % (key, kind.__name__))


def from_dict(d):
    """Workload from a parsed spec (see the module docstring)."""
    if not isinstance(d, dict):
        raise SpecError("spec: a JSON object is expected")
    if "generator" in d:
        g = _require(d, "generator", str)
        if g == "scaled":
            w = I.scaled(_require(d, "base", str), _require(d, "n_atoms", int), d.get("seed", 77))
        elif g in I.WORKLOADS:
            w = I.WORKLOADS[g](d["seed"]) if "seed" in d else I.WORKLOADS[g]()
        else:
            raise SpecError("spec: unknown generator '%s'" % g)
        if "precision" in d:
            w.precision = _precision(d["precision"])
        return w
    h = _require(d, "h", float)
    if not h > 0:
        raise SpecError("spec: h must be positive")
    atoms = d.get("atoms")
    if not isinstance(atoms, list) or not atoms:
        raise SpecError("spec: 'atoms' must be a non-empty list")
    pos, rl, rf, ns = [], [], [], []
    for k, a in enumerate(atoms):
        if not isinstance(a, dict):
            raise SpecError("spec: atom %d is not an object" % k)
        p = a.get("pos")
        if not (isinstance(p, list) and len(p) == 3 and all(isinstance(x, (int, float)) for x in p)):
            raise SpecError("spec: atom %d: 'pos' must be three numbers" % k)
        pos.append([float(x) for x in p])
        rl.append(_require(a, "r_loc", float))
        rf.append(_require(a, "r_fine", float))
        n = _require(a, "n_sf", int)
        if n < 0:
            raise SpecError("spec: atom %d: n_sf must be >= 0" % k)
        ns.append(n)
    pos = np.array(pos)
    if np.any(pos < 0):
        raise SpecError("spec: positions are box coordinates (>= 0)")
    if "N" in d:
        N = d["N"]
        if not (isinstance(N, list) and len(N) == 3 and all(isinstance(x, int) and x > 0 for x in N)):
            raise SpecError("spec: 'N' must be three positive integers")
        N = tuple(N)
    else:
        ext = float(np.max(pos)) + max(rl)
        n = int(math.ceil(ext / h)) + 1
        N = (n, n, n)
    pair_mode = 1 if d.get("pair_cutoff") == "sum_of_radii" else 0
    cutoff = 0.0 if pair_mode else _require(d, "pair_cutoff", float)
    seed = d.get("seed", 1)
    fine_mode = d.get("fine_mode", "union")
    if fine_mode not in ("union", "own"):
        raise SpecError("spec: fine_mode is 'union' or 'own'")
    wells = np.column_stack([pos, np.full(len(pos), 2.0), np.full(len(pos), 1.0)])
    if "wells" in d:
        wells = np.asarray(d["wells"], np.float64).reshape(-1, 5)
    return I.Workload(d.get("name", "spec"), N, h, pos, np.array(rl), np.array(rf),
                      np.array(ns, np.int64), cutoff, pair_mode, wells, int(seed),
                      lprime_margin=float(d.get("lprime_margin", 8.0)), fine_mode=fine_mode,
                      precision=_precision(d.get("precision", "fp64")))


def _precision(p):
    if p not in PRECISIONS:
        raise SpecError("spec: precision is one of %s" % (PRECISIONS,))
    return p


def to_dict(w):
    """Explicit spec of a workload (every atom listed)."""
    return {"name": w.name, "h": w.h, "N": [int(x) for x in w.N],
            "atoms": [{"pos": [float(x) for x in w.pos[k]], "r_loc": float(w.r_loc[k]),
                       "r_fine": float(w.r_fine[k]), "n_sf": int(w.nsf[k])} for k in range(len(w.pos))],
            "pair_cutoff": "sum_of_radii" if w.pair_mode == 1 else float(w.pair_cutoff),
            "lprime_margin": float(w.lprime_margin), "fine_mode": w.fine_mode,
            "precision": w.precision, "seed": int(w.seed),
            "wells": np.asarray(w.wells, np.float64).tolist()}


def load(path):
    with open(path) as f:
        try:
            d = json.load(f)
        except json.JSONDecodeError as e:
            raise SpecError("spec: not valid JSON (%s)" % e) from None
    return from_dict(d)


def dump(w, path):
    with open(path, "w") as f:
        json.dump(to_dict(w), f, indent=1)
