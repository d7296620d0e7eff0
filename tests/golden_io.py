"""Readers for the text fixtures under tests/golden/ (values the paper prints)."""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _num(tok: str) -> Fraction:
    return Fraction(tok)


def _lines(fname):
    with open(os.path.join(GOLDEN, fname)) as f:
        for raw in f:
            line = raw.strip()
            if line and not line.startswith("#"):
                yield line


def _matrix(spec: str):
    return [[_num(t) for t in row.split()] for row in spec.split(";")]


def toy_tree(fname: str = "toy_tree.txt"):
    """dict: 'A','b','solution' (Fractions) and per-quantity lists over rounds.
    ``toy_tree_damped.txt`` (rounds 1 and 2 under damping) adds 'gamma'."""
    out = {}
    for line in _lines(fname):
        key, rest = line.split(None, 1)
        if key == "matrix":
            out["A"] = _matrix(rest)
        else:
            out[key] = [_num(t) for t in rest.split()]
    return out


def paper_systems():
    """dict name -> dict with 'A' (float array, scale applied), 'A_exact' and
    optional 'b', 'solution', 'spectral_radius', 'parallel_gabp_iterations',
    'serial_gabp_iterations'."""
    systems, cur = {}, None
    for line in _lines("paper_systems.txt"):
        key, rest = line.split(None, 1)
        if key == "name":
            cur = systems.setdefault(rest, {})
        elif key == "matrix":
            cur["matrix"] = _matrix(rest)
        elif key == "scale":
            cur["scale"] = _num(rest)
        elif key in ("rhs", "solution"):
            cur[key] = [_num(t) for t in rest.split()]
        elif key == "spectral_radius":
            cur[key] = float(rest)
        elif key in ("parallel_gabp_iterations", "serial_gabp_iterations"):
            cur[key] = int(rest)
    for s in systems.values():
        exact = [[v * s.get("scale", 1) for v in row] for row in s["matrix"]]
        s["A_exact"] = exact
        s["A"] = np.array([[float(v) for v in row] for row in exact])
        s["b"] = np.array([float(v) for v in s["rhs"]])
    return systems
