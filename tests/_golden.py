"""Readers for the closed-form fixtures under tests/golden/ (shared by the
oracle pins and the GPU parity tests)."""
from __future__ import annotations

import math
from pathlib import Path

import numpy as np

from synthetic import Problem

GOLDEN = Path(__file__).resolve().parent / "golden"


def delta_cases():
    """Yield (name, Problem, late_mode, prim_mode, expected) for each line of
    delta_basis.txt.  The problem has w_l = 1, one radial point, and the
    radial weight 1 is supplied separately by the caller (xw = [1])."""
    for line in (GOLDEN / "delta_basis.txt").read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = [t.strip() for t in line.split("|")]
        name, l_min, l_max = f[0], int(f[1]), int(f[2])
        late_l = [int(v) for v in f[3].split(",")]
        prim_l = [int(v) for v in f[4].split(",")]
        lm = np.array([int(v) for v in f[5].split(",")], dtype=np.int32).reshape(1, 3)
        pm = np.array([int(v) for v in f[6].split(",")], dtype=np.int32).reshape(1, 3)
        num, den = int(f[7]), int(f[8])
        L = l_max - l_min + 1
        q = np.zeros((len(late_l), L))
        for a, l in enumerate(late_l):
            q[a, l - l_min] = 1.0
        qt = np.zeros((1, len(prim_l), L))
        for p, l in enumerate(prim_l):
            qt[0, p, l - l_min] = 1.0
        P = Problem(l_min=l_min, l_max=l_max, nb_late=len(late_l), nb_prim=len(prim_l),
                    n_x=1, q=q, qt=qt, w_l=np.ones(L), x=np.array([1.0]),
                    phi=np.zeros(len(prim_l)), late_modes=lm, prim_modes=pm, name=name)
        yield name, P, num / (den * math.pi)
