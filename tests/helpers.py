"""Test-only helpers: golden fixture loading and tolerances."""
import json
import os

import numpy as np
import scipy.sparse as sp

from instances import BlockLP

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _mat(rows, m, n):
    a = np.array(rows, dtype=float).reshape(m, n) if m * n else np.zeros((m, n))
    return sp.csc_matrix(a)


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        d = json.load(f)
    N, n0, mg = d["N"], d["n0"], d["mg"]
    A = [sp.csc_matrix(np.array(a, dtype=float)) for a in d["A"]]
    ms = [a.shape[0] for a in A]
    ns = [a.shape[1] for a in A]
    W = [_mat(d["W"][i], ms[i], n0) for i in range(N)]
    l = np.array(d["l"], dtype=np.int64)
    FL = [_mat(d["FL"][j], int(l[j]), ns[j]) for j in range(N - 1)]
    FR = [_mat(d["FR"][j], int(l[j]), ns[j + 1]) for j in range(N - 1)]
    F0 = [_mat(d["F0"][j], int(l[j]), n0) for j in range(N - 1)]
    Fg = [_mat(d["Fg"][i], mg, ns[i]) for i in range(N)]
    Fg0 = _mat(d["Fg0"], mg, n0)
    lp = BlockLP(N=N, n0=n0, mg=mg, A=A, W=W,
                 b=[np.array(v, float) for v in d["b"]],
                 c=[np.array(v, float) for v in d["c"]],
                 c0=np.array(d["c0"], float), l=l, FL=FL, FR=FR, F0=F0,
                 blink=[np.array(v, float) for v in d["blink"]], Fg=Fg, Fg0=Fg0,
                 bg=np.array(d["bg"], float), name=name)
    return lp, d


GOLDEN_FILES = sorted(f for f in os.listdir(GOLDEN) if f.endswith(".json"))
