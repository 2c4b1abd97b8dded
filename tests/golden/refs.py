"""Reader of the oracle reference fixtures written by ``make_large_golden.py`` and the error
measures a solver result is judged by.

A fixture stores, per right-hand side, the oracle's compliance, ||u||_2, ||u||_inf, the
projections u . g_i on 8 seeded N(0,1) vectors and u at sampled DOFs (see the script).  For a
candidate solution u:
  * rel_compliance_error = |c - c_ref| / |c_ref|;
  * rel_u_error_est = sqrt(mean_i ((u - u_ref) . g_i)^2) / ||u_ref||_2, an unbiased estimate of
    ||u - u_ref||_2^2 / ||u_ref||_2^2 under the square root (E[(g . d)^2] = ||d||^2 for
    g ~ N(0, I)), so it sees errors anywhere in the vector;
  * rel_u_error_sampled = ||(u - u_ref)[S]|| / ||u_ref[S]|| over the uniformly sampled DOFs S;
  * max_abs_error_rel_inf = max over all stored DOFs of |u - u_ref| / ||u_ref||_inf.
This module holds no arithmetic of the method; it reads text and compares vectors.
"""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
N_PROJ = 8


def projections(n):
    """The seeded N(0,1) probe vectors g_i (numpy default_rng(1000 + i))."""
    return [np.random.default_rng(1000 + i).standard_normal(n) for i in range(N_PROJ)]


def path(name):
    return os.path.join(HERE, name + ".txt")


def load(name):
    """List of per-right-hand-side dicts of the fixture ``name`` (file name without .txt)."""
    out, cur, mode, left = [], None, None, 0
    for line in open(path(name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        t = line.split()
        if left > 0:
            cur[mode].append((int(t[0]), float(t[1])))
            left -= 1
            continue
        if t[0] == "rhs":
            cur = dict(rhs=int(t[1]), n=int(t[3]), iterations=int(t[5]),
                       true_rel_residual=float(t[7]), uniform=[], extra=[])
            out.append(cur)
        elif t[0] in ("compliance", "norm2", "norminf"):
            cur[t[0]] = float(t[1])
        elif t[0] == "proj":
            cur["proj"] = np.array([float(v) for v in t[1:]])
        elif t[0] == "crosscheck":
            cur["crosscheck"] = {t[i]: float(t[i + 1]) for i in range(2, len(t) - 1, 2)}
        elif t[0] in ("uniform", "extra"):
            mode, left = t[0], int(t[1])
        else:
            raise ValueError("unexpected line in %s: %s" % (name, line))
    return out


def accuracy(u, compliance, ref, G=None):
    """Error measures of solution u (host array) with compliance ``compliance`` against one
    right-hand side ``ref`` of a fixture.  G: the probe vectors (computed if not given)."""
    u = np.asarray(u, dtype=np.float64)
    if G is None:
        G = projections(u.size)
    dp = np.array([g @ u for g in G]) - ref["proj"]
    iu = np.array([i for i, _ in ref["uniform"]], dtype=np.int64)
    vu = np.array([v for _, v in ref["uniform"]])
    ia = np.array([i for i, _ in ref["uniform"] + ref["extra"]], dtype=np.int64)
    va = np.array([v for _, v in ref["uniform"] + ref["extra"]])
    return {
        "rel_compliance_error": abs(compliance - ref["compliance"]) / abs(ref["compliance"]),
        "rel_u_error_est": float(np.sqrt(np.mean(dp ** 2)) / ref["norm2"]),
        "rel_u_error_sampled": float(np.linalg.norm(u[iu] - vu) / np.linalg.norm(vu)),
        "max_abs_error_rel_inf": float(np.abs(u[ia] - va).max() / ref["norminf"]),
        "rel_norm2_diff": abs(float(np.linalg.norm(u)) - ref["norm2"]) / ref["norm2"],
    }
