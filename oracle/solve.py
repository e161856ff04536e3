"""End-to-end oracle solve of a workload.  Test infrastructure only."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import gll as _gll
from .discretize import Level, lift
from .krylov import fcg, gmres
from .multigrid import Hierarchy


@dataclass
class OracleResult:
    u: np.ndarray           # full nodal solution (boundary included), per rhs
    iterations: list
    history: list
    f0: np.ndarray
    hierarchy: Hierarchy


def build(workload, order=None, smoother="gll", restriction="interp"):
    """Fine level and hierarchy of a workload (coordinates at the oracle's own
    GLL nodes)."""
    p = workload.order if order is None else order
    xi, _ = _gll.gll(p)
    coords = workload.coords(xi)
    fine = Level(workload.dim, workload.nelem, p, coords)
    return fine, Hierarchy(fine, smoother=smoother, restriction=restriction)


def solve(workload, gamma=2, alpha=2.0 / 3.0, tol=1e-10, maxit=200, method="fcg",
          m=1, hierarchy=None, rhs_index=None):
    if hierarchy is None:
        fine, hier = build(workload)
    else:
        hier = hierarchy
        fine = hier.levels[-1]
    coords = fine.coords
    F = workload.sample_rhs(coords)
    g = workload.sample_dirichlet(coords)
    idx = range(workload.nrhs) if rhs_index is None else rhs_index
    us, its, hists, f0s = [], [], [], []
    for j in idx:
        f0, v = lift(fine, F[j], g)
        M = lambda r: hier.precondition(r, gamma, alpha, m)
        if method in ("fcg", "pcg"):
            w, k, h = fcg(fine.apply, M, f0, tol, maxit, flexible=(method == "fcg"))
        elif method == "gmres":
            w, k, h = gmres(fine.apply, M, f0, tol, maxit)
        else:
            raise ValueError(method)
        us.append(w + v)
        its.append(k)
        hists.append(h)
        f0s.append(f0)
    return OracleResult(np.stack(us), its, hists, np.stack(f0s), hier)
