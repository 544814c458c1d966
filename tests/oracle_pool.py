"""The oracle's per-shell work spread over worker processes (test
infrastructure).

In the oracle, the interior right-hand side (Deriv, Jacobian, GHEqns) and the
filters act on each shell separately; only ApplyBCs couples the shells.  For
domains where one oracle right-hand side takes minutes, ShellPool runs those
per-shell steps one shell per task in a pool of spawned processes (spawned,
never forked: the parent has a CUDA context) and is installed in place of
evolve.rhs_interior and evolve.apply_filters, so that the oracle's own
rk4_step and apply_boundaries orchestrate the result.  Each task computes
exactly what the oracle computes for that shell: the same functions on the
same arrays.
"""
import multiprocessing as mp
import types

import numpy as np

from oracle import evolve, grid


def _interior(task):
    spec, H, dH, gammas, us = task
    one = types.SimpleNamespace(grids=[grid.shell_grid(*spec)], H=[H], dH=[dH],
                                gamma0=gammas[0], gamma1=gammas[1], gamma2=gammas[2])
    return evolve.rhs_interior(one, [us])[0]


def _filters(task):
    spec, params, us = task
    one = types.SimpleNamespace(grids=[grid.shell_grid(*spec)], **params)
    return evolve.apply_filters(one, [us])[0]


class ShellPool:
    """Worker processes that evaluate the oracle's per-shell steps of a domain."""

    def __init__(self, processes):
        self.pool = mp.get_context("spawn").Pool(processes)

    def close(self):
        self.pool.close()
        self.pool.join()

    def rhs_interior(self, dom, u):
        gam = (dom.gamma0, dom.gamma1, dom.gamma2)
        return self.pool.map(_interior, [(spec, dom.H[s], dom.dH[s], gam, np.asarray(u[s]))
                                         for s, spec in enumerate(dom.specs)], chunksize=1)

    def apply_filters(self, dom, u):
        params = dict(radial_filter_on=dom.radial_filter_on, filt_alpha=dom.filt_alpha,
                      filt_order=dom.filt_order, sh_keep_l=dom.sh_keep_l, sh_filter=dom.sh_filter)
        return self.pool.map(_filters, [(spec, params, np.asarray(u[s])) for s, spec in enumerate(dom.specs)],
                             chunksize=1)

    def install(self, monkeypatch):
        """Use the pool for the oracle's per-shell steps (undone with the
        monkeypatch)."""
        monkeypatch.setattr(evolve, "rhs_interior", self.rhs_interior)
        monkeypatch.setattr(evolve, "apply_filters", self.apply_filters)
