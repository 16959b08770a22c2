"""Resampled phase-space points and the Monte Carlo estimate of sigma-hat.

Oracle module (test infrastructure only).

Eq. 4 integrated over Eq. 5 with the point density of the generator:

    sigma-hat = (1/N_try) sum_{accepted i} w_i ,
    w_i = 1/(2 s-hat) * W_PS,i * |M|^2_avg,i * S_ident * 0.3893793721e9 pb GeV^2

where W_PS is the generator's weight (the phase-space volume for RAMBO),
N_try counts every draw (accepted or not) and S_ident = 1/k! for k identical
final-state particles.  The error is the standard error of the mean over the
N_try draws (rejected draws contribute w = 0).
"""
import math
import numpy as np

from . import phasespace as ps
from .sm import GEV2_TO_PB


def draw(kin, par, u):
    """One draw for every row of u: (P, W_PS, ok, s-hat).  Kinds: 2to2, rambo, ttbar, rambo_bw and
    ypt (the paper's parametrisation: objects with absolute leg indices, as phasespace.ypt_phi)."""
    kind = kin["kind"]
    N = u.shape[0]
    if kind == "2to2":
        w = kin["sqrt_s"]
        P, wt = ps.two_to_two_massless(w, u)
        return P, wt, np.ones(N, dtype=bool), np.full(N, w * w)
    if kind == "rambo":
        w = kin["sqrt_s"]
        masses = kin.get("masses")
        nf = kin["n_final"]
        if masses and any(m > 0 for m in masses):
            pf, wt = ps.rambo_massive(w, masses, u)
        else:
            pf, wt = ps.rambo_massless(w, nf, u)
        P = np.zeros((N, nf + 2, 4))
        P[:, 0], P[:, 1] = ps.incoming(w, N)
        P[:, 2:] = pf
        return P, wt, np.ones(N, dtype=bool), np.full(N, w * w)
    if kind == "ttbar":
        return ps.ttbar_dilepton(u, par, kin["sqrt_s_range"])
    if kind == "ypt":
        w = kin["sqrt_s"]
        nf = kin["n_final"]
        objs = [dict(o, legs=tuple(l - 2 for l in o["legs"])) for o in kin["objects"]]
        pf, wt, ok = ps.ypt_phi(w, objs, nf, u)
        P = np.zeros((N, nf + 2, 4))
        P[:, 0], P[:, 1] = ps.incoming(w, N)
        P[:, 2:] = pf
        return P, wt, ok, np.full(N, w * w)
    if kind == "rambo_bw":
        w = kin["sqrt_s"]
        nf = kin["n_final"]
        pf, wt, ok = ps.rambo_resonance(w, nf, kin["res_mass"], kin["res_width"], u)
        P = np.zeros((N, nf + 2, 4))
        P[:, 0], P[:, 1] = ps.incoming(w, N)
        P[:, 2:] = pf
        return P, wt, ok, np.full(N, w * w)
    raise ValueError(kind)


def grid_dims(kin):
    """Uniform variables a draw uses (also the dimensions of an adaptive grid, oracle.vegas)."""
    if kin["kind"] == "2to2":
        return 2
    if kin["kind"] == "rambo":
        return 4 * kin["n_final"]
    if kin["kind"] == "rambo_bw":
        return 4 * kin["n_final"] - 1
    if kin["kind"] == "ypt":
        return 3 * kin["n_final"] - 3
    return 15


def generate(kin, par, seed, events, max_attempts=10000):
    """Accepted points for the given event indices, redrawing failed ones.

    Returns (P [N, n, 4], W_PS [N], s-hat [N], tries [N]) where tries is the
    number of draws the event used (accepted attempt index + 1).
    """
    return _generate(kin, par, seed, events, max_attempts, None)[:4]


def generate_grid(kin, par, seed, events, grid, max_attempts=10000):
    """generate() with the uniforms of every draw mapped through an adaptive grid
    (oracle.vegas.vegas_map on the first grid_dims(kin) uniforms): the weight
    carries the map's Jacobian.  Returns (P, W, s-hat, tries, bins [N, D])."""
    return _generate(kin, par, seed, events, max_attempts, np.asarray(grid, dtype=np.float64))


def _generate(kin, par, seed, events, max_attempts, grid):
    from . import vegas
    events = np.asarray(events, dtype=np.uint64)
    N = events.shape[0]
    attempt = np.zeros(N, dtype=np.uint64)
    pending = np.ones(N, dtype=bool)
    P = None
    W = np.zeros(N)
    S = np.zeros(N)
    nu = grid_dims(kin)
    cut = kin.get("cuts")
    bins = None
    if grid is not None:
        assert grid.shape[0] == grid_dims(kin)
        bins = np.zeros((N, grid.shape[0]), dtype=np.int64)
    while pending.any():
        idx = np.nonzero(pending)[0]
        u = ps.uniforms(seed, events[idx], attempt[idx], nu)
        if grid is not None:
            D = grid.shape[0]
            x, jac, b = vegas.vegas_map(grid, u[:, :D])
            u = u.copy()
            u[:, :D] = x
        Pn, Wn, ok, Sn = draw(kin, par, u)
        if grid is not None:
            Wn = Wn * jac
        if cut is not None:
            ok = ok & ps.pass_cuts(Pn, cut["legs"], cut["pt_min"], cut["eta_max"], cut["dr_min"])
        if kin.get("paper_cuts") is not None:
            pc = kin["paper_cuts"]
            ok = ok & ps.pass_paper_cuts(Pn, pc["leg_class"], pc["thresholds"])
        if P is None:
            P = np.zeros((N,) + Pn.shape[1:])
        acc = idx[ok]
        P[acc] = Pn[ok]
        W[acc] = Wn[ok]
        S[acc] = Sn[ok]
        if grid is not None:
            bins[acc] = b[ok]
        pending[acc] = False
        attempt[idx[~ok]] += np.uint64(1)
        if int(attempt.max()) >= max_attempts:
            raise RuntimeError("phase-space resampling did not converge")
    return P, W, S, attempt.astype(np.int64) + 1, bins


def accumulate(me2, W, S, tries, s_ident):
    """(sum w, sum w^2, n_acc, n_try) over the accepted points."""
    w = (1.0 / (2.0 * S)) * W * me2 * s_ident * GEV2_TO_PB
    return float(w.sum()), float((w * w).sum()), int(w.shape[0]), int(tries.sum())


def estimate(sum_w, sum_w2, n_try):
    """sigma-hat and its standard error in pb."""
    mean = sum_w / n_try
    var = max(sum_w2 / n_try - mean * mean, 0.0)
    return mean, math.sqrt(var / max(n_try - 1, 1))
