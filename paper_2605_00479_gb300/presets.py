"""Reaction networks and seeded input generators.

This module holds only model *tables* (species, reactant orders, stoichiometry,
rate constants, laws) and seeded parameter draws.  It contains none of the
simulation arithmetic, imports nothing else from this package, and is the one
module shared by the CUDA engine's callers and the test oracle.

Rate constants follow Gillespie's c-convention: the propensity of a
mass-action reaction is c_j times the number of distinct reactant
combinations, prod_i C(x_i, r_ij).  The paper's k-constants absorb the 1/r!
factors (Sec. 4.2: k1 = c1/2, k2 = c2/6 for the Schloegl model).

Models (paper section in brackets):
  birth_death   0 -> X (k), X -> 0 (gamma)                        [Sec. 4.1]
  schlogl       A + 2X <-> 3X, B <-> X, reservoirs A and B fixed   [Sec. 4.2]
  telegraph     Goff <-> Gon, Gon -> Gon + M, M -> 0               [Sec. 4.3]
  dimer         2A <-> D                                          [Sec. 4.4]
  repressilator three mRNAs, three proteins, Hill repression       [Sec. 4.5]
  hill_self     0 -> X at alpha0 + alpha/(1+X^h), X -> 0 (gamma)   (pin model)
"""
from __future__ import annotations

import numpy as np

MASS_ACTION = 0
HILL_REPRESSION = 1


def _model(order, stoich, rate, law=None, hill=None, constant=None, names=None):
    order = np.asarray(order, dtype=np.int32)
    M, N = order.shape
    return {
        "order": order,
        "stoich": np.asarray(stoich, dtype=np.int32).reshape(M, N),
        "rate": np.asarray(rate, dtype=np.float64).reshape(M),
        "law": np.zeros(M, np.int32) if law is None else np.asarray(law, dtype=np.int32),
        "hill": None if hill is None else np.asarray(hill, dtype=np.float64).reshape(M, 4),
        "constant": None if constant is None else np.asarray(constant, dtype=np.uint8),
        "names": names,
    }


def birth_death(k=10.0, gamma=0.1):
    """0 -> X at rate k; X -> 0 at rate gamma*X.  Stationary law Poisson(k/gamma)."""
    return _model(order=[[0], [1]], stoich=[[1], [-1]], rate=[k, gamma], names=["X"])


def schlogl(c1=3e-7, c2=1e-4, c3=1e-3, c4=3.5, A=1e5, B=2e5):
    """Schloegl model with species (X, A, B); A and B are held fixed.

    Defaults: the classic bistable set in c-convention (k1 = c1/2 = 1.5e-7,
    k2 = c2/6 = 1.667e-5, k3 = 1e-3, k4 = 3.5, A = 1e5, B = 2e5).
    """
    m = _model(
        order=[[2, 1, 0], [3, 0, 0], [0, 0, 1], [1, 0, 0]],
        stoich=[[1, -1, 0], [-1, 1, 0], [1, 0, -1], [-1, 0, 1]],
        rate=[c1, c2, c3, c4], constant=[0, 1, 1], names=["X", "A", "B"])
    m["reservoirs"] = (int(A), int(B))
    return m


def schlogl_x0(model, X0=250):
    A, B = model["reservoirs"]
    return np.array([X0, A, B], dtype=np.int32)


def schlogl_rescaled():
    """The paper's rescaled parameter set: k1 = 1.5e-4 with A = 100, k3 = 1 with B = 200."""
    return schlogl(c1=3e-4, c2=1e-4, c3=1.0, c4=3.5, A=100, B=200)


def telegraph(kon=0.05, koff=0.05, km=20.0, gamma=1.0):
    """Species (Goff, Gon, M): Goff -> Gon (kon), Gon -> Goff (koff),
    Gon -> Gon + M (km), M -> 0 (gamma).  Start: gene off, no mRNA."""
    return _model(
        order=[[1, 0, 0], [0, 1, 0], [0, 1, 0], [0, 0, 1]],
        stoich=[[-1, 1, 0], [1, -1, 0], [0, 0, 1], [0, 0, -1]],
        rate=[kon, koff, km, gamma], names=["Goff", "Gon", "M"])


TELEGRAPH_X0 = np.array([1, 0, 0], dtype=np.int32)


def dimer(k1=1e-3, k2=0.1):
    """Species (M, D): 2M -> D (k1, propensity k1 M(M-1)/2), D -> 2M (k2 D)."""
    return _model(order=[[2, 0], [0, 1]], stoich=[[-2, 1], [2, -1]], rate=[k1, k2], names=["M", "D"])


def dimer_x0(M0=300):
    return np.array([M0, 0], dtype=np.int32)


def repressilator(alpha0=0.216, alpha=216.0, h=2, beta=5.0, mdecay=1.0, pdecay=5.0):
    """Species (MA, MB, MC, PA, PB, PC).  Per gene i in (A, B, C), in order:
    transcription 0 -> M_i at alpha0 + alpha/(1 + P_j^h) with repressor
    j = (C, A, B)[i]; mRNA decay M_i -> 0; translation M_i -> M_i + P_i (beta);
    protein decay P_i -> 0."""
    order, stoich, rate, law, hill = [], [], [], [], []
    repressor = {0: 5, 1: 3, 2: 4}  # A <- P_C, B <- P_A, C <- P_B
    for g in range(3):
        o = [0] * 6; s = [0] * 6; s[g] = 1
        order.append(o); stoich.append(s); rate.append(1.0); law.append(HILL_REPRESSION)
        hill.append([alpha0, alpha, float(h), float(repressor[g])])
        o = [0] * 6; o[g] = 1; s = [0] * 6; s[g] = -1
        order.append(o); stoich.append(s); rate.append(mdecay); law.append(MASS_ACTION); hill.append([0, 0, 0, 0])
        o = [0] * 6; o[g] = 1; s = [0] * 6; s[3 + g] = 1
        order.append(o); stoich.append(s); rate.append(beta); law.append(MASS_ACTION); hill.append([0, 0, 0, 0])
        o = [0] * 6; o[3 + g] = 1; s = [0] * 6; s[3 + g] = -1
        order.append(o); stoich.append(s); rate.append(pdecay); law.append(MASS_ACTION); hill.append([0, 0, 0, 0])
    return _model(order, stoich, rate, law=law, hill=hill, names=["MA", "MB", "MC", "PA", "PB", "PC"])


REPRESSILATOR_X0 = np.array([0, 0, 0, 5, 0, 0], dtype=np.int32)


def repressilator_paper():
    """Parameter set printed in Sec. 4.5: alpha0 = 1, delta_p = 1."""
    return repressilator(alpha0=1.0, alpha=216.0, h=2, beta=5.0, mdecay=1.0, pdecay=1.0)


def hill_self(alpha0=1.0, alpha=30.0, h=2, gamma=1.0):
    """One species repressing its own production: 0 -> X at alpha0 + alpha/(1+X^h),
    X -> 0 at gamma*X.  A birth-death chain with a closed-form stationary law."""
    return _model(order=[[0], [1]], stoich=[[1], [-1]], rate=[1.0, gamma],
                  law=[HILL_REPRESSION, MASS_ACTION], hill=[[alpha0, alpha, float(h), 0.0], [0, 0, 0, 0]],
                  names=["X"])


def even_samples(t_end, K):
    """K evenly spaced sample times 0 .. t_end inclusive."""
    if K == 1:
        return np.array([t_end], dtype=np.float64)
    return np.linspace(0.0, t_end, K, dtype=np.float64)


# ---------------------------------------------------------------- sweeps
def log_uniform(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))


def telegraph_sweep(n_sets, seed=2024, gamma_range=None):
    """Rate tables [n_sets, 4] = (kon, koff, km, gamma): kon, koff log-uniform in
    [0.05, 5], km log-uniform in [5, 100]; gamma = 1 or log-uniform in gamma_range."""
    rng = np.random.default_rng(seed)
    kon = log_uniform(rng, 0.05, 5.0, n_sets)
    koff = log_uniform(rng, 0.05, 5.0, n_sets)
    km = log_uniform(rng, 5.0, 100.0, n_sets)
    gamma = np.ones(n_sets) if gamma_range is None else log_uniform(rng, gamma_range[0], gamma_range[1], n_sets)
    return np.stack([kon, koff, km, gamma], axis=1)


def dimer_sweep(n_sets, seed=2025):
    """(k1, k2) log-uniform in [x0.5, x2] around (1e-3, 0.1)."""
    rng = np.random.default_rng(seed)
    return np.stack([log_uniform(rng, 0.5e-3, 2e-3, n_sets), log_uniform(rng, 0.05, 0.2, n_sets)], axis=1)


def repressilator_sweep(n_sets, seed=2026):
    """Rate tables [n_sets, 12] and Hill tables [n_sets, 12, 4] for the
    repressilator with alpha and beta log-uniform in [x0.5, x2] around
    (216, 5) and the other constants as in repressilator()."""
    rng = np.random.default_rng(seed)
    alpha = log_uniform(rng, 108.0, 432.0, n_sets)
    beta = log_uniform(rng, 2.5, 10.0, n_sets)
    base = repressilator()
    rates = np.repeat(base["rate"][None, :], n_sets, axis=0)
    hills = np.repeat(base["hill"][None, :, :], n_sets, axis=0)
    for g in range(3):
        hills[:, 4 * g, 1] = alpha
        rates[:, 4 * g + 2] = beta
        rates[:, 4 * g + 3] = beta
    return rates, hills
