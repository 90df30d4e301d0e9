"""Chemical master equation on a truncated state space (test infrastructure only).

The direct method samples exact paths of the continuous-time Markov chain whose
forward equation is the chemical master equation (Sec. 2: the SSA "generates
exact realisations" of it).  On a small truncated state space the CME can be
solved directly, p(t) = p(0) exp(Q t), which pins the oracle's fp64 mode: its
empirical law at each sample time must match p(t).

Propensities are written from their definitions with exact combinatorics:
mass action a_j = c_j * prod_i C(x_i, r_ij) (Gillespie's c-convention; Sec. 2,
Sec. 4.2 and Sec. 4.4 of the paper) and Hill repression
a_j = alpha0 + alpha / (1 + P^h) (Sec. 4.5).  Constant species keep their count.
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg


def propensity(model, j, x):
    """a_j(x) in binary64 from the definitions above."""
    if int(model["law"][j]) == 1:
        alpha0, alpha, h, reg = model["hill"][j]
        P = float(x[int(reg)])
        return alpha0 + alpha / (1.0 + P ** int(h))
    a = float(model["rate"][j])
    for i, r in enumerate(model["order"][j]):
        if r:
            a *= math.comb(int(x[i]), int(r))
    return a


def enumerate_states(model, x0, bounds):
    """States reachable from x0 with every species i kept in [0, bounds[i]].

    Transitions that would leave the box are returned with target -1 (an
    absorbing sink), so the probability lost to the truncation is measurable."""
    x0 = tuple(int(v) for v in x0)
    const = model.get("constant")
    index = {x0: 0}
    states = [x0]
    edges = []
    q = deque([x0])
    M = len(model["rate"])
    while q:
        x = q.popleft()
        for j in range(M):
            a = propensity(model, j, x)
            if a <= 0.0:
                continue
            y = list(x)
            for i, s in enumerate(model["stoich"][j]):
                if const is not None and const[i]:
                    continue
                y[i] += int(s)
            y = tuple(y)
            if any(v < 0 or v > b for v, b in zip(y, bounds)):
                edges.append((index[x], -1, a))   # leaves the truncated space: goes to the sink
                continue
            if y not in index:
                index[y] = len(states)
                states.append(y)
                q.append(y)
            edges.append((index[x], index[y], a))
    return states, index, edges


def generator(n, edges):
    """Sparse generator Q (rows: from, cols: to) with diagonal -sum of outflow;
    index n is the absorbing sink for mass leaving the truncated space."""
    rows = [e[0] for e in edges]
    cols = [e[1] if e[1] >= 0 else n for e in edges]
    n = n + 1
    vals = [e[2] for e in edges]
    Q = scipy.sparse.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    out = np.asarray(Q.sum(axis=1)).ravel()
    return (Q - scipy.sparse.diags(out)).tocsc()


def transient(model, x0, bounds, times):
    """p(t) for each t in times (ascending), with p(0) = delta_{x0}.

    Returns (states, P) where P has shape [len(times), n_states]; the mass
    lost to the truncation at time t is 1 - P[t].sum()."""
    states, index, edges = enumerate_states(model, x0, bounds)
    Q = generator(len(states), edges)
    p0 = np.zeros(len(states) + 1)
    p0[0] = 1.0
    out = []
    for t in times:
        if t == 0.0:
            out.append(p0.copy())
        else:
            out.append(scipy.sparse.linalg.expm_multiply(Q.T * t, p0))
    return states, np.array(out)[:, :-1]


def marginal(states, p, species):
    """Marginal law of one species: (support values, probabilities)."""
    vals = np.array([s[species] for s in states])
    hi = vals.max()
    m = np.zeros(hi + 1)
    np.add.at(m, vals, p)
    return np.arange(hi + 1), m


def stationary_birth_death_chain(birth, death, n_max):
    """Stationary law of a 1-D birth-death chain by detailed balance:
    pi(n+1)/pi(n) = birth(n)/death(n+1)."""
    logp = np.zeros(n_max + 1)
    for n in range(n_max):
        logp[n + 1] = logp[n] + math.log(birth(n)) - math.log(death(n + 1))
    p = np.exp(logp - logp.max())
    return p / p.sum()
