"""Passive advection by a truncated Taylor exponential and its adjoints, fp64.
Oracle -- test infrastructure only.

Sec. 3.1, Eq. Adv: rho_{i+1} = A[rho_i, v_i] = sum_k (dt^k / k!) A(v_i)^k rho_i,
truncated at the first order K >= 1 whose term is small.  Reading (the paper
only says the term must be "< 1e-5"): the term's max-norm is compared with
``tol * scale``, where ``scale`` is the problem's max |rho_0|; the small term
itself is included in the sum; K > kmax is an error.

Adjoints (Eq. KKTPO / Alg. 1) are written as the plain derivative of that
finite sum with K held fixed (the order recorded by the forward pass).
"""
import math

import numpy as np

from . import mac


class TaylorOrderError(RuntimeError):
    pass


def taylor_forward(grid, v, rho, dt, tol, scale, kmax=64):
    """Return (rho_next, K, terms) with terms[k] = (dt^k/k!) A(v)^k rho, k = 0..K."""
    A = mac.advection_matrix(grid, v)
    terms = [rho.copy()]
    t = rho
    for k in range(1, kmax + 1):
        t = (dt / k) * (A @ t)
        terms.append(t)
        if np.max(np.abs(t)) < tol * scale:
            return np.sum(terms, axis=0), k, terms
    raise TaylorOrderError("Taylor series did not reach tolerance within kmax=%d" % kmax)


def taylor_apply(grid, v, rho, dt, K):
    """sum_{k=0}^{K} (dt^k/k!) A(v)^k rho with a fixed order K."""
    A = mac.advection_matrix(grid, v)
    out = rho.copy()
    t = rho
    for k in range(1, K + 1):
        t = (dt / k) * (A @ t)
        out = out + t
    return out


def taylor_adjoint_rho(grid, v, mu, dt, K):
    """(d A[rho, v] / d rho)^T mu = sum_{k=0}^{K} (dt^k/k!) (A(v)^T)^k mu."""
    AT = mac.advection_matrix(grid, v).T.tocsr()
    out = mu.copy()
    t = mu
    for k in range(1, K + 1):
        t = (dt / k) * (AT @ t)
        out = out + t
    return out


def taylor_adjoint_v(grid, v, rho, mu, dt, K):
    """(d A[rho, v] / d v)^T mu with K fixed.

    d/dv sum_k c_k A^k rho = sum_{k=1}^{K} c_k sum_{m=0}^{k-1} A^{k-1-m} B(A^m rho),
    with c_k = dt^k / k! and B(x) dv = d(A(v) x)/dv dv, so the transpose applied
    to mu is the double sum  sum_k c_k sum_m B(A^m rho)^T (A^T)^{k-1-m} mu,
    evaluated here term by term exactly as written.
    """
    A = mac.advection_matrix(grid, v)
    AT = A.T.tocsr()
    powers = [rho]                      # A^m rho, m = 0..K-1
    for m in range(1, K):
        powers.append(A @ powers[-1])
    adj = [mu]                          # (A^T)^j mu, j = 0..K-1
    for j in range(1, K):
        adj.append(AT @ adj[-1])
    out = np.zeros(grid.F)
    for k in range(1, K + 1):
        ck = dt ** k / math.factorial(k)
        for m in range(k):
            out += ck * mac.advection_v_derivative_T(grid, v, powers[m], adj[k - 1 - m])
    return out
