"""Independent audits of a solved step, FP64 (test infrastructure only).

* ``kkt_direct``    -- Eq. 2 solved directly (least squares on the full KKT matrix) for worlds
                       without contacts; u+ is unique even when lambda is not (redundant loops).
* ``ncp_residual``  -- natural-map residual of the dual problem (Eq. 3) at a returned lambda,
                       in the Jacobi-scaled units of Sec. 4.1: for every contact block
                       ||lam_k - Pi_K(lam_k - (v_k + Gamma(v_k)))||_inf, and for the bilateral
                       block the part of the constraint velocity that lies in the range of the
                       scaled Jacobian (the rest is the inconsistent bias of redundant rows,
                       which no impulse can remove).
"""
from __future__ import annotations

import numpy as np

from . import padmm as PA


def kkt_direct(J, M, u_minus_plus_dt_h, v_star, R=None):
    """Solve [[M, J^T], [J, -R]] [u+; -lambda] = [M u- + dt h; -v*] (Eq. 2) by least squares.
    ``u_minus_plus_dt_h`` is M u- + dt h.  Returns (u+, lambda)."""
    n = M.shape[0]
    m = J.shape[0]
    R = np.zeros((m, m)) if R is None else R
    K = np.block([[M, J.T], [J, -R]])
    rhs = np.concatenate([u_minus_plus_dt_h, -v_star])
    sol, *_ = np.linalg.lstsq(K, rhs, rcond=1e-13)
    return sol[:n], -sol[n:]


def ncp_residual(J, u_plus, v_star, lam, p, n_bilateral, mu, reg=None, unilateral=()):
    """Natural-map NCP residual (scaled units) of (lambda, u+).  Returns (r_contact, r_bilateral).
    The row velocity is v = J u+ + R lambda + v* (Eq. 2's second block row).  Contact triples and
    unilateral rows (joint limits, lambda >= 0 ⟂ v >= 0) enter r_contact through the natural map;
    regularised rows need v = 0 and rigid bilateral rows v = 0 on the range of J (r_bilateral)."""
    v = J @ u_plus + v_star
    if reg is not None:
        v = v + reg * lam
    vs = p * v
    ls = lam / p
    mus = np.array(mu, dtype=np.float64)
    for k in range(len(mu)):
        i = n_bilateral + 3 * k
        mus[k] = mu[k] * p[i + 2] / p[i]
    r_c = 0.0
    if len(mu):
        w = vs + PA.desaxce(vs, n_bilateral, mus)
        nat = ls - PA.project_cone(ls - w, n_bilateral, mus)
        r_c = float(np.max(np.abs(nat[n_bilateral:])))
    uni = np.zeros(len(lam), bool)
    uni[list(unilateral)] = True
    if uni.any():
        nat = ls[uni] - np.maximum(ls[uni] - vs[uni], 0.0)
        r_c = max(r_c, float(np.max(np.abs(nat))))
    soft = np.zeros(len(lam), bool) if reg is None else reg > 0
    rigid = np.zeros(len(lam), bool)
    rigid[:n_bilateral] = True
    rigid &= ~uni & ~soft
    r_b = float(np.max(np.abs(vs[soft]))) if soft.any() else 0.0
    if rigid.any():
        Jb = p[rigid, None] * J[rigid]
        U, S, _ = np.linalg.svd(Jb, full_matrices=False)
        rank = int(np.sum(S > S.max() * 1e-10)) if S.size else 0
        Q = U[:, :rank]
        r_b = max(r_b, float(np.max(np.abs(Q @ (Q.T @ vs[rigid])))))
    return r_c, r_b


def null_space_bias(J, v_star, p, n_bilateral):
    """Size of the part of the scaled bilateral bias that no velocity can produce (the residual
    floor of redundant loops): ||(I - Q Q^T) P v*_b||_inf with Q a basis of range(P J_b)."""
    if not n_bilateral:
        return 0.0
    Jb = p[:n_bilateral, None] * J[:n_bilateral]
    U, S, _ = np.linalg.svd(Jb, full_matrices=False)
    rank = int(np.sum(S > S.max() * 1e-10))
    Q = U[:, :rank]
    b = p[:n_bilateral] * v_star[:n_bilateral]
    return float(np.max(np.abs(b - Q @ (Q.T @ b))))
