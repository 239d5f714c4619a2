"""Dual problem and Proximal-ADMM (Sec. 4: Eq. 3, Eq. 4, Alg. 1 and Sec. 4.1), FP64.

Test infrastructure only (see ``oracle/__init__``).

Conventions.  Constraint rows are the joint rows (bilateral; regularised drive rows; unilateral
joint-limit rows, listed in ``unilateral``) followed by one (t1, t2, n) triple per active contact;
``n_bilateral`` counts every row before the contacts.  ``cone_mu[k]`` is the friction coefficient of contact k.  All iterates live in
the Jacobi-scaled space of Sec. 4.1: x~ = P^-1 x, v~ = P v, D~ = P D P.  The two tangential
rows of a contact share one scale so the cone stays circular with mu~ = mu p_n / p_t.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.linalg import solve_triangular


# ----------------------------------------------------------------------------- Eq. 4
def delassus(J, Minv, R=None):
    """Eq. 4: D = J M^-1 J^T + R, R the diagonal regularisation of the joint-space dynamics rows
    (a vector, or None for none)."""
    D = J @ Minv @ J.T
    return D if R is None else D + np.diag(R)


def delassus_matrix_free(J, Minv, p, R=None):
    """Sec. 5.1's sparse formulation: the scaled Delassus operator v -> P (J M^-1 J^T + R) P v as
    the chain of products with J^T, M^-1 and J, without forming D."""
    def apply(v):
        out = p * (J @ (Minv @ (J.T @ (p * v))))
        return out if R is None else out + p * R * p * v
    return apply


def delassus_diagonal(J, Minv, R=None):
    """diag(D) of Eq. 4 row by row, d_r = J_r M^-1 J_r^T + R_r, without forming D."""
    d = np.array([J[r] @ Minv @ J[r] for r in range(J.shape[0])])
    return d if R is None else d + R


def free_velocity(J, u_free, v_star):
    """Eq. 4: v_f = J (u^- + dt M^-1 h) + v*, with u_free = u^- + dt M^-1 h."""
    return J @ u_free + v_star


def jacobi_scaling(D, n_bilateral, n_contacts, precond=True):
    """Sec. 4.1: P = diag(D)^-1/2, once per step.  Tangential rows of a contact share
    p_t = ((D_t1t1 + D_t2t2) / 2)^-1/2 so that the scaled friction cone stays a circular cone.
    ``D`` is the Delassus matrix or, for the matrix-free path, its diagonal as a vector."""
    m = D.shape[0]
    if not precond:
        return np.ones(m)
    d = (np.diag(D) if D.ndim == 2 else D).copy()
    p = 1.0 / np.sqrt(d)
    for k in range(n_contacts):
        i = n_bilateral + 3 * k
        pt = 1.0 / math.sqrt(0.5 * (d[i] + d[i + 1]))
        p[i] = p[i + 1] = pt
    return p


# ----------------------------------------------------------------------------- cones
def desaxce(v, n_bilateral, mu):
    """De Saxce operator (Sec. 4, Eq. 3): Gamma(v)_k = (0, 0, mu_k ||v_k,t||) on every contact
    triple (t1, t2, n), zero on bilateral rows."""
    s = np.zeros_like(v)
    if len(mu):
        vc = v[n_bilateral:].reshape(-1, 3)
        s[n_bilateral + 2::3] = np.asarray(mu) * np.hypot(vc[:, 0], vc[:, 1])
    return s


def project_cone(x, n_bilateral, mu, unilateral=None):
    """Projection onto K = R^(bilateral) x prod_k K_mu_k, K_mu = {(t, n): ||t|| <= mu n}: the
    closed-form Euclidean projection onto a second-order cone, contact by contact:
    inside K -> unchanged; inside the polar cone (mu ||t|| <= -n) -> 0; otherwise onto the
    boundary ray, n' = (mu ||t|| + n) / (1 + mu^2), t' = mu n' t / ||t||.
    ``unilateral`` lists rows before the contacts whose set is the ray R+ (joint limits, Sec. 3):
    they are clamped at zero."""
    y = x.copy()
    if unilateral is not None and len(unilateral):
        y[unilateral] = np.maximum(x[unilateral], 0.0)
    if not len(mu):
        return y
    mu = np.asarray(mu, dtype=np.float64)
    xc = x[n_bilateral:].reshape(-1, 3)
    yc = y[n_bilateral:].reshape(-1, 3)
    tn = np.hypot(xc[:, 0], xc[:, 1])
    n = xc[:, 2]
    inside = tn <= mu * n
    polar = (~inside) & (mu * tn <= -n)
    side = ~(inside | polar)
    yc[polar] = 0.0
    nn = (mu * tn + n) / (1.0 + mu * mu)
    scale = np.where(side, mu * nn / np.where(tn > 0, tn, 1.0), 0.0)
    yc[side, 0] = scale[side] * xc[side, 0]
    yc[side, 1] = scale[side] * xc[side, 1]
    yc[side, 2] = nn[side]
    return y


# ----------------------------------------------------------------------------- Alg. 1
@dataclass
class PadmmResult:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    iterations: int
    r_p: float
    r_d: float
    r_c: float
    converged: bool
    restarts: int


def residuals(x, x_prev, y, y_hat_prev, z, eta, rho, n_bilateral, n_contacts, lin_res=None, unilateral=None):
    """Infinity-norm residuals of Sec. 4.1.  Primal: x - y.  Dual: the deviation of the x-step's
    stationarity condition once the new iterates are substituted,
    eta (x^i - x^{i-1}) + rho (y^i - y^_{i-1}).  Complementarity: max over contacts |y_k . z_k|.

    ``lin_res`` is the residual A x^i + b^i that an inexact x-step left (Conjugate Residual); the
    dual residual then subtracts it, which makes it D x + v_f + Gamma - z, the stationarity of the
    dual problem at the new iterates (the exact x-step has lin_res = 0 and the formula above).
    Unilateral rows (joint limits) add |y_i z_i| to the complementarity residual."""
    r_p = float(np.max(np.abs(x - y))) if x.size else 0.0
    dev = eta * (x - x_prev) + rho * (y - y_hat_prev)
    if lin_res is not None:
        dev = dev - lin_res
    r_d = float(np.max(np.abs(dev))) if x.size else 0.0
    r_c = 0.0
    if n_contacts:
        yc = y[n_bilateral:].reshape(-1, 3)
        zc = z[n_bilateral:].reshape(-1, 3)
        r_c = float(np.max(np.abs(np.sum(yc * zc, axis=1))))
    if unilateral is not None and len(unilateral):
        r_c = max(r_c, float(np.max(np.abs(y[unilateral] * z[unilateral]))))
    return r_p, r_d, r_c


def conjugate_residual(apply_A, c, x0, iters):
    """Conjugate Residual iterations for A x = c with A symmetric (Sec. 5.1 pairs it with the
    matrix-free Delassus operator; the method is the textbook one, e.g. Saad, "Iterative Methods
    for Sparse Linear Systems", Sec. 6.8).  From x0, each iteration takes the step along the search
    direction p that minimises ||c - A x||_2, then makes the next direction A-orthogonal in the
    A^2 inner product:
      r0 = c - A x0, p0 = r0
      alpha_j = (r_j, A r_j) / (A p_j, A p_j);  x_{j+1} = x_j + alpha_j p_j;  r_{j+1} = r_j - alpha_j A p_j
      beta_j  = (r_{j+1}, A r_{j+1}) / (r_j, A r_j);  p_{j+1} = r_{j+1} + beta_j p_j,
    with A p_{j+1} = A r_{j+1} + beta_j A p_j, so one operator application per iteration.  Runs
    ``iters`` iterations (a fixed budget), fewer only if the residual vanishes exactly."""
    x = np.array(x0, dtype=np.float64)
    r = c - apply_A(x)
    Ar = apply_A(r)
    p, Ap = r.copy(), Ar.copy()
    rAr = float(r @ Ar)
    for _ in range(iters):
        ApAp = float(Ap @ Ap)
        if rAr == 0.0 or ApAp == 0.0:
            break
        alpha = rAr / ApAp
        x = x + alpha * p
        r = r - alpha * Ap
        Ar = apply_A(r)
        rAr_next = float(r @ Ar)
        beta = rAr_next / rAr
        rAr = rAr_next
        p = r + beta * p
        Ap = Ar + beta * Ap
    return x


def nesterov_coefficient(a):
    """Sec. 4.1's Nesterov step (Goldstein et al. 2014): the next momentum parameter
    a' = (1 + sqrt(1 + 4 a^2)) / 2 and the extrapolation weight (a - 1) / a'."""
    a_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * a * a))
    return a_next, (a - 1.0) / a_next


def padmm(D, v_f, n_bilateral, mu, eta, rho, eps, n_max, x0=None, z0=None, nesterov=True,
          restart_factor=0.999, cr_iters=None, unilateral=None):
    """Alg. 1 (one time step), on an already scaled problem (D, v_f, mu).

    Steps per iteration i (hats are the Nesterov-extrapolated iterates, equal to the plain ones
    without acceleration):
      s^i  = Gamma(z^_{i-1})
      x^i  = -(D + (eta + rho) I)^-1 (v_f + s^i - eta x^{i-1} - rho y^_{i-1} - z^_{i-1})
      y^i  = Pi_K(x^i - z^_{i-1} / rho)
      z^i  = z^_{i-1} - rho (x^i - y^i)
      Nesterov with adaptive restart (O'Donoghue & Candes; Fast ADMM of Goldstein et al. 2014):
      c^i = ||z^i - z^_{i-1}||^2 / rho + rho ||y^i - y^_{i-1}||^2; if c^i < 0.999 c^{i-1} then
      a' = (1 + sqrt(1 + 4 a^2)) / 2 and (y^, z^) = (y, z)^i + (a - 1)/a' ((y, z)^i - (y, z)^{i-1}),
      otherwise a = 1, (y^, z^) = (y, z)^{i-1} and c^i = c^{i-1} / 0.999.
      stop when r_p, r_d, r_c < eps.
    The factorisation of D + (eta + rho) I is computed once (Sec. 4: the left-hand side is
    constant across iterations).  Returns y^N as lambda~.

    With ``cr_iters`` set, ``D`` is the matrix-free operator v -> D v instead (Sec. 5.1's sparse
    formulation) and the x-step is ``cr_iters`` Conjugate Residual iterations on
    (D + (eta + rho) I) x = -b started from the previous iterate x^{i-1}; the dual residual then
    includes what the x-step left of that system (see ``residuals``).
    """
    n_contacts = len(mu)
    if cr_iters is None:
        m = D.shape[0]
        A = D + (eta + rho) * np.eye(m)
        L = np.linalg.cholesky(A) if m else np.zeros((0, 0))

        def solve_x(b, x_prev):
            t = _forward(L, b)
            return -_backward(L, t)
    else:
        m = v_f.shape[0]

        def apply_A(v):
            return D(v) + (eta + rho) * v

        def solve_x(b, x_prev):
            return conjugate_residual(apply_A, -b, x_prev, cr_iters)

    x = np.zeros(m) if x0 is None else x0.copy()
    y = x.copy()
    z = np.zeros(m) if z0 is None else z0.copy()
    y_hat, z_hat = y.copy(), z.copy()
    a = 1.0
    c_prev = math.inf
    it = 0
    r_p = r_d = r_c = math.inf
    converged = False
    restarts = 0
    for it in range(1, n_max + 1):
        s = desaxce(z_hat, n_bilateral, mu)
        b = v_f + s - eta * x - rho * y_hat - z_hat
        x_new = solve_x(b, x)
        y_new = project_cone(x_new - z_hat / rho, n_bilateral, mu, unilateral)
        z_new = z_hat - rho * (x_new - y_new)
        lin_res = None if cr_iters is None else apply_A(x_new) + b
        r_p, r_d, r_c = residuals(x_new, x, y_new, y_hat, z_new, eta, rho, n_bilateral, n_contacts, lin_res,
                                  unilateral)
        if nesterov:
            c = float(np.dot(z_new - z_hat, z_new - z_hat) / rho + rho * np.dot(y_new - y_hat, y_new - y_hat))
            if c < restart_factor * c_prev:
                a_next, beta = nesterov_coefficient(a)
                y_hat_next = y_new + beta * (y_new - y)
                z_hat_next = z_new + beta * (z_new - z)
                a = a_next
                c_prev = c
            else:
                restarts += 1
                a = 1.0
                y_hat_next, z_hat_next = y.copy(), z.copy()
                c_prev = c_prev / restart_factor
        else:
            y_hat_next, z_hat_next = y_new, z_new
        x, y, z = x_new, y_new, z_new
        y_hat, z_hat = y_hat_next, z_hat_next
        if r_p < eps and r_d < eps and r_c < eps:
            converged = True
            break
    return PadmmResult(x=x, y=y, z=z, iterations=it, r_p=r_p, r_d=r_d, r_c=r_c, converged=converged,
                       restarts=restarts)


def _forward(L, b):
    """Solve L t = b (forward substitution; library triangular solve)."""
    return solve_triangular(L, b, lower=True, check_finite=False)


def _backward(L, t):
    """Solve L^T x = t (backward substitution; library triangular solve)."""
    return solve_triangular(L, t, lower=True, trans="T", check_finite=False)
