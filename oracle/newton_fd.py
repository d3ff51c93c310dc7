"""Finite differences of the solution map by re-solving R(z, theta) = 0.

A pin for problems with second-order cone blocks, where no closed form
exists: the solution map theta -> (x, y, s) is evaluated at theta +- h dtheta
by Newton's method on the residual map of eq. (residual-map) (a root z of R
with z_N = 1 gives the optimum through phi, Sec. 2.3-2.4), started from the
root at theta.  Only R is used: the Newton Jacobian is itself a central
finite difference of R, so this pin does not rely on the formula for F.
z_N stays 1 (R is positively homogeneous, so its roots form rays) and the
N equations are solved in least squares over the first N - 1 coordinates.
"""
import numpy as np

from . import embedding as E


def _theta(prob, d, h):
    P = E.P_full(prob) + h * E.sym_from_upper_values(prob, d.dP)
    A = E.A_dense(prob) + h * E.dense_on_A_pattern(prob, d.dA)
    return {"P": P, "A": A, "q": prob.q + h * d.dq, "b": prob.b + h * d.db}


def _jac_fd(fun, z, eps=1e-7):
    N = z.shape[0]
    J = np.empty((N, N - 1))
    for j in range(N - 1):
        e = np.zeros(N)
        e[j] = eps
        J[:, j] = (fun(z + e) - fun(z - e)) / (2 * eps)
    return J


def resolve(prob, theta, z0, tol=1e-14, maxit=30):
    fun = lambda z: E.residual_map(prob, z, theta)
    z = z0.copy()
    for _ in range(maxit):
        r = fun(z)
        if np.linalg.norm(r) <= tol * max(1.0, np.linalg.norm(z)):
            break
        J = _jac_fd(fun, z)
        step = np.linalg.lstsq(J, -r, rcond=None)[0]
        z[:-1] += step
    return z, float(np.linalg.norm(fun(z)))


def jvp_fd(prob, d, h=1e-6):
    """Central difference of phi(z(theta +- h dtheta))."""
    z0 = E.solution_to_z(prob)
    zp, rp = resolve(prob, _theta(prob, d, h), z0)
    zm, rm = resolve(prob, _theta(prob, d, -h), z0)
    out = (E.phi(prob, zp) - E.phi(prob, zm)) / (2 * h)
    n, m = prob.n, prob.m
    return out[:n], out[n:n + m], out[n + m:], {"res_plus": rp, "res_minus": rm}
