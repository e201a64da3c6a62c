"""Oracle test surface: the two-dimensional Mueller-Brown potential.

TEST INFRASTRUCTURE ONLY.  Mueller and Brown, Theor. Chim. Acta 53, 75 (1979):
V(x, y) = sum_k A_k exp[a_k (x-x0_k)^2 + b_k (x-x0_k)(y-y0_k) + c_k (y-y0_k)^2]
with the published constants below.  Used to pin the NEB/CI/FIRE logic of
the oracle on a surface whose saddle points are known.
"""
import numpy as np

A = np.array([-200.0, -100.0, -170.0, 15.0])
a = np.array([-1.0, -1.0, -6.5, 0.7])
b = np.array([0.0, 0.0, 11.0, 0.6])
c = np.array([-10.0, -10.0, -6.5, 0.7])
x0 = np.array([1.0, 0.0, -0.5, -1.0])
y0 = np.array([0.0, 0.5, 1.5, 1.0])


def energy(p):
    x, y = p
    dx, dy = x - x0, y - y0
    return float(np.sum(A * np.exp(a * dx * dx + b * dx * dy + c * dy * dy)))


def gradient(p):
    x, y = p
    dx, dy = x - x0, y - y0
    ex = A * np.exp(a * dx * dx + b * dx * dy + c * dy * dy)
    return np.array([np.sum(ex * (2 * a * dx + b * dy)), np.sum(ex * (b * dx + 2 * c * dy))])


def image(X):
    """Band image function: (E, force = -grad, info)."""
    X = np.asarray(X, dtype=np.float64)
    return energy(X), -gradient(X), {}
