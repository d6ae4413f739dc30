"""Exact periodic solutions of the viscous Burgers' equation u_t + u u_x = alpha u_xx by the Cole-Hopf transform:
u = -2 alpha phi_x / phi with phi_t = alpha phi_xx,  phi = 1 + sum_m a_m cos(m x + theta_m) exp(-alpha m^2 t)
(sum |a_m| < 1 keeps phi > 0).  A test helper: the reference against which Burgers runs converge."""
import numpy as np

A = (0.3, 0.2, 0.15)
M = (1, 2, 3)
THETA = (0.4, 2.0, 4.1)


def cole_hopf(n: int, t: float, alpha: float, a=A, m=M, theta=THETA) -> np.ndarray:
    x = 2.0 * np.pi * np.arange(n) / n
    phi = 1.0 + sum(ai * np.cos(mi * x + ti) * np.exp(-alpha * mi * mi * t) for ai, mi, ti in zip(a, m, theta))
    dphi = -sum(ai * mi * np.sin(mi * x + ti) * np.exp(-alpha * mi * mi * t) for ai, mi, ti in zip(a, m, theta))
    return -2.0 * alpha * dphi / phi
