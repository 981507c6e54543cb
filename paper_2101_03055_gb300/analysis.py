"""Heat and mass transfer of the double-diffusive cavity (Sec. 3.2).

Local Nusselt and Sherwood numbers on the hot, high-concentration wall x = 0:
Nu(y) = -(dT/dx + D_CT dC/dx), Sh(y) = -(S_TC dT/dx + dC/dx), with the sign
chosen so that heat leaving the hot wall counts positive (the paper prints the
derivatives without it), and their averages over the wall, (1/A) int Nu dy.
The wall derivative is the second-order one-sided (upwind) difference through
the wall value and the first two nodes, which sit half a spacing and one and a
half spacings from the half-way wall: q'(0) = (9 q_1 - q_2 - 8 q_w) / (3 dx).
Lengths are scaled by the cavity width L, so dx = 1 / nx.
"""
from __future__ import annotations

import numpy as np


def wall_derivative(q1, q2, qw, dx):
    return (9.0 * q1 - q2 - 8.0 * qw) / (3.0 * dx)


def nusselt_sherwood(M, D_CT: float, S_TC: float, T_wall: float = 1.0, C_wall: float = 1.0, east: bool = False):
    """Average Nu and Sh (flux in +x) on the west wall, or on the east wall, of a moment stack [T, C, u_x, u_y, p][ny][nx]; returns (Nu, Sh, Nu(y), Sh(y))."""
    T, C = M[0], M[1]
    nx = T.shape[1]
    dx = 1.0 / nx
    if east:
        dT = -wall_derivative(T[:, -1], T[:, -2], T_wall, dx)
        dC = -wall_derivative(C[:, -1], C[:, -2], C_wall, dx)
    else:
        dT = wall_derivative(T[:, 0], T[:, 1], T_wall, dx)
        dC = wall_derivative(C[:, 0], C[:, 1], C_wall, dx)
    Nu_y = -(dT + D_CT * dC)  # the flux in +x: out of the hot wall, into the cold wall
    Sh_y = -(S_TC * dT + dC)
    return float(Nu_y.mean()), float(Sh_y.mean()), Nu_y, Sh_y
