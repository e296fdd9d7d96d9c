"""Matrix-form brute force of one double-MRT step, for tiny grids.

TEST INFRASTRUCTURE ONLY (used by the oracle pin tests).

A second, independent restatement of Sec. 3 that shares nothing with
``dmrt_oracle.c``: the whole grid is one state vector, streaming is a dense
linear map built from the geometry (an affine map for the thermal lattice,
whose anti-bounce-back adds a constant), and the collisions use dense
matrices from the paper inverted with ``numpy.linalg.inv``.

Matrices come in as arguments so that the caller supplies the paper's
printed values (the test fixtures), with the reading of Eq. 37 applied.
"""
from __future__ import annotations

import math

import numpy as np


def velocities_d2q9():
    """Eq. 23 evaluated with c = 1."""
    e = [(0.0, 0.0)]
    for i in range(2, 6):
        e.append((-math.cos(i * math.pi / 2), -math.sin(i * math.pi / 2)))
    for i in range(6, 10):
        ang = (2 * i + 1) * math.pi / 4
        e.append((-math.sqrt(2) * math.cos(ang), -math.sqrt(2) * math.sin(ang)))
    return np.rint(np.array(e)).astype(int)


def velocities_d2q5():
    """Eq. 35 evaluated with c = 1."""
    e = [(0.0, 0.0)]
    for i in range(2, 6):
        e.append((-math.cos(i * math.pi / 2), -math.sin(i * math.pi / 2)))
    return np.rint(np.array(e)).astype(int)


def _opposite(e):
    return [int(np.nonzero((e == -e[k]).all(axis=1))[0][0]) for k in range(len(e))]


def stream_maps(e, nx, ny, wall_kind):
    """Dense streaming map (P, c) with out = P @ in + c.

    ``wall_kind(side, j) -> (sign, const)`` gives the reflected value
    sign * in[opposite, node] + const for a link leaving through ``side``
    ('left', 'right', 'bottom', 'top').
    Index of (k, j, i) in the state vector: (k * ny + j) * nx + i.
    """
    q = len(e)
    n = q * nx * ny
    P = np.zeros((n, n))
    c = np.zeros(n)
    opp = _opposite(e)

    def idx(k, j, i):
        return (k * ny + j) * nx + i

    for k in range(q):
        for j in range(ny):
            for i in range(nx):
                si, sj = i - e[k][0], j - e[k][1]
                dst = idx(k, j, i)
                if 0 <= si < nx and 0 <= sj < ny:
                    P[dst, idx(k, sj, si)] = 1.0
                else:
                    side = "left" if si < 0 else "right" if si >= nx else "bottom" if sj < 0 else "top"
                    sign, const = wall_kind(side, j)
                    P[dst, idx(opp[k], j, i)] = sign
                    c[dst] = const
    return P, c


class BruteForce:
    def __init__(self, M, N, nx, ny, rates9, rates5, a, gbeta, theta_ref,
                 theta_hot, theta_cold, abb_coef, rho0=1.0):
        self.M = np.asarray(M, dtype=float)
        self.N = np.asarray(N, dtype=float)
        self.Minv = np.linalg.inv(self.M)
        self.Ninv = np.linalg.inv(self.N)
        self.S = np.diag(rates9)
        self.Q = np.diag(rates5)
        self.nx, self.ny = nx, ny
        self.a, self.gbeta, self.theta_ref = a, gbeta, theta_ref
        self.rho0 = rho0
        self.e9 = velocities_d2q9()
        self.e5 = velocities_d2q5()
        self.w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
        self.theta_hot, self.theta_cold = theta_hot, theta_cold
        self.Pf, self.cf = stream_maps(self.e9, nx, ny, lambda side, j: (1.0, 0.0))

        def thermal(side, j):
            if side == "left":
                return (-1.0, abb_coef * theta_hot)
            if side == "right":
                return (-1.0, abb_coef * theta_cold)
            return (1.0, 0.0)

        self.Pg, self.cg = stream_maps(self.e5, nx, ny, thermal)

    def step(self, fs, gs):
        nx, ny = self.nx, self.ny
        f = (self.Pf @ fs.reshape(-1) + self.cf).reshape(9, ny, nx)
        g = (self.Pg @ gs.reshape(-1) + self.cg).reshape(5, ny, nx)
        fo = np.empty_like(f)
        go = np.empty_like(g)
        theta = np.empty((ny, nx))
        cs2 = 1.0 / 3.0
        for j in range(ny):
            for i in range(nx):
                fl = f[:, j, i]
                gl = g[:, j, i]
                drho = fl.sum()
                u = (fl * self.e9[:, 0]).sum() / self.rho0
                v = (fl * self.e9[:, 1]).sum() / self.rho0
                th = gl.sum()
                uu = u * u + v * v
                r0 = self.rho0
                meq = np.array([drho, r0 * u, r0 * v, -2 * drho + 3 * r0 * uu, r0 * (u * u - v * v),
                                r0 * u * v, -r0 * u, -r0 * v, drho - 3 * r0 * uu])
                m = self.M @ fl
                fc = self.Minv @ (m - self.S @ (m - meq))
                G = np.array([0.0, self.gbeta * (th - self.theta_ref)])
                eu = self.e9 @ np.array([u, v])
                feq = self.w9 * r0 * (1 + eu / cs2 + eu ** 2 / (2 * cs2 ** 2) - uu / (2 * cs2))
                F = ((self.e9 - np.array([u, v])) @ G) / (r0 * cs2) * feq
                fo[:, j, i] = fc + F
                neq = np.array([th, u * th, v * th, self.a * th, 0.0])
                n = self.N @ gl
                go[:, j, i] = self.Ninv @ (n - self.Q @ (n - neq))
                theta[j, i] = th
        return fo, go, theta
