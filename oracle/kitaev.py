"""Kitaev honeycomb model in its Majorana / Z2-gauge form (Sec. IV, Eqs. 15-16).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Lattice reading (the paper fixes only that eta lives on z-bonds, Eq. 16, and
that both directions are periodic in its proof of concept, Sec. IV):
unit cells r = (i, j) in Z_L^2, each with one black site b(r) and one white
site w(r), index b(r) = w(r) = i*L + j.  Bonds: z: b(r)-w(r) with u = eta_r;
x: b(r)-w(r+e1), e1 = (1,0); y: b(r)-w(r+e2), e2 = (0,1); u = +1 on x and y
(a fixed gauge).  The CRBM's visible unit v_ij is (eta_ij + 1) / 2.

With H = (i/4) sum A_jk c_j c_k and c^2 = 1, Eq. (16) gives A_bw = -2 J_a u_bw.
The single-fermion energies eps_l >= 0 are the positive eigenvalues of iA,
i.e. the singular values of the N x N block M_bw = 2 J_a u_bw.  The paper's
configuration free energy F(eta) = -T sum_l log 2cosh(beta eps_l / 2) gives the
target log-weight log pi(eta) = -beta F(eta) = sum_l log 2cosh(beta eps_l / 2).
"""
from __future__ import annotations

import numpy as np


def hopping_matrix(v, J, open_cols=False):
    """M(eta) per chain: (C, N, N) FP64 with M[b(r), w(r)] = 2 Jz eta_r,
    M[b(r), w(r+e1)] = 2 Jx, M[b(r), w(r+e2)] = 2 Jy (entries add if bonds coincide).
    open_cols: the lattice is open along j -- the y-bonds from column L-1 to
    column 0 are absent (a cylinder, periodic along i; the reading of the
    paper's open boundary conditions, Sec. IV)."""
    v = np.asarray(v)
    C, L, _ = v.shape
    N = L * L
    Jx, Jy, Jz = (float(x) for x in J)
    eta = 2.0 * v.astype(np.float64) - 1.0
    M = np.zeros((C, N, N))
    for i in range(L):
        for j in range(L):
            b = i * L + j
            M[:, b, b] += 2.0 * Jz * eta[:, i, j]
            M[:, b, ((i + 1) % L) * L + j] += 2.0 * Jx
            if not (open_cols and j == L - 1):
                M[:, b, i * L + (j + 1) % L] += 2.0 * Jy
    return M


def energies(v, J, open_cols=False):
    """Single-fermion energies eps_l >= 0 (singular values of M, LAPACK), (C, N)."""
    return np.linalg.svd(hopping_matrix(v, J, open_cols), compute_uv=False)


def log2cosh(x):
    """log(2 cosh x) for x >= 0, as x + log1p(e^{-2x})."""
    x = np.abs(x)
    return x + np.log1p(np.exp(-2.0 * x))


def log_weight_from_eps(eps, beta):
    """log pi = sum_l log 2cosh(beta eps_l / 2)   (Sec. IV, text after Eq. 16)."""
    beta = np.asarray(beta, dtype=np.float64).reshape(-1, 1)
    return log2cosh(beta * eps / 2.0).sum(axis=1)


def log_weight(v, beta, J, open_cols=False):
    return log_weight_from_eps(energies(v, J, open_cols), beta)


def thermal_terms(eps, beta):
    """Per-configuration energy e(eta) = -sum (eps/2) tanh(beta eps/2) and fermionic
    heat-capacity term c_f(eta) = sum (beta eps/2)^2 sech^2(beta eps/2).

    Both follow from differentiating ln Z = ln sum_eta prod_l 2cosh(beta eps_l/2)
    with respect to beta:  <E> = <e>,  C = beta^2 (<e^2> - <e>^2) + <c_f>.
    """
    beta = np.asarray(beta, dtype=np.float64).reshape(-1, 1)
    x = beta * eps / 2.0
    e = -(eps / 2.0 * np.tanh(x)).sum(axis=1)
    q = np.exp(-2.0 * np.abs(x))                  # sech^2 x = 4 q / (1 + q)^2
    cf = (x * x * 4.0 * q / (1.0 + q) ** 2).sum(axis=1)
    return e, cf


def vison_density(v, open_cols=False):
    """Fraction of hexagons with flux -1: the hexagon of cell r carries the two
    z-bonds r and r - e1 + e2, so its flux is eta_r * eta_{r-e1+e2}.  With
    open columns the hexagons of column L-1 (which would cross the cut) do not
    exist: L (L-1) hexagons."""
    v = np.asarray(v).astype(np.int64)
    other = np.roll(np.roll(v, 1, axis=1), -1, axis=2)   # v[(i-1) % L, (j+1) % L]
    L = v.shape[1]
    diff = v != other
    if open_cols:
        return diff[:, :, :L - 1].sum(axis=(1, 2)) / float(L * (L - 1))
    return diff.sum(axis=(1, 2)) / float(L * L)


def bloch_energies(L: int, J, eta: float = 1.0):
    """Closed form at uniform eta: eps(k) = 2 |Jz eta + Jx e^{i k1} + Jy e^{i k2}|,
    k = 2 pi (m1, m2) / L -- M is then a 2D circulant diagonalised by plane waves."""
    Jx, Jy, Jz = (float(x) for x in J)
    m = np.arange(L)
    k1, k2 = np.meshgrid(2 * np.pi * m / L, 2 * np.pi * m / L, indexing="ij")
    return np.sort((2.0 * np.abs(Jz * eta + Jx * np.exp(1j * k1) + Jy * np.exp(1j * k2))).ravel())


def majorana_spectrum(v, J, open_cols=False):
    """Eigenvalues of the 2N x 2N Hermitian iA (A_bw = -2 J u_bw, A_wb = -A_bw)."""
    M = hopping_matrix(v, J, open_cols)
    C, N, _ = M.shape
    A = np.zeros((C, 2 * N, 2 * N))
    A[:, :N, N:] = -M
    A[:, N:, :N] = np.transpose(M, (0, 2, 1))
    return np.linalg.eigvalsh(1j * A)
