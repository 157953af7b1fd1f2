"""Brute-force dense Tikhonov solve of the discretised tomography problem.

An independent route to what SAFR computes, used only to pin the oracle on
tiny grids.  Everything is built in the spatial domain from the problem
statement, without the per-frequency factorisation:

* unknowns: the L layers sampled on their own grids x^l_p = c_l x_p (Section 3.2),
  each the band-limited (|n| <= M/2-1) trigonometric interpolant of its samples;
* forward model (Section 2, Eq. defAperonly): star g sees
  sum_l phi_l(c_l x_p + alpha_g h_l), i.e. layer l read at the fractional
  layer index p + alpha_g h_l / (c_l delta), evaluated with the Nyquist-free
  Dirichlet kernel K(t) = (1 + 2 sum_{n=1}^{M/2-1} cos(2 pi n t / M)) / M;
* data term: right-rectangle quadrature of the L2(Omega_T) norm over the full
  zero-padded M x M grid (Appendix A), i.e. a plain sum of squares;
* penalty: the H^beta(c_l Omega_T, gamma_l) norm of Section 2/3.1, which on the
  samples is (c_l^2 / gamma_l) M^-2 sum_n (1 + tau_l |n|^2)^beta |DFT2(phi_l)(n)|^2
  with tau_l = pi^2 / (c_l T)^2, written here as a cosine kernel in the sample
  differences;
* minimiser of  sum_g ||A_g phi - Psi_g||^2 + alpha sum_l ||phi_l||^2_{H^beta}
  from the normal equations, solved densely in FP64.
"""
from __future__ import annotations

import math

import numpy as np


def dirichlet(t: np.ndarray, M: int) -> np.ndarray:
    n = np.arange(1, M // 2)
    return (1.0 + 2.0 * np.cos(2.0 * math.pi * np.multiply.outer(t, n) / M).sum(-1)) / M


def cone_coeffs(h, h_lgs, lgs):
    h = np.asarray(h, np.float64)
    return 1.0 - h / h_lgs if lgs else np.ones_like(h)


def forward_operator(M, pitch, h, dirs_x, dirs_y, c):
    """Dense (G M^2) x (L M^2) operator, rows (g,p,q), columns (l,a,b)."""
    G, L = len(dirs_x), len(h)
    idx = np.arange(M, dtype=np.float64)
    A = np.zeros((G * M * M, L * M * M))
    for g in range(G):
        for l in range(L):
            sx = dirs_x[g] * h[l] / (c[l] * pitch)
            sy = dirs_y[g] * h[l] / (c[l] * pitch)
            Kx = dirichlet(idx[:, None] + sx - idx[None, :], M)
            Ky = dirichlet(idx[:, None] + sy - idx[None, :], M)
            A[g * M * M:(g + 1) * M * M, l * M * M:(l + 1) * M * M] = np.kron(Kx, Ky)
    return A


def penalty_operator(M, pitch, c, gamma, beta):
    """Dense (L M^2)^2 block-diagonal H^beta Gram matrix on the layer samples."""
    T = M * pitch / 2.0
    L = len(c)
    j = np.arange(M)
    lab = np.where(j < M // 2, j, j - M).astype(np.float64)  # label of the Nyquist bin: -M/2
    nx, ny = np.meshgrid(lab, lab, indexing="ij")
    d = np.arange(M)
    DA = (d[:, None] - d[None, :]) % M
    R = np.zeros((L * M * M, L * M * M))
    for l in range(L):
        tau = math.pi ** 2 / (c[l] * T) ** 2
        w = (1.0 + tau * (nx ** 2 + ny ** 2)) ** beta
        kern = np.empty((M, M))
        for dx in range(M):
            for dy in range(M):
                kern[dx, dy] = (w * np.cos(2.0 * math.pi * (nx * dx + ny * dy) / M)).sum() / M ** 2
        # block[(a,b),(a',b')] = kern[(a-a') mod M, (b-b') mod M]
        blk = kern[DA[:, None, :, None], DA[None, :, None, :]].reshape(M * M, M * M)
        R[l * M * M:(l + 1) * M * M, l * M * M:(l + 1) * M * M] = (c[l] ** 2 / gamma[l]) * blk
    return R


def solve(M, pitch, h, cn2, dirs_x, dirs_y, lgs, h_lgs, alpha, beta, psi_padded):
    """Layers [L][M][M] (native grids) minimising the Tikhonov functional."""
    gamma = np.asarray(cn2, np.float64) / np.sum(cn2)
    c = cone_coeffs(h, h_lgs, lgs)
    A = forward_operator(M, pitch, h, dirs_x, dirs_y, c)
    R = penalty_operator(M, pitch, c, gamma, beta)
    H = A.T @ A + alpha * R
    phi = np.linalg.solve(H, A.T @ np.asarray(psi_padded, np.float64).ravel())
    return phi.reshape(len(h), M, M), A, R
