"""Hartree and LDA exchange-correlation potentials from rho on the grid (FP64, numpy).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

V in Eq. 2 has three parts: the atoms' local pseudopotentials, the
electrostatic (Hartree) potential of rho, and the exchange-correlation
potential (Section 2.2, the text after Eq. 2).  This module writes out the two parts that follow from
rho alone, as plain definitions, so that a rho -> V -> H^V loop can be closed
(the pseudopotential part needs data this work does not have):

  hartree(rho, cell)  V_H with  lap V_H = -4 pi (rho - mean rho)  on the periodic
                      grid, solved in reciprocal space (numpy's FFT as a step):
                      V_H(G) = 4 pi rho(G) / |G|^2, V_H(G = 0) = 0 (a neutralising
                      background); E_H = 1/2 sum_g rho_g V_H,g dV.
  lda_xc(rho)         Slater exchange and the Perdew-Zunger (1981) fit of the
                      Ceperley-Alder correlation energy, spin unpolarised, in
                      hartree: per point eps_xc (energy per electron) and
                      v_xc = d(rho eps_xc)/d rho.  The paper does not name its
                      functional; LDA is the reading taken here.  Points with
                      rho <= 0 (a seeded, non-physical D can give them) get
                      eps_xc = v_xc = 0.

Grid convention as everywhere: r_g = sum_i (g_i / n_i) a_i, C order
[n1][n2][n3], dV = Omega / (n1 n2 n3); cell rows are a1, a2, a3 (bohr).
"""
from __future__ import annotations

import numpy as np

# Perdew-Zunger (1981), unpolarised: rs >= 1 and rs < 1 branches (hartree)
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def reciprocal_vectors(cell):
    """Rows b_j with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(cell, dtype=np.float64)).T


def g_squared(shape, cell):
    """|G|^2 on numpy's FFT grid: G = sum_i m_i b_i with m_i the FFT frequencies of axis i."""
    b = reciprocal_vectors(cell)
    m = np.meshgrid(*[np.fft.fftfreq(n, 1.0 / n) for n in shape], indexing="ij")
    gx = m[0] * b[0, 0] + m[1] * b[1, 0] + m[2] * b[2, 0]
    gy = m[0] * b[0, 1] + m[1] * b[1, 1] + m[2] * b[2, 1]
    gz = m[0] * b[0, 2] + m[1] * b[1, 2] + m[2] * b[2, 2]
    return gx * gx + gy * gy + gz * gz


def hartree(rho, cell):
    """(V_H, E_H) of the periodic density rho [n1][n2][n3] (electrons per bohr^3)."""
    rho = np.asarray(rho, dtype=np.float64)
    omega = abs(np.linalg.det(np.asarray(cell, dtype=np.float64)))
    dv = omega / rho.size
    g2 = g_squared(rho.shape, cell)
    rg = np.fft.fftn(rho)
    vg = np.zeros_like(rg)
    nz = g2 > 0.0
    vg[nz] = 4.0 * np.pi * rg[nz] / g2[nz]
    v = np.fft.ifftn(vg).real
    e = 0.5 * float(np.sum(rho * v)) * dv
    return v, e


def wigner_seitz_radius(rho):
    """rs = (3 / (4 pi rho))^(1/3) for rho > 0."""
    return (3.0 / (4.0 * np.pi * rho)) ** (1.0 / 3.0)


def lda_exchange(rs):
    """Slater exchange: eps_x = -(3/4) (3/pi)^(1/3) rho^(1/3) = -(3/4) (9/(4 pi^2))^(1/3) / rs; v_x = 4/3 eps_x."""
    ex = -0.75 * (9.0 / (4.0 * np.pi * np.pi)) ** (1.0 / 3.0) / rs
    return ex, 4.0 / 3.0 * ex


def pz81_correlation(rs):
    """Perdew-Zunger (1981) correlation per electron and its potential v_c = eps_c - (rs/3) d eps_c/d rs."""
    rs = np.asarray(rs, dtype=np.float64)
    ec = np.empty_like(rs)
    vc = np.empty_like(rs)
    hi = rs >= 1.0
    r = rs[hi]
    sq = np.sqrt(r)
    den = 1.0 + PZ_BETA1 * sq + PZ_BETA2 * r
    ec[hi] = PZ_GAMMA / den
    vc[hi] = ec[hi] * (1.0 + 7.0 / 6.0 * PZ_BETA1 * sq + 4.0 / 3.0 * PZ_BETA2 * r) / den
    r = rs[~hi]
    lr = np.log(r)
    ec[~hi] = PZ_A * lr + PZ_B + PZ_C * r * lr + PZ_D * r
    vc[~hi] = PZ_A * lr + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * r * lr + (2.0 * PZ_D - PZ_C) / 3.0 * r
    return ec, vc


def lda_xc(rho):
    """(eps_xc, v_xc) per grid point; zero where rho <= 0."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    pos = rho > 0.0
    rs = wigner_seitz_radius(rho[pos])
    ex, vx = lda_exchange(rs)
    ec, vc = pz81_correlation(rs)
    eps[pos] = ex + ec
    v[pos] = vx + vc
    return eps, v
