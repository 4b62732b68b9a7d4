"""Local thermostat (Appendix C): oracle.

TEST INFRASTRUCTURE ONLY (tests/, __graft_entry__.smoke(), bench.py's CPU legs).

When the switching parameters change from lambda^c (the conservative reference:
the values of the previous step) to lambda^d (the updated values), the applied
force F^d of Eq. F_i_d neglects grad lambda and the energy is not conserved.
Appendix C measures the error per atom at the end of the step and corrects it
by rescaling relative momenta of a group of atoms:

  Delta V_i = (lambda_i^c - lambda_i^d) (E_i^(f) - E_i^(p))                  (Eq. Delta_V_i)
  Delta T_i = sum_a [ dt^2/(8 m_i) (F^c_ia^2 - F^d_ia^2) + (F^c_ia - F^d_ia) v_ia(t+dt/2) dt/2 ]
                                                                              (Eq. Delta_T_i)
  Delta E_i = Delta T_i + Delta V_i                                          (Eq. Delta_E_i)
  p_j <- m_j v_cm(Omega_i) + beta p_rel,j,  beta = sqrt(Delta E_i / sum_j p_rel,j^2/(2 m_j) + 1)
                                                          (Eqs. p_resc_omega, beta_omega_i)

F^c and F^d are the interatomic forces only (no external force).  Units: eV, A,
fs, amu; velocities in A/fs, so a kinetic energy is m v^2 / (2 ACC).

Readings (the paper leaves them open):
  * Omega_i = {i} plus every distinct mobile atom of i's neighbour row (all images
    within r_row = r_EAM + skin at the positions of the step); the paper draws at
    most 800 atoms at random from the neighbour list, and these rows are shorter,
    so every row atom is taken and no draw is needed.  Members in the order i,
    then ascending index.
  * Order of the corrections: beta depends on the momenta before the rescaling,
    so corrections that share atoms do not commute.  They are applied in the
    sub-domain order the paper calls for but does not specify: the box is cut
    into cells of edge >= 2 (r_row + skin) (an even number along every periodic
    dimension, or one), the cells are swept in 8 colours (the parities of the
    cell coordinates, colour = px + 2 py + 4 pz), cells of one colour in
    ascending cell id (x fastest), atoms of a cell in ascending index.  Two atoms
    in different cells of one colour are at least one cell apart, so their groups
    are disjoint and the order among them does not matter.
  * Atoms with Delta E_i = 0 (exactly) or fixed atoms get no correction.  A
    negative radicand leaves the velocities unchanged and is reported.
"""
from __future__ import annotations

import numpy as np

from . import ACC, neighbors as _neighbors


def delta_v(lam_c, lam_d, e_fast, e_prec) -> np.ndarray:
    """Eq. Delta_V_i."""
    return (np.asarray(lam_c) - np.asarray(lam_d)) * (np.asarray(e_fast) - np.asarray(e_prec))


def delta_t(f_c, f_d, v_half, mass, dt: float) -> np.ndarray:
    """Eq. Delta_T_i (the kinetic-energy difference at the end of the step between
    the two forces, from the half-step velocity)."""
    f_c, f_d, v_half = (np.asarray(a, float) for a in (f_c, f_d, v_half))
    m = np.asarray(mass, float)[:, None]
    a = dt * dt * ACC / (8.0 * m) * (f_c * f_c - f_d * f_d) + (f_c - f_d) * v_half * (0.5 * dt)
    return a.sum(1)


def thermostat_cells(x, box, r_row: float, skin: float):
    """Cell coordinates (n, 3) and counts (3,) of the correction sweep."""
    x = np.asarray(x, float)
    L = np.asarray(box.hi, float) - np.asarray(box.lo, float)
    h_min = 2.0 * (r_row + skin)
    nc = np.maximum(1, np.floor(L / h_min).astype(int))
    for d in range(3):
        if box.periodic[d] and nc[d] > 1 and nc[d] % 2 == 1:
            nc[d] -= 1
    s = x - np.asarray(box.lo, float)
    for d in range(3):
        if box.periodic[d]:
            s[:, d] = np.mod(s[:, d], L[d])
    c = np.floor(s / (L / nc)).astype(int)
    c = np.clip(c, 0, nc - 1)
    return c, nc


def correction_order(x, box, r_row: float, skin: float, candidates) -> list:
    """The atoms of `candidates` in the order the corrections are applied."""
    c, nc = thermostat_cells(x, box, r_row, skin)
    cand = np.asarray(sorted(int(i) for i in candidates), int)
    if cand.size == 0:
        return []
    cc = c[cand]
    color = (cc[:, 0] & 1) + 2 * (cc[:, 1] & 1) + 4 * (cc[:, 2] & 1)
    cid = (cc[:, 2] * nc[1] + cc[:, 1]) * nc[0] + cc[:, 0]
    order = np.lexsort((cand, cid, color))
    return cand[order].tolist()


def rescale_group(v, mass, omega, dE: float):
    """Eqs. p_resc_omega and beta_omega_i on the atoms omega (in place); returns
    (beta, ok).  ok is False (and v unchanged) for a negative radicand."""
    m = np.asarray(mass, float)[omega]
    vv = v[omega]
    vcm = (m[:, None] * vv).sum(0) / m.sum()
    rel = vv - vcm
    krel = float((0.5 * m * (rel * rel).sum(1)).sum() / ACC)
    # zero relative kinetic energy can absorb no change: a failure unless dE == 0
    rad = dE / krel + 1.0 if krel > 0 else (1.0 if dE == 0 else -1.0)
    if rad < 0:
        return float("nan"), False
    beta = float(np.sqrt(rad))
    v[omega] = vcm + beta * rel
    return beta, True


def groups(x, box, r_row: float, fixed=None) -> list:
    """Omega_i for every atom: i, then the distinct mobile atoms within r_row (all images), ascending."""
    nl = _neighbors(x, box, r_row)
    n = np.asarray(x).shape[0]
    out = []
    for i in range(n):
        js = sorted({int(j) for j in nl.j[i, :int(nl.cnt[i])]} - {i})
        if fixed is not None:
            js = [j for j in js if not fixed[j]]
        out.append([i] + js)
    return out


def correct(x, box, v_end, mass, dE, r_row: float, skin: float, fixed=None):
    """Apply the corrections of Delta E (per atom) to the end-of-step velocities.
    Returns (v_corrected, n_corrected, n_negative_radicand)."""
    v = np.array(v_end, float, copy=True)
    dE = np.asarray(dE, float)
    fx = np.zeros(len(dE), bool) if fixed is None else np.asarray(fixed) != 0
    cand = [i for i in range(len(dE)) if dE[i] != 0.0 and not fx[i]]
    om = groups(x, box, r_row, fx)
    n_ok = n_bad = 0
    for i in correction_order(x, box, r_row, skin, cand):
        _, ok = rescale_group(v, mass, om[i], float(dE[i]))
        n_ok += ok
        n_bad += not ok
    return v, n_ok, n_bad
