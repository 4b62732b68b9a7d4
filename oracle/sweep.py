"""Oracle of the switching-zone parameter study (the paper's appendix on the switching
function: force and energy error against the precise potential as a function of
r_lambda,lo, r_lambda,hi; and its sensitivity study of the CSP thresholds, section 3.3).

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing on the product path).

One study point, as the paper defines it:
- one lambda update with lambda = lambda_min (Eq. lambda_2_i) as the switching
  parameter: one-sample windows (CSP_avg = CSP, lambda_avg = lambda_min) and no
  minimum step, no local thermostat;
- hybrid energies and forces (Eqs. energy_hyb, F_i_d) against the precise potential
  evaluated for every atom;
- atoms whose force has both an EAM and an ACE contribution ("mixed" atoms) grouped
  by CSP_avg; per group the RMSE of the force components and of the site energy.
  Atoms with purely EAM or purely ACE contributions are left out, as the paper does.

An atom i has an EAM contribution when it has a neighbour within the EAM cutoff and
lambda_k > 0 for some k in {i} and its EAM neighbours (the gradient of lambda_k E_k^f
with respect to x_i is nonzero exactly then); likewise an ACE contribution with the
ACE cutoff and 1 - lambda_k > 0.  Only changeable atoms are grouped.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import ACE, LambdaState, classify, eam_any, hybrid, neighbors

CSP_EDGES = (0.0, 0.5, 1.0, 2.0, 3.0, 4.5, 6.0, 8.0, 12.0, 20.0, np.inf)


def one_sample(hyb):
    """The study's switching parameters: lambda = lambda_min after one update."""
    return dataclasses.replace(hyb, n_csp_avg=1, n_lam_avg=1, dlam_min=0.0)


def contributes(x, box, rc: float, weight: np.ndarray) -> np.ndarray:
    """True where x_i enters some weight_k E_k with weight_k > 0 through a pair within rc."""
    nl = neighbors(x, box, rc)
    out = np.zeros(x.shape[0], bool)
    for i in range(x.shape[0]):
        c = int(nl.cnt[i])
        if c == 0:
            continue
        js = nl.j[i, :c]
        out[i] = weight[i] > 0 or bool((weight[js] > 0).any())
    return out


def grouped_rmse(d: np.ndarray, csp: np.ndarray, mask: np.ndarray, edges=CSP_EDGES):
    """(count, RMSE) per CSP group of the rows of d selected by mask; d is (n,) or (n,3)
    (RMSE over the components); NaN for an empty group."""
    d = np.asarray(d, np.float64).reshape(d.shape[0], -1)
    cnt, rmse = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = mask & (csp >= lo) & (csp < hi)
        k = int(m.sum())
        cnt.append(k)
        rmse.append(float(np.sqrt((d[m] ** 2).mean())) if k else float("nan"))
    return np.array(cnt), np.array(rmse)


def reference(x, box, eam_p, ace_p):
    """Precise site energies and forces of every atom, and the fast forces of every atom."""
    e_p, f_p = ACE(ace_p).eval(x, box)
    _, f_f, _, _ = eam_any(x, box, eam_p)
    return e_p, f_p, f_f


def study(x, box, changeable, hyb, eam_p, ace_p, ref=None, edges=CSP_EDGES) -> dict:
    """One study point; ref = reference(...) may be passed to share it between points."""
    n = x.shape[0]
    h = one_sample(hyb)
    st = LambdaState(n, 1, 1)
    lam, lam0, csp_s, csp_avg, lam_min, _ = classify(st, x, box, h, changeable)
    e_h, f_h, _, _ = hybrid(x, box, lam, eam_p, ACE(ace_p))
    e_p, f_p, f_f = ref if ref is not None else reference(x, box, eam_p, ace_p)
    mob = np.asarray(changeable, bool)
    has_f = contributes(x, box, float(eam_p.rc), lam)
    has_p = contributes(x, box, float(ace_p.rc), 1.0 - lam)
    mixed = mob & has_f & has_p
    cnt, f_rmse = grouped_rmse(f_h - f_p, csp_avg, mixed, edges)
    _, e_rmse = grouped_rmse(e_h - e_p, csp_avg, mixed, edges)
    ref_cnt, ref_rmse = grouped_rmse(f_f - f_p, csp_avg, mob, edges)
    d = (f_h - f_p)[mixed]
    return {
        "lam": lam, "lam0": lam0, "csp": csp_avg, "mixed": mixed,
        "n_precise": int((lam < 1).sum()), "n_detected": int((lam0 < 1).sum()), "n_mixed": int(mixed.sum()),
        "group_count": cnt, "force_rmse": f_rmse, "energy_rmse": e_rmse,
        "ref_count": ref_cnt, "ref_force_rmse": ref_rmse,
        "force_rmse_mixed": float(np.sqrt((d ** 2).mean())) if d.size else float("nan"),
    }
