"""Fit the linear ACE coefficients to the synthetic EAM on bulk snapshots.

TEST/INPUT INFRASTRUCTURE: calls only the oracle.  It writes the stored
coefficients ap_inputs/ace_anchor.npz that the molecular-dynamics workloads use
as their precise potential ("EAM-anchored ACE"): c = c_fit + eps_perp, where
c_fit minimises

    sum_s 1/N_s [ sum_i ((E_i^ACE - E_i^EAM)/0.01 eV)^2 + sum_i |F_i^ACE - F_i^EAM|^2/(0.01 eV/A)^2 ]
      + ridge |c|^2

over FCC bulk cells with thermal-like displacements and small strains.  The
paper fits its fast potential to the precise one on bulk MD snapshots only
(section 3), so the two agree in the bulk and part at surfaces and defects; here
the roles are reversed because only the analytic EAM exists.

eps_perp is the seeded N(0, 0.01^2) coefficient vector with its components along
the bulk design's leading right-singular vectors (singular values above
SV_KEEP x the largest) removed, times EPS_SCALE, so that it leaves the bulk fit
alone.  The structure dependence of the precise/fast discrepancy comes from
fitting on bulk only (held-out per-atom |F_ACE - F_EAM| medians: ~11 meV/A in
300 K-like bulk, ~65 meV/A at a (100) surface, ~140 meV/A in strongly disordered
cells; printed per class by this script).

    python oracle/fit_ace_anchor.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import ap_inputs as I  # noqa: E402
import oracle as O  # noqa: E402

EPS_SCALE = 1.0
SV_KEEP = 1e-2
RIDGE = 1e-6
OUT = os.path.join(ROOT, "ap_inputs", "ace_anchor.npz")


def periodic_box(n, a):
    return I.Box(lo=np.zeros(3), hi=np.full(3, n * a), periodic=np.array([True, True, True]))


def bulk(seed: int):
    """FCC 4x4x4 cells: 5 lattice constants (strain) x 3 displacement widths."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for a in (3.57, 3.595, 3.615, 3.635, 3.66):
        for sigma in (0.04, 0.08, 0.12):
            out.append((I.fcc_lattice(4, 4, 4, a) + sigma * g.standard_normal((256, 3)), periodic_box(4, a)))
    return out


def defects(seed: int):
    """Held-out structure classes: (100) slab, vacancy cell, disordered cell."""
    g = np.random.Generator(np.random.PCG64(seed))
    a = I.A_CU
    x = I.fcc_lattice(4, 4, 5, a) + 0.07 * g.standard_normal((320, 3))
    slab = (x, I.Box(lo=np.array([0.0, 0.0, -15.0]), hi=np.array([4 * a, 4 * a, 5 * a + 15.0]),
                     periodic=np.array([True, True, False])))
    x = np.delete(I.fcc_lattice(4, 4, 4, a), 0, axis=0)
    vac = (x + 0.07 * g.standard_normal(x.shape), periodic_box(4, a))
    dis = (I.fcc_lattice(4, 4, 4, a) + 0.25 * g.standard_normal((256, 3)), periodic_box(4, a))
    return {"slab": slab, "vac": vac, "dis": dis}


def design(structs, ace_unit):
    eam = I.eam_params(0)
    rows, y = [], []
    for x, box in structs:
        n = x.shape[0]
        e_eam, f_eam, _, _ = O.eam(x, box, eam)
        _, B = ace_unit[0].basis(x, box, np.arange(n))
        nl = O.neighbors(x, box, 7.0)
        cols = [a.eval(x, box, nl=nl)[1].reshape(-1) for a in ace_unit]
        rows += [B / np.sqrt(n) / 0.01, np.stack(cols, 1) / np.sqrt(n) / 0.01]
        y += [e_eam / np.sqrt(n) / 0.01, f_eam.reshape(-1) / np.sqrt(n) / 0.01]
    return np.concatenate(rows, 0), np.concatenate(y, 0)


def force_gap(ace, x, box):
    _, fa = ace.eval(x, box)
    _, fe, _, _ = O.eam(x, box, I.eam_params(0))
    return np.linalg.norm(fa - fe, axis=1)


def main():
    t0 = time.time()
    base = I.ace_params(0)
    nb = O.ACE(base).nbasis
    ace_unit = []
    for v in range(nb):
        c = np.zeros(512)
        c[v] = 1.0
        ace_unit.append(O.ACE(I.ACEParams(W=base.W, c=c, rc=base.rc, n0=base.n0)))
    X, y = design(bulk(I.seed_for(6, 0)), ace_unit)
    c_fit = np.linalg.solve(X.T @ X + RIDGE * np.eye(nb), X.T @ y)
    _, s, vt = np.linalg.svd(X, full_matrices=False)
    keep = vt[s > SV_KEEP * s[0]]
    eps = base.c[:nb] - keep.T @ (keep @ base.c[:nb])
    c = np.zeros(512)
    c[:nb] = c_fit + EPS_SCALE * eps
    ace = O.ACE(I.ACEParams(W=base.W, c=c, rc=base.rc, n0=base.n0))
    # held-out residuals by class (per-atom |F_ACE - F_EAM| in meV/A)
    rep = {}
    g = np.random.Generator(np.random.PCG64(I.seed_for(6, 2)))
    for sg in (0.04, 0.07, 0.1):
        x, box = I.fcc_lattice(4, 4, 4) + sg * g.standard_normal((256, 3)), periodic_box(4, I.A_CU)
        d = force_gap(ace, x, box) * 1e3
        rep[f"bulk_s{sg}"] = (float(np.median(d)), float(np.percentile(d, 90)))
    dd = defects(I.seed_for(6, 3))
    x, box = dd["slab"]
    d = force_gap(ace, x, box) * 1e3
    z = x[:, 2]
    surf = (z < 1.0) | (z > z.max() - 1.0 - 0.3)
    rep["slab_surface"] = (float(np.median(d[surf])), float(np.percentile(d[surf], 10)))
    rep["slab_interior"] = (float(np.median(d[~surf])), float(np.percentile(d[~surf], 90)))
    x, box = dd["vac"]
    d = force_gap(ace, x, box) * 1e3
    L = box.hi - box.lo
    r = np.linalg.norm((x + L / 2) % L - L / 2, axis=1)                   # distance to the vacant site at 0
    rep["vacancy_nn"] = (float(np.median(d[r < 3.0])), float(np.percentile(d[r < 3.0], 10)))
    x, box = dd["dis"]
    d = force_gap(ace, x, box) * 1e3
    rep["disordered"] = (float(np.median(d)), float(np.percentile(d, 10)))
    report = {"per_atom_dF_meV_A(median,p10|p90)": rep, "kept_singular_directions": int(keep.shape[0]),
              "eps_perp_norm": float(np.linalg.norm(eps)), "eps_scale": EPS_SCALE, "sv_keep": SV_KEEP,
              "ridge": RIDGE, "n_equations": int(X.shape[0]), "seconds": time.time() - t0}
    np.savez(OUT, c=c, W=base.W, report=np.array([EPS_SCALE, SV_KEEP, RIDGE]))
    print(report)


if __name__ == "__main__":
    main()
