"""Fit the linear ACE coefficients to the synthetic EAM on bulk snapshots.

TEST/INPUT INFRASTRUCTURE: calls only the oracle.  It writes the stored
coefficients ap_inputs/ace_anchor.npz that the molecular-dynamics workloads use
as their precise potential ("EAM-anchored ACE"): c = c_fit + eps, where c_fit
minimises

    sum_s 1/N_s [ sum_i ((E_i^ACE - E_i^EAM)/0.01 eV)^2 + sum_i |F_i^ACE - F_i^EAM|^2/(0.01 eV/A)^2 ]
      + ridge |c|^2

over FCC bulk cells with thermal-like displacements and small strains (the
paper fits its fast potential to the precise one on bulk MD snapshots with
these tolerances; here the roles are reversed because only the analytic EAM
exists), and eps is the seeded N(0, 0.01^2) coefficient vector scaled by
EPS_SCALE, so that ACE and EAM agree in bulk and differ at surfaces and defects.

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
RIDGE = 1e-5
OUT = os.path.join(ROOT, "ap_inputs", "ace_anchor.npz")


def structures(seed: int):
    """Bulk cells (strain x thermal-like displacement) first, then (100) slabs,
    vacancy cells and strongly disordered cells, so that the fit stays bound
    where the molecular-dynamics workloads leave the bulk."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for a in (3.57, 3.595, 3.615, 3.635, 3.66):
        for sigma in (0.04, 0.08, 0.12):
            x = I.fcc_lattice(4, 4, 4, a) + sigma * g.standard_normal((256, 3))
            box = I.Box(lo=np.zeros(3), hi=np.full(3, 4 * a), periodic=np.array([True, True, True]))
            out.append((x, box))
    a = I.A_CU
    for sigma in (0.05, 0.1, 0.2):
        x = I.fcc_lattice(4, 4, 5, a) + sigma * g.standard_normal((320, 3))
        box = I.Box(lo=np.array([0.0, 0.0, -15.0]), hi=np.array([4 * a, 4 * a, 5 * a + 15.0]),
                    periodic=np.array([True, True, False]))
        out.append((x, box))
    for sigma in (0.05, 0.1):
        x = I.fcc_lattice(4, 4, 4, a)
        x = np.delete(x, g.choice(256, 3, replace=False), axis=0)
        x = x + sigma * g.standard_normal(x.shape)
        out.append((x, I.Box(lo=np.zeros(3), hi=np.full(3, 4 * a), periodic=np.array([True, True, True]))))
    for sigma in (0.2, 0.3):
        x = I.fcc_lattice(4, 4, 4, a) + sigma * g.standard_normal((256, 3))
        out.append((x, I.Box(lo=np.zeros(3), hi=np.full(3, 4 * a), periodic=np.array([True, True, True]))))
    return out


def design(structs, ace_unit, with_forces):
    eam = I.eam_params(0)
    rows_e, ye, rows_f, yf = [], [], [], []
    for k, (x, box) in enumerate(structs):
        n = x.shape[0]
        e_eam, f_eam, _, _ = O.eam(x, box, eam)
        ace0 = ace_unit[0]
        _, B = ace0.basis(x, box, np.arange(n))
        rows_e.append(B / np.sqrt(n) / 0.01)
        ye.append(e_eam / np.sqrt(n) / 0.01)
        if with_forces[k]:
            nl = O.neighbors(x, box, 7.0)
            cols = []
            for a in ace_unit:
                _, f = a.eval(x, box, nl=nl)
                cols.append(f.reshape(-1))
            rows_f.append(np.stack(cols, 1) / np.sqrt(n) / 0.01)
            yf.append(f_eam.reshape(-1) / np.sqrt(n) / 0.01)
    X = np.concatenate(rows_e + rows_f, 0)
    y = np.concatenate(ye + yf, 0)
    return X, y


def main():
    t0 = time.time()
    base = I.ace_params(0)
    nb = O.ACE(base).nbasis
    ace_unit = []
    for v in range(nb):
        c = np.zeros(512)
        c[v] = 1.0
        ace_unit.append(O.ACE(I.ACEParams(W=base.W, c=c, rc=base.rc, n0=base.n0)))
    train = structures(I.seed_for(6, 0))
    with_f = [True] * len(train)
    X, y = design(train, ace_unit, with_f)
    A = X.T @ X + RIDGE * np.eye(nb)
    c_fit = np.linalg.solve(A, X.T @ y)
    c = np.zeros(512)
    c[:nb] = c_fit + EPS_SCALE * base.c[:nb]
    # report residuals on held-out structures with the final coefficients
    test = structures(I.seed_for(6, 1))
    ace = O.ACE(I.ACEParams(W=base.W, c=c, rc=base.rc, n0=base.n0))
    de, df, by_sigma = [], [], {}
    for k, (x, box) in enumerate(test):
        e_eam, f_eam, _, _ = O.eam(x, box, I.eam_params(0))
        e_ace, f_ace = ace.eval(x, box)
        de.append(e_ace - e_eam)
        df.append(f_ace - f_eam)
        by_sigma.setdefault((0.04, 0.08, 0.12)[k % 3] if k < 15 else ("slab", "slab", "slab", "vac", "vac", "dis", "dis")[k - 15], []).append(f_ace - f_eam)
    de = np.concatenate(de)
    df = np.concatenate(df)
    report = {"rms_dF_by_sigma_eV_A": {s_: float(np.sqrt((np.concatenate(v) ** 2).mean())) for s_, v in by_sigma.items()},
              "rms_dE_eV": float(np.sqrt((de ** 2).mean())), "rms_dF_eV_A": float(np.sqrt((df ** 2).mean())),
              "max_dF_eV_A": float(np.abs(df).max()), "eps_scale": EPS_SCALE, "ridge": RIDGE,
              "n_equations": int(X.shape[0]), "seconds": time.time() - t0}
    np.savez(OUT, c=c, W=base.W, report=np.array([report["rms_dE_eV"], report["rms_dF_eV_A"],
                                                   report["max_dF_eV_A"], EPS_SCALE, RIDGE]))
    print(report)


if __name__ == "__main__":
    main()
