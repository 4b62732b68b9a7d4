"""Pins of the switching-zone study oracle (oracle/sweep.py) on the CPU.

- The energy error of atoms with lambda = 0 vanishes (the paper notes that it does by
  design, since E_i then is the precise site energy), and atoms with lambda_k = 0 for
  every k within the ACE cutoff carry no force error at all.
- Limits: thresholds above every CSP make no atom precise and no atom mixed; a zone
  narrower than every interatomic distance keeps lambda = lambda_0.
- The contribution sets agree with a brute-force scan over all periodic images.
- grouped_rmse against a hand computation.
"""
import numpy as np
import pytest

import ap_inputs as I
import oracle as O
import oracle.sweep as OS


@pytest.fixture(scope="module")
def snap():
    w = I.config_c6(12, 10)
    eam, ace = I.eam_params(0), I.ace_for_config(5)
    ch = (w.fixed == 0).astype(np.uint8)
    return w, eam, ace, ch, OS.reference(w.x, w.box, eam, ace)


def test_precise_atoms_have_the_precise_energy_and_pure_ace_atoms_no_force_error(snap):
    w, eam, ace, ch, ref = snap
    o = OS.study(w.x, w.box, ch, I.HYB1, eam, ace, ref=ref)
    lam = o["lam"]
    e_h, f_h, _, _ = O.hybrid(w.x, w.box, lam, eam, O.ACE(ace))
    e_p, f_p, _ = ref
    p = lam == 0
    assert p.sum() > 100
    assert np.abs(e_h[p] - e_p[p]).max() < 1e-12
    # lambda_k = 0 for every k within the ACE cutoff (which contains the EAM cutoff):
    # the force is the precise one
    pure = (ch == 1) & ~OS.contributes(w.x, w.box, ace.rc, lam)
    assert pure.sum() > 50
    assert np.abs(f_h[pure] - f_p[pure]).max() < 1e-12
    # and the mixed atoms do carry an error
    assert o["force_rmse_mixed"] > 1e-4


def test_limits(snap):
    w, eam, ace, ch, ref = snap
    o = OS.study(w.x, w.box, ch, I.HybridParams(csp_lo=1e6, csp_hi=2e6), eam, ace, ref=ref)
    assert o["n_precise"] == 0 and o["n_mixed"] == 0
    assert np.all(np.isnan(o["force_rmse"]))
    o = OS.study(w.x, w.box, ch, I.HybridParams(r_lo=0.0, r_hi=1.0), eam, ace, ref=ref)
    assert np.array_equal(o["lam"], o["lam0"])         # no neighbour is closer than 1 A


def test_contribution_sets_against_a_pair_scan():
    w = I.config_c1()
    g = I.rng_for(1, 11)
    lam = np.where(g.uniform(size=w.n) < 0.9, 1.0, g.uniform(size=w.n))
    lam[g.uniform(size=w.n) < 0.05] = 0.0
    L = w.box.hi - w.box.lo
    for rc, wt in ((5.5, lam), (7.0, 1.0 - lam)):
        got = OS.contributes(w.x, w.box, rc, wt)
        want = np.zeros(w.n, bool)
        for i in range(w.n):
            d = w.x - w.x[i]
            # every periodic image within rc (the cell is 14.46 A wide, rc < L)
            near = np.zeros(w.n, bool)
            for s in np.ndindex(3, 3, 3):
                dd = d + (np.array(s) - 1) * L
                r = np.linalg.norm(dd, axis=1)
                near |= (r < rc) & (r > 0)
            want[i] = near.any() and (wt[i] > 0 or (wt[near] > 0).any())
        assert np.array_equal(got, want)


def test_grouped_rmse_by_hand():
    d = np.array([[1.0, 0, 0], [0, 2.0, 0], [0, 0, 3.0], [4.0, 0, 0]])
    csp = np.array([0.1, 0.2, 5.0, 0.3])
    mask = np.array([True, True, True, False])
    cnt, r = OS.grouped_rmse(d, csp, mask, edges=(0.0, 1.0, 10.0, np.inf))
    assert cnt.tolist() == [2, 1, 0]
    assert r[0] == pytest.approx(np.sqrt((1 + 4) / 6))
    assert r[1] == pytest.approx(np.sqrt(9 / 3))
    assert np.isnan(r[2])
