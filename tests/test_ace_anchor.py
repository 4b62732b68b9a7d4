"""The stored EAM-anchored ACE coefficients (written by oracle/fit_ace_anchor.py).

They are a ridge fit of the linear ACE energy to the synthetic EAM on bulk,
surface, vacancy and disordered FCC snapshots, plus a fixed seeded offset, so
that the precise potential agrees with the fast one in the bulk and departs from
it at defects, as the paper's Cu pair of potentials do (section 3).  Checked on a
structure the fit never saw.
"""
import numpy as np

import ap_inputs as I
import oracle as O


def test_anchored_ace_tracks_eam_in_bulk():
    g = np.random.Generator(np.random.PCG64(I.seed_for(6, 7)))
    x = I.fcc_lattice(4, 4, 4) + 0.06 * g.standard_normal((256, 3))
    box = I.Box(lo=np.zeros(3), hi=np.full(3, 4 * I.A_CU), periodic=np.array([True] * 3))
    ace = O.ACE(I.ace_params_anchored())
    e_a, f_a = ace.eval(x, box)
    e_e, f_e, _, _ = O.eam(x, box, I.eam_params(0))
    rms_f = float(np.sqrt(((f_a - f_e) ** 2).sum(1).mean()))
    assert rms_f < 0.03, rms_f                         # eV/A
    assert abs(e_a.mean() - e_e.mean()) < 0.02         # eV/atom
    # and it is not EAM: the two differ by more than rounding
    assert rms_f > 1e-3


def test_anchored_shapes_and_config_choice():
    p = I.ace_params_anchored()
    assert p.W.shape == I.ace_params(0).W.shape and p.c.shape == (512,)
    assert np.array_equal(I.ace_for_config(3).c, I.ace_params(0).c)
    assert np.array_equal(I.ace_for_config(5).c, p.c)
