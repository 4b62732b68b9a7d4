"""Switching-zone parameter study on the GPU against oracle.sweep (needs a GPU).

On the 4,846-atom indented-slab snapshot (12 x 12 x 10 cells) at three study points
(the paper's r_lambda = (4, 12) A, a narrow zone (0, 2) A, and raised thresholds with
the widest zone (8, 20) A):
- lambda, lambda_0, the mixed-atom set and the per-group counts are bit-exact (FP64
  classification on both sides; the GPU's nonzero-force test against the oracle's
  structural definition);
- per-group force RMSE within 1e-7 eV/A (FP64) or 1 meV/A (mixed); energy RMSE within
  1e-8 eV (FP64) or 1e-5 eV (mixed); the EAM-vs-ACE reference RMSE likewise.
"""
import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle.sweep as OS

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap
    from paper_2411_03002_gb300 import sweep as S

POINTS = [(2.5, 3.0, 4.0, 12.0), (2.5, 3.0, 0.0, 2.0), (3.0, 3.5, 8.0, 20.0)]


@pytest.fixture(scope="module")
def snapshot():
    w = I.config_c6(12, 10)
    eam, ace = I.eam_params(0), I.ace_for_config(5)
    ch = (w.fixed == 0).astype(np.uint8)
    ref = OS.reference(w.x, w.box, eam, ace)
    return w, eam, ace, ch, ref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_study_points_match_oracle(snapshot, precision):
    w, eam, ace, ch, ref = snapshot
    prec = ap.PREC_FP64 if precision == "fp64" else ap.PREC_MIXED
    st = S.Study(eam, ace, w.hyb, torch.as_tensor(w.x, device="cuda"), w.box,
                 torch.as_tensor(ch, device="cuda"), precision=prec, reps=1)
    assert tuple(S.CSP_EDGES) == tuple(OS.CSP_EDGES)
    tol_f, tol_e = (1e-7, 1e-8) if prec == ap.PREC_FP64 else (1e-3, 1e-5)
    for (clo, chi, rlo, rhi) in POINTS:
        g = st.point(S.Point(clo, chi, rlo, rhi))
        hyb = I.HybridParams(csp_lo=clo, csp_hi=chi, r_lo=rlo, r_hi=rhi)
        o = OS.study(w.x, w.box, ch, hyb, eam, ace, ref=ref)
        assert np.array_equal(st.last["lam"], o["lam"])
        assert np.array_equal(st.last["lam0"], o["lam0"])
        assert np.array_equal(st.last["mixed"], o["mixed"])
        assert g["n_precise"] == o["n_precise"] and g["n_mixed"] == o["n_mixed"] > 0
        assert g["group_count"] == o["group_count"].tolist()
        for key, okey, tol in (("force_rmse_meV_A", "force_rmse", tol_f), ("energy_rmse_meV", "energy_rmse", tol_e),
                               ("ref_force_rmse_meV_A", "ref_force_rmse", tol_f)):
            a, b = np.array(g[key]) * 1e-3, o[okey]
            both = np.isfinite(b)
            assert np.array_equal(np.isfinite(a), both), key
            assert np.abs(a[both] - b[both]).max() <= tol, (key, np.abs(a[both] - b[both]).max())
        assert g["t_forces_ms"] > 0 and g["speedup_vs_full_ace"] > 0


def test_wider_zone_costs_more_and_is_more_precise(snapshot):
    """The paper's trade-off on this snapshot: a wider zone at fixed r_lambda,lo makes
    more atoms precise and lowers the force error of the mixed atoms (oracle only)."""
    w, eam, ace, ch, ref = snapshot
    a = OS.study(w.x, w.box, ch, I.HybridParams(r_lo=4.0, r_hi=6.0), eam, ace, ref=ref)
    b = OS.study(w.x, w.box, ch, I.HybridParams(r_lo=4.0, r_hi=12.0), eam, ace, ref=ref)
    assert b["n_precise"] > a["n_precise"]
    assert b["force_rmse_mixed"] < a["force_rmse_mixed"]
