"""What the learned selector gains over the centro-symmetry detector (needs a GPU).

On a held-out 32,000-atom slab (ap_inputs.config_c2 variant 4: free (100) surfaces and
a 0.3 A-disordered hemisphere; the selector never saw it), with the stored model:
* labels: |F_ACE - F_EAM| > 25 meV/A from full potentials (the selector's label);
* detection: the selector's detected set (p_avg > p_lo) holds at least 90 % of the
  label-positive atoms with at least 95 % precision; the CSP detector holds at most
  45 % at every threshold pair from (2.5, 3.0) down to (0.4, 0.9) A^2.  The positives it
  misses lie under the surfaces, where the lattice is intact and CSP ~ 0;
* force error at a matched cost: with the switching zone r_lambda = (4, 10) A the
  selector (p_lo, p_hi) = (0.9, 0.95) makes no more atoms precise than CSP with the
  paper's Hyb1 zone (4, 12) A, and its RMS force error against full ACE on the
  label-positive atoms is at least 20 % lower.
The thermalised slab (150 EAM MD steps) is measured too: there a CSP run whose zone is
re-tuned matches the selector at equal cost, so no gain is asserted on it.
"""
import dataclasses
import os

import numpy as np
import pytest
import torch

import ap_inputs as I

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap

TAU = 0.025
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def slab():
    w = I.config_c2(variant=4)
    x = torch.as_tensor(w.x, device="cuda")
    sel = np.load(os.path.join(ROOT, "paper_2411_03002_gb300", "selector_cu.npz"))
    ctx = context(w, x, I.HYB1, sel)
    n = w.n
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    allq = torch.arange(n, dtype=torch.int32, device="cuda")
    na = torch.tensor([n], dtype=torch.int64, device="cuda")
    _, fa = ctx.eval_eam(x, z)
    _, fa = ctx.eval_ace(x, z, allq, na, f=fa)
    _, fe = ctx.eval_eam(x)
    ctx.close()
    pos = torch.linalg.vector_norm(fa - fe, dim=1) > TAU
    return w, x, sel, fa, pos


def context(w, x, hyb, sel, detector=None, p_lo=0.5, p_hi=0.9):
    det = ap.DETECT_CSP if detector is None else detector
    ctx = ap.Context(ap.make_config(I.eam_params(0), I.ace_for_config(2), hyb, precision=ap.PREC_MIXED, detector=det,
                                    sel_p_lo=p_lo, sel_p_hi=p_hi))
    if det == ap.DETECT_SELECTOR:
        ctx.sel_set_model(sel["params"], sel["mu"], sel["inv_sigma"])
    ctx.build_neighbors(x, w.box)
    return ctx


def evaluate(ctx, x, fa, pos):
    lam, q, nq = ctx.classify(x)
    detected = ctx.get_lambda_state()["lam0"] < 1.0
    _, f = ctx.eval_eam(x, lam)
    _, f = ctx.eval_ace(x, lam, q, nq, f=f)
    d = torch.linalg.vector_norm(f - fa, dim=1)
    ctx.close()
    return {"precise": float((lam < 1.0).float().mean()),
            "recall": float((detected & pos).sum() / pos.sum()),
            "precision": float((detected & pos).sum() / detected.sum()),
            "rms_pos_meV": float(torch.sqrt((d[pos] ** 2).mean()) * 1e3)}


def test_selector_detects_what_csp_cannot(slab):
    w, x, sel, fa, pos = slab
    assert 0.1 < float(pos.float().mean()) < 0.3
    s = evaluate(context(w, x, I.HYB1, sel, ap.DETECT_SELECTOR, float(sel["p_lo"]), float(sel["p_hi"])), x, fa, pos)
    print("selector detection", s)
    assert s["recall"] >= 0.90 and s["precision"] >= 0.95, s
    for lo in (2.5, 1.5, 1.0, 0.6, 0.4):
        c = evaluate(context(w, x, dataclasses.replace(I.HYB1, csp_lo=lo, csp_hi=lo + 0.5), sel), x, fa, pos)
        print("csp", lo, c)
        assert c["recall"] <= 0.45, (lo, c)


def test_selector_lower_error_at_no_more_cost_than_csp_hyb1(slab):
    w, x, sel, fa, pos = slab
    c = evaluate(context(w, x, I.HYB1, sel), x, fa, pos)
    zone = dataclasses.replace(I.HYB1, r_lo=4.0, r_hi=10.0)
    s = evaluate(context(w, x, zone, sel, ap.DETECT_SELECTOR, 0.9, 0.95), x, fa, pos)
    print("matched point: csp Hyb1", c, "selector (0.9, 0.95) zone 4/10", s)
    assert s["precise"] <= c["precise"], (s, c)
    assert s["rms_pos_meV"] <= 0.8 * c["rms_pos_meV"], (s, c)
