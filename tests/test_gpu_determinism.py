"""Bitwise reproducible forces with the fixed-point ACE reduction (needs a GPU).

With ace_deterministic = 1 the ACE force contributions are rounded to multiples of
2^-36 eV/A and summed with integer atomics, which are exact and independent of the
order in which warps finish; the EAM forces are gathered and every energy is reduced
in a fixed order.  So:
* two identical 50-step mixed-precision MD runs of the 32,000-atom slab (lambda
  updates, rebuilds) end with bit-identical positions, velocities and forces;
* the fixed-point forces still meet the parity bars against the oracle on the
  2,048-atom forced-lambda cell: FP64 |dF_i| <= 1e-5 (|F_i| + 0.01 eV/A), mixed
  1 meV/A.
"""
import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap


def md(w, steps):
    cfg = ap.make_config(I.eam_params(0), I.ace_for_config(2), w.hyb, precision=ap.PREC_MIXED, dt=w.dt,
                         lambda_every=10, rebuild_every=5, deterministic=True)
    ctx = ap.Context(cfg)
    x = torch.as_tensor(w.x, device="cuda").clone()
    v = torch.as_tensor(w.v, device="cuda").clone()
    f = torch.zeros_like(x)
    lam = torch.empty(w.n, dtype=torch.float64, device="cuda")
    ctx.build_neighbors(x, w.box)
    ctx.step(x, v, f, torch.as_tensor(w.mass, device="cuda"), None, lam, 0)
    s = ctx.step(x, v, f, torch.as_tensor(w.mass, device="cuda"), None, lam, steps)
    ctx.close()
    return x.cpu().numpy(), v.cpu().numpy(), f.cpu().numpy(), s


def test_two_runs_are_bitwise_equal():
    w = I.config_c2()
    x1, v1, f1, s1 = md(w, 50)
    x2, v2, f2, s2 = md(w, 50)
    assert s1.n_precise > 0 and s1.rebuilds >= 10
    assert np.array_equal(f1, f2) and np.array_equal(x1, x2) and np.array_equal(v1, v2)
    assert s1.e_pot == s2.e_pot and s1.e_kin == s2.e_kin


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fixed_point_forces_match_oracle(precision):
    w = I.config_c3()
    prec = ap.PREC_FP64 if precision == "fp64" else ap.PREC_MIXED
    ctx = ap.Context(ap.make_config(I.eam_params(0), I.ace_params(0), w.hyb, precision=prec, deterministic=True))
    x = torch.as_tensor(w.x, device="cuda")
    lam = torch.as_tensor(w.lam, device="cuda")
    ctx.build_neighbors(x, w.box)
    q, nq = ctx.precise_queue(lam)
    _, f = ctx.eval_eam(x, lam)
    _, f = ctx.eval_ace(x, lam, q, nq, f=f)
    _, f_o, _, _ = O.hybrid(w.x, w.box, w.lam, I.eam_params(0), O.ACE(I.ace_params(0)))
    d = np.linalg.norm(f.cpu().numpy() - f_o, axis=1)
    if prec == ap.PREC_FP64:
        assert np.all(d <= 1e-5 * (np.linalg.norm(f_o, axis=1) + 0.01)), d.max()
    else:
        assert d.max() <= 1e-3, d.max()
