"""Mishin EAM2 as the fast potential (Appendix E forms) on the GPU against the oracle
(needs a GPU).  Both of the paper's parameter sets (original EAM2 and the 300 K fit),
in three cases chosen so that every branch of the forms is taken:

* c3: the 2,048-atom cell with lambda forced to {0, 1, U(0,1)}; densities on both
  sides of x = 1 (polynomial and rational embedding branches).
* compressed: the same cell scaled by 0.96; every density above 1.
* close_pair: the 237-atom void cell with one neighbour pulled to 2.0 A of atom 0,
  inside rs1, so the (rs - r)^4 core terms contribute; lambda ~ U(0,1).

Bars as for the analytic EAM: FP64 |dF_i| <= 1e-5 (|F_i| + 0.01 eV/A), mixed
max |dF_i| <= 1 meV/A, total energy within 1e-6 eV/atom; in FP64 also the EAM site
energies E_i^f to 1e-10 eV.  Then energy conservation of fixed-lambda velocity
Verlet with the Mishin potential, and the configurations the library refuses.
"""
import dataclasses

import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap

SETS = {"original": I.MISHIN_ORIGINAL, "fit": I.MISHIN_FIT_300K}


def T(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def make_case(name):
    w = I.config_c3()
    if name == "c3":
        return w.x, w.box, w.lam
    if name == "compressed":
        s = 0.96
        return w.x * s, dataclasses.replace(w.box, lo=w.box.lo * s, hi=w.box.hi * s), w.lam
    w1 = I.config_c1()
    x = w1.x.copy()
    L = w1.box.hi - w1.box.lo
    d = x - x[0]
    d -= L * np.round(d / L)
    r = np.linalg.norm(d, axis=1)
    r[0] = np.inf
    j = int(np.argmin(r))
    x[j] = x[0] + d[j] * (2.0 / r[j])
    return x, w1.box, I.rng_for(1, 7).uniform(0.0, 1.0, w1.n)


def evaluate(p, x, box, lam, prec):
    ctx = ap.Context(ap.make_config(p, I.ace_params(0), I.SINGLE_EVAL, precision=prec))
    xt = T(x)
    ctx.build_neighbors(xt, box)
    lt = T(lam)
    q = np.nonzero(lam < 1)[0]
    cnt = torch.tensor([len(q)], dtype=torch.int64, device="cuda")
    ef, f = ctx.eval_eam(xt, lt)
    ep, f = ctx.eval_ace(xt, lt, T(q, torch.int32), cnt, f=f)
    _, e_tot = ctx.blend_forces(lt, ef, ep)
    return ef.cpu().numpy(), f.cpu().numpy(), e_tot.item()


@pytest.mark.parametrize("case", ["c3", "compressed", "close_pair"])
@pytest.mark.parametrize("pset", ["original", "fit"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mishin_hybrid_matches_oracle(case, pset, precision):
    p = SETS[pset]
    x, box, lam = make_case(case)
    prec = ap.PREC_FP64 if precision == "fp64" else ap.PREC_MIXED
    e_o, f_o, ef_o, _ = O.hybrid(x, box, lam, p, O.ACE(I.ace_params(0)))
    ef, f, e_tot = evaluate(p, x, box, lam, prec)
    d = np.linalg.norm(f - f_o, axis=1)
    if prec == ap.PREC_FP64:
        lim = 1e-5 * (np.linalg.norm(f_o, axis=1) + 0.01)
        assert np.all(d <= lim), (d / lim).max()
        assert np.abs(ef - ef_o).max() < 1e-10
    else:
        assert d.max() <= 1e-3, d.max()
    assert abs(e_tot - e_o.sum()) / len(x) <= 1e-6


def test_mishin_case_coverage():
    """The cases above take every branch (checked on the oracle, host only)."""
    p = I.MISHIN_ORIGINAL
    _, _, rho, _ = O.eam_mishin(*make_case("c3")[:2], p)
    assert (rho > 1).any() and (rho <= 1).any()
    _, _, rho, _ = O.eam_mishin(*make_case("compressed")[:2], p)
    assert (rho > 1).all()
    x, box, _ = make_case("close_pair")
    L = box.hi - box.lo
    d = x - x[0]
    d -= L * np.round(d / L)
    assert np.sort(np.linalg.norm(d, axis=1))[1] == pytest.approx(2.0) and 2.0 < p.rs1


@pytest.mark.parametrize("pset", ["original", "fit"])
def test_mishin_fixed_lambda_nve_fp64(pset):
    """Fixed lambda makes the hybrid conservative (section 2.3); 200 steps of 1 fs at
    300 K on the void cell with the Mishin fast potential."""
    w = I.config_c1()
    hyb = I.HybridParams(r_lo=2.0, r_hi=3.5, n_csp_avg=1, n_lam_avg=1, sample_every=100000)
    cfg = ap.make_config(SETS[pset], I.ace_params(0), hyb, precision=ap.PREC_FP64, dt=1.0, rebuild_every=10)
    ctx = ap.Context(cfg)
    v0 = I.maxwell_boltzmann(w.mass, np.ones(w.n, bool), 300.0, I.rng_for(1, 3))
    x, v = T(w.x), T(v0)
    f = torch.zeros_like(x)
    lam = torch.empty(w.n, dtype=torch.float64, device="cuda")
    ctx.build_neighbors(x, w.box)
    s0 = ctx.step(x, v, f, T(w.mass), None, lam, 0)
    s1 = ctx.step(x, v, f, T(w.mass), None, lam, 200)
    drift = abs(s1.e_pot + s1.e_kin - s0.e_pot - s0.e_kin) / w.n
    assert drift < 1e-5, drift
    assert s1.n_precise > 0 and s1.n_precise < w.n


def test_mishin_rejected_where_analytic_only():
    """The selector detector and too short an eam_rc are refused with eam_type Mishin."""
    cfg = ap.make_config(I.MISHIN_ORIGINAL, I.ace_params(0), I.SINGLE_EVAL, detector=ap.DETECT_SELECTOR)
    with pytest.raises(ap.ApError):
        ap.Context(cfg)
    cfg = ap.make_config(I.MISHIN_ORIGINAL, I.ace_params(0), I.SINGLE_EVAL)
    cfg.eam_rc = I.MISHIN_ORIGINAL.rc - 0.1
    with pytest.raises(ap.ApError):
        ap.Context(cfg)
