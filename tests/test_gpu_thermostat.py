"""Local thermostat (Appendix C) on the GPU against the oracle (needs a GPU).

* One lambda-update step in FP64 from the seeded start, on the 237-atom cell (one
  sweep cell) and the 32,000-atom slab (many cells, all 8 colours): the corrected
  end-of-step velocities match the oracle's step (forces from the oracle, the same
  classification, Delta E, and the corrections in the same sweep order) within
  1e-9 relative, and so does the corrected energy.
* MD of the 237-atom cell at 900 K with lambda re-sampled every step: with the
  thermostat the total energy stays at the conservative system's level; without it,
  it follows the lambda changes.
"""
import dataclasses

import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle as O
import oracle.thermostat as TH

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap


def fresh_hyb(h):
    """lambda re-sampled from scratch at every update (no averaging, no hysteresis)."""
    return dataclasses.replace(h, n_csp_avg=1, n_lam_avg=1, dlam_min=0.0)


def gpu_step(w, hyb, v0, ace_p, thermostat, nsteps=1, eam_p=None):
    cfg = ap.make_config(eam_p or I.eam_params(0), ace_p, hyb, precision=ap.PREC_FP64, dt=w.dt, lambda_every=1,
                         thermostat=thermostat)
    ctx = ap.Context(cfg)
    x = torch.as_tensor(w.x, device="cuda").clone()
    v = torch.as_tensor(v0, device="cuda").clone()
    f = torch.zeros_like(x)
    lam = torch.empty(w.n, dtype=torch.float64, device="cuda")
    m = torch.as_tensor(w.mass, device="cuda")
    ctx.build_neighbors(x, w.box)
    s0 = ctx.step(x, v, f, m, None, lam, 0)
    s1 = ctx.step(x, v, f, m, None, lam, nsteps)
    return s0, s1, v.cpu().numpy()


def oracle_step(w, hyb, v0, ace_p, eam_p=None):
    eam = eam_p or I.eam_params(0)
    ace = O.ACEFS(ace_p) if getattr(ace_p, "c2", None) is not None else O.ACE(ace_p)
    m, dt = w.mass, w.dt
    st = O.LambdaState(w.n, hyb.n_csp_avg, hyb.n_lam_avg)
    lam0, *_ = O.classify(st, w.x, w.box, hyb)
    _, f0, _, _ = O.hybrid(w.x, w.box, lam0, eam, ace)
    vh = v0 + 0.5 * dt * f0 * O.ACC / m[:, None]
    x1 = w.x + dt * vh
    lam1, *_ = O.classify(st, x1, w.box, hyb)
    _, fd, ef, _ = O.hybrid(x1, w.box, lam1, eam, ace)
    _, fc, _, _ = O.hybrid(x1, w.box, lam0, eam, ace)
    ep, _ = ace.eval(x1, w.box)
    dE = TH.delta_v(lam0, lam1, ef, ep) + TH.delta_t(fc, fd, vh, m, dt)
    v1 = vh + 0.5 * dt * fd * O.ACC / m[:, None]
    v1c, n_ok, n_bad = TH.correct(x1, w.box, v1, m, dE, float(eam.rc) + 1.0, 1.0)   # rows at eam_rc + skin
    return v1, v1c, dE, n_ok, n_bad, float(np.abs(lam1 - lam0).sum())


@pytest.mark.parametrize("case", ["c1", "slab"])
def test_one_update_step_matches_oracle(case):
    if case == "c1":
        w = I.config_c1()
        hyb = dataclasses.replace(fresh_hyb(I.SINGLE_EVAL), csp_lo=1.0, csp_hi=4.0)
        v0 = I.maxwell_boltzmann(w.mass, np.ones(w.n, bool), 900.0, np.random.Generator(np.random.PCG64(I.seed_for(9, 6))))
        ace_p = I.ace_params(0)
    else:
        w = I.config_c2()
        hyb = fresh_hyb(w.hyb)
        v0 = w.v
        ace_p = I.ace_for_config(2)
    w = dataclasses.replace(w, hyb=hyb)
    v1, v1c, dE, n_ok, n_bad, changes = oracle_step(w, hyb, v0, ace_p)
    assert changes > 0 and n_ok > 0 and n_bad == 0
    _, s1, v_gpu = gpu_step(w, hyb, v0, ace_p, thermostat=True)
    assert s1.th_refused == 0 and s1.th_corrected == n_ok
    scale = np.abs(v1c).max()
    assert np.abs(v_gpu - v1c).max() <= 1e-9 * scale, np.abs(v_gpu - v1c).max() / scale
    # the corrections matter: the uncorrected velocities are further away
    assert np.abs(v1 - v1c).max() > 100 * np.abs(v_gpu - v1c).max()
    assert s1.th_energy == pytest.approx(float(dE.sum()), rel=1e-9, abs=1e-12)


def test_thermostat_conserves_energy_with_changing_lambda():
    w = I.config_c1()
    hyb = dataclasses.replace(fresh_hyb(I.SINGLE_EVAL), csp_lo=1.0, csp_hi=4.0)
    v0 = I.maxwell_boltzmann(w.mass, np.ones(w.n, bool), 900.0, np.random.Generator(np.random.PCG64(I.seed_for(9, 6))))

    def run(thermostat):
        cfg = ap.make_config(I.eam_params(0), I.ace_params(0), hyb, precision=ap.PREC_FP64, dt=w.dt, lambda_every=1,
                             thermostat=thermostat)
        ctx = ap.Context(cfg)
        x = torch.as_tensor(w.x, device="cuda").clone()
        v = torch.as_tensor(v0, device="cuda").clone()
        f = torch.zeros_like(x)
        lam = torch.empty(w.n, dtype=torch.float64, device="cuda")
        m = torch.as_tensor(w.mass, device="cuda")
        ctx.build_neighbors(x, w.box)
        s = ctx.step(x, v, f, m, None, lam, 0)
        e = [s.e_pot + s.e_kin]
        for _ in range(30):
            s = ctx.step(x, v, f, m, None, lam, 1)
            e.append(s.e_pot + s.e_kin)
        return np.array(e), s

    e_off, _ = run(False)
    e_on, s_on = run(True)
    assert s_on.th_corrected > 0 and s_on.th_refused == 0
    drift_off = np.abs(e_off - e_off[0]).max()
    drift_on = np.abs(e_on - e_on[0]).max()
    assert drift_on < 0.01 * drift_off, (drift_on, drift_off)


@pytest.mark.parametrize("eam_kind", ["analytic", "mishin"])
@pytest.mark.parametrize("ace_kind", ["linear", "fs"])
def test_one_update_step_other_potentials(eam_kind, ace_kind):
    """The same one-update step with the Mishin EAM2 fast potential and/or the
    Finnis-Sinclair ACE form: the thermostat's difference forces and Delta V go through
    both potentials' kernels (the 237-atom cell, FP64, 1e-9 relative)."""
    w = I.config_c1()
    hyb = dataclasses.replace(fresh_hyb(I.SINGLE_EVAL), csp_lo=1.0, csp_hi=4.0)
    v0 = I.maxwell_boltzmann(w.mass, np.ones(w.n, bool), 900.0, np.random.Generator(np.random.PCG64(I.seed_for(9, 6))))
    ace_p = I.ace_params(0) if ace_kind == "linear" else I.ace_params_fs(0, c2_scale=0.1)
    eam_p = I.eam_params(0) if eam_kind == "analytic" else I.MISHIN_ORIGINAL
    w = dataclasses.replace(w, hyb=hyb)
    v1, v1c, dE, n_ok, n_bad, changes = oracle_step(w, hyb, v0, ace_p, eam_p)
    assert changes > 0 and n_ok > 0 and n_bad == 0
    _, s1, v_gpu = gpu_step(w, hyb, v0, ace_p, thermostat=True, eam_p=eam_p)
    assert s1.th_refused == 0 and s1.th_corrected == n_ok
    scale = np.abs(v1c).max()
    assert np.abs(v_gpu - v1c).max() <= 1e-9 * scale, np.abs(v_gpu - v1c).max() / scale
    assert s1.th_energy == pytest.approx(float(dE.sum()), rel=1e-9, abs=1e-12)
