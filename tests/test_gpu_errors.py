"""Error paths of the C-ABI from host-made inputs, and capacity growth (needs a GPU).

Every input here is ordinary, valid device memory; the library's own checks turn
it into a status.  Nothing faults or hangs the GPU.
* a NaN position -> AP_ERR_NONFINITE from ap_build_neighbors, and a NaN velocity
  (non-finite positions after the drift) -> AP_ERR_NONFINITE from ap_step;
* an atom moved by more than skin/2 since the last list build -> AP_ERR_SKIN;
* a compressed crystal whose rows overflow the default EAM and ACE capacities and
  whose atoms have more neighbours inside the ACE cutoff than the kernel caches:
  the rows grow, and energies and forces still match the oracle;
* the local thermostat (Appendix C) when the only mobile atom changes lambda with
  all its row neighbours fixed: its group has no relative kinetic energy, so the
  correction cannot be made -> AP_ERR_RADICAND, velocities as without the thermostat.
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

AP_ERR_NONFINITE, AP_ERR_RADICAND, AP_ERR_SKIN = 4, 7, 9


def T(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def md_setup(w, precision=None, **kw):
    cfg = ap.make_config(I.eam_params(0), I.ace_params(0), w.hyb, precision=precision or ap.PREC_FP64, dt=1.0,
                         lambda_every=10, **kw)
    ctx = ap.Context(cfg)
    x, v = T(w.x).clone(), torch.zeros((w.n, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros_like(x)
    lam = torch.empty(w.n, dtype=torch.float64, device="cuda")
    m = T(np.full(w.n, I.MASS_CU))
    ctx.build_neighbors(x, w.box)
    ctx.step(x, v, f, m, None, lam, 0)
    return ctx, x, v, f, m, lam


def test_nan_position_is_reported_by_the_build():
    w = I.config_c1()
    x = w.x.copy()
    x[5, 1] = np.nan
    ctx = ap.Context(ap.make_config(I.eam_params(0), I.ace_params(0), w.hyb, precision=ap.PREC_MIXED))
    with pytest.raises(ap.ApError) as e:
        ctx.build_neighbors(T(x), w.box)
    assert e.value.status == AP_ERR_NONFINITE


def test_nan_velocity_is_reported_by_the_step():
    w = I.config_c1()
    ctx, x, v, f, m, lam = md_setup(w)
    v[7, 2] = float("nan")
    with pytest.raises(ap.ApError) as e:
        ctx.step(x, v, f, m, None, lam, 3)
    assert e.value.status == AP_ERR_NONFINITE


def test_displacement_beyond_half_the_skin_is_reported():
    w = I.config_c1()
    ctx, x, v, f, m, lam = md_setup(w)      # skin 1 A: the limit is 0.5 A
    ctx.step(x, v, f, m, None, lam, 1)      # within the limit: fine
    x[3, 0] += 0.6
    with pytest.raises(ap.ApError) as e:
        ctx.step(x, v, f, m, None, lam, 1)
    assert e.value.status == AP_ERR_SKIN


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dense_cluster_grows_the_rows_and_matches_the_oracle(precision):
    """FCC at a = 3.0 A (0.83 of copper's): about 170 neighbours within the EAM rows'
    6.5 A (default capacity 160), about 320 within the ACE rows' 8 A (default 288) and
    about 215 inside the 7 A ACE cutoff (more than the 192 records the kernel keeps in
    shared memory).  lambda forced to {0, 1, U(0, 1)} thirds, every atom in the queue."""
    g = np.random.Generator(np.random.PCG64(I.seed_for(3, 40)))
    a = 3.0
    x = I.fcc_lattice(5, 5, 5, a) + 0.03 * g.standard_normal((500, 3))
    box = I.Box(lo=np.zeros(3), hi=np.full(3, 5 * a), periodic=np.array([True, True, True]))
    n = x.shape[0]
    cat = g.integers(0, 3, n)
    lam = np.where(cat == 0, 0.0, np.where(cat == 1, 1.0, g.uniform(0.0, 1.0, n)))
    prec = ap.PREC_FP64 if precision == "fp64" else ap.PREC_MIXED
    ctx = ap.Context(ap.make_config(I.eam_params(0), I.ace_params(0), I.SINGLE_EVAL, precision=prec))
    xt, lt = T(x), T(lam)
    ctx.build_neighbors(xt, box)
    cnt, _, _ = ctx.get_neighbors(0, cap=400)
    assert int(cnt.max()) > 160
    q = torch.arange(n, dtype=torch.int32, device="cuda")
    nq = torch.tensor([n], dtype=torch.int64, device="cuda")
    ef, fg = ctx.eval_eam(xt, lt)
    ep, fg = ctx.eval_ace(xt, lt, q, nq, f=fg)
    cnt_a, _, _ = ctx.get_neighbors(1, cap=400)
    assert int(cnt_a.max()) > 288
    e_o, f_o, ef_o, ep_o = O.hybrid(x, box, lam, I.eam_params(0), O.ACE(I.ace_params(0)))
    fgn = fg.cpu().numpy()
    d = np.linalg.norm(fgn - f_o, axis=1)
    if prec == ap.PREC_FP64:
        assert np.all(d <= 1e-5 * (np.linalg.norm(f_o, axis=1) + 0.01)), d.max()
        m = lam < 1.0                            # the oracle reports E^p only where lambda < 1
        assert np.abs(ep.cpu().numpy()[m] - ep_o[m]).max() < 1e-9
    else:
        assert d.max() <= 1e-3, d.max()
    e_gpu = (lam * ef.cpu().numpy() + (1 - lam) * ep.cpu().numpy()).sum()
    assert abs(e_gpu - e_o.sum()) / n <= 1e-6


def test_thermostat_without_relative_kinetic_energy_reports_the_radicand():
    """Perfect FCC 4x4x4 with one vacancy.  Only one vacancy neighbour is mobile; its
    CSP (a^2/2 = 6.53 A^2) lies between csp_lo = 6 and csp_hi = 7, so its lambda_0 is
    interior and moves with it.  Its group {i} has no relative kinetic energy."""
    a = I.A_CU
    x = I.fcc_lattice(4, 4, 4)
    vac = 0
    d = x - x[vac]
    L = 4 * a
    d -= L * np.round(d / L)
    r = np.linalg.norm(d, axis=1)
    mobile_atom = int(np.nonzero(np.abs(r - a / np.sqrt(2)) < 1e-6)[0][0])
    keep = np.arange(len(x)) != vac
    x = x[keep]
    mobile_atom -= 1 if mobile_atom > vac else 0
    n = x.shape[0]
    fixed = np.ones(n, np.uint8)
    fixed[mobile_atom] = 0
    box = I.Box(lo=np.zeros(3), hi=np.full(3, L), periodic=np.array([True, True, True]))
    hyb = dataclasses.replace(I.SINGLE_EVAL, csp_lo=6.0, csp_hi=7.0, r_lo=0.0, r_hi=0.5, dlam_min=0.0)

    def run(thermostat):
        cfg = ap.make_config(I.eam_params(0), I.ace_params(0), hyb, precision=ap.PREC_FP64, dt=1.0,
                             lambda_every=1, thermostat=thermostat)
        ctx = ap.Context(cfg)
        xt = T(x).clone()
        v = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        f = torch.zeros_like(xt)
        lam = torch.empty(n, dtype=torch.float64, device="cuda")
        m, fx = T(np.full(n, I.MASS_CU)), T(fixed, torch.uint8)
        ctx.build_neighbors(xt, box)
        ctx.step(xt, v, f, m, fx, lam, 0)
        l0 = float(lam[mobile_atom])
        err = None
        try:
            ctx.step(xt, v, f, m, fx, lam, 1)
        except ap.ApError as e:
            err = e.status
        return err, v.cpu().numpy(), l0, float(lam[mobile_atom])

    err_on, v_on, l0, l1 = run(True)
    err_off, v_off, _, _ = run(False)
    assert 0.0 < l0 < 1.0 and l1 != l0          # the mobile atom's lambda is interior and moved
    assert err_off is None
    assert err_on == AP_ERR_RADICAND
    # the refused correction left the velocities alone (FP64 ACE forces are summed with
    # atomics, so the two runs agree to rounding)
    assert np.allclose(v_on, v_off, rtol=1e-10, atol=1e-18)
    assert np.any(v_on[mobile_atom] != 0.0)
