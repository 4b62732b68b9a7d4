"""Pins of the local-thermostat oracle (oracle/thermostat.py, Appendix C)."""
import dataclasses

import numpy as np
import pytest

import ap_inputs as I
import oracle as O
import oracle.thermostat as TH


def rng(k):
    return np.random.Generator(np.random.PCG64(I.seed_for(9, k)))


def test_rescale_conserves_momentum_and_sets_the_energy_change():
    g = rng(1)
    v = g.standard_normal((50, 3)) * 0.01
    m = 60 + 10 * g.random(50)
    om = list(range(3, 40))
    p0 = (m[:, None] * v).sum(0)
    ke = lambda vv: float((0.5 * m[:, None] * vv * vv).sum() / O.ACC)
    for dE in (3e-3, -2e-3, 0.0):
        w = v.copy()
        beta, ok = TH.rescale_group(w, m, om, dE)
        assert ok
        assert np.allclose((m[:, None] * w).sum(0), p0, rtol=0, atol=1e-14)
        assert ke(w) - ke(v) == pytest.approx(dE, abs=1e-14 * ke(v))      # rounding of the totals
        assert np.array_equal(np.delete(w, om, 0), np.delete(v, om, 0))     # only Omega moves
        if dE == 0.0:
            assert beta == 1.0


def test_negative_radicand_leaves_velocities_alone():
    g = rng(2)
    v = g.standard_normal((10, 3)) * 0.01
    m = np.full(10, 63.546)
    rel = v - (m[:, None] * v).sum(0) / m.sum()
    krel = float((0.5 * m[:, None] * rel * rel).sum() / O.ACC)
    w = v.copy()
    _, ok = TH.rescale_group(w, m, list(range(10)), -1.5 * krel)
    assert not ok and np.array_equal(w, v)


def test_delta_t_is_the_end_of_step_kinetic_energy_difference():
    g = rng(3)
    n, dt = 40, 1.0
    m = 60 + 10 * g.random(n)
    vh = g.standard_normal((n, 3)) * 0.02
    fc, fd = g.standard_normal((n, 3)), g.standard_normal((n, 3))
    vc = vh + 0.5 * dt * fc * O.ACC / m[:, None]
    vd = vh + 0.5 * dt * fd * O.ACC / m[:, None]
    direct = 0.5 * m * ((vc * vc).sum(1) - (vd * vd).sum(1)) / O.ACC
    assert np.allclose(TH.delta_t(fc, fd, vh, m, dt), direct, rtol=1e-11, atol=1e-16)


def test_delta_v_is_the_site_energy_difference():
    w = I.config_c1()
    g = rng(4)
    lam_c = np.clip(g.random(w.n) * 1.4 - 0.2, 0, 1)
    lam_d = np.where(g.random(w.n) < 0.5, lam_c, np.clip(lam_c + 0.1 * g.standard_normal(w.n), 0, 1))
    ace = O.ACE(I.ace_params(0))
    ec, *_ = O.hybrid(w.x, w.box, lam_c, I.eam_params(0), ace)
    ed, *_ = O.hybrid(w.x, w.box, lam_d, I.eam_params(0), ace)
    ef, _, _, _ = O.eam(w.x, w.box, I.eam_params(0))
    ep, _ = ace.eval(w.x, w.box)
    assert np.allclose(ec - ed, TH.delta_v(lam_c, lam_d, ef, ep), rtol=1e-10, atol=1e-13)


def test_groups_of_one_colour_in_different_cells_are_disjoint():
    w = I.config_c2()
    x, box = w.x, w.box
    c, nc = TH.thermostat_cells(x, box, 6.5, 1.0)
    assert np.all(nc[:2] % 2 == 0) and np.all(nc >= 1)
    L = box.hi - box.lo
    assert np.all(L / nc >= 15.0 - 1e-12)
    g = rng(5)
    pick = g.choice(w.n, 400, replace=False)
    color = (c[:, 0] & 1) + 2 * (c[:, 1] & 1) + 4 * (c[:, 2] & 1)
    cid = (c[:, 2] * nc[1] + c[:, 1]) * nc[0] + c[:, 0]
    for a in pick[:200]:
        for b in pick[200:]:
            if color[a] == color[b] and cid[a] != cid[b]:
                d = x[b] - x[a]
                d[:2] -= L[:2] * np.round(d[:2] / L[:2])
                assert np.linalg.norm(d) >= 15.0 - 1e-9       # Omega radius 6.5 + skin each
    order = TH.correction_order(x, box, 6.5, 1.0, pick)
    assert sorted(order) == sorted(pick.tolist())


@pytest.mark.slow
def test_corrections_restore_energy_conservation_with_changing_lambda():
    """Oracle MD of the 237-atom cell at 900 K with lambda re-sampled every step:
    without the correction the total energy follows the lambda changes; with it,
    it stays at the conservative system's level (Appendix C)."""
    w = I.config_c1()
    hyb = dataclasses.replace(I.SINGLE_EVAL, csp_lo=1.0, csp_hi=4.0, dlam_min=0.0)
    eam, ace = I.eam_params(0), O.ACE(I.ace_params(0))
    m = w.mass
    v0 = I.maxwell_boltzmann(m, np.ones(w.n, bool), 900.0, rng(6))
    dt, steps = 1.0, 30

    def run(correct: bool):
        x, v = w.x.copy(), v0.copy()
        st = O.LambdaState(w.n, 1, 1)
        lam, *_ = O.classify(st, x, w.box, hyb)
        _, f, _, _ = O.hybrid(x, w.box, lam, eam, ace)
        energies, changes = [], 0.0
        for _ in range(steps):
            vh = v + 0.5 * dt * f * O.ACC / m[:, None]
            x = x + dt * vh
            lam_c = lam
            lam, *_ = O.classify(st, x, w.box, hyb)
            e_d, f_d, ef, _ = O.hybrid(x, w.box, lam, eam, ace)
            v = vh + 0.5 * dt * f_d * O.ACC / m[:, None]
            changes += float(np.abs(lam - lam_c).sum())
            if correct:
                _, f_c, _, _ = O.hybrid(x, w.box, lam_c, eam, ace)
                ep, _ = ace.eval(x, w.box)
                dE = TH.delta_v(lam_c, lam, ef, ep) + TH.delta_t(f_c, f_d, vh, m, dt)
                v, n_ok, n_bad = TH.correct(x, w.box, v, m, dE, 6.5, 1.0)
                assert n_bad == 0
            f = f_d
            energies.append(float(e_d.sum()) + O.kinetic(v, m))
        return np.array(energies), changes

    e_off, ch = run(False)
    e_on, _ = run(True)
    assert ch > 1.0                                            # lambda did change
    drift_off = np.abs(e_off - e_off[0]).max()
    drift_on = np.abs(e_on - e_on[0]).max()
    assert drift_on < 0.01 * drift_off, (drift_on, drift_off)      # measured ratio ~1e-4
