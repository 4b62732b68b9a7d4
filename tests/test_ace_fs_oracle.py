"""Pins of the Finnis-Sinclair ACE form E = phi^(1) + F(phi^(2)) in the oracle
(Eq. energy_ace with the regularised square root F of oracle.fs_embed)."""
import dataclasses

import numpy as np
import pytest

import ap_inputs as I
import oracle as O


def test_embedding_closed_forms():
    eps = 0.01
    F, dF = O.fs_embed(np.array([0.0, 3 * eps * eps, -3 * eps * eps, 1.0, 1e6]), eps)
    assert F[0] == 0.0 and dF[0] == pytest.approx(1 / (2 * eps))
    assert F[1] == pytest.approx(eps, rel=1e-14) and F[2] == pytest.approx(-eps, rel=1e-14)   # sqrt(4 eps^2) - eps
    assert F[3] == pytest.approx(np.sqrt(1 + eps * eps) - eps, rel=1e-15)
    assert F[4] + eps - 1e3 == pytest.approx(eps * eps / 2e3, rel=1e-4)  # sqrt(phi) - eps + eps^2/(2 sqrt(phi))
    xs = np.linspace(-0.01, 0.01, 41)
    h = 1e-7
    fp, _ = O.fs_embed(xs + h, eps)
    fm, _ = O.fs_embed(xs - h, eps)
    _, d = O.fs_embed(xs, eps)
    nz = xs != 0
    assert np.allclose(((fp - fm) / (2 * h))[nz], d[nz], rtol=1e-6)
    # at 0, F' is continuous and F'' jumps: the central difference is off by h / (4 eps^2)
    assert ((fp - fm) / (2 * h))[~nz][0] == pytest.approx(d[~nz][0] * (1 - h / (4 * eps * eps)), rel=1e-6)


def test_zero_c2_reduces_to_the_linear_ace():
    w = I.config_c1()
    p = dataclasses.replace(I.ace_params(0), c2=np.zeros(512), fs_eps=0.01)
    e_fs, f_fs = O.ACEFS(p).eval(w.x, w.box)
    e_l, f_l = O.ACE(I.ace_params(0)).eval(w.x, w.box)
    assert np.array_equal(e_fs, e_l) and np.allclose(f_fs, f_l, rtol=0, atol=1e-15)


@pytest.mark.parametrize("scale", [-0.1, 0.1, -0.001])
def test_fs_forces_are_the_gradient_of_the_weighted_energy(scale):
    w = I.config_c1()
    p = I.ace_params_fs(0, c2_scale=scale)
    ace = O.ACEFS(p)
    g = np.random.Generator(np.random.PCG64(I.seed_for(1, 41)))
    wt = g.random(w.n)
    _, f = ace.eval(w.x, w.box, weights=wt)
    h = 1e-5
    for i in g.choice(w.n, 6, replace=False):
        for a in range(3):
            xp, xm = w.x.copy(), w.x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            ep, _ = ace.eval(xp, w.box)
            em, _ = ace.eval(xm, w.box)
            fd = -((wt * ep).sum() - (wt * em).sum()) / (2 * h)
            assert f[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_phi2_regimes_of_the_test_parameters():
    w = I.config_c1()
    for scale, lo, hi in ((-0.1, 0.02, 0.1), (0.1, -0.1, -0.02), (-0.001, 1e-4, 1e-3)):
        _, p2 = O.ACEFS(I.ace_params_fs(0, c2_scale=scale)).phis(w.x, w.box)
        assert lo < p2.min() and p2.max() < hi, (scale, p2.min(), p2.max())
