"""Pins of the Mishin EAM2 oracle (Appendix E forms, the paper's two parameter sets)
against the FCC properties the paper prints (tests/golden/mishin_eam2.txt) and
against finite differences."""
import os

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import ap_inputs as I
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "mishin_eam2.txt")
GPA = 160.21766208        # eV/A^3 -> GPa


def golden():
    out = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        s, q, v = line.split()
        out[(s, q)] = float(v)
    return out


SETS = {"original": I.MISHIN_ORIGINAL, "fit": I.MISHIN_FIT_300K}


def energy(p, x, L):
    box = I.Box(lo=np.zeros(3), hi=np.asarray(L, float), periodic=np.array([True] * 3))
    e, *_ = O.eam_mishin(x, box, p)
    return e.sum()


def lattice(p):
    f = lambda a: energy(p, I.fcc_lattice(3, 3, 3, a), [3 * a] * 3) / 108
    r = minimize_scalar(f, bounds=(3.5, 3.75), method="bounded", options={"xatol": 1e-11})
    return r.x, r.fun


@pytest.mark.parametrize("name", ["original", "fit"])
def test_lattice_constant_and_cohesive_energy(name):
    g = golden()
    a0, ecoh = lattice(SETS[name])
    assert a0 == pytest.approx(g[(name, "a0_A")], abs=5e-5)
    assert ecoh == pytest.approx(g[(name, "ecoh_eV")], abs=1e-4)


@pytest.mark.parametrize("name", ["original", "fit"])
def test_elastic_constants(name):
    g = golden()
    p = SETS[name]
    a0, _ = lattice(p)
    x0 = I.fcc_lattice(3, 3, 3, a0)
    L0 = np.array([3 * a0] * 3)
    V = L0.prod()
    h = 1e-4

    def e_strain(eps):                      # diagonal strain
        s = 1.0 + np.asarray(eps)
        return energy(p, x0 * s, L0 * s)

    e0 = e_strain([0, 0, 0])
    c11 = (e_strain([h, 0, 0]) + e_strain([-h, 0, 0]) - 2 * e0) / (h * h * V)
    cpp = (e_strain([h, h, 0]) + e_strain([-h, -h, 0]) - 2 * e0) / (h * h * V)   # = 2 C11 + 2 C12
    c12 = 0.5 * cpp - c11
    # C44 from the [110]-oriented cell: C'33 = (C11 + C12 + 2 C44) / 2
    xo, Lo = I.fcc_oriented(110, 4, 6, 6, a0)
    Vo = Lo.prod()
    eo = lambda e3: energy(p, xo * np.array([1, 1, 1 + e3]), Lo * np.array([1, 1, 1 + e3]))
    c33p = (eo(h) + eo(-h) - 2 * eo(0.0)) / (h * h * Vo)
    c44 = c33p - 0.5 * (c11 + c12)
    assert c11 * GPA == pytest.approx(g[(name, "c11_GPa")], rel=2e-3)
    assert c12 * GPA == pytest.approx(g[(name, "c12_GPa")], rel=2e-3)
    assert c44 * GPA == pytest.approx(g[(name, "c44_GPa")], rel=2e-3)


def test_forces_are_minus_the_energy_gradient():
    p = I.MISHIN_FIT_300K
    gen = np.random.Generator(np.random.PCG64(I.seed_for(7, 3)))
    x = I.fcc_lattice(3, 3, 3) + 0.15 * gen.standard_normal((108, 3))
    box = I.Box(lo=np.zeros(3), hi=np.full(3, 3 * I.A_CU), periodic=np.array([True] * 3))
    w = gen.random(108)
    _, f, _, _ = O.eam_mishin(x, box, p, weights=w)
    hh = 1e-5
    for i in gen.choice(108, 5, replace=False):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += hh
            xm[i, a] -= hh
            ep, *_ = O.eam_mishin(xp, box, p)
            em, *_ = O.eam_mishin(xm, box, p)
            assert f[i, a] == pytest.approx(-((w * ep).sum() - (w * em).sum()) / (2 * hh), rel=1e-6, abs=1e-8)


def test_core_terms_and_guarded_density():
    p = I.MISHIN_ORIGINAL
    phi, dphi, z, dz = O.mishin_terms(p, 1.0)            # inside all three core terms
    assert np.isfinite([phi, dphi, z, dz]).all()
    # the second density exponent underflows: zeta is a exp(-b1 (r - r03)^2) psi
    r = 2.5
    u = (r - p.rc) / p.h
    psi = u ** 4 / (1 + u ** 4)
    _, _, z, _ = O.mishin_terms(p, r)
    assert z == pytest.approx(p.a * np.exp(-p.b1 * (r - p.r03) ** 2) * psi, rel=1e-14)
    assert O.mishin_terms(p, p.rc)[:3] == (0.0, 0.0, 0.0) or abs(O.mishin_terms(p, p.rc)[0]) < 1e-300
    xi, dxi = O.mishin_embed(p, 1.0)
    assert xi == pytest.approx(p.xi0) and dxi == 0.0
