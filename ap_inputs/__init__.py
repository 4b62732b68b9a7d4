"""Seeded synthetic workloads for the adaptive-precision EAM/ACE force evaluation.

This module is shared by the CUDA path, the CPU oracle and the tests.  It only
builds inputs: lattices, displacements, masks, velocities and the random
potential parameters.  It contains none of the method's arithmetic (no
neighbour search, no centro-symmetry, no switching function, no potential).

Units: eV, Angstrom, fs, amu.  Every random draw uses numpy's PCG64 generator
seeded with ``seed_for(config, k) = 2411030020 + 100*config + k``.

Workloads (all copper-like FCC, a = 3.615 A):
  * c1  4x4x4 periodic cell, sigma = 0.05 A, spherical void r = 4 A -> 237 atoms.
  * c2  20x20x20 slab (x/y periodic, z free), hemispherical 0.3 A disorder of
        radius 15 A under the top surface, 300 K Maxwell-Boltzmann velocities.
  * c3  8x8x8 periodic cell, sigma = 0.1 A, lambda forced to a seeded mix of
        0, 1 and U(0,1); plus a batch of 64 cells of 4*n1*n2*n3 atoms.
  * c5  100x100x100 slab (4,000,000 atoms), bottom 3 (200) layers fixed, a
        spherical indenter (R = 50 A, k = 10 eV/A^3, 20 m/s) above the top surface.
  * c6  indented-slab snapshot of the c5 geometry (crater, graded disorder, vacancies,
        thermal noise) for the switching-zone parameter study.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SEED_BASE = 2411030020
A_CU = 3.615            # lattice parameter (A)
MASS_CU = 63.546        # amu
KB_EV = 8.617333262e-5  # eV/K
# 1 eV/(A amu) expressed in A/fs^2, from 1 eV = 1.602176634e-19 J, 1 amu = 1.66053906660e-27 kg
ACC_EV_A_AMU = 1.602176634e-19 / 1.66053906660e-27 * 1e-20 / 1e-10


def seed_for(config: int, k: int = 0) -> int:
    return SEED_BASE + 100 * config + k


def rng_for(config: int, k: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_for(config, k)))


@dataclasses.dataclass
class Box:
    lo: np.ndarray          # (3,) float64
    hi: np.ndarray          # (3,) float64
    periodic: np.ndarray    # (3,) bool

    @property
    def length(self) -> np.ndarray:
        return self.hi - self.lo


@dataclasses.dataclass
class HybridParams:
    """Switching-function parameters (Table 'model_parameters' of the paper)."""
    csp_lo: float = 2.5
    csp_hi: float = 3.0
    r_lo: float = 4.0
    r_hi: float = 12.0
    n_csp_avg: int = 11          # samples in the CSP window
    n_lam_avg: int = 11          # samples in the lambda window
    dlam_min: float = 1.0 / 110.0
    sample_every: int = 10       # lambda update period (MD steps)
    fcut_mode: int = 0           # 0 = polynomial as printed, 1 = C2-symmetric reading


HYB1 = HybridParams()
HYB2 = HybridParams(r_lo=8.0, r_hi=20.0)
# Single-evaluation parameter set used for the 237-atom cell (r_hi < L/2).
SINGLE_EVAL = HybridParams(r_lo=2.0, r_hi=3.5, n_csp_avg=1, n_lam_avg=1, sample_every=1)


@dataclasses.dataclass
class EAMParams:
    """Analytic EAM: exponential density, square-root embedding, Morse pair."""
    beta: float
    alpha: float
    A: float
    D: float
    rp: float
    r0: float = A_CU / math.sqrt(2.0)
    rc: float = 5.5
    h: float = 0.5

    def as_array(self) -> np.ndarray:
        return np.array([self.beta, self.alpha, self.A, self.D, self.rp, self.r0, self.rc, self.h])


EAM_NOMINAL = EAMParams(beta=3.0, alpha=1.6, A=0.42398, D=0.23925, rp=2.81322)


@dataclasses.dataclass
class MishinParams:
    """Mishin EAM2 copper (the paper's Appendix E functional forms).  Field order is
    the oracle's and the library's parameter order."""
    E1: float
    E2: float
    delta: float
    F0: float
    xi0: float
    xi2: float
    h: float
    q1: float
    q2: float
    q3: float
    q4: float
    Q1: float
    Q2: float
    S1: float
    S2: float
    S3: float
    a: float
    a1: float
    a2: float
    b1: float
    b2: float
    r01: float
    r02: float
    r03: float
    r04: float
    rs1: float
    rs2: float
    rs3: float
    rc: float

    def as_array(self) -> np.ndarray:
        return np.array([getattr(self, f.name) for f in dataclasses.fields(self)])


# The two parameter sets printed in the paper's table of the optimised EAM (Appendix E):
# the original EAM2 values and the values fitted at 300 K to the ACE potential.
MISHIN_ORIGINAL = MishinParams(
    E1=2.01458e+02, E2=6.59288e-03, delta=8.62250e-03, F0=0.0, xi0=-2.30000, xi2=1.40000, h=5.00370e-01,
    q1=-1.30000, q2=-9.00000e-01, q3=1.80000, q4=3.00000, Q1=4.00000e-01, Q2=3.00000e-01, S1=4.0, S2=40.0,
    S3=1150.0, a=3.80362, a1=2.97758, a2=1.54927, b1=1.73940e-01, b2=5.35661e+02, r01=8.35910e-01,
    r02=4.46867, r03=-2.19885, r04=-2.61984e+02, rs1=2.24, rs2=1.80, rs3=1.20, rc=5.50679)
MISHIN_FIT_300K = MishinParams(
    E1=2.01486e+02, E2=6.44057e-03, delta=2.18016e-02, F0=-1.50036e-01, xi0=-2.30089, xi2=1.39912, h=5.00370e-01,
    q1=-1.29894, q2=-8.99672e-01, q3=1.79940, q4=2.99944, Q1=3.99178e-01, Q2=3.00455e-01, S1=4.0, S2=40.0,
    S3=1150.0, a=3.80541, a1=2.96972, a2=1.55510, b1=1.66589e-01, b2=5.35661e+02, r01=8.36347e-01,
    r02=4.46690, r03=-2.19834, r04=-2.61984e+02, rs1=2.24, rs2=1.80, rs3=1.20, rc=5.50679)


@dataclasses.dataclass
class ACEParams:
    """Single-species ACE: radial mixing W[l][n][k] and coefficients c[v] of phi^(1);
    with c2, the Finnis-Sinclair form E = phi^(1) + F(phi^(2)) (phi^(2) = sum c2_v B_v)."""
    W: np.ndarray            # (5, 8, 8) float64, indexed [l][n][k]
    c: np.ndarray            # (512,) float64; the first n_basis entries are used
    rc: float = 7.0
    n0: float = 10.0         # A-basis normalisation N0
    c2: Optional[np.ndarray] = None   # (512,) coefficients of phi^(2), or None (linear ACE)
    fs_eps: float = 0.1      # regularisation of the square-root embedding


@dataclasses.dataclass
class Indenter:
    center0: np.ndarray      # (3,) initial centre (A)
    velocity: np.ndarray     # (3,) A/fs
    radius: float = 50.0
    k: float = 10.0          # eV/A^3


@dataclasses.dataclass
class Workload:
    name: str
    x: np.ndarray                    # (N,3) float64
    box: Box
    mass: np.ndarray                 # (N,) float64
    fixed: np.ndarray                # (N,) uint8: 1 = fixed atom (lambda = 1, v = 0)
    v: Optional[np.ndarray] = None   # (N,3) float64, A/fs
    lam: Optional[np.ndarray] = None # (N,) float64 forced lambda, or None
    indenter: Optional[Indenter] = None
    dt: float = 1.0
    hyb: HybridParams = dataclasses.field(default_factory=HybridParams)

    @property
    def n(self) -> int:
        return self.x.shape[0]


# ----------------------------------------------------------------------------- lattices
_FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


def fcc_lattice(nx: int, ny: int, nz: int, a: float = A_CU) -> np.ndarray:
    """FCC positions, z-layer-major order (k outer, j, i, basis inner)."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + _FCC_BASIS[None, :, :]).reshape(-1, 3) * a
    return pos


def eam_params(seed_config: int = 0, k: int = 1) -> EAMParams:
    """Nominal parameters times (1 + 0.02 N(0,1)), seeded."""
    if seed_config < 0:
        return dataclasses.replace(EAM_NOMINAL)
    g = rng_for(seed_config, k)
    f = 1.0 + 0.02 * g.standard_normal(5)
    n = EAM_NOMINAL
    return EAMParams(beta=n.beta * f[0], alpha=n.alpha * f[1], A=n.A * f[2], D=n.D * f[3], rp=n.rp * f[4])


def ace_params(seed_config: int = 0, k: int = 2, c_std: float = 0.01) -> ACEParams:
    """W_l = I + 0.1 N(0,1) for l = 0..4, and c ~ N(0, c_std^2) (512 draws)."""
    g = rng_for(seed_config, k)
    W = np.eye(8)[None, :, :] + 0.1 * g.standard_normal((5, 8, 8))
    c = c_std * g.standard_normal(512)
    return ACEParams(W=W, c=c)


def ace_params_fs(seed_config: int = 0, k: int = 2, c2_scale: float = -0.1, fs_eps: float = 0.01) -> ACEParams:
    """ace_params plus seeded phi^(2) coefficients c2 = c2_scale N(0, 1) (512 draws).  With
    this seed phi^(2) keeps one sign over FCC-like cells: c2_scale = -0.1 puts it near
    +0.05 (the square-root branch), +0.1 near -0.05 (the odd extension), -0.001 near
    +5e-4 (the transition, |phi| ~ 5 eps^2)."""
    p = ace_params(seed_config, k)
    g = rng_for(seed_config, k + 40)
    return dataclasses.replace(p, c2=c2_scale * g.standard_normal(512), fs_eps=fs_eps)


ANCHOR_FILE = __import__("os").path.join(__import__("os").path.dirname(__file__), "ace_anchor.npz")


def ace_params_anchored() -> ACEParams:
    """EAM-anchored ACE for the molecular-dynamics workloads: the stored
    coefficients c = c_fit + N(0, 0.01^2) written by oracle/fit_ace_anchor.py (a
    ridge fit of the linear ACE to the synthetic EAM on bulk snapshots) with the
    same radial mixing W as ace_params(0).  Loaded from a data file; nothing is
    computed here."""
    d = np.load(ANCHOR_FILE)
    return ACEParams(W=np.array(d["W"]), c=np.array(d["c"]))


def ace_for_config(config: int) -> ACEParams:
    """Random coefficients for the single-evaluation cells (1, 3), anchored ones
    for the dynamics workloads (2, 4, 5)."""
    return ace_params_anchored() if config in (2, 4, 5) else ace_params(0)


def maxwell_boltzmann(mass: np.ndarray, mobile: np.ndarray, T: float, g: np.random.Generator) -> np.ndarray:
    """v ~ N(0, kT/m) per component, COM removed, rescaled to T with 3N_mobile - 3 DOF."""
    n = mass.shape[0]
    sig = np.sqrt(KB_EV * T * ACC_EV_A_AMU / mass)
    v = g.standard_normal((n, 3)) * sig[:, None]
    v[~mobile] = 0.0
    m = mass[mobile]
    vcm = (m[:, None] * v[mobile]).sum(0) / m.sum()
    v[mobile] -= vcm
    ke = 0.5 * (m[:, None] * v[mobile] ** 2).sum() / ACC_EV_A_AMU
    dof = 3 * int(mobile.sum()) - 3
    t_now = 2.0 * ke / (dof * KB_EV)
    v[mobile] *= math.sqrt(T / t_now)
    return v


def _periodic_box(nx: int, ny: int, nz: int, a: float = A_CU) -> Box:
    return Box(lo=np.zeros(3), hi=np.array([nx, ny, nz], float) * a, periodic=np.array([True, True, True]))


def _slab_box(nx: int, ny: int, nz: int, a: float = A_CU, pad: float = 10.0) -> Box:
    ztop = (nz - 0.5) * a
    return Box(lo=np.array([0.0, 0.0, -pad]), hi=np.array([nx * a, ny * a, ztop + pad]),
               periodic=np.array([True, True, False]))


# ----------------------------------------------------------------------------- configs
def config_c1() -> Workload:
    """237-atom periodic cell with a 4 A void at a lattice site, sigma = 0.05 A."""
    g = rng_for(1, 0)
    x = fcc_lattice(4, 4, 4)
    box = _periodic_box(4, 4, 4)
    centre = np.array([2.0, 2.0, 2.0]) * A_CU          # a lattice site
    keep = np.linalg.norm(x - centre, axis=1) >= 4.0
    x = x[keep]
    x = x + 0.05 * g.standard_normal(x.shape)
    n = x.shape[0]
    return Workload("c1_fcc4_void", x, box, np.full(n, MASS_CU), np.zeros(n, np.uint8), hyb=SINGLE_EVAL)


def config_c2(hyb: HybridParams = HYB1, variant: int = 0) -> Workload:
    """32,000-atom slab with a hemispherical 0.3 A disordered region; 300 K velocities.
    variant > 0 draws the disorder and velocities from other seeds (held-out slabs)."""
    g = rng_for(2, 0 if variant == 0 else 20 + 2 * variant)
    nx = ny = nz = 20
    x = fcc_lattice(nx, ny, nz)
    box = _slab_box(nx, ny, nz)
    ztop = (nz - 0.5) * A_CU
    centre = np.array([nx * A_CU / 2, ny * A_CU / 2, ztop])
    dis = (np.linalg.norm(x - centre, axis=1) < 15.0) & (x[:, 2] <= ztop + 1e-9)
    x[dis] += 0.3 * g.standard_normal((int(dis.sum()), 3))
    n = x.shape[0]
    mass = np.full(n, MASS_CU)
    v = maxwell_boltzmann(mass, np.ones(n, bool), 300.0, rng_for(2, 1 if variant == 0 else 21 + 2 * variant))
    name = "c2_slab20" if variant == 0 else f"c2_slab20_v{variant}"
    return Workload(name, x, box, mass, np.zeros(n, np.uint8), v=v, hyb=hyb)


def config_c3() -> Workload:
    """2,048-atom periodic cell, sigma = 0.1 A, lambda forced to {0, 1, U(0,1)} thirds."""
    g = rng_for(3, 0)
    x = fcc_lattice(8, 8, 8)
    x = x + 0.1 * g.standard_normal(x.shape)
    n = x.shape[0]
    cat = g.integers(0, 3, n)
    lam = np.where(cat == 0, 0.0, np.where(cat == 1, 1.0, g.uniform(0.0, 1.0, n)))
    return Workload("c3_fcc8", x, _periodic_box(8, 8, 8), np.full(n, MASS_CU), np.zeros(n, np.uint8),
                    lam=lam, hyb=SINGLE_EVAL)


def config_c3_batch(n_cells: int = 64) -> list:
    """Independent periodic cells of 4*n1*n2*n3 atoms, n_i in {5..10} (500-4,000 atoms)."""
    g = rng_for(3, 1)
    out = []
    for c in range(n_cells):
        nn = g.integers(5, 11, 3)
        x = fcc_lattice(*nn)
        x = x + 0.1 * g.standard_normal(x.shape)
        n = x.shape[0]
        cat = g.integers(0, 3, n)
        lam = np.where(cat == 0, 0.0, np.where(cat == 1, 1.0, g.uniform(0.0, 1.0, n)))
        out.append(Workload(f"c3_cell{c}", x, _periodic_box(*nn), np.full(n, MASS_CU),
                            np.zeros(n, np.uint8), lam=lam, hyb=SINGLE_EVAL))
    return out


def config_c5(ncell: int = 100, hyb: HybridParams = HYB2, T: float = 300.0, nxy: Optional[int] = None) -> Workload:
    """Nanoindentation-shaped slab: ncell^3 FCC cells (4,000,000 atoms at ncell = 100).
    nxy < ncell cuts a laterally periodic column of the same depth (nxy x nxy x ncell)."""
    nx = ny = ncell if nxy is None else nxy
    nz = ncell
    x = fcc_lattice(nx, ny, nz)
    box = _slab_box(nx, ny, nz)
    n = x.shape[0]
    fixed = (x[:, 2] < 1.25 * A_CU).astype(np.uint8)      # bottom three (200) layers
    mass = np.full(n, MASS_CU)
    v = maxwell_boltzmann(mass, fixed == 0, T, rng_for(5, 1))
    ztop = (nz - 0.5) * A_CU
    R = 50.0
    ind = Indenter(center0=np.array([nx * A_CU / 2, ny * A_CU / 2, ztop + R]),
                   velocity=np.array([0.0, 0.0, -2.0e-4]), radius=R, k=10.0)
    return Workload(f"c5_indent{ncell}", x, box, mass, fixed, v=v, indenter=ind, hyb=hyb)


def config_c6(nxy: int = 100, nz: int = 100, depth: float = 8.0) -> Workload:
    """Indented-slab snapshot for the switching-zone parameter study (a stand-in for the
    paper's nanoindentation snapshot with dislocations): the c5 slab geometry with
    - the atoms inside the R = 50 A indenter sphere, its tip `depth` below the surface, removed;
    - a graded disordered zone under the contact: extra Gaussian displacement of width
      0.3 exp(-d / 12 A) for atoms within d < 40 A of the contact point;
    - 0.2 % of the atoms within 45 A of the contact point removed (vacancies);
    - thermal Gaussian displacement of width 0.06 A on every mobile atom.
    Bottom three (200) layers fixed; no velocities (a single-step study).  4,000,000
    lattice sites at nxy = nz = 100."""
    g = rng_for(6, 0)
    x = fcc_lattice(nxy, nxy, nz)
    box = _slab_box(nxy, nxy, nz)
    ztop = (nz - 0.5) * A_CU
    R = 50.0
    contact = np.array([nxy * A_CU / 2, nxy * A_CU / 2, ztop - depth])
    centre = contact + np.array([0.0, 0.0, R])
    keep = np.linalg.norm(x - centre, axis=1) >= R
    d = np.linalg.norm(x - contact, axis=1)
    keep &= ~((d < 45.0) & (g.uniform(size=x.shape[0]) < 0.002))
    x, d = x[keep], d[keep]
    fixed = (x[:, 2] < 1.25 * A_CU).astype(np.uint8)
    mobile = fixed == 0
    sig = np.where(mobile, 0.06, 0.0)
    sig = np.where(mobile & (d < 40.0), np.hypot(sig, 0.3 * np.exp(-d / 12.0)), sig)
    x = x + sig[:, None] * g.standard_normal(x.shape)
    n = x.shape[0]
    return Workload(f"c6_snapshot{nxy}x{nz}", x, box, np.full(n, MASS_CU), fixed, hyb=HYB1)


# ----------------------------------------------------------------------------- selector data (c4)
# Orthorhombic repeat cells of FCC with a (100), (110) or (111) surface normal to z:
# unit vectors of x, y, z in cubic coordinates, repeat lengths (units of a), atoms per cell.
_ORIENT = {
    100: (np.eye(3), np.array([1.0, 1.0, 1.0]), 4),
    110: (np.array([[0.0, 0.0, 1.0], [1.0, -1.0, 0.0] / np.sqrt(2.0), [1.0, 1.0, 0.0] / np.sqrt(2.0)]),
          np.array([1.0, 1.0 / np.sqrt(2.0), 1.0 / np.sqrt(2.0)]), 2),
    111: (np.array([[1.0, -1.0, 0.0] / np.sqrt(2.0), [1.0, 1.0, -2.0] / np.sqrt(6.0), [1.0, 1.0, 1.0] / np.sqrt(3.0)]),
          np.array([1.0 / np.sqrt(2.0), np.sqrt(6.0) / 2.0, np.sqrt(3.0)]), 6),
}


def fcc_oriented(surface: int, nx: int, ny: int, nz: int, a: float = A_CU):
    """FCC sites of nx x ny x nz orthorhombic repeat cells whose z axis is the
    [100], [110] or [111] direction.  Returns (positions sorted by z, y, x; box lengths)."""
    E, per, per_cell = _ORIENT[surface]
    L = per * a * np.array([nx, ny, nz])
    m = int(np.ceil(np.linalg.norm(L) / a)) + 2
    c = np.arange(-m, m + 1)
    k, j, i = np.meshgrid(c, c, c, indexing="ij")
    cells = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    sites = ((cells[:, None, :] + _FCC_BASIS[None, :, :]).reshape(-1, 3) * a) @ E.T
    eps = 1e-6
    keep = np.all((sites >= -eps) & (sites < L - eps), axis=1)
    x = sites[keep]
    if x.shape[0] != per_cell * nx * ny * nz:
        raise RuntimeError("oriented FCC cell count mismatch")
    order = np.lexsort((np.round(x[:, 0], 6), np.round(x[:, 1], 6), np.round(x[:, 2], 6)))
    return x[order], L


def config_c4(k: int) -> Workload:
    """Selector training structure k in [0, 200), about 5,000 atoms, 40 per category:
    0 bulk with thermal-like Gaussian displacements (sigma 0.05-0.09 A);
    1 bulk with 0.5-2 % vacancies (sigma 0.04-0.09 A);
    2 slabs with (100), (110), (111) surfaces in turn (sigma 0.04-0.09 A, 10 A vacuum);
    3 bulk with disorder sigma 0.05-0.5 A;
    4 starting points of 300-1200 K EAM molecular dynamics (bulk for even k, (100)
      slab for odd k; lattice sites plus sigma 0.02 A, Maxwell-Boltzmann velocities at T).
    Categories 0-3 carry no velocities."""
    if not 0 <= k < 200:
        raise ValueError("k in [0, 200)")
    g = rng_for(4, k)
    cat = k // 40
    mass_of = lambda x: np.full(x.shape[0], MASS_CU)
    if cat in (0, 1, 3):
        x = fcc_lattice(11, 11, 10)
        box = _periodic_box(11, 11, 10)
        if cat == 1:
            nv = int(round(g.uniform(0.005, 0.02) * x.shape[0]))
            x = np.delete(x, g.choice(x.shape[0], nv, replace=False), axis=0)
        sigma = g.uniform(0.05, 0.5) if cat == 3 else g.uniform(0.04 if cat == 1 else 0.05, 0.09)
        x = x + sigma * g.standard_normal(x.shape)
        return Workload(f"c4_{k}", x, box, mass_of(x), np.zeros(x.shape[0], np.uint8), hyb=HYB1)
    if cat == 2:
        surface = (100, 110, 111)[k % 3]
        dims = {100: (11, 11, 10), 110: (10, 14, 18), 111: (12, 7, 10)}[surface]
        x, L = fcc_oriented(surface, *dims)
        x = x + g.uniform(0.04, 0.09) * g.standard_normal(x.shape)
        box = Box(lo=np.array([0.0, 0.0, -10.0]), hi=np.array([L[0], L[1], L[2] + 10.0]),
                  periodic=np.array([True, True, False]))
        return Workload(f"c4_{k}_s{surface}", x, box, mass_of(x), np.zeros(x.shape[0], np.uint8), hyb=HYB1)
    T = g.uniform(300.0, 1200.0)
    if k % 2 == 0:
        x = fcc_lattice(11, 11, 10)
        box = _periodic_box(11, 11, 10)
    else:
        x = fcc_lattice(11, 11, 10)
        box = _slab_box(11, 11, 10)
    x = x + 0.02 * g.standard_normal(x.shape)
    m = mass_of(x)
    v = maxwell_boltzmann(m, np.ones(x.shape[0], bool), T, g)
    return Workload(f"c4_{k}_md{int(T)}", x, box, m, np.zeros(x.shape[0], np.uint8), v=v, hyb=HYB1)


def sample_atoms(n: int, count: int, config: int, k: int = 7) -> np.ndarray:
    """Seeded sorted sample of atom indices (for sampled parity checks)."""
    g = rng_for(config, k)
    return np.sort(g.choice(n, size=min(count, n), replace=False))
