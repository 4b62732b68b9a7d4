"""CPU oracle of the adaptive-precision force evaluation (arXiv 2411.03002).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The product path (the
CUDA library and its binding) never does, and the two share no code.

Everything is FP64 and follows the paper's definitions in the paper's order:
  * neighbour sets, centro-symmetry (Appendix A, Eq. csp_1_i), f_cut, lambda_0
    (Eq. lambda_1_i), lambda_min (Eq. lambda_2_i): ``ap_oracle.c``;
  * time averages (Eqs. csp_2_i, lambda_3_i) and the minimum-step hysteresis
    (Eq. lambda_4_i): ``LambdaState`` below;
  * EAM site energy (Eq. energy_eam) and linear ACE site energy (Eq. energy_ace):
    ``ap_oracle.c``;
  * blended energy (Eq. energy_hyb) and the applied force at fixed lambda
    (Eq. F_i_d): ``hybrid``;
  * velocity Verlet with the lambda step (Eq. vv): ``md_step``.

Readings where the paper is ambiguous:
  * lambda_0 = 1 - f_cut((CSP_hi - CSP_avg)/(CSP_hi - CSP_lo)): the printed argument
    is oriented so that it is 0 for precise and 1 for fast atoms, as Appendix B
    states in words.
  * the averaging windows include the current sample; histories start filled
    with the first sample; the canonical sum runs oldest to newest.
  * atoms with fewer than 12 neighbours inside the CSP search radius get CSP = +inf.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ap_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
ACC = 1.602176634e-19 / 1.66053906660e-27 * 1e-20 / 1e-10   # A/fs^2 per eV/(A amu)
KB = 8.617333262e-5


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O2 -ffp-contract=off, OpenMP over atoms)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-D_DEFAULT_SOURCE", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("periodic", ctypes.c_int * 3)]


class _EAM(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("beta", "alpha", "A", "D", "rp", "r0", "rc", "h")]


_MISHIN_FIELDS = ("E1", "E2", "delta", "F0", "xi0", "xi2", "h", "q1", "q2", "q3", "q4", "Q1", "Q2", "S1", "S2",
                  "S3", "a", "a1", "a2", "b1", "b2", "r01", "r02", "r03", "r04", "rs1", "rs2", "rs3", "rc")


class _Mishin(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in _MISHIN_FIELDS]


def _mishin(p) -> _Mishin:
    return _Mishin(*[float(getattr(p, k)) for k in _MISHIN_FIELDS])


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.orc_neighbors.restype = ctypes.c_int
        _lib.orc_neighbors.argtypes = [ctypes.c_int, P, P, ctypes.c_double, ctypes.c_int, P, P, P]
        _lib.orc_neighbors_of.restype = ctypes.c_int
        _lib.orc_neighbors_of.argtypes = [ctypes.c_int, P, P, ctypes.c_double, ctypes.c_int, P, ctypes.c_int, P, P, P]
        _lib.orc_csp.argtypes = [ctypes.c_int, P, P, P, P, P, ctypes.c_int, P, P]
        _lib.orc_fcut.restype = ctypes.c_double
        _lib.orc_fcut.argtypes = [ctypes.c_double, ctypes.c_int]
        _lib.orc_dfcut.restype = ctypes.c_double
        _lib.orc_dfcut.argtypes = [ctypes.c_double, ctypes.c_int]
        _lib.orc_lambda0.argtypes = [ctypes.c_int, P, ctypes.c_double, ctypes.c_double, ctypes.c_int, P, P]
        _lib.orc_lambda_min.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int, P]
        _lib.orc_eam.argtypes = [ctypes.c_int, P, P, P, P, P, ctypes.c_int, P, P, P, P, P, P]
        _lib.orc_eam_pair.argtypes = [P, ctypes.c_int, P, P, P, P, P]
        _lib.orc_eam_mishin.argtypes = [ctypes.c_int, P, P, P, P, P, ctypes.c_int, P, P, P, P, P, P]
        _lib.orc_mishin_pair.argtypes = [P, ctypes.c_double, P, P, P, P]
        _lib.orc_mishin_embed.argtypes = [P, ctypes.c_double, P, P]
        _lib.orc_ace_create.restype = P
        _lib.orc_ace_create.argtypes = [P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        _lib.orc_ace_destroy.argtypes = [P]
        _lib.orc_ace_nbasis.restype = ctypes.c_int
        _lib.orc_ace_nbasis.argtypes = [P]
        _lib.orc_ace_basis_desc.argtypes = [P, P]
        _lib.orc_ace_gaunt.argtypes = [P, P]
        _lib.orc_ylm.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P]
        _lib.orc_ace_basis.argtypes = [P, ctypes.c_int, P, P, P, P, P, P, ctypes.c_int, P, P]
        _lib.orc_ace_eval.argtypes = [P, ctypes.c_int, P, P, P, P, P, ctypes.c_int, P, P, P]
        _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def num_threads() -> int:
    return lib().orc_num_threads()


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _box(box) -> _Box:
    b = _Box()
    for k in range(3):
        b.lo[k] = float(box.lo[k])
        b.hi[k] = float(box.hi[k])
        b.periodic[k] = int(bool(box.periodic[k]))
    return b


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------- neighbours
class NeighborList:
    """Rows of (j, s) with |x_j + s L - x_i| < rc, ordered by j then s."""

    def __init__(self, cnt, j, s, cap, rc, ids=None):
        self.cnt, self.j, self.s, self.cap, self.rc, self.ids = cnt, j, s, cap, rc, ids

    def pairs(self, row: int) -> set:
        c = int(self.cnt[row])
        return {(int(self.j[row, q]), *map(int, self.s[row, q])) for q in range(c)}


def neighbors(x, box, rc: float, cap: int = 256) -> NeighborList:
    x = _f64(x)
    n = x.shape[0]
    b = _box(box)
    while True:
        cnt = np.zeros(n, np.int32)
        j = np.zeros((n, cap), np.int32)
        s = np.zeros((n, cap, 3), np.int32)
        m = lib().orc_neighbors(n, _p(x), ctypes.byref(b), rc, cap, _p(cnt), _p(j), _p(s))
        if m <= cap:
            return NeighborList(cnt, j, s, cap, rc)
        cap = m + 16


def neighbors_of(x, box, rc: float, ids, cap: int = 256) -> NeighborList:
    x = _f64(x)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    b = _box(box)
    while True:
        m_ = ids.shape[0]
        cnt = np.zeros(m_, np.int32)
        j = np.zeros((m_, cap), np.int32)
        s = np.zeros((m_, cap, 3), np.int32)
        m = lib().orc_neighbors_of(x.shape[0], _p(x), ctypes.byref(b), rc, m_, _p(ids), cap, _p(cnt), _p(j), _p(s))
        if m <= cap:
            return NeighborList(cnt, j, s, cap, rc, ids)
        cap = m + 16


# ----------------------------------------------------------------------------- switching
def fcut(x: float, mode: int = 0) -> float:
    return lib().orc_fcut(float(x), int(mode))


def dfcut(x: float, mode: int = 0) -> float:
    return lib().orc_dfcut(float(x), int(mode))


def csp(x, box, r_search: float = 6.5, changeable=None, nl: Optional[NeighborList] = None) -> np.ndarray:
    """CSP_i (LAMMPS definition, N = 12) over every image within r_search."""
    x = _f64(x)
    if nl is None:
        nl = neighbors(x, box, r_search)
    ch = None if changeable is None else np.ascontiguousarray(changeable, dtype=np.uint8)
    out = np.zeros(x.shape[0])
    lib().orc_csp(x.shape[0], _p(x), ctypes.byref(_box(box)), _p(nl.cnt), _p(nl.j), _p(nl.s), nl.cap, _p(ch),
                  _p(out))
    return out


def lambda0(csp_avg, csp_lo: float, csp_hi: float, mode: int = 0, changeable=None) -> np.ndarray:
    c = _f64(csp_avg)
    ch = None if changeable is None else np.ascontiguousarray(changeable, dtype=np.uint8)
    out = np.zeros(c.shape[0])
    lib().orc_lambda0(c.shape[0], _p(c), csp_lo, csp_hi, mode, _p(ch), _p(out))
    return out


def lambda_min(x, box, lam0, r_lo: float, r_hi: float, mode: int = 0, changeable=None) -> np.ndarray:
    x = _f64(x)
    l0 = _f64(lam0)
    ch = None if changeable is None else np.ascontiguousarray(changeable, dtype=np.uint8)
    out = np.zeros(x.shape[0])
    lib().orc_lambda_min(x.shape[0], _p(x), ctypes.byref(_box(box)), _p(l0), _p(ch), r_lo, r_hi, mode, _p(out))
    return out


def canonical_mean(hist: np.ndarray, newest: int) -> np.ndarray:
    """Mean of a ring buffer [n_s, N], summed oldest -> newest in FP64, divided by n_s."""
    ns = hist.shape[0]
    s = hist[(newest + 1) % ns].copy()
    for q in range(1, ns):
        s = s + hist[(newest + 1 + q) % ns]
    return s / float(ns)


def msz_update(lam_avg, lam_prev, dlam_min: float) -> np.ndarray:
    """Eq. lambda_4_i: take lambda_avg if |lambda_avg - previous| >= dlam_min or
    lambda_avg is exactly 0 or 1, else keep the previous value."""
    take = (np.abs(lam_avg - lam_prev) >= dlam_min) | (lam_avg == 0.0) | (lam_avg == 1.0)
    return np.where(take, lam_avg, lam_prev)


class LambdaState:
    """Histories of CSP and lambda_min and the previous lambda (Appendix B)."""

    def __init__(self, n: int, n_csp: int, n_lam: int):
        self.csp_hist = np.zeros((n_csp, n))
        self.lam_hist = np.zeros((n_lam, n))
        self.lam_prev = np.ones(n)
        self.pos_csp = -1
        self.pos_lam = -1
        self.started = False

    def push(self, hist: np.ndarray, pos: int, sample: np.ndarray) -> int:
        if not self.started:
            hist[:] = sample[None, :]
            return 0
        pos = (pos + 1) % hist.shape[0]
        hist[pos] = sample
        return pos


def classify(state: LambdaState, x, box, hyb, changeable=None, r_search: float = 6.5, score=None,
             score_lo: float = 0.0, score_hi: float = 1.0):
    """One lambda update (Appendix B): CSP -> CSP_avg -> lambda_0 -> lambda_min ->
    lambda_avg -> lambda_avg,msz.  Returns (lam, lam0, csp_sample, csp_avg, lam_min, lam_avg).
    With ``score`` (another detector's per-atom score, larger = more in need of the
    precise potential), that score replaces CSP in the history and in the f_cut
    argument, with thresholds (score_lo, score_hi) in place of (CSP_lo, CSP_hi)."""
    x = _f64(x)
    ch = None if changeable is None else np.ascontiguousarray(changeable, dtype=np.uint8)
    c = csp(x, box, r_search, ch) if score is None else _f64(score)
    lo, hi = (hyb.csp_lo, hyb.csp_hi) if score is None else (score_lo, score_hi)
    state.pos_csp = state.push(state.csp_hist, state.pos_csp, c)
    cavg = canonical_mean(state.csp_hist, state.pos_csp)
    l0 = lambda0(cavg, lo, hi, hyb.fcut_mode, ch)
    lmin = lambda_min(x, box, l0, hyb.r_lo, hyb.r_hi, hyb.fcut_mode, ch)
    state.pos_lam = state.push(state.lam_hist, state.pos_lam, lmin)
    lavg = canonical_mean(state.lam_hist, state.pos_lam)
    if not state.started:
        prev = lavg.copy()
        state.started = True
    else:
        prev = state.lam_prev
    lam = msz_update(lavg, prev, hyb.dlam_min)
    if ch is not None:
        lam = np.where(ch == 0, 1.0, lam)
    state.lam_prev = lam.copy()
    return lam, l0, c, cavg, lmin, lavg


# ----------------------------------------------------------------------------- potentials
def eam(x, box, p, weights=None, nl: Optional[NeighborList] = None):
    """EAM site energies and F = -grad sum_i w_i E_i^f.  p: ap_inputs.EAMParams."""
    x = _f64(x)
    n = x.shape[0]
    if nl is None:
        nl = neighbors(x, box, p.rc)
    e = np.zeros(n)
    f = np.zeros((n, 3))
    rho = np.zeros(n)
    dxi = np.zeros(n)
    pp = _EAM(p.beta, p.alpha, p.A, p.D, p.rp, p.r0, p.rc, p.h)
    w = None if weights is None else _f64(weights)
    lib().orc_eam(n, _p(x), ctypes.byref(_box(box)), _p(nl.cnt), _p(nl.j), _p(nl.s), nl.cap, ctypes.byref(pp),
                  _p(w), _p(e), _p(f), _p(rho), _p(dxi))
    return e, f, rho, dxi


def eam_mishin(x, box, p, weights=None, nl: Optional[NeighborList] = None):
    """Mishin EAM2 site energies and F = -grad sum_i w_i E_i^f (Appendix E forms).
    p: ap_inputs.MishinParams.  Returns (E, F, rho, xi'(rho))."""
    x = _f64(x)
    n = x.shape[0]
    if nl is None:
        nl = neighbors(x, box, p.rc)
    e, f, rho, dxi = np.zeros(n), np.zeros((n, 3)), np.zeros(n), np.zeros(n)
    w = None if weights is None else _f64(weights)
    pp = _mishin(p)
    lib().orc_eam_mishin(n, _p(x), ctypes.byref(_box(box)), _p(nl.cnt), _p(nl.j), _p(nl.s), nl.cap, ctypes.byref(pp),
                         _p(w), _p(e), _p(f), _p(rho), _p(dxi))
    return e, f, rho, dxi


def mishin_terms(p, r: float):
    """(Phi, Phi', zeta, zeta') of the Mishin EAM2 at distance r."""
    out = [ctypes.c_double() for _ in range(4)]
    lib().orc_mishin_pair(ctypes.byref(_mishin(p)), float(r), *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def mishin_embed(p, x: float):
    """(xi, xi') of the Mishin EAM2 at density x (including the fitted offset F0)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().orc_mishin_embed(ctypes.byref(_mishin(p)), float(x), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def eam_any(x, box, p, weights=None, nl: Optional[NeighborList] = None):
    """EAM with either parameter type (analytic synthetic or Mishin EAM2)."""
    if hasattr(p, "E1"):
        return eam_mishin(x, box, p, weights, nl)
    return eam(x, box, p, weights, nl)


def eam_pair(p, r):
    """zeta(r), zeta'(r), Phi(r), Phi'(r) of the analytic EAM at the distances r."""
    r = _f64(r).reshape(-1)
    out = [np.zeros(r.shape[0]) for _ in range(4)]
    pp = _EAM(p.beta, p.alpha, p.A, p.D, p.rp, p.r0, p.rc, p.h)
    lib().orc_eam_pair(ctypes.byref(pp), r.shape[0], _p(r), *[_p(o) for o in out])
    return tuple(out)


class ACE:
    """Linear ACE with the project-defined basis (radial Chebyshev x f_cut, real
    spherical harmonics l <= 4, nu = 1, 2, 3 products, Gaunt couplings)."""

    def __init__(self, params, fcut_mode: int = 0):
        W = _f64(params.W).reshape(5, 8, 8)
        c = _f64(params.c)
        self.rc = float(params.rc)
        self.h = lib().orc_ace_create(_p(W), _p(c), c.shape[0], self.rc, float(params.n0), fcut_mode)
        self._keep = (W, c)

    def __del__(self):
        try:
            if self.h:
                lib().orc_ace_destroy(self.h)
        except Exception:
            pass

    @property
    def nbasis(self) -> int:
        return lib().orc_ace_nbasis(self.h)

    def basis_desc(self) -> np.ndarray:
        d = np.zeros((self.nbasis, 7), np.int32)
        lib().orc_ace_basis_desc(self.h, _p(d))
        return d

    def gaunt(self) -> np.ndarray:
        g = np.zeros((4, 7, 4, 7, 4, 7))
        lib().orc_ace_gaunt(self.h, _p(g))
        return g

    def ylm(self, l: int, m: int, u):
        u = _f64(u)
        y = ctypes.c_double()
        gy = np.zeros(3)
        lib().orc_ylm(self.h, l, m, _p(u), ctypes.byref(y), _p(gy))
        return y.value, gy

    def basis(self, x, box, ids):
        """A (len(ids), 200) and B (len(ids), nbasis) for the given atoms."""
        x = _f64(x)
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        nl = neighbors_of(x, box, self.rc, ids)
        A = np.zeros((ids.shape[0], 200))
        B = np.zeros((ids.shape[0], self.nbasis))
        lib().orc_ace_basis(self.h, ids.shape[0], _p(ids), _p(x), ctypes.byref(_box(box)), _p(nl.cnt), _p(nl.j),
                            _p(nl.s), nl.cap, _p(A), _p(B))
        return A, B

    def eval(self, x, box, weights=None, nl: Optional[NeighborList] = None):
        """Site energies (0 where weight == 0) and F = -grad sum_i w_i E_i^p."""
        x = _f64(x)
        n = x.shape[0]
        if nl is None:
            nl = neighbors(x, box, self.rc)
        e = np.zeros(n)
        f = np.zeros((n, 3))
        w = None if weights is None else _f64(weights)
        lib().orc_ace_eval(self.h, n, _p(x), ctypes.byref(_box(box)), _p(nl.cnt), _p(nl.j), _p(nl.s), nl.cap,
                           _p(w), _p(e), _p(f))
        return e, f


def fs_embed(phi, eps: float):
    """Embedding of the Finnis-Sinclair ACE form (Eq. energy_ace: E = phi^(1) + sqrt(phi^(2))),
    regularised so that it is defined and C1 for every real phi:
    F(phi) = sign(phi) (sqrt(|phi| + eps^2) - eps),  F'(phi) = 1 / (2 sqrt(|phi| + eps^2)).
    For phi >> eps^2, F = sqrt(phi) - eps + O(eps^2/sqrt(phi)).  Returns (F, F')."""
    phi = _f64(phi)
    s = np.sqrt(np.abs(phi) + eps * eps)
    return np.sign(phi) * (s - eps), 0.5 / s


class ACEFS:
    """ACE with the Finnis-Sinclair form E_i = phi_i^(1) + F(phi_i^(2)), phi^(p) = sum_v
    c^(p)_v B_iv.  Forces at fixed weights: -grad sum_i w_i E_i = -grad sum_i w_i phi_i^(1)
    - grad sum_i (w_i F'(phi_i^(2))) phi_i^(2), i.e. two linear ACE evaluations."""

    def __init__(self, params, fcut_mode: int = 0):
        import dataclasses as _dc
        self.eps = float(params.fs_eps)
        self.rc = float(params.rc)
        self.a1 = ACE(_dc.replace(params, c2=None), fcut_mode)
        self.a2 = ACE(_dc.replace(params, c=params.c2, c2=None), fcut_mode)

    def phis(self, x, box, nl=None):
        if nl is None:
            nl = neighbors(x, box, self.rc)
        p1, _ = self.a1.eval(x, box, nl=nl)
        p2, _ = self.a2.eval(x, box, nl=nl)
        return p1, p2

    def eval(self, x, box, weights=None, nl: Optional[NeighborList] = None):
        """Site energies (0 where weight == 0) and F = -grad sum_i w_i E_i."""
        x = _f64(x)
        if nl is None:
            nl = neighbors(x, box, self.rc)
        p1, p2 = self.phis(x, box, nl)
        fv, dfv = fs_embed(p2, self.eps)
        w = np.ones(x.shape[0]) if weights is None else _f64(weights)
        _, f1 = self.a1.eval(x, box, weights=w, nl=nl)
        _, f2 = self.a2.eval(x, box, weights=w * dfv, nl=nl)
        e = np.where(w != 0.0, p1 + fv, 0.0)
        return e, f1 + f2


def ace_for(params, fcut_mode: int = 0):
    """The oracle ACE for a parameter set: linear, or Finnis-Sinclair when params.c2 is set."""
    return ACEFS(params, fcut_mode) if getattr(params, "c2", None) is not None else ACE(params, fcut_mode)


def hybrid(x, box, lam, eam_p, ace: ACE):
    """Eq. energy_hyb and Eq. F_i_d: E_i = lam E^f + (1-lam) E^p and
    F = -grad sum_k [lam_k E_k^f + (1-lam_k) E_k^p] at fixed lam.
    Returns (E_site, F, E_fast, E_prec); E_prec is 0 where lam == 1."""
    lam = _f64(lam)
    ef, ff, _, _ = eam_any(x, box, eam_p, weights=lam)
    w = 1.0 - lam
    ep, fp = ace.eval(x, box, weights=w)
    e = lam * ef + w * ep
    return e, ff + fp, ef, ep


def indenter(x, center, radius: float, k: float):
    """Repulsive sphere: F = k (R - r)^2 (x - c)/r and E = k (R - r)^3 / 3 for r < R."""
    d = _f64(x) - np.asarray(center)[None, :]
    r = np.sqrt((d * d).sum(1))
    inside = r < radius
    f = np.zeros_like(d)
    rr = r[inside]
    f[inside] = (k * (radius - rr) ** 2 / rr)[:, None] * d[inside]
    e = np.zeros(r.shape[0])
    e[inside] = k * (radius - rr) ** 3 / 3.0
    return e, f


def md_step(x, v, f, mass, dt: float, force_fn, fixed=None):
    """Velocity Verlet (Eq. vv).  force_fn(x_new) performs the lambda step and returns
    the new forces (and anything else).  Fixed atoms keep v = 0 and do not move."""
    a = f * (ACC / mass)[:, None]
    v = v + 0.5 * dt * a
    if fixed is not None:
        v[fixed != 0] = 0.0
    x = x + dt * v
    out = force_fn(x)
    f_new = out[0]
    a = f_new * (ACC / mass)[:, None]
    v = v + 0.5 * dt * a
    if fixed is not None:
        v[fixed != 0] = 0.0
    return x, v, out


def kinetic(v, mass) -> float:
    return float(0.5 * (mass[:, None] * v * v).sum() / ACC)


def extract_cluster(x, box, center_idx: int, radius: float):
    """Atoms (all images) within radius of atom center_idx, as unwrapped coordinates
    around it, for local evaluation in an open box.  Returns (xc, src, k0)."""
    x = _f64(x)
    d0 = x - x[center_idx][None, :]
    L = box.hi - box.lo
    for k in range(3):
        if box.periodic[k]:
            d0[:, k] -= L[k] * np.round(d0[:, k] / L[k])
    r = np.sqrt((d0 * d0).sum(1))
    sel = np.nonzero(r < radius)[0]
    xc = x[center_idx][None, :] + d0[sel]
    k0 = int(np.nonzero(sel == center_idx)[0][0])
    return xc, sel, k0
