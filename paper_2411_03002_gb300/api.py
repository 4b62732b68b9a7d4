"""Python binding of the C-ABI (include/ap.h): the same calls, marshalled from
torch tensors.  Every step of the computation runs in libap.so's CUDA kernels;
this module only passes device pointers, sizes and the current stream.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional, Sequence

import numpy as np
import torch

from . import _native as N
from ._native import ApBox, ApConfig, ApError, ApStepStats


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_box(lo, hi, periodic) -> ApBox:
    b = ApBox()
    for k in range(3):
        b.lo[k] = float(lo[k])
        b.hi[k] = float(hi[k])
        b.periodic[k] = int(bool(periodic[k]))
    return b


def make_config(eam, ace, hyb, precision: int = N.PREC_MIXED, skin: float = 1.0, dt: float = 1.0,
                indenter=None, cap_eam: int = 0, cap_ace: int = 0, lambda_every: Optional[int] = None,
                rebuild_every: int = 0, detector: int = N.DETECT_CSP, sel_p_lo: float = 0.5,
                sel_p_hi: float = 0.9, thermostat: bool = False, deterministic: bool = False) -> ApConfig:
    """Fill an ap_config from parameter objects with the attribute names of
    the EAM (beta, alpha, A, D, rp, r0, rc, h), ACE (W, c, rc, n0) and switching
    (csp_lo, csp_hi, r_lo, r_hi, dlam_min, n_csp_avg, n_lam_avg, fcut_mode,
    sample_every) parameter sets.  An EAM object with the 29 Mishin EAM2
    parameters (E1 .. rc, Appendix E; ap_inputs.MishinParams) selects that potential."""
    c = ApConfig()
    if hasattr(eam, "E1"):
        m = np.asarray(eam.as_array(), dtype=np.float64)
        if m.size != 29:
            raise ValueError("Mishin EAM2 needs 29 parameters")
        c.eam_type = N.EAM_MISHIN
        for i in range(29):
            c.eam_mishin[i] = m[i]
        c.eam_rc, c.eam_h = float(eam.rc), float(eam.h)
    else:
        for k in ("beta", "alpha", "A", "D", "rp", "r0", "rc", "h"):
            setattr(c, "eam_" + k, float(getattr(eam, k)))
    W = np.ascontiguousarray(ace.W, dtype=np.float64).reshape(-1)
    if W.size != 320:
        raise ValueError("ACE W must have 5*8*8 entries")
    cc = np.ascontiguousarray(ace.c, dtype=np.float64).reshape(-1)
    for i in range(320):
        c.ace_W[i] = W[i]
    nc = min(512, cc.size)
    for i in range(nc):
        c.ace_c[i] = cc[i]
    c.ace_nc = nc
    c.ace_rc = float(ace.rc)
    c.ace_n0 = float(ace.n0)
    c2 = getattr(ace, "c2", None)
    if c2 is not None:   # Finnis-Sinclair form E = phi1 + F(phi2)
        c2 = np.ascontiguousarray(c2, dtype=np.float64).reshape(-1)
        c.ace_fs_on = 1
        c.ace_fs_eps = float(ace.fs_eps)
        for i in range(min(512, c2.size)):
            c.ace_c2[i] = c2[i]
    c.csp_lo, c.csp_hi = float(hyb.csp_lo), float(hyb.csp_hi)
    c.r_lo, c.r_hi = float(hyb.r_lo), float(hyb.r_hi)
    c.dlam_min = float(hyb.dlam_min)
    c.n_csp_avg, c.n_lam_avg = int(hyb.n_csp_avg), int(hyb.n_lam_avg)
    c.fcut_mode = int(hyb.fcut_mode)
    c.skin = float(skin)
    c.cap_eam, c.cap_ace = int(cap_eam), int(cap_ace)
    c.precision = int(precision)
    c.dt = float(dt)
    c.lambda_every = int(lambda_every if lambda_every is not None else hyb.sample_every)
    c.rebuild_every = int(rebuild_every)
    c.detector = int(detector)
    c.sel_p_lo, c.sel_p_hi = float(sel_p_lo), float(sel_p_hi)
    c.thermostat_on = 1 if thermostat else 0
    if indenter is not None:
        c.indenter_on = 1
        for k in range(3):
            c.ind_c0[k] = float(indenter.center0[k])
            c.ind_v[k] = float(indenter.velocity[k])
        c.ind_R = float(indenter.radius)
        c.ind_k = float(indenter.k)
    c.ace_deterministic = 1 if deterministic else 0
    return c


def ace_nbasis() -> int:
    return N.lib().ap_ace_nbasis(None)


def ace_basis_desc() -> np.ndarray:
    d = np.zeros((ace_nbasis(), 7), np.int32)
    _check(None, N.lib().ap_ace_basis_desc(None, d.ctypes.data_as(ctypes.c_void_p)))
    return d


def ace_gaunt() -> np.ndarray:
    g = np.zeros((4, 7, 4, 7, 4, 7))
    _check(None, N.lib().ap_ace_gaunt(None, g.ctypes.data_as(ctypes.c_void_p)))
    return g


PEAK_FFMA = 0
PEAK_TF32_MMA = 1


def probe_peak(which: int = PEAK_FFMA, reps: int = 6, stream=None):
    """(TFLOP/s, SM MHz) measured on the current device by ap_probe_peak: the FP32
    FFMA rate (which = PEAK_FFMA) or the warp-level TF32 tensor-core rate
    (PEAK_TF32_MMA), best of reps - 1 timed runs."""
    tf, mhz = ctypes.c_double(), ctypes.c_double()
    _check(None, N.lib().ap_probe_peak(int(which), int(reps), _stream(stream), ctypes.byref(tf), ctypes.byref(mhz)))
    return tf.value, mhz.value


def _check(ctx, st: int):
    if st != N.AP_OK:
        msg = N.lib().ap_last_error(ctx).decode() if ctx else ""
        raise ApError(st, msg)


@dataclasses.dataclass
class StepStats:
    step: int
    n_precise: int
    n_detected: int
    rebuilds: int
    e_pot: float
    e_kin: float
    max_disp: float
    error_bits: int
    th_corrected: int = 0
    th_refused: int = 0
    th_energy: float = 0.0
    kept: int = 0
    ace_rebuilds: int = 0


class Context:
    """One ap_ctx on the current CUDA device."""

    def __init__(self, cfg: ApConfig):
        self.lib = N.lib()
        h = ctypes.c_void_p()
        st = self.lib.ap_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != N.AP_OK:
            raise ApError(st, "ap_create failed")
        self.h = h
        self.cfg = cfg
        self.n = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.ap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        _check(self.h, st)

    @property
    def nbasis(self) -> int:
        return self.lib.ap_ace_nbasis(self.h)

    def need(self) -> int:
        return self.lib.ap_need(self.h)

    # ---------------------------------------------------------------- neighbours
    def build_neighbors(self, x: torch.Tensor, box, species: Optional[torch.Tensor] = None, stream=None):
        b = box if isinstance(box, ApBox) else make_box(box.lo, box.hi, box.periodic)
        self.n = x.shape[0]
        self._ck(self.lib.ap_build_neighbors(self.h, self.n, _ptr(x), _ptr(species), ctypes.byref(b),
                                             _stream(stream)))

    def build_neighbors_batch(self, x: torch.Tensor, offsets: Sequence[int], boxes: Sequence, species=None,
                              stream=None):
        ns = len(boxes)
        off = (ctypes.c_int64 * (ns + 1))(*[int(o) for o in offsets])
        arr = (ApBox * ns)(*[b if isinstance(b, ApBox) else make_box(b.lo, b.hi, b.periodic) for b in boxes])
        self.n = int(offsets[-1])
        self._ck(self.lib.ap_build_neighbors_batch(self.h, ns, off, arr, _ptr(x), _ptr(species), _stream(stream)))

    def neighbor_total(self, which: int = 0) -> int:
        """Total entries of the current EAM (0) or ACE (1) rows, or of the EAM row prefixes
        the last EAM force pass walked (2) (synchronises)."""
        t = ctypes.c_int64()
        self._ck(self.lib.ap_neighbor_total(self.h, which, ctypes.byref(t)))
        return t.value

    def spatial_order(self, stream=None) -> torch.Tensor:
        """The atoms in the cell order of the last build (int32 [n]): x[order], v[order], ...
        put neighbours close in memory (ap_spatial_order)."""
        order = torch.empty(max(self.n, 1), dtype=torch.int32, device="cuda")
        self._ck(self.lib.ap_spatial_order(self.h, _ptr(order), _stream(stream)))
        return order[:self.n]

    def get_neighbors(self, which: int = 0, cap: int = 320):
        """(cnt [rows], idx [rows, cap], shift [rows, cap, 3]) as CUDA int32 tensors."""
        rows = ctypes.c_int64()
        dev = torch.device("cuda")
        nrows = self.n
        cnt = torch.zeros(max(nrows, 1), dtype=torch.int32, device=dev)
        idx = torch.zeros((max(nrows, 1), cap), dtype=torch.int32, device=dev)
        sh = torch.zeros((max(nrows, 1), cap, 3), dtype=torch.int32, device=dev)
        self._ck(self.lib.ap_get_neighbors(self.h, which, _ptr(cnt), _ptr(idx), _ptr(sh), cap, ctypes.byref(rows)))
        r = rows.value
        return cnt[:r], idx[:r], sh[:r]

    # ---------------------------------------------------------------- lambda
    def classify(self, x: torch.Tensor, changeable: Optional[torch.Tensor] = None, sample_now: bool = True,
                 stream=None):
        n = x.shape[0]
        lam = torch.empty(n, dtype=torch.float64, device=x.device)
        idx = torch.empty(max(n, 1), dtype=torch.int32, device=x.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=x.device)
        self._ck(self.lib.ap_classify(self.h, n, _ptr(x), _ptr(changeable), 1 if sample_now else 0, _ptr(lam),
                                      _ptr(idx), _ptr(cnt), _stream(stream)))
        return lam, idx, cnt

    def precise_queue(self, lam, stream=None):
        """(queue int32 [max(n,1)], count int64 [1]) of the atoms with lambda < 1."""
        n = lam.shape[0]
        idx = torch.empty(max(n, 1), dtype=torch.int32, device=lam.device)
        cnt = torch.empty(1, dtype=torch.int64, device=lam.device)
        self._ck(self.lib.ap_precise_queue(self.h, n, _ptr(lam), _ptr(idx), _ptr(cnt), _stream(stream)))
        return idx, cnt

    def reset_lambda(self):
        self._ck(self.lib.ap_reset_lambda(self.h))

    def get_lambda_state(self, stream=None):
        n = self.n
        dev = torch.device("cuda")
        out = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(5)]
        self._ck(self.lib.ap_get_lambda_state(self.h, *[_ptr(t) for t in out], _stream(stream)))
        return dict(zip(("csp", "csp_avg", "lam0", "lam_min", "lam_avg"), out))

    # ---------------------------------------------------------------- potentials
    def eval_eam(self, x, lam=None, e_fast=None, f=None, feat=None, stream=None):
        """(e_fast, f); feat, a [n, 24] float32 CUDA tensor, also receives the selector features."""
        n = x.shape[0]
        if e_fast is None:
            e_fast = torch.empty(n, dtype=torch.float64, device=x.device)
        if f is None:
            f = torch.zeros((n, 3), dtype=torch.float64, device=x.device)
        self._ck(self.lib.ap_eval_eam(self.h, n, _ptr(x), _ptr(lam), _ptr(e_fast), _ptr(f), _ptr(feat),
                                      _stream(stream)))
        return e_fast, f

    def eval_ace(self, x, lam, precise_idx, n_precise, e_prec=None, f=None, forces: bool = True, stream=None):
        n = x.shape[0]
        if e_prec is None:
            e_prec = torch.empty(n, dtype=torch.float64, device=x.device)
        if f is None and forces:
            f = torch.zeros((n, 3), dtype=torch.float64, device=x.device)
        self._ck(self.lib.ap_eval_ace(self.h, n, _ptr(x), _ptr(lam), _ptr(precise_idx), _ptr(n_precise),
                                      _ptr(e_prec), _ptr(f), _stream(stream)))
        return e_prec, f

    def blend_forces(self, lam, e_fast, e_prec, stream=None):
        n = e_fast.shape[0]
        e_atom = torch.empty(n, dtype=torch.float64, device=e_fast.device)
        e_tot = torch.zeros(1, dtype=torch.float64, device=e_fast.device)
        self._ck(self.lib.ap_blend_forces(self.h, n, _ptr(lam), _ptr(e_fast), _ptr(e_prec), _ptr(e_atom),
                                          _ptr(e_tot), _stream(stream)))
        return e_atom, e_tot

    # ---------------------------------------------------------------- dynamics
    def step(self, x, v, f, mass, fixed, lam, nsteps: int, stream=None) -> StepStats:
        st = ApStepStats()
        n = x.shape[0]
        self._ck(self.lib.ap_step(self.h, n, _ptr(x), _ptr(v), _ptr(f), _ptr(mass), _ptr(fixed), _ptr(lam),
                                  int(nsteps), ctypes.byref(st), _stream(stream)))
        return StepStats(st.step, st.n_precise, st.n_detected, st.rebuilds, st.e_pot, st.e_kin, st.max_disp,
                         st.error_bits, st.th_corrected, st.th_refused, st.th_energy, st.kept, st.ace_rebuilds)

    PHASES = ("neighbors", "classify", "eam", "ace", "other", "thermostat", "ace_adjoint", "eam_force", "ace_basis")

    def profile_enable(self, on: bool = True):
        self._ck(self.lib.ap_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        ms = (ctypes.c_double * len(self.PHASES))()
        calls = (ctypes.c_int64 * len(self.PHASES))()
        kern, pairs, atoms = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._ck(self.lib.ap_profile_read(self.h, ms, calls, ctypes.byref(kern), ctypes.byref(pairs),
                                          ctypes.byref(atoms)))
        mma = ctypes.c_int64()
        self._ck(self.lib.ap_profile_mma(self.h, ctypes.byref(mma)))
        return {"phases": {p: (ms[k], calls[k]) for k, p in enumerate(self.PHASES)}, "kernels": kern.value,
                "ace_pairs": pairs.value, "ace_atoms": atoms.value, "ace_mma": mma.value}

    def state_export(self) -> bytes:
        ln = ctypes.c_size_t()
        self._ck(self.lib.ap_state_export(self.h, None, ctypes.byref(ln)))
        buf = ctypes.create_string_buffer(ln.value)
        self._ck(self.lib.ap_state_export(self.h, buf, ctypes.byref(ln)))
        return buf.raw

    def state_import(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        self._ck(self.lib.ap_state_import(self.h, buf, len(data)))

    # ---------------------------------------------------------------- selector
    def sel_set_model(self, params, mu, inv_sigma):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        m = np.ascontiguousarray(mu, dtype=np.float32).reshape(-1)
        s = np.ascontiguousarray(inv_sigma, dtype=np.float32).reshape(-1)
        if p.size != N.SEL_NPARAMS or m.size != N.SEL_NFEAT or s.size != N.SEL_NFEAT:
            raise ValueError("selector model: expected 5825 parameters and 24 mu / inv_sigma values")
        self._ck(self.lib.ap_sel_set_model(self.h, p.ctypes.data, m.ctypes.data, s.ctypes.data))

    def sel_get_model(self):
        p = np.zeros(N.SEL_NPARAMS, np.float32)
        m = np.zeros(N.SEL_NFEAT, np.float32)
        s = np.zeros(N.SEL_NFEAT, np.float32)
        self._ck(self.lib.ap_sel_get_model(self.h, p.ctypes.data, m.ctypes.data, s.ctypes.data))
        return p, m, s

    def sel_features(self, x, changeable=None, feat=None, stream=None) -> torch.Tensor:
        n = x.shape[0]
        if feat is None:
            feat = torch.empty((n, N.SEL_NFEAT), dtype=torch.float32, device=x.device)
        self._ck(self.lib.ap_sel_features(self.h, n, _ptr(x), _ptr(changeable), _ptr(feat), _stream(stream)))
        return feat

    def sel_predict(self, feat, p=None, logit=None, stream=None):
        n = feat.shape[0]
        if p is None:
            p = torch.empty(n, dtype=torch.float32, device=feat.device)
        if logit is None:
            logit = torch.empty(n, dtype=torch.float32, device=feat.device)
        self._ck(self.lib.ap_sel_predict(self.h, n, _ptr(feat), _ptr(p), _ptr(logit), _stream(stream)))
        return p, logit

    def sel_train_step(self, feat, label, weight, idx=None, b: Optional[int] = None, lr: float = 1e-3,
                       beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, loss=None, stream=None):
        bb = int(b if b is not None else (idx.shape[0] if idx is not None else feat.shape[0]))
        self._ck(self.lib.ap_sel_train_step(self.h, bb, _ptr(feat), _ptr(idx), _ptr(label), _ptr(weight),
                                            float(lr), float(beta1), float(beta2), float(eps), _ptr(loss),
                                            _stream(stream)))

    def sel_get_grad(self):
        g = np.zeros(N.SEL_NPARAMS, np.float32)
        loss = ctypes.c_float()
        self._ck(self.lib.ap_sel_get_grad(self.h, g.ctypes.data, ctypes.byref(loss)))
        return g, float(loss.value)


# Module-level calls with the C-ABI names.
def ap_create(cfg: ApConfig) -> Context:
    return Context(cfg)


def ap_build_neighbors(ctx: Context, x, box, species=None, stream=None):
    return ctx.build_neighbors(x, box, species, stream)


def ap_classify(ctx: Context, x, changeable=None, sample_now=True, stream=None):
    return ctx.classify(x, changeable, sample_now, stream)


def ap_eval_eam(ctx: Context, x, lam=None, e_fast=None, f=None, feat=None, stream=None):
    return ctx.eval_eam(x, lam, e_fast, f, feat, stream)


def ap_eval_ace(ctx: Context, x, lam, precise_idx, n_precise, e_prec=None, f=None, stream=None):
    return ctx.eval_ace(x, lam, precise_idx, n_precise, e_prec, f, stream=stream)


def ap_blend_forces(ctx: Context, lam, e_fast, e_prec, stream=None):
    return ctx.blend_forces(lam, e_fast, e_prec, stream)


def ap_step(ctx: Context, x, v, f, mass, fixed, lam, nsteps: int, stream=None) -> StepStats:
    return ctx.step(x, v, f, mass, fixed, lam, nsteps, stream)


def ap_sel_set_model(ctx: Context, params, mu, inv_sigma):
    return ctx.sel_set_model(params, mu, inv_sigma)


def ap_sel_get_model(ctx: Context):
    return ctx.sel_get_model()


def ap_sel_features(ctx: Context, x, changeable=None, feat=None, stream=None):
    return ctx.sel_features(x, changeable, feat, stream)


def ap_sel_predict(ctx: Context, feat, p=None, logit=None, stream=None):
    return ctx.sel_predict(feat, p, logit, stream)


def ap_sel_train_step(ctx: Context, feat, label, weight, idx=None, **kw):
    return ctx.sel_train_step(feat, label, weight, idx, **kw)


def ap_sel_get_grad(ctx: Context):
    return ctx.sel_get_grad()
