"""Switching-zone parameter study on the GPU: force and energy error against the
precise potential, and the cost of the adaptive evaluation, as functions of
r_lambda,lo, r_lambda,hi (the paper's switching-zone width study in its appendix on
the switching function) and of the CSP thresholds (its sensitivity study, section 3.3).

One study point follows the paper's definition:
- one lambda update with lambda = lambda_min (Eq. lambda_2_i) as the switching
  parameter (one-sample CSP and lambda windows, no minimum step, no thermostat);
- hybrid energies and forces (Eqs. energy_hyb, F_i_d) compared with the precise
  potential evaluated for every atom;
- atoms whose force has both an EAM and an ACE contribution ("mixed" atoms) grouped
  by CSP_avg, with the RMSE of the force components and of the site energy per group.
  Here an atom has a contribution from a potential when the library's weighted force
  of that potential on it is nonzero: the EAM force gathers lambda_k-weighted terms of
  every pair within the EAM cutoff, the ACE force (1 - lambda_k)-weighted terms of
  every precise atom within the ACE cutoff, so it is zero exactly when every weight
  in reach is zero.

Every evaluation runs through the library (ap_classify, ap_eval_eam, ap_eval_ace,
ap_blend_forces); numpy only groups the returned per-atom arrays.  The timings are
CUDA-event times of the library calls on the current stream.

    python -m paper_2411_03002_gb300.sweep --nxy 100 --nz 100 --out sweep.json
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import time
from typing import Iterable, Optional, Sequence

import numpy as np
import torch

from . import api
from ._native import PREC_FP64, PREC_MIXED

# CSP_avg group edges (A^2): thermal fluctuations below CSP_hi = 3, then defects.
CSP_EDGES = (0.0, 0.5, 1.0, 2.0, 3.0, 4.5, 6.0, 8.0, 12.0, 20.0, float("inf"))


@dataclasses.dataclass(frozen=True)
class Point:
    csp_lo: float
    csp_hi: float
    r_lo: float
    r_hi: float


def default_points() -> list:
    """r_lambda,lo in {0, 2, 4, 8} x width in {2, 4, 8, 12} A at the paper's CSP
    thresholds (2.5, 3) A^2, then thresholds (1.5, 2), (3, 3.5) (+0.5 A^2 as in the
    sensitivity study) and (4, 4.5) at the paper's r_lambda = (4, 12) A."""
    pts = [Point(2.5, 3.0, lo, lo + w) for lo in (0.0, 2.0, 4.0, 8.0) for w in (2.0, 4.0, 8.0, 12.0)]
    pts += [Point(lo, lo + 0.5, 4.0, 12.0) for lo in (1.5, 3.0, 4.0)]
    return pts


def one_sample(hyb, p: Optional[Point] = None):
    """Switching parameters of a study point: one-sample windows and no minimum step,
    so that lambda = lambda_min after one update."""
    kw = dict(n_csp_avg=1, n_lam_avg=1, dlam_min=0.0, sample_every=1)
    if p is not None:
        kw.update(csp_lo=p.csp_lo, csp_hi=p.csp_hi, r_lo=p.r_lo, r_hi=p.r_hi)
    return dataclasses.replace(hyb, **kw)


def grouped_rmse(d: np.ndarray, csp: np.ndarray, mask: np.ndarray, edges: Sequence[float] = CSP_EDGES):
    """(count, RMSE) per CSP group of the rows of d selected by mask (NaN when empty)."""
    d = np.asarray(d, np.float64).reshape(d.shape[0], -1)
    cnt, rmse = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = mask & (csp >= lo) & (csp < hi)
        k = int(m.sum())
        cnt.append(k)
        rmse.append(float(np.sqrt((d[m] ** 2).mean())) if k else float("nan"))
    return np.array(cnt), np.array(rmse)


class _Timer:
    def __init__(self):
        self.s = torch.cuda.current_stream()
        self.a = torch.cuda.Event(enable_timing=True)
        self.b = torch.cuda.Event(enable_timing=True)

    def __enter__(self):
        self.a.record(self.s)
        return self

    def __exit__(self, *exc):
        self.b.record(self.s)

    @property
    def ms(self) -> float:
        self.b.synchronize()
        return self.a.elapsed_time(self.b)


class Study:
    """Study points on one configuration.  x: (n,3) FP64 CUDA tensor; changeable:
    (n,) uint8 CUDA tensor (1 = mobile) or None; eam/ace/hyb: parameter objects as
    for make_config (hyb supplies the f_cut mode; its radii and thresholds are
    replaced per point)."""

    def __init__(self, eam, ace, hyb, x: torch.Tensor, box, changeable: Optional[torch.Tensor] = None,
                 precision: int = PREC_MIXED, skin: float = 1.0, reps: int = 3, lambda_every: int = 10):
        self.eam, self.ace, self.hyb = eam, ace, hyb
        self.x, self.box, self.precision, self.skin = x, box, precision, skin
        self.n = x.shape[0]
        self.changeable = changeable
        self.mobile = (np.ones(self.n, bool) if changeable is None
                       else changeable.cpu().numpy().astype(bool))
        self.reps, self.lambda_every = max(1, reps), lambda_every
        self._reference()

    def _ctx(self, hyb):
        c = api.Context(api.make_config(self.eam, self.ace, hyb, precision=self.precision, skin=self.skin))
        c.build_neighbors(self.x, self.box)
        return c

    def _reference(self):
        """Precise energies and forces of every atom; fast forces of every atom."""
        ctx = self._ctx(one_sample(self.hyb))
        dev = self.x.device
        zero = torch.zeros(self.n, dtype=torch.float64, device=dev)
        one = torch.ones(self.n, dtype=torch.float64, device=dev)
        q = torch.arange(self.n, dtype=torch.int32, device=dev)
        nq = torch.tensor([self.n], dtype=torch.int64, device=dev)
        ctx.eval_ace(self.x, zero, q, nq)                       # warm-up (rows, tables)
        ms = []
        for _ in range(self.reps):
            with _Timer() as t:
                e_p, f_p = ctx.eval_ace(self.x, zero, q, nq)
            ms.append(t.ms)
        self.t_full_ace_ms = float(np.median(ms))
        ms = []
        for _ in range(self.reps):
            with _Timer() as t:
                _, f_f = ctx.eval_eam(self.x, one)
            ms.append(t.ms)
        self.t_full_eam_ms = float(np.median(ms))
        self.e_p, self.f_p, self.f_f = e_p.cpu().numpy(), f_p.cpu().numpy(), f_f.cpu().numpy()
        ctx.close()

    def point(self, p: Point) -> dict:
        ctx = self._ctx(one_sample(self.hyb, p))
        lam, q, nq = ctx.classify(self.x, self.changeable)
        ef, f_f = ctx.eval_eam(self.x, lam)
        ep, f_p = ctx.eval_ace(self.x, lam, q, nq)
        e_atom, _ = ctx.blend_forces(lam, ef, ep)
        st = ctx.get_lambda_state()
        lam_h = lam.cpu().numpy()
        lam0_h = st["lam0"].cpu().numpy()
        csp = st["csp_avg"].cpu().numpy()
        ff, fp = f_f.cpu().numpy(), f_p.cpu().numpy()
        e_h = e_atom.cpu().numpy()
        # timing: the lambda update and the force evaluation, each on its own (one-sample
        # windows: repeated updates at the same positions give the same lambda)
        t_cls, t_frc = [], []
        for _ in range(self.reps):
            with _Timer() as t:
                lam2, q2, nq2 = ctx.classify(self.x, self.changeable)
            t_cls.append(t.ms)
            with _Timer() as t:
                _, f2 = ctx.eval_eam(self.x, lam2)
                ctx.eval_ace(self.x, lam2, q2, nq2, f=f2)
            t_frc.append(t.ms)
        mixed = self.mobile & (np.abs(ff).sum(1) > 0) & (np.abs(fp).sum(1) > 0)
        fh = ff + fp
        cnt, f_rmse = grouped_rmse(fh - self.f_p, csp, mixed)
        _, e_rmse = grouped_rmse(e_h - self.e_p, csp, mixed)
        ref_cnt, ref_rmse = grouped_rmse(self.f_f - self.f_p, csp, self.mobile)
        d = (fh - self.f_p)[mixed]
        t_cls_ms, t_frc_ms = float(np.median(t_cls)), float(np.median(t_frc))
        out = {
            "point": dataclasses.asdict(p),
            "n": self.n,
            "n_precise": int((lam_h < 1).sum()),
            "n_detected": int((lam0_h < 1).sum()),
            "n_mixed": int(mixed.sum()),
            "group_count": cnt.tolist(),
            "force_rmse_meV_A": (f_rmse * 1e3).tolist(),
            "energy_rmse_meV": (e_rmse * 1e3).tolist(),
            "ref_count": ref_cnt.tolist(),
            "ref_force_rmse_meV_A": (ref_rmse * 1e3).tolist(),
            "force_rmse_mixed_meV_A": float(np.sqrt((d ** 2).mean()) * 1e3) if d.size else float("nan"),
            "t_classify_ms": t_cls_ms,
            "t_forces_ms": t_frc_ms,
            "t_full_ace_ms": self.t_full_ace_ms,
            "t_full_eam_ms": self.t_full_eam_ms,
            "speedup_vs_full_ace": self.t_full_ace_ms / (t_frc_ms + t_cls_ms / self.lambda_every),
        }
        self.last = {"lam": lam_h, "lam0": lam0_h, "csp": csp, "mixed": mixed}
        ctx.close()
        return out

    def run(self, points: Iterable[Point]) -> list:
        return [self.point(p) for p in points]


def main(argv=None):
    import ap_inputs as I
    ap_ = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap_.add_argument("--nxy", type=int, default=100)
    ap_.add_argument("--nz", type=int, default=100)
    ap_.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap_.add_argument("--reps", type=int, default=5)
    ap_.add_argument("--out", default=None)
    a = ap_.parse_args(argv)
    t0 = time.time()
    w = I.config_c6(a.nxy, a.nz)
    x = torch.as_tensor(w.x, device="cuda")
    ch = torch.as_tensor((w.fixed == 0).astype(np.uint8), device="cuda")
    prec = PREC_MIXED if a.precision == "mixed" else PREC_FP64
    s = Study(I.eam_params(0), I.ace_for_config(5), w.hyb, x, w.box, ch, precision=prec, reps=a.reps)
    res = s.run(default_points())
    doc = {"workload": w.name, "n_atoms": w.n, "precision": a.precision, "csp_edges": list(CSP_EDGES)[:-1],
           "points": res, "wall_s": time.time() - t0}
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(json.dumps(doc, indent=1))
    print("%s, %d atoms, %s; full ACE %.2f ms, full EAM %.2f ms" % (w.name, w.n, a.precision, s.t_full_ace_ms,
                                                                     s.t_full_eam_ms))
    for r in res:
        p = r["point"]
        print("csp %.1f-%.1f r %4.1f-%4.1f  precise %6.2f%%  mixed %7d  rmse %7.2f meV/A  forces %7.3f ms"
              "  classify %7.3f ms  speedup %6.2f" % (p["csp_lo"], p["csp_hi"], p["r_lo"], p["r_hi"],
                                                      100 * r["n_precise"] / w.n, r["n_mixed"],
                                                      r["force_rmse_mixed_meV_A"], r["t_forces_ms"],
                                                      r["t_classify_ms"], r["speedup_vs_full_ace"]))


if __name__ == "__main__":
    main()
