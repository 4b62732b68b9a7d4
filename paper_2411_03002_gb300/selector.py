"""Training and evaluation of the selector with this library's kernels.

The selector is a learned detection score that replaces the centro-symmetry
argument of f_cut (Appendix B: any detector whose f_cut argument is 0 for atoms
to be computed precisely and 1 for atoms to be computed fast); its features,
network and training step are defined in include/ap.h (ap_sel_*).

Data (the selector workload).  200 structures of about 5,000 atoms from
``ap_inputs.config_c4``: bulk at 300 K-like displacements, vacancies,
(100)/(110)/(111) slabs, disorder up to 0.5 A, and snapshots of 300-1200 K
EAM molecular dynamics (run here with ap_step at lambda = 1).  Each atom's label is
y = 1 when the precise and the fast potential disagree on its force by more than
TAU: |F_i^ACE - F_i^EAM| > TAU with both potentials evaluated in full (every atom
precise for the ACE, lambda = 1 for the EAM) in FP64.  This is the paper's reason
to treat an atom precisely (section 3: the fast potential is accurate in the bulk
and not at defects and surfaces).  Held-out data: three 32,000-atom slabs with
disordered hemispheres (``ap_inputs.config_c2`` variants 1-3).

Training.  Weighted binary cross-entropy with class weights 1/(2 f_y) (f_y the
class frequency), features standardised by the training mean and standard
deviation, Adam on batches of BATCH samples with a step learning-rate schedule,
all on the device through ap_sel_train_step.

    python -m paper_2411_03002_gb300.selector OUT.npz OUT.json
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np
import torch

import ap_inputs as I

from . import _native as N
from .api import Context, make_config

TAU = 0.025            # eV/A: label threshold on |F_ACE - F_EAM|
BATCH = 8192
EPOCHS = 40
MD_STEPS = 400         # EAM MD steps behind each snapshot of category 4
P_LO, P_HI = 0.5, 0.9  # default score thresholds of the deployed selector
SIZES = ((24, 64), (64,), (64, 64), (64,), (64,), (1,))


def _dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a) if dtype is None else np.ascontiguousarray(a, dtype), device="cuda")


def _fast_only(hyb):
    """Switching parameters whose CSP threshold no atom reaches (lambda = 1 everywhere)."""
    import dataclasses
    return dataclasses.replace(hyb, csp_lo=1e6, csp_hi=2e6)


def run_eam_md(w, steps: int) -> np.ndarray:
    """Positions after `steps` of EAM molecular dynamics (lambda = 1) from w.x, w.v."""
    cfg = make_config(I.eam_params(0), I.ace_params_anchored(), _fast_only(w.hyb), precision=N.PREC_MIXED,
                      dt=w.dt, lambda_every=10, rebuild_every=5)
    ctx = Context(cfg)
    x = _dev(w.x).clone()
    v = _dev(w.v).clone()
    f = torch.zeros_like(x)
    lam = torch.empty(w.n, dtype=torch.float64, device="cuda")
    ctx.build_neighbors(x, w.box)
    ctx.step(x, v, f, _dev(w.mass), None, lam, steps)
    out = x.cpu().numpy()
    ctx.close()
    return out


def label_structure(x, box, tau: float = TAU):
    """Features (device [n,24]), labels and |F_ACE - F_EAM| (host) of one structure."""
    n = x.shape[0]
    cfg = make_config(I.eam_params(0), I.ace_params_anchored(), I.HYB1, precision=N.PREC_FP64)
    ctx = Context(cfg)
    xd = _dev(x)
    ctx.build_neighbors(xd, box)
    feat = ctx.sel_features(xd)
    _, f_eam = ctx.eval_eam(xd)
    lam0 = _dev(np.zeros(n))
    queue = _dev(np.arange(n, dtype=np.int32))
    cnt = _dev(np.array([n], np.int64))
    _, f_ace = ctx.eval_ace(xd, lam0, queue, cnt)
    df = np.linalg.norm(f_ace.cpu().numpy() - f_eam.cpu().numpy(), axis=1)
    ctx.close()
    return feat, (df > tau).astype(np.float32), df


def build_dataset(ks=range(200), md_steps: int = MD_STEPS, log=None):
    feats, ys, dfs, cats = [], [], [], []
    for k in ks:
        w = I.config_c4(k)
        x = run_eam_md(w, md_steps) if w.v is not None else w.x
        f, y, df = label_structure(x, w.box)
        feats.append(f)
        ys.append(y)
        dfs.append(df)
        cats.append(np.full(w.n, k // 40, np.int8))
        if log:
            log(f"  {w.name}: n={w.n} positives={y.mean():.3f}")
    return torch.cat(feats), np.concatenate(ys), np.concatenate(dfs), np.concatenate(cats)


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases, in the flat layout of include/ap.h."""
    g = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for shape in SIZES:
        k = int(np.prod(shape))
        parts.append(np.zeros(k) if len(shape) == 1 else g.standard_normal(k) * np.sqrt(2.0 / shape[0]))
    return np.concatenate(parts).astype(np.float32)


def lr_at(epoch: int, epochs: int) -> float:
    return 3e-3 if epoch < 0.6 * epochs else (1e-3 if epoch < 0.85 * epochs else 3e-4)


def train(feat: torch.Tensor, y: np.ndarray, epochs: int = EPOCHS, batch: int = BATCH, seed: int = 7, log=None):
    """Returns (params, mu, inv_sigma, per-epoch mean loss, seconds)."""
    fh = feat.cpu().numpy().astype(np.float64)
    mu = fh.mean(0).astype(np.float32)
    sd = fh.std(0)
    inv = (1.0 / np.where(sd > 1e-12, sd, 1.0)).astype(np.float32)
    f1 = float(y.mean())
    c = np.where(y > 0.5, 0.5 / f1, 0.5 / (1.0 - f1)) / batch
    ctx = Context(make_config(I.eam_params(0), I.ace_params(0), I.HYB1))
    ctx.sel_set_model(init_params(seed), mu, inv)
    yd, wd = _dev(y, np.float32), _dev(c, np.float32)
    n = y.shape[0]
    steps = n // batch
    losses = torch.zeros(epochs * steps, dtype=torch.float32, device="cuda")
    g = np.random.Generator(np.random.PCG64(seed))
    torch.cuda.synchronize()
    t0 = time.time()
    for e in range(epochs):
        perm = _dev(g.permutation(n).astype(np.int32))
        lr = lr_at(e, epochs)
        for s in range(steps):
            q = e * steps + s
            ctx.sel_train_step(feat, yd, wd, idx=perm[s * batch:(s + 1) * batch], lr=lr, loss=losses[q:q + 1])
        if log and (e % 5 == 4 or e == epochs - 1):
            ep = losses[e * steps:(e + 1) * steps].mean().item()
            log(f"  epoch {e + 1}: loss {ep:.4f} lr {lr:g}")
    torch.cuda.synchronize()
    seconds = time.time() - t0
    params, mu, inv = ctx.sel_get_model()
    hist = losses.view(epochs, steps).mean(1).cpu().numpy()
    ctx.close()
    return params, mu, inv, hist, seconds


def roc_auc(score: np.ndarray, y: np.ndarray) -> float:
    """Area under the ROC curve (probability a positive outranks a negative; ties count half)."""
    order = np.argsort(score, kind="mergesort")
    s = score[order]
    ranks = np.empty(len(s))
    i = 0
    while i < len(s):
        j = i
        while j + 1 < len(s) and s[j + 1] == s[i]:
            j += 1
        ranks[order[i:j + 1]] = 0.5 * (i + j) + 1
        i = j + 1
    npos = y.sum()
    nneg = len(y) - npos
    return float((ranks[y > 0.5].sum() - npos * (npos + 1) / 2) / (npos * nneg))


def hybrid_errors(w, params, mu, inv, p_lo: float, p_hi: float, tau: float = TAU):
    """One classification with CSP and with the selector on a held-out slab; the
    hybrid force of each against full ACE.  Returns a dict of metrics."""
    n = w.n
    xd = _dev(w.x)
    full = make_config(I.eam_params(0), I.ace_params_anchored(), w.hyb, precision=N.PREC_FP64)
    ctx = Context(full)
    ctx.build_neighbors(xd, w.box)
    queue = _dev(np.arange(n, dtype=np.int32))
    cnt = _dev(np.array([n], np.int64))
    _, f_ace = ctx.eval_ace(xd, _dev(np.zeros(n)), queue, cnt)
    _, f_eam = ctx.eval_eam(xd)
    f_ace = f_ace.cpu().numpy()
    df = np.linalg.norm(f_ace - f_eam.cpu().numpy(), axis=1)
    pos = df > tau
    ctx.close()
    out = {"n": n, "label_positive_fraction": float(pos.mean())}
    for name, det in (("csp", N.DETECT_CSP), ("selector", N.DETECT_SELECTOR)):
        cfg = make_config(I.eam_params(0), I.ace_params_anchored(), w.hyb, precision=N.PREC_FP64, detector=det,
                          sel_p_lo=p_lo, sel_p_hi=p_hi)
        ctx = Context(cfg)
        if det == N.DETECT_SELECTOR:
            ctx.sel_set_model(params, mu, inv)
        ctx.build_neighbors(xd, w.box)
        lam, idx, npre = ctx.classify(xd)
        st = ctx.get_lambda_state()
        detected = st["lam0"].cpu().numpy() < 1.0
        _, f = ctx.eval_eam(xd, lam)
        _, f = ctx.eval_ace(xd, lam, idx, npre, f=f)
        err = f.cpu().numpy() - f_ace
        lam_h = lam.cpu().numpy()
        out[name] = {
            "precise_fraction": float((lam_h < 1.0).mean()),
            "detected_fraction": float(detected.mean()),
            "recall_of_label_positives_by_detected": float((detected & pos).sum() / max(pos.sum(), 1)),
            "precision_of_detected": float((detected & pos).sum() / max(detected.sum(), 1)),
            "force_err_rms_meV_A_label_positive": float(np.sqrt((err[pos] ** 2).mean()) * 1e3) if pos.any() else 0.0,
            "force_err_rms_meV_A_all": float(np.sqrt((err ** 2).mean()) * 1e3),
            "force_err_max_meV_A": float(np.abs(err).max() * 1e3),
        }
        ctx.close()
    return out


def evaluate(params, mu, inv, variants=(1, 2, 3), p_lo: float = P_LO, p_hi: float = P_HI, tau: float = TAU):
    rep = {"per_slab": []}
    aucs = []
    for v in variants:
        w = I.config_c2(variant=v)
        feat, y, _ = label_structure(w.x, w.box, tau)
        ctx = Context(make_config(I.eam_params(0), I.ace_params(0), I.HYB1))
        ctx.sel_set_model(params, mu, inv)
        p, _ = ctx.sel_predict(feat)
        ph = p.cpu().numpy()
        ctx.close()
        auc = roc_auc(ph, y)
        aucs.append(auc)
        m = hybrid_errors(w, params, mu, inv, p_lo, p_hi, tau)
        m.update({"variant": v, "auc": auc, "recall_at_p_lo": float(((ph > p_lo) & (y > 0.5)).sum() / max(y.sum(), 1)),
                  "precision_at_p_lo": float(((ph > p_lo) & (y > 0.5)).sum() / max((ph > p_lo).sum(), 1))})
        rep["per_slab"].append(m)
    rep["auc_mean"] = float(np.mean(aucs))
    return rep


def main(out_npz: str, out_json: str, epochs: int = EPOCHS):
    log = lambda m: print(m, flush=True)
    t0 = time.time()
    log("building the selector training set (200 structures)")
    feat, y, df, cats = build_dataset(log=log)
    t_data = time.time() - t0
    log(f"{feat.shape[0]} samples, positive fraction {y.mean():.3f}, {t_data:.1f} s")
    params, mu, inv, hist, t_train = train(feat, y, epochs=epochs, log=log)
    rep = evaluate(params, mu, inv)
    rep.update({"samples": int(feat.shape[0]), "positive_fraction": float(y.mean()),
                "positive_fraction_by_category": [float(y[cats == c].mean()) for c in range(5)],
                "tau_eV_A": TAU, "epochs": epochs, "batch": BATCH, "loss_by_epoch": hist.tolist(),
                "seconds_data": t_data, "seconds_train": t_train, "p_lo": P_LO, "p_hi": P_HI})
    np.savez(out_npz, params=params, mu=mu, inv_sigma=inv, p_lo=P_LO, p_hi=P_HI, tau=TAU)
    with open(out_json, "w") as fh:
        json.dump(rep, fh, indent=1)
    log(json.dumps({k: v for k, v in rep.items() if k != "loss_by_epoch"}, indent=1))


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2], *(int(a) for a in sys.argv[3:4]))
