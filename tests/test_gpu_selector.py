"""Selector kernels (features, tcgen05 MLP, training step, classification) against
the oracle in oracle/selector.py (needs a GPU).

Tolerances.  Features are FP32 on the GPU and FP64 in the oracle: each feature
within 2e-5 relative plus 1e-4 of its typical size; counts and shell membership
exactly, except for atoms with a pair distance within 1e-4 A of a cut (excluded,
as FP32 and FP64 may put the pair on different sides).  The MLP accumulates in
FP32 on the tensor cores and in FP64 in the oracle with the same bf16 rounding
points; an accumulation-order difference can move an h1 value across a bf16
rounding boundary (one bf16 ulp, 2^-8 relative), which moves the logit by
~1e-3: logits within 0.05 everywhere and 1e-4 at the median.
"""
import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle as O
import oracle.selector as S

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap

CUTS = (5.5,) + S.SHELL_CUTS
COUNT_FEATURES = (4, 5, 6, 22)


def context(w, prec=None):
    cfg = ap.make_config(I.eam_params(0), I.ace_params(0), w.hyb, precision=ap.PREC_MIXED if prec is None else prec)
    return ap.Context(cfg)


def near_cut(x, box, ids):
    """Atoms of ids with a pair distance within 1e-4 A of a feature cut."""
    nl = O.neighbors_of(x, box, 5.6, ids)
    L = box.hi - box.lo
    bad = np.zeros(len(ids), bool)
    for q in range(len(ids)):
        m = int(nl.cnt[q])
        d = x[nl.j[q, :m]] + nl.s[q, :m] * L - x[ids[q]]
        r = np.sqrt((d * d).sum(1))
        bad[q] = any(np.any(np.abs(r - c) < 1e-4) for c in CUTS)
    return bad


def compare_features(fg, fo):
    scale = np.maximum(np.median(np.abs(fo), axis=0), 1e-2)
    err = np.abs(fg - fo)
    tol = 2e-5 * np.abs(fo) + 1e-4 * scale
    bad = err > tol
    assert not bad.any(), [(int(a), int(f), fg[a, f], fo[a, f]) for a, f in zip(*np.nonzero(bad))][:10]
    assert np.array_equal(fg[:, COUNT_FEATURES], fo[:, COUNT_FEATURES])


def test_features_c1_all_atoms_fp32_and_stored_offsets():
    w = I.config_c1()
    ctx = context(w)
    x = torch.as_tensor(w.x, device="cuda")
    ctx.build_neighbors(x, w.box)
    fg = ctx.sel_features(x).cpu().numpy().astype(np.float64)
    fo = S.features(w.x, w.box, I.eam_params(0))
    ok = ~near_cut(w.x, w.box, np.arange(w.n))
    assert ok.sum() > 200
    compare_features(fg[ok], fo[ok])


def test_features_slab_sampled_atoms():
    w = I.config_c2()
    ctx = context(w)
    x = torch.as_tensor(w.x, device="cuda")
    ctx.build_neighbors(x, w.box)
    fg = ctx.sel_features(x).cpu().numpy().astype(np.float64)
    g = np.random.Generator(np.random.PCG64(I.seed_for(2, 11)))
    L = w.box.hi - w.box.lo
    z = w.x[:, 2]
    # surface layers, the disordered hemisphere and bulk, away from the periodic x/y edges
    inner = (w.x[:, 0] > 15) & (w.x[:, 0] < L[0] - 15) & (w.x[:, 1] > 15) & (w.x[:, 1] < L[1] - 15)
    groups = [np.nonzero(inner & (z > z.max() - 1.0))[0], np.nonzero(inner & (z < z.min() + 1.0))[0],
              np.nonzero(inner & (np.abs(z - np.median(z)) < 10))[0]]
    centre = np.array([L[0] / 2, L[1] / 2, z.max()])
    groups.append(np.nonzero(np.linalg.norm(w.x - centre, axis=1) < 14)[0])
    pick = np.concatenate([g.choice(gr, min(40, len(gr)), replace=False) for gr in groups])
    fo = np.zeros((len(pick), 24))
    keep = np.ones(len(pick), bool)
    for q, i in enumerate(pick):
        d = w.x - w.x[i]
        sel = np.nonzero((d * d).sum(1) < 13.5 ** 2)[0]
        xc = w.x[sel]
        box = I.Box(lo=xc.min(0) - 10, hi=xc.max(0) + 10, periodic=np.array([False] * 3))
        k0 = int(np.nonzero(sel == i)[0][0])
        fo[q] = S.features(xc, box, I.eam_params(0), ids=[k0])[0]
        keep[q] = not near_cut(xc, box, np.array([k0]))[0]
    assert keep.sum() > 0.9 * len(pick)
    compare_features(fg[pick][keep], fo[keep])


def random_model(seed=21):
    g = np.random.Generator(np.random.PCG64(seed))
    theta = S.init_params(g)
    theta[1536:1600] = 0.1 * g.standard_normal(64)                     # b1
    theta[5696:5760] = 0.1 * g.standard_normal(64)                     # b2
    theta[-1] = -0.2
    mu = g.standard_normal(24).astype(np.float32)
    inv = (1.0 / (0.5 + g.random(24))).astype(np.float32)
    return theta.astype(np.float32), mu, inv


def random_features(n, seed=22):
    g = np.random.Generator(np.random.PCG64(seed))
    return (g.standard_normal((n, 24)) * 2.0 + 0.5).astype(np.float32)


@pytest.mark.parametrize("n", [1, 127, 128, 129, 1037, 40000])
def test_mlp_matches_oracle(n):
    theta, mu, inv = random_model()
    feat = random_features(n)
    w = I.config_c1()
    ctx = context(w)
    ctx.sel_set_model(theta, mu, inv)
    p, z = ctx.sel_predict(torch.as_tensor(feat, device="cuda"))
    torch.cuda.synchronize()
    zo = S.forward(theta.astype(np.float64), S.standardise(feat, mu, inv))["z"]
    dz = np.abs(z.cpu().numpy() - zo)
    assert dz.max() < 0.05 and np.median(dz) < 1e-4, (dz.max(), np.median(dz))
    assert np.abs(p.cpu().numpy() - S.sigmoid(zo)).max() < 0.0125


def test_mlp_zero_weights_give_sigmoid_of_b3():
    theta = np.zeros(S.N_PARAMS, np.float32)
    theta[-1] = 0.75
    ctx = context(I.config_c1())
    ctx.sel_set_model(theta, np.zeros(24, np.float32), np.ones(24, np.float32))
    p, z = ctx.sel_predict(torch.as_tensor(random_features(300), device="cuda"))
    assert torch.all(z == 0.75)
    assert torch.allclose(p, torch.full_like(p, 1 / (1 + np.exp(-0.75))), rtol=1e-6, atol=0)
    got, mu, inv = ctx.sel_get_model()
    assert np.array_equal(got, theta) and np.all(mu == 0) and np.all(inv == 1)


def train_problem(b, seed=23):
    g = np.random.Generator(np.random.PCG64(seed))
    feat = random_features(b + 500, seed)
    y = (g.random(b + 500) < 0.3).astype(np.float32)
    wt = (g.random(b + 500) + 0.5).astype(np.float32)
    idx = np.sort(g.choice(b + 500, b, replace=False)).astype(np.int32)
    wt[idx] /= wt[idx].sum()
    return feat, y, wt, idx


@pytest.mark.parametrize("gather", [False, True])
def test_train_step_gradient_matches_oracle(gather):
    b = 3000
    theta, mu, inv = random_model()
    feat, y, wt, idx = train_problem(b)
    if not gather:
        feat, y, wt = feat[idx], y[idx], wt[idx]
        idx = None
    ctx = context(I.config_c1())
    ctx.sel_set_model(theta, mu, inv)
    dev = lambda a: None if a is None else torch.as_tensor(a, device="cuda")
    ctx.sel_train_step(dev(feat), dev(y), dev(wt), idx=dev(idx), b=b, lr=0.0)
    g, loss = ctx.sel_get_grad()
    rows = np.arange(b) if idx is None else idx
    fw = S.forward(theta.astype(np.float64), S.standardise(feat[rows], mu, inv))
    go = S.backward(fw, y[rows].astype(np.float64), wt[rows].astype(np.float64))
    lo = S.loss(fw["z"], y[rows], wt[rows])
    assert abs(loss - lo) <= 1e-4 * abs(lo), (loss, lo)
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    assert rel < 2e-3, rel
    got, _, _ = ctx.sel_get_model()
    assert np.array_equal(got, theta)                                  # lr = 0 leaves the master alone


def test_adam_training_tracks_oracle():
    b = 2048
    theta, mu, inv = random_model(31)
    feat, y, wt, idx = train_problem(b, 32)
    feat, y, wt = feat[idx], y[idx], wt[idx]
    ctx = context(I.config_c1())
    ctx.sel_set_model(theta, mu, inv)
    tf, ty, tw = (torch.as_tensor(a, device="cuda") for a in (feat, y, wt))
    th = theta.astype(np.float64)
    opt = S.Adam(S.N_PARAMS, lr=3e-3)
    xt = S.standardise(feat, mu, inv)
    for step in range(12):
        ctx.sel_train_step(tf, ty, tw, lr=3e-3)
        _, loss = ctx.sel_get_grad()
        fw = S.forward(th, xt)
        lo = S.loss(fw["z"], y, wt)
        assert abs(loss - lo) <= 2e-3 * abs(lo), (step, loss, lo)
        th = opt.step(th, S.backward(fw, y.astype(np.float64), wt.astype(np.float64)))
    got, _, _ = ctx.sel_get_model()
    assert np.abs(got - th).max() < 12 * 3e-3


def test_classification_with_the_selector_matches_oracle():
    w = I.config_c1()
    theta, mu, inv = random_model(41)
    fo = S.features(w.x, w.box, I.eam_params(0))
    po = S.score(theta.astype(np.float64), fo, mu, inv)
    p_lo, p_hi = np.quantile(po, [0.6, 0.85])
    cfg = ap.make_config(I.eam_params(0), I.ace_params(0), w.hyb, precision=ap.PREC_MIXED,
                         detector=ap.DETECT_SELECTOR, sel_p_lo=p_lo, sel_p_hi=p_hi)
    ctx = ap.Context(cfg)
    ctx.sel_set_model(theta, mu, inv)
    x = torch.as_tensor(w.x, device="cuda")
    ctx.build_neighbors(x, w.box)
    lam, idx, npre = ctx.classify(x)
    st = ctx.get_lambda_state()
    l0g = st["lam0"].cpu().numpy()
    sto = O.LambdaState(w.n, w.hyb.n_csp_avg, w.hyb.n_lam_avg)
    lam_o, l0o, *_ = O.classify(sto, w.x, w.box, w.hyb, score=po, score_lo=p_lo, score_hi=p_hi)
    band = (np.abs(po - p_lo) < 0.0125) | (np.abs(po - p_hi) < 0.0125)
    det_g, det_o = l0g < 1.0, l0o < 1.0
    assert np.array_equal(det_g[~band], det_o[~band])
    assert det_o.sum() > 10
    # interior lambda_0 within |f_cut'| <= 1.875 times the score difference over the window
    assert np.abs(l0g - l0o)[~band].max() <= 1.875 * 0.0125 / (p_hi - p_lo) + 1e-12
    # the CSP sample is still the exact one (kept as the reference detector)
    assert np.array_equal(st["csp"].cpu().numpy(), O.csp(w.x, w.box))
