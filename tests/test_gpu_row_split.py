"""EAM rows split at the potential cutoff (needs a GPU).

The row build puts the entries inside r_c first and the skin entries after them;
the density pass marks where the in-range entries end and the force pass walks only
that prefix (Eq. F_i_d at fixed lambda).  Checked here:
* the exported rows are ordered so: no entry beyond r_c (FP64 distance, outside a
  1e-4 A band that the build's FP32 test may place either way) comes before an entry
  inside r_c;
* after every atom moves by up to 0.45 A without a rebuild (skin/2 = 0.5 A), pairs
  from the skin part come within r_c; the lambda-weighted EAM energies and forces
  still match the oracle at the moved positions (FP64 and mixed precision), on the
  stored-offset path (the 237-atom cell) and the packed-cell-code path (the
  32,000-atom slab);
* the prefix total that ap_neighbor_total(which = 2) reports matches the rows.
"""
import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def workload(name):
    return I.config_c1() if name == "cell237" else I.config_c2()


@pytest.mark.parametrize("name", ["cell237", "slab32k"])
def test_rows_put_the_in_range_entries_first(name):
    w = workload(name)
    p = I.eam_params(0)
    ctx = ap.Context(ap.make_config(p, I.ace_params(0), w.hyb, precision=ap.PREC_MIXED))
    ctx.build_neighbors(T(w.x), w.box)
    cnt, idx, sh = (a.cpu().numpy() for a in ctx.get_neighbors(0))
    L = w.box.hi - w.box.lo
    band = 1e-4
    rows = range(w.n) if w.n < 1000 else range(0, w.n, 7)
    for i in rows:
        c = int(cnt[i])
        d = w.x[idx[i, :c]] + sh[i, :c] * L - w.x[i]
        r = np.sqrt((d * d).sum(1))
        inside = np.nonzero(r < p.rc - band)[0]
        outside = np.nonzero(r > p.rc + band)[0]
        if len(inside) and len(outside):
            assert outside.min() > inside.max(), i
    ctx.close()


@pytest.mark.parametrize("name", ["cell237", "slab32k"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_eam_after_moves_without_rebuild(name, precision):
    w = workload(name)
    p = I.eam_params(0)
    prec = ap.PREC_FP64 if precision == "fp64" else ap.PREC_MIXED
    ctx = ap.Context(ap.make_config(p, I.ace_params(0), w.hyb, precision=prec))
    ctx.build_neighbors(T(w.x), w.box)
    g = np.random.Generator(np.random.PCG64(I.seed_for(2, 71)))
    u = g.standard_normal((w.n, 3))
    u *= (0.45 * g.uniform(0.0, 1.0, w.n) ** (1.0 / 3.0) / np.linalg.norm(u, axis=1))[:, None]
    x1 = w.x + u
    lam = g.uniform(0.0, 1.0, w.n)
    with pytest.raises(Exception):
        ctx.neighbor_total(2)        # no EAM evaluation on these rows yet
    # pairs that came inside r_c from the skin part of the rows
    n0, n1 = O.neighbors(w.x, w.box, p.rc), O.neighbors(x1, w.box, p.rc)
    came_in = sum(len(n1.pairs(i) - n0.pairs(i)) for i in range(0, w.n, 1 if w.n < 1000 else 5))
    assert came_in > 0
    ef, f = ctx.eval_eam(T(x1), T(lam))
    torch.cuda.synchronize()
    e_o, f_o, _, _ = O.eam(x1, w.box, p, weights=lam)
    d = np.linalg.norm(f.cpu().numpy() - f_o, axis=1)
    if prec == ap.PREC_FP64:
        assert np.all(d <= 1e-5 * (np.linalg.norm(f_o, axis=1) + 0.01)), d.max()
        assert np.abs(ef.cpu().numpy() - e_o).max() < 1e-10
        # the force pass walked, per atom, up to the last row entry inside r_c at x1
        cnt, idx, sh = (a.cpu().numpy() for a in ctx.get_neighbors(0))
        L = w.box.hi - w.box.lo
        want = 0
        for i in range(w.n):
            c = int(cnt[i])
            dd = x1[idx[i, :c]] + sh[i, :c] * L - x1[i]
            inside = np.nonzero((dd * dd).sum(1) < p.rc * p.rc)[0]
            want += int(inside.max()) + 1 if len(inside) else 0
        assert abs(ctx.neighbor_total(2) - want) <= 2
        assert ctx.neighbor_total(2) < ctx.neighbor_total(0)
    else:
        # FP32 pair terms: about 54 per atom of up to ~5 eV at the closest displaced
        # pairs, so one site energy may carry 54 x 5 x 6e-8 ~ 2e-5 eV of rounding; the
        # bound is 1e-4 eV per atom and 1e-6 eV per atom on the total
        assert d.max() <= 1e-3, d.max()
        efn = ef.cpu().numpy()
        assert np.abs(efn - e_o).max() < 1e-4
        assert abs(efn.sum() - e_o.sum()) / w.n < 1e-6
    ctx.close()


def test_csp_on_fresh_rows_matches_the_full_row_walk():
    """ap_step classifies on rows built at the same positions, where the CSP may stop after
    a row's in-range part; ap_classify walks whole rows.  Both, and the oracle, agree bit
    for bit on the 32,000-atom slab (with its disordered hemisphere)."""
    w = I.config_c2()
    cfg = ap.make_config(I.eam_params(0), I.ace_params(0), w.hyb, precision=ap.PREC_MIXED, dt=w.dt)
    ctx = ap.Context(cfg)
    x = T(w.x)
    v = T(w.v)
    f = torch.zeros_like(x)
    lam = torch.empty(w.n, dtype=torch.float64, device="cuda")
    ctx.build_neighbors(x, w.box)
    ctx.step(x, v, f, T(w.mass), None, lam, 0)
    csp_step = ctx.get_lambda_state()["csp"].cpu().numpy()
    ctx2 = ap.Context(cfg)
    ctx2.build_neighbors(x, w.box)
    ctx2.classify(x)
    csp_full = ctx2.get_lambda_state()["csp"].cpu().numpy()
    assert np.array_equal(csp_step, csp_full)
    assert np.array_equal(csp_step, O.csp(x.cpu().numpy(), w.box))
    ctx.close()
    ctx2.close()
