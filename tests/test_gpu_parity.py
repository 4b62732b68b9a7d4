"""CUDA path against the oracle on the same seeded inputs (needs a GPU).

Bars (stated with the method's tolerances):
  * neighbour rows, CSP, lambda_0, lambda_min, lambda and the precise set: bit-exact
    (pairs within 1e-12 r_c^2 of the cutoff are reported and excluded);
  * FP64 mode: per atom |dF_i| <= 1e-5 (|F_i| + 0.01 eV/A), |dE_tot|/N <= 1e-6 eV;
  * mixed mode: max_i |dF_i| <= 1 meV/A, |dE_tot|/N <= 1e-6 eV.
"""
import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap

DEV = "cuda"


def ctx_for(w, precision, hyb=None, ace_seed=0, **kw):
    cfg = ap.make_config(I.eam_params(0), I.ace_params(ace_seed), hyb or w.hyb, precision=precision, **kw)
    return ap.Context(cfg)


def T(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def force_ok(f_gpu, f_or, precision):
    d = np.linalg.norm(f_gpu - f_or, axis=1)
    if precision == ap.PREC_FP64:
        lim = 1e-5 * (np.linalg.norm(f_or, axis=1) + 0.01)
        return bool(np.all(d <= lim)), float((d / lim).max())
    return bool(d.max() <= 1e-3), float(d.max())


def near_cutoff(x, box, i, j, s, rc):
    L = box.hi - box.lo
    d = (x[j] + np.asarray(s) * L) - x[i]
    return abs(float(d @ d) - rc * rc) < 1e-12 * rc * rc


def compare_rows(x, box, rc, cnt, idx, sh, nl_or, ids=None):
    """Rows as sets of (j, s); returns the number of excluded near-cutoff pairs."""
    excluded = 0
    rows = range(len(cnt)) if ids is None else range(len(ids))
    for r in rows:
        i = r if ids is None else int(ids[r])
        g = {(int(idx[r, q]), *map(int, sh[r, q])) for q in range(int(cnt[r]))}
        o = nl_or.pairs(i if nl_or.ids is None else r)
        for (j, *s) in g ^ o:
            assert near_cutoff(x, box, i, j, s, rc), (i, j, s, (j, *s) in g)
            excluded += 1
    return excluded


@pytest.fixture(scope="module")
def c1():
    return I.config_c1()


# ------------------------------------------------------------------ neighbours
def test_neighbor_rows_bit_exact_c1(c1):
    ctx = ctx_for(c1, ap.PREC_FP64)
    x = T(c1.x)
    ctx.build_neighbors(x, c1.box)
    cnt, idx, sh = ctx.get_neighbors(0)
    nl = O.neighbors(c1.x, c1.box, 6.5)
    ex = compare_rows(c1.x, c1.box, 6.5, cnt.cpu().numpy(), idx.cpu().numpy(), sh.cpu().numpy(), nl)
    assert ex <= 2


def test_neighbor_rows_bit_exact_slab_unwrapped():
    # x/y periodic, z free, positions shifted by whole and partial box lengths
    w = I.config_c2()
    sel = np.nonzero(w.x[:, 0] < 40.0)[0][:4000]
    x = w.x[sel].copy()
    L = w.box.hi - w.box.lo
    g = np.random.Generator(np.random.PCG64(77))
    x[:, 0] += L[0] * g.integers(-2, 3, x.shape[0])
    x[:, 1] += L[1] * g.integers(-1, 2, x.shape[0])
    ctx = ctx_for(w, ap.PREC_MIXED)
    ctx.build_neighbors(T(x), w.box)
    cnt, idx, sh = ctx.get_neighbors(0)
    ids = np.arange(0, x.shape[0], 37)
    nl = O.neighbors_of(x, w.box, 6.5, ids)
    cn, ix, s_ = cnt.cpu().numpy(), idx.cpu().numpy(), sh.cpu().numpy()
    compare_rows(x, w.box, 6.5, cn[ids], ix[ids], s_[ids], nl, ids=ids)


# ------------------------------------------------------------------ classification
@pytest.mark.parametrize("hyb", [I.SINGLE_EVAL, I.HybridParams(r_lo=2.0, r_hi=3.5, n_csp_avg=1, n_lam_avg=1,
                                                                 fcut_mode=1)])
def test_classify_bit_exact_c1(c1, hyb):
    ctx = ctx_for(c1, ap.PREC_MIXED, hyb=hyb)
    x = T(c1.x)
    ctx.build_neighbors(x, c1.box)
    lam, qidx, cnt = ctx.classify(x)
    st = ctx.get_lambda_state()
    ost = O.LambdaState(c1.n, 1, 1)
    lam_o, l0_o, csp_o, cavg_o, lmin_o, lavg_o = O.classify(ost, c1.x, c1.box, hyb)
    assert np.array_equal(st["csp"].cpu().numpy(), csp_o)
    assert np.array_equal(st["lam0"].cpu().numpy(), l0_o)
    assert np.array_equal(st["lam_min"].cpu().numpy(), lmin_o)
    assert np.array_equal(lam.cpu().numpy(), lam_o)
    n_p = int(cnt.item())
    assert np.array_equal(qidx[:n_p].cpu().numpy(), np.nonzero(lam_o < 1.0)[0])
    detected = int((l0_o < 1.0).sum())
    assert detected > 0 and n_p >= detected


def test_classify_history_sequence_bit_exact():
    # three lambda updates on a moving 237-atom cell with windows of 3
    w = I.config_c1()
    hyb = I.HybridParams(r_lo=2.0, r_hi=3.5, n_csp_avg=3, n_lam_avg=3, dlam_min=0.05)
    ctx = ctx_for(w, ap.PREC_MIXED, hyb=hyb)
    ost = O.LambdaState(w.n, 3, 3)
    g = np.random.Generator(np.random.PCG64(12))
    x = w.x.copy()
    for it in range(4):
        ctx.build_neighbors(T(x), w.box)
        lam, qidx, cnt = ctx.classify(T(x))
        lam_o, *_ = O.classify(ost, x, w.box, hyb)
        assert np.array_equal(lam.cpu().numpy(), lam_o), it
        x = x + 0.04 * g.standard_normal(x.shape)
        # without a sample (sample_now = 0): the last update's lambda and queue, at moved
        # positions, and the histories untouched (the next update still matches the oracle)
        ctx.build_neighbors(T(x), w.box)
        lam2, q2, cnt2 = ctx.classify(T(x), sample_now=False)
        assert np.array_equal(lam2.cpu().numpy(), lam_o), it
        n2 = int(cnt2.item())
        assert n2 == int(cnt.item()) and np.array_equal(q2[:n2].cpu().numpy(), np.nonzero(lam_o < 1.0)[0])


def test_classify_without_sample_needs_an_update():
    w = I.config_c1()
    ctx = ctx_for(w, ap.PREC_MIXED)
    ctx.build_neighbors(T(w.x), w.box)
    with pytest.raises(ap.ApError) as e:
        ctx.classify(T(w.x), sample_now=False)
    assert e.value.status == 6          # AP_ERR_STATE


def test_eval_eam_features_equal_sel_features():
    """ap_eval_eam's optional feature output is the selector's 24 features of every atom,
    the same values ap_sel_features gives (same kernels, all atoms changeable)."""
    w = I.config_c2()
    ctx = ctx_for(w, ap.PREC_MIXED)
    x = T(w.x)
    ctx.build_neighbors(x, w.box)
    feat = torch.empty((w.n, 24), dtype=torch.float32, device=DEV)
    ef, f = ctx.eval_eam(x, feat=feat)
    ref = ctx.sel_features(x)
    assert torch.equal(feat, ref)
    ef2, f2 = ctx.eval_eam(x)
    assert torch.equal(ef, ef2) and torch.equal(f, f2)


# ------------------------------------------------------------------ potentials
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_eam_ace_hybrid_c1(c1, precision):
    prec = ap.PREC_FP64 if precision == "fp64" else ap.PREC_MIXED
    ctx = ctx_for(c1, prec)
    x = T(c1.x)
    ctx.build_neighbors(x, c1.box)
    lam, qidx, cnt = ctx.classify(x)
    lam_np = lam.cpu().numpy()
    ef, f = ctx.eval_eam(x, lam)
    ep, f = ctx.eval_ace(x, lam, qidx, cnt, f=f)
    e_atom, e_tot = ctx.blend_forces(lam, ef, ep)
    torch.cuda.synchronize()
    ace = O.ACE(I.ace_params(0))
    e_o, f_o, ef_o, ep_o = O.hybrid(c1.x, c1.box, lam_np, I.eam_params(0), ace)
    ok, worst = force_ok(f.cpu().numpy(), f_o, prec)
    assert ok, worst
    assert abs(e_tot.item() - e_o.sum()) / c1.n <= 1e-6
    tol = 1e-10 if prec == ap.PREC_FP64 else 1e-5
    assert np.abs(ef.cpu().numpy() - ef_o).max() < tol
    mask = lam_np < 1
    assert np.abs(ep.cpu().numpy()[mask] - ep_o[mask]).max() < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_ace_and_full_eam_limits(c1, precision):
    prec = ap.PREC_FP64 if precision == "fp64" else ap.PREC_MIXED
    ctx = ctx_for(c1, prec)
    x = T(c1.x)
    ctx.build_neighbors(x, c1.box)
    n = c1.n
    ace = O.ACE(I.ace_params(0))
    # lambda = 0: pure ACE
    lam0 = torch.zeros(n, dtype=torch.float64, device=DEV)
    allidx = torch.arange(n, dtype=torch.int32, device=DEV)
    cnt = torch.tensor([n], dtype=torch.int64, device=DEV)
    ef, f = ctx.eval_eam(x, lam0)
    ep, f = ctx.eval_ace(x, lam0, allidx, cnt, f=f)
    e_o, f_o = ace.eval(c1.x, c1.box)
    assert force_ok(f.cpu().numpy(), f_o, prec)[0]
    assert abs(ep.sum().item() - e_o.sum()) / n < 1e-6
    # lambda = 1: pure EAM, empty queue
    lam1 = torch.ones(n, dtype=torch.float64, device=DEV)
    zero = torch.zeros(1, dtype=torch.int64, device=DEV)
    ef, f = ctx.eval_eam(x, lam1)
    ep, f = ctx.eval_ace(x, lam1, allidx, zero, f=f)
    e_o, f_o, _, _ = O.eam(c1.x, c1.box, I.eam_params(0))
    assert force_ok(f.cpu().numpy(), f_o, prec)[0]
    assert float(ep.abs().max()) == 0.0


def test_forced_lambda_mix_c3_fp64_and_mixed():
    w = I.config_c3()
    ace = O.ACE(I.ace_params(0))
    e_o, f_o, _, _ = O.hybrid(w.x, w.box, w.lam, I.eam_params(0), ace)
    for prec in (ap.PREC_FP64, ap.PREC_MIXED):
        ctx = ctx_for(w, prec)
        x = T(w.x)
        ctx.build_neighbors(x, w.box)
        lam = T(w.lam)
        q = np.nonzero(w.lam < 1)[0]
        qidx = T(q, torch.int32)
        cnt = torch.tensor([len(q)], dtype=torch.int64, device=DEV)
        ef, f = ctx.eval_eam(x, lam)
        ep, f = ctx.eval_ace(x, lam, qidx, cnt, f=f)
        e_atom, e_tot = ctx.blend_forces(lam, ef, ep)
        ok, worst = force_ok(f.cpu().numpy(), f_o, prec)
        assert ok, (prec, worst)
        assert abs(e_tot.item() - e_o.sum()) / w.n <= 1e-6


def test_batched_cells_one_launch():
    cells = I.config_c3_batch(64)
    sizes = [c.n for c in cells]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    x = np.concatenate([c.x for c in cells])
    lam = np.concatenate([c.lam for c in cells])
    ctx = ctx_for(cells[0], ap.PREC_MIXED)
    ctx.build_neighbors_batch(T(x), offs.tolist(), [c.box for c in cells])
    q = np.nonzero(lam < 1)[0]
    ef, f = ctx.eval_eam(T(x), T(lam))
    ep, f = ctx.eval_ace(T(x), T(lam), T(q, torch.int32), torch.tensor([len(q)], dtype=torch.int64, device=DEV),
                         f=f)
    e_atom, _ = ctx.blend_forces(T(lam), ef, ep)
    f, e_atom = f.cpu().numpy(), e_atom.cpu().numpy()
    ace = O.ACE(I.ace_params(0))
    for k, c in enumerate(cells):         # every cell: forces and the cell's energy
        e_o, f_o, _, _ = O.hybrid(c.x, c.box, c.lam, I.eam_params(0), ace)
        ok, worst = force_ok(f[offs[k]:offs[k + 1]], f_o, ap.PREC_MIXED)
        assert ok, (k, worst)
        assert abs(e_atom[offs[k]:offs[k + 1]].sum() - e_o.sum()) / c.n <= 1e-6, k


# ------------------------------------------------------------------ dynamics
def test_md_fixed_lambda_energy_conservation_fp64():
    # lambda held constant (update period longer than the run): conservative (section 2.3)
    w = I.config_c1()
    hyb = I.HybridParams(r_lo=2.0, r_hi=3.5, n_csp_avg=1, n_lam_avg=1, sample_every=100000)
    ctx = ctx_for(w, ap.PREC_FP64, hyb=hyb, dt=1.0, rebuild_every=10)
    v0 = I.maxwell_boltzmann(w.mass, np.ones(w.n, bool), 300.0, I.rng_for(1, 3))
    x, v = T(w.x), T(v0)
    f = torch.zeros_like(x)
    mass = T(w.mass)
    lam = torch.empty(w.n, dtype=torch.float64, device=DEV)
    ctx.build_neighbors(x, w.box)
    s0 = ctx.step(x, v, f, mass, None, lam, 0)
    e0 = s0.e_pot + s0.e_kin
    s1 = ctx.step(x, v, f, mass, None, lam, 200)
    drift = abs(s1.e_pot + s1.e_kin - e0) / w.n
    assert drift < 1e-5, drift
    assert s1.n_precise > 0


def test_md_matches_oracle_trajectory_fp64():
    # 20 velocity-Verlet steps with the lambda step every 5 steps, against the oracle
    w = I.config_c1()
    hyb = I.HybridParams(r_lo=2.0, r_hi=3.5, n_csp_avg=2, n_lam_avg=2, dlam_min=0.01, sample_every=5)
    ctx = ctx_for(w, ap.PREC_FP64, hyb=hyb, dt=1.0)
    v0 = I.maxwell_boltzmann(w.mass, np.ones(w.n, bool), 300.0, I.rng_for(1, 5))
    x, v = T(w.x), T(v0)
    f = torch.zeros_like(x)
    lam = torch.empty(w.n, dtype=torch.float64, device=DEV)
    ctx.build_neighbors(x, w.box)
    ctx.step(x, v, f, T(w.mass), None, lam, 20)
    # oracle
    ace = O.ACE(I.ace_params(0))
    p = I.eam_params(0)
    st = O.LambdaState(w.n, 2, 2)
    lam_o = O.classify(st, w.x, w.box, hyb)[0]
    xo, vo = w.x.copy(), v0.copy()
    fo = O.hybrid(xo, w.box, lam_o, p, ace)[1]
    for k in range(1, 21):
        def force(xn, k=k):
            nonlocal lam_o
            if k % 5 == 0:
                lam_o = O.classify(st, xn, w.box, hyb)[0]
            return (O.hybrid(xn, w.box, lam_o, p, ace)[1],)
        xo, vo, out = O.md_step(xo, vo, fo, w.mass, 1.0, force)
        fo = out[0]
    L = w.box.hi - w.box.lo
    dx = x.cpu().numpy() - xo
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-9
    # the trajectories differ at round-off level, so compare lambda to tolerance and the sets exactly
    lg = lam.cpu().numpy()
    assert np.abs(lg - lam_o).max() < 1e-8
    assert np.array_equal(lg < 1.0, lam_o < 1.0)


def test_precise_queue_from_lambda(c1):
    ctx = ctx_for(c1, ap.PREC_MIXED)
    ctx.build_neighbors(T(c1.x), c1.box)
    g = np.random.Generator(np.random.PCG64(I.seed_for(1, 31)))
    lam = np.where(g.random(c1.n) < 0.5, 1.0, g.random(c1.n))
    lam[[0, 5, c1.n - 1]] = [1.0, np.nextafter(1.0, 0.0), 0.0]     # exact edges
    idx, cnt = ctx.precise_queue(T(lam))
    k = int(cnt.item())
    assert np.array_equal(idx[:k].cpu().numpy(), np.nonzero(lam < 1.0)[0])
    idx, cnt = ctx.precise_queue(T(np.ones(c1.n)))
    assert int(cnt.item()) == 0


def test_neighbor_total_is_the_sum_of_the_row_counts(c1):
    """ap_neighbor_total (instrumentation) against the exported EAM and ACE row counts."""
    w = c1
    ctx = ctx_for(w, ap.PREC_FP64)
    x = T(w.x)
    ctx.build_neighbors(x, w.box)
    cnt, _, _ = ctx.get_neighbors(0)
    assert ctx.neighbor_total(0) == int(cnt.sum().item()) > 0
    lam, q, nq = ctx.classify(x)
    ctx.eval_ace(x, lam, q, nq)
    cnt1, _, _ = ctx.get_neighbors(1)
    assert ctx.neighbor_total(1) == int(cnt1.sum().item())
