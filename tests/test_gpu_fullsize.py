"""Parity at the full benchmark size, through the timed region's path (needs a GPU).

The 4,000,000-atom nanoindentation-shaped slab is prepared and integrated exactly as
bench.py times it (mixed precision, Hyb2, lambda updated every 10 MD steps, the lists
on the skin criterion with the bench's 0.7 A skin, indenter, fixed bottom layers): ap_step(0) prepares, then
ap_step runs 10, 10 and 5 MD steps.  The lambda updates at steps 10 and 20 push the
second and third CSP and lambda_min samples into the 11-sample windows (Eqs. csp_2_i,
lambda_3_i).  At 300 K no atom moves 0.45 skin = 0.315 A in 10 fs, so the update at step 10
keeps the lists of step 0: its CSP comes from rows 10 steps older than the positions,
its spread from old cells, and its ACE rows are built from those cells; the forces at
step 25 are evaluated on rows older still (the EAM force pass walks the prefix the
density pass found).

About 1,000 sampled atoms are checked against the oracle run on local clusters with
the GPU's own positions at each step:
* CSP, lambda_0 and lambda bit-exact at steps 0, 10 and 20 (the oracle replays the
  same sequence of samples with one LambdaState per cluster);
* forces (EAM + ACE at the GPU's lambda, + indenter at t = step dt) within 1 meV/A
  at steps 0, 10 and 25.
Samples are stratified: 6 clusters under the top surface (one beneath the indenter)
give detected atoms (lambda_0 < 1), other atoms with lambda = 0, interior lambda and
lambda = 1; 2 clusters above the fixed bottom layers give mobile and fixed atoms there.
A classification cluster has radius 45 A around its centre, samples lie within 16 A
of it: a sample's lambda depends on lambda_0 within r_hi = 20 A, whose CSP depends on
neighbours within r_c + skin = 6.2 A, so 16 + 20 + 6.2 leaves a 2.8 A margin to the cut.  Force
clusters have radius 32 A (EAM densities within 2 x 5.5 A, ACE site energies within
7 A of a sample and their neighbours within 7 A: 16 + 14 A, plus 2 A for the motion
over 25 steps), with lambda from the GPU (checked above).  Cluster centres keep
50 A from the periodic x/y edges, so no image shift enters the cluster coordinates.
"""
import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap

R_CLASSIFY, R_FORCE, R_SAMPLE = 45.0, 32.0, 16.0
STEPS = (0, 10, 20, 25)            # MD step after each ap_step call
SKIN = 0.7                         # the bench's neighbour-list skin (A)


def _open_box(xc):
    return I.Box(lo=xc.min(0) - 20.0, hi=xc.max(0) + 20.0, periodic=np.array([False, False, False]))


@pytest.fixture(scope="module")
def run():
    w = I.config_c5(100, hyb=I.HYB2)
    cfg = ap.make_config(I.eam_params(0), I.ace_for_config(5), w.hyb, precision=ap.PREC_MIXED, indenter=w.indenter,
                         lambda_every=10, dt=w.dt, skin=SKIN, rebuild_every=ap.REBUILD_SKIN)
    ctx = ap.Context(cfg)
    dev = "cuda"
    x = torch.as_tensor(w.x, device=dev).clone()
    v = torch.as_tensor(w.v, device=dev).clone()
    f = torch.zeros((w.n, 3), dtype=torch.float64, device=dev)
    lam = torch.empty(w.n, dtype=torch.float64, device=dev)
    mass, fixed = torch.as_tensor(w.mass, device=dev), torch.as_tensor(w.fixed, device=dev)
    ctx.build_neighbors(x, w.box)
    snaps = {}
    stats = None
    for step, k in zip(STEPS, (0, 10, 10, 5)):
        stats = ctx.step(x, v, f, mass, fixed, lam, k)
        st = ctx.get_lambda_state()
        snaps[step] = dict(x=x.cpu().numpy(), f=f.cpu().numpy(), lam=lam.cpu().numpy(), csp=st["csp"].cpu().numpy(),
                           lam0=st["lam0"].cpu().numpy())
        if step == 0:
            stats0 = stats
    ctx.close()
    torch.cuda.empty_cache()
    return dict(w=w, snaps=snaps, stats=stats, stats0=stats0)


def clusters(p):
    """(centre, sample indices) of the 8 clusters, samples drawn from the step-0 state."""
    w, s0 = p["w"], p["snaps"][0]
    x, lam, lam0 = s0["x"], s0["lam"], s0["lam0"]
    L = w.box.hi - w.box.lo
    ztop = float(x[:, 2].max())
    zfix = float(x[w.fixed != 0, 2].max())
    g = np.random.Generator(np.random.PCG64(I.seed_for(5, 9)))
    centres = [np.array([L[0] / 2, L[1] / 2, ztop - 12.0])]          # beneath the indenter
    for _ in range(5):
        centres.append(np.array([g.uniform(60.0, L[0] - 60.0), g.uniform(60.0, L[1] - 60.0), ztop - 12.0]))
    for _ in range(2):
        centres.append(np.array([g.uniform(60.0, L[0] - 60.0), g.uniform(60.0, L[1] - 60.0), zfix + 4.0]))
    out = []
    for k, c in enumerate(centres):
        d = x - c
        near = ((d * d).sum(1) < R_SAMPLE * R_SAMPLE)
        if k < 6:
            strata = [(near & (lam0 < 1.0), 35),                                   # detected
                      (near & (lam0 == 1.0) & (lam == 0.0), 35),                   # lambda = 0, not detected
                      (near & (lam > 0.0) & (lam < 1.0), 35),                      # switching zone
                      (near & (lam == 1.0), 25)]                                   # fast
        else:
            strata = [(near & (w.fixed == 0) & (x[:, 2] < zfix + 10.0), 90),       # mobile, by the fixed layers
                      (near & (w.fixed != 0), 30)]                                 # fixed
        idx = []
        for mask, count in strata:
            cand = np.nonzero(mask)[0]
            if len(cand):
                idx.extend(g.choice(cand, size=min(count, len(cand)), replace=False).tolist())
        out.append((c, np.array(sorted(set(idx)))))
    return out


@pytest.fixture(scope="module")
def plan(run):
    return clusters(run)


def test_sample_count_and_strata(run, plan):
    s0 = run["snaps"][0]
    idx = np.concatenate([s for _, s in plan])
    assert len(idx) >= 1000
    lam, lam0, fixed = s0["lam"][idx], s0["lam0"][idx], run["w"].fixed[idx]
    for name, m in (("detected", lam0 < 1.0), ("lambda=0", lam == 0.0), ("interior", (lam > 0) & (lam < 1)),
                    ("lambda=1", lam == 1.0), ("fixed", fixed != 0)):
        assert m.sum() >= 50, name


def test_updates_kept_the_lists(run):
    st = run["stats"]
    print(f"4M run: kept {st.kept} of 2 updates, rebuilds {st.rebuilds}, max displacement {st.max_disp:.3f} A")
    assert st.kept >= 1 and st.error_bits == 0


def test_precise_fraction_in_expected_range(run):
    for s in (run["stats0"], run["stats"]):
        frac = s.n_precise / run["w"].n
        assert 0.02 < frac < 0.10, frac
        assert s.n_detected > 0


def test_lambda_bit_exact_at_steps_0_10_20(run, plan):
    w, snaps = run["w"], run["snaps"]
    for c, samples in plan:
        x0 = snaps[0]["x"]
        d = x0 - c
        sel = np.nonzero((d * d).sum(1) < R_CLASSIFY * R_CLASSIFY)[0]
        pos = np.searchsorted(sel, samples)
        assert np.array_equal(sel[pos], samples)
        ch = (w.fixed[sel] == 0).astype(np.uint8)
        st = O.LambdaState(len(sel), w.hyb.n_csp_avg, w.hyb.n_lam_avg)
        for step in (0, 10, 20):
            xc = snaps[step]["x"][sel]
            lam_o, l0_o, csp_o, *_ = O.classify(st, xc, _open_box(xc), w.hyb, changeable=ch,
                                                r_search=I.eam_params(0).rc + SKIN)
            assert np.array_equal(csp_o[pos], snaps[step]["csp"][samples]), step
            assert np.array_equal(l0_o[pos], snaps[step]["lam0"][samples]), step
            assert np.array_equal(lam_o[pos], snaps[step]["lam"][samples]), step


def test_forces_within_1_meV_at_steps_0_10_25(run, plan):
    w, snaps = run["w"], run["snaps"]
    ace, p = O.ACE(I.ace_for_config(5)), I.eam_params(0)
    worst = 0.0
    checked = 0
    for c, samples in plan:
        mobile = samples[w.fixed[samples] == 0]
        for step in (0, 10, 25):
            s = snaps[step]
            x0 = snaps[0]["x"]
            d = x0 - c
            sel = np.nonzero((d * d).sum(1) < R_FORCE * R_FORCE)[0]
            pos = np.searchsorted(sel, mobile)
            xc = s["x"][sel]
            _, f_o, _, _ = O.hybrid(xc, _open_box(xc), s["lam"][sel], p, ace)
            centre_t = w.indenter.center0 + w.indenter.velocity * (step * w.dt)
            _, f_ind = O.indenter(xc[pos], centre_t, w.indenter.radius, w.indenter.k)
            dd = np.linalg.norm(s["f"][mobile] - (f_o[pos] + f_ind), axis=1)
            worst = max(worst, float(dd.max()))
            checked += len(mobile)
    assert checked >= 3 * 850
    assert worst <= 1e-3, worst
