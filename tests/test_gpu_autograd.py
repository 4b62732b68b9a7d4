"""torch.autograd.Function over the energy kernels, backward = adjoint kernels
(needs a GPU).  Workload: the 2,048-atom cell with lambda forced to thirds of
{0, 1, U(0,1)}, and a batch of 64 cells of 500-4,000 atoms in one launch.

Bars: FP64 backward vs central finite differences of the FP64 forward energy
(h = 1e-4 A, 64 seeded atoms x 3 components): |dF| <= 1e-6 |F| + 1e-7 eV/A;
backward vs the oracle gradient: FP64 |dF_i| <= 1e-5 (|F_i| + 0.01), FP32 1 meV/A;
forward energy vs oracle: 1e-6 eV/atom.
"""
import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap
    from paper_2411_03002_gb300.autograd import energy


@pytest.fixture(scope="module")
def c3():
    w = I.config_c3()
    e_o, f_o, _, _ = O.hybrid(w.x, w.box, w.lam, I.eam_params(0), O.ACE(I.ace_params(0)))
    return w, e_o, f_o


def ctx_for(w, prec):
    return ap.Context(ap.make_config(I.eam_params(0), I.ace_params(0), w.hyb, precision=prec))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_backward_matches_oracle_gradient(c3, prec):
    w, e_o, f_o = c3
    p = ap.PREC_FP64 if prec == "fp64" else ap.PREC_MIXED
    ctx = ctx_for(w, p)
    x = torch.as_tensor(w.x, device="cuda").requires_grad_(True)
    lam = torch.as_tensor(w.lam, device="cuda")
    e = energy(x, lam, ctx, box=w.box)
    e.backward()
    f = -x.grad.cpu().numpy()
    assert abs(e.item() - e_o.sum()) / w.n <= 1e-6
    d = np.linalg.norm(f - f_o, axis=1)
    if p == ap.PREC_FP64:
        assert np.all(d <= 1e-5 * (np.linalg.norm(f_o, axis=1) + 0.01)), d.max()
    else:
        assert d.max() <= 1e-3, d.max()


def test_backward_matches_finite_differences_fp64(c3):
    w, _, _ = c3
    ctx = ctx_for(w, ap.PREC_FP64)
    lam = torch.as_tensor(w.lam, device="cuda")
    x0 = torch.as_tensor(w.x, device="cuda")
    x = x0.clone().requires_grad_(True)
    energy(x, lam, ctx, box=w.box).backward()
    f = -x.grad.cpu().numpy()
    g = np.random.Generator(np.random.PCG64(I.seed_for(3, 5)))
    atoms = g.choice(w.n, size=64, replace=False)
    h = 1e-4
    worst = 0.0
    for i in atoms:
        for k in range(3):
            xp = x0.clone()
            xp[i, k] += h
            xm = x0.clone()
            xm[i, k] -= h
            with torch.no_grad():
                ep = energy(xp, lam, ctx, box=w.box).item()
                em = energy(xm, lam, ctx, box=w.box).item()
            fd = -(ep - em) / (2 * h)
            err = abs(fd - f[i, k]) / (1e-6 * abs(f[i, k]) + 1e-7)
            worst = max(worst, err)
    assert worst <= 1.0, worst


def test_batch_of_64_cells_in_one_launch():
    cells = I.config_c3_batch(64)
    offs = np.concatenate([[0], np.cumsum([c.n for c in cells])])
    x = torch.as_tensor(np.concatenate([c.x for c in cells]), device="cuda").requires_grad_(True)
    lam = torch.as_tensor(np.concatenate([c.lam for c in cells]), device="cuda")
    ctx = ctx_for(cells[0], ap.PREC_MIXED)
    e = energy(x, lam, ctx, batch=(offs.tolist(), [c.box for c in cells]))
    e.backward()
    f = -x.grad.cpu().numpy()
    # per-cell energies: the site energies of the same context on the same rows
    idx, cnt = ctx.precise_queue(lam)
    ef, _ = ctx.eval_eam(x.detach(), lam)
    ep, _ = ctx.eval_ace(x.detach(), lam, idx, cnt, forces=False)
    e_atom = ctx.blend_forces(lam, ef, ep)[0].cpu().numpy()
    ace = O.ACE(I.ace_params(0))
    e_sum, n_sum = 0.0, 0
    for k, c in enumerate(cells):         # every cell: forces from backward, the cell's energy
        e_o, f_o, _, _ = O.hybrid(c.x, c.box, c.lam, I.eam_params(0), ace)
        d = np.linalg.norm(f[offs[k]:offs[k + 1]] - f_o, axis=1)
        assert d.max() <= 1e-3, (k, d.max())
        assert abs(e_atom[offs[k]:offs[k + 1]].sum() - e_o.sum()) / c.n <= 1e-6, k
        e_sum += e_o.sum()
        n_sum += c.n
    assert abs(e.item() - e_sum) / n_sum <= 1e-6
