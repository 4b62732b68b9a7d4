"""ap_spatial_order: the atoms in the cell order of the last build (needs a GPU).

* On a randomly shuffled 32,000-atom slab the order is a permutation, and consecutive
  atoms in it are neighbours in space (mean distance below 5 A, against tens of A in the
  shuffled order);
* the EAM energies and forces of the reordered system, mapped back, equal the original
  ones within the FP64 bar (the order changes only the memory layout);
* with a batch of cells every system's atoms stay inside that system's index range.
"""
import numpy as np
import pytest
import torch

import ap_inputs as I

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap


def test_order_of_a_shuffled_slab():
    w = I.config_c2()
    p = np.random.Generator(np.random.PCG64(I.seed_for(2, 60))).permutation(w.n)
    xs = w.x[p]
    ctx = ap.Context(ap.make_config(I.eam_params(0), I.ace_params(0), w.hyb, precision=ap.PREC_FP64))
    x = torch.as_tensor(xs, device="cuda")
    ctx.build_neighbors(x, w.box)
    order = ctx.spatial_order().cpu().numpy().astype(np.int64)
    assert np.array_equal(np.sort(order), np.arange(w.n))
    gap_shuffled = np.linalg.norm(np.diff(xs, axis=0), axis=1).mean()
    gap_ordered = np.linalg.norm(np.diff(xs[order], axis=0), axis=1).mean()
    assert gap_ordered < 5.0 < gap_shuffled, (gap_ordered, gap_shuffled)
    lam = np.random.Generator(np.random.PCG64(3)).uniform(0.0, 1.0, w.n)
    e1, f1 = ctx.eval_eam(x, torch.as_tensor(lam, device="cuda"))
    x2 = torch.as_tensor(np.ascontiguousarray(xs[order]), device="cuda")
    ctx.build_neighbors(x2, w.box)
    e2, f2 = ctx.eval_eam(x2, torch.as_tensor(np.ascontiguousarray(lam[order]), device="cuda"))
    e1, f1, e2, f2 = (t.cpu().numpy() for t in (e1, f1, e2, f2))
    d = np.linalg.norm(f2 - f1[order], axis=1)
    assert np.all(d <= 1e-5 * (np.linalg.norm(f1[order], axis=1) + 0.01)), d.max()
    assert np.abs(e2 - e1[order]).max() < 1e-10


def test_batch_order_keeps_each_system_in_its_range():
    cells = I.config_c3_batch(8)
    offs = np.concatenate([[0], np.cumsum([c.n for c in cells])])
    x = np.concatenate([c.x for c in cells])
    ctx = ap.Context(ap.make_config(I.eam_params(0), I.ace_params(0), I.SINGLE_EVAL, precision=ap.PREC_MIXED))
    ctx.build_neighbors_batch(torch.as_tensor(x, device="cuda"), offs.tolist(), [c.box for c in cells])
    order = ctx.spatial_order().cpu().numpy()
    for s in range(len(cells)):
        part = order[offs[s]:offs[s + 1]]
        assert np.array_equal(np.sort(part), np.arange(offs[s], offs[s + 1])), s
