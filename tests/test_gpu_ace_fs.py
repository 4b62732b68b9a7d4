"""Finnis-Sinclair ACE form E = phi^(1) + F(phi^(2)) (Eq. energy_ace) on the GPU
against oracle.ACEFS (needs a GPU).  Same bars as the linear ACE parity tests:
FP64 |dF_i| <= 1e-5 (|F_i| + 0.01 eV/A), mixed max |dF_i| <= 1 meV/A, total energy
within 1e-6 eV/atom; in three phi^(2) regimes (square root, odd extension,
transition) on the 2,048-atom cell with lambda forced to {0, 1, U(0,1)}."""
import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap


def T(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("scale", [-0.1, 0.1, -0.001])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fs_hybrid_matches_oracle(scale, precision):
    w = I.config_c3()
    p = I.ace_params_fs(0, c2_scale=scale)
    prec = ap.PREC_FP64 if precision == "fp64" else ap.PREC_MIXED
    e_o, f_o, _, ep_o = O.hybrid(w.x, w.box, w.lam, I.eam_params(0), O.ACEFS(p))
    ctx = ap.Context(ap.make_config(I.eam_params(0), p, w.hyb, precision=prec))
    x = T(w.x)
    ctx.build_neighbors(x, w.box)
    lam = T(w.lam)
    q = np.nonzero(w.lam < 1)[0]
    qidx = T(q, torch.int32)
    cnt = torch.tensor([len(q)], dtype=torch.int64, device="cuda")
    ef, f = ctx.eval_eam(x, lam)
    ep, f = ctx.eval_ace(x, lam, qidx, cnt, f=f)
    _, e_tot = ctx.blend_forces(lam, ef, ep)
    fg = f.cpu().numpy()
    d = np.linalg.norm(fg - f_o, axis=1)
    if prec == ap.PREC_FP64:
        lim = 1e-5 * (np.linalg.norm(f_o, axis=1) + 0.01)
        assert np.all(d <= lim), (d / lim).max()
        assert np.abs(ep.cpu().numpy()[q] - ep_o[q]).max() < 1e-10
    else:
        assert d.max() <= 1e-3, d.max()
    assert abs(e_tot.item() - e_o.sum()) / w.n <= 1e-6


def test_fs_energy_only_path_and_autograd():
    """The autograd forward (energy-only ACE) and backward (adjoint) of the FS form."""
    from paper_2411_03002_gb300 import autograd
    w = I.config_c3()
    p = I.ace_params_fs(0, c2_scale=-0.1)
    ctx = ap.Context(ap.make_config(I.eam_params(0), p, w.hyb, precision=ap.PREC_FP64))
    x = T(w.x).requires_grad_(True)
    e = autograd.energy(x, T(w.lam), ctx, box=w.box)
    e.backward()
    e_o, f_o, _, _ = O.hybrid(w.x, w.box, w.lam, I.eam_params(0), O.ACEFS(p))
    assert abs(e.item() - e_o.sum()) / w.n <= 1e-6
    d = np.linalg.norm(-x.grad.cpu().numpy() - f_o, axis=1)
    assert np.all(d <= 1e-5 * (np.linalg.norm(f_o, axis=1) + 0.01))
