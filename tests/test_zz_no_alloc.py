"""ap_eval_eam_static: the allocation-free EAM entry point, for callers that
cannot allocate device memory themselves (their device memory belongs to
another runtime's pool, or their memory budget is fixed up front).

It is called here through the C-ABI (ctypes) and compared, on two calls in a
row, with the regular context-based ap_eval_eam in FP64 mode and with the FP64
oracle's EAM, with the FP64 force tolerance used by the other parity tests:
|dF_i| <= 1e-5 (|F_i| + 0.01 eV/A), and site energies within 1e-10 eV.  Also: no
lambda (NULL = all 1), and a periodic cell shorter than twice the cutoff, where
an atom's own images are its neighbours.
This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap
    from paper_2411_03002_gb300 import _native as N


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def reference(w, cfg, lam):
    ctx = ap.Context(cfg)
    x = torch.as_tensor(w.x, device="cuda")
    ctx.build_neighbors(x, w.box)
    e, f = ctx.eval_eam(x, lam)
    torch.cuda.synchronize()
    return e.cpu().numpy(), f.cpu().numpy()


def static_call(w, cfg, lam):
    lib = N.lib()
    x = torch.as_tensor(w.x, device="cuda")
    e = torch.full((w.n,), np.nan, dtype=torch.float64, device="cuda")
    f = torch.zeros((w.n, 3), dtype=torch.float64, device="cuda")
    box = ap.make_box(w.box.lo, w.box.hi, w.box.periodic)
    st = lib.ap_eval_eam_static(ctypes.byref(cfg), w.n, _p(x), ctypes.byref(box), _p(lam), _p(e), _p(f),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return e.cpu().numpy(), f.cpu().numpy()


@pytest.mark.parametrize("name", ["c1", "c3", "slab"])
def test_static_matches_context_twice(name):
    if name == "c1":
        w = I.config_c1()
    elif name == "c3":
        w = I.config_c3()
    else:
        full = I.config_c2()
        keep = (full.x[:, 0] < 25.0) & (full.x[:, 1] < 25.0)
        w = I.Workload("slab_piece", full.x[keep], I.Box(lo=full.box.lo, hi=full.box.hi,
                       periodic=np.array([False, False, False])), full.mass[keep], full.fixed[keep])
    cfg = ap.make_config(I.eam_params(0), I.ace_params(0), I.SINGLE_EVAL, precision=ap.PREC_FP64)
    lam_np = np.random.Generator(np.random.PCG64(31)).uniform(0.0, 1.0, w.n)
    lam = torch.as_tensor(lam_np, device="cuda")
    e_ref, f_ref = reference(w, cfg, lam)
    e_o, f_o, _, _ = O.eam(w.x, w.box, I.eam_params(0), weights=lam_np)
    for _ in range(2):
        e, f = static_call(w, cfg, lam)
        for er, fr in ((e_ref, f_ref), (e_o, f_o)):
            d = np.linalg.norm(f - fr, axis=1)
            assert np.all(d <= 1e-5 * (np.linalg.norm(fr, axis=1) + 0.01)), d.max()
            assert np.abs(e - er).max() < 1e-10


def test_static_without_lambda_weighs_every_atom_by_one():
    w = I.config_c3()
    cfg = ap.make_config(I.eam_params(0), I.ace_params(0), I.SINGLE_EVAL, precision=ap.PREC_FP64)
    e_ref, f_ref = reference(w, cfg, torch.ones(w.n, dtype=torch.float64, device="cuda"))
    e_o, f_o, _, _ = O.eam(w.x, w.box, I.eam_params(0))
    for _ in range(2):
        e, f = static_call(w, cfg, None)
        for er, fr in ((e_ref, f_ref), (e_o, f_o)):
            d = np.linalg.norm(f - fr, axis=1)
            assert np.all(d <= 1e-5 * (np.linalg.norm(fr, axis=1) + 0.01)), d.max()
            assert np.abs(e - er).max() < 1e-10


def test_static_small_periodic_cell_counts_own_images():
    """2x2x2 FCC cells (32 atoms), L = 7.23 A < 2 r_c = 11 A: every atom sees images of
    itself and several images of each other atom inside the cutoff."""
    g = np.random.Generator(np.random.PCG64(I.seed_for(0, 41)))
    x = I.fcc_lattice(2, 2, 2) + 0.05 * g.standard_normal((32, 3))
    box = I.Box(lo=np.zeros(3), hi=np.full(3, 2 * I.A_CU), periodic=np.array([True, True, True]))
    w = I.Workload("fcc2", x, box, np.full(32, I.MASS_CU), np.zeros(32, np.uint8))
    lam_np = g.uniform(0.0, 1.0, 32)
    cfg = ap.make_config(I.eam_params(0), I.ace_params(0), I.SINGLE_EVAL, precision=ap.PREC_FP64)
    e_o, f_o, _, _ = O.eam(x, box, I.eam_params(0), weights=lam_np)
    for _ in range(2):
        e, f = static_call(w, cfg, torch.as_tensor(lam_np, device="cuda"))
        d = np.linalg.norm(f - f_o, axis=1)
        assert np.all(d <= 1e-5 * (np.linalg.norm(f_o, axis=1) + 0.01)), d.max()
        assert np.abs(e - e_o).max() < 1e-10


def test_static_rejects_too_many_atoms():
    lib = N.lib()
    cfg = ap.make_config(I.eam_params(0), I.ace_params(0), I.SINGLE_EVAL, precision=ap.PREC_FP64)
    box = ap.make_box([0, 0, 0], [10, 10, 10], [1, 1, 1])
    dummy = torch.zeros(3, dtype=torch.float64, device="cuda")
    st = lib.ap_eval_eam_static(ctypes.byref(cfg), 32769, _p(dummy), ctypes.byref(box), None, _p(dummy), _p(dummy),
                                None)
    assert st == 1
