"""ap_step with rebuild_every = AP_REBUILD_SKIN (needs a GPU).

The lists are checked after every drift and rebuilt when an atom has moved more than
skin/2 since the last build; a lambda update keeps them while no atom has moved more
than 0.45 skin, takes the CSP from the kept rows where they decide it and builds the new
ACE rows from the kept cells.  Every force and every lambda must be those of a run that
rebuilds at each update:

* thermal 32,000-atom slab (FCC sites, 300 K), FP64: the same trajectory and lambda as
  the default policy (rebuild at each lambda update) to roundoff, with fewer rebuilds
  and at least two kept updates; five steps after a kept update the forces of all
  atoms equal the oracle's at the GPU's positions and lambda (FP64 bar), so the ACE
  rows built from the kept cells are complete;
* the same in mixed precision against the oracle (1 meV/A, the bar of the other
  mixed-precision MD tests);
* the slab with the melting hemisphere (atoms move ~0.05 A/fs): rebuilds between
  lambda updates, no skin error, and the trajectory of a run that rebuilds every step;
* a lone atom 7.5 A above the surface (fewer than 12 atoms within reach): the kept rows
  cannot decide its CSP, so every update rebuilds (no update is kept) and the run
  equals the default one;
* the precise queue's ACE rows (ace_rc + skin) are checked against their own build: after
  an outside neighbour build they are rebuilt alone, and the forces stay the oracle's.
"""
import dataclasses

import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap


class Run:
    def __init__(self, w, prec, rebuild_every, skin=1.0, lambda_every=10):
        cfg = ap.make_config(I.eam_params(0), I.ace_for_config(2), w.hyb, precision=prec, dt=w.dt, skin=skin,
                             lambda_every=lambda_every, rebuild_every=rebuild_every)
        self.ctx = ap.Context(cfg)
        self.box = w.box
        self.x = torch.as_tensor(w.x, device="cuda").clone()
        self.v = torch.as_tensor(w.v, device="cuda").clone()
        self.f = torch.zeros_like(self.x)
        self.lam = torch.empty(w.n, dtype=torch.float64, device="cuda")
        self.m = torch.as_tensor(w.mass, device="cuda")
        self.ctx.build_neighbors(self.x, w.box)
        self.s0 = self.ctx.step(self.x, self.v, self.f, self.m, None, self.lam, 0)

    def step(self, k):
        return self.ctx.step(self.x, self.v, self.f, self.m, None, self.lam, k)


def thermal_slab():
    w0 = I.config_c2()
    return dataclasses.replace(w0, x=I.fcc_lattice(20, 20, 20))


def image_gap(xa, xb, box):
    d = xa - xb
    L = box.hi - box.lo
    for a in range(3):
        if box.periodic[a]:
            d[:, a] -= L[a] * np.round(d[:, a] / L[a])
    return np.linalg.norm(d, axis=1)


def wrapped(x, box):
    x = x.copy()
    L = box.hi - box.lo
    for a in range(3):
        if box.periodic[a]:
            x[:, a] = box.lo[a] + np.mod(x[:, a] - box.lo[a], L[a])
    return x


def oracle_forces(w, x, lam):
    _, fo, _, _ = O.hybrid(wrapped(x, w.box), w.box, lam, I.eam_params(0), O.ACE(I.ace_for_config(2)))
    return fo


def run_to_kept_update(a, b=None, min_kept=2, max_calls=12):
    """Calls of 10 steps until the last call ended on a kept update and at least
    min_kept updates were kept; returns the per-call (lambda, x) gaps to b."""
    gaps = []
    kept = 0
    for _ in range(max_calls):
        sa = a.step(10)
        k0, kept = kept, sa.kept
        if b is not None:
            sb = b.step(10)
            lam_gap = (a.lam - b.lam).abs().max().item()
            gaps.append((lam_gap, image_gap(a.x.cpu().numpy(), b.x.cpu().numpy(), b.box).max(),
                         sa.n_precise, sb.n_precise, sa, sb))
        if kept > k0 and kept >= min_kept:
            break
    return sa, gaps


def test_kept_updates_match_rebuilt_ones_fp64():
    w = thermal_slab()
    a = Run(w, ap.PREC_FP64, ap.REBUILD_SKIN)
    b = Run(w, ap.PREC_FP64, 0)
    sa, gaps = run_to_kept_update(a, b)
    for lam_gap, x_gap, npa, npb, _, _ in gaps:
        assert lam_gap < 1e-9 and x_gap < 1e-9 and npa == npb, (lam_gap, x_gap, npa, npb)
    sb = gaps[-1][5]
    print(f"thermal slab FP64: {len(gaps)} updates, kept {sa.kept}, rebuilds {sa.rebuilds} vs {sb.rebuilds}, "
          f"max disp {sa.max_disp:.3f} A, precise {sa.n_precise}")
    assert sa.kept >= 2 and sa.rebuilds < sb.rebuilds and sa.error_bits == 0
    # five steps on the ACE rows built from the kept cells
    sa = a.step(5)
    assert sa.error_bits == 0
    fo = oracle_forces(w, a.x.cpu().numpy(), a.lam.cpu().numpy())
    err = np.linalg.norm(a.f.cpu().numpy() - fo, axis=1)
    lim = 1e-5 * (np.linalg.norm(fo, axis=1) + 0.01)
    print(f"forces after a kept update vs oracle: max {err.max() * 1e3:.3g} meV/A")
    assert np.all(err <= lim), (err / lim).max()


def test_kept_updates_mixed_forces_match_oracle():
    w = thermal_slab()
    a = Run(w, ap.PREC_MIXED, ap.REBUILD_SKIN)
    sa, _ = run_to_kept_update(a)
    assert sa.kept >= 2 and sa.error_bits == 0
    sa = a.step(5)
    fo = oracle_forces(w, a.x.cpu().numpy(), a.lam.cpu().numpy())
    err = np.linalg.norm(a.f.cpu().numpy() - fo, axis=1)
    print(f"mixed: kept {sa.kept}, rebuilds {sa.rebuilds}, max |dF| {err.max() * 1e3:.3g} meV/A")
    assert err.max() <= 1e-3, err.max()


def test_rebuilds_between_updates_on_the_melting_slab():
    w = I.config_c2()
    a = Run(w, ap.PREC_FP64, ap.REBUILD_SKIN)
    b = Run(w, ap.PREC_FP64, 1)
    updates = 0
    for _ in range(4):
        sa = a.step(10)
        sb = b.step(10)
        updates += 1
        assert sa.error_bits == 0
        assert (a.lam - b.lam).abs().max().item() < 1e-8
        assert image_gap(a.x.cpu().numpy(), b.x.cpu().numpy(), w.box).max() < 1e-8
    print(f"melting slab: rebuilds {sa.rebuilds} (every step: {sb.rebuilds}), kept {sa.kept}")
    # more rebuilds than the initial build plus the updates that were not kept: some
    # happened between updates, when an atom passed skin/2
    assert sa.rebuilds > 1 + updates - sa.kept


def test_lone_atom_sends_every_update_to_a_rebuild():
    w0 = thermal_slab()
    lone = np.array([[w0.box.hi[0] / 2 + 0.3, w0.box.hi[1] / 2 + 0.2, w0.x[:, 2].max() + 7.5]])
    assert lone[0, 2] < w0.box.hi[2]
    w = dataclasses.replace(w0, x=np.concatenate([w0.x, lone]), v=np.concatenate([w0.v, np.zeros((1, 3))]),
                            mass=np.concatenate([w0.mass, w0.mass[:1]]),
                            fixed=np.concatenate([w0.fixed, np.zeros(1, np.uint8)]))
    a = Run(w, ap.PREC_FP64, ap.REBUILD_SKIN)
    b = Run(w, ap.PREC_FP64, 0)
    for _ in range(3):
        sa = a.step(10)
        sb = b.step(10)
        assert (a.lam - b.lam).abs().max().item() < 1e-9
        assert image_gap(a.x.cpu().numpy(), b.x.cpu().numpy(), w.box).max() < 1e-9
    assert sa.kept == 0 and sa.rebuilds == sb.rebuilds, (sa.kept, sa.rebuilds, sb.rebuilds)


def test_ace_rows_rebuilt_alone_after_an_outside_build():
    """ap_build_neighbors between ap_step calls builds new cells and EAM rows but not the
    precise queue's ACE rows: their displacement reference no longer applies, so the next
    step rebuilds them alone (from the new cells), and the forces stay the oracle's."""
    w = thermal_slab()
    a = Run(w, ap.PREC_FP64, ap.REBUILD_SKIN)
    sa = a.step(15)
    a.ctx.build_neighbors(a.x, w.box)
    sb = a.step(3)
    assert sb.ace_rebuilds >= sa.ace_rebuilds + 1 and sb.error_bits == 0, (sa.ace_rebuilds, sb.ace_rebuilds)
    fo = oracle_forces(w, a.x.cpu().numpy(), a.lam.cpu().numpy())
    err = np.linalg.norm(a.f.cpu().numpy() - fo, axis=1)
    lim = 1e-5 * (np.linalg.norm(fo, axis=1) + 0.01)
    print(f"ACE rows rebuilt alone: {sb.ace_rebuilds}, max |dF| {err.max() * 1e3:.3g} meV/A")
    assert np.all(err <= lim), (err / lim).max()
