"""Pins of the selector oracle (oracle/selector.py) against facts that do not
come from the oracle itself: lattice geometry, library routines (torch's bf16
conversion, BCE with logits and Adam), finite differences and invariances."""
import numpy as np
import pytest
import torch

import ap_inputs as I
import oracle as O
import oracle.selector as S

A = I.A_CU


def periodic_box(n, a=A):
    return I.Box(lo=np.zeros(3), hi=np.full(3, n * a), periodic=np.array([True] * 3))


# ----------------------------------------------------------------------------- precision points
def test_bf16_matches_torch_round_to_nearest_even():
    g = np.random.Generator(np.random.PCG64(1))
    x = np.concatenate([g.standard_normal(20000).astype(np.float32) * 10.0 ** g.integers(-6, 6, 20000),
                        np.float32([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 0.0, -0.0, 65504.0])])
    ours = S.bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))
    assert S.bf16(np.float32([1.0 + 2 ** -8]))[0] == 1.0            # tie to even
    assert S.bf16(np.float32([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6


def test_standardise_is_fp32_then_bf16():
    g = np.random.Generator(np.random.PCG64(2))
    f = g.standard_normal((500, 24)) * 3 + 1
    mu = g.standard_normal(24).astype(np.float32)
    inv = (1.0 / (0.5 + g.random(24))).astype(np.float32)
    t = (torch.from_numpy(f.astype(np.float32)) - torch.from_numpy(mu)) * torch.from_numpy(inv)
    ref = t.to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(S.standardise(f, mu, inv), ref)


# ----------------------------------------------------------------------------- features
def fcc_features():
    x = I.fcc_lattice(4, 4, 4)
    return S.features(x, periodic_box(4), I.EAM_NOMINAL)


def test_perfect_fcc_features_follow_the_shell_structure():
    f = fcc_features()
    assert np.allclose(f, f[0], atol=1e-12)                       # every site equivalent
    f = f[0]
    # FCC shells: 12 at a/sqrt2, 6 at a, 24 at a sqrt(3/2), 12 at a sqrt2 (all < 5.5 A)
    shells = np.array([A / np.sqrt(2), A, A * np.sqrt(1.5), A * np.sqrt(2)])
    mult = np.array([12, 6, 24, 12])
    assert (f[4], f[5], f[6], f[22]) == (12, 6, 24, 54)
    assert abs(f[7]) < 1e-20 and abs(f[8]) < 1e-20                # CSP and second-shell CSP
    assert np.all(np.abs(f[[9, 10, 11, 12, 13, 23]]) < 1e-12)     # vector sums, neighbour contrasts
    assert np.allclose(f[[14, 16, 17]], A / np.sqrt(2), rtol=1e-14) and abs(f[15]) < 1e-12
    r = np.repeat(shells, mult)
    mu = r.mean()
    assert np.isclose(f[18], mu, rtol=1e-14)
    assert np.isclose(f[19], np.sqrt(((r - mu) ** 2).mean()), rtol=1e-12)
    assert np.isclose(f[20], ((r - mu) ** 3).mean(), rtol=1e-11)
    assert np.isclose(f[21], ((r - mu) ** 4).mean(), rtol=1e-12)
    z, _, ph, _ = O.eam_pair(I.EAM_NOMINAL, shells)
    rho = (mult * z).sum()
    assert np.isclose(f[0], rho, rtol=1e-13)
    assert np.isclose(f[1], -I.EAM_NOMINAL.A * np.sqrt(rho), rtol=1e-13)
    assert np.isclose(f[2], -0.5 * I.EAM_NOMINAL.A / np.sqrt(rho), rtol=1e-13)
    assert np.isclose(f[3], 0.5 * (mult * ph).sum(), rtol=1e-13)


def test_unrelaxed_100_surface_atom():
    x = I.fcc_lattice(4, 4, 4)
    box = I.Box(lo=np.array([0.0, 0.0, -10.0]), hi=np.array([4 * A, 4 * A, 4 * A + 10.0]),
                periodic=np.array([True, True, False]))
    f = S.features(x, box, I.EAM_NOMINAL)
    top = np.nonzero(np.isclose(x[:, 2], x[:, 2].max()))[0]
    ft = f[top]
    assert np.all(ft[:, 4] == 8) and np.all(ft[:, 5] == 5)
    # first shell: 4 in-plane neighbours cancel, the 4 below sum to (0, 0, -2a)
    assert np.allclose(ft[:, 9], 2 * A, rtol=1e-12)
    # second shell: +-a x, +-a y cancel pairwise, -a z has no partner -> its own r^2 = a^2
    assert np.allclose(ft[:, 10], A, rtol=1e-12)
    assert np.allclose(ft[:, 8], A * A, rtol=1e-12)
    # CSP: 8 nearest plus 4 of the 5 equidistant second-shell atoms -> a^2 or 3a^2/2
    assert set(np.unique(np.round(ft[:, 7] / (A * A), 12))) <= {1.0, 1.5}


def test_vacancy_neighbour():
    x = np.delete(I.fcc_lattice(4, 4, 4), 0, axis=0)
    f = S.features(x, periodic_box(4), I.EAM_NOMINAL)
    L = 4 * A
    r = np.linalg.norm((x + L / 2) % L - L / 2, axis=1)
    nn = np.nonzero(np.isclose(r, A / np.sqrt(2)))[0]
    assert len(nn) == 12
    assert np.all(f[nn, 4] == 11)
    assert np.allclose(f[nn, 9], A / np.sqrt(2), rtol=1e-12)      # the missing bond vector
    assert np.allclose(f[nn, 7], A * A / 2, rtol=1e-12)           # CSP = a^2/2 next to a vacancy


def test_features_are_rotation_invariant():
    g = np.random.Generator(np.random.PCG64(3))
    x = I.fcc_lattice(3, 3, 3) + 0.15 * g.standard_normal((108, 3))
    box = I.Box(lo=x.min(0) - 10, hi=x.max(0) + 10, periodic=np.array([False] * 3))
    q, _ = np.linalg.qr(g.standard_normal((3, 3)))
    xr = x @ q.T
    boxr = I.Box(lo=xr.min(0) - 10, hi=xr.max(0) + 10, periodic=np.array([False] * 3))
    f0 = S.features(x, box, I.EAM_NOMINAL)
    f1 = S.features(xr, boxr, I.EAM_NOMINAL)
    assert np.allclose(f0, f1, rtol=1e-9, atol=1e-9)


# ----------------------------------------------------------------------------- network
def small_problem(seed=4, b=40):
    g = np.random.Generator(np.random.PCG64(seed))
    theta = S.init_params(g)
    theta[S.N_PARAMS - 1] = 0.3
    xt = g.standard_normal((b, S.N_FEAT))
    y = (g.random(b) < 0.3).astype(float)
    w = g.random(b) + 0.5
    return theta, xt, y, w / w.sum()


def test_loss_matches_torch_bce_with_logits():
    theta, xt, y, w = small_problem()
    z = S.forward(theta, xt, rounding=False)["z"]
    ref = torch.nn.functional.binary_cross_entropy_with_logits(torch.from_numpy(z), torch.from_numpy(y),
                                                               weight=torch.from_numpy(w), reduction="sum")
    assert np.isclose(S.loss(z, y, w), float(ref), rtol=1e-13)


def test_forward_matches_a_torch_mlp_without_rounding():
    theta, xt, _, _ = small_problem()
    P = S.unpack(theta)
    t = lambda a: torch.from_numpy(np.asarray(a, np.float64))
    h1 = torch.relu(t(xt) @ t(P["W1"]) + t(P["b1"]))
    h2 = torch.relu(h1 @ t(P["W2"]) + t(P["b2"]))
    z = h2 @ t(P["w3"]) + t(P["b3"])
    assert np.allclose(S.forward(theta, xt, rounding=False)["z"], z.numpy(), rtol=1e-13, atol=1e-13)


def test_gradient_matches_central_differences():
    theta, xt, y, w = small_problem()
    g = S.backward(S.forward(theta, xt, rounding=False), y, w)
    rng = np.random.Generator(np.random.PCG64(5))
    picks = np.concatenate([rng.choice(S.N_PARAMS, 60, replace=False), [S.N_PARAMS - 1, 1536, 5696, 5760]])
    h = 1e-6
    for p in picks:
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd = (S.loss(S.forward(tp, xt, False)["z"], y, w) - S.loss(S.forward(tm, xt, False)["z"], y, w)) / (2 * h)
        assert abs(fd - g[p]) <= 1e-7 + 1e-5 * abs(fd), (p, fd, g[p])


def test_gradient_matches_torch_autograd():
    theta, xt, y, w = small_problem(6)
    g = S.backward(S.forward(theta, xt, rounding=False), y, w)
    th = torch.tensor(theta, requires_grad=True)
    P = {}
    o = 0
    for name, shape in S.SIZES:
        k = int(np.prod(shape))
        P[name] = th[o:o + k].reshape(shape)
        o += k
    h1 = torch.relu(torch.from_numpy(xt) @ P["W1"] + P["b1"])
    h2 = torch.relu(h1 @ P["W2"] + P["b2"])
    z = h2 @ P["w3"] + P["b3"]
    loss = torch.nn.functional.binary_cross_entropy_with_logits(z, torch.from_numpy(y), weight=torch.from_numpy(w),
                                                                reduction="sum")
    loss.backward()
    assert np.allclose(g, th.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_adam_first_step_closed_form_and_torch():
    g = np.random.Generator(np.random.PCG64(7))
    theta = g.standard_normal(50)
    grads = [g.standard_normal(50) for _ in range(6)]
    opt = S.Adam(50, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
    t1 = opt.step(theta, grads[0])
    assert np.allclose(t1, theta - 1e-2 * grads[0] / (np.abs(grads[0]) + 1e-8), rtol=1e-12, atol=1e-15)
    tp = torch.tensor(theta, requires_grad=True)
    ref = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    ours = theta.copy()
    opt = S.Adam(50, lr=1e-2)
    for gr in grads:
        ours = opt.step(ours, gr)
        tp.grad = torch.tensor(gr)
        ref.step()
    assert np.allclose(ours, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------------------------- score -> lambda_0
def test_score_replaces_csp_in_lambda0():
    x = I.fcc_lattice(3, 3, 3)
    box = periodic_box(3)
    hyb = I.SINGLE_EVAL
    p = np.linspace(0.0, 1.0, x.shape[0])
    st = O.LambdaState(x.shape[0], 1, 1)
    lam, l0, *_ = O.classify(st, x, box, hyb, score=p, score_lo=0.3, score_hi=0.7)
    assert np.all(l0[p <= 0.3] == 1.0) and np.all(l0[p >= 0.7] == 0.0)
    mid = (p > 0.3) & (p < 0.7)
    assert np.all((l0[mid] > 0) & (l0[mid] < 1))
    assert np.all(np.diff(l0) <= 0)                               # larger score -> more precise
