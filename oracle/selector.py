"""Learned detection score (the selector): oracle.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may import this module; it shares no code with the
CUDA library.

The paper leaves the detection mechanism open: the argument of f_cut in
Eq. lambda_1_i may come from any detector, provided it is 0 for atoms to be
treated precisely and 1 for atoms to be treated fast (Appendix B, the remark after
the definition of f_cut).  The project's learned detector is defined here; the
centro-symmetry parameter stays in the loop as one feature and as the reference
detector the selector is evaluated against.

Score.  p_i = sigmoid(MLP(standardised features_i)); it is pushed into the same
history as the CSP samples would be, averaged over the same window (Eq. csp_2_i
with p in place of CSP), and mapped to the f_cut argument
(p_hi - p_avg)/(p_hi - p_lo): p_avg >= p_hi gives lambda_0 = 0, p_avg <= p_lo
gives lambda_0 = 1.

Features (24 per atom; N_i = every image (j, s) with r_ij < R_FEAT = 5.5 A, the
EAM cutoff; shells S1 = {r < 3.09}, S2 = {3.09 <= r < 4.02}, S3 = {4.02 <= r <
4.77} A, the midpoints between the first four FCC shells at a = 3.615 A):
   0 rho_i = sum_N zeta(r)          1 xi(rho_i)            2 xi'(rho_i)
   3 1/2 sum_N Phi(r)               4 |S1|  5 |S2|  6 |S3|
   7 min(CSP_i, 100)  (centro-symmetry, N = 12, as the classification computes it)
   8 second-shell centro-symmetry: sum_{j in S2} min(r_ij^2, min_{k in S2, k != j} |r_ij + r_ik|^2)
   9 |sum_S1 r_ij|   10 |sum_S2 r_ij|   11 |sum_N r_ij|
  12 |sum_N zeta'(r_ij) r_ij / r_ij|
  13 rho_i - mean_{j in S1} rho_j
  14-17 mean, standard deviation, min, max of r_ij over S1
  18-21 mean, standard deviation, third and fourth central moments of r_ij over N
  22 |N|
  23 mean_{j in N} xi'_j - xi'_i
Empty sets give 0 for every statistic over them.  Standard deviations and
central moments are population moments about the mean (two passes).

Network (the kernel's precision points, which decide the lambda_0 = 1 set, so the
oracle takes them too): x~ = bf16(fp32(fp32(x - mu) * inv_sigma));
h1 = bf16(relu(x~ W1 + b1)); h2 = relu(h1 W2 + b2); z = h2 . w3 + b3 with W1, W2,
w3 rounded to bf16 and the biases kept in FP32; the sums themselves run in FP64
here (FP32 on the tensor cores).  Training minimises the weighted binary
cross-entropy sum_b w_b BCE(z_b, y_b) / sum_b w_b with Adam (FP32 master
weights, bf16 copies for the forward pass); the gradient passes straight through
the bf16 roundings.
"""
from __future__ import annotations

import numpy as np

from . import csp as _csp, eam as _eam, eam_pair as _eam_pair, neighbors as _neighbors

R_FEAT = 5.5
SHELL_CUTS = (3.09, 4.02, 4.77)
CSP_CAP = 100.0
N_FEAT = 24
N_HID = 64
# flat parameter layout: W1 [24][64] (input-major), b1 [64], W2 [64][64], b2 [64], w3 [64], b3 [1]
SIZES = (("W1", (N_FEAT, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("w3", (N_HID,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


# ----------------------------------------------------------------------------- features
def features(x, box, eam_p, csp_search: float = 6.5, nl=None, ids=None) -> np.ndarray:
    """The 24 features, FP64, from their definitions (module docstring), of the
    atoms ids (default: every atom), in that order."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    if nl is None:
        nl = _neighbors(x, box, R_FEAT)
    _, _, rho, dxi = _eam(x, box, eam_p, nl=nl)
    cspv = _csp(x, box, csp_search)
    L = np.asarray(box.hi, float) - np.asarray(box.lo, float)
    c1, c2, c3 = SHELL_CUTS
    ids = np.arange(n) if ids is None else np.asarray(ids)
    out = np.zeros((ids.shape[0], N_FEAT))
    for row, i in enumerate(ids):
        m = int(nl.cnt[i])
        js = nl.j[i, :m]
        d = x[js] + nl.s[i, :m] * L - x[i]
        r = np.sqrt((d * d).sum(1))
        keep = r < R_FEAT
        js, d, r = js[keep], d[keep], r[keep]
        z, dz, ph, _ = _eam_pair(eam_p, r)
        s1, s2, s3 = r < c1, (r >= c1) & (r < c2), (r >= c2) & (r < c3)
        xi = -eam_p.A * np.sqrt(rho[i]) if rho[i] > 0 else 0.0
        f = out[row]
        f[0] = rho[i]
        f[1] = xi
        f[2] = dxi[i]
        f[3] = 0.5 * ph.sum()
        f[4], f[5], f[6] = s1.sum(), s2.sum(), s3.sum()
        f[7] = min(cspv[i], CSP_CAP)
        d2 = d[s2]
        acc = 0.0
        for a in range(d2.shape[0]):
            best = float(d2[a] @ d2[a])
            for b in range(d2.shape[0]):
                if b != a:
                    v = d2[a] + d2[b]
                    best = min(best, float(v @ v))
            acc += best
        f[8] = acc
        f[9] = np.linalg.norm(d[s1].sum(0))
        f[10] = np.linalg.norm(d[s2].sum(0))
        f[11] = np.linalg.norm(d.sum(0))
        f[12] = np.linalg.norm(((dz / r)[:, None] * d).sum(0)) if r.size else 0.0
        if s1.any():
            f[13] = rho[i] - rho[js[s1]].mean()
            r1 = r[s1]
            f[14] = r1.mean()
            f[15] = np.sqrt(((r1 - r1.mean()) ** 2).mean())
            f[16] = r1.min()
            f[17] = r1.max()
        if r.size:
            mu = r.mean()
            f[18] = mu
            f[19] = np.sqrt(((r - mu) ** 2).mean())
            f[20] = ((r - mu) ** 3).mean()
            f[21] = ((r - mu) ** 4).mean()
            f[23] = dxi[js].mean() - dxi[i]
        f[22] = r.size
    return out


# ----------------------------------------------------------------------------- precision points
def bf16(a) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even), returned as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def unpack(theta) -> dict:
    theta = np.asarray(theta)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def standardise(feat, mu, inv_sigma) -> np.ndarray:
    """x~ = bf16(fp32(fp32(x - mu) * inv_sigma)), every step in FP32."""
    f = np.asarray(feat, np.float32)
    return bf16((f - np.asarray(mu, np.float32)) * np.asarray(inv_sigma, np.float32))


def forward(theta, xt, rounding: bool = True) -> dict:
    """MLP on standardised inputs xt [B, 24] (already bf16-valued when rounding).
    FP64 sums; rounding=False gives the plain FP64 network (used to pin the gradient)."""
    P = unpack(np.asarray(theta, np.float64))
    rnd = (lambda a: bf16(a).astype(np.float64)) if rounding else (lambda a: a)
    W1, W2, w3 = rnd(P["W1"]), rnd(P["W2"]), rnd(P["w3"])
    xt = np.asarray(xt, np.float64)
    z1 = xt @ W1 + P["b1"]
    h1 = np.maximum(z1, 0.0)
    if rounding:
        h1 = bf16(h1.astype(np.float32)).astype(np.float64)
    z2 = h1 @ W2 + P["b2"]
    h2 = np.maximum(z2, 0.0)
    z = h2 @ w3 + P["b3"][0]
    return dict(xt=xt, z1=z1, h1=h1, z2=z2, h2=h2, z=z, W1=W1, W2=W2, w3=w3)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-np.asarray(z, np.float64)))


def loss(z, y, w) -> float:
    """Weighted mean binary cross-entropy on logits: sum w [softplus(z) - y z] / sum w."""
    z = np.asarray(z, np.float64)
    sp = np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))
    return float((w * (sp - y * z)).sum() / w.sum())


def backward(fw: dict, y, w) -> np.ndarray:
    """Gradient of loss(z, y, w) w.r.t. the flat parameters (straight through the
    bf16 roundings of the weights and of h1)."""
    gz = w * (sigmoid(fw["z"]) - y) / w.sum()                  # dL/dz [B]
    dw3 = fw["h2"].T @ gz
    db3 = np.array([gz.sum()])
    dz2 = np.outer(gz, fw["w3"]) * (fw["z2"] > 0)
    dW2 = fw["h1"].T @ dz2
    db2 = dz2.sum(0)
    dz1 = (dz2 @ fw["W2"].T) * (fw["z1"] > 0)
    dW1 = fw["xt"].T @ dz1
    db1 = dz1.sum(0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, db3])


class Adam:
    """Adam (Kingma and Ba 2015) with bias correction; eps outside the square root."""

    def __init__(self, n: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, theta, g) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)


def init_params(seed_rng: np.random.Generator) -> np.ndarray:
    """He-normal weights, zero biases (the trainer's starting point)."""
    parts = []
    for name, shape in SIZES:
        if name.startswith("b"):
            parts.append(np.zeros(int(np.prod(shape))))
        else:
            fan_in = shape[0]
            parts.append(seed_rng.standard_normal(int(np.prod(shape))) * np.sqrt(2.0 / fan_in))
    return np.concatenate(parts)


def score(theta, feat, mu, inv_sigma) -> np.ndarray:
    """p_i = sigmoid(z_i) for raw features [N, 24]."""
    return sigmoid(forward(theta, standardise(feat, mu, inv_sigma))["z"])
