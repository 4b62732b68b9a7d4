"""Host-side pieces of the selector training (no GPU): the ROC-AUC used in its
evaluation, the parameter layout, the learning-rate schedule, and the seeded
structure generators of the training set."""
import numpy as np
import pytest

import ap_inputs as I
import oracle as O
from paper_2411_03002_gb300 import selector as T
from paper_2411_03002_gb300 import SEL_NPARAMS


def test_roc_auc_matches_pairwise_definition():
    g = np.random.Generator(np.random.PCG64(1))
    y = (g.random(400) < 0.3).astype(float)
    s = np.round(g.random(400) + 0.5 * y, 2)              # ties included
    pos, neg = s[y > 0.5], s[y < 0.5]
    brute = ((pos[:, None] > neg[None, :]).sum() + 0.5 * (pos[:, None] == neg[None, :]).sum()) / (len(pos) * len(neg))
    assert T.roc_auc(s, y) == pytest.approx(brute, rel=1e-12)


def test_roc_auc_matches_sklearn():
    metrics = pytest.importorskip("sklearn.metrics")
    g = np.random.Generator(np.random.PCG64(2))
    y = (g.random(2000) < 0.2).astype(float)
    s = g.random(2000) + 0.3 * y
    assert T.roc_auc(s, y) == pytest.approx(metrics.roc_auc_score(y, s), rel=1e-12)


def test_init_params_layout_and_schedule():
    p = T.init_params(3)
    assert p.shape == (SEL_NPARAMS,) and p.dtype == np.float32
    assert np.all(p[1536:1600] == 0) and np.all(p[5696:5760] == 0) and p[-1] == 0     # biases
    assert abs(p[:1536].std() - np.sqrt(2 / 24)) < 0.02
    assert [T.lr_at(e, 40) for e in (0, 23, 24, 33, 34, 39)] == [3e-3, 3e-3, 1e-3, 1e-3, 3e-4, 3e-4]


@pytest.mark.parametrize("surface", [100, 110, 111])
def test_oriented_fcc_has_fcc_shells(surface):
    dims = {100: (3, 3, 3), 110: (4, 5, 5), 111: (5, 3, 2)}[surface]
    x, L = I.fcc_oriented(surface, *dims)
    box = I.Box(lo=np.zeros(3), hi=L, periodic=np.array([True] * 3))
    n1 = O.neighbors(x, box, 3.0).cnt
    n2 = O.neighbors(x, box, 3.7).cnt
    assert np.all(n1 == 12) and np.all(n2 - n1 == 6)
    # the z axis is the surface normal: one (hkl) layer spacing a/2, a/(2 sqrt 2), a/sqrt 3
    dz = np.diff(np.unique(np.round(x[:, 2], 6)))
    assert np.allclose(dz, {100: 0.5, 110: 0.5 / np.sqrt(2), 111: 1 / np.sqrt(3)}[surface] * I.A_CU)


def test_selector_structures_are_seeded_and_categorised():
    a, b = I.config_c4(17), I.config_c4(17)
    assert np.array_equal(a.x, b.x)
    n = [I.config_c4(k).n for k in (0, 40, 80, 81, 82, 120, 160, 161)]
    assert all(4500 <= m <= 5100 for m in n)
    assert I.config_c4(40).n < I.config_c4(0).n                 # vacancies removed
    assert I.config_c4(160).v is not None and I.config_c4(0).v is None
    with pytest.raises(ValueError):
        I.config_c4(200)
