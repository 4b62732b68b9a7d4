"""Selector training and the stored model, end to end on the GPU.

* The stored model (paper_2411_03002_gb300/selector_cu.npz, trained by
  ``python -m paper_2411_03002_gb300.selector``) separates atoms whose ACE and EAM
  forces differ by more than 25 meV/A from the rest on a 32,000-atom slab that
  neither its training nor its stored evaluation used (variant 4).
* A short training run on a subset of the training structures lowers the loss
  and separates the classes on a held-out slab.
* Training is bitwise reproducible: the gradient reduction has a fixed order.
"""
import os

import numpy as np
import pytest
import torch

import ap_inputs as I

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2411_03002_gb300 as ap
    from paper_2411_03002_gb300 import selector as T

MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2411_03002_gb300",
                     "selector_cu.npz")


def predict(params, mu, inv, feat):
    ctx = ap.Context(ap.make_config(I.eam_params(0), I.ace_params(0), I.HYB1))
    ctx.sel_set_model(params, mu, inv)
    p, _ = ctx.sel_predict(feat)
    out = p.cpu().numpy()
    ctx.close()
    return out


def test_stored_model_on_an_unseen_slab():
    d = np.load(MODEL)
    w = I.config_c2(variant=4)
    feat, y, _ = T.label_structure(w.x, w.box)
    p = predict(d["params"], d["mu"], d["inv_sigma"], feat)
    assert 0.1 < y.mean() < 0.3
    assert T.roc_auc(p, y) > 0.98
    hit = (p > float(d["p_lo"])) & (y > 0.5)
    assert hit.sum() / y.sum() > 0.9 and hit.sum() / (p > float(d["p_lo"])).sum() > 0.9


@pytest.fixture(scope="module")
def small_set():
    return T.build_dataset(ks=(0, 5, 40, 45, 80, 81, 82, 120, 125, 160, 161), md_steps=200)


def test_short_training_separates_classes(small_set):
    feat, y, _, _ = small_set
    params, mu, inv, hist, _ = T.train(feat, y, epochs=12, batch=2048, seed=3)
    assert hist[-1] < 0.8 * hist[0], hist
    w = I.config_c2(variant=5)
    f2, y2, _ = T.label_structure(w.x, w.box)
    assert T.roc_auc(predict(params, mu, inv, f2), y2) > 0.95


def test_training_is_bitwise_reproducible(small_set):
    feat, y, _, _ = small_set
    a = T.train(feat, y, epochs=2, batch=2048, seed=5)
    b = T.train(feat, y, epochs=2, batch=2048, seed=5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[3], b[3])
