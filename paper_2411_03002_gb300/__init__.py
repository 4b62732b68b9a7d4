"""GB300-native adaptive-precision EAM/ACE force evaluation (arXiv 2411.03002).

The computation lives in libap.so (hand-written CUDA for sm_103a, C-ABI in
include/ap.h).  This package is its Python binding.
"""
from .api import (Context, StepStats, ace_basis_desc, ace_gaunt, ace_nbasis, ap_blend_forces, ap_build_neighbors,
                  ap_classify, ap_create, ap_eval_ace, ap_eval_eam, ap_sel_features, ap_sel_get_grad,
                  ap_sel_get_model, ap_sel_predict, ap_sel_set_model, ap_sel_train_step, ap_step, make_box,
                  make_config, probe_peak, PEAK_FFMA, PEAK_TF32_MMA)
from ._native import (ApConfig, ApError, DETECT_CSP, DETECT_SELECTOR, EAM_ANALYTIC, EAM_MISHIN, PREC_FP64,
                      PREC_MIXED, REBUILD_SKIN, SEL_NFEAT, SEL_NPARAMS)
from . import autograd

__all__ = ["Context", "StepStats", "ApConfig", "ApError", "PREC_FP64", "PREC_MIXED", "DETECT_CSP",
           "DETECT_SELECTOR", "EAM_ANALYTIC", "EAM_MISHIN", "SEL_NFEAT", "SEL_NPARAMS", "make_box", "make_config", "ace_nbasis",
           "ace_basis_desc", "ace_gaunt", "ap_create", "ap_build_neighbors", "ap_classify", "ap_eval_eam",
           "ap_eval_ace", "ap_blend_forces", "ap_step", "ap_sel_set_model", "ap_sel_get_model", "ap_sel_features",
           "ap_sel_predict", "ap_sel_train_step", "ap_sel_get_grad", "autograd", "probe_peak", "PEAK_FFMA",
           "PEAK_TF32_MMA", "REBUILD_SKIN"]
