"""C-ABI checks that need no GPU: symbols, struct layouts, host-side tables."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import ap_inputs as I
import oracle as O
from paper_2411_03002_gb300 import _native as N
from paper_2411_03002_gb300 import api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ap.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ap_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = N.lib()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    # the binding declares exactly the header's functions
    assert sorted(n for n, _, _ in N.SIGNATURES) == names


def test_struct_layouts_match_header(tmp_path):
    """sizeof of the three structs and offsetof of every ap_config and ap_step_stats
    field agree between the header and the ctypes binding."""
    fields = [("ap_config", N.ApConfig, f[0]) for f in N.ApConfig._fields_]
    fields += [("ap_step_stats", N.ApStepStats, f[0]) for f in N.ApStepStats._fields_]
    body = 'printf("%zu %zu %zu\\n", sizeof(ap_config), sizeof(ap_box), sizeof(ap_step_stats));'
    body += "".join(f'printf("%zu\\n", offsetof({t}, {k}));' for t, _, k in fields)
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ap.h"\nint main(){' + body + "return 0;}")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sz = list(map(int, out))
    assert sz[0] == ctypes.sizeof(N.ApConfig)
    assert sz[1] == ctypes.sizeof(N.ApBox)
    assert sz[2] == ctypes.sizeof(N.ApStepStats)
    for (t, cls, k), off in zip(fields, sz[3:]):
        assert getattr(cls, k).offset == off, (t, k)


def test_basis_enumeration_matches_oracle():
    desc_lib = api.ace_basis_desc()
    ace = O.ACE(I.ace_params(0))
    desc_or = ace.basis_desc()
    assert desc_lib.shape == desc_or.shape == (325, 7)
    # the oracle leaves unused slots of nu=1,2 entries at 0 except l for nu=2; compare used fields
    for v in range(325):
        nu = desc_or[v, 0]
        assert desc_lib[v, 0] == nu
        assert list(desc_lib[v, 1:1 + nu]) == list(desc_or[v, 1:1 + nu])
        if nu >= 2:
            assert list(desc_lib[v, 4:4 + nu]) == list(desc_or[v, 4:4 + nu])


def test_racah_gaunt_matches_quadrature():
    g_lib = api.ace_gaunt()
    g_or = O.ACE(I.ace_params(0)).gaunt()
    assert np.abs(g_lib - g_or).max() < 1e-13
    assert np.abs(g_or).max() > 0.1


def test_config_validation_rejects_bad_values():
    cfg = api.make_config(I.EAM_NOMINAL, I.ace_params(0), I.HybridParams(csp_lo=3.0, csp_hi=2.5))
    h = ctypes.c_void_p()
    assert N.lib().ap_create(ctypes.byref(cfg), ctypes.byref(h)) == 1   # AP_ERR_ARG before any device call
    assert N.lib().ap_create(None, ctypes.byref(h)) == 1
    # rebuild_every: a period >= 0 or the skin criterion (-1), nothing below
    cfg = api.make_config(I.EAM_NOMINAL, I.ace_params(0), I.HybridParams(), rebuild_every=-2)
    assert N.lib().ap_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    assert N.REBUILD_SKIN == -1


def test_null_context_calls_fail_cleanly():
    lib = N.lib()
    assert lib.ap_build_neighbors(None, 0, None, None, None, None) == 1
    assert lib.ap_classify(None, 0, None, None, 1, None, None, None, None) == 1
    assert lib.ap_step(None, 0, None, None, None, None, None, None, 0, None, None) == 1
    assert lib.ap_last_error(None) == b"null context"


def test_generated_nu3_code_matches_the_basis(tmp_path):
    """ace_nu3.inc (the straight-line nu = 3 code) is the generator's output for
    the basis enumeration compiled into the library."""
    csrc = os.path.join(ROOT, "paper_2411_03002_gb300", "csrc")
    exe = tmp_path / "gen_nu3"
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "include"), os.path.join(csrc, "gen_nu3.cpp"),
                    os.path.join(csrc, "ace_tables.cpp"), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    with open(os.path.join(csrc, "ace_nu3.inc")) as fh:
        assert fh.read() == out


def test_profile_phase_names_match_the_header():
    """Context.PHASES lists one name per AP_PHASE_* constant, in index order, and
    AP_NUM_PHASES entries in all (ap_profile_read fills that many)."""
    src = open(HEADER).read()
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (AP_PHASE_[A-Z_0-9]+) (\d+)", src)}
    num = int(re.search(r"#define AP_NUM_PHASES (\d+)", src).group(1))
    assert len(consts) == num == len(api.Context.PHASES)
    for name, idx in consts.items():
        assert api.Context.PHASES[idx] == name[len("AP_PHASE_"):].lower(), name
