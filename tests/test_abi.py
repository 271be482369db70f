"""Host-side checks of the C ABI (no GPU needed): the header is plain C, the
library builds for sm_103a, loads, and exports every entry point the header
declares; the ctypes binding covers the same set."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")
HEADERS = sorted(os.path.join(INCLUDE, h) for h in os.listdir(INCLUDE) if h.endswith(".h"))


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:rf_status|void|int|const char\s*\*)\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                            src, re.M)
    return sorted(set(names))


@pytest.mark.parametrize("header", HEADERS)
def test_header_is_plain_c(header):
    # no CUDA, torch or C++ types in the signatures: a C compiler accepts it alone
    subprocess.check_call(["gcc", "-fsyntax-only", "-std=c99", "-Wall", "-Werror", "-I", INCLUDE, "-x", "c", header])


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("pst_create", "tsdf_integrate", "fitness_eval", "pfo_track_frame", "rf_mlp_train_step",
                 "rf_learned_step"):
        assert must in names


@pytest.fixture(scope="module")
def built_lib():
    from paper_2105_05600_gb300 import build

    return build.build()


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(built_lib):
    from paper_2105_05600_gb300 import _native

    assert sorted(_native.EXPORTS) == declared_functions()
    assert _native.rf_version().startswith("librosefusion")


def test_structs_match_the_header(built_lib):
    # the ctypes mirrors must have the C sizes (checked by compiling a probe against the header)
    from paper_2105_05600_gb300 import _native

    probe = r"""
#include <stdio.h>
#include "rf_proposal.h"
int main(void) { printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(rf_intrinsics), sizeof(rf_pose),
                        sizeof(rf_params), sizeof(rf_iter_stats), sizeof(rf_frame_stats), sizeof(rf_track_options),
                        sizeof(rf_proposal_params), sizeof(rf_learned_stats)); return 0; }
"""
    import tempfile

    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(probe)
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(x) for x in subprocess.check_output([exe]).split()]
    mine = [ctypes.sizeof(t) for t in (_native.rf_intrinsics, _native.rf_pose, _native.rf_params,
                                       _native.rf_iter_stats, _native.rf_frame_stats, _native.rf_track_options,
                                       _native.rf_proposal_params, _native.rf_learned_stats)]
    assert sizes == mine


def test_argument_errors_need_no_gpu(built_lib):
    # argument validation happens before any CUDA call and never throws
    from paper_2105_05600_gb300 import _native as n

    assert n.lib.pst_create(0, 1, 0, None, None) == n.RF_ERR_ARG
    assert "n must be >= 1" in n.lib.rf_last_error().decode() or "null" in n.lib.rf_last_error().decode()
    h = ctypes.c_void_p()
    org = (ctypes.c_float * 3)(0, 0, 0)
    assert n.lib.rf_volume_create(12, 16, 16, 0.01, 0.03, org, 0, ctypes.byref(h)) == n.RF_ERR_ARG
    assert n.lib.fitness_eval(None, None, 0, None, 0, None, None, None, None, None, None, None) == n.RF_ERR_ARG
    assert n.lib.rf_tracker_create(None, None, 0, None, 0, 0, ctypes.byref(h)) == n.RF_ERR_ARG


def test_proposal_argument_errors_need_no_gpu(built_lib):
    from paper_2105_05600_gb300 import _native as n

    h = ctypes.c_void_p()
    assert n.lib.rf_mlp_num_params() == 348944
    assert n.lib.rf_mlp_create(0, ctypes.byref(h)) == n.RF_ERR_ARG
    assert n.lib.rf_mlp_create(n.RF_MLP_MAX_BATCH + 1, ctypes.byref(h)) == n.RF_ERR_ARG
    assert n.lib.rf_mlp_forward(None, None, 1, None, None) == n.RF_ERR_ARG
    assert n.lib.rf_mlp_train_step(None, None, None, None, 8, 8, 1e-3, None, None) == n.RF_ERR_ARG
    p = n.proposal_params()
    assert (p.k_learned, p.k_fallback, p.resume, p.stuck) == (5, 20, 1, 1)
    assert abs(p.kappa - 0.25) < 1e-7 and abs(p.theta - 0.95) < 1e-7
    bad_stuck = n.proposal_params(stuck=3)
    assert n.lib.rf_learned_create(None, None, None, ctypes.byref(bad_stuck), 8, 8, ctypes.byref(h)) == n.RF_ERR_ARG
    assert n.lib.rf_proposal_apply(None, None, None, ctypes.byref(p), None, None, None) == n.RF_ERR_ARG
    bad = n.proposal_params(k_learned=0)
    assert n.lib.rf_learned_create(None, None, None, ctypes.byref(bad), 8, 8, ctypes.byref(h)) == n.RF_ERR_ARG
    o = n.rf_track_options(None, None, None, n.RF_MAX_ITERS + 1, 0)
    assert n.lib.pfo_track_frame_ex_async(None, None, None, None, None, None, None, ctypes.byref(o),
                                          None) == n.RF_ERR_ARG


def test_binding_constants_match_the_header(built_lib):
    # flag bits, error codes and size limits of the binding equal the header's #defines
    from paper_2105_05600_gb300 import _native as n

    src = open(os.path.join(INCLUDE, "rosefusion.h")).read()
    defs = dict(re.findall(r"^#define\s+(RF_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src, re.M))
    assert "RF_CELL_MARGIN" in defs
    checked = 0
    for name, val in defs.items():
        if hasattr(n, name):
            assert getattr(n, name) == int(val), name
            checked += 1
    assert checked >= 12
    combo = re.search(r"#define RF_DEFAULT_FLAGS \(([^)]*)\)", src).group(1)
    assert n.RF_DEFAULT_FLAGS == sum(int(defs[t.strip()]) for t in combo.split("|"))
