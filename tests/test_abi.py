"""The C ABI library: builds, loads, exports every declared entry point, and
rejects invalid arguments on the host before touching the GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "safr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(safr_[a-z_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_19542_gb300 import safr
    return safr.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 10, names
    for n in names:
        assert hasattr(lib, n), f"libsafr.so does not export {n}"


def test_binding_names_match_the_abi():
    from paper_2510_19542_gb300 import safr
    for n in _declared_functions():
        assert callable(getattr(safr, n, None)), f"binding lacks {n}"


def test_status_strings(lib):
    from paper_2510_19542_gb300 import safr
    for s in range(10):
        assert safr.safr_status_string(s).startswith("SAFR_")
    assert "unknown" in safr.safr_status_string(99)


def _geom(**kw):
    from paper_2510_19542_gb300 import synth
    g = synth.scaled(synth.config(2), M=64, P=20)
    g.update(kw)
    return g


@pytest.mark.parametrize("change,status", [
    (dict(M=48), 2),                       # not a power of two
    (dict(M=2048, P=20), 2),               # above the maximum grid
    (dict(M=4, P=4), 2),                   # below the minimum grid
    (dict(h=np.linspace(0, 16000.0, 65), cn2=np.full(65, 1 / 65)), 2),  # SAFR_MAX_L + 1 layers
    (dict(dir_x=np.linspace(-5e-4, 5e-4, 33), dir_y=np.zeros(33),       # SAFR_MAX_G + 1 stars
          kind=np.array([1] * 16 + [0] * 17, np.int32)), 2),
    (dict(dir_x=np.linspace(-5e-4, 5e-4, 20), dir_y=np.zeros(20),       # 17 LGS in one group
          kind=np.array([1] * 17 + [0] * 3, np.int32)), 2),
    (dict(dir_x=np.linspace(-5e-4, 5e-4, 17), dir_y=np.zeros(17),       # 17 NGS in one group
          kind=np.zeros(17, np.int32), output_metric=0), 2),
    (dict(P=65), 1),                       # pupil larger than the grid
    (dict(pitch=0.0), 1),
    (dict(alpha=0.0), 1),
    (dict(beta=-1.0), 1),
    (dict(h=np.array([0.0, 8000, 4000, 9000, 10000, 11000, 12000, 13000, 14000])), 1),  # not ascending
    (dict(h=np.linspace(0, 95000.0, 9)), 1),  # above the sodium layer
    (dict(cn2=np.zeros(9)), 1),
    (dict(output_metric=0), 1),            # mixed plan needs the metric grid
    (dict(alpha_tt=0.0), 1),
    (dict(kind=np.array([0, 1, 2, 0, 0, 0, 0, 0, 0], np.int32)), 1),
    (dict(precision=7), 1),
])
def test_plan_create_rejects_bad_geometry(lib, change, status):
    from paper_2510_19542_gb300 import safr
    g = _geom(**change)
    with pytest.raises(safr.SafrError) as ei:
        safr.safr_plan_create(g, 0)
    assert ei.value.status == status


def test_null_arguments(lib):
    from paper_2510_19542_gb300 import safr
    assert lib.safr_plan_create(None, 0, None) == safr.SAFR_ERR_INVALID_ARG
    out = C.c_void_p()
    assert lib.safr_plan_create(None, 0, C.byref(out)) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_precompute(None, None) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_reconstruct(None, None, None, None, None, None) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_destroy(None) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_launches_per_frame(None) == 0
    assert lib.safr_filter_train(None, None, None, None, None) == safr.SAFR_ERR_INVALID_ARG
    cfg = safr.safr_filter_config(0.15, 25.0, 0.01, 1000, 256, 1, 2e-3, 5)
    assert lib.safr_filter_train(None, C.byref(cfg), None, None, None) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_filter_apply(None, None, 0.01, None) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_filter_reset(None, None) == safr.SAFR_ERR_INVALID_ARG


def test_filter_parameter_count_matches_the_header():
    """SAFR_FILTER_PARAMS = 4*64 + 64 + 2*(64*64 + 64) + 64 + 1 (MLP 4-64-64-64-1)."""
    from paper_2510_19542_gb300 import safr
    src = open(os.path.join(ROOT, "include", "safr.h")).read()
    declared = int(re.search(r"#define SAFR_FILTER_PARAMS (\d+)", src).group(1))
    assert declared == safr.SAFR_FILTER_PARAMS == 4 * 64 + 64 + 2 * (64 * 64 + 64) + 64 + 1


def test_plan_create_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2510_19542_gb300 import safr
    with pytest.raises(safr.SafrError) as ei:
        safr.safr_plan_create(_geom(), 0)
    assert ei.value.status == safr.SAFR_ERR_CUDA
