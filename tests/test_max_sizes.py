"""The largest plans the header allows, against the FP64 oracle, element by element.

SAFR_MAX_M (1024) in every precision, SAFR_MAX_L (64), SAFR_MAX_G (32 stars, SAFR_MAX_GROUP_G = 16
in each group) and both at once, on every schedule that takes the plan: the three-pass schedule
must hold each of these shapes, the persistent kernel the FP32 ones; the one-cluster kernel is
tried where the grid allows it.  A shape whose three-pass kernels would need more shared memory
than an SM has is refused at plan creation with SAFR_ERR_UNSUPPORTED_SIZE, and the device stays
usable.  Tolerances and per-layer bounds as in test_gpu_parity.py (layer_errors.py).
"""
import numpy as np
import pytest
from layer_errors import assert_layers

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp32": 1e-5, "fp16": 1e-3, "fp64": 1e-12}
DT = {"fp32": np.float32, "fp64": np.float64}
FUSED, PASSES, CLUSTER = 1, 2, 3


@pytest.fixture(scope="module")
def safr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr as s
    s.load()
    return s


def _ring(n, radius_arcmin, phase_deg):
    a = np.deg2rad(phase_deg + 360.0 * np.arange(n) / n)
    t = np.tan(np.deg2rad(radius_arcmin / 60.0))
    return t * np.cos(a), t * np.sin(a)


def _geometry(name):
    from paper_2510_19542_gb300 import synth
    if name == "ngs-1024-fp32":      # SAFR_MAX_M, odd pupil (a ragged row pair)
        return dict(synth.scaled(synth.config(3), M=1024, P=301, L=2), precision="fp32")
    if name == "mixed-1024-fp32":    # SAFR_MAX_M, 6 LGS + 3 NGS: resample, removeTT, group sum
        return synth.scaled(synth.config(2), M=1024, P=300, L=3)
    if name == "ngs-1024-fp16":      # SAFR_MAX_M, full pupil, FP16 storage with per-layer scales
        return synth.scaled(synth.config(3), M=1024, P=1024, L=4)
    if name == "ngs-1024-fp64":      # SAFR_MAX_M in FP64
        return dict(synth.scaled(synth.config(3), M=1024, P=256, L=2), precision="fp64")
    if name == "ngs-32-L64":         # SAFR_MAX_L
        return dict(synth.scaled(synth.config(3), M=32, P=32, L=64), precision="fp32")
    if name.startswith("mixed-64-G32"):  # SAFR_MAX_G = 16 LGS + 16 NGS (SAFR_MAX_GROUP_G each)
        L = 64 if name.endswith("L64") else 4
        g = synth.scaled(synth.config(2), M=64, P=40, L=L)
        lx, ly = _ring(16, 2.0, 0.0)
        nx, ny = _ring(16, 1.3, 11.25)
        g.update(dir_x=np.concatenate([lx, nx]), dir_y=np.concatenate([ly, ny]),
                 kind=np.array([1] * 16 + [0] * 16, np.int32), name=name)
        return g
    raise ValueError(name)


_REF = {}


def _case(name, oracle_mod):
    """Geometry, frame (as passed to the GPU), input scales and the oracle's layers (once per session)."""
    if name not in _REF:
        from paper_2510_19542_gb300 import synth
        g = _geometry(name)
        x = synth.random_frame(g, 17)
        if g.get("precision", "fp32") == "fp16":
            h, sc = synth.to_fp16_storage(x)
            ref = oracle_mod.OraclePlan(g).reconstruct(synth.from_fp16_storage(h, sc))
            _REF[name] = (g, h, sc, ref)
        else:
            _REF[name] = (g, x, None, oracle_mod.OraclePlan(g).reconstruct(x))
    return _REF[name]


def _run(safr, g, x, sc, path):
    prec = g.get("precision", "fp32")
    plan = safr.Plan(g, device=0)
    try:
        safr.safr_set_path(plan.handle, path)
    except safr.SafrError as e:
        plan.close()
        if e.status != safr.SAFR_ERR_UNSUPPORTED_SIZE:
            raise
        return None
    assert safr.safr_get_path(plan.handle) == path
    if prec == "fp16":
        xin = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        layers, scales = plan.reconstruct(xin, in_scales=torch.from_numpy(sc).cuda())
        torch.cuda.synchronize()
        got = layers.double().cpu().numpy() * scales.double().cpu().numpy()[:, None, None]
    else:
        xin = torch.from_numpy(np.ascontiguousarray(x.astype(DT[prec]))).cuda()
        got = plan.reconstruct(xin)
        torch.cuda.synchronize()
        got = got.double().cpu().numpy()
    assert safr.safr_get_status(plan.handle) == 0
    plan.close()
    return got


# which schedules must hold each shape (the others are tried and may decline)
MUST = {
    "ngs-1024-fp32": (FUSED, PASSES),
    "mixed-1024-fp32": (FUSED, PASSES),
    "ngs-1024-fp16": (FUSED, PASSES),
    "ngs-1024-fp64": (PASSES,),
    "ngs-32-L64": (FUSED, PASSES),
    "mixed-64-G32": (FUSED, PASSES),
    "mixed-64-G32-L64": (FUSED, PASSES),
}


@pytest.mark.parametrize("name", list(MUST))
def test_largest_plans_match_the_oracle(safr, oracle_mod, name):
    g, x, sc, ref = _case(name, oracle_mod)
    tol = TOL[g.get("precision", "fp32")]
    paths = (FUSED, PASSES, CLUSTER) if g["M"] <= 64 else (FUSED, PASSES)
    ran = []
    for path in paths:
        got = _run(safr, g, x, sc, path)
        if got is None:
            assert path not in MUST[name], (name, path, "declined")
            continue
        assert got.shape == ref.shape
        assert_layers(got, ref, tol, f"{name} path {path}")
        ran.append(path)
    assert set(MUST[name]) <= set(ran)


def test_shape_beyond_the_three_pass_kernels_is_refused(safr):
    """M = 1024 with 16 stars in one group: the column pass would need (3 x 16 + 1) x 1024 complex
    of shared memory, more than an SM has; plan creation refuses it and frees what it allocated."""
    from paper_2510_19542_gb300 import synth
    g = dict(synth.scaled(synth.config(3), M=1024, P=64, L=1), precision="fp32")
    x, y = _ring(16, 1.0, 0.0)
    g.update(dir_x=x, dir_y=y, kind=np.zeros(16, np.int32))
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(safr.SafrError) as ei:
        safr.safr_plan_create(g, 0)
    assert ei.value.status == safr.SAFR_ERR_UNSUPPORTED_SIZE
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)
    # the device is still usable: a small plan runs
    small = synth.scaled(synth.config(2), M=32, P=12)
    plan = safr.Plan(small, device=0)
    out = plan.reconstruct(torch.from_numpy(synth.frame(small).astype(np.float32)).cuda())
    torch.cuda.synchronize()
    assert torch.isfinite(out).all() and safr.safr_get_status(plan.handle) == 0
    plan.close()
