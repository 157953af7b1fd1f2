"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: relative L2 error <= 1e-5 for FP32, <= 1e-3 for FP16 storage,
<= 1e-12 for the FP64 instantiation, overall and per layer (both relative to
the whole output and to each layer's own RMS, as layer_errors.py states).  B
from the GPU precompute (a Cholesky solve) is compared with the oracle's (a
Jacobi SVD) at 1e-12 in FP64.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def safr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr as s
    s.load()
    return s


@pytest.fixture(scope="module")
def synth():
    from paper_2510_19542_gb300 import synth as s
    return s


TOL = {"fp32": 1e-5, "fp16": 1e-3, "fp64": 1e-12}
DT = {"fp32": np.float32, "fp16": np.float16, "fp64": np.float64}


from layer_errors import assert_layers, rel_errors  # noqa: E402,F401


PATHS = {"fused": 1, "passes": 2, "cluster": 3}


@pytest.fixture(params=["fused", "passes", "cluster"])
def path(request):
    return PATHS[request.param]


def skip_unless_path_holds(geom, path):
    """The one-cluster schedule holds grids up to 64 only."""
    if path == PATHS["cluster"] and geom["M"] > 64:
        pytest.skip("the one-cluster kernel holds grids up to 64")


def run_gpu(safr, geom, x, in_scales=None, path=None):
    prec = geom.get("precision", "fp32")
    skip_unless_path_holds(geom, path)
    plan = safr.Plan(geom, device=0, path=path)
    if path is not None:
        assert safr.safr_get_path(plan.handle) == path
    xin = torch.from_numpy(np.ascontiguousarray(x.astype(DT[prec]))).cuda()
    sc = torch.from_numpy(in_scales).cuda() if in_scales is not None else None
    out = plan.reconstruct(xin, in_scales=sc)
    torch.cuda.synchronize()
    assert safr.safr_get_status(plan.handle) == 0
    if isinstance(out, tuple):
        layers, scales = out
        got = layers.double().cpu().numpy() * scales.double().cpu().numpy()[:, None, None]
    else:
        got = out.double().cpu().numpy()
    return plan, got


def check(safr, oracle_mod, geom, x, tol=None, in_scales=None, x_oracle=None, path=None):
    prec = geom.get("precision", "fp32")
    tol = TOL[prec] if tol is None else tol
    ref = oracle_mod.OraclePlan(geom).reconstruct(x if x_oracle is None else x_oracle)
    plan, got = run_gpu(safr, geom, x, in_scales, path)
    plan.close()
    return assert_layers(got, ref, tol)


# ----------------------------------------------------------------------------
# B: GPU Cholesky route vs oracle Jacobi-SVD route
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("k,M,P,L", [(1, 32, 32, None), (2, 64, 20, None), (3, 64, 64, 35), (2, 32, 10, 4)])
def test_precompute_B_matches_oracle(safr, synth, oracle_mod, k, M, P, L):
    geom = synth.scaled(synth.config(k), M=M, P=P, L=L)
    geom["precision"] = "fp64"
    pl = safr.Plan(geom, device=0)
    orc = oracle_mod.OraclePlan(geom)
    for gi in range(pl.info["ngroups"]):
        Bg = safr.safr_copy_B(pl.handle, gi)              # [k][l][g][j]
        _, stars, _, Bo = orc.group(gi)                   # [j][k][l][g]
        Bo = np.transpose(Bo[:, :M // 2], (1, 2, 3, 0))
        err = np.abs(Bg - Bo).max() / np.abs(Bo).max()
        assert err <= 1e-12, (gi, err)
        assert np.all(Bg[:, :, :, M // 2] == 0)           # Nyquist row
    pl.close()


def test_precompute_B_fp32_rounding(safr, synth, oracle_mod):
    geom = synth.scaled(synth.config(2), M=64, P=20)
    pl = safr.Plan(geom, device=0)
    orc = oracle_mod.OraclePlan(geom)
    for gi in range(2):
        Bg = safr.safr_copy_B(pl.handle, gi)
        Bo = np.transpose(orc.group(gi)[3][:, :32], (1, 2, 3, 0))
        assert np.abs(Bg - Bo).max() <= 1e-6 * np.abs(Bo).max()
    pl.close()


# ----------------------------------------------------------------------------
# Whole frames
# ----------------------------------------------------------------------------
def test_tiny_ngs_fp64(safr, synth, oracle_mod, path):
    g = synth.config(1)
    check(safr, oracle_mod, g, synth.frame(g), path=path)


def test_tiny_ngs_fp32(safr, synth, oracle_mod, path):
    g = dict(synth.config(1), precision="fp32")
    check(safr, oracle_mod, g, synth.frame(g), path=path)


@pytest.mark.parametrize("M,P,L", [(64, 20, None), (128, 40, None), (64, 37, 5), (32, 9, 3), (8, 8, 2),
                                   (16, 5, 9), (256, 80, 12), (512, 160, 6), (64, 20, 35)])
def test_mixed_lgs_ngs_fp32(safr, synth, oracle_mod, M, P, L, path):
    """Split tomography with removeTT and the metric resample; odd P gives a
    ragged last row pair and an odd pad offset.  The 512 grid runs the
    transforms with 16 values per lane (loaded 8 at a time) and B unstaged;
    the 64 grid with 35 layers has B unstaged in the one-cluster kernel."""
    g = synth.scaled(synth.config(2), M=M, P=P, L=L)
    check(safr, oracle_mod, g, synth.frame(g), path=path)


def test_mixed_lgs_ngs_fp64(safr, synth, oracle_mod, path):
    g = dict(synth.scaled(synth.config(2), M=64, P=21), precision="fp64")
    check(safr, oracle_mod, g, synth.frame(g), path=path)


def test_lgs_only_native_and_metric(safr, synth, oracle_mod, path):
    base = synth.scaled(synth.config(2), M=64, P=20)
    lgs = [i for i in range(9) if base["kind"][i] == 1]
    for metric in (0, 1):
        g = dict(base, dir_x=base["dir_x"][lgs], dir_y=base["dir_y"][lgs], kind=base["kind"][lgs],
                 output_metric=metric)
        check(safr, oracle_mod, g, synth.frame(g), path=path)


def test_many_layers_chunked(safr, synth, oracle_mod, path):
    """L = 35 on a 512 grid: the column pass runs the inverse FFTs in layer chunks."""
    g = dict(synth.scaled(synth.config(3), M=512, P=160, L=35), precision="fp32")
    x = synth.random_frame(g, 5)
    check(safr, oracle_mod, g, x, path=path)


def test_fp16_storage(safr, synth, oracle_mod, path):
    g = synth.scaled(synth.config(3), M=64, P=64, L=35)
    x = synth.frame(g)
    h, sc = synth.to_fp16_storage(x)
    check(safr, oracle_mod, g, h, in_scales=sc, x_oracle=synth.from_fp16_storage(h, sc), path=path)


def test_degenerate_layers_and_single_star(safr, synth, oracle_mod, path):
    rng = np.random.default_rng(0)
    # every layer at the ground: A(n) has rank one at every n
    g = dict(synth.scaled(synth.config(1), M=32, P=32), h=np.array([0.0, 1e-6, 2e-6]), precision="fp64")
    check(safr, oracle_mod, g, rng.standard_normal((3, 32, 32)), path=path)
    # one star, one layer, beta = 0
    g = dict(synth.scaled(synth.config(1), M=16, P=12), h=np.array([5000.0]), cn2=np.array([1.0]),
             dir_x=np.array([2e-4]), dir_y=np.array([-1e-4]), kind=np.zeros(1, np.int32), beta=0.0,
             precision="fp64")
    check(safr, oracle_mod, g, rng.standard_normal((1, 12, 12)), path=path)


def test_asymmetric_asterism_no_transpose(safr, synth, oracle_mod, path):
    rng = np.random.default_rng(4)
    g = synth.scaled(synth.config(2), M=64, P=24)
    g["dir_x"] = rng.uniform(-6e-4, 6e-4, 9)
    g["dir_y"] = rng.uniform(-2e-4, 2e-4, 9)
    check(safr, oracle_mod, g, synth.random_frame(g, 3), path=path)


def test_full_size_morfeo_frame(safr, synth, oracle_mod, path):
    """The benchmarked workload at full size: 256 grid, 80 pupil, 6 LGS + 3 NGS, 9 layers."""
    g = synth.config(2)
    check(safr, oracle_mod, g, synth.frame(g), path=path)


_FP16_512 = {}


def _fp16_512_reference(synth, oracle_mod):
    """The 512-grid 35-layer FP16-storage frame and its full FP64 oracle layers
    (computed once per session: one full oracle run takes seconds)."""
    if not _FP16_512:
        g = synth.config(3)
        x = synth.random_frame(g, 11) * 5.0
        h, sc = synth.to_fp16_storage(x)
        _FP16_512.update(g=g, h=h, sc=sc, ref=oracle_mod.OraclePlan(g).reconstruct(synth.from_fp16_storage(h, sc)))
    return _FP16_512


def test_full_size_fp16_512(safr, synth, oracle_mod, path):
    """512 grid, 35 layers, FP16 storage with per-layer scales, at full size:
    every output against the full FP64 oracle (35 IDFT2s of 512^2), with the
    per-layer errors (relative to the whole output and to each layer's own RMS)
    asserted for all 35 layers."""
    w = _fp16_512_reference(synth, oracle_mod)
    plan, got = run_gpu(safr, w["g"], w["h"], w["sc"], path)
    plan.close()
    overall, per_layer, own = assert_layers(got, w["ref"], TOL["fp16"])
    assert len(own) == 35


# ----------------------------------------------------------------------------
# Properties of the GPU path
# ----------------------------------------------------------------------------
def test_deterministic_and_host_entry(safr, synth, path):
    g = synth.scaled(synth.config(2), M=64, P=20)
    x = synth.frame(g).astype(np.float32)
    skip_unless_path_holds(g, path)
    plan = safr.Plan(g, device=0, path=path)
    xin = torch.from_numpy(x).cuda()
    a = plan.reconstruct(xin).cpu().numpy()
    b = plan.reconstruct(xin).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    host_out = np.empty_like(a)
    safr.safr_reconstruct_host(plan.handle, np.ascontiguousarray(x), host_out)
    np.testing.assert_array_equal(host_out, a)
    plan.close()


def test_runtime_argument_errors(safr, synth):
    g = synth.scaled(synth.config(2), M=32, P=10)
    h = safr.safr_plan_create(g, 0)
    x = torch.zeros((9, 10, 10), device="cuda")
    out = torch.zeros((9, 32, 32), device="cuda")
    with pytest.raises(safr.SafrError) as ei:
        safr.safr_reconstruct(h, x, out)
    assert ei.value.status == safr.SAFR_ERR_NOT_PRECOMPUTED
    safr.safr_precompute(h)
    with pytest.raises(safr.SafrError) as ei:
        safr.safr_reconstruct(h, x.data_ptr() + 4, out)
    assert ei.value.status == safr.SAFR_ERR_MISALIGNED
    with pytest.raises(safr.SafrError) as ei:
        safr.safr_reconstruct(h, x, out, out_scales=torch.zeros(9, device="cuda"))
    assert ei.value.status == safr.SAFR_ERR_INVALID_ARG
    safr.safr_reconstruct(h, x, out)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0  # linear map of a zero frame
    assert safr.safr_get_status(h) == 0
    info = safr.safr_get_plan_info(h)
    assert info["ngroups"] == 2 and info["group_G"] == [6, 3] and info["precomputed"] == 1
    safr.safr_destroy(h)


def test_trace_phases(safr, synth, path):
    g = synth.config(2) if path != PATHS["cluster"] else synth.scaled(synth.config(2), M=64, P=20)
    plan = safr.Plan(g, device=0, path=path)
    x = torch.from_numpy(synth.random_frame(g, 1).astype(np.float32)).cuda()
    safr.safr_trace(plan.handle, True)
    plan.reconstruct(x)
    ms = safr.safr_trace_read(plan.handle)
    assert len(ms) == safr.safr_launches_per_frame(plan.handle) and all(m > 0 for m in ms)
    plan.close()


def test_cluster_kernel_path_selection(safr, synth):
    """SAFR_PATH_CLUSTER is accepted on grids up to 64 and refused above (choice
    unchanged); SAFR_PATH_AUTO runs the one-cluster kernel on the small 32-grid
    frame and the persistent kernel on grids above 64."""
    g = synth.config(1)
    plan = safr.Plan(g, device=0)
    assert safr.safr_get_path(plan.handle) == PATHS["cluster"]
    assert safr.safr_launches_per_frame(plan.handle) == 1
    plan.close()
    for M in (8, 16, 32, 64, 128):
        g = synth.scaled(synth.config(2), M=M, P=max(4, M // 3))
        plan = safr.Plan(g, device=0)
        auto = safr.safr_get_path(plan.handle)
        if M > 64:
            assert auto == PATHS["fused"]
            with pytest.raises(safr.SafrError) as ei:
                safr.safr_set_path(plan.handle, PATHS["cluster"])
            assert ei.value.status == safr.SAFR_ERR_UNSUPPORTED_SIZE
            assert safr.safr_get_path(plan.handle) == auto
        else:
            assert auto in (PATHS["cluster"], PATHS["fused"])
            safr.safr_set_path(plan.handle, PATHS["cluster"])
            assert safr.safr_get_path(plan.handle) == PATHS["cluster"]
        plan.close()


def test_paths_agree(safr, synth):
    """Both schedules on the full-size workload: same layers to FP32 rounding."""
    g = synth.config(2)
    x = torch.from_numpy(synth.frame(g).astype(np.float32)).cuda()
    a = safr.Plan(g, device=0, path=1)
    b = safr.Plan(g, device=0, path=2)
    ya = a.reconstruct(x).double().cpu().numpy()
    yb = b.reconstruct(x).double().cpu().numpy()
    assert np.linalg.norm(ya - yb) / np.linalg.norm(yb) < 2e-6
    a.close()
    b.close()


def test_grid_barrier_timeout_is_reported_not_hung(safr, synth):
    """One CTA leaves before the first grid barrier: the others' bounded waits run
    out, the kernel records SAFR_ERR_TIMEOUT, and the plan keeps working after
    the status is read."""
    g = synth.scaled(synth.config(2), M=64, P=20)
    plan = safr.Plan(g, device=0, path=1)
    x = torch.from_numpy(synth.frame(g).astype(np.float32)).cuda()
    good = plan.reconstruct(x).clone()
    safr.safr_debug_skip_barrier(plan.handle, 0, 0.02)
    plan.reconstruct(x)
    torch.cuda.synchronize()
    assert safr.safr_get_status(plan.handle) == safr.SAFR_ERR_TIMEOUT
    assert safr.safr_get_status(plan.handle) == 0  # cleared, barrier re-armed
    safr.safr_debug_skip_barrier(plan.handle, -1, 0.0)
    again = plan.reconstruct(x)
    torch.cuda.synchronize()
    assert safr.safr_get_status(plan.handle) == 0
    assert torch.equal(again, good)
    plan.close()


def test_plans_created_later_do_not_break_earlier_ones(safr, synth):
    """A kernel's shared-memory limit is shared by every plan that launches it: a
    plan with a smaller need, created later, must not make an earlier plan's
    launch fail (both schedules)."""
    big_g = synth.scaled(synth.config(2), M=128, P=41)
    small_g = synth.scaled(synth.config(2), M=16, P=6)
    for path in (1, 2):
        big = safr.Plan(big_g, device=0, path=path)
        x = torch.from_numpy(synth.random_frame(big_g, 2).astype(np.float32)).cuda()
        ref = big.reconstruct(x).clone()
        small = safr.Plan(small_g, device=0, path=path)
        small.reconstruct(torch.zeros((9, 6, 6), device="cuda"))
        again = big.reconstruct(x)
        torch.cuda.synchronize()
        assert torch.equal(again, ref)
        big_same_m = safr.Plan(synth.scaled(synth.config(2), M=128, P=12, L=3), device=0, path=path)
        big_same_m.reconstruct(torch.zeros((9, 12, 12), device="cuda"))
        assert torch.equal(big.reconstruct(x), ref)
        for p in (big, small, big_same_m):
            p.close()
