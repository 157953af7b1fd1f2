"""safr_reconstruct_frames: n frames of one plan (contiguous arrays).

On the persistent kernel the frames run in one launch; frame f's layers must
equal safr_reconstruct's for frame f bit for bit (the same arithmetic, the
same workspaces, one frame after the other).  On the other schedules the
frames are launched one by one.  The first frame is also checked against the
FP64 oracle (per layer, layer_errors.py).
"""
import numpy as np
import pytest
from layer_errors import assert_layers

torch = pytest.importorskip("torch")


def test_frames_argument_errors_without_a_gpu():
    from paper_2510_19542_gb300 import safr
    lib = safr.load()
    fake = 1 << 20
    assert lib.safr_reconstruct_frames(None, 2, fake, None, fake, None, None) == safr.SAFR_ERR_INVALID_ARG


def _case(safr, synth, g, n, path, seed0):
    prec = g.get("precision", "fp32")
    dev = torch.device("cuda:0")
    plan = safr.Plan(g, device=0, path=path)
    L, M, G, P = len(g["h"]), g["M"], len(g["dir_x"]), g["P"]
    xs = [synth.random_frame(g, seed0 + f) for f in range(n)]
    if prec == "fp16":
        hs = [synth.to_fp16_storage(x) for x in xs]
        xin = torch.from_numpy(np.stack([h for h, _ in hs])).to(dev)
        isc = torch.from_numpy(np.stack([s for _, s in hs])).to(dev)
        osc = torch.full((n, L), float("nan"), dtype=torch.float32, device=dev)
        out = torch.full((n, L, M, M), float("nan"), dtype=torch.float16, device=dev)
    else:
        dt = torch.float64 if prec == "fp64" else torch.float32
        xin = torch.from_numpy(np.stack(xs)).to(dev, dt)
        isc = osc = None
        out = torch.full((n, L, M, M), float("nan"), dtype=dt, device=dev)
    safr.safr_reconstruct_frames(plan.handle, n, xin, out, in_scales=isc, out_scales=osc)
    torch.cuda.synchronize(dev)
    assert safr.safr_get_status(plan.handle) == 0
    for f in range(n):  # each frame alone (copied: a frame inside the array need not be 16-byte aligned)
        one = plan.empty_layers()
        if prec == "fp16":
            o_sc = torch.empty(L, dtype=torch.float32, device=dev)
            safr.safr_reconstruct(plan.handle, xin[f].clone(), one, in_scales=isc[f].clone(), out_scales=o_sc)
            torch.cuda.synchronize(dev)
            assert torch.equal(osc[f], o_sc), (g["name"], f)
        else:
            safr.safr_reconstruct(plan.handle, xin[f].clone(), one)
            torch.cuda.synchronize(dev)
        assert torch.equal(out[f], one), (g["name"], f)
    return plan, xs, xin, isc, out, osc


@pytest.mark.gpu
@pytest.mark.parametrize("which", ["mixed-64", "morfeo", "tiny-fp64", "fp16-64", "ngs-512-L6"])
def test_frames_equal_frame_by_frame(which, oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    g = {"mixed-64": synth.scaled(synth.config(2), M=64, P=21),
         "morfeo": synth.config(2),
         "tiny-fp64": synth.config(1),
         "fp16-64": synth.scaled(synth.config(3), M=64, P=64, L=35),
         "ngs-512-L6": dict(synth.scaled(synth.config(3), M=512, P=160, L=6), precision="fp32")}[which]
    n = 5
    plan, xs, xin, isc, out, osc = _case(safr, synth, g, n, safr.SAFR_PATH_FUSED, 40)
    # frame 0 against the oracle (FP16 storage: the decoded inputs and the decoded layers)
    prec = g.get("precision", "fp32")
    if prec == "fp16":
        x0 = synth.from_fp16_storage(xin[0].cpu().numpy(), isc[0].cpu().numpy())
        got = out[0].double().cpu().numpy() * osc[0].double().cpu().numpy()[:, None, None]
        tol = 1e-3
    else:
        x0 = xin[0].double().cpu().numpy()
        got = out[0].double().cpu().numpy()
        tol = 1e-12 if prec == "fp64" else 1e-5
    assert_layers(got, oracle_mod.OraclePlan(g).reconstruct(x0), tol, which)
    plan.close()


@pytest.mark.gpu
def test_frames_on_other_schedules_and_one_frame():
    """The three-pass and one-cluster schedules launch frame by frame; n = 1 is one frame."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    g = synth.scaled(synth.config(2), M=64, P=20)  # 20 x 20 x 4 B and 9 x 64 x 64 x 4 B: aligned frames
    for path in (safr.SAFR_PATH_PASSES, safr.SAFR_PATH_CLUSTER):
        plan, *_ = _case(safr, synth, g, 3, path, 60)
        plan.close()
    plan, *_ = _case(safr, synth, g, 1, safr.SAFR_PATH_FUSED, 70)
    plan.close()
    # frames whose byte size is not a multiple of 16 on a frame-by-frame schedule: refused
    odd = synth.scaled(synth.config(2), M=64, P=21)
    plan = safr.Plan(odd, device=0, path=safr.SAFR_PATH_PASSES)
    x = torch.zeros((2, 9, 21, 21), device="cuda")
    out = torch.zeros((2, 9, 64, 64), device="cuda")
    with pytest.raises(safr.SafrError) as ei:
        safr.safr_reconstruct_frames(plan.handle, 2, x, out)
    assert ei.value.status == safr.SAFR_ERR_MISALIGNED
    plan.close()
