"""Batched frames and the schedule autotuner, through the C ABI.

A batch must give, for every frame, exactly the layers that safr_reconstruct
gives for that frame's plan: the batch replays a CUDA graph of the frames' own
launches.  The autotuner changes only the tiling of the last phase, so its
layers agree with the untuned plan to FP32 rounding.
"""
import numpy as np
import pytest
from layer_errors import assert_layers

torch = pytest.importorskip("torch")


def test_batch_and_autotune_reject_bad_arguments_without_a_gpu():
    from paper_2510_19542_gb300 import safr
    lib = safr.load()
    import ctypes as C
    out = C.c_void_p()
    assert lib.safr_batch_create(None, 3, C.byref(out)) == safr.SAFR_ERR_INVALID_ARG
    arr = (C.c_void_p * 1)(None)
    assert lib.safr_batch_create(arr, 1, C.byref(out)) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_batch_create(arr, 0, C.byref(out)) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_autotune(None, None) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_batch_reconstruct(None, None, None, None, None, None) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_batch_destroy(None) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_batch_launches(None) == 0


def _geometries(synth):
    base = synth.scaled(synth.config(2), M=64, P=20)
    lgs = [i for i in range(9) if base["kind"][i] == 1]
    return [
        ("mixed-64", base),
        ("ngs-32", dict(synth.config(1), precision="fp32")),
        ("lgs-64-native", dict(base, dir_x=base["dir_x"][lgs], dir_y=base["dir_y"][lgs], kind=base["kind"][lgs],
                               output_metric=0)),
        ("mixed-128-L5", synth.scaled(synth.config(2), M=128, P=41, L=5)),
        ("mixed-64-again", synth.scaled(synth.config(2), M=64, P=21)),
        ("ngs-32-fp64", synth.config(1)),                                # FP64
        ("mixed-64-passes", synth.scaled(synth.config(2), M=64, P=20)),  # three-pass schedule
        ("mixed-16", synth.scaled(synth.config(2), M=16, P=6)),
    ]


@pytest.mark.gpu
def test_batch_equals_frame_by_frame():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    dev = torch.device("cuda:0")
    geoms = _geometries(synth)
    plans = []
    for name, g in geoms:
        p = safr.Plan(g, device=0)
        if name.endswith("passes"):
            safr.safr_set_path(p.handle, safr.SAFR_PATH_PASSES)
        plans.append(p)
    batch = safr.safr_batch_create([p.handle for p in plans])
    assert safr.safr_batch_launches(batch) == sum(safr.safr_launches_per_frame(p.handle) for p in plans)
    dts = {"fp32": torch.float32, "fp64": torch.float64}
    for call, seed0 in enumerate((31, 57)):  # new buffers each call: captured again each time
        xs = [torch.from_numpy(synth.random_frame(g, seed0 + i)).to(dev, dts[g.get("precision", "fp32")])
              for i, (_, g) in enumerate(geoms)]
        outs = [p.empty_layers().fill_(float("nan")) for p in plans]
        safr.safr_batch_reconstruct(batch, xs, outs)
        torch.cuda.synchronize(dev)
        assert safr.safr_batch_get_status(batch) == 0
        assert safr.safr_batch_graph(batch) == 1
        for (name, g), p, x, out in zip(geoms, plans, xs, outs):
            ref = p.reconstruct(x)
            torch.cuda.synchronize(dev)
            assert torch.equal(out, ref), (call, name)
    # same buffers, new data: the captured graph is replayed
    for x in xs:
        x.mul_(-0.5)
    safr.safr_batch_reconstruct(batch, xs, outs)
    torch.cuda.synchronize(dev)
    for (name, g), p, x, out in zip(geoms, plans, xs, outs):
        assert torch.equal(out, p.reconstruct(x)), ("replay", name)
    safr.safr_batch_destroy(batch)
    for p in plans:
        p.close()


@pytest.mark.gpu
def test_every_chain_count_equals_frame_by_frame():
    """The batch graph with its chain count forced to K = 1, 2, 4, 8 (frames of grids up to 256 on
    1/K of the SMs each, one-cluster frames on their own cluster) gives every frame's layers bit
    for bit as frame-by-frame safr_reconstruct."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    dev = torch.device("cuda:0")
    geoms = [g for _, g in _geometries(synth) if g.get("precision", "fp32") == "fp32"]
    geoms += [synth.scaled(synth.config(2), M=128, P=40, L=4), synth.scaled(synth.config(2), M=256, P=80, L=3)]
    plans = [safr.Plan(g, device=0) for g in geoms]
    xs = [torch.from_numpy(synth.random_frame(g, 300 + i).astype(np.float32)).to(dev) for i, g in enumerate(geoms)]
    refs = [p.reconstruct(x).clone() for p, x in zip(plans, xs)]
    batch = safr.safr_batch_create([p.handle for p in plans])
    for K in (1, 2, 4, 8):
        safr.safr_batch_set_chains(batch, K)
        outs = [p.empty_layers().fill_(float("nan")) for p in plans]
        safr.safr_batch_reconstruct(batch, xs, outs)
        torch.cuda.synchronize(dev)
        assert safr.safr_batch_chains(batch) == K
        assert safr.safr_batch_graph(batch) == 1
        for i, (o, r) in enumerate(zip(outs, refs)):
            assert torch.equal(o, r), (K, geoms[i]["name"])
    with pytest.raises(safr.SafrError):
        safr.safr_batch_set_chains(batch, 3)
    assert safr.safr_batch_get_status(batch) == 0
    safr.safr_batch_destroy(batch)
    for p in plans:
        p.close()


@pytest.mark.gpu
def test_batch_frame_against_oracle(oracle_mod):
    """One batched frame of the seeded uneven-geometry workload (scaled down) against the FP64 oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    dev = torch.device("cuda:0")
    geoms = synth.batch_configs(n=6, seed=4, grids=(32, 64))
    plans = [safr.Plan(g, device=0) for g in geoms]
    batch = safr.safr_batch_create([p.handle for p in plans])
    xs_np = [synth.frame(g) for g in geoms]
    xs = [torch.from_numpy(x.astype(np.float32)).to(dev) for x in xs_np]
    outs = [p.empty_layers() for p in plans]
    safr.safr_batch_reconstruct(batch, xs, outs)
    torch.cuda.synchronize(dev)
    assert safr.safr_batch_get_status(batch) == 0
    for g, x, out in zip(geoms, xs_np, outs):
        ref = oracle_mod.OraclePlan(g).reconstruct(x)
        got = out.double().cpu().numpy()
        assert_layers(got, ref, 1e-5, g["name"])
    safr.safr_batch_destroy(batch)
    for p in plans:
        p.close()


@pytest.mark.gpu
def test_autotune_keeps_the_layers_and_caches_by_shape():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    dev = torch.device("cuda:0")
    g = synth.scaled(synth.config(2), M=128, P=40)
    x = torch.from_numpy(synth.frame(g).astype(np.float32)).to(dev)
    p = safr.Plan(g, device=0)
    before = p.reconstruct(x).double().cpu().numpy()
    safr.safr_autotune(p.handle)
    info = safr.safr_get_plan_info(p.handle)
    assert info["autotuned"] == 1 and info["path"] in (safr.SAFR_PATH_FUSED, safr.SAFR_PATH_PASSES,
                                                       safr.SAFR_PATH_CLUSTER)
    after = p.reconstruct(x).double().cpu().numpy()
    assert np.linalg.norm(after - before) / np.linalg.norm(before) <= 2e-6
    assert safr.safr_get_status(p.handle) == 0
    q = safr.Plan(g, device=0)  # same shape: the cached schedule, no timing
    safr.safr_autotune(q.handle)
    iq = safr.safr_get_plan_info(q.handle)
    assert (iq["path"], iq["tile_rows"], iq["autotuned"]) == (info["path"], info["tile_rows"], 1)
    p.close()
    q.close()


@pytest.mark.gpu
def test_batch_with_a_repeated_plan_stays_in_one_chain():
    """Two frames on one plan share its workspaces, so the batch keeps them in one chain."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    dev = torch.device("cuda:0")
    g = synth.scaled(synth.config(2), M=64, P=20)
    p, q = safr.Plan(g, device=0), safr.Plan(g, device=0)
    batch = safr.safr_batch_create([p.handle, q.handle, p.handle])
    xs = [torch.from_numpy(synth.random_frame(g, 90 + i).astype(np.float32)).to(dev) for i in range(3)]
    outs = [p.empty_layers() for _ in range(3)]
    safr.safr_batch_reconstruct(batch, xs, outs)
    torch.cuda.synchronize(dev)
    assert safr.safr_batch_chains(batch) == 1
    for plan, x, out in zip((p, q, p), xs, outs):
        assert torch.equal(out, plan.reconstruct(x))
    assert safr.safr_batch_get_status(batch) == 0
    safr.safr_batch_destroy(batch)
    p.close()
    q.close()
