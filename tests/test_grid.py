"""The persistent kernel's grid size (safr_set_grid): every phase shares its
work among the CTAs launched, so the layers must not depend on it beyond
rounding, and two plans with half grids may run at the same time on two
streams."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_set_grid_rejects_bad_arguments_without_a_gpu():
    from paper_2510_19542_gb300 import safr
    lib = safr.load()
    assert lib.safr_set_grid(None, 0) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_get_grid(None) == 0


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.gpu
def test_layers_do_not_depend_on_the_grid(oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    for g in [synth.scaled(synth.config(2), M=64, P=20), synth.config(1), synth.config(2)]:
        x = synth.frame(g)
        ref = oracle_mod.OraclePlan(g).reconstruct(x)
        dt = torch.float64 if g.get("precision") == "fp64" else torch.float32
        tol = 1e-12 if g.get("precision") == "fp64" else 1e-5
        p = safr.Plan(g, device=0, path=safr.SAFR_PATH_FUSED)
        xin = torch.from_numpy(x).to("cuda:0", dt)
        first = None
        # launches on one plan alternate grid sizes: each launch's grid barrier counts its own CTAs
        for ctas in (0, nsm // 2, nsm // 4, nsm // 8, 7, nsm // 2, 0):
            safr.safr_set_grid(p.handle, ctas)
            assert safr.safr_get_grid(p.handle) == (ctas or nsm)
            out = p.reconstruct(xin)
            got = out.double().cpu().numpy()
            assert _rel(got, ref) <= tol, (g["name"], ctas, _rel(got, ref))
            if ctas == 0:
                if first is None:
                    first = out.clone()
                else:
                    assert torch.equal(out, first), g["name"]
        assert safr.safr_get_status(p.handle) == 0
        p.close()


@pytest.mark.gpu
def test_two_half_grid_plans_on_two_streams():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    g = synth.config(2)
    plans = [safr.Plan(g, device=0) for _ in range(2)]
    for p in plans:
        safr.safr_set_grid(p.handle, nsm // 2)
    xs = [torch.from_numpy(synth.frame(g, seed=80 + i).astype(np.float32)).cuda() for i in range(2)]
    seq = [p.reconstruct(x) for p, x in zip(plans, xs)]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(2)]
    outs = [p.empty_layers() for p in plans]
    for _ in range(3):
        for p, x, o, s in zip(plans, xs, outs, streams):
            safr.safr_reconstruct(p.handle, x, o, stream=s)
        torch.cuda.synchronize()
        for a, b in zip(outs, seq):
            assert torch.equal(a, b)
    for p in plans:
        assert safr.safr_get_status(p.handle) == 0
        p.close()
