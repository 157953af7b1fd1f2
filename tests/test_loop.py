"""The AO-loop steps around SAFR (Algorithm 3) on the GPU, through the C ABI,
against the FP64 oracle: pseudo open loop control (safr_polc), the
integrator (safr_integrate) and the whole loop iteration (safr_loop_step) on
two iterations in a row.  Tolerances: relative L2 1e-6 for POLC and the
integrator in FP32 (a sum of L bilinear interpolations), 1e-5 for the loop
step in FP32 (it contains a SAFR frame), 1e-12 in FP64.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_loop_entry_points_reject_bad_arguments_without_a_gpu():
    from paper_2510_19542_gb300 import safr
    lib = safr.load()
    assert lib.safr_polc(None, None, None, None, None) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_integrate(None, None, None, C.c_double(0.5), None) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_loop_step(None, None, None, C.c_double(0.5), None) == safr.SAFR_ERR_INVALID_ARG


DT = {"fp32": (torch.float32, np.float32), "fp64": (torch.float64, np.float64)}
TOL = {"fp32": (1e-6, 1e-5), "fp64": (1e-12, 1e-12)}


def _geometries(synth):
    base = synth.scaled(synth.config(2), M=64, P=20)
    lgs = [i for i in range(9) if base["kind"][i] == 1]
    return [
        ("mixed-64-metric", base),
        ("lgs-64-native", dict(base, dir_x=base["dir_x"][lgs], dir_y=base["dir_y"][lgs], kind=base["kind"][lgs],
                               output_metric=0)),
        ("tiny-ngs-32-fp64", synth.config(1)),
        ("morfeo-256", synth.config(2)),
    ]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.gpu
def test_polc_and_integrator_match_oracle(oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    dev = torch.device("cuda:0")
    for name, g in _geometries(synth):
        prec = g.get("precision", "fp32")
        tdt, ndt = DT[prec]
        tol = TOL[prec][0]
        plan = safr.Plan(g, device=0)
        L, M, G, P = len(g["h"]), g["M"], len(g["dir_x"]), g["P"]
        rng = np.random.default_rng(11)
        psi = (rng.standard_normal((G, P, P)) * synth.pupil(g)).astype(ndt)
        a = rng.standard_normal((L, M, M)).astype(ndt)
        out = torch.full((G, P, P), float("nan"), dtype=tdt, device=dev)
        safr.safr_polc(plan.handle, torch.from_numpy(psi).to(dev), torch.from_numpy(a).to(dev), out)
        ref = oracle_mod.polc(g, psi.astype(np.float64), a.astype(np.float64))
        got = out.double().cpu().numpy()
        assert np.all(np.isfinite(got)), name
        assert _rel(got, ref) <= tol, (name, _rel(got, ref))
        # the integrator, in place
        phi = rng.standard_normal((L, M, M)).astype(ndt)
        at = torch.from_numpy(a).to(dev)
        safr.safr_integrate(plan.handle, torch.from_numpy(phi).to(dev), at, 0.5)
        ref = oracle_mod.integrate(phi.astype(np.float64), a.astype(np.float64), 0.5)
        assert _rel(at.double().cpu().numpy(), ref) <= tol, name
        with pytest.raises(safr.SafrError):
            safr.safr_integrate(plan.handle, torch.from_numpy(phi).to(dev), at, 1.5)
        torch.cuda.synchronize(dev)
        assert safr.safr_get_status(plan.handle) == 0
        plan.close()


@pytest.mark.gpu
def test_loop_steps_in_a_row_match_oracle(oracle_mod):
    """Two loop iterations: a1 = (1-k) a0 + k SAFR(POLC(psi1, a0)), then a2 from a1 and psi2."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    dev = torch.device("cuda:0")
    for name, g in _geometries(synth)[:3]:
        prec = g.get("precision", "fp32")
        tdt, ndt = DT[prec]
        plan = safr.Plan(g, device=0)
        orc = oracle_mod.OraclePlan(g)
        L, M = len(g["h"]), g["M"]
        gain = 0.5
        a_ref = np.random.default_rng(5).standard_normal((L, M, M)) * 0.1
        a = torch.from_numpy(a_ref.astype(ndt)).to(dev)
        a_ref = a_ref.astype(ndt).astype(np.float64)
        for it, seed in enumerate((31, 32)):
            psi = synth.frame(g, seed=seed).astype(ndt)
            safr.safr_loop_step(plan.handle, torch.from_numpy(psi).to(dev), a, gain)
            polc = oracle_mod.polc(g, psi.astype(np.float64), a_ref)
            a_ref = oracle_mod.integrate(orc.reconstruct(polc), a_ref, gain)
            got = a.double().cpu().numpy()
            assert np.all(np.isfinite(got)), (name, it)
            assert _rel(got, a_ref) <= TOL[prec][1], (name, it, _rel(got, a_ref))
        assert safr.safr_get_status(plan.handle) == 0
        plan.close()


@pytest.mark.gpu
def test_loop_refuses_fp16_storage_plans():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    g = dict(synth.scaled(synth.config(3), M=64, P=64, L=5), precision="fp16")
    plan = safr.Plan(g, device=0)
    x = torch.zeros((3, 64, 64), dtype=torch.float16, device="cuda:0")
    a = torch.zeros((5, 64, 64), dtype=torch.float16, device="cuda:0")
    with pytest.raises(safr.SafrError) as ei:
        safr.safr_loop_step(plan.handle, x, a, 0.5)
    assert ei.value.status == safr.SAFR_ERR_UNSUPPORTED_SIZE
    plan.close()


@pytest.mark.gpu
def test_loop_steps_on_the_three_pass_schedule_match_oracle(oracle_mod):
    """The same two iterations when the plan runs the three-pass schedule: POLC,
    the frame and the integrator are then three separate kernels."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    dev = torch.device("cuda:0")
    g = synth.scaled(synth.config(2), M=64, P=20)
    plan = safr.Plan(g, device=0, path=safr.SAFR_PATH_PASSES)
    orc = oracle_mod.OraclePlan(g)
    L, M = len(g["h"]), g["M"]
    a_ref = np.random.default_rng(6).standard_normal((L, M, M)).astype(np.float32).astype(np.float64) * 0.1
    a = torch.from_numpy(a_ref.astype(np.float32)).to(dev)
    for seed in (41, 42):
        psi = synth.frame(g, seed=seed).astype(np.float32)
        safr.safr_loop_step(plan.handle, torch.from_numpy(psi).to(dev), a, 0.25)
        a_ref = oracle_mod.integrate(orc.reconstruct(oracle_mod.polc(g, psi.astype(np.float64), a_ref)), a_ref, 0.25)
        assert _rel(a.double().cpu().numpy(), a_ref) <= 1e-5
    assert safr.safr_get_status(plan.handle) == 0
    plan.close()
