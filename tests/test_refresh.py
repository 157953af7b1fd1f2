"""Soft real-time refresh of B (Algorithm 2 rerun in place when the turbulence
profile, the star positions or alpha change) and plan files, through the C ABI.

A refreshed plan must hold exactly the B, and give exactly the layers and loop
steps, of a plan created from the new geometry: the same host arithmetic
feeds the same precompute kernel.  A plan file round trip must give back B and
the layers bit for bit.  The file parser is checked on the CPU with files
written here from the documented format (FNV-1a-64 hashes computed in Python).
"""
import ctypes as C
import os
import struct

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def fnv1a(data: bytes) -> int:
    h = 0xcbf29ce484222325
    for b in data:
        h ^= b
        h = (h * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def plan_file(g, B: bytes, learned=0, version=1, magic=b"SAFRPLN1"):
    L, G = len(g["h"]), len(g["dir_x"])
    prec = {"fp32": 0, "fp16": 1, "fp64": 2}[g.get("precision", "fp32")]
    head = magic + struct.pack("<I", version)
    head += struct.pack("<8i", g["M"], g["P"], L, G, prec, int(g.get("output_metric", 1)), int(g.get("remove_tt", 1)),
                        learned)
    head += struct.pack("<7d", g["pitch"], g.get("diameter", 0.0), g.get("obstruction", 0.0), g.get("h_lgs", 90e3),
                        g["alpha"], g.get("alpha_tt", g["alpha"]), g["beta"])
    for arr in (g["h"], g["cn2"], g["dir_x"], g["dir_y"]):
        head += np.ascontiguousarray(arr, dtype="<f8").tobytes()
    head += np.ascontiguousarray(g["kind"], dtype="<i4").tobytes()
    return head + struct.pack("<Q", fnv1a(head)) + struct.pack("<Q", len(B)) + B + struct.pack("<Q", fnv1a(B))


def test_plan_files_are_checked_before_any_device_work(tmp_path):
    from paper_2510_19542_gb300 import safr, synth
    lib = safr.load()
    out = C.c_void_p()
    assert lib.safr_plan_save(None, b"x") == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_plan_load(None, 0, C.byref(out)) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_refresh(None, None, None) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_plan_load(os.fsencode(str(tmp_path / "missing")), 0, C.byref(out)) == safr.SAFR_ERR_IO
    g = synth.config(1)
    M, L, G = g["M"], 3, 3
    nb = (M // 2) * L * G * M * 16  # FP64 complex B
    B = np.random.default_rng(1).standard_normal(nb // 8).tobytes()
    good = plan_file(g, B)
    cases = {
        "magic": plan_file(g, B, magic=b"SAFRPLN0"),
        "version": plan_file(g, B, version=2),
        "truncated": good[:-9],
        "geometry": good[:40] + bytes([good[40] ^ 1]) + good[41:],
        "B": good[:-20] + bytes([good[-20] ^ 1]) + good[-19:],
        "trailing": good + b"\0",
    }
    for name, data in cases.items():
        path = tmp_path / name
        path.write_bytes(data)
        assert lib.safr_plan_load(os.fsencode(str(path)), 0, C.byref(out)) == safr.SAFR_ERR_IO, name
    path = tmp_path / "good"
    path.write_bytes(good)
    st = lib.safr_plan_load(os.fsencode(str(path)), 0, C.byref(out))
    if torch.cuda.is_available():
        assert st == safr.SAFR_OK
        safr.safr_destroy(out.value)
    else:
        assert st == safr.SAFR_ERR_CUDA  # the file passed every check; only plan creation needs the GPU


@pytest.mark.gpu
def test_plan_file_round_trip(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    dev = torch.device("cuda:0")
    for name, g in [("mixed-64", synth.scaled(synth.config(2), M=64, P=20)), ("ngs-32-fp64", synth.config(1))]:
        p = safr.Plan(g, device=0)
        path = str(tmp_path / f"{name}.safr")
        safr.safr_plan_save(p.handle, path)
        q = safr.Plan.load(path, 0)
        assert np.array_equal(safr.safr_copy_B(q.handle, 0), safr.safr_copy_B(p.handle, 0))
        dt = torch.float64 if g.get("precision") == "fp64" else torch.float32
        x = torch.from_numpy(synth.frame(g)).to(dev, dt)
        assert torch.equal(p.reconstruct(x), q.reconstruct(x)), name
        with open(path, "rb") as f:
            data = f.read()
        head = len(plan_file(g, b"")) - 8                  # geometry, its hash and the byte count of B
        assert len(data) == head + p.info["b_bytes"] + 8
        assert data == plan_file(g, data[head:-8]), name   # exactly the documented format
        p.close()
        q.close()


@pytest.mark.gpu
def test_learned_B_survives_a_plan_file(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    g = synth.config(5)
    p = safr.Plan(g, device=0)
    rng = np.random.default_rng(3)
    w = (rng.standard_normal(safr.SAFR_FILTER_PARAMS) * 0.1).astype(np.float32)
    safr.safr_filter_apply(p.handle, w, 0.01)
    path = str(tmp_path / "learned.safr")
    safr.safr_plan_save(p.handle, path)
    q = safr.Plan.load(path, 0)
    assert np.array_equal(safr.safr_copy_B(q.handle, 0), safr.safr_copy_B(p.handle, 0))
    p.close()
    q.close()


def _changed(g):
    rng = np.random.default_rng(9)
    L, G = len(g["h"]), len(g["dir_x"])
    cn2 = np.asarray(g["cn2"]) * rng.uniform(0.5, 1.5, L)
    rot = np.deg2rad(7.0)
    dx = np.cos(rot) * np.asarray(g["dir_x"]) - np.sin(rot) * np.asarray(g["dir_y"])
    dy = np.sin(rot) * np.asarray(g["dir_x"]) + np.cos(rot) * np.asarray(g["dir_y"])
    return dict(g, cn2=cn2, dir_x=dx * 1.05, dir_y=dy * 1.05, alpha=g["alpha"] * 3.0,
                alpha_tt=g.get("alpha_tt", g["alpha"]) * 0.5)


@pytest.mark.gpu
def test_refresh_equals_a_new_plan():
    """Profile, asterism rotation and alphas changed in place: B, the layers and a
    loop step equal those of a plan created from the new geometry, bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    dev = torch.device("cuda:0")
    for g in [synth.scaled(synth.config(2), M=64, P=20), synth.config(1), synth.config(2)]:
        h = _changed(g)
        p = safr.Plan(g, device=0)
        safr.safr_refresh(p.handle, cn2=h["cn2"], dir_x=h["dir_x"], dir_y=h["dir_y"], alpha=h["alpha"],
                          alpha_tt=h["alpha_tt"])
        q = safr.Plan(h, device=0)
        for gi in range(p.info["ngroups"]):
            assert np.array_equal(safr.safr_copy_B(p.handle, gi), safr.safr_copy_B(q.handle, gi)), (g["name"], gi)
        assert safr.safr_get_plan_info(p.handle)["warnings"] == safr.safr_get_plan_info(q.handle)["warnings"]
        dt = torch.float64 if g.get("precision") == "fp64" else torch.float32
        x = torch.from_numpy(synth.frame(h)).to(dev, dt)
        assert torch.equal(p.reconstruct(x), q.reconstruct(x)), g["name"]
        a = torch.from_numpy(np.random.default_rng(2).standard_normal((p.info["L"], g["M"], g["M"]))).to(dev, dt)
        a2 = a.clone()
        safr.safr_loop_step(p.handle, x, a, 0.5)
        safr.safr_loop_step(q.handle, x, a2, 0.5)
        assert torch.equal(a, a2), g["name"]
        assert safr.safr_get_status(p.handle) == 0
        p.close()
        q.close()


@pytest.mark.gpu
def test_refresh_rejects_bad_values_and_keeps_B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    g = synth.config(1)
    p = safr.Plan(g, device=0)
    B0 = safr.safr_copy_B(p.handle, 0)
    for kw in [dict(cn2=[0.5, 0.0, 0.5]), dict(dir_x=[0.0, np.nan, 0.0], dir_y=[0.0, 0.0, 0.0]),
               dict(alpha=np.inf)]:
        with pytest.raises(safr.SafrError) as ei:
            safr.safr_refresh(p.handle, **kw)
        assert ei.value.status == safr.SAFR_ERR_INVALID_ARG
    lib = safr.load()
    u = safr.safr_update(None, np.zeros(3).ctypes.data_as(C.POINTER(C.c_double)), None, 0.0, 0.0)
    assert lib.safr_refresh(p.handle, C.byref(u), None) == safr.SAFR_ERR_INVALID_ARG  # dir_x without dir_y
    assert np.array_equal(safr.safr_copy_B(p.handle, 0), B0)
    p.close()
