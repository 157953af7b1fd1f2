"""safr_reconstruct_noalloc: the reconstruction for callers that cannot call
cudaMalloc.

A hard-real-time thread, a plugin whose host framework owns all device
memory, or code that may not allocate after start-up cannot create a plan,
because a plan allocates.  The no-allocation entry point takes every input
(wavefronts and B) and every output (layers and a status word) from the
caller.  It keeps the kernel's scratch in a static device array of the
library.  These tests check it through the C ABI against the plan-based
safr_reconstruct on the same inputs, at the FP32 tolerance of the other GPU
tests (relative L2 1e-5), on calls made back to back, so that the second call
runs on the scratch the first one left behind.

The file name makes pytest collect it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

TOL_FP32 = 1e-5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_rejects_sizes_beyond_the_scratch_without_a_gpu():
    """The size checks run before any CUDA call (fake, aligned pointers are never touched)."""
    from paper_2510_19542_gb300 import safr
    lib = safr.load()
    fake = 1 << 20
    # 35 layers on a 512 grid need 35 * 256 * 512 * 8 B = 36.7 MB of layer spectra: more than 8 MiB
    st = lib.safr_reconstruct_noalloc(0, 512, 512, 35, 3, fake, fake, fake, fake, None)
    assert st == safr.SAFR_ERR_UNSUPPORTED_SIZE
    assert lib.safr_reconstruct_noalloc(0, 48, 8, 3, 3, fake, fake, fake, fake, None) == \
        safr.SAFR_ERR_UNSUPPORTED_SIZE                                   # M not a power of two
    assert lib.safr_reconstruct_noalloc(0, 64, 8, 3, 3, None, fake, fake, fake, None) == safr.SAFR_ERR_INVALID_ARG
    assert lib.safr_reconstruct_noalloc(0, 64, 8, 3, 3, fake + 4, fake, fake, fake, None) == \
        safr.SAFR_ERR_MISALIGNED


def _kernel_order(B):
    """B from safr_copy_B (natural j, last axis) in the frame kernel's frequency
    order along j: pos(j) = (j mod R) * LW + brev(j div R), LW = min(M, 32),
    R = M / LW, brev reversing log2(LW) bits."""
    M = B.shape[-1]
    LW = min(M, 32)
    R, bits = M // LW, LW.bit_length() - 1
    j = np.arange(M)
    m = j // R
    brev = np.zeros_like(m)
    for i in range(bits):
        brev |= ((m >> i) & 1) << (bits - 1 - i)
    out = np.empty_like(B)
    out[..., (j % R) * LW + brev] = B
    return out


def _geometries(synth):
    ngs = dict(synth.scaled(synth.config(3), M=256, P=256, L=9), precision="fp32")
    tiny = dict(synth.config(1), precision="fp32")
    base = synth.scaled(synth.config(2), M=64, P=20)
    lgs = [i for i in range(9) if base["kind"][i] == 1]
    lgs_native = dict(base, dir_x=base["dir_x"][lgs], dir_y=base["dir_y"][lgs], kind=base["kind"][lgs],
                      output_metric=0)
    # 512 grid with 16 stars: B (64 rows of 4 KB per column) is too large to stage in shared memory, the
    # case where the persistent kernel could take two phase-2 columns per pass; the entry point lays out
    # shared memory for the one-column kernel it launches.  Scratch: 16 * 256 * 64 * 8 B of row spectra
    # and 4 * 256 * 512 * 8 B of layer spectra fit in 8 MiB.
    az = np.deg2rad(22.5 * np.arange(16))
    ngs512 = dict(synth.scaled(synth.config(3), M=512, P=64, L=4), precision="fp32",
                  dir_x=2.9e-4 * np.cos(az), dir_y=2.9e-4 * np.sin(az), kind=np.zeros(16, np.int32))
    return [("ngs-256-L9", ngs), ("tiny-ngs-32", tiny), ("lgs-64-native", lgs_native), ("ngs-512-L4-G16", ngs512)]


@pytest.mark.gpu
def test_noalloc_matches_plan_entry_point_on_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    safr.load()
    dev = torch.device("cuda:0")
    for name, g in _geometries(synth):
        plan = safr.Plan(g, device=0, path=safr.SAFR_PATH_FUSED)
        info = plan.info
        assert info["ngroups"] == 1
        M, P, L, G = info["M"], info["P"], info["L"], info["G"]
        # B of the single group, [k][l][g][j], rounded to FP32 like the plan's own copy
        B = torch.from_numpy(np.ascontiguousarray(_kernel_order(safr.safr_copy_B(plan.handle, 0)).astype(np.complex64)))
        B = B.to(dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        for seed in (21, 22):  # two calls in a row on the shared scratch
            x = torch.from_numpy(synth.random_frame(g, seed).astype(np.float32)).to(dev)
            ref = plan.reconstruct(x).double().cpu().numpy()
            out = torch.full((L, M, M), float("nan"), dtype=torch.float32, device=dev)
            safr.safr_reconstruct_noalloc(0, M, P, L, G, B, x, out, status)
            torch.cuda.synchronize(dev)
            assert int(status.item()) == 0, (name, seed)
            got = out.double().cpu().numpy()
            assert np.all(np.isfinite(got)), (name, seed)
            assert _rel(got, ref) <= TOL_FP32, (name, seed, _rel(got, ref))
        assert safr.safr_get_status(plan.handle) == 0
        plan.close()
