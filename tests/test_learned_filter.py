"""Learned spectral filter on the GPU (through the C ABI) against the FP64 oracle.

Inference: B built by safr_filter_apply from seeded parameters (rounded to
BF16, so both sides use identical values) against the oracle's
group_B_learned; the MLP runs in FP32 on the GPU and B is stored in FP32, so
the bar is a max error of 2e-5 of max|B|.  Training: the held-out error of
plain SAFR that safr_filter_train reports is recomputed by the oracle on the
same Philox frames, built through the pupil (relative 1e-4), and so is the
learned filter's, from the parameters the call returns.  The fallback: non-finite MLP output or a learned
filter that does not beat plain SAFR leaves plain SAFR's B in the plan.
"""
import math

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


def bf16(x):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy()


def seeded_params(seed, gain=1.0):
    rng = np.random.default_rng(seed)
    H = 64
    parts = [rng.standard_normal(H * 4) * gain / 2.0, rng.standard_normal(H) * 0.1,
             rng.standard_normal(H * H) * gain / 8.0, rng.standard_normal(H) * 0.1,
             rng.standard_normal(H * H) * gain / 8.0, rng.standard_normal(H) * 0.1,
             rng.standard_normal(H) * gain / 8.0, rng.standard_normal(1) * 0.1]
    return bf16(np.concatenate(parts))


def oracle_args(g):
    M = g["M"]
    T = M * g["pitch"] / 2.0
    cn2 = np.asarray(g["cn2"], np.float64)
    return dict(M=M, T=T, h=np.asarray(g["h"], np.float64), c=np.ones(len(g["h"])), gamma=cn2 / cn2.sum(),
                ax=np.asarray(g["dir_x"], np.float64), ay=np.asarray(g["dir_y"], np.float64))


def oracle_learned_B(oracle_mod, g, params, noise):
    a = oracle_args(g)
    return oracle_mod.group_B_learned(a["M"], a["T"], a["h"], a["c"], a["gamma"], a["ax"], a["ay"], g["beta"],
                                      params.astype(np.float64), noise)


def as_gpu_layout(Bo):
    """oracle [j][k][l][g] over the full spectrum -> safr_copy_B's [k < M/2][l][g][j]."""
    M = Bo.shape[0]
    return np.transpose(Bo[:, :M // 2], (1, 2, 3, 0))


def frames_loss(oracle_mod, g, B, r0, L0, noise, key, nframes):
    a = oracle_args(g)
    return oracle_mod.filter_frames_loss(a["M"], a["T"], a["h"], a["c"], a["gamma"], a["ax"], a["ay"], B, g["P"],
                                         g.get("diameter", 0.0), g.get("obstruction", 0.0), r0, L0, noise, key, 0,
                                         nframes, nframes)


def test_apply_matches_oracle(safr, synth, oracle_mod):
    g = synth.config(5)
    plan = safr.Plan(g, device=0)
    for seed, noise in [(1, 0.01), (2, 0.05)]:
        p = seeded_params(seed)
        safr.safr_filter_apply(plan.handle, p, noise)
        Bg = safr.safr_copy_B(plan.handle, 0)
        Bo = as_gpu_layout(oracle_learned_B(oracle_mod, g, p, noise))
        err = np.abs(Bg - Bo).max() / np.abs(Bo).max()
        assert err <= 2e-5, (seed, err)
        assert np.all(Bg[..., g["M"] // 2] == 0)
    assert safr.safr_get_status(plan.handle) == 0
    plan.close()


def test_frames_with_learned_B_match_oracle_composition(safr, synth, oracle_mod):
    """Layers from the unchanged frame kernels with a learned B equal
    IDFT2(sum_g B_lg DFT2(psi_g)) (Algorithm 1) built from oracle routines."""
    g = synth.config(5)
    plan = safr.Plan(g, device=0)
    p = seeded_params(3)
    safr.safr_filter_apply(plan.handle, p, 0.01)
    x = synth.frame(g)
    got = plan.reconstruct(torch.from_numpy(x.astype(np.float32)).cuda()).double().cpu().numpy()
    Bo = oracle_learned_B(oracle_mod, g, p, 0.01)            # [j][k][l][g]
    d = np.stack([oracle_mod.dft2(x[i]) for i in range(x.shape[0])])  # [g][j][k]
    b = np.einsum("jklg,gjk->ljk", Bo, d)
    ref = np.stack([oracle_mod.idft2(b[l]).real for l in range(b.shape[0])])
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    plan.close()


def test_reset_and_nonfinite_fallback(safr, synth):
    g = synth.config(5)
    plan = safr.Plan(g, device=0)
    B0 = safr.safr_copy_B(plan.handle, 0)
    safr.safr_filter_apply(plan.handle, seeded_params(4), 0.01)
    assert not np.array_equal(safr.safr_copy_B(plan.handle, 0), B0)
    safr.safr_filter_reset(plan.handle)
    assert np.array_equal(safr.safr_copy_B(plan.handle, 0), B0)
    # parameters that make the MLP overflow to inf - inf = NaN: plain SAFR stays, SAFR_ERR_DEVICE
    p = np.zeros(safr.SAFR_FILTER_PARAMS, np.float32)
    p[:256] = 3.0e38                                    # W0: every hidden unit of layer 1 -> +inf
    W1 = np.full((64, 64), 3.0e38, np.float32)
    W1[:, 1::2] *= -1                                  # inf - inf in layer 2
    p[256 + 64:256 + 64 + 4096] = W1.ravel()
    safr.safr_filter_apply(plan.handle, seeded_params(5), 0.01)
    with pytest.raises(safr.SafrError) as ei:
        safr.safr_filter_apply(plan.handle, p, 0.01)
    assert ei.value.status == safr.SAFR_ERR_DEVICE
    assert np.array_equal(safr.safr_copy_B(plan.handle, 0), B0)
    bad = seeded_params(6)
    bad[10] = np.nan
    with pytest.raises(safr.SafrError) as ei:
        safr.safr_filter_apply(plan.handle, bad, 0.01)
    assert ei.value.status == safr.SAFR_ERR_INVALID_ARG
    plan.close()


def test_split_plans_are_refused(safr, synth):
    g = synth.scaled(synth.config(2), M=32, P=10)  # LGS + NGS: two star groups
    plan = safr.Plan(g, device=0)
    with pytest.raises(safr.SafrError) as ei:
        safr.safr_filter_apply(plan.handle, seeded_params(1), 0.01)
    assert ei.value.status == safr.SAFR_ERR_UNSUPPORTED_SIZE
    plan.close()


@pytest.mark.parametrize("alpha_scale", [1.0, 300.0])
def test_training_against_oracle(safr, synth, oracle_mod, alpha_scale):
    """A short run: the training error falls, the reported held-out errors are
    the oracle's on the same frames, and B is the learned one exactly when it
    won.  With alpha 300x too large plain SAFR is badly over-regularised and
    the learned filter must win."""
    g = dict(synth.config(5), alpha=synth.config(5)["alpha"] * alpha_scale)
    plan = safr.Plan(g, device=0)
    B0 = safr.safr_copy_B(plan.handle, 0)
    seed, nv, noise = 9, 512, 0.01
    w, res = safr.safr_filter_train(plan.handle, r0=0.15, L0=25.0, noise_level=noise, train_frames=4096,
                                    valid_frames=nv, epochs=3, lr=3e-3, seed=seed)
    assert res["nonfinite"] == 0 and res["steps"] == 3 * 16
    assert all(math.isfinite(res[k]) for k in ("train_loss_first", "train_loss_last", "valid_loss_learned",
                                                "valid_loss_plain"))
    assert res["train_loss_last"] < res["train_loss_first"]
    key = (seed + 1, (seed >> 32) ^ 0x5AFE)                 # held-out key
    Bp = oracle_mod.OraclePlan(g).group(0)[3]
    lp, ep = frames_loss(oracle_mod, g, Bp, 0.15, 25.0, noise, key, nv)
    assert abs(lp / ep / res["valid_loss_plain"] - 1) <= 1e-4, (lp / ep, res["valid_loss_plain"])
    Bl = oracle_learned_B(oracle_mod, g, w, noise)
    ll, el = frames_loss(oracle_mod, g, Bl, 0.15, 25.0, noise, key, nv)
    assert abs(ll / el / res["valid_loss_learned"] - 1) <= 1e-3, (ll / el, res["valid_loss_learned"])
    Bg = safr.safr_copy_B(plan.handle, 0)
    if res["used_learned"]:
        assert res["valid_loss_learned"] < res["valid_loss_plain"]
        assert np.abs(Bg - as_gpu_layout(Bl)).max() <= 2e-5 * np.abs(Bg).max()
    else:
        assert np.array_equal(Bg, B0)
    if alpha_scale > 1:
        assert res["used_learned"] == 1
    assert safr.safr_get_status(plan.handle) == 0
    plan.close()
