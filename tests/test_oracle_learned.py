"""Pins of the learned spectral filter's oracle routines (CPU only).

The learned filter replaces Section 3.1's Tikhonov factor g(s) = s / (s^2 +
alpha) by phi / s, phi from an MLP.  Each check reaches its expected value by
another route than the oracle's own code: a library pseudo-inverse and SVD
(numpy/LAPACK), a closed form of a network with one active path, published
generator vectors, an exact identity (zero reconstruction, exact inverse of
noise-free data) or a statistical expectation of the frame generator.
"""
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
H = 64


def _params(**entries):
    """Parameter vector (layout W0[64][4] b0 W1[64][64] b1 W2[64][64] b2 W3[64] b3)
    with the named single entries set: W0=(i, q, v), W1=(i, j, v), W2=(i, j, v), W3=(j, v), b3=v."""
    p = np.zeros(4 * H + H + 2 * (H * H + H) + H + 1)
    oW0, ob0 = 0, 4 * H
    oW1 = ob0 + H
    ob1 = oW1 + H * H
    oW2 = ob1 + H
    ob2 = oW2 + H * H
    oW3 = ob2 + H
    ob3 = oW3 + H
    for i, q, v in entries.get("W0", []):
        p[oW0 + i * 4 + q] = v
    for i, j, v in entries.get("W1", []):
        p[oW1 + i * H + j] = v
    for i, j, v in entries.get("W2", []):
        p[oW2 + i * H + j] = v
    for j, v in entries.get("W3", []):
        p[oW3 + j] = v
    p[ob3] = entries.get("b3", 0.0)
    return p


def _gelu(z):
    return 0.5 * z * (1.0 + math.erf(z / math.sqrt(2.0)))


def _one_path(q, a=3, b=5, c=7):
    """phi(x) = logistic(gelu(gelu(gelu(x_q)))) through hidden units a, b, c."""
    return _params(W0=[(a, q, 1.0)], W1=[(b, a, 1.0)], W2=[(c, b, 1.0)], W3=[(c, 1.0)])


def test_philox_known_answer_vectors(oracle_mod):
    kat = json.load(open(os.path.join(HERE, "golden", "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        ctr = [int(w, 16) for w in v["ctr"]]
        key = [int(w, 16) for w in v["key"]]
        out = [int(w, 16) for w in v["out"]]
        assert list(oracle_mod.philox4x32_10(ctr, key)) == out


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_mlp_single_path_closed_form(oracle_mod, q):
    """Row-major W[out][in], layer order and the exact (erf) GELU: a network with
    one active path through off-diagonal entries has a closed form."""
    p = _one_path(q)
    rng = np.random.default_rng(q)
    for _ in range(5):
        x = rng.uniform(-2, 2, 4)
        z = _gelu(_gelu(_gelu(x[q])))
        assert abs(oracle_mod.mlp_phi(p, x) - 1.0 / (1.0 + math.exp(-z))) < 1e-15
    # transposing any weight matrix breaks the path: phi = logistic(0) = 1/2
    bad = _params(W0=[(q, 3, 1.0)], W1=[(3, 5, 1.0)], W2=[(5, 7, 1.0)], W3=[(7, 1.0)]) if q != 3 else None
    if bad is not None:
        assert oracle_mod.mlp_phi(bad, np.full(4, 0.7)) != oracle_mod.mlp_phi(p, np.full(4, 0.7))


def _geometry(G, L, M=8, seed=0):
    rng = np.random.default_rng(seed)
    T = 4.0
    h = np.sort(rng.uniform(0, 15e3, L))
    h[0] = 0.0
    gamma = rng.uniform(0.1, 1.0, L)
    gamma /= gamma.sum()
    ax = rng.uniform(-3e-4, 3e-4, G)
    ay = rng.uniform(-3e-4, 3e-4, G)
    return dict(M=M, T=T, h=h, c=np.ones(L), gamma=gamma, ax=ax, ay=ay, beta=1.5)


def _A(g, j, k):
    """A_n[g][l] = s_l(n) exp(i pi n.(alpha_g h_l) / (c_l T)) (Section 3.1)."""
    M, T = g["M"], g["T"]
    nx = j if j < M // 2 else j - M
    ny = k if k < M // 2 else k - M
    tau = math.pi ** 2 / (g["c"] * T) ** 2
    s = np.sqrt(g["gamma"]) / g["c"] * (1 + tau * (nx * nx + ny * ny)) ** (-g["beta"] / 2)
    th = math.pi / T * (nx * np.outer(g["ax"], g["h"]) + ny * np.outer(g["ay"], g["h"])) / g["c"][None, :]
    return s, s[None, :] * np.exp(1j * th)


def _learned(oracle_mod, g, p, noise):
    return oracle_mod.group_B_learned(g["M"], g["T"], g["h"], g["c"], g["gamma"], g["ax"], g["ay"], g["beta"], p,
                                      noise)


@pytest.mark.parametrize("G,L", [(4, 3), (3, 5), (3, 3)])
def test_learned_B_with_phi_one_is_the_pseudo_inverse(oracle_mod, G, L):
    """phi = 1 (logistic(40) rounds to 1): B_n = diag(s) A_n^+ with A_n^+ from
    LAPACK's SVD, singular values below 1e-13 sigma_max dropped on both sides."""
    g = _geometry(G, L, seed=G * 10 + L)
    p = _params(b3=40.0)
    assert oracle_mod.mlp_phi(p, np.zeros(4)) == 1.0
    B = _learned(oracle_mod, g, p, 0.01)
    M = g["M"]
    for j in range(M):
        for k in range(M):
            if j == M // 2 or k == M // 2:
                assert np.all(B[j, k] == 0)
                continue
            s, A = _A(g, j, k)
            ref = s[:, None] * np.linalg.pinv(A, rcond=1e-13)
            assert np.max(np.abs(B[j, k] - ref)) <= 1e-10 * np.max(np.abs(ref)), (j, k)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_learned_B_feature_dependence(oracle_mod, q):
    """phi depending on |n| (q=0), on the layer height (q=1) or on sigma_r (q=2)
    through the one-path network: B_n[l] = s_l sum_r V_lr phi(x_q) / sigma_r
    conj(U_gr) with U, sigma, V from numpy's SVD and the features
    (|n| / (M/2), h_l / 20 km, (log10 sigma_r + 4) / 4, noise / 0.05)."""
    g = _geometry(4, 3, seed=7)
    p = _one_path(q)
    B = _learned(oracle_mod, g, p, 0.02)
    M = g["M"]

    def phi(x):
        z = _gelu(_gelu(_gelu(x)))
        return 1.0 / (1.0 + math.exp(-z))

    for j, k in [(1, 0), (0, 3), (2, 5), (7, 6), (3, 1)]:
        s, A = _A(g, j, k)
        U, S, Vh = np.linalg.svd(A, full_matrices=False)
        V = Vh.conj().T
        nx = j if j < M // 2 else j - M
        ny = k if k < M // 2 else k - M
        ref = np.zeros((len(s), A.shape[0]), complex)
        for l in range(len(s)):
            for r in range(len(S)):
                if S[r] <= 1e-13 * S.max():
                    continue
                x = [math.hypot(nx, ny) / (M / 2), g["h"][l] / 20e3, (math.log10(max(S[r], 1e-12)) + 4) / 4,
                     0.02 / 0.05][q]
                ref[l] += s[l] * V[l, r] * phi(x) / S[r] * U[:, r].conj()
        assert np.max(np.abs(B[j, k] - ref)) <= 1e-10 * np.max(np.abs(ref)), (j, k)


def _frames_loss(oracle_mod, g, B, noise, nframes, key=(11, 22), P=None, D=0.0, obstruction=0.0):
    """Loss over nframes training frames; by default no aperture (P = M, D = 0)."""
    return oracle_mod.filter_frames_loss(g["M"], g["T"], g["h"], g["c"], g["gamma"], g["ax"], g["ay"], B,
                                         P or g["M"], D, obstruction, 0.15, 25.0, noise, key, 0, 1 << 20, nframes)


def _frame(oracle_mod, g, F, noise, P=None, D=0.0, obstruction=0.0, key=(5, 6)):
    return oracle_mod.filter_frame(g["M"], g["T"], g["h"], g["c"], g["gamma"], g["ax"], g["ay"], P or g["M"], D,
                                   obstruction, 0.15, 25.0, noise, key, F)


def test_frames_zero_reconstruction_loses_all_energy(oracle_mod):
    g = _geometry(3, 4, M=16, seed=3)
    B = np.zeros((16, 16, 4, 3), complex)
    loss, energy = _frames_loss(oracle_mod, g, B, 0.05, 6)
    assert energy > 0 and loss == energy


def test_frames_exact_inverse_recovers_noise_free_layers(oracle_mod):
    """G >= L, full column rank: B = diag(s) A^+ = the left inverse of the frames'
    phase matrix e^{i theta}, so noise-free frames are reconstructed exactly.
    A sign or index slip in the frames' phases breaks this."""
    g = _geometry(5, 3, M=16, seed=4)
    B = _learned(oracle_mod, g, _params(b3=40.0), 0.0)
    loss, energy = _frames_loss(oracle_mod, g, B, 0.0, 4)
    assert energy > 0 and loss <= 1e-20 * energy


def _von_karman_energy(g, r0=0.15, L0=25.0):
    """Expected sum over the full spectrum of E|phi_l(n)|^2: DFT of a real von
    Karman screen (PSD 0.023 r0_l^-5/3 (f^2 + L0^-2)^-11/6, r0_l = r0 gamma_l^-3/5)
    with half the power per complex coefficient, sampled at pitch 2 c_l T / M."""
    M, T = g["M"], g["T"]
    tot = 0.0
    for l in range(len(g["h"])):
        per = 2 * g["c"][l] * T
        r0l = r0 * g["gamma"][l] ** (-0.6)
        for j in range(M):
            for k in range(M // 2):
                if j == M // 2 or (j == 0 and k == 0):
                    continue
                nx = j if j < M // 2 else j - M
                f2 = (nx * nx + k * k) / per ** 2
                psd = 0.023 * r0l ** (-5 / 3) * (f2 + L0 ** -2) ** (-11 / 6)
                tot += (1 if k == 0 else 2) * M ** 4 * 0.5 * psd / per ** 2
    return tot


def test_frames_energy_and_noise_statistics(oracle_mod):
    """Mean frame energy matches the von Karman expectation, and the error of an
    exact inverse on noisy frames matches E|B eta|^2 = noise^2 E_f / M^2 sum_n w_n ||B_n||_F^2
    (statistical: 400 frames, a few percent)."""
    g = _geometry(5, 3, M=16, seed=5)
    M = g["M"]
    B = _learned(oracle_mod, g, _params(b3=40.0), 0.0)
    nf, nu = 400, 0.1
    loss, energy = _frames_loss(oracle_mod, g, B, nu, nf)
    Ef = _von_karman_energy(g)
    assert abs(energy / nf / Ef - 1) < 0.03
    fro = 0.0
    for j in range(M):
        for k in range(M // 2):
            if j == M // 2:
                continue
            fro += (1 if k == 0 else 2) * np.sum(abs(B[j, k]) ** 2)
    expect = nu ** 2 * Ef / M ** 2 * fro
    assert abs(loss / nf / expect - 1) < 0.05


def test_frame_layers_are_real_screens(oracle_mod):
    """phi_l(-n) = conj(phi_l(n)) on the stored row k = 0; nothing at n = 0 or on the Nyquist row."""
    g = _geometry(3, 4, M=16, seed=8)
    phi, _ = _frame(oracle_mod, g, 3, 0.0)
    M = g["M"]
    for j in range(1, M // 2):
        assert np.array_equal(phi[0, M - j], phi[0, j].conj())
    assert np.all(phi[0, 0] == 0) and np.all(phi[:, M // 2] == 0)
    assert np.all(np.abs(phi[1:, 1]) > 0)


def test_frame_data_without_aperture_is_the_layered_model(oracle_mod):
    """No aperture, no noise: d_g(n) = sum_l exp(i pi n.(alpha_g h_l) / (c_l T)) phi_l(n)
    (Section 2 in the Fourier domain) and the wavefront numpy's ifft2 gives is real."""
    g = _geometry(3, 4, M=16, seed=9)
    M = g["M"]
    phi, d = _frame(oracle_mod, g, 7, 0.0)
    for j in range(M):
        for k in range(1, M // 2):
            if j == M // 2:
                continue
            s, A = _A(g, j, k)
            ref = (A / s[None, :]) @ phi[k, j]
            assert np.max(np.abs(d[:, j, k] - ref)) <= 1e-9 * np.max(np.abs(ref))
    for gi in range(3):
        w = np.fft.ifft2(d[gi])
        assert np.max(np.abs(w.imag)) <= 1e-12 * np.max(np.abs(w.real))


def test_frame_aperture_and_noise(oracle_mod):
    """With a pupil (P < M, annulus of diameter D): numpy's ifft2 of d is real,
    zero off the pupil (the mask of synth.pupil placed at (M-P)/2), and equals
    the aperture-free wavefront on it.  With noise, the difference is white
    noise on the pupil only, of std noise x RMS of the noise-free wavefront."""
    from paper_2510_19542_gb300 import synth
    g = _geometry(3, 4, M=32, seed=10)
    M, P, D, obs = g["M"], 28, 6.5, 0.1
    pitch = 2 * g["T"] / M
    pm = synth.pupil(dict(P=P, pitch=pitch, diameter=D, obstruction=obs))
    mask = np.zeros((M, M), bool)
    o = (M - P) // 2
    mask[o:o + P, o:o + P] = pm
    _, d_free = _frame(oracle_mod, g, 4, 0.0)
    _, d_clean = _frame(oracle_mod, g, 4, 0.0, P=P, D=D, obstruction=obs)
    _, d_noisy = _frame(oracle_mod, g, 4, 0.2, P=P, D=D, obstruction=obs)
    for gi in range(3):
        free = np.fft.ifft2(d_free[gi]).real
        clean = np.fft.ifft2(d_clean[gi])
        noisy = np.fft.ifft2(d_noisy[gi])
        scale = np.max(np.abs(free))
        assert np.max(np.abs(clean.imag)) <= 1e-12 * scale and np.max(np.abs(noisy.imag)) <= 1e-12 * scale
        assert np.max(np.abs(clean.real - free * mask)) <= 1e-12 * scale
        eta = noisy.real - clean.real
        assert np.max(np.abs(eta[~mask])) <= 1e-12 * scale
        rms = np.sqrt(np.mean(free[mask] ** 2))
        assert abs(np.std(eta[mask]) / rms / 0.2 - 1) < 0.1
        assert abs(np.mean(eta[mask])) < 0.15 * 0.2 * rms


def test_frames_loss_sums_the_frames(oracle_mod):
    """The loss of two frames is the weighted squared error of B d against phi
    over the stored frequencies (k = 0 weight 1, k > 0 weight 2, no Nyquist row)."""
    g = _geometry(3, 4, M=16, seed=11)
    M = g["M"]
    B = _learned(oracle_mod, g, _one_path(2), 0.01)
    loss, energy = _frames_loss(oracle_mod, g, B, 0.05, 2, key=(5, 6), P=14, D=3.5)
    tl = te = 0.0
    for F in range(2):
        phi, d = _frame(oracle_mod, g, F, 0.05, P=14, D=3.5)
        for k in range(M // 2):
            for j in range(M):
                if j == M // 2:
                    continue
                wn = 1 if k == 0 else 2
                e = B[j, k] @ d[:, j, k] - phi[k, j]
                tl += wn * np.sum(abs(e) ** 2)
                te += wn * np.sum(abs(phi[k, j]) ** 2)
    assert abs(loss / tl - 1) < 1e-12 and abs(energy / te - 1) < 1e-12
