"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks re-types the oracle's own formulas: each one reaches the
expected value by another route (direct definition sums on tiny inputs, a
library routine, a closed form, an invariant, or the dense spatial-domain
Tikhonov solve in dense_tikhonov.py).
"""
import cmath
import json
import math
import os

import numpy as np
import pytest

import dense_tikhonov as dt

HERE = os.path.dirname(os.path.abspath(__file__))


# --------------------------------------------------------------------------
# DFT2 / IDFT2 (Section 3.2)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("M", [4, 6])
def test_dft2_matches_direct_definition(oracle_mod, M):
    """Brute-force four-fold sum of the DFT2 definition, in pure Python."""
    rng = np.random.default_rng(M)
    X = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    Y = oracle_mod.dft2(X)
    Z = oracle_mod.idft2(X)
    for j in range(M):
        for k in range(M):
            s = sum(X[p, q] * cmath.exp(-2j * math.pi * (j * p + k * q) / M)
                    for p in range(M) for q in range(M))
            t = sum(X[p, q] * cmath.exp(2j * math.pi * (j * p + k * q) / M)
                    for p in range(M) for q in range(M)) / M ** 2
            assert abs(Y[j, k] - s) < 1e-12
            assert abs(Z[j, k] - t) < 1e-13


@pytest.mark.parametrize("M", [8, 16, 32])
def test_dft2_library_parseval_shift(oracle_mod, M):
    rng = np.random.default_rng(M)
    X = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    Y = oracle_mod.dft2(X)
    np.testing.assert_allclose(Y, np.fft.fft2(X), rtol=0, atol=1e-12 * M * M)
    # Parseval
    assert abs(np.sum(abs(X) ** 2) - np.sum(abs(Y) ** 2) / M ** 2) < 1e-12 * np.sum(abs(X) ** 2)
    # inverse
    np.testing.assert_allclose(oracle_mod.idft2(Y), X, rtol=0, atol=1e-13)
    # shift theorem: DFT2(roll(X, (a, b)))(j, k) = e^{-2 pi i (ja + kb)/M} DFT2(X)(j, k)
    a, b = 3, M - 2
    j = np.arange(M)
    ph = np.exp(-2j * math.pi * (np.outer(j, np.ones(M)) * a + np.outer(np.ones(M), j) * b) / M)
    np.testing.assert_allclose(oracle_mod.dft2(np.roll(X, (a, b), axis=(0, 1))), ph * Y,
                               rtol=0, atol=1e-11 * M)


# --------------------------------------------------------------------------
# Jacobi SVD (Algorithm 2 step 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(3, 3), (6, 9), (9, 6), (3, 35), (35, 3), (1, 5), (5, 1), (9, 9)])
def test_jacobi_svd(oracle_mod, shape):
    rng = np.random.default_rng(sum(shape))
    A = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    U, S, V, sweeps = oracle_mod.svd(A)
    assert sweeps < 100
    np.testing.assert_allclose(U @ np.diag(S) @ V.conj().T, A, rtol=0, atol=1e-13 * np.abs(A).max())
    np.testing.assert_allclose(V.conj().T @ V, np.eye(shape[1]), atol=1e-13)
    big = S > 1e-12 * S.max()
    Ub = U[:, big]
    np.testing.assert_allclose(Ub.conj().T @ Ub, np.eye(big.sum()), atol=1e-13)
    ref = np.linalg.svd(A, compute_uv=False)  # LAPACK, an independent routine
    np.testing.assert_allclose(np.sort(S)[::-1][:len(ref)], ref, rtol=1e-13, atol=1e-13 * ref[0])


def test_jacobi_svd_rank_deficient(oracle_mod):
    rng = np.random.default_rng(7)
    u = rng.standard_normal((6, 1)) + 1j * rng.standard_normal((6, 1))
    v = rng.standard_normal((1, 4)) + 1j * rng.standard_normal((1, 4))
    A = u @ v
    U, S, V, _ = oracle_mod.svd(A)
    np.testing.assert_allclose(U @ np.diag(S) @ V.conj().T, A, atol=1e-13 * np.abs(A).max())
    s = np.sort(S)[::-1]
    assert abs(s[0] - np.linalg.norm(u) * np.linalg.norm(v)) < 1e-12 * s[0]
    assert np.all(s[1:] < 1e-13 * s[0])


# --------------------------------------------------------------------------
# B (Algorithm 2): closed forms and identities
# --------------------------------------------------------------------------
def _geometry(rng, L, G, lgs, M=16, pitch=0.5):
    h = np.sort(rng.uniform(0, 15000, L))
    h[0] = 0.0
    cn2 = rng.uniform(0.2, 1.0, L)
    dx = rng.uniform(-1, 1, G) * 3e-4
    dy = rng.uniform(-1, 1, G) * 3e-4
    return dict(M=M, P=M, pitch=pitch, diameter=0.0, obstruction=0.0, h=h, cn2=cn2,
                dir_x=dx, dir_y=dy, kind=np.full(G, lgs, np.int32), h_lgs=90e3,
                alpha=0.05, alpha_tt=0.05, beta=1.5, output_metric=0, remove_tt=0)


@pytest.mark.parametrize("L,G,lgs", [(3, 3, 0), (9, 6, 1), (4, 9, 1), (35, 3, 0)])
def test_B_dc_closed_form(oracle_mod, L, G, lgs):
    """n = 0: A(0) = 1_G s^T has rank one, so by Sherman-Morrison
    B_lg(0) = s_l^2 / (G sum_l' s_l'^2 + alpha) with s_l(0) = gamma_l^{1/2} / c_l."""
    rng = np.random.default_rng(L * 100 + G)
    g = _geometry(rng, L, G, lgs)
    gam = g["cn2"] / g["cn2"].sum()
    c = 1 - g["h"] / 90e3 if lgs else np.ones(L)
    T = g["M"] * g["pitch"] / 2
    B = oracle_mod.group_B(g["M"], T, g["h"], c, gam, g["dir_x"], g["dir_y"], g["alpha"], g["beta"])
    s2 = gam / c ** 2
    expect = np.repeat((s2 / (G * s2.sum() + g["alpha"]))[:, None], G, axis=1)
    np.testing.assert_allclose(B[0, 0], expect, rtol=1e-12, atol=1e-15)


def test_B_single_layer_closed_form(oracle_mod):
    """L = 1: A(n) = s e^{i theta_g} is a column, B_g = s^2 e^{-i theta_g} / (G s^2 + alpha).
    theta_g is the Fourier shift of the layer as seen from star g."""
    M, pitch = 16, 0.5
    T = M * pitch / 2
    h = np.array([7000.0])
    gam = np.array([1.0])
    c = 1 - h / 90e3
    dx = np.array([1e-4, -2.5e-4, 3e-4])
    dy = np.array([2e-4, 0.5e-4, -1e-4])
    alpha, beta = 0.02, 1.5
    B = oracle_mod.group_B(M, T, h, c, gam, dx, dy, alpha, beta)
    j = np.arange(M)
    lab = np.where(j < M // 2, j, j - M)
    for jj in range(M):
        for kk in range(M):
            if jj == M // 2 or kk == M // 2:
                continue
            nx, ny = lab[jj], lab[kk]
            # layer shift in layer pixels, seen in the Fourier series of period 2 c T
            s = (1.0 / c[0]) * (1 + (math.pi / (c[0] * T)) ** 2 * (nx * nx + ny * ny)) ** (-beta / 2)
            theta = 2 * math.pi * (nx * dx * h[0] + ny * dy * h[0]) / (c[0] * M * pitch)
            expect = s * s * np.exp(-1j * theta) / (3 * s * s + alpha)
            np.testing.assert_allclose(B[jj, kk, 0], expect, rtol=1e-12, atol=1e-15)


def test_B_nyquist_and_hermitian(oracle_mod):
    rng = np.random.default_rng(11)
    g = _geometry(rng, 5, 4, 1)
    M = g["M"]
    T = M * g["pitch"] / 2
    c = 1 - g["h"] / 90e3
    B = oracle_mod.group_B(M, T, g["h"], c, g["cn2"] / g["cn2"].sum(), g["dir_x"], g["dir_y"], 0.01, 1.5)
    assert np.all(B[M // 2, :] == 0) and np.all(B[:, M // 2] == 0)
    neg = (-np.arange(M)) % M
    np.testing.assert_allclose(B[neg][:, neg], np.conj(B), rtol=0, atol=1e-13 * np.abs(B).max())


def test_B_tikhonov_identity(oracle_mod):
    """R_alpha(A) = V g_alpha(Sigma^T) U^H with the Tikhonov filter equals
    (A^H A + alpha I)^-1 A^H (Section 3.1); the right side is a LAPACK solve.
    As in the oracle's B, the Jacobi SVD runs on A when it has no more columns
    than rows and on A^H = V Sigma U^H otherwise."""
    rng = np.random.default_rng(3)
    alpha = 0.005
    for (m, n) in [(6, 9), (9, 6), (3, 35), (4, 4), (1, 7)]:
        A = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
        if m >= n:
            U, S, V, _ = oracle_mod.svd(A)
        else:
            V, S, U, _ = oracle_mod.svd(A.conj().T)
        filt = S / (S ** 2 + alpha)
        R = V @ np.diag(filt) @ U.conj().T
        # the smaller of the two equivalent linear systems keeps the reference accurate
        if m >= n:
            ref = np.linalg.solve(A.conj().T @ A + alpha * np.eye(n), A.conj().T)
        else:
            ref = A.conj().T @ np.linalg.inv(A @ A.conj().T + alpha * np.eye(m))
        np.testing.assert_allclose(R, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


# --------------------------------------------------------------------------
# Whole reconstruction vs the dense spatial-domain Tikhonov solve (main pin)
# --------------------------------------------------------------------------
DENSE_CASES = [
    # M, L, G, lgs, alpha, beta
    (8, 2, 3, 0, 0.05, 1.5),
    (8, 3, 2, 1, 0.005, 1.5),
    (16, 3, 3, 1, 0.005, 1.5),
    (16, 2, 4, 0, 0.01, 11.0 / 6.0),
    (16, 4, 2, 1, 0.1, 0.0),
]


@pytest.mark.parametrize("M,L,G,lgs,alpha,beta", DENSE_CASES)
def test_reconstruction_equals_dense_tikhonov(oracle_mod, M, L, G, lgs, alpha, beta):
    rng = np.random.default_rng(M * 1000 + L * 10 + G)
    g = _geometry(rng, L, G, lgs, M=M)
    g["alpha"] = alpha
    g["beta"] = beta
    psi = rng.standard_normal((G, M, M))
    ref, _, _ = dt.solve(M, g["pitch"], g["h"], g["cn2"], g["dir_x"], g["dir_y"], lgs, 90e3,
                         alpha, beta, psi)
    out, imag = oracle_mod.OraclePlan(g).reconstruct(psi, return_imag=True)
    assert np.abs(out - ref).max() <= 1e-10 * np.abs(ref).max()
    assert imag <= 1e-13 * np.abs(out).max()  # real output (Hermitian B, Nyquist zeroed)


def test_reconstruction_with_padding_equals_dense(oracle_mod):
    """P < M: the pupil is zero-extended to the periodic grid (Section 2)."""
    rng = np.random.default_rng(99)
    M, P, L, G = 16, 10, 3, 3
    g = _geometry(rng, L, G, 1, M=M)
    g["P"] = P
    psi = rng.standard_normal((G, P, P))
    pad = np.zeros((G, M, M))
    o = (M - P) // 2
    pad[:, o:o + P, o:o + P] = psi
    ref, _, _ = dt.solve(M, g["pitch"], g["h"], g["cn2"], g["dir_x"], g["dir_y"], 1, 90e3,
                         g["alpha"], g["beta"], pad)
    out = oracle_mod.OraclePlan(g).reconstruct(psi)
    assert np.abs(out - ref).max() <= 1e-10 * np.abs(ref).max()


def test_exact_recovery_as_alpha_to_zero(oracle_mod):
    """Noise-free data in the range of the operator: the data misfit vanishes
    as O(alpha) and the layers tend to the minimum-H^beta-norm solution."""
    rng = np.random.default_rng(21)
    M, L, G = 8, 3, 2
    g = _geometry(rng, L, G, 1, M=M)
    gam = g["cn2"] / g["cn2"].sum()
    c = 1 - g["h"] / 90e3
    A = dt.forward_operator(M, g["pitch"], g["h"], g["dir_x"], g["dir_y"], c)
    R = dt.penalty_operator(M, g["pitch"], c, gam, g["beta"])
    phi_true = rng.standard_normal(L * M * M)
    y = A @ phi_true
    # minimum-norm (in the R metric) solution of A phi = A phi_true, via LAPACK pinv
    w, Q = np.linalg.eigh(R)
    Rmh = Q @ np.diag(w ** -0.5) @ Q.T
    phi_star = Rmh @ np.linalg.pinv(A @ Rmh, rcond=1e-10) @ y
    res, err = [], []
    for alpha in (1e-8, 1e-10):
        g["alpha"] = alpha
        out = oracle_mod.OraclePlan(g).reconstruct(y.reshape(G, M, M))
        res.append(np.linalg.norm(A @ out.ravel() - y) / np.linalg.norm(y))
        err.append(np.linalg.norm(out.ravel() - phi_star) / np.linalg.norm(phi_star))
    # O(alpha) convergence: both errors shrink by the factor alpha shrinks by
    assert 50 < res[0] / res[1] < 200 and 50 < err[0] / err[1] < 200
    assert res[1] < 1e-6 and err[1] < 1e-5


def test_unit_gain_and_shift_theorem(oracle_mod):
    """G = L = 1, beta = 0, alpha -> 0: the layer is the wavefront moved back by the
    star's integer pixel shift, minus the wavefront's Nyquist components."""
    M, pitch = 16, 0.5
    rng = np.random.default_rng(4)
    psi = rng.standard_normal((1, M, M))
    F = np.fft.fft2(psi[0])
    F[M // 2, :] = 0
    F[:, M // 2] = 0
    band = np.fft.ifft2(F).real
    for (sx, sy) in [(0, 0), (3, -2), (5, 1)]:
        h = 10000.0
        g = dict(M=M, P=M, pitch=pitch, h=np.array([h]), cn2=np.array([1.0]),
                 dir_x=np.array([sx * pitch / h]), dir_y=np.array([sy * pitch / h]),
                 kind=np.zeros(1, np.int32), alpha=1e-13, beta=0.0, output_metric=0, remove_tt=0)
        out = oracle_mod.OraclePlan(g).reconstruct(psi)[0]
        # layer(x) = psi(x - alpha h): layer[p] = psi[p - s]
        np.testing.assert_allclose(out, np.roll(band, (sx, sy), axis=(0, 1)), atol=1e-10)


def test_translation_equivariance(oracle_mod):
    rng = np.random.default_rng(8)
    g = _geometry(rng, 3, 4, 1, M=16)
    psi = rng.standard_normal((4, 16, 16))
    pl = oracle_mod.OraclePlan(g)
    a = pl.reconstruct(psi)
    b = pl.reconstruct(np.roll(psi, (3, -5), axis=(1, 2)))
    np.testing.assert_allclose(b, np.roll(a, (3, -5), axis=(1, 2)), atol=1e-12 * np.abs(a).max())


def test_linearity(oracle_mod):
    rng = np.random.default_rng(9)
    g = _geometry(rng, 3, 3, 0, M=16)
    pl = oracle_mod.OraclePlan(g)
    x, y = rng.standard_normal((2, 3, 16, 16))
    np.testing.assert_allclose(pl.reconstruct(2.5 * x - 0.5 * y),
                               2.5 * pl.reconstruct(x) - 0.5 * pl.reconstruct(y), atol=1e-12)


# --------------------------------------------------------------------------
# removeTT and the metric resample
# --------------------------------------------------------------------------
def test_remove_tt_plane_and_orthogonality(oracle_mod):
    P, d = 24, 0.5
    mask = oracle_mod.pupil_mask(P, d, 11.5, 0.11)
    x = (np.arange(P) - (P - 1) / 2) * d
    X, Y = np.meshgrid(x, x, indexing="ij")
    plane = (0.7 + 1.3 * X - 0.4 * Y) * mask
    out, abc = oracle_mod.remove_tt(plane, d, mask)
    np.testing.assert_allclose(abc, [0.7, 1.3, -0.4], atol=1e-12)
    np.testing.assert_allclose(out, 0.7 * mask, atol=1e-12)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal((P, P)) * mask
    out, _ = oracle_mod.remove_tt(psi, d, mask)
    assert abs(np.sum(out * X * mask)) < 1e-10 and abs(np.sum(out * Y * mask)) < 1e-10
    np.testing.assert_array_equal(out[mask == 0], 0.0)
    assert abs(np.sum(out) - np.sum(psi)) < 1e-10  # piston kept (centred symmetric mask)


def test_resample_identity_and_ramp(oracle_mod):
    M = 32
    rng = np.random.default_rng(2)
    src = rng.standard_normal((M, M))
    np.testing.assert_array_equal(oracle_mod.resample(src, 1.0), src)
    i = np.arange(M, dtype=np.float64)
    ramp = 0.3 * i[:, None] - 1.7 * i[None, :]
    c = 0.85
    out = oracle_mod.resample(ramp, c)
    u = M / 2 + (i - M / 2) / c
    ok = (u >= 0) & (u < M - 1)  # away from the periodic seam
    expect = 0.3 * u[:, None] - 1.7 * u[None, :]
    np.testing.assert_allclose(out[np.ix_(ok, ok)], expect[np.ix_(ok, ok)], atol=1e-12)


def test_mixed_plan_is_sum_of_split_groups(oracle_mod):
    """Split tomography (Algorithm 3, line 4): LGS group after removeTT, resampled
    to the metric grid, plus the NGS group with alpha_TT."""
    rng = np.random.default_rng(31)
    M, P = 16, 12
    gl = _geometry(rng, 3, 3, 1, M=M)
    gl.update(P=P, diameter=P * gl["pitch"], obstruction=0.2, alpha=0.005)
    gn = dict(gl, dir_x=rng.uniform(-1, 1, 2) * 3e-4, dir_y=rng.uniform(-1, 1, 2) * 3e-4,
              kind=np.zeros(2, np.int32), alpha=0.01)
    mixed = dict(gl, dir_x=np.concatenate([gn["dir_x"][:1], gl["dir_x"], gn["dir_x"][1:]]),
                 dir_y=np.concatenate([gn["dir_y"][:1], gl["dir_y"], gn["dir_y"][1:]]),
                 kind=np.array([0, 1, 1, 1, 0], np.int32), alpha=0.005, alpha_tt=0.01,
                 output_metric=1, remove_tt=1)
    mask = oracle_mod.pupil_mask(P, gl["pitch"], gl["diameter"], 0.2)
    psi = rng.standard_normal((5, P, P)) * mask
    out = oracle_mod.OraclePlan(mixed).reconstruct(psi)
    lgs_in = np.stack([oracle_mod.remove_tt(psi[i], gl["pitch"], mask)[0] for i in (1, 2, 3)])
    lgs_native = oracle_mod.OraclePlan(dict(gl, output_metric=0)).reconstruct(lgs_in)
    c = 1 - gl["h"] / 90e3
    lgs_metric = np.stack([oracle_mod.resample(lgs_native[l], c[l]) for l in range(3)])
    ngs = oracle_mod.OraclePlan(gn).reconstruct(psi[[0, 4]])
    np.testing.assert_allclose(out, lgs_metric + ngs, atol=1e-12 * np.abs(out).max())


# --------------------------------------------------------------------------
# Paper parameters and the stored oracle regression values
# --------------------------------------------------------------------------
def test_paper_parameters_in_workloads():
    from paper_2510_19542_gb300 import synth
    with open(os.path.join(HERE, "golden", "paper_parameters.json")) as f:
        paper = json.load(f)
    for k in (1, 2, 3):
        g = synth.config(k)
        assert g["alpha"] == paper["safr"]["alpha"]["value"]
        assert g["beta"] == paper["safr"]["beta"]["value"]
        assert g["h_lgs"] == paper["system"]["na_layer_height_m"]["value"]
    g2 = synth.config(2)
    assert g2["obstruction"] == paper["system"]["central_obstruction"]["value"]
    assert g2["alpha_tt"] == paper["safr"]["alpha_tt_highflux"]["value"]


def test_oracle_regression_values(oracle_mod):
    """Values written by tests/golden/make_golden.py (oracle only) for the 32x32 workload."""
    from paper_2510_19542_gb300 import synth
    with open(os.path.join(HERE, "golden", "oracle_tiny_ngs_32.json")) as f:
        gold = json.load(f)
    g = synth.config(1)
    out = oracle_mod.OraclePlan(g).reconstruct(synth.frame(g))
    np.testing.assert_allclose(np.sqrt(np.mean(out ** 2, axis=(1, 2))), gold["layer_rms"], rtol=1e-12)
    idx = np.array(gold["sample_lpq"])
    np.testing.assert_allclose(out[idx[:, 0], idx[:, 1], idx[:, 2]], gold["sample_values"],
                               rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# Sampled reconstruction (the full-size point checks) against the full one
# --------------------------------------------------------------------------
def _sample_plans(M):
    from paper_2510_19542_gb300 import synth
    mixed = synth.scaled(synth.config(2), M=M, P=max(4, (5 * M) // 16 + 1), L=4)   # odd P: odd pad offset
    lgs_metric = dict(mixed, kind=np.ones(9, np.int32), name=f"lgs-metric-{M}")
    lgs_native = dict(lgs_metric, output_metric=0, name=f"lgs-native-{M}")
    ngs = synth.scaled(synth.config(1), M=M, P=M // 2, L=3)
    ngs["precision"] = "fp32"
    return mixed, lgs_metric, lgs_native, ngs


@pytest.mark.parametrize("M", [16, 32, 64])
def test_samples_equal_full_reconstruction(oracle_mod, M):
    """oracle_plan_reconstruct_samples (an IDFT2 sum at each point plus its own
    bilinear indexing) equals oracle_plan_reconstruct (the whole IDFT2 of
    Algorithm 1 and the separate resample, Section 3.2 / 3.3) at every sampled
    (l, p, q).  The points cover the whole grid at M <= 32 and, at M = 64, the
    rows and columns of the wrap seam (0, 1, M-2, M-1), the centre row M/2
    (integer source position for every c_l) and random points; the ground
    layer (c = 1) and the NGS group sample integer source positions, the
    upper LGS layers of the metric plans wrap around the periodic grid."""
    from paper_2510_19542_gb300 import synth
    rng = np.random.default_rng(M)
    for g in _sample_plans(M):
        orc = oracle_mod.OraclePlan(g)
        x = synth.random_frame(g, 17 + M)
        full = orc.reconstruct(x)
        L = full.shape[0]
        if M <= 32:
            l, p, q = np.meshgrid(np.arange(L), np.arange(M), np.arange(M), indexing="ij")
            lpq = np.stack([l.ravel(), p.ravel(), q.ravel()], 1)
        else:
            edge = np.array([0, 1, M // 2, M - 2, M - 1])
            pts = [(l, p, q) for l in range(L) for p in edge for q in range(M)]
            pts += [(l, p, q) for l in range(L) for p in range(M) for q in edge]
            pts += [tuple(v) for v in np.stack([rng.integers(0, L, 400), rng.integers(0, M, 400),
                                                rng.integers(0, M, 400)], 1)]
            lpq = np.array(pts)
        got = orc.reconstruct_samples(x, lpq)
        ref = full[lpq[:, 0], lpq[:, 1], lpq[:, 2]]
        scale = np.abs(full).max()
        assert np.abs(got - ref).max() <= 1e-12 * scale, (g["name"], np.abs(got - ref).max() / scale)
