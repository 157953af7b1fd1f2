"""Pins of the oracle's loop steps around SAFR (Algorithm 3): pseudo open loop
control, psi~ = mask (psi + A a), with the tomography operator of Section 2
evaluated by bilinear interpolation, and the integrator.

Expected values come from other routes: np.roll for integer shifts (bilinear
interpolation is then exact), the closed form of Eq. (defAperonly) for
layers linear in the physical coordinates (also exact under bilinear
interpolation), the exact Fourier-series layered model of synth.py, and the
closed form of the integrator's recursion.
"""
import math

import numpy as np
import pytest

from paper_2510_19542_gb300 import synth


def _ngs_integer_geometry(M=32, P=24, output_metric=1):
    """Three NGS whose shifts alpha_g h_l / delta are whole pixels."""
    d = 0.25
    h = np.array([0.0, 4000.0, 8000.0])
    ax = np.array([3, -2, 1]) * d / 4000.0
    ay = np.array([-2, 1, 4]) * d / 4000.0
    return dict(name="ngs-int", M=M, P=P, pitch=d, diameter=P * d, obstruction=0.1, h=h,
                cn2=np.array([0.5, 0.3, 0.2]), dir_x=ax, dir_y=ay, kind=np.zeros(3, np.int32), h_lgs=90e3,
                alpha=0.005, alpha_tt=0.01, beta=1.5, output_metric=output_metric, remove_tt=0)


def _mask_on_pupil(g):
    return synth.pupil(g)


def test_polc_constant_layers(oracle_mod):
    g = synth.scaled(synth.config(2), M=64, P=20)
    L, G, M, P = len(g["h"]), len(g["dir_x"]), g["M"], g["P"]
    kappa = np.linspace(-1.0, 2.0, L)
    a = np.broadcast_to(kappa[:, None, None], (L, M, M)).copy()
    psi = np.random.default_rng(1).standard_normal((G, P, P))
    out = oracle_mod.polc(g, psi, a)
    m = _mask_on_pupil(g)
    np.testing.assert_allclose(out, m * (psi + kappa.sum()), rtol=0, atol=1e-12)


@pytest.mark.parametrize("output_metric", [0, 1])
def test_polc_integer_shifts_are_rolls(oracle_mod, output_metric):
    g = _ngs_integer_geometry(output_metric=output_metric)
    M, P, L, G = g["M"], g["P"], 3, 3
    o = (M - P) // 2
    rng = np.random.default_rng(2)
    a = rng.standard_normal((L, M, M))
    psi = rng.standard_normal((G, P, P))
    out = oracle_mod.polc(g, psi, a)
    m = _mask_on_pupil(g)
    for s in range(G):
        ref = psi[s].copy()
        for l in range(L):
            sx = int(round(g["dir_x"][s] * g["h"][l] / g["pitch"]))
            sy = int(round(g["dir_y"][s] * g["h"][l] / g["pitch"]))
            ref += np.roll(a[l], (-(o + sx), -(o + sy)), axis=(0, 1))[:P, :P]
        np.testing.assert_allclose(out[s], m * ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("output_metric", [0, 1])
def test_polc_linear_layers_follow_the_operator(oracle_mod, output_metric):
    """Layers linear in metres, f_l(x, y) = b_l x + e_l y + k_l, sampled on the
    output grid; bilinear interpolation is exact, so A_g a at pupil point r is
    sum_l f_l(c_l r + alpha_g h_l) (Eq. defAperonly) for LGS (c_l < 1)."""
    M, P, d = 64, 16, 0.5
    h = np.array([0.0, 5000.0, 12000.0])
    lx, ly = np.array([1e-4, -2e-4]), np.array([0.5e-4, 1.5e-4])
    g = dict(name="lgs-lin", M=M, P=P, pitch=d, diameter=0.0, obstruction=0.0, h=h, cn2=np.array([.5, .3, .2]),
             dir_x=lx, dir_y=ly, kind=np.ones(2, np.int32), h_lgs=90e3, alpha=0.005, alpha_tt=0.01, beta=1.5,
             output_metric=output_metric, remove_tt=0)
    rng = np.random.default_rng(3)
    b, e, k = rng.standard_normal(3), rng.standard_normal(3), rng.standard_normal(3)
    c = 1.0 - h / 90e3
    u = np.arange(M) - M / 2.0
    a = np.empty((3, M, M))
    for l in range(3):
        pitch = d if output_metric else c[l] * d
        a[l] = b[l] * pitch * u[:, None] + e[l] * pitch * u[None, :] + k[l]
    out = oracle_mod.polc(g, np.zeros((2, P, P)), a)
    o = (M - P) // 2
    r = d * (o + np.arange(P) - M / 2.0)
    for s in range(2):
        ref = np.zeros((P, P))
        for l in range(3):
            X = c[l] * r[:, None] + lx[s] * h[l]
            Y = c[l] * r[None, :] + ly[s] * h[l]
            ref += b[l] * X + e[l] * Y + k[l]
        np.testing.assert_allclose(out[s], ref, rtol=0, atol=1e-10)


def _polc_truth_error(oracle_mod, g, stars=None):
    x, coeffs = synth.frame(g, noise=0.0, return_truth=True)
    a = synth.truth_layers(g, coeffs)
    out = oracle_mod.polc(g, np.zeros_like(x), a)
    s = slice(None) if stars is None else stars
    return np.linalg.norm(out[s] - x[s]) / np.linalg.norm(x[s])


def test_polc_against_exact_layered_model_whole_pixel_shifts(oracle_mod):
    """Whole-pixel shifts (NGS, c_l = 1): POLC of the true screens equals synth's
    exact Fourier-series evaluation of sum_l phi_l(r + alpha_g h_l)."""
    g = dict(_ngs_integer_geometry(), r0=0.15, L0=25.0, noise=0.0, seed=3)
    assert _polc_truth_error(oracle_mod, g) <= 1e-10


def test_polc_against_exact_layered_model_cone(oracle_mod):
    """Mixed LGS + NGS on the metric grid: against synth's exact evaluation of
    sum_l phi_l(c_l r + alpha_g h_l), the only error is bilinear interpolation of
    the screens.  So it is alike for LGS (c_l < 1) and NGS stars (a wrong cone
    factor would misplace every LGS sample) and it falls as the grid is refined."""
    errs = {}
    for M, P in [(64, 20), (128, 40)]:
        g = synth.scaled(synth.config(2), M=M, P=P)
        lgs = np.asarray(g["kind"]) == 1
        e_l, e_n = _polc_truth_error(oracle_mod, g, lgs), _polc_truth_error(oracle_mod, g, ~lgs)
        assert e_l <= 0.15 and e_n <= 0.15, (M, e_l, e_n)
        assert 0.7 <= e_l / e_n <= 1.4, (M, e_l, e_n)
        errs[M] = max(e_l, e_n)
    assert errs[128] < 0.75 * errs[64], errs
    assert _polc_truth_error(oracle_mod, synth.config(1)) <= 0.05


def test_integrator_closed_form(oracle_mod):
    rng = np.random.default_rng(4)
    a0, phi = rng.standard_normal(100), rng.standard_normal(100)
    np.testing.assert_array_equal(oracle_mod.integrate(phi, a0, 0.0), a0)
    np.testing.assert_array_equal(oracle_mod.integrate(phi, a0, 1.0), phi)
    a, g = a0.copy(), 0.3
    for n in range(1, 8):
        a = oracle_mod.integrate(phi, a, g)
        np.testing.assert_allclose(a, phi + (1 - g) ** n * (a0 - phi), rtol=0, atol=1e-14)
