"""Seeded synthetic inputs for SAFR: geometries and guide-star wavefronts.

This module only draws inputs.  It holds none of the reconstruction's
arithmetic (no B, no regularisation, no inverse transform) and imports neither
the CUDA binding nor the oracle, so the tests, the oracle and the library all
consume identical bytes from it.

Wavefronts follow the layered model of Section 2: each layer is a periodic
von Karman phase screen, and star g sees (A_g phi)(r) = sum_l phi_l(c_l r +
alpha_g h_l) (Section 2).  The screens are band-limited Fourier series of
period 2T, so the sum is evaluated exactly at the shifted and scaled sample
points by two small complex matrix products per (star, layer).  Units are
radians of phase at 500 nm.  The phase power spectrum is the standard von
Karman form 0.023 r0^(-5/3) (f^2 + L0^-2)^(-11/6) with r0_l = r0 gamma_l^(-3/5).
Noise is i.i.d. Gaussian on the pupil pixels with standard deviation equal to
a fraction of the noise-free wavefront's RMS over the pupil, per star.
"""
from __future__ import annotations

import math

import numpy as np

ARCMIN = math.pi / (180.0 * 60.0)

NGS, LGS = 0, 1


def _ring(radius_arcmin: float, azimuths_deg) -> tuple[np.ndarray, np.ndarray]:
    """Direction vectors alpha_g = tan(theta) (cos phi, sin phi) (Section 2)."""
    t = math.tan(radius_arcmin * ARCMIN)
    az = np.deg2rad(np.asarray(azimuths_deg, dtype=np.float64))
    return t * np.cos(az), t * np.sin(az)


def _exp_profile(h: np.ndarray, scale_m: float = 3000.0) -> np.ndarray:
    w = np.exp(-h / scale_m)
    return w / w.sum()


def config(k: int) -> dict:
    """Geometry of the named workloads.

    1: 8 m telescope, 32x32 grid (0.25 m), 3 NGS at 1 arcmin, 3 layers 0/4/12 km
       with Cn2 0.6/0.25/0.15, r0 0.15 m, 1% noise, FP64.
    2: MORFEO-like: 39 m aperture (11% obstruction), 80x80 pupil samples on a
       256x256 grid, 6 LGS at 90 km on a 2 arcmin ring + 3 NGS at 1.3 arcmin,
       9 layers 0-16 km with an exponential Cn2 profile, r0 0.157 m, 2% noise, FP32.
    3: 8 m pupil filling a 512x512 grid, 3 NGS at 1 arcmin, 35 layers 0-20 km,
       exponential Cn2, r0 0.15 m, 1% noise, FP16 storage with per-layer scales.
    5: the geometry of 1 (8 m, 32x32 grid, 3 NGS at 1 arcmin) with 35 layers
       0-20 km on the exponential Cn2 profile, r0 0.15 m, 1% noise, FP32: the
       learned spectral filter's workload.
    """
    if k == 1:
        ax, ay = _ring(1.0, [0.0, 120.0, 240.0])
        h = np.array([0.0, 4000.0, 12000.0])
        return dict(name="tiny-ngs-32", M=32, P=32, pitch=0.25, diameter=8.0, obstruction=0.0,
                    h=h, cn2=np.array([0.6, 0.25, 0.15]), dir_x=ax, dir_y=ay,
                    kind=np.zeros(3, np.int32), h_lgs=90e3, alpha=0.005, alpha_tt=0.01, beta=1.5,
                    output_metric=1, remove_tt=1, precision="fp64", r0=0.15, L0=25.0, noise=0.01,
                    seed=1)
    if k == 2:
        lx, ly = _ring(2.0, [60.0 * g for g in range(6)])
        nx, ny = _ring(1.3, [60.0 + 120.0 * g for g in range(3)])
        h = np.linspace(0.0, 16000.0, 9)
        return dict(name="morfeo-256", M=256, P=80, pitch=39.0 / 80.0, diameter=39.0,
                    obstruction=0.11, h=h, cn2=_exp_profile(h), dir_x=np.concatenate([lx, nx]),
                    dir_y=np.concatenate([ly, ny]),
                    kind=np.array([LGS] * 6 + [NGS] * 3, np.int32), h_lgs=90e3, alpha=0.005,
                    alpha_tt=0.01, beta=1.5, output_metric=1, remove_tt=1, precision="fp32",
                    r0=0.157, L0=25.0, noise=0.02, seed=2)
    if k == 3:
        ax, ay = _ring(1.0, [0.0, 120.0, 240.0])
        h = np.linspace(0.0, 20000.0, 35)
        return dict(name="ngs-512-L35-fp16", M=512, P=512, pitch=8.0 / 512.0, diameter=8.0,
                    obstruction=0.0, h=h, cn2=_exp_profile(h), dir_x=ax, dir_y=ay,
                    kind=np.zeros(3, np.int32), h_lgs=90e3, alpha=0.005, alpha_tt=0.01, beta=1.5,
                    output_metric=1, remove_tt=1, precision="fp16", r0=0.15, L0=25.0,
                    noise=0.01, seed=3)
    if k == 5:
        h = np.linspace(0.0, 20000.0, 35)
        return dict(config(1), name="learned-ngs-32-L35", h=h, cn2=_exp_profile(h), precision="fp32", seed=5)
    raise ValueError(f"no workload {k}")


def scaled(geom: dict, M: int, P: int | None = None, L: int | None = None) -> dict:
    """The same asterism and profile shape on a smaller grid (fast parity cases).

    The pitch is rescaled so the pupil keeps its diameter in metres."""
    g = dict(geom)
    P = P if P is not None else max(2, int(round(geom["P"] * M / geom["M"])))
    g["M"], g["P"] = M, P
    g["pitch"] = geom["pitch"] * geom["P"] / P
    if L is not None and L != len(geom["h"]):
        h = np.linspace(float(geom["h"][0]), float(geom["h"][-1]), L)
        g["h"] = h
        g["cn2"] = _exp_profile(h)
    g["name"] = f'{geom["name"]}@M{M}P{P}L{len(g["h"])}'
    return g


def pupil(geom: dict) -> np.ndarray:
    """Annular pupil mask [P][P] (bool), pixel centres at (a-(P-1)/2)*pitch."""
    P, d = geom["P"], geom["pitch"]
    x = (np.arange(P) - (P - 1) / 2.0) * d
    r2 = x[:, None] ** 2 + x[None, :] ** 2
    D = geom.get("diameter", 0.0)
    if D <= 0:
        return np.ones((P, P), bool)
    ro, ri = D / 2.0, geom.get("obstruction", 0.0) * D / 2.0
    return (r2 <= ro * ro) & (r2 >= ri * ri)


def _screen_coeffs(rng, M: int, T: float, r0: float, L0: float) -> np.ndarray:
    """Fourier coefficients C[nx, ny] (nx, ny in -(M/2-1)..M/2-1) of a real
    periodic von Karman screen of period 2T, Hermitian so the series is real."""
    n = np.arange(-(M // 2 - 1), M // 2)
    f = n / (2.0 * T)
    f2 = f[:, None] ** 2 + f[None, :] ** 2
    psd = 0.023 * r0 ** (-5.0 / 3.0) * (f2 + L0 ** -2) ** (-11.0 / 6.0)
    df = 1.0 / (2.0 * T)
    amp = np.sqrt(psd) * df
    xi = (rng.standard_normal(amp.shape) + 1j * rng.standard_normal(amp.shape)) / math.sqrt(2.0)
    c = amp * xi
    c = 0.5 * (c + np.conj(c[::-1, ::-1]))  # C[-n] = conj C[n]
    c[M // 2 - 1, M // 2 - 1] = 0.0         # no piston
    return c


def frame(geom: dict, seed: int | None = None, noise: float | None = None,
          return_truth: bool = False):
    """Wavefronts [G][P][P] (float64) for geometry ``geom``.

    The screens use ``seed`` (default: geom['seed']) and the noise uses
    seed + 1000.  With return_truth the layer coefficients are returned too."""
    M, P, d = geom["M"], geom["P"], geom["pitch"]
    T = M * d / 2.0
    seed = geom.get("seed", 0) if seed is None else seed
    noise = geom.get("noise", 0.0) if noise is None else noise
    h = np.asarray(geom["h"], np.float64)
    gam = np.asarray(geom["cn2"], np.float64)
    gam = gam / gam.sum()
    r0, L0 = geom.get("r0", 0.15), geom.get("L0", 25.0)
    rng = np.random.default_rng(seed)
    coeffs = [_screen_coeffs(rng, M, T, r0 * g ** (-3.0 / 5.0), L0) for g in gam]
    o = (M - P) // 2
    xp = -T + (o + np.arange(P)) * d            # pupil sample coordinates
    n = np.arange(-(M // 2 - 1), M // 2)
    omega = math.pi / T
    mask = pupil(geom)
    G = len(geom["dir_x"])
    out = np.zeros((G, P, P))
    for g in range(G):
        lgs = int(geom["kind"][g]) == LGS
        for l in range(len(h)):
            c = 1.0 - h[l] / geom.get("h_lgs", 90e3) if lgs else 1.0
            ex = np.exp(1j * omega * np.outer(c * xp + geom["dir_x"][g] * h[l], n))
            ey = np.exp(1j * omega * np.outer(c * xp + geom["dir_y"][g] * h[l], n))
            out[g] += (ex @ coeffs[l] @ ey.T).real
    out *= mask
    if noise > 0:
        nrng = np.random.default_rng(seed + 1000)
        for g in range(G):
            rms = math.sqrt(float(np.mean(out[g][mask] ** 2)))
            out[g] += noise * rms * nrng.standard_normal((P, P)) * mask
    if return_truth:
        return out, coeffs
    return out


def truth_layers(geom: dict, coeffs) -> np.ndarray:
    """The screens of frame(..., return_truth=True) on the M x M grid x_p =
    -T + p * pitch (layer pitch = pupil pitch: NGS geometry), [L][M][M]."""
    M, d = geom["M"], geom["pitch"]
    T = M * d / 2.0
    x = -T + np.arange(M) * d
    n = np.arange(-(M // 2 - 1), M // 2)
    e = np.exp(1j * (math.pi / T) * np.outer(x, n))
    return np.stack([(e @ c @ e.T).real for c in coeffs])


def random_frame(geom: dict, seed: int) -> np.ndarray:
    """Plain N(0,1) pupil samples (masked): cheap inputs for structural checks."""
    rng = np.random.default_rng(seed)
    G, P = len(geom["dir_x"]), geom["P"]
    return rng.standard_normal((G, P, P)) * pupil(geom)


def to_fp16_storage(x: np.ndarray):
    """(half values, per-star power-of-two scales) with x ~= half * scale."""
    G = x.shape[0]
    scales = np.empty(G, np.float32)
    for g in range(G):
        rms = float(np.sqrt(np.mean(x[g] ** 2))) or 1.0
        scales[g] = 2.0 ** math.floor(math.log2(rms))
    h = (x / scales[:, None, None]).astype(np.float16)
    return h, scales


def from_fp16_storage(h: np.ndarray, scales: np.ndarray) -> np.ndarray:
    return h.astype(np.float64) * scales.astype(np.float64)[:, None, None]


def batch_configs(n: int = 64, seed: int = 4, grids=(128, 256, 512)) -> list:
    """Geometries of the batched workload: n frames of uneven geometry drawn from
    ``seed``.  Per frame: grid M from ``grids``, P = ceil(0.3125 M) pupil samples
    across a 39 m aperture (11% obstruction), G in [3, 9] stars that are all LGS
    (90 km, 2 arcmin ring), all NGS (1.3 arcmin ring) or a mix of both, L in
    [3, 35] layers on 0-16 km with the exponential Cn2 profile, FP32.  Frame f's
    inputs use seed 4000 + f."""
    rng = np.random.default_rng(seed)
    out = []
    for f in range(n):
        M = int(rng.choice(grids))
        G = int(rng.integers(3, 10))
        L = int(rng.integers(3, 36))
        mix = int(rng.integers(0, 3))  # 0 LGS only, 1 NGS only, 2 mixed
        n_lgs = G if mix == 0 else (0 if mix == 1 else int(rng.integers(1, G)))
        n_ngs = G - n_lgs
        P = int(math.ceil(0.3125 * M))
        lx, ly = _ring(2.0, [360.0 * i / max(n_lgs, 1) for i in range(n_lgs)])
        nx, ny = _ring(1.3, [60.0 + 360.0 * i / max(n_ngs, 1) for i in range(n_ngs)])
        h = np.linspace(0.0, 16000.0, L)
        out.append(dict(name=f"batch-{f}", M=M, P=P, pitch=39.0 / P, diameter=39.0, obstruction=0.11,
                        h=h, cn2=_exp_profile(h), dir_x=np.concatenate([lx, nx]), dir_y=np.concatenate([ly, ny]),
                        kind=np.array([LGS] * n_lgs + [NGS] * n_ngs, np.int32), h_lgs=90e3, alpha=0.005,
                        alpha_tt=0.01, beta=1.5, output_metric=1, remove_tt=1, precision="fp32",
                        r0=0.157, L0=25.0, noise=0.02, seed=4000 + f))
    return out
