"""ctypes marshalling for the FP64 SAFR oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Each wrapper names the
paper passage its C routine follows; the arithmetic is all in ``oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_cp = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_bp = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (FP64, IEEE, OpenMP over independent loops)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        lib.oracle_dft2.argtypes = [C.c_int, _cp, _cp, C.c_int]
        lib.oracle_svd.argtypes = [C.c_int, C.c_int, _cp, _cp, _dp, _cp]
        lib.oracle_svd.restype = C.c_int
        lib.oracle_cone.argtypes = [C.c_int, _dp, C.c_double, C.c_int, _dp]
        lib.oracle_group_B.argtypes = [C.c_int, C.c_double, C.c_int, _dp, _dp, _dp, C.c_int,
                                       _dp, _dp, C.c_double, C.c_double, _cp]
        lib.oracle_remove_tt.argtypes = [C.c_int, C.c_double, _bp, _dp, _dp]
        lib.oracle_resample.argtypes = [C.c_int, C.c_double, _dp, _dp]
        lib.oracle_pupil_mask.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, _bp]
        lib.oracle_plan_new.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                        C.c_int, _dp, _dp, C.c_int, _dp, _dp, _ip,
                                        C.c_double, C.c_double, C.c_double, C.c_double,
                                        C.c_int, C.c_int]
        lib.oracle_plan_new.restype = C.c_void_p
        lib.oracle_plan_free.argtypes = [C.c_void_p]
        lib.oracle_plan_ngroups.argtypes = [C.c_void_p]
        lib.oracle_plan_group.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                          C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.c_void_p]
        lib.oracle_plan_reconstruct.argtypes = [C.c_void_p, _dp, _dp, C.POINTER(C.c_double)]
        lib.oracle_plan_reconstruct_samples.argtypes = [C.c_void_p, _dp, C.c_int, _ip, _dp]
        lib.oracle_mlp_phi.argtypes = [_dp, _dp]
        lib.oracle_mlp_phi.restype = C.c_double
        lib.oracle_group_B_learned.argtypes = [C.c_int, C.c_double, C.c_int, _dp, _dp, _dp, C.c_int, _dp, _dp,
                                               C.c_double, _dp, C.c_double, _cp]
        lib.oracle_philox4x32_10.argtypes = [_up, _up, _up]
        lib.oracle_filter_frames_loss.argtypes = [C.c_int, C.c_double, C.c_int, _dp, _dp, _dp, C.c_int, _dp, _dp,
                                                  _cp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                                  C.c_double, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                                  C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.oracle_polc.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, _dp, C.c_int,
                                    _dp, _dp, _ip, C.c_double, C.c_int, _dp, _dp, _dp]
        lib.oracle_integrate.argtypes = [C.c_long, _dp, _dp, C.c_double]
        lib.oracle_filter_frame.argtypes = [C.c_int, C.c_double, C.c_int, _dp, _dp, _dp, C.c_int, _dp, _dp,
                                            C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                            C.c_uint32, C.c_uint32, C.c_uint32, _cp, _cp]
        _lib = lib
        return lib


def threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all cores)."""
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def dft2(x: np.ndarray) -> np.ndarray:
    """DFT2 of Section 3.2 (unnormalised, e^{-2 pi i (jp+kq)/M})."""
    x = _c128(x)
    y = np.empty_like(x)
    _load().oracle_dft2(x.shape[0], x, y, 0)
    return y


def idft2(y: np.ndarray) -> np.ndarray:
    """IDFT2 of Section 3.2 (1/M^2, e^{+2 pi i (jp+kq)/M})."""
    y = _c128(y)
    x = np.empty_like(y)
    _load().oracle_dft2(y.shape[0], y, x, 1)
    return x


def svd(A: np.ndarray):
    """Hestenes one-sided Jacobi SVD: A (m x n) = U diag(S) V^H, U m x n, V n x n."""
    A = _c128(A)
    m, n = A.shape
    U = np.empty((m, n), np.complex128)
    S = np.empty(n, np.float64)
    V = np.empty((n, n), np.complex128)
    sweeps = _load().oracle_svd(m, n, A, U, S, V)
    return U, S, V, sweeps


def cone(h, h_lgs: float, lgs: bool) -> np.ndarray:
    """c_l of Section 2."""
    h = _f64(h)
    c = np.empty_like(h)
    _load().oracle_cone(len(h), h, float(h_lgs), int(bool(lgs)), c)
    return c


def group_B(M, T, h, c, gamma, ax, ay, alpha, beta) -> np.ndarray:
    """Algorithm 2 for one star group: B [M][M][L][G] over the full spectrum."""
    h, c, gamma, ax, ay = map(_f64, (h, c, gamma, ax, ay))
    L, G = len(h), len(ax)
    B = np.empty((M, M, L, G), np.complex128)
    rc = _load().oracle_group_B(M, float(T), L, h, c, gamma, G, ax, ay, float(alpha), float(beta), B)
    if rc:
        raise ValueError("oracle_group_B: bad arguments")
    return B


MLP_PARAMS = 4 * 64 + 64 + 2 * (64 * 64 + 64) + 64 + 1


def mlp_phi(params: np.ndarray, x) -> float:
    """Filter factor phi in (0, 1) of the learned filter's MLP at features x[4]."""
    return _load().oracle_mlp_phi(_f64(params), _f64(x))


def group_B_learned(M, T, h, c, gamma, ax, ay, beta, params, noise_level) -> np.ndarray:
    """Section 3.1's filtered inverse with the learned filter phi / sigma: B [M][M][L][G]."""
    h, c, gamma, ax, ay, params = map(_f64, (h, c, gamma, ax, ay, params))
    if params.size != MLP_PARAMS:
        raise ValueError("wrong parameter count")
    L, G = len(h), len(ax)
    B = np.empty((M, M, L, G), np.complex128)
    if _load().oracle_group_B_learned(M, float(T), L, h, c, gamma, G, ax, ay, float(beta), params,
                                      float(noise_level), B):
        raise ValueError("oracle_group_B_learned: bad arguments")
    return B


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al., SC 2011): 4 output words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, np.uint32)
    _load().oracle_philox4x32_10(c, k, out)
    return out


def filter_frame(M, T, h, c, gamma, ax, ay, P, D, obstruction, r0, L0, noise_level, key, F):
    """One training frame of the learned filter (Section 2's layered model through
    the aperture): layer spectra phi [M/2][M][L] (k < M/2, j, l) and data spectra
    d [G][M][M] (j, k)."""
    h, c, gamma, ax, ay = map(_f64, (h, c, gamma, ax, ay))
    L, G = len(h), len(ax)
    phi = np.empty((M // 2, M, L), np.complex128)
    d = np.empty((G, M, M), np.complex128)
    if _load().oracle_filter_frame(M, float(T), L, h, c, gamma, G, ax, ay, int(P), float(D), float(obstruction),
                                   float(r0), float(L0), float(noise_level), int(key[0]) & 0xFFFFFFFF,
                                   int(key[1]) & 0xFFFFFFFF, int(F), phi, d):
        raise ValueError("oracle_filter_frame: bad arguments")
    return phi, d


def filter_frames_loss(M, T, h, c, gamma, ax, ay, B, P, D, obstruction, r0, L0, noise_level, key, frame0, nwrap,
                       nframes):
    """(loss, energy) of reconstruction B [M][M][L][G] on the learned filter's
    training frames (frame0 + i) mod nwrap, i < nframes."""
    h, c, gamma, ax, ay = map(_f64, (h, c, gamma, ax, ay))
    B = _c128(B)
    L, G = len(h), len(ax)
    loss, energy = C.c_double(), C.c_double()
    if _load().oracle_filter_frames_loss(M, float(T), L, h, c, gamma, G, ax, ay, B, int(P), float(D),
                                         float(obstruction), float(r0), float(L0), float(noise_level),
                                         int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF, int(frame0),
                                         int(nwrap), int(nframes), C.byref(loss), C.byref(energy)):
        raise ValueError("oracle_filter_frames_loss: bad arguments")
    return loss.value, energy.value


def polc(geom: dict, wavefronts: np.ndarray, a: np.ndarray) -> np.ndarray:
    """Pseudo open loop data (Algorithm 3, line 2): mask * (wavefronts + A(a)),
    A the tomography operator of Section 2 on the bilinearly interpolated layers
    a [L][M][M] of the plan's output grid (metric unless output_metric is 0)."""
    g = geom
    M, P = int(g["M"]), int(g["P"])
    L, G = len(g["h"]), len(g["dir_x"])
    psi = _f64(wavefronts).reshape(G, P, P)
    a = _f64(a).reshape(L, M, M)
    out = np.empty((G, P, P), np.float64)
    if _load().oracle_polc(M, P, float(g["pitch"]), float(g.get("diameter", 0.0)), float(g.get("obstruction", 0.0)),
                           L, _f64(g["h"]), G, _f64(g["dir_x"]), _f64(g["dir_y"]),
                           np.ascontiguousarray(g["kind"], dtype=np.int32), float(g.get("h_lgs", 90e3)),
                           int(g.get("output_metric", 1)), psi, a, out):
        raise ValueError("oracle_polc: bad arguments")
    return out


def integrate(phi: np.ndarray, a: np.ndarray, gain: float) -> np.ndarray:
    """Integrator (Algorithm 3, line 5): returns (1 - gain) a + gain phi."""
    out = _f64(a).copy()
    _load().oracle_integrate(out.size, _f64(phi).reshape(-1), out.reshape(-1), float(gain))
    return out


def pupil_mask(P: int, delta: float, D: float, obstruction: float) -> np.ndarray:
    m = np.empty((P, P), np.uint8)
    _load().oracle_pupil_mask(P, float(delta), float(D), float(obstruction), m)
    return m


def remove_tt(psi: np.ndarray, delta: float, mask: np.ndarray):
    """removeTT of Algorithm 3 (least-squares plane over the mask); returns (psi', (a,b,c))."""
    out = _f64(psi).copy()
    abc = np.empty(3, np.float64)
    rc = _load().oracle_remove_tt(out.shape[0], float(delta), np.ascontiguousarray(mask, np.uint8), out, abc)
    if rc:
        raise ValueError("oracle_remove_tt: singular normal equations")
    return out, abc


def resample(src: np.ndarray, c: float) -> np.ndarray:
    """Bilinear, periodic resample of a pitch c*delta layer onto the pitch delta grid."""
    src = _f64(src)
    dst = np.empty_like(src)
    _load().oracle_resample(src.shape[0], float(c), src, dst)
    return dst


class OraclePlan:
    """Geometry + per-group B (Algorithm 2) + per-frame reconstruction (Algorithm 1).

    ``geom`` is a dict with keys M, P, pitch, diameter, obstruction, h, cn2,
    dir_x, dir_y, kind, h_lgs, alpha, alpha_tt, beta, output_metric, remove_tt.
    """

    def __init__(self, geom: dict):
        lib = _load()
        self.geom = dict(geom)
        g = self.geom
        self.M, self.P = int(g["M"]), int(g["P"])
        self.L, self.G = len(g["h"]), len(g["dir_x"])
        self._h = _f64(g["h"])
        self._cn2 = _f64(g["cn2"])
        self._ax = _f64(g["dir_x"])
        self._ay = _f64(g["dir_y"])
        self._kind = np.ascontiguousarray(g["kind"], dtype=np.int32)
        self._ptr = lib.oracle_plan_new(
            self.M, self.P, float(g["pitch"]), float(g.get("diameter", 0.0)),
            float(g.get("obstruction", 0.0)), self.L, self._h, self._cn2, self.G,
            self._ax, self._ay, self._kind, float(g.get("h_lgs", 90e3)), float(g["alpha"]),
            float(g.get("alpha_tt", g["alpha"])), float(g["beta"]),
            int(g.get("output_metric", 1)), int(g.get("remove_tt", 1)))
        if not self._ptr:
            raise ValueError("oracle_plan_new: invalid geometry")

    def __del__(self):
        p = getattr(self, "_ptr", None)
        if p:
            _load().oracle_plan_free(p)
            self._ptr = None

    @property
    def ngroups(self) -> int:
        return _load().oracle_plan_ngroups(self._ptr)

    def group(self, gi: int):
        """(kind, star indices, c_l, B[M][M][L][Gg]) of group gi (LGS first)."""
        kind, Gg = C.c_int(), C.c_int()
        lib = _load()
        if lib.oracle_plan_group(self._ptr, gi, C.byref(kind), C.byref(Gg), None, None, None):
            raise IndexError(gi)
        B = np.empty((self.M, self.M, self.L, Gg.value), np.complex128)
        stars = np.empty(Gg.value, np.int32)
        c = np.empty(self.L, np.float64)
        lib.oracle_plan_group(self._ptr, gi, None, None, stars.ctypes.data, c.ctypes.data,
                              B.ctypes.data)
        return kind.value, stars, c, B

    def reconstruct(self, wavefronts: np.ndarray, return_imag: bool = False):
        """Layers [L][M][M] from wavefronts [G][P][P] (FP64)."""
        w = _f64(wavefronts).reshape(self.G, self.P, self.P)
        out = np.empty((self.L, self.M, self.M), np.float64)
        im = C.c_double(0.0)
        _load().oracle_plan_reconstruct(self._ptr, w, out, C.byref(im))
        return (out, im.value) if return_imag else out

    def reconstruct_samples(self, wavefronts: np.ndarray, lpq: np.ndarray) -> np.ndarray:
        """Layer values at the (l, p, q) rows of lpq only (direct IDFT2 sums)."""
        w = _f64(wavefronts).reshape(self.G, self.P, self.P)
        lpq = np.ascontiguousarray(lpq, dtype=np.int32).reshape(-1, 3)
        out = np.empty(len(lpq), np.float64)
        _load().oracle_plan_reconstruct_samples(self._ptr, w, len(lpq), lpq, out)
        return out
