"""FP64 CPU oracle for the image-source method (ISM) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this module.  The product library never calls
it, and it shares no code with the CUDA path: it wraps ``ism_oracle.c`` (plain
C, double precision, image-major direct sums) through ctypes.

Functions map one to one onto passages of the paper (Diaz-Guerra et al.,
"gpuRIR"):

* ``enumerate_images``  -- Section 2.1, eq. (1)-(4)
* ``rir``               -- eq. (5) with the windowed sinc of eq. (6)
* ``t60_sabine``        -- eq. (7);  ``beta_sabine`` its inverse (Section 4 helper)
* ``nb_img_from_t``, ``att2t_sabine`` -- Section 4 helpers
* ``noise`` / ``tail`` / ``envelope_amp`` -- Section 2.2 "Diffuse reverberation",
  eq. (8) read as a 60 dB decay over T60, Philox4x32-10 driven logistic noise
* ``lj_energy`` / ``envelope_amp_lj`` / ``tail_lj`` -- the Lehmann-Johansson
  energy-decay envelope that Section 2.2 cites (a reading: the energy arrival
  rate of the image lattice, averaged over directions)
* ``rir_grad``          -- derivative of eq. (1)-(6) (not in the paper)
* ``simulate``          -- the library call of Section 4 (ISM up to Tdiff, tail after)

Parity pins for every function live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ism_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libism_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ism_oracle.c with gcc (-O2 -fopenmp -ffp-contract=off)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        D = ctypes.c_double
        Dp = ctypes.POINTER(ctypes.c_double)
        Ip = ctypes.POINTER(ctypes.c_int)
        U32p = ctypes.POINTER(ctypes.c_uint32)
        Fp = ctypes.POINTER(ctypes.c_float)
        lib.oracle_enumerate_images.restype = ctypes.c_long
        lib.oracle_enumerate_images.argtypes = [Dp, Dp, D, Dp, Dp, Ip, Ip, Dp, Ip, Dp, Dp, Dp]
        lib.oracle_rir_list.restype = None
        lib.oracle_rir_list.argtypes = [Dp, Dp, D, D, D, Dp, Dp, ctypes.c_int, Ip, ctypes.c_int,
                                        Dp, ctypes.c_int]
        lib.oracle_rir_list_pattern.restype = None
        lib.oracle_rir_list_pattern.argtypes = [Dp, Dp, D, D, D, Dp, Dp, Dp, D, ctypes.c_int, Ip, ctypes.c_int,
                                                Dp, ctypes.c_int]
        lib.oracle_pattern_gain.restype = D
        lib.oracle_pattern_gain.argtypes = [D, Dp, Dp, Dp]
        lib.oracle_delta_prime.restype = D
        lib.oracle_delta_prime.argtypes = [D, D, D]
        lib.oracle_image_coord.restype = D
        lib.oracle_image_coord.argtypes = [ctypes.c_int, D, D]
        lib.oracle_image_exponents.restype = None
        lib.oracle_image_exponents.argtypes = [ctypes.c_int, Ip, Ip]
        lib.oracle_grid_bounds.restype = None
        lib.oracle_grid_bounds.argtypes = [ctypes.c_int, Ip, Ip]
        lib.oracle_t60_sabine.restype = D
        lib.oracle_t60_sabine.argtypes = [Dp, Dp]
        lib.oracle_beta_sabine.restype = ctypes.c_int
        lib.oracle_beta_sabine.argtypes = [Dp, D, Dp, ctypes.c_int, Dp]
        lib.oracle_att2t_sabine.restype = D
        lib.oracle_att2t_sabine.argtypes = [D, D]
        lib.oracle_nb_img_from_t.restype = None
        lib.oracle_nb_img_from_t.argtypes = [D, Dp, D, D, Ip]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_philox4x32_10.argtypes = [U32p, U32p, U32p]
        lib.oracle_noise_word.restype = ctypes.c_uint32
        lib.oracle_noise_word.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        lib.oracle_uniform_f32.restype = ctypes.c_float
        lib.oracle_uniform_f32.argtypes = [ctypes.c_uint32]
        lib.oracle_ln_f32.restype = ctypes.c_float
        lib.oracle_ln_f32.argtypes = [ctypes.c_float]
        lib.oracle_ln_f32_array.restype = None
        lib.oracle_ln_f32_array.argtypes = [Fp, Fp, ctypes.c_long]
        lib.oracle_logistic_f32.restype = ctypes.c_float
        lib.oracle_logistic_f32.argtypes = [ctypes.c_float]
        lib.oracle_noise.restype = None
        lib.oracle_noise.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, Fp]
        lib.oracle_envelope_amp.restype = D
        lib.oracle_envelope_amp.argtypes = [Dp, ctypes.c_int, D, D]
        lib.oracle_envelope_sqrt.restype = D
        lib.oracle_envelope_sqrt.argtypes = [D, ctypes.c_int, ctypes.c_int, D, D]
        lib.oracle_tail.restype = None
        lib.oracle_tail.argtypes = [ctypes.c_uint64, ctypes.c_uint32, D, ctypes.c_int, ctypes.c_int,
                                    D, D, Dp]
        lib.oracle_lj_energy.restype = D
        lib.oracle_lj_energy.argtypes = [Dp, Dp, D, D, Dp, Dp, ctypes.c_int]
        lib.oracle_lj_energy_many.restype = None
        lib.oracle_lj_energy_many.argtypes = [Dp, Dp, D, Dp, ctypes.c_int, Dp, Dp, ctypes.c_int, Dp]
        lib.oracle_rir_grad.restype = None
        lib.oracle_rir_grad.argtypes = [Dp, Dp, D, D, D, Dp, Dp, Ip, ctypes.c_int, Dp, Dp, Dp, Dp]
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_max_threads.argtypes = []
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _d(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        a = a.reshape(n)
    return a


def max_threads() -> int:
    return int(_load().oracle_max_threads())


# --------------------------------------------------------------------------- #
# Section 2.1, eq. (1)-(4)
# --------------------------------------------------------------------------- #
def grid_bounds(N: int):
    """ceil(-N/2) <= n < ceil(N/2) (Section 2.1). Returns (lo, hi_exclusive)."""
    lo, hi = ctypes.c_int(), ctypes.c_int()
    _load().oracle_grid_bounds(int(N), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def image_coord(n: int, L: float, xs: float) -> float:
    """Eq. (1)."""
    return float(_load().oracle_image_coord(int(n), float(L), float(xs)))


def image_exponents(n: int):
    """Number of hits of the near (x0) and far (x1) wall for image index n."""
    e0, e1 = ctypes.c_int(), ctypes.c_int()
    _load().oracle_image_exponents(int(n), ctypes.byref(e0), ctypes.byref(e1))
    return e0.value, e1.value


def delta_prime(x: float, fs: float, Tw: float) -> float:
    """Eq. (6) at time offset x/fs (x in samples), f_c = fs/2."""
    return float(_load().oracle_delta_prime(float(x), float(fs), float(Tw)))


def enumerate_images(L, beta, c, ps, pr, N):
    """All images of one pair: dict of n[M,3], pos[M,3], e[M,6], d, tau, A."""
    L, beta, ps, pr = _d(L, 3), _d(beta, 6), _d(ps, 3), _d(pr, 3)
    Nn = np.ascontiguousarray(np.asarray(N, dtype=np.int32).reshape(3))
    M = int(Nn[0]) * int(Nn[1]) * int(Nn[2])
    n = np.zeros((M, 3), np.int32)
    pos = np.zeros((M, 3), np.float64)
    e = np.zeros((M, 6), np.int32)
    d = np.zeros(M, np.float64)
    tau = np.zeros(M, np.float64)
    A = np.zeros(M, np.float64)
    cnt = _load().oracle_enumerate_images(_dp(L), _dp(beta), float(c), _dp(ps), _dp(pr), _ip(Nn),
                                          _ip(n), _dp(pos), _ip(e), _dp(d), _dp(tau), _dp(A))
    return dict(count=int(cnt), n=n, pos=pos, e=e, d=d, tau=tau, A=A)


# --------------------------------------------------------------------------- #
# Eq. (5)-(6)
# --------------------------------------------------------------------------- #
def rir_list(L, beta, c, fs, Tw, ps_list, pr_list, N, n_ism, n_threads: int = 0):
    """ISM part h[0:n_ism] for each pair (ps_list[i], pr_list[i]); [n_pairs, n_ism] FP64."""
    L, beta = _d(L, 3), _d(beta, 6)
    ps = np.ascontiguousarray(np.asarray(ps_list, dtype=np.float64).reshape(-1, 3))
    pr = np.ascontiguousarray(np.asarray(pr_list, dtype=np.float64).reshape(-1, 3))
    assert ps.shape == pr.shape
    Nn = np.ascontiguousarray(np.asarray(N, dtype=np.int32).reshape(3))
    out = np.zeros((ps.shape[0], int(n_ism)), np.float64)
    if ps.shape[0] and n_ism > 0:
        _load().oracle_rir_list(_dp(L), _dp(beta), float(c), float(fs), float(Tw), _dp(ps), _dp(pr),
                                int(ps.shape[0]), _ip(Nn), int(n_ism), _dp(out), int(n_threads))
    return out


# Receiver polar patterns (Section 4; the formula is a reading, see
# oracle_pattern_gain): alpha of g(theta) = alpha + (1 - alpha) cos(theta).
PATTERN_ALPHA = {"omni": 1.0, "subcardioid": 0.75, "cardioid": 0.5, "hypercardioid": 0.25, "bidirectional": 0.0}


def pattern_gain(pattern, orient, pr, p_img) -> float:
    """Gain of one image for a receiver at pr oriented along orient."""
    return _load().oracle_pattern_gain(float(PATTERN_ALPHA[pattern]), _dp(_d(orient, 3)), _dp(_d(pr, 3)),
                                       _dp(_d(p_img, 3)))


def rir_list_pattern(L, beta, c, fs, Tw, ps_list, pr_list, orient_list, pattern, N, n_ism, n_threads: int = 0):
    """As rir_list, each image's amplitude scaled by the receiver's polar pattern."""
    L, beta = _d(L, 3), _d(beta, 6)
    ps = np.ascontiguousarray(np.asarray(ps_list, dtype=np.float64).reshape(-1, 3))
    pr = np.ascontiguousarray(np.asarray(pr_list, dtype=np.float64).reshape(-1, 3))
    orient = np.ascontiguousarray(np.asarray(orient_list, dtype=np.float64).reshape(-1, 3))
    assert ps.shape == pr.shape == orient.shape
    Nn = np.ascontiguousarray(np.asarray(N, dtype=np.int32).reshape(3))
    out = np.zeros((ps.shape[0], int(n_ism)), np.float64)
    if ps.shape[0] and n_ism > 0:
        _load().oracle_rir_list_pattern(_dp(L), _dp(beta), float(c), float(fs), float(Tw), _dp(ps), _dp(pr),
                                        _dp(orient), float(PATTERN_ALPHA[pattern]), int(ps.shape[0]), _ip(Nn),
                                        int(n_ism), _dp(out), int(n_threads))
    return out


# --------------------------------------------------------------------------- #
# Section 4, simulating moving sources: the source signal is cut into one
# segment per trajectory point, each segment is filtered by the RIRs of its
# point (one per microphone) and the filtered segments are overlap-added.
# Reading: segment p covers the samples [start_p, start_(p+1)), by default
# start_p = floor(p n_x / n_points); the output has n_x + n_S - 1 samples.
# --------------------------------------------------------------------------- #
def segment_starts(n_x: int, n_points: int):
    """Uniform segmentation: start_p = floor(p n_x / n_points), p = 0 .. n_points."""
    return [(p * int(n_x)) // int(n_points) for p in range(int(n_points) + 1)]


def auralize(signal, rirs, starts=None):
    """y[m] = sum_p conv(x[start_p:start_(p+1)], h[p, m]) placed at start_p (FP64).

    signal [n_x]; rirs [n_points, n_mics, n_S]; returns [n_mics, n_x + n_S - 1]."""
    x = np.asarray(signal, dtype=np.float64).ravel()
    h = np.asarray(rirs, dtype=np.float64)
    n_points, n_mics, n_s = h.shape
    if starts is None:
        starts = segment_starts(x.size, n_points)
    y = np.zeros((n_mics, x.size + n_s - 1), np.float64)
    for p in range(n_points):
        a, b = int(starts[p]), int(starts[p + 1])
        if b <= a:
            continue
        for m in range(n_mics):
            y[m, a:b + n_s - 1] += np.convolve(x[a:b], h[p, m])
    return y


def rir(L, beta, c, fs, Tw, ps, pr, N, n_ism, n_threads: int = 0):
    """ISM part of one RIR, eq. (5) with eq. (6)."""
    return rir_list(L, beta, c, fs, Tw, [ps], [pr], N, n_ism, n_threads)[0]


# --------------------------------------------------------------------------- #
# Eq. (7) and the Section 4 helpers
# --------------------------------------------------------------------------- #
def t60_sabine(L, beta) -> float:
    return float(_load().oracle_t60_sabine(_dp(_d(L, 3)), _dp(_d(beta, 6))))


def beta_sabine(L, T60, weights=None, negative: bool = False):
    """Reflection coefficients for a wanted T60; None if infeasible (alpha >= 1)."""
    w = _d(np.ones(6) if weights is None else weights, 6)
    out = np.zeros(6, np.float64)
    rc = _load().oracle_beta_sabine(_dp(_d(L, 3)), float(T60), _dp(w), int(bool(negative)), _dp(out))
    return None if rc != 0 else out


def att2t_sabine(att_dB, T60) -> float:
    return float(_load().oracle_att2t_sabine(float(att_dB), float(T60)))


def nb_img_from_t(T, L, c, Tw):
    out = np.zeros(3, np.int32)
    _load().oracle_nb_img_from_t(float(T), _dp(_d(L, 3)), float(c), float(Tw), _ip(out))
    return out


# --------------------------------------------------------------------------- #
# Diffuse tail (Section 2.2, eq. (8)), Philox4x32-10 noise
# --------------------------------------------------------------------------- #
def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    _load().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def noise_word(seed: int, rir: int, k: int) -> int:
    return int(_load().oracle_noise_word(int(seed), int(rir), int(k)))


def uniform_f32(x: int) -> np.float32:
    return np.float32(_load().oracle_uniform_f32(int(x) & 0xFFFFFFFF))


def ln_f32(x) -> np.float32:
    return np.float32(_load().oracle_ln_f32(float(np.float32(x))))


def ln_f32_array(x) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    y = np.empty_like(x)
    Fp = ctypes.POINTER(ctypes.c_float)
    _load().oracle_ln_f32_array(x.ctypes.data_as(Fp), y.ctypes.data_as(Fp), int(x.size))
    return y


def logistic_f32(u) -> np.float32:
    return np.float32(_load().oracle_logistic_f32(float(np.float32(u))))


def noise(seed: int, rir: int, k0: int, n: int) -> np.ndarray:
    """Logistic noise z for samples k0..k0+n-1 of RIR `rir` (FP32, bit-exact spec)."""
    z = np.zeros(int(n), np.float32)
    if n:
        _load().oracle_noise(int(seed), int(rir), int(k0), int(n),
                             z.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return z


def envelope_amp(h_ism, n_ism: int, fs: float, T60: float) -> float:
    h = np.ascontiguousarray(np.asarray(h_ism, dtype=np.float64))
    assert h.shape[0] >= n_ism
    return float(_load().oracle_envelope_amp(_dp(h), int(n_ism), float(fs), float(T60)))


def envelope_sqrt(A, k, n_ism, fs, T60) -> float:
    return float(_load().oracle_envelope_sqrt(float(A), int(k), int(n_ism), float(fs), float(T60)))


def tail(seed: int, rir: int, A: float, n_ism: int, n_s: int, fs: float, T60: float) -> np.ndarray:
    """Returns h[0:n_s] with zeros below n_ism and the diffuse tail above."""
    h = np.zeros(int(n_s), np.float64)
    _load().oracle_tail(int(seed), int(rir), float(A), int(n_ism), int(n_s), float(fs), float(T60), _dp(h))
    return h


# --------------------------------------------------------------------------- #
# Lehmann-Johansson energy-decay envelope (Section 2.2 cites it; a reading)
# --------------------------------------------------------------------------- #
LJ_NODES = 96   # Gauss-Legendre nodes per angle (quadrature error < 1e-11 while c t sum_a -ln(rho_a) / L_a < 300)


def _gauss_legendre(n):
    x, w = np.polynomial.legendre.leggauss(int(n))
    return np.ascontiguousarray(x), np.ascontiguousarray(w)


def lj_energy(L, beta, c, t, nodes: int = LJ_NODES):
    """E(t): the energy arriving at time t from the images of the room, relative
    to t = 0 (the average over directions of prod_a rho_a^(c t |u_a| / L_a),
    rho_a = |beta_a0 beta_a1|).  t: scalar or array (seconds)."""
    x, w = _gauss_legendre(nodes)
    tt = np.ascontiguousarray(np.atleast_1d(np.asarray(t, np.float64)))
    out = np.zeros(tt.shape[0], np.float64)
    _load().oracle_lj_energy_many(_dp(_d(L, 3)), _dp(_d(beta, 6)), float(c), _dp(tt), int(tt.shape[0]), _dp(x),
                                  _dp(w), int(nodes), _dp(out))
    return out if np.ndim(t) else float(out[0])


def envelope_amp_lj(h_ism, n_ism: int, fs: float, L, beta, c, nodes: int = LJ_NODES) -> float:
    """Envelope amplitude at t0 = n_ism / fs for the Lehmann-Johansson decay: the
    mean over the last W = ceil(0.02 fs) image-source samples of
    h[k]^2 E(t0) / E(t_k) (their power brought forward to t0 along the same
    decay; 0 if E(t0) = 0)."""
    h = np.asarray(h_ism, np.float64)
    W = min(int(math.ceil(0.02 * fs)), int(n_ism))
    if W <= 0:
        return 0.0
    k = np.arange(n_ism - W, n_ism)
    E = lj_energy(L, beta, c, np.concatenate([[n_ism / fs], k / fs]), nodes)
    if not E[0] > 0.0:
        return 0.0
    acc = 0.0
    for i in range(W):   # fixed order, one sample at a time
        acc += h[k[i]] ** 2 * (E[0] / E[1 + i])
    return acc / W


def tail_lj(seed: int, rir: int, A: float, n_ism: int, n_s: int, fs: float, L, beta, c, ks=None,
            nodes: int = LJ_NODES) -> np.ndarray:
    """The diffuse tail with the Lehmann-Johansson envelope: h[k] = z_k sqrt(A E(t_k) / E(t0))
    for n_ism <= k < n_s (z_k the noise of ``noise``); returns h[0:n_s] with zeros
    below n_ism, or, when ``ks`` lists sample indices, the tail at those samples only."""
    ks_arr = np.arange(n_ism, n_s) if ks is None else np.asarray(ks, np.int64)
    E = lj_energy(L, beta, c, np.concatenate([[n_ism / fs], ks_arr / fs]), nodes)
    z = np.array([noise(seed, rir, int(k), 1)[0] for k in ks_arr], np.float64) if ks is not None else \
        noise(seed, rir, n_ism, n_s - n_ism).astype(np.float64)
    env = np.zeros_like(E[1:]) if not E[0] > 0.0 else np.sqrt(A * E[1:] / E[0])
    if ks is not None:
        return z * env
    h = np.zeros(int(n_s), np.float64)
    h[n_ism:] = z * env
    return h


# --------------------------------------------------------------------------- #
# Gradient (not in the paper): derivative of eq. (1)-(6)
# --------------------------------------------------------------------------- #
def rir_grad(L, beta, c, fs, Tw, ps, pr, N, n_ism, g):
    """dLoss/d(beta[6], ps[3], pr[3]) for one pair given g = dLoss/dh[0:n_ism]."""
    g = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
    assert g.shape[0] >= n_ism
    db, dps, dpr = np.zeros(6), np.zeros(3), np.zeros(3)
    Nn = np.ascontiguousarray(np.asarray(N, dtype=np.int32).reshape(3))
    _load().oracle_rir_grad(_dp(_d(L, 3)), _dp(_d(beta, 6)), float(c), float(fs), float(Tw),
                            _dp(_d(ps, 3)), _dp(_d(pr, 3)), _ip(Nn), int(n_ism), _dp(g),
                            _dp(db), _dp(dps), _dp(dpr))
    return db, dps, dpr


# --------------------------------------------------------------------------- #
# The library call of Section 4
# --------------------------------------------------------------------------- #
def n_samples(T: float, fs: float) -> int:
    """Samples covering [0, T): ceil(T fs (1 - 1e-6)), in FP64 from the FP32 inputs.

    The relative slack absorbs the FP32 rounding of T (1.2 s is stored as
    1.20000005 s, which would otherwise add a sample at 48 kHz)."""
    return int(math.ceil(float(T) * float(fs) * (1.0 - 1e-6)))


def simulate(L, beta, c, fs, pos_src, pos_rcv, N, Tmax, Tdiff=None, Tw=None, seed: int = 0,
             pairs=None, n_threads: int = 0, env_amp=None, envelope: str = "sabine"):
    """RIRs for all (source, receiver) pairs, [n_src, n_rcv, n_S] FP64.

    ISM (eq. (5)-(6)) for samples k < n_ism = ceil(Tdiff fs), diffuse tail
    (eq. (8)) for n_ism <= k < n_S = ceil(Tmax fs).  RIR index r = i_src * n_rcv
    + i_rcv keys the noise.  ``pairs`` restricts the work to a list of
    (i_src, i_rcv); the result is then [len(pairs), n_S].  ``env_amp`` maps an
    RIR index to an externally supplied envelope amplitude (for comparing tails
    given the same A).  ``envelope``: "sabine" (eq. (7)-(8)) or "lj" (the
    Lehmann-Johansson energy decay, ``lj_energy``).
    """
    ps_all = np.asarray(pos_src, dtype=np.float64).reshape(-1, 3)
    pr_all = np.asarray(pos_rcv, dtype=np.float64).reshape(-1, 3)
    n_rcv = pr_all.shape[0]
    if Tw is None:
        Tw = 4e-3
    n_S = n_samples(Tmax, fs)
    if Tdiff is None or Tdiff <= 0 or Tdiff >= Tmax:
        n_ism = n_S
    else:
        n_ism = n_samples(Tdiff, fs)
    if pairs is None:
        pairs = [(i, j) for i in range(ps_all.shape[0]) for j in range(n_rcv)]
    ps = np.array([ps_all[i] for i, _ in pairs]).reshape(-1, 3)
    pr = np.array([pr_all[j] for _, j in pairs]).reshape(-1, 3)
    h_ism = rir_list(L, beta, c, fs, Tw, ps, pr, N, n_ism, n_threads)
    out = np.zeros((len(pairs), n_S), np.float64)
    out[:, :n_ism] = h_ism
    if n_ism < n_S:
        T60 = t60_sabine(L, beta)
        for idx, (i, j) in enumerate(pairs):
            r = i * n_rcv + j
            if envelope == "lj":
                A = envelope_amp_lj(h_ism[idx], n_ism, fs, L, beta, c) if env_amp is None else float(env_amp[r])
                out[idx, n_ism:] = tail_lj(seed, r, A, n_ism, n_S, fs, L, beta, c)[n_ism:]
                continue
            A = envelope_amp(h_ism[idx], n_ism, fs, T60) if env_amp is None else float(env_amp[r])
            out[idx, n_ism:] = tail(seed, r, A, n_ism, n_S, fs, T60)[n_ism:]
    if len(pairs) == ps_all.shape[0] * n_rcv and pairs == [(i, j) for i in range(ps_all.shape[0])
                                                          for j in range(n_rcv)]:
        return out.reshape(ps_all.shape[0], n_rcv, n_S)
    return out
