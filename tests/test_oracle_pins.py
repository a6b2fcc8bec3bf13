"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-derived
fixtures (tests/golden/), closed forms, invariants, an independent naive
enumeration (Allen-Berkley (m, q) form), brute force, a vendor library
(cuRAND's host Philox generator) or finite differences.  CPU only.
"""
import ctypes
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append([float(v) for v in line.split()])
    return out


# --------------------------------------------------------------------------- #
# Section 2.1: the grid and eq. (1)-(4)
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 22, 73, 87, 141])
def test_grid_bounds_count(N):
    lo, hi = oracle.grid_bounds(N)
    assert hi - lo == N
    assert lo == math.ceil(-N / 2) and hi == math.ceil(N / 2)


def test_image_count_closed_form():
    N = [5, 4, 3]
    res = oracle.enumerate_images([3, 4, 2.5], [0.7] * 6, 343.0, [1, 1.5, 1.2], [2, 2.5, 1.5], N)
    assert res["count"] == 5 * 4 * 3
    assert len({tuple(r) for r in res["n"]}) == 60


def test_exponents_hand_fixture():
    for n, e0, e1 in _rows("exponents_hand.txt"):
        assert oracle.image_exponents(int(n)) == (int(e0), int(e1))


def test_exponents_by_plane_crossings():
    """Count the mirror planes x = kL crossed between image and receiver."""
    L, xs, xr = 3.0, 0.7, 2.1
    for n in range(-9, 10):
        x = oracle.image_coord(n, L, xs)
        assert x == pytest.approx(n * L + xs if n % 2 == 0 else (n + 1) * L - xs)
        lo, hi = sorted((x, xr))
        ks = [k for k in range(-20, 21) if lo < k * L < hi]
        hits0 = sum(1 for k in ks if k % 2 == 0)
        hits1 = sum(1 for k in ks if k % 2 != 0)
        assert oracle.image_exponents(n) == (hits0, hits1), n


def _allen_berkley_images(L, beta, ps, pr, M):
    """Independent naive enumeration in the (m, q) form of Allen and Berkley:
    coordinate 2 m L + (1 - 2 q) x_s, weight beta_0^|m-q| beta_1^|m| per axis."""
    out = []
    rng = range(-M, M + 1)
    for mx in rng:
        for qx in (0, 1):
            for my in rng:
                for qy in (0, 1):
                    for mz in rng:
                        for qz in (0, 1):
                            m, q = (mx, my, mz), (qx, qy, qz)
                            pos, e, w = [], [], 1.0
                            for a in range(3):
                                pos.append(2 * m[a] * L[a] + (1 - 2 * q[a]) * ps[a])
                                e0, e1 = abs(m[a] - q[a]), abs(m[a])
                                e += [e0, e1]
                                w *= beta[2 * a] ** e0 * beta[2 * a + 1] ** e1
                            d = math.sqrt(sum((pr[a] - pos[a]) ** 2 for a in range(3)))
                            out.append((tuple(pos), tuple(e), w, d))
    return out


def test_bijection_with_allen_berkley():
    """Paper grid N = 2(2M+1) per axis is the (m, q) grid m in [-M, M], q in {0,1}."""
    L, beta = [3.0, 4.0, 2.5], [0.7, 0.6, 0.5, 0.8, 0.9, 0.4]
    ps, pr = [1.0, 1.5, 1.2], [2.0, 2.5, 1.5]
    M = 2
    N = [2 * (2 * M + 1)] * 3
    res = oracle.enumerate_images(L, beta, 343.0, ps, pr, N)
    ab = _allen_berkley_images(L, beta, ps, pr, M)
    assert res["count"] == len(ab) == 1000
    key = lambda pos, e: (tuple(round(v, 9) for v in pos), tuple(e))
    mine = {key(res["pos"][i], res["e"][i]): (res["A"][i], res["d"][i]) for i in range(res["count"])}
    theirs = {key(p, e): (w / (4 * math.pi * d), d) for p, e, w, d in ab}
    assert mine.keys() == theirs.keys()
    for k in mine:
        assert mine[k][0] == pytest.approx(theirs[k][0], rel=1e-13, abs=1e-300)
        assert mine[k][1] == pytest.approx(theirs[k][1], rel=1e-13)


def _windowed_sinc_plain(x, Nw):
    """Eq. (6) in the sample variable, written from the textbook forms
    cos^2 window and sin(pi x)/(pi x)."""
    if abs(x) >= Nw / 2:
        return 0.0
    w = math.cos(math.pi * x / Nw) ** 2
    s = 1.0 if x == 0 else math.sin(math.pi * x) / (math.pi * x)
    return w * s


def test_brute_force_tiny_room():
    """Eq. (5)-(6) summed over every sample and every image of the (m, q) grid."""
    L, beta = [3.0, 4.0, 2.5], [0.7, 0.6, 0.5, 0.8, 0.9, 0.4]
    ps, pr = [1.0, 1.5, 1.2], [2.0, 2.5, 1.5]
    c, fs, Tw = 343.0, 16000.0, 32 / 16000.0
    M = 1
    N = [2 * (2 * M + 1)] * 3
    n_ism = 700
    h = oracle.rir(L, beta, c, fs, Tw, ps, pr, N, n_ism)
    ref = np.zeros(n_ism)
    for pos, e, w, d in _allen_berkley_images(L, beta, ps, pr, M):
        s = fs * d / c
        A = w / (4 * math.pi * d)
        for k in range(n_ism):
            ref[k] += A * _windowed_sinc_plain(k - s, Tw * fs)
    peak = np.max(np.abs(ref))
    assert peak > 0
    assert np.max(np.abs(h - ref)) <= 1e-13 * peak


def test_direct_path_integer_delay_fixture():
    (k, val), = _rows("direct_path.txt")
    h = oracle.rir([6, 5, 4], [0.0] * 6, 300.0, 1000.0, 32 / 1000.0, [1, 1, 1], [4, 1, 1], [7, 7, 7], 40)
    k = int(k)
    assert h[k] == pytest.approx(val, rel=1e-15)
    others = np.delete(h, k)
    assert np.all(others == 0.0)


def test_beta_zero_leaves_direct_path():
    L, ps, pr = [5.0, 4.0, 3.0], [1.1, 2.3, 0.9], [3.7, 1.2, 2.2]
    c, fs, Tw = 343.0, 16000.0, 32 / 16000.0
    h = oracle.rir(L, [0.0] * 6, c, fs, Tw, ps, pr, [9, 9, 9], 400)
    d = math.dist(ps, pr)
    s = fs * d / c
    ref = np.array([_windowed_sinc_plain(k - s, 32.0) / (4 * math.pi * d) for k in range(400)])
    assert np.max(np.abs(h - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_swap_invariance():
    L, beta = [4.0, 3.5, 2.7], [0.8, 0.7, 0.9, 0.6, 0.75, 0.85]
    ps, pr = [1.2, 0.8, 1.9], [3.1, 2.6, 0.7]
    c, fs, Tw = 343.0, 16000.0, 32 / 16000.0
    N = [11, 11, 11]
    a = oracle.rir(L, beta, c, fs, Tw, ps, pr, N, 1200)
    b = oracle.rir(L, beta, c, fs, Tw, pr, ps, N, 1200)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


def test_negative_beta_sign_pattern():
    """Section 2.2: with beta -> -beta every image is weighted by (-1)^(hits)."""
    L, beta = [4.0, 3.5, 2.7], [0.8, 0.7, 0.9, 0.6, 0.75, 0.85]
    ps, pr = [1.2, 0.8, 1.9], [3.1, 2.6, 0.7]
    pos = oracle.enumerate_images(L, beta, 343.0, ps, pr, [5, 5, 5])
    neg = oracle.enumerate_images(L, [-b for b in beta], 343.0, ps, pr, [5, 5, 5])
    sign = (-1.0) ** pos["e"].sum(axis=1)
    np.testing.assert_allclose(neg["A"], sign * pos["A"], rtol=1e-15)


def test_delta_prime_properties():
    fs, Tw = 16000.0, 32 / 16000.0
    assert oracle.delta_prime(0.0, fs, Tw) == 1.0
    for j in range(1, 16):
        assert oracle.delta_prime(float(j), fs, Tw) == 0.0
        assert oracle.delta_prime(float(-j), fs, Tw) == 0.0
    for x in [0.3, 1.7, 5.25, 15.9]:
        assert oracle.delta_prime(x, fs, Tw) == pytest.approx(oracle.delta_prime(-x, fs, Tw), rel=1e-15)
        assert oracle.delta_prime(x, fs, Tw) == pytest.approx(_windowed_sinc_plain(x, 32.0), rel=1e-13)
    assert oracle.delta_prime(16.0, fs, Tw) == 0.0
    assert oracle.delta_prime(16.5, fs, Tw) == 0.0


# --------------------------------------------------------------------------- #
# eq. (7) and the Section 4 helpers
# --------------------------------------------------------------------------- #
def test_sabine_hand_fixture():
    for Lx, Ly, Lz, b, T60 in _rows("sabine_hand.txt"):
        assert oracle.t60_sabine([Lx, Ly, Lz], [b] * 6) == pytest.approx(T60, rel=1e-13)


def test_sabine_roundtrip_and_infeasible():
    for L, T in [([6, 5, 3], 0.6), ([10, 8, 3.5], 1.2), ([3, 4, 2.5], 0.7), ([7.3, 4.1, 3.3], 0.25)]:
        b = oracle.beta_sabine(L, T)
        assert b is not None
        assert oracle.t60_sabine(L, b) == pytest.approx(T, rel=1e-12)
        bn = oracle.beta_sabine(L, T, negative=True)
        np.testing.assert_array_equal(bn, -b)
    w = [1, 1, 0.5, 0.5, 2, 2]
    b = oracle.beta_sabine([6, 5, 3], 0.6, weights=w)
    assert oracle.t60_sabine([6, 5, 3], b) == pytest.approx(0.6, rel=1e-12)
    # alpha >= 1 is infeasible: tiny T60 in a small room
    assert oracle.beta_sabine([3, 3, 3], 0.01) is None


def test_att2t():
    assert oracle.att2t_sabine(60.0, 0.8) == pytest.approx(0.8)
    assert oracle.att2t_sabine(13.0, 0.6) == pytest.approx(0.13)


def test_nb_img_config_values_and_completeness():
    assert list(oracle.nb_img_from_t(0.6, [6, 5, 3], 343.0, 32 / 16000)) == [73, 87, 141]
    # no image that reaches the receiver before T is missing: a larger grid
    # changes nothing in [0, T)
    L, beta = [3.0, 2.5, 2.2], [0.9] * 6
    ps, pr = [1.0, 0.7, 1.1], [2.1, 1.8, 0.6]
    c, fs, Tw, T = 343.0, 8000.0, 32 / 8000.0, 0.06
    N = oracle.nb_img_from_t(T, L, c, Tw)
    n = oracle.n_samples(T, fs)
    a = oracle.rir(L, beta, c, fs, Tw, ps, pr, N, n)
    b = oracle.rir(L, beta, c, fs, Tw, ps, pr, [x + 4 for x in N], n)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


# --------------------------------------------------------------------------- #
# Diffuse tail: Philox4x32-10, the FP32 uniform / ln / logistic spec, eq. (8)
# --------------------------------------------------------------------------- #
def _curand_host():
    for p in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    """cuRAND's host PHILOX4_32_10 generator (default ordering) emits, as its
    b-th block of four words, Philox4x32-10 of counter (b div 65536, 0,
    b mod 65536, 0) under key (seed low, seed high)."""
    cr = _curand_host()
    if cr is None:
        pytest.skip("libcurand not available")
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    for seed in (0x123456789ABCDEF0, 7, 0xFFFFFFFFFFFFFFFF):
        gen = ctypes.c_void_p()
        assert cr.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
        try:
            assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            n_blocks = 65536 + 64
            buf = np.zeros(4 * n_blocks, np.uint32)
            assert cr.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(buf.size)) == 0
            blocks = buf.reshape(-1, 4)
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for b in list(range(0, 40)) + list(range(65530, 65536 + 64)):
                ctr = [b // 65536, 0, b % 65536, 0]
                assert oracle.philox4x32_10(ctr, key) == [int(v) for v in blocks[b]], (seed, b)
        finally:
            cr.curandDestroyGenerator(gen)


def test_noise_word_layout():
    seed, rir = 0xDEADBEEF12345678, 17
    for k in range(0, 40):
        blk = oracle.philox4x32_10([k // 4, rir, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle.noise_word(seed, rir, k) == blk[k % 4]


def test_uniform_exact_and_symmetric():
    assert oracle.uniform_f32(0) == np.float32(2.0 ** -24)
    assert oracle.uniform_f32(0xFFFFFFFF) == np.float32(1 - 2.0 ** -24)
    rng = np.random.default_rng(1)
    for x in rng.integers(0, 2 ** 32, 200, dtype=np.uint64):
        u = oracle.uniform_f32(int(x))
        m = int(x) >> 9
        assert float(u) == (2 * m + 1) * 2.0 ** -24
        v = oracle.uniform_f32(int(x) ^ 0xFFFFFE00)
        assert float(u) + float(v) == 1.0


def test_ln_f32_exhaustive_over_noise_domain():
    """Every ratio u/(1-u) the noise transform can produce: <= 2 ulp of ln."""
    m = np.arange(0, 1 << 23, dtype=np.float64)
    u = ((2 * m + 1) * 2.0 ** -24).astype(np.float32)
    x = (u / (np.float32(1) - u)).astype(np.float32)
    y = oracle.ln_f32_array(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    err = np.abs(y - ref) / ulp
    assert err.max() <= 2.0, err.max()


def test_logistic_distribution_moments():
    seed = 99
    z = np.concatenate([oracle.noise(seed, r, 0, 50000) for r in range(4)]).astype(np.float64)
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.02
    # logistic CDF with unit variance: F(z) = 1 / (1 + exp(-pi z / sqrt 3))
    zs = np.sort(z)
    F = 1.0 / (1.0 + np.exp(-math.pi * zs / math.sqrt(3)))
    ks = np.max(np.abs(F - (np.arange(1, zs.size + 1) / zs.size)))
    assert ks < 1.63 / math.sqrt(zs.size) * 1.5


def test_tail_decay_slope_and_level():
    """Eq. (8) read as a 60 dB decay in T60: the fitted energy slope of the
    tail is -60/T60 dB/s and its power at t0 continues A."""
    fs, T60, n_ism, n_s, A = 8000.0, 0.8, 800, 8000, 2.5e-4
    rirs = [oracle.tail(5, r, A, n_ism, n_s, fs, T60)[n_ism:] for r in range(16)]
    p = np.mean(np.stack(rirs) ** 2, axis=0)
    blocks = p[: (p.size // 400) * 400].reshape(-1, 400).mean(axis=1)
    t = (np.arange(blocks.size) * 400 + 200) / fs
    slope, icpt = np.polyfit(t, 10 * np.log10(blocks), 1)
    assert slope == pytest.approx(-60.0 / T60, rel=0.03)
    assert 10 ** (icpt / 10) == pytest.approx(A, rel=0.1)


def test_envelope_amp_on_exact_exponential():
    """If the ISM part already decays as eq. (8), the estimate returns its level at t0."""
    fs, T60, n_ism, A0 = 16000.0, 0.5, 4000, 3e-3
    k = np.arange(n_ism)
    h = np.sqrt(A0 * 10 ** (-6 * (k - n_ism) / fs / T60))
    assert oracle.envelope_amp(h, n_ism, fs, T60) == pytest.approx(A0, rel=1e-12)


# --------------------------------------------------------------------------- #
# Lehmann-Johansson energy-decay envelope (Section 2.2 cites it; a reading)
# --------------------------------------------------------------------------- #
def test_lj_energy_rigid_walls_do_not_decay():
    """|beta| = 1 on every wall: no image loses energy, E(t) = 1 at all times."""
    for beta in ([1, 1, 1, 1, 1, 1], [-1, 1, 1, -1, -1, -1]):
        np.testing.assert_allclose(oracle.lj_energy([5.0, 4.0, 3.0], beta, 343.0, [0.0, 0.05, 0.7, 3.0]), 1.0,
                                   rtol=1e-13)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_lj_energy_one_absorbing_axis_closed_form(axis):
    """Only the walls of one axis absorb (rho = |b0 b1| < 1): |u_a| is uniform on
    [0, 1] over the sphere, so E(t) = int_0^1 rho^(k mu) dmu = (1 - e^-K) / K with
    K = -ln(rho) c t / L_a."""
    L = [4.3, 3.1, 2.6]
    beta = [1.0] * 6
    beta[2 * axis], beta[2 * axis + 1] = 0.6, -0.85
    rho = 0.6 * 0.85
    for t in (0.01, 0.1, 0.45, 1.3):
        K = -math.log(rho) * 343.0 * t / L[axis]
        assert oracle.lj_energy(L, beta, 343.0, t) == pytest.approx((1 - math.exp(-K)) / K, rel=1e-11)


def test_lj_energy_depends_on_wall_products_and_axis_symmetry():
    """The energy of an image depends on the two walls of an axis through their
    product only (each is hit half of the time), and the directional average
    does not prefer an axis: permuting the axes with their walls changes nothing."""
    L = [6.0, 5.0, 3.0]
    a = oracle.lj_energy(L, [0.5, 0.8, 0.9, 0.7, 0.6, 0.95], 343.0, [0.05, 0.3])
    b = oracle.lj_energy(L, [0.8, 0.5, -0.7, -0.9, 0.95, 0.6], 343.0, [0.05, 0.3])
    c = oracle.lj_energy(L, [math.sqrt(0.4)] * 2 + [math.sqrt(0.63)] * 2 + [math.sqrt(0.57)] * 2, 343.0, [0.05, 0.3])
    np.testing.assert_allclose(a, b, rtol=1e-12)
    np.testing.assert_allclose(a, c, rtol=1e-12)
    d = oracle.lj_energy([3.0, 6.0, 5.0], [0.6, 0.95, 0.5, 0.8, 0.9, 0.7], 343.0, [0.05, 0.3])
    np.testing.assert_allclose(a, d, rtol=1e-11)


def test_lj_energy_initial_decay_is_eyring():
    """For short times E(t) ~ 1 - t c sum_a (-ln rho_a) <|u_a|> / L_a with <|u_a|> = 1/2 over
    the sphere; with one absorption alpha on every wall (rho = 1 - alpha) that is
    Eyring's energy decay rate c S (-ln(1 - alpha)) / (4 V)."""
    L = np.array([7.0, 5.0, 3.2])
    alpha = 0.3
    b = math.sqrt(1 - alpha)
    V = float(np.prod(L))
    S = 2 * (L[0] * L[1] + L[1] * L[2] + L[0] * L[2])
    rate = 343.0 * S * (-math.log(1 - alpha)) / (4 * V)
    h = 1e-6
    slope = (oracle.lj_energy(L, [b] * 6, 343.0, h) - oracle.lj_energy(L, [b] * 6, 343.0, 0.0)) / h
    assert slope == pytest.approx(-rate, rel=1e-4)
    # and it falls monotonically, log-convex (a mixture of exponentials)
    t = np.linspace(0.0, 1.0, 41)
    E = oracle.lj_energy(L, [b] * 6, 343.0, t)
    assert np.all(np.diff(E) < 0)
    assert np.all(np.diff(np.log(E), 2) >= -1e-12)


def test_lj_energy_follows_the_energy_decay_of_the_images():
    """Brute force: the energy sum A_n^2 of the images whose delay falls in each
    20 ms window (eq. (1)-(4), enumerated by the oracle) decays with the slope
    of E(t) within 2 %, and its level is c / (4 pi V) E(t) on average within 10 %;
    the Sabine exponential misses the slope of this room with unequal walls by
    more than 25 %."""
    L = np.array([5.0, 4.0, 3.0])
    beta = np.array([0.9, 0.85, 0.95, 0.8, 0.7, 0.9])
    c, T = 343.0, 0.6
    N = oracle.nb_img_from_t(T, L, c, 0.0)
    im = oracle.enumerate_images(L, beta, c, [1.2, 1.7, 1.1], [3.9, 2.2, 1.8], N)
    edges = np.arange(0.02, T, 0.02)
    E_img = np.histogram(im["tau"], bins=edges, weights=im["A"] ** 2)[0] / np.diff(edges)
    mid = 0.5 * (edges[1:] + edges[:-1])
    pred = c / (4 * math.pi * np.prod(L)) * oracle.lj_energy(L, beta, c, mid)
    sel = (mid > 0.05) & (mid < 0.56)
    s_img = np.polyfit(mid[sel], np.log(E_img[sel]), 1)[0]
    s_lj = np.polyfit(mid[sel], np.log(pred[sel]), 1)[0]
    assert s_lj == pytest.approx(s_img, rel=0.02)
    assert math.exp(np.mean(np.log(E_img[sel] / pred[sel]))) == pytest.approx(1.0, abs=0.1)
    s_sabine = -6 * math.log(10) / oracle.t60_sabine(L, beta)
    assert abs(s_sabine / s_img - 1) > 0.25


def test_lj_envelope_amp_and_tail_level():
    """If the image-source part already follows the decay E(t), the amplitude
    fit returns its level at t0; the tail continues it: mean z^2 E(t) / E(t0) A."""
    L, beta, c, fs, n_ism = [6.0, 5.0, 3.0], [0.9, 0.8, 0.85, 0.9, 0.7, 0.95], 343.0, 8000.0, 1600
    k = np.arange(n_ism)
    E = oracle.lj_energy(L, beta, c, np.concatenate([[n_ism / fs], k / fs]))
    A0 = 2e-3
    h = np.sqrt(A0 * E[1:] / E[0])
    assert oracle.envelope_amp_lj(h, n_ism, fs, L, beta, c) == pytest.approx(A0, rel=1e-12)
    n_s = 8000
    rirs = np.stack([oracle.tail_lj(3, r, A0, n_ism, n_s, fs, L, beta, c)[n_ism:] for r in range(8)])
    Et = oracle.lj_energy(L, beta, c, np.arange(n_ism, n_s) / fs) / E[0]
    ratio = np.mean(rirs ** 2, axis=0) / (A0 * Et)   # unit-variance noise: mean 1
    assert np.mean(ratio) == pytest.approx(1.0, abs=0.03)
    # the noise is the bit-exact stream of the Sabine tail, only the envelope differs
    z = oracle.noise(3, 5, n_ism, 50).astype(np.float64)
    np.testing.assert_allclose(oracle.tail_lj(3, 5, A0, n_ism, n_s, fs, L, beta, c, ks=np.arange(n_ism, n_ism + 50)),
                               z * np.sqrt(A0 * Et[:50]), rtol=1e-14)


# --------------------------------------------------------------------------- #
# Gradient: FP64 central finite differences of the oracle's own forward
# --------------------------------------------------------------------------- #
def test_gradient_matches_central_differences():
    L = [4.0, 3.5, 2.7]
    beta = np.array([0.8, 0.7, 0.9, 0.6, 0.75, 0.85])
    ps, pr = np.array([1.2, 0.8, 1.9]), np.array([3.1, 2.6, 0.7])
    c, fs, Tw, N, n = 343.0, 8000.0, 32 / 8000.0, [7, 7, 7], 500
    rng = np.random.default_rng(3)
    target = rng.standard_normal(n) * 1e-3

    def loss(b, s, r):
        h = oracle.rir(L, b, c, fs, Tw, s, r, N, n)
        return float(np.sum((h - target) ** 2))

    h = oracle.rir(L, beta, c, fs, Tw, ps, pr, N, n)
    g = 2 * (h - target)
    db, dps, dpr = oracle.rir_grad(L, beta, c, fs, Tw, ps, pr, N, n, g)
    eps = 1e-6

    def fd(vec, i, which):
        vp, vm = vec.copy(), vec.copy()
        vp[i] += eps
        vm[i] -= eps
        args_p = {"b": beta, "s": ps, "r": pr}
        args_m = dict(args_p)
        args_p[which], args_m[which] = vp, vm
        return (loss(args_p["b"], args_p["s"], args_p["r"]) - loss(args_m["b"], args_m["s"], args_m["r"])) / (2 * eps)

    for i in range(6):
        assert db[i] == pytest.approx(fd(beta, i, "b"), rel=1e-5, abs=1e-9)
    for i in range(3):
        assert dps[i] == pytest.approx(fd(ps, i, "s"), rel=1e-5, abs=1e-9)
        assert dpr[i] == pytest.approx(fd(pr, i, "r"), rel=1e-5, abs=1e-9)


def test_gradient_at_beta_zero_product_rule():
    """At beta = 0 only first-order images have non-zero d/dbeta (product form)."""
    L = [4.0, 3.5, 2.7]
    ps, pr = np.array([1.2, 0.8, 1.9]), np.array([3.1, 2.6, 0.7])
    c, fs, Tw, N, n = 343.0, 8000.0, 32 / 8000.0, [5, 5, 5], 300
    g = np.ones(n)
    db, _, _ = oracle.rir_grad(L, [0.0] * 6, c, fs, Tw, ps, pr, N, n, g)
    eps = 1e-7
    for w in range(6):
        b = np.zeros(6)
        b[w] = eps
        fd = (oracle.rir(L, b, c, fs, Tw, ps, pr, N, n).sum() - oracle.rir(L, np.zeros(6), c, fs, Tw, ps, pr, N, n).sum()) / eps
        assert db[w] == pytest.approx(fd, rel=1e-5)


# --------------------------------------------------------------------------- #
# Receiver polar patterns (Section 4 names them; the first-order formula
# g = alpha + (1 - alpha) cos(theta) is the reading taken)
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("pattern,front,side,back", [
    ("omni", 1.0, 1.0, 1.0),
    ("subcardioid", 1.0, 0.75, 0.5),
    ("cardioid", 1.0, 0.5, 0.0),
    ("hypercardioid", 1.0, 0.25, -0.5),
    ("bidirectional", 1.0, 0.0, -1.0),
])
def test_pattern_gain_textbook_values(pattern, front, side, back):
    """A receiver at pr looking along +x: an image straight ahead, at 90 degrees
    and straight behind gives the textbook gains of each first-order pattern
    (cardioid null behind, figure-eight nulls at the sides and inverted rear
    lobe, hypercardioid rear lobe -1/2); the length of the orientation vector
    does not matter."""
    pr = np.array([1.0, 2.0, 1.5])
    for o in ([1.0, 0.0, 0.0], [3.5, 0.0, 0.0]):
        assert oracle.pattern_gain(pattern, o, pr, pr + [4.0, 0, 0]) == pytest.approx(front, abs=1e-15)
        assert oracle.pattern_gain(pattern, o, pr, pr + [0, -2.5, 0]) == pytest.approx(side, abs=1e-15)
        assert oracle.pattern_gain(pattern, o, pr, pr + [0, 0, 7.0]) == pytest.approx(side, abs=1e-15)
        assert oracle.pattern_gain(pattern, o, pr, pr + [-0.3, 0, 0]) == pytest.approx(back, abs=1e-15)
    # 60 degrees off axis: cos = 1/2
    a = {"omni": 1.0, "subcardioid": 0.75, "cardioid": 0.5, "hypercardioid": 0.25, "bidirectional": 0.0}[pattern]
    img = pr + [1.0, math.sqrt(3.0), 0.0]
    assert oracle.pattern_gain(pattern, [1, 0, 0], pr, img) == pytest.approx(a + (1 - a) * 0.5, abs=1e-15)


def test_pattern_direct_path_only_scales_by_the_gain():
    """With beta = 0 only the direct path remains, so every sample of a patterned
    RIR is the omnidirectional one times the gain toward the source, computed
    here from the positions alone."""
    L = [4.0, 3.5, 2.7]
    ps, pr = np.array([1.2, 0.8, 1.9]), np.array([3.1, 2.6, 0.7])
    c, fs, Tw, N, n = 343.0, 8000.0, 32 / 8000.0, [5, 5, 5], 200
    h0 = oracle.rir(L, [0.0] * 6, c, fs, Tw, ps, pr, N, n)
    o = np.array([0.3, -1.0, 0.4])
    u = (ps - pr) / np.linalg.norm(ps - pr)
    cos_t = float(np.dot(o / np.linalg.norm(o), u))
    for pat, a in oracle.PATTERN_ALPHA.items():
        h = oracle.rir_list_pattern(L, [0.0] * 6, c, fs, Tw, [ps], [pr], [o], pat, N, n)[0]
        np.testing.assert_allclose(h, (a + (1 - a) * cos_t) * h0, rtol=1e-12, atol=1e-15)


def test_pattern_linear_in_alpha_and_omni_is_no_pattern():
    """g is affine in alpha, so every pattern's RIR is alpha times the
    omnidirectional RIR plus (1 - alpha) times the figure-eight one; omni is
    bit for bit the RIR without a pattern, and flipping the orientation
    negates the figure-eight RIR exactly."""
    L = [3.7, 2.9, 2.3]
    beta = [0.9, 0.8, 0.85, -0.7, 0.95, 0.6]
    ps, pr = [[1.0, 1.1, 0.7], [2.9, 2.2, 1.5]], [[2.0, 1.4, 1.2], [0.6, 0.5, 2.0]]
    o = [[0.2, 0.9, -0.3], [-1.0, 0.1, 0.5]]
    c, fs, Tw, N, n = 343.0, 16000.0, 32 / 16000, [9, 9, 11], 900
    h = {p: oracle.rir_list_pattern(L, beta, c, fs, Tw, ps, pr, o, p, N, n) for p in oracle.PATTERN_ALPHA}
    h_plain = oracle.rir_list(L, beta, c, fs, Tw, ps, pr, N, n)
    assert np.array_equal(h["omni"], h_plain)
    for p, a in oracle.PATTERN_ALPHA.items():
        np.testing.assert_allclose(h[p], a * h["omni"] + (1 - a) * h["bidirectional"], rtol=1e-9,
                                   atol=1e-12 * np.max(np.abs(h_plain)))
    flipped = oracle.rir_list_pattern(L, beta, c, fs, Tw, ps, pr, -np.asarray(o), "bidirectional", N, n)
    assert np.array_equal(flipped, -h["bidirectional"])


# --------------------------------------------------------------------------- #
# Moving sources (Section 4): segment-wise filtering with overlap-add
# --------------------------------------------------------------------------- #
def test_auralize_brute_force_tiny():
    """Against a plain double loop over (segment, sample, tap) on tiny inputs."""
    rng = np.random.default_rng(3)
    x = rng.normal(size=23)
    h = rng.normal(size=(4, 2, 6))
    starts = oracle.segment_starts(23, 4)
    assert starts == [0, 5, 11, 17, 23]
    y = oracle.auralize(x, h, starts)
    ref = np.zeros((2, 23 + 6 - 1))
    for p in range(4):
        for s in range(starts[p], starts[p + 1]):
            for m in range(2):
                for k in range(6):
                    ref[m, s + k] += x[s] * h[p, m, k]
    np.testing.assert_allclose(y, ref, rtol=1e-13, atol=1e-13)


def test_auralize_delayed_impulses_closed_form():
    """RIRs that are single scaled impulses: each microphone hears each segment
    delayed and scaled by its point's impulse, so the output is a sum of shifted
    copies of the segments, written here by indexing alone."""
    rng = np.random.default_rng(4)
    n_x, n_points, n_s = 300, 7, 40
    x = rng.normal(size=n_x)
    d = rng.integers(0, n_s, size=(n_points, 3))
    g = rng.normal(size=(n_points, 3))
    h = np.zeros((n_points, 3, n_s))
    for p in range(n_points):
        for m in range(3):
            h[p, m, d[p, m]] = g[p, m]
    starts = oracle.segment_starts(n_x, n_points)
    ref = np.zeros((3, n_x + n_s - 1))
    for p in range(n_points):
        a, b = starts[p], starts[p + 1]
        for m in range(3):
            ref[m, a + d[p, m]:b + d[p, m]] += g[p, m] * x[a:b]
    np.testing.assert_allclose(oracle.auralize(x, h), ref, rtol=1e-14, atol=1e-14)


def test_auralize_static_source_is_one_filter():
    """Identical RIRs at every point (a static source): the segments partition
    the signal, so the result is the signal filtered once, for any cut."""
    rng = np.random.default_rng(5)
    x = rng.normal(size=257)
    h1 = rng.normal(size=(2, 31))
    one = oracle.auralize(x, h1[None])
    for n_points in (2, 5, 16):
        many = oracle.auralize(x, np.repeat(h1[None], n_points, axis=0))
        np.testing.assert_allclose(many, one, rtol=1e-12, atol=1e-12)
    # explicit, uneven cut
    many = oracle.auralize(x, np.repeat(h1[None], 3, axis=0), [0, 10, 200, 257])
    np.testing.assert_allclose(many, one, rtol=1e-12, atol=1e-12)
