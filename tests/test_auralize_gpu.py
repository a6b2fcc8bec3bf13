"""Moving sources on the GPU (Section 4): segment-wise filtering of a source
signal by the RIRs of the trajectory points, overlap-added (ism_auralize),
against the FP64 oracle (oracle.auralize, pinned in test_oracle_pins.py).

FP32 multiply-adds in a fixed order: the error bound used is 1e-5 of the
largest sum of the terms' magnitudes, (|x| * |h|)[t], which bounds the FP32
accumulation error of up to ~60k terms with a wide margin (the measured error
is printed).  The FFT form (ism_auralize_ex, ISM_AURALIZE_FFT) is held to the
same bound: an FP32 FFT's error is a few units of 2^-24 times log2 N of the
transformed energy, spread over every output, so it is measured against the
largest magnitude sum, not each output's own.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1810_11359_gb300 import ism, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def check(got, x, h, starts=None, tol=1e-5):
    x64 = np.asarray(x, np.float32).astype(np.float64)
    h64 = np.asarray(h, np.float32).astype(np.float64)
    ref = oracle.auralize(x64, h64, starts)
    mag = oracle.auralize(np.abs(x64), np.abs(h64), starts)
    assert got.shape == ref.shape and np.all(np.isfinite(got))
    err = np.max(np.abs(got.astype(np.float64) - ref)) / np.max(mag)
    print(f"auralize {h.shape} n_x={x.size}: max|err| / max(|x|*|h|) = {err:.3e}")
    assert err <= tol
    return err


def run(x, h, starts=None, method=None, workspace=None):
    out = ism.ism_auralize(x, h, starts=starts, method=method, workspace=workspace)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("n_x,n_points,n_mics,n_s", [(1000, 7, 3, 300), (257, 1, 9, 1), (4099, 64, 8, 517),
                                                     (300, 300, 2, 129), (50, 3, 1, 2000), (1500, 11, 9, 1024)])
def test_random_shapes_against_oracle(n_x, n_points, n_mics, n_s):
    """Ragged sizes: tails of the 128-output tiles and 128-tap chunks, mic groups
    of 8 plus a remainder, one segment, one sample per segment, RIRs longer
    than the signal; RIR lengths that are multiples of 4 take the 128-bit tap
    staging, the others the scalar one."""
    rng = np.random.default_rng(n_x + n_points)
    x = rng.normal(size=n_x).astype(np.float32)
    h = rng.normal(size=(n_points, n_mics, n_s)).astype(np.float32)
    check(run(x, h), x, h)


def test_explicit_uneven_segments():
    rng = np.random.default_rng(8)
    x = rng.normal(size=2000).astype(np.float32)
    h = rng.normal(size=(5, 4, 700)).astype(np.float32)
    starts = [0, 3, 900, 901, 1700]
    got = run(x, h, starts)
    check(got, x, h, starts + [2000])
    # samples before the first start are not emitted
    got2 = run(x, h, [100, 300, 900, 901, 1700])
    x2 = x.copy()
    x2[:100] = 0.0
    check(got2, x2, h, [0, 300, 900, 901, 1700, 2000])


def test_run_to_run_bit_identical():
    rng = np.random.default_rng(9)
    x = rng.normal(size=5000).astype(np.float32)
    h = rng.normal(size=(10, 8, 3000)).astype(np.float32)
    a, b = run(x, h), run(x, h)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_trajectory_workload_moving_source():
    """The 48 kHz workload end to end: 64 trajectory points x 8 microphones,
    1.2 s RIRs (image sources and tail) from the library, a 1.2 s seeded
    noise burst as the source signal; outputs sampled across the whole
    length are checked one by one against the definition (the full oracle
    would take minutes)."""
    room = workloads.trajectory_array()
    beta = ism.ism_beta_sabine(room.L, room.rt60)
    N = ism.ism_nb_img_from_t(room.Tdiff, room.L, room.c, room.window())
    h = ism.ism_simulate(room.L, beta, room.pos_src, room.pos_rcv, N, room.Tmax, room.fs, room.Tdiff, room.window(),
                         seed=room.seed)
    rng = np.random.default_rng(12)
    n_x = h.shape[2]
    x = rng.normal(size=n_x).astype(np.float32)
    y = ism.ism_auralize(x, h)
    torch.cuda.synchronize()
    y = y.cpu().numpy()
    hh = h.cpu().numpy().astype(np.float64)
    x64 = x.astype(np.float64)
    starts = oracle.segment_starts(n_x, hh.shape[0])
    seg = np.searchsorted(starts, np.arange(n_x), side="right") - 1
    worst = 0.0
    for m, t in [(0, 0), (3, 777), (7, 14400), (1, 57599), (5, 60000), (2, 115198), (6, 90001)]:
        s = np.arange(max(0, t - hh.shape[2] + 1), min(t, n_x - 1) + 1)
        terms = x64[s] * hh[seg[s], m, t - s]
        ref, mag = terms.sum(), np.abs(terms).sum()
        if mag == 0:
            assert y[m, t] == 0.0
            continue
        worst = max(worst, abs(float(y[m, t]) - ref) / mag)
    print(f"trajectory auralization: max|err| / sum|terms| = {worst:.3e}")
    assert worst <= 1e-5


# --------------------------------------------------------------------------- #
# FFT form (four-step FFTs in shared memory, frequency-domain overlap-add)
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("n_x,n_points,n_mics,n_s", [(1000, 7, 3, 300), (257, 1, 9, 1), (4099, 64, 8, 517),
                                                     (300, 300, 2, 129), (50, 3, 1, 2000), (1500, 11, 9, 1024),
                                                     (20000, 20, 17, 3000)])
def test_fft_random_shapes_against_oracle(n_x, n_points, n_mics, n_s):
    """The direct form's shapes and one with 9 microphone pairs (two pair
    groups in the row pass): DFT lengths 2^11 .. 2^15, odd and even powers
    (a radix-2 stage or not), an odd microphone count (a pair with an empty
    imaginary part), one point, one sample per segment."""
    rng = np.random.default_rng(n_x + n_points + 7)
    x = rng.normal(size=n_x).astype(np.float32)
    h = rng.normal(size=(n_points, n_mics, n_s)).astype(np.float32)
    check(run(x, h, method="fft"), x, h)


def test_fft_explicit_uneven_segments_and_chunks():
    """Caller-given segment starts (repeated and clamped ones); a workspace
    that holds only a few points per chunk gives bitwise the same result as
    one chunk (the spectra are summed in ascending point order either way)."""
    rng = np.random.default_rng(18)
    x = rng.normal(size=2000).astype(np.float32)
    h = rng.normal(size=(5, 4, 700)).astype(np.float32)
    starts = [0, 3, 900, 901, 1700]
    got = run(x, h, starts, method="fft")
    check(got, x, h, starts + [2000])
    got2 = run(x, h, [100, 300, 900, 901, 1700], method="fft")
    x2 = x.copy()
    x2[:100] = 0.0
    check(got2, x2, h, [0, 300, 900, 901, 1700, 2000])
    h2 = rng.normal(size=(23, 6, 900)).astype(np.float32)
    x3 = rng.normal(size=3000).astype(np.float32)
    one = run(x3, h2, method="fft")
    # a workspace of the spectra plus two points: 12 chunks (the sizes of one and two points give both)
    s1 = ism.ism_auralize_workspace_size(3000, 1, 6, 900, "fft")
    s2 = ism.ism_auralize_workspace_size(3000, 2, 6, 900, "fft")
    assert ism.ism_auralize_workspace_size(3000, 23, 6, 900, "fft") >= s1 + 22 * (s2 - s1)   # one chunk by default
    ws = torch.empty(s2, dtype=torch.uint8, device="cuda")
    xd, hd = torch.as_tensor(x3).cuda(), torch.as_tensor(h2).cuda()
    many_t = torch.empty((6, 3000 + 900 - 1), device="cuda")
    lib = ism.load()
    st = lib.ism_auralize_ex(ctypes.c_void_p(xd.data_ptr()), 3000, ctypes.c_void_p(hd.data_ptr()), 23, 6, 900, None,
                             ctypes.c_void_p(many_t.data_ptr()), ism.AURALIZE_METHODS["fft"],
                             ctypes.c_void_p(ws.data_ptr()), s2, None)
    assert st == 0, lib.ism_last_error_message().decode()
    torch.cuda.synchronize()
    many = many_t.cpu().numpy()
    assert np.array_equal(one.view(np.uint32), many.view(np.uint32))
    check(many, x3, h2)
    # a workspace below one point is refused
    st = lib.ism_auralize_ex(ctypes.c_void_p(xd.data_ptr()), 3000, ctypes.c_void_p(hd.data_ptr()), 23, 6, 900, None,
                             ctypes.c_void_p(many_t.data_ptr()), ism.AURALIZE_METHODS["fft"],
                             ctypes.c_void_p(ws.data_ptr()), s1 - 256, None)
    assert st == 3


def test_fft_run_to_run_bit_identical_and_close_to_direct():
    rng = np.random.default_rng(19)
    x = rng.normal(size=5000).astype(np.float32)
    h = rng.normal(size=(10, 8, 3000)).astype(np.float32)
    a, b = run(x, h, method="fft"), run(x, h, method="fft")
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    d = run(x, h, method="direct")
    assert np.array_equal(d.view(np.uint32), run(x, h).view(np.uint32))   # "direct" is ism_auralize
    check(a, x, h)


def test_fft_trajectory_workload_moving_source():
    """The 48 kHz array (64 points x 8 microphones, 1.2 s RIRs with tails, a 1.2 s
    signal) through the automatic choice, which takes the FFT form here: outputs
    sampled over the whole length against the definition, and every output
    against the direct form."""
    room = workloads.trajectory_array()
    beta = ism.ism_beta_sabine(room.L, room.rt60)
    N = ism.ism_nb_img_from_t(room.Tdiff, room.L, room.c, room.window())
    h = ism.ism_simulate(room.L, beta, room.pos_src, room.pos_rcv, N, room.Tmax, room.fs, room.Tdiff, room.window(),
                         seed=room.seed)
    rng = np.random.default_rng(12)
    n_x = h.shape[2]
    x = rng.normal(size=n_x).astype(np.float32)
    assert ism.ism_auralize_workspace_size(n_x, 64, 8, n_x, "auto") > 0   # the automatic choice is the FFT form
    y = run(x, h, method="auto")
    yd = run(x, h)
    hh = h.cpu().numpy().astype(np.float64)
    x64 = x.astype(np.float64)
    starts = oracle.segment_starts(n_x, hh.shape[0])
    seg = np.searchsorted(starts, np.arange(n_x), side="right") - 1
    errs, mags = [], []
    for m, t in [(0, 0), (3, 777), (7, 14400), (1, 57599), (5, 60000), (2, 115198), (6, 90001), (4, 30000)]:
        s = np.arange(max(0, t - hh.shape[2] + 1), min(t, n_x - 1) + 1)
        terms = x64[s] * hh[seg[s], m, t - s]
        errs.append(abs(float(y[m, t]) - terms.sum()))
        mags.append(np.abs(terms).sum())
    scale = max(mags)
    print(f"trajectory auralization (FFT): max|err| / max sum|terms| = {max(errs) / scale:.3e}")
    assert max(errs) <= 1e-5 * scale
    diff = np.max(np.abs(y.astype(np.float64) - yd)) / scale
    print(f"FFT vs direct form over all outputs: {diff:.3e} of the largest magnitude sum")
    assert diff <= 1e-5


@pytest.mark.parametrize("n_x,n_s,n_mics", [(30000, 20000, 8), (100000, 90000, 5), (150000, 150001, 8),
                                             (400000, 300000, 3)])
def test_fft_long_signals_sampled_against_the_definition(n_x, n_s, n_mics):
    """DFT lengths 2^16 (rows of 256, one warp per row sequence), 2^18 (rows of
    512, three pairs in one group), 2^19 (columns of 1024, rows of 512: three
    microphone pairs per row-pass CTA, so 4 pairs take two groups, the second
    with idle warps) and 2^20 (rows of 1024, the CTA-wide row pass: one pair per
    CTA), three trajectory points: outputs sampled over the whole length against
    the definition (scaled by the largest magnitude sum among them), and every
    output against the direct form."""
    rng = np.random.default_rng(n_x)
    x = rng.normal(size=n_x).astype(np.float32)
    h = (rng.normal(size=(3, n_mics, n_s)) * np.exp(-np.arange(n_s) / (n_s / 4.0))).astype(np.float32)
    y = run(x, h, method="fft")
    x64, h64 = x.astype(np.float64), h.astype(np.float64)
    starts = oracle.segment_starts(n_x, 3)
    seg = np.searchsorted(starts, np.arange(n_x), side="right") - 1
    n_out = n_x + n_s - 1
    errs, mags = [], []
    for t in rng.integers(0, n_out, 12).tolist() + [0, n_out - 1, n_x - 1]:
        m = t % n_mics
        s = np.arange(max(0, t - n_s + 1), min(t, n_x - 1) + 1)
        terms = x64[s] * h64[seg[s], m, t - s]
        errs.append(abs(float(y[m, t]) - terms.sum()))
        mags.append(np.abs(terms).sum())
    scale = max(mags)
    print(f"FFT n_out={n_out}: max|err| / max sum|terms| = {max(errs) / scale:.3e}")
    assert max(errs) <= 1e-5 * scale
    d = run(x, h, method="direct")
    assert np.max(np.abs(y.astype(np.float64) - d)) <= 1e-5 * scale
