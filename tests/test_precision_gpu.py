"""GPU parity of the other arithmetic forms of the accumulation kernel.

FP32_DIRECT evaluates every image tap in FP32 (the default FP32 form uses the
Chebyshev moments for 32-tap windows); its bound is the FP32 one, 1e-5.

The window and the sinc of eq. (6) are evaluated in packed FP16 (FP16X2) or
read from the windowed-sinc table of eq. (9) (LUT, and LUT_TEX through the
texture unit); every form accumulates in FP32, and the image enumeration,
distances and delays stay in FP32 / float-float.  Each result is compared with
the FP64 oracle: max|err| <= 2e-3 x max|h|, the reduced-precision bound.

BF16X2 is not one of the delivered reduced-precision forms: BF16 keeps 8
significant bits, so rounding a single tap to BF16 may already move it by
2^-8 = 3.9e-3 of its value, and the peak sample of an RIR is one tap of the
direct path: no BF16 tap evaluation can guarantee 2e-3 of the peak.  The form
is kept for the comparison the paper's mixed-precision section invites; its
test checks that it runs, is reproducible, and stays within the error its
arithmetic allows (three roundings of 2^-8 on the largest tap, below 1.2e-2),
and prints the error it reaches.
"""
import numpy as np
import pytest

import oracle
from paper_1810_11359_gb300 import ism, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp16x2": 2e-3, "lut": 2e-3, "fp32_direct": 1e-5, "lut_tex": 2e-3,
       "bf16x2": 1.2e-2}   # bf16x2: not a delivered form (see above); its arithmetic's own bound
PRECS = ["fp16x2", "bf16x2", "lut", "fp32_direct", "lut_tex"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def f32(x):
    return np.float32(x)


def lib_run(L, beta, ps, pr, N, Tmax, fs, prec, Tdiff=0.0, Tw=0.0, c=343.0, seed=0):
    ps_t = torch.as_tensor(np.asarray(ps, np.float32).reshape(-1, 3)).cuda()
    pr_t = torch.as_tensor(np.asarray(pr, np.float32).reshape(-1, 3)).cuda()
    out = ism.ism_simulate(L, beta, ps_t, pr_t, N, Tmax, fs, Tdiff, Tw, c, prec=prec, seed=seed)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def oracle_ism(L, beta, ps, pr, N, n_ism, fs, Tw, c=343.0):
    beta32 = np.asarray(beta, np.float32).astype(np.float64)
    ps = np.asarray(ps, np.float32).reshape(-1, 3).astype(np.float64)
    pr = np.asarray(pr, np.float32).reshape(-1, 3).astype(np.float64)
    pairs_s = np.repeat(ps, pr.shape[0], axis=0)
    pairs_r = np.tile(pr, (ps.shape[0], 1))
    return oracle.rir_list(L, beta32, float(f32(c)), float(f32(fs)), float(f32(Tw)), pairs_s, pairs_r, N, n_ism)


def rel_err(got, ref):
    peak = np.max(np.abs(ref))
    assert peak > 0
    assert np.all(np.isfinite(got))
    return float(np.max(np.abs(got.astype(np.float64) - ref)) / peak)


@pytest.mark.parametrize("prec", PRECS)
def test_single_rir(prec):
    room = workloads.single_rir()
    n = oracle.n_samples(room.Tmax, room.fs)
    got = lib_run(room.L, room.beta, room.pos_src, room.pos_rcv, room.nb_img, room.Tmax, room.fs, prec,
                  Tw=room.window())
    ref = oracle_ism(room.L, room.beta, room.pos_src, room.pos_rcv, room.nb_img, n, room.fs, room.window())
    e = rel_err(got.reshape(1, -1), ref)
    print(f"{prec} single RIR: max|err|/peak = {e:.3e}")
    assert e <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("fs,Tw", [(16000.0, 32 / 16000), (16000.0, 6 / 16000), (8000.0, 40 / 8000),
                                   (16000.0, 110.25 / 16000), (8000.0, 256 / 8000)])
def test_window_lengths_and_ragged_rooms(prec, fs, Tw):
    """Integral and non-integral windows of 1 to 8 taps per lane; 2 x 3 pairs
    in a small room with unequal walls, a length that is not a multiple of
    the 256-sample tile."""
    L = np.array([3.7, 2.9, 2.3])
    beta = np.array([0.9, 0.8, 0.85, -0.7, 0.95, 0.6], np.float32)
    ps = np.array([[1.0, 1.1, 0.7], [2.9, 2.2, 1.5]], np.float32)
    pr = np.array([[2.0, 1.4, 1.2], [0.6, 0.5, 2.0], [3.1, 2.4, 0.4]], np.float32)
    Tmax = 0.0731
    N = oracle.nb_img_from_t(Tmax, L, 343.0, Tw)
    n = oracle.n_samples(f32(Tmax), fs)
    got = lib_run(L, beta, ps, pr, N, Tmax, fs, prec, Tw=Tw).reshape(6, n)
    ref = oracle_ism(L, beta, ps, pr, N, n, fs, Tw)
    e = rel_err(got, ref)
    print(f"{prec} fs={fs} Nw={Tw * fs}: max|err|/peak = {e:.3e}")
    assert e <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_trajectory_workload_sampled_rirs_and_tail(prec):
    """The 512-RIR trajectory / 8-microphone workload at 48 kHz in full, in
    the launch the bench times; six RIRs against the oracle, and the tail
    against the oracle's tail for the same fitted amplitude (the tail does
    not depend on the precision form)."""
    room = workloads.trajectory_array()
    beta = oracle.beta_sabine(room.L, room.rt60)
    N = oracle.nb_img_from_t(room.Tdiff, room.L, room.c, room.window())
    n_S = oracle.n_samples(f32(room.Tmax), room.fs)
    n_ism = oracle.n_samples(f32(room.Tdiff), room.fs)
    ps = torch.as_tensor(room.pos_src).cuda()
    pr = torch.as_tensor(room.pos_rcv).cuda()
    out = torch.empty((64, 8, n_S), device="cuda")
    amp = torch.empty(512, device="cuda")
    job = ism.make_job(room.L, beta, ps, pr, N, room.Tmax, room.fs, out, Tdiff=room.Tdiff, Tw=room.window(),
                       seed=room.seed, env_amp=amp)
    ism.ism_simulate_batch([job], prec=prec)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(512, n_S)
    A = amp.cpu().numpy()
    T60 = oracle.t60_sabine(room.L, np.asarray(beta, np.float32).astype(np.float64))
    worst = 0.0
    for r in [0, 7, 100, 255, 301, 511]:
        i, j = divmod(r, 8)
        ref = oracle_ism(room.L, beta, room.pos_src[i:i + 1], room.pos_rcv[j:j + 1], N, n_ism, room.fs,
                         room.window())
        worst = max(worst, rel_err(got[r:r + 1, :n_ism], ref))
        tail_ref = oracle.tail(room.seed, r, float(A[r]), n_ism, n_S, float(f32(room.fs)), T60)[n_ism:]
        np.testing.assert_allclose(got[r, n_ism:].astype(np.float64), tail_ref, rtol=1e-6,
                                   atol=1e-12 * np.sqrt(A[r]))
    print(f"{prec} trajectory workload: max|err|/peak = {worst:.3e}")
    assert worst <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_reduced_precision_run_to_run_bit_identical(prec):
    r = workloads.single_rir()
    args = (r.L, r.beta, r.pos_src, r.pos_rcv, r.nb_img, r.Tmax, r.fs, prec)
    a = lib_run(*args, Tw=r.window())
    b = lib_run(*args, Tw=r.window())
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("prec", PRECS)
def test_reduced_precision_against_fp32_path_on_batched_workload(prec):
    """The 128-RIR 6 x 5 x 3 m workload: each reduced form against the FP32
    path on the same GPU, and one RIR against the oracle."""
    room = workloads.batched_fp32()
    beta = oracle.beta_sabine(room.L, room.rt60)
    N = oracle.nb_img_from_t(room.Tmax, room.L, room.c, room.window())
    ref32 = lib_run(room.L, beta, room.pos_src, room.pos_rcv, N, room.Tmax, room.fs, "fp32", Tw=room.window())
    got = lib_run(room.L, beta, room.pos_src, room.pos_rcv, N, room.Tmax, room.fs, prec, Tw=room.window())
    e32 = rel_err(got.reshape(128, -1), ref32.reshape(128, -1).astype(np.float64))
    ref = oracle_ism(room.L, beta, room.pos_src[1:2], room.pos_rcv[17:18], N, 9600, room.fs, room.window())
    e = rel_err(got[1, 17][None], ref)
    print(f"{prec} batched workload: vs FP32 path {e32:.3e}, vs oracle {e:.3e}")
    assert e <= TOL[prec] and e32 <= TOL[prec]
