"""GPU parity of the Lehmann-Johansson tail envelope (ISM_ENVELOPE_LJ).

The envelope is E(t) / E(t0), E the energy arrival rate of the image sources
averaged over directions (the reading of the energy-decay prediction that
Section 2.2 cites; the oracle's ``lj_energy``).  The GPU evaluates it once per
job with a Gauss-Legendre product rule in FP32 with float-float rates and
compensated sums; the oracle with a 96-node rule in FP64.  Bounds:
* image-source part: the FP32 bound, 1e-5 of the peak (the envelope does not
  touch it);
* envelope amplitude A against the oracle's fit on the oracle's own image-source
  part: 2e-3 relative (A is a mean of squares of the FP32 image-source samples);
* tail given the same A: 1e-6 relative per sample (the noise is bit-exact;
  the envelope carries exp2f's 2 ulp, the compensated sums' 2 ulp and four
  roundings: < 6e-7).
"""
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


def f32(x):
    return np.float32(x)


def _run(L, beta, ps, pr, N, Tmax, fs, Tdiff, Tw, seed, envelope="lj", prec="fp32"):
    ps_t = torch.as_tensor(np.asarray(ps, np.float32).reshape(-1, 3)).cuda()
    pr_t = torch.as_tensor(np.asarray(pr, np.float32).reshape(-1, 3)).cuda()
    n_S = ism.ism_rir_length(Tmax, fs)
    out = torch.full((ps_t.shape[0], pr_t.shape[0], n_S), float("nan"), device="cuda")
    amp = torch.empty(ps_t.shape[0] * pr_t.shape[0], device="cuda")
    job = ism.make_job(L, beta, ps_t, pr_t, N, Tmax, fs, out, Tdiff=Tdiff, Tw=Tw, seed=seed, env_amp=amp,
                       envelope=envelope)
    ism.ism_simulate_batch([job], prec=prec)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(-1, n_S), amp.cpu().numpy()


def _check(L, beta, ps, pr, N, Tmax, fs, Tdiff, Tw, seed, rirs, ks=None, c=343.0):
    got, A = _run(L, beta, ps, pr, N, Tmax, fs, Tdiff, Tw, seed)
    n_S = oracle.n_samples(f32(Tmax), fs)
    n_ism = oracle.n_samples(f32(Tdiff), fs)
    b32 = np.asarray(beta, np.float32).astype(np.float64)
    ps = np.asarray(ps, np.float32).reshape(-1, 3)
    pr = np.asarray(pr, np.float32).reshape(-1, 3)
    fs32, c32 = float(f32(fs)), float(f32(c))
    for r in rirs:
        i, j = divmod(r, pr.shape[0])
        h = oracle.rir(L, b32, c32, fs32, float(f32(Tw)), ps[i], pr[j], N, n_ism)
        peak = np.max(np.abs(h))
        assert np.max(np.abs(got[r, :n_ism] - h)) <= 1e-5 * peak, r
        A_ref = oracle.envelope_amp_lj(h, n_ism, fs32, L, b32, c32)
        assert A[r] == pytest.approx(A_ref, rel=2e-3), r
        kk = np.arange(n_ism, n_S) if ks is None else np.asarray(ks)
        ref = oracle.tail_lj(seed, r, float(A[r]), n_ism, n_S, fs32, L, b32, c32, ks=kk)
        np.testing.assert_allclose(got[r, kk].astype(np.float64), ref, rtol=1e-6, atol=0.0)
    return got, A


def test_lj_tail_small_room_unequal_walls_every_sample():
    """A 4.1 x 3.3 x 2.7 m room with six different walls (one negative), 2 x 3
    pairs, 16 kHz, images to 60 ms, tail to 0.45 s (several envelope chunks and
    a ragged last one): every tail sample against the oracle."""
    L = np.array([4.1, 3.3, 2.7])
    beta = np.array([0.92, 0.85, -0.9, 0.8, 0.75, 0.95], np.float32)
    ps = np.array([[1.0, 1.1, 0.7], [3.0, 2.2, 1.5]], np.float32)
    pr = np.array([[2.0, 1.4, 1.2], [0.6, 0.5, 2.0], [3.1, 2.4, 0.4]], np.float32)
    Tw = 32 / 16000
    N = oracle.nb_img_from_t(0.06, L, 343.0, Tw)
    _check(L, beta, ps, pr, N, 0.45, 16000.0, 0.06, Tw, 21, rirs=range(6))


def test_lj_tail_trajectory_workload_full_launch_sampled():
    """The 512-RIR 48 kHz array workload with the LJ envelope in the launch the
    bench times: six RIRs' image-source parts, amplitudes and 4,000 tail
    samples each against the oracle."""
    room = workloads.trajectory_array()
    beta = oracle.beta_sabine(room.L, room.rt60)
    N = oracle.nb_img_from_t(room.Tdiff, room.L, room.c, room.window())
    n_S = oracle.n_samples(f32(room.Tmax), room.fs)
    n_ism = oracle.n_samples(f32(room.Tdiff), room.fs)
    ks = np.unique(np.concatenate([np.arange(n_ism, n_ism + 1000), np.linspace(n_ism, n_S - 1, 3000).astype(int),
                                   np.arange(n_S - 64, n_S)]))
    _check(room.L, beta, room.pos_src, room.pos_rcv, N, room.Tmax, room.fs, room.Tdiff, room.window(), room.seed,
           rirs=[0, 7, 100, 301, 511], ks=ks)


def test_lj_tail_with_an_absorbing_wall_is_zero_and_batches_are_bitwise():
    """beta = 0 on one wall: every image beyond the first reflections of that
    axis has zero energy, E(t) = 0 after t = 0, so the tail and A are zero.
    Mixed launch set: a Sabine job and an LJ job in one ism_simulate_batch
    equal their separate calls bit for bit."""
    L = np.array([3.7, 2.9, 2.3])
    beta = np.array([0.9, 0.0, 0.85, 0.7, 0.95, 0.6], np.float32)
    ps = np.array([[1.0, 1.1, 0.7]], np.float32)
    pr = np.array([[2.0, 1.4, 1.2]], np.float32)
    Tw = 32 / 16000
    N = oracle.nb_img_from_t(0.05, L, 343.0, Tw)
    got, A = _run(L, beta, ps, pr, N, 0.2, 16000.0, 0.05, Tw, 3)
    n_ism = oracle.n_samples(f32(0.05), 16000.0)
    assert A[0] == 0.0 and np.all(got[0, n_ism:] == 0.0)
    assert np.max(np.abs(got[0, :n_ism])) > 0.0

    beta2 = np.array([0.9, 0.8, 0.85, 0.7, 0.95, 0.6], np.float32)
    a_lj, _ = _run(L, beta2, ps, pr, N, 0.2, 16000.0, 0.05, Tw, 3, envelope="lj")
    a_sb, _ = _run(L, beta2, ps, pr, N, 0.2, 16000.0, 0.05, Tw, 3, envelope="sabine")
    n_S = a_lj.shape[1]
    assert np.array_equal(a_lj[:, :n_ism].view(np.uint32), a_sb[:, :n_ism].view(np.uint32))
    ps_t, pr_t = torch.as_tensor(ps).cuda(), torch.as_tensor(pr).cuda()
    o1 = torch.empty((1, 1, n_S), device="cuda")
    o2 = torch.empty((1, 1, n_S), device="cuda")
    jobs = [ism.make_job(L, beta2, ps_t, pr_t, N, 0.2, 16000.0, o1, Tdiff=0.05, Tw=Tw, seed=3, envelope="sabine"),
            ism.make_job(L, beta2, ps_t, pr_t, N, 0.2, 16000.0, o2, Tdiff=0.05, Tw=Tw, seed=3, envelope="lj")]
    ism.ism_simulate_batch(jobs)
    torch.cuda.synchronize()
    assert np.array_equal(o1.cpu().numpy().reshape(-1).view(np.uint32), a_sb.reshape(-1).view(np.uint32))
    assert np.array_equal(o2.cpu().numpy().reshape(-1).view(np.uint32), a_lj.reshape(-1).view(np.uint32))
    # the noise is the same stream: the two tails differ by a positive, smooth factor only
    ratio = a_lj[0, n_ism:] / a_sb[0, n_ism:]
    assert np.all(ratio > 0)


def test_lj_tail_through_the_server_equals_the_direct_call():
    L = np.array([5.2, 4.4, 3.1])
    beta = ism.ism_beta_sabine(L, 0.7)
    ps = np.array([[1.3, 2.1, 1.4]], np.float32)
    pr = np.array([[3.9, 1.2, 1.7], [2.2, 3.3, 0.9]], np.float32)
    Tw = 32 / 16000
    N = ism.ism_nb_img_from_t(0.2, L, 343.0, Tw)
    ref = ism.ism_simulate(L, beta, ps, pr, N, 0.7, 16000.0, 0.2, Tw, seed=9, envelope="lj").cpu().numpy()
    with ism.Server(hbm_budget=1 << 30) as srv:
        t, out = srv.submit(L, beta, ps, pr, N, 0.7, 16000.0, Tdiff=0.2, Tw=Tw, seed=9, envelope="lj")
        srv.wait(t)
    assert np.array_equal(out.view(np.uint32), ref.view(np.uint32))


def test_lj_tail_with_coefficients_in_device_memory_is_bitwise_the_host_form():
    """beta read in place from device memory (ism_job.beta_dev): the envelope's
    quadrature is built on the device from those values, bitwise as from room.beta."""
    L = np.array([5.3, 4.1, 2.9])
    beta = np.array([0.9, 0.82, 0.88, 0.75, 0.93, 0.7], np.float32)
    ps = torch.as_tensor(np.array([[1.2, 1.9, 1.1]], np.float32)).cuda()
    pr = torch.as_tensor(np.array([[3.7, 2.6, 1.8], [0.9, 3.1, 2.2]], np.float32)).cuda()
    Tw = 32 / 16000
    N = oracle.nb_img_from_t(0.08, L, 343.0, Tw)
    n_S = ism.ism_rir_length(0.5, 16000.0)
    outs = []
    for b in (beta, torch.as_tensor(beta).cuda()):
        out = torch.empty((1, 2, n_S), device="cuda")
        job = ism.make_job(L, b, ps, pr, N, 0.5, 16000.0, out, Tdiff=0.08, Tw=Tw, seed=5, envelope="lj")
        ism.ism_simulate_batch([job])
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    assert np.max(np.abs(outs[0])) > 0
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))
