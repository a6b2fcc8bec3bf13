"""GPU parity: libism (through its C ABI) against the FP64 oracle.

Floating point: max|err| <= 1e-5 x max|h| of the oracle RIR (FP32 bound).
Integer work (noise words, the logistic transform): bit-exact.
Run-to-run and batch-vs-alone: bit-identical.
"""
import numpy as np
import pytest

import oracle
from paper_1810_11359_gb300 import ism, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def f32(x):
    return np.float32(x)


def lib_run(L, beta, ps, pr, N, Tmax, fs, Tdiff=0.0, Tw=0.0, c=343.0, seed=0):
    ps_t = torch.as_tensor(np.asarray(ps, np.float32).reshape(-1, 3)).cuda()
    pr_t = torch.as_tensor(np.asarray(pr, np.float32).reshape(-1, 3)).cuda()
    out = ism.ism_simulate(L, beta, ps_t, pr_t, N, Tmax, fs, Tdiff, Tw, c, seed=seed)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def oracle_ism(L, beta, ps, pr, N, n_ism, fs, Tw, c=343.0):
    """Oracle ISM part for every pair, from the FP32 values the library sees."""
    beta32 = np.asarray(beta, np.float32).astype(np.float64)
    ps = np.asarray(ps, np.float32).reshape(-1, 3).astype(np.float64)
    pr = np.asarray(pr, np.float32).reshape(-1, 3).astype(np.float64)
    pairs_s = np.repeat(ps, pr.shape[0], axis=0)
    pairs_r = np.tile(pr, (ps.shape[0], 1))
    return oracle.rir_list(L, beta32, float(f32(c)), float(f32(fs)), float(f32(Tw)), pairs_s, pairs_r, N, n_ism)


def assert_close(got, ref, tol=TOL_FP32, what=""):
    peak = np.max(np.abs(ref))
    err = np.max(np.abs(got.astype(np.float64) - ref))
    assert peak > 0, what
    assert err <= tol * peak, f"{what}: max|err|/peak = {err / peak:.3e} > {tol:.1e}"
    return err / peak


def test_single_rir_plain():
    room = workloads.single_rir()
    n = oracle.n_samples(room.Tmax, room.fs)
    got = lib_run(room.L, room.beta, room.pos_src, room.pos_rcv, room.nb_img, room.Tmax, room.fs, Tw=room.window())
    ref = oracle_ism(room.L, room.beta, room.pos_src, room.pos_rcv, room.nb_img, n, room.fs, room.window())
    assert got.shape == (1, 1, 4800)
    assert_close(got.reshape(1, -1), ref, what="single RIR")


@pytest.mark.parametrize("beta", [[0.9, 0.8, 0.85, 0.7, 0.95, 0.6], [-0.9, 0.8, -0.85, 0.7, 0.95, -0.6],
                                  [1.0, 1.0, 0.99, 0.99, 1.0, 0.98]])
def test_small_room_many_pairs_ragged(beta):
    rng = np.random.default_rng(11)
    L = np.array([4.3, 3.7, 2.9])
    ps = (0.3 + rng.random((3, 3)) * (L - 0.6)).astype(np.float32)
    pr = (0.3 + rng.random((5, 3)) * (L - 0.6)).astype(np.float32)
    fs, Tmax, Tw = 16000.0, 0.0531, 32 / 16000
    N = oracle.nb_img_from_t(Tmax, L, 343.0, Tw)
    n = oracle.n_samples(f32(Tmax), fs)
    got = lib_run(L, beta, ps, pr, N, Tmax, fs, Tw=Tw)
    ref = oracle_ism(L, beta, ps, pr, N, n, fs, Tw)
    assert got.shape == (3, 5, n)
    assert_close(got.reshape(15, -1), ref, what="small room")


@pytest.mark.parametrize("fs,Tw", [(16000.0, 4e-3),          # 64 taps: two taps per lane
                                   (16000.0, 40 / 16000),    # 40 taps: masked window
                                   (44100.0, 2.5e-3),        # 110.25 taps: non-integer window
                                   (16000.0, 6 / 16000),     # 6 taps
                                   (8000.0, 256 / 8000)])    # 256 taps: widest window
def test_window_lengths(fs, Tw):
    L = np.array([3.3, 4.1, 2.6])
    beta = [0.8, 0.75, 0.9, 0.7, 0.85, 0.65]
    ps = np.array([[1.1, 0.9, 1.3], [2.9, 3.5, 0.4]], np.float32)
    pr = np.array([[2.2, 2.8, 1.9]], np.float32)
    Tmax = 0.04
    N = oracle.nb_img_from_t(Tmax, L, 343.0, Tw)
    n = oracle.n_samples(f32(Tmax), f32(fs))
    got = lib_run(L, beta, ps, pr, N, Tmax, fs, Tw=Tw)
    ref = oracle_ism(L, beta, ps, pr, N, n, fs, Tw)
    assert_close(got.reshape(2, -1), ref, what=f"Tw={Tw} fs={fs}")


def test_beta_zero_is_direct_path_only():
    L = np.array([5.0, 4.0, 3.0])
    ps, pr = np.array([[1.1, 2.3, 0.9]], np.float32), np.array([[3.7, 1.2, 2.2]], np.float32)
    N = [9, 9, 9]
    got = lib_run(L, [0.0] * 6, ps, pr, N, 0.05, 16000.0, Tw=32 / 16000)[0, 0]
    ref = oracle_ism(L, [0.0] * 6, ps, pr, N, got.size, 16000.0, 32 / 16000)[0]
    assert_close(got, ref, what="beta=0")
    nz = np.nonzero(got)[0]
    assert nz.size <= 32


def test_integer_delay_fixture_on_gpu():
    # c = 300, fs = 1000, d = 3: direct path exactly at sample 10, A = 1/(12 pi)
    got = lib_run([6.0, 5.0, 4.0], [0.0] * 6, [[1, 1, 1]], [[4, 1, 1]], [7, 7, 7], 0.04, 1000.0, Tw=32 / 1000,
                  c=300.0)[0, 0]
    assert got[10] == pytest.approx(1 / (12 * np.pi), rel=2e-6)
    others = np.delete(got, 10)
    assert np.max(np.abs(others)) <= 1e-6 * got[10]


def test_grid_of_one_image_per_axis():
    L = np.array([3.0, 4.0, 2.5])
    ps, pr = np.array([[1.0, 1.5, 1.2]], np.float32), np.array([[2.0, 2.5, 1.5]], np.float32)
    got = lib_run(L, [0.7] * 6, ps, pr, [1, 1, 1], 0.02, 16000.0, Tw=32 / 16000)[0, 0]
    ref = oracle_ism(L, [0.7] * 6, ps, pr, [1, 1, 1], got.size, 16000.0, 32 / 16000)[0]
    assert_close(got, ref, what="N=1")


def test_very_short_rirs():
    L = np.array([3.0, 4.0, 2.5])
    ps, pr = np.array([[0.2, 0.2, 0.2]], np.float32), np.array([[0.25, 0.21, 0.2]], np.float32)
    for Tmax in (1 / 16000, 3 / 16000, 17 / 16000, 33 / 16000):
        got = lib_run(L, [0.7] * 6, ps, pr, [5, 5, 5], Tmax, 16000.0, Tw=32 / 16000)[0, 0]
        n = oracle.n_samples(f32(Tmax), 16000.0)
        assert got.size == n
        ref = oracle_ism(L, [0.7] * 6, ps, pr, [5, 5, 5], n, 16000.0, 32 / 16000)[0]
        assert np.max(np.abs(got - ref)) <= TOL_FP32 * max(np.max(np.abs(ref)), 1e-3)


def test_bit_identical_run_to_run():
    room = workloads.batched_fp32()
    beta = oracle.beta_sabine(room.L, room.rt60)
    N = [21, 25, 39]
    outs = [lib_run(room.L, beta, room.pos_src, room.pos_rcv[:8], N, 0.1, room.fs, Tw=room.window())
            for _ in range(5)]
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))


def test_batch_equals_separate_calls_bitwise():
    rooms = workloads.differentiation_rooms(6, seed=21)
    ref_outs, jobs, keep = [], [], []
    for i, r in enumerate(rooms):
        beta = oracle.beta_sabine(r.L, r.rt60)
        N = oracle.nb_img_from_t(0.08, r.L, 343.0, r.window())
        Tdiff = 0.05 if i % 2 else 0.0
        alone = lib_run(r.L, beta, r.pos_src, r.pos_rcv, N, 0.08, r.fs, Tdiff=Tdiff, Tw=r.window(), seed=100 + i)
        ref_outs.append(alone)
        ps = torch.as_tensor(r.pos_src).cuda()
        pr = torch.as_tensor(r.pos_rcv).cuda()
        out = torch.empty_like(torch.as_tensor(alone)).cuda()
        keep.append((ps, pr, out))
        jobs.append(ism.make_job(r.L, beta, ps, pr, N, 0.08, r.fs, out, Tdiff=Tdiff, Tw=r.window(), seed=100 + i))
    ism.ism_simulate_batch(jobs)
    torch.cuda.synchronize()
    for (ps, pr, out), alone in zip(keep, ref_outs):
        assert np.array_equal(out.cpu().numpy().view(np.uint32), alone.view(np.uint32))


@pytest.mark.parametrize("order", ["alike", "different"])
def test_fused_and_direct_jobs_in_one_set_equal_separate_calls(order):
    """One launch set mixing fused jobs (dense rooms) and a direct job (a sparse
    48 kHz room) between them: with the fused jobs' shell counts alike the
    fused CTAs go by shell rank over all their RIRs, with different counts job
    by job; either way every job's RIRs are bitwise those of its own call."""
    dense = [(np.array([4.0, 3.5, 2.8]), [[1.1, 2.4, 1.3]], [[2.9, 0.8, 1.7], [0.7, 3.0, 2.2]]),
             (np.array([3.6, 4.2, 2.9]), [[2.5, 1.0, 0.9]], [[0.9, 3.1, 2.0]])]
    Tmax_dense = [0.2, 0.2] if order == "alike" else [0.2, 0.35]
    sparse = (np.array([10.0, 8.0, 3.5]), [[2.0, 3.0, 1.2]], [[7.5, 5.0, 1.6], [7.6, 5.1, 1.6]])
    specs = [(dense[0], Tmax_dense[0], 16000.0), (sparse, 0.05, 48000.0), (dense[1], Tmax_dense[1], 16000.0)]
    jobs, keep, refs = [], [], []
    for (L, src, rcv), Tmax, fs in specs:
        beta = oracle.beta_sabine(L, 0.5)
        Tw = 32 / fs
        N = oracle.nb_img_from_t(Tmax, L, 343.0, Tw)
        refs.append(lib_run(L, beta, src, rcv, N, Tmax, fs, Tw=Tw))
        ps = torch.as_tensor(np.asarray(src, np.float32)).cuda()
        pr = torch.as_tensor(np.asarray(rcv, np.float32)).cuda()
        out = torch.full(refs[-1].shape, float("nan"), device="cuda")
        keep.append((ps, pr, out))
        jobs.append(ism.make_job(L, beta, ps, pr, N, Tmax, fs, out, Tw=Tw))
    ism.ism_simulate_batch(jobs)
    torch.cuda.synchronize()
    for (ps, pr, out), ref in zip(keep, refs):
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_batched_config_full_size_sampled_rirs():
    """The 128-RIR 6 x 5 x 3 m workload at full size, in the bench's launch;
    four RIRs compared in full against the oracle."""
    room = workloads.batched_fp32()
    beta = oracle.beta_sabine(room.L, room.rt60)
    N = oracle.nb_img_from_t(room.Tmax, room.L, room.c, room.window())
    assert list(N) == [73, 87, 141]
    got = lib_run(room.L, beta, room.pos_src, room.pos_rcv, N, room.Tmax, room.fs, Tw=room.window())
    assert got.shape == (4, 32, 9600)
    assert np.all(np.isfinite(got))
    for (i, j) in [(0, 0), (1, 17), (2, 31), (3, 5)]:
        ref = oracle_ism(room.L, beta, room.pos_src[i:i + 1], room.pos_rcv[j:j + 1], N, 9600, room.fs, room.window())
        assert_close(got[i, j][None], ref, what=f"pair {i},{j}")


def test_noise_bit_exact():
    for seed, rir, k0, n in [(0, 0, 0, 4096), (0xDEADBEEF12345678, 511, 14398, 1 << 20), (7, 3, 1, 1001)]:
        z = ism.ism_diffuse_noise(seed, rir, k0, n).cpu().numpy()
        ref = oracle.noise(seed, rir, k0, n)
        assert np.array_equal(z.view(np.uint32), ref.view(np.uint32)), (seed, rir, k0)


def test_tail_and_envelope_given_same_amplitude():
    room = workloads.trajectory_array()
    beta = oracle.beta_sabine(room.L, room.rt60)
    N = oracle.nb_img_from_t(room.Tdiff, room.L, room.c, room.window())
    assert list(N) == [25, 29, 63]
    sel_src = room.pos_src[[0, 37]]
    ps = torch.as_tensor(sel_src).cuda()
    pr = torch.as_tensor(room.pos_rcv).cuda()
    n_S = oracle.n_samples(f32(room.Tmax), room.fs)
    n_ism = oracle.n_samples(f32(room.Tdiff), room.fs)
    out = torch.empty((2, 8, n_S), device="cuda")
    amp = torch.empty(16, device="cuda")
    job = ism.make_job(room.L, beta, ps, pr, N, room.Tmax, room.fs, out, Tdiff=room.Tdiff, Tw=room.window(),
                       seed=room.seed, env_amp=amp)
    ism.ism_simulate_batch([job])
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(16, n_S)
    A = amp.cpu().numpy()
    ism_ref = oracle_ism(room.L, beta, sel_src, room.pos_rcv, N, n_ism, room.fs, room.window())
    assert_close(got[:, :n_ism], ism_ref, what="ISM part")
    T60 = oracle.t60_sabine(room.L, np.asarray(beta, np.float32).astype(np.float64))
    for r in range(16):
        A_ref = oracle.envelope_amp(ism_ref[r], n_ism, float(f32(room.fs)), T60)
        assert A[r] == pytest.approx(A_ref, rel=2e-3), r
        tail_ref = oracle.tail(room.seed, r, float(A[r]), n_ism, n_S, float(f32(room.fs)), T60)[n_ism:]
        tail = got[r, n_ism:].astype(np.float64)
        np.testing.assert_allclose(tail, tail_ref, rtol=1e-6, atol=1e-12 * np.sqrt(A[r]))


def test_invalid_positions_flagged_on_device():
    L = np.array([3.0, 4.0, 2.5])
    ps = torch.tensor([[1.0, 1.5, 1.2], [1.0, 1.5, 3.1]], device="cuda")   # second source above the ceiling
    pr = torch.tensor([[2.0, 2.5, 1.5]], device="cuda")
    ws = ism.Workspace()
    out = ism.ism_simulate(L, [0.7] * 6, ps, pr, [9, 9, 9], 0.05, 16000.0, Tw=32 / 16000, workspace=ws)
    flags = ism.ism_workspace_status(ws.buf)
    assert flags & ism.DEVICE_FLAG_POSITION
    o = out.cpu().numpy()
    assert np.all(o[1] == 0.0)
    assert np.max(np.abs(o[0])) > 0.0
    ok = ism.ism_simulate(L, [0.7] * 6, ps[:1], pr, [9, 9, 9], 0.05, 16000.0, Tw=32 / 16000, workspace=ws)
    assert ism.ism_workspace_status(ws.buf) == 0
    assert np.array_equal(ok.cpu().numpy()[0], o[0])


def test_workspace_too_small_rejected():
    import ctypes
    L = np.array([3.0, 4.0, 2.5])
    ps = torch.tensor([[1.0, 1.5, 1.2]], device="cuda")
    pr = torch.tensor([[2.0, 2.5, 1.5]], device="cuda")
    need = ism.ism_workspace_size(L, [0.7] * 6, 1, 1, [9, 9, 9], 0.05, 16000.0, Tw=32 / 16000)
    buf = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.full((1, 1, 800), 7.0, device="cuda")
    r = ism._room(L, [0.7] * 6, 343.0)
    st = ism.load().ism_simulate(ctypes.byref(r), ctypes.c_void_p(ps.data_ptr()), 1, ctypes.c_void_p(pr.data_ptr()), 1,
                                 ism._nb([9, 9, 9]), 0.05, 16000.0, 0.0, 32 / 16000, 0, 0,
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(buf.data_ptr()), need - 256, None)
    assert st == 3
    assert torch.all(out == 7.0)


def test_host_entry_matches_device_entry():
    room = workloads.single_rir()
    dev = lib_run(room.L, room.beta, room.pos_src, room.pos_rcv, room.nb_img, room.Tmax, room.fs, Tw=room.window())
    host = ism.ism_simulate_host(room.L, room.beta, room.pos_src, room.pos_rcv, room.nb_img, room.Tmax, room.fs,
                                 Tw=room.window())
    assert np.array_equal(dev.view(np.uint32), host.view(np.uint32))


@pytest.mark.parametrize("pinned", [True, False])
def test_host_entry_large_result_in_pieces_matches_device_entry(pinned):
    """A 118 MB result (the 48 kHz array workload: 64 source points x 8
    microphones, 1.2 s with a diffuse tail) into a pinned or a pageable host
    buffer: bitwise the device entry point's RIRs."""
    room = workloads.trajectory_array()
    beta = ism.ism_beta_sabine(room.L, room.rt60)
    N = ism.ism_nb_img_from_t(room.Tdiff, room.L, room.c, room.window())
    n_S = ism.ism_rir_length(room.Tmax, room.fs)
    ps = torch.as_tensor(room.pos_src).cuda()
    pr = torch.as_tensor(room.pos_rcv).cuda()
    dev = torch.empty((ps.shape[0], pr.shape[0], n_S), device="cuda")
    ism.ism_simulate(room.L, beta, ps, pr, N, room.Tmax, room.fs, Tdiff=room.Tdiff, Tw=room.window(), seed=room.seed,
                     out=dev)
    out = torch.empty((ps.shape[0], pr.shape[0], n_S), dtype=torch.float32)
    if pinned:
        out = out.pin_memory()
    out.numpy()[:] = np.nan
    host = ism.ism_simulate_host(room.L, beta, room.pos_src, room.pos_rcv, N, room.Tmax, room.fs, Tdiff=room.Tdiff,
                                 Tw=room.window(), seed=room.seed, out=out.numpy())
    assert np.array_equal(dev.cpu().numpy().view(np.uint32), host.view(np.uint32))


def test_host_entry_repeated_calls_equal_fresh_calls():
    """Repeated host-entry calls with the same arguments and a page-locked result
    replay a CUDA graph of the first call's launches; only the positions change
    from call to call.  Every result must equal, bit for bit, the device entry's
    for the same positions -- including positions seen before, and a dense and a
    sparse room on two lanes and on one."""
    rng = np.random.default_rng(21)
    for room, Tdiff in ((workloads.batched_fp32(), None), (workloads.trajectory_array(), "tdiff")):
        beta = ism.ism_beta_sabine(room.L, room.rt60)
        Td = room.Tdiff if Tdiff else 0.0
        N = ism.ism_nb_img_from_t(Td if Tdiff else room.Tmax, room.L, room.c, room.window())
        n_S = ism.ism_rir_length(room.Tmax, room.fs)
        n_src, n_rcv = room.pos_src.shape[0], room.pos_rcv.shape[0]
        out = torch.empty((n_src, n_rcv, n_S), dtype=torch.float32).pin_memory()
        ws = ism.Workspace()
        pos_sets = [(room.pos_src, room.pos_rcv)]
        for _ in range(2):
            pos_sets.append((workloads._uniform_inside(rng, room.L, n_src), workloads._uniform_inside(rng, room.L, n_rcv)))
        pos_sets.append(pos_sets[0])
        for ps, pr in pos_sets:
            out.numpy()[:] = np.nan
            host = ism.ism_simulate_host(room.L, beta, ps, pr, N, room.Tmax, room.fs, Tdiff=Td, Tw=room.window(),
                                         seed=room.seed, out=out.numpy(), workspace=ws)
            dev = torch.empty((n_src, n_rcv, n_S), device="cuda")
            ism.ism_simulate(room.L, beta, torch.as_tensor(ps).cuda(), torch.as_tensor(pr).cuda(), N, room.Tmax,
                             room.fs, Tdiff=Td, Tw=room.window(), seed=room.seed, out=dev)
            assert np.array_equal(dev.cpu().numpy().view(np.uint32), host.view(np.uint32))


def test_repeated_device_calls_replay_graphs_bitwise():
    """From the second identical call on, ism_simulate_batch (and ism_simulate)
    replays a CUDA graph of the launches; the position buffers keep their
    addresses and get new values between calls.  Every result must equal, bit
    for bit, an eager call (the stage profiler on: no graphs) on the same
    positions; and the call captured in the caller's own CUDA graph after the
    library has cached it must replay the same RIRs."""
    rng = np.random.default_rng(33)
    room = workloads.batched_fp32()
    beta = ism.ism_beta_sabine(room.L, room.rt60)
    N = ism.ism_nb_img_from_t(0.3, room.L, room.c, room.window())
    n_S = ism.ism_rir_length(0.3, room.fs)
    ps = torch.empty((2, 3), device="cuda")
    pr = torch.empty((5, 3), device="cuda")
    out = torch.empty((2, 5, n_S), device="cuda")
    ws = ism.Workspace()
    pos = [(workloads._uniform_inside(rng, room.L, 2), workloads._uniform_inside(rng, room.L, 5)) for _ in range(5)]
    got = []
    for a, b in pos:
        ps.copy_(torch.as_tensor(a))
        pr.copy_(torch.as_tensor(b))
        ism.ism_simulate(room.L, beta, ps, pr, N, 0.3, room.fs, Tw=room.window(), out=out, workspace=ws)
        got.append(out.cpu().numpy().copy())
    ref_out = torch.empty_like(out)
    ws_ref = ism.Workspace()
    ism.ism_profile_enable(True)
    try:
        for (a, b), g in zip(pos, got):
            ism.ism_simulate(room.L, beta, torch.as_tensor(a).cuda(), torch.as_tensor(b).cuda(), N, 0.3, room.fs,
                             Tw=room.window(), out=ref_out, workspace=ws_ref)
            assert np.array_equal(ref_out.cpu().numpy().view(np.uint32), g.view(np.uint32))
    finally:
        ism.ism_profile_enable(False)
    # the caller's own capture of the (cached) call
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            ism.ism_simulate(room.L, beta, ps, pr, N, 0.3, room.fs, Tw=room.window(), out=out, workspace=ws)
    for (a, b), g in zip(pos[:2], got[:2]):
        ps.copy_(torch.as_tensor(a))
        pr.copy_(torch.as_tensor(b))
        out.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), g.view(np.uint32))


def test_thin_shells_of_a_small_call_equal_the_batched_result():
    """A launch set with few fused CTAs (the single-RIR workload: 19 shells of
    8 bins) takes thinner Chebyshev shells, down to one bin per CTA, so that it
    fills the GPU; the moment sums are exact integers with per-bin scales, so
    the RIR must equal, bit for bit, the same job run beside a large one (8-bin
    shells), and stay within the FP32 tolerance of the oracle."""
    room = workloads.single_rir()
    big = workloads.batched_fp32()
    beta_b = ism.ism_beta_sabine(big.L, big.rt60)
    N_b = ism.ism_nb_img_from_t(big.Tmax, big.L, big.c, big.window())
    ps = torch.as_tensor(room.pos_src).cuda()
    pr = torch.as_tensor(room.pos_rcv).cuda()
    alone = torch.empty((1, 1, 4800), device="cuda")
    ism.ism_simulate(room.L, room.beta, ps, pr, room.nb_img, room.Tmax, room.fs, Tw=room.window(), out=alone)
    ps_b = torch.as_tensor(big.pos_src).cuda()
    pr_b = torch.as_tensor(big.pos_rcv).cuda()
    out_b = torch.empty((4, 32, ism.ism_rir_length(big.Tmax, big.fs)), device="cuda")
    mixed = torch.empty((1, 1, 4800), device="cuda")
    jobs = [ism.make_job(big.L, beta_b, ps_b, pr_b, N_b, big.Tmax, big.fs, out_b, Tw=big.window()),
            ism.make_job(room.L, room.beta, ps, pr, room.nb_img, room.Tmax, room.fs, mixed, Tw=room.window())]
    ism.ism_simulate_batch(jobs)
    torch.cuda.synchronize()
    a, m = alone.cpu().numpy(), mixed.cpu().numpy()
    assert np.array_equal(a.view(np.uint32), m.view(np.uint32))
    ref = oracle_ism(room.L, room.beta, room.pos_src, room.pos_rcv, room.nb_img, 4800, room.fs, room.window())
    assert np.max(np.abs(a.reshape(-1) - ref.reshape(-1))) <= TOL_FP32 * np.max(np.abs(ref))


def test_sabine_on_device_fp64():
    rooms = workloads.serving_requests(64, seed=9)
    L = torch.tensor(np.stack([r.room.L for r in rooms]), dtype=torch.float64, device="cuda")
    T = torch.tensor([r.room.rt60 for r in rooms], dtype=torch.float64, device="cuda")
    beta, st = ism.ism_beta_sabine_device(L, T)
    beta, st = beta.cpu().numpy(), st.cpu().numpy()
    for i, r in enumerate(rooms):
        ref = oracle.beta_sabine(r.room.L, r.room.rt60)
        if ref is None:
            assert st[i] == 2
        else:
            assert st[i] == 0
            np.testing.assert_allclose(beta[i], ref, rtol=1e-14)


def test_large_call_on_two_lanes_equals_per_source_calls_bitwise():
    """A call with enough work runs as two halves (split by source) on two
    internal streams; every RIR must equal, bit for bit, the same RIR from a
    call on one source alone (too small to be split)."""
    room = workloads.batched_fp32()
    beta = oracle.beta_sabine(room.L, room.rt60)
    N = oracle.nb_img_from_t(room.Tmax, room.L, room.c, room.window())
    full = lib_run(room.L, beta, room.pos_src, room.pos_rcv, N, room.Tmax, room.fs, Tw=room.window())
    for i in range(4):
        one = lib_run(room.L, beta, room.pos_src[i:i + 1], room.pos_rcv, N, room.Tmax, room.fs, Tw=room.window())
        assert np.array_equal(full[i].view(np.uint32), one[0].view(np.uint32)), i


def test_split_call_keeps_the_noise_index_of_every_rir():
    """A call with a diffuse tail large enough to be split: the tail of RIRs
    of the second half still uses their index in the whole call (Philox
    counter), checked against the oracle's tail for the same amplitude."""
    room = workloads.trajectory_array()
    beta = oracle.beta_sabine(room.L, room.rt60)
    Tdiff, Tmax = 0.6, 0.9
    N = oracle.nb_img_from_t(Tdiff, room.L, room.c, room.window())
    n_S = oracle.n_samples(f32(Tmax), room.fs)
    n_ism = oracle.n_samples(f32(Tdiff), room.fs)
    ps = torch.as_tensor(room.pos_src).cuda()
    pr = torch.as_tensor(room.pos_rcv).cuda()
    out = torch.empty((64, 8, n_S), device="cuda")
    amp = torch.empty(512, device="cuda")
    job = ism.make_job(room.L, beta, ps, pr, N, Tmax, room.fs, out, Tdiff=Tdiff, Tw=room.window(), seed=11,
                       env_amp=amp)
    ism.ism_simulate_batch([job])
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(512, n_S)
    A = amp.cpu().numpy()
    T60 = oracle.t60_sabine(room.L, np.asarray(beta, np.float32).astype(np.float64))
    for r in [3, 255, 256, 300, 511]:
        tail_ref = oracle.tail(11, r, float(A[r]), n_ism, n_S, float(f32(room.fs)), T60)[n_ism:]
        np.testing.assert_allclose(got[r, n_ism:].astype(np.float64), tail_ref, rtol=1e-6,
                                   atol=1e-12 * np.sqrt(A[r]))


def test_degenerate_distances_exceed_the_density_estimate():
    """A cube room with the receiver at its centre and the source next to it puts
    the images on a near-cubic lattice around the receiver: many share one
    integer delay, far more than the smooth density estimate (4 pi s^2 / (k^3
    V)) that sets the first fixed-point scales of the fused FP32 form.  The
    exact counts per integer delay are computed here: above 1016 images on one
    integer delay, no first scale (terms of at least 2^21 for a term cap of
    2^22) can pass the kernel's overflow check, so the kernel must redo that
    shell with scales from its exact counts.  The result must match the oracle
    at the FP32 tolerance."""
    L = np.array([4.0, 4.0, 4.0])
    beta = np.full(6, 0.95, np.float32)
    ps = np.array([[2.0, 2.0, 2.0009765625]], np.float32)   # 2 + 2^-10 m: exactly representable
    pr = np.array([[2.0, 2.0, 2.0]], np.float32)
    fs, Tmax, Tw = 16000.0, 0.7, 32 / 16000
    N = oracle.nb_img_from_t(Tmax, L, 343.0, Tw)
    n = oracle.n_samples(f32(Tmax), fs)
    # exact delays (FP64) of every image and the largest count per integer delay
    k = float(f32(fs)) / float(f32(343.0))
    coords = []
    for a in range(3):
        nn = np.arange(-(N[a] // 2), -(N[a] // 2) + N[a])
        even = nn % 2 == 0
        x = np.where(even, nn * L[a] + float(ps[0, a]), (nn + 1) * L[a] - float(ps[0, a]))
        coords.append(((x - float(pr[0, a])) * k) ** 2)
    s = np.sqrt(coords[0][:, None, None] + coords[1][None, :, None] + coords[2][None, None, :]).ravel()
    b = np.floor(s).astype(np.int64)
    counts = np.bincount(b[b <= n + 14])
    assert counts.max() > 1016, counts.max()
    got = lib_run(L, beta, ps, pr, N, Tmax, fs, Tw=Tw).reshape(1, -1)
    ref = oracle_ism(L, beta, ps, pr, N, n, fs, Tw)
    assert np.all(np.isfinite(got))
    err = np.max(np.abs(got.astype(np.float64) - ref)) / np.max(np.abs(ref))
    assert err <= TOL_FP32, err
