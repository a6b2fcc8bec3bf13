"""Receiver polar patterns and orientation on the GPU (Section 4 names them;
the first-order family g = alpha + (1 - alpha) cos(theta) is the reading
taken, pinned in the oracle's tests).

Every patterned RIR is compared with the FP64 oracle's patterned RIR at the
FP32 tolerance (1e-5 of the peak), in both FP32 forms: the fused Chebyshev
form (dense delay bins: the 128-RIR 6 x 5 x 3 m workload) and the direct form
(sparse bins: a small room with short RIRs, the 48 kHz trajectory workload),
and in the reduced-precision forms at theirs.
"""
import numpy as np
import pytest

import oracle
from paper_1810_11359_gb300 import ism, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp32_direct": 1e-5, "fp16x2": 2e-3, "lut": 2e-3, "bf16x2": 1e-2}
PATTERNS = ["subcardioid", "cardioid", "hypercardioid", "bidirectional"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def f32(x):
    return np.float32(x)


def run(L, beta, ps, pr, N, Tmax, fs, pattern, orient, Tw, prec="fp32", Tdiff=0.0, seed=0):
    out = ism.ism_simulate(L, beta, np.asarray(ps, np.float32), np.asarray(pr, np.float32), N, Tmax, fs, Tdiff, Tw,
                           prec=prec, seed=seed, mic_pattern=pattern, orient_rcv=np.asarray(orient, np.float32))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def oracle_pattern(L, beta, ps, pr, orient, pattern, N, n_ism, fs, Tw, pairs=None):
    b32 = np.asarray(beta, np.float32).astype(np.float64)
    ps = np.asarray(ps, np.float32).reshape(-1, 3).astype(np.float64)
    pr = np.asarray(pr, np.float32).reshape(-1, 3).astype(np.float64)
    orient = np.asarray(orient, np.float32).reshape(-1, 3).astype(np.float64)
    if pairs is None:
        pairs = [(i, j) for i in range(ps.shape[0]) for j in range(pr.shape[0])]
    return oracle.rir_list_pattern(L, b32, float(f32(343.0)), float(f32(fs)), float(f32(Tw)),
                                   [ps[i] for i, _ in pairs], [pr[j] for _, j in pairs], [orient[j] for _, j in pairs],
                                   pattern, N, n_ism)


def rel_err(got, ref):
    peak = np.max(np.abs(ref))
    assert peak > 0 and np.all(np.isfinite(got))
    return float(np.max(np.abs(got.astype(np.float64) - ref)) / peak)


@pytest.mark.parametrize("pattern", PATTERNS)
def test_small_room_sparse_bins(pattern):
    """2 x 3 pairs in a 3.7 x 2.9 x 2.3 m room, 73 ms at 16 kHz (the direct
    form, sparse bins), receivers looking in three different directions."""
    L = np.array([3.7, 2.9, 2.3])
    beta = np.array([0.9, 0.8, 0.85, -0.7, 0.95, 0.6], np.float32)
    ps = np.array([[1.0, 1.1, 0.7], [2.9, 2.2, 1.5]], np.float32)
    pr = np.array([[2.0, 1.4, 1.2], [0.6, 0.5, 2.0], [3.1, 2.4, 0.4]], np.float32)
    orient = np.array([[1.0, 0.0, 0.0], [0.3, -0.8, 0.5], [0.0, 0.0, -2.0]], np.float32)
    Tw, Tmax, fs = 32 / 16000, 0.0731, 16000.0
    N = oracle.nb_img_from_t(Tmax, L, 343.0, Tw)
    n = oracle.n_samples(f32(Tmax), fs)
    got = run(L, beta, ps, pr, N, Tmax, fs, pattern, orient, Tw).reshape(6, n)
    e = rel_err(got, oracle_pattern(L, beta, ps, pr, orient, pattern, N, n, fs, Tw))
    print(f"{pattern} small room: {e:.3e}")
    assert e <= TOL["fp32"]


@pytest.mark.parametrize("pattern", ["cardioid", "bidirectional"])
def test_batched_workload_fused_form(pattern):
    """The 128-RIR workload at full size (the fused Chebyshev form), each
    receiver oriented toward the room centre; four RIRs against the oracle."""
    room = workloads.batched_fp32()
    beta = oracle.beta_sabine(room.L, room.rt60)
    N = oracle.nb_img_from_t(room.Tmax, room.L, room.c, room.window())
    orient = (np.asarray(room.L) / 2 - room.pos_rcv).astype(np.float32)
    got = run(room.L, beta, room.pos_src, room.pos_rcv, N, room.Tmax, room.fs, pattern, orient, room.window())
    pairs = [(0, 0), (1, 17), (2, 9), (3, 31)]
    ref = oracle_pattern(room.L, beta, room.pos_src, room.pos_rcv, orient, pattern, N, 9600, room.fs, room.window(),
                         pairs=pairs)
    e = rel_err(np.stack([got[i, j] for i, j in pairs]), ref)
    print(f"{pattern} batched workload: {e:.3e}")
    assert e <= TOL["fp32"]


def test_trajectory_workload_cardioid_array():
    """The 48 kHz 512-RIR trajectory workload (direct form, sparse bins) with an
    outward-looking cardioid circle array; six RIRs against the oracle."""
    room = workloads.trajectory_array()
    beta = oracle.beta_sabine(room.L, room.rt60)
    N = oracle.nb_img_from_t(room.Tdiff, room.L, room.c, room.window())
    n_ism = oracle.n_samples(f32(room.Tdiff), room.fs)
    centre = room.pos_rcv.mean(axis=0)
    orient = (room.pos_rcv - centre).astype(np.float32)
    got = run(room.L, beta, room.pos_src, room.pos_rcv, N, room.Tmax, room.fs, "cardioid", orient, room.window(),
              Tdiff=room.Tdiff, seed=room.seed)
    pairs = [(0, 0), (7, 3), (33, 5), (63, 7)]
    ref = oracle_pattern(room.L, beta, room.pos_src, room.pos_rcv, orient, "cardioid", N, n_ism, room.fs,
                         room.window(), pairs=pairs)
    e = rel_err(np.stack([got[i, j, :n_ism] for i, j in pairs]), ref)
    print(f"cardioid trajectory: {e:.3e}")
    assert e <= TOL["fp32"]


@pytest.mark.parametrize("prec", ["fp32_direct", "fp16x2", "bf16x2", "lut"])
def test_patterns_in_every_precision_form(prec):
    L = np.array([4.3, 3.7, 2.9])
    beta = ism.ism_beta_sabine(L, 0.4)
    ps = np.array([[1.1, 0.9, 1.3]], np.float32)
    pr = np.array([[2.2, 2.8, 1.9], [3.6, 0.8, 1.0]], np.float32)
    orient = np.array([[-1.0, -1.0, 0.0], [0.0, 1.0, 0.2]], np.float32)
    Tw, Tmax, fs = 32 / 16000, 0.2, 16000.0
    N = oracle.nb_img_from_t(Tmax, L, 343.0, Tw)
    n = oracle.n_samples(f32(Tmax), fs)
    got = run(L, beta, ps, pr, N, Tmax, fs, "hypercardioid", orient, Tw, prec=prec).reshape(2, n)
    e = rel_err(got, oracle_pattern(L, beta, ps, pr, orient, "hypercardioid", N, n, fs, Tw))
    print(f"hypercardioid {prec}: {e:.3e}")
    assert e <= TOL[prec]


def test_omni_through_the_job_struct_equals_the_plain_call_bitwise():
    room = workloads.single_rir()
    ps = torch.as_tensor(room.pos_src).cuda()
    pr = torch.as_tensor(room.pos_rcv).cuda()
    plain = ism.ism_simulate(room.L, room.beta, ps, pr, room.nb_img, room.Tmax, room.fs, Tw=room.window())
    out = torch.empty_like(plain)
    orient = torch.tensor([[0.0, 0.0, 1.0]], device="cuda")
    job = ism.make_job(room.L, room.beta, ps, pr, room.nb_img, room.Tmax, room.fs, out, Tw=room.window(),
                       mic_pattern="omni", orient_rcv=orient)
    ism.ism_simulate_batch([job])
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), plain.cpu().numpy().view(np.uint32))


def test_zero_orientation_flagged_on_device():
    L = np.array([3.0, 4.0, 2.5])
    ps = torch.tensor([[1.0, 1.5, 1.2]], device="cuda")
    pr = torch.tensor([[2.0, 2.5, 1.5], [1.5, 1.0, 0.8]], device="cuda")
    orient = torch.tensor([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0]], device="cuda")
    out = torch.empty((1, 2, 800), device="cuda")
    ws = ism.Workspace()
    job = ism.make_job(L, [0.7] * 6, ps, pr, [9, 9, 9], 0.05, 16000.0, out, Tw=32 / 16000, mic_pattern="cardioid",
                       orient_rcv=orient)
    ism.ism_simulate_batch([job], workspace=ws)
    assert ism.ism_workspace_status(ws.buf) & ism.DEVICE_FLAG_POSITION
    o = out.cpu().numpy()
    assert np.all(o[0, 1] == 0.0) and np.max(np.abs(o[0, 0])) > 0.0


def test_gradient_of_a_patterned_job_is_rejected():
    L = np.array([3.0, 4.0, 2.5])
    ps = torch.tensor([[1.0, 1.5, 1.2]], device="cuda")
    pr = torch.tensor([[2.0, 2.5, 1.5]], device="cuda")
    orient = torch.tensor([[1.0, 0.0, 0.0]], device="cuda")
    out = torch.empty((1, 1, 800), device="cuda")
    job = ism.make_job(L, [0.7] * 6, ps, pr, [9, 9, 9], 0.05, 16000.0, out, Tw=32 / 16000, mic_pattern="cardioid",
                       orient_rcv=orient)
    g = ism.make_grad_job(job, torch.zeros_like(out), torch.zeros(6, device="cuda"), torch.zeros(1, 3, device="cuda"),
                          torch.zeros(1, 3, device="cuda"))
    with pytest.raises(ism.IsmError) as e:
        ism.ism_backward_workspace_size([g])
    assert e.value.status == ism.STATUS_CODES["ISM_ERR_UNSUPPORTED"]


def test_server_patterned_requests_alone_and_in_the_mix():
    rng = np.random.default_rng(11)
    reqs = []
    for k in range(12):
        L = rng.uniform(3.0, 7.0, 3)
        n_rcv = int(rng.integers(1, 5))
        ps = rng.uniform(0.5, L - 0.5, (1, 3)).astype(np.float32)
        pr = rng.uniform(0.5, L - 0.5, (n_rcv, 3)).astype(np.float32)
        orient = rng.normal(size=(n_rcv, 3)).astype(np.float32)
        beta = ism.ism_beta_sabine(L, 0.4)
        N = ism.ism_nb_img_from_t(0.2, L, 343.0, 32 / 16000)
        pat = PATTERNS[k % 4] if k % 3 else "omni"
        reqs.append((L, beta, ps, pr, N, pat, orient))
    with ism.Server(hbm_budget=1 << 30, max_inflight=3, max_batch=8) as srv:
        tickets = [srv.submit(L, b, ps, pr, N, 0.2, 16000.0, Tw=32 / 16000, mic_pattern=pat, orient_rcv=o)
                   for L, b, ps, pr, N, pat, o in reqs]
        for t, _ in tickets:
            srv.wait(t)
    for (t, out), (L, b, ps, pr, N, pat, o) in zip(tickets, reqs):
        alone = ism.ism_simulate(L, b, ps, pr, N, 0.2, 16000.0, 0.0, 32 / 16000, mic_pattern=pat,
                                 orient_rcv=o).cpu().numpy()
        assert np.array_equal(out.view(np.uint32), alone.view(np.uint32))
    L, b, ps, pr, N, pat, o = reqs[1]
    ref = oracle_pattern(L, b, ps, pr, o, pat, N, 3200, 16000.0, 32 / 16000)
    assert rel_err(tickets[1][1].reshape(-1, 3200), ref) <= TOL["fp32"]
