"""Reflection coefficients read from device memory (ism_job.beta_dev).

The kernels read the coefficients in place and the diffuse tail's Sabine T60
is evaluated on the device with the host's FP64 operations, so every output
must be bitwise the one of the same coefficients passed in room.beta: the
fused FP32 form, the direct form with a diffuse tail, the gradients, and the
autograd front end with a CUDA beta.  A coefficient outside [-1, 1] in device
memory is flagged by the geometry kernel (ISM_DEVICE_FLAG_BETA) and its job
gets no image.  With the training state on the device a whole training step
can be captured in a CUDA graph; a replay is bitwise the eager step.
"""
import numpy as np
import pytest

from paper_1810_11359_gb300 import ism, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _run(room, beta, N, Tdiff, host_beta: bool, seed=7):
    ps = torch.as_tensor(np.asarray(room.pos_src, np.float32)).cuda()
    pr = torch.as_tensor(np.asarray(room.pos_rcv, np.float32)).cuda()
    n_S = ism.ism_rir_length(room.Tmax, room.fs)
    out = torch.full((ps.shape[0], pr.shape[0], n_S), float("nan"), device="cuda")
    b = beta if host_beta else torch.as_tensor(np.asarray(beta, np.float32)).cuda()
    job = ism.make_job(room.L, b, ps, pr, N, room.Tmax, room.fs, out, Tdiff=Tdiff, Tw=room.window(), seed=seed)
    ws = ism.ism_simulate_batch([job])
    flags = ism.ism_workspace_status(ws)
    return out.cpu().numpy(), flags


@pytest.mark.parametrize("case", ["fused_no_tail", "direct_with_tail"])
def test_device_beta_is_bitwise_the_host_beta(case):
    if case == "fused_no_tail":
        room = workloads.batched_fp32()
        room.pos_src, room.pos_rcv = room.pos_src[:1], room.pos_rcv[:6]
        beta = ism.ism_beta_sabine(room.L, room.rt60)
        Tdiff = 0.0
        N = ism.ism_nb_img_from_t(room.Tmax, room.L, room.c, room.window())
    else:
        room = workloads.trajectory_array()
        room.pos_src = room.pos_src[:3]
        beta = np.array([0.93, 0.91, 0.95, -0.9, 0.92, 0.94])
        Tdiff = room.Tdiff
        N = ism.ism_nb_img_from_t(Tdiff, room.L, room.c, room.window())
    a, fa = _run(room, beta, N, Tdiff, True)
    b, fb = _run(room, beta, N, Tdiff, False)
    assert fa == 0 and fb == 0
    assert np.isfinite(a).all() and np.abs(a).max() > 0
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_device_beta_gradients_are_bitwise_the_host_beta_gradients():
    rooms = workloads.differentiation_rooms(6)
    n_S = ism.ism_rir_length(0.4, 16000.0)
    g = np.random.default_rng(41).standard_normal((len(rooms), n_S)).astype(np.float32)
    res = []
    for host in (True, False):
        keep, gjobs, outs = [], [], []
        for i, r in enumerate(rooms):
            beta = ism.ism_beta_sabine(r.L, r.rt60)
            N = ism.ism_nb_img_from_t(0.4, r.L, r.c, r.window())
            ps = torch.as_tensor(r.pos_src).cuda()
            pr = torch.as_tensor(r.pos_rcv).cuda()
            go = torch.as_tensor(g[i]).cuda()
            bt = beta if host else torch.as_tensor(beta.astype(np.float32)).cuda()
            gb, gs, gr = torch.empty(6, device="cuda"), torch.empty((1, 3), device="cuda"), torch.empty((1, 3), device="cuda")
            job = ism.make_job(r.L, bt, ps, pr, N, 0.4, 16000.0, go, Tw=r.window())
            gjobs.append(ism.make_grad_job(job, go, gb, gs, gr))
            keep.append((ps, pr, go, bt))
            outs.append((gb, gs, gr))
        ism.ism_simulate_backward_batch(gjobs)
        torch.cuda.synchronize()
        res.append([[t.cpu().numpy() for t in o] for o in outs])
    for x, y in zip(res[0], res[1]):
        for a, b in zip(x, y):
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_device_beta_outside_the_unit_interval_is_flagged():
    room = workloads.single_rir()
    beta = np.array([0.7, 0.7, 1.5, 0.7, 0.7, 0.7])
    out, flags = _run(room, beta, room.nb_img, 0.0, False)
    assert flags & ism.ISM_DEVICE_FLAG_BETA
    assert not flags & ism.ISM_DEVICE_FLAG_POSITION
    assert np.all(out == 0.0)


def test_autograd_with_cuda_beta_matches_cpu_beta():
    from paper_1810_11359_gb300 import torch_ism
    rooms = workloads.differentiation_rooms(8)
    L = np.stack([r.L for r in rooms])
    beta0 = np.stack([ism.ism_beta_sabine(r.L, r.rt60) for r in rooms]).astype(np.float32)
    ps0 = np.stack([r.pos_src for r in rooms])
    pr0 = np.stack([r.pos_rcv for r in rooms])
    Tw = rooms[0].window()
    nb = np.stack([ism.ism_nb_img_from_t(0.4, r.L, 343.0, Tw) for r in rooms])
    target = torch.randn((8, 1, 1, ism.ism_rir_length(0.4, 16000.0)), device="cuda") * 1e-3
    got = []
    for dev in ("cpu", "cuda"):
        beta = torch.tensor(beta0, device=dev, requires_grad=True)
        ps = torch.tensor(ps0, device="cuda", requires_grad=True)
        pr = torch.tensor(pr0, device="cuda", requires_grad=True)
        h = torch_ism.rir(L, beta, ps, pr, 0.4, 16000.0, Tw=Tw, nb_img=nb)
        ((h - target) ** 2).sum().backward()
        torch.cuda.synchronize()
        assert beta.grad.device.type == dev
        got.append([h.detach().cpu().numpy(), beta.grad.cpu().numpy(), ps.grad.cpu().numpy(), pr.grad.cpu().numpy()])
    for a, b in zip(*got):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_training_step_captured_in_a_cuda_graph_matches_eager():
    """The library makes no synchronous call and no allocation inside its
    calls, so a whole training step (forward batch, loss, autograd backward
    through the adjoint) can be captured in a CUDA graph; a replay gives
    bitwise the eager step's loss and gradients."""
    from paper_1810_11359_gb300 import torch_ism
    rooms = workloads.differentiation_rooms(70)   # two launch sets of jobs
    L = np.stack([r.L for r in rooms])
    beta0 = np.stack([ism.ism_beta_sabine(r.L, r.rt60) for r in rooms]).astype(np.float32)
    Tw = rooms[0].window()
    nb = np.stack([ism.ism_nb_img_from_t(0.4, r.L, 343.0, Tw) for r in rooms])
    beta = torch.tensor(beta0, device="cuda", requires_grad=True)
    ps = torch.tensor(np.stack([r.pos_src for r in rooms]), device="cuda", requires_grad=True)
    pr = torch.tensor(np.stack([r.pos_rcv for r in rooms]), device="cuda", requires_grad=True)
    target = torch.randn((70, 1, 1, ism.ism_rir_length(0.4, 16000.0)), device="cuda") * 1e-3
    ws = ism.Workspace()

    def step():
        h = torch_ism.rir(L, beta, ps, pr, 0.4, 16000.0, Tw=Tw, nb_img=nb, workspace=ws)
        loss = ((h - target) ** 2).sum()
        beta.grad = ps.grad = pr.grad = None
        loss.backward()
        return loss

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            eager_loss = step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    eager = [eager_loss.detach().clone(), beta.grad.clone(), ps.grad.clone(), pr.grad.clone()]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        g_loss = step()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, [g_loss, beta.grad, ps.grad, pr.grad]):
        assert torch.equal(a, b)


def test_simulate_with_device_beta_pattern_and_envelope_is_bitwise_the_host_beta():
    """ism.ism_simulate with the coefficients as a CUDA tensor, a cardioid
    receiver pattern and the Lehmann-Johansson tail (the batch entry point of
    the binding): bitwise the same call with host coefficients, and the same
    again on a repeated call."""
    rng = np.random.default_rng(8)
    L = np.array([5.0, 4.0, 3.0])
    beta_h = np.array([0.9, 0.8, 0.85, 0.7, 0.6, 0.75], np.float32)
    ps = workloads._uniform_inside(rng, L, 2)
    pr = workloads._uniform_inside(rng, L, 3)
    orient = rng.normal(size=(3, 3)).astype(np.float32)
    N = ism.ism_nb_img_from_t(0.2, L, 343.0, 32 / 16000)
    kw = dict(Tdiff=0.1, Tw=32 / 16000, mic_pattern="cardioid", orient_rcv=orient, envelope="lj", seed=3)
    host = ism.ism_simulate(L, beta_h, ps, pr, N, 0.4, 16000.0, **kw).cpu().numpy()
    beta_d = torch.as_tensor(beta_h).cuda()
    for _ in range(2):
        dev = ism.ism_simulate(L, beta_d, ps, pr, N, 0.4, 16000.0, **kw).cpu().numpy()
        assert np.array_equal(dev.view(np.uint32), host.view(np.uint32))
