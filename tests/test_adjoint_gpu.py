"""GPU parity of the adjoint (gradients through eq. (1)-(6)) against the FP64
oracle's analytic gradient and FP64 central finite differences of the
oracle's forward sum.

The adjoint is linear in dLoss/dh, so the parity cases feed seeded random
fields as dLoss/dh; the autograd test uses a real loss and checks that the
torch.autograd.Function returns what the C entry point returns for the same
dLoss/dh.  Bound: for each gradient group (dbeta [6], dp_s, dp_r) max|err|
<= 1e-4 x max|reference| -- FP32 taps (reciprocal and sin/cos to a few ulp)
summed over 1e4-1e6 image-tap terms of both signs.
"""
import numpy as np
import pytest

import oracle
from paper_1810_11359_gb300 import ism, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def f32(x):
    return np.float32(x)


def oracle_grads(L, beta, ps, pr, N, n_ism, fs, Tw, g, c=343.0):
    """Oracle gradient of sum_k g[i, j, k] h_ij[k] over all pairs."""
    b32 = np.asarray(beta, np.float32).astype(np.float64)
    ps = np.asarray(ps, np.float32).reshape(-1, 3).astype(np.float64)
    pr = np.asarray(pr, np.float32).reshape(-1, 3).astype(np.float64)
    db = np.zeros(6)
    dps = np.zeros_like(ps)
    dpr = np.zeros_like(pr)
    for i in range(ps.shape[0]):
        for j in range(pr.shape[0]):
            a, b, cc = oracle.rir_grad(L, b32, float(f32(c)), float(f32(fs)), float(f32(Tw)), ps[i], pr[j], N, n_ism,
                                       np.asarray(g[i, j], np.float64))
            db += a
            dps[i] += b
            dpr[j] += cc
    return db, dps, dpr


def gpu_grads(L, beta, ps, pr, N, Tmax, fs, Tw, g, Tdiff=0.0, c=343.0):
    gb, gs, gr = ism.ism_simulate_backward(L, beta, ps, pr, N, Tmax, fs, torch.as_tensor(g, dtype=torch.float32),
                                           Tdiff=Tdiff, Tw=Tw, c=c)
    torch.cuda.synchronize()
    return gb.cpu().numpy(), gs.cpu().numpy(), gr.cpu().numpy()


def check(got, ref, what):
    errs = []
    for name, a, b in zip(("dbeta", "dp_s", "dp_r"), got, ref):
        scale = np.max(np.abs(b))
        assert scale > 0, (what, name)
        e = float(np.max(np.abs(np.asarray(a, np.float64) - b)) / scale)
        errs.append(e)
        assert np.all(np.isfinite(a)), (what, name)
        assert e <= TOL, f"{what} {name}: max|err|/max|ref| = {e:.3e}"
    print(f"{what}: rel err dbeta {errs[0]:.2e} dp_s {errs[1]:.2e} dp_r {errs[2]:.2e}")
    return errs


@pytest.mark.parametrize("fs,Tw", [(16000.0, 32 / 16000), (16000.0, 6 / 16000), (8000.0, 110.25 / 8000)])
def test_backward_matches_oracle_gradient(fs, Tw):
    L = np.array([3.7, 2.9, 2.3])
    beta = np.array([0.9, 0.8, 0.85, -0.7, 0.95, 0.6], np.float32)
    ps = np.array([[1.0, 1.1, 0.7], [2.9, 2.2, 1.5]], np.float32)
    pr = np.array([[2.0, 1.4, 1.2], [0.6, 0.5, 2.0], [3.1, 2.4, 0.4]], np.float32)
    Tmax = 0.0731
    N = oracle.nb_img_from_t(Tmax, L, 343.0, Tw)
    n = oracle.n_samples(f32(Tmax), fs)
    g = np.random.default_rng(11).standard_normal((2, 3, n)).astype(np.float32)
    got = gpu_grads(L, beta, ps, pr, N, Tmax, fs, Tw, g)
    ref = oracle_grads(L, beta, ps, pr, N, n, fs, Tw, g)
    check(got, ref, f"fs={fs} Nw={Tw * fs}")


def test_backward_against_finite_differences_of_oracle_forward():
    """Central differences (h = 1e-6, FP64) of sum_k g[k] h[k] computed by the
    oracle's forward sum, at a point exactly representable in FP32."""
    L = np.array([3.0, 4.0, 2.5])
    beta = np.array([0.75, 0.875, 0.8125, 0.6875, 0.9375, 0.5], np.float64)
    ps = np.array([1.25, 1.5, 0.875])
    pr = np.array([2.125, 2.625, 1.375])
    fs, Tw, c = 16000.0, 32 / 16000, 343.0
    N = [7, 7, 5]
    n = 800
    g = np.random.default_rng(12).standard_normal(n)

    def loss(b, s, r):
        return float(np.dot(g, oracle.rir(L, b, float(f32(c)), fs, float(f32(Tw)), s, r, N, n)))

    h = 1e-6
    fd = []
    for which in range(3):
        base = [beta.copy(), ps.copy(), pr.copy()][which]
        out = np.zeros(base.shape[0])
        for k in range(base.shape[0]):
            args_p = [beta.copy(), ps.copy(), pr.copy()]
            args_m = [beta.copy(), ps.copy(), pr.copy()]
            args_p[which][k] += h
            args_m[which][k] -= h
            out[k] = (loss(*args_p) - loss(*args_m)) / (2 * h)
        fd.append(out)
    got = gpu_grads(L, beta.astype(np.float32), ps[None], pr[None], N, n / fs, fs, Tw,
                    g.astype(np.float32)[None, None])
    check((got[0], got[1][0], got[2][0]), fd, "finite differences")


def test_differentiation_workload_full_launch_sampled_rooms():
    """All 256 rooms (sides 4-8 m, T60 0.3-0.8 s, 16 kHz, 0.4 s) in one
    backward batch, the launch the bench times; six rooms against the oracle."""
    rooms = workloads.differentiation_rooms()
    n_S = oracle.n_samples(f32(0.4), 16000.0)
    g_all = np.random.default_rng(13).standard_normal((len(rooms), n_S)).astype(np.float32)
    keep, gjobs, meta = [], [], []
    for b, r in enumerate(rooms):
        beta = ism.ism_beta_sabine(r.L, r.rt60)
        N = ism.ism_nb_img_from_t(r.Tmax, r.L, r.c, r.window())
        ps = torch.as_tensor(r.pos_src).cuda()
        pr = torch.as_tensor(r.pos_rcv).cuda()
        go = torch.as_tensor(g_all[b]).cuda()
        gb = torch.empty(6, device="cuda")
        gs = torch.empty((1, 3), device="cuda")
        gr = torch.empty((1, 3), device="cuda")
        job = ism.make_job(r.L, beta, ps, pr, N, r.Tmax, r.fs, go, Tw=r.window())
        gjobs.append(ism.make_grad_job(job, go, gb, gs, gr))
        keep.append((ps, pr, go, gb, gs, gr))
        meta.append((beta, N))
    ism.ism_simulate_backward_batch(gjobs)
    torch.cuda.synchronize()
    for b in [0, 1, 77, 128, 200, 255]:
        r = rooms[b]
        beta, N = meta[b]
        _, _, _, gb, gs, gr = keep[b]
        ref = oracle_grads(r.L, beta, r.pos_src, r.pos_rcv, N, n_S, r.fs, r.window(), g_all[b][None, None])
        check((gb.cpu().numpy(), gs.cpu().numpy(), gr.cpu().numpy()), ref, f"room {b}")


def test_autograd_function_matches_c_entry_point():
    from paper_1810_11359_gb300 import torch_ism
    rooms = workloads.differentiation_rooms(8)
    scale, dps, dpr = workloads.differentiation_perturbation(8)
    L = np.stack([r.L for r in rooms])
    beta0 = np.stack([ism.ism_beta_sabine(r.L, r.rt60) for r in rooms])
    ps0 = np.stack([r.pos_src for r in rooms])
    pr0 = np.stack([r.pos_rcv for r in rooms])
    Tw = rooms[0].window()
    nb = np.stack([ism.ism_nb_img_from_t(0.4, r.L, 343.0, Tw) for r in rooms])
    with torch.no_grad():
        target = torch_ism.rir(L, torch.as_tensor(beta0 * scale, dtype=torch.float32),
                               torch.as_tensor(ps0 + dps[:, None].astype(np.float32)).cuda(),
                               torch.as_tensor(pr0 + dpr[:, None].astype(np.float32)).cuda(), 0.4, 16000.0, Tw=Tw,
                               nb_img=nb)
    beta = torch.tensor(beta0, dtype=torch.float32, requires_grad=True)
    ps = torch.tensor(ps0, device="cuda", requires_grad=True)
    pr = torch.tensor(pr0, device="cuda", requires_grad=True)
    h = torch_ism.rir(L, beta, ps, pr, 0.4, 16000.0, Tw=Tw, nb_img=nb)
    loss = ((h - target) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    assert beta.grad.shape == (8, 6) and ps.grad.shape == (8, 1, 3) and pr.grad.shape == (8, 1, 3)
    # the same dLoss/dh through the C entry point, room by room
    g = (2.0 * (h - target)).detach()
    for b in range(8):
        gb, gs, gr = ism.ism_simulate_backward(L[b], beta0[b], ps0[b], pr0[b], nb[b], 0.4, 16000.0,
                                               g[b].contiguous(), Tw=Tw)
        torch.cuda.synchronize()
        assert np.array_equal(gb.cpu().numpy(), beta.grad[b].numpy())
        assert np.array_equal(gs.cpu().numpy(), ps.grad[b].cpu().numpy())
        assert np.array_equal(gr.cpu().numpy(), pr.grad[b].cpu().numpy())


def test_backward_bit_identical_run_to_run():
    r = workloads.single_rir()
    n = oracle.n_samples(r.Tmax, r.fs)
    g = np.random.default_rng(14).standard_normal((1, 1, n)).astype(np.float32)
    a = gpu_grads(r.L, r.beta, r.pos_src, r.pos_rcv, r.nb_img, r.Tmax, r.fs, r.window(), g)
    b = gpu_grads(r.L, r.beta, r.pos_src, r.pos_rcv, r.nb_img, r.Tmax, r.fs, r.window(), g)
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


def test_tail_samples_carry_no_gradient():
    L = np.array([5.0, 4.0, 3.0])
    beta = ism.ism_beta_sabine(L, 0.5)
    ps = np.array([[1.2, 1.3, 1.1]], np.float32)
    pr = np.array([[3.1, 2.2, 1.9]], np.float32)
    fs, Tw, Tmax, Tdiff = 16000.0, 32 / 16000, 0.2, 0.05
    N = ism.ism_nb_img_from_t(Tdiff, L, 343.0, Tw)
    n_S, n_ism = oracle.n_samples(f32(Tmax), fs), oracle.n_samples(f32(Tdiff), fs)
    g = np.random.default_rng(15).standard_normal((1, 1, n_S)).astype(np.float32)
    g0 = g.copy()
    g0[..., n_ism:] = 0.0
    a = gpu_grads(L, beta, ps, pr, N, Tmax, fs, Tw, g, Tdiff=Tdiff)
    b = gpu_grads(L, beta, ps, pr, N, Tmax, fs, Tw, g0, Tdiff=Tdiff)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    ref = oracle_grads(L, beta, ps, pr, N, n_ism, fs, Tw, g0)
    check(a, ref, "with tail")


def _grad_job(L, beta, ps, pr, N, Tmax, fs, Tw, g, keep):
    ps_t = torch.as_tensor(np.asarray(ps, np.float32)).cuda()
    pr_t = torch.as_tensor(np.asarray(pr, np.float32)).cuda()
    go = torch.as_tensor(np.asarray(g, np.float32)).cuda()
    gb = torch.empty(6, device="cuda")
    gs = torch.empty((ps_t.shape[0], 3), device="cuda")
    gr = torch.empty((pr_t.shape[0], 3), device="cuda")
    keep.append((ps_t, pr_t, go))
    job = ism.make_job(L, beta, ps_t, pr_t, N, Tmax, fs, go, Tw=Tw)
    return ism.make_grad_job(job, go, gb, gs, gr), (gb, gs, gr)


def test_mixed_window_batch_matches_single_calls_and_oracle():
    """One backward call over a 32-tap job (fused Chebyshev adjoint), a 6-tap
    job and a 110.25-tap job (per-tap adjoint over binned ids): each job's
    gradients are bitwise those of its own call, and within the bound of the
    oracle."""
    L = np.array([4.1, 3.3, 2.7])
    beta = np.array([0.85, 0.9, 0.8, 0.75, 0.95, 0.7], np.float32)
    ps = np.array([[1.0, 1.1, 0.7], [2.9, 2.2, 1.5]], np.float32)
    pr = np.array([[2.0, 1.4, 1.2], [0.6, 0.5, 2.0]], np.float32)
    cases = [(16000.0, 32 / 16000), (16000.0, 6 / 16000), (8000.0, 110.25 / 8000)]
    Tmax = 0.0617
    keep, gjobs, outs, gs_in, meta = [], [], [], [], []
    for k, (fs, Tw) in enumerate(cases):
        N = oracle.nb_img_from_t(Tmax, L, 343.0, Tw)
        n = oracle.n_samples(f32(Tmax), fs)
        g = np.random.default_rng(20 + k).standard_normal((2, 2, n)).astype(np.float32)
        gj, o = _grad_job(L, beta, ps, pr, N, Tmax, fs, Tw, g, keep)
        gjobs.append(gj)
        outs.append(o)
        gs_in.append(g)
        meta.append((fs, Tw, N, n))
    ism.ism_simulate_backward_batch(gjobs)
    torch.cuda.synchronize()
    for k, (fs, Tw, N, n) in enumerate(meta):
        got = tuple(x.cpu().numpy() for x in outs[k])
        single = gpu_grads(L, beta, ps, pr, N, Tmax, fs, Tw, gs_in[k])
        for x, y in zip(got, single):
            assert np.array_equal(x.view(np.uint32), y.view(np.uint32)), (fs, Tw)
        check(got, oracle_grads(L, beta, ps, pr, N, n, fs, Tw, gs_in[k]), f"mixed batch fs={fs} Nw={Tw * fs}")


@pytest.mark.parametrize("case", ["cube_centre", "near_walls", "shared_xy"])
def test_fused_adjoint_edge_geometries(case):
    """Geometries that stress the shell enumeration of the fused adjoint: a
    cube with the receiver at its centre (images on a near-cubic lattice, many
    per integer delay), source and receiver 1 cm from walls, and a pair that
    shares x and y (the images of a column straddle the receiver)."""
    fs, Tw = 16000.0, 32 / 16000
    if case == "cube_centre":
        L = np.array([3.0, 3.0, 3.0])
        ps = np.array([[0.75, 1.1, 2.2]], np.float32)
        pr = np.array([[1.5, 1.5, 1.5]], np.float32)
    elif case == "near_walls":
        L = np.array([4.0, 3.5, 2.8])
        ps = np.array([[0.01, 3.49, 1.4]], np.float32)
        pr = np.array([[3.99, 0.01, 2.79]], np.float32)
    else:
        L = np.array([5.0, 4.0, 3.0])
        ps = np.array([[2.0, 1.5, 0.6]], np.float32)
        pr = np.array([[2.0, 1.5, 2.4]], np.float32)
    beta = np.array([0.92, 0.88, 0.9, 0.85, 0.8, 0.95], np.float32)
    Tmax = 0.09
    N = oracle.nb_img_from_t(Tmax, L, 343.0, Tw)
    n = oracle.n_samples(f32(Tmax), fs)
    g = np.random.default_rng(31).standard_normal((1, 1, n)).astype(np.float32)
    got = gpu_grads(L, beta, ps, pr, N, Tmax, fs, Tw, g)
    check(got, oracle_grads(L, beta, ps, pr, N, n, fs, Tw, g), case)


def test_backward_batch_invariance():
    """A room's gradients do not depend on the other rooms of the batch (the
    fused adjoint's sums have a fixed order per RIR)."""
    rooms = workloads.differentiation_rooms(4)
    n_S = oracle.n_samples(f32(0.4), 16000.0)
    g_all = np.random.default_rng(33).standard_normal((4, n_S)).astype(np.float32)
    keep, gjobs, outs = [], [], []
    for b, r in enumerate(rooms):
        beta = ism.ism_beta_sabine(r.L, r.rt60)
        N = ism.ism_nb_img_from_t(r.Tmax, r.L, r.c, r.window())
        gj, o = _grad_job(r.L, beta, r.pos_src, r.pos_rcv, N, r.Tmax, r.fs, r.window(), g_all[b], keep)
        gjobs.append(gj)
        outs.append(o)
    ism.ism_simulate_backward_batch(gjobs)
    torch.cuda.synchronize()
    for b in (0, 3):
        r = rooms[b]
        beta = ism.ism_beta_sabine(r.L, r.rt60)
        N = ism.ism_nb_img_from_t(r.Tmax, r.L, r.c, r.window())
        single = gpu_grads(r.L, beta, r.pos_src, r.pos_rcv, N, r.Tmax, r.fs, r.window(), g_all[b][None, None])
        for x, y in zip((o.cpu().numpy() for o in outs[b]), single):
            assert np.array_equal(x.reshape(-1).view(np.uint32), y.reshape(-1).view(np.uint32))
