"""The allocation-free entry point (ism_simulate_noalloc).

Callers that cannot allocate device memory (a real-time audio callback, a
thread inside a framework that owns every allocation) use this variant: it
runs the ordinary simulation in a fixed scratch area that the library keeps
in device memory.  These tests call it through the C ABI twice in a row and
check each result against ism_simulate with a caller-owned workspace.  Both
run the same launches with the same arithmetic (only the scratch differs), so
the results must agree bit for bit -- tighter than the FP32 tolerance (1e-5 of
the peak) of the parity tests.  The file is collected last so that a failure
here leaves every other test already run.
"""
import ctypes

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


def _noalloc_c_abi(L, beta, ps, pr, N, Tmax, fs, Tdiff, Tw, seed, c=343.0):
    """Direct C-ABI call: device positions and output, no workspace."""
    lib = ism.load()
    ps_t = torch.as_tensor(np.asarray(ps, np.float32).reshape(-1, 3)).cuda()
    pr_t = torch.as_tensor(np.asarray(pr, np.float32).reshape(-1, 3)).cuda()
    n_S = ism.ism_rir_length(Tmax, fs)
    out = torch.full((ps_t.shape[0], pr_t.shape[0], n_S), float("nan"), device="cuda")
    room = ism._room(L, beta, c)
    stream = torch.cuda.current_stream()
    st = lib.ism_simulate_noalloc(ctypes.byref(room), ctypes.c_void_p(ps_t.data_ptr()), ps_t.shape[0],
                                  ctypes.c_void_p(pr_t.data_ptr()), pr_t.shape[0], ism._nb(N), float(Tmax), float(fs),
                                  float(Tdiff), float(Tw), 0, int(seed), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, lib.ism_last_error_message().decode()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _with_workspace(L, beta, ps, pr, N, Tmax, fs, Tdiff, Tw, seed, c=343.0):
    out = ism.ism_simulate(L, beta, torch.as_tensor(np.asarray(ps, np.float32)).cuda(),
                           torch.as_tensor(np.asarray(pr, np.float32)).cuda(), N, Tmax, fs, Tdiff, Tw, c, seed=seed)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _close(a, b):
    assert np.max(np.abs(b)) > 0
    assert np.all(np.isfinite(a))
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_noalloc_matches_workspace_entry_two_calls_in_a_row():
    # call 1: the single-RIR workload
    r1 = workloads.single_rir()
    args1 = (r1.L, r1.beta, r1.pos_src, r1.pos_rcv, r1.nb_img, r1.Tmax, r1.fs, 0.0, r1.window(), 0)
    # call 2: another room, several pairs and a diffuse tail (reuses the scratch left by call 1)
    L2 = np.array([4.3, 3.7, 2.9])
    beta2 = ism.ism_beta_sabine(L2, 0.5)
    ps2 = np.array([[1.1, 0.9, 1.3], [2.9, 3.0, 0.4]], np.float32)
    pr2 = np.array([[2.2, 2.8, 1.9], [0.7, 1.5, 2.1], [3.6, 0.8, 1.0]], np.float32)
    N2 = ism.ism_nb_img_from_t(0.05, L2, 343.0, 32 / 16000)
    args2 = (L2, beta2, ps2, pr2, N2, 0.12, 16000.0, 0.05, 32 / 16000, 77)

    got1 = _noalloc_c_abi(*args1)
    got2 = _noalloc_c_abi(*args2)
    _close(got1, _with_workspace(*args1))
    _close(got2, _with_workspace(*args2))
    # and once more in the opposite order
    _close(_noalloc_c_abi(*args1), _with_workspace(*args1))


def test_noalloc_rejects_simulations_above_its_scratch():
    # the direct evaluation of the 128-RIR workload with a 40-tap window bins
    # 0.5 GB of image ids: more than the 64 MiB scratch
    room = workloads.batched_fp32()
    beta = ism.ism_beta_sabine(room.L, room.rt60)
    N = ism.ism_nb_img_from_t(room.Tmax, room.L, room.c, 40 / 16000)
    out = torch.full((4, 32, 9600), 7.0, device="cuda")
    ps = torch.as_tensor(room.pos_src).cuda()
    pr = torch.as_tensor(room.pos_rcv).cuda()
    r = ism._room(room.L, beta, 343.0)
    lib = ism.load()
    st = lib.ism_simulate_noalloc(ctypes.byref(r), ctypes.c_void_p(ps.data_ptr()), 4, ctypes.c_void_p(pr.data_ptr()),
                                  32, ism._nb(N), 0.6, 16000.0, 0.0, 40 / 16000, ism.PRECISIONS["fp32_direct"], 0,
                                  ctypes.c_void_p(out.data_ptr()), None)
    assert st == 8
    assert "scratch" in lib.ism_last_error_message().decode()
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)


def test_noalloc_runs_the_fused_fp32_form_of_the_128_rir_workload():
    # the fused Chebyshev form keeps no image ids: the same workload fits the scratch
    room = workloads.batched_fp32()
    beta = ism.ism_beta_sabine(room.L, room.rt60)
    N = ism.ism_nb_img_from_t(room.Tmax, room.L, room.c, room.window())
    args = (room.L, beta, room.pos_src, room.pos_rcv, N, room.Tmax, room.fs, 0.0, room.window(), 0)
    _close(_noalloc_c_abi(*args), _with_workspace(*args))
