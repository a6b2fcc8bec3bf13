"""The C ABI: the library loads on a machine without a GPU, exports every
symbol include/ism.h declares, and its host-only helpers (sizing, Sabine,
image counts) agree with the oracle and reject bad arguments.  No device
work is done here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1810_11359_gb300 import build as libbuild
from paper_1810_11359_gb300 import ism

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return ism.load()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ism_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 15
    for name in sorted(declared):
        assert hasattr(lib, name), name
        assert name in ism._SIGS, f"binding lacks {name}"


def test_status_strings_and_version(lib):
    assert lib.ism_version() == 101
    for code, name in ism.STATUS_NAMES.items():
        assert lib.ism_status_string(code).decode() == name


def test_rir_length_rule():
    assert ism.ism_rir_length(np.float32(0.3), 16000.0) == 4800 == oracle.n_samples(np.float32(0.3), 16000.0)
    assert ism.ism_rir_length(np.float32(1.2), 48000.0) == 57600
    assert ism.ism_rir_length(np.float32(0.6), 16000.0) == 9600
    for T, fs in [(0.123457, 16000.0), (0.77, 44100.0), (1e-3, 8000.0)]:
        assert ism.ism_rir_length(T, fs) == oracle.n_samples(np.float32(T), np.float32(fs))
    with pytest.raises(ism.IsmError):
        ism.ism_rir_length(0.0, 16000.0)


def test_sabine_helpers_match_oracle():
    for L, T in [([6, 5, 3], 0.6), ([10, 8, 3.5], 1.2), ([3, 4, 2.5], 0.7)]:
        b = ism.ism_beta_sabine(L, T)
        np.testing.assert_allclose(b, oracle.beta_sabine(L, T), rtol=1e-15)
        assert ism.ism_t60_sabine(L, b) == pytest.approx(oracle.t60_sabine(L, b), rel=1e-15)
        np.testing.assert_array_equal(ism.ism_beta_sabine(L, T, negative=True), -b)
    w = [1, 1, 0.5, 0.5, 2, 2]
    np.testing.assert_allclose(ism.ism_beta_sabine([6, 5, 3], 0.6, w), oracle.beta_sabine([6, 5, 3], 0.6, w), rtol=1e-15)
    with pytest.raises(ism.IsmError) as e:
        ism.ism_beta_sabine([3, 3, 3], 0.01)
    assert e.value.status == 2


def test_nb_img_and_att2t_match_oracle():
    for T, L, Tw in [(0.6, [6, 5, 3], 32 / 16000), (0.3, [10, 8, 3.5], 32 / 48000), (0.4, [4.5, 7.1, 5.2], 4e-3)]:
        assert list(ism.ism_nb_img_from_t(T, L, 343.0, Tw)) == list(oracle.nb_img_from_t(T, L, 343.0, Tw))
    assert ism.ism_att2t_sabine(13.0, 0.6) == pytest.approx(oracle.att2t_sabine(13.0, 0.6))


def test_workspace_size_and_validation(lib):
    L, beta = [6.0, 5.0, 3.0], [0.9] * 6
    # the direct evaluation of a window other than 32 taps bins image ids: at least
    # the worst-case id buffer, 128 RIRs x 895,491 images x 4 B
    n = ism.ism_workspace_size(L, beta, 4, 32, [73, 87, 141], 0.6, 16000.0, Tw=40 / 16000, prec="fp32_direct")
    assert n >= 128 * 73 * 87 * 141 * 4
    assert n % 256 == 0
    # with a 32-tap window the direct evaluation enumerates its images in the
    # accumulating CTA: tables and window rows only
    nd = ism.ism_workspace_size(L, beta, 4, 32, [73, 87, 141], 0.6, 16000.0, Tw=32 / 16000, prec="fp32_direct")
    assert 128 * 301 * 64 * 4 <= nd < 32 << 20
    # the fused Chebyshev form enumerates its images itself: per-bin counts,
    # tables and window rows only (128 x 301 bins x 64 FP32 rows = 9.9 MB)
    n32 = ism.ism_workspace_size(L, beta, 4, 32, [73, 87, 141], 0.6, 16000.0, Tw=32 / 16000)
    assert 128 * 301 * 64 * 4 <= n32 < 32 << 20
    assert n32 % 256 == 0
    bad = [
        dict(L=[0, 5, 3]),
        dict(beta=[1.5] + [0.9] * 5),
        dict(nb_img=[0, 3, 3]),
        dict(fs=-1.0),
        dict(Tmax=0.0),
        dict(Tw=1.0 / 16000),           # one tap
    ]
    base = dict(L=L, beta=beta, n_src=1, n_rcv=1, nb_img=[5, 5, 5], Tmax=0.1, fs=16000.0, Tw=32 / 16000)
    for b in bad:
        kw = dict(base, **b)
        with pytest.raises(ism.IsmError) as e:
            ism.ism_workspace_size(**kw)
        assert e.value.status == 1, b
    with pytest.raises(ism.IsmError) as e:
        ism.ism_workspace_size(**dict(base, nb_img=[2000, 3, 3]))
    assert e.value.status == 8
    with pytest.raises(ism.IsmError) as e:
        ism.ism_workspace_size(**dict(base, Tw=300 / 16000))
    assert e.value.status == 8
    assert lib.ism_last_error_message().decode() != ""


def test_host_entry_rejects_outside_positions_without_device_work(lib):
    r = ism._room([3, 4, 2.5], [0.7] * 6, 343.0)
    ps = np.array([[1.0, 1.5, 3.0]], np.float32)  # z above the ceiling
    pr = np.array([[2.0, 2.5, 1.5]], np.float32)
    out = np.zeros(4800, np.float32)
    st = lib.ism_simulate_host(ctypes.byref(r), ctypes.c_void_p(ps.ctypes.data), 1, ctypes.c_void_p(pr.ctypes.data), 1,
                               ism._nb([5, 5, 5]), 0.3, 16000.0, 0.0, 0.0, 0, 0, ctypes.c_void_p(out.ctypes.data),
                               None, 0, None)
    assert st == 1
    assert "outside" in lib.ism_last_error_message().decode()


def test_server_config_is_checked_before_any_device_work(lib):
    cfg = ism.ism_server_config(64 << 20, 0, 99, 32, 0, 0)        # max_inflight out of range
    h = ctypes.c_void_p()
    assert lib.ism_server_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg = ism.ism_server_config(1 << 20, 0, 2, 32, 0, 0)          # budget below 16 MiB
    assert lib.ism_server_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    assert h.value is None
    assert lib.ism_server_submit(None, None, None) == 1
    assert lib.ism_server_destroy(None) == 1


def test_backward_validates_like_the_forward(lib):
    gj = ism.ism_grad_job()
    gj.job.room = ism._room([3, 4, 2.5], [0.7] * 6, 343.0)
    gj.job.n_src = gj.job.n_rcv = 1
    for a in range(3):
        gj.job.nb_img[a] = 5
    gj.job.Tmax, gj.job.fs, gj.job.Tw = 0.1, 16000.0, 32 / 16000
    b = ctypes.c_size_t()
    assert lib.ism_backward_workspace_size(ctypes.byref(gj), 1, ctypes.byref(b)) == 0
    assert b.value > 0
    # missing grad_out / positions: rejected before any launch
    assert lib.ism_simulate_backward_batch(ctypes.byref(gj), 1, None, 0, None) == 1
    gj.job.fs = -1.0
    assert lib.ism_backward_workspace_size(ctypes.byref(gj), 1, ctypes.byref(b)) == 1


def test_strided_job_arrays_match_per_room_jobs():
    """The vectorised job arrays of the autograd front end hold, byte for
    byte, what make_job / make_grad_job build room by room (host tensors only
    give the pointers here; nothing is launched)."""
    import ctypes
    import numpy as np
    import torch
    from paper_1810_11359_gb300 import ism
    rng = np.random.default_rng(7)
    B, S, M, n_S = 5, 2, 3, 17
    L = rng.uniform(3, 9, (B, 3))
    beta = rng.uniform(0.1, 0.99, (B, 6))
    nb = rng.integers(1, 40, (B, 3)).astype(np.int32)
    ps = torch.zeros((B, S, 3))
    pr = torch.zeros((B, M, 3))
    out = torch.zeros((B, S, M, n_S))
    gb, gs, gr = torch.zeros((B, 6)), torch.zeros((B, S, 3)), torch.zeros((B, M, 3))
    arr = ism.make_jobs_strided(L, beta, ps, pr, nb, 0.25, 16000.0, out, Tdiff=0.1, Tw=0.002, c=340.0, seed=2 ** 63 + 5)
    garr = ism.make_grad_jobs_strided(arr, out, gb, gs, gr)
    for b in range(B):
        j = ism.make_job(L[b], beta[b], ps[b], pr[b], nb[b], 0.25, 16000.0, out[b], Tdiff=0.1, Tw=0.002, c=340.0,
                         seed=2 ** 63 + 5)
        assert bytes(arr[b]) == bytes(j)
        g = ism.make_grad_job(j, out[b], gb[b], gs[b], gr[b])
        assert bytes(garr[b]) == bytes(g)
    assert ctypes.sizeof(arr) == B * ctypes.sizeof(ism.ism_job)


def test_binding_struct_layouts_match_the_header(tmp_path):
    """The ctypes structs of the binding have the sizes and field offsets the
    C compiler gives the structs of include/ism.h (a C program built here
    prints them)."""
    import ctypes
    import os
    import shutil
    import subprocess
    import pytest
    from paper_1810_11359_gb300 import ism
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"ism_room": ism.ism_room, "ism_job": ism.ism_job, "ism_grad_job": ism.ism_grad_job,
               "ism_server_config": ism.ism_server_config, "ism_server_stats": ism.ism_server_stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ism.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert got[(name, f[0])] == getattr(cls, f[0]).offset, (name, f[0])


def test_plan_takes_the_fused_forms_for_32_tap_windows():
    """Host-side planning (no GPU needed): 32-tap windows take a kernel that
    enumerates its own images -- the Chebyshev one for a dense room, the fused
    per-tap one for FP32_DIRECT and for the sparse 48 kHz array (~36 images per
    delay bin) -- and need no image-id buffer; another window length bins image
    ids (the per-tap form over a 40-tap window); a backward call over a 32-tap
    window takes the fused adjoint (no ids either), over a 6-tap window the
    per-tap adjoint over binned ids."""
    from paper_1810_11359_gb300 import ism
    L = [6.0, 5.0, 3.0]
    beta = ism.ism_beta_sabine(L, 0.6)
    N = ism.ism_nb_img_from_t(0.6, L, 343.0, 32 / 16000)
    fused = ism.ism_workspace_size(L, beta, 4, 32, N, 0.6, 16000.0, Tw=32 / 16000, prec="fp32")
    direct = ism.ism_workspace_size(L, beta, 4, 32, N, 0.6, 16000.0, Tw=32 / 16000, prec="fp32_direct")
    N40 = ism.ism_nb_img_from_t(0.6, L, 343.0, 40 / 16000)
    binned = ism.ism_workspace_size(L, beta, 4, 32, N40, 0.6, 16000.0, Tw=40 / 16000, prec="fp32_direct")
    ids = 128 * int(np.prod(N)) * 4
    assert fused == direct and fused < ids / 10 and binned > ids
    L2 = [10.0, 8.0, 3.5]
    b2 = ism.ism_beta_sabine(L2, 1.2)
    N2 = ism.ism_nb_img_from_t(0.3, L2, 343.0, 32 / 48000)
    a = ism.ism_workspace_size(L2, b2, 64, 8, N2, 1.2, 48000.0, Tdiff=0.3, Tw=32 / 48000, prec="fp32")
    b = ism.ism_workspace_size(L2, b2, 64, 8, N2, 1.2, 48000.0, Tdiff=0.3, Tw=32 / 48000, prec="fp32_direct")
    assert a == b and a < 512 * int(np.prod(N2)) * 4
    # backward: host tensors only lend the pointers the host-side checks look at
    import torch
    ps, pr = torch.ones((1, 3)), torch.ones((1, 3))
    sizes = []
    for Tw in (32 / 16000, 6 / 16000):
        N3 = ism.ism_nb_img_from_t(0.4, L, 343.0, Tw)
        go = torch.zeros(ism.ism_rir_length(0.4, 16000.0))
        job = ism.make_job(L, beta, ps, pr, N3, 0.4, 16000.0, go, Tw=Tw)
        gj = ism.make_grad_job(job, go, torch.zeros(6), torch.zeros((1, 3)), torch.zeros((1, 3)))
        sizes.append((ism.ism_backward_workspace_size([gj]), int(np.prod(N3)) * 4))
    (fused_b, _), (direct_b, ids_b) = sizes
    assert fused_b < ids_b and direct_b > ids_b
