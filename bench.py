"""Throughput benchmark of the image-source-method hot path on GB300.

Workload (one "step", default --workload batched): 128 RIRs (4 sources x 32
receivers) in a 6 x 5 x 3 m room, beta from Sabine for T60 = 0.6 s, 16 kHz,
0.6 s RIRs (9600 samples), 32-tap windowed sinc, images per axis from Tmax
([73, 87, 141] = 895,491 images per RIR).  One step is one ism_simulate
call: geometry, enumeration, binning, accumulation, finalize.

--workload trajectory: 512 RIRs (64-point source trajectory x 8-microphone
circle) in a 10 x 8 x 3.5 m room, T60 = 1.2 s, 48 kHz, image sources to
0.3 s and the Philox diffuse tail to 1.2 s (57,600 samples per RIR); the
line adds the HBM roofline of the tail kernel.

--prec fp32|fp16x2|bf16x2|lut|lut_tex|fp32_direct selects the tap arithmetic of the
accumulation kernel (the image enumeration and delays are FP32 in all).

Prints one JSON line (rank 0).  `value` is RIRs/s of the whole job; the line
also carries image-contributions/s, the live roofline of the accumulation
kernel, an end-to-end number through the host-buffer C entry point, the
oracle timed on the host cores and on one core (cpu_baseline) and the SM
clocks sampled during the timed region and 1.5 s of untimed repeats after it.
On one GPU the default workload's line adds `extras`, measured in the same
run: every tap arithmetic against the FP32 path on this workload and on the
48 kHz array (with the Sabine and the Lehmann-Johansson tail), the serving
stream's p50/p99 latency at 0.5x and 0.8x load, the single-RIR latency, the
moving-source filtering (FFT and direct forms) and the training step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batched|trajectory] [--prec fp32|fp16x2|bf16x2|lut|lut_tex|fp32_direct]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1810_11359_gb300 import workloads  # noqa: E402

METRIC = "RIRs/sec"
UNIT = "RIR/s"
FMA_OPS_PER_CONTRIBUTION = 5   # FADD (j - f), 2 FFMA (window), FMUL, FFMA (accumulate)
OPS_PER_IMAGE = 42             # per image: the geometry of its delay and amplitude (~40), sin(pi f), the window phase
L2_BYTES = 129 * 1024 * 1024
DTYPES = {"fp32": "f32", "fp16x2": "f16x2 taps, f32 accumulation", "bf16x2": "bf16x2 taps, f32 accumulation",
          "lut": "f32 windowed-sinc table, f32 accumulation", "fp32_direct": "f32 (every tap evaluated)",
          "lut_tex": "f32 windowed-sinc table through the texture unit (8-bit filter weights), f32 accumulation"}
# tap arithmetic of the direct accumulation kernel instantiated for each form (its PREC template value)
PREC_ID = {"fp32": 0, "fp16x2": 1, "bf16x2": 2, "lut": 3, "fp32_direct": 0, "lut_tex": 4}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def workload(name="batched"):
    """(room, Tdiff, T_img): T_img is the length the images are enumerated for."""
    if name == "trajectory":
        room = workloads.trajectory_array()
        return room, room.Tdiff, room.Tdiff
    room = workloads.batched_fp32()
    return room, 0.0, room.Tmax


def contributions(room, beta, N, n_ism):
    """(image-tap contributions, contributing images) of the step: for every
    RIR and every image, the samples 0 <= k < n_ism with |k - s| < N_w/2, and
    the images with at least one such sample (FP64, numpy)."""
    L = np.asarray(room.L, np.float64)
    fs, c = float(np.float32(room.fs)), float(np.float32(room.c))
    Nw = round(float(np.float32(room.window())) * fs)
    half = Nw / 2.0
    axes = []
    for a in range(3):
        lo = -(int(N[a]) // 2)
        n = np.arange(lo, lo + int(N[a]))
        axes.append(n)
    total = 0
    images = 0
    for ps in room.pos_src.astype(np.float64):
        for pr in room.pos_rcv.astype(np.float64):
            sq = []
            for a in range(3):
                n = axes[a]
                m = np.where(n % 2 == 0, n, n + 1).astype(np.float64)
                off = np.where(n % 2 == 0, ps[a] - pr[a], -ps[a] - pr[a])
                sq.append(((m * L[a] + off) * fs / c) ** 2)
            s = np.sqrt(sq[0][:, None, None] + sq[1][None, :, None] + sq[2][None, None, :]).ravel()
            k_lo = np.maximum(np.floor(s - half) + 1, 0)
            k_hi = np.minimum(np.ceil(s + half) - 1, n_ism - 1)
            taps = np.maximum(k_hi - k_lo + 1, 0)
            total += int(np.sum(taps))
            images += int(np.count_nonzero(taps))
    return total, images


class ClockSampler:
    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_from_profiles():
    """DRAM bytes per accumulation launch from the committed ncu summary, or
    None when the kernel source changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "shell_batched_128rir.txt")
    try:
        from paper_1810_11359_gb300 import build as b
        import hashlib
        h = hashlib.sha256()
        for f in ("ism_accum_cheb.cu", "ism_shell.cuh", "ism_accum.cuh", "ism_device.cuh", "ism_internal.h"):
            h.update(open(os.path.join(b.CSRC, f), "rb").read())
        dig = h.hexdigest()[:16]
        vals = {}
        for line in open(path):
            if "=" in line and line.strip().startswith("bench_"):
                k, v = line.strip().split("=", 1)
                vals[k.strip()] = v.strip()
        if vals.get("bench_kernel_source_sha256_16") != dig:
            return None
        return float(vals["bench_dram_bytes_per_launch"])
    except Exception:
        return None


def _oracle_pairs(room, beta, N, Tdiff, pairs, cores):
    """The oracle's RIRs (image sources, then the tail when Tdiff < Tmax) for a
    list of (source, receiver) pairs."""
    import oracle
    b32 = np.asarray(beta, np.float32).astype(np.float64)
    return oracle.simulate(room.L, b32, float(np.float32(room.c)), float(np.float32(room.fs)), room.pos_src,
                           room.pos_rcv, N, float(np.float32(room.Tmax)),
                           Tdiff=float(np.float32(Tdiff)) if Tdiff else None, Tw=float(np.float32(room.window())),
                           seed=room.seed, pairs=pairs, n_threads=cores)


_CORES = []


def host_cores():
    """OpenMP threads of the oracle on this host, read once (an oracle call with an
    explicit thread count changes what OpenMP reports afterwards)."""
    if not _CORES:
        import oracle
        _CORES.append(int(oracle.max_threads()))
    return _CORES[0]


def cpu_baseline(room, beta, N, Tdiff, budget_s=15.0):
    """The FP64 oracle, as it stands, on the host cores over a bounded sample
    of the step's RIRs."""
    import oracle
    oracle.build()
    cores = host_cores()
    all_pairs = [(i, j) for i in range(room.pos_src.shape[0]) for j in range(room.pos_rcv.shape[0])]
    # calibrate on one RIR per core, then size the sample to the budget
    n = max(1, min(cores, len(all_pairs)))
    t0 = time.perf_counter()
    _oracle_pairs(room, beta, N, Tdiff, all_pairs[:n], cores)
    dt = time.perf_counter() - t0
    total_rirs, total_t = n, dt
    more = int(max(0, (budget_s - dt) / max(dt / n, 1e-6)))
    more = min(more, len(all_pairs) - n)
    more = (more // cores) * cores
    if more > 0:
        t0 = time.perf_counter()
        _oracle_pairs(room, beta, N, Tdiff, all_pairs[n:n + more], cores)
        total_t += time.perf_counter() - t0
        total_rirs += more
    return {"value": total_rirs / total_t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{total_rirs} of the step's {len(all_pairs)} RIRs (full length, FP64 direct sum), "
                      f"{total_t:.1f} s"}


def cpu_single_core(room, beta, N, Tdiff, budget_s=5.0):
    """The FP64 oracle on one host core over a bounded sample of the step's RIRs."""
    all_pairs = [(i, j) for i in range(room.pos_src.shape[0]) for j in range(room.pos_rcv.shape[0])]
    t0 = time.perf_counter()
    done = 0
    while done < len(all_pairs) and time.perf_counter() - t0 < budget_s:
        _oracle_pairs(room, beta, N, Tdiff, all_pairs[done:done + 1], 1)
        done += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} of the step's {len(all_pairs)} RIRs on one core, {dt:.1f} s"}


def _setup(name):
    """(room, beta, N, Tdiff, n_S, n_ism, ps, pr) of a named workload, on the device."""
    import torch
    from paper_1810_11359_gb300 import ism
    room, Tdiff, T_img = workload(name)
    beta = ism.ism_beta_sabine(room.L, room.rt60)
    N = ism.ism_nb_img_from_t(T_img, room.L, room.c, room.window())
    n_S = ism.ism_rir_length(room.Tmax, room.fs)
    n_ism = ism.ism_rir_length(Tdiff, room.fs) if Tdiff else n_S
    dev = torch.device("cuda", torch.cuda.current_device())
    ps = torch.from_numpy(room.pos_src).to(dev)
    pr = torch.from_numpy(room.pos_rcv).to(dev)
    return room, beta, N, Tdiff, n_S, n_ism, ps, pr


def measure_forms(name, forms, steps, flush, peak_tops, envelope="sabine", counts=None):
    """Each tap arithmetic on one workload, against the FP32 path on the same
    GPU: RIRs/s of the whole step (CUDA events around each step, L2 flushed
    before it, default internal lanes), the accumulation stage timed with every
    launch on one stream (useful ops / time against the FP32 FMA peak), the
    tail stage, and max|err| / peak of the image-source part against the FP32
    path's (all RIRs) and against the FP64 oracle (one RIR)."""
    import torch
    import oracle
    from paper_1810_11359_gb300 import ism
    room, beta, N, Tdiff, n_S, n_ism, ps, pr = _setup(name)
    dev = ps.device
    n_rir = ps.shape[0] * pr.shape[0]
    n_contrib, n_images = counts if counts is not None else contributions(room, beta, N, n_ism)
    alg_ops = FMA_OPS_PER_CONTRIBUTION * n_contrib + OPS_PER_IMAGE * n_images
    ws = ism.Workspace(dev)
    outs = {}
    res = {}
    r_or = min(n_rir - 1, 301)
    i_or, j_or = divmod(r_or, pr.shape[0])
    ref_or = oracle.rir(room.L, np.asarray(beta, np.float32).astype(np.float64), float(np.float32(room.c)),
                        float(np.float32(room.fs)), float(np.float32(room.window())), room.pos_src[i_or],
                        room.pos_rcv[j_or], N, n_ism, n_threads=host_cores())
    for form in ["fp32"] + [f for f in forms if f != "fp32"]:
        out = torch.empty((ps.shape[0], pr.shape[0], n_S), dtype=torch.float32, device=dev)

        def step():
            ism.ism_simulate(room.L, beta, ps, pr, N, room.Tmax, room.fs, Tdiff=Tdiff, Tw=room.window(), c=room.c,
                             prec=form, seed=room.seed, out=out, workspace=ws, envelope=envelope)

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in evs:
            flush.zero_()
            a.record()
            step()
            b.record()
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
        ism.ism_set_lanes(1)
        step()
        torch.cuda.synchronize()
        ism.ism_profile_reset()
        ism.ism_profile_enable(True)
        k = 5
        for _ in range(k):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        ism.ism_profile_enable(False)
        prof = ism.ism_profile_read()
        ism.ism_set_lanes(2)
        acc_ms = prof["accum"][0] / k
        got = out.cpu().numpy().reshape(n_rir, n_S)
        outs[form] = got
        e_or = float(np.max(np.abs(got[r_or, :n_ism].astype(np.float64) - ref_or)) / np.max(np.abs(ref_or)))
        d = {"rirs_per_s": n_rir / (ms * 1e-3), "ms_per_step": ms, "accum_ms": acc_ms,
             "accum_frac_of_fp32_peak": alg_ops / (acc_ms * 1e-3) / 1e12 / peak_tops,
             "stage_ms": {kk: v[0] / k for kk, v in prof.items() if v[0] > 0},
             "max_err_vs_oracle_rir": e_or, "oracle_rir": r_or}
        if form != "fp32":
            ref = outs["fp32"][:, :n_ism].astype(np.float64)
            d["max_err_vs_fp32_path"] = float(np.max(np.abs(got[:, :n_ism] - ref)) / np.max(np.abs(ref)))
            d["speed_vs_fp32"] = res["fp32"]["ms_per_step"] / ms
        res[form] = d
    return {"workload": room.name, "rirs_per_step": n_rir, "envelope": envelope,
            "timing": "CUDA events per step, L2 flushed before each; accumulation stage with every launch on one "
                      "stream; errors over the image-source part, relative to its peak",
            "forms": res}


def single_rir_latency(calls=50):
    """The single-RIR workload (3 x 4 x 2.5 m, 10,648 images, 4800 samples): time per
    call on the device (CUDA events, positions resident) and end to end through
    the host-buffer entry point (wall clock), the FP32 error against the oracle,
    and the oracle's own time for the RIR on one core."""
    import torch
    import oracle
    from paper_1810_11359_gb300 import ism
    room = workloads.single_rir()
    dev = torch.device("cuda", torch.cuda.current_device())
    ps = torch.from_numpy(room.pos_src).to(dev)
    pr = torch.from_numpy(room.pos_rcv).to(dev)
    ws = ism.Workspace(dev)
    out = torch.empty((1, 1, 4800), dtype=torch.float32, device=dev)

    def call():
        ism.ism_simulate(room.L, room.beta, ps, pr, room.nb_img, room.Tmax, room.fs, Tw=room.window(), c=room.c,
                         out=out, workspace=ws)

    for _ in range(5):
        call()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(calls):
        call()
    b.record()
    torch.cuda.synchronize()
    dev_ms = a.elapsed_time(b) / calls
    h_ps = torch.from_numpy(room.pos_src).pin_memory()
    h_pr = torch.from_numpy(room.pos_rcv).pin_memory()
    h_out = torch.empty((1, 1, 4800), dtype=torch.float32).pin_memory()
    ws_h = ism.Workspace(dev)
    for _ in range(5):
        ism.ism_simulate_host(room.L, room.beta, h_ps.numpy(), h_pr.numpy(), room.nb_img, room.Tmax, room.fs,
                              Tw=room.window(), c=room.c, out=h_out.numpy(), workspace=ws_h)
    walls = []
    for _ in range(calls):
        t0 = time.perf_counter()
        ism.ism_simulate_host(room.L, room.beta, h_ps.numpy(), h_pr.numpy(), room.nb_img, room.Tmax, room.fs,
                              Tw=room.window(), c=room.c, out=h_out.numpy(), workspace=ws_h)
        walls.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    ref = oracle.rir(room.L, room.beta.astype(np.float32), np.float32(room.c), np.float32(room.fs),
                     np.float32(room.window()), room.pos_src[0], room.pos_rcv[0], room.nb_img, 4800, n_threads=1)
    or_s = time.perf_counter() - t0
    got = h_out.numpy().reshape(-1).astype(np.float64)
    return {"workload": room.name, "images": int(np.prod(room.nb_img)), "samples": 4800,
            "device_ms_per_call": dev_ms, "host_entry_ms_per_call_p50": float(np.median(walls)) * 1e3,
            "host_entry_ms_per_call_p99": float(np.percentile(walls, 99)) * 1e3,
            "max_err_vs_oracle": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))),
            "oracle_ms_one_core": or_s * 1e3, "calls": calls}


def sustain_clocks(step, seconds=1.5):
    """Untimed repeats of the step for `seconds` after the timed region, so that
    the clock sampler sees the GPU under load for several samples."""
    import torch
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds:
        for _ in range(20):
            step()
        torch.cuda.synchronize()
        n += 20
    return n


def run_reference(args, rank):
    if rank != 0:
        return
    room, Tdiff, T_img = workload(args.workload)
    import oracle
    beta = oracle.beta_sabine(room.L, room.rt60)
    N = oracle.nb_img_from_t(T_img, room.L, room.c, room.window())
    oracle.build()
    cores = host_cores()
    all_pairs = [(i, j) for i in range(room.pos_src.shape[0]) for j in range(room.pos_rcv.shape[0])]
    sample = max(1, min(len(all_pairs), cores))
    pairs = all_pairs[:sample]

    def step():
        _oracle_pairs(room, beta, N, Tdiff, pairs, cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    value = sample / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": room.name, "rirs_per_step": sample, "of_rirs": len(all_pairs)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample} of the {len(all_pairs)} RIRs per step, full length"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _pct(v, q):
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


def serving_measure(args):
    """The serving stream: rooms with sides U(3, 10) m, T60 U(0.2, 1.0) s, one
    source and 1-16 receivers, 16 kHz, Tdiff = min(0.25 s, T60), Tmax = T60,
    through the continuous-batching server.  Three arrival patterns of
    `--requests` requests each: all at once (saturated), then Poisson at 0.5x
    and 0.8x the saturated request rate.  The client hands the server, in one
    ism_server_submit_batch call, every request that has arrived (all of them
    at once when saturated), into output buffers it allocated beforehand.
    Latency = arrival to RIRs in the caller's host buffer: the client's delay
    in submitting (its clock) plus the server's submission-to-ready time.  The
    client's buffers are page-locked, so the server copies results straight
    into them."""
    import threading
    from paper_1810_11359_gb300 import ism

    def feasible(L, rt):
        try:
            ism.ism_beta_sabine(L, rt)
            return True
        except ism.IsmError:
            return False

    def prepared(rate):
        out = []
        for r in workloads.serving_requests(args.requests, seed=4, rate_hz=rate, feasible=feasible):
            room = r.room
            Tdiff = min(0.25, room.rt60)
            out.append((r.arrival_s, dict(L=room.L, beta=ism.ism_beta_sabine(room.L, room.rt60), pos_src=room.pos_src,
                                          pos_rcv=room.pos_rcv,
                                          nb_img=ism.ism_nb_img_from_t(Tdiff, room.L, room.c, room.window()),
                                          Tmax=room.Tmax, fs=room.fs, Tdiff=Tdiff, Tw=room.window(), seed=i_seed(r))))
        return out

    def i_seed(r):
        return int(r.arrival_s * 1e6) & 0xFFFFFFFF

    import torch
    pool = {"block": None}

    def outputs(reqs):
        # the client's result buffers: views of one page-locked block allocated before the
        # run (the server copies results straight into page-locked buffers)
        shapes = [(a["pos_src"].shape[0], a["pos_rcv"].shape[0], ism.ism_rir_length(a["Tmax"], a["fs"]))
                  for _, a in reqs]
        sizes = [s0 * s1 * s2 for s0, s1, s2 in shapes]
        total = int(sum(sizes))
        if pool["block"] is None or pool["block"].numel() < total:
            pool["block"] = None
            pool["block"] = torch.zeros(int(total * 1.25), dtype=torch.float32).pin_memory()
        flat = pool["block"].numpy()
        outs, o = [], 0
        for shp, n in zip(shapes, sizes):
            outs.append(flat[o:o + n].reshape(shp))
            o += n
        return outs

    def run(srv, reqs):
        n = len(reqs)
        outs = outputs(reqs)
        tickets = [None] * n
        lag = [0.0] * n
        lat = [0.0] * n
        submitted = threading.Semaphore(0)

        def waiter():
            for i in range(n):
                submitted.acquire()
                lat[i] = lag[i] + srv.wait(tickets[i])

        th = threading.Thread(target=waiter)
        th.start()
        t0 = time.perf_counter()
        i = 0
        while i < n:
            now = time.perf_counter() - t0
            if reqs[i][0] > now:   # nothing has arrived: wait for the next arrival
                dt = reqs[i][0] - now
                if dt > 2e-3:
                    time.sleep(dt - 1e-3)
                continue
            j = i
            while j < n and j - i < 1024 and reqs[j][0] <= now:
                j += 1
            got = srv.submit_many([a for _, a in reqs[i:j]], outs=outs[i:j])
            ts = time.perf_counter() - t0
            for k in range(i, j):
                tickets[k] = got[k - i][0]
                lag[k] = ts - reqs[k][0]
                submitted.release()
            i = j
        th.join()
        dur = time.perf_counter() - t0
        rirs = sum(a["pos_src"].shape[0] * a["pos_rcv"].shape[0] for _, a in reqs)
        return {"requests": n, "rirs": rirs, "seconds": dur, "rirs_per_s": rirs / dur, "requests_per_s": n / dur,
                "p50_ms": _pct(lat, 50) * 1e3, "p99_ms": _pct(lat, 99) * 1e3, "max_ms": max(lat) * 1e3}

    srv = ism.Server(hbm_budget=8 << 30, max_inflight=6, max_batch=32, prec=args.prec)
    warm = prepared(None)[:300]
    run(srv, warm)
    sat_reqs = prepared(None)
    ism.ism_profile_reset()
    sat = run(srv, sat_reqs)
    st_sat = srv.stats()
    res = {"saturated": sat}
    for f in (0.5, 0.8):
        res[f"poisson_{f}x"] = run(srv, prepared(f * sat["requests_per_s"]))
    st = srv.stats()
    srv.close()
    return res, st, st_sat


def run_serving(args):
    """Prints the serving line (see serving_measure)."""
    res, st, st_sat = serving_measure(args)
    sat = res["saturated"]
    line = {
        "metric": METRIC, "value": sat["rirs_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": sat["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.prec], "data": "synthetic (seeded serving stream)",
        "config": {"workload": "serving_3-10m_rt0.2-1.0_1-16rcv_16k", "requests_per_pattern": args.requests,
                   "hbm_budget_bytes": 8 << 30, "max_inflight": 6, "max_batch": 32,
                   "latency": "arrival to RIRs in the caller's host buffer (client submit delay + server time)",
                   "client": "arrived requests handed over in one ism_server_submit_batch call, "
                             "page-locked result buffers"},
        "serving": res,
        "p50_ms": res["poisson_0.8x"]["p50_ms"], "p99_ms": res["poisson_0.8x"]["p99_ms"],
        "server_stats": {"batches": st["batches"], "inflight_peak": st["inflight_peak"],
                         "dev_peak_bytes": st["dev_peak"], "batches_saturated": st_sat["batches"]},
        "e2e": {"value": sat["rirs_per_s"], "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "entry": "ism_server_submit_batch / ism_server_wait (host positions in, host RIRs out)"},
    }
    print(json.dumps(line), flush=True)


def run_differentiation(args, world, rank, dist, quiet=False):
    """One training step per timed step: 256 rooms (sides U(4, 8) m, T60
    U(0.3, 0.8) s, 1 source + 1 receiver, 16 kHz, 0.4 s) forward through the
    autograd front end, L2 loss against fixed targets (the RIRs of the rooms
    with beta x 0.97 and positions moved by N(0, 5 cm)), backward through the
    adjoint kernel.  beta and the positions live on the device (the kernels
    read beta in place), so nothing waits for the GPU and the whole step --
    the library's launches, the loss and the autograd backward -- is captured
    once in a CUDA graph and replayed; the end-to-end line reads the loss to
    the host after each replay."""
    import torch
    from paper_1810_11359_gb300 import ism, torch_ism

    rooms = workloads.differentiation_rooms()
    scale, dps, dpr = workloads.differentiation_perturbation()
    B = len(rooms)
    L = np.stack([r.L for r in rooms])
    beta0 = np.stack([ism.ism_beta_sabine(r.L, r.rt60) for r in rooms])
    ps0 = np.stack([r.pos_src for r in rooms]).astype(np.float32)
    pr0 = np.stack([r.pos_rcv for r in rooms]).astype(np.float32)
    Tw = rooms[0].window()
    nb = np.stack([ism.ism_nb_img_from_t(0.4, r.L, 343.0, Tw) for r in rooms])
    dev = torch.device("cuda", torch.cuda.current_device())
    ws_f, ws_b = ism.Workspace(dev), ism.Workspace(dev)
    with torch.no_grad():
        target = torch_ism.rir(L, torch.as_tensor(beta0 * scale, dtype=torch.float32),
                               torch.as_tensor(ps0 + dps[:, None].astype(np.float32)).to(dev),
                               torch.as_tensor(pr0 + dpr[:, None].astype(np.float32)).to(dev), 0.4, 16000.0, Tw=Tw,
                               nb_img=nb)
    # the training state lives on the device: beta is read by the kernels in place
    beta = torch.tensor(beta0, dtype=torch.float32, device=dev, requires_grad=True)
    ps = torch.tensor(ps0, device=dev, requires_grad=True)
    pr = torch.tensor(pr0, device=dev, requires_grad=True)

    def step():
        h = torch_ism.rir(L, beta, ps, pr, 0.4, 16000.0, Tw=Tw, nb_img=nb, workspace=ws_f)
        loss = ((h - target) ** 2).sum()
        beta.grad = ps.grad = pr.grad = None
        loss.backward()
        return loss

    # warm-up on a side stream, then the step captured once as a CUDA graph (every launch of
    # the library and of the loss, the autograd backward included) to be replayed below
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(max(args.warmup, 3)):
            step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        g_loss = step()
    torch.cuda.synchronize()
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ism.ism_profile_reset()
    ism.ism_profile_enable(True)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # steps back to back as a training loop runs them (nothing waits for the GPU); the L2
    # flush before each step lies outside its pair of events
    torch.cuda.synchronize()
    for a, b in evs:
        flush.zero_()
        a.record()
        loss = step()
        b.record()
    torch.cuda.synchronize()
    ism.ism_profile_enable(False)
    prof = ism.ism_profile_read()
    eager_ms = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
    dev_ms = sum(v[0] for v in prof.values()) / args.steps
    # graph replays: the launch gaps of the step's ~30 kernels go away
    graph.replay()
    torch.cuda.synchronize()
    for a, b in evs:
        flush.zero_()
        a.record()
        graph.replay()
        b.record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
    # end to end: replays reading the loss to the host after every step
    walls = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        graph.replay()
        loss_h = float(g_loss.item())
        walls.append(time.perf_counter() - w0)
    wall = sum(walls) / len(walls)
    from paper_1810_11359_gb300 import replicas
    ms = replicas.max_over_ranks(ms, device=dev)           # the slowest rank's step (replicas)
    wall = replicas.max_over_ranks(wall, device=dev)
    line = {
        "metric": METRIC, "value": replicas.whole_job_rate(B, world, ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded rooms and perturbed targets)",
        "config": {"workload": "differentiation_256rooms_4-8m_rt0.3-0.8_16k_0.4s", "rooms_per_step": B,
                   "step": "forward + L2 loss + backward (beta, source, receiver gradients)",
                   "l2": "flushed between timed steps (256 MB write)"},
        "training_steps_per_sec": 1e3 / ms,
        "eager_ms_per_step": eager_ms,
        "library_device_ms_per_step": dev_ms,
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": int(sum(v[1] for v in prof.values())),
        "e2e": {"value": replicas.whole_job_rate(B, world, wall), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 4,
                "ms_per_step": wall * 1e3,
                "entry": "torch_ism.rir + loss.backward() captured in a CUDA graph, training state on "
                         "the device, loss read to the host after every replay"},
        "timing": "the step captured once in a CUDA graph; replays back to back, CUDA events around each, "
                  "L2 flushed before each (eager_ms_per_step: the same steps launched one by one)",
        "loss": loss_h,
    }
    if quiet:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_moving_source(args, world, rank, dist, quiet=False):
    """One step renders a moving source recorded by the 8-microphone array
    (Section 4): the 512 RIRs of the 48 kHz trajectory workload (64 points x 8
    microphones, image sources to 0.3 s, Philox tail to 1.2 s), then a 1.2 s
    source signal (seeded noise) cut into 64 segments, each filtered by its
    point's RIRs and overlap-added (ism_auralize).  Inputs resident on the
    device; the roofline line is the filtering kernel's useful multiply-adds
    (8 x n_x x n_S per step) against the FP32 FMA peak."""
    import torch
    from paper_1810_11359_gb300 import ism

    room = workloads.trajectory_array()
    beta = ism.ism_beta_sabine(room.L, room.rt60)
    N = ism.ism_nb_img_from_t(room.Tdiff, room.L, room.c, room.window())
    dev = torch.device("cuda", torch.cuda.current_device())
    ps = torch.as_tensor(room.pos_src).to(dev)
    pr = torch.as_tensor(room.pos_rcv).to(dev)
    n_s = ism.ism_rir_length(room.Tmax, room.fs)
    rng = np.random.default_rng(13)
    x = torch.as_tensor(rng.normal(size=n_s).astype(np.float32)).to(dev)
    h = torch.empty((ps.shape[0], pr.shape[0], n_s), dtype=torch.float32, device=dev)
    y = torch.empty((pr.shape[0], x.numel() + n_s - 1), dtype=torch.float32, device=dev)
    ws = ism.Workspace(dev)
    ws_au = ism.Workspace(dev)

    def step():
        ism.ism_simulate(room.L, beta, ps, pr, N, room.Tmax, room.fs, room.Tdiff, room.window(), seed=room.seed,
                         out=h, workspace=ws)
        ism.ism_auralize(x, h, out=y, method="auto", workspace=ws_au)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, m, b in evs:
        flush.zero_()
        a.record()
        ism.ism_simulate(room.L, beta, ps, pr, N, room.Tmax, room.fs, room.Tdiff, room.window(), seed=room.seed,
                         out=h, workspace=ws)
        m.record()
        ism.ism_auralize(x, h, out=y, method="auto", workspace=ws_au)
        b.record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, _, b in evs) / len(evs)
    au_ms = sum(m.elapsed_time(b) for _, m, b in evs) / len(evs)
    # the direct form on the same RIRs, for comparison
    y_d = torch.empty_like(y)
    for _ in range(2):
        ism.ism_auralize(x, h, out=y_d)
    torch.cuda.synchronize()
    ed = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in ed:
        flush.zero_()
        a.record()
        ism.ism_auralize(x, h, out=y_d)
        b.record()
    torch.cuda.synchronize()
    direct_ms = sum(a.elapsed_time(b) for a, b in ed) / len(ed)
    fft_vs_direct = float((y - y_d).abs().max() / y_d.abs().max())
    peaks, peak_kind = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tops = n_sm * 128 * sm_mhz * 1e6 / 1e12
    macs = pr.shape[0] * x.numel() * n_s
    rirs = ps.shape[0] * pr.shape[0]
    # the FFT form's own work: one length-N complex DFT per segment, per point and
    # microphone pair and per pair's inverse (5 N log2 N flops each, the radix-2
    # count), and one complex multiply-add (8 flops) per point, pair and bin
    n_out = x.numel() + n_s - 1
    logN = max(4, int(math.ceil(math.log2(n_out))))
    Nf = 1 << logN
    pairs = (pr.shape[0] + 1) // 2
    n_dft = ps.shape[0] * (1 + pairs) + pairs
    fft_flops = 5.0 * Nf * logN * n_dft + 8.0 * ps.shape[0] * pairs * Nf
    peak_tflops = 2.0 * peak_tops
    from paper_1810_11359_gb300 import replicas
    ms = replicas.max_over_ranks(ms, device=dev)           # the slowest rank's step (replicas)
    line = {
        "metric": METRIC, "value": replicas.whole_job_rate(rirs, world, ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded trajectory and source signal)",
        "config": {"workload": "moving_source_10x8x3.5_rt1.2_64x8_48k_1.2s_signal1.2s", "rirs_per_step": rirs,
                   "signal_samples": int(x.numel()), "segments": int(ps.shape[0]),
                   "l2": "flushed between timed steps (256 MB write)"},
        "seconds_of_audio_per_sec": (x.numel() / room.fs) / (ms * 1e-3),
        "auralize_ms_per_step": au_ms,
        "auralize_method": "fft (automatic choice)",
        "direct_form_ms": direct_ms,
        "fft_speedup_vs_direct": direct_ms / au_ms,
        "fft_vs_direct_max_err_rel_peak": fft_vs_direct,
        "roofline": {"bound": "alu", "kernel": "af_cols_kernel + af_rows_warp_kernel + af_combine_kernel + af_icols_kernel (FFT form)",
                     "achieved": fft_flops / (au_ms * 1e-3) / 1e12, "peak": peak_tflops, "unit": "TFLOP/s (FP32)",
                     "frac": fft_flops / (au_ms * 1e-3) / 1e12 / peak_tflops, "flops_per_step": fft_flops,
                     "dft_length": Nf, "dfts_per_step": n_dft,
                     "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 flops x {sm_mhz:.0f} MHz ({peak_kind} max SM "
                                   f"clock); flops counted as 5 N log2 N per complex DFT",
                     "traffic": None},
        "direct_roofline": {"bound": "alu", "kernel": "auralize_kernel", "achieved": macs / (direct_ms * 1e-3) / 1e12,
                            "peak": peak_tops, "unit": "T multiply-adds/s (FP32 FMA pipe)",
                            "frac": macs / (direct_ms * 1e-3) / 1e12 / peak_tops, "useful_macs_per_step": macs},
    }
    if quiet:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "trajectory", "serving", "differentiation", "moving_source"])
    ap.add_argument("--requests", type=int, default=20000, help="serving: requests per arrival pattern")
    ap.add_argument("--prec", default="fp32", choices=list(PREC_ID))
    ap.add_argument("--envelope", default="sabine", choices=["sabine", "lj"],
                    help="power envelope of the diffuse tail (workloads with a tail)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the precision forms, the 48 kHz array, serving and single-RIR lines")
    ap.add_argument("--serving-requests", type=int, default=3000,
                    help="default workload: requests per arrival pattern of the serving line")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist

    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        torch.cuda.set_device(local_rank)   # before the process group, so NCCL binds this rank's GPU
        dist.init_process_group("nccl")
        dist.barrier()
        __graft_entry__.build()
    else:
        torch.cuda.set_device(0)
    from paper_1810_11359_gb300 import ism

    if args.workload == "serving":
        if rank == 0:
            run_serving(args)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.workload == "moving_source":
        run_moving_source(args, world, rank, dist)
        if world > 1:
            dist.destroy_process_group()
        return
    if args.workload == "differentiation":
        run_differentiation(args, world, rank, dist)
        if world > 1:
            dist.destroy_process_group()
        return

    room, Tdiff, T_img = workload(args.workload)
    beta = ism.ism_beta_sabine(room.L, room.rt60)
    N = ism.ism_nb_img_from_t(T_img, room.L, room.c, room.window())
    n_S = ism.ism_rir_length(room.Tmax, room.fs)
    n_ism = ism.ism_rir_length(Tdiff, room.fs) if Tdiff else n_S
    dev = torch.device("cuda", torch.cuda.current_device())
    ps = torch.from_numpy(room.pos_src).to(dev)
    pr = torch.from_numpy(room.pos_rcv).to(dev)
    out = torch.empty((ps.shape[0], pr.shape[0], n_S), dtype=torch.float32, device=dev)
    ws = ism.Workspace(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ism.ism_simulate(room.L, beta, ps, pr, N, room.Tmax, room.fs, Tdiff=Tdiff, Tw=room.window(), c=room.c,
                         prec=args.prec, seed=room.seed, out=out, workspace=ws, envelope=args.envelope)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for a, b in evs:
        flush.zero_()                     # evict L2 between timed steps (outside the events)
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # the timed region lasts ~10 ms: keep the GPU on the same step for 1.5 s more,
    # untimed, so that the clock record holds several samples under this load
    sustained = sustain_clocks(step)
    clk = clocks.stop()
    if clk is not None:
        clk["window"] = f"the timed steps and {sustained} untimed repeats of the step (1.5 s) right after them"
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    # the per-stage breakdown and the launch count from the same steps run again with the
    # library's stage timers on (their events stay out of the timed region above)
    ism.ism_profile_reset()
    ism.ism_profile_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ism.ism_profile_enable(False)
    prof = ism.ism_profile_read()

    # the kernel roofline: the same steps with every launch on one stream, so
    # that the accumulation kernel's events bracket it alone
    ism.ism_set_lanes(1)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    k_roof = max(5, min(args.steps, 20))
    ism.ism_profile_reset()
    ism.ism_profile_enable(True)
    for _ in range(k_roof):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ism.ism_profile_enable(False)
    prof_roof = ism.ism_profile_read()
    ism.ism_set_lanes(2)
    from paper_1810_11359_gb300 import replicas
    ms = replicas.max_over_ranks(ms, device=dev)           # the slowest rank's step
    rirs = ps.shape[0] * pr.shape[0] * world
    value = replicas.whole_job_rate(ps.shape[0] * pr.shape[0], world, ms * 1e-3)

    # end to end through the host-buffer entry point: pinned inputs in, RIRs out
    h_ps = torch.from_numpy(room.pos_src).pin_memory()
    h_pr = torch.from_numpy(room.pos_rcv).pin_memory()
    h_out = torch.empty((ps.shape[0], pr.shape[0], n_S), dtype=torch.float32).pin_memory()
    ws_h = ism.Workspace(dev)

    def step_host():
        ism.ism_simulate_host(room.L, beta, h_ps.numpy(), h_pr.numpy(), N, room.Tmax, room.fs, Tdiff=Tdiff,
                              Tw=room.window(), c=room.c, prec=args.prec, seed=room.seed, out=h_out.numpy(),
                              workspace=ws_h)

    for _ in range(2):
        step_host()
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step_host()
    e2e_dt = (time.perf_counter() - t0) / e2e_steps
    e2e_dt = replicas.max_over_ranks(e2e_dt, device=dev)

    if rank != 0:
        dist.destroy_process_group()
        return

    n_contrib, n_images = contributions(room, beta, N, n_ism)
    acc_ms, acc_launches, acc_calls = prof_roof["accum"]
    # the accumulation stage of one step, timed with every launch on one
    # stream (the coefficient table and the accumulation kernel)
    acc_ms_per_step = acc_ms / k_roof
    peaks, peak_kind = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peak_tops = n_sm * 128 * sm_mhz * 1e6 / 1e12          # FP32 FMA-pipe lane operations / s
    # the accumulation kernels compute each image's delay and amplitude (eq. (1)-(4))
    # and its taps (eq. (5)-(6)); the fused FP32 kernel also enumerates the images
    alg_ops = FMA_OPS_PER_CONTRIBUTION * n_contrib + OPS_PER_IMAGE * n_images
    achieved_tops = alg_ops / (acc_ms_per_step * 1e-3) / 1e12
    launches_per_step = sum(v[1] for v in prof.values()) / max(args.steps, 1)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.prec], "data": "synthetic (seeded positions, Sabine beta)",
        "config": {"workload": room.name, "rirs_per_step": int(ps.shape[0] * pr.shape[0]), "n_samples": n_S,
                   "n_ism_samples": n_ism, "images_per_rir": int(np.prod(N)), "nb_img": [int(v) for v in N],
                   "taps": 32, "precision": args.prec, "l2": "flushed between timed steps (256 MB write)"},
        "image_contributions_per_sec": n_contrib * world / (ms * 1e-3),
        "contributions_per_step": n_contrib,
        "images_in_reach_per_step": n_images,
        "stage_ms_per_step": {k: v[0] / max(args.steps, 1) for k, v in prof.items()},
        "roofline": {"bound": "alu",
                     "kernel": ("shell_kernel (fused enumeration, exact delays, Chebyshev moments)"
                                if args.prec == "fp32" and args.workload == "batched"
                                else ("shell_direct_kernel (fused enumeration, every tap evaluated)"
                                      if args.prec in ("fp32", "fp32_direct")
                                      else f"accum_kernel<1,false,{PREC_ID[args.prec]}> over binned ids")),
                     "achieved": achieved_tops,
                     "peak": peak_tops, "unit": "Tops/s (FP32 FMA-pipe lane ops)",
                     "frac": achieved_tops / peak_tops,
                     "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz ({peak_kind} max SM clock)",
                     "ops_per_contribution": FMA_OPS_PER_CONTRIBUTION, "ops_per_image": OPS_PER_IMAGE,
                     "ops_per_step": alg_ops,
                     "kernel_ms": acc_ms_per_step,
                     "kernel_launches_per_step": acc_launches / k_roof,
                     "timing": "CUDA events around the accumulation stage, launches on one stream, L2 flushed",
                     "traffic": traffic_from_profiles() if (args.prec == "fp32" and args.workload == "batched")
                     else None},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "e2e": {"value": rirs / e2e_dt, "unit": UNIT,
                "h2d_bytes_per_step": int(room.pos_src.nbytes + room.pos_rcv.nbytes),
                "d2h_bytes_per_step": int(h_out.numel() * 4), "ms_per_step": e2e_dt * 1e3,
                "entry": "ism_simulate_host (pinned host positions in, host RIRs out)"},
        "clocks": clk,
    }
    if n_ism < n_S:
        tail_ms, tail_launches, _ = prof_roof["tail"]
        tail_bytes = 4.0 * (n_S - n_ism) * ps.shape[0] * pr.shape[0]   # one FP32 store per tail sample
        tail_ms_launch = tail_ms / k_roof                              # one stream, summed over the step's launches
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        # the tail kernel is issue-bound (ncu: 81 % issue, 21 % of the copy bandwidth): count
        # the operations of its specification per sample -- Philox4x32-10 (100 integer ops per
        # 4 samples), the uniform (4), the ratio u / (1 - u) (2), the FP32 ln (22), the
        # logistic scale (1), the envelope (4) and the product (1)
        tail_ops = 59.0 * (n_S - n_ism) * ps.shape[0] * pr.shape[0]
        tail_tops = tail_ops / (tail_ms_launch * 1e-3) / 1e12
        line["tail_roofline"] = {"bound": "alu", "kernel": "tail_kernel", "achieved": tail_tops, "peak": peak_tops,
                                 "unit": "Tops/s (lane ops)", "frac": tail_tops / peak_tops, "ops_per_sample": 59,
                                 "kernel_ms_per_step": tail_ms_launch,
                                 "hbm_gbs": tail_bytes / tail_ms_launch / 1e6, "hbm_frac": tail_bytes / tail_ms_launch / 1e6 / hbm,
                                 "bytes_per_step": tail_bytes,
                                 "peak_basis": f"{n_sm} SMs x 128 lanes x {sm_mhz:.0f} MHz; HBM {peak_kind} copy bandwidth"}
    if world == 1 and not args.no_extras:
        host_cores()   # before any oracle call that sets its own thread count
        # the rest of the metric, measured in the same run: the reduced-precision forms against
        # the FP32 path on this workload and on the 48 kHz array with its diffuse tail, the
        # serving stream's latency percentiles, and the single-RIR latency
        extras = {}
        t_x = time.perf_counter()
        forms = ["fp32_direct", "fp16x2", "lut", "lut_tex", "bf16x2"]
        extras["precision_forms"] = measure_forms(args.workload, forms, 10, flush, peak_tops,
                                                  counts=(n_contrib, n_images))
        extras["trajectory_48k_array"] = measure_forms("trajectory", ["fp32"] + forms, 10, flush, peak_tops)
        lj = measure_forms("trajectory", ["fp32"], 10, flush, peak_tops, envelope="lj")
        extras["trajectory_48k_array_lj_envelope"] = lj
        extras["single_rir"] = single_rir_latency()
        sv_args = argparse.Namespace(requests=args.serving_requests, prec="fp32")
        res, st, _ = serving_measure(sv_args)
        extras["serving"] = {"workload": "serving_3-10m_rt0.2-1.0_1-16rcv_16k", "requests_per_pattern":
                             args.serving_requests, "patterns": res,
                             "server": {"hbm_budget_bytes": 8 << 30, "max_inflight": 6, "max_batch": 32,
                                        "batches": st["batches"], "inflight_peak": st["inflight_peak"]},
                             "latency": "arrival to RIRs in the caller's page-locked host buffer",
                             "entry": "ism_server_submit_batch / ism_server_wait"}
        sub = argparse.Namespace(steps=10, warmup=3)
        ms_line = run_moving_source(sub, 1, 0, None, quiet=True)
        extras["moving_source_48k_array"] = {
            k: ms_line[k] for k in ("value", "unit", "ms_per_step", "config", "seconds_of_audio_per_sec",
                                    "auralize_ms_per_step", "auralize_method", "direct_form_ms",
                                    "fft_speedup_vs_direct", "fft_vs_direct_max_err_rel_peak", "roofline",
                                    "direct_roofline")}
        df_line = run_differentiation(sub, 1, 0, None, quiet=True)
        extras["differentiation_256rooms"] = {
            k: df_line[k] for k in ("value", "unit", "ms_per_step", "config", "training_steps_per_sec",
                                    "eager_ms_per_step", "library_device_ms_per_step", "stage_ms_per_step", "e2e",
                                    "timing")}
        extras["seconds"] = time.perf_counter() - t_x
        line["extras"] = extras
        line["p50_ms"] = res["poisson_0.8x"]["p50_ms"]
        line["p99_ms"] = res["poisson_0.8x"]["p99_ms"]
    if not args.no_cpu_baseline and world >= 1:
        line["cpu_baseline"] = cpu_baseline(room, beta, N, Tdiff)
        line["cpu_baseline"]["single_core"] = cpu_single_core(room, beta, N, Tdiff)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
