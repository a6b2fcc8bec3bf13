"""Seeded synthetic inputs for the five measured workloads.

This module only draws numbers: room sizes, target reverberation times,
source/receiver positions, sample rates and durations.  It holds none of the
image-source arithmetic (no reflection coefficients, image counts or delays):
every consumer -- the CUDA library, the CPU oracle, the tests and the bench --
derives those itself from what is drawn here.  Positions are FP32 because that
is the library's input type; room sizes are FP64 for the same reason.

The paper measures only synthetic shoebox rooms (its Fig. 4/5 workloads: a
3 x 4 x 2.5 m room, T60 0.3-1.9 s, 1-1024 RIRs); these generators follow that
style at the sizes named for each workload.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

C_SOUND = 343.0


@dataclass
class Room:
    """One simulation call: a shoebox, its walls and all source/receiver pairs."""
    L: np.ndarray                      # (3,) float64, metres
    pos_src: np.ndarray                # (n_src, 3) float32
    pos_rcv: np.ndarray                # (n_rcv, 3) float32
    fs: float
    Tmax: float
    Tdiff: Optional[float] = None      # None: image sources up to Tmax, no tail
    Tw: Optional[float] = None         # window length, seconds (32 taps if None)
    c: float = C_SOUND
    rt60: Optional[float] = None       # target T60 when beta comes from Sabine
    beta: Optional[np.ndarray] = None  # (6,) explicit reflection coefficients
    nb_img: Optional[np.ndarray] = None  # explicit images per axis (paper units)
    seed: int = 0                      # noise seed of the diffuse tail
    name: str = ""

    def window(self) -> float:
        return self.Tw if self.Tw is not None else 32.0 / self.fs

    @property
    def n_rir(self) -> int:
        return int(self.pos_src.shape[0] * self.pos_rcv.shape[0])


def _uniform_inside(rng, L, n, margin=0.5):
    lo = np.full(3, margin)
    hi = np.asarray(L, dtype=np.float64) - margin
    return (lo + (hi - lo) * rng.random((n, 3))).astype(np.float32)


def single_rir() -> Room:
    """Single RIR, plain method: 3 x 4 x 2.5 m, beta 0.7 everywhere, 4800 samples.
    The 10,648-image grid (m in -5..5 with two parities per axis) is 22 images
    per axis in the paper's own units."""
    return Room(L=np.array([3.0, 4.0, 2.5]),
                pos_src=np.array([[1.0, 1.5, 1.2]], np.float32),
                pos_rcv=np.array([[2.0, 2.5, 1.5]], np.float32),
                fs=16000.0, Tmax=0.3, beta=np.full(6, 0.7), nb_img=np.array([22, 22, 22]),
                name="single_rir_3x4x2.5_beta0.7_16k_0.3s")


def batched_fp32(seed: int = 2) -> Room:
    """128 RIRs (4 sources x 32 receivers) in a 6 x 5 x 3 m room, T60 = 0.6 s,
    16 kHz, full image-source RIR up to 0.6 s (9600 samples)."""
    rng = np.random.default_rng(seed)
    L = np.array([6.0, 5.0, 3.0])
    return Room(L=L, pos_src=_uniform_inside(rng, L, 4), pos_rcv=_uniform_inside(rng, L, 32),
                fs=16000.0, Tmax=0.6, rt60=0.6, name="batched_6x5x3_rt0.6_4x32_16k_0.6s")


def trajectory_array(seed: int = 3) -> Room:
    """512 RIRs: a 64-point straight source trajectory x an 8-mic circular
    array (r = 5 cm, xy-plane), 10 x 8 x 3.5 m, T60 = 1.2 s, 48 kHz, image
    sources to 0.3 s then the diffuse tail to 1.2 s."""
    rng = np.random.default_rng(seed)
    L = np.array([10.0, 8.0, 3.5])
    a, b = _uniform_inside(rng, L, 2).astype(np.float64)
    t = np.linspace(0.0, 1.0, 64)[:, None]
    src = (a[None, :] * (1 - t) + b[None, :] * t).astype(np.float32)
    centre = _uniform_inside(rng, L, 1, margin=0.6)[0].astype(np.float64)
    ang = 2 * np.pi * np.arange(8) / 8
    mics = np.stack([centre[0] + 0.05 * np.cos(ang), centre[1] + 0.05 * np.sin(ang),
                     np.full(8, centre[2])], axis=1).astype(np.float32)
    return Room(L=L, pos_src=src, pos_rcv=mics, fs=48000.0, Tmax=1.2, Tdiff=0.3, rt60=1.2,
                seed=seed, name="trajectory_10x8x3.5_rt1.2_64x8_48k_1.2s_tdiff0.3")


@dataclass
class Request:
    room: Room
    arrival_s: float


def serving_requests(n: int = 20000, seed: int = 4, rate_hz: Optional[float] = None,
                     feasible: Optional[Callable[[np.ndarray, float], bool]] = None) -> List[Request]:
    """Serving stream: shoebox sides U(3, 10) m, T60 U(0.2, 1.0) s, one source and
    U{1..16} receivers >= 0.5 m from the walls, 16 kHz, Tdiff = min(0.25, T60),
    Tmax = T60.  Poisson arrivals at `rate_hz` (all at t = 0 if None).
    `feasible(L, T60)` lets the caller reject rooms whose walls would need an
    absorption >= 1 (the rejected draw is redrawn with the same generator)."""
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for i in range(n):
        while True:
            L = rng.uniform(3.0, 10.0, 3)
            rt = float(rng.uniform(0.2, 1.0))
            if feasible is None or feasible(L, rt):
                break
        n_rcv = int(rng.integers(1, 17))
        src = _uniform_inside(rng, L, 1)
        rcv = _uniform_inside(rng, L, n_rcv)
        if rate_hz:
            t += float(rng.exponential(1.0 / rate_hz))
        room = Room(L=L, pos_src=src, pos_rcv=rcv, fs=16000.0, Tmax=rt, Tdiff=min(0.25, rt), rt60=rt,
                    seed=seed * 1000003 + i, name=f"req{i}")
        out.append(Request(room=room, arrival_s=t))
    return out


def differentiation_rooms(n: int = 256, seed: int = 5) -> List[Room]:
    """256 rooms, sides U(4, 8) m, T60 U(0.3, 0.8) s, one source and one
    receiver each, 16 kHz, 0.4 s, no tail."""
    rng = np.random.default_rng(seed)
    rooms = []
    for i in range(n):
        L = rng.uniform(4.0, 8.0, 3)
        rt = float(rng.uniform(0.3, 0.8))
        rooms.append(Room(L=L, pos_src=_uniform_inside(rng, L, 1), pos_rcv=_uniform_inside(rng, L, 1),
                          fs=16000.0, Tmax=0.4, rt60=rt, name=f"diff{i}"))
    return rooms


def differentiation_perturbation(n: int = 256, seed: int = 6):
    """Target perturbation per room: beta scale 0.97 and N(0, 5 cm) position
    offsets for source and receiver."""
    rng = np.random.default_rng(seed)
    return 0.97, rng.normal(0.0, 0.05, (n, 3)), rng.normal(0.0, 0.05, (n, 3))
