"""Seeded synthetic inputs for the multi-cell MU-MIMO WSR problem.

This module draws channels, user weights, noise powers, power budgets and the
random initial precoders. It holds none of the method's arithmetic: it is the
one module that both the FP64 oracle and the GPU path read their inputs from.

Notation (the paper's letters in brackets):
  C cells / base stations (K), K users per cell (I), Nt BS antennas (M),
  Nr receive antennas per user (N), d streams per user (d).
  User r = k*K + i is user i of cell k (i_k).

Array layout of one instance (the C-ABI layout, complex, row-major):
  H      (C, C*K*Nr, Nt): H[j, r*Nr:(r+1)*Nr, :] is the channel H_{r j} from
         BS j to user r (system model of Sec. II).  Block H[j] stacks the
         channels of every user in the system seen from BS j.
  G0     (C, Nt, K*d): raw CN(0,1) draws for the initial precoders;
         G0[k][:, i*d:(i+1)*d] belongs to user i of cell k.  The method
         projects them onto the power ball itself (Sec. VII-A setup).
  alpha  (C*K,) priority weights, sigma2 (C*K,) noise powers, P (C,) budgets.

Every instance b of a workload draws from numpy's PCG64 generator seeded with
``base_seed * 1_000_003 + b``, so any single instance can be regenerated on
its own.  CN(0,1) means (x + i y)/sqrt(2) with x, y standard normal.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

SEED_STRIDE = 1_000_003


@dataclasses.dataclass
class Instance:
    """One channel realization with its scalars and initial-precoder draw."""

    C: int
    K: int
    Nt: int
    Nr: int
    d: int
    H: np.ndarray       # (C, C*K*Nr, Nt) complex
    G0: np.ndarray      # (C, Nt, K*d) complex, unprojected CN(0,1)
    alpha: np.ndarray   # (C*K,) float64
    sigma2: np.ndarray  # (C*K,) float64
    P: np.ndarray       # (C,) float64

    @property
    def dims(self):
        return (self.C, self.K, self.Nt, self.Nr, self.d)

    def astype(self, complex_dtype) -> "Instance":
        return dataclasses.replace(self, H=self.H.astype(complex_dtype),
                                   G0=self.G0.astype(complex_dtype))


def cn01(rng: np.random.Generator, shape) -> np.ndarray:
    """Circularly symmetric CN(0,1) samples, complex128."""
    x = rng.standard_normal(shape)
    y = rng.standard_normal(shape)
    return (x + 1j * y) / math.sqrt(2.0)


def instance_rng(base_seed: int, b: int) -> np.random.Generator:
    return np.random.default_rng(base_seed * SEED_STRIDE + b)


def rayleigh_instance(rng: np.random.Generator, C: int, K: int, Nt: int,
                      Nr: int, d: int, P, sigma2=1.0, alpha=1.0) -> Instance:
    """i.i.d. CN(0,1) channels on every BS-user link (Sec. VII-A setup).

    ``P``, ``sigma2`` and ``alpha`` may be scalars, arrays of the right length
    or callables ``f(rng, n) -> array`` drawn after the channel.
    """
    H = cn01(rng, (C, C * K * Nr, Nt))
    G0 = cn01(rng, (C, Nt, K * d))

    def fill(v, n):
        if callable(v):
            return np.asarray(v(rng, n), dtype=np.float64)
        return np.broadcast_to(np.asarray(v, dtype=np.float64), (n,)).copy()

    alpha_a = fill(alpha, C * K)
    sigma2_a = fill(sigma2, C * K)
    P_a = fill(P, C)
    return Instance(C, K, Nt, Nr, d, H, G0, alpha_a, sigma2_a, P_a)


# --------------------------------------------------------------------------
# Seven-cell hexagonal layout with path loss and shadowing (the large-scale
# fading workload).  Builder's choices: circumradius 500 m, BSs at hexagon
# centres (inter-site distance sqrt(3)*500 m), no wrap-around, users uniform
# in their own hexagon at >= 35 m from their BS.
# --------------------------------------------------------------------------
HEX_RADIUS_M = 500.0
HEX_MIN_DIST_M = 35.0
PATHLOSS_A_DB = 128.1
PATHLOSS_B_DB = 37.6
SHADOW_STD_DB = 8.0
NOISE_DBM_PER_HZ = -174.0
BANDWIDTH_HZ = 10e6
BS_POWER_DBM = 46.0


def dbm_to_watt(dbm: float) -> float:
    return 10.0 ** ((dbm - 30.0) / 10.0)


def hex_centres(R: float = HEX_RADIUS_M) -> np.ndarray:
    """Centres of a 7-cell cluster of flat-top hexagons with circumradius R."""
    isd = math.sqrt(3.0) * R
    pts = [(0.0, 0.0)]
    for q in range(6):
        a = math.radians(30.0 + 60.0 * q)
        pts.append((isd * math.cos(a), isd * math.sin(a)))
    return np.asarray(pts)


def in_flat_hex(x, y, R: float) -> np.ndarray:
    ax, ay = np.abs(x), np.abs(y)
    return (ay <= math.sqrt(3.0) / 2.0 * R) & (math.sqrt(3.0) * ax + ay <= math.sqrt(3.0) * R)


def hex_instance(rng: np.random.Generator, K: int = 10, Nt: int = 128,
                 Nr: int = 2, d: int = 2) -> Instance:
    C = 7
    R = HEX_RADIUS_M
    centres = hex_centres(R)
    users = np.zeros((C * K, 2))
    for k in range(C):
        got = 0
        while got < K:
            x, y = rng.uniform(-R, R, size=2)
            if in_flat_hex(x, y, R) and math.hypot(x, y) >= HEX_MIN_DIST_M:
                users[k * K + got] = centres[k] + (x, y)
                got += 1
    # distance user r -> BS j, path loss and shadowing per link
    dist_km = np.linalg.norm(users[:, None, :] - centres[None, :, :], axis=2) / 1000.0
    pl_db = PATHLOSS_A_DB + PATHLOSS_B_DB * np.log10(dist_km)
    shadow_db = SHADOW_STD_DB * rng.standard_normal((C * K, C))
    gain = 10.0 ** (-(pl_db + shadow_db) / 10.0)          # (CK, C) power gain
    small = cn01(rng, (C, C * K * Nr, Nt))
    amp = np.sqrt(gain).T                                  # (C, CK)
    H = small * np.repeat(amp, Nr, axis=1)[:, :, None]
    G0 = cn01(rng, (C, Nt, K * d))
    noise = dbm_to_watt(NOISE_DBM_PER_HZ) * BANDWIDTH_HZ
    return Instance(C, K, Nt, Nr, d, H, G0,
                    np.ones(C * K), np.full(C * K, noise),
                    np.full(C, dbm_to_watt(BS_POWER_DBM)))


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
SNR_SWEEP_DB = (0, 5, 10, 15, 20, 25, 30)


def tiny_fp64(n: int = 100, base_seed: int = 1) -> List[Instance]:
    """Single cell, Nt=8, K=4, Nr=2, d=2, sigma2=1, P=10 dB, alpha=1."""
    return [rayleigh_instance(instance_rng(base_seed, b), 1, 4, 8, 2, 2, P=10.0)
            for b in range(n)]


def single_cell_64(n_per_p: int = 1024, base_seed: int = 2,
                   p_db: Sequence[float] = SNR_SWEEP_DB,
                   first: int = 0, count: Optional[int] = None) -> List[Instance]:
    """Single cell, Nt=64, K=16, Nr=4, d=4, sigma2=1, alpha~U(0.5,1.5).

    Instance b has P = 10^(p_db[b // n_per_p]/10); the batch holds
    len(p_db)*n_per_p instances.  ``first``/``count`` select a slice.
    """
    total = n_per_p * len(p_db)
    count = total - first if count is None else count
    out = []
    for b in range(first, first + count):
        P = 10.0 ** (p_db[b // n_per_p] / 10.0)
        out.append(rayleigh_instance(instance_rng(base_seed, b), 1, 16, 64, 4, 4, P=P,
                                     alpha=lambda g, n: g.uniform(0.5, 1.5, n)))
    return out


def hex7(n: int = 256, base_seed: int = 3, first: int = 0,
         count: Optional[int] = None) -> List[Instance]:
    """7-cell hexagonal layout, Nt=128, K=10, Nr=2, d=2, 46 dBm, -104 dBm noise."""
    count = n - first if count is None else count
    return [hex_instance(instance_rng(base_seed, b)) for b in range(first, first + count)]


UNEVEN_NT = (16, 32, 64, 128, 256)
UNEVEN_NR = (1, 2, 4)


def uneven(n: int = 4096, base_seed: int = 4, first: int = 0,
           count: Optional[int] = None) -> List[Instance]:
    """Uneven single-cell batch: Nt~U{16..256}, K~U[4,64], Nr~U{1,2,4},
    d=min(Nr,2), sigma2=1, P=10^U[0,3], alpha=1."""
    count = n - first if count is None else count
    out = []
    for b in range(first, first + count):
        g = instance_rng(base_seed, b)
        Nt = int(g.choice(UNEVEN_NT))
        K = int(g.integers(4, 65))
        Nr = int(g.choice(UNEVEN_NR))
        d = min(Nr, 2)
        P = 10.0 ** g.uniform(0.0, 3.0)
        out.append(rayleigh_instance(g, 1, K, Nt, Nr, d, P=P))
    return out


def unrolled_64(n: int = 1024, base_seed: int = 5, first: int = 0,
                count: Optional[int] = None) -> List[Instance]:
    """Single cell, Nt=64, K=16, Nr=2, d=2, P=20 dB, sigma2=1, alpha=1."""
    count = n - first if count is None else count
    return [rayleigh_instance(instance_rng(base_seed, b), 1, 16, 64, 2, 2, P=100.0)
            for b in range(first, first + count)]


def paper_snr_sigma2(inst_H: np.ndarray, C: int, K: int, Nr: int, snr_db: float) -> float:
    """Noise power from the paper's SNR rule (Sec. VII-A): the geometric mean over
    users of ||H_{r r}||_F^2 / Nr, scaled by 10^(-SNR/10)."""
    acc = 0.0
    for r in range(C * K):
        k = r // K
        Hrr = inst_H[k, r * Nr:(r + 1) * Nr, :]
        acc += math.log10(float(np.sum(np.abs(Hrr) ** 2)) / Nr)
    return 10.0 ** (acc / (C * K)) * 10.0 ** (-snr_db / 10.0)


def paper_shape(rng: np.random.Generator, C: int, K: int, Nt: int, Nr: int, d: int,
                snr_db: float, P: float = 10.0) -> Instance:
    """The paper's experiment shapes: P = 10 W and sigma2 from the SNR rule."""
    inst = rayleigh_instance(rng, C, K, Nt, Nr, d, P=P)
    s2 = paper_snr_sigma2(inst.H, C, K, Nr, snr_db)
    inst.sigma2[:] = s2
    return inst


def random_small(rng: np.random.Generator, C: int, K: int, Nt: int, Nr: int, d: int,
                 P=10.0, alpha_range=(0.5, 1.5), sigma2_range=(0.5, 2.0)) -> Instance:
    """Small random instance with heterogeneous alpha, sigma2 and per-cell P."""
    return rayleigh_instance(
        rng, C, K, Nt, Nr, d,
        P=(lambda g, n: P * g.uniform(0.5, 1.5, n)) if np.isscalar(P) else P,
        sigma2=lambda g, n: g.uniform(*sigma2_range, n),
        alpha=lambda g, n: g.uniform(*alpha_range, n))


# --------------------------------------------------------------------------
# Packing into the C-ABI layout (instances back to back; no arithmetic)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Packed:
    dims: List[tuple]          # (C, K, Nt, Nr, d) per instance
    H: np.ndarray              # (h_elems,) complex
    G0: np.ndarray             # (v_elems,) complex
    alpha: np.ndarray          # (n_users,) float32
    sigma2: np.ndarray         # (n_users,) float32
    P: np.ndarray              # (n_cells,) float32
    h_off: np.ndarray          # complex offsets per instance
    v_off: np.ndarray

    @property
    def uniform(self) -> bool:
        return all(d == self.dims[0] for d in self.dims)


def pack(instances: Sequence[Instance], complex_dtype=np.complex64) -> Packed:
    h_off, v_off = [], []
    h = v = 0
    for inst in instances:
        h_off.append(h)
        v_off.append(v)
        h += inst.H.size
        v += inst.G0.size
    return Packed(
        dims=[inst.dims for inst in instances],
        H=np.concatenate([inst.H.reshape(-1) for inst in instances]).astype(complex_dtype),
        G0=np.concatenate([inst.G0.reshape(-1) for inst in instances]).astype(complex_dtype),
        alpha=np.concatenate([inst.alpha for inst in instances]).astype(np.float32),
        sigma2=np.concatenate([inst.sigma2 for inst in instances]).astype(np.float32),
        P=np.concatenate([inst.P for inst in instances]).astype(np.float32),
        h_off=np.asarray(h_off, dtype=np.int64), v_off=np.asarray(v_off, dtype=np.int64))


def unpack_V(packed: Packed, V: np.ndarray) -> List[np.ndarray]:
    """Split a packed V buffer into per-instance (C, Nt, K*d) arrays."""
    out = []
    for (C, K, Nt, Nr, d), off in zip(packed.dims, packed.v_off):
        out.append(V[off:off + C * Nt * K * d].reshape(C, Nt, K * d))
    return out
