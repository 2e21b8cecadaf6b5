"""Seeded synthetic workloads for the matched filter of arXiv:0906.4175.

This module draws random numbers and lays out the configurations; it holds
none of the method's arithmetic (no PSD, no template, no FFT).  Both the CUDA
path and the FP64 oracle consume exactly these draws:

* ``normals``: 2*(N/2) standard normals per segment (g1_k = g[2k], g2_k = g[2k+1]);
  each side colours them with its own Eq. (2) PSD and inverse FFT.
* injections: (m1, m2, snr, j0, phi) records; each side builds the
  2PN template itself.

The geometry follows the paper's workloads (Sec. 1.1): f_low = 40 Hz, 256 s
segments at 4096 Hz (2^20 samples), component masses of a few solar masses.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

INJ_DTYPE = np.dtype([("m1", "f8"), ("m2", "f8"), ("snr", "f8"), ("j0", "i8"), ("phi", "f8")])

F_LOW = 40.0      # Hz, Sec. 1.1
F0_PSD = 150.0    # Hz, Eq. (2)


@dataclass
class SegmentSpec:
    N: int
    fs: float
    seed: int
    injections: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=INJ_DTYPE))

    @property
    def T(self) -> float:
        return self.N / self.fs

    def normals(self) -> np.ndarray:
        """2*(N/2) standard normals (float64), reproducible from ``seed``."""
        rng = np.random.default_rng([self.seed, 0x5E6])
        return rng.standard_normal(2 * (self.N // 2))


@dataclass
class Workload:
    name: str
    m1: np.ndarray
    m2: np.ndarray
    segments: list
    f_low: float = F_LOW
    threshold: float = 6.0
    description: str = ""

    @property
    def n_templates(self) -> int:
        return int(self.m1.size)


def _injections(rng, n, N, m_lo, m_hi, snr_lo, snr_hi, masses=None, max_total=None):
    inj = np.zeros(n, dtype=INJ_DTYPE)
    for i in range(n):
        if masses is not None and i < len(masses):
            a, b = masses[i]
        else:
            while True:
                a, b = rng.uniform(m_lo, m_hi, size=2)
                if max_total is None or a + b <= max_total:
                    break
        inj[i] = (a, b, rng.uniform(snr_lo, snr_hi), int(rng.integers(0, N)),
                  rng.uniform(0.0, 2.0 * np.pi))
    return inj


def tiny(seed: int = 0) -> Workload:
    """16 templates, m ~ U[1.2, 1.6], fs = 2048 Hz, one N = 2^16 segment (32 s),
    one 1.4+1.4 injection at SNR 10 with a uniform coalescence sample."""
    rng = np.random.default_rng([seed, 1])
    m1 = rng.uniform(1.2, 1.6, 16)
    m2 = rng.uniform(1.2, 1.6, 16)
    N, fs = 1 << 16, 2048.0
    inj = np.zeros(1, dtype=INJ_DTYPE)
    inj[0] = (1.4, 1.4, 10.0, int(rng.integers(0, N)), rng.uniform(0, 2 * np.pi))
    seg = SegmentSpec(N, fs, seed * 1000 + 11, inj)
    return Workload("tiny: 16 templates, N=2^16, fs=2048", m1, m2, [seg])


def lattice_bank(n_side: int = 32, lo: float = 1.0, hi: float = 3.0, seed: int = 0):
    """n_side x n_side lattice of cell centres over [lo, hi]^2 (mirrored pairs kept),
    in a seeded random order."""
    c = lo + (np.arange(n_side) + 0.5) * (hi - lo) / n_side
    a, b = np.meshgrid(c, c, indexing="ij")
    m1 = a.ravel().copy()
    m2 = b.ravel().copy()
    perm = np.random.default_rng([seed, 2]).permutation(m1.size)
    return m1[perm], m2[perm]


def scale(seed: int = 0, n_templates: int = 1024) -> Workload:
    """1024 templates on a 32x32 lattice over [1, 3]^2 Msun, fs = 4096 Hz, one
    N = 2^20 segment (256 s) with 8 injections at SNR U[8, 20]: 4 at lattice
    masses, 4 off the lattice; threshold rho = 6."""
    n_side = int(round(np.sqrt(n_templates)))
    m1, m2 = lattice_bank(n_side, 1.0, 3.0, seed)
    rng = np.random.default_rng([seed, 3])
    N, fs = 1 << 20, 4096.0
    on = [(m1[i], m2[i]) for i in rng.choice(m1.size, 4, replace=False)]
    inj = _injections(rng, 8, N, 1.0, 3.0, 8.0, 20.0, masses=on)
    seg = SegmentSpec(N, fs, seed * 1000 + 21, inj)
    return Workload("scale: 1024 templates, N=2^20, fs=4096", m1, m2, [seg])


def uneven(seed: int = 0, n_templates: int = 4096) -> Workload:
    """4096 templates, m ~ U[1, 34] with M <= 35 (ISCO cut-offs 126..2199 Hz),
    8 segments: two each of N = 2^18, 2^19, 2^20, 2^21 at 4096 Hz, two
    injections per segment."""
    rng = np.random.default_rng([seed, 4])
    m1 = np.empty(n_templates)
    m2 = np.empty(n_templates)
    i = 0
    while i < n_templates:
        a, b = rng.uniform(1.0, 34.0, size=2)
        if a + b <= 35.0:
            m1[i], m2[i] = a, b
            i += 1
    segs = []
    for si, lg in enumerate([18, 18, 19, 19, 20, 20, 21, 21]):
        N = 1 << lg
        inj = _injections(rng, 2, N, 1.0, 34.0, 8.0, 20.0, max_total=35.0)
        segs.append(SegmentSpec(N, 4096.0, seed * 1000 + 31 + si, inj))
    return Workload("uneven: 4096 templates, 8 segments N=2^18..2^21", m1, m2, segs)


def refine_bank(seed: int = 0, n_segments: int = 32, inj_per_segment: int = 8) -> Workload:
    """1-Msun-spaced bank m in {1..20}, m1 >= m2 (210 templates); 32 segments of
    N = 2^20 with 8 injections each (m ~ U[1, 20], SNR ~ U[8, 15])."""
    ms = np.arange(1, 21, dtype=np.float64)
    a, b = np.meshgrid(ms, ms, indexing="ij")
    keep = a >= b
    m1 = a[keep].ravel().copy()
    m2 = b[keep].ravel().copy()
    rng = np.random.default_rng([seed, 5])
    N, fs = 1 << 20, 4096.0
    segs = []
    for si in range(n_segments):
        inj = _injections(rng, inj_per_segment, N, 1.0, 20.0, 8.0, 15.0)
        # keep injections apart in time so each has its own coarse peak
        inj["j0"] = (np.arange(inj_per_segment) * (N // inj_per_segment)
                     + rng.integers(0, N // (4 * inj_per_segment), inj_per_segment))
        segs.append(SegmentSpec(N, fs, seed * 1000 + 51 + si, inj))
    return Workload("refine: 210-template 1-Msun bank, 32 x N=2^20", m1, m2, segs)


def small(seed: int = 0, N: int = 1 << 12, fs: float = 4096.0, n_templates: int = 8,
          m_lo: float = 1.2, m_hi: float = 3.0, n_inj: int = 1, snr: float = 12.0) -> Workload:
    """A small case for fast tests: n_templates in U[m_lo, m_hi], one segment."""
    rng = np.random.default_rng([seed, 6, N])
    m1 = rng.uniform(m_lo, m_hi, n_templates)
    m2 = rng.uniform(m_lo, m_hi, n_templates)
    inj = _injections(rng, n_inj, N, m_lo, m_hi, snr, snr)
    return Workload("small", m1, m2, [SegmentSpec(N, fs, seed * 1000 + 61, inj)])
