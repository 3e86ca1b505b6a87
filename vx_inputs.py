"""Seeded synthetic inputs for the periodic vertex model.

This module holds no vertex-model arithmetic.  It only draws random numbers
and arranges them into the arrays that both the CUDA path and the FP64
oracle take as inputs: Voronoi seed points, per-edge line tensions, per-cell
target shape indices and per-tissue cell counts.  Both sides import it; it
imports neither.

Random stream
-------------
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the state advances by the golden-gamma constant
0x9E3779B97F4A7C15 and each output is the state passed through the
variant-13 finaliser (xor-shift 30, multiply 0xBF58476D1CE4E5B9, xor-shift
27, multiply 0x94D049BB133111EB, xor-shift 31).  A uniform double in [0, 1)
is ``(z >> 11) * 2**-53``.  Stream ``s`` starts from state ``s``; sub-stream
``i`` of stream ``s`` (one per tissue of a batch) starts from state
``s * 2**32 + i``.

Workloads
---------
The five synthetic workloads mirror the paper's synthetic benchmark (random
periodic Voronoi tissues, Methods "Mesh initialization"; Fig. 2 uses a box of
side sqrt(N) with A0 = 1).  Moduli are given in the dimensionless units of
Eq. (Energy1) (areas in units of A0, lengths in units of sqrt(A0)) with the
energy measured in units of A0, so a tissue of target area A0 has the
dimensional moduli K_A = k_A / A0, K_P = k_P and Lambda = lambda sqrt(A0);
forces then scale with sqrt(A0).  ``dimensional`` does that conversion.

* ``tissue_c1``  100 cells, unit box, A0 = 0.01, p0 = 3.7, k_A = k_P = 1,
  lambda_e ~ U(0, 0.1) per edge (seeds: stream 0, tensions: stream 1).
* ``tissue_c2``  10,000 cells, unit box, A0 = 1e-4, p0 in {3.5, 3.7, 3.9},
  uniform lambda = 0.05 (stream 2).
* ``batch_c3``   512 tissues, n_i = round(exp(U(ln 200, ln 5000))), box
  sqrt(n_i), A0 = 1, p0_i ~ U(3.5, 4.0), Lambda_e ~ U(0, 0.1) (stream 3,
  tissue i on sub-stream i).
* ``tissue_c4``  1,000 cells, box sqrt(1000), A0 = 1, p0 = 3.7, hidden
  tensions Lambda* ~ U(0.02, 0.1) and trial tensions ~ U(0.02, 0.1)
  (stream 4).
* ``batch_c5``   64 tissues of 10,000 cells, box 100, A0 = 1 per cell,
  Lambda_e ~ U(0, 0.1) (stream 5, tissue i on sub-stream i).

Per-edge draws are taken in canonical edge order (edge id 0, 1, 2, ...), so a
tensor array of length E is the next E uniforms of the stream after the seeds
when the two share a stream, or the first E of their own stream otherwise.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64 stream producing uint64 words and doubles."""

    def __init__(self, state: int):
        self.state = np.uint64(state % (1 << 64))

    def next_u64(self, count: int) -> np.ndarray:
        k = np.arange(1, count + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = self.state + k * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
            self.state = self.state + np.uint64(count) * _GAMMA
        return z

    def uniform(self, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        z = self.next_u64(count)
        u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u


def substream(stream: int, index: int) -> SplitMix64:
    return SplitMix64(stream * (1 << 32) + index)


def uniform_seeds(n: int, Lx: float, Ly: float, rng: SplitMix64) -> np.ndarray:
    """n seed points, uniform in [0, Lx) x [0, Ly); row i = (x_i, y_i)."""
    u = rng.uniform(2 * n).reshape(n, 2)
    return np.stack([u[:, 0] * Lx, u[:, 1] * Ly], axis=1)


def lattice_seeds(m: int, k: int, a: float = 1.0, shift=(0.1, 0.13)):
    """Triangular lattice of m x k seeds (k even) with spacing a.

    Its periodic Voronoi tessellation is the regular honeycomb of side
    s = a / sqrt(3) in a box Lx = m a, Ly = k a sqrt(3) / 2.  The whole
    lattice is shifted by ``shift`` (in units of a) so that no Voronoi vertex
    falls on a box edge.  Returns (seeds, Lx, Ly).
    """
    if k % 2:
        raise ValueError("k must be even for a periodic triangular lattice")
    h = a * math.sqrt(3.0) / 2.0
    Lx, Ly = m * a, k * h
    pts = []
    for j in range(k):
        for i in range(m):
            x = (i + 0.5 * (j % 2) + shift[0]) * a
            y = j * h + shift[1] * a
            pts.append((x % Lx, y % Ly))
    return np.asarray(pts, dtype=np.float64), Lx, Ly


def dimensional(A0: float, kA: float, kP: float, p0: float, lam):
    """Dimensional (K_A, K_P, A0, P0, Lambda) of a tissue of target area A0
    whose moduli are given in cell units (energy unit A0)."""
    r = math.sqrt(A0)
    return dict(KA=kA / A0, KP=kP, A0=A0, P0=p0 * r, lam=np.asarray(lam) * r)


def tissue_c1():
    """100-cell tissue of the FP64 plain-method workload."""
    n, L = 100, 1.0
    seeds = uniform_seeds(n, L, L, SplitMix64(0))
    lam = SplitMix64(1).uniform(3 * n, 0.0, 0.1)
    return dict(seeds=seeds, Lx=L, Ly=L, n=n, **dimensional(0.01, 1.0, 1.0, 3.7, lam))


def tissue_c2(p0: float = 3.7):
    """10,000-cell tissue of the FP32 single-large-tissue workload."""
    n, L = 10_000, 1.0
    seeds = uniform_seeds(n, L, L, SplitMix64(2))
    return dict(seeds=seeds, Lx=L, Ly=L, n=n,
                **dimensional(1e-4, 1.0, 1.0, p0, np.full(3 * n, 0.05)))


C2_P0_SWEEP = (3.5, 3.7, 3.9)


def batch_c3(count: int = 512):
    """512 tissues of log-uniform size in [200, 5000] cells."""
    out = []
    for i in range(count):
        rng = substream(3, i)
        n = int(round(math.exp(rng.uniform(1, math.log(200), math.log(5000))[0])))
        L = math.sqrt(n)
        p0 = float(rng.uniform(1, 3.5, 4.0)[0])
        seeds = uniform_seeds(n, L, L, rng)
        lam = rng.uniform(3 * n, 0.0, 0.1)
        out.append(dict(seeds=seeds, Lx=L, Ly=L, n=n, A0=1.0, KA=1.0, KP=1.0,
                        P0=p0, lam=lam))
    return out


def tissue_c4():
    """1,000-cell tissue of the parameter-inference workload."""
    n = 1000
    L = math.sqrt(n)
    rng = SplitMix64(4)
    seeds = uniform_seeds(n, L, L, rng)
    lam_hidden = rng.uniform(3 * n, 0.02, 0.1)
    lam_trial = rng.uniform(3 * n, 0.02, 0.1)
    fd_edges = (rng.next_u64(20) % np.uint64(3 * n)).astype(np.int64)
    return dict(seeds=seeds, Lx=L, Ly=L, n=n, A0=1.0, KA=1.0, KP=1.0,
                P0=3.7, lam_hidden=lam_hidden, lam=lam_trial, fd_edges=fd_edges)


def batch_c5(count: int = 64, n: int = 10_000):
    """64 tissues of 10,000 cells for the batched inverse-design workload."""
    L = math.sqrt(n)
    out = []
    for i in range(count):
        rng = substream(5, i)
        seeds = uniform_seeds(n, L, L, rng)
        lam = rng.uniform(3 * n, 0.0, 0.1)
        out.append(dict(seeds=seeds, Lx=L, Ly=L, n=n, A0=1.0, KA=1.0, KP=1.0,
                        P0=3.7, lam=lam, q_target=(0.1, 0.0)))
    return out


def small_tissue(n: int, stream: int, A0: float = 1.0, p0: float = 3.7,
                 lam_range=(0.0, 0.1), aspect: float = 1.0):
    """A small random tissue for tests: n cells of target area A0 in a box of
    area n A0 (Lx / Ly = aspect)."""
    Ly = math.sqrt(n * A0 / aspect)
    Lx = n * A0 / Ly
    rng = SplitMix64(stream)
    seeds = uniform_seeds(n, Lx, Ly, rng)
    lam = rng.uniform(3 * n, *lam_range)
    return dict(seeds=seeds, Lx=Lx, Ly=Ly, n=n, **dimensional(A0, 1.0, 1.0, p0, lam))
