"""Seeded synthetic instances shaped like the paper's workloads.

This module holds input generators only -- lattices, coupling values and their seeds --
and none of the method's arithmetic.  Both the CUDA path and the CPU oracle take their
instances from here.  Start vectors are not generated here: the library draws them on
the device from SplitMix64 and the oracle implements the same published generator on
its own.

The systems are spin rings with nearest- and next-nearest-neighbour exchange and s = 1
random regular graphs, the kinds of Heisenberg systems the paper treats (Sec. 2, and
the applications it cites in Sec. 1).  Sites are numbered 0..N-1; the site number is the
digit position of the subspace coding (position N-1 most significant).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Instance:
    name: str
    n_sites: int
    two_s: int
    two_m: int
    u: np.ndarray
    v: np.ndarray
    J: np.ndarray
    steps: int = 0
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def A(self) -> int:
        t = self.n_sites * self.two_s - self.two_m
        assert t % 2 == 0
        return t // 2

    @property
    def n_bonds(self) -> int:
        return int(self.u.shape[0])


def ring_bonds(n_sites: int, j1: float, j2: float | None = None):
    """Nearest-neighbour bonds (i, i+1 mod N) with coupling j1, then, if j2 is given,
    next-nearest-neighbour bonds (i, i+2 mod N) with coupling j2."""
    u, v, J = [], [], []
    for i in range(n_sites):
        u.append(i); v.append((i + 1) % n_sites); J.append(j1)
    if j2 is not None:
        for i in range(n_sites):
            u.append(i); v.append((i + 2) % n_sites); J.append(j2)
    return (np.array(u, dtype=np.int32), np.array(v, dtype=np.int32),
            np.array(J, dtype=np.float64))


def random_regular_graph(n_sites: int, degree: int, seed: int):
    """Edges of a simple random `degree`-regular graph: configuration-model pairing of
    n_sites*degree stubs with numpy's PCG64, redrawn until no self-loop or multi-edge
    remains.  Returned sorted as (u < v) pairs."""
    assert (n_sites * degree) % 2 == 0
    rng = np.random.Generator(np.random.PCG64(seed))
    stubs = np.repeat(np.arange(n_sites), degree)
    for _ in range(100000):
        perm = rng.permutation(stubs)
        pairs = perm.reshape(-1, 2)
        a = np.minimum(pairs[:, 0], pairs[:, 1])
        b = np.maximum(pairs[:, 0], pairs[:, 1])
        if np.any(a == b):
            continue
        keys = a * n_sites + b
        if len(np.unique(keys)) != len(keys):
            continue
        order = np.lexsort((b, a))
        return a[order].astype(np.int32), b[order].astype(np.int32)
    raise RuntimeError("no simple regular graph found")


def uniform_couplings(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=n).astype(np.float64)


# ---- the five workloads -----------------------------------------------------------------

def ring16() -> Instance:
    """s = 1/2 ring, N = 16, J = -1 (antiferromagnetic), M = 0, 100 steps, start seed 1001."""
    u, v, J = ring_bonds(16, -1.0)
    return Instance("ring16_s12_M0", 16, 1, 0, u, v, J, steps=100, seed=1001)


def j1j2_ring32() -> Instance:
    """s = 1/2 J1-J2 ring, N = 32, J1 = -1, J2 = -0.5, M = 0 (dim C(32,16)), 60 steps."""
    u, v, J = ring_bonds(32, -1.0, -0.5)
    return Instance("j1j2_ring32_s12_M0", 32, 1, 0, u, v, J, steps=60, seed=1002)


def j1j2_ring(n_sites: int, j2: float = -0.5, seed: int = 1002) -> Instance:
    """s = 1/2 J1-J2 ring of any even N (J1 = -1), M = 0 -- mid-size cases for profiling."""
    u, v, J = ring_bonds(n_sites, -1.0, j2)
    return Instance(f"j1j2_ring{n_sites}_s12_M0", n_sites, 1, 0, u, v, J, steps=60, seed=seed)


def s1_random_graph(n_sites: int = 20, graph_seed: int = 3) -> Instance:
    """s = 1, each site bonded to 4 random partners, J ~ U[-1.5, -0.5], M = 0, 80 steps."""
    a, b = random_regular_graph(n_sites, 4, graph_seed)
    J = uniform_couplings(len(a), -1.5, -0.5, graph_seed)
    return Instance(f"s1_rrg{n_sites}_M0", n_sites, 2, 0, a, b, J, steps=80, seed=1003,
                    meta={"graph_seed": graph_seed})


def s1_random_graph_small() -> Instance:
    """The N = 12 companion of s1_random_graph (graph seed 13, dim 73,789)."""
    return s1_random_graph(12, 13)


def ring24_random_j() -> Instance:
    """s = 1/2 ring N = 24, nearest and next-nearest bonds with J ~ U[-1.2, -0.8]
    (48 couplings, seed 4), M = 0."""
    u, v, _ = ring_bonds(24, 0.0, 0.0)
    J = uniform_couplings(len(u), -1.2, -0.8, 4)
    return Instance("ring24_randJ_s12_M0", 24, 1, 0, u, v, J, steps=80, seed=1004)


def ftlm_ring24() -> Instance:
    """s = 1/2 ring N = 24, J1 = -1, J2 = -0.3; all sectors, R = 32 +-1 vectors, 80 steps."""
    u, v, J = ring_bonds(24, -1.0, -0.3)
    return Instance("ftlm_ring24_j1j2", 24, 1, 0, u, v, J, steps=80, seed=1005,
                    meta={"R": 32})


def arnoldi_ring24() -> Instance:
    """s = 1/2 J1-J2 ring N = 24 (J1 = -1, J2 = -0.3), M = 0, 60 Arnoldi steps, seed 1006."""
    u, v, J = ring_bonds(24, -1.0, -0.3)
    return Instance("arnoldi_ring24_j1j2", 24, 1, 0, u, v, J, steps=60, seed=1006)


def small_ring(n_sites: int, j1: float = -1.0, j2: float | None = None, two_s: int = 1,
               two_m: int | None = None) -> Instance:
    """A small ring for tests (M = lowest |M| unless given)."""
    u, v, J = ring_bonds(n_sites, j1, j2)
    if two_m is None:
        two_m = (n_sites * two_s) % 2
    return Instance(f"ring{n_sites}", n_sites, two_s, two_m, u, v, J, steps=60, seed=7)
