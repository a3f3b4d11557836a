"""Discrete-velocity lattices for the oracle (test infrastructure only).

The paper works on D3Q19 (Sec. III A, "adopted in the present investigation");
the two-component workloads also run on D3Q27.  Both are built here by
enumerating the 27 vectors of {-1, 0, 1}^3 and keeping those whose squared
length is allowed, with the standard weights of each shell:

    D3Q19: |c|^2 = 0, 1, 2          w = 1/3, 1/18, 1/36
    D3Q27: |c|^2 = 0, 1, 2, 3       w = 8/27, 2/27, 1/54, 1/216

Both lattices have sound speed c_s^2 = 1/3 (Sec. II, after the momentum
equation: c_s = 1/sqrt(3)).

These tables are written independently of the CUDA library's own tables;
nothing here is shared with the GPU path.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

CS2 = 1.0 / 3.0  # c_s^2, Sec. II

_SHELL_WEIGHTS = {
    19: {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0},
    27: {0: 8.0 / 27.0, 1: 2.0 / 27.0, 2: 1.0 / 54.0, 3: 1.0 / 216.0},
}


@dataclass(frozen=True)
class Lattice:
    """A 3D lattice: velocities ``c`` (Q x 3 int) and weights ``w`` (Q float64)."""

    name: str
    c: np.ndarray
    w: np.ndarray

    @property
    def Q(self) -> int:
        return int(self.c.shape[0])


def make_lattice(q: int) -> Lattice:
    """Build D3Q19 (``q=19``) or D3Q27 (``q=27``).

    Velocities are ordered by shell (rest first), and inside a shell by the
    lexicographic order of itertools.product over (-1, 0, 1); the order does
    not matter to any result of the oracle.
    """
    if q not in _SHELL_WEIGHTS:
        raise ValueError(f"unsupported lattice D3Q{q}; use 19 or 27")
    weights = _SHELL_WEIGHTS[q]
    vecs = [v for v in itertools.product((-1, 0, 1), repeat=3) if sum(a * a for a in v) in weights]
    vecs.sort(key=lambda v: sum(a * a for a in v))
    c = np.array(vecs, dtype=np.int64)
    w = np.array([weights[int((v * v).sum())] for v in c], dtype=np.float64)
    assert c.shape[0] == q
    return Lattice(name=f"D3Q{q}", c=c, w=w)


D3Q19 = make_lattice(19)
D3Q27 = make_lattice(27)


def lattice(q: int) -> Lattice:
    return D3Q19 if q == 19 else D3Q27 if q == 27 else make_lattice(q)
