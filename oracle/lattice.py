"""Lattice tables for the oracle (Sec. 3, lattice definitions).

D2Q9: e0=(0,0), e1,3=(+-1,0), e2,4=(0,+-1), e5,6=(+-1,1), e7,8=(-+1,-1);
w0=4/9, w1..4=1/9, w5..8=1/36; cs^2=1/3.
D3Q7: e1..e6 the six unit axis vectors; w0=1/4, w1..6=1/8; cs^2 = sum_i w_i e_ix^2
= 1/4 (the paper's "e^2 = 1/4").
D3Q19: D3Q7's axis vectors plus the twelve face diagonals in the order
e7,8=(+-1,1,0), e9,10=(+-1,-1,0), e11,12=(+-1,0,1), e13,14=(+-1,0,-1),
e15,16=(0,+-1,1), e17,18=(0,+-1,-1); w0=1/3, w1..6=1/18, w7..18=1/36; cs^2=1/3.

The paper lists only e1=(1,0,0), e2=(0,1,0) and e6=(0,0,-1) of the axis
vectors; the order e3=(0,0,1), e4=(-1,0,0), e5=(0,-1,0) is a reading taken
here (it mirrors the D2Q9 pattern).  The order only fixes the summation order.
"""
from dataclasses import dataclass
from fractions import Fraction

import numpy as np


@dataclass(frozen=True)
class Lattice:
    name: str
    e: np.ndarray          # (Q, D) integer velocities
    w: tuple               # Q weights as Fractions (exact)
    cs2: Fraction          # lattice sound speed squared

    @property
    def Q(self):
        return self.e.shape[0]

    @property
    def D(self):
        return self.e.shape[1]

    @property
    def opposite(self):
        """Index i' with e_i' = -e_i, found by search (no table)."""
        out = []
        for i in range(self.Q):
            for j in range(self.Q):
                if np.array_equal(self.e[j], -self.e[i]):
                    out.append(j)
                    break
        return tuple(out)

    def wf(self, i):
        return float(self.w[i])


def _frac(*vals):
    return tuple(Fraction(v) for v in vals)


D2Q9 = Lattice(
    "D2Q9",
    np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1),
              (1, 1), (-1, 1), (-1, -1), (1, -1)], dtype=np.int64),
    _frac("4/9", "1/9", "1/9", "1/9", "1/9", "1/36", "1/36", "1/36", "1/36"),
    Fraction(1, 3),
)

_AXES3 = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0), (0, -1, 0), (0, 0, -1)]

D3Q7 = Lattice(
    "D3Q7",
    np.array([(0, 0, 0)] + _AXES3, dtype=np.int64),
    _frac("1/4", *(["1/8"] * 6)),
    Fraction(1, 4),
)

D3Q19 = Lattice(
    "D3Q19",
    np.array([(0, 0, 0)] + _AXES3 + [
        (1, 1, 0), (-1, 1, 0), (1, -1, 0), (-1, -1, 0),
        (1, 0, 1), (-1, 0, 1), (1, 0, -1), (-1, 0, -1),
        (0, 1, 1), (0, -1, 1), (0, 1, -1), (0, -1, -1)], dtype=np.int64),
    _frac("1/3", *(["1/18"] * 6), *(["1/36"] * 12)),
    Fraction(1, 3),
)


def lattices_for(dim):
    """(flow/heat lattice, phase-field lattice, stencil lattice) per dimension.

    2D: D2Q9 for f, g and s (Sec. 5.1).  3D: D3Q19 for f and s, D3Q7 for g,
    and the D3Q19 neighbours for the finite-difference stencils.
    """
    if dim == 2:
        return D2Q9, D2Q9, D2Q9
    if dim == 3:
        return D3Q19, D3Q7, D3Q19
    raise ValueError("dim must be 2 or 3")
