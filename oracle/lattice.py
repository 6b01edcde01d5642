"""Discrete velocity sets (Sec. 2.1, Fig. 1; weights in the paragraph after Eq. feq).

Pins: tests/test_oracle_lattice.py checks the exact rational isotropy identities
(sum w = 1, sum w c = 0, sum w c c = c_s^2 I, fourth-order isotropy) that any
dropped or mis-signed velocity would break.

The D2Q9 and D3Q27 orderings are those of Fig. 1.  D3Q19 (not printed in the
paper) keeps the D3Q27 ordering of the 6 axis and 12 edge velocities and puts
the rest velocity last, with the textbook weights 1/3, 1/18, 1/36.
"""
import numpy as np

CS2 = 1.0 / 3.0  # lattice speed of sound squared (dx = dt = 1)


class Lattice:
    def __init__(self, name, c, w):
        self.name = name
        self.c = np.array(c, dtype=np.int64)
        self.cf = self.c.astype(np.float64)
        self.w = np.array(w, dtype=np.float64)
        self.Q, self.D = self.c.shape
        self.opp = np.array(
            [int(np.flatnonzero((self.c == -self.c[i]).all(1))[0]) for i in range(self.Q)]
        )
        self.rest = int(np.flatnonzero((self.c == 0).all(1))[0])
        self.norm = np.sqrt((self.cf ** 2).sum(1))
        # mirror[i, m]: the velocity c_i with the components of the axes in bit mask m negated
        # (specular reflection at slip walls normal to those axes)
        self.mirror = np.zeros((self.Q, 2 ** self.D), dtype=np.int64)
        for i in range(self.Q):
            for m in range(2 ** self.D):
                sgn = np.array([-1 if (m >> a) & 1 else 1 for a in range(self.D)])
                self.mirror[i, m] = int(np.flatnonzero((self.c == sgn * self.c[i]).all(1))[0])


_D2 = [(-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (-1, 1), (1, 1), (1, -1), (0, 0)]
D2Q9 = Lattice("D2Q9", _D2, [1 / 9] * 4 + [1 / 36] * 4 + [4 / 9])

_AX3 = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
_ED3 = [(-1, -1, 0), (-1, 1, 0), (1, -1, 0), (1, 1, 0),
        (-1, 0, -1), (-1, 0, 1), (1, 0, -1), (1, 0, 1),
        (0, -1, -1), (0, -1, 1), (0, 1, -1), (0, 1, 1)]
_CO3 = [(-1, -1, -1), (-1, -1, 1), (-1, 1, -1), (-1, 1, 1),
        (1, -1, -1), (1, -1, 1), (1, 1, -1), (1, 1, 1)]
D3Q19 = Lattice("D3Q19", _AX3 + _ED3 + [(0, 0, 0)], [1 / 18] * 6 + [1 / 36] * 12 + [1 / 3])
D3Q27 = Lattice("D3Q27", _AX3 + _ED3 + _CO3 + [(0, 0, 0)],
                [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8 + [8 / 27])

LATTICES = {"D2Q9": D2Q9, "D3Q19": D3Q19, "D3Q27": D3Q27}


def get(name):
    return LATTICES[name]
