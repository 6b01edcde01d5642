"""Dense Cartesian level geometry used by the oracle.

A level is a box of ``dims`` = (nx, ny[, nz]) cells, flat index x fastest
(idx = x + nx*(y + ny*z)).  Cell centres sit at (i + 1/2) in that level's cell
units, so box walls lie on cell faces and every wall link has q = 1/2
(half-way bounce-back, Eq. bb with q = 1/2).  Axes are periodic or walled;
a walled axis is no-slip (bounce-back) or slip (specular reflection: the
velocity component normal to the wall changes sign, the tangential motion
goes on; the paper's lateral walls of Sec. 3.2, u.n = 0 and no shear).

Blocks tile the level in ``block`` cells per axis (the last block of an axis may
be ragged); they are the unit of refinement (Sec. 2.6).
"""
import numpy as np


class LevelGeom:
    def __init__(self, dims, periodic, block, slip=None):
        self.dims = tuple(int(d) for d in dims)
        self.D = len(self.dims)
        self.periodic = tuple(bool(p) for p in periodic)
        self.slip = tuple(bool(s) and not p for s, p in zip(slip or (False,) * self.D, self.periodic))
        self.block = tuple(int(b) for b in block)
        self.N = int(np.prod(self.dims))
        idx = np.arange(self.N)
        coord = []
        rem = idx
        for a in range(self.D):
            coord.append(rem % self.dims[a])
            rem = rem // self.dims[a]
        self.coord = np.stack(coord)  # (D, N)
        self.bdims = tuple((d + b - 1) // b for d, b in zip(self.dims, self.block))
        self.NB = int(np.prod(self.bdims))
        bc = self.coord // np.array(self.block)[:, None]
        self.block_of = self.flat_block(bc)

    def flat(self, coord):
        out = np.zeros(coord.shape[1:], dtype=np.int64)
        mul = 1
        for a in range(self.D):
            out = out + coord[a] * mul
            mul *= self.dims[a]
        return out

    def flat_block(self, bcoord):
        out = np.zeros(bcoord.shape[1:], dtype=np.int64)
        mul = 1
        for a in range(self.D):
            out = out + bcoord[a] * mul
            mul *= self.bdims[a]
        return out

    def block_coord(self, b):
        b = np.asarray(b)
        out = []
        for a in range(self.D):
            out.append(b % self.bdims[a])
            b = b // self.bdims[a]
        return np.stack(out)

    def _off(self, offset, cells):
        off = np.asarray(offset)
        if off.ndim == 1:
            return off.reshape(-1, *([1] * cells.ndim))
        return off  # one offset per cell, shape (D, *cells.shape)

    def shift(self, cells, offset):
        """Flat index of cell + offset, wrapping periodic axes.

        Returns (index, wall_axis): index is -1 where the target leaves the box
        through a walled axis; wall_axis is the first such axis (x, y, z order)
        times 2 plus 1 for the upper face, else -1.
        """
        cells = np.asarray(cells)
        co = self.coord[:, cells] + self._off(offset, cells)
        bad = np.zeros(cells.shape, dtype=bool)
        face = np.full(cells.shape, -1, dtype=np.int64)
        for a in range(self.D):
            n = self.dims[a]
            if self.periodic[a]:
                co[a] = co[a] % n
            else:
                lo = co[a] < 0
                hi = co[a] >= n
                newf = (~bad) & (lo | hi)
                face = np.where(newf & lo, 2 * a, face)
                face = np.where(newf & hi, 2 * a + 1, face)
                bad |= lo | hi
                co[a] = np.clip(co[a], 0, n - 1)
        idx = self.flat(co)
        return np.where(bad, -1, idx), face

    def pull(self, cells, ck):
        """Where the population that streams into ``cells`` with velocity ``ck`` comes from.

        Returns (src, face, flip).  Through a slip wall the population was
        reflected: its source keeps the cell's coordinate along that axis and it
        left the source with that component negated (bit a of ``flip``).  Through
        a no-slip wall (which wins where a link crosses both kinds) src is -1 and
        face is the first such face (2 a, + 1 for the upper one), as in ``shift``.
        """
        cells = np.asarray(cells)
        co = self.coord[:, cells] - np.asarray(ck).reshape(-1, *([1] * cells.ndim))
        bad = np.zeros(cells.shape, dtype=bool)
        face = np.full(cells.shape, -1, dtype=np.int64)
        flip = np.zeros(cells.shape, dtype=np.int64)
        for a in range(self.D):
            n = self.dims[a]
            if self.periodic[a]:
                co[a] = co[a] % n
                continue
            lo = co[a] < 0
            hi = co[a] >= n
            out = lo | hi
            if self.slip[a]:
                flip = np.where(out, flip | (1 << a), flip)
                co[a] = np.where(out, self.coord[a, cells], co[a])
            else:
                newf = (~bad) & out
                face = np.where(newf & lo, 2 * a, face)
                face = np.where(newf & hi, 2 * a + 1, face)
                bad |= out
                co[a] = np.clip(co[a], 0, n - 1)
        idx = self.flat(co)
        flip = np.where(bad, 0, flip)
        return np.where(bad, -1, idx), face, flip

    def clamp_shift(self, cells, offset):
        """Like shift, but walled axes clamp to the box (zero-gradient ghosts)."""
        cells = np.asarray(cells)
        co = self.coord[:, cells] + self._off(offset, cells)
        for a in range(self.D):
            n = self.dims[a]
            co[a] = co[a] % n if self.periodic[a] else np.clip(co[a], 0, n - 1)
        return self.flat(co)

    def centers(self, scale=1.0):
        """Cell centres, optionally scaled to another level's cell units."""
        return (self.coord.astype(np.float64) + 0.5) * scale

    def block_neighbors(self, b):
        """Flat indices of the 3^D block neighbourhood of block b (incl. b)."""
        bc = self.block_coord(np.array([b]))[:, 0]
        out = []
        for off in np.ndindex(*([3] * self.D)):
            c = bc + np.array(off) - 1
            ok = True
            for a in range(self.D):
                if self.periodic[a]:
                    c[a] %= self.bdims[a]
                elif c[a] < 0 or c[a] >= self.bdims[a]:
                    ok = False
            if ok:
                out.append(int(self.flat_block(c.reshape(-1, 1))[0]))
        return sorted(set(out))
