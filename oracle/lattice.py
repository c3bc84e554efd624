"""D2Q9 and D3Q19 velocity sets (Sec. 2; weights are the textbook values the
paper relies on without printing them).

Velocity order is the library's documented population order:
  D2Q9 : 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+x+y), 6 (-x+y), 7 (-x-y), 8 (+x-y)
  D3Q19: 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z,
         7 (+x+y), 8 (-x-y), 9 (+x-y), 10 (-x+y),
         11 (+x+z), 12 (-x-z), 13 (+x-z), 14 (-x+z),
         15 (+y+z), 16 (-y-z), 17 (+y-z), 18 (-y+z)
Weights depend only on |c|^2: D2Q9 4/9, 1/9, 1/36; D3Q19 1/3, 1/18, 1/36.
c_s^2 = 1/3 for both.
"""

import numpy as np

CS2 = 1.0 / 3.0

_D2Q9 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0), (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)]
_D3Q19 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
          (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
          (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
          (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


class Lattice:
    def __init__(self, dim):
        self.dim = dim
        if dim == 2:
            self.c = np.array(_D2Q9, dtype=np.int64)
            by_norm = {0: 4.0 / 9.0, 1: 1.0 / 9.0, 2: 1.0 / 36.0}
        elif dim == 3:
            self.c = np.array(_D3Q19, dtype=np.int64)
            by_norm = {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}
        else:
            raise ValueError("dim must be 2 or 3")
        self.q = len(self.c)
        self.w = np.array([by_norm[int(np.dot(ci, ci))] for ci in self.c])
        self.opp = np.array([int(np.where((self.c == -ci).all(axis=1))[0][0]) for ci in self.c])
        self.cf = self.c.astype(np.float64)
