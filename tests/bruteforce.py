"""Naive per-output re-evaluation of the right-hand side L(U), for tiny grids.

Every output value is computed on its own from the definitions: each interface
flux, each edge field and each derivative is rebuilt from explicit stencils with
explicit periodic coordinates, memoised only so the run stays short.  It uses the
oracle's point-wise routines (each pinned on its own in test_oracle_pointwise.py)
and none of the oracle's grid loops, so it checks their assembly: positions,
offsets, orientation and signs of every stencil.
"""
import numpy as np

from oracle import oracle as orc


class BruteRHS:
    def __init__(self, cons, bf, W, L=(1.0, 1.0, 1.0), gam=4.0 / 3.0, ho=1, tol=1e-6):
        self.cons, self.bf, self.W = cons, bf, W
        self.nz, self.ny, self.nx = cons.shape[1:]
        self.N = (self.nx, self.ny, self.nz)
        self.h = [L[d] / self.N[d] for d in range(3)]
        self.gam, self.ho, self.tol = gam, ho, tol
        self._prim = {}
        self._face = {}
        self._edge = {}

    # value of a grid array at integer coordinates (x, y, z), periodic
    def _get(self, arr, x, y, z):
        return arr[z % self.nz, y % self.ny, x % self.nx]

    @staticmethod
    def _shift(pos, d, s):
        p = list(pos)
        p[d] += s
        return tuple(p)

    def prim(self, pos):
        """rho, vx, vy, vz, p, Bx, By, Bz at the centre of cell pos."""
        key = tuple(q % n for q, n in zip(pos, self.N))
        if key in self._prim:
            return self._prim[key]
        B = np.zeros(3)
        for d in range(3):
            # faces at d-3/2, d-1/2, d+1/2, d+3/2 are the face arrays at offsets -2..1
            s = [self._get(self.bf[d], *self._shift(key, d, o)) for o in (-2, -1, 0, 1)]
            B[d] = orc.interp(s, self.ho)
        u = np.array([self._get(self.cons[v], *key) for v in range(5)])
        p, _, _, bad = orc.c2p(u, B, self.gam, self._get(self.W, *key), tol=self.tol)
        assert bad == 0
        out = np.concatenate([p, B])
        self._prim[key] = out
        return out

    def face(self, d, pos):
        """Flux (8), a+, a- and the L/R velocity states on the face above pos along d."""
        key = (d,) + tuple(q % n for q, n in zip(pos, self.N))
        if key in self._face:
            return self._face[key]
        cells = [self.prim(self._shift(pos, d, o)) for o in range(-2, 4)]
        L = np.array([orc.mp5([cells[m][v] for m in range(0, 5)]) for v in range(8)])
        R = np.array([orc.mp5([cells[m][v] for m in range(5, 0, -1)]) for v in range(8)])
        bn = self._get(self.bf[d], *pos)
        L[5 + d] = bn
        R[5 + d] = bn
        f, ap, am = orc.hll(L[:5], L[5:], R[:5], R[5:], self.gam, d)
        out = (f, ap, am, L[1:4].copy(), R[1:4].copy())
        self._face[key] = out
        return out

    def edge(self, c, pos):
        """UCT field on the edge along c half a cell above pos along a and b."""
        key = (c,) + tuple(q % n for q, n in zip(pos, self.N))
        if key in self._edge:
            return self._edge[key]
        a, b = (c + 1) % 3, (c + 2) % 3
        # a-faces along b (offsets -2..3), each with L and R velocity states
        af = [self.face(a, self._shift(pos, b, o)) for o in range(-2, 4)]
        va = np.zeros((2, 2))
        vb = np.zeros((2, 2))
        for s, slot in ((0, 3), (1, 4)):
            comp_a = [af[m][slot][a] for m in range(6)]
            comp_b = [af[m][slot][b] for m in range(6)]
            va[s] = [orc.mp5(comp_a[0:5]), orc.mp5(comp_a[5:0:-1])]
            vb[s] = [orc.mp5(comp_b[0:5]), orc.mp5(comp_b[5:0:-1])]
        Ba_line = [self._get(self.bf[a], *self._shift(pos, b, o)) for o in range(-2, 4)]
        Bb_line = [self._get(self.bf[b], *self._shift(pos, a, o)) for o in range(-2, 4)]
        Ba = [orc.mp5(Ba_line[0:5]), orc.mp5(Ba_line[5:0:-1])]
        Bb = [orc.mp5(Bb_line[0:5]), orc.mp5(Bb_line[5:0:-1])]
        fa0, fa1 = af[2], af[3]                      # a-faces at b and b+1
        fb0 = self.face(b, pos)
        fb1 = self.face(b, self._shift(pos, a, 1))   # b-faces at a and a+1
        E = orc.uct_point(va, vb, Ba, Bb, max(fa0[1], fa1[1]), max(fa0[2], fa1[2]),
                          max(fb0[1], fb1[1]), max(fb0[2], fb1[2]))
        self._edge[key] = E
        return E

    def rhs_cell(self, pos):
        out = np.zeros(5)
        for d in range(3):
            fl = [self.face(d, self._shift(pos, d, o))[0] for o in range(-3, 3)]
            for c in range(5):
                out[c] -= orc.der([fl[m][c] for m in range(6)], self.h[d], self.ho)
        return out

    def rhs_face(self, a, pos):
        b, c = (a + 1) % 3, (a + 2) % 3
        ec = [self.edge(c, self._shift(pos, b, o)) for o in range(-3, 3)]
        eb = [self.edge(b, self._shift(pos, c, o)) for o in range(-3, 3)]
        return -(orc.der(ec, self.h[b], self.ho) - orc.der(eb, self.h[c], self.ho))
