"""Structured box mesh of quads/hexes and dense per-element basis matrices.

Follows the operator decomposition A = P^T G^T B^T D B G P of Sec. 2.2, Eq. (8), in its
plainest form: G is an explicit element-to-node connectivity array and B is a dense
(Q^d x D^d) matrix per reference element (the Kronecker product of the 1D tables,
written out entry by entry).  P is the identity (one subdomain).

Numbering (shared convention with the CUDA path; the index arithmetic is re-derived
independently there):

* elements lexicographic, x fastest: e = ex + nx*(ey + ny*ez);
* H1 nodes on the global (k*nx+1) x (k*ny+1) [x (k*nz+1)] lattice, x fastest;
* element-local H1 node a = a0 + D*(a1 + D*a2), L2 dof j = j0 + L*(j1 + L*j2),
  quadrature point q = q0 + Q*(q1 + Q*q2), D = k+1, L = k, Q = 2k;
* state vectors U = [x | v | e]: x and v stored by component (all nodes of component 0,
  then 1, ...), e element-major.
"""
import itertools
import numpy as np

from . import quadrature as qr


class Mesh:
    """Box [lo, hi] split into n[0] x n[1] (x n[2]) equal elements, H1 order k."""

    def __init__(self, n, lo, hi, k, nq1d=None):
        self.d = len(n)
        self.n = tuple(int(v) for v in n)
        self.lo = np.asarray(lo, dtype=float)
        self.hi = np.asarray(hi, dtype=float)
        self.k = int(k)
        self.D = self.k + 1
        self.L = self.k
        self.Q = int(nq1d) if nq1d else 2 * self.k
        self.h = (self.hi - self.lo) / np.asarray(self.n)
        self.NE = int(np.prod(self.n))
        self.lat = tuple(self.k * m + 1 for m in self.n)     # H1 lattice extents
        self.NV = int(np.prod(self.lat))
        self.ND = self.D ** self.d                           # H1 dofs per element
        self.NL = self.L ** self.d                           # L2 dofs per element
        self.NQ = self.Q ** self.d                           # qp per element
        self.NEd = self.NE * self.NL                         # L2 unknowns
        self.n_unknowns = 2 * self.d * self.NV + self.NEd
        self._build_1d()
        self._build_dense()
        self._build_connectivity()

    # -- 1D tables -------------------------------------------------------------------
    def _build_1d(self):
        self.zq, self.wq = qr.gauss_legendre(self.Q)
        self.zh = qr.h1_nodes(self.k)
        self.zl = qr.l2_nodes(self.k)
        self.b1 = qr.lagrange(self.zh, self.zq)          # [Q, D]
        self.g1 = qr.lagrange_deriv(self.zh, self.zq)    # [Q, D]
        self.l1 = qr.lagrange(self.zl, self.zq)          # [Q, L]

    # -- dense reference-element matrices ---------------------------------------------
    def _multi(self, m):
        """Multi-indices (i0, i1[, i2]) in x-fastest order."""
        return [tuple(reversed(t)) for t in itertools.product(range(m), repeat=self.d)]

    def _build_dense(self):
        d, qs, hs, ls = self.d, self._multi(self.Q), self._multi(self.D), self._multi(self.L)
        self.Bh = np.zeros((self.NQ, self.ND))            # value of H1 basis a at qp q
        self.Gh = np.zeros((self.NQ, d, self.ND))         # reference gradient
        self.Bl = np.zeros((self.NQ, self.NL))            # value of L2 basis j at qp q
        self.alpha = np.zeros(self.NQ)                    # reference quadrature weight
        for iq, q in enumerate(qs):
            self.alpha[iq] = np.prod([self.wq[q[c]] for c in range(d)])
            for ia, a in enumerate(hs):
                self.Bh[iq, ia] = np.prod([self.b1[q[c], a[c]] for c in range(d)])
                for r in range(d):
                    self.Gh[iq, r, ia] = np.prod(
                        [(self.g1 if c == r else self.b1)[q[c], a[c]] for c in range(d)])
            for ij, j in enumerate(ls):
                self.Bl[iq, ij] = np.prod([self.l1[q[c], j[c]] for c in range(d)])
        self.qref = np.array([[self.zq[q[c]] for c in range(d)] for q in qs])   # [NQ, d]
        self.lref = np.array([[self.zl[j[c]] for c in range(d)] for j in ls])   # [NL, d]
        self.href = np.array([[self.zh[a[c]] for c in range(d)] for a in hs])   # [ND, d]

    # -- connectivity (the G operator) -----------------------------------------------------
    def _build_connectivity(self):
        d, k = self.d, self.k
        self.conn = np.zeros((self.NE, self.ND), dtype=np.int64)
        self.ecoord = np.zeros((self.NE, d), dtype=np.int64)
        hs = self._multi(self.D)
        for e, ec in enumerate(self._multi_el()):
            self.ecoord[e] = ec
            for ia, a in enumerate(hs):
                g = [ec[c] * k + a[c] for c in range(d)]
                idx, stride = 0, 1
                for c in range(d):
                    idx += g[c] * stride
                    stride *= self.lat[c]
                self.conn[e, ia] = idx

    def _multi_el(self):
        ranges = [range(m) for m in reversed(self.n)]
        return [tuple(reversed(t)) for t in itertools.product(*ranges)]

    # -- geometry ------------------------------------------------------------------------
    def initial_nodes(self):
        """x0 on the undeformed box: component-major array [d, NV]."""
        x0 = np.zeros((self.d, self.NV))
        for e in range(self.NE):
            for ia in range(self.ND):
                x0[:, self.conn[e, ia]] = self.lo + self.h * (self.ecoord[e] + self.href[ia])
        return x0

    def l2_node_positions(self):
        """Physical positions of the L2 nodes on the undeformed box: [NE*NL, d]."""
        pos = np.zeros((self.NE, self.NL, self.d))
        for e in range(self.NE):
            pos[e] = self.lo + self.h * (self.ecoord[e] + self.lref)
        return pos.reshape(-1, self.d)

    def element_centres(self):
        return self.lo + self.h * (self.ecoord + 0.5)

    def boundary_mask(self, bc_mask):
        """Boolean [d, NV]: True where velocity component c is fixed (v.n = 0).

        Bit 2*c + s of ``bc_mask`` selects the face of axis c at the low (s=0) or high
        (s=1) end of the box.
        """
        fixed = np.zeros((self.d, self.NV), dtype=bool)
        ids = np.arange(self.NV)
        for c in range(self.d):
            stride = int(np.prod(self.lat[:c]))
            coord = (ids // stride) % self.lat[c]
            if bc_mask & (1 << (2 * c)):
                fixed[c] |= coord == 0
            if bc_mask & (1 << (2 * c + 1)):
                fixed[c] |= coord == self.lat[c] - 1
        return fixed

    # -- vector views ----------------------------------------------------------------------
    def split(self, U):
        """U = [x | v | e] -> (x [d, NV], v [d, NV], e [NE, NL])."""
        n1 = self.d * self.NV
        x = U[:n1].reshape(self.d, self.NV)
        v = U[n1:2 * n1].reshape(self.d, self.NV)
        e = U[2 * n1:].reshape(self.NE, self.NL)
        return x, v, e

    def join(self, x, v, e):
        return np.concatenate([np.ravel(x), np.ravel(v), np.ravel(e)])

    def gather(self, f):
        """H1 field [d, NV] -> element values [NE, d, ND] (the G operator)."""
        return np.transpose(f[:, self.conn], (1, 0, 2))

    def scatter(self, fe):
        """Element values [NE, d, ND] -> summed H1 field [d, NV] (G^T)."""
        dt = np.result_type(fe.dtype, np.float64)
        out = np.zeros((self.d, self.NV), dtype=dt)
        for c in range(self.d):
            np.add.at(out[c], self.conn, fe[:, c, :])
        return out
