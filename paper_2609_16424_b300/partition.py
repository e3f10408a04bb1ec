"""Two-slab decomposition of a box mesh, emulated on one GPU (paper Sec. 2.2, Eq. (8) with
the parallel prolongation P != I).

The box is cut across its last axis into two sub-box meshes with separate buffers.  Each
evaluates its operators on its own elements; the velocity rows of the nodes on the cut
then hold partial sums, and one exchange (pack the face, copy it to the other side, add it
into the free rows: the P^T of the paper) completes them.  Interface nodes are stored on
both sides and owned by the lower slab; L2 rows are element-local and need no exchange.
On several GPUs the copy would be a point-to-point transfer between ranks; here it is a
device copy between the two buffers.
"""
import torch

from .hydro import Mesh


def slab_maps(dim, n, k, cut, device="cpu"):
    """Global row of every local row of the two slabs ([x | v | e] layout of both), and
    the rows each slab owns (the cut plane belongs to the lower slab).  Returns
    (n_global, [rows_0, rows_1], [owned_0, owned_1])."""
    axis = dim - 1
    ext = [k * n[c] + 1 for c in range(dim)]
    nv_g = 1
    for e in ext:
        nv_g *= e
    plane = nv_g // ext[axis]                       # nodes per lattice plane of the last axis
    ne_plane = 1
    for c in range(dim - 1):
        ne_plane *= n[c]
    nl = k ** dim
    ne_g = ne_plane * n[axis]
    n_g = 2 * dim * nv_g + ne_g * nl
    rows, owned = [], []
    for p, (z0, nz, e0) in enumerate(((0, cut, 0), (k * cut, n[axis] - cut, cut * ne_plane))):
        nv = plane * (k * nz + 1)
        ne = ne_plane * nz
        nodes = torch.arange(nv, device=device) + z0 * plane   # the same plane layout on both sides
        erows = torch.arange(ne * nl, device=device) + 2 * dim * nv_g + e0 * nl
        rows.append(torch.cat([nodes + c * nv_g for c in range(2 * dim)] + [erows]))
        own_node = torch.ones(nv, dtype=torch.bool, device=device)
        if p == 1:
            own_node[:plane] = False
        owned.append(torch.cat([own_node] * (2 * dim) + [torch.ones(ne * nl, dtype=torch.bool, device=device)]))
    return n_g, rows, owned


class SlabPair:
    def __init__(self, dim, n, lo, hi, order, cut, rho0=1.0, gamma=1.4, bc_mask=None, device=None, **kw):
        axis = dim - 1
        n = [int(x) for x in n]
        if not 0 < cut < n[axis]:
            raise ValueError("cut must split the last axis into two non-empty slabs")
        self.dim, self.n, self.order, self.axis, self.cut = dim, n, order, axis, cut
        self.device = torch.device(device or "cuda")
        bc = (1 << (2 * dim)) - 1 if bc_mask is None else int(bc_mask)
        h_ax = (hi[axis] - lo[axis]) / n[axis]
        z_cut = lo[axis] + cut * h_ax
        vol = 1.0
        ne = 1
        for c in range(dim):
            vol *= hi[c] - lo[c]
            ne *= n[c]
        h0 = kw.pop("h0", 0.0) or (vol / ne) ** (1.0 / dim)
        h_coarse = kw.pop("h_coarse", 0.0) or h0
        ne_plane = ne // n[axis]
        self.face_hi, self.face_lo = 2 * axis + 1, 2 * axis
        self.parts = []
        for p, (za, zb, nz) in enumerate(((lo[axis], z_cut, cut), (z_cut, hi[axis], n[axis] - cut))):
            lo_p, hi_p, n_p = list(lo), list(hi), list(n)
            lo_p[axis], hi_p[axis], n_p[axis] = za, zb, nz
            e0 = 0 if p == 0 else cut * ne_plane
            e1 = cut * ne_plane if p == 0 else ne
            mat = {name: (val[e0:e1] if hasattr(val, "__len__") else val)
                   for name, val in (("rho0", rho0), ("gamma", gamma))}
            bc_p = bc & ~(1 << (self.face_hi if p == 0 else self.face_lo))
            self.parts.append(Mesh(dim, n_p, lo_p, hi_p, order, rho0=mat["rho0"], gamma=mat["gamma"],
                                   bc_mask=bc_p, h0=h0, h_coarse=h_coarse, device=self.device, **kw))
        self._maps()

    def _maps(self):
        self.n_g, self.rows, self.owned = slab_maps(self.dim, self.n, self.order, self.cut, self.device)

    def split(self, v):
        """Local copies of a global vector (interface nodes on both sides)."""
        return [v[r].contiguous() for r in self.rows]

    def join(self, parts):
        """Global vector from the owned rows of each part."""
        out = torch.empty(self.n_g, dtype=parts[0].dtype, device=self.device)
        for r, o, x in zip(self.rows, self.owned, parts):
            out[r[o]] = x[o]
        return out

    def exchange(self, parts):
        """The halo sum: both sides pack their face, the packs are swapped (device copies),
        each side adds the other's pack into its free velocity rows."""
        m0, m1 = self.parts
        b0 = m0.halo_pack(self.face_hi, parts[0])
        b1 = m1.halo_pack(self.face_lo, parts[1])
        recv0, recv1 = b1.clone(), b0.clone()
        m0.halo_add(self.face_hi, recv0, parts[0])
        m1.halo_add(self.face_lo, recv1, parts[1])
        return parts

    def residual(self, u, k, tau):
        us, ks = self.split(u), self.split(k)
        return self.join(self.exchange([m.residual(a, b, tau) for m, a, b in zip(self.parts, us, ks)]))

    def jvp(self, u, k, tau, dk):
        us, ks, ds = self.split(u), self.split(k), self.split(dk)
        return self.join(self.exchange([m.jvp(a, b, tau, d) for m, a, b, d in zip(self.parts, us, ks, ds)]))

    def jvp_record(self, u, k, tau, dk, tc=None):
        """Float J.w from each part's linearisation record (FP32 CUDA cores or tensor cores)."""
        us, ks, ds = self.split(u), self.split(k), self.split(dk)
        outs = []
        for m, a, b, d in zip(self.parts, us, ks, ds):
            m.linearize(a, b, tau)
            outs.append(m.jvp(a, b, tau, d, lin=True, tc=tc))
        return self.join(self.exchange(outs))

    def energies(self, u):
        """(kinetic, internal): sums over the parts (mass partial sums on the cut add up)."""
        ke, ie = 0.0, 0.0
        for m, a in zip(self.parts, self.split(u)):
            k1, i1 = m.energies(a)
            ke += k1
            ie += i1
        return ke, ie

    def dt_estimate(self, u):
        return min(m.dt_estimate(a) for m, a in zip(self.parts, self.split(u)))
