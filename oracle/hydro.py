"""Stage residual R(k; tau, u) of the implicit Lagrangian hydrodynamics method.

Paper passages followed (section / equation numbers of the paper):

* Sec. 2.1, Eqs. (6a)-(6b): M_V dv/dt = -F.1, M_E de/dt = F^T.v, dx/dt = v;
* Sec. 2.1, Eq. (7): M_V = int rho w w^T, M_E = int rho phi phi^T,
  F_ij = int (sigma : grad w_i) phi_j, all over the current domain;
* Sec. 2.1 (after Eq. (7)): rho = rho0 / |J_{x<-x0}| pointwise at quadrature points,
  so rho |J| dx-weights are constant in time and the mass matrices are formed once;
* Sec. 3.4, Eqs. (11), (13)-(20): sigma = -p I + mu eps(v), mu = mu_imp with the
  smooth length scale, compression measure, smooth |.|, smooth switch and
  the regularised energy e+;
* Sec. 3.5, Eq. (21): R(k; tau, u) evaluated at the stage state w = u + tau k.

Readings where the paper is silent (the same readings are used by the CUDA path):

* R is written in mass-weighted form (no mass inverse), matching the blocks
  M_V + tau dF/dv and M_E - tau dF^T/de of Eq. (23):
      R_x = k_x - w_v
      R_v = M_V k_v + F(w).1          (rows of fixed normal velocity: R_v = k_v)
      R_e = M_E k_e - F(w)^T w_v - b(w)
* b is the manufactured Taylor-Green energy source (only when enabled):
  b_j = int_{Omega(w)} s(x) phi_j dx with s = v.grad p / (gamma - 1) of the steady
  vortex, s = (3 pi / 8) [cos 3 pi x cos pi y - cos pi x cos 3 pi y] for gamma = 5/3.

All arithmetic is written so that it also runs in complex128, which lets
``jvp_complex_step`` differentiate it (the residual is analytic in k).
"""
import numpy as np


class Params:
    """Physical and model parameters (defaults from Sec. 3.4)."""

    def __init__(self, mesh, rho0=1.0, gamma=1.4, visc=True, q1=0.5, q2=1.0, psi0=0.5,
                 eps_e=1e-6, h0=None, h_coarse=None, bc_mask=None, tg_source=False,
                 visc_model='imp', q1_exp=0.5, q2_exp=2.0, vorticity=False):
        ne = mesh.NE
        self.rho0 = np.broadcast_to(np.asarray(rho0, dtype=float), (ne,)).copy()
        self.gamma = np.broadcast_to(np.asarray(gamma, dtype=float), (ne,)).copy()
        self.visc = bool(visc)
        self.q1, self.q2, self.psi0, self.eps_e = float(q1), float(q2), float(psi0), float(eps_e)
        vol = float(np.prod(mesh.hi - mesh.lo))
        self.h0 = float(h0) if h0 else (vol / mesh.NE) ** (1.0 / mesh.d)
        self.h_coarse = float(h_coarse) if h_coarse else self.h0
        self.bc_mask = (1 << (2 * mesh.d)) - 1 if bc_mask is None else int(bc_mask)
        self.tg_source = bool(tg_source)
        # the original tensor viscosity mu_exp (Sec. 3.4) for explicit runs: 'exp'
        if visc_model not in ('imp', 'exp'):
            raise ValueError("visc_model must be 'imp' or 'exp'")
        self.visc_model = visc_model
        self.q1_exp, self.q2_exp = float(q1_exp), float(q2_exp)
        self.l0_exp = self.h0 / mesh.k
        self.vorticity = bool(vorticity)


def det(J):
    """Determinant of a batch of d x d matrices [..., d, d] (cofactor expansion)."""
    if J.shape[-1] == 2:
        return J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
    return (J[..., 0, 0] * (J[..., 1, 1] * J[..., 2, 2] - J[..., 1, 2] * J[..., 2, 1])
            - J[..., 0, 1] * (J[..., 1, 0] * J[..., 2, 2] - J[..., 1, 2] * J[..., 2, 0])
            + J[..., 0, 2] * (J[..., 1, 0] * J[..., 2, 1] - J[..., 1, 1] * J[..., 2, 0]))


def inv(J):
    """Inverse of a batch of d x d matrices (adjugate over determinant)."""
    dt = det(J)
    A = np.empty_like(J)
    if J.shape[-1] == 2:
        A[..., 0, 0] = J[..., 1, 1]
        A[..., 0, 1] = -J[..., 0, 1]
        A[..., 1, 0] = -J[..., 1, 0]
        A[..., 1, 1] = J[..., 0, 0]
    else:
        for i in range(3):
            for j in range(3):
                r = [m for m in range(3) if m != j]
                c = [m for m in range(3) if m != i]
                minor = J[..., r[0], c[0]] * J[..., r[1], c[1]] - J[..., r[0], c[1]] * J[..., r[1], c[0]]
                A[..., i, j] = (-1) ** (i + j) * minor
    return A / dt[..., None, None]


def stress(grad_v, detJ, rho, e, gamma, prm, d, return_mu=False):
    """Total stress sigma = -p I + mu_imp eps(v) at quadrature points (Sec. 3.4).

    grad_v: physical velocity gradient [..., d, d] ((grad v)_{cb} = dv_c/dx_b);
    detJ, rho, e, gamma: [...]; returns sigma [..., d, d].
    """
    # Eq. (19): smooth positive part of the specific internal energy.  For e < 0 the same
    # quantity is evaluated as eps^2 / (2 (sqrt(e^2 + eps^2) - e)) (multiply and divide by
    # the conjugate), which avoids the cancellation of e + sqrt(e^2 + eps^2)
    root = np.sqrt(e * e + prm.eps_e ** 2)
    neg = np.real(e) < 0
    e_plus = np.where(neg, 0.5 * prm.eps_e ** 2 / np.where(neg, root - e, 1.0), 0.5 * (e + root))
    # Eq. (20): ideal-gas pressure and sound speed
    p = (gamma - 1.0) * rho * e_plus
    c_s = np.sqrt(gamma * (gamma - 1.0) * e_plus)
    eye = np.eye(d)
    sigma = -p[..., None, None] * eye
    mu = np.zeros_like(p)
    if prm.visc:
        # Eq. (14): isotropic current length scale by volume scaling
        h = prm.h0 * (detJ / prm.detJ0) ** (1.0 / d)
        # Eq. (15): compression measure
        delta_v = h * np.trace(grad_v, axis1=-2, axis2=-1)
        # Eq. (18): smoothing scale
        delta_s = 2.0 * (h / prm.h_coarse) * c_s
        # Eq. (16): smooth absolute value
        abs_dv = np.sqrt(delta_v ** 2 + delta_s ** 2)
        # Eq. (17): smooth compression switch with psi(0) = psi0
        shift = 2.0 * delta_s * np.arctanh(1.0 - 2.0 * prm.psi0)
        psi = 0.5 + 0.5 * np.tanh((-delta_v - shift) / (2.0 * delta_s))
        # Eq. (13): smooth viscosity coefficient
        mu = rho * h * (prm.q2 * abs_dv + prm.q1 * c_s * psi)
        # Eq. (11): sigma_a = mu eps(v), eps(v) = sym(grad v)
        eps_v = 0.5 * (grad_v + np.swapaxes(grad_v, -1, -2))
        sigma = sigma + mu[..., None, None] * eps_v
    return (sigma, mu) if return_mu else sigma


def stress_exp(grad_v, J, J0inv, rho, e, gamma, prm, d, return_mu=False):
    """Total stress sigma = -p I + mu_exp eps(v) with the original tensor viscosity (Sec. 3.4,
    the equation for mu_exp; its ingredients are defined in Dobrev et al. 2012, Sec. 6.2,
    which the paper cites and does not print; the readings here):

      (lambda_1, s_1): smallest eigenvalue of eps(v) and its unit eigenvector;
      l = l0 |J J0^{-1} s_1|: the initial length l0 = h0 / k carried by the deformation
          (J J0^{-1} = dx / dx0) along s_1;
      psi_1 = 1 if lambda_1 < 0 (compression) else 0;
      psi_0 = 1, or |div v| / (sqrt(d) |grad v|_F) in [0, 1] with the vorticity switch on
          (1 for isotropic compression, 0 for divergence-free flow);
      mu_exp = rho (q2 l^2 |lambda_1| + q1 psi_1 psi_0 l c_s).

    e+, p and c_s as in Eqs. (19)-(20).  grad_v, J, J0inv: [..., d, d]; rho, e, gamma: [...].
    Real arithmetic only (the eigen-decomposition is not analytic)."""
    root = np.sqrt(e * e + prm.eps_e ** 2)
    e_plus = np.where(e < 0, 0.5 * prm.eps_e ** 2 / np.where(e < 0, root - e, 1.0), 0.5 * (e + root))
    p = (gamma - 1.0) * rho * e_plus
    c_s = np.sqrt(gamma * (gamma - 1.0) * e_plus)
    sigma = -p[..., None, None] * np.eye(d)
    if not prm.visc:
        return (sigma, np.zeros_like(p)) if return_mu else sigma
    eps_v = 0.5 * (grad_v + np.swapaxes(grad_v, -1, -2))
    lam, vec = np.linalg.eigh(eps_v)                  # ascending eigenvalues
    lam1, s1 = lam[..., 0], vec[..., :, 0]
    Fd = np.einsum('...ij,...jk->...ik', J, J0inv)
    ell = prm.l0_exp * np.linalg.norm(np.einsum('...ij,...j->...i', Fd, s1), axis=-1)
    psi1 = (lam1 < 0).astype(float)
    if prm.vorticity:
        gnorm = np.sqrt(np.sum(grad_v * grad_v, axis=(-2, -1)))
        psi0 = np.where(gnorm > 0, np.abs(np.trace(grad_v, axis1=-2, axis2=-1))
                        / (np.sqrt(d) * np.where(gnorm > 0, gnorm, 1.0)), 1.0)
    else:
        psi0 = 1.0
    mu = rho * (prm.q2_exp * ell ** 2 * np.abs(lam1) + prm.q1_exp * psi1 * psi0 * ell * c_s)
    sigma = sigma + mu[..., None, None] * eps_v
    return (sigma, mu) if return_mu else sigma


def tg_source(xq):
    """Taylor-Green manufactured energy source s(x) (per unit volume), gamma = 5/3.

    From the steady vortex v = (sin pi x cos pi y, -cos pi x sin pi y),
    p = 100 + (cos 2 pi x + cos 2 pi y) / 4, rho = 1: momentum balances exactly and
    rho de/dt = v.grad e = v.grad p / (gamma - 1) must be supplied by the source.
    """
    x, y = xq[..., 0], xq[..., 1]
    pi = np.pi
    return (3.0 * pi / 8.0) * (np.cos(3 * pi * x) * np.cos(pi * y) - np.cos(pi * x) * np.cos(3 * pi * y))


class Hydro:
    """Discrete operators of Eq. (7) on a Mesh, with the stage residual of Eq. (21)."""

    def __init__(self, mesh, prm):
        self.m, self.p = mesh, prm
        x0 = mesh.initial_nodes()
        J0 = np.einsum('ecn,qrn->eqcr', mesh.gather(x0), mesh.Gh)
        self.detJ0 = det(J0)                                 # [NE, NQ]
        self.J0inv = inv(J0)
        prm.detJ0 = self.detJ0
        # rho |J| is conserved pointwise: rho alpha detJ = rho0 alpha detJ0 (Sec. 2.1)
        self.mq = prm.rho0[:, None] * mesh.alpha[None, :] * self.detJ0   # [NE, NQ]
        self.fixed = mesh.boundary_mask(prm.bc_mask)        # [d, NV]
        self.x0 = x0

    # -- mass matrices (Eq. (7)), formed once -------------------------------------------
    def mass_v_elem(self):
        """Element H1 mass matrices [NE, ND, ND] = sum_q rho alpha detJ w_a w_b."""
        B = self.m.Bh
        return np.einsum('eq,qa,qb->eab', self.mq, B, B)

    def mass_e_elem(self):
        """Element L2 mass matrices [NE, NL, NL] = sum_q rho alpha detJ phi_i phi_j."""
        B = self.m.Bl
        return np.einsum('eq,qa,qb->eab', self.mq, B, B)

    def mass_v_dense(self):
        """Assembled scalar H1 mass matrix [NV, NV] (dense; small meshes only)."""
        M = np.zeros((self.m.NV, self.m.NV))
        Me = self.mass_v_elem()
        for e in range(self.m.NE):
            c = self.m.conn[e]
            M[np.ix_(c, c)] += Me[e]
        return M

    def mass_v_sparse(self):
        import scipy.sparse as sp
        Me = self.mass_v_elem()
        c = self.m.conn
        rows = np.repeat(c[:, :, None], self.m.ND, axis=2).ravel()
        cols = np.repeat(c[:, None, :], self.m.ND, axis=1).ravel()
        return sp.csr_matrix((Me.ravel(), (rows, cols)), shape=(self.m.NV, self.m.NV))

    def apply_mass_v(self, f):
        """M_V f for an H1 field [d, NV] (same scalar matrix per component)."""
        fe = self.m.gather(f)
        fq = np.einsum('ecn,qn->ecq', fe, self.m.Bh)
        return self.m.scatter(np.einsum('eq,ecq,qa->eca', self.mq, fq, self.m.Bh))

    def apply_mass_e(self, g):
        """M_E g for an L2 field [NE, NL] (block diagonal)."""
        return np.einsum('eab,eb->ea', self.mass_e_elem(), g)

    # -- force matrix (Eq. (7)) ---------------------------------------------------------
    def qp_state(self, x, v, e):
        """Geometry, density, velocity gradient and energy at the quadrature points."""
        m = self.m
        J = np.einsum('ecn,qrn->eqcr', m.gather(x), m.Gh)          # dx_c / dxhat_r
        detJ = det(J)
        Jinv = inv(J)                                               # dxhat_r / dx_b
        # physical gradients of the H1 basis: grad w_a = J^{-T} ghat w_a
        gradw = np.einsum('eqrb,qrn->eqbn', Jinv, m.Gh)             # [NE, NQ, d, ND]
        grad_v = np.einsum('ecn,eqbn->eqcb', m.gather(v), gradw)    # dv_c / dx_b
        eq = np.einsum('ej,qj->eq', e, m.Bl)
        # pointwise mass conservation: rho = rho0 / |J_{x<-x0}| = rho0 detJ0 / detJ
        rho = self.p.rho0[:, None] * self.detJ0 / detJ
        return J, detJ, gradw, grad_v, eq, rho

    def force_matrix(self, x, v, e):
        """Element force matrices F_e[(c, a), j] = int (sigma : grad w_{c,a}) phi_j.

        Returns F [NE, d, ND, NL] together with detJ [NE, NQ] for the line search.
        """
        m = self.m
        J, detJ, gradw, grad_v, eq, rho = self.qp_state(x, v, e)
        if self.p.visc_model == 'exp':
            sigma = stress_exp(grad_v, J, self.J0inv, rho, eq, self.p.gamma[:, None], self.p, m.d)
        else:
            sigma = stress(grad_v, detJ, rho, eq, self.p.gamma[:, None], self.p, m.d)
        # sigma : grad w_{c,a} = sum_b sigma_{cb} (grad w_a)_b for the vector basis w_a e_c
        sig_gw = np.einsum('eqcb,eqbn->eqcn', sigma, gradw)
        dx = m.alpha[None, :] * detJ                              # current-domain weights
        F = np.einsum('eq,eqcn,qj->ecnj', dx, sig_gw, m.Bl)
        return F, detJ

    def source(self, x):
        """Element vector b_j = int_{Omega(x)} s phi_j dx for the Taylor-Green source."""
        m = self.m
        xq = np.einsum('ecn,qn->eqc', m.gather(x), m.Bh)
        detJ = det(np.einsum('ecn,qrn->eqcr', m.gather(x), m.Gh))
        return np.einsum('eq,eq,qj->ej', m.alpha[None, :] * detJ, tg_source(xq), m.Bl)

    # -- stage residual (Eq. (21)) ----------------------------------------------------------
    def residual(self, u, k, tau, return_detj=False):
        m = self.m
        w = u + tau * k
        wx, wv, we = m.split(w)
        kx, kv, ke = m.split(k)
        F, detJ = self.force_matrix(wx, wv, we)
        ones = np.ones(m.NL)
        F1 = m.scatter(np.einsum('ecnj,j->ecn', F, ones))                  # F . 1
        FTv = np.einsum('ecnj,ecn->ej', F, m.gather(wv))                   # F^T . w_v
        Rx = kx - wv
        Rv = self.apply_mass_v(kv) + F1
        Rv = np.where(self.fixed, kv, Rv)
        Re = self.apply_mass_e(ke) - FTv
        if self.p.tg_source:
            Re = Re - self.source(wx)
        R = m.join(Rx, Rv, Re)
        return (R, detJ) if return_detj else R

    def min_detj(self, x):
        m = self.m
        return float(np.min(det(np.einsum('ecn,qrn->eqcr', m.gather(x), m.Gh)).real))

    # -- Jacobian actions ---------------------------------------------------------------------
    def jvp_complex_step(self, u, k, tau, dk, h=1e-30):
        """J dk with J = dR/dk by the complex-step derivative Im R(k + i h dk) / h."""
        return self.residual(u.astype(complex), k + 1j * h * dk, tau).imag / h

    def jvp_fd(self, u, k, tau, dk, h=1e-7):
        """Central finite difference (R(k + h dk) - R(k - h dk)) / 2h."""
        return (self.residual(u, k + h * dk, tau) - self.residual(u, k - h * dk, tau)) / (2 * h)

    def jacobian(self, u, k, tau, method='cs'):
        """Dense Jacobian, column by column (small meshes only)."""
        n = k.size
        Jm = np.zeros((n, n))
        for j in range(n):
            ej = np.zeros(n)
            ej[j] = 1.0
            if method == 'cs':
                Jm[:, j] = self.jvp_complex_step(u, k, tau, ej)
            else:
                hj = 1e-7 * max(1.0, abs(k[j]))
                Jm[:, j] = self.jvp_fd(u, k, tau, ej, hj)
        return Jm

    # -- energies ------------------------------------------------------------------------------
    def kinetic_energy(self, u):
        _, v, _ = self.m.split(u)
        return 0.5 * float(np.sum(v * self.apply_mass_v(v)))

    def internal_energy(self, u):
        _, _, e = self.m.split(u)
        return float(np.sum(self.apply_mass_e(e)))

    def total_mass(self):
        return float(np.sum(self.mq))


def coupling_pattern(mesh):
    """Sparse boolean pattern of dR/dk: dofs couple when they share an element.

    Every unknown (x and v components of an H1 node, an L2 dof) belongs to the elements
    that contain it; R at any row depends only on unknowns of the elements containing
    that row's dof (R_x couples x_i and v_i of the same node, which share elements too).
    Returns a CSC matrix (n x n) with a 1 where a row and a column share an element.
    """
    import scipy.sparse as sp
    m = mesh
    rows, cols = [], []
    n1 = m.d * m.NV
    for e in range(m.NE):
        dofs = []
        for c in range(m.d):
            dofs.append(c * m.NV + m.conn[e])            # x components
            dofs.append(n1 + c * m.NV + m.conn[e])       # v components
        dofs.append(2 * n1 + e * m.NL + np.arange(m.NL))
        dofs = np.concatenate(dofs)
        rows.append(np.full(dofs.size, e))
        cols.append(dofs)
    P = sp.csr_matrix((np.ones(sum(r.size for r in rows)), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(m.NE, m.n_unknowns))
    pat = (P.T @ P).tocsc()
    pat.data[:] = 1.0
    return pat


def column_colors(mesh):
    """Colour of every unknown so that same-coloured columns share no row.

    H1 dofs: a node at lattice position i reaches rows within lattice distance k, so two
    nodes with the same i mod (2k+1) in every direction share no row.  L2 dofs of
    elements whose positions agree mod 2 in every direction share no node.  x, v and e
    columns and the components get separate colour ranges.
    """
    m = mesh
    colors = np.zeros(m.n_unknowns, dtype=np.int64)
    ids = np.arange(m.NV)
    mod = 2 * m.k + 1
    hcol = np.zeros(m.NV, dtype=np.int64)
    stride_c = 1
    for c in range(m.d):
        stride = int(np.prod(m.lat[:c]))
        hcol += ((ids // stride) % m.lat[c] % mod) * stride_c
        stride_c *= mod
    nh = stride_c
    base = 0
    for field in range(2):
        for c in range(m.d):
            off = (field * m.d + c) * m.NV
            colors[off:off + m.NV] = base + hcol
            base += nh
    ecol = np.zeros(m.NE, dtype=np.int64)
    stride_c = 1
    for c in range(m.d):
        ecol += (m.ecoord[:, c] % 2) * stride_c
        stride_c *= 2
    off = 2 * m.d * m.NV
    colors[off:] = base + (ecol[:, None] * m.NL + np.arange(m.NL)[None, :]).ravel()
    return colors


def jacobian_sparse(hyd, u, k, tau, pattern=None, colors=None):
    """Sparse Jacobian by compressed complex-step columns (Curtis-Powell-Reid).

    For each colour the sum of its unit vectors is differentiated once; the rows of
    each column are read off the coupling pattern.  Exact to rounding, like the dense
    complex-step Jacobian.
    """
    import scipy.sparse as sp
    m = hyd.m
    pat = coupling_pattern(m) if pattern is None else pattern
    col = column_colors(m) if colors is None else colors
    n = m.n_unknowns
    indptr, indices = pat.indptr, pat.indices
    data = np.zeros(indices.size)
    for c in range(int(col.max()) + 1):
        members = np.nonzero(col == c)[0]
        if members.size == 0:
            continue
        seed = np.zeros(n)
        seed[members] = 1.0
        Js = hyd.jvp_complex_step(u, k, tau, seed)
        for j in members:
            sl = slice(indptr[j], indptr[j + 1])
            data[sl] = Js[indices[sl]]
    return sp.csc_matrix((data, indices.copy(), indptr.copy()), shape=(n, n))
