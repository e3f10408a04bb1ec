"""Python view of a mesh and its operators (argument marshalling over include/lh.h)."""
import ctypes as C

import torch

from . import _lib
from . import lib as _L


class LHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def newton_opts(**kw):
    """lh_newton_opts with the library defaults, overridden by keyword arguments
    (newton_rtol, newton_atol, gmres_rtol, newton_maxit, gmres_maxit, restart,
    max_halvings, jvp_prec in {'fp64', 'fp32', 'tf32', 'bf16'}, precond in {'jacobi', 'kron',
    'jvv_diag', 'cheb'}, forcing, eta_max, scaled_norm, cheb_degree, cheb_ratio, arnoldi);
    'tf32' and 'bf16' run the element contractions of J.w on the tensor cores."""
    o = _lib.NewtonOpts()
    _L.lh_newton_opts_init(C.byref(o))
    fields = {f for f, _ in _lib.NewtonOpts._fields_}
    for key, val in kw.items():
        if key not in fields:
            raise TypeError(f"unknown Newton option {key!r}")
        if key == "jvp_prec":
            val = {"fp64": _lib.LH_FP64, "fp32": _lib.LH_FP32, "tf32": _lib.LH_TF32,
                   "bf16": _lib.LH_BF16}.get(val, val)
        if key == "precond":
            val = {"jacobi": 0, "kron": 1, "jvv_diag": 2, "cheb": 3}.get(val, val)
        setattr(o, key, val)
    return o


def advance_opts(**kw):
    """lh_advance_opts with the library defaults, overridden by keyword arguments (scheme,
    fs_cfl, dt0, grow, shrink, grow_its, reject_its, enlarge, max_steps, max_attempts, dt_min)."""
    a = _lib.AdvanceOpts()
    _L.lh_advance_opts_init(C.byref(a))
    fields = {f for f, _ in _lib.AdvanceOpts._fields_}
    for key, val in kw.items():
        if key not in fields:
            raise TypeError(f"unknown time-loop option {key!r}")
        setattr(a, key, val)
    return a


def explicit_opts(**kw):
    """lh_explicit_opts with the library defaults, overridden by keyword arguments (scheme,
    visc_model in {'imp', 'exp', 0, 1}, q1_exp, q2_exp, l0_exp, vorticity, cfl, mass_rtol,
    mass_maxit)."""
    o = _lib.ExplicitOpts()
    _L.lh_explicit_opts_init(C.byref(o))
    fields = {f for f, _ in _lib.ExplicitOpts._fields_}
    for key, val in kw.items():
        if key not in fields:
            raise TypeError(f"unknown explicit option {key!r}")
        if key == "visc_model":
            val = {"imp": 0, "exp": 1}.get(val, val)
        setattr(o, key, val)
    return o


def _stats_dict(st):
    return {f: getattr(st, f) for f, _ in st._fields_}


def _attempts(hist, count):
    return [(hist[i].dt, hist[i].h, None if hist[i].newton_its < 0 else hist[i].newton_its, bool(hist[i].accepted))
            for i in range(count)]


def advance_replay(counts, dt_est, t_end, hist_cap=100000, **kw):
    """The time loop of Mesh.advance on the host with scripted Newton counts (None: a failed
    solve), no mesh and no GPU (lh_advance_replay).  Returns (steps, rejected, attempts, t)."""
    arr = (C.c_int * max(1, len(counts)))(*[-1 if c is None else int(c) for c in counts])
    hist = (_lib.AdvanceAttempt * hist_cap)()
    stats = _lib.AdvanceStats()
    a = advance_opts(**kw)
    st = _L.lh_advance_replay(arr, len(counts), float(dt_est), float(t_end), C.byref(a), C.byref(stats), hist,
                              hist_cap)
    if st != _lib.LH_OK:
        raise LHError(st, _L.lh_last_error(None).decode())
    return stats.steps, stats.rejected, _attempts(hist, min(stats.attempts, hist_cap)), stats.t


def launch_count():
    """CUDA kernels launched by liblh.so in this process so far."""
    return int(_L.lh_launch_count())


def probe_fma(prec="fp64"):
    """Measured FMA-pipe throughput (TFLOP/s) of the current device."""
    out = C.c_double()
    st = _L.lh_probe_fma(_lib.LH_FP64 if prec == "fp64" else _lib.LH_FP32, C.byref(out))
    if st != _lib.LH_OK:
        raise LHError(st, _L.lh_last_error(None).decode())
    return out.value


class Mesh:
    """Box mesh of quads (dim 2) or hexes (dim 3) with Q_k - Q_{k-1} spaces.

    rho0 and gamma may be scalars or per-element sequences (element order x-fastest).
    All vector arguments are CUDA tensors in the layout of include/lh.h.
    """

    def __init__(self, dim, n, lo, hi, order, rho0=1.0, gamma=1.4, bc_mask=None, visc=True,
                 q1=0.5, q2=1.0, psi0=0.5, eps_e=1e-6, h0=0.0, h_coarse=0.0, tg_source=False,
                 device=None):
        self.device = torch.device(device or "cuda")
        d = _lib.MeshDesc()
        _L.lh_mesh_desc_init(C.byref(d))
        d.dim = dim
        for c in range(dim):
            d.n[c] = int(n[c])
            d.lo[c] = float(lo[c])
            d.hi[c] = float(hi[c])
        d.order = order
        ne = 1
        for c in range(dim):
            ne *= int(n[c])
        keep = []
        for name, val in (("rho0", rho0), ("gamma", gamma)):
            if hasattr(val, "__len__"):
                arr = (C.c_double * ne)(*[float(x) for x in val])
                keep.append(arr)
                setattr(d, name, C.cast(arr, C.POINTER(C.c_double)))
            else:
                setattr(d, name + "_value", float(val))
        d.bc_mask = (1 << (2 * dim)) - 1 if bc_mask is None else int(bc_mask)
        d.visc = int(bool(visc))
        d.q1, d.q2, d.psi0, d.eps_e = q1, q2, psi0, eps_e
        d.h0, d.h_coarse = h0, h_coarse
        d.tg_source = int(bool(tg_source))
        with torch.cuda.device(self.device):
            d.stream = torch.cuda.current_stream().cuda_stream
            h = C.c_void_p()
            st = _L.lh_mesh_create(C.byref(d), C.byref(h))
        if st != _lib.LH_OK:
            raise LHError(st, _L.lh_last_error(None).decode())
        self._h = h
        s = (C.c_longlong * 6)()
        self._check(_L.lh_sizes(self._h, s))
        self.NE, self.NV, self.NEd, self.n, self.NQ, self.dim = (int(x) for x in s)
        self.order = order

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _L.lh_mesh_destroy(h)
            self._h = None

    # -- helpers ---------------------------------------------------------------------
    def _check(self, st):
        if st != _lib.LH_OK:
            raise LHError(st, _L.lh_last_error(self._h).decode())

    def _stream(self):
        _L.lh_set_stream(self._h, C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))

    def _vec(self, t, name, dtype=torch.float64, n=None):
        n = self.n if n is None else n
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
                and t.numel() == n):
            raise ValueError(f"{name}: expected a contiguous CUDA {dtype} tensor of {n} entries")
        return t

    def new(self, dtype=torch.float64):
        return torch.empty(self.n, dtype=dtype, device=self.device)

    # -- operators -------------------------------------------------------------------------
    def initial_nodes(self):
        x0 = torch.empty(self.dim * self.NV, dtype=torch.float64, device=self.device)
        self._stream()
        self._check(_L.lh_initial_nodes(self._h, _ptr(x0)))
        return x0

    def residual(self, u, k, tau, out=None, min_detj=False):
        """R(k; tau, u) (Eq. (21)); with min_detj=True also returns min det J at w."""
        self._vec(u, "u")
        self._vec(k, "k")
        out = self.new() if out is None else self._vec(out, "out")
        self._stream()
        md = C.c_double()
        self._check(_L.lh_residual(self._h, _ptr(u), _ptr(k), float(tau), _ptr(out),
                                   C.byref(md) if min_detj else None))
        return (out, md.value) if min_detj else out

    def linearize(self, u, k, tau):
        """Evaluate the residual at w = u + tau k and keep the linearisation of the point map
        (float) for jvp(lin=True) and jvp(tc=...)."""
        self._vec(u, "u")
        self._vec(k, "k")
        self._stream()
        self._check(_L.lh_linearize(self._h, _ptr(u), _ptr(k), float(tau)))

    # -- box decomposition (halo of a shared face) -----------------------------------------
    def halo_len(self, face):
        n = C.c_longlong()
        st = _L.lh_halo_len(self._h, int(face), C.byref(n))
        if st != _lib.LH_OK:
            raise LHError(st, _L.lh_last_error(None).decode())
        return int(n.value)

    def halo_pack(self, face, r, buf=None):
        """Velocity rows of the nodes of a face of r (partial sums of this side)."""
        self._vec(r, "r", r.dtype)
        buf = torch.empty(self.halo_len(face), dtype=r.dtype, device=self.device) if buf is None else buf
        self._vec(buf, "buf", r.dtype, self.halo_len(face))
        self._stream()
        prec = _lib.LH_FP64 if r.dtype == torch.float64 else _lib.LH_FP32
        self._check(_L.lh_halo_pack(self._h, int(face), _ptr(r), _ptr(buf), prec))
        return buf

    def halo_add(self, face, buf, r):
        """r[free velocity rows of the face] += buf (the other side's packed rows)."""
        self._vec(r, "r", r.dtype)
        self._vec(buf, "buf", r.dtype, self.halo_len(face))
        self._stream()
        prec = _lib.LH_FP64 if r.dtype == torch.float64 else _lib.LH_FP32
        self._check(_L.lh_halo_add(self._h, int(face), _ptr(buf), _ptr(r), prec))
        return r

    def tc_status(self):
        """Raise LHError if a bounded tensor-core wait of the TF32/BF16 J.w timed out."""
        self._check(_L.lh_tc_status(self._h))

    def jvp(self, u, k, tau, dk, out=None, lin=False, tc=None):
        """(dR/dk) dk; float64 dk -> FP64 kernel, float32 dk -> FP32 kernel (lin=True: from
        the record of linearize(u, k, tau)); tc='tf32' or 'bf16': from the record, element
        contractions on the tensor cores."""
        self._vec(u, "u")
        self._vec(k, "k")
        prec = _lib.LH_FP32 if dk.dtype == torch.float32 else _lib.LH_FP64
        if lin or tc:
            if dk.dtype != torch.float32:
                raise ValueError("record-based J.w needs a float32 direction")
            prec = {None: _lib.LH_FP32_LIN, "tf32": _lib.LH_TF32, "bf16": _lib.LH_BF16}[tc]
        self._vec(dk, "dk", dk.dtype)
        out = self.new(dk.dtype) if out is None else self._vec(out, "out", dk.dtype)
        self._stream()
        self._check(_L.lh_jvp(self._h, _ptr(u), _ptr(k), float(tau), _ptr(dk), _ptr(out), prec))
        return out

    def jtvp(self, u, k, tau, y, out=None, lin=False):
        """(dR/dk)^T y: FP64 (float64 y), or FP32 from the record of linearize(u, k, tau)
        (lin=True, float32 y)."""
        self._vec(u, "u")
        self._vec(k, "k")
        dt = torch.float32 if lin else torch.float64
        self._vec(y, "y", dt)
        out = self.new(dt) if out is None else self._vec(out, "out", dt)
        self._stream()
        prec = _lib.LH_FP32_LIN if lin else _lib.LH_FP64
        self._check(_L.lh_jtvp(self._h, _ptr(u), _ptr(k), float(tau), _ptr(y), _ptr(out), prec))
        return out

    def mass_apply(self, which, f):
        n = self.dim * self.NV if which == 0 else self.NEd
        self._vec(f, "f", n=n)
        out = torch.empty(n, dtype=torch.float64, device=self.device)
        self._stream()
        self._check(_L.lh_mass_apply(self._h, int(which), _ptr(f), _ptr(out)))
        return out

    def mass_solve(self, which, rhs, rtol=1e-12, maxit=500):
        n = self.dim * self.NV if which == 0 else self.NEd
        self._vec(rhs, "rhs", n=n)
        sol = torch.empty(n, dtype=torch.float64, device=self.device)
        its = C.c_int()
        self._stream()
        self._check(_L.lh_mass_solve(self._h, int(which), _ptr(rhs), _ptr(sol), float(rtol), int(maxit),
                                     C.byref(its)))
        return sol, its.value

    def precond(self, r, tau, kind="kron"):
        """z = P^-1 r with the Newton-GMRES block preconditioner (kind 'jacobi' or 'kron')."""
        self._vec(r, "r")
        z = self.new()
        self._stream()
        self._check(_L.lh_precond(self._h, {"jacobi": 0, "kron": 1}[kind], float(tau), _ptr(r), _ptr(z)))
        return z

    def dt_estimate(self, u):
        self._vec(u, "u")
        dt = C.c_double()
        self._stream()
        self._check(_L.lh_dt_estimate(self._h, _ptr(u), C.byref(dt)))
        return dt.value

    def jvv_diagonal(self, u, k, tau, out=None):
        """Diagonal of the velocity block dR_v/dk_v = M_V + tau dF/dv at (u, k, tau), [dim * NV]
        (1 on fixed rows; the viscous part from the FP32 linearisation record)."""
        self._vec(u, "u")
        self._vec(k, "k")
        out = torch.empty(self.dim * self.NV, dtype=torch.float64, device=self.device) if out is None else out
        self._stream()
        self._check(_L.lh_jvv_diagonal(self._h, _ptr(u), _ptr(k), float(tau), _ptr(out)))
        return out

    def tg_velocity_error(self, u):
        """L1 velocity error of the 2D Taylor-Green vortex at state u (Sec. 4.1)."""
        self._vec(u, "u")
        out = C.c_double()
        self._stream()
        self._check(_L.lh_tg_velocity_error(self._h, _ptr(u), C.byref(out)))
        return out.value

    def energies(self, u):
        self._vec(u, "u")
        ke, ie = C.c_double(), C.c_double()
        self._stream()
        self._check(_L.lh_energies(self._h, _ptr(u), C.byref(ke), C.byref(ie)))
        return ke.value, ie.value

    def profile(self, enable=True):
        """Enable (and reset) or disable the per-kind element-kernel event timers."""
        self._stream()
        self._check(_L.lh_profile_enable(self._h, int(bool(enable))))

    def profile_read(self):
        """{kind: (total device ms, launches)} since the last profile(True)."""
        ms = (C.c_double * len(_lib.PROF_KINDS))()
        cnt = (C.c_longlong * len(_lib.PROF_KINDS))()
        self._check(_L.lh_profile_read(self._h, ms, cnt))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(_lib.PROF_KINDS)}

    def advance(self, u, t_end, fs_cfl=2.0, k=None, max_steps=1000000, scheme=2, max_attempts=None, grow=True,
                hist_cap=None, **kw):
        """SDIRK steps (scheme 2: implicit midpoint, 3: SD3, 4: SD4) from t = 0 to t_end with
        the Newton-count time step control of the paper's Sec. 4, run by lh_advance: the first
        dt is fs_cfl times the explicit estimate; after a step with <= 1 Newton iteration dt
        grows by 5%, with 2-3 it is kept, with >= 4 the step is rejected and repeated with
        0.85 dt (also after a failed solve).  A multi-stage step counts the most iterations
        any of its stages took.  grow=False never enlarges dt.  u (and k, the first initial
        guess, if given) advance in place; the loop also ends after max_attempts attempts.
        kw: Newton-GMRES options.  Returns (steps, rejected, attempts) with attempts =
        [(controller dt, step taken, Newton iterations or None, accepted)]."""
        self._vec(u, "u")
        if k is not None:
            self._vec(k, "k")
        a = advance_opts(scheme=scheme, fs_cfl=fs_cfl, enlarge=int(bool(grow)), max_steps=max_steps,
                         max_attempts=max_attempts or 0)
        cap = hist_cap or (max_attempts or 100000)
        hist = (_lib.AdvanceAttempt * cap)()
        stats = _lib.AdvanceStats()
        o = newton_opts(**kw)
        self._stream()
        st = _L.lh_advance(self._h, _ptr(u), _ptr(k) if k is not None else None, float(t_end), C.byref(o),
                           C.byref(a), C.byref(stats), hist, cap)
        self._check(st)
        return stats.steps, stats.rejected, _attempts(hist, min(stats.attempts, cap))

    def force(self, u, w=None, estimate=False, **kw):
        """F(u).1 [dim NV] and F(u)^T w + b [N_E] (w = the velocity of u if None), and with
        estimate=True the explicit time-step estimate, for the explicit path (kw: explicit
        options, e.g. visc_model='exp').  Returns (f1, ftw) or (f1, ftw, dt_est)."""
        self._vec(u, "u")
        if w is not None:
            self._vec(w, "w", n=self.dim * self.NV)
        f1 = torch.empty(self.dim * self.NV, dtype=torch.float64, device=self.device)
        ftw = torch.empty(self.NEd, dtype=torch.float64, device=self.device)
        est = C.c_double()
        o = explicit_opts(**kw)
        self._stream()
        self._check(_L.lh_force(self._h, _ptr(u), _ptr(w) if w is not None else None, C.byref(o), _ptr(f1),
                                _ptr(ftw), C.byref(est) if estimate else None))
        return (f1, ftw, est.value) if estimate else (f1, ftw)

    def explicit_step(self, u, dt, **kw):
        """One explicit step (scheme 2: RK2-average, 3: RK3 SSP, 4: RK4) in place on u."""
        self._vec(u, "u")
        o, st = explicit_opts(**kw), _lib.ExplicitStats()
        self._stream()
        self._check(_L.lh_explicit_step(self._h, _ptr(u), float(dt), C.byref(o), C.byref(st)))
        return _stats_dict(st)

    def explicit_advance(self, u, t_end, max_steps=10000000, **kw):
        """Explicit run from t = 0 to t_end in place on u with the explicit step control
        (first dt = cfl x estimate; repeat with 0.85 dt when the estimate at the new state is
        below the step; grow 2% when it is above 1.25 dt).  Returns the run statistics."""
        self._vec(u, "u")
        o, st = explicit_opts(**kw), _lib.ExplicitStats()
        self._stream()
        self._check(_L.lh_explicit_advance(self._h, _ptr(u), float(t_end), int(max_steps), C.byref(o),
                                           C.byref(st)))
        return _stats_dict(st)

    def newton_step(self, u, k_prev, dt, opts=None, **kw):
        """One implicit midpoint step in place on u (and k_prev, if given).  Returns the
        step statistics as a dict; raises LHError (state unchanged) on failure."""
        self._vec(u, "u")
        if k_prev is not None:
            self._vec(k_prev, "k_prev")
        o = opts if opts is not None else newton_opts(**kw)
        stats = _lib.StepStats()
        self._stream()
        st = _L.lh_newton_step(self._h, _ptr(u), _ptr(k_prev) if k_prev is not None else None, float(dt),
                               C.byref(o), C.byref(stats))
        out = {f: getattr(stats, f) for f, _ in _lib.StepStats._fields_}
        if st != _lib.LH_OK:
            err = LHError(st, _L.lh_last_error(self._h).decode())
            err.stats = out
            raise err
        return out

    def _stats_call(self, fn, *args):
        stats = _lib.StepStats()
        self._stream()
        st = fn(*args, C.byref(stats))
        out = {f: getattr(stats, f) for f, _ in _lib.StepStats._fields_}
        if st != _lib.LH_OK:
            err = LHError(st, _L.lh_last_error(self._h).decode())
            err.stats = out
            raise err
        return out

    def stage_solve(self, u_base, k, tau, opts=None, **kw):
        """Solve the stage system R(k; tau, u_base) = 0 (Eq. (21)) in place on k (the initial
        guess on entry); u_base is not changed.  Returns the solve statistics as a dict;
        raises LHError (k unchanged) on failure."""
        self._vec(u_base, "u_base")
        self._vec(k, "k")
        o = opts if opts is not None else newton_opts(**kw)
        return self._stats_call(_L.lh_stage_solve, self._h, _ptr(u_base), _ptr(k), float(tau), C.byref(o))

    def sdirk_step(self, u, k_prev, dt, scheme=3, opts=None, **kw):
        """One SDIRK step in place on u: scheme 2 (implicit midpoint), 3 (SD3, order 3,
        L-stable) or 4 (SD4, order 4, A-stable), each stage solved by Newton-GMRES.  k_prev
        (or None) is the first stage's initial guess and receives the last stage's k.
        Returns the statistics summed over the stages (newton_its_max: the largest stage
        count); raises LHError (state unchanged) on failure."""
        self._vec(u, "u")
        if k_prev is not None:
            self._vec(k_prev, "k_prev")
        o = opts if opts is not None else newton_opts(**kw)
        return self._stats_call(_L.lh_sdirk_step, self._h, int(scheme), _ptr(u),
                                _ptr(k_prev) if k_prev is not None else None, float(dt), C.byref(o))
