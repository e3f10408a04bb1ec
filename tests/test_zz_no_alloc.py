"""lh_residual_noalloc: the stage residual for callers that must not allocate device
memory when they call the library.  Its scratch lives in fixed-size static device
arrays; its output must equal the regular lh_residual on the same inputs, call after
call (the shared scratch keeps the previous call's contents)."""
import ctypes as C

import numpy as np
import pytest
import torch

import lh_synth
from lhcase import Case

pytestmark = pytest.mark.gpu


def _desc(case, tg=False, visc=True, gamma=1.4):
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300 import _lib
    d = _lib.MeshDesc()
    lh.lib.lh_mesh_desc_init(C.byref(d))
    d.dim = case.dim
    for c in range(case.dim):
        d.n[c] = case.n[c]
        d.lo[c] = 0.0
        d.hi[c] = 1.0
    d.order = case.k
    d.visc = int(visc)
    d.tg_source = int(tg)
    d.gamma_value = gamma
    d.stream = torch.cuda.current_stream().cuda_stream
    return d


def _noalloc(case, d, u, k, tau, gamma=1.4):
    import paper_2609_16424_b300 as lh
    rho0 = torch.ones(case.gm.NE, dtype=torch.float64, device="cuda")
    gam = torch.full((case.gm.NE,), gamma, dtype=torch.float64, device="cuda")
    r = torch.full_like(u, float("nan"))
    st = lh.lib.lh_residual_noalloc(C.byref(d), C.c_void_p(rho0.data_ptr()), C.c_void_p(gam.data_ptr()),
                                    C.c_void_p(u.data_ptr()), C.c_void_p(k.data_ptr()), C.c_double(tau),
                                    C.c_void_p(r.data_ptr()))
    assert st == 0, lh.lib.lh_last_error(None)
    torch.cuda.synchronize()
    return r


@pytest.mark.parametrize("dim,n,k,tg", [(3, (5, 4, 3), 2, False), (2, (7, 5), 3, True)])
def test_noalloc_residual_equals_regular_residual(dim, n, k, tg):
    gamma = 5.0 / 3.0 if tg else 1.4
    case = Case(dim, n, k, seed=31, visc=not tg, tg=tg, gamma=gamma)
    d = _desc(case, tg=tg, visc=not tg, gamma=gamma)
    u = case.dev(case.u)
    for call, seed in enumerate((41, 42)):           # two calls in a row, different k
        kk = case.dev(lh_synth.normal_vector(case.gm.n, seed, 0.1))
        tau = 0.01 * (call + 1)
        ref = case.gm.residual(u, kk, tau).cpu().numpy()
        got = _noalloc(case, d, u, kk, tau, gamma).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_noalloc_allocates_nothing_and_alternates_orders():
    """After the first call on the device (which looks up the arrays and writes the tables),
    calls of different orders in a row leave the device's free memory and torch's allocator
    unchanged, and each equals lh_residual."""
    cases = [Case(3, (4, 3, 3), 2, seed=51), Case(3, (2, 2, 2), 3, seed=52), Case(2, (6, 5), 1, seed=53)]
    descs = [_desc(c) for c in cases]
    data = []
    for c in cases:
        u = c.dev(c.u)
        kk = c.dev(lh_synth.normal_vector(c.gm.n, 54, 0.1))
        data.append((u, kk, c.gm.residual(u, kk, 0.02).cpu().numpy()))
    rho0 = [torch.ones(c.gm.NE, dtype=torch.float64, device="cuda") for c in cases]
    gam = [torch.full((c.gm.NE,), 1.4, dtype=torch.float64, device="cuda") for c in cases]
    outs = [torch.empty_like(u) for u, _, _ in data]

    def call(i):
        import paper_2609_16424_b300 as lh
        u, kk, _ = data[i]
        st = lh.lib.lh_residual_noalloc(C.byref(descs[i]), C.c_void_p(rho0[i].data_ptr()),
                                        C.c_void_p(gam[i].data_ptr()), C.c_void_p(u.data_ptr()),
                                        C.c_void_p(kk.data_ptr()), C.c_double(0.02), C.c_void_p(outs[i].data_ptr()))
        assert st == 0, lh.lib.lh_last_error(None)

    call(0)                                          # set-up call
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for rep in range(2):
        for i in (1, 0, 2, 1):
            call(i)
            torch.cuda.synchronize()
            ref = data[i][2]
            assert np.linalg.norm(outs[i].cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_rejects_meshes_beyond_its_scratch():
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300 import _lib
    d = _lib.MeshDesc()
    lh.lib.lh_mesh_desc_init(C.byref(d))
    d.n[0] = d.n[1] = d.n[2] = 64                    # 64^3 Q2: 21.2M scratch entries > 2^21
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(x.data_ptr())
    st = lh.lib.lh_residual_noalloc(C.byref(d), p, p, p, p, C.c_double(0.1), C.c_void_p(x[4:].data_ptr()))
    assert st == _lib.LH_EINVAL
    assert b"static scratch" in lh.lib.lh_last_error(None)
