"""C ABI checks that need no GPU: the library loads, exports every symbol that
include/lh.h declares, and the ctypes structures match the C layout."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lh.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lh_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300 import _lib
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lh.lib, name), name
    assert sorted(_lib.SYMBOLS) == names


def test_struct_layout_matches_header(tmp_path):
    from paper_2609_16424_b300 import _lib
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "lh.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(lh_mesh_desc), offsetof(lh_mesh_desc, rho0),
         offsetof(lh_mesh_desc, bc_mask), offsetof(lh_mesh_desc, tg_source), offsetof(lh_mesh_desc, stream));
  printf("%zu %zu %zu\n", sizeof(lh_newton_opts), offsetof(lh_newton_opts, jvp_prec),
         offsetof(lh_newton_opts, arnoldi));
  printf("%zu %zu %zu\n", sizeof(lh_step_stats), offsetof(lh_step_stats, min_detj),
         offsetof(lh_step_stats, newton_its_max));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(lh_advance_opts), offsetof(lh_advance_opts, dt0),
         offsetof(lh_advance_opts, max_attempts), offsetof(lh_advance_opts, dt_min), sizeof(lh_advance_attempt),
         offsetof(lh_advance_attempt, accepted));
  printf("%zu %zu %zu\n", sizeof(lh_advance_stats), offsetof(lh_advance_stats, t),
         offsetof(lh_advance_stats, gmres_its));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    D = _lib.MeshDesc
    assert [int(x) for x in out[0].split()] == [C.sizeof(D), D.rho0.offset, D.bc_mask.offset,
                                                 D.tg_source.offset, D.stream.offset]
    N = _lib.NewtonOpts
    assert [int(x) for x in out[1].split()] == [C.sizeof(N), N.jvp_prec.offset, N.arnoldi.offset]
    S = _lib.StepStats
    assert [int(x) for x in out[2].split()] == [C.sizeof(S), S.min_detj.offset, S.newton_its_max.offset]
    A, H, T = _lib.AdvanceOpts, _lib.AdvanceAttempt, _lib.AdvanceStats
    assert [int(x) for x in out[3].split()] == [C.sizeof(A), A.dt0.offset, A.max_attempts.offset, A.dt_min.offset,
                                                 C.sizeof(H), H.accepted.offset]
    assert [int(x) for x in out[4].split()] == [C.sizeof(T), T.t.offset, T.gmres_its.offset]


def test_defaults_and_argument_checks_without_gpu():
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300 import _lib
    d = _lib.MeshDesc()
    lh.lib.lh_mesh_desc_init(C.byref(d))
    assert (d.dim, d.order, d.visc, d.q1, d.q2, d.psi0, d.eps_e) == (3, 2, 1, 0.5, 1.0, 0.5, 1e-6)
    o = _lib.NewtonOpts()
    lh.lib.lh_newton_opts_init(C.byref(o))
    assert (o.newton_rtol, o.gmres_rtol, o.restart) == (1e-10, 1e-12, 30)
    assert (o.precond, o.forcing, o.eta_max, o.scaled_norm) == (1, 0, 0.1, 0)
    # the binding maps option names and rejects unknown ones (a typo must not pass silently)
    o2 = lh.newton_opts(precond="jvv_diag", jvp_prec="bf16", scaled_norm=1)
    assert (o2.precond, o2.jvp_prec, o2.scaled_norm) == (2, _lib.LH_BF16, 1)
    with pytest.raises(TypeError):
        lh.newton_opts(newton_rtoll=1e-6)
    # invalid descriptions are rejected before any CUDA call
    h = C.c_void_p()
    d.order = 7
    assert lh.lib.lh_mesh_create(C.byref(d), C.byref(h)) == _lib.LH_EINVAL
    assert b"order" in lh.lib.lh_last_error(None)
    d.order, d.dim = 2, 4
    assert lh.lib.lh_mesh_create(C.byref(d), C.byref(h)) == _lib.LH_EINVAL
    assert lh.lib.lh_mesh_create(None, C.byref(h)) == _lib.LH_EINVAL
    assert h.value is None


@pytest.mark.parametrize("fn", ["lh_residual", "lh_jvp", "lh_jtvp", "lh_newton_step", "lh_stage_solve",
                                "lh_sdirk_step", "lh_jvv_diagonal", "lh_tg_velocity_error", "lh_advance"])
def test_null_mesh_is_rejected(fn):
    import paper_2609_16424_b300 as lh
    f = getattr(lh.lib, fn)
    nargs = len(f.argtypes)
    args = [None] * nargs
    if fn in ("lh_residual", "lh_jvp", "lh_jtvp", "lh_newton_step", "lh_stage_solve", "lh_jvv_diagonal",
              "lh_advance"):
        args[3] = 0.1
    if fn == "lh_advance":
        args[8] = 0
    if fn == "lh_sdirk_step":
        args[1], args[4] = 3, 0.1
    if fn in ("lh_jvp", "lh_jtvp"):
        args[6] = 0
    assert f(*args) == 1     # LH_EINVAL
