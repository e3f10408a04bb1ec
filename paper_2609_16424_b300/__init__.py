"""B300-native implicit high-order Lagrangian hydrodynamics (arxiv 2609.16424).

Thin Python binding over the C ABI of ``liblh.so`` (include/lh.h).  Every operator runs
in the library's CUDA kernels; this package only marshals torch tensors (device memory
and the current stream) into the C calls.  There is no CPU fallback: importing the
package fails if the compiled library is missing.
"""
import os

from . import _lib

if not os.path.exists(_lib.LIB_PATH):
    raise ImportError(
        "liblh.so is missing: build it with `python paper_2609_16424_b300/build.py` "
        "(or __graft_entry__.build()); the package has no fallback path")

lib = _lib.load()

from .hydro import Mesh, LHError, probe_fma, newton_opts, advance_opts, advance_replay, launch_count  # noqa: E402
from .autograd import StageResidual  # noqa: E402

__all__ = ["Mesh", "LHError", "probe_fma", "newton_opts", "advance_opts", "advance_replay", "launch_count",
           "StageResidual", "lib"]
