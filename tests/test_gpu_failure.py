"""Failure detection on the GPU without a fault: a bounded device wait is made
to run out and the host reads the status; the context stays usable.

mx_inject_wait_timeout makes the two-CTA plane kernel arm its bulk-copy
barrier without issuing the copies, so the barrier never completes (no copy is
ever in flight).  The kernel's wait gives up after about one second, sets the
context's timeout flag and runs to its end; mx_sync reports MX_ERR_TIMEOUT and
clears the flag.  The next evaluation without the hook gives the oracle's
field again.
"""
import time

import numpy as np
import pytest

from helpers import cfg_of, context, problem, random_m, rel_l2, t64
from oracle import micromag as mm

pytestmark = pytest.mark.gpu


def test_bulk_copy_wait_runs_out_and_the_context_recovers():
    from paper_2602_12242_gb300 import MX_TERM_DEMAG, MxError, _lib
    from paper_2602_12242_gb300.solver import from_dev4, to_dev4
    c = cfg_of(nx=64, ny=32, nz=4)  # Px/2 = 64, Py/2 = 32 (even ny: bulk copies), Pz = 8
    ctx = context(c, demag_path=_lib.MX_DEMAG_PLANE_PAIR)
    assert ctx.kernel_name("yz_fused") == "yzh_kernel"
    m = np.asarray(random_m(c, 91), dtype=np.float32).astype(np.float64)
    ref = mm.demag_field(problem(c), t64(m)).numpy()
    dm = to_dev4(m)
    ctx.heff(dm, terms=MX_TERM_DEMAG)
    ctx.sync()
    _lib.mx_inject_wait_timeout(ctx.h, 1)
    t0 = time.time()
    ctx.heff(dm, terms=MX_TERM_DEMAG)
    with pytest.raises(MxError) as ei:
        ctx.sync()
    elapsed = time.time() - t0
    assert ei.value.status == _lib.MX_ERR_TIMEOUT
    assert 0.5 < elapsed < 60, elapsed
    _lib.mx_inject_wait_timeout(ctx.h, 0)
    h = from_dev4(ctx.heff(dm, terms=MX_TERM_DEMAG))
    ctx.sync()
    assert rel_l2(h, ref) <= 1e-5


def test_wait_timeout_hook_needs_the_two_cta_kernel():
    from paper_2602_12242_gb300 import MxError, _lib
    c = cfg_of(nx=64, ny=512, nz=16)  # four-CTA plane kernel: no bulk-copy barrier
    ctx = context(c, demag_path=_lib.MX_DEMAG_PLANE)
    assert ctx.kernel_name("yz_fused") == "yzq_kernel"
    with pytest.raises(MxError) as ei:
        _lib.mx_inject_wait_timeout(ctx.h, 1)
    assert ei.value.status == _lib.MX_ERR_UNSUPPORTED
